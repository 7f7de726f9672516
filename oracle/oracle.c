/*
 * oracle.c -- plain, serial, FP64 CPU oracle for the Parareal stencil path.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header or constant with the CUDA path.
 *
 * Every routine is the textbook definition written out with plain loops, in
 * double precision, with no blocking, fusion or reordering:
 *
 *   - the advection-diffusion right-hand side u_t = -a.grad u + nu(t) Lap u
 *     of the benchmark problem (Sec. 3, Eq. adv_diff_eq) on the periodic unit
 *     cube, discretised three ways:
 *       ORC_C2      second-order centred: the 7-point Laplacian of Sec. 2.3
 *                   and centred first differences for advection;
 *       ORC_C4      fourth-order centred differences for both terms (the
 *                   paper's fine propagator, Sec. 2.3 / Sec. 3.1);
 *       ORC_UPWIND  7-point Laplacian plus first-order upwind advection (the
 *                   paper's coarse propagator, Algorithm 2);
 *   - classical four-stage Runge-Kutta (Sec. 2.3, fine propagator) with the
 *     stage times t, t+dt/2, t+dt/2, t+dt, or with nu frozen at the step start;
 *   - forward Euler (Algorithm 2);
 *   - box restriction and trilinear prolongation between a grid and one
 *     coarsened by an integer factor (the spatial coarsening of Sec. 2.2.2);
 *   - a periodic integer shift;
 *   - a periodic 3x3x3 convolution with its two gradients, and GELU.
 *
 * Grid: n^3 points x_i = i/n, i = 0..n-1 per axis, h = 1/n, stored
 * [z][y][x] with x fastest.  Time of step j of a run that starts at integer
 * step index s0 with step dt is (s0 + j) * dt.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

enum { ORC_C2 = 0, ORC_C4 = 1, ORC_UPWIND = 2 };

typedef struct {
    int n;          /* grid edge */
    int scheme;     /* ORC_C2, ORC_C4 or ORC_UPWIND */
    double a[3];    /* advection velocity (x, y, z) */
    double nu0;     /* nu(t) = nu0 * (1 + nu_amp * sin(nu_omega * t)) */
    double nu_amp;
    double nu_omega;
} orc_problem;

static long idx3(int n, int i, int j, int k)
{
    /* periodic wrap of each index into 0..n-1 */
    i = ((i % n) + n) % n;
    j = ((j % n) + n) % n;
    k = ((k % n) + n) % n;
    return ((long)k * n + j) * n + i;
}

/* Diffusion coefficient of Sec. 3: nu(t) = nu0 + (nu0/2) sin(omega t) when
 * nu_amp = 1/2. */
double orc_nu(const orc_problem *p, double t)
{
    return p->nu0 * (1.0 + p->nu_amp * sin(p->nu_omega * t));
}

/* out = A(nu) u, the semi-discrete right-hand side for a given nu. */
void orc_apply_A(const orc_problem *p, double nu, const double *u, double *out)
{
    const int n = p->n;
    const double h = 1.0 / n;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                const double c = u[idx3(n, i, j, k)];
                /* neighbours at distance 1 and 2 along each axis */
                double m1[3], p1[3], m2[3], p2[3];
                m1[0] = u[idx3(n, i - 1, j, k)]; p1[0] = u[idx3(n, i + 1, j, k)];
                m1[1] = u[idx3(n, i, j - 1, k)]; p1[1] = u[idx3(n, i, j + 1, k)];
                m1[2] = u[idx3(n, i, j, k - 1)]; p1[2] = u[idx3(n, i, j, k + 1)];
                m2[0] = u[idx3(n, i - 2, j, k)]; p2[0] = u[idx3(n, i + 2, j, k)];
                m2[1] = u[idx3(n, i, j - 2, k)]; p2[1] = u[idx3(n, i, j + 2, k)];
                m2[2] = u[idx3(n, i, j, k - 2)]; p2[2] = u[idx3(n, i, j, k + 2)];
                double lap = 0.0, adv = 0.0;
                for (int d = 0; d < 3; ++d) {
                    if (p->scheme == ORC_C4) {
                        /* fourth-order centred second and first derivatives */
                        lap += (-m2[d] + 16.0 * m1[d] - 30.0 * c + 16.0 * p1[d] - p2[d])
                               / (12.0 * h * h);
                        adv += p->a[d] * (m2[d] - 8.0 * m1[d] + 8.0 * p1[d] - p2[d])
                               / (12.0 * h);
                    } else {
                        /* 7-point Laplacian, one axis at a time */
                        lap += (m1[d] - 2.0 * c + p1[d]) / (h * h);
                        if (p->scheme == ORC_C2) {
                            adv += p->a[d] * (p1[d] - m1[d]) / (2.0 * h);
                        } else { /* ORC_UPWIND: difference taken on the upstream side */
                            if (p->a[d] > 0.0)
                                adv += p->a[d] * (c - m1[d]) / h;
                            else
                                adv += p->a[d] * (p1[d] - c) / h;
                        }
                    }
                }
                out[idx3(n, i, j, k)] = nu * lap - adv;
            }
}

/* Classical RK4, nsteps steps of size dt, in place.  Step j runs from
 * t = (s0 + j) dt.  frozen != 0 evaluates nu at the step start for all four
 * stages; otherwise at the classical stage times t, t+dt/2, t+dt/2, t+dt. */
void orc_rk4(const orc_problem *p, double *u, long s0, double dt, int nsteps, int frozen)
{
    const long N = (long)p->n * p->n * p->n;
    double *k1 = malloc(N * sizeof(double));
    double *k2 = malloc(N * sizeof(double));
    double *k3 = malloc(N * sizeof(double));
    double *k4 = malloc(N * sizeof(double));
    double *y = malloc(N * sizeof(double));
    for (int j = 0; j < nsteps; ++j) {
        const double t = (double)(s0 + j) * dt;
        const double nu1 = orc_nu(p, t);
        const double nu2 = frozen ? nu1 : orc_nu(p, t + 0.5 * dt);
        const double nu4 = frozen ? nu1 : orc_nu(p, t + dt);
        orc_apply_A(p, nu1, u, k1);
        for (long q = 0; q < N; ++q) y[q] = u[q] + 0.5 * dt * k1[q];
        orc_apply_A(p, nu2, y, k2);
        for (long q = 0; q < N; ++q) y[q] = u[q] + 0.5 * dt * k2[q];
        orc_apply_A(p, nu2, y, k3);
        for (long q = 0; q < N; ++q) y[q] = u[q] + dt * k3[q];
        orc_apply_A(p, nu4, y, k4);
        for (long q = 0; q < N; ++q)
            u[q] = u[q] + dt / 6.0 * (k1[q] + 2.0 * k2[q] + 2.0 * k3[q] + k4[q]);
    }
    free(k1); free(k2); free(k3); free(k4); free(y);
}

/* Forward Euler (Algorithm 2): u <- u + dt A(nu(t)) u with t the step start. */
void orc_euler(const orc_problem *p, double *u, long s0, double dt, int nsteps)
{
    const long N = (long)p->n * p->n * p->n;
    double *r = malloc(N * sizeof(double));
    for (int j = 0; j < nsteps; ++j) {
        const double t = (double)(s0 + j) * dt;
        orc_apply_A(p, orc_nu(p, t), u, r);
        for (long q = 0; q < N; ++q) u[q] = u[q] + dt * r[q];
    }
    free(r);
}

/* Box restriction by factor r: each coarse value is the plain average of the
 * r^3 fine values of its cell, fine indices I*r .. I*r+r-1 per axis. */
void orc_restrict_box(const double *f, int n, int r, double *c)
{
    const int nc = n / r;
    for (int K = 0; K < nc; ++K)
        for (int J = 0; J < nc; ++J)
            for (int I = 0; I < nc; ++I) {
                double s = 0.0;
                for (int dk = 0; dk < r; ++dk)
                    for (int dj = 0; dj < r; ++dj)
                        for (int di = 0; di < r; ++di)
                            s += f[idx3(n, I * r + di, J * r + dj, K * r + dk)];
                c[idx3(nc, I, J, K)] = s / ((double)r * r * r);
            }
}

/* Periodic trilinear prolongation by factor r.  Coarse value I sits at the
 * centroid of its cell, fine-index coordinate I*r + (r-1)/2, so fine point i
 * has coarse coordinate s = (i - (r-1)/2) / r and takes the linear blend of
 * its two bracketing coarse values along each axis. */
void orc_prolong_trilinear(const double *c, int nc, int r, double *f)
{
    const int n = nc * r;
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i) {
                const int q[3] = {i, j, k};
                int lo[3];
                double w[3];
                for (int d = 0; d < 3; ++d) {
                    const double s = (q[d] - 0.5 * (r - 1)) / r;
                    lo[d] = (int)floor(s);
                    w[d] = s - lo[d];
                }
                double v = 0.0;
                for (int ck = 0; ck < 2; ++ck)
                    for (int cj = 0; cj < 2; ++cj)
                        for (int ci = 0; ci < 2; ++ci) {
                            const double wt = (ci ? w[0] : 1.0 - w[0])
                                            * (cj ? w[1] : 1.0 - w[1])
                                            * (ck ? w[2] : 1.0 - w[2]);
                            v += wt * c[idx3(nc, lo[0] + ci, lo[1] + cj, lo[2] + ck)];
                        }
                f[idx3(n, i, j, k)] = v;
            }
}

/* Periodic integer shift: out(x) = u(x - s h), i.e. out[i] = u[i - s]. */
void orc_shift(const double *u, int n, int sx, int sy, int sz, double *out)
{
    for (int k = 0; k < n; ++k)
        for (int j = 0; j < n; ++j)
            for (int i = 0; i < n; ++i)
                out[idx3(n, i, j, k)] = u[idx3(n, i - sx, j - sy, k - sz)];
}

/* Periodic 3x3x3 cross-correlation, channel-first layout:
 *   out[co][p] = b[co] + sum_ci sum_{dz,dy,dx in -1..1}
 *                W[co][ci][dz+1][dy+1][dx+1] * in[ci][p + (dx,dy,dz)]          */
void orc_conv3d_fwd(const double *in, int n, int cin, int cout,
                    const double *W, const double *b, double *out)
{
    const long N = (long)n * n * n;
    for (int co = 0; co < cout; ++co)
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double s = b ? b[co] : 0.0;
                    for (int ci = 0; ci < cin; ++ci)
                        for (int dz = -1; dz <= 1; ++dz)
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx) {
                                    const double w =
                                        W[(((long)co * cin + ci) * 3 + dz + 1) * 9 + (dy + 1) * 3 + dx + 1];
                                    s += w * in[ci * N + idx3(n, i + dx, j + dy, k + dz)];
                                }
                    out[co * N + idx3(n, i, j, k)] = s;
                }
}

/* Gradient of orc_conv3d_fwd with respect to its input:
 *   din[ci][q] = sum_co sum_tap W[co][ci][tap] * dout[co][q - tap]           */
void orc_conv3d_dgrad(const double *dout, int n, int cin, int cout,
                      const double *W, double *din)
{
    const long N = (long)n * n * n;
    for (int ci = 0; ci < cin; ++ci)
        for (int k = 0; k < n; ++k)
            for (int j = 0; j < n; ++j)
                for (int i = 0; i < n; ++i) {
                    double s = 0.0;
                    for (int co = 0; co < cout; ++co)
                        for (int dz = -1; dz <= 1; ++dz)
                            for (int dy = -1; dy <= 1; ++dy)
                                for (int dx = -1; dx <= 1; ++dx) {
                                    const double w =
                                        W[(((long)co * cin + ci) * 3 + dz + 1) * 9 + (dy + 1) * 3 + dx + 1];
                                    s += w * dout[co * N + idx3(n, i - dx, j - dy, k - dz)];
                                }
                    din[ci * N + idx3(n, i, j, k)] = s;
                }
}

/* Gradient of orc_conv3d_fwd with respect to its weights and bias:
 *   dW[co][ci][tap] = sum_p dout[co][p] * in[ci][p + tap],  db[co] = sum_p dout[co][p] */
void orc_conv3d_wgrad(const double *in, const double *dout, int n, int cin, int cout,
                      double *dW, double *db)
{
    const long N = (long)n * n * n;
    for (int co = 0; co < cout; ++co) {
        double sb = 0.0;
        for (long q = 0; q < N; ++q) sb += dout[co * N + q];
        if (db) db[co] = sb;
        for (int ci = 0; ci < cin; ++ci)
            for (int dz = -1; dz <= 1; ++dz)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dx = -1; dx <= 1; ++dx) {
                        double s = 0.0;
                        for (int k = 0; k < n; ++k)
                            for (int j = 0; j < n; ++j)
                                for (int i = 0; i < n; ++i)
                                    s += dout[co * N + idx3(n, i, j, k)]
                                       * in[ci * N + idx3(n, i + dx, j + dy, k + dz)];
                        dW[(((long)co * cin + ci) * 3 + dz + 1) * 9 + (dy + 1) * 3 + dx + 1] = s;
                    }
    }
}

/* GELU with the exact Gaussian CDF: g(x) = x * Phi(x). */
void orc_gelu(const double *x, long N, double *y)
{
    for (long q = 0; q < N; ++q)
        y[q] = 0.5 * x[q] * (1.0 + erf(x[q] / sqrt(2.0)));
}

/* dg/dx = Phi(x) + x * phi(x). */
void orc_gelu_grad(const double *x, long N, double *g)
{
    const double inv_sqrt_2pi = 1.0 / sqrt(2.0 * M_PI);
    for (long q = 0; q < N; ++q)
        g[q] = 0.5 * (1.0 + erf(x[q] / sqrt(2.0))) + x[q] * inv_sqrt_2pi * exp(-0.5 * x[q] * x[q]);
}
