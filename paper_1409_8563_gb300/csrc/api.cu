// api.cu -- the C ABI of include/parareal.h: context, workspace, and the
// orchestration of Parareal (Eq. parareal, Algorithm 1) on one GPU.
//
// HBM layout of a context (P = n^3, Pc = (n/r)^3, N = n_slices, T = the
// arithmetic type of F and G):
//   U      (N+1) x P  FP64   the iterate U^k[0..N]
//   Fv     (N+1) x P  T      Fv[n+1] = F(U^k[n]) of the current iteration
//   Gold   N pointers to P (r = 1, FP64) or Pc (r > 1, T) fields: G(U^k[n])
//   gspare one more such field: the newest G output, swapped into Gold
//   wA,wB  N x P      T      ping-pong state of the batched fine sweep
//   wC     N x P      T      (staged RK4 path only) RK4 accumulator
//   cA..cD            T      coarse-propagator state
//   wS     P          T      state of the serial fine run
//   tmpd   2P         FP64   host/device conversions, propagate() scratch
//   ref    P          FP64   u_fine(T) for the defect d^k (optional)
#include <algorithm>
#include <array>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "ctx.cuh"
#include "net.cuh"

using namespace pr;

thread_local std::string g_create_error;

parareal_status fail(parareal_ctx *c, parareal_status s, const std::string &msg)
{
    if (c) c->err = msg;
    else g_create_error = msg;
    return s;
}

static bool is_integer_ratio(double a, double b, long long *q)
{
    if (!(b > 0.0) || !(a > 0.0)) return false;
    const double x = a / b;
    const long long r = std::llround(x);
    if (r < 1 || std::fabs(x - (double)r) > 1e-9 * x) return false;
    *q = r;
    return true;
}

// Largest |R(dt lambda)| over Fourier modes and sampled nu: R the RK4
// polynomial (rk4) or 1 + z (forward Euler), lambda = nu L(k) + D(k) the
// symbol of the operator op on the periodic grid (every Fourier mode is an
// eigenvector of these circulant stencils).
static double step_growth(bool rk4, int op, int n, double dt, const double a[3], double nu_lo,
                          double nu_hi)
{
    const int stride = n <= 64 ? 1 : n / 64;
    using cplx = std::complex<double>;
    std::vector<double> L1(n);
    std::vector<cplx> D1[3];
    for (int ax = 0; ax < 3; ++ax) D1[ax].resize(n);
    const double hn = (double)n;   // 1/h
    for (int k = 0; k < n; ++k) {
        const double th = 2.0 * M_PI * k / n;
        const double c1 = std::cos(th), s1 = std::sin(th), c2 = std::cos(2 * th), s2 = std::sin(2 * th);
        // second difference per axis
        L1[k] = (op == OP_C4 ? (-2.0 * c2 + 32.0 * c1 - 30.0) / 12.0 : 2.0 * c1 - 2.0) * hn * hn;
        for (int ax = 0; ax < 3; ++ax) {
            // symbol of -a d/dx as discretised
            if (op == OP_C4)
                D1[ax][k] = cplx(0.0, -a[ax] * (8.0 * s1 - s2) / 6.0 * hn);
            else if (op == OP_C2)
                D1[ax][k] = cplx(0.0, -a[ax] * s1 * hn);
            else if (a[ax] > 0.0)   // (u - u_{-1})/h
                D1[ax][k] = -a[ax] * hn * cplx(1.0 - c1, s1);
            else                    // (u_{+1} - u)/h
                D1[ax][k] = -a[ax] * hn * cplx(c1 - 1.0, s1);
        }
    }
    double g = 0.0;
    const double nus[5] = {nu_lo, 0.75 * nu_lo + 0.25 * nu_hi, 0.5 * (nu_lo + nu_hi),
                           0.25 * nu_lo + 0.75 * nu_hi, nu_hi};
    auto scan = [&](int kx, int ky, int kz) {
        const double L = L1[kx] + L1[ky] + L1[kz];
        const cplx D = D1[0][kx] + D1[1][ky] + D1[2][kz];
        for (double nu : nus) {
            const cplx z = dt * (nu * L + D);
            const cplx R = rk4 ? 1.0 + z + z * z / 2.0 + z * z * z / 6.0 + z * z * z * z / 24.0
                               : 1.0 + z;
            g = std::max(g, std::abs(R));
        }
    };
    for (int kz = 0; kz < n; kz += stride)
        for (int ky = 0; ky < n; ky += stride)
            for (int kx = 0; kx < n; kx += stride) scan(kx, ky, kz);
    scan(n / 2, n / 2, n / 2);
    return g;
}

static parareal_status validate(const parareal_config *cfg, long long *Nf, long long *Nc,
                                std::string *msg)
{
    if (!cfg) { *msg = "null config"; return PARAREAL_E_INVALID; }
    if (cfg->n < 8 || cfg->n > 1024 || cfg->n % 4) { *msg = "n must be a multiple of 4 in 8..1024"; return PARAREAL_E_INVALID; }
    if (cfg->n_slices < 1 || cfg->n_slices > 4096) { *msg = "n_slices must be in 1..4096"; return PARAREAL_E_INVALID; }
    if (!(cfg->T > 0.0)) { *msg = "T must be positive"; return PARAREAL_E_INVALID; }
    if (cfg->coarse_factor < 1 || cfg->n % cfg->coarse_factor || cfg->n / cfg->coarse_factor < 4) {
        *msg = "coarse_factor must divide n and leave a coarse edge of at least 4";
        return PARAREAL_E_INVALID;
    }
    if (cfg->fine_dtype != PARAREAL_F32 && cfg->fine_dtype != PARAREAL_F64) { *msg = "fine_dtype"; return PARAREAL_E_INVALID; }
    if (cfg->nu_mode != PARAREAL_NU_STAGE && cfg->nu_mode != PARAREAL_NU_FROZEN) { *msg = "nu_mode"; return PARAREAL_E_INVALID; }
    if (cfg->coarse_kind < PARAREAL_COARSE_STENCIL || cfg->coarse_kind > PARAREAL_COARSE_EULER_UPWIND) { *msg = "coarse_kind"; return PARAREAL_E_INVALID; }
    if (cfg->coarse_kind == PARAREAL_COARSE_EULER_UPWIND && cfg->coarse_factor != 1) { *msg = "the Euler/upwind coarse propagator runs on the fine grid (coarse_factor 1)"; return PARAREAL_E_INVALID; }
    if (cfg->fine_scheme != PARAREAL_SCHEME_C2 && cfg->fine_scheme != PARAREAL_SCHEME_C4) { *msg = "fine_scheme"; return PARAREAL_E_INVALID; }
    if (cfg->learned_act != PARAREAL_ACT_GELU && cfg->learned_act != PARAREAL_ACT_LINEAR) { *msg = "learned_act"; return PARAREAL_E_INVALID; }
    if (cfg->correction_form != PARAREAL_CORRECTION_STANDARD && cfg->correction_form != PARAREAL_CORRECTION_DIFFERENCE) { *msg = "correction_form"; return PARAREAL_E_INVALID; }
    if (cfg->correction_form == PARAREAL_CORRECTION_DIFFERENCE && cfg->coarse_kind == PARAREAL_COARSE_LEARNED &&
        cfg->learned_act != PARAREAL_ACT_LINEAR) {
        *msg = "the difference form of the correction needs a linear coarse propagator";
        return PARAREAL_E_INVALID;
    }
    if (cfg->learned_skip != PARAREAL_SKIP_SHIFT && cfg->learned_skip != PARAREAL_SKIP_STENCIL) { *msg = "learned_skip"; return PARAREAL_E_INVALID; }
    if (cfg->learned_eval != PARAREAL_EVAL_LAYERS && cfg->learned_eval != PARAREAL_EVAL_COMPOSED &&
        cfg->learned_eval != PARAREAL_EVAL_POLYPHASE) { *msg = "learned_eval"; return PARAREAL_E_INVALID; }
    if (cfg->learned_eval != PARAREAL_EVAL_LAYERS && cfg->learned_act != PARAREAL_ACT_LINEAR) {
        *msg = "learned_eval COMPOSED / POLYPHASE needs learned_act LINEAR (a GELU network is not one convolution)";
        return PARAREAL_E_INVALID;
    }
    if (cfg->learned_eval == PARAREAL_EVAL_POLYPHASE && cfg->coarse_kind == PARAREAL_COARSE_LEARNED &&
        (cfg->learned_skip != PARAREAL_SKIP_STENCIL || (cfg->coarse_factor != 2 && cfg->coarse_factor != 4 &&
                                                        cfg->coarse_factor != 8) ||
         cfg->coarse_transfer != PARAREAL_TRANSFER_BOX || cfg->n % 16)) {
        *msg = "learned_eval POLYPHASE needs the stencil skip, coarse_factor 2, 4 or 8, box transfers and n a multiple of 16";
        return PARAREAL_E_INVALID;
    }
    if (cfg->coarse_transfer != PARAREAL_TRANSFER_BOX && cfg->coarse_transfer != PARAREAL_TRANSFER_SPECTRAL) { *msg = "coarse_transfer"; return PARAREAL_E_INVALID; }
    if (cfg->coarse_transfer == PARAREAL_TRANSFER_SPECTRAL) {
        if (cfg->coarse_kind != PARAREAL_COARSE_STENCIL || cfg->coarse_factor < 2) {
            *msg = "spectral transfers need the stencil coarse propagator on a coarsened grid";
            return PARAREAL_E_INVALID;
        }
        const size_t mat = (size_t)cfg->n * (cfg->n / cfg->coarse_factor) *
                           (cfg->fine_dtype == PARAREAL_F64 ? 8 : 4);
        if (mat > 160 * 1024) { *msg = "spectral transfer matrices larger than 160 KiB"; return PARAREAL_E_INVALID; }
    }
    if (cfg->pipeline_blocks < 0) { *msg = "pipeline_blocks < 0"; return PARAREAL_E_INVALID; }
    if (cfg->pipeline_blocks > 0 &&
        (cfg->fine_dtype != PARAREAL_F32 || cfg->fine_scheme != PARAREAL_SCHEME_C2 || cfg->n_slices < 2)) {
        *msg = "pipelined iterations need the FP32 fused fine sweep (F32, scheme C2) and n_slices >= 2";
        return PARAREAL_E_INVALID;
    }
    const double slice = cfg->T / cfg->n_slices;
    if (!is_integer_ratio(slice, cfg->dt_fine, Nf)) { *msg = "T/(n_slices dt_fine) must be an integer"; return PARAREAL_E_INVALID; }
    if (!is_integer_ratio(slice, cfg->dt_coarse, Nc)) { *msg = "T/(n_slices dt_coarse) must be an integer"; return PARAREAL_E_INVALID; }
    if (!(cfg->nu0 > 0.0) || !(std::fabs(cfg->nu_amp) < 1.0)) { *msg = "need nu0 > 0 and |nu_amp| < 1"; return PARAREAL_E_INVALID; }
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_stability(const parareal_config *cfg, double *growth2)
{
    long long Nf, Nc;
    std::string msg;
    parareal_status s = validate(cfg, &Nf, &Nc, &msg);
    if (s != PARAREAL_OK) return fail(nullptr, s, msg);
    const double lo = cfg->nu0 * (1.0 - std::fabs(cfg->nu_amp));
    const double hi = cfg->nu0 * (1.0 + std::fabs(cfg->nu_amp));
    const double gf = step_growth(true, cfg->fine_scheme == PARAREAL_SCHEME_C4 ? OP_C4 : OP_C2,
                                  cfg->n, cfg->dt_fine, cfg->a, lo, hi);
    double gc = 0.0;
    if (cfg->coarse_kind == PARAREAL_COARSE_EULER_UPWIND)
        gc = step_growth(false, OP_UPWIND, cfg->n, cfg->dt_coarse, cfg->a, lo, hi);
    else if (cfg->coarse_kind == PARAREAL_COARSE_STENCIL || cfg->learned_skip == PARAREAL_SKIP_STENCIL)
        gc = step_growth(true, OP_C2, cfg->n / cfg->coarse_factor, cfg->dt_coarse, cfg->a, lo, hi);
    if (growth2) { growth2[0] = gf; growth2[1] = gc; }
    if (gf > 1.0 + 1e-12 || gc > 1.0 + 1e-12) {
        g_create_error = "stability pre-check: per-step growth fine " + std::to_string(gf) +
                         ", coarse " + std::to_string(gc);
        return PARAREAL_E_UNSTABLE;
    }
    return PARAREAL_OK;
}

// Pick tile shapes: fused path for FP32 (bandwidth-bound; halo recompute is
// cheap), staged path for FP64 (FP64 throughput-bound; no recompute).
static void default_tiles(int dtype, int n, int count, int *path, int *tx, int *ty, int *zc)
{
    // FP64: no halo recomputation (the FP64 rate bounds the step); a small
    // batch is a few microseconds of work per stage, so one persistent launch
    // per sweep replaces four launches per step
    *path = dtype == PARAREAL_F64
                ? ((long long)count * n * n * n <= (1ll << 22) ? PATH_PERSIST : PATH_STAGED)
                : PATH_FUSED;
    const int cand[][2] = {{64, 16}, {32, 16}, {32, 8}, {16, 16}};
    const int candd[][2] = {{32, 8}, {16, 16}, {16, 8}};
    *tx = *ty = 0;
    // a tile that divides n; failing that (FP32), the one that wastes least
    if (dtype == PARAREAL_F32) {
        for (auto &t : cand)
            if (n % t[0] == 0 && n % t[1] == 0) { *tx = t[0]; *ty = t[1]; break; }
        if (*tx == 0) {
            long long best = -1;
            for (auto &t : cand) {
                const long long cover = (long long)((n + t[0] - 1) / t[0] * t[0]) * ((n + t[1] - 1) / t[1] * t[1]);
                if (best < 0 || cover < best) { best = cover; *tx = t[0]; *ty = t[1]; }
            }
        }
    } else {
        for (auto &t : candd)
            if (n % t[0] == 0 && n % t[1] == 0) { *tx = t[0]; *ty = t[1]; break; }
    }
    if (*tx == 0) { *path = *path == PATH_PERSIST ? PATH_PERSIST : PATH_STAGED; *tx = 16; *ty = 8; }
    // z chunk: whole columns unless the launch would leave SMs idle
    int z = n;
    while (z > 16 && (long long)count * (n / *tx) * (n / *ty) * ((n + z - 1) / z) < 2ll * sm_count()) z /= 2;
    *zc = z;
}

static bool tile_override(const char *var, int dtype, int n, int *path, int *tx, int *ty, int *zc)
{
    const char *e = std::getenv(var);
    if (!e || !*e) return true;
    int p, x, y, z;
    if (std::sscanf(e, "%d,%d,%d,%d", &p, &x, &y, &z) != 4) return false;
    if (!is_fused(p) && p != PATH_STAGED && p != PATH_PERSIST && p != PATH_CLUSTER) return false;
    if (is_fused(p) && (!rk4_fused_supported(dtype, n, x, y, fused_rows(p)) || z < 1)) return false;
    if (p == PATH_CLUSTER && rk4_cluster_size(dtype, n) == 0) return false;
    *path = p; *tx = x; *ty = y; *zc = z;
    return true;
}

// Record the start event of one timed launch (its stop event is the next in the pool).
static parareal_status prof_begin(parareal_ctx *c)
{
    while (c->ev_pool.size() < c->ev_used + 2) {
        cudaEvent_t e;
        CK(cudaEventCreate(&e));
        c->ev_pool.push_back(e);
    }
    CK(cudaEventRecord(c->ev_pool[c->ev_used], c->st));
    c->ev_used += 2;
    return PARAREAL_OK;
}

template <typename T>
parareal_status rk4_batch(parareal_ctx *c, int m, const T *in, T *out, int first_slice, int count,
                          long long nsteps, double dt, int path, int tx, int ty, int zc, T *ws1,
                          T *ws2, T *ws3, int slice_stride, int op, const int *cancel)
{
    if (is_fused(path) && op != OP_C2)
        return fail(c, PARAREAL_E_INVALID, "the fused RK4 kernel implements the 7-point operator only");
    StepArgs a{};
    a.op = op;
    a.n = m;
    a.P = (long long)m * m * m;
    a.count = count;
    a.first_slice = first_slice;
    a.slice_stride = slice_stride;
    a.steps_per_slice = nsteps;
    a.dt = dt;
    for (int d = 0; d < 3; ++d) a.a[d] = c->cfg.a[d];
    a.nu0 = c->cfg.nu0;
    a.nu_amp = c->cfg.nu_amp;
    a.nu_omega = c->cfg.nu_omega;
    a.frozen = c->cfg.nu_mode == PARAREAL_NU_FROZEN;
    a.cancel = cancel;
    if (is_fused(path)) {
        const T *src = in;
        const bool timed = c->prof && m == c->n;
        for (long long j = 0; j < nsteps; ++j) {
            T *dst = (j == nsteps - 1) ? out : ((j & 1) ? ws2 : ws1);
            a.j = j;
            if (timed) {
                parareal_status ps = prof_begin(c);
                if (ps != PARAREAL_OK) return ps;
            }
            LK((launch_rk4_fused<T>(a, src, dst, tx, ty, zc, fused_rows(path), c->st)));
            if (timed) {
                CK(cudaEventRecord(c->ev_pool[c->ev_used - 1], c->st));
                c->prof_bytes += 2.0 * (double)count * (double)a.P * sizeof(T);
                c->prof_launches++;
            }
            src = dst;
        }
    } else if (path == PATH_CLUSTER) {
        if (op_radius(op) != 1)
            return fail(c, PARAREAL_E_INVALID, "the cluster RK4 kernel implements radius-1 operators only");
        LK(launch_rk4_cluster<T>(a, in, out, nsteps, c->st));
    } else if (path == PATH_PERSIST) {
        if (in != out)
            CK(cudaMemcpyAsync(out, in, (size_t)count * a.P * sizeof(T), cudaMemcpyDeviceToDevice, c->st));
        LK(launch_rk4_persist<T>(a, out, ws1, ws2, ws3, nsteps, c->bar, c->st));
        c->persist_used = true;
    } else {
        if (in != out)
            CK(cudaMemcpyAsync(out, in, (size_t)count * a.P * sizeof(T), cudaMemcpyDeviceToDevice, c->st));
        for (long long j = 0; j < nsteps; ++j) {
            a.j = j;
            LK(launch_rk4_stage<T>(a, 1, out, out, ws1, ws3, c->st));
            LK(launch_rk4_stage<T>(a, 2, ws1, out, ws2, ws3, c->st));
            LK(launch_rk4_stage<T>(a, 3, ws2, out, ws1, ws3, c->st));
            LK(launch_rk4_stage<T>(a, 4, ws1, out, nullptr, ws3, c->st));
        }
    }
    return PARAREAL_OK;
}

template parareal_status rk4_batch<float>(parareal_ctx *, int, const float *, float *, int, int,
                                          long long, double, int, int, int, int, float *, float *,
                                          float *, int, int, const int *);
template parareal_status rk4_batch<double>(parareal_ctx *, int, const double *, double *, int, int,
                                           long long, double, int, int, int, int, double *,
                                           double *, double *, int, int, const int *);

template <typename T>
parareal_status euler_batch(parareal_ctx *c, int m, const T *in, T *out, int first_slice,
                            int count, long long nsteps, double dt, int op, T *ws1, T *ws2)
{
    StepArgs a{};
    a.op = op;
    a.n = m;
    a.P = (long long)m * m * m;
    a.count = count;
    a.first_slice = first_slice;
    a.slice_stride = 1;
    a.steps_per_slice = nsteps;
    a.dt = dt;
    for (int d = 0; d < 3; ++d) a.a[d] = c->cfg.a[d];
    a.nu0 = c->cfg.nu0;
    a.nu_amp = c->cfg.nu_amp;
    a.nu_omega = c->cfg.nu_omega;
    a.frozen = 1;
    if (nsteps == 0) {
        if (in != out)
            CK(cudaMemcpyAsync(out, in, (size_t)count * a.P * sizeof(T), cudaMemcpyDeviceToDevice, c->st));
        return PARAREAL_OK;
    }
    // ping-pong between the two workspaces, the last step written to out; a
    // step never reads the buffer it writes
    const T *src = in;
    if (in == out || in == ws1) {
        CK(cudaMemcpyAsync(ws2, in, (size_t)count * a.P * sizeof(T), cudaMemcpyDeviceToDevice, c->st));
        src = ws2;
    }
    for (long long j = 0; j < nsteps; ++j) {
        T *dst = (j == nsteps - 1) ? out : ((j & 1) ? ws2 : ws1);
        a.j = j;
        LK(launch_rk4_stage<T>(a, 0, src, nullptr, dst, nullptr, c->st));
        src = dst;
    }
    return PARAREAL_OK;
}
template parareal_status euler_batch<float>(parareal_ctx *, int, const float *, float *, int, int,
                                            long long, double, int, float *, float *);
template parareal_status euler_batch<double>(parareal_ctx *, int, const double *, double *, int,
                                             int, long long, double, int, double *, double *);

// ------------------------------------------------------------ propagators

// fvb[s+1] = F(U[s]) for s in [first, first+count) on c->st, in the given
// launch shape.  conv (if set) is recorded once U has been read; cancel as in
// StepArgs.
template <typename T>
static parareal_status fine_sweep_range(parareal_ctx *c, int first, int count, void *fvb, int path,
                                        int tx, int ty, int zc, cudaEvent_t conv, const int *cancel)
{
    const long long P = c->P;
    T *Fv = static_cast<T *>(fvb) + (long long)(first + 1) * P;
    const T *in;
    if (std::is_same<T, float>::value) {
        LK(launch_convert_f64_to_f32(c->U + (long long)first * P, reinterpret_cast<float *>(c->wC ? c->wC : c->wA),
                                     (long long)count * P, c->st));
        in = static_cast<const T *>(c->wC ? c->wC : c->wA);
    } else {
        in = reinterpret_cast<const T *>(c->U + (long long)first * P);
    }
    if (conv) CK(cudaEventRecord(conv, c->st));
    // the fused path must not read and write the same buffer
    T *ws1 = static_cast<T *>(c->wA), *ws2 = static_cast<T *>(c->wB), *ws3 = static_cast<T *>(c->wC);
    if (is_fused(path) && in == ws1) std::swap(ws1, ws3);
    return rk4_batch<T>(c, c->n, in, Fv, first, count, c->Nf, c->cfg.dt_fine, path, tx, ty, zc, ws1,
                        ws2, ws3, 1, c->fine_op, cancel);
}

// F(U^k[s]) into fv_of(k)[s+1] for s in [first, first+count), k = k_total.
template <typename T>
static parareal_status fine_sweep_t(parareal_ctx *c, int first, int count)
{
    c->spec_valid = false;
    return fine_sweep_range<T>(c, first, count, fv_of(c, c->k_total), c->fine_path, c->fine_tx,
                               c->fine_ty, c->fine_zc, nullptr, nullptr);
}

// The stencil coarse propagator of slice s on the fine grid, in FP64: RK4 on
// the grid coarsened by r (box restriction before, trilinear prolongation
// after) or on the fine grid itself when r = 1.
template <typename T>
static parareal_status stencil_g_fine_t(parareal_ctx *c, const double *u, int s, double *out)
{
    T *cA = static_cast<T *>(c->cA), *cB = static_cast<T *>(c->cB), *cC = static_cast<T *>(c->cC),
      *cD = static_cast<T *>(c->cD);
    parareal_status ps;
    if (c->r > 1) {
        LK(launch_restrict<T>(u, c->n, c->r, cA, c->st));
        ps = rk4_batch<T>(c, c->nc, cA, cB, s, 1, c->Nc, c->cfg.dt_coarse, c->coarse_path,
                          c->coarse_tx, c->coarse_ty, c->coarse_zc, cC, cD, cA);
        if (ps != PARAREAL_OK) return ps;
        // prolongation of the coarse result (the correction kernel with no
        // fine value and no old coarse value writes exactly that)
        LK((launch_correct<T, T>(nullptr, cB, nullptr, out, c->n, c->r, c->partials, c->nblk, c->st)));
        return PARAREAL_OK;
    }
    if (std::is_same<T, float>::value) {
        LK(launch_convert_f64_to_f32(u, reinterpret_cast<float *>(cA), c->P, c->st));
        ps = rk4_batch<T>(c, c->n, cA, cB, s, 1, c->Nc, c->cfg.dt_coarse, c->coarse_path,
                          c->coarse_tx, c->coarse_ty, c->coarse_zc, cC, cD, cA);
        if (ps != PARAREAL_OK) return ps;
        LK(launch_convert_f32_to_f64(reinterpret_cast<const float *>(cB), out, c->P, c->st));
        return PARAREAL_OK;
    }
    return rk4_batch<T>(c, c->n, reinterpret_cast<const T *>(u), reinterpret_cast<T *>(out), s, 1,
                        c->Nc, c->cfg.dt_coarse, c->coarse_path, c->coarse_tx, c->coarse_ty,
                        c->coarse_zc, cB, cC, cD);
}

parareal_status stencil_g_fine(parareal_ctx *c, const double *u, int s, double *out)
{
    return c->f64 ? stencil_g_fine_t<double>(c, u, s, out) : stencil_g_fine_t<float>(c, u, s, out);
}

// G(U_in) for slice s into `out` (Pc T fields when G's output is coarse,
// else P doubles).
template <typename T>
static parareal_status coarse_apply_t(parareal_ctx *c, const double *Uin, int s, void *out)
{
    T *cA = static_cast<T *>(c->cA), *cB = static_cast<T *>(c->cB), *cC = static_cast<T *>(c->cC),
      *cD = static_cast<T *>(c->cD);
    if (c->cfg.coarse_kind == PARAREAL_COARSE_EULER_UPWIND) {
        // forward Euler / upwind (Algorithm 2) on the fine grid, FP64 out
        if (std::is_same<T, float>::value) {
            LK(launch_convert_f64_to_f32(Uin, reinterpret_cast<float *>(cA), c->P, c->st));
            parareal_status ps = euler_batch<T>(c, c->n, cA, cB, s, 1, c->Nc, c->cfg.dt_coarse,
                                                OP_UPWIND, cC, cD);
            if (ps != PARAREAL_OK) return ps;
            LK(launch_convert_f32_to_f64(reinterpret_cast<const float *>(cB), static_cast<double *>(out), c->P, c->st));
            return PARAREAL_OK;
        }
        return euler_batch<T>(c, c->n, reinterpret_cast<const T *>(Uin), static_cast<T *>(out), s, 1,
                              c->Nc, c->cfg.dt_coarse, OP_UPWIND, cB, cC);
    }
    // the phase-kernel learned G: its coarse part is the stencil propagator's
    if (c->cfg.coarse_kind != PARAREAL_COARSE_STENCIL && !c->net.poly) {
        if (c->cfg.learned_skip == PARAREAL_SKIP_STENCIL) {
            // the net corrects the stencil propagator's output on the fine grid
            double *gs = c->tmpd + c->P;
            parareal_status ps = stencil_g_fine(c, Uin, s, gs);
            if (ps != PARAREAL_OK) return ps;
            return net_apply<double, double>(c, gs, s, static_cast<double *>(out));
        }
        // shift + convolution net, on the fine grid or on the restricted grid
        if (c->r == 1) return net_apply<double, double>(c, Uin, s, static_cast<double *>(out));
        LK(launch_restrict<T>(Uin, c->n, c->r, cA, c->st));
        return net_apply<T, T>(c, cA, s, static_cast<T *>(out));
    }
    if (c->r > 1) {
        if (c->spectral) {
            LK(launch_restrict_spectral<T>(Uin, c->n, c->r, static_cast<const T *>(c->sp_R),
                                           static_cast<const T *>(c->sp_Rt), static_cast<T *>(c->sp_work),
                                           cA, c->st));
        } else {
            LK(launch_restrict<T>(Uin, c->n, c->r, cA, c->st));
        }
        return rk4_batch<T>(c, c->nc, cA, static_cast<T *>(out), s, 1, c->Nc, c->cfg.dt_coarse,
                            c->coarse_path, c->coarse_tx, c->coarse_ty, c->coarse_zc, cB, cC, cD);
    }
    if (std::is_same<T, float>::value) {
        LK(launch_convert_f64_to_f32(Uin, reinterpret_cast<float *>(cA), c->P, c->st));
        parareal_status ps = rk4_batch<T>(c, c->n, cA, cB, s, 1, c->Nc, c->cfg.dt_coarse,
                                          c->coarse_path, c->coarse_tx, c->coarse_ty, c->coarse_zc,
                                          cC, cD, cA);
        if (ps != PARAREAL_OK) return ps;
        LK(launch_convert_f32_to_f64(reinterpret_cast<const float *>(cB), static_cast<double *>(out), c->P, c->st));
        return PARAREAL_OK;
    }
    return rk4_batch<T>(c, c->n, reinterpret_cast<const T *>(Uin), static_cast<T *>(out), s, 1,
                        c->Nc, c->cfg.dt_coarse, c->coarse_path, c->coarse_tx, c->coarse_ty,
                        c->coarse_zc, cB, cC, cD);
}

// The correction with a coarse-grid G: U[p] <- Fv[p] + P(cnew - cold)[p]
// (trilinear inside the correction kernel, or the spectral prolongation into
// a fine T field first).  Fv / cold may be null.
template <typename T>
static parareal_status correct_coarse(parareal_ctx *c, int s, const T *Fv, const T *cnew, const T *cold,
                                      double *U, double *dU)
{
    if (c->net.poly) {
        // the learned G's change through slice s's phase kernels
        T *fine = static_cast<T *>(c->sp_fine);
        LK(launch_poly_prolong<T>(cnew, cold, c->net.wpoly + poly_weights_floats(c->r, s), c->n, c->r, fine,
                                  c->st));
        LK((launch_correct<T, T>(Fv, fine, nullptr, U, c->n, 1, c->partials, c->nblk, c->st, dU)));
        return PARAREAL_OK;
    }
    if (!c->spectral) {
        LK((launch_correct<T, T>(Fv, cnew, cold, U, c->n, c->r, c->partials, c->nblk, c->st, dU)));
        return PARAREAL_OK;
    }
    T *fine = static_cast<T *>(c->sp_fine);
    LK(launch_prolong_spectral<T>(cnew, cold, c->n, c->r, static_cast<const T *>(c->sp_P),
                                  static_cast<const T *>(c->sp_Pt), static_cast<T *>(c->sp_work), fine,
                                  c->st));
    LK((launch_correct<T, T>(Fv, fine, nullptr, U, c->n, 1, c->partials, c->nblk, c->st, dU)));
    return PARAREAL_OK;
}

// U[s+1] <- Fv[s+1] + (gnew - gold) with norms into slice_norms[s+1].
// Fv / gold may be null (read as zero).
template <typename T>
static parareal_status correct_t(parareal_ctx *c, int s, const void *gnew, const void *gold,
                                 bool with_fine, double *dU = nullptr)
{
    const T *Fv = with_fine ? static_cast<const T *>(fv_of(c, c->k_total)) + (long long)(s + 1) * c->P
                            : nullptr;
    double *U = c->U + (long long)(s + 1) * c->P;
    if (!c->g_fine) {
        parareal_status ps = correct_coarse<T>(c, s, Fv, static_cast<const T *>(gnew),
                                               static_cast<const T *>(gold), U, dU);
        if (ps != PARAREAL_OK) return ps;
    } else {
        LK((launch_correct<T, double>(Fv, static_cast<const double *>(gnew),
                                      static_cast<const double *>(gold), U, c->n, 1, c->partials,
                                      c->nblk, c->st, dU)));
    }
    LK(launch_reduce_partials(c->partials, c->nblk, c->slice_norms + 5ll * (s + 1), c->st));
    return PARAREAL_OK;
}

#define DISPATCH(c, fn, ...) ((c)->f64 ? fn<double>(c, __VA_ARGS__) : fn<float>(c, __VA_ARGS__))

// Serial coarse start-up (Algorithm 1, initialisation) for slices first..first+count-1.
static parareal_status coarse_chain(parareal_ctx *c, int first, int count, bool chain)
{
    for (int s = first; s < first + count; ++s) {
        void *g = g_next(c, s + 1);
        parareal_status ps = DISPATCH(c, coarse_apply_t, c->U + (long long)s * c->P, s, g);
        if (ps != PARAREAL_OK) return ps;
        if (chain) {
            ps = DISPATCH(c, correct_t, s, g, nullptr, false);
            if (ps != PARAREAL_OK) return ps;
        }
        c->gcur[s + 1] ^= 1;
    }
    return PARAREAL_OK;
}

// F(U^k[n]) of the open slices n = k_total..N-1 into fv_of(k_total), on c->st.
parareal_status fine_sweep_open(parareal_ctx *c)
{
    return DISPATCH(c, fine_sweep_t, c->k_total, c->N - c->k_total);
}

parareal_status pipe_join(parareal_ctx *c)
{
    if (!c->st_f) return PARAREAL_OK;
    CK(cudaEventRecord(c->ev_join, c->st_f));
    CK(cudaStreamWaitEvent(c->st, c->ev_join, 0));
    return PARAREAL_OK;
}

namespace {

// The speculative sweep of one iteration (pipelined iterations): F(U^{k+1}[n])
// for n in [K+1, N), in blocks launched on st_f as the chain finalises them.
struct PipeSpec {
    parareal_ctx *c;
    int p = 0;                 // parity of K+1: the buffers and events it fills
    int nb = 0;                // number of blocks (0: nothing to speculate)
    int next = 0;              // next block to launch

    PipeSpec(parareal_ctx *cc, int K) : c(cc)
    {
        const int cnt = c->N - (K + 1);
        if (!c->Fv2 || cnt <= 0) return;
        nb = std::min(c->cfg.pipeline_blocks, cnt);
        p = (K + 1) & 1;
        c->spec_lo[p].assign(nb, 0);
        c->spec_hi[p].assign(nb, 0);
        for (int j = 0; j < nb; ++j) {
            c->spec_lo[p][j] = K + 1 + (int)((long long)j * cnt / nb);
            c->spec_hi[p][j] = K + 1 + (int)((long long)(j + 1) * cnt / nb);
        }
    }

    // After the correction that made U[m] final: launch every block whose
    // last slice is m.
    parareal_status after_final(int m)
    {
        while (next < nb && c->spec_hi[p][next] - 1 == m) {
            parareal_status s = launch(next);
            if (s != PARAREAL_OK) return s;
            ++next;
        }
        return PARAREAL_OK;
    }

    parareal_status launch(int j)
    {
        CK(cudaEventRecord(c->ev_fork, c->st));
        CK(cudaStreamWaitEvent(c->st_f, c->ev_fork, 0));
        if (j == 0) CK(cudaMemsetAsync(c->cancel, 0, sizeof(int), c->st_f));
        const int lo = c->spec_lo[p][j], hi = c->spec_hi[p][j];
        const cudaStream_t main_st = c->st;
        c->st = c->st_f;
        parareal_status s = fine_sweep_range<float>(c, lo, hi - lo, fv_of(c, p), c->pipe_path,
                                                    c->pipe_tx, c->pipe_ty, c->pipe_zc,
                                                    c->ev_conv[p][j], c->cancel);
        c->st = main_st;
        if (s != PARAREAL_OK) return s;
        CK(cudaEventRecord(c->ev_done[p][j], c->st_f));
        return PARAREAL_OK;
    }
};

// Waits of an iteration's chain on the speculative sweep that produced its
// Fv (host loop, events recorded by the previous enqueue).
struct PipeWait {
    parareal_ctx *c;
    int p = 0, nb = 0;
    int done_upto = -1, conv_upto = -1;   // blocks already waited on

    PipeWait(parareal_ctx *cc, int K, bool active) : c(cc)
    {
        if (!active) return;
        p = K & 1;
        nb = (int)c->spec_lo[p].size();
    }

    int block_of(int s) const
    {
        for (int j = 0; j < nb; ++j)
            if (s >= c->spec_lo[p][j] && s < c->spec_hi[p][j]) return j;
        return -1;
    }

    // Before the correction of chain step n (reads Fv[n+1] = F(U[n]), writes U[n+1]).
    parareal_status before_step(int n)
    {
        if (nb == 0) return PARAREAL_OK;
        const int jd = block_of(n);
        for (; jd >= 0 && done_upto < jd; ++done_upto) CK(cudaStreamWaitEvent(c->st, c->ev_done[p][done_upto + 1], 0));
        const int jc = block_of(n + 1);
        for (; jc >= 0 && conv_upto < jc; ++conv_upto) CK(cudaStreamWaitEvent(c->st, c->ev_conv[p][conv_upto + 1], 0));
        return PARAREAL_OK;
    }
};

}  // namespace

// Device work of one Parareal iteration (Algorithm 1 loop body for every
// open slice), enqueued on c->st without any host synchronisation:
// fine sweep of slices K..N-1, then the serial coarse sweep with the
// correction and per-slice norms, then (with a reference) the defect norms
// into slot N+1 of slice_norms.  K = c->k_total: U[0..K] are already exact.
// with_fine = false leaves out the fine sweep (the caller has put F(U^k[n])
// into Fv[n+1] another way); copy_norms = false leaves the norms on the device.
//
// Pipelined iterations: the fine sweep of this iteration was started by the
// previous one (or runs here when it was not), and this iteration starts the
// next one's, F(U^{k+1}[n]) into fv_of(K+1), block by block on st_f right
// after the correction that makes a block's last slice final.  The chain
// waits for a block of the previous speculation before it reads the block's
// F values and before it overwrites the U values the block reads.
parareal_status iter_enqueue(parareal_ctx *c, bool copy_norms, bool with_fine, bool capture,
                             void (*stop_eval)(parareal_ctx *, void *), void *stop_arg)
{
    const int K = c->k_total;
    const bool pipe = c->Fv2 != nullptr;
    parareal_status s = PARAREAL_OK;
    // a graph body assumes the speculative Fv of its iteration (the host
    // provides it before the first body)
    const bool have_fv = pipe && (capture || c->spec_valid);
    if (with_fine && !have_fv) {
        s = fine_sweep_open(c);
        if (s != PARAREAL_OK) return s;
    }
    PipeWait wait(c, K, pipe && !capture && c->spec_valid && c->spec_events);
    PipeSpec spec(c, K);
    auto step_done = [&](int n) -> parareal_status {     // U[n+1] is final
        return spec.after_final(n + 1);
    };
    if (c->cfg.correction_form == PARAREAL_CORRECTION_DIFFERENCE) {
        // U[n+1] = Fv[n+1] + G(D_n), D_n = U^{k+1}[n] - U^k[n] (G linear); the
        // correction of slice n writes D_{n+1}.  D_K = 0: slice K+1 takes Fv alone.
        double *Din = c->dA, *Dout = c->dB;
        if ((s = wait.before_step(K)) != PARAREAL_OK) return s;
        s = DISPATCH(c, correct_t, K, g_cur(c, K + 1), g_cur(c, K + 1), true, Din);
        if (s != PARAREAL_OK) return s;
        if ((s = step_done(K)) != PARAREAL_OK) return s;
        for (int n = K + 1; n < c->N; ++n) {
            s = DISPATCH(c, coarse_apply_t, Din, n, c->gspare);
            if (s != PARAREAL_OK) return s;
            if ((s = wait.before_step(n)) != PARAREAL_OK) return s;
            s = DISPATCH(c, correct_t, n, c->gspare, nullptr, true, Dout);
            if (s != PARAREAL_OK) return s;
            if ((s = step_done(n)) != PARAREAL_OK) return s;
            std::swap(Din, Dout);
        }
    } else {
        // slice K+1: its input U[K] did not change, so G's difference is zero
        if ((s = wait.before_step(K)) != PARAREAL_OK) return s;
        s = DISPATCH(c, correct_t, K, g_cur(c, K + 1), g_cur(c, K + 1), true);
        if (s != PARAREAL_OK) return s;
        if ((s = step_done(K)) != PARAREAL_OK) return s;
        for (int n = K + 1; n < c->N; ++n) {
            void *g = g_next(c, n + 1);
            s = DISPATCH(c, coarse_apply_t, c->U + (long long)n * c->P, n, g);
            if (s != PARAREAL_OK) return s;
            if ((s = wait.before_step(n)) != PARAREAL_OK) return s;
            s = DISPATCH(c, correct_t, n, g, g_cur(c, n + 1), true);
            if (s != PARAREAL_OK) return s;
            if ((s = step_done(n)) != PARAREAL_OK) return s;
            c->gcur[n + 1] ^= 1;
        }
    }
    if (c->has_ref) {
        LK(launch_diff_norms<double>(c->U + (long long)c->N * c->P, c->ref, c->P, c->partials, c->nblk, c->st));
        LK(launch_reduce_partials(c->partials, c->nblk, c->slice_norms + 5ll * (c->N + 1), c->st));
    }
    c->spec_pending = spec.nb > 0;
    if (pipe && capture && spec.nb > 0) {
        // inside a graph body: decide on the device whether the speculative
        // sweep is still needed, then join its branch
        if (stop_eval) stop_eval(c, stop_arg);
        s = pipe_join(c);
        if (s != PARAREAL_OK) return s;
    }
    if (copy_norms)
        CK(cudaMemcpyAsync(c->h_norms, c->slice_norms, sizeof(double) * 5 * (c->N + 2),
                           cudaMemcpyDeviceToHost, c->st));
    return PARAREAL_OK;
}

// Host side of one iteration, after c->st has been synchronised: per-slice
// and maximal relative changes, the defect (or -1), NaN/Inf detection.
parareal_status iter_finish(parareal_ctx *c, double *dmax, double *l2max, double *d)
{
    const int K = c->k_total;
    *dmax = 0.0;
    *l2max = 0.0;
    for (int s = 0; s <= c->N; ++s) {
        if (s < K + 1) { c->diff_inf[s] = 0.0; c->diff_l2[s] = 0.0; continue; }
        const double *q = c->h_norms + 5 * s;
        if (q[4] != 0.0) return fail(c, PARAREAL_E_DIVERGED, "non-finite value in slice " + std::to_string(s));
        c->diff_inf[s] = q[1] > 0 ? q[0] / q[1] : q[0];
        c->diff_l2[s] = q[3] > 0 ? std::sqrt(q[2] / q[3]) : std::sqrt(q[2]);
        *dmax = std::max(*dmax, c->diff_inf[s]);
        *l2max = std::max(*l2max, c->diff_l2[s]);
    }
    *d = -1.0;
    if (c->has_ref) {
        const double *q = c->h_norms + 5 * (c->N + 1);
        if (q[4] != 0.0) return fail(c, PARAREAL_E_DIVERGED, "non-finite value in the last slice");
        *d = q[1] > 0 ? q[0] / q[1] : q[0];
    }
    c->k_total++;
    return PARAREAL_OK;
}

static parareal_status defect(parareal_ctx *c, double *d)
{
    LK(launch_diff_norms<double>(c->U + (long long)c->N * c->P, c->ref, c->P, c->partials, c->nblk, c->st));
    LK(launch_reduce_partials(c->partials, c->nblk, c->slice_norms + 5ll * (c->N + 1), c->st));
    double h[5];
    CK(cudaMemcpyAsync(h, c->slice_norms + 5ll * (c->N + 1), sizeof h, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (h[4] != 0.0) return fail(c, PARAREAL_E_DIVERGED, "non-finite value in the last slice");
    *d = h[1] > 0 ? h[0] / h[1] : h[0];
    return PARAREAL_OK;
}

// ------------------------------------------------------------------- ABI

extern "C" parareal_status parareal_create(const parareal_config *cfg, void *stream,
                                           parareal_ctx **out)
{
    if (!out) return fail(nullptr, PARAREAL_E_INVALID, "null out");
    *out = nullptr;
    long long Nf, Nc;
    std::string msg;
    parareal_status s = validate(cfg, &Nf, &Nc, &msg);
    if (s != PARAREAL_OK) return fail(nullptr, s, msg);
    double growth[2];
    parareal_status warn = PARAREAL_OK;
    if (parareal_stability(cfg, growth) == PARAREAL_E_UNSTABLE) {
        if (!cfg->allow_unstable) return PARAREAL_E_UNSTABLE;
        warn = PARAREAL_W_MARGINAL;
    }
    {
        // shared-memory opt-ins, once per device and process
        static std::vector<int> configured;
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess) return fail(nullptr, PARAREAL_E_CUDA, "no CUDA device");
        if (std::find(configured.begin(), configured.end(), dev) == configured.end()) {
            if (configure_rk4_kernels() != cudaSuccess || configure_spectral_kernels() != cudaSuccess ||
                configure_queue_kernels() != cudaSuccess || configure_cluster_kernels() != cudaSuccess)
                return fail(nullptr, PARAREAL_E_CUDA, "kernel configuration failed");
            configured.push_back(dev);
        }
    }
    parareal_ctx *c = new parareal_ctx();
    c->cfg = *cfg;
    c->st = static_cast<cudaStream_t>(stream);
    c->n = cfg->n;
    c->N = cfg->n_slices;
    c->r = cfg->coarse_factor;
    c->nc = c->n / c->r;
    c->P = (long long)c->n * c->n * c->n;
    c->Pc = (long long)c->nc * c->nc * c->nc;
    c->Nf = Nf;
    c->Nc = Nc;
    c->f64 = cfg->fine_dtype == PARAREAL_F64;
    c->esz = c->f64 ? 8 : 4;
    c->diff_inf.assign(c->N + 1, 0.0);
    c->diff_l2.assign(c->N + 1, 0.0);
    default_tiles(cfg->fine_dtype, c->n, c->N, &c->fine_path, &c->fine_tx, &c->fine_ty, &c->fine_zc);
    default_tiles(cfg->fine_dtype, c->n, 1, &c->ser_path, &c->ser_tx, &c->ser_ty, &c->ser_zc);
    default_tiles(cfg->fine_dtype, c->nc, 1, &c->coarse_path, &c->coarse_tx, &c->coarse_ty, &c->coarse_zc);
    // explicit launch shapes ("path,tile_x,tile_y,zchunk"), e.g. from the autotuner
    if (!tile_override("PARAREAL_FINE_TILE", cfg->fine_dtype, c->n, &c->fine_path, &c->fine_tx,
                       &c->fine_ty, &c->fine_zc) ||
        !tile_override("PARAREAL_SERIAL_TILE", cfg->fine_dtype, c->n, &c->ser_path, &c->ser_tx,
                       &c->ser_ty, &c->ser_zc) ||
        !tile_override("PARAREAL_COARSE_TILE", cfg->fine_dtype, c->nc, &c->coarse_path,
                       &c->coarse_tx, &c->coarse_ty, &c->coarse_zc)) {
        delete c;
        return fail(nullptr, PARAREAL_E_INVALID, "unsupported launch shape override");
    }
    // pipelined: no cooperative persistent launch beside the side stream's sweep
    if (cfg->pipeline_blocks > 0 && c->coarse_path == PATH_PERSIST) c->coarse_path = PATH_STAGED;
    c->fine_op = cfg->fine_scheme == PARAREAL_SCHEME_C4 ? OP_C4 : OP_C2;
    if (c->fine_op != OP_C2) {
        // the fused kernels implement the 7-point operator only
        if (is_fused(c->fine_path)) c->fine_path = PATH_STAGED;
        if (is_fused(c->ser_path)) c->ser_path = PATH_STAGED;
    }

    auto alloc = [&](void **p, size_t bytes) -> bool {
        if (cudaMalloc(p, bytes) != cudaSuccess) { cudaGetLastError(); *p = nullptr; return false; }
        return true;
    };
    const size_t e = c->esz;
    const size_t P = (size_t)c->P, Pc = (size_t)c->Pc, N = (size_t)c->N;
    // G's output: a coarse T field when G ends on the coarse grid (stencil G,
    // or a net on the restricted grid), else a fine FP64 field
    const bool poly = cfg->coarse_kind == PARAREAL_COARSE_LEARNED && cfg->learned_eval == PARAREAL_EVAL_POLYPHASE;
    c->g_fine = c->r == 1 || (cfg->coarse_kind != PARAREAL_COARSE_STENCIL &&
                              cfg->learned_skip == PARAREAL_SKIP_STENCIL && !poly);
    const size_t gbytes = c->g_fine ? P * sizeof(double) : Pc * e;
    bool ok = cudaGetDevice(&c->dev) == cudaSuccess;
    ok = ok && alloc((void **)&c->U, (N + 1) * P * sizeof(double));
    ok = ok && alloc(&c->Fv, (N + 1) * P * e);
    if (cfg->pipeline_blocks > 0) {
        // the second F buffer, the side stream (lowest priority: the serial
        // chain on the context's stream goes first), the cancel flag, events
        int lo = 0, hi = 0;
        ok = ok && alloc(&c->Fv2, (N + 1) * P * e) && alloc((void **)&c->cancel, sizeof(int)) &&
             cudaMemset(c->cancel, 0, sizeof(int)) == cudaSuccess &&
             cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess &&
             cudaStreamCreateWithPriority(&c->st_f, cudaStreamNonBlocking, lo) == cudaSuccess &&
             cudaStreamCreateWithPriority(&c->st_hi, cudaStreamNonBlocking, hi) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_in, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&c->ev_out, cudaEventDisableTiming) == cudaSuccess;
        const int nb = std::min(cfg->pipeline_blocks, c->N - 1);
        for (int p = 0; p < 2 && ok; ++p) {
            c->ev_conv[p].assign(nb, nullptr);
            c->ev_done[p].assign(nb, nullptr);
            for (int j = 0; j < nb && ok; ++j)
                ok = cudaEventCreateWithFlags(&c->ev_conv[p][j], cudaEventDisableTiming) == cudaSuccess &&
                     cudaEventCreateWithFlags(&c->ev_done[p][j], cudaEventDisableTiming) == cudaSuccess;
        }
        // launch shape of a block: the fused shape for its slice count
        default_tiles(PARAREAL_F32, c->n, (c->N - 1 + nb - 1) / nb, &c->pipe_path, &c->pipe_tx,
                      &c->pipe_ty, &c->pipe_zc);
        if (!is_fused(c->pipe_path)) { c->pipe_path = c->fine_path; c->pipe_tx = c->fine_tx; c->pipe_ty = c->fine_ty; c->pipe_zc = c->fine_zc; }
        ok = ok && tile_override("PARAREAL_PIPE_TILE", PARAREAL_F32, c->n, &c->pipe_path, &c->pipe_tx,
                                 &c->pipe_ty, &c->pipe_zc) && is_fused(c->pipe_path);
    }
    c->gold.assign(N + 1, nullptr);
    c->gold2.assign(N + 1, nullptr);
    c->gcur.assign(N + 1, 0);
    for (size_t i = 1; ok && i <= N; ++i) ok = alloc(&c->gold[i], gbytes) && alloc(&c->gold2[i], gbytes);
    ok = ok && alloc(&c->gspare, gbytes);
    ok = ok && alloc(&c->wA, N * P * e) && alloc(&c->wB, N * P * e) && alloc(&c->wC, N * P * e);
    const size_t cbytes = (c->r > 1 ? Pc : P) * e;
    ok = ok && alloc(&c->cA, cbytes) && alloc(&c->cB, cbytes) && alloc(&c->cC, cbytes) && alloc(&c->cD, cbytes);
    ok = ok && alloc((void **)&c->tmpd, 2 * P * sizeof(double));
    if (cfg->correction_form == PARAREAL_CORRECTION_DIFFERENCE)
        ok = ok && alloc((void **)&c->dA, P * sizeof(double)) && alloc((void **)&c->dB, P * sizeof(double));
    ok = ok && alloc(&c->wS, P * e);
    ok = ok && alloc((void **)&c->bar, sizeof(pr::GridBarrier)) &&
         cudaMemset(c->bar, 0, sizeof(pr::GridBarrier)) == cudaSuccess;
    c->spectral = cfg->coarse_transfer == PARAREAL_TRANSFER_SPECTRAL;
    // the fine field a coarse G's change is prolonged into before the correction
    if (poly) ok = ok && alloc(&c->sp_fine, P * e);
    if (c->spectral) {
        const size_t me = (size_t)c->n * c->nc * e;
        ok = ok && alloc(&c->sp_R, me) && alloc(&c->sp_Rt, me) && alloc(&c->sp_P, me) &&
             alloc(&c->sp_Pt, me) && alloc(&c->sp_work, spectral_work_elems(c->n, c->r) * e) &&
             alloc(&c->sp_fine, P * e);
        if (ok) {
            std::vector<double> m4[4];
            spectral_matrices(c->n, c->r, &m4[0], &m4[1], &m4[2], &m4[3]);
            void *dst[4] = {c->sp_R, c->sp_Rt, c->sp_P, c->sp_Pt};
            for (int i = 0; i < 4 && ok; ++i) {
                if (c->f64) {
                    ok = cudaMemcpy(dst[i], m4[i].data(), me, cudaMemcpyHostToDevice) == cudaSuccess;
                } else {
                    std::vector<float> f(m4[i].begin(), m4[i].end());
                    ok = cudaMemcpy(dst[i], f.data(), me, cudaMemcpyHostToDevice) == cudaSuccess;
                }
            }
        }
    }
    c->nblk = correct_blocks(c->P);
    ok = ok && alloc((void **)&c->partials, 5 * sizeof(double) * (size_t)c->nblk);
    ok = ok && alloc((void **)&c->slice_norms, 5 * sizeof(double) * (N + 2));
    ok = ok && cudaMallocHost((void **)&c->h_norms, 5 * sizeof(double) * (N + 2)) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        parareal_destroy(c);
        return fail(nullptr, PARAREAL_E_NOMEM, "device allocation failed");
    }
    if (cudaMemsetAsync(c->slice_norms, 0, 5 * sizeof(double) * (N + 2), c->st) != cudaSuccess) {
        parareal_destroy(c);
        return fail(nullptr, PARAREAL_E_CUDA, "memset failed");
    }
    if (cfg->coarse_kind == PARAREAL_COARSE_LEARNED || cfg->coarse_kind == PARAREAL_COARSE_SHIFT) {
        parareal_status ns = net_setup(c);
        if (ns != PARAREAL_OK) {
            const std::string msg = c->err;
            parareal_destroy(c);
            return fail(nullptr, ns, msg);
        }
    }
    *out = c;
    return warn;
}

extern "C" void parareal_destroy(parareal_ctx *c)
{
    if (!c) return;
    cudaStreamSynchronize(c->st);
    if (c->st_f) cudaStreamSynchronize(c->st_f);
    if (c->st_hi) cudaStreamSynchronize(c->st_hi);
    void *ptrs[] = {c->U, c->Fv, c->Fv2, c->cancel, c->gspare, c->wA, c->wB, c->wC, c->cA, c->cB, c->cC, c->cD,
                    c->tmpd, c->wS, c->ref, c->partials, c->slice_norms, c->dA, c->dB,
                    c->sp_R, c->sp_Rt, c->sp_P, c->sp_Pt, c->sp_work, c->sp_fine, c->bar};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (void *p : c->gold)
        if (p) cudaFree(p);
    for (void *p : c->gold2)
        if (p) cudaFree(p);
    if (c->h_norms) cudaFreeHost(c->h_norms);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    for (int p = 0; p < 2; ++p) {
        for (cudaEvent_t e : c->ev_conv[p]) if (e) cudaEventDestroy(e);
        for (cudaEvent_t e : c->ev_done[p]) if (e) cudaEventDestroy(e);
    }
    if (c->ev_fork) cudaEventDestroy(c->ev_fork);
    if (c->ev_join) cudaEventDestroy(c->ev_join);
    if (c->ev_in) cudaEventDestroy(c->ev_in);
    if (c->ev_out) cudaEventDestroy(c->ev_out);
    solve_graph_free(c);
    if (c->st_f) cudaStreamDestroy(c->st_f);
    if (c->st_hi) cudaStreamDestroy(c->st_hi);
    net_free(c);
    delete c;
}

extern "C" const char *parareal_last_error(const parareal_ctx *c)
{
    return c ? c->err.c_str() : g_create_error.c_str();
}

extern "C" long long parareal_launch_count(const parareal_ctx *c) { return c ? c->launches : 0; }

extern "C" parareal_status parareal_profile(parareal_ctx *c, int enable)
{
    if (!c) return PARAREAL_E_INVALID;
    CK(cudaStreamSynchronize(c->st));
    c->prof = enable != 0;
    c->ev_used = 0;
    c->prof_bytes = 0.0;
    c->prof_launches = 0;
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_profile_read(parareal_ctx *c, double *ms, long long *launches,
                                                 double *bytes)
{
    if (!c) return PARAREAL_E_INVALID;
    CK(cudaStreamSynchronize(c->st));
    double total = 0.0;
    for (size_t i = 0; i + 1 < c->ev_used; i += 2) {
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, c->ev_pool[i], c->ev_pool[i + 1]));
        total += t;
    }
    if (ms) *ms = total;
    if (launches) *launches = c->prof_launches;
    if (bytes) *bytes = c->prof_bytes;
    c->ev_used = 0;
    c->prof_bytes = 0.0;
    c->prof_launches = 0;
    return PARAREAL_OK;
}

// Copy n^3 values of `dtype` at src (host or device) into the FP64 field dst.
static parareal_status load_field(parareal_ctx *c, double *dst, const void *src, int dtype, int mem)
{
    if (!src) return fail(c, PARAREAL_E_INVALID, "null field pointer");
    if (dtype != PARAREAL_F32 && dtype != PARAREAL_F64) return fail(c, PARAREAL_E_INVALID, "dtype");
    if (mem != PARAREAL_MEM_DEVICE && mem != PARAREAL_MEM_HOST) return fail(c, PARAREAL_E_INVALID, "mem");
    const size_t bytes = (size_t)c->P * (dtype == PARAREAL_F64 ? 8 : 4);
    const cudaMemcpyKind kind = mem == PARAREAL_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
    if (dtype == PARAREAL_F64) {
        CK(cudaMemcpyAsync(dst, src, bytes, kind, c->st));
    } else {
        float *stage = reinterpret_cast<float *>(c->tmpd) + c->P;   // upper half of tmpd
        CK(cudaMemcpyAsync(stage, src, bytes, kind, c->st));
        LK(launch_convert_f32_to_f64(stage, dst, c->P, c->st));
    }
    CK(cudaStreamSynchronize(c->st));   // the caller's buffer is borrowed for this call only
    return PARAREAL_OK;
}

static parareal_status store_field(parareal_ctx *c, void *dst, const double *src, int dtype, int mem)
{
    if (!dst) return fail(c, PARAREAL_E_INVALID, "null field pointer");
    if (dtype != PARAREAL_F32 && dtype != PARAREAL_F64) return fail(c, PARAREAL_E_INVALID, "dtype");
    if (mem != PARAREAL_MEM_DEVICE && mem != PARAREAL_MEM_HOST) return fail(c, PARAREAL_E_INVALID, "mem");
    const cudaMemcpyKind kind = mem == PARAREAL_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
    if (dtype == PARAREAL_F64) {
        CK(cudaMemcpyAsync(dst, src, (size_t)c->P * 8, kind, c->st));
    } else {
        float *stage = reinterpret_cast<float *>(c->tmpd) + c->P;
        LK(launch_convert_f64_to_f32(src, stage, c->P, c->st));
        CK(cudaMemcpyAsync(dst, stage, (size_t)c->P * 4, kind, c->st));
    }
    CK(cudaStreamSynchronize(c->st));   // the caller's buffer is borrowed for this call only
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_set_problem(parareal_ctx *c, const void *u0, int dtype, int mem)
{
    if (!c) return PARAREAL_E_INVALID;
    c->spec_valid = false;      // U, F or the sweep workspaces change
    parareal_status s = load_field(c, c->U, u0, dtype, mem);
    if (s != PARAREAL_OK) return s;
    c->has_problem = true;
    c->started = false;
    c->k_total = 0;
    std::fill(c->diff_inf.begin(), c->diff_inf.end(), 0.0);
    std::fill(c->diff_l2.begin(), c->diff_l2.end(), 0.0);
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_set_reference(parareal_ctx *c, const void *ref, int dtype, int mem)
{
    if (!c) return PARAREAL_E_INVALID;
    if (!c->ref && cudaMalloc((void **)&c->ref, (size_t)c->P * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->ref = nullptr;
        return fail(c, PARAREAL_E_NOMEM, "reference allocation failed");
    }
    parareal_status s = load_field(c, c->ref, ref, dtype, mem);
    if (s == PARAREAL_OK) c->has_ref = true;
    return s;
}

extern "C" parareal_status parareal_get_slice(parareal_ctx *c, int slice, void *dst, int dtype, int mem)
{
    if (!c) return PARAREAL_E_INVALID;
    if (slice < 0 || slice > c->N) return fail(c, PARAREAL_E_INVALID, "slice out of range");
    return store_field(c, dst, c->U + (long long)slice * c->P, dtype, mem);
}

extern "C" parareal_status parareal_set_slice(parareal_ctx *c, int slice, const void *src, int dtype, int mem)
{
    if (!c) return PARAREAL_E_INVALID;
    c->spec_valid = false;      // U, F or the sweep workspaces change
    if (slice < 0 || slice > c->N) return fail(c, PARAREAL_E_INVALID, "slice out of range");
    return load_field(c, c->U + (long long)slice * c->P, src, dtype, mem);
}

extern "C" parareal_status parareal_selftest_grid_barrier(void *cuda_stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    pr::GridBarrier *b = nullptr;
    if (cudaMalloc((void **)&b, sizeof *b) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, PARAREAL_E_NOMEM, "self-test barrier allocation failed");
    }
    pr::GridBarrier h{};
    cudaError_t e = cudaMemsetAsync(b, 0, sizeof *b, st);
    if (e == cudaSuccess) e = launch_grid_barrier_selftest(b, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, b, sizeof h, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(b);
    if (e != cudaSuccess) return fail(nullptr, PARAREAL_E_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    if (h.err == 1) return fail(nullptr, PARAREAL_E_TIMEOUT, "grid barrier gave up as designed (self-test)");
    return PARAREAL_OK;
}

parareal_status device_check(parareal_ctx *c)
{
    if (c->persist_used) {
        pr::GridBarrier h{};
        CK(cudaMemcpyAsync(&h, c->bar, sizeof h, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        c->persist_used = false;
        if (h.err) {
            // blocks may have left a barrier half counted: start the next launch clean
            CK(cudaMemsetAsync(c->bar, 0, sizeof h, c->st));
            return fail(c, PARAREAL_E_TIMEOUT, "a grid barrier of the persistent RK4 kernel gave up waiting");
        }
    }
    return net_check(c);
}

// ----------------------------------------------------------- checkpoint

namespace {
// Layout of a saved iteration state: this header, then U[0..N] (FP64), the
// N stored coarse outputs G(U^k[n]), then u_fine(T) when a reference is set.
struct StateHeader {
    char magic[8];
    int n, N, r, f64, g_fine, k_total, started, has_ref;
    long long P, gbytes;
    unsigned long long cfg_hash;   // fingerprint of every config field the iteration depends on
    unsigned long long model_hash; // learned G: fingerprint of its FP32 master weights (else 0)
};
constexpr char STATE_MAGIC[8] = {'P', 'R', 'L', 'S', 'T', 'A', 'T', '3'};

// FNV-1a over the bytes of one value.
template <typename V>
void fnv(unsigned long long &h, const V &v)
{
    const unsigned char *b = reinterpret_cast<const unsigned char *>(&v);
    for (size_t i = 0; i < sizeof(V); ++i) h = (h ^ b[i]) * 1099511628211ull;
}

unsigned long long config_hash(const parareal_config &c)
{
    unsigned long long h = 1469598103934665603ull;
    fnv(h, c.n); fnv(h, c.n_slices); fnv(h, c.T); fnv(h, c.dt_fine); fnv(h, c.dt_coarse);
    fnv(h, c.coarse_factor);
    for (int d = 0; d < 3; ++d) fnv(h, c.a[d]);
    fnv(h, c.nu0); fnv(h, c.nu_amp); fnv(h, c.nu_omega); fnv(h, c.fine_dtype); fnv(h, c.nu_mode);
    fnv(h, c.coarse_kind); fnv(h, c.learned_skip); fnv(h, c.fine_scheme); fnv(h, c.learned_act);
    fnv(h, c.correction_form); fnv(h, c.learned_eval); fnv(h, c.coarse_transfer);
    return h;
}
}  // namespace

// Fingerprint of the learned propagator's weights (0 for the other coarse
// propagators).  A learned context without a model gives E_STATE.
static parareal_status model_hash(parareal_ctx *c, unsigned long long *h)
{
    *h = 0;
    const int k = c->cfg.coarse_kind;
    if (k != PARAREAL_COARSE_LEARNED) return PARAREAL_OK;
    if (!c->net.has_model || !c->net.master)
        return fail(c, PARAREAL_E_STATE, "learned coarse propagator has no model: set or train one first");
    std::vector<float> w(NET_PARAMS);
    CK(cudaMemcpyAsync(w.data(), c->net.master, NET_PARAMS * sizeof(float), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    unsigned long long v = 1469598103934665603ull;
    for (float x : w) fnv(v, x);
    *h = v | 1ull;     // never 0 for a learned model
    return PARAREAL_OK;
}

static bool alloc_ref(parareal_ctx *c)
{
    if (cudaMalloc((void **)&c->ref, (size_t)c->P * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        c->ref = nullptr;
        return false;
    }
    return true;
}

static size_t gold_bytes(const parareal_ctx *c)
{
    return c->g_fine ? (size_t)c->P * sizeof(double) : (size_t)c->Pc * c->esz;
}

static size_t state_bytes(const parareal_ctx *c)
{
    return sizeof(StateHeader) + (size_t)(c->N + 1) * c->P * sizeof(double) +
           (size_t)c->N * gold_bytes(c) + (c->has_ref ? (size_t)c->P * sizeof(double) : 0);
}

extern "C" parareal_status parareal_save_state(parareal_ctx *c, void *host, size_t bytes, size_t *needed)
{
    if (!c) return PARAREAL_E_INVALID;
    const size_t need = state_bytes(c);
    if (needed) *needed = need;
    if (!host) return PARAREAL_OK;
    if (!c->has_problem) return fail(c, PARAREAL_E_STATE, "no problem set: nothing to save");
    if (bytes < need) return fail(c, PARAREAL_E_INVALID, "state buffer smaller than parareal_save_state's size");
    StateHeader h{};
    std::memcpy(h.magic, STATE_MAGIC, sizeof h.magic);
    h.n = c->n; h.N = c->N; h.r = c->r; h.f64 = c->f64; h.g_fine = c->g_fine;
    h.k_total = c->k_total; h.started = c->started; h.has_ref = c->has_ref;
    h.P = c->P; h.gbytes = (long long)gold_bytes(c);
    h.cfg_hash = config_hash(c->cfg);
    parareal_status ms = model_hash(c, &h.model_hash);
    if (ms != PARAREAL_OK) return ms;
    char *p = static_cast<char *>(host);
    std::memcpy(p, &h, sizeof h);
    p += sizeof h;
    const size_t ub = (size_t)(c->N + 1) * c->P * sizeof(double);
    CK(cudaMemcpyAsync(p, c->U, ub, cudaMemcpyDeviceToHost, c->st));
    p += ub;
    for (int i = 1; i <= c->N; ++i, p += gold_bytes(c))
        CK(cudaMemcpyAsync(p, g_cur(c, i), gold_bytes(c), cudaMemcpyDeviceToHost, c->st));
    if (c->has_ref) CK(cudaMemcpyAsync(p, c->ref, (size_t)c->P * sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_load_state(parareal_ctx *c, const void *host, size_t bytes)
{
    if (!c) return PARAREAL_E_INVALID;
    c->spec_valid = false;      // U, F or the sweep workspaces change
    if (!host || bytes < sizeof(StateHeader)) return fail(c, PARAREAL_E_INVALID, "state buffer too small");
    StateHeader h;
    std::memcpy(&h, host, sizeof h);
    if (std::memcmp(h.magic, STATE_MAGIC, sizeof h.magic) != 0)
        return fail(c, PARAREAL_E_INVALID, "not a saved Parareal state");
    if (h.n != c->n || h.N != c->N || h.r != c->r || h.f64 != (int)c->f64 || h.g_fine != (int)c->g_fine ||
        h.P != c->P || h.gbytes != (long long)gold_bytes(c) || h.cfg_hash != config_hash(c->cfg))
        return fail(c, PARAREAL_E_INVALID, "saved state belongs to a different configuration");
    unsigned long long mh = 0;
    parareal_status ms = model_hash(c, &mh);
    if (ms != PARAREAL_OK) return ms;
    if (mh != h.model_hash)
        return fail(c, PARAREAL_E_STATE, "saved state was iterated with other coarse-model weights");
    if (h.has_ref && !c->ref && !alloc_ref(c)) return fail(c, PARAREAL_E_NOMEM, "reference allocation failed");
    const bool had_ref = c->has_ref;
    c->has_ref = h.has_ref != 0;
    if (bytes < state_bytes(c)) {
        c->has_ref = had_ref;
        return fail(c, PARAREAL_E_INVALID, "state buffer shorter than its header says");
    }
    const char *p = static_cast<const char *>(host) + sizeof h;
    const size_t ub = (size_t)(c->N + 1) * c->P * sizeof(double);
    CK(cudaMemcpyAsync(c->U, p, ub, cudaMemcpyHostToDevice, c->st));
    p += ub;
    for (int i = 1; i <= c->N; ++i, p += gold_bytes(c))
        CK(cudaMemcpyAsync(g_cur(c, i), p, gold_bytes(c), cudaMemcpyHostToDevice, c->st));
    if (c->has_ref) CK(cudaMemcpyAsync(c->ref, p, (size_t)c->P * sizeof(double), cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->k_total = h.k_total;
    c->started = h.started != 0;
    c->has_problem = true;
    std::fill(c->diff_inf.begin(), c->diff_inf.end(), 0.0);
    std::fill(c->diff_l2.begin(), c->diff_l2.end(), 0.0);
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_fine_sweep(parareal_ctx *c, int first, int count)
{
    if (!c) return PARAREAL_E_INVALID;
    if (first < 0 || count < 0 || first + count > c->N) return fail(c, PARAREAL_E_INVALID, "slice range");
    if (count == 0) return PARAREAL_OK;
    return DISPATCH(c, fine_sweep_t, first, count);
}

extern "C" parareal_status parareal_coarse_sweep(parareal_ctx *c, int first, int count, int chain)
{
    if (!c) return PARAREAL_E_INVALID;
    c->spec_valid = false;      // U, F or the sweep workspaces change
    if (first < 0 || count < 0 || first + count > c->N) return fail(c, PARAREAL_E_INVALID, "slice range");
    return coarse_chain(c, first, count, chain != 0);
}

extern "C" parareal_status parareal_iterate(parareal_ctx *c, int k_max, double tol, int stop_rule,
                                            int *k_done, double *hist)
{
    if (!c) return PARAREAL_E_INVALID;
    if (k_done) *k_done = 0;
    if (!c->has_problem) return fail(c, PARAREAL_E_STATE, "set_problem first");
    if (k_max < 0) return fail(c, PARAREAL_E_INVALID, "k_max < 0");
    if (stop_rule == PARAREAL_STOP_DEFECT && !c->has_ref) return fail(c, PARAREAL_E_STATE, "no reference set");
    if (stop_rule < 0 || stop_rule > 2) return fail(c, PARAREAL_E_INVALID, "stop_rule");
    ChainStream chain_stream(c);
    parareal_status s;
    if (!c->started) {
        std::fill(c->gcur.begin(), c->gcur.end(), 0);
        s = coarse_chain(c, 0, c->N, true);
        if (s != PARAREAL_OK) return s;
        c->started = true;
    }
    const auto t0 = std::chrono::steady_clock::now();
    int done = 0;
    bool stopped = false;
    for (; done < k_max && c->k_total < c->N; ++done) {
        s = iter_enqueue(c);
        if (s == PARAREAL_OK) {
            c->spec_valid = false;
            if (cudaStreamSynchronize(c->st) != cudaSuccess) s = fail(c, PARAREAL_E_CUDA, "iteration failed");
        }
        if (s == PARAREAL_OK) s = device_check(c);
        double dmax = 0.0, l2max = 0.0, d = -1.0;
        if (s == PARAREAL_OK) s = iter_finish(c, &dmax, &l2max, &d);
        if (s != PARAREAL_OK) {
            // a failed iteration leaves no usable speculative sweep
            if (c->st_f) {
                cudaMemsetAsync(c->cancel, 1, sizeof(int), c->st);
                pipe_join(c);
            }
            return s;
        }
        // the next iteration's F, if this one started it (pipelined)
        c->spec_valid = c->spec_pending;
        c->spec_events = c->spec_pending;
        if (hist) {
            hist[4 * done + 0] = dmax;
            hist[4 * done + 1] = l2max;
            hist[4 * done + 2] = d;
            hist[4 * done + 3] =
                std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        }
        if ((stop_rule == PARAREAL_STOP_DIFF && dmax <= tol) ||
            (stop_rule == PARAREAL_STOP_DEFECT && d <= tol)) {
            ++done;
            stopped = true;
            break;
        }
    }
    if (c->st_f) {
        if (stopped && c->spec_valid) {
            // the speculative sweep is not needed: its remaining launches exit
            CK(cudaMemsetAsync(c->cancel, 1, sizeof(int), c->st));
            c->spec_valid = false;
        }
        s = pipe_join(c);
        if (s != PARAREAL_OK) return s;
    }
    if (k_done) *k_done = done;
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_residual(parareal_ctx *c, int kind, double *out)
{
    if (!c || !out) return PARAREAL_E_INVALID;
    std::fill(out, out + c->N + 1, 0.0);
    if (kind == PARAREAL_RES_DIFF_INF || kind == PARAREAL_RES_DIFF_L2) {
        for (int n = 0; n <= c->N; ++n)
            out[n] = kind == PARAREAL_RES_DIFF_INF ? c->diff_inf[n] : c->diff_l2[n];
        return PARAREAL_OK;
    }
    if (!c->has_problem) return fail(c, PARAREAL_E_STATE, "set_problem first");
    if (kind == PARAREAL_RES_DEFECT) {
        if (!c->has_ref) return fail(c, PARAREAL_E_STATE, "no reference set");
        return defect(c, &out[c->N]);
    }
    if (kind != PARAREAL_RES_FINE && kind != PARAREAL_RES_FINE_L2) return fail(c, PARAREAL_E_INVALID, "kind");
    // ||F(U[n-1]) - U[n]||_inf / ||U[n]||_inf: one fine sweep into Fv, then
    // the norm of Fv[n] - U[n] per slice.
    parareal_status s = DISPATCH(c, fine_sweep_t, 0, c->N);
    if (s != PARAREAL_OK) return s;
    for (int n = 1; n <= c->N; ++n) {
        if (c->f64) {
            LK(launch_diff_norms<double>(static_cast<const double *>(c->Fv) + (long long)n * c->P,
                                         c->U + (long long)n * c->P, c->P, c->partials, c->nblk, c->st));
        } else {
            LK(launch_diff_norms<float>(static_cast<const float *>(c->Fv) + (long long)n * c->P,
                                        c->U + (long long)n * c->P, c->P, c->partials, c->nblk, c->st));
        }
        LK(launch_reduce_partials(c->partials, c->nblk, c->slice_norms + 5ll * n, c->st));
    }
    CK(cudaMemcpyAsync(c->h_norms, c->slice_norms, sizeof(double) * 5 * (c->N + 1), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    for (int n = 1; n <= c->N; ++n) {
        const double *q = c->h_norms + 5 * n;
        if (kind == PARAREAL_RES_FINE) out[n] = q[1] > 0 ? q[0] / q[1] : q[0];
        else out[n] = q[3] > 0 ? std::sqrt(q[2] / q[3]) : std::sqrt(q[2]);
    }
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_serial_fine(parareal_ctx *c, void *dst, int dtype, int mem,
                                                int as_reference)
{
    if (!c) return PARAREAL_E_INVALID;
    c->spec_valid = false;      // U, F or the sweep workspaces change
    if (!c->has_problem) return fail(c, PARAREAL_E_STATE, "set_problem first");
    // march slice after slice in the fine arithmetic type; slice boundaries
    // pass through Fv[1] (F's output of one slice is the next slice's input)
    const long long P = c->P;
    parareal_status s = PARAREAL_OK;
    if (c->f64) {
        double *cur = static_cast<double *>(c->wS);
        CK(cudaMemcpyAsync(cur, c->U, P * 8, cudaMemcpyDeviceToDevice, c->st));
        double *Fv1 = static_cast<double *>(c->Fv) + P;
        for (int n = 0; n < c->N && s == PARAREAL_OK; ++n) {
            s = rk4_batch<double>(c, c->n, cur, Fv1, n, 1, c->Nf, c->cfg.dt_fine, c->ser_path,
                                  c->ser_tx, c->ser_ty, c->ser_zc, static_cast<double *>(c->wA),
                                  static_cast<double *>(c->wB), static_cast<double *>(c->wC), 1,
                                  c->fine_op);
            if (s == PARAREAL_OK) CK(cudaMemcpyAsync(cur, Fv1, P * 8, cudaMemcpyDeviceToDevice, c->st));
        }
        if (s != PARAREAL_OK) return s;
        CK(cudaMemcpyAsync(c->tmpd, cur, P * 8, cudaMemcpyDeviceToDevice, c->st));
    } else {
        float *cur = static_cast<float *>(c->wS);
        LK(launch_convert_f64_to_f32(c->U, cur, P, c->st));
        float *Fv1 = static_cast<float *>(c->Fv) + P;
        for (int n = 0; n < c->N && s == PARAREAL_OK; ++n) {
            s = rk4_batch<float>(c, c->n, cur, Fv1, n, 1, c->Nf, c->cfg.dt_fine, c->ser_path,
                                 c->ser_tx, c->ser_ty, c->ser_zc, static_cast<float *>(c->wA),
                                 static_cast<float *>(c->wB), static_cast<float *>(c->wC), 1,
                                 c->fine_op);
            if (s == PARAREAL_OK) CK(cudaMemcpyAsync(cur, Fv1, P * 4, cudaMemcpyDeviceToDevice, c->st));
        }
        if (s != PARAREAL_OK) return s;
        LK(launch_convert_f32_to_f64(cur, c->tmpd, P, c->st));
    }
    if (as_reference) {
        if (!c->ref && cudaMalloc((void **)&c->ref, (size_t)P * sizeof(double)) != cudaSuccess) {
            cudaGetLastError();
            c->ref = nullptr;
            return fail(c, PARAREAL_E_NOMEM, "reference allocation failed");
        }
        CK(cudaMemcpyAsync(c->ref, c->tmpd, P * 8, cudaMemcpyDeviceToDevice, c->st));
        c->has_ref = true;
    }
    if (dst) {
        // tmpd holds the result; store_field stages through tmpd's upper half
        // only for FP32, which does not overlap the FP64 values in use.
        if (dtype == PARAREAL_F64) {
            CK(cudaMemcpyAsync(dst, c->tmpd, P * 8, mem == PARAREAL_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                             : cudaMemcpyDeviceToDevice, c->st));
            CK(cudaStreamSynchronize(c->st));
        } else {
            float *stage = static_cast<float *>(c->wA);
            LK(launch_convert_f64_to_f32(c->tmpd, stage, P, c->st));
            CK(cudaMemcpyAsync(dst, stage, P * 4, mem == PARAREAL_MEM_HOST ? cudaMemcpyDeviceToHost
                                                                          : cudaMemcpyDeviceToDevice, c->st));
            CK(cudaStreamSynchronize(c->st));
        }
    }
    return c->persist_used ? device_check(c) : PARAREAL_OK;
}

template <typename T>
static parareal_status propagate_t(parareal_ctx *c, int which, const void *src, void *dst,
                                   int dtype, int first, int count)
{
    const long long P = c->P;
    const size_t es = dtype == PARAREAL_F64 ? 8 : 4;
    for (int f = 0; f < count; ++f) {
        const char *sp = static_cast<const char *>(src) + (size_t)f * P * es;
        char *dp = static_cast<char *>(dst) + (size_t)f * P * es;
        double *in64 = c->tmpd;          // input as FP64
        double *res64 = c->tmpd + P;     // result as FP64
        if (dtype == PARAREAL_F64) {
            CK(cudaMemcpyAsync(in64, sp, P * 8, cudaMemcpyDeviceToDevice, c->st));
        } else {
            LK(launch_convert_f32_to_f64(reinterpret_cast<const float *>(sp), in64, P, c->st));
        }
        parareal_status s;
        if (which == 0) {
            // input in the serial-state buffer, output in the unused Fv[0]
            // slot, fine-sized workspaces wA..wC
            T *tin = static_cast<T *>(c->wS), *tout = static_cast<T *>(c->Fv);
            if (std::is_same<T, float>::value)
                LK(launch_convert_f64_to_f32(in64, reinterpret_cast<float *>(tin), P, c->st));
            else
                CK(cudaMemcpyAsync(tin, in64, P * 8, cudaMemcpyDeviceToDevice, c->st));
            s = rk4_batch<T>(c, c->n, tin, tout, first + f, 1, c->Nf, c->cfg.dt_fine, c->ser_path,
                             c->ser_tx, c->ser_ty, c->ser_zc, static_cast<T *>(c->wA),
                             static_cast<T *>(c->wB), static_cast<T *>(c->wC), 1, c->fine_op);
            if (s != PARAREAL_OK) return s;
            if (std::is_same<T, float>::value)
                LK(launch_convert_f32_to_f64(reinterpret_cast<const float *>(tout), res64, P, c->st));
            else
                CK(cudaMemcpyAsync(res64, tout, P * 8, cudaMemcpyDeviceToDevice, c->st));
        } else {
            s = coarse_apply_t<T>(c, in64, first + f, c->gspare);
            if (s != PARAREAL_OK) return s;
            // res64 = G output on the fine grid: U-style correction with
            // null F and null old value, written into res64
            CK(cudaMemsetAsync(res64, 0, P * 8, c->st));
            const T *nullT = nullptr;
            if (!c->g_fine) {
                s = correct_coarse<T>(c, first + f, nullT, static_cast<const T *>(c->gspare), nullptr, res64,
                                      nullptr);
                if (s != PARAREAL_OK) return s;
            } else {
                LK((launch_correct<T, double>(nullT, static_cast<const double *>(c->gspare), nullptr,
                                              res64, c->n, 1, c->partials, c->nblk, c->st)));
            }
        }
        if (dtype == PARAREAL_F64) {
            CK(cudaMemcpyAsync(dp, res64, P * 8, cudaMemcpyDeviceToDevice, c->st));
        } else {
            LK(launch_convert_f64_to_f32(res64, reinterpret_cast<float *>(dp), P, c->st));
        }
    }
    CK(cudaStreamSynchronize(c->st));   // src and dst are borrowed for this call only
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_propagate(parareal_ctx *c, int which, const void *src,
                                              void *dst, int dtype, int first, int count)
{
    if (!c) return PARAREAL_E_INVALID;
    c->spec_valid = false;      // U, F or the sweep workspaces change
    if (!src || !dst || (which != 0 && which != 1)) return fail(c, PARAREAL_E_INVALID, "arguments");
    if (dtype != PARAREAL_F32 && dtype != PARAREAL_F64) return fail(c, PARAREAL_E_INVALID, "dtype");
    if (first < 0 || count < 0 || first + count > c->N) return fail(c, PARAREAL_E_INVALID, "slice range");
    parareal_status s = DISPATCH(c, propagate_t, which, src, dst, dtype, first, count);
    return s != PARAREAL_OK ? s : device_check(c);
}

// ----------------------------------------------------------------- autotune

// Time `reps` RK4 steps of `count` fields on an m^3 grid with one launch
// shape; returns ms per step (min over 3 trials).
template <typename T>
static parareal_status time_shape(parareal_ctx *c, int m, int count, int path, int tx, int ty, int zc,
                                  double dt, double *ms)
{
    T *in = static_cast<T *>(c->wC), *out = static_cast<T *>(c->Fv) + c->P;
    T *w1 = static_cast<T *>(c->wA), *w2 = static_cast<T *>(c->wB);
    T *w3 = reinterpret_cast<T *>(c->U);   // scratch: autotune overwrites the iterate
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    CK(cudaEventCreate(&e1));
    const int reps = 4;
    double best = 1e30;
    parareal_status s = PARAREAL_OK;
    for (int trial = 0; trial < 3 && s == PARAREAL_OK; ++trial) {
        CK(cudaEventRecord(e0, c->st));
        s = rk4_batch<T>(c, m, in, out, 0, count, reps, dt, path, tx, ty, zc, w1, w2, w3);
        CK(cudaEventRecord(e1, c->st));
        CK(cudaEventSynchronize(e1));
        float t = 0.f;
        CK(cudaEventElapsedTime(&t, e0, e1));
        if (trial > 0) best = std::min(best, (double)t / reps);   // trial 0 warms up
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = best;
    return s;
}

// Candidates: every compiled fused shape (one and two rows per thread) that
// divides m, whole-column and chunked z marches, the per-stage path, the
// persistent path, and the cluster path where the field fits one cluster.
enum { NO_STAGED = 1, NO_PERSIST = 2 };

static void candidates(int dtype, int m, std::vector<std::array<int, 4>> *out, int exclude = 0)
{
    const int shapes[][2] = {{64, 32}, {64, 16}, {64, 8}, {32, 32}, {32, 16}, {32, 8}, {16, 16}, {16, 8}};
    for (int path : {PATH_FUSED, PATH_FUSED2})
        for (auto &sh : shapes) {
            if (!rk4_fused_supported(dtype, m, sh[0], sh[1], fused_rows(path))) continue;
            for (int zc = m; zc >= 8; zc /= 2) {
                out->push_back({path, sh[0], sh[1], zc});
                if (zc <= m / 8) break;
            }
        }
    if (!(exclude & NO_STAGED)) out->push_back({PATH_STAGED, 16, 8, m});
    if (!(exclude & NO_PERSIST)) out->push_back({PATH_PERSIST, 16, 8, m});
    if (!(exclude & NO_STAGED) && rk4_cluster_size(dtype, m) > 0)
        out->push_back({PATH_CLUSTER, 0, 0, m});
}

static std::string tune_key(int dtype, int m, int count, int exclude)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    char k[128];
    // "paths=5": the candidate set includes launch paths 0-4 (a cached pick
    // made from fewer paths is not reused)
    std::snprintf(k, sizeof k, "n=%d dtype=%d count=%d sms=%d paths=5%s%s", m, dtype, count, sms,
                  (exclude & NO_STAGED) ? " nostaged" : "", (exclude & NO_PERSIST) ? " nopersist" : "");
    return k;
}

// Cache lines: {"key": "...", "shape": [path, tx, ty, zc], "ms": t}
static bool cache_lookup(const char *path, const std::string &key, int *sh)
{
    if (!path) return false;
    FILE *f = std::fopen(path, "r");
    if (!f) return false;
    char line[512];
    bool found = false;
    while (std::fgets(line, sizeof line, f)) {
        const std::string l(line);
        if (l.find("\"" + key + "\"") == std::string::npos) continue;
        const size_t p = l.find("\"shape\": [");
        if (p == std::string::npos) continue;
        if (std::sscanf(l.c_str() + p + 10, "%d, %d, %d, %d", &sh[0], &sh[1], &sh[2], &sh[3]) == 4) found = true;
    }
    std::fclose(f);
    return found;
}

static void cache_store(const char *path, const std::string &key, const int *sh, double ms)
{
    if (!path) return;
    FILE *f = std::fopen(path, "a");
    if (!f) return;
    std::fprintf(f, "{\"key\": \"%s\", \"shape\": [%d, %d, %d, %d], \"ms\": %.6f}\n", key.c_str(),
                 sh[0], sh[1], sh[2], sh[3], ms);
    std::fclose(f);
}

template <typename T>
static parareal_status tune_one(parareal_ctx *c, const char *cache, int m, int count, double dt,
                                int *path, int *tx, int *ty, int *zc, double *best_ms, int exclude = 0)
{
    const int dtype = c->f64 ? PARAREAL_F64 : PARAREAL_F32;
    const std::string key = tune_key(dtype, m, count, exclude);
    int sh[4];
    if (cache_lookup(cache, key, sh) &&
        ((sh[0] == PATH_STAGED && !(exclude & NO_STAGED)) ||
         (sh[0] == PATH_PERSIST && !(exclude & NO_PERSIST)) ||
         (sh[0] == PATH_CLUSTER && !(exclude & NO_STAGED) && rk4_cluster_size(dtype, m) > 0) ||
         (is_fused(sh[0]) && rk4_fused_supported(dtype, m, sh[1], sh[2], fused_rows(sh[0]))))) {
        *path = sh[0]; *tx = sh[1]; *ty = sh[2]; *zc = sh[3];
        *best_ms = -1.0;
        return PARAREAL_OK;
    }
    std::vector<std::array<int, 4>> cand;
    candidates(dtype, m, &cand, exclude);
    double best = 1e30;
    std::array<int, 4> pick = cand.back();
    for (auto &k : cand) {
        double ms;
        parareal_status s = time_shape<T>(c, m, count, k[0], k[1], k[2], k[3], dt, &ms);
        if (s != PARAREAL_OK) return s;
        if (ms < best) { best = ms; pick = k; }
    }
    *path = pick[0]; *tx = pick[1]; *ty = pick[2]; *zc = pick[3];
    *best_ms = best;
    const int store[4] = {pick[0], pick[1], pick[2], pick[3]};
    cache_store(cache, key, store, best);
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_autotune(parareal_ctx *c, const char *cache_path, double *ms2)
{
    if (!c) return PARAREAL_E_INVALID;
    c->spec_valid = false;      // U, F or the sweep workspaces change
    CK(cudaMemsetAsync(c->wC, 0, (size_t)c->N * c->P * c->esz, c->st));
    CK(cudaMemsetAsync(c->cA, 0, (size_t)(c->r > 1 ? c->Pc : c->P) * c->esz, c->st));
    double fms = 0.0, cms = 0.0;
    parareal_status s = PARAREAL_OK;
    if (c->fine_op != OP_C2) {
        // F runs on the per-stage kernels, which have no launch shape to tune
    } else if (c->f64)
        s = tune_one<double>(c, cache_path, c->n, c->N, c->cfg.dt_fine, &c->fine_path, &c->fine_tx,
                             &c->fine_ty, &c->fine_zc, &fms);
    else
        s = tune_one<float>(c, cache_path, c->n, c->N, c->cfg.dt_fine, &c->fine_path, &c->fine_tx,
                            &c->fine_ty, &c->fine_zc, &fms);
    if (s != PARAREAL_OK) return s;
    if (c->fine_op != OP_C2) {
    } else if (c->N > 1) {
        // one fine field at a time (serial fine run, propagate)
        double sms = 0.0;
        if (c->f64)
            s = tune_one<double>(c, cache_path, c->n, 1, c->cfg.dt_fine, &c->ser_path, &c->ser_tx,
                                 &c->ser_ty, &c->ser_zc, &sms);
        else
            s = tune_one<float>(c, cache_path, c->n, 1, c->cfg.dt_fine, &c->ser_path, &c->ser_tx,
                                &c->ser_ty, &c->ser_zc, &sms);
        if (s != PARAREAL_OK) return s;
    } else {
        c->ser_path = c->fine_path; c->ser_tx = c->fine_tx; c->ser_ty = c->fine_ty; c->ser_zc = c->fine_zc;
    }
    if ((c->cfg.coarse_kind == PARAREAL_COARSE_STENCIL ||
         c->cfg.learned_skip == PARAREAL_SKIP_STENCIL) && c->nc >= 8) {
        // the coarse sweep runs one field at a time on the coarse grid
        // (pipelined: no cooperative persistent launch beside the side stream's sweep)
        const int ex = c->Fv2 ? NO_PERSIST : 0;
        void *saveC = c->wC;
        c->wC = c->cA;   // input of the timed coarse steps
        if (c->f64)
            s = tune_one<double>(c, cache_path, c->nc, 1, c->cfg.dt_coarse, &c->coarse_path,
                                 &c->coarse_tx, &c->coarse_ty, &c->coarse_zc, &cms, ex);
        else
            s = tune_one<float>(c, cache_path, c->nc, 1, c->cfg.dt_coarse, &c->coarse_path,
                                &c->coarse_tx, &c->coarse_ty, &c->coarse_zc, &cms, ex);
        c->wC = saveC;
        if (s != PARAREAL_OK) return s;
    }
    const char *pipe_env = std::getenv("PARAREAL_PIPE_TILE");
    if (c->Fv2 && !(pipe_env && *pipe_env)) {
        // the speculative sweep's blocks: fused shapes only (they honour the cancel flag)
        const int nb = (int)c->ev_done[0].size();
        double pms = 0.0;
        s = tune_one<float>(c, cache_path, c->n, (c->N - 1 + nb - 1) / nb, c->cfg.dt_fine,
                            &c->pipe_path, &c->pipe_tx, &c->pipe_ty, &c->pipe_zc, &pms,
                            NO_STAGED | NO_PERSIST);
        if (s != PARAREAL_OK) return s;
    }
    if (ms2) { ms2[0] = fms; ms2[1] = cms; }
    c->has_problem = false;   // the iterate was used as scratch
    c->started = false;
    return PARAREAL_OK;
}

extern "C" int parareal_cluster_size(int dtype, int n)
{
    if ((dtype != PARAREAL_F32 && dtype != PARAREAL_F64) || n < 4) return 0;
    return rk4_cluster_size(dtype, n);
}

extern "C" parareal_status parareal_get_launch_shape(const parareal_ctx *c, int *fine4, int *coarse4,
                                                     int *serial4)
{
    if (!c) return PARAREAL_E_INVALID;
    if (fine4) { fine4[0] = c->fine_path; fine4[1] = c->fine_tx; fine4[2] = c->fine_ty; fine4[3] = c->fine_zc; }
    if (serial4) { serial4[0] = c->ser_path; serial4[1] = c->ser_tx; serial4[2] = c->ser_ty; serial4[3] = c->ser_zc; }
    if (coarse4) { coarse4[0] = c->coarse_path; coarse4[1] = c->coarse_tx; coarse4[2] = c->coarse_ty; coarse4[3] = c->coarse_zc; }
    return PARAREAL_OK;
}
