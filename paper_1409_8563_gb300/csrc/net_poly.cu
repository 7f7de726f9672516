// net_poly.cu -- the LINEAR learned coarse propagator with the stencil skip,
// evaluated on the coarse grid (learned_eval POLYPHASE).
//
// With the stencil skip the learned propagator is G(u) = x + K * x, x the
// stencil propagator's output prolonged to the fine grid, x = P c with c its
// coarse result and P the trilinear prolongation, K = K_0 + nu_hat K_1 the
// composed 9^3 kernel of the four linear layers (net_composed.cu).  Both P
// and the cross-correlation are linear, and P commutes with shifts by r fine
// cells, so G's fine output at p = X r + rho (X a coarse cell, rho in
// [0, r)^3) is a short coarse cross-correlation whose taps depend only on
// the phase rho:
//
//   G(u)[X r + rho] = sum_t W_rho[t] c[X + s(rho) + t],   t in [0, TT)^3,
//   W_rho[t] = sum_e (delta + K)[e] P3(rho + e, s(rho) + t),
//
// P3(x', C) the trilinear weight of fine point x' (relative to the cell's
// origin) on coarse cell C, s(rho) = floor((rho - 4 - (r-1)/2) / r) per axis
// the first coarse cell any tap reaches.  TT = 4 taps per axis for r = 4
// (64 multiply-adds per fine point instead of 729 + 8), 3 for r = 8, 6 for
// r = 2.  The phase kernels are built in FP64 from the composed kernels
// whenever the model changes, per slice in FP32, and applied to the coarse
// change of G's output inside the correction, as the trilinear prolongation
// is for the stencil propagator; G's coarse part is the stencil propagator's.
#include <algorithm>
#include <cmath>

#include "internal.cuh"
#include "net.cuh"

namespace pr {
namespace {

constexpr int PP_THREADS = 256;
constexpr int PP_B = 16;                 // fine brick edge of one CTA

// floor(a / b) for b > 0
__host__ __device__ inline int floordiv(int a, int b) { return a >= 0 ? a / b : -((-a + b - 1) / b); }

// First coarse cell (relative to the point's own cell) that the taps of
// phase rho reach: floor((rho - 4 - (r-1)/2) / r) = floor((2 rho - 7 - r) / (2 r)).
__host__ __device__ inline int phase_start(int rho, int r) { return floordiv(2 * rho - 7 - r, 2 * r); }

// Trilinear weight of fine coordinate x (relative to a coarse cell's first
// fine point) on coarse cell C (relative to that cell): the fine point lies
// at coarse coordinate (x - (r-1)/2) / r, between cells f and f + 1 (the
// weights of the prolongation inside the correction kernel).
__device__ inline double lin1(int x, int r, int C)
{
    const double sv = ((double)x - 0.5 * (double)(r - 1)) / (double)r;
    const double f = floor(sv);
    const double w = sv - f;
    const int fi = (int)f;
    return C == fi ? 1.0 - w : (C == fi + 1 ? w : 0.0);
}

// W2[c][rho][t] for the two composed kernels K (c = 0: K_0 plus the skip's
// identity, c = 1: K_1), in FP64.  K[c][(ez+4) 81 + (ey+4) 9 + (ex+4)].
__global__ void compose_poly_kernel(const double *__restrict__ K, int r, int TT, double *__restrict__ W2)
{
    const int R3 = r * r * r, T3 = TT * TT * TT;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;          // (c * R3 + rho) * T3 + t
    if (j >= 2 * R3 * T3) return;
    const int t = j % T3, rho = (j / T3) % R3, c = j / (T3 * R3);
    const int tx = t % TT, ty = (t / TT) % TT, tz = t / (TT * TT);
    const int rx = rho % r, ry = (rho / r) % r, rz = rho / (r * r);
    const int Cx = phase_start(rx, r) + tx, Cy = phase_start(ry, r) + ty, Cz = phase_start(rz, r) + tz;
    double wx[9], wy[9], wz[9];
    for (int e = 0; e < 9; ++e) {
        wx[e] = lin1(rx + e - 4, r, Cx);
        wy[e] = lin1(ry + e - 4, r, Cy);
        wz[e] = lin1(rz + e - 4, r, Cz);
    }
    const double *Kc = K + (size_t)c * NET_K9;
    double s = 0.0;
    for (int ez = 0; ez < 9; ++ez) {
        if (wz[ez] == 0.0) continue;
        double sy = 0.0;
        for (int ey = 0; ey < 9; ++ey) {
            if (wy[ey] == 0.0) continue;
            double sx = 0.0;
            for (int ex = 0; ex < 9; ++ex) {
                double k = Kc[(ez * 9 + ey) * 9 + ex];
                if (c == 0 && ez == 4 && ey == 4 && ex == 4) k += 1.0;    // the skip x itself
                sx += k * wx[ex];
            }
            sy += sx * wy[ey];
        }
        s += sy * wz[ez];
    }
    W2[j] = s;
}

// Wn[n][rho][t] = W2[0][rho][t] + nu_hat[n] W2[1][rho][t] in FP32, rows of
// T3 + 1 (the pad keeps the rows of neighbouring phases in distinct banks).
__global__ void compose_poly_slices(const double *__restrict__ W2, const float *__restrict__ nu_hat,
                                    int n_slices, int R3, int T3, float *__restrict__ Wn)
{
    const int row = T3 + 1;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;          // (n * R3 + rho) * row + t
    if (j >= n_slices * R3 * row) return;
    const int t = j % row, rho = (j / row) % R3, n = j / (row * R3);
    Wn[j] = t < T3 ? (float)(W2[rho * T3 + t] + (double)nu_hat[n] * W2[(R3 + rho) * T3 + t]) : 0.f;
}

// out[p] = sum_t W_rho(p)[t] dc[X(p) + s(rho(p)) + t], dc = cnew - cold (cold
// may be null), on the coarse grid of edge nc = n / r, periodic.  One CTA per
// 16^3 fine brick: the brick's coarse window of dc and the slice's phase
// kernels in shared memory; thread t owns the x-row (t % 16, t / 16) of the
// brick and sums every tap in a fixed order.
template <typename T>
__global__ void __launch_bounds__(PP_THREADS)
poly_prolong_kernel(const T *__restrict__ cnew, const T *__restrict__ cold, const float *__restrict__ W,
                    int n, int r, int TT, int lo_off, int win, T *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char pp_smem[];
    const int R3 = r * r * r, T3 = TT * TT * TT, row = T3 + 1;
    float *ws = reinterpret_cast<float *>(pp_smem);
    T *dcw = reinterpret_cast<T *>(pp_smem + (((size_t)R3 * row * sizeof(float) + 15) & ~(size_t)15));
    const int nc = n / r, nb = n / PP_B;
    const int bx = blockIdx.x % nb, by = (blockIdx.x / nb) % nb, bz = blockIdx.x / (nb * nb);
    const int cx0 = bx * PP_B / r + lo_off, cy0 = by * PP_B / r + lo_off, cz0 = bz * PP_B / r + lo_off;
    for (int i = threadIdx.x; i < R3 * row; i += blockDim.x) ws[i] = W[i];
    auto wrap = [nc](int v) { v %= nc; return v < 0 ? v + nc : v; };
    const int w3 = win * win * win;
    for (int i = threadIdx.x; i < w3; i += blockDim.x) {
        const int ix = i % win, iy = (i / win) % win, iz = i / (win * win);
        const long long q = ((long long)wrap(cz0 + iz) * nc + wrap(cy0 + iy)) * nc + wrap(cx0 + ix);
        dcw[i] = cold ? cnew[q] - cold[q] : cnew[q];
    }
    __syncthreads();
    const int x = threadIdx.x % PP_B, y = threadIdx.x / PP_B;
    const int rx = x % r, ry = y % r;
    const int wx0 = x / r + phase_start(rx, r) - lo_off, wy0 = y / r + phase_start(ry, r) - lo_off;
    const long long gx = (long long)bx * PP_B + x, gy = (long long)by * PP_B + y;
    for (int z = 0; z < PP_B; ++z) {
        const int rz = z % r;
        const int wz0 = z / r + phase_start(rz, r) - lo_off;
        const float *wp = ws + ((rz * r + ry) * r + rx) * row;
        T acc = (T)0;
        for (int tz = 0; tz < TT; ++tz)
            for (int ty = 0; ty < TT; ++ty) {
                const T *dr = dcw + ((wz0 + tz) * win + (wy0 + ty)) * win + wx0;
                const float *wr = wp + (tz * TT + ty) * TT;
                for (int tx = 0; tx < TT; ++tx) acc = fma((T)wr[tx], dr[tx], acc);
            }
        out[((long long)(bz * PP_B + z) * n + gy) * n + gx] = acc;
    }
}

// The same sum for TT taps per axis known at compile time (r = 4: 4, r = 8:
// 3), with a thread's phase kernel in registers: thread t takes phase
// t % min(r^3, 256) and whole x-rows of the brick's CB coarse cells (rows
// t / min(r^3, 256), + 256 / min(r^3, 256), ...), so the 32 lanes of a warp
// are 32 phases of the same cells and read at most 2^3 distinct window
// entries per load.  The CB cells of a row share their window: per (tz, ty)
// a thread loads CB + TT - 1 entries for CB x TT FMAs.  Each cell's taps are
// summed in the order of the generic kernel, so both give the same value.
template <typename T, int TT, int CB>
__global__ void __launch_bounds__(PP_THREADS)
poly_prolong_reg_kernel(const T *__restrict__ cnew, const T *__restrict__ cold, const float *__restrict__ W,
                        int n, int r, int lo_off, int win, T *__restrict__ out)
{
    constexpr int T3 = TT * TT * TT;
    constexpr int RW = CB + TT - 1;                  // window entries of one row of cells
    extern __shared__ __align__(16) unsigned char pp_smem[];
    T *dcw = reinterpret_cast<T *>(pp_smem);
    const int R3 = r * r * r, nc = n / r, nb = n / PP_B;
    const int bx = blockIdx.x % nb, by = (blockIdx.x / nb) % nb, bz = blockIdx.x / (nb * nb);
    const int cx0 = bx * CB + lo_off, cy0 = by * CB + lo_off, cz0 = bz * CB + lo_off;
    auto wrap = [nc](int v) { v %= nc; return v < 0 ? v + nc : v; };
    const int w3 = win * win * win;
    for (int i = threadIdx.x; i < w3; i += blockDim.x) {
        const int ix = i % win, iy = (i / win) % win, iz = i / (win * win);
        const long long q = ((long long)wrap(cz0 + iz) * nc + wrap(cy0 + iy)) * nc + wrap(cx0 + ix);
        dcw[i] = cold ? cnew[q] - cold[q] : cnew[q];
    }
    __syncthreads();
    const int rs = R3 < PP_THREADS ? R3 : PP_THREADS;
    const int g = threadIdx.x / rs, per = PP_THREADS / rs;
    for (int rho = threadIdx.x % rs; rho < R3; rho += PP_THREADS) {
        const int rx = rho % r, ry = (rho / r) % r, rz = rho / (r * r);
        T w[T3];
#pragma unroll
        for (int k = 0; k < T3; ++k) w[k] = (T)W[rho * (T3 + 1) + k];
        const int sx = phase_start(rx, r) - lo_off, sy = phase_start(ry, r) - lo_off,
                  sz = phase_start(rz, r) - lo_off;
        for (int row = g; row < CB * CB; row += per) {
            const int cy = row % CB, cz = row / CB;
            const T *d0 = dcw + ((cz + sz) * win + (cy + sy)) * win + sx;
            T acc[CB];
#pragma unroll
            for (int c = 0; c < CB; ++c) acc[c] = (T)0;
#pragma unroll
            for (int tz = 0; tz < TT; ++tz)
#pragma unroll
                for (int ty = 0; ty < TT; ++ty) {
                    T v[RW];
#pragma unroll
                    for (int e = 0; e < RW; ++e) v[e] = d0[(tz * win + ty) * win + e];
#pragma unroll
                    for (int tx = 0; tx < TT; ++tx)
#pragma unroll
                        for (int c = 0; c < CB; ++c)
                            acc[c] = fma(w[(tz * TT + ty) * TT + tx], v[c + tx], acc[c]);
                }
            const long long gy = (long long)by * PP_B + cy * r + ry, gz = (long long)bz * PP_B + cz * r + rz;
#pragma unroll
            for (int c = 0; c < CB; ++c)
                out[(gz * n + gy) * n + (long long)bx * PP_B + c * r + rx] = acc[c];
        }
    }
}

}  // namespace

void poly_geometry(int r, int *TT, int *lo_off, int *win)
{
    int tt = 0, lo = 0, hi = 0;
    for (int rho = 0; rho < r; ++rho) {
        const int s = phase_start(rho, r);
        // the last coarse cell a tap of this phase reaches: the upper
        // trilinear neighbour of fine coordinate rho + 4
        const int e = floordiv(2 * (rho + 4) - (r - 1), 2 * r) + 1;
        tt = std::max(tt, e - s + 1);
        lo = rho == 0 ? s : std::min(lo, s);
    }
    for (int rho = 0; rho < r; ++rho) hi = std::max(hi, phase_start(rho, r) + tt - 1);
    *TT = tt;
    *lo_off = lo;
    *win = (PP_B / r - 1) + hi - lo + 1;
}

size_t poly_smem_bytes(int r, size_t e)
{
    int TT, lo, win;
    poly_geometry(r, &TT, &lo, &win);
    const size_t wbytes = ((size_t)r * r * r * (TT * TT * TT + 1) * sizeof(float) + 15) & ~(size_t)15;
    return wbytes + (size_t)win * win * win * e;
}

size_t poly_weights_floats(int r, int n_slices)
{
    int TT, lo, win;
    poly_geometry(r, &TT, &lo, &win);
    return (size_t)n_slices * r * r * r * (TT * TT * TT + 1);
}

size_t poly_scratch_doubles(int r)
{
    int TT, lo, win;
    poly_geometry(r, &TT, &lo, &win);
    return (size_t)2 * r * r * r * TT * TT * TT;
}

cudaError_t configure_poly_kernels(int r)
{
    const int bytes = (int)poly_smem_bytes(r, sizeof(double));
    cudaError_t e = cudaFuncSetAttribute(poly_prolong_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(poly_prolong_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    return e;
}

template <typename T, int TT, int CB>
static void launch_reg(const T *cnew, const T *cold, const float *W, int n, int r, int lo, int win, T *out,
                       cudaStream_t st)
{
    const int nb = n / PP_B;
    poly_prolong_reg_kernel<T, TT, CB><<<nb * nb * nb, PP_THREADS, (size_t)win * win * win * sizeof(T), st>>>(
        cnew, cold, W, n, r, lo, win, out);
}

cudaError_t launch_compose_poly(const double *K2, int r, const float *nu_hat, int n_slices, double *W2,
                                float *Wn, cudaStream_t st)
{
    int TT, lo, win;
    poly_geometry(r, &TT, &lo, &win);
    const int R3 = r * r * r, T3 = TT * TT * TT;
    compose_poly_kernel<<<(2 * R3 * T3 + 127) / 128, 128, 0, st>>>(K2, r, TT, W2);
    compose_poly_slices<<<(n_slices * R3 * (T3 + 1) + 255) / 256, 256, 0, st>>>(W2, nu_hat, n_slices, R3, T3, Wn);
    return cudaGetLastError();
}

template <typename T>
cudaError_t launch_poly_prolong(const T *cnew, const T *cold, const float *W, int n, int r, T *out,
                                cudaStream_t st)
{
    if (n % PP_B || PP_B % r) return cudaErrorInvalidValue;
    int TT, lo, win;
    poly_geometry(r, &TT, &lo, &win);
    if (TT == 4 && r == 4) {
        launch_reg<T, 4, PP_B / 4>(cnew, cold, W, n, r, lo, win, out, st);
    } else if (TT == 3 && r == 8) {
        launch_reg<T, 3, PP_B / 8>(cnew, cold, W, n, r, lo, win, out, st);
    } else {
        const int nb = n / PP_B;
        poly_prolong_kernel<T><<<nb * nb * nb, PP_THREADS, poly_smem_bytes(r, sizeof(T)), st>>>(
            cnew, cold, W, n, r, TT, lo, win, out);
    }
    return cudaGetLastError();
}
template cudaError_t launch_poly_prolong<float>(const float *, const float *, const float *, int, int,
                                                float *, cudaStream_t);
template cudaError_t launch_poly_prolong<double>(const double *, const double *, const float *, int, int,
                                                 double *, cudaStream_t);

}  // namespace pr
