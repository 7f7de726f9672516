// correct.cu -- the Parareal correction (Eq. parareal; Algorithm 1,
// "Correction") with the convergence norms of Sec. 2.2.4, in FP64.
//
//   U^{k+1}[n+1] = F(U^k[n]) + (G(U^{k+1}[n]) - G(U^k[n]))
//
// G's two outputs enter only through their difference.  A null Fv or gold
// reads as zero (the start-up chain writes U[n+1] = G(U[n]) this way).  For a coarse-grid G
// (factor r > 1) the difference of the two coarse results, taken in G's
// precision, is prolonged (trilinear; a linear map, so P(c_new) - P(c_old) =
// P(c_new - c_old)) and an unchanged input still gives an exactly zero
// correction.  Every block also
// produces partial norms of dU = U^{k+1} - U^k and of U^{k+1}:
//   {max|dU|, max|U|, sum dU^2, sum U^2, non-finite flag},
// reduced per block with warp shuffles and then across blocks in a fixed
// order, so results are bitwise reproducible.
#include "internal.cuh"

namespace pr {

static constexpr int RED_THREADS = 256;

// Non-negative finite doubles order like their bit patterns; max of |x| is
// taken on the integer bits so the FP64 pipe is spent only on the sums.
__device__ __forceinline__ unsigned long long abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool nonfinite_bits(unsigned long long b)
{
    return (b & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
}

struct Partial {
    unsigned long long mx_d, mx_u;   // bit patterns of max|dU|, max|U|
    double s_d, s_u;
    int bad;
};

__device__ __forceinline__ void warp_reduce(Partial &p)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, p.mx_d, o);
        const unsigned long long b = __shfl_xor_sync(0xffffffffu, p.mx_u, o);
        p.mx_d = a > p.mx_d ? a : p.mx_d;
        p.mx_u = b > p.mx_u ? b : p.mx_u;
        p.s_d += __shfl_xor_sync(0xffffffffu, p.s_d, o);
        p.s_u += __shfl_xor_sync(0xffffffffu, p.s_u, o);
        p.bad |= __shfl_xor_sync(0xffffffffu, p.bad, o);
    }
}

// Block reduction in a fixed order; thread 0 writes 5 doubles at out.
__device__ void block_reduce_store(Partial p, double *out)
{
    __shared__ Partial sh[RED_THREADS / 32];
    warp_reduce(p);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        Partial t = sh[0];
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            t.mx_d = sh[w].mx_d > t.mx_d ? sh[w].mx_d : t.mx_d;
            t.mx_u = sh[w].mx_u > t.mx_u ? sh[w].mx_u : t.mx_u;
            t.s_d += sh[w].s_d;
            t.s_u += sh[w].s_u;
            t.bad |= sh[w].bad;
        }
        out[0] = __longlong_as_double((long long)t.mx_d);
        out[1] = __longlong_as_double((long long)t.mx_u);
        out[2] = t.s_d;
        out[3] = t.s_u;
        out[4] = t.bad ? 1.0 : 0.0;
    }
}

// Trilinear weights along one axis: fine index i, factor r; coarse centroid
// of cell I at fine coordinate I*r + (r-1)/2.  Arithmetic in TP (the coarse
// field's precision).
template <typename TP>
__device__ __forceinline__ void lin_weights(int i, int r, int nc, int &lo, int &hi, TP &w)
{
    const TP s = ((TP)i - (TP)0.5 * (TP)(r - 1)) * ((TP)1 / (TP)r);
    const TP f = floor(s);
    w = s - f;
    lo = (int)f;
    hi = lo + 1;
    lo = lo < 0 ? lo + nc : lo;
    hi = hi >= nc ? hi - nc : hi;
}

// Work is handed out in groups of R = max(1, RED_THREADS / n) rows of n
// points: thread t owns x = t % n of row (t / n) of each group, so x and its
// prolongation weights stay fixed per thread and no point index is divided.
template <typename TF, typename TG>
__global__ void __launch_bounds__(RED_THREADS)
correct_kernel(const TF *__restrict__ Fv, const TG *__restrict__ gnew, const TG *__restrict__ gold,
               double *__restrict__ U, int n, int r, double *__restrict__ partials,
               double *__restrict__ dU)
{
    Partial acc{0ull, 0ull, 0.0, 0.0, 0};
    const int nc = n / r;
    const int R = n >= (int)blockDim.x ? 1 : (int)blockDim.x / n;   // rows per group
    const int lanes = R * n;
    const long long rows = (long long)n * n;
    for (int xs = threadIdx.x % n; xs < n; xs += blockDim.x) {
        if (threadIdx.x >= lanes && n < (int)blockDim.x) break;
        const int x = n >= (int)blockDim.x ? xs : (int)threadIdx.x % n;
        const int rsub = n >= (int)blockDim.x ? 0 : (int)threadIdx.x / n;
        int x0 = 0, x1 = 0;
        TG wx = (TG)0;
        if (r > 1) lin_weights<TG>(x, r, nc, x0, x1, wx);
        for (long long g = blockIdx.x; g * R < rows; g += gridDim.x) {
            const long long row = g * R + rsub;
            if (row >= rows) break;
            const long long p = row * n + x;
            double dg = 0.0;
            if (r == 1) {
                dg = (double)gnew[p] - (gold ? (double)gold[p] : 0.0);
            } else {
                // G's output change on the fine grid: trilinear prolongation
                // of the difference of the two coarse results, taken in the
                // coarse precision TG (one correctly rounded subtraction per
                // corner; no FP64 conversions, which run on the narrow FP64
                // pipe)
                const int z = (int)(row / n), y = (int)(row - (long long)z * n);
                int y0, y1, z0, z1;
                TG wy, wz;
                lin_weights<TG>(y, r, nc, y0, y1, wy);
                lin_weights<TG>(z, r, nc, z0, z1, wz);
                auto dc = [&](int I, int J, int K) -> TG {
                    const long long q = ((long long)K * nc + J) * nc + I;
                    return gold ? gnew[q] - gold[q] : gnew[q];
                };
                const TG c00 = fma(wx, dc(x1, y0, z0) - dc(x0, y0, z0), dc(x0, y0, z0));
                const TG c10 = fma(wx, dc(x1, y1, z0) - dc(x0, y1, z0), dc(x0, y1, z0));
                const TG c01 = fma(wx, dc(x1, y0, z1) - dc(x0, y0, z1), dc(x0, y0, z1));
                const TG c11 = fma(wx, dc(x1, y1, z1) - dc(x0, y1, z1), dc(x0, y1, z1));
                const TG c0 = fma(wy, c10 - c00, c00);
                const TG c1 = fma(wy, c11 - c01, c01);
                dg = (double)fma(wz, c1 - c0, c0);
            }
            const double un = (Fv ? (double)Fv[p] : 0.0) + dg;
            const double du = un - U[p];
            U[p] = un;
            if (dU) dU[p] = du;
            const unsigned long long bu = abs_bits(un), bd = abs_bits(du);
            acc.bad |= nonfinite_bits(bu) ? 1 : 0;
            acc.mx_u = bu > acc.mx_u ? bu : acc.mx_u;
            acc.mx_d = bd > acc.mx_d ? bd : acc.mx_d;
            acc.s_d = fma(du, du, acc.s_d);
            acc.s_u = fma(un, un, acc.s_u);
        }
        if (n < (int)blockDim.x) break;
    }
    block_reduce_store(acc, partials + 5ll * blockIdx.x);
}

int correct_blocks(long long P)
{
    long long b = (P + RED_THREADS - 1) / RED_THREADS;
    const long long cap = 8ll * sm_count();
    return (int)(b < cap ? (b < 1 ? 1 : b) : cap);
}

template <typename TF, typename TG>
cudaError_t launch_correct(const TF *Fv, const TG *gnew, const TG *gold, double *U, int n, int r,
                           double *partials, int nblocks, cudaStream_t st, double *dU)
{
    correct_kernel<TF, TG><<<nblocks, RED_THREADS, 0, st>>>(Fv, gnew, gold, U, n, r, partials, dU);
    return cudaGetLastError();
}
template cudaError_t launch_correct<float, float>(const float *, const float *, const float *,
                                                  double *, int, int, double *, int, cudaStream_t,
                                                  double *);
template cudaError_t launch_correct<float, double>(const float *, const double *, const double *,
                                                   double *, int, int, double *, int, cudaStream_t,
                                                  double *);
template cudaError_t launch_correct<double, double>(const double *, const double *,
                                                    const double *, double *, int, int, double *,
                                                    int, cudaStream_t, double *);
template cudaError_t launch_correct<double, float>(const double *, const float *, const float *,
                                                   double *, int, int, double *, int, cudaStream_t,
                                                  double *);

// max|a - b| and max|b| (the defect d^k of Eq. defect), same partial layout.
template <typename TA>
__global__ void __launch_bounds__(RED_THREADS)
diff_norms_kernel(const TA *__restrict__ a, const double *__restrict__ b, long long P,
                  double *__restrict__ partials)
{
    Partial acc{0ull, 0ull, 0.0, 0.0, 0};
    for (long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x; p < P;
         p += (long long)gridDim.x * blockDim.x) {
        const double bv = b[p];
        const double d = (double)a[p] - bv;
        const unsigned long long bb = abs_bits(bv), bd = abs_bits(d);
        acc.bad |= nonfinite_bits(bd) ? 1 : 0;
        acc.mx_u = bb > acc.mx_u ? bb : acc.mx_u;
        acc.mx_d = bd > acc.mx_d ? bd : acc.mx_d;
        acc.s_d = fma(d, d, acc.s_d);
        acc.s_u = fma(bv, bv, acc.s_u);
    }
    block_reduce_store(acc, partials + 5ll * blockIdx.x);
}

template <typename TA>
cudaError_t launch_diff_norms(const TA *a, const double *b, long long P, double *partials,
                              int nblocks, cudaStream_t st)
{
    diff_norms_kernel<TA><<<nblocks, RED_THREADS, 0, st>>>(a, b, P, partials);
    return cudaGetLastError();
}
template cudaError_t launch_diff_norms<float>(const float *, const double *, long long, double *,
                                              int, cudaStream_t);
template cudaError_t launch_diff_norms<double>(const double *, const double *, long long, double *,
                                               int, cudaStream_t);

// One block: thread t folds blocks t, t+256, ... in order, then a fixed tree.
__global__ void __launch_bounds__(RED_THREADS)
reduce_partials_kernel(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    Partial acc{0ull, 0ull, 0.0, 0.0, 0};
    for (int b = threadIdx.x; b < nb; b += blockDim.x) {
        const double *q = partials + 5ll * b;
        const unsigned long long md = (unsigned long long)__double_as_longlong(q[0]);
        const unsigned long long mu = (unsigned long long)__double_as_longlong(q[1]);
        acc.mx_d = md > acc.mx_d ? md : acc.mx_d;
        acc.mx_u = mu > acc.mx_u ? mu : acc.mx_u;
        acc.s_d += q[2];
        acc.s_u += q[3];
        acc.bad |= q[4] != 0.0;
    }
    block_reduce_store(acc, out);
}

cudaError_t launch_reduce_partials(const double *partials, int nblocks, double *out,
                                   cudaStream_t st)
{
    reduce_partials_kernel<<<1, RED_THREADS, 0, st>>>(partials, nblocks, out);
    return cudaGetLastError();
}

}  // namespace pr
