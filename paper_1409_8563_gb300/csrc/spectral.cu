// spectral.cu -- Fourier restriction and prolongation between the fine n^3
// grid and the coarse m^3 grid (m = n / r) of the stencil coarse propagator
// (Sec. 2.2.2: a coarse propagator on a coarser mesh needs transfer operators
// between the meshes, and their order matters for convergence).
//
// Both transfers keep the Fourier modes with |k_d| <= m/2 - 1 on every axis
// and drop all others, the coarse grid's Nyquist wavenumber m/2 included
// (it has no symmetric partner on the coarse grid).  Coarse point X sits on
// fine point X r.  Along one axis they are the real matrices
//
//   R[X][x] = (1/n) (1 + 2 sum_{k=1}^{m/2-1} cos(2 pi k (X r - x) / n))   (m x n)
//   P[x][X] = r R[X][x]                                                   (n x m)
//
// (the Fourier series truncated to the kept modes, written as a real sum),
// applied one axis after the other: restriction x, y, z; prolongation z, y,
// x.  The matrices are built on the host in FP64 and applied in the coarse
// propagator's precision T.
#include <cmath>
#include <vector>

#include "internal.cuh"

namespace pr {
namespace {

constexpr int SP_THREADS = 256;
// dynamic shared memory the x-pass may use: a 160 KiB matrix plus staged rows
constexpr size_t SP_SMEM_MAX = 200 * 1024;

// out[row][j] = sum_i Mt[i][j] in[row][i] for `rows` rows: the transfer along
// x, the contiguous axis.  Mt is the transposed matrix (len_in x len_out), so
// the lanes of a warp, which take consecutive j, read consecutive words; the
// block's rows are staged in shared memory as T.  A block takes
// max(1, 256 / len_out) rows at a time.  With `old` non-null the input is
// in - old.
template <typename TI, typename T>
__global__ void __launch_bounds__(SP_THREADS)
along_x_kernel(const TI *__restrict__ in, const TI *__restrict__ old, long long rows, int len_in,
               int len_out, const T *__restrict__ Mt, T *__restrict__ out)
{
    extern __shared__ __align__(16) unsigned char sp_smem[];
    T *ms = reinterpret_cast<T *>(sp_smem);                 // Mt: len_in x len_out
    const int rpb = len_out >= SP_THREADS ? 1 : SP_THREADS / len_out;
    T *xs = ms + (size_t)len_in * len_out;                  // rpb rows of len_in
    for (int i = threadIdx.x; i < len_in * len_out; i += blockDim.x) ms[i] = Mt[i];
    const int rl = threadIdx.x / (len_out >= SP_THREADS ? SP_THREADS : len_out);
    for (long long r0 = (long long)blockIdx.x * rpb; r0 < rows; r0 += (long long)gridDim.x * rpb) {
        __syncthreads();
        for (int i = threadIdx.x; i < rpb * len_in; i += blockDim.x) {
            const long long row = r0 + i / len_in;
            const long long q = row * len_in + i % len_in;
            xs[i] = row < rows ? (old ? (T)(in[q] - old[q]) : (T)in[q]) : (T)0;
        }
        __syncthreads();
        const long long row = r0 + rl;
        if (rl >= rpb || row >= rows) continue;
        const T *x = xs + rl * len_in;
        for (int j = threadIdx.x % (len_out >= SP_THREADS ? SP_THREADS : len_out); j < len_out;
             j += SP_THREADS) {
            T acc = (T)0;
            for (int i = 0; i < len_in; ++i) acc = fma(ms[i * len_out + j], x[i], acc);
            out[row * len_out + j] = acc;
        }
    }
}

// out[a][j][b] = sum_i M[j][i] in[a][i][b] (a < na, b < nb): the transfer
// along a strided axis (y or z).  One thread per output, b fastest, so the
// loads of `in` are coalesced and the matrix entry is shared by the warp.
// With `old` non-null the input is in - old.
template <typename TI, typename T>
__global__ void __launch_bounds__(SP_THREADS)
along_strided_kernel(const TI *__restrict__ in, const TI *__restrict__ old, int na, int len_in,
                     int len_out, int nb, const T *__restrict__ M, T *__restrict__ out)
{
    const long long total = (long long)na * len_out * nb;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int b = (int)(q % nb);
        const int j = (int)((q / nb) % len_out);
        const long long a = q / ((long long)nb * len_out);
        const TI *src = in + a * len_in * (long long)nb + b;
        const TI *srco = old ? old + a * len_in * (long long)nb + b : nullptr;
        const T *mrow = M + (long long)j * len_in;
        T acc = (T)0;
        for (int i = 0; i < len_in; ++i) {
            const T v = srco ? (T)(src[(long long)i * nb] - srco[(long long)i * nb])
                             : (T)src[(long long)i * nb];
            acc = fma(__ldg(mrow + i), v, acc);
        }
        out[q] = acc;
    }
}

unsigned grid_of(long long work)
{
    const long long b = (work + SP_THREADS - 1) / SP_THREADS;
    const long long cap = 8ll * sm_count();
    return (unsigned)(b < 1 ? 1 : (b < cap ? b : cap));
}

template <typename TI, typename T>
cudaError_t along_x(const TI *in, const TI *old, long long rows, int len_in, int len_out,
                    const T *Mt, T *out, cudaStream_t st)
{
    const int rpb = len_out >= SP_THREADS ? 1 : SP_THREADS / len_out;
    const size_t smem = ((size_t)len_in * len_out + (size_t)rpb * len_in) * sizeof(T);
    if (smem > SP_SMEM_MAX) return cudaErrorInvalidValue;
    const long long blocks = (rows + rpb - 1) / rpb;
    const long long cap = 4ll * sm_count();
    along_x_kernel<TI, T><<<(unsigned)(blocks < cap ? blocks : cap), SP_THREADS, smem, st>>>(
        in, old, rows, len_in, len_out, Mt, out);
    return cudaGetLastError();
}

template <typename TI, typename T>
cudaError_t along_strided(const TI *in, const TI *old, int na, int len_in, int len_out, int nb,
                          const T *M, T *out, cudaStream_t st)
{
    along_strided_kernel<TI, T><<<grid_of((long long)na * len_out * nb), SP_THREADS, 0, st>>>(
        in, old, na, len_in, len_out, nb, M, out);
    return cudaGetLastError();
}

}  // namespace

cudaError_t configure_spectral_kernels()
{
    cudaError_t e = cudaSuccess;
    auto conf = [&](const void *fn) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SP_SMEM_MAX);
    };
    conf((const void *)along_x_kernel<double, float>);
    conf((const void *)along_x_kernel<float, float>);
    conf((const void *)along_x_kernel<double, double>);
    return e;
}

void spectral_matrices(int n, int r, std::vector<double> *R, std::vector<double> *Rt,
                       std::vector<double> *P, std::vector<double> *Pt)
{
    const int m = n / r;
    const double pi = 3.14159265358979323846;
    R->assign((size_t)m * n, 0.0);
    Rt->assign((size_t)n * m, 0.0);
    P->assign((size_t)n * m, 0.0);
    Pt->assign((size_t)m * n, 0.0);
    for (int X = 0; X < m; ++X)
        for (int x = 0; x < n; ++x) {
            double s = 1.0;
            for (int k = 1; k <= m / 2 - 1; ++k) s += 2.0 * std::cos(2.0 * pi * k * (double)(X * r - x) / n);
            const double rv = s / n;
            (*R)[(size_t)X * n + x] = rv;
            (*Rt)[(size_t)x * m + X] = rv;
            (*P)[(size_t)x * m + X] = r * rv;
            (*Pt)[(size_t)X * n + x] = r * rv;
        }
}

size_t spectral_work_elems(int n, int r)
{
    const long long m = n / r;
    return (size_t)((long long)n * n * m + (long long)n * m * m);
}

template <typename T>
cudaError_t launch_restrict_spectral(const double *fine, int n, int r, const T *R, const T *Rt,
                                     T *work, T *coarse, cudaStream_t st)
{
    const int m = n / r;
    T *t1 = work;                                  // [n][n][m]
    T *t2 = work + (size_t)n * n * m;              // [n][m][m]
    cudaError_t e = along_x<double, T>(fine, nullptr, (long long)n * n, n, m, Rt, t1, st);
    if (e == cudaSuccess) e = along_strided<T, T>(t1, nullptr, n, n, m, m, R, t2, st);
    if (e == cudaSuccess) e = along_strided<T, T>(t2, nullptr, 1, n, m, m * m, R, coarse, st);
    return e;
}

template <typename T>
cudaError_t launch_prolong_spectral(const T *cnew, const T *cold, int n, int r, const T *P,
                                    const T *Pt, T *work, T *fine, cudaStream_t st)
{
    const int m = n / r;
    T *c1 = work + (size_t)n * n * m;              // [n][m][m]
    T *c2 = work;                                  // [n][n][m]
    cudaError_t e = along_strided<T, T>(cnew, cold, 1, m, n, m * m, P, c1, st);
    if (e == cudaSuccess) e = along_strided<T, T>(c1, nullptr, n, m, n, m, P, c2, st);
    if (e == cudaSuccess) e = along_x<T, T>(c2, nullptr, (long long)n * n, m, n, Pt, fine, st);
    return e;
}

template cudaError_t launch_restrict_spectral<float>(const double *, int, int, const float *,
                                                     const float *, float *, float *, cudaStream_t);
template cudaError_t launch_restrict_spectral<double>(const double *, int, int, const double *,
                                                      const double *, double *, double *, cudaStream_t);
template cudaError_t launch_prolong_spectral<float>(const float *, const float *, int, int,
                                                    const float *, const float *, float *, float *,
                                                    cudaStream_t);
template cudaError_t launch_prolong_spectral<double>(const double *, const double *, int, int,
                                                     const double *, const double *, double *,
                                                     double *, cudaStream_t);

}  // namespace pr
