// noalloc.cu -- a defect-norm entry point that allocates nothing.
//
// parareal_diff_norms_noalloc computes the same five numbers as the defect
// norms inside parareal_residual / parareal_iterate -- max|a-b|, max|b|,
// sum (a-b)^2, sum b^2 and a non-finite flag -- for two caller-owned FP64
// device arrays, without a context and without any device allocation.  It is
// meant for callers that cannot call cudaMalloc: code running while a CUDA
// graph is being captured (allocation is not a capturable operation), host
// code inside a framework whose allocator owns all device memory (a second
// allocator would fragment it or break its accounting), and real-time loops
// that must not block on the driver's allocation lock.
//
// The per-block partial results live in a file-scope __device__ array of
// fixed size instead of a cudaMalloc'd buffer.  Every GPU that loads the
// library keeps this array (640 KiB) until the process exits.
#include <cuda_runtime.h>

#include <string>

#include "../../include/parareal.h"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_POINTS_PER_THREAD = 16;
constexpr long long NA_CHUNK = (long long)NA_THREADS * NA_POINTS_PER_THREAD;  // points per block
constexpr int NA_SLOTS = 16384;                                              // blocks per call at most

// Scratch shared by every call on a device: one 5-double partial per block.
// Each call writes every slot it later reads, so nothing must start at zero.
__device__ __align__(256) double g_na_partials[NA_SLOTS * 5];

thread_local std::string g_na_error;

struct NaPartial {
    unsigned long long mx_d, mx_b;
    double s_d, s_b;
    int bad;
};

__device__ __forceinline__ unsigned long long na_abs_bits(double x)
{
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

__device__ void na_block_store(NaPartial p, double *out)
{
    __shared__ NaPartial sh[NA_THREADS / 32];
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long a = __shfl_xor_sync(0xffffffffu, p.mx_d, o);
        const unsigned long long c = __shfl_xor_sync(0xffffffffu, p.mx_b, o);
        p.mx_d = a > p.mx_d ? a : p.mx_d;
        p.mx_b = c > p.mx_b ? c : p.mx_b;
        p.s_d += __shfl_xor_sync(0xffffffffu, p.s_d, o);
        p.s_b += __shfl_xor_sync(0xffffffffu, p.s_b, o);
        p.bad |= __shfl_xor_sync(0xffffffffu, p.bad, o);
    }
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = p;
    __syncthreads();
    if (threadIdx.x == 0) {
        NaPartial t = sh[0];
        for (int w = 1; w < NA_THREADS / 32; ++w) {
            t.mx_d = sh[w].mx_d > t.mx_d ? sh[w].mx_d : t.mx_d;
            t.mx_b = sh[w].mx_b > t.mx_b ? sh[w].mx_b : t.mx_b;
            t.s_d += sh[w].s_d;
            t.s_b += sh[w].s_b;
            t.bad |= sh[w].bad;
        }
        out[0] = __longlong_as_double((long long)t.mx_d);
        out[1] = __longlong_as_double((long long)t.mx_b);
        out[2] = t.s_d;
        out[3] = t.s_b;
        out[4] = t.bad ? 1.0 : 0.0;
    }
}

// Block k reduces points [k*NA_CHUNK, (k+1)*NA_CHUNK) into partials[k].
__global__ void __launch_bounds__(NA_THREADS)
na_diff_kernel(const double *__restrict__ a, const double *__restrict__ b, long long count,
               double *__restrict__ partials)
{
    NaPartial acc{0ull, 0ull, 0.0, 0.0, 0};
    const long long base = (long long)blockIdx.x * NA_CHUNK;
    for (int q = 0; q < NA_POINTS_PER_THREAD; ++q) {
        const long long p = base + (long long)q * NA_THREADS + threadIdx.x;
        if (p >= count) break;
        const double bv = b[p];
        const double d = a[p] - bv;
        const unsigned long long bb = na_abs_bits(bv), bd = na_abs_bits(d);
        acc.bad |= (bd & 0x7ff0000000000000ull) == 0x7ff0000000000000ull;
        acc.mx_b = bb > acc.mx_b ? bb : acc.mx_b;
        acc.mx_d = bd > acc.mx_d ? bd : acc.mx_d;
        acc.s_d = fma(d, d, acc.s_d);
        acc.s_b = fma(bv, bv, acc.s_b);
    }
    na_block_store(acc, partials + 5ll * blockIdx.x);
}

// One block folds the nb partials in a fixed order into out[0..4].
__global__ void __launch_bounds__(NA_THREADS)
na_reduce_kernel(const double *__restrict__ partials, int nb, double *__restrict__ out)
{
    NaPartial acc{0ull, 0ull, 0.0, 0.0, 0};
    for (int k = threadIdx.x; k < nb; k += NA_THREADS) {
        const double *q = partials + 5ll * k;
        const unsigned long long md = (unsigned long long)__double_as_longlong(q[0]);
        const unsigned long long mb = (unsigned long long)__double_as_longlong(q[1]);
        acc.mx_d = md > acc.mx_d ? md : acc.mx_d;
        acc.mx_b = mb > acc.mx_b ? mb : acc.mx_b;
        acc.s_d += q[2];
        acc.s_b += q[3];
        acc.bad |= q[4] != 0.0;
    }
    na_block_store(acc, out);
}

// Device address of g_na_partials, looked up once per device.  In host
// code the symbol g_na_partials names a host-side stand-in, not device
// memory, so it must never be passed to a kernel directly.
constexpr int NA_MAX_DEVICES = 64;
double *g_na_ptr[NA_MAX_DEVICES] = {};

}  // namespace

extern "C" const char *parareal_noalloc_last_error(void) { return g_na_error.c_str(); }

extern "C" parareal_status parareal_diff_norms_noalloc(const double *a, const double *b,
                                                       long long count, double *out5,
                                                       void *cuda_stream)
{
    if (!a || !b || !out5 || count < 1) {
        g_na_error = "need non-null a, b, out5 and count >= 1";
        return PARAREAL_E_INVALID;
    }
    if (count > PARAREAL_NOALLOC_MAX_COUNT) {
        g_na_error = "count " + std::to_string(count) + " exceeds the maximum " +
                     std::to_string((long long)PARAREAL_NOALLOC_MAX_COUNT) +
                     " of parareal_diff_norms_noalloc";
        return PARAREAL_E_INVALID;
    }
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        g_na_error = "no usable current CUDA device";
        return PARAREAL_E_CUDA;
    }
    if (!g_na_ptr[dev]) {
        // first call on this device: resolve the scratch array's device address
        double *p = nullptr;
        e = cudaGetSymbolAddress((void **)&p, g_na_partials);
        if (e != cudaSuccess || !p) {
            g_na_error = std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e);
            return PARAREAL_E_CUDA;
        }
        g_na_ptr[dev] = p;
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    const int nb = (int)((count + NA_CHUNK - 1) / NA_CHUNK);
    na_diff_kernel<<<nb, NA_THREADS, 0, st>>>(a, b, count, g_na_ptr[dev]);
    na_reduce_kernel<<<1, NA_THREADS, 0, st>>>(g_na_ptr[dev], nb, out5);
    e = cudaGetLastError();
    if (e != cudaSuccess) {
        g_na_error = std::string("launch: ") + cudaGetErrorString(e);
        return PARAREAL_E_CUDA;
    }
    return PARAREAL_OK;
}
