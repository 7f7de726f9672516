// net_composed.cu -- the LINEAR learned coarse propagator evaluated as one
// 9x9x9 periodic cross-correlation.
//
// With identity activations and no biases the four layers are linear maps,
// and cross-correlations compose by adding offsets:
//   (W2 (W1 x))[p] = sum_{d1,d2} W2[d2] W1[d1] x[p + d1 + d2]
// (channels contracted in between).  The second input channel is
// nu_hat * S(u), so
//   Net(S(u))[p] = sum_e K[e] S(u)[p + e],  e in [-4,4]^3,  K = K_0 + nu_hat K_1,
// K_c the kernel of input channel c of layer 1 carried through layers 2-4.
// compose_* build K_0 and K_1 in FP64 from the FP32 master weights (once per
// model) and the per-slice kernels in FP32; net_lin9_kernel applies one of
// them with FP32 accumulation: 729 multiply-adds per point against the
// ~14.7k of the four layers.  The result is the same linear operator as the
// layer-by-layer evaluation, without its BF16 rounding of weights and
// activations.
#include "internal.cuh"
#include "net.cuh"

namespace pr {

// Edges of the composed kernels after layers 1..4: 3, 5, 7, 9.
constexpr int COMPOSE_MAX = 2 * 16 * 7 * 7 * 7;   // largest intermediate (after layer 3)

// A[c][co][tap] = W1[co][c][tap] (c = input channel 0 / 1, radius 1).
__global__ void compose_first(const float *__restrict__ master, double *__restrict__ A)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;   // (c * 16 + co) * 27 + tap
    if (j >= 2 * 16 * 27) return;
    const int tap = j % 27, co = (j / 27) % 16, c = j / (27 * 16);
    A[j] = (double)master[NET_W1 + (co * 2 + c) * 27 + tap];
}

// One more layer: B[c][co][b] = sum_ci sum_d W[co][ci][d] A[c][ci][b - d],
// A of edge ea = 2R+1 (index a = e + R), B of edge ea + 2 (index b = e' + R + 1),
// d = tap offset + 1 in {0,1,2}^3.  W in master order [co][ci][27].
__global__ void compose_next(const double *__restrict__ A, int ea, int cin,
                             const float *__restrict__ W, int cout, double *__restrict__ B)
{
    const int eb = ea + 2;
    const int nb = eb * eb * eb;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;   // (c * cout + co) * nb + b
    if (j >= 2 * cout * nb) return;
    const int q = j % nb, co = (j / nb) % cout, c = j / (nb * cout);
    const int bx = q % eb, by = (q / eb) % eb, bz = q / (eb * eb);
    double s = 0.0;
    for (int ci = 0; ci < cin; ++ci) {
        const double *Ac = A + (size_t)(c * cin + ci) * ea * ea * ea;
        const float *Wc = W + (co * cin + ci) * 27;
        for (int dz = 0; dz < 3; ++dz) {
            const int az = bz - dz;
            if (az < 0 || az >= ea) continue;
            for (int dy = 0; dy < 3; ++dy) {
                const int ay = by - dy;
                if (ay < 0 || ay >= ea) continue;
                for (int dx = 0; dx < 3; ++dx) {
                    const int ax = bx - dx;
                    if (ax < 0 || ax >= ea) continue;
                    s += (double)Wc[(dz * 3 + dy) * 3 + dx] * Ac[(az * ea + ay) * ea + ax];
                }
            }
        }
    }
    B[j] = s;
}

// keff[n][e] = K_0[e] + nu_hat[n] K_1[e] for every slice n (K: [2][729]).
__global__ void compose_slices(const double *__restrict__ K, const float *__restrict__ nu_hat,
                               int n_slices, float *__restrict__ keff)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n_slices * NET_K9) return;
    const int e = j % NET_K9, n = j / NET_K9;
    keff[j] = (float)(K[e] + (double)nu_hat[n] * K[NET_K9 + e]);
}

cudaError_t launch_compose_linear(const float *master, const float *nu_hat, int n_slices,
                                  double *scratch, float *keff, cudaStream_t st)
{
    double *A = scratch, *B = scratch + COMPOSE_MAX;
    compose_first<<<(2 * 16 * 27 + 255) / 256, 256, 0, st>>>(master, A);
    // layer 2 (16 -> 16), layer 3 (16 -> 16), layer 4 (16 -> 1)
    compose_next<<<(2 * 16 * 125 + 127) / 128, 128, 0, st>>>(A, 3, 16, master + NET_W2, 16, B);
    compose_next<<<(2 * 16 * 343 + 127) / 128, 128, 0, st>>>(B, 5, 16, master + NET_W3, 16, A);
    compose_next<<<(2 * NET_K9 + 127) / 128, 128, 0, st>>>(A, 7, 16, master + NET_W4, 1, B);
    compose_slices<<<(n_slices * NET_K9 + 255) / 256, 256, 0, st>>>(B, nu_hat, n_slices, keff);
    return cudaGetLastError();
}

size_t compose_scratch_doubles() { return 2 * (size_t)COMPOSE_MAX; }

const double *composed_kernels(const double *scratch) { return scratch + COMPOSE_MAX; }

// out[p] = x[p] + sum_e K[e] x[p + e], x = S(u), S(u)[q] = u[q - s] (periodic
// shift s in [0, m)^3), K the slice's kernel in device memory.  One CTA of
// 128 threads per 8 x 8 x 16 output tile: the 16 x 16 x 24 halo of x in
// shared memory as FP32 (wrapped coordinates from per-axis tables), rows
// padded to 20 values so that the 16-byte loads of the 8 threads of a
// quarter warp (8 consecutive rows) hit distinct banks, and the 729 weights
// in rows of 12.  Each thread accumulates one x row of 8 points: per kernel
// row 4 vector loads of x, 3 broadcast loads of weights and 72 FMAs.  Only
// the y and x offsets are unrolled (the loop over z offsets keeps the code
// within the instruction cache).  The skip term is added in FP64 from u.
template <typename TU, typename TG>
__global__ void __launch_bounds__(128)
net_lin9_kernel(const TU *__restrict__ u, int m, int sx, int sy, int sz, const float *__restrict__ K,
                TG *__restrict__ out)
{
    constexpr int SX = 20, HY = 16, HZ = 24;
    __shared__ __align__(16) float xs[HZ * HY * SX];
    __shared__ __align__(16) float ws[81 * 12];
    __shared__ int gtab[3][24];                    // wrapped halo coordinates per axis
    const int mt = m >> 3, mz = m >> 4;
    const int ox = (blockIdx.x % mt) * 8, oy = ((blockIdx.x / mt) % mt) * 8, oz = (blockIdx.x / (mt * mt)) * 16;
    (void)mz;
    auto wrapm = [m](int v) { v %= m; return v < 0 ? v + m : v; };
    if (threadIdx.x < 72) {
        const int ax = threadIdx.x / 24, h = threadIdx.x % 24;
        const int o = ax == 0 ? ox - sx : (ax == 1 ? oy - sy : oz - sz);
        gtab[ax][h] = wrapm(o - 4 + h);
    }
    for (int i = threadIdx.x; i < 81 * 12; i += blockDim.x) {
        const int r = i / 12, k = i % 12;
        ws[i] = k < 9 ? K[r * 9 + k] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int i = threadIdx.x; i < HZ * HY * 16; i += blockDim.x) {
        const int hx = i & 15, hy = (i >> 4) & 15, hz = i >> 8;
        xs[(hz * HY + hy) * SX + hx] = (float)u[((long long)gtab[2][hz] * m + gtab[1][hy]) * m + gtab[0][hx]];
    }
    __syncthreads();
    const int y = threadIdx.x & 7, z = threadIdx.x >> 3;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll 1
    for (int dz = 0; dz < 9; ++dz) {
        const float *plane = xs + (z + dz) * HY * SX;
        const float *wplane = ws + dz * 9 * 12;
#pragma unroll
        for (int dy = 0; dy < 9; ++dy) {
            const float4 *row = reinterpret_cast<const float4 *>(plane + (y + dy) * SX);
            const float4 q0 = row[0], q1 = row[1], q2 = row[2], q3 = row[3];
            const float v[16] = {q0.x, q0.y, q0.z, q0.w, q1.x, q1.y, q1.z, q1.w,
                                 q2.x, q2.y, q2.z, q2.w, q3.x, q3.y, q3.z, q3.w};
            const float4 *wr = reinterpret_cast<const float4 *>(wplane + dy * 12);
            const float4 w0 = wr[0], w1 = wr[1], w2 = wr[2];
            const float w[9] = {w0.x, w0.y, w0.z, w0.w, w1.x, w1.y, w1.z, w1.w, w2.x};
#pragma unroll
            for (int dx = 0; dx < 9; ++dx)
#pragma unroll
                for (int i = 0; i < 8; ++i) acc[i] = fmaf(w[dx], v[i + dx], acc[i]);
        }
    }
    const long long row = ((long long)(oz + z) * m + (oy + y)) * m + ox;
    const long long qrow = ((long long)gtab[2][z + 4] * m + gtab[1][y + 4]) * m;
#pragma unroll
    for (int i = 0; i < 8; ++i)
        out[row + i] = (TG)((double)u[qrow + gtab[0][i + 4]] + (double)acc[i]);
}

template <typename TU, typename TG>
cudaError_t launch_net_lin9(const TU *u, int m, const int s[3], const float *K, TG *out, cudaStream_t st)
{
    if (m % 16) return cudaErrorInvalidValue;
    const unsigned tiles = (unsigned)((m / 8) * (m / 8) * (m / 16));
    net_lin9_kernel<TU, TG><<<tiles, 128, 0, st>>>(u, m, s[0], s[1], s[2], K, out);
    return cudaGetLastError();
}
template cudaError_t launch_net_lin9<double, double>(const double *, int, const int *, const float *, double *, cudaStream_t);
template cudaError_t launch_net_lin9<float, float>(const float *, int, const int *, const float *, float *, cudaStream_t);
template cudaError_t launch_net_lin9<double, float>(const double *, int, const int *, const float *, float *, cudaStream_t);
template cudaError_t launch_net_lin9<float, double>(const float *, int, const int *, const float *, double *, cudaStream_t);

}  // namespace pr
