// net.cu -- the learned coarse propagator's kernels (forward, backward, Adam).
//
//   G(u, t_n) = S(u) + Net([S(u), nu(t_n)/nu0]),
//   Net = conv3(2->16) GELU conv3(16->16) GELU conv3(16->16) GELU conv3(16->1)
//
// with S the skip propagator (periodic integer shift, or the stencil
// propagator) and conv3 a periodic 3x3x3 cross-correlation.  Linear mode
// (lin != 0): identity activations, no biases, and the second input channel
// nu_hat * S(u) instead of the constant nu_hat, so that G is linear in u with
// a kernel that depends on nu(t_n).  Storage: activations channels-last in BF16
// ([point][16], 32 bytes per point), pre-activations in FP32, weights as FP32
// masters with BF16 operand copies; all accumulation in FP32.
//
// The 16->16 layers (and their input gradients) are implicit GEMMs with
// M = points, N = 16 output channels, K = 27 taps x 16 input channels: one
// CTA stages an 8x8x8 output tile plus halo (10^3 points) in shared memory
// and each warp runs mma.sync m16n8k16 BF16 over 4 row tiles of 16 points,
// gathering the 16 rows of each tap with ldmatrix (one row = one point's 16
// channels).  The weight gradient is the transposed GEMM (M = 16 input
// channels, N = 16 output channels, K = points) per tap, split over CTAs with
// a fixed-order reduction.  The thin layers (2->16, 16->1) run on CUDA cores.
//
// Shared-memory rows are swizzled: 16-byte chunk h (0/1) of halo point q sits
// at chunk 2q + (h ^ ((q >> 2) & 1)), so 8 consecutive points hit 8 distinct
// bank groups.
#include <cuda_bf16.h>

#include "internal.cuh"
#include "net.cuh"

namespace pr {

using bf16 = __nv_bfloat16;

__device__ __forceinline__ float gelu_f(float x)
{
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
           x * 0.39894228040143268f * __expf(-0.5f * x * x);
}
__device__ __forceinline__ float bf16r(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }

__device__ __forceinline__ int wrap(int i, int m) { return i < 0 ? i + m : (i >= m ? i - m : i); }

__device__ __forceinline__ int chunk(int q, int h) { return 2 * q + (h ^ ((q >> 2) & 1)); }

// Tile decomposition: blockIdx.x = tile within a sample, blockIdx.y = sample.
struct Tile {
    int ox, oy, oz;
};
__device__ __forceinline__ Tile tile_of(int t, int m)
{
    const int mt = m >> 3;
    Tile r;
    r.ox = (t % mt) * 8;
    r.oy = ((t / mt) % mt) * 8;
    r.oz = (t / (mt * mt)) * 8;
    return r;
}

__device__ __forceinline__ unsigned smem_u32(const void *p)
{
    return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void ldsm_x4(unsigned addr, unsigned (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x2(unsigned addr, unsigned (&r)[2])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n"
                 : "=r"(r[0]), "=r"(r[1])
                 : "r"(addr));
}
__device__ __forceinline__ void ldsm_x4_t(unsigned addr, unsigned (&r)[4])
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
                 : "r"(addr));
}
__device__ __forceinline__ void mma_bf16(float (&d)[4], const unsigned (&a)[4], unsigned b0,
                                         unsigned b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Load the 10^3 halo of a [P][16] BF16 field (swizzled chunks) into smem:
// 16-byte asynchronous copies, all in flight before the thread waits for its
// own (the caller's barrier then publishes them to the block).
__device__ __forceinline__ void load_halo16(uint4 *sm, const bf16 *__restrict__ in, const Tile &T,
                                            int m)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(in);
    for (int i = threadIdx.x; i < 2000; i += blockDim.x) {
        const int q = i >> 1, h = i & 1;
        const int hx = q % 10, hy = (q / 10) % 10, hz = q / 100;
        const int gx = wrap(T.ox + hx - 1, m), gy = wrap(T.oy + hy - 1, m), gz = wrap(T.oz + hz - 1, m);
        const long long p = ((long long)gz * m + gy) * m + gx;
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n"
                     ::"r"((unsigned)__cvta_generic_to_shared(sm + chunk(q, h))), "l"(src + 2 * p + h)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
}

// ---------------------------------------------------------------- layer 1

// z1 = conv(x0, W1) + b1, a1 = bf16(gelu(z1)), x0 = [bf16(S(u)), bf16(nu_hat)].
// Linear mode: x0 = [bf16(S(u)), bf16(nu_hat) bf16(S(u))], no bias, a1 = bf16(z1);
// the two channels share their input, so their weights are combined per sample.
// 128 threads per 8^3 tile, 4 consecutive x points per thread, so each weight
// read from shared memory feeds four FMAs.
template <typename TU>
__global__ void __launch_bounds__(128)
net_in_fwd(const TU *__restrict__ u, int m, int sx, int sy, int sz, const float *__restrict__ nu_hat,
           const float *__restrict__ W1q, const float *__restrict__ b1, float *__restrict__ z1,
           bf16 *__restrict__ a1, int lin)
{
    __shared__ float xs[1000];
    __shared__ __align__(16) float w[27 * 16];     // [tap][channel]
    __shared__ float beff[16];
    const int s = blockIdx.y;
    const long long P = (long long)m * m * m;
    const Tile T = tile_of(blockIdx.x, m);
    const TU *us = u + s * P;
    for (int i = threadIdx.x; i < 1000; i += blockDim.x) {
        const int hx = i % 10, hy = (i / 10) % 10, hz = i / 100;
        const int gx = wrap(wrap(T.ox + hx - 1, m) - sx + m, m);
        const int gy = wrap(wrap(T.oy + hy - 1, m) - sy + m, m);
        const int gz = wrap(wrap(T.oz + hz - 1, m) - sz + m, m);
        xs[i] = bf16r((float)us[((long long)gz * m + gy) * m + gx]);
    }
    const float nq = bf16r(nu_hat[s]);
    for (int i = threadIdx.x; i < 16 * 27; i += blockDim.x) {
        const int c = i / 27, t = i % 27;
        w[t * 16 + c] = lin ? fmaf(nq, W1q[c * 54 + 27 + t], W1q[c * 54 + t]) : W1q[c * 54 + t];
    }
    if (threadIdx.x < 16) {
        float acc = lin ? 0.f : b1[threadIdx.x];
        if (!lin)
            for (int t = 0; t < 27; ++t) acc = fmaf(W1q[threadIdx.x * 54 + 27 + t], nq, acc);
        beff[threadIdx.x] = acc;
    }
    __syncthreads();
    const int lx0 = (threadIdx.x & 1) * 4, ly = (threadIdx.x >> 1) & 7, lz = threadIdx.x >> 4;
    float acc[4][16];
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[k][c] = beff[c];
    for (int dz = 0; dz < 3; ++dz)
        for (int dy = 0; dy < 3; ++dy) {
            const float *row = xs + ((lz + dz) * 10 + (ly + dy)) * 10 + lx0;
            float v[6];
#pragma unroll
            for (int i = 0; i < 6; ++i) v[i] = row[i];
#pragma unroll
            for (int dx = 0; dx < 3; ++dx) {
                const float4 *wt = reinterpret_cast<const float4 *>(w + ((dz * 3 + dy) * 3 + dx) * 16);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float4 wq = wt[q];
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
                        acc[k][4 * q + 0] = fmaf(wq.x, v[k + dx], acc[k][4 * q + 0]);
                        acc[k][4 * q + 1] = fmaf(wq.y, v[k + dx], acc[k][4 * q + 1]);
                        acc[k][4 * q + 2] = fmaf(wq.z, v[k + dx], acc[k][4 * q + 2]);
                        acc[k][4 * q + 3] = fmaf(wq.w, v[k + dx], acc[k][4 * q + 3]);
                    }
                }
            }
        }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const long long p = s * P + ((long long)(T.oz + lz) * m + (T.oy + ly)) * m + T.ox + lx0 + k;
        if (z1) {
            float4 *zp = reinterpret_cast<float4 *>(z1 + 16 * p);
#pragma unroll
            for (int c = 0; c < 4; ++c)
                zp[c] = make_float4(acc[k][4 * c], acc[k][4 * c + 1], acc[k][4 * c + 2], acc[k][4 * c + 3]);
        }
        __align__(16) bf16 o[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(lin ? acc[k][c] : gelu_f(acc[k][c]));
        uint4 *ap = reinterpret_cast<uint4 *>(a1 + 16 * p);
        ap[0] = reinterpret_cast<const uint4 *>(o)[0];
        ap[1] = reinterpret_cast<const uint4 *>(o)[1];
    }
}

// --------------------------------------------------------- 16 -> 16 layers

// MODE 0 (forward):  out = bf16(gelu(acc + bias)), zout = acc + bias (if non-null)
// MODE 1 (dgrad):    out = bf16(acc * gelu'(zaux))
// (linear mode: no bias, identity activation, so out = bf16(acc) in both)
// acc[p][n] = sum_tap sum_k in[p + tap][k] * Bt[tap][n][k]
template <int MODE>
__global__ void __launch_bounds__(256)
net_mid(const bf16 *__restrict__ in, int m, const bf16 *__restrict__ Bt, const float *__restrict__ bias,
        const float *__restrict__ zaux, float *__restrict__ zout, bf16 *__restrict__ out, int lin)
{
    extern __shared__ uint4 sm_mid[];
    uint4 *act = sm_mid;               // 2000 chunks: [1000 points][2]
    uint4 *bs = sm_mid + 2000;         // 864 chunks:  [27][16 n][2]
    const int s = blockIdx.y;
    const long long P = (long long)m * m * m;
    const Tile T = tile_of(blockIdx.x, m);
    load_halo16(act, in + 16 * s * P, T, m);
    for (int i = threadIdx.x; i < 864; i += blockDim.x) bs[i] = reinterpret_cast<const uint4 *>(Bt)[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float acc[4][2][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;

    const int arow = (lane & 7) + ((lane >> 3) & 1) * 8;   // A row this lane addresses
    const int akh = lane >> 4;                             // its K half
    const int bj = lane >> 3, br = lane & 7;               // B matrix / row this lane addresses
    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        unsigned b[4];
        ldsm_x4(smem_u32(bs + (t * 16 + (bj >> 1) * 8 + br) * 2 + (bj & 1)), b);
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int x = arow & 7, y = 2 * mt + (arow >> 3), z = w;
            const int q = ((z + 1 + dz) * 10 + (y + 1 + dy)) * 10 + (x + 1 + dx);
            unsigned a[4];
            ldsm_x4(smem_u32(act + chunk(q, akh)), a);
            mma_bf16(acc[mt][0], a, b[0], b[1]);
            mma_bf16(acc[mt][1], a, b[2], b[3]);
        }
    }

    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int mt = 0; mt < 4; ++mt)
#pragma unroll
        for (int hh = 0; hh < 2; ++hh) {
            const int row = g + 8 * hh;
            const int x = row & 7, y = 2 * mt + (row >> 3), z = w;
            const long long p = s * P + ((long long)(T.oz + z) * m + (T.oy + y)) * m + T.ox + x;
#pragma unroll
            for (int nt = 0; nt < 2; ++nt) {
                const int co = nt * 8 + 2 * tq;
                float v0 = acc[mt][nt][2 * hh], v1 = acc[mt][nt][2 * hh + 1];
                if (lin) {
                    if (MODE == 0 && zout)
                        *reinterpret_cast<float2 *>(zout + 16 * p + co) = make_float2(v0, v1);
                } else if (MODE == 0) {
                    v0 += bias[co];
                    v1 += bias[co + 1];
                    if (zout) *reinterpret_cast<float2 *>(zout + 16 * p + co) = make_float2(v0, v1);
                    v0 = gelu_f(v0);
                    v1 = gelu_f(v1);
                } else {
                    const float2 zz = *reinterpret_cast<const float2 *>(zaux + 16 * p + co);
                    v0 *= gelu_grad_f(zz.x);
                    v1 *= gelu_grad_f(zz.y);
                }
                *reinterpret_cast<__nv_bfloat162 *>(out + 16 * p + co) = __floats2bfloat162_rn(v0, v1);
            }
        }
}

// dW[tap][ci][co] += sum_p x[p + tap][ci] dz[p][co]; db[co] += sum_p dz[p][co].
// Each CTA walks tiles t = blockIdx.x, + gridDim.x, ... over all samples and
// writes one partial [27*256 + 16] at partials + blockIdx.x * NET_MID_PARTIAL.
__global__ void __launch_bounds__(256)
net_mid_wgrad(const bf16 *__restrict__ x, const bf16 *__restrict__ dz, int m, int tiles_total,
              float *__restrict__ partials)
{
    extern __shared__ uint4 sm_wg[];
    uint4 *xs = sm_wg;                 // 2000 chunks (halo of x)
    uint4 *ds = sm_wg + 2000;          // 1024 chunks (tile of dz, 512 points)
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long P = (long long)m * m * m;
    const int tiles = (m >> 3) * (m >> 3) * (m >> 3);
    // taps of this warp: w, w+8, w+16, w+24 (< 27)
    float acc[4][2][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[a][b][c] = 0.f;
    float dbias = 0.f;
    const int j = lane >> 3, r = lane & 7;
    for (int tt = blockIdx.x; tt < tiles_total; tt += gridDim.x) {
        const int s = tt / tiles;
        const Tile T = tile_of(tt % tiles, m);
        __syncthreads();
        load_halo16(xs, x + 16 * s * P, T, m);
        for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
            const int q = i >> 1, h = i & 1;
            const int lx = q & 7, ly = (q >> 3) & 7, lz = q >> 6;
            const long long p = s * P + ((long long)(T.oz + lz) * m + (T.oy + ly)) * m + T.ox + lx;
            ds[chunk(q, h)] = reinterpret_cast<const uint4 *>(dz)[2 * p + h];
        }
        __syncthreads();
        if (threadIdx.x < 16) {
            const bf16 *d16 = reinterpret_cast<const bf16 *>(ds);
            for (int q = 0; q < 512; ++q) {
                const int c = threadIdx.x;
                dbias += __bfloat162float(d16[chunk(q, c >> 3) * 8 + (c & 7)]);
            }
        }
        for (int ks = 0; ks < 32; ++ks) {
            // B: rows = 16 points (k), cols = 16 output channels (n)
            unsigned b[4];
            {
                const int q = ks * 16 + r + 8 * (j & 1);
                ldsm_x4_t(smem_u32(ds + chunk(q, j >> 1)), b);
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const int t = w + 8 * k;
                if (t < 27) {
                    const int dz_ = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                    const int q = ks * 16 + r + 8 * (j >> 1);
                    const int lx = q & 7, ly = (q >> 3) & 7, lz = q >> 6;
                    const int hq = ((lz + 1 + dz_) * 10 + (ly + 1 + dy)) * 10 + (lx + 1 + dx);
                    unsigned a[4];
                    ldsm_x4_t(smem_u32(xs + chunk(hq, j & 1)), a);
                    mma_bf16(acc[k][0], a, b[0], b[1]);
                    mma_bf16(acc[k][1], a, b[2], b[3]);
                }
            }
        }
    }
    float *out = partials + (long long)blockIdx.x * NET_MID_PARTIAL;
    const int g = lane >> 2, tq = lane & 3;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int t = w + 8 * k;
        if (t >= 27) continue;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int ci = g + 8 * hh, co = nt * 8 + 2 * tq;
                out[t * 256 + ci * 16 + co] = acc[k][nt][2 * hh];
                out[t * 256 + ci * 16 + co + 1] = acc[k][nt][2 * hh + 1];
            }
    }
    if (threadIdx.x < 16) out[27 * 256 + threadIdx.x] = dbias;
}

// ---------------------------------------------------------------- layer 4

// The last layer on the tensor cores: the 16 -> 1 convolution as an implicit
// GEMM with N = 8 (output channel 0; B rows 1-7 are zero), the same tiling as
// net_mid, and the epilogue g = S(u) + z4, z4 = acc + b4 (no bias in linear
// mode), written in TG if g_out is non-null.  With a target (training):
// r = g - tgt, dz4 = bf16(r * grad_scale), and the block's sum of r^2 (fixed
// order) into loss_partials[tile].
template <typename TU, typename TG>
__global__ void __launch_bounds__(256)
net_out_mma(const bf16 *__restrict__ a3, int m, const bf16 *__restrict__ B4, const float *__restrict__ b4,
            const TU *__restrict__ u, int sx, int sy, int sz, TG *__restrict__ g_out, int lin,
            const float *__restrict__ tgt, float grad_scale, bf16 *__restrict__ dz4,
            double *__restrict__ loss_partials)
{
    __shared__ double red[8];
    extern __shared__ uint4 sm_om[];
    uint4 *act = sm_om;                // 2000 chunks
    uint4 *bs = sm_om + 2000;          // 432 chunks: [27][8 n][2]
    const int s = blockIdx.y;
    const long long P = (long long)m * m * m;
    const Tile T = tile_of(blockIdx.x, m);
    load_halo16(act, a3 + 16 * s * P, T, m);
    for (int i = threadIdx.x; i < 432; i += blockDim.x) bs[i] = reinterpret_cast<const uint4 *>(B4)[i];
    __syncthreads();

    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    float acc[4][4];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[a][c] = 0.f;
    const int arow = (lane & 7) + ((lane >> 3) & 1) * 8;
    const int akh = lane >> 4;
    const int bh = (lane >> 3) & 1, br = lane & 7;
    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        unsigned b[2];
        ldsm_x2(smem_u32(bs + (t * 8 + br) * 2 + bh), b);
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            const int x = arow & 7, y = 2 * mt + (arow >> 3), z = w;
            const int q = ((z + 1 + dz) * 10 + (y + 1 + dy)) * 10 + (x + 1 + dx);
            unsigned a[4];
            ldsm_x4(smem_u32(act + chunk(q, akh)), a);
            mma_bf16(acc[mt], a, b[0], b[1]);
        }
    }
    // output channel 0 sits in column 0 of the accumulator: lanes with tq == 0
    const int g = lane >> 2, tq = lane & 3;
    const float bias = lin ? 0.f : b4[0];
    double l = 0.0;
    if (tq == 0) {
#pragma unroll
        for (int mt = 0; mt < 4; ++mt)
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const int row = g + 8 * hh;
                const int x = row & 7, y = 2 * mt + (row >> 3), z = w;
                const int gx = T.ox + x, gy = T.oy + y, gz = T.oz + z;
                const long long p = ((long long)gz * m + gy) * m + gx;
                const long long ps = ((long long)wrap(gz - sz + m, m) * m + wrap(gy - sy + m, m)) * m +
                                     wrap(gx - sx + m, m);
                const float z4 = acc[mt][2 * hh] + bias;
                const double gv = (double)u[s * P + ps] + (double)z4;
                if (g_out) g_out[s * P + p] = (TG)gv;
                if (tgt) {
                    const double rr = gv - (double)tgt[s * P + p];
                    dz4[s * P + p] = __float2bfloat16_rn((float)rr * grad_scale);
                    l += rr * rr;
                }
            }
    }
    if (tgt) {
        for (int o = 16; o > 0; o >>= 1) l += __shfl_xor_sync(0xffffffffu, l, o);
        if (lane == 0) red[w] = l;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int k = 0; k < 8; ++k) t += red[k];
            loss_partials[(long long)blockIdx.y * gridDim.x + blockIdx.x] = t;
        }
    }
}

// dz3[p][ci] = bf16( (sum_tap dz4[p - tap] W4[ci][tap]) * gelu'(z3[p][ci]) )
__global__ void __launch_bounds__(512)
net_out_dgrad(const bf16 *__restrict__ dz4, int m, const float *__restrict__ W4q,
              const float *__restrict__ z3, bf16 *__restrict__ dz3, int lin)
{
    __shared__ float ds[1000];
    __shared__ float w[432];
    const int s = blockIdx.y;
    const long long P = (long long)m * m * m;
    const Tile T = tile_of(blockIdx.x, m);
    for (int i = threadIdx.x; i < 1000; i += blockDim.x) {
        const int hx = i % 10, hy = (i / 10) % 10, hz = i / 100;
        const int gx = wrap(T.ox + hx - 1, m), gy = wrap(T.oy + hy - 1, m), gz = wrap(T.oz + hz - 1, m);
        ds[i] = __bfloat162float(dz4[s * P + ((long long)gz * m + gy) * m + gx]);
    }
    for (int i = threadIdx.x; i < 432; i += blockDim.x) w[i] = W4q[i];
    __syncthreads();
    const int lx = threadIdx.x & 7, ly = (threadIdx.x >> 3) & 7, lz = threadIdx.x >> 6;
    float acc[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) acc[c] = 0.f;
    for (int t = 0; t < 27; ++t) {
        const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
        const float v = ds[((lz + 1 - dz) * 10 + (ly + 1 - dy)) * 10 + lx + 1 - dx];
#pragma unroll
        for (int c = 0; c < 16; ++c) acc[c] = fmaf(w[c * 27 + t], v, acc[c]);
    }
    const long long p = s * P + ((long long)(T.oz + lz) * m + (T.oy + ly)) * m + T.ox + lx;
    const float4 *zp = reinterpret_cast<const float4 *>(z3 + 16 * p);
    __align__(16) bf16 o[16];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 zz = lin ? make_float4(0.f, 0.f, 0.f, 0.f) : zp[c];
        o[4 * c + 0] = __float2bfloat16_rn(lin ? acc[4 * c + 0] : acc[4 * c + 0] * gelu_grad_f(zz.x));
        o[4 * c + 1] = __float2bfloat16_rn(lin ? acc[4 * c + 1] : acc[4 * c + 1] * gelu_grad_f(zz.y));
        o[4 * c + 2] = __float2bfloat16_rn(lin ? acc[4 * c + 2] : acc[4 * c + 2] * gelu_grad_f(zz.z));
        o[4 * c + 3] = __float2bfloat16_rn(lin ? acc[4 * c + 3] : acc[4 * c + 3] * gelu_grad_f(zz.w));
    }
    uint4 *op = reinterpret_cast<uint4 *>(dz3 + 16 * p);
    op[0] = reinterpret_cast<const uint4 *>(o)[0];
    op[1] = reinterpret_cast<const uint4 *>(o)[1];
}

// dW4[ci][tap] = sum_p a3[p + tap][ci] dz4[p], db4 = sum_p dz4[p]; per-CTA
// partials of NET_OUT_PARTIAL = 433 floats over a grid-stride set of tiles.
// Work is split into warp-sized workers: worker j < 54 owns tap j >> 1 and
// the eight channels of half j & 1 (one 16-byte chunk per point, eight FMAs
// per shared-memory load), worker 54 the bias; warp w runs workers w, w + 16,
// ... and its lanes take the tile's points lane, lane + 32, ... (consecutive
// lanes read consecutive, swizzled chunks: no bank conflicts).  Lane partial
// sums are folded by a fixed shuffle tree at the end.
constexpr int OW_WARPS = 16, OW_WORKERS = 55, OW_PER_WARP = (OW_WORKERS + OW_WARPS - 1) / OW_WARPS;
__global__ void __launch_bounds__(OW_WARPS * 32)
net_out_wgrad(const bf16 *__restrict__ a3, const bf16 *__restrict__ dz4, int m, int tiles_total,
              float *__restrict__ partials)
{
    extern __shared__ uint4 sm_ow[];
    uint4 *act = sm_ow;                                   // 2000 chunks
    float *ds = reinterpret_cast<float *>(sm_ow + 2000);  // 512
    const long long P = (long long)m * m * m;
    const int tiles = (m >> 3) * (m >> 3) * (m >> 3);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[OW_PER_WARP][8];
#pragma unroll
    for (int k = 0; k < OW_PER_WARP; ++k)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[k][c] = 0.f;
    for (int tt = blockIdx.x; tt < tiles_total; tt += gridDim.x) {
        const int s = tt / tiles;
        const Tile T = tile_of(tt % tiles, m);
        __syncthreads();
        load_halo16(act, a3 + 16 * s * P, T, m);
        for (int i = threadIdx.x; i < 512; i += blockDim.x) {
            const int lx = i & 7, ly = (i >> 3) & 7, lz = i >> 6;
            ds[i] = __bfloat162float(dz4[s * P + ((long long)(T.oz + lz) * m + (T.oy + ly)) * m + T.ox + lx]);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < OW_PER_WARP; ++k) {
            const int j = warp + OW_WARPS * k;
            if (j < 54) {
                const int t = j >> 1, h = j & 1;
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                for (int i = 0; i < 16; ++i) {
                    const int q = lane + 32 * i;
                    const int lx = q & 7, ly = (q >> 3) & 7, lz = q >> 6;
                    const int hq = ((lz + 1 + dz) * 10 + (ly + 1 + dy)) * 10 + lx + 1 + dx;
                    const uint4 v = act[chunk(hq, h)];
                    const bf16 *e = reinterpret_cast<const bf16 *>(&v);
                    const float d = ds[q];
#pragma unroll
                    for (int c = 0; c < 8; ++c) acc[k][c] = fmaf(__bfloat162float(e[c]), d, acc[k][c]);
                }
            } else if (j == 54) {
                for (int i = 0; i < 16; ++i) acc[k][0] += ds[lane + 32 * i];
            }
        }
    }
    float *out = partials + (long long)blockIdx.x * NET_OUT_PARTIAL;
#pragma unroll
    for (int k = 0; k < OW_PER_WARP; ++k) {
        const int j = warp + OW_WARPS * k;
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc[k][c] += __shfl_xor_sync(0xffffffffu, acc[k][c], o);
        if (lane == 0) {
            if (j < 54) {
                const int t = j >> 1, h = j & 1;
#pragma unroll
                for (int c = 0; c < 8; ++c) out[(8 * h + c) * 27 + t] = acc[k][c];
            } else if (j == 54) {
                out[432] = acc[k][0];
            }
        }
    }
}

// dW1[co][0][tap] = sum_p x0[p + tap] dz1[p][co]   (x0 = bf16(S(u)))
// dW1[co][1][tap] = sum_samples bf16(nu_hat_s) sum_p dz1[p][co],  db1[co] = sum_p dz1[p][co]
// (linear mode: dW1[co][1][tap] = sum_samples bf16(nu_hat_s) sum_p x0[p + tap] dz1[p][co])
// partial layout: [16][2][27] then [16] (NET_IN_PARTIAL = 880 floats).
// Warp-sized workers as in net_out_wgrad: worker j < 54 owns tap j >> 1 and
// output channels 8 (j & 1) .. + 7 (one chunk of dz1 per point, eight FMAs
// per pair of loads), workers 54 and 55 the channel sums of each half; the
// per-tile lane sums are weighted by the tile's sample's nu_hat for channel 2.
constexpr int IW_WARPS = 16, IW_WORKERS = 56, IW_PER_WARP = (IW_WORKERS + IW_WARPS - 1) / IW_WARPS;
template <typename TU>
__global__ void __launch_bounds__(IW_WARPS * 32)
net_in_wgrad(const TU *__restrict__ u, int m, int sx, int sy, int sz, const float *__restrict__ nu_hat,
             const bf16 *__restrict__ dz1, int tiles_total, float *__restrict__ partials, int lin)
{
    __shared__ float xs[1000];
    __shared__ uint4 dzs[1024];        // dz1 of the tile's 512 points, swizzled chunks
    const long long P = (long long)m * m * m;
    const int tiles = (m >> 3) * (m >> 3) * (m >> 3);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    float acc[IW_PER_WARP][8], accnu[IW_PER_WARP][8];
#pragma unroll
    for (int k = 0; k < IW_PER_WARP; ++k)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[k][c] = accnu[k][c] = 0.f;
    for (int tt = blockIdx.x; tt < tiles_total; tt += gridDim.x) {
        const int s = tt / tiles;
        const Tile T = tile_of(tt % tiles, m);
        __syncthreads();
        for (int i = threadIdx.x; i < 1000; i += blockDim.x) {
            const int hx = i % 10, hy = (i / 10) % 10, hz = i / 100;
            const int gx = wrap(wrap(T.ox + hx - 1, m) - sx + m, m);
            const int gy = wrap(wrap(T.oy + hy - 1, m) - sy + m, m);
            const int gz = wrap(wrap(T.oz + hz - 1, m) - sz + m, m);
            xs[i] = bf16r((float)u[s * P + ((long long)gz * m + gy) * m + gx]);
        }
        const uint4 *dsrc = reinterpret_cast<const uint4 *>(dz1);
        for (int i = threadIdx.x; i < 1024; i += blockDim.x) {
            const int q = i >> 1, h = i & 1;
            const int lx = q & 7, ly = (q >> 3) & 7, lz = q >> 6;
            const long long p = s * P + ((long long)(T.oz + lz) * m + (T.oy + ly)) * m + T.ox + lx;
            dzs[chunk(q, h)] = dsrc[2 * p + h];
        }
        __syncthreads();
        const float nus = bf16r(nu_hat[s]);
#pragma unroll
        for (int k = 0; k < IW_PER_WARP; ++k) {
            const int j = warp + IW_WARPS * k;
            if (j >= IW_WORKERS) continue;
            const int h = j & 1;
            float part[8];
#pragma unroll
            for (int c = 0; c < 8; ++c) part[c] = 0.f;
            if (j < 54) {
                const int t = j >> 1;
                const int dz = t / 9 - 1, dy = (t / 3) % 3 - 1, dx = t % 3 - 1;
                for (int i = 0; i < 16; ++i) {
                    const int q = lane + 32 * i;
                    const int lx = q & 7, ly = (q >> 3) & 7, lz = q >> 6;
                    const float x = xs[((lz + 1 + dz) * 10 + (ly + 1 + dy)) * 10 + lx + 1 + dx];
                    const uint4 v = dzs[chunk(q, h)];
                    const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
                    for (int c = 0; c < 8; ++c) part[c] = fmaf(x, __bfloat162float(e[c]), part[c]);
                }
                if (lin) {
#pragma unroll
                    for (int c = 0; c < 8; ++c) accnu[k][c] = fmaf(nus, part[c], accnu[k][c]);
                }
            } else {
                for (int i = 0; i < 16; ++i) {
                    const uint4 v = dzs[chunk(lane + 32 * i, h)];
                    const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
                    for (int c = 0; c < 8; ++c) part[c] += __bfloat162float(e[c]);
                }
#pragma unroll
                for (int c = 0; c < 8; ++c) accnu[k][c] = fmaf(nus, part[c], accnu[k][c]);
            }
#pragma unroll
            for (int c = 0; c < 8; ++c) acc[k][c] += part[c];
        }
    }
    float *out = partials + (long long)blockIdx.x * NET_IN_PARTIAL;
#pragma unroll
    for (int k = 0; k < IW_PER_WARP; ++k) {
        const int j = warp + IW_WARPS * k;
        if (j >= IW_WORKERS) continue;
#pragma unroll
        for (int c = 0; c < 8; ++c)
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc[k][c] += __shfl_xor_sync(0xffffffffu, acc[k][c], o);
                accnu[k][c] += __shfl_xor_sync(0xffffffffu, accnu[k][c], o);
            }
        if (lane != 0) continue;
        const int h = j & 1;
        if (j < 54) {
            const int t = j >> 1;
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                out[(8 * h + c) * 54 + t] = acc[k][c];
                if (lin) out[(8 * h + c) * 54 + 27 + t] = accnu[k][c];
            }
        } else {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                if (!lin)
                    for (int q = 0; q < 27; ++q) out[(8 * h + c) * 54 + 27 + q] = accnu[k][c];
                out[864 + 8 * h + c] = acc[k][c];
            }
        }
    }
}

// out[j] = sum over b of partials[b * stride + j], fixed order, FP64 accumulation.
__global__ void reduce_cols(const float *__restrict__ partials, int nb, int stride, int L,
                            float *__restrict__ out)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= L) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += (double)partials[(long long)b * stride + j];
    out[j] = (float)s;
}

// out[0] = sum of parts[0 .. nb): one block; thread i sums i, i + 1024, ...,
// then a fixed tree folds the 1024 sums (the same order on every call).
__global__ void __launch_bounds__(1024)
reduce_loss(const double *__restrict__ parts, int nb, double *__restrict__ out)
{
    __shared__ double red[1024];
    double s = 0.0;
    for (int b = threadIdx.x; b < nb; b += 1024) s += parts[b];
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = 512; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = red[0];
}

// Adam (Kingma & Ba 2015) on FP32 masters with bias correction.
__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ g, float *__restrict__ mo,
                            float *__restrict__ vo, int L, float lr, float b1, float b2, float eps,
                            float c1, float c2)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= L) return;
    const float gj = g[j];
    const float mm = b1 * mo[j] + (1.f - b1) * gj;
    const float vv = b2 * vo[j] + (1.f - b2) * gj * gj;
    mo[j] = mm;
    vo[j] = vv;
    p[j] -= lr * (mm / c1) / (sqrtf(vv / c2) + eps);
}

// Operand copies from the FP32 masters (layout of NetLayout).
__global__ void prepare_operands(const float *__restrict__ master, float *__restrict__ W1q,
                                 bf16 *__restrict__ B2f, bf16 *__restrict__ B3f,
                                 bf16 *__restrict__ B2b, bf16 *__restrict__ B3b, float *__restrict__ W4q,
                                 bf16 *__restrict__ B4f)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < 864) W1q[j] = bf16r(master[NET_W1 + j]);
    if (j < 432) W4q[j] = bf16r(master[NET_W4 + j]);
    if (j < 27 * 8 * 16) {
        // last-layer operand [tap][n][k = ci]: row n = 0 holds W4[ci][tap], rows 1-7 zero
        const int k = j % 16, n = (j / 16) % 8, tap = j / 128;
        B4f[j] = __float2bfloat16_rn(n == 0 ? master[NET_W4 + k * 27 + tap] : 0.f);
    }
    if (j < 6912) {
        // j = (co * 16 + ci) * 27 + tap  (master order)
        const int tap = j % 27, ci = (j / 27) % 16, co = j / (27 * 16);
        const bf16 v2 = __float2bfloat16_rn(master[NET_W2 + j]);
        const bf16 v3 = __float2bfloat16_rn(master[NET_W3 + j]);
        // forward operand: [tap][n = co][k = ci]
        B2f[(tap * 16 + co) * 16 + ci] = v2;
        B3f[(tap * 16 + co) * 16 + ci] = v3;
        // input-gradient operand: taps mirrored, [tap'][n = ci][k = co], tap' = 26 - tap
        B2b[((26 - tap) * 16 + ci) * 16 + co] = v2;
        B3b[((26 - tap) * 16 + ci) * 16 + co] = v3;
    }
}

// ----------------------------------------------------------------- launchers

static unsigned tiles_of(int m) { return (unsigned)((m / 8) * (m / 8) * (m / 8)); }

template <typename TU>
cudaError_t launch_net_in_fwd(const TU *u, int m, const int s[3], const float *nu_hat, int batch,
                              const float *W1q, const float *b1, float *z1, bf16 *a1, cudaStream_t st,
                              int lin)
{
    net_in_fwd<TU><<<dim3(tiles_of(m), batch), 128, 0, st>>>(u, m, s[0], s[1], s[2], nu_hat, W1q, b1, z1, a1,
                                                             lin);
    return cudaGetLastError();
}
template cudaError_t launch_net_in_fwd<float>(const float *, int, const int *, const float *, int,
                                              const float *, const float *, float *, bf16 *, cudaStream_t,
                                              int);
template cudaError_t launch_net_in_fwd<double>(const double *, int, const int *, const float *, int,
                                               const float *, const float *, float *, bf16 *, cudaStream_t,
                                               int);

static constexpr size_t MID_SMEM = (2000 + 864) * 16;
static constexpr size_t WG_SMEM = (2000 + 1024) * 16;
static constexpr size_t OW_SMEM = 2000 * 16 + 512 * 4;

cudaError_t configure_net_kernels()
{
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(net_mid<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MID_SMEM))) return e;
    if ((e = cudaFuncSetAttribute(net_mid<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MID_SMEM))) return e;
    if ((e = cudaFuncSetAttribute(net_mid_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM))) return e;
    if ((e = cudaFuncSetAttribute(net_out_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)OW_SMEM))) return e;
    return cudaSuccess;
}

cudaError_t launch_net_mid(int mode, const bf16 *in, int m, int batch, const bf16 *Bt, const float *bias,
                           const float *zaux, float *zout, bf16 *out, cudaStream_t st, int lin)
{
    if (mode == 0)
        net_mid<0><<<dim3(tiles_of(m), batch), 256, MID_SMEM, st>>>(in, m, Bt, bias, zaux, zout, out, lin);
    else
        net_mid<1><<<dim3(tiles_of(m), batch), 256, MID_SMEM, st>>>(in, m, Bt, bias, zaux, zout, out, lin);
    return cudaGetLastError();
}

int net_partial_blocks(int m, int batch)
{
    const long long t = (long long)tiles_of(m) * batch;
    const long long cap = 4ll * sm_count();
    return (int)(t < cap ? t : cap);
}

cudaError_t launch_net_mid_wgrad(const bf16 *x, const bf16 *dz, int m, int batch, float *partials,
                                 int nblocks, cudaStream_t st)
{
    net_mid_wgrad<<<nblocks, 256, WG_SMEM, st>>>(x, dz, m, (int)tiles_of(m) * batch, partials);
    return cudaGetLastError();
}

cudaError_t launch_net_out_dgrad(const bf16 *dz4, int m, int batch, const float *W4q, const float *z3,
                                 bf16 *dz3, cudaStream_t st, int lin)
{
    net_out_dgrad<<<dim3(tiles_of(m), batch), 512, 0, st>>>(dz4, m, W4q, z3, dz3, lin);
    return cudaGetLastError();
}

cudaError_t launch_net_out_wgrad(const bf16 *a3, const bf16 *dz4, int m, int batch, float *partials,
                                 int nblocks, cudaStream_t st)
{
    net_out_wgrad<<<nblocks, OW_WARPS * 32, OW_SMEM, st>>>(a3, dz4, m, (int)tiles_of(m) * batch, partials);
    return cudaGetLastError();
}

template <typename TU>
cudaError_t launch_net_in_wgrad(const TU *u, int m, int batch, const int s[3], const float *nu_hat,
                                const bf16 *dz1, float *partials, int nblocks, cudaStream_t st, int lin)
{
    net_in_wgrad<TU><<<nblocks, IW_WARPS * 32, 0, st>>>(u, m, s[0], s[1], s[2], nu_hat, dz1,
                                              (int)tiles_of(m) * batch, partials, lin);
    return cudaGetLastError();
}
template cudaError_t launch_net_in_wgrad<float>(const float *, int, int, const int *, const float *,
                                                const bf16 *, float *, int, cudaStream_t, int);
template cudaError_t launch_net_in_wgrad<double>(const double *, int, int, const int *, const float *,
                                                 const bf16 *, float *, int, cudaStream_t, int);

cudaError_t launch_reduce_cols(const float *partials, int nb, int stride, int L, float *out, cudaStream_t st)
{
    reduce_cols<<<(L + 255) / 256, 256, 0, st>>>(partials, nb, stride, L, out);
    return cudaGetLastError();
}

cudaError_t launch_reduce_loss(const double *parts, int nb, double *out, cudaStream_t st)
{
    reduce_loss<<<1, 1024, 0, st>>>(parts, nb, out);
    return cudaGetLastError();
}

cudaError_t launch_adam(float *p, const float *g, float *mo, float *vo, int L, float lr, float b1, float b2,
                        float eps, float c1, float c2, cudaStream_t st)
{
    adam_kernel<<<(L + 255) / 256, 256, 0, st>>>(p, g, mo, vo, L, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t launch_prepare_operands(const float *master, float *W1q, bf16 *B2f, bf16 *B3f, bf16 *B2b,
                                    bf16 *B3b, float *W4q, bf16 *B4f, cudaStream_t st)
{
    prepare_operands<<<(6912 + 255) / 256, 256, 0, st>>>(master, W1q, B2f, B3f, B2b, B3b, W4q, B4f);
    return cudaGetLastError();
}

static constexpr size_t OM_SMEM = (2000 + 432) * 16;

template <typename TU, typename TG>
cudaError_t launch_net_out_mma(const bf16 *a3, int m, int batch, const bf16 *B4f, const float *b4,
                               const TU *u, const int s[3], TG *g_out, cudaStream_t st, int lin)
{
    net_out_mma<TU, TG><<<dim3(tiles_of(m), batch), 256, OM_SMEM, st>>>(a3, m, B4f, b4, u, s[0], s[1],
                                                                       s[2], g_out, lin, nullptr, 0.f,
                                                                       nullptr, nullptr);
    return cudaGetLastError();
}

cudaError_t launch_net_out_mma_train(const bf16 *a3, int m, int batch, const bf16 *B4f, const float *b4,
                                     const float *u, const int s[3], const float *tgt, float grad_scale,
                                     bf16 *dz4, double *loss_partials, cudaStream_t st, int lin)
{
    net_out_mma<float, float><<<dim3(tiles_of(m), batch), 256, OM_SMEM, st>>>(
        a3, m, B4f, b4, u, s[0], s[1], s[2], nullptr, lin, tgt, grad_scale, dz4, loss_partials);
    return cudaGetLastError();
}
template cudaError_t launch_net_out_mma<float, float>(const bf16 *, int, int, const bf16 *, const float *,
                                                      const float *, const int *, float *, cudaStream_t, int);
template cudaError_t launch_net_out_mma<double, double>(const bf16 *, int, int, const bf16 *, const float *,
                                                        const double *, const int *, double *, cudaStream_t,
                                                        int);
template cudaError_t launch_net_out_mma<float, double>(const bf16 *, int, int, const bf16 *, const float *,
                                                       const float *, const int *, double *, cudaStream_t, int);
template cudaError_t launch_net_out_mma<double, float>(const bf16 *, int, int, const bf16 *, const float *,
                                                       const double *, const int *, float *, cudaStream_t, int);

}  // namespace pr

namespace pr {

// Mid-layer gradient: partial layout dW[tap][ci][co] + db[co] -> master
// layout W[co][ci][tap] and b[co], summed over blocks in a fixed order.
__global__ void reduce_mid(const float *__restrict__ partials, int nb, float *__restrict__ W,
                           float *__restrict__ b)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= NET_MID_PARTIAL) return;
    double s = 0.0;
    for (int q = 0; q < nb; ++q) s += (double)partials[(long long)q * NET_MID_PARTIAL + j];
    if (j < 6912) {
        const int t = j / 256, ci = (j / 16) % 16, co = j % 16;
        W[(co * 16 + ci) * 27 + t] = (float)s;
    } else {
        b[j - 6912] = (float)s;
    }
}

cudaError_t launch_reduce_mid(const float *partials, int nb, float *W, float *b, cudaStream_t st)
{
    reduce_mid<<<(NET_MID_PARTIAL + 255) / 256, 256, 0, st>>>(partials, nb, W, b);
    return cudaGetLastError();
}

}  // namespace pr
