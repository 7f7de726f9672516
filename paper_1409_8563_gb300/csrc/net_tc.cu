// net_tc.cu -- the learned propagator's 16 -> 16 convolution layers (forward,
// inference) on the 5th-generation tensor cores: tcgen05.mma with the
// accumulator in tensor memory.
//
// One MMA computes D[128 x 16] += A[128 x 16] * B[16 x 16] (BF16 in, FP32
// accumulate).  An output plane tile is 8 x 16 points (M = 128, row m = x + 8 y);
// it is 27 MMAs, one per tap, each with K = 16 input channels:
//   D[m][co] = sum_tap sum_ci act[p(m) + tap][ci] * W[tap][co][ci].
// The A operands are not copied: the activations of the tile's halo (10 x 18
// x (ZB + 2) points for ZB output planes) sit in shared memory in the layout
//   chunk(z, y, h, x) = ((z * 18 + y) * 2 + h) * 10 + x     (16-byte chunks,
//   h = channel half),
// so the 8 points x .. x+7 of one halo row and channel half form one 8 x 16 B
// core matrix, and the operand of tap (dx, dy, dz) is a shared-memory
// descriptor whose start moves by the tap's offset: stride between 8-row
// groups (y) 320 B, between the two channel halves 160 B (K-major, no
// swizzle).  B (the tap's 16 x 16 weights) is stored [tap][h][co] the same way.
//
// Each CTA (4 warps) allocates 32 tensor-memory columns once (one 16-column
// accumulator per output plane), loops over tiles, and reads D back with
// tcgen05.ld (warp w owns lanes 32w .. 32w+31, i.e. tile rows 32w .. 32w+31).
// The same MMA loop serves training: the forward pass that also keeps the
// FP32 pre-activations, and the input gradient (the layer's adjoint: taps
// mirrored and the channel matrix transposed, which only changes B), whose
// epilogue multiplies by the activation's derivative at the stored
// pre-activation.
// Completion of the MMAs is signalled on an mbarrier whose wait is bounded: on
// timeout the kernel records an error flag, waits once more (bounded), frees
// its tensor memory and returns.
#include <cuda_bf16.h>
#include <stdint.h>

#include "internal.cuh"
#include "net.cuh"

namespace pr {

using bf16 = __nv_bfloat16;

namespace {

constexpr int ZB = 2;                             // output planes per tile (one accumulator each)
constexpr int HX = 10, HY = 18, HZ = ZB + 2;
constexpr int HALO_CHUNKS = HZ * HY * 2 * HX;     // 1440 chunks, 23040 B
constexpr int HALO_ALLOC = HALO_CHUNKS + 32;      // per buffer, 16-byte chunks
constexpr int B_CHUNKS = 27 * 2 * 16;             // 864 chunks, 13824 B
constexpr int TC_THREADS = 128;
constexpr uint32_t TMEM_COLS = 32;                // ZB accumulators of 16 columns
constexpr long long WAIT_LIMIT = 1ll << 22;

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Shared-memory matrix descriptor: K-major, no swizzle; byte address, leading
// (K-direction) and stride (M/N-direction) byte offsets, all multiples of 16.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;   // descriptor version of the 5th-generation tensor cores
    return d;                 // base offset 0, no swizzle
}

// Instruction descriptor: kind::f16, A and B BF16 (K-major), D FP32, M x N.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4)                      // D format: F32
           | (1u << 7)                    // A format: BF16
           | (1u << 10)                   // B format: BF16
           | ((uint32_t)(N >> 3) << 17)   // N / 8
           | ((uint32_t)(M >> 4) << 24);  // M / 16
}

__device__ __forceinline__ void mma_tc(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n"
        ::"r"(tmem_d), "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits for the phase of `parity` to complete, giving up (false) after
// `limit` tries; the caller then records the failure and returns.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t mbar, uint32_t parity,
                                                  long long limit = WAIT_LIMIT)
{
    for (long long i = 0; i < limit; ++i)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void cp_async16_tc(uint32_t saddr, const void *g)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(saddr), "l"(g) : "memory");
}

__device__ __forceinline__ float gelu_tc(float x)
{
    return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
// d gelu / dx = Phi(x) + x phi(x)
__device__ __forceinline__ float gelu_grad_tc(float x)
{
    return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
           x * 0.39894228040143268f * __expf(-0.5f * x * x);
}

__device__ __forceinline__ int wrapi(int i, int m) { return i < 0 ? i + m : (i >= m ? i - m : i); }

struct TileTC {
    int s, ox, oy, oz;
};
__device__ __forceinline__ TileTC tile_tc(long long tt, int m)
{
    const int tx_n = m / 8, ty_n = m / 16, tz_n = m / ZB;
    const long long per = (long long)tx_n * ty_n * tz_n;
    TileTC T;
    T.s = (int)(tt / per);
    const long long r = tt % per;
    T.ox = (int)(r % tx_n) * 8;
    T.oy = (int)((r / tx_n) % ty_n) * 16;
    T.oz = (int)(r / ((long long)tx_n * ty_n)) * ZB;
    return T;
}

// Queue the halo of tile T into the buffer at shared address `buf`
// (chunk(z, y, h, x) = ((z * HY + y) * 2 + h) * HX + x; 16-byte copies).
__device__ __forceinline__ void halo_async(uint32_t buf, const bf16 *__restrict__ in, const TileTC &T,
                                           int m, long long P)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(in + 16 * T.s * P);
    for (int i = threadIdx.x; i < HALO_CHUNKS; i += TC_THREADS) {
        const int x = i % HX, h = (i / HX) & 1, y = (i / (2 * HX)) % HY, z = i / (2 * HX * HY);
        const int gx = wrapi(T.ox + x - 1, m), gy = wrapi(T.oy + y - 1, m), gz = wrapi(T.oz + z - 1, m);
        cp_async16_tc(buf + (uint32_t)i * 16u, src + 2 * (((long long)gz * m + gy) * m + gx) + h);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

}  // namespace

// acc[p][n] = sum_tap sum_k in[p + tap][k] Bt[tap][n][k], then
//   MODE 0 (forward):  z = acc + bias[n], zout[p][n] = z (if zout is non-null),
//                      out[p][n] = bf16(gelu(z));
//   MODE 1 (dgrad):    out[p][n] = bf16(acc * gelu'(zaux[p][n]))
// (linear mode: no bias, identity activation, so out = bf16(acc) in both and
// zout = acc).  Bt: [tap][n][k] BF16, the forward taps W[tap][co][ci] for
// MODE 0, the mirrored transposed taps W[-tap][co][ci] (n = ci, k = co) for
// MODE 1.  A tile is 8 x 16 x ZB points: ZB GEMMs of M = 128 on one halo,
// accumulators at columns 16 zp .. 16 zp + 15.  Persistent CTAs: the halo of
// the next tile streams in (cp.async, double buffer) while the current tile's
// MMAs and epilogue run.  m must be a multiple of 16.
template <int MODE>
__global__ void __launch_bounds__(TC_THREADS)
net_mid_tc(const bf16 *__restrict__ in, int m, int batch, const bf16 *__restrict__ Bt,
           const float *__restrict__ bias, const float *__restrict__ zaux, float *__restrict__ zout,
           bf16 *__restrict__ out, int lin, int *__restrict__ errflag)
{
    extern __shared__ __align__(1024) uint4 sm_tc[];
    uint4 *halo0 = sm_tc;
    uint4 *bs = sm_tc + 2 * HALO_ALLOC;
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)m * m * m;
    const long long tiles = (long long)(m / 8) * (m / 16) * (m / ZB) * batch;

    // B: [tap][co][ci] (two chunks per co row) -> [tap][h][co]
    const uint4 *bsrc = reinterpret_cast<const uint4 *>(Bt);
    for (int i = tid; i < B_CHUNKS; i += TC_THREADS) {
        const int t = i / 32, h = (i / 16) & 1, co = i & 15;
        bs[i] = bsrc[(t * 16 + co) * 2 + h];
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_addr(&tmem_slot)), "r"(TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    const uint32_t halo_a[2] = {smem_addr(halo0), smem_addr(halo0 + HALO_ALLOC)};
    long long tt = blockIdx.x;
    if (tt < tiles) halo_async(halo_a[0], in, tile_tc(tt, m), m, P);
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = tmem_slot;
    const uint32_t mbar_a = smem_addr(&mbar);
    const uint32_t bs_a = smem_addr(bs);
    constexpr uint32_t IDESC = idesc_bf16(128, 16);

    uint32_t parity = 0;
    int buf = 0;
    for (; tt < tiles; tt += gridDim.x, buf ^= 1) {
        const TileTC T = tile_tc(tt, m);
        // the next tile's halo goes to the other buffer, whose last reader
        // (the previous tile's MMAs) has completed
        const long long nt = tt + gridDim.x;
        if (nt < tiles) halo_async(halo_a[buf ^ 1], in, tile_tc(nt, m), m, P);
        else asm volatile("cp.async.commit_group;\n" ::: "memory");
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        // this thread's copies -> visible to the tensor core's async proxy
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        if (tid == 0) {
            // descriptors of the halo and weight bases; each tap adds its offset
            // (in 16-byte units) to the start-address field, which stays below
            // 2^14 for any shared-memory address
            const uint64_t a0 = smem_desc(halo_a[buf], HX * 16, 2 * HX * 16);
            const uint64_t b0 = smem_desc(bs_a, 256, 128);
#pragma unroll
            for (int zp = 0; zp < ZB; ++zp)
#pragma unroll
                for (int t = 0; t < 27; ++t) {
                    const int dz = t / 9, dy = (t / 3) % 3, dx = t % 3;     // offsets + 1
                    const uint32_t a_chunk = (uint32_t)((((zp + dz) * HY + dy) * 2) * HX + dx);
                    mma_tc(tmem + 16u * zp, a0 + a_chunk, b0 + (uint64_t)(t * 32), IDESC, t > 0 ? 1u : 0u);
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         ::"r"(mbar_a) : "memory");
        }
        // every thread waits (bounded) for the MMAs, then the block takes one
        // decision: if any thread gave up, all leave the tile loop together,
        // so no warp-collective tensor-memory load or barrier below runs with
        // part of the block gone.  After a give-up the block waits once more
        // (bounded, again block-wide) for the MMAs in flight before the
        // tensor memory they write is freed.
        if (__syncthreads_or(mbar_wait_bounded(mbar_a, parity) ? 0 : 1)) {
            if (tid == 0) atomicExch(errflag, 1);
            (void)__syncthreads_or(mbar_wait_bounded(mbar_a, parity) ? 0 : 1);
            break;
        }
        parity ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        const int row = warp * 32 + lane;
#pragma unroll
        for (int zp = 0; zp < ZB; ++zp) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + 16u * zp;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            const long long p = T.s * P + ((long long)(T.oz + zp) * m + (T.oy + (row >> 3))) * m + T.ox + (row & 7);
            __align__(16) bf16 o[16];
            if (MODE == 0) {
                float z[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) z[c] = lin ? __uint_as_float(v[c]) : __uint_as_float(v[c]) + bias[c];
                if (zout) {
                    float4 *zp4 = reinterpret_cast<float4 *>(zout + 16 * p);
#pragma unroll
                    for (int c = 0; c < 4; ++c) zp4[c] = make_float4(z[4 * c], z[4 * c + 1], z[4 * c + 2], z[4 * c + 3]);
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(lin ? z[c] : gelu_tc(z[c]));
            } else {
                float g[16];
#pragma unroll
                for (int c = 0; c < 16; ++c) g[c] = __uint_as_float(v[c]);
                if (!lin) {
                    const float4 *za4 = reinterpret_cast<const float4 *>(zaux + 16 * p);
#pragma unroll
                    for (int c = 0; c < 4; ++c) {
                        const float4 zz = za4[c];
                        g[4 * c] *= gelu_grad_tc(zz.x);
                        g[4 * c + 1] *= gelu_grad_tc(zz.y);
                        g[4 * c + 2] *= gelu_grad_tc(zz.z);
                        g[4 * c + 3] *= gelu_grad_tc(zz.w);
                    }
                }
#pragma unroll
                for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16_rn(g[c]);
            }
            uint4 *op = reinterpret_cast<uint4 *>(out + 16 * p);
            op[0] = reinterpret_cast<const uint4 *>(o)[0];
            op[1] = reinterpret_cast<const uint4 *>(o)[1];
        }
        // every warp's tensor-memory reads precede the next tile's MMAs
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(TMEM_COLS));
}

// ------------------------------------------------ weight gradient (tcgen05)
//
// dW[tap][ci][co] = sum_p x[p + tap][ci] dz[p][co] as MMAs with K = 16 points
// (the 8 x-points of two tile rows), N = 16 output channels and M = 128 rows
// (dyi, h, i): input channel ci = 8 h + i seen at the y offset dy = dyi - 1.
// Both operands are read MN-major straight from the [point][16] layouts: one
// 16-byte chunk holds 8 channels of one point, and 8 consecutive x-points of
// one halo row are 8 consecutive chunks, i.e. one core matrix (8 K-rows x 8
// MN-elements).  In the halo, row groups (dyi, h) sit HX chunks apart
// uniformly (the channel half moves by HX, the y row by 2 HX), so one MMA
// covers the dy offsets -1 .. 6 for one (dz, dx) pair; rows with dyi > 2 fall
// outside the stencil, read slack or other rows of shared memory, and are
// never stored.  Nine accumulators of 16 columns (one per (dz, dx)) stay in
// tensor memory over all of a CTA's tiles; the epilogue writes the CTA's
// partial sum [27][16 ci][16 co] + db[16], reduced in a fixed order after.
namespace {
constexpr int DZ_CHUNKS = ZB * 16 * 2 * 8;        // dz tile: 8 x 16 x ZB points, 2 chunks each
// chunks after the buffers: rows dyi > 2 read up to ~1700 chunks past a halo
// base; the slack also holds the CTA at ~100 KB of shared memory, so at most
// two CTAs (2 x 256 tensor-memory columns) share an SM
constexpr int WG_SLACK = 2368;
constexpr uint32_t WG_TMEM_COLS = 256;            // 9 accumulators of 16 columns
constexpr size_t WG_SMEM = (size_t)(2 * HALO_ALLOC + 2 * DZ_CHUNKS + WG_SLACK) * 16 + 128 * 16 * 4;

// dz tile of T: chunk(z, y, h, x) = ((z * 16 + y) * 2 + h) * 8 + x
__device__ __forceinline__ void dz_async(uint32_t buf, const bf16 *__restrict__ dz, const TileTC &T, int m,
                                         long long P)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(dz + 16 * T.s * P);
    for (int i = threadIdx.x; i < DZ_CHUNKS; i += TC_THREADS) {
        const int x = i & 7, h = (i >> 3) & 1, y = (i >> 4) & 15, z = i >> 8;
        cp_async16_tc(buf + (uint32_t)i * 16u,
                      src + 2 * (((long long)(T.oz + z) * m + (T.oy + y)) * m + T.ox + x) + h);
    }
}
}  // namespace

__global__ void __launch_bounds__(TC_THREADS)
net_mid_wgrad_tc(const bf16 *__restrict__ x, const bf16 *__restrict__ dz, int m, int batch,
                 float *__restrict__ partials, int *__restrict__ errflag)
{
    extern __shared__ __align__(1024) uint4 sm_wg[];
    uint4 *halo0 = sm_wg;
    uint4 *dz0 = sm_wg + 2 * HALO_ALLOC;
    float *red = reinterpret_cast<float *>(sm_wg + 2 * HALO_ALLOC + 2 * DZ_CHUNKS + WG_SLACK);
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_slot;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long P = (long long)m * m * m;
    const long long tiles = (long long)(m / 8) * (m / 16) * (m / ZB) * batch;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_addr(&tmem_slot)), "r"(WG_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::);
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_addr(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::);
    }
    const uint32_t halo_a[2] = {smem_addr(halo0), smem_addr(halo0 + HALO_ALLOC)};
    const uint32_t dz_a[2] = {smem_addr(dz0), smem_addr(dz0 + DZ_CHUNKS)};
    long long tt = blockIdx.x;
    // one cp.async group per tile: dz's copies, then the halo's, which
    // halo_async commits together
    if (tt < tiles) {
        const TileTC T = tile_tc(tt, m);
        dz_async(dz_a[0], dz, T, m, P);
        halo_async(halo_a[0], x, T, m, P);
    } else {
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    const uint32_t tmem = tmem_slot;
    const uint32_t mbar_a = smem_addr(&mbar);
    // MN-major A and B (transpose bits 15 and 16 of the instruction descriptor)
    constexpr uint32_t IDESC = idesc_bf16(128, 16) | (1u << 15) | (1u << 16);

    float dbias[16];                                // bias-gradient sums of this thread's points
#pragma unroll
    for (int c = 0; c < 16; ++c) dbias[c] = 0.f;
    uint32_t parity = 0;
    int buf = 0, ntile = 0;
    bool failed = false;
    for (; tt < tiles; tt += gridDim.x, buf ^= 1, ++ntile) {
        // the MMAs of the previous tile read the buffer the next tile goes to
        if (ntile > 0) {
            if (__syncthreads_or(mbar_wait_bounded(mbar_a, parity) ? 0 : 1)) {
                failed = true;
                break;
            }
            parity ^= 1u;
        }
        const long long nt = tt + gridDim.x;
        if (nt < tiles) {
            const TileTC N = tile_tc(nt, m);
            dz_async(dz_a[buf ^ 1], dz, N, m, P);
            halo_async(halo_a[buf ^ 1], x, N, m, P);
        } else {
            asm volatile("cp.async.commit_group;\n" ::: "memory");
        }
        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
        if (tid == 0) {
#pragma unroll 1
            for (int zp = 0; zp < ZB; ++zp)
#pragma unroll 1
                for (int y0 = 0; y0 < 16; y0 += 2) {
                    // B: K rows = points (x, y0 + kb), N = co; K groups 16 chunks apart, N groups 8
                    const uint32_t b_chunk = (uint32_t)(((zp * 16 + y0) * 2) * 8);
                    const uint64_t bdesc = smem_desc(dz_a[buf] + b_chunk * 16u, 16 * 16, 8 * 16);
#pragma unroll
                    for (int j = 0; j < 9; ++j) {
                        const int dzo = j / 3, dxo = j % 3;     // halo offsets of (dz, dx) + 1
                        // A: K rows = points, M = (dyi, h, i); K groups 2 HX chunks apart, M groups HX
                        const uint32_t a_chunk = (uint32_t)((((zp + dzo) * HY + y0) * 2) * HX + dxo);
                        const uint64_t adesc = smem_desc(halo_a[buf] + a_chunk * 16u, 2 * HX * 16, HX * 16);
                        const uint32_t acc = (ntile > 0 || zp > 0 || y0 > 0) ? 1u : 0u;
                        mma_tc(tmem + 16u * j, adesc, bdesc, IDESC, acc);
                    }
                }
            asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                         ::"r"(mbar_a) : "memory");
        }
        // bias gradient on the CUDA cores: thread tid sums all 16 channels of
        // the tile points tid and tid + 128 (two 16-byte loads each; the 8
        // lanes of a quarter warp read 8 consecutive chunks)
        {
            const uint4 *dt = dz0 + buf * DZ_CHUNKS;
#pragma unroll
            for (int k = 0; k < 8 * 16 * ZB / TC_THREADS; ++k) {
                const int q = tid + TC_THREADS * k;
                const int xq = q & 7, yq = (q >> 3) & 15, zq = q >> 7;
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const uint4 v = dt[((zq * 16 + yq) * 2 + h) * 8 + xq];
                    const bf16 *e = reinterpret_cast<const bf16 *>(&v);
#pragma unroll
                    for (int c = 0; c < 8; ++c) dbias[8 * h + c] += __bfloat162float(e[c]);
                }
            }
        }
    }
    // the last tile's MMAs
    if (!failed && ntile > 0 && __syncthreads_or(mbar_wait_bounded(mbar_a, parity) ? 0 : 1)) failed = true;
    if (failed) {
        if (tid == 0) atomicExch(errflag, 1);
        // MMAs may still be in flight: wait once more (bounded) before the
        // tensor memory they write is freed
        (void)__syncthreads_or(mbar_wait_bounded(mbar_a, parity) ? 0 : 1);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    float *out = partials + (long long)blockIdx.x * NET_MID_PARTIAL;
    if (!failed) {
        const int row = warp * 32 + lane;
        const int g = row >> 3, dyi = g >> 1, ci = 8 * (g & 1) + (row & 7);
#pragma unroll 1
        for (int j = 0; j < 9; ++j) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(warp * 32) << 16) + 16u * j;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
                  "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
                  "=r"(v[14]), "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
            if (dyi <= 2) {
                const int t = (j / 3) * 9 + dyi * 3 + (j % 3);
#pragma unroll
                for (int co = 0; co < 16; ++co)
                    out[t * 256 + ci * 16 + co] = ntile > 0 ? __uint_as_float(v[co]) : 0.f;
            }
        }
    }
    // bias gradient: the threads' sums in a fixed order
#pragma unroll
    for (int c = 0; c < 16; ++c) red[tid * 16 + c] = dbias[c];
    __syncthreads();
    if (tid < 16) {
        float sacc = 0.f;
        for (int k = 0; k < TC_THREADS; ++k) sacc += red[k * 16 + tid];
        out[27 * 256 + tid] = sacc;
    }
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::);
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::);
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(WG_TMEM_COLS));
}

static constexpr size_t TC_SMEM = (size_t)(2 * HALO_ALLOC + B_CHUNKS) * 16;

cudaError_t configure_net_tc()
{
    cudaError_t e = cudaFuncSetAttribute(net_mid_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(net_mid_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TC_SMEM);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(net_mid_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)WG_SMEM);
}

bool net_tc_supported(int m) { return m >= 16 && m % 16 == 0; }

cudaError_t launch_net_mid_tc(int mode, const bf16 *in, int m, int batch, const bf16 *Bt, const float *bias,
                              const float *zaux, float *zout, bf16 *out, int lin, int *errflag,
                              cudaStream_t st)
{
    const long long tiles = (long long)(m / 8) * (m / 16) * (m / ZB) * batch;
    const long long cap = 3ll * sm_count();   // three CTAs of 60 KB shared memory per SM
    const int grid = (int)(tiles < cap ? tiles : cap);
    if (mode == 0)
        net_mid_tc<0><<<grid, TC_THREADS, TC_SMEM, st>>>(in, m, batch, Bt, bias, zaux, zout, out, lin, errflag);
    else
        net_mid_tc<1><<<grid, TC_THREADS, TC_SMEM, st>>>(in, m, batch, Bt, bias, zaux, zout, out, lin, errflag);
    return cudaGetLastError();
}

// Failure-detection self-test: the bounded wait above on an mbarrier that
// no thread ever arrives on.  The wait gives up after `limit` tries and the
// kernel sets *flag; nothing else is touched, so the device stays usable.
__global__ void wait_selftest_kernel(long long limit, int *flag)
{
    __shared__ __align__(8) unsigned long long mbar;
    const uint32_t a = smem_addr(&mbar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(a) : "memory");
    __syncthreads();
    if (threadIdx.x == 0) {
        *flag = mbar_wait_bounded(a, 0u, limit) ? 0 : 1;
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];\n" ::"r"(a) : "memory");
    }
}

cudaError_t launch_wait_selftest(long long limit, int *flag, cudaStream_t st)
{
    wait_selftest_kernel<<<1, 32, 0, st>>>(limit, flag);
    return cudaGetLastError();
}

// One CTA per partial slot (nblocks of them, the caller's reduction count);
// a CTA without tiles writes zeros.  At most two CTAs hold tensor memory on
// one SM at a time (256 of its 512 columns each); later CTAs start as
// earlier ones finish.
cudaError_t launch_net_mid_wgrad_tc(const bf16 *x, const bf16 *dz, int m, int batch, float *partials,
                                    int nblocks, int *errflag, cudaStream_t st)
{
    net_mid_wgrad_tc<<<nblocks, TC_THREADS, WG_SMEM, st>>>(x, dz, m, batch, partials, errflag);
    return cudaGetLastError();
}

}  // namespace pr
