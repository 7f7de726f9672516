// stencil.cu -- RK4 time steps of the periodic advection-diffusion operator
// A(t) y = nu(t) Lap_7 y - a . D_2 y   (7-point Laplacian of Sec. 2.3,
// centred first differences), classical RK4 (Sec. 2.3 fine propagator):
//
//   d1 = dt A(t1) u,        y2 = u + d1/2
//   d2 = dt A(t2) y2,       y3 = u + d2/2
//   d3 = dt A(t2) y3,       y4 = u + d3
//   d4 = dt A(t4) y4,       u' = u + (d1/6 + d2/3 + d3/3 + d4/6)
//
// with t1 = t, t2 = t + dt/2, t4 = t + dt (or all t when nu is frozen), t the
// step start (s * dt for global step index s).
//
// Two kernels:
//   rk4_fused_kernel  one full step per launch.  Each CTA owns a TX x TY
//                     column of the grid plus a 4-point halo in x and y and
//                     marches along z; the four stages are software-pipelined
//                     along z (stage s works on plane z-s), each stage's
//                     current plane sits in shared memory for its x/y
//                     neighbours and its z neighbours sit in registers.  HBM
//                     traffic: one read and one write of the field per step.
//   rk4_stage_kernel  one stage per launch, one point per thread; no halo
//                     recomputation, so the fewest arithmetic operations per
//                     step (the right trade where FP64 throughput, not
//                     bandwidth, bounds the step).
#include <type_traits>

#include "internal.cuh"

namespace pr {

template <typename T> struct VecT;
template <> struct VecT<float> {
    static constexpr int V = 4;
    using type = float4;
};
template <> struct VecT<double> {
    static constexpr int V = 2;
    using type = double2;
};

template <typename T>
__device__ __forceinline__ void ldv(const T *p, T (&r)[VecT<T>::V]);
template <>
__device__ __forceinline__ void ldv<float>(const float *p, float (&r)[4])
{
    const float4 q = *reinterpret_cast<const float4 *>(p);
    r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
}
template <>
__device__ __forceinline__ void ldv<double>(const double *p, double (&r)[2])
{
    const double2 q = *reinterpret_cast<const double2 *>(p);
    r[0] = q.x; r[1] = q.y;
}
template <typename T>
__device__ __forceinline__ void ldg_v(const T *p, T (&r)[VecT<T>::V]);
template <>
__device__ __forceinline__ void ldg_v<float>(const float *p, float (&r)[4])
{
    const float4 q = __ldg(reinterpret_cast<const float4 *>(p));
    r[0] = q.x; r[1] = q.y; r[2] = q.z; r[3] = q.w;
}
template <>
__device__ __forceinline__ void ldg_v<double>(const double *p, double (&r)[2])
{
    const double2 q = __ldg(reinterpret_cast<const double2 *>(p));
    r[0] = q.x; r[1] = q.y;
}
template <typename T>
__device__ __forceinline__ void stv(T *p, const T (&r)[VecT<T>::V]);
template <>
__device__ __forceinline__ void stv<float>(float *p, const float (&r)[4])
{
    *reinterpret_cast<float4 *>(p) = make_float4(r[0], r[1], r[2], r[3]);
}
template <>
__device__ __forceinline__ void stv<double>(double *p, const double (&r)[2])
{
    *reinterpret_cast<double2 *>(p) = make_double2(r[0], r[1]);
}

__device__ __forceinline__ double nu_at(const StepArgs &a, double t)
{
    return a.nu0 * (1.0 + a.nu_amp * sin(a.nu_omega * t));
}

template <typename T, int TX, int TY>
struct FusedShape {
    static constexpr int V = VecT<T>::V;
    static constexpr int RX = TX + 8;          // region width incl. 4-point halo per side
    static constexpr int RY = TY + 8;
    static constexpr int QX = RX / V;          // vectors per region row
    static constexpr int NT = QX * RY;         // threads per CTA
    static constexpr int PL = RX * RY;         // values per shared plane
    static constexpr int EL = QX * RY;         // entries per edge array
    static constexpr int D = 4;                // planes of u in flight ahead of use
    static constexpr int RING = 6;             // u planes resident (divides the unroll of 12)
    // u ring [RING][PL], stage planes [2][3][PL], u edges [RING][2][EL], stage edges [2][3][2][EL]
    static constexpr size_t SMEM = ((size_t)(RING + 6) * PL + (size_t)(2 * RING + 12) * EL) * sizeof(T);
    // CTAs per SM the register allocation is held to: as many as 64K
    // registers allow at >= 128 registers per thread (latency hiding comes
    // from independent CTAs: every CTA waits at a barrier once per plane)
    static constexpr int MINB = NT * 2 * 128 <= 65536 ? 2 : 1;
};

// 16-byte asynchronous global->shared copy (L2 only, bypassing L1) and its
// group bookkeeping.
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Per-thread constants of the fused kernel: shared-memory offsets of the own
// vector, of the vectors one row up/down (y neighbours) and of the edge
// entries of the vectors to the left/right (x neighbours).  At the region
// border the offsets are clamped in bounds; the values read there only feed
// halo points that never reach an output.
struct FusedLane {
    int own, ym, yp, eo, el, er;
};

// delta[i] = dt * A(nu_s) y at the V points of this thread's vector: c, zm,
// zp are the vector at planes p, p-1, p+1 (registers); the y neighbours come
// from the shared plane Sp, the x neighbours from its edge arrays
// (E[1] = last element of each vector, E[0] = first element).
template <typename T>
__device__ __forceinline__ void stage_delta(T (&d)[VecT<T>::V], const T *__restrict__ Sp,
                                            const T *__restrict__ E, int EL, const FusedLane &L,
                                            const T (&c)[VecT<T>::V], const T (&zm)[VecT<T>::V],
                                            const T (&zp)[VecT<T>::V], const T (&w)[7])
{
    constexpr int V = VecT<T>::V;
    T ym[V], yp[V];
    ldv<T>(Sp + L.ym, ym);
    ldv<T>(Sp + L.yp, yp);
    const T left = E[EL + L.el];
    const T right = E[L.er];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const T l = (i == 0) ? left : c[i - 1];
        const T r = (i == V - 1) ? right : c[i + 1];
        T acc = w[0] * c[i];
        acc = fma(w[1], l, acc);
        acc = fma(w[2], r, acc);
        acc = fma(w[3], ym[i], acc);
        acc = fma(w[4], yp[i], acc);
        acc = fma(w[5], zm[i], acc);
        acc = fma(w[6], zp[i], acc);
        d[i] = acc;
    }
}

// y[i] = base[i] + (w . stencil)[i]: the weighted 7-point sum of stage_delta
// accumulated onto base in one FMA chain (the stage's RK4 factor is folded
// into w).
template <typename T>
__device__ __forceinline__ void stage_axpy(T (&y)[VecT<T>::V], const T *__restrict__ Sp,
                                           const T *__restrict__ E, int EL, const FusedLane &L,
                                           const T (&c)[VecT<T>::V], const T (&zm)[VecT<T>::V],
                                           const T (&zp)[VecT<T>::V], const T (&w)[7],
                                           const T (&base)[VecT<T>::V])
{
    constexpr int V = VecT<T>::V;
    T ym[V], yp[V];
    ldv<T>(Sp + L.ym, ym);
    ldv<T>(Sp + L.yp, yp);
    const T left = E[EL + L.el];
    const T right = E[L.er];
#pragma unroll
    for (int i = 0; i < V; ++i) {
        const T l = (i == 0) ? left : c[i - 1];
        const T r = (i == V - 1) ? right : c[i + 1];
        T acc = fma(w[0], c[i], base[i]);
        acc = fma(w[1], l, acc);
        acc = fma(w[2], r, acc);
        acc = fma(w[3], ym[i], acc);
        acc = fma(w[4], yp[i], acc);
        acc = fma(w[5], zm[i], acc);
        acc = fma(w[6], zp[i], acc);
        y[i] = acc;
    }
}

// Elementwise helpers over a thread's vector: z = fma(a, x, y), z = x + y.
template <typename T>
__device__ __forceinline__ void vfma(T (&z)[VecT<T>::V], T a, const T (&x)[VecT<T>::V],
                                     const T (&y)[VecT<T>::V])
{
#pragma unroll
    for (int i = 0; i < VecT<T>::V; ++i) z[i] = fma(a, x[i], y[i]);
}
// z[i] = x[i] + y[i]
template <typename T>
__device__ __forceinline__ void vadd(T (&z)[VecT<T>::V], const T (&x)[VecT<T>::V],
                                     const T (&y)[VecT<T>::V])
{
#pragma unroll
    for (int i = 0; i < VecT<T>::V; ++i) z[i] = x[i] + y[i];
}

// Register windows of one thread, indexed by iteration modulo their period:
// u of iteration j in U[j % 4], y2 produced at iteration j in Y2[j % 4],
// y3/y4 produced at iteration j in Y3[j % 3] / Y4[j % 3].  The step's result
// is formed from the stage values of its plane,
//   u' = u + ((y2 - u) + 2 (y3 - u) + (y4 - u)) / 3 + d4 / 6,
// which equals u + d1/6 + d2/3 + d3/3 + d4/6 (y2 = u + d1/2, y3 = u + d2/2,
// y4 = u + d3) and needs no running increment sum; the differences y - u
// are exact where y is within a factor 2 of u.
template <typename T>
struct FusedRegs {
    T U[4][VecT<T>::V];
    T Y2[4][VecT<T>::V], Y3[3][VecT<T>::V], Y4[3][VecT<T>::V];
};

// Everything one z-iteration needs besides the registers.
template <typename T>
struct FusedIter {
    T *ring, *planes, *ering, *eplanes;   // shared memory
    const T *src;                          // global: this thread's column, plane 0
    T *dst;
    long long plane;                       // n*n
    int n, n_it, zreq;                     // iterations, wrapped plane of the next request
    long long ooff;                        // output offset of the current iteration
    bool act1, act2, act3, act4, owner;
};

// One z-iteration at compile-time phase PH = it % 12 (see the kernel).
template <typename T, int TX, int TY, int PH>
__device__ __forceinline__ void fused_step(FusedIter<T> &I, FusedRegs<T> &R, const FusedLane &L,
                                           int it, const T (&w1)[7], const T (&w2)[7],
                                           const T (&w4)[7])
{
    using S = FusedShape<T, TX, TY>;
    constexpr int V = S::V, PL = S::PL, EL = S::EL, D = S::D, RING = S::RING;
    constexpr T c3 = (T)(1.0 / 3.0);
    if (it >= I.n_it) return;
    // request the u plane of iteration it + D
    if (it + D < I.n_it)
        cp_async16(I.ring + ((PH + D) % RING) * PL + L.own, I.src + (long long)I.zreq * I.plane);
    cp_async_commit();
    I.zreq = I.zreq + 1 == I.n ? 0 : I.zreq + 1;
    cp_async_wait<D>();
    T un[V];
    ldv<T>(I.ring + (PH % RING) * PL + L.own, un);
    // edges of u(it) for the x neighbours of stage 1 in the next iteration
    T *eu = I.ering + (PH % RING) * 2 * EL;
    eu[L.eo] = un[0];
    eu[EL + L.eo] = un[V - 1];

    const T *Su = I.ring + ((PH + RING - 1) % RING) * PL;
    const T *Eu = I.ering + ((PH + RING - 1) % RING) * 2 * EL;
    const T *Sc = I.planes + (PH & 1) * 3 * PL;
    const T *Ec = I.eplanes + (PH & 1) * 6 * EL;
    T *Sn = I.planes + ((PH + 1) & 1) * 3 * PL;
    T *En = I.eplanes + ((PH + 1) & 1) * 6 * EL;

    // w1, w2 carry the factor 1/2 of y2 = u + d1/2 and y3 = u + d2/2, w4 the
    // factor 1/6 of d4 in the result, so each stage is one FMA chain
    T y2n[V] = {}, y3n[V] = {}, y4n[V] = {};
    // stage 1 at the plane of iteration it-1
    if (I.act1)
        stage_axpy<T>(y2n, Su, Eu, EL, L, R.U[(PH + 3) % 4], R.U[(PH + 2) % 4], un, w1,
                      R.U[(PH + 3) % 4]);
    // stage 2 at the plane of iteration it-2
    if (I.act2)
        stage_axpy<T>(y3n, Sc, Ec, EL, L, R.Y2[(PH + 3) % 4], R.Y2[(PH + 2) % 4], y2n, w2,
                      R.U[(PH + 2) % 4]);
    // stage 3 at the plane of iteration it-3: y4 = u + d3 = u + 2 (d3 / 2)
    if (I.act3) {
        T h[V];
        stage_delta<T>(h, Sc + PL, Ec + 2 * EL, EL, L, R.Y3[(PH + 2) % 3], R.Y3[(PH + 1) % 3], y3n, w2);
        vfma<T>(y4n, (T)2, h, R.U[(PH + 1) % 4]);
    }
    // stage 4 at the plane of iteration it-4: the finished step
    //   u' = u + ((y2 - u) + 2 (y3 - u) + (y4 - u)) / 3 + d4 / 6
    if (I.act4 && it >= 8) {
        const T(&u4)[V] = R.U[PH % 4];
        const T(&y2c)[V] = R.Y2[(PH + 1) % 4];
        const T(&y3c)[V] = R.Y3[(PH + 1) % 3];
        const T(&y4c)[V] = R.Y4[(PH + 2) % 3];
        T b[V], o[V];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const T s = fma((T)2, y3c[i] - u4[i], (y2c[i] - u4[i]) + (y4c[i] - u4[i]));
            b[i] = fma(c3, s, u4[i]);
        }
        stage_axpy<T>(o, Sc + 2 * PL, Ec + 4 * EL, EL, L, y4c, R.Y4[(PH + 1) % 3], y4n, w4, b);
        if (I.owner) stv<T>(I.dst + I.ooff, o);
    }
    I.ooff += I.plane;
    stv<T>(Sn + L.own, y2n);
    stv<T>(Sn + PL + L.own, y3n);
    stv<T>(Sn + 2 * PL + L.own, y4n);
    En[L.eo] = y2n[0];
    En[EL + L.eo] = y2n[V - 1];
    En[2 * EL + L.eo] = y3n[0];
    En[3 * EL + L.eo] = y3n[V - 1];
    En[4 * EL + L.eo] = y4n[0];
    En[5 * EL + L.eo] = y4n[V - 1];
    __syncthreads();
#pragma unroll
    for (int i = 0; i < V; ++i) {
        R.U[PH % 4][i] = un[i];
        R.Y2[PH % 4][i] = y2n[i];
        R.Y3[PH % 3][i] = y3n[i];
        R.Y4[PH % 3][i] = y4n[i];
    }
}

// One RK4 step of `count` fields.  Each CTA owns a TX x TY column (plus a
// 4-point halo in x and y) of one field and a z range [z_lo, z_hi); it runs
// n_it = (z_hi - z_lo) + 8 iterations, iteration it loading plane
// z_lo - 4 + it and finishing plane z_lo - 8 + it (stage s works on plane
// z_lo - 4 + it - s).  The z loop is unrolled by 12, a multiple of every
// register window's period, so the windows never move between registers.
template <typename T, int TX, int TY>
__global__ void __launch_bounds__(FusedShape<T, TX, TY>::NT, FusedShape<T, TX, TY>::MINB)
rk4_fused_kernel(StepArgs a, const T *__restrict__ in, T *__restrict__ out, int tiles_x,
                 int tiles_y, int zchunk, int nzc)
{
    using S = FusedShape<T, TX, TY>;
    constexpr int V = S::V, RX = S::RX, RY = S::RY, QX = S::QX, PL = S::PL, EL = S::EL;
    constexpr int D = S::D, RING = S::RING;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);
    T *planes = ring + RING * PL;
    T *ering = planes + 6 * PL;
    T *eplanes = ering + 2 * RING * EL;
    __shared__ T s_w[3][7];                        // stage 1, stages 2-3, stage 4

    const int tid = threadIdx.x;
    // Rows in order of the stages they need: the TY inner rows (all four)
    // first, then the halo rows 3, RY-4 (three stages), 2, RY-3, 1, RY-2 and
    // 0, RY-1 (none), so the halo rows share warps and those warps skip
    // whole stages.
    const int qx = tid % QX;
    const int ri = tid / QX;
    const int hj = ri - TY;
    const int ry = ri < TY ? 4 + ri : ((hj & 1) ? RY - 4 + (hj >> 1) : 3 - (hj >> 1));
    int b = blockIdx.x;
    const int zc = b % nzc; b /= nzc;
    const int tx = b % tiles_x; b /= tiles_x;
    const int ty = b % tiles_y; b /= tiles_y;
    const int f = b;
    const int n = a.n;

    if (tid < 3) {
        const long long s = (long long)(a.first_slice + f * a.slice_stride) * a.steps_per_slice + a.j;
        const double t = (double)s * a.dt;
        const double ts = a.frozen ? t : (tid == 0 ? t : (tid == 1 ? t + 0.5 * a.dt : t + a.dt));
        double w[7];
        stage_weights(nu_at(a, ts), a.dt, n, a.a, w);
        // the stage factors of the fused step: 1/2 (stage 1, and stages 2-3,
        // where stage 3 doubles it back), 1/6 (stage 4)
        const double f = tid == 2 ? 1.0 / 6.0 : 0.5;
#pragma unroll
        for (int k = 0; k < 7; ++k) s_w[tid][k] = (T)(f * w[k]);
    }
    __syncthreads();
    T w1[7], w2[7], w4[7];
#pragma unroll
    for (int k = 0; k < 7; ++k) {
        w1[k] = s_w[0][k];
        w2[k] = s_w[1][k];
        w4[k] = s_w[2][k];
    }

    FusedLane L;
    L.own = ry * RX + qx * V;
    L.ym = (ry > 0 ? ry - 1 : 0) * RX + qx * V;
    L.yp = (ry < RY - 1 ? ry + 1 : RY - 1) * RX + qx * V;
    L.eo = ry * QX + qx;
    L.el = ry * QX + (qx > 0 ? qx - 1 : 0);          // right edge of the left vector
    L.er = ry * QX + (qx < QX - 1 ? qx + 1 : QX - 1); // left edge of the right vector

    const int gx = ((tx * TX - 4 + qx * V) % n + n) % n;
    const int gy = ((ty * TY - 4 + ry) % n + n) % n;
    FusedIter<T> I;
    I.ring = ring;
    I.planes = planes;
    I.ering = ering;
    I.eplanes = eplanes;
    I.plane = (long long)n * n;
    I.src = in + (long long)f * a.P + (long long)gy * n + gx;
    I.dst = out + (long long)f * a.P + (long long)gy * n + gx;
    I.n = n;
    const int z_lo = zc * zchunk;
    const int z_hi = min(z_lo + zchunk, n);
    I.n_it = z_hi - z_lo + 8;
    I.ooff = (long long)(z_lo - 8) * I.plane;
    // stage s is needed on rows [s, RY-s) and elements [s, RX-s) of the region
    auto active = [&](int s) {
        return ry >= s && ry < RY - s && (qx + 1) * V > s && qx * V < RX - s;
    };
    // warp-uniform stage flags: a warp takes a stage when any of its lanes
    // needs it (the other lanes' results there are never read), so the
    // stage branches never diverge
    const unsigned lanes = __activemask();
    I.act1 = __any_sync(lanes, active(1));
    I.act2 = __any_sync(lanes, active(2));
    I.act3 = __any_sync(lanes, active(3));
    I.act4 = __any_sync(lanes, active(4));
    I.owner = ry >= 4 && ry < 4 + TY && qx * V >= 4 && qx * V < 4 + TX;

    // prologue: planes of iterations 0 .. D-1 into ring slots 0 .. D-1
    int z0 = z_lo - 4;
    z0 = ((z0 % n) + n) % n;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        if (q < I.n_it) cp_async16(ring + q * PL + L.own, I.src + (long long)z0 * I.plane);
        cp_async_commit();
        z0 = z0 + 1 == n ? 0 : z0 + 1;
    }
    I.zreq = z0;

    FusedRegs<T> R;
#pragma unroll
    for (int i = 0; i < V; ++i) {
#pragma unroll
        for (int k = 0; k < 4; ++k) R.U[k][i] = R.Y2[k][i] = (T)0;
#pragma unroll
        for (int k = 0; k < 3; ++k) R.Y3[k][i] = R.Y4[k][i] = (T)0;
    }
    for (int base = 0; base < I.n_it; base += 12) {
        fused_step<T, TX, TY, 0>(I, R, L, base + 0, w1, w2, w4);
        fused_step<T, TX, TY, 1>(I, R, L, base + 1, w1, w2, w4);
        fused_step<T, TX, TY, 2>(I, R, L, base + 2, w1, w2, w4);
        fused_step<T, TX, TY, 3>(I, R, L, base + 3, w1, w2, w4);
        fused_step<T, TX, TY, 4>(I, R, L, base + 4, w1, w2, w4);
        fused_step<T, TX, TY, 5>(I, R, L, base + 5, w1, w2, w4);
        fused_step<T, TX, TY, 6>(I, R, L, base + 6, w1, w2, w4);
        fused_step<T, TX, TY, 7>(I, R, L, base + 7, w1, w2, w4);
        fused_step<T, TX, TY, 8>(I, R, L, base + 8, w1, w2, w4);
        fused_step<T, TX, TY, 9>(I, R, L, base + 9, w1, w2, w4);
        fused_step<T, TX, TY, 10>(I, R, L, base + 10, w1, w2, w4);
        fused_step<T, TX, TY, 11>(I, R, L, base + 11, w1, w2, w4);
    }
    cp_async_wait<0>();
}

template <typename T, int TX, int TY>
static cudaError_t launch_fused_shape(const StepArgs &a, const T *in, T *out, int zchunk,
                                      cudaStream_t st)
{
    using S = FusedShape<T, TX, TY>;
    const int tiles_x = a.n / TX, tiles_y = a.n / TY;
    const int nzc = (a.n + zchunk - 1) / zchunk;
    const long long blocks = (long long)a.count * tiles_x * tiles_y * nzc;
    rk4_fused_kernel<T, TX, TY><<<(unsigned)blocks, S::NT, S::SMEM, st>>>(a, in, out, tiles_x,
                                                                         tiles_y, zchunk, nzc);
    return cudaGetLastError();
}

template <typename T, int TX, int TY>
static cudaError_t configure_shape()
{
    return cudaFuncSetAttribute(rk4_fused_kernel<T, TX, TY>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FusedShape<T, TX, TY>::SMEM);
}

// Tile shapes compiled for the fused kernel.
#define PR_FUSED_SHAPES(X) \
    X(float, 64, 32)       \
    X(float, 64, 16)       \
    X(float, 64, 8)        \
    X(float, 32, 16)       \
    X(float, 32, 8)        \
    X(float, 16, 16)       \
    X(double, 32, 8)       \
    X(double, 16, 16)      \
    X(double, 16, 8)

// Shared-memory opt-in of every compiled shape (once per device, before any
// launch or stream capture).
cudaError_t configure_rk4_kernels()
{
    cudaError_t e = cudaSuccess;
#define PR_CONF(T, TX, TY) \
    if (e == cudaSuccess) e = configure_shape<T, TX, TY>();
    PR_FUSED_SHAPES(PR_CONF)
#undef PR_CONF
    return e;
}

bool rk4_fused_supported(int dtype, int n, int tile_x, int tile_y)
{
    if (n % tile_x || n % tile_y) return false;
#define PR_SUP(T, TX, TY)                                                                   \
    if ((dtype == PARAREAL_F64) == (sizeof(T) == 8) && tile_x == TX && tile_y == TY) return true;
    PR_FUSED_SHAPES(PR_SUP)
#undef PR_SUP
    return false;
}

template <typename T>
cudaError_t launch_rk4_fused(const StepArgs &a, const T *in, T *out, int tile_x, int tile_y,
                             int zchunk, cudaStream_t st)
{
    if (zchunk <= 0 || a.n % tile_x || a.n % tile_y) return cudaErrorInvalidValue;
#define PR_DISPATCH(TT, TX, TY)                                                             \
    if constexpr (std::is_same<T, TT>::value)                                                \
        if (tile_x == TX && tile_y == TY) return launch_fused_shape<TT, TX, TY>(a, in, out, zchunk, st);
    PR_FUSED_SHAPES(PR_DISPATCH)
#undef PR_DISPATCH
    return cudaErrorInvalidValue;
}
template cudaError_t launch_rk4_fused<float>(const StepArgs &, const float *, float *, int, int,
                                             int, cudaStream_t);
template cudaError_t launch_rk4_fused<double>(const StepArgs &, const double *, double *, int,
                                              int, int, cudaStream_t);

// ------------------------------------------------------------ staged RK4

// One stage of one step, one point per thread, any operator of radius R
// (weights from op_weights).  Stages 1-4 are the RK4 stages of the file
// header (ysrc = y_s, u = the step's start value, acc = running increment
// sum); stage 0 is a forward Euler step ydst = ysrc + dt A(nu(t)) ysrc.
template <typename T, int R>
__global__ void __launch_bounds__(256)
rk4_stage_kernel(StepArgs a, int stage, const T *__restrict__ ysrc, T *__restrict__ u,
                 T *__restrict__ ydst, T *__restrict__ acc)
{
    constexpr int NW = 1 + 6 * R;
    __shared__ T s_w[NW];
    const int f = blockIdx.y;
    if (threadIdx.x == 0) {
        const long long s = (long long)(a.first_slice + f * a.slice_stride) * a.steps_per_slice + a.j;
        const double t = (double)s * a.dt;
        const double c = (stage <= 1 || a.frozen) ? 0.0 : (stage == 4 ? 1.0 : 0.5);
        double w[13];
        op_weights(a.op, nu_at(a, t + c * a.dt), a.dt, a.n, a.a, w);
        for (int k = 0; k < NW; ++k) s_w[k] = (T)w[k];
    }
    __syncthreads();
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= a.P) return;
    const int n = a.n;
    const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / ((long long)n * n));
    const T *Y = ysrc + (long long)f * a.P;
    const long long nn = (long long)n * n;
    // periodic neighbour index at distance k (|k| <= R < n) along one axis
    auto wrap = [n](int i, int k) { i += k; return i < 0 ? i + n : (i >= n ? i - n : i); };
    const long long row = (long long)z * nn + (long long)y * n;
    T d = s_w[0] * Y[row + x];
#pragma unroll
    for (int r = 1; r <= R; ++r) {
        const int b = 1 + 6 * (r - 1);
        d = fma(s_w[b + 0], Y[row + wrap(x, -r)], d);
        d = fma(s_w[b + 1], Y[row + wrap(x, r)], d);
        d = fma(s_w[b + 2], Y[(long long)z * nn + (long long)wrap(y, -r) * n + x], d);
        d = fma(s_w[b + 3], Y[(long long)z * nn + (long long)wrap(y, r) * n + x], d);
        d = fma(s_w[b + 4], Y[(long long)wrap(z, -r) * nn + (long long)y * n + x], d);
        d = fma(s_w[b + 5], Y[(long long)wrap(z, r) * nn + (long long)y * n + x], d);
    }
    const long long q = (long long)f * a.P + p;
    if (stage == 0) {
        ydst[q] = Y[p] + d;
        return;
    }
    const T uq = u[q];
    if (stage == 1) {
        ydst[q] = fma((T)0.5, d, uq);
        acc[q] = d * (T)(1.0 / 6.0);
    } else if (stage == 2) {
        ydst[q] = fma((T)0.5, d, uq);
        acc[q] = fma((T)(1.0 / 3.0), d, acc[q]);
    } else if (stage == 3) {
        ydst[q] = uq + d;
        acc[q] = fma((T)(1.0 / 3.0), d, acc[q]);
    } else {
        u[q] = uq + fma((T)(1.0 / 6.0), d, acc[q]);
    }
}

template <typename T>
cudaError_t launch_rk4_stage(const StepArgs &a, int stage, const T *ysrc, T *u, T *ydst, T *acc,
                             cudaStream_t st)
{
    const unsigned bx = (unsigned)((a.P + 255) / 256);
    dim3 grid(bx, (unsigned)a.count);
    if (op_radius(a.op) == 2)
        rk4_stage_kernel<T, 2><<<grid, 256, 0, st>>>(a, stage, ysrc, u, ydst, acc);
    else
        rk4_stage_kernel<T, 1><<<grid, 256, 0, st>>>(a, stage, ysrc, u, ydst, acc);
    return cudaGetLastError();
}
template cudaError_t launch_rk4_stage<float>(const StepArgs &, int, const float *, float *,
                                             float *, float *, cudaStream_t);
template cudaError_t launch_rk4_stage<double>(const StepArgs &, int, const double *, double *,
                                              double *, double *, cudaStream_t);

// ------------------------------------------------- conversion, restriction

__global__ void convert_d2f_kernel(const double *__restrict__ s, float *__restrict__ d, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        d[i] = (float)s[i];
}
__global__ void convert_f2d_kernel(const float *__restrict__ s, double *__restrict__ d, long long N)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (long long)gridDim.x * blockDim.x)
        d[i] = (double)s[i];
}

static unsigned grid_for(long long N)
{
    long long b = (N + 255) / 256;
    return (unsigned)(b < 152 * 16 ? (b < 1 ? 1 : b) : 152 * 16);
}

cudaError_t launch_convert_f64_to_f32(const double *src, float *dst, long long N, cudaStream_t st)
{
    convert_d2f_kernel<<<grid_for(N), 256, 0, st>>>(src, dst, N);
    return cudaGetLastError();
}
cudaError_t launch_convert_f32_to_f64(const float *src, double *dst, long long N, cudaStream_t st)
{
    convert_f2d_kernel<<<grid_for(N), 256, 0, st>>>(src, dst, N);
    return cudaGetLastError();
}

// Box average over the r^3 fine points I*r..I*r+r-1 of each coarse cell.
template <typename T>
__global__ void restrict_kernel(const double *__restrict__ fine, int n, int r, T *__restrict__ coarse)
{
    const int nc = n / r;
    const long long Pc = (long long)nc * nc * nc;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < Pc;
         q += (long long)gridDim.x * blockDim.x) {
        const int I = (int)(q % nc), J = (int)((q / nc) % nc), K = (int)(q / ((long long)nc * nc));
        double s = 0.0;
        for (int dk = 0; dk < r; ++dk)
            for (int dj = 0; dj < r; ++dj) {
                const double *row = fine + ((long long)(K * r + dk) * n + (J * r + dj)) * n + I * r;
                for (int di = 0; di < r; ++di) s += row[di];
            }
        coarse[q] = (T)(s / ((double)r * r * r));
    }
}

template <typename T>
cudaError_t launch_restrict(const double *fine, int n, int r, T *coarse, cudaStream_t st)
{
    const long long Pc = (long long)(n / r) * (n / r) * (n / r);
    restrict_kernel<T><<<grid_for(Pc), 256, 0, st>>>(fine, n, r, coarse);
    return cudaGetLastError();
}
template cudaError_t launch_restrict<float>(const double *, int, int, float *, cudaStream_t);
template cudaError_t launch_restrict<double>(const double *, int, int, double *, cudaStream_t);

}  // namespace pr
