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
//                     A thread owns a vector of points in R = 1 or 2 rows;
//                     shared-memory traffic, not HBM, bounds the step, and
//                     R = 2 cuts it by a quarter.
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


template <typename T, int TX, int TY, int R>
struct FusedShape {
    static constexpr int V = VecT<T>::V;
    static constexpr int RX = TX + 8;          // region width incl. 4-point halo per side
    static constexpr int RY = TY + 8;
    static constexpr int QX = RX / V;          // vectors per region row
    static constexpr int NT = QX * RY / R;     // threads per CTA (R rows each)
    static constexpr int PL = RX * RY;         // values per shared plane
    static constexpr int EL = QX * RY;         // entries per edge array
    static constexpr int D = 4;                // planes of u in flight ahead of use
    static constexpr int RING = 6;             // u planes resident (divides the unroll of 12)
    // u ring [RING][PL], stage planes [2][3][PL], u edges [RING][2][EL], stage edges [2][3][2][EL]
    static constexpr size_t SMEM = ((size_t)(RING + 6) * PL + (size_t)(2 * RING + 12) * EL) * sizeof(T);
    // CTAs per SM the register allocation is held to: two where 64K
    // registers still give every thread its working set (~128 registers at
    // one row per thread, ~168 at two), else one (latency hiding comes from
    // independent CTAs: every CTA waits at a barrier once per plane)
    static constexpr int MINB = NT * 2 * (R == 1 ? 128 : 168) <= 65536 ? 2 : 1;
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

// Per-thread constants of the fused kernel for a thread owning R consecutive
// region rows: shared-memory offsets of its vector in each row, of the
// vectors above its first row and below its last row (its other y
// neighbours are its own rows, in registers), and of the edge entries of
// the vectors left/right of it in each row (x neighbours).  At the region
// border the offsets are clamped in bounds; the values read there only feed
// halo points that never reach an output.
template <int R>
struct FusedLane {
    int own[R], ym, yp, eo[R], el[R], er[R];
};

// d[r][i] = dt * A(nu_s) y at the V points of row r of this thread: c, zm,
// zp are the rows' vectors at planes p, p-1, p+1 (registers); the y
// neighbours outside the thread's rows come from the shared plane Sp, the x
// neighbours from its edge arrays (E[1] = last element of each vector, E[0]
// = first element).  The seven terms are summed in a fixed order (centre,
// x-1, x+1, y-1, y+1, z-1, z+1) whatever the thread's row count.
template <typename T, int R>
__device__ __forceinline__ void stage_delta(T (&d)[R][VecT<T>::V], const T *__restrict__ Sp,
                                            const T *__restrict__ E, int EL, const FusedLane<R> &L,
                                            const T (&c)[R][VecT<T>::V], const T (&zm)[R][VecT<T>::V],
                                            const T (&zp)[R][VecT<T>::V], const T (&w)[7])
{
    constexpr int V = VecT<T>::V;
    T ym[V], yp[V];
    ldv<T>(Sp + L.ym, ym);
    ldv<T>(Sp + L.yp, yp);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const T left = E[EL + L.el[r]];
        const T right = E[L.er[r]];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const T l = (i == 0) ? left : c[r][i > 0 ? i - 1 : 0];
            const T rt = (i == V - 1) ? right : c[r][i < V - 1 ? i + 1 : 0];
            const T up = (r == 0) ? ym[i] : c[r > 0 ? r - 1 : 0][i];
            const T dn = (r == R - 1) ? yp[i] : c[r < R - 1 ? r + 1 : 0][i];
            T acc = w[0] * c[r][i];
            acc = fma(w[1], l, acc);
            acc = fma(w[2], rt, acc);
            acc = fma(w[3], up, acc);
            acc = fma(w[4], dn, acc);
            acc = fma(w[5], zm[r][i], acc);
            acc = fma(w[6], zp[r][i], acc);
            d[r][i] = acc;
        }
    }
}

// y[r][i] = base[r][i] + (w . stencil)[r][i]: the weighted 7-point sum of
// stage_delta accumulated onto base in one FMA chain (the stage's RK4 factor
// is folded into w).
template <typename T, int R>
__device__ __forceinline__ void stage_axpy(T (&y)[R][VecT<T>::V], const T *__restrict__ Sp,
                                           const T *__restrict__ E, int EL, const FusedLane<R> &L,
                                           const T (&c)[R][VecT<T>::V], const T (&zm)[R][VecT<T>::V],
                                           const T (&zp)[R][VecT<T>::V], const T (&w)[7],
                                           const T (&base)[R][VecT<T>::V])
{
    constexpr int V = VecT<T>::V;
    T ym[V], yp[V];
    ldv<T>(Sp + L.ym, ym);
    ldv<T>(Sp + L.yp, yp);
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const T left = E[EL + L.el[r]];
        const T right = E[L.er[r]];
#pragma unroll
        for (int i = 0; i < V; ++i) {
            const T l = (i == 0) ? left : c[r][i > 0 ? i - 1 : 0];
            const T rt = (i == V - 1) ? right : c[r][i < V - 1 ? i + 1 : 0];
            const T up = (r == 0) ? ym[i] : c[r > 0 ? r - 1 : 0][i];
            const T dn = (r == R - 1) ? yp[i] : c[r < R - 1 ? r + 1 : 0][i];
            T acc = fma(w[0], c[r][i], base[r][i]);
            acc = fma(w[1], l, acc);
            acc = fma(w[2], rt, acc);
            acc = fma(w[3], up, acc);
            acc = fma(w[4], dn, acc);
            acc = fma(w[5], zm[r][i], acc);
            acc = fma(w[6], zp[r][i], acc);
            y[r][i] = acc;
        }
    }
}

// Register windows of one thread, indexed by iteration modulo their period:
// u of iteration j in U[j % 4], y2 produced at iteration j in Y2[j % 4],
// y3/y4 produced at iteration j in Y3[j % 3] / Y4[j % 3].  The step's result
// is formed from the stage values of its plane,
//   u' = u + ((y2 - u) + 2 (y3 - u) + (y4 - u)) / 3 + d4 / 6,
// which equals u + d1/6 + d2/3 + d3/3 + d4/6 (y2 = u + d1/2, y3 = u + d2/2,
// y4 = u + d3) and needs no running increment sum; the differences y - u
// are exact where y is within a factor 2 of u.
template <typename T, int R>
struct FusedRegs {
    T U[4][R][VecT<T>::V];
    T Y2[4][R][VecT<T>::V], Y3[3][R][VecT<T>::V], Y4[3][R][VecT<T>::V];
};

// Everything one z-iteration needs besides the registers.
template <typename T, int R>
struct FusedIter {
    T *ring, *planes, *ering, *eplanes;   // shared memory
    const T *src[R];                       // global: this thread's column in each row, plane 0
    T *dst[R];
    long long plane;                       // n*n
    int n, n_it, zreq;                     // iterations, wrapped plane of the next request
    long long ooff;                        // output offset of the current iteration
    bool act1, act2, act3, act4, owner;
};

// One z-iteration at compile-time phase PH = it % 12 (see the kernel).
template <typename T, int TX, int TY, int R, int PH>
__device__ __forceinline__ void fused_step(FusedIter<T, R> &I, FusedRegs<T, R> &G,
                                           const FusedLane<R> &L, int it, const T (&w1)[7],
                                           const T (&w2)[7], const T (&w4)[7])
{
    using S = FusedShape<T, TX, TY, R>;
    constexpr int V = S::V, PL = S::PL, EL = S::EL, D = S::D, RING = S::RING;
    constexpr T c3 = (T)(1.0 / 3.0);
    if (it >= I.n_it) return;
    // request the u plane of iteration it + D
    if (it + D < I.n_it) {
#pragma unroll
        for (int r = 0; r < R; ++r)
            cp_async16(I.ring + ((PH + D) % RING) * PL + L.own[r], I.src[r] + (long long)I.zreq * I.plane);
    }
    cp_async_commit();
    I.zreq = I.zreq + 1 == I.n ? 0 : I.zreq + 1;
    cp_async_wait<D>();
    T un[R][V];
    T *eu = I.ering + (PH % RING) * 2 * EL;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        ldv<T>(I.ring + (PH % RING) * PL + L.own[r], un[r]);
        // edges of u(it) for the x neighbours of stage 1 in the next iteration
        eu[L.eo[r]] = un[r][0];
        eu[EL + L.eo[r]] = un[r][V - 1];
    }

    const T *Su = I.ring + ((PH + RING - 1) % RING) * PL;
    const T *Eu = I.ering + ((PH + RING - 1) % RING) * 2 * EL;
    const T *Sc = I.planes + (PH & 1) * 3 * PL;
    const T *Ec = I.eplanes + (PH & 1) * 6 * EL;
    T *Sn = I.planes + ((PH + 1) & 1) * 3 * PL;
    T *En = I.eplanes + ((PH + 1) & 1) * 6 * EL;

    // w1, w2 carry the factor 1/2 of y2 = u + d1/2 and y3 = u + d2/2, w4 the
    // factor 1/6 of d4 in the result, so each stage is one FMA chain
    T y2n[R][V] = {}, y3n[R][V] = {}, y4n[R][V] = {};
    // stage 1 at the plane of iteration it-1
    if (I.act1)
        stage_axpy<T, R>(y2n, Su, Eu, EL, L, G.U[(PH + 3) % 4], G.U[(PH + 2) % 4], un, w1,
                         G.U[(PH + 3) % 4]);
    // stage 2 at the plane of iteration it-2
    if (I.act2)
        stage_axpy<T, R>(y3n, Sc, Ec, EL, L, G.Y2[(PH + 3) % 4], G.Y2[(PH + 2) % 4], y2n, w2,
                         G.U[(PH + 2) % 4]);
    // stage 3 at the plane of iteration it-3: y4 = u + d3 = u + 2 (d3 / 2)
    if (I.act3) {
        T h[R][V];
        stage_delta<T, R>(h, Sc + PL, Ec + 2 * EL, EL, L, G.Y3[(PH + 2) % 3], G.Y3[(PH + 1) % 3],
                          y3n, w2);
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int i = 0; i < V; ++i) y4n[r][i] = fma((T)2, h[r][i], G.U[(PH + 1) % 4][r][i]);
    }
    // stage 4 at the plane of iteration it-4: the finished step
    //   u' = u + ((y2 - u) + 2 (y3 - u) + (y4 - u)) / 3 + d4 / 6
    if (I.act4 && it >= 8) {
        const T(&u4)[R][V] = G.U[PH % 4];
        const T(&y2c)[R][V] = G.Y2[(PH + 1) % 4];
        const T(&y3c)[R][V] = G.Y3[(PH + 1) % 3];
        const T(&y4c)[R][V] = G.Y4[(PH + 2) % 3];
        T b[R][V], o[R][V];
#pragma unroll
        for (int r = 0; r < R; ++r)
#pragma unroll
            for (int i = 0; i < V; ++i) {
                const T s = fma((T)2, y3c[r][i] - u4[r][i], (y2c[r][i] - u4[r][i]) + (y4c[r][i] - u4[r][i]));
                b[r][i] = fma(c3, s, u4[r][i]);
            }
        stage_axpy<T, R>(o, Sc + 2 * PL, Ec + 4 * EL, EL, L, y4c, G.Y4[(PH + 1) % 3], y4n, w4, b);
        if (I.owner) {
#pragma unroll
            for (int r = 0; r < R; ++r) stv<T>(I.dst[r] + I.ooff, o[r]);
        }
    }
    I.ooff += I.plane;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        stv<T>(Sn + L.own[r], y2n[r]);
        stv<T>(Sn + PL + L.own[r], y3n[r]);
        stv<T>(Sn + 2 * PL + L.own[r], y4n[r]);
        En[L.eo[r]] = y2n[r][0];
        En[EL + L.eo[r]] = y2n[r][V - 1];
        En[2 * EL + L.eo[r]] = y3n[r][0];
        En[3 * EL + L.eo[r]] = y3n[r][V - 1];
        En[4 * EL + L.eo[r]] = y4n[r][0];
        En[5 * EL + L.eo[r]] = y4n[r][V - 1];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < V; ++i) {
            G.U[PH % 4][r][i] = un[r][i];
            G.Y2[PH % 4][r][i] = y2n[r][i];
            G.Y3[PH % 3][r][i] = y3n[r][i];
            G.Y4[PH % 3][r][i] = y4n[r][i];
        }
}

// One RK4 step of `count` fields.  Each CTA owns a TX x TY column (plus a
// 4-point halo in x and y) of one field and a z range [z_lo, z_hi); each
// thread owns one V-vector in each of R consecutive region rows.  The CTA
// runs n_it = (z_hi - z_lo) + 8 iterations, iteration it loading plane
// z_lo - 4 + it and finishing plane z_lo - 8 + it (stage s works on plane
// z_lo - 4 + it - s).  The z loop is unrolled by 12, a multiple of every
// register window's period, so the windows never move between registers.
// With R = 2 a thread's own rows are each other's y neighbours, so per
// stage it reads one shared-memory row above and one below for two rows of
// results: a quarter less shared-memory traffic per point than R = 1.
// The RK4 step of one tile column (tile tx, ty of field f, z chunk zc) by one
// CTA of FusedShape::NT threads in the dynamic shared memory smem_raw.  A
// tile that reaches past the grid's edge (n not a multiple of the tile)
// wraps periodically like the halo and writes only the points of its own
// [tx TX, min((tx+1) TX, n)) x [ty TY, ...) range.
template <typename T, int TX, int TY, int R>
__device__ __forceinline__ void fused_tile_step(const StepArgs &a, const T *__restrict__ in,
                                                T *__restrict__ out, int f, int tx, int ty, int zc,
                                                int zchunk, unsigned char *smem_raw)
{
    using S = FusedShape<T, TX, TY, R>;
    constexpr int V = S::V, RX = S::RX, RY = S::RY, QX = S::QX, PL = S::PL, EL = S::EL;
    constexpr int D = S::D, RING = S::RING;
    constexpr int H = 4 / R;                       // halo row groups per side
    constexpr int RG = RY / R;                     // row groups in the region
    static_assert(TY % R == 0 && 4 % R == 0, "row groups must tile the region");
    T *ring = reinterpret_cast<T *>(smem_raw);
    T *planes = ring + RING * PL;
    T *ering = planes + 6 * PL;
    T *eplanes = ering + 2 * RING * EL;
    __shared__ T s_w[3][7];                        // stage 1, stages 2-3, stage 4

    const int tid = threadIdx.x;
    // Row groups (R rows each) in order of the stages they need: the TY/R
    // inner groups (all four) first, then the halo groups from the innermost
    // outwards, alternating top and bottom, so the halo groups share warps
    // and those warps skip whole stages.
    const int qx = tid % QX;
    const int gi = tid / QX;
    const int hj = gi - TY / R;
    const int grp = gi < TY / R ? H + gi : ((hj & 1) ? RG - H + (hj >> 1) : H - 1 - (hj >> 1));
    const int ry = grp * R;                        // first region row of this thread
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

    // Shared-memory row of region row y: rows are stored grouped by their
    // position within a row group (y % R), so when a warp's lanes span
    // consecutive row groups, each of its accesses covers consecutive stored
    // rows, as with one row per thread (no bank conflicts between groups).
    auto prow = [](int y) { return (y % R) * RG + y / R; };
    FusedLane<R> L;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int pr = prow(ry + r);
        L.own[r] = pr * RX + qx * V;
        L.eo[r] = pr * QX + qx;
        L.el[r] = pr * QX + (qx > 0 ? qx - 1 : 0);          // right edge of the left vector
        L.er[r] = pr * QX + (qx < QX - 1 ? qx + 1 : QX - 1); // left edge of the right vector
    }
    L.ym = prow(ry > 0 ? ry - 1 : 0) * RX + qx * V;
    L.yp = prow(ry + R < RY ? ry + R : RY - 1) * RX + qx * V;

    const int gx = ((tx * TX - 4 + qx * V) % n + n) % n;
    FusedIter<T, R> I;
    I.ring = ring;
    I.planes = planes;
    I.ering = ering;
    I.eplanes = eplanes;
    I.plane = (long long)n * n;
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int gy = ((ty * TY - 4 + ry + r) % n + n) % n;
        I.src[r] = in + (long long)f * a.P + (long long)gy * n + gx;
        I.dst[r] = out + (long long)f * a.P + (long long)gy * n + gx;
    }
    I.n = n;
    const int z_lo = zc * zchunk;
    const int z_hi = min(z_lo + zchunk, n);
    I.n_it = z_hi - z_lo + 8;
    I.ooff = (long long)(z_lo - 8) * I.plane;
    // stage s is needed on rows [s, RY-s) and elements [s, RX-s) of the region
    auto active = [&](int s) {
        return ry + R - 1 >= s && ry < RY - s && (qx + 1) * V > s && qx * V < RX - s;
    };
    // warp-uniform stage flags: a warp takes a stage when any of its lanes
    // needs it (the other lanes' results there are never read), so the
    // stage branches never diverge
    const unsigned lanes = __activemask();
    I.act1 = __any_sync(lanes, active(1));
    I.act2 = __any_sync(lanes, active(2));
    I.act3 = __any_sync(lanes, active(3));
    I.act4 = __any_sync(lanes, active(4));
    // the region's inner rows [4, 4+TY) are whole row groups (4 and TY are
    // multiples of R), so a thread owns outputs in all of its rows or none
    // (n is a multiple of 4, so the edge of a wrapped tile falls between row
    // groups and between vectors)
    I.owner = ry >= 4 && ry < 4 + TY && qx * V >= 4 && qx * V < 4 + TX &&
              tx * TX + qx * V - 4 < n && ty * TY + ry - 4 < n;

    // prologue: planes of iterations 0 .. D-1 into ring slots 0 .. D-1
    int z0 = z_lo - 4;
    z0 = ((z0 % n) + n) % n;
#pragma unroll
    for (int q = 0; q < D; ++q) {
        if (q < I.n_it) {
#pragma unroll
            for (int r = 0; r < R; ++r)
                cp_async16(ring + q * PL + L.own[r], I.src[r] + (long long)z0 * I.plane);
        }
        cp_async_commit();
        z0 = z0 + 1 == n ? 0 : z0 + 1;
    }
    I.zreq = z0;

    FusedRegs<T, R> G;
#pragma unroll
    for (int r = 0; r < R; ++r)
#pragma unroll
        for (int i = 0; i < V; ++i) {
#pragma unroll
            for (int k = 0; k < 4; ++k) G.U[k][r][i] = G.Y2[k][r][i] = (T)0;
#pragma unroll
            for (int k = 0; k < 3; ++k) G.Y3[k][r][i] = G.Y4[k][r][i] = (T)0;
        }
    for (int base = 0; base < I.n_it; base += 12) {
        fused_step<T, TX, TY, R, 0>(I, G, L, base + 0, w1, w2, w4);
        fused_step<T, TX, TY, R, 1>(I, G, L, base + 1, w1, w2, w4);
        fused_step<T, TX, TY, R, 2>(I, G, L, base + 2, w1, w2, w4);
        fused_step<T, TX, TY, R, 3>(I, G, L, base + 3, w1, w2, w4);
        fused_step<T, TX, TY, R, 4>(I, G, L, base + 4, w1, w2, w4);
        fused_step<T, TX, TY, R, 5>(I, G, L, base + 5, w1, w2, w4);
        fused_step<T, TX, TY, R, 6>(I, G, L, base + 6, w1, w2, w4);
        fused_step<T, TX, TY, R, 7>(I, G, L, base + 7, w1, w2, w4);
        fused_step<T, TX, TY, R, 8>(I, G, L, base + 8, w1, w2, w4);
        fused_step<T, TX, TY, R, 9>(I, G, L, base + 9, w1, w2, w4);
        fused_step<T, TX, TY, R, 10>(I, G, L, base + 10, w1, w2, w4);
        fused_step<T, TX, TY, R, 11>(I, G, L, base + 11, w1, w2, w4);
    }
    cp_async_wait<0>();
}

template <typename T, int TX, int TY, int R>
__global__ void __launch_bounds__(FusedShape<T, TX, TY, R>::NT, FusedShape<T, TX, TY, R>::MINB)
rk4_fused_kernel(StepArgs a, const T *__restrict__ in, T *__restrict__ out, int tiles_x,
                 int tiles_y, int zchunk, int nzc)
{
    extern __shared__ __align__(16) unsigned char smem_fused[];
    if (a.cancel && *(volatile const int *)a.cancel) return;    // uniform: no barrier is skipped
    int b = blockIdx.x;
    const int zc = b % nzc; b /= nzc;
    const int tx = b % tiles_x; b /= tiles_x;
    const int ty = b % tiles_y; b /= tiles_y;
    fused_tile_step<T, TX, TY, R>(a, in, out, b, tx, ty, zc, zchunk, smem_fused);
}

// ------------------------------------------------------- tile-step queue

__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void red_add_release_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("red.add.release.gpu.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

constexpr long long QUEUE_WAIT_LIMIT = 1ll << 22;

// Persistent CTAs that take the batch's tile steps from the queue in order.
// An item only waits for items taken before it (its problem's previous
// step), so the queue drains whatever the number of resident CTAs.
template <int TX, int TY, int R>
__global__ void __launch_bounds__(FusedShape<float, TX, TY, R>::NT, 1)
rk4_queue_kernel(const __grid_constant__ QueueParams q, unsigned long long *head,
                 unsigned long long *done, int *err)
{
    extern __shared__ __align__(16) unsigned char smem_queue[];
    __shared__ long long s_item;
    __shared__ int s_ok;
    int seg = 0;                      // the item order only grows: cursors move forward
    for (;;) {
        __syncthreads();              // the previous item's threads are all done
        if (threadIdx.x == 0) s_item = (long long)atomicAdd(head, 1ull);
        __syncthreads();
        const long long item = s_item;
        if (item >= q.total) break;
        while (seg + 1 < q.n_segs && q.seg_first_item[seg + 1] <= item) ++seg;
        const long long per_step = q.items_prefix[q.seg_active[seg]];
        const long long rel = item - q.seg_first_item[seg];
        const long long j = q.seg_first_step[seg] + rel / per_step;
        const long long r = rel % per_step;
        int i = 0;
        while (q.items_prefix[i + 1] <= r) ++i;
        const QueueEntry &E = q.e[i];
        long long local = r - q.items_prefix[i];
        // the problem's previous step must be complete
        if (threadIdx.x == 0) {
            int ok = 1;
            const unsigned long long need = (unsigned long long)(j * E.items);
            long long it = 0;
            while (ld_acquire_u64(&done[i]) < need) {
                if (++it >= QUEUE_WAIT_LIMIT || *(volatile int *)err) {
                    atomicExch(err, 1);
                    ok = 0;
                    break;
                }
                if (it > 64) __nanosleep(64);
            }
            s_ok = ok;
        }
        __syncthreads();
        if (!s_ok) break;
        const int zc = (int)(local % E.nzc); local /= E.nzc;
        const int tx = (int)(local % E.tiles_x); local /= E.tiles_x;
        const int ty = (int)(local % E.tiles_y); local /= E.tiles_y;
        const int f = (int)local;
        StepArgs a = E.a;
        a.j = j;
        const float *src = j == 0 ? E.in : ((j - 1) & 1 ? E.ws2 : E.ws1);
        float *dst = j == E.nsteps - 1 ? E.out : ((j & 1) ? E.ws2 : E.ws1);
        fused_tile_step<float, TX, TY, R>(a, src, dst, f, tx, ty, zc, E.zchunk, smem_queue);
        __syncthreads();              // every thread's stores of this tile precede the release
        if (threadIdx.x == 0) red_add_release_u64(&done[i], 1ull);
    }
}

#define PR_QUEUE_SHAPES(X) \
    X(64, 32, 1)           \
    X(64, 16, 1)           \
    X(32, 16, 1)           \
    X(64, 32, 2)

cudaError_t configure_queue_kernels()
{
    cudaError_t e = cudaSuccess;
#define PR_QCONF(TX, TY, R)                                                                      \
    if (e == cudaSuccess)                                                                        \
        e = cudaFuncSetAttribute(rk4_queue_kernel<TX, TY, R>,                                    \
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,                    \
                                 (int)FusedShape<float, TX, TY, R>::SMEM);
    PR_QUEUE_SHAPES(PR_QCONF)
#undef PR_QCONF
    return e;
}

bool rk4_queue_supported(int tile_x, int tile_y, int rows)
{
#define PR_QSUP(TX, TY, R) \
    if (tile_x == TX && tile_y == TY && rows == R) return true;
    PR_QUEUE_SHAPES(PR_QSUP)
#undef PR_QSUP
    return false;
}

cudaError_t launch_rk4_queue(const QueueParams &q, int tile_x, int tile_y, int rows,
                             unsigned long long *head, unsigned long long *done, int *err,
                             cudaStream_t st)
{
    if (q.total <= 0) return cudaSuccess;
#define PR_QLAUNCH(TX, TY, R)                                                                    \
    if (tile_x == TX && tile_y == TY && rows == R) {                                             \
        using S = FusedShape<float, TX, TY, R>;                                                  \
        int per_sm = 0;                                                                          \
        cudaError_t oe = cudaOccupancyMaxActiveBlocksPerMultiprocessor(                          \
            &per_sm, rk4_queue_kernel<TX, TY, R>, S::NT, S::SMEM);                               \
        if (oe != cudaSuccess) return oe;                                                        \
        long long grid = (long long)(per_sm < 1 ? 1 : per_sm) * sm_count();                     \
        if (grid > q.total) grid = q.total;                                                      \
        rk4_queue_kernel<TX, TY, R><<<(unsigned)grid, S::NT, S::SMEM, st>>>(q, head, done, err);  \
        return cudaGetLastError();                                                               \
    }
    PR_QUEUE_SHAPES(PR_QLAUNCH)
#undef PR_QLAUNCH
    return cudaErrorInvalidValue;
}

template <typename T, int TX, int TY, int R>
static cudaError_t launch_fused_shape(const StepArgs &a, const T *in, T *out, int zchunk,
                                      cudaStream_t st)
{
    using S = FusedShape<T, TX, TY, R>;
    // a tile that reaches past the grid's edge wraps and owns only its part
    const int tiles_x = (a.n + TX - 1) / TX, tiles_y = (a.n + TY - 1) / TY;
    const int nzc = (a.n + zchunk - 1) / zchunk;
    const long long blocks = (long long)a.count * tiles_x * tiles_y * nzc;
    rk4_fused_kernel<T, TX, TY, R><<<(unsigned)blocks, S::NT, S::SMEM, st>>>(a, in, out, tiles_x,
                                                                            tiles_y, zchunk, nzc);
    return cudaGetLastError();
}

template <typename T, int TX, int TY, int R>
static cudaError_t configure_shape()
{
    return cudaFuncSetAttribute(rk4_fused_kernel<T, TX, TY, R>,
                                cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)FusedShape<T, TX, TY, R>::SMEM);
}

// Tile shapes compiled for the fused kernel: element type, tile, rows per thread.
#define PR_FUSED_SHAPES(X) \
    X(float, 64, 32, 1)    \
    X(float, 64, 16, 1)    \
    X(float, 64, 8, 1)     \
    X(float, 32, 16, 1)    \
    X(float, 32, 8, 1)     \
    X(float, 16, 16, 1)    \
    X(float, 64, 32, 2)    \
    X(float, 64, 16, 2)    \
    X(float, 32, 32, 2)    \
    X(float, 32, 16, 2)    \
    X(double, 32, 8, 1)    \
    X(double, 16, 16, 1)   \
    X(double, 16, 8, 1)

// Shared-memory opt-in of every compiled shape (once per device, before any
// launch or stream capture).
cudaError_t configure_rk4_kernels()
{
    cudaError_t e = cudaSuccess;
#define PR_CONF(T, TX, TY, R) \
    if (e == cudaSuccess) e = configure_shape<T, TX, TY, R>();
    PR_FUSED_SHAPES(PR_CONF)
#undef PR_CONF
    return e;
}

bool rk4_fused_supported(int dtype, int n, int tile_x, int tile_y, int rows)
{
    if (n % 4) return false;
#define PR_SUP(T, TX, TY, R)                                                                 \
    if ((dtype == PARAREAL_F64) == (sizeof(T) == 8) && tile_x == TX && tile_y == TY && rows == R) \
        return true;
    PR_FUSED_SHAPES(PR_SUP)
#undef PR_SUP
    return false;
}

template <typename T>
cudaError_t launch_rk4_fused(const StepArgs &a, const T *in, T *out, int tile_x, int tile_y,
                             int zchunk, int rows, cudaStream_t st)
{
    if (zchunk <= 0 || a.n % 4) return cudaErrorInvalidValue;
#define PR_DISPATCH(TT, TX, TY, R)                                                          \
    if constexpr (std::is_same<T, TT>::value)                                                \
        if (tile_x == TX && tile_y == TY && rows == R)                                       \
            return launch_fused_shape<TT, TX, TY, R>(a, in, out, zchunk, st);
    PR_FUSED_SHAPES(PR_DISPATCH)
#undef PR_DISPATCH
    return cudaErrorInvalidValue;
}
template cudaError_t launch_rk4_fused<float>(const StepArgs &, const float *, float *, int, int,
                                             int, int, cudaStream_t);
template cudaError_t launch_rk4_fused<double>(const StepArgs &, const double *, double *, int,
                                              int, int, int, cudaStream_t);

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

// ------------------------------------------------------ persistent RK4

// Grid-wide barrier of a cooperative launch.  The last block to arrive
// resets the count and advances the generation; the others wait for the
// generation to change, for at most BARRIER_LIMIT polls, after which they
// set the error flag and every block leaves at its next barrier.
constexpr long long BARRIER_LIMIT = 1ll << 20;

__device__ __forceinline__ unsigned atom_add_acq_rel(unsigned *p, unsigned v)
{
    unsigned old;
    asm volatile("atom.add.acq_rel.gpu.u32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
    return old;
}
__device__ __forceinline__ void atom_add_release(unsigned *p, unsigned v)
{
    asm volatile("red.add.release.gpu.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned ld_acquire(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// The block's writes before the barrier reach the other blocks through the
// CTA barrier followed by thread 0's acquire-release arrival; the waiting
// blocks acquire the new generation.
__device__ __forceinline__ bool grid_sync_bounded(GridBarrier *b, unsigned nblocks, unsigned &gen)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned g = gen;
        if (atom_add_acq_rel(&b->count, 1u) == nblocks - 1) {
            atomicExch(&b->count, 0u);
            atom_add_release(&b->gen, 1u);
        } else {
            long long i = 0;
            while (ld_acquire(&b->gen) == g) {
                if (++i >= BARRIER_LIMIT) {
                    atomicExch(&b->err, 1);
                    ok = 0;
                    break;
                }
                if (i > 64) __nanosleep(20);
            }
        }
        s_ok = ok && *(volatile int *)&b->err == 0;
        gen = g + 1;
    }
    __syncthreads();
    return s_ok != 0;
}

// All nsteps RK4 steps of `count` fields in one cooperative launch: the four
// stages of each step are grid-wide passes over every point, separated by
// grid barriers (the per-stage arithmetic of rk4_stage_kernel, operand for
// operand, so the two paths agree bitwise).  u holds the state (updated in
// place at stage 4), y1/y2 the stage values, acc the running increment sum.
// The per-stage weights of every field are computed in FP64 once per step
// per block (count <= PERSIST_MAX_FIELDS).  For grids small enough that a
// step is a few microseconds of work, this replaces 4 launches per step by
// 4 barriers.
template <typename T, int R>
__global__ void __launch_bounds__(256)
rk4_persist_kernel(StepArgs a, T *__restrict__ u, T *__restrict__ y1, T *__restrict__ y2,
                   T *__restrict__ acc, long long nsteps, GridBarrier *bar)
{
    constexpr int NW = 1 + 6 * R;
    __shared__ T sw[PERSIST_MAX_FIELDS * 4 * NW];
    unsigned gen = *(volatile unsigned *)&bar->gen;
    const int n = a.n;
    const long long nn = (long long)n * n;
    const long long total = (long long)a.count * a.P;
    const long long stride = (long long)gridDim.x * blockDim.x;
    auto wrap = [n](int i, int k) { i += k; return i < 0 ? i + n : (i >= n ? i - n : i); };
    for (long long j = 0; j < nsteps; ++j) {
        __syncthreads();      // the previous step's readers of sw are done
        for (int i = threadIdx.x; i < a.count * 4; i += blockDim.x) {
            const int f = i / 4, stage = i % 4 + 1;
            const long long s = (long long)(a.first_slice + f * a.slice_stride) * a.steps_per_slice + j;
            const double t = (double)s * a.dt;
            const double c = (stage <= 1 || a.frozen) ? 0.0 : (stage == 4 ? 1.0 : 0.5);
            double w[13];
            op_weights(a.op, nu_at(a, t + c * a.dt), a.dt, n, a.a, w);
            for (int k = 0; k < NW; ++k) sw[i * NW + k] = (T)w[k];
        }
        __syncthreads();
        for (int stage = 1; stage <= 4; ++stage) {
            const T *ys = stage == 1 ? u : (stage == 3 ? y2 : y1);
            T *yd = stage == 2 ? y2 : y1;
            for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += stride) {
                const int f = (int)(q / a.P);
                const long long p = q - (long long)f * a.P;
                const T *w = sw + (f * 4 + stage - 1) * NW;
                const int x = (int)(p % n), y = (int)((p / n) % n), z = (int)(p / nn);
                const T *Y = ys + (long long)f * a.P;
                const long long row = (long long)z * nn + (long long)y * n;
                T d = w[0] * Y[row + x];
#pragma unroll
                for (int r = 1; r <= R; ++r) {
                    const int b = 1 + 6 * (r - 1);
                    d = fma(w[b + 0], Y[row + wrap(x, -r)], d);
                    d = fma(w[b + 1], Y[row + wrap(x, r)], d);
                    d = fma(w[b + 2], Y[(long long)z * nn + (long long)wrap(y, -r) * n + x], d);
                    d = fma(w[b + 3], Y[(long long)z * nn + (long long)wrap(y, r) * n + x], d);
                    d = fma(w[b + 4], Y[(long long)wrap(z, -r) * nn + (long long)y * n + x], d);
                    d = fma(w[b + 5], Y[(long long)wrap(z, r) * nn + (long long)y * n + x], d);
                }
                const T uq = u[q];
                if (stage == 1) {
                    yd[q] = fma((T)0.5, d, uq);
                    acc[q] = d * (T)(1.0 / 6.0);
                } else if (stage == 2) {
                    yd[q] = fma((T)0.5, d, uq);
                    acc[q] = fma((T)(1.0 / 3.0), d, acc[q]);
                } else if (stage == 3) {
                    yd[q] = uq + d;
                    acc[q] = fma((T)(1.0 / 3.0), d, acc[q]);
                } else {
                    u[q] = uq + fma((T)(1.0 / 6.0), d, acc[q]);
                }
            }
            if (j == nsteps - 1 && stage == 4) break;      // the launch's end is the last barrier
            if (!grid_sync_bounded(bar, gridDim.x, gen)) return;
        }
    }
}

// Failure-detection self-test of the grid barrier: block 0 leaves without
// arriving, so every other block's wait must give up and set the flag.
__global__ void grid_barrier_selftest_kernel(GridBarrier *b)
{
    unsigned gen = *(volatile unsigned *)&b->gen;
    if (blockIdx.x == 0) return;
    grid_sync_bounded(b, gridDim.x, gen);
}

cudaError_t launch_grid_barrier_selftest(GridBarrier *b, cudaStream_t st)
{
    void *args[] = {&b};
    return cudaLaunchCooperativeKernel((const void *)grid_barrier_selftest_kernel, dim3(sm_count()),
                                       dim3(32), args, 0, st);
}

template <typename T, int R>
static int persist_grid()
{
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev >= 0 && dev < 64 && cached[dev] > 0) return cached[dev];
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, rk4_persist_kernel<T, R>, 256, 0) !=
            cudaSuccess || per_sm < 1)
        per_sm = 1;
    const int g = per_sm * sm_count();
    if (dev >= 0 && dev < 64) cached[dev] = g;
    return g;
}

template <typename T>
cudaError_t launch_rk4_persist(const StepArgs &a0, T *u, T *y1, T *y2, T *acc, long long nsteps,
                               GridBarrier *bar, cudaStream_t st)
{
    if (nsteps <= 0) return cudaSuccess;
    for (int f0 = 0; f0 < a0.count; f0 += PERSIST_MAX_FIELDS) {
        StepArgs a = a0;
        a.count = a0.count - f0 < PERSIST_MAX_FIELDS ? a0.count - f0 : PERSIST_MAX_FIELDS;
        a.first_slice = a0.first_slice + f0 * a0.slice_stride;
        a.j = 0;
        const long long off = (long long)f0 * a0.P;
        T *pu = u + off, *p1 = y1 + off, *p2 = y2 + off, *pa = acc + off;
        const long long total = (long long)a.count * a.P;
        const bool r2 = op_radius(a.op) == 2;
        const int cap = r2 ? persist_grid<T, 2>() : persist_grid<T, 1>();
        // one block per SM at least: the stage work is FP64-rate bound, so every
        // SM takes a share even when that leaves threads idle
        long long want = (total + 255) / 256;
        if (want < sm_count()) want = sm_count();
        const int grid = (int)(want < cap ? want : cap);
        void *args[] = {&a, &pu, &p1, &p2, &pa, &nsteps, &bar};
        const void *fn = r2 ? (const void *)rk4_persist_kernel<T, 2> : (const void *)rk4_persist_kernel<T, 1>;
        const cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(256), args, 0, st);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}
template cudaError_t launch_rk4_persist<float>(const StepArgs &, float *, float *, float *, float *,
                                               long long, GridBarrier *, cudaStream_t);
template cudaError_t launch_rk4_persist<double>(const StepArgs &, double *, double *, double *,
                                                double *, long long, GridBarrier *, cudaStream_t);

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
    const long long cap = 16ll * sm_count();
    return (unsigned)(b < cap ? (b < 1 ? 1 : b) : cap);
}

int sm_count()
{
    // per device, queried once (device ordinals beyond the table are queried each time)
    static int cache[64] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) dev = 0;
    if (dev >= 0 && dev < 64 && cache[dev] > 0) return cache[dev];
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
    if (dev >= 0 && dev < 64) cache[dev] = n;
    return n;
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
