// internal.cuh -- shared declarations of the GB300 Parareal library.
//
// Layout of every field in HBM: n^3 values, index (z*n + y)*n + x, x fastest.
// A batch of fields (time slices) is contiguous: field s starts at s*n^3.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>
#include <vector>

#include "../../include/parareal.h"

namespace pr {

// ---------------------------------------------------------------- problem

// Parameters of one RK4 step launch over a batch of fields.
struct StepArgs {
    int n;                    // grid edge of this launch's fields
    long long P;              // n^3
    int count;                // number of fields (time slices) in the batch
    int first_slice;          // slice index of field 0 (for the time of each step)
    int slice_stride;         // field f runs on slice first_slice + f * slice_stride
    long long steps_per_slice;// N_f or N_c: step index of slice s, step j = s*steps_per_slice + j
    long long j;              // step number within the slice
    double dt;
    double a[3];
    double nu0, nu_amp, nu_omega;
    int frozen;               // nu at step start for all stages
    int op;                   // OP_*: spatial operator (the fused kernel is OP_C2 only)
    const int *cancel;        // fused kernel: non-null and nonzero at a CTA's start -> the
                              // CTA returns at once (a speculative sweep no longer needed)
};

// Spatial operators.  OP_C2: 7-point Laplacian, centred first differences.
// OP_C4: fourth-order centred differences (radius 2, 13 points).  OP_UPWIND:
// 7-point Laplacian, first-order upwind first differences.
enum { OP_C2 = 0, OP_C4 = 1, OP_UPWIND = 2 };

// Stencil radius of an operator.
__host__ __device__ inline int op_radius(int op) { return op == OP_C4 ? 2 : 1; }

// Per-stage 7-point weights of delta = dt * A(nu_s) y:
// w[0] centre, w[1] x-1, w[2] x+1, w[3] y-1, w[4] y+1, w[5] z-1, w[6] z+1.
__host__ __device__ inline void stage_weights(double nu, double dt, int n, const double a[3],
                                              double w[7])
{
    const double inv_h = (double)n;
    const double d = dt * nu * inv_h * inv_h;   // dt nu / h^2
    w[0] = -6.0 * d;
    for (int ax = 0; ax < 3; ++ax) {
        const double e = 0.5 * dt * a[ax] * inv_h;  // dt a / (2h)
        w[1 + 2 * ax] = d + e;   // minus-side neighbour:  + a (u_{-})/(2h)
        w[2 + 2 * ax] = d - e;   // plus-side neighbour:   - a (u_{+})/(2h)
    }
}

// Weights of delta = dt * A(nu) y for any operator: w[0] centre, then the
// radius-1 neighbours in the order of stage_weights (x-1, x+1, y-1, y+1, z-1,
// z+1), then for OP_C4 the radius-2 neighbours in the same order.
__host__ __device__ inline void op_weights(int op, double nu, double dt, int n, const double a[3],
                                           double w[13])
{
    const double inv_h = (double)n;
    if (op == OP_C2) {
        stage_weights(nu, dt, n, a, w);
        return;
    }
    if (op == OP_C4) {
        const double d = dt * nu * inv_h * inv_h / 12.0;   // dt nu / (12 h^2)
        w[0] = -90.0 * d;                                  // three axes of -30
        for (int ax = 0; ax < 3; ++ax) {
            const double e = dt * a[ax] * inv_h / 12.0;    // dt a / (12 h)
            w[1 + 2 * ax] = 16.0 * d + 8.0 * e;            // u_{-1}
            w[2 + 2 * ax] = 16.0 * d - 8.0 * e;            // u_{+1}
            w[7 + 2 * ax] = -d - e;                        // u_{-2}
            w[8 + 2 * ax] = -d + e;                        // u_{+2}
        }
        return;
    }
    // OP_UPWIND: a > 0 differences (u - u_{-1})/h, a < 0 (u_{+1} - u)/h
    const double d = dt * nu * inv_h * inv_h;
    w[0] = -6.0 * d;
    for (int ax = 0; ax < 3; ++ax) {
        const double e = dt * a[ax] * inv_h;               // dt a / h
        w[1 + 2 * ax] = d + (e > 0.0 ? e : 0.0);
        w[2 + 2 * ax] = d - (e < 0.0 ? e : 0.0);
        w[0] -= (e > 0.0 ? e : -e);
    }
}

// nu(t) = nu0 (1 + nu_amp sin(nu_omega t)) (Sec. 3), in FP64.
__device__ __forceinline__ double nu_at(const StepArgs &a, double t)
{
    return a.nu0 * (1.0 + a.nu_amp * sin(a.nu_omega * t));
}

// Streaming multiprocessors of the current device (cached per device).
int sm_count();

// ------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return cudaGetLastError().

// Fused z-marching RK4 step (one full step per launch, all stages on chip);
// `rows` = region rows per thread (1 or 2).  The tile need not divide n:
// tiles at the grid's edge wrap periodically and write only their own points.
template <typename T>
cudaError_t launch_rk4_fused(const StepArgs &a, const T *in, T *out, int tile_x, int tile_y,
                             int zchunk, int rows, cudaStream_t st);
bool rk4_fused_supported(int dtype, int n, int tile_x, int tile_y, int rows);
cudaError_t configure_rk4_kernels();


// One RK4 stage per launch (no halo recomputation; state kept in HBM/L2),
// any operator.  Stage 0 is one forward Euler step: ydst = ysrc + dt A ysrc
// (u and acc unused).
template <typename T>
cudaError_t launch_rk4_stage(const StepArgs &a, int stage, const T *ysrc, T *u, T *ydst,
                             T *acc, cudaStream_t st);

// A batch of independent problems' fine sweeps of one Parareal round as one
// persistent launch over a queue of tile steps (launch_rk4_queue).  Entry i
// is the batched RK4 sweep of one problem: a.count fields of a.n^3 points,
// nsteps steps from `in` into `out` through ws1/ws2 (the ping-pong of
// rk4_batch), tiles of the queue's shape with z chunks of zchunk planes.
struct QueueEntry {
    StepArgs a;
    const float *in;
    float *out, *ws1, *ws2;
    long long nsteps;
    int tiles_x, tiles_y, nzc, zchunk;
    long long items;                  // tiles of one step: count * tiles_x * tiles_y * nzc
};
// Queue order: step by step; within a step the problems still stepping, in
// entry order (entries sorted by nsteps, longest first, so the problems
// active at step j are a prefix).  seg_first_step[s] .. [s+1] are the steps
// with `seg_active[s]` problems; items_prefix[i] sums the items of entries
// 0..i-1.
constexpr int QUEUE_MAX = 64;
struct QueueParams {
    QueueEntry e[QUEUE_MAX];
    int n_entries, n_segs;
    long long seg_first_step[QUEUE_MAX + 1];
    int seg_active[QUEUE_MAX];
    long long seg_first_item[QUEUE_MAX + 1];
    long long items_prefix[QUEUE_MAX + 1];
    long long total;
};

// Grid-wide barrier state of the persistent RK4 kernel (device memory,
// zero-initialised; err becomes 1 when a barrier wait gave up).
struct GridBarrier {
    unsigned count, gen;
    int err, pad;
};
constexpr int PERSIST_MAX_FIELDS = 64;

// All nsteps RK4 steps of `count` fields in one cooperative launch (per 64
// fields), the per-stage arithmetic of launch_rk4_stage with a grid barrier
// between stages: u is advanced in place; y1, y2, acc are workspaces of the
// same size.  a.j is ignored (steps 0..nsteps-1 of the slice).
template <typename T>
cudaError_t launch_rk4_persist(const StepArgs &a, T *u, T *y1, T *y2, T *acc, long long nsteps,
                               GridBarrier *bar, cudaStream_t st);

// Self-test: a cooperative launch in which one block never reaches the grid
// barrier (every other block's bounded wait gives up and sets b->err).
cudaError_t launch_grid_barrier_selftest(GridBarrier *b, cudaStream_t st);

// All nsteps RK4 steps of `count` small fields (7-point operator) in one
// launch, each field held in the distributed shared memory of one
// thread-block cluster (planes split along z over the cluster's CTAs, z
// neighbours of a CTA's edge planes read from its neighbours' shared
// memory, a cluster barrier between stages): the per-point arithmetic of
// launch_rk4_stage, so the result equals the per-stage path's bit for bit.
// in may equal out.  a.j is ignored (steps 0..nsteps-1 of the slice).
template <typename T>
cudaError_t launch_rk4_cluster(const StepArgs &a, const T *in, T *out, long long nsteps,
                               cudaStream_t st);
// The cluster size for an n^3 field of `dtype` (0: the field does not fit).
int rk4_cluster_size(int dtype, int n);
cudaError_t configure_cluster_kernels();

// The fine sweeps of up to QUEUE_MAX problems in one launch: CTAs take tile
// steps from the queue in order (head: a device counter, zeroed before the
// launch); a step of problem i waits, bounded, until done[i] counts every
// tile of the problem's previous step (done zeroed before the launch; err
// set when a wait gives up, after which the CTA stops).  FP32, the fused
// kernel's tile arithmetic, so each field's result equals launch_rk4_fused's.
cudaError_t launch_rk4_queue(const QueueParams &q, int tile_x, int tile_y, int rows,
                             unsigned long long *head, unsigned long long *done, int *err,
                             cudaStream_t st);
bool rk4_queue_supported(int tile_x, int tile_y, int rows);
cudaError_t configure_queue_kernels();

// Elementwise conversions / copies of a batch of fields.
cudaError_t launch_convert_f64_to_f32(const double *src, float *dst, long long count,
                                      cudaStream_t st);
cudaError_t launch_convert_f32_to_f64(const float *src, double *dst, long long count,
                                      cudaStream_t st);

// Box restriction (factor r) of one FP64 fine field to a T coarse field.
template <typename T>
cudaError_t launch_restrict(const double *fine, int n, int r, T *coarse, cudaStream_t st);

// Spectral transfers (spectral.cu): the per-axis matrices in FP64 -- R (m x
// n), its transpose, P = r R^T (n x m) and its transpose -- and the two
// transfers, each three passes through `work` (spectral_work_elems(n, r)
// elements of T).  Restriction reads a fine FP64 field and writes the coarse
// T field; prolongation writes the fine T field P (cnew - cold) (cold may be
// null).
void spectral_matrices(int n, int r, std::vector<double> *R, std::vector<double> *Rt,
                       std::vector<double> *P, std::vector<double> *Pt);
size_t spectral_work_elems(int n, int r);
cudaError_t configure_spectral_kernels();
template <typename T>
cudaError_t launch_restrict_spectral(const double *fine, int n, int r, const T *R, const T *Rt,
                                     T *work, T *coarse, cudaStream_t st);
template <typename T>
cudaError_t launch_prolong_spectral(const T *cnew, const T *cold, int n, int r, const T *P,
                                    const T *Pt, T *work, T *fine, cudaStream_t st);

// Correction of Eq. (parareal) for one slice, with per-block norm partials:
//   U[p] <- Fv[p] + (g_new[p] - g_old[p]),  g = trilinear prolongation of the
//   coarse T fields cnew/cold by factor r (r == 1: plain FP64 fields gnew/gold).
// Partials per block: {max|dU|, max|U|, sum dU^2, sum U^2, nan}.  A non-null
// dU receives the change U_new - U_old of every point.
template <typename TF, typename TG>
cudaError_t launch_correct(const TF *Fv, const TG *gnew, const TG *gold, double *U, int n, int r,
                           double *partials, int nblocks, cudaStream_t st, double *dU = nullptr);
int correct_blocks(long long P);

// Max-abs of (a - b) and of b over one field (defect d^k), per-block partials.
template <typename TA>
cudaError_t launch_diff_norms(const TA *a, const double *b, long long P, double *partials,
                              int nblocks, cudaStream_t st);

// Fixed-order reduction of `nblocks` partial 5-tuples into out[5].
cudaError_t launch_reduce_partials(const double *partials, int nblocks, double *out,
                                   cudaStream_t st);

}  // namespace pr
