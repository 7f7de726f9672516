// internal.cuh -- shared declarations of the GB300 Parareal library.
//
// Layout of every field in HBM: n^3 values, index (z*n + y)*n + x, x fastest.
// A batch of fields (time slices) is contiguous: field s starts at s*n^3.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string>

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
};

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

// ------------------------------------------------------------- launchers
// All launchers enqueue on `st` and return cudaGetLastError().

// Fused z-marching RK4 step (one full step per launch, all stages on chip).
template <typename T>
cudaError_t launch_rk4_fused(const StepArgs &a, const T *in, T *out, int tile_x, int tile_y,
                             int zchunk, cudaStream_t st);
bool rk4_fused_supported(int dtype, int n, int tile_x, int tile_y);
cudaError_t configure_rk4_kernels();

// One RK4 stage per launch (no halo recomputation; state kept in HBM/L2).
template <typename T>
cudaError_t launch_rk4_stage(const StepArgs &a, int stage, const T *ysrc, T *u, T *ydst,
                             T *acc, cudaStream_t st);

// Elementwise conversions / copies of a batch of fields.
cudaError_t launch_convert_f64_to_f32(const double *src, float *dst, long long count,
                                      cudaStream_t st);
cudaError_t launch_convert_f32_to_f64(const float *src, double *dst, long long count,
                                      cudaStream_t st);

// Box restriction (factor r) of one FP64 fine field to a T coarse field.
template <typename T>
cudaError_t launch_restrict(const double *fine, int n, int r, T *coarse, cudaStream_t st);

// Correction of Eq. (parareal) for one slice, with per-block norm partials:
//   U[p] <- Fv[p] + (g_new[p] - g_old[p]),  g = trilinear prolongation of the
//   coarse T fields cnew/cold by factor r (r == 1: plain FP64 fields gnew/gold).
// Partials per block: {max|dU|, max|U|, sum dU^2, sum U^2, nan}.
template <typename TF, typename TG>
cudaError_t launch_correct(const TF *Fv, const TG *gnew, const TG *gold, double *U, int n, int r,
                           double *partials, int nblocks, cudaStream_t st);
int correct_blocks(long long P);

// Max-abs of (a - b) and of b over one field (defect d^k), per-block partials.
template <typename TA>
cudaError_t launch_diff_norms(const TA *a, const double *b, long long P, double *partials,
                              int nblocks, cudaStream_t st);

// Fixed-order reduction of `nblocks` partial 5-tuples into out[5].
cudaError_t launch_reduce_partials(const double *partials, int nblocks, double *out,
                                   cudaStream_t st);

}  // namespace pr
