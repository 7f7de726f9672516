// cluster.cu -- RK4 sweeps of small fields held in the distributed shared
// memory of one thread-block cluster per field (launch path 4).
//
// The coarse propagator of the benchmark configurations runs N_c RK4 steps
// on a 32^3 (or smaller) grid for every slice, one slice after the other:
// a sweep of a few hundred microseconds of latency and almost no work.  Here
// the whole sweep is one launch.  The n^3 field is split along z over the C
// CTAs of a cluster: CTA rank q owns planes q P .. q P + P - 1 (P = n / C) of
// four arrays in shared memory -- u, the stage inputs y1 and y2, and the
// increment sum acc.  Every stage reads the x/y neighbours of its input from
// the CTA's own shared memory and the z neighbours of its first and last
// plane from the neighbouring CTAs' (distributed shared memory, periodic in
// z), writes its own points, and ends with a cluster barrier.  The field
// crosses HBM once in and once out per sweep.
//
// The per-point arithmetic is that of rk4_stage_kernel: the same weights
// (op_weights at the stage times, rounded to T), the same operations in the
// same order, so this path and the per-stage and persistent paths give
// bitwise the same fields.  Clusters have up to 16 CTAs (8 where the device
// does not schedule 16).
#include <cooperative_groups.h>

#include "internal.cuh"

namespace cg = cooperative_groups;

namespace pr {
namespace {

constexpr int CL_THREADS = 1024;
constexpr size_t CL_SMEM_MAX = 200 * 1024;    // dynamic shared memory of one CTA

// Shared memory of one CTA: u, y1, y2 with a ghost plane below and above its
// `planes` own planes (the neighbouring CTAs' edge planes), and acc.
__host__ __device__ inline size_t cluster_smem(int n, int planes, size_t e)
{
    return ((size_t)3 * (planes + 2) + planes) * n * n * e;
}

// Thread t owns the (x, y) columns t, t + blockDim.x, ... of every own plane.
// Every stage reads only the CTA's own shared memory (ghost planes included);
// the values of its first and last plane also go, by remote stores, into the
// ghost planes of the CTA below and above, where the next stage reads them.
template <typename T>
__global__ void __launch_bounds__(CL_THREADS)
rk4_cluster_kernel(StepArgs a, const T *__restrict__ in, T *__restrict__ out, long long nsteps)
{
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int q = (int)cl.block_rank();
    const int f = (int)(blockIdx.x / C);                 // the cluster's field
    const int n = a.n, nn = n * n, planes = n / C;
    const int ext = (planes + 2) * nn;                   // one array with its ghost planes
    extern __shared__ __align__(16) unsigned char smem_cl[];
    T *arr[3];
    arr[0] = reinterpret_cast<T *>(smem_cl);             // u
    arr[1] = arr[0] + ext;                               // y1
    arr[2] = arr[1] + ext;                               // y2
    T *acc = arr[2] + ext;                               // own planes only
    __shared__ T sw[4 * 7];
    const unsigned qm = (unsigned)((q + C - 1) % C), qp = (unsigned)((q + 1) % C);
    // the neighbours' ghost planes that receive this CTA's edge planes: the
    // first own plane is the top ghost of the CTA below, the last own plane
    // the bottom ghost of the CTA above
    T *gdn[3], *gup[3];
    for (int k = 0; k < 3; ++k) {
        gdn[k] = cl.map_shared_rank(arr[k], qm) + (planes + 1) * nn;
        gup[k] = cl.map_shared_rank(arr[k], qp);
    }
    const long long base = (long long)f * a.P + (long long)q * planes * nn;
    for (int c = threadIdx.x; c < nn; c += blockDim.x)
        for (int zl = 0; zl < planes; ++zl) {
            const T v = in[base + (long long)zl * nn + c];
            arr[0][(zl + 1) * nn + c] = v;
            if (zl == 0) gdn[0][c] = v;
            if (zl == planes - 1) gup[0][c] = v;
        }
    cl.sync();      // every ghost plane of u is filled
    for (long long j = 0; j < nsteps; ++j) {
        // the step's four stage weights (the readers of the previous step's
        // are past the last stage's cluster barrier)
        if (threadIdx.x < 4) {
            const int stage = (int)threadIdx.x + 1;
            const long long s = (long long)(a.first_slice + f * a.slice_stride) * a.steps_per_slice + j;
            const double t = (double)s * a.dt;
            const double cc = (stage <= 1 || a.frozen) ? 0.0 : (stage == 4 ? 1.0 : 0.5);
            double w[13];
            op_weights(a.op, nu_at(a, t + cc * a.dt), a.dt, n, a.a, w);
            for (int k = 0; k < 7; ++k) sw[threadIdx.x * 7 + k] = (T)w[k];
        }
        __syncthreads();
        for (int stage = 1; stage <= 4; ++stage) {
            const int is = stage == 1 ? 0 : (stage == 3 ? 2 : 1);      // input array
            const int id = stage == 4 ? 0 : (stage == 2 ? 2 : 1);      // output array
            const T *ys = arr[is];
            T *yd = arr[id];
            const T *u = arr[0];
            const T *w = sw + (stage - 1) * 7;
            for (int c = threadIdx.x; c < nn; c += blockDim.x) {
                const int y = c / n, x = c - y * n;
                const int xm = c - x + (x == 0 ? n - 1 : x - 1), xp = c - x + (x == n - 1 ? 0 : x + 1);
                const int ym = (y == 0 ? n - 1 : y - 1) * n + x, yp = (y == n - 1 ? 0 : y + 1) * n + x;
                for (int zl = 0; zl < planes; ++zl) {
                    const int pl = (zl + 1) * nn;
                    const int i = pl + c;
                    T d = w[0] * ys[i];
                    d = fma(w[1], ys[pl + xm], d);
                    d = fma(w[2], ys[pl + xp], d);
                    d = fma(w[3], ys[pl + ym], d);
                    d = fma(w[4], ys[pl + yp], d);
                    d = fma(w[5], ys[i - nn], d);
                    d = fma(w[6], ys[i + nn], d);
                    const T uq = u[i];
                    const int ia = zl * nn + c;
                    T v;
                    if (stage == 1) {
                        v = fma((T)0.5, d, uq);
                        acc[ia] = d * (T)(1.0 / 6.0);
                    } else if (stage == 2) {
                        v = fma((T)0.5, d, uq);
                        acc[ia] = fma((T)(1.0 / 3.0), d, acc[ia]);
                    } else if (stage == 3) {
                        v = uq + d;
                        acc[ia] = fma((T)(1.0 / 3.0), d, acc[ia]);
                    } else {
                        v = uq + fma((T)(1.0 / 6.0), d, acc[ia]);
                    }
                    yd[i] = v;
                    if (zl == 0) gdn[id][c] = v;
                    if (zl == planes - 1) gup[id][c] = v;
                }
            }
            // the stage's outputs, ghost planes included, are complete
            // everywhere before the next stage reads them; after the last
            // stage no CTA touches another's shared memory, so every CTA may
            // leave
            cl.sync();
        }
    }
    for (int c = threadIdx.x; c < nn; c += blockDim.x)
        for (int zl = 0; zl < planes; ++zl)
            out[base + (long long)zl * nn + c] = arr[0][(zl + 1) * nn + c];
}

}  // namespace

int rk4_cluster_size(int dtype, int n)
{
    const size_t e = dtype == PARAREAL_F64 ? 8 : 4;
    static int max16 = -1;            // 16-CTA clusters schedulable on this device
    if (max16 < 0) {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(16);
        cfg.blockDim = dim3(CL_THREADS);
        cfg.dynamicSmemBytes = CL_SMEM_MAX;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = 16;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int clusters = 0;
        max16 = (configure_cluster_kernels() == cudaSuccess &&
                 cudaOccupancyMaxActiveClusters(&clusters, rk4_cluster_kernel<double>, &cfg) == cudaSuccess &&
                 clusters > 0) ? 1 : 0;
        cudaGetLastError();
    }
    for (int C : {16, 8, 4, 2, 1}) {
        if (n % C || (C == 16 && !max16)) continue;
        // the most CTAs that divide n; fewer would only hold more planes each
        return cluster_smem(n, n / C, e) <= CL_SMEM_MAX ? C : 0;
    }
    return 0;
}

cudaError_t configure_cluster_kernels()
{
    cudaError_t e = cudaSuccess;
    auto conf = [&](const void *fn) {
        if (e == cudaSuccess)
            e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)CL_SMEM_MAX);
        // clusters of 16 CTAs (beyond the portable 8) where the device schedules them
        if (e == cudaSuccess) e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    };
    conf((const void *)rk4_cluster_kernel<float>);
    conf((const void *)rk4_cluster_kernel<double>);
    return e;
}

template <typename T>
cudaError_t launch_rk4_cluster(const StepArgs &a, const T *in, T *out, long long nsteps,
                               cudaStream_t st)
{
    const int C = rk4_cluster_size(sizeof(T) == 8 ? PARAREAL_F64 : PARAREAL_F32, a.n);
    if (C == 0 || op_radius(a.op) != 1 || a.count < 1) return cudaErrorInvalidValue;
    if (nsteps <= 0)
        return in == out ? cudaSuccess
                         : cudaMemcpyAsync(out, in, (size_t)a.count * a.P * sizeof(T),
                                           cudaMemcpyDeviceToDevice, st);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(a.count * C));
    const int nn = a.n * a.n;
    cfg.blockDim = dim3((unsigned)(nn < CL_THREADS ? nn : CL_THREADS));
    cfg.dynamicSmemBytes = cluster_smem(a.n, a.n / C, sizeof(T));
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)C;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, rk4_cluster_kernel<T>, a, in, out, nsteps);
}
template cudaError_t launch_rk4_cluster<float>(const StepArgs &, const float *, float *, long long,
                                               cudaStream_t);
template cudaError_t launch_rk4_cluster<double>(const StepArgs &, const double *, double *,
                                                long long, cudaStream_t);

}  // namespace pr
