// ctx.cuh -- the context behind the opaque parareal_ctx handle, shared by
// the host-side translation units (api.cu, learned.cu).
#pragma once

#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "internal.cuh"

// Launch paths of an RK4 sweep: the fused kernel with one region row per
// thread, the per-stage kernels, the fused kernel with two rows per thread,
// and the per-stage arithmetic as one persistent cooperative launch per
// sweep (grid barriers between stages; small grids).
enum { PATH_FUSED = 0, PATH_STAGED = 1, PATH_FUSED2 = 2, PATH_PERSIST = 3, PATH_CLUSTER = 4 };
// region rows per thread of a fused launch path
inline int fused_rows(int path) { return path == PATH_FUSED2 ? 2 : 1; }
inline bool is_fused(int path) { return path == PATH_FUSED || path == PATH_FUSED2; }

// Device state of the learned coarse propagator (allocated on demand).
struct NetState {
    int m = 0;                 // grid edge the net runs on (n / coarse_factor)
    long long Pm = 0;
    int shift[3] = {0, 0, 0};  // periodic shift S, in cells, normalised to [0, m)
    int bmax = 0;              // batch capacity of the training buffers
    float *master = nullptr, *grad = nullptr, *mom1 = nullptr, *mom2 = nullptr;
    float *W1q = nullptr, *W4q = nullptr;
    __nv_bfloat16 *B2f = nullptr, *B3f = nullptr, *B2b = nullptr, *B3b = nullptr, *B4f = nullptr;
    float *nu_slices = nullptr;               // nu(t_n)/nu0 per slice
    __nv_bfloat16 *ia = nullptr, *ib = nullptr;   // inference activations, 1 field each
    // training buffers (bmax fields each)
    float *z1 = nullptr, *z2 = nullptr, *z3 = nullptr;
    __nv_bfloat16 *a1 = nullptr, *a2 = nullptr, *a3 = nullptr, *dzA = nullptr, *dzB = nullptr,
                  *dz4 = nullptr;
    float *ub = nullptr, *fb = nullptr, *nub = nullptr;
    float *partials = nullptr;
    double *loss_parts = nullptr, *loss_sum = nullptr;
    float *h_nub = nullptr;                   // pinned staging for nu of a batch
    double *h_loss = nullptr;
    int adam_t = 0;
    int lin = 0;               // linear mode (PARAREAL_ACT_LINEAR)
    bool composed = false;     // linear mode evaluated as one 9^3 kernel per slice
    double *kscratch = nullptr;             // composition scratch (device)
    float *keff = nullptr;                  // per-slice 9^3 kernels (device)
    bool poly = false;         // ... folded with the prolongation into phase kernels
    double *wpoly2 = nullptr;               // FP64 phase kernels of K_0 (+ skip) and K_1
    float *wpoly = nullptr;                 // per-slice FP32 phase kernels
    bool tc = false;           // 16 -> 16 layers on tcgen05 (grid edge a multiple of 16)
    int *tc_err = nullptr;     // device flag: a tensor-core completion wait ran out
    bool has_model = false;
};

struct SolveGraph;                // solve_graph.cu: the captured iteration loop

struct parareal_ctx {
    parareal_config cfg{};
    cudaStream_t st = nullptr;
    int dev = 0;
    int n = 0, N = 0, r = 1, nc = 0;
    long long P = 0, Pc = 0, Nf = 0, Nc = 0;
    bool f64 = false;
    size_t esz = 4;
    bool g_fine = true;           // G's output is a fine FP64 field (else coarse T)

    double *U = nullptr;
    void *Fv = nullptr;
    // pipelined iterations (cfg.pipeline_blocks > 0): F(U^k[n]) of iteration
    // k lives in Fv for even k and in Fv2 for odd k; the next iteration's
    // sweep runs on st_f, block by block, while the serial chain corrects
    void *Fv2 = nullptr;
    cudaStream_t st_f = nullptr;
    int *cancel = nullptr;            // device flag read by the speculative sweep's launches
    bool spec_valid = false;          // fv_of(k_total) holds F(U^k[n]) for the open slices
    bool spec_events = false;         // ... with the block events of a host-loop enqueue
    bool spec_pending = false;        // the last enqueue started the next iteration's sweep
    std::vector<int> spec_lo[2], spec_hi[2];           // block slice ranges, by parity of k
    std::vector<cudaEvent_t> ev_conv[2], ev_done[2];   // per block: input read / sweep done
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    // the serial chain of pipelined iterations runs on st_hi (highest
    // priority), ordered after / before the caller's stream by ev_in / ev_out
    cudaStream_t st_hi = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    int pipe_path = PATH_FUSED, pipe_tx = 64, pipe_ty = 16, pipe_zc = 0;   // block launch shape
    // G(U^k[s-1]) for s = 1..N (index 0 unused) lives in gold[s] or gold2[s]:
    // gcur[s] names the current one, the other receives the next G output.
    // The roles follow from the iteration count alone (no pointer swaps), so
    // work enqueued for a given iteration is the same whenever it is built.
    std::vector<void *> gold, gold2;
    std::vector<int> gcur;
    void *gspare = nullptr;       // scratch G output (difference form, propagate)
    void *wA = nullptr, *wB = nullptr, *wC = nullptr;
    void *cA = nullptr, *cB = nullptr, *cC = nullptr, *cD = nullptr;
    double *tmpd = nullptr;       // 2P doubles: conversions and propagate() scratch
    double *dA = nullptr, *dB = nullptr;   // U^{k+1}[n] - U^k[n] (difference-form correction)
    void *wS = nullptr;           // P of T: state of the serial fine run
    double *ref = nullptr;
    pr::GridBarrier *bar = nullptr;   // barrier state of the persistent RK4 kernel
    bool persist_used = false;        // a persistent launch ran since the last check
    // spectral transfers (coarse_transfer SPECTRAL): matrices R, R^T, P, P^T
    // in G's precision, three-pass workspace, and the prolonged fine change
    bool spectral = false;
    void *sp_R = nullptr, *sp_Rt = nullptr, *sp_P = nullptr, *sp_Pt = nullptr;
    void *sp_work = nullptr, *sp_fine = nullptr;
    double *partials = nullptr;
    int nblk = 0;
    double *slice_norms = nullptr;  // (N+1) x 5 on device
    double *h_norms = nullptr;      // pinned copy

    bool has_problem = false, started = false, has_ref = false;
    int k_total = 0;
    std::vector<double> diff_inf, diff_l2;   // last iteration, per slice

    // launch shapes: the batched fine sweep (N fields), one fine field (serial
    // fine run, propagate) and one coarse field
    int fine_op = pr::OP_C2;      // operator of F (the fused path needs OP_C2)
    int fine_path = PATH_FUSED, fine_tx = 64, fine_ty = 16, fine_zc = 0;
    int ser_path = PATH_FUSED, ser_tx = 64, ser_ty = 16, ser_zc = 0;
    int coarse_path = PATH_FUSED, coarse_tx = 32, coarse_ty = 8, coarse_zc = 0;

    NetState net;
    SolveGraph *sgraph = nullptr;

    std::string err;
    long long launches = 0;

    // kernel timing (parareal_profile)
    bool prof = false;
    std::vector<cudaEvent_t> ev_pool;   // pairs: start, stop
    size_t ev_used = 0;
    double prof_bytes = 0.0;
    long long prof_launches = 0;
};

parareal_status fail(parareal_ctx *c, parareal_status s, const std::string &msg);

// The buffer of F(U^k[n]) for iteration k.
inline void *fv_of(const parareal_ctx *c, int k) { return (c->Fv2 && (k & 1)) ? c->Fv2 : c->Fv; }

// The current and the next buffer of the stored G output of slice s.
inline void *g_cur(parareal_ctx *c, int s) { return c->gcur[s] ? c->gold2[s] : c->gold[s]; }
inline void *g_next(parareal_ctx *c, int s) { return c->gcur[s] ? c->gold[s] : c->gold2[s]; }

#define CK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(c, PARAREAL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

#define LK(call)                                                                              \
    do {                                                                                      \
        ++c->launches;                                                                        \
        CK(call);                                                                             \
    } while (0)

template <typename T>
parareal_status rk4_batch(parareal_ctx *c, int m, const T *in, T *out, int first_slice, int count,
                          long long nsteps, double dt, int path, int tx, int ty, int zc, T *ws1,
                          T *ws2, T *ws3, int slice_stride = 1, int op = pr::OP_C2,
                          const int *cancel = nullptr);

// api.cu: nsteps forward Euler steps (Algorithm 2) of `count` fields with
// operator op; in may equal out; ws1/ws2 are count*m^3 workspaces.
template <typename T>
parareal_status euler_batch(parareal_ctx *c, int m, const T *in, T *out, int first_slice,
                            int count, long long nsteps, double dt, int op, T *ws1, T *ws2);

// api.cu: one Parareal iteration split into device work and host bookkeeping.
// With pipelining, `capture` marks an enqueue inside a graph capture: the
// side branch is joined before return, no event of an earlier enqueue is
// waited on, and `stop_eval` (if set) is enqueued on the main branch after
// the norms and before the join (it sets the cancel flag).
parareal_status iter_enqueue(parareal_ctx *c, bool copy_norms = true, bool with_fine = true,
                             bool capture = false, void (*stop_eval)(parareal_ctx *, void *) = nullptr,
                             void *stop_arg = nullptr);
// api.cu: order the context's stream after the pipelined side stream
parareal_status pipe_join(parareal_ctx *c);

// Pipelined iterations run their serial chain on the context's high-priority
// stream, so that the chain's small kernels take SMs ahead of the queued CTAs
// of the speculative sweep: for the lifetime of this guard c->st is that
// stream, ordered after the caller's stream on entry; on exit the caller's
// stream is ordered after it.
struct ChainStream {
    parareal_ctx *c;
    cudaStream_t user = nullptr;
    bool on = false;
    explicit ChainStream(parareal_ctx *cc) : c(cc)
    {
        if (!c->st_hi || c->st == c->st_hi) return;
        user = c->st;
        if (cudaEventRecord(c->ev_in, user) != cudaSuccess ||
            cudaStreamWaitEvent(c->st_hi, c->ev_in, 0) != cudaSuccess)
            return;
        c->st = c->st_hi;
        on = true;
    }
    ~ChainStream()
    {
        if (!on) return;
        cudaEventRecord(c->ev_out, c->st_hi);
        cudaStreamWaitEvent(user, c->ev_out, 0);
        c->st = user;
    }
    ChainStream(const ChainStream &) = delete;
    ChainStream &operator=(const ChainStream &) = delete;
};
// api.cu: F(U^k[n]) of the open slices into fv_of(k) on the context's stream
parareal_status fine_sweep_open(parareal_ctx *c);
parareal_status iter_finish(parareal_ctx *c, double *dmax, double *l2max, double *d);

// api.cu: the stencil coarse propagator of slice s, prolonged to the fine
// grid in FP64 (the skip path of the stencil-corrected learned propagator)
parareal_status stencil_g_fine(parareal_ctx *c, const double *u, int s, double *out);

// solve_graph.cu
void solve_graph_free(parareal_ctx *c);

// api.cu: status of the device-side waits since the last check (persistent
// RK4 grid barriers, tensor-core completion waits); synchronises the stream
parareal_status device_check(parareal_ctx *c);

// learned.cu
parareal_status net_check(parareal_ctx *c);
parareal_status net_compose(parareal_ctx *c);
parareal_status net_setup(parareal_ctx *c);
void net_free(parareal_ctx *c);
template <typename TU, typename TG>
parareal_status net_apply(parareal_ctx *c, const TU *u, int slice, TG *out);
