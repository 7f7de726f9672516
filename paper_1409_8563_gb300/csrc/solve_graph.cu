// solve_graph.cu -- Parareal iterations (Eq. parareal, Algorithm 1) as one
// CUDA graph launch, with the stopping test of Sec. 2.2.4 evaluated on the
// device.
//
// parareal_iterate runs one iteration per host round trip: it enqueues the
// fine sweep, the serial coarse sweep with the corrections and the norms,
// waits for them, and decides on the host whether to go on.  Here the loop
// itself is on the device:
//
//   WHILE (go) { pre --> SWITCH (K) { body[0] | body[1] | ... | body[N-1] } --> post }
//
// body[K] is the iteration with K slices already exact (slices 0..K are
// final), captured once with its launch shapes fixed: the batched fine
// sweep of slices K..N-1, the coarse sweep with the corrections of slices
// K..N-1, the norms.  The one-thread pre kernel selects K = K0 + (iterations
// run); the one-thread post kernel reads the norms the iteration produced,
// applies the stopping rule of parareal_iterate, appends the iteration's
// record to a device history and sets the loop condition go.  The
// host reads the history once, after the whole graph ran.  The iterates are
// the ones parareal_iterate produces, bit for bit: the same kernels in the
// same order on the same buffers (the roles of the double-buffered coarse
// outputs follow from the iteration count alone).
#include <chrono>
#include <cmath>
#include <cstring>

#include "ctx.cuh"

namespace {

// Device-side state of one graph solve.
struct DevSolve {
    int k_max, stop_rule, K0, N;
    int done, status;               // iterations run; 1 = non-finite value seen
    double tol;
    unsigned long long t0;          // %globaltimer at the start, ns
    int cancelled;                  // pipelined: the last speculative sweep was cancelled
    int pad;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// First node of every loop pass: the iteration to run is K = K0 + done.
__global__ void solve_pre_kernel(DevSolve *d, cudaGraphConditionalHandle which)
{
    if (threadIdx.x != 0) return;
    if (d->done == 0) d->t0 = global_ns();
    cudaGraphSetConditional(which, (unsigned)(d->K0 + d->done));
}

// The norms of the iteration with K = K0 + done exact slices: the largest
// relative changes of slices K+1..N, the defect (or -1), non-finite values.
__device__ void iteration_norms(const DevSolve *d, const double *__restrict__ norms, int has_ref,
                                double *dmax, double *l2max, double *defect, int *bad)
{
    const int N = d->N, K = d->K0 + d->done;
    *dmax = 0.0;
    *l2max = 0.0;
    *defect = -1.0;
    *bad = 0;
    for (int s = K + 1; s <= N; ++s) {
        const double *q = norms + 5 * s;
        *bad |= q[4] != 0.0;
        const double di = q[1] > 0.0 ? q[0] / q[1] : q[0];
        const double dl = q[3] > 0.0 ? sqrt(q[2] / q[3]) : sqrt(q[2]);
        *dmax = di > *dmax ? di : *dmax;
        *l2max = dl > *l2max ? dl : *l2max;
    }
    if (has_ref) {
        const double *q = norms + 5 * (N + 1);
        *bad |= q[4] != 0.0;
        *defect = q[1] > 0.0 ? q[0] / q[1] : q[0];
    }
}

// Pipelined iterations: on the main branch of a body, after the norms.  If
// the stopping rule will end the loop after this iteration (or a value is
// non-finite), the next iteration's speculative sweep is not needed: the
// cancel flag makes its remaining launches exit.
__global__ void solve_eval_kernel(DevSolve *d, const double *__restrict__ norms, int has_ref,
                                  int *cancel)
{
    if (threadIdx.x != 0) return;
    double dmax, l2max, defect;
    int bad;
    iteration_norms(d, norms, has_ref, &dmax, &l2max, &defect, &bad);
    const bool stop = bad || (d->stop_rule == PARAREAL_STOP_DIFF && dmax <= d->tol) ||
                      (d->stop_rule == PARAREAL_STOP_DEFECT && defect <= d->tol);
    if (stop) {
        *(volatile int *)cancel = 1;
        d->cancelled = 1;
    }
}

// Last node of every loop pass: the stopping test after the iteration with
// K = K0 + done exact slices -- per-slice relative changes of slices K+1..N
// (slot s of `norms` holds {max|dU|, max|U|, sum dU^2, sum U^2,
// non-finite}), the defect in slot N+1 when a reference is set, and the
// rules of parareal_iterate.
__global__ void solve_post_kernel(DevSolve *d, const double *__restrict__ norms,
                                  double *__restrict__ hist, int has_ref,
                                  cudaGraphConditionalHandle go)
{
    if (threadIdx.x != 0) return;
    const int N = d->N, K = d->K0 + d->done;
    double dmax, l2max, defect;
    int bad;
    iteration_norms(d, norms, has_ref, &dmax, &l2max, &defect, &bad);
    const int i = d->done;
    hist[4 * i + 0] = dmax;
    hist[4 * i + 1] = l2max;
    hist[4 * i + 2] = defect;
    hist[4 * i + 3] = (double)(global_ns() - d->t0) * 1e-6;
    d->done = i + 1;
    bool stop = bad || d->done >= d->k_max || K + 1 >= N;
    if (d->stop_rule == PARAREAL_STOP_DIFF && dmax <= d->tol) stop = true;
    if (d->stop_rule == PARAREAL_STOP_DEFECT && defect <= d->tol) stop = true;
    if (bad) d->status = 1;
    cudaGraphSetConditional(go, stop ? 0u : 1u);
}

}  // namespace

// Graph state kept in the context between solves.
struct SolveGraph {
    cudaGraphExec_t exec = nullptr;
    cudaGraph_t graph = nullptr;
    cudaStream_t cap = nullptr;     // capture stream (the legacy stream cannot be captured)
    DevSolve *dev = nullptr;
    double *hist = nullptr;         // 4 doubles per iteration, device
    std::vector<long long> body_launches;
    bool has_ref = false;
    int shape[16] = {0};            // launch shapes the bodies were captured with
};

// Pipelined bodies: the device-side stopping test that may cancel the
// speculative sweep, enqueued by iter_enqueue before it joins the side branch.
static void enqueue_eval(parareal_ctx *c, void *arg)
{
    SolveGraph *g = static_cast<SolveGraph *>(arg);
    solve_eval_kernel<<<1, 32, 0, c->st>>>(g->dev, c->slice_norms, g->has_ref ? 1 : 0, c->cancel);
    ++c->launches;
}

void solve_graph_free(parareal_ctx *c)
{
    SolveGraph *g = c->sgraph;
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->cap) cudaStreamDestroy(g->cap);
    if (g->dev) cudaFree(g->dev);
    if (g->hist) cudaFree(g->hist);
    delete g;
    c->sgraph = nullptr;
}

// Role of slice i's stored coarse output after the start-up and k
// iterations: the start-up writes every slot once; an iteration with K exact
// slices of the standard form writes slots K+2..N (the difference form
// writes none).
static int expected_gcur(const parareal_ctx *c, int i, int k)
{
    if (c->cfg.correction_form == PARAREAL_CORRECTION_DIFFERENCE) return 1;
    return (1 + std::max(0, std::min(k, i - 1))) & 1;
}

static void shapes_of(const parareal_ctx *c, int *sh)
{
    const int v[16] = {c->fine_path, c->fine_tx, c->fine_ty, c->fine_zc,
                       c->ser_path, c->ser_tx, c->ser_ty, c->ser_zc,
                       c->coarse_path, c->coarse_tx, c->coarse_ty, c->coarse_zc,
                       c->pipe_path, c->pipe_tx, c->pipe_ty, c->pipe_zc};
    std::memcpy(sh, v, sizeof v);
}

// Capture body[K] for every K, starting from the canonical state right after
// the coarse start-up (every stored coarse output written once).
static parareal_status build_graph(parareal_ctx *c)
{
    solve_graph_free(c);
    SolveGraph *g = new SolveGraph();
    c->sgraph = g;
    const int N = c->N;
    // pipelined bodies: the chain is captured at the highest priority, the
    // speculative sweep (side stream) at the lowest, and the graph runs with
    // these per-node priorities
    int lo = 0, hi = 0;
    CK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    CK(cudaStreamCreateWithPriority(&g->cap, cudaStreamNonBlocking, c->Fv2 ? hi : lo));
    CK(cudaMalloc((void **)&g->dev, sizeof(DevSolve)));
    CK(cudaMalloc((void **)&g->hist, sizeof(double) * 4 * (size_t)N));
    g->has_ref = c->has_ref;
    shapes_of(c, g->shape);

    cudaGraph_t top;
    CK(cudaGraphCreate(&top, 0));
    g->graph = top;
    // go is 1 at every launch; the post kernel of each pass sets it
    cudaGraphConditionalHandle go, which;
    CK(cudaGraphConditionalHandleCreate(&go, top, 1, cudaGraphCondAssignDefault));
    cudaGraphNodeParams wp{};
    wp.type = cudaGraphNodeTypeConditional;
    wp.conditional.handle = go;
    wp.conditional.type = cudaGraphCondTypeWhile;
    wp.conditional.size = 1;
    cudaGraphNode_t wnode;
    CK(cudaGraphAddNode(&wnode, top, nullptr, nullptr, 0, &wp));
    cudaGraph_t wbody = wp.conditional.phGraph_out[0];
    CK(cudaGraphConditionalHandleCreate(&which, wbody, 0, 0));
    // one loop pass: pre kernel -> SWITCH over K -> post kernel
    cudaGraphNode_t pre, snode, post;      // post: the last node of a pass
    {
        void *args[2] = {&g->dev, &which};
        cudaKernelNodeParams kp{};
        kp.func = (void *)solve_pre_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = args;
        CK(cudaGraphAddKernelNode(&pre, wbody, nullptr, 0, &kp));
    }
    cudaGraphNodeParams sp{};
    sp.type = cudaGraphNodeTypeConditional;
    sp.conditional.handle = which;
    sp.conditional.type = cudaGraphCondTypeSwitch;
    sp.conditional.size = (unsigned)N;
    CK(cudaGraphAddNode(&snode, wbody, &pre, nullptr, 1, &sp));
    {
        int has_ref = c->has_ref ? 1 : 0;
        double *norms = c->slice_norms;
        void *args[5] = {&g->dev, &norms, &g->hist, &has_ref, &go};
        cudaKernelNodeParams kp{};
        kp.func = (void *)solve_post_kernel;
        kp.gridDim = dim3(1);
        kp.blockDim = dim3(32);
        kp.kernelParams = args;
        CK(cudaGraphAddKernelNode(&post, wbody, &snode, 1, &kp));
    }

    // capture the bodies with the context's own enqueue code on the capture
    // stream, iteration after iteration from the post-start-up state
    const cudaStream_t st = c->st;
    const int k_save = c->k_total;
    const std::vector<int> gcur_save = c->gcur;
    const bool prof_save = c->prof;
    c->prof = false;
    c->st = g->cap;
    std::fill(c->gcur.begin(), c->gcur.end(), 1);
    c->gcur[0] = 0;
    g->body_launches.assign(N, 0);
    parareal_status ps = PARAREAL_OK;
    for (int K = 0; K < N && ps == PARAREAL_OK; ++K) {
        cudaGraph_t body = sp.conditional.phGraph_out[K];
        if (cudaStreamBeginCaptureToGraph(g->cap, body, nullptr, nullptr, 0,
                                          cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            ps = fail(c, PARAREAL_E_CUDA, "graph capture could not start");
            break;
        }
        c->k_total = K;
        const long long l0 = c->launches;
        ps = iter_enqueue(c, false, true, true, enqueue_eval, g);
        g->body_launches[K] = c->launches - l0 + 2;      // with the pre and post kernels
        cudaGraph_t out = nullptr;
        const cudaError_t ee = cudaStreamEndCapture(g->cap, &out);
        if (ps == PARAREAL_OK && ee != cudaSuccess)
            ps = fail(c, PARAREAL_E_CUDA, std::string("graph capture: ") + cudaGetErrorString(ee));
    }
    c->st = st;
    c->k_total = k_save;
    c->gcur = gcur_save;
    c->prof = prof_save;
    if (ps != PARAREAL_OK) {
        cudaGetLastError();
        solve_graph_free(c);
        return ps;
    }

    CK(cudaGraphInstantiate(&g->exec, top, c->Fv2 ? cudaGraphInstantiateFlagUseNodePriority : 0));
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_iterate_device(parareal_ctx *c, int k_max, double tol,
                                                   int stop_rule, int *k_done, double *hist)
{
    if (!c) return PARAREAL_E_INVALID;
    if (k_done) *k_done = 0;
    if (!c->has_problem) return fail(c, PARAREAL_E_STATE, "set_problem first");
    if (k_max < 0) return fail(c, PARAREAL_E_INVALID, "k_max < 0");
    if (stop_rule == PARAREAL_STOP_DEFECT && !c->has_ref) return fail(c, PARAREAL_E_STATE, "no reference set");
    if (stop_rule < 0 || stop_rule > 2) return fail(c, PARAREAL_E_INVALID, "stop_rule");
    ChainStream chain_stream(c);
    parareal_status s;
    if (!c->started) {
        // the coarse start-up, as parareal_iterate runs it
        s = parareal_iterate(c, 0, tol, stop_rule, nullptr, nullptr);
        if (s != PARAREAL_OK) return s;
    }
    if (k_max == 0 || c->k_total >= c->N) return PARAREAL_OK;
    // the stored coarse outputs must be in the roles the bodies were captured with
    for (int i = 1; i <= c->N; ++i) {
        if (c->gcur[i] != expected_gcur(c, i, c->k_total))
            return fail(c, PARAREAL_E_STATE, "iteration state not reached by parareal_iterate / "
                                             "parareal_iterate_device from set_problem");
    }
    int sh[16];
    shapes_of(c, sh);
    SolveGraph *g = c->sgraph;
    if (!g || g->has_ref != c->has_ref || std::memcmp(sh, g->shape, sizeof sh) != 0) {
        s = build_graph(c);
        if (s != PARAREAL_OK) {
            solve_graph_free(c);
            return s;
        }
        g = c->sgraph;
    }
    // pipelined: every body reads the F values of its iteration from the
    // previous body's speculative sweep; the first one's come from here
    if (c->Fv2 && !c->spec_valid) {
        s = fine_sweep_open(c);
        if (s != PARAREAL_OK) return s;
    }
    c->spec_valid = false;
    DevSolve h{};
    h.k_max = k_max;
    h.stop_rule = stop_rule;
    h.K0 = c->k_total;
    h.N = c->N;
    h.tol = tol;
    CK(cudaMemcpyAsync(g->dev, &h, sizeof h, cudaMemcpyHostToDevice, c->st));
    CK(cudaGraphLaunch(g->exec, c->st));
    std::vector<double> hd(4 * (size_t)c->N);
    CK(cudaMemcpyAsync(&h, g->dev, sizeof h, cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(hd.data(), g->hist, sizeof(double) * hd.size(), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(c->h_norms, c->slice_norms, sizeof(double) * 5 * (c->N + 2),
                       cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->persist_used = true;      // the bodies may hold persistent launches
    s = device_check(c);
    if (s != PARAREAL_OK) return s;
    const int K0 = c->k_total;
    for (int i = 0; i < h.done; ++i) c->launches += g->body_launches[K0 + i];
    // host bookkeeping of the last iteration run, as parareal_iterate keeps it
    const int ran = h.status ? h.done - 1 : h.done;
    c->k_total = K0 + ran;
    for (int i = 1; i <= c->N; ++i) c->gcur[i] = expected_gcur(c, i, c->k_total);
    // the last body's speculative sweep, unless cancelled, holds F(U^k) of the
    // next iteration (complete: the graph joined it)
    c->spec_valid = c->Fv2 && !h.status && !h.cancelled && h.done > 0 && c->k_total < c->N;
    c->spec_events = false;
    if (h.done > 0) {
        const int Kl = K0 + h.done - 1;          // K of the last iteration run
        for (int sl = 0; sl <= c->N; ++sl) {
            if (sl < Kl + 1) { c->diff_inf[sl] = 0.0; c->diff_l2[sl] = 0.0; continue; }
            const double *q = c->h_norms + 5 * sl;
            c->diff_inf[sl] = q[1] > 0 ? q[0] / q[1] : q[0];
            c->diff_l2[sl] = q[3] > 0 ? std::sqrt(q[2] / q[3]) : std::sqrt(q[2]);
        }
    }
    if (h.status) return fail(c, PARAREAL_E_DIVERGED, "non-finite value in the iterate");
    if (hist)
        for (int i = 0; i < ran; ++i)
            for (int j = 0; j < 4; ++j) hist[4 * i + j] = hd[4 * i + j];
    if (k_done) *k_done = ran;
    return PARAREAL_OK;
}
