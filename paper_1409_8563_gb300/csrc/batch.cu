// batch.cu -- many independent Parareal problems of uneven sizes advanced
// together.
//
// Each instance is a full context (its own grid edge, nu0, time steps and
// workspace) bound to a stream of its own.  One round of Parareal for the
// whole batch -- the coarse start-up, or one iteration of every instance
// still running -- is captured into a single CUDA graph in which every
// instance is a parallel branch (fork from the batch stream, join back), so
// the GPU schedules the small instances' kernels side by side.  After the
// graph ran, one host pass reads every instance's norms and applies its
// stopping rule.
#include <string>
#include <vector>

#include "ctx.cuh"

struct parareal_batch {
    std::vector<parareal_ctx *> ctx;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> join;
    cudaEvent_t fork = nullptr;
    cudaStream_t main = nullptr;
    bool own_main = false;        // the legacy default stream cannot be captured
    std::vector<int> stopped;
    std::string err;
    long long graph_launches = 0;
};

static parareal_status bfail(parareal_batch *b, parareal_status s, const std::string &m)
{
    b->err = m;
    return s;
}

#define BK(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return bfail(b, PARAREAL_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

extern "C" void parareal_batch_destroy(parareal_batch *b)
{
    if (!b) return;
    if (b->main) cudaStreamSynchronize(b->main);
    for (parareal_ctx *c : b->ctx) parareal_destroy(c);
    for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
    for (cudaEvent_t e : b->join) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->own_main && b->main) cudaStreamDestroy(b->main);
    delete b;
}

extern "C" parareal_status parareal_batch_create(const parareal_config *cfgs, int count, void *stream,
                                                 parareal_batch **out)
{
    if (!out || !cfgs || count < 1) return PARAREAL_E_INVALID;
    *out = nullptr;
    parareal_batch *b = new parareal_batch();
    b->main = static_cast<cudaStream_t>(stream);
    if (!b->main) {
        if (cudaStreamCreateWithFlags(&b->main, cudaStreamNonBlocking) != cudaSuccess) {
            b->main = nullptr;
            parareal_batch_destroy(b);
            return PARAREAL_E_CUDA;
        }
        b->own_main = true;
    }
    if (cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) != cudaSuccess) {
        parareal_batch_destroy(b);
        return PARAREAL_E_CUDA;
    }
    for (int i = 0; i < count; ++i) {
        cudaStream_t s;
        cudaEvent_t e;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            parareal_batch_destroy(b);
            return PARAREAL_E_CUDA;
        }
        b->streams.push_back(s);
        b->join.push_back(e);
        parareal_ctx *c = nullptr;
        parareal_status st = parareal_create(&cfgs[i], s, &c);
        if (st < 0) {
            parareal_batch_destroy(b);
            return st;
        }
        b->ctx.push_back(c);
    }
    b->stopped.assign(count, 0);
    *out = b;
    return PARAREAL_OK;
}

extern "C" const char *parareal_batch_last_error(const parareal_batch *b)
{
    if (!b) return "";
    if (!b->err.empty()) return b->err.c_str();
    for (parareal_ctx *c : b->ctx) {
        const char *e = parareal_last_error(c);
        if (e && *e) return e;
    }
    return "";
}

extern "C" parareal_ctx *parareal_batch_context(parareal_batch *b, int i)
{
    if (!b || i < 0 || i >= (int)b->ctx.size()) return nullptr;
    return b->ctx[i];
}

extern "C" parareal_status parareal_batch_set_problem(parareal_batch *b, int i, const void *u0,
                                                      int dtype, int mem)
{
    if (!b || i < 0 || i >= (int)b->ctx.size()) return PARAREAL_E_INVALID;
    b->stopped[i] = 0;
    return parareal_set_problem(b->ctx[i], u0, dtype, mem);
}

extern "C" parareal_status parareal_batch_serial_fine(parareal_batch *b, int as_reference)
{
    if (!b) return PARAREAL_E_INVALID;
    // every instance on its own stream, concurrently
    for (parareal_ctx *c : b->ctx) {
        parareal_status s = parareal_serial_fine(c, nullptr, PARAREAL_F64, PARAREAL_MEM_DEVICE, as_reference);
        if (s != PARAREAL_OK) return s;
    }
    for (cudaStream_t s : b->streams) BK(cudaStreamSynchronize(s));
    return PARAREAL_OK;
}

// Capture fn(ctx) for every selected instance as parallel branches of one
// graph on b->main, then launch it and wait.
template <typename Fn>
static parareal_status run_round(parareal_batch *b, const std::vector<int> &sel, Fn fn)
{
    if (sel.empty()) return PARAREAL_OK;
    BK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
    parareal_status s = PARAREAL_OK;
    cudaError_t ce = cudaEventRecord(b->fork, b->main);
    for (size_t q = 0; q < sel.size() && s == PARAREAL_OK && ce == cudaSuccess; ++q) {
        const int i = sel[q];
        ce = cudaStreamWaitEvent(b->streams[i], b->fork, 0);
        if (ce != cudaSuccess) break;
        s = fn(b->ctx[i]);
        if (s != PARAREAL_OK) break;
        ce = cudaEventRecord(b->join[i], b->streams[i]);
        if (ce == cudaSuccess) ce = cudaStreamWaitEvent(b->main, b->join[i], 0);
    }
    cudaGraph_t g = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(b->main, &g);
    if (s != PARAREAL_OK) {
        if (g) cudaGraphDestroy(g);
        return s;
    }
    if (ce != cudaSuccess || ee != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return bfail(b, PARAREAL_E_CUDA, std::string("graph capture: ") +
                                             cudaGetErrorString(ce != cudaSuccess ? ce : ee));
    }
    cudaGraphExec_t x = nullptr;
    const cudaError_t ie = cudaGraphInstantiate(&x, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) return bfail(b, PARAREAL_E_CUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
    const cudaError_t le = cudaGraphLaunch(x, b->main);
    const cudaError_t se = le == cudaSuccess ? cudaStreamSynchronize(b->main) : le;
    cudaGraphExecDestroy(x);
    if (se != cudaSuccess) return bfail(b, PARAREAL_E_CUDA, std::string("graph launch: ") + cudaGetErrorString(se));
    b->graph_launches++;
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_batch_iterate(parareal_batch *b, int k_max, double tol,
                                                  int stop_rule, int *k_done, double *defect)
{
    if (!b || k_max < 0 || stop_rule < 0 || stop_rule > 2) return PARAREAL_E_INVALID;
    const int M = (int)b->ctx.size();
    for (int i = 0; i < M; ++i) {
        if (!b->ctx[i]->has_problem) return bfail(b, PARAREAL_E_STATE, "set_problem for every instance first");
        if (stop_rule == PARAREAL_STOP_DEFECT && !b->ctx[i]->has_ref)
            return bfail(b, PARAREAL_E_STATE, "no reference set");
        if (k_done) k_done[i] = 0;
        if (defect) defect[i] = -1.0;
    }
    // coarse start-up of every instance that needs it
    std::vector<int> sel;
    for (int i = 0; i < M; ++i)
        if (!b->ctx[i]->started) sel.push_back(i);
    parareal_status s = run_round(b, sel, [](parareal_ctx *c) {
        const parareal_status r = parareal_coarse_sweep(c, 0, c->N, 1);
        if (r == PARAREAL_OK) c->started = true;
        return r;
    });
    if (s != PARAREAL_OK) return s;
    for (int round = 0; round < k_max; ++round) {
        sel.clear();
        for (int i = 0; i < M; ++i)
            if (!b->stopped[i] && b->ctx[i]->k_total < b->ctx[i]->N) sel.push_back(i);
        if (sel.empty()) break;
        s = run_round(b, sel, [](parareal_ctx *c) { return iter_enqueue(c); });
        if (s != PARAREAL_OK) return s;
        for (int i : sel) {
            parareal_ctx *c = b->ctx[i];
            double dmax, l2, d;
            s = iter_finish(c, &dmax, &l2, &d);
            if (s != PARAREAL_OK) return s;
            if (k_done) k_done[i]++;
            if (defect) defect[i] = d;
            if ((stop_rule == PARAREAL_STOP_DIFF && dmax <= tol) ||
                (stop_rule == PARAREAL_STOP_DEFECT && d <= tol))
                b->stopped[i] = 1;
        }
    }
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_batch_autotune(parareal_batch *b, const char *cache_path)
{
    if (!b) return PARAREAL_E_INVALID;
    // tune the first instance of each (grid edge, coarse edge, dtype, slices);
    // the others take its shapes
    std::vector<parareal_ctx *> done;
    for (parareal_ctx *c : b->ctx) {
        parareal_ctx *same = nullptr;
        for (parareal_ctx *d : done)
            if (d->n == c->n && d->nc == c->nc && d->f64 == c->f64 && d->N == c->N) same = d;
        if (!same) {
            parareal_status s = parareal_autotune(c, cache_path, nullptr);
            if (s != PARAREAL_OK) return s;
            done.push_back(c);
            continue;
        }
        c->fine_path = same->fine_path; c->fine_tx = same->fine_tx;
        c->fine_ty = same->fine_ty; c->fine_zc = same->fine_zc;
        c->ser_path = same->ser_path; c->ser_tx = same->ser_tx;
        c->ser_ty = same->ser_ty; c->ser_zc = same->ser_zc;
        c->coarse_path = same->coarse_path; c->coarse_tx = same->coarse_tx;
        c->coarse_ty = same->coarse_ty; c->coarse_zc = same->coarse_zc;
        c->has_problem = false;
        c->started = false;
    }
    return PARAREAL_OK;
}

extern "C" long long parareal_batch_graph_launches(const parareal_batch *b)
{
    return b ? b->graph_launches : 0;
}
