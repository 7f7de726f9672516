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
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "ctx.cuh"

struct parareal_batch {
    // fine sweeps of a round: 0 = each instance's own launches in its graph
    // branch; 1 = one persistent launch over a queue of every instance's tile
    // steps (queue tile shape qtx x qty, qrows rows per thread)
    int fine_mode = 0;
    int qtx = 64, qty = 32, qrows = 1;
    unsigned long long *qhead = nullptr, *qdone = nullptr;
    int *qerr = nullptr;
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
    if (b->qhead) cudaFree(b->qhead);
    if (b->qdone) cudaFree(b->qdone);
    if (b->qerr) cudaFree(b->qerr);
    if (b->own_main && b->main) cudaStreamDestroy(b->main);
    delete b;
}

extern "C" parareal_status parareal_batch_create(const parareal_config *cfgs, int count, void *stream,
                                                 parareal_batch **out)
{
    if (!out || !cfgs || count < 1) return PARAREAL_E_INVALID;
    *out = nullptr;
    // the round graph overlaps instances already; pipelined instances are not supported
    for (int i = 0; i < count; ++i)
        if (cfgs[i].pipeline_blocks != 0) return PARAREAL_E_INVALID;
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
    if (cudaMalloc((void **)&b->qhead, sizeof(unsigned long long)) != cudaSuccess ||
        cudaMalloc((void **)&b->qdone, sizeof(unsigned long long) * pr::QUEUE_MAX) != cudaSuccess ||
        cudaMalloc((void **)&b->qerr, sizeof(int)) != cudaSuccess ||
        cudaMemset(b->qerr, 0, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        parareal_batch_destroy(b);
        return PARAREAL_E_NOMEM;
    }
    *out = b;
    return PARAREAL_OK;
}

// The queue of one round: the fine sweep of the open slices of every
// selected instance (steps and tiles as rk4_batch lays them out), entries
// sorted by step count, longest first.  Input: each instance's U[K..N-1] in
// FP32 in its wC (converted by the caller), output Fv[K+1..N].
static void build_queue(parareal_batch *b, const std::vector<int> &sel, int nsteps_override,
                        pr::QueueParams *q)
{
    std::vector<int> order(sel);
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
        return b->ctx[x]->Nf > b->ctx[y]->Nf;
    });
    std::memset(q, 0, sizeof *q);
    q->n_entries = (int)order.size();
    q->items_prefix[0] = 0;
    for (int k = 0; k < q->n_entries; ++k) {
        parareal_ctx *c = b->ctx[order[k]];
        pr::QueueEntry &E = q->e[k];
        const int K = c->k_total;
        pr::StepArgs &a = E.a;
        a.op = pr::OP_C2;
        a.n = c->n;
        a.P = c->P;
        a.count = c->N - K;
        a.first_slice = K;
        a.slice_stride = 1;
        a.steps_per_slice = c->Nf;
        a.dt = c->cfg.dt_fine;
        for (int d = 0; d < 3; ++d) a.a[d] = c->cfg.a[d];
        a.nu0 = c->cfg.nu0;
        a.nu_amp = c->cfg.nu_amp;
        a.nu_omega = c->cfg.nu_omega;
        a.frozen = c->cfg.nu_mode == PARAREAL_NU_FROZEN;
        E.in = static_cast<const float *>(c->wC);
        E.out = static_cast<float *>(c->Fv) + (long long)(K + 1) * c->P;
        E.ws1 = static_cast<float *>(c->wA);
        E.ws2 = static_cast<float *>(c->wB);
        E.nsteps = nsteps_override > 0 ? nsteps_override : c->Nf;
        E.tiles_x = (c->n + b->qtx - 1) / b->qtx;
        E.tiles_y = (c->n + b->qty - 1) / b->qty;
        E.zchunk = c->n <= 64 ? c->n : 64;
        E.nzc = (c->n + E.zchunk - 1) / E.zchunk;
        E.items = (long long)a.count * E.tiles_x * E.tiles_y * E.nzc;
        q->items_prefix[k + 1] = q->items_prefix[k] + E.items;
    }
    // segments of steps with the same active prefix of entries
    q->n_segs = 0;
    long long step = 0, item = 0;
    for (int active = q->n_entries; active > 0; --active) {
        const long long last = q->e[active - 1].nsteps;    // steps while `active` entries run
        if (last <= step) continue;
        q->seg_first_step[q->n_segs] = step;
        q->seg_active[q->n_segs] = active;
        q->seg_first_item[q->n_segs] = item;
        item += (last - step) * q->items_prefix[active];
        step = last;
        ++q->n_segs;
    }
    q->seg_first_step[q->n_segs] = step;
    q->seg_first_item[q->n_segs] = item;
    q->total = item;
}

// Enqueue the queue launch of a round on b->main: zeroed counters, every
// selected instance's U[K..N-1] converted to FP32 into its wC, one launch.
static parareal_status enqueue_queue(parareal_batch *b, const std::vector<int> &sel, int nsteps_override)
{
    static pr::QueueParams q;      // ~14 KB: kept off the stack
    build_queue(b, sel, nsteps_override, &q);
    BK(cudaMemsetAsync(b->qhead, 0, sizeof(unsigned long long), b->main));
    BK(cudaMemsetAsync(b->qdone, 0, sizeof(unsigned long long) * pr::QUEUE_MAX, b->main));
    for (int i : sel) {
        parareal_ctx *c = b->ctx[i];
        const int K = c->k_total;
        BK(pr::launch_convert_f64_to_f32(c->U + (long long)K * c->P, static_cast<float *>(c->wC),
                                         (long long)(c->N - K) * c->P, b->main));
        c->launches++;
    }
    BK(pr::launch_rk4_queue(q, b->qtx, b->qty, b->qrows, b->qhead, b->qdone, b->qerr, b->main));
    return PARAREAL_OK;
}

// The queue's device-side waits since the last check.
static parareal_status queue_check(parareal_batch *b)
{
    int h = 0;
    BK(cudaMemcpyAsync(&h, b->qerr, sizeof h, cudaMemcpyDeviceToHost, b->main));
    BK(cudaStreamSynchronize(b->main));
    if (h) {
        BK(cudaMemsetAsync(b->qerr, 0, sizeof h, b->main));
        return bfail(b, PARAREAL_E_TIMEOUT, "a tile step of the batch queue gave up waiting for its problem's previous step");
    }
    return PARAREAL_OK;
}

// With the queue, every instance's batched and single-field fine launches
// use the queue's tile shape too: the serial fine run (the reference) then
// takes the same arithmetic as the queue's sweeps.
// The instances' own fine launches take the queue's shape.  The fused tile
// step computes every point by the same expression whatever the tile, rows
// per thread or z chunk, so a serial sweep already on a fused shape (the
// autotuned one) keeps it and its result stays bitwise the queue's; any
// other serial path moves to the queue's shape.
static void queue_shapes_to_instances(parareal_batch *b)
{
    const int path = b->qrows == 2 ? PATH_FUSED2 : PATH_FUSED;
    for (parareal_ctx *c : b->ctx) {
        c->fine_path = path;
        c->fine_tx = b->qtx;
        c->fine_ty = b->qty;
        c->fine_zc = c->n <= 64 ? c->n : 64;
        if (c->ser_path != PATH_FUSED && c->ser_path != PATH_FUSED2) {
            c->ser_path = path;
            c->ser_tx = b->qtx;
            c->ser_ty = b->qty;
            c->ser_zc = c->fine_zc;
        }
    }
}

extern "C" parareal_status parareal_batch_set_fine_mode(parareal_batch *b, int mode, int tile_x,
                                                         int tile_y, int rows)
{
    if (!b || (mode != 0 && mode != 1)) return PARAREAL_E_INVALID;
    if (mode == 1) {
        if ((int)b->ctx.size() > pr::QUEUE_MAX) return bfail(b, PARAREAL_E_INVALID, "at most 64 instances in the queue");
        if (!pr::rk4_queue_supported(tile_x, tile_y, rows))
            return bfail(b, PARAREAL_E_INVALID, "tile shape not compiled for the queue");
        for (parareal_ctx *c : b->ctx)
            if (c->f64 || c->fine_op != pr::OP_C2)
                return bfail(b, PARAREAL_E_INVALID, "the queue runs FP32 instances of the 7-point operator");
        b->qtx = tile_x;
        b->qty = tile_y;
        b->qrows = rows;
        queue_shapes_to_instances(b);
    }
    b->fine_mode = mode;
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_batch_get_fine_mode(const parareal_batch *b, int *mode4)
{
    if (!b || !mode4) return PARAREAL_E_INVALID;
    mode4[0] = b->fine_mode;
    mode4[1] = b->qtx;
    mode4[2] = b->qty;
    mode4[3] = b->qrows;
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
static parareal_status run_round(parareal_batch *b, const std::vector<int> &sel, Fn fn,
                                 bool queue = false)
{
    if (sel.empty()) return PARAREAL_OK;
    BK(cudaStreamBeginCapture(b->main, cudaStreamCaptureModeThreadLocal));
    // the fine sweeps of every selected instance first, as one queue launch
    parareal_status s = queue ? enqueue_queue(b, sel, 0) : PARAREAL_OK;
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
    return queue ? queue_check(b) : PARAREAL_OK;
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
        const bool queue = b->fine_mode == 1;
        s = run_round(b, sel, [queue](parareal_ctx *c) { return iter_enqueue(c, true, !queue); },
                      queue);
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
    if (b->fine_mode == 1) {
        // the queue's tile shape: two steps of every instance's full sweep per
        // candidate, timed with events (best of three after a warm-up)
        std::vector<int> all;
        for (int i = 0; i < (int)b->ctx.size(); ++i) {
            b->ctx[i]->k_total = 0;
            all.push_back(i);
        }
        const int shapes[][3] = {{64, 32, 1}, {64, 16, 1}, {32, 16, 1}, {64, 32, 2}};
        cudaEvent_t e0, e1;
        BK(cudaEventCreate(&e0));
        BK(cudaEventCreate(&e1));
        double best = 1e30;
        int pick = 0;
        for (int k = 0; k < 4; ++k) {
            b->qtx = shapes[k][0];
            b->qty = shapes[k][1];
            b->qrows = shapes[k][2];
            double t_best = 1e30;
            for (int trial = 0; trial < 4; ++trial) {
                BK(cudaEventRecord(e0, b->main));
                parareal_status s = enqueue_queue(b, all, 2);
                if (s != PARAREAL_OK) return s;
                BK(cudaEventRecord(e1, b->main));
                BK(cudaEventSynchronize(e1));
                float ms = 0.f;
                BK(cudaEventElapsedTime(&ms, e0, e1));
                if (trial > 0) t_best = std::min(t_best, (double)ms);
            }
            parareal_status s = queue_check(b);
            if (s != PARAREAL_OK) return s;
            if (t_best < best) { best = t_best; pick = k; }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        b->qtx = shapes[pick][0];
        b->qty = shapes[pick][1];
        b->qrows = shapes[pick][2];
        queue_shapes_to_instances(b);
        for (parareal_ctx *c : b->ctx) {
            c->has_problem = false;
            c->started = false;
        }
    }
    return PARAREAL_OK;
}

extern "C" long long parareal_batch_graph_launches(const parareal_batch *b)
{
    return b ? b->graph_launches : 0;
}
