// learned.cu -- host side of the learned coarse propagator: parameter state,
// the network inside G, training-pair generation by the fine solver, and
// training (forward, backward, fixed-order gradient reduction, Adam).
//
//   G(u, t_n) = S(u) + Net([S(u), nu(t_n)/nu0])   on the grid n / coarse_factor
//
// S shifts by round(a_d * Delta t_slice * m) cells per axis (the exact
// transport of one slice when that is a whole number of cells).  Training
// minimises the mean squared error between G(u_n) and F(u_n) over pairs the
// fine propagator generates from seeded fields; with coarse_factor r > 1 both
// sides of a pair are box-restricted to the net's grid.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "ctx.cuh"
#include "net.cuh"

using namespace pr;
using bf16 = __nv_bfloat16;

static double nu_of(const parareal_config &cfg, double t)
{
    return cfg.nu0 * (1.0 + cfg.nu_amp * std::sin(cfg.nu_omega * t));
}

static bool dalloc(void **p, size_t bytes)
{
    if (cudaMalloc(p, bytes) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

parareal_status net_setup(parareal_ctx *c)
{
    NetState &S = c->net;
    // SHIFT skip: the net runs on the grid n/r after the shift S; STENCIL
    // skip: the net corrects the stencil propagator's prolonged output on the
    // fine grid (no shift: the stencil propagator already transports)
    const bool stencil_skip = c->cfg.learned_skip == PARAREAL_SKIP_STENCIL;
    S.m = stencil_skip ? c->n : c->n / c->r;
    S.lin = c->cfg.learned_act == PARAREAL_ACT_LINEAR;
    if (S.m % 8) return fail(c, PARAREAL_E_INVALID, "the learned propagator needs a grid edge that is a multiple of 8");
    S.Pm = (long long)S.m * S.m * S.m;
    const double slice = c->cfg.T / c->N;
    for (int d = 0; d < 3; ++d) {
        const long long k = stencil_skip ? 0 : std::llround(c->cfg.a[d] * slice * S.m);
        S.shift[d] = (int)(((k % S.m) + S.m) % S.m);
    }
    CK(configure_net_kernels());
    S.tc = net_tc_supported(S.m);
    if (S.tc) CK(configure_net_tc());
    bool ok = dalloc((void **)&S.master, NET_PARAMS * 4) && dalloc((void **)&S.grad, NET_PARAMS * 4) &&
              dalloc((void **)&S.mom1, NET_PARAMS * 4) && dalloc((void **)&S.mom2, NET_PARAMS * 4) &&
              dalloc((void **)&S.W1q, 864 * 4) && dalloc((void **)&S.W4q, 432 * 4) &&
              dalloc((void **)&S.B2f, 6912 * 2) && dalloc((void **)&S.B3f, 6912 * 2) &&
              dalloc((void **)&S.B2b, 6912 * 2) && dalloc((void **)&S.B3b, 6912 * 2) &&
              dalloc((void **)&S.B4f, 27 * 8 * 16 * 2) && dalloc((void **)&S.tc_err, sizeof(int)) &&
              dalloc((void **)&S.nu_slices, sizeof(float) * c->N) &&
              dalloc((void **)&S.ia, (size_t)S.Pm * 32) && dalloc((void **)&S.ib, (size_t)S.Pm * 32);
    S.composed = S.lin && c->cfg.learned_eval != PARAREAL_EVAL_LAYERS;
    S.poly = S.lin && c->cfg.learned_eval == PARAREAL_EVAL_POLYPHASE && stencil_skip && c->r > 1;
    if (S.composed && S.m % 16)
        return fail(c, PARAREAL_E_INVALID, "the composed learned propagator needs a grid edge that is a multiple of 16");
    if (ok && S.composed)
        ok = dalloc((void **)&S.kscratch, compose_scratch_doubles() * sizeof(double)) &&
             dalloc((void **)&S.keff, sizeof(float) * NET_K9 * c->N);
    if (ok && S.poly) {
        ok = dalloc((void **)&S.wpoly2, poly_scratch_doubles(c->r) * sizeof(double)) &&
             dalloc((void **)&S.wpoly, poly_weights_floats(c->r, c->N) * sizeof(float));
        CK(configure_poly_kernels(c->r));
    }
    if (!ok) return fail(c, PARAREAL_E_NOMEM, "learned propagator allocation failed");
    std::vector<float> nus(c->N);
    for (int s = 0; s < c->N; ++s) nus[s] = (float)(nu_of(c->cfg, s * slice) / c->cfg.nu0);
    CK(cudaMemcpy(S.nu_slices, nus.data(), sizeof(float) * c->N, cudaMemcpyHostToDevice));
    // Net = 0 until a model is set: G = S (the shift-only propagator)
    CK(cudaMemsetAsync(S.master, 0, NET_PARAMS * 4, c->st));
    CK(cudaMemsetAsync(S.tc_err, 0, sizeof(int), c->st));
    CK(cudaMemsetAsync(S.mom1, 0, NET_PARAMS * 4, c->st));
    CK(cudaMemsetAsync(S.mom2, 0, NET_PARAMS * 4, c->st));
    LK(launch_prepare_operands(S.master, S.W1q, S.B2f, S.B3f, S.B2b, S.B3b, S.W4q, S.B4f, c->st));
    S.has_model = c->cfg.coarse_kind == PARAREAL_COARSE_SHIFT;
    return net_compose(c);
}

// Composed evaluation: rebuild the per-slice 9^3 kernels from the master
// weights (stream-ordered; called whenever the model changes).
parareal_status net_compose(parareal_ctx *c)
{
    NetState &S = c->net;
    if (!S.composed) return PARAREAL_OK;
    LK(launch_compose_linear(S.master, S.nu_slices, c->N, S.kscratch, S.keff, c->st));
    if (S.poly)
        LK(launch_compose_poly(composed_kernels(S.kscratch), c->r, S.nu_slices, c->N, S.wpoly2, S.wpoly, c->st));
    return PARAREAL_OK;
}

void net_free(parareal_ctx *c)
{
    NetState &S = c->net;
    void *p[] = {S.master, S.grad, S.mom1, S.mom2, S.W1q, S.W4q, S.B2f, S.B3f, S.B2b, S.B3b, S.B4f, S.tc_err,
                 S.nu_slices, S.ia, S.ib, S.z1, S.z2, S.z3, S.a1, S.a2, S.a3, S.dzA, S.dzB, S.dz4,
                 S.ub, S.fb, S.nub, S.partials, S.loss_parts, S.loss_sum, S.kscratch, S.keff,
                 S.wpoly2, S.wpoly};
    for (void *q : p)
        if (q) cudaFree(q);
    if (S.h_nub) cudaFreeHost(S.h_nub);
    if (S.h_loss) cudaFreeHost(S.h_loss);
    S = NetState();
}

// Status of the tensor-core layers since the last check (synchronises the stream).
parareal_status net_check(parareal_ctx *c)
{
    NetState &S = c->net;
    if (!S.tc || !S.tc_err) return PARAREAL_OK;
    int h = 0;
    CK(cudaMemcpyAsync(&h, S.tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (h) {
        // clear the flag so that later calls on this context report only their own timeouts
        CK(cudaMemsetAsync(S.tc_err, 0, sizeof(int), c->st));
        return fail(c, PARAREAL_E_TIMEOUT, "tensor-core completion wait ran out in the learned propagator");
    }
    return PARAREAL_OK;
}

// G for one field of slice `slice`: u on the net's grid (TU), out on it (TG).
template <typename TU, typename TG>
parareal_status net_apply(parareal_ctx *c, const TU *u, int slice, TG *out)
{
    NetState &S = c->net;
    if (S.composed) {
        // the four linear layers as one 9^3 cross-correlation (net_composed.cu)
        LK((launch_net_lin9<TU, TG>(u, S.m, S.shift, S.keff + (size_t)slice * NET_K9, out, c->st)));
        return PARAREAL_OK;
    }
    const float *b = S.master;
    LK(launch_net_in_fwd<TU>(u, S.m, S.shift, S.nu_slices + slice, 1, S.W1q, b + NET_B1, nullptr, S.ia, c->st,
                             S.lin));
    if (S.tc) {
        LK(launch_net_mid_tc(0, S.ia, S.m, 1, S.B2f, b + NET_B2, nullptr, nullptr, S.ib, S.lin, S.tc_err, c->st));
        LK(launch_net_mid_tc(0, S.ib, S.m, 1, S.B3f, b + NET_B3, nullptr, nullptr, S.ia, S.lin, S.tc_err, c->st));
    } else {
        LK(launch_net_mid(0, S.ia, S.m, 1, S.B2f, b + NET_B2, nullptr, nullptr, S.ib, c->st, S.lin));
        LK(launch_net_mid(0, S.ib, S.m, 1, S.B3f, b + NET_B3, nullptr, nullptr, S.ia, c->st, S.lin));
    }
    LK((launch_net_out_mma<TU, TG>(S.ia, S.m, 1, S.B4f, b + NET_B4, u, S.shift, out, c->st, S.lin)));
    return PARAREAL_OK;
}
template parareal_status net_apply<double, double>(parareal_ctx *, const double *, int, double *);
template parareal_status net_apply<float, float>(parareal_ctx *, const float *, int, float *);
template parareal_status net_apply<double, float>(parareal_ctx *, const double *, int, float *);
template parareal_status net_apply<float, double>(parareal_ctx *, const float *, int, double *);

static parareal_status net_training_buffers(parareal_ctx *c, int batch)
{
    NetState &S = c->net;
    if (S.bmax >= batch) return PARAREAL_OK;
    void *p[] = {S.z1, S.z2, S.z3, S.a1, S.a2, S.a3, S.dzA, S.dzB, S.dz4, S.ub, S.fb, S.nub,
                 S.partials, S.loss_parts, S.loss_sum};
    for (void *q : p)
        if (q) cudaFree(q);
    if (S.h_nub) cudaFreeHost(S.h_nub);
    if (S.h_loss) cudaFreeHost(S.h_loss);
    const size_t F = (size_t)batch * S.Pm;
    const int nb = net_partial_blocks(S.m, batch);
    const size_t tiles = (size_t)batch * (S.m / 8) * (S.m / 8) * (S.m / 8);
    bool ok = dalloc((void **)&S.z1, F * 64) && dalloc((void **)&S.z2, F * 64) && dalloc((void **)&S.z3, F * 64) &&
              dalloc((void **)&S.a1, F * 32) && dalloc((void **)&S.a2, F * 32) && dalloc((void **)&S.a3, F * 32) &&
              dalloc((void **)&S.dzA, F * 32) && dalloc((void **)&S.dzB, F * 32) && dalloc((void **)&S.dz4, F * 2) &&
              dalloc((void **)&S.ub, F * 4) && dalloc((void **)&S.fb, F * 4) &&
              dalloc((void **)&S.nub, sizeof(float) * batch) &&
              dalloc((void **)&S.partials, sizeof(float) * (size_t)nb * NET_MID_PARTIAL) &&
              dalloc((void **)&S.loss_parts, sizeof(double) * tiles) &&
              dalloc((void **)&S.loss_sum, sizeof(double) * 4096);
    ok = ok && cudaMallocHost((void **)&S.h_nub, sizeof(float) * batch) == cudaSuccess &&
         cudaMallocHost((void **)&S.h_loss, sizeof(double) * 4096) == cudaSuccess;
    if (!ok) {
        cudaGetLastError();
        S.bmax = 0;
        return fail(c, PARAREAL_E_NOMEM, "training buffers");
    }
    S.bmax = batch;
    return PARAREAL_OK;
}

// One 16 -> 16 layer of training, forward (mode 0, pre-activations into zout)
// or input gradient (mode 1, mirrored operand, times gelu'(zaux)): on the
// tensor cores (tcgen05) where the grid edge allows their tiles, else the
// mma.sync kernel.
static cudaError_t mid_layer(parareal_ctx *c, int mode, const __nv_bfloat16 *in, int batch,
                             const __nv_bfloat16 *Bt, const float *bias, const float *zaux, float *zout,
                             __nv_bfloat16 *out)
{
    NetState &S = c->net;
    if (S.tc)
        return launch_net_mid_tc(mode, in, S.m, batch, Bt, bias, zaux, zout, out, S.lin, S.tc_err, c->st);
    return launch_net_mid(mode, in, S.m, batch, Bt, bias, zaux, zout, out, c->st, S.lin);
}

// Weight-gradient partials of a 16 -> 16 layer (input x, output gradient dz),
// on the tensor cores where the forward runs there.
static cudaError_t mid_wgrad(parareal_ctx *c, const __nv_bfloat16 *x, const __nv_bfloat16 *dz, int batch,
                             int nb)
{
    NetState &S = c->net;
    if (S.tc) return launch_net_mid_wgrad_tc(x, dz, S.m, batch, S.partials, nb, S.tc_err, c->st);
    return launch_net_mid_wgrad(x, dz, S.m, batch, S.partials, nb, c->st);
}

// Loss and gradient of one batch already staged in S.ub / S.fb / S.nub;
// the loss sum lands in loss_slot (device).  grad = d(mean squared error)/dparams.
static parareal_status net_loss_grad(parareal_ctx *c, int batch, double *loss_slot)
{
    NetState &S = c->net;
    const float *b = S.master;
    const int m = S.m;
    const long long F = (long long)batch * S.Pm;
    const int tiles = (int)((long long)batch * (m / 8) * (m / 8) * (m / 8));
    // forward, keeping pre-activations
    LK(launch_net_in_fwd<float>(S.ub, m, S.shift, S.nub, batch, S.W1q, b + NET_B1, S.z1, S.a1, c->st,
                                S.lin));
    LK(mid_layer(c, 0, S.a1, batch, S.B2f, b + NET_B2, nullptr, S.z2, S.a2));
    LK(mid_layer(c, 0, S.a2, batch, S.B3f, b + NET_B3, nullptr, S.z3, S.a3));
    const float gscale = (float)(2.0 / (double)F);
    LK(launch_net_out_mma_train(S.a3, m, batch, S.B4f, b + NET_B4, S.ub, S.shift, S.fb, gscale, S.dz4,
                                S.loss_parts, c->st, S.lin));
    LK(launch_reduce_loss(S.loss_parts, tiles, loss_slot, c->st));
    // backward
    const int nb = net_partial_blocks(m, batch);
    LK(launch_net_out_wgrad(S.a3, S.dz4, m, batch, S.partials, nb, c->st));
    LK(launch_reduce_cols(S.partials, nb, NET_OUT_PARTIAL, NET_OUT_PARTIAL, S.grad + NET_W4, c->st));
    LK(launch_net_out_dgrad(S.dz4, m, batch, S.W4q, S.z3, S.dzA, c->st, S.lin));   // dz3
    LK(mid_wgrad(c, S.a2, S.dzA, batch, nb));
    LK(launch_reduce_mid(S.partials, nb, S.grad + NET_W3, S.grad + NET_B3, c->st));
    LK(mid_layer(c, 1, S.dzA, batch, S.B3b, nullptr, S.z2, nullptr, S.dzB));  // dz2
    LK(mid_wgrad(c, S.a1, S.dzB, batch, nb));
    LK(launch_reduce_mid(S.partials, nb, S.grad + NET_W2, S.grad + NET_B2, c->st));
    LK(mid_layer(c, 1, S.dzB, batch, S.B2b, nullptr, S.z1, nullptr, S.dzA));  // dz1
    LK(launch_net_in_wgrad<float>(S.ub, m, batch, S.shift, S.nub, S.dzA, S.partials, nb, c->st, S.lin));
    LK(launch_reduce_cols(S.partials, nb, NET_IN_PARTIAL, NET_IN_PARTIAL, S.grad + NET_W1, c->st));
    if (S.lin) {
        // the linear net has no biases: their gradients are zero and Adam leaves them
        CK(cudaMemsetAsync(S.grad + NET_B1, 0, 16 * 4, c->st));
        CK(cudaMemsetAsync(S.grad + NET_B2, 0, 16 * 4, c->st));
        CK(cudaMemsetAsync(S.grad + NET_B3, 0, 16 * 4, c->st));
        CK(cudaMemsetAsync(S.grad + NET_B4, 0, 4, c->st));
    }
    return PARAREAL_OK;
}

// Stage batch fields (device FP32, Pm each) and their nu values.
static parareal_status stage_batch(parareal_ctx *c, const float *const *us, const float *const *fs,
                                   const int *slices, int batch)
{
    NetState &S = c->net;
    const size_t bytes = (size_t)S.Pm * 4;
    for (int i = 0; i < batch; ++i) {
        CK(cudaMemcpyAsync(S.ub + i * S.Pm, us[i], bytes, cudaMemcpyDeviceToDevice, c->st));
        if (fs) CK(cudaMemcpyAsync(S.fb + i * S.Pm, fs[i], bytes, cudaMemcpyDeviceToDevice, c->st));
    }
    CK(cudaStreamSynchronize(c->st));   // h_nub reuse
    const double slice = c->cfg.T / c->N;
    for (int i = 0; i < batch; ++i)
        S.h_nub[i] = (float)(nu_of(c->cfg, slices[i] * slice) / c->cfg.nu0);
    CK(cudaMemcpyAsync(S.nub, S.h_nub, sizeof(float) * batch, cudaMemcpyHostToDevice, c->st));
    return PARAREAL_OK;
}

static parareal_status need_learned(parareal_ctx *c)
{
    if (!c) return PARAREAL_E_INVALID;
    if ((c->cfg.coarse_kind != PARAREAL_COARSE_LEARNED && c->cfg.coarse_kind != PARAREAL_COARSE_SHIFT) ||
        !c->net.master)
        return fail(c, PARAREAL_E_STATE, "context was not created with a learned coarse propagator");
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_set_coarse_model(parareal_ctx *c, const float *w, int mem)
{
    parareal_status s = need_learned(c);
    if (s != PARAREAL_OK) return s;
    if (!w) return fail(c, PARAREAL_E_INVALID, "null weights");
    NetState &S = c->net;
    CK(cudaMemcpyAsync(S.master, w, NET_PARAMS * 4,
                       mem == PARAREAL_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemsetAsync(S.mom1, 0, NET_PARAMS * 4, c->st));
    CK(cudaMemsetAsync(S.mom2, 0, NET_PARAMS * 4, c->st));
    S.adam_t = 0;
    LK(launch_prepare_operands(S.master, S.W1q, S.B2f, S.B3f, S.B2b, S.B3b, S.W4q, S.B4f, c->st));
    if (mem == PARAREAL_MEM_HOST) CK(cudaStreamSynchronize(c->st));
    s = net_compose(c);
    if (s != PARAREAL_OK) return s;
    S.has_model = true;
    c->started = false;   // G changed: the next iterate restarts from the coarse chain
    c->k_total = 0;
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_get_coarse_model(parareal_ctx *c, float *w, int mem)
{
    parareal_status s = need_learned(c);
    if (s != PARAREAL_OK) return s;
    if (!w) return fail(c, PARAREAL_E_INVALID, "null weights");
    CK(cudaMemcpyAsync(w, c->net.master, NET_PARAMS * 4,
                       mem == PARAREAL_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    return PARAREAL_OK;
}

extern "C" parareal_status parareal_coarse_model_grad(parareal_ctx *c, const float *u,
                                                      const float *target, const int *slices,
                                                      int count, float *grad_out, double *loss)
{
    if (c) c->spec_valid = false;      // U, F or the sweep workspaces may change
    parareal_status s = need_learned(c);
    if (s != PARAREAL_OK) return s;
    if (!u || !target || !slices || count < 1 || !grad_out) return fail(c, PARAREAL_E_INVALID, "arguments");
    for (int i = 0; i < count; ++i)
        if (slices[i] < 0 || slices[i] >= c->N) return fail(c, PARAREAL_E_INVALID, "slice index");
    if ((s = net_training_buffers(c, count)) != PARAREAL_OK) return s;
    NetState &S = c->net;
    std::vector<const float *> us(count), fs(count);
    for (int i = 0; i < count; ++i) {
        us[i] = u + (size_t)i * S.Pm;
        fs[i] = target + (size_t)i * S.Pm;
    }
    if ((s = stage_batch(c, us.data(), fs.data(), slices, count)) != PARAREAL_OK) return s;
    if ((s = net_loss_grad(c, count, S.loss_sum)) != PARAREAL_OK) return s;
    CK(cudaMemcpyAsync(grad_out, S.grad, NET_PARAMS * 4, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(S.h_loss, S.loss_sum, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if ((s = net_check(c)) != PARAREAL_OK) return s;      // tensor-core completion waits
    if (loss) *loss = S.h_loss[0] / ((double)count * S.Pm);
    return PARAREAL_OK;
}

// splitmix64 (Steele, Lea & Flood 2014): the shuffling generator of training.
static uint64_t splitmix64(uint64_t &x)
{
    uint64_t z = (x += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

extern "C" parareal_status parareal_train_coarse(parareal_ctx *c, const float *pairs_u,
                                                 const float *pairs_f, const int *pair_slice,
                                                 int n_pairs, const parareal_train_config *tc,
                                                 double *loss_hist)
{
    if (c) c->spec_valid = false;      // U, F or the sweep workspaces may change
    parareal_status s = need_learned(c);
    if (s != PARAREAL_OK) return s;
    if (!pairs_u || !pairs_f || !pair_slice || !tc || n_pairs < 1 || tc->epochs < 0 || tc->batch < 1)
        return fail(c, PARAREAL_E_INVALID, "arguments");
    for (int i = 0; i < n_pairs; ++i)
        if (pair_slice[i] < 0 || pair_slice[i] >= c->N) return fail(c, PARAREAL_E_INVALID, "slice index");
    const int B = std::min(tc->batch, n_pairs);
    if ((s = net_training_buffers(c, B)) != PARAREAL_OK) return s;
    NetState &S = c->net;
    const int nbat = n_pairs / B;   // the remainder of a shuffled epoch is dropped
    if (nbat > 4096) return fail(c, PARAREAL_E_INVALID, "too many batches per epoch (max 4096)");
    std::vector<int> perm(n_pairs);
    uint64_t rng = tc->seed;
    std::vector<const float *> us(B), fs(B);
    std::vector<int> sl(B);
    for (int e = 0; e < tc->epochs; ++e) {
        for (int i = 0; i < n_pairs; ++i) perm[i] = i;
        for (int i = n_pairs - 1; i > 0; --i) {    // Fisher-Yates
            const int j = (int)(splitmix64(rng) % (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        for (int bi = 0; bi < nbat; ++bi) {
            for (int k = 0; k < B; ++k) {
                const int q = perm[bi * B + k];
                us[k] = pairs_u + (size_t)q * S.Pm;
                fs[k] = pairs_f + (size_t)q * S.Pm;
                sl[k] = pair_slice[q];
            }
            if ((s = stage_batch(c, us.data(), fs.data(), sl.data(), B)) != PARAREAL_OK) return s;
            if ((s = net_loss_grad(c, B, S.loss_sum + bi)) != PARAREAL_OK) return s;
            S.adam_t++;
            const double c1 = 1.0 - std::pow(tc->beta1, S.adam_t);
            const double c2 = 1.0 - std::pow(tc->beta2, S.adam_t);
            LK(launch_adam(S.master, S.grad, S.mom1, S.mom2, NET_PARAMS, (float)tc->lr, (float)tc->beta1,
                           (float)tc->beta2, (float)tc->eps, (float)c1, (float)c2, c->st));
            LK(launch_prepare_operands(S.master, S.W1q, S.B2f, S.B3f, S.B2b, S.B3b, S.W4q, S.B4f, c->st));
        }
        CK(cudaMemcpyAsync(S.h_loss, S.loss_sum, sizeof(double) * nbat, cudaMemcpyDeviceToHost, c->st));
        CK(cudaStreamSynchronize(c->st));
        if ((s = net_check(c)) != PARAREAL_OK) return s;  // tensor-core completion waits
        double tot = 0.0;
        for (int bi = 0; bi < nbat; ++bi) tot += S.h_loss[bi];
        if (!std::isfinite(tot)) return fail(c, PARAREAL_E_DIVERGED, "training loss is not finite");
        if (loss_hist) loss_hist[e] = tot / ((double)nbat * B * S.Pm);
    }
    if ((s = net_compose(c)) != PARAREAL_OK) return s;
    S.has_model = true;
    c->started = false;
    c->k_total = 0;
    return PARAREAL_OK;
}

// Training pairs from the fine solver: for each of n_ics seeded fields the
// serial fine trajectory over all slices gives pairs (u_n, F(u_n)), n = 0..N-1,
// stored at pair index ic * N + n (restricted to the net's grid when r > 1).
template <typename T>
static parareal_status make_pairs_t(parareal_ctx *c, const float *ics, int n_ics, float *pu, float *pf,
                                    int *pair_slice)
{
    const long long P = c->P;
    const size_t fb = (size_t)n_ics * P * sizeof(T);
    T *st = nullptr, *w1 = nullptr, *w2 = nullptr, *w3 = nullptr, *nx = nullptr;
    double *tmp = nullptr;
    const bool restrict_pairs = c->net.m != c->n;          // net on the restricted grid
    const bool stencil_skip = c->cfg.learned_skip == PARAREAL_SKIP_STENCIL;
    bool ok = dalloc((void **)&st, fb) && dalloc((void **)&w1, fb) && dalloc((void **)&w2, fb) &&
              dalloc((void **)&w3, fb) && dalloc((void **)&nx, fb) &&
              (!(restrict_pairs || stencil_skip) || dalloc((void **)&tmp, (size_t)P * 8));
    auto cleanup = [&]() {
        for (void *q : {(void *)st, (void *)w1, (void *)w2, (void *)w3, (void *)nx, (void *)tmp})
            if (q) cudaFree(q);
    };
    if (!ok) {
        cleanup();
        return fail(c, PARAREAL_E_NOMEM, "pair generation buffers");
    }
    const long long Pm = c->net.Pm;
    auto emit = [&](const T *field, float *dst) -> parareal_status {
        // one field on the fine grid -> the net's grid, FP32
        if (!restrict_pairs) {
            if (std::is_same<T, float>::value)
                CK(cudaMemcpyAsync(dst, field, P * 4, cudaMemcpyDeviceToDevice, c->st));
            else
                LK(launch_convert_f64_to_f32(reinterpret_cast<const double *>(field), dst, P, c->st));
        } else {
            if (std::is_same<T, float>::value)
                LK(launch_convert_f32_to_f64(reinterpret_cast<const float *>(field), tmp, P, c->st));
            else
                CK(cudaMemcpyAsync(tmp, field, P * 8, cudaMemcpyDeviceToDevice, c->st));
            LK(launch_restrict<float>(tmp, c->n, c->r, dst, c->st));
        }
        return PARAREAL_OK;
    };
    parareal_status s = PARAREAL_OK;
    if (std::is_same<T, float>::value)
        CK(cudaMemcpyAsync(st, ics, fb, cudaMemcpyDeviceToDevice, c->st));
    else
        LK(launch_convert_f32_to_f64(ics, reinterpret_cast<double *>(st), (long long)n_ics * P, c->st));
    // STENCIL skip: the net's input is the stencil propagator's output Gs(u_n)
    auto emit_skip = [&](const T *field, int slice, float *dst) -> parareal_status {
        if (std::is_same<T, float>::value)
            LK(launch_convert_f32_to_f64(reinterpret_cast<const float *>(field), tmp, P, c->st));
        else
            CK(cudaMemcpyAsync(tmp, field, P * 8, cudaMemcpyDeviceToDevice, c->st));
        double *gs = c->tmpd + P;
        parareal_status ps = stencil_g_fine(c, tmp, slice, gs);
        if (ps != PARAREAL_OK) return ps;
        LK(launch_convert_f64_to_f32(gs, dst, P, c->st));
        return PARAREAL_OK;
    };
    for (int n = 0; n < c->N && s == PARAREAL_OK; ++n) {
        for (int i = 0; i < n_ics && s == PARAREAL_OK; ++i) {
            float *dst = pu + ((size_t)i * c->N + n) * Pm;
            s = stencil_skip ? emit_skip(st + (size_t)i * P, n, dst) : emit(st + (size_t)i * P, dst);
            if (pair_slice) pair_slice[i * c->N + n] = n;
        }
        if (s != PARAREAL_OK) break;
        s = rk4_batch<T>(c, c->n, st, nx, n, n_ics, c->Nf, c->cfg.dt_fine, c->fine_path, c->fine_tx,
                         c->fine_ty, c->fine_zc, w1, w2, w3, 0, c->fine_op);
        if (s != PARAREAL_OK) break;
        for (int i = 0; i < n_ics && s == PARAREAL_OK; ++i)
            s = emit(nx + (size_t)i * P, pf + ((size_t)i * c->N + n) * Pm);
        std::swap(st, nx);
    }
    cudaStreamSynchronize(c->st);
    cleanup();
    return s;
}

extern "C" parareal_status parareal_make_pairs(parareal_ctx *c, const float *ics, int n_ics,
                                               float *pairs_u, float *pairs_f, int *pair_slice)
{
    if (c) c->spec_valid = false;      // U, F or the sweep workspaces may change
    parareal_status s = need_learned(c);
    if (s != PARAREAL_OK) return s;
    if (!ics || n_ics < 1 || !pairs_u || !pairs_f) return fail(c, PARAREAL_E_INVALID, "arguments");
    return c->f64 ? make_pairs_t<double>(c, ics, n_ics, pairs_u, pairs_f, pair_slice)
                  : make_pairs_t<float>(c, ics, n_ics, pairs_u, pairs_f, pair_slice);
}

extern "C" parareal_status parareal_selftest_timeout(void *cuda_stream)
{
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    int *flag = nullptr;
    if (cudaMalloc((void **)&flag, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return fail(nullptr, PARAREAL_E_NOMEM, "self-test flag allocation failed");
    }
    int h = -1;
    cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
    if (e == cudaSuccess) e = launch_wait_selftest(1ll << 18, flag, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, flag, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(flag);
    if (e != cudaSuccess) return fail(nullptr, PARAREAL_E_CUDA, std::string("self-test: ") + cudaGetErrorString(e));
    if (h == 1) return fail(nullptr, PARAREAL_E_TIMEOUT, "bounded wait gave up as designed (self-test)");
    return PARAREAL_OK;
}
