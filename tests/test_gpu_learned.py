"""GPU parity of the learned coarse propagator (forward, gradients, Adam,
pair generation) against the FP64 oracle, and what training buys Parareal.

Tolerances: the oracle rounds to bfloat16 at the same points as the GPU
(weights, network input, activations, pre-activation gradients), so the two
differ only where FP32 and FP64 accumulation put a value on different sides
of a bfloat16 rounding boundary (one bf16 ulp = 2^-8 relative on those
elements).  Relative L2 of the network output and of each layer's gradient is
therefore held to 1e-2; FP32-only arithmetic (Adam, pairs) to 1e-5 / 1e-6.
"""
import math

import numpy as np
import pytest

from oracle import core, net
from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import oracle_F, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NET_TOL = 1e-2


def learned_cfg(n=16, N=4, kind=native.COARSE_LEARNED, r=1):
    base, _ = configs.small(n=n, n_slices=N, dtype=native.F32, nf=8, nc=2)
    base.coarse_kind = kind
    base.coarse_factor = r
    return base


def to_master(params):
    flat = []
    for W, b in params:
        flat.append(W.ravel())
        flat.append(b.ravel())
    out = np.concatenate(flat).astype(np.float32)
    assert out.size == native.MODEL_PARAMS
    return out


def from_master(v):
    params, off = [], 0
    for ci, co in net.LAYERS:
        W = v[off:off + co * ci * 27].reshape(co, ci, 3, 3, 3).astype(np.float64)
        off += co * ci * 27
        b = v[off:off + co].astype(np.float64)
        off += co
        params.append([W, b])
    return params


def shift_of(cfg):
    m = cfg.n // cfg.coarse_factor
    return tuple(int(round(a * cfg.T / cfg.n_slices * m)) % m for a in cfg.a)


def nu_hat(cfg, s):
    t = s * cfg.T / cfg.n_slices
    return float(np.float32((1 + cfg.nu_amp * math.sin(cfg.nu_omega * t))))


def test_forward_matches_oracle():
    cfg = learned_cfg()
    ctx = native.Parareal(cfg)
    params = net.init_params(seed=3, scale=0.15)
    w = to_master(params)
    ctx.set_coarse_model(w)
    params = from_master(w)           # the FP32 values the GPU holds
    u = inputs.spectral_ic(16, seed=5, kmax=4)
    src = torch.from_numpy(u).float().cuda().contiguous()
    dst = torch.empty_like(src)
    s = 2
    ctx.propagate(1, src, dst, s, 1)
    got = dst.double().cpu().numpy()
    u32 = u.astype(np.float32).astype(np.float64)
    ref, _ = net.forward(u32, nu_hat(cfg, s), params, shift_of(cfg), bf16_emul=True)
    su = core.shift(u32, shift_of(cfg))
    assert np.max(np.abs(ref - su)) > 1e-2          # the net contributes
    err = rel_l2(got - su, ref - su)
    assert err < NET_TOL, err
    ctx.close()


def test_shift_only_propagator_is_the_exact_shift():
    cfg = learned_cfg(kind=native.COARSE_SHIFT)
    ctx = native.Parareal(cfg)
    u = inputs.spectral_ic(16, seed=6, kmax=4)
    src = torch.from_numpy(u).cuda().contiguous()
    dst = torch.empty_like(src)
    ctx.propagate(1, src, dst, 1, 1)
    assert np.array_equal(dst.cpu().numpy(), core.shift(u, shift_of(cfg)))
    ctx.close()


def test_gradients_match_oracle():
    cfg = learned_cfg()
    ctx = native.Parareal(cfg)
    params = net.init_params(seed=4, scale=0.15)
    w = to_master(params)
    ctx.set_coarse_model(w)
    params = from_master(w)
    us = [inputs.spectral_ic(16, seed=10 + i, kmax=4) for i in range(2)]
    tg = [core.shift(x, shift_of(cfg)) * 0.9 + 0.05 * inputs.spectral_ic(16, seed=20 + i, kmax=6)
          for i, x in enumerate(us)]
    us32 = [x.astype(np.float32) for x in us]
    tg32 = [x.astype(np.float32) for x in tg]
    slices = [1, 3]
    U = torch.from_numpy(np.stack(us32)).cuda()
    Tg = torch.from_numpy(np.stack(tg32)).cuda()
    g = torch.empty(native.MODEL_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctx.coarse_model_grad(U, Tg, slices, g)
    ref_loss, ref_g = net.loss_and_grads([x.astype(np.float64) for x in us32],
                                         [nu_hat(cfg, s) for s in slices],
                                         [x.astype(np.float64) for x in tg32], params,
                                         shift_of(cfg), bf16_emul=True)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss, (loss, ref_loss)
    got = from_master(g.cpu().numpy())
    for li in range(4):
        for k in range(2):
            e = rel_l2(got[li][k], ref_g[li][k])
            assert e < 2 * NET_TOL, (li, k, e)
    ctx.close()


def test_adam_step_is_the_textbook_update_of_the_gpu_gradient():
    cfg = learned_cfg()
    ctx = native.Parareal(cfg)
    w0 = to_master(net.init_params(seed=7, scale=0.1))
    ctx.set_coarse_model(w0)
    u = np.stack([inputs.spectral_ic(16, seed=30, kmax=4)]).astype(np.float32)
    f = np.stack([inputs.spectral_ic(16, seed=31, kmax=4)]).astype(np.float32)
    U, Fd = torch.from_numpy(u).cuda(), torch.from_numpy(f).cuda()
    g = torch.empty(native.MODEL_PARAMS, dtype=torch.float32, device="cuda")
    ctx.coarse_model_grad(U, Fd, [2], g)
    grad = g.cpu().numpy().astype(np.float64)
    ctx.train_coarse(U, Fd, [2], epochs=1, batch=1, lr=1e-3, eps=1e-8)
    w1 = ctx.get_coarse_model().astype(np.float64)
    p = [[w0.astype(np.float64).copy(), np.zeros(1)]]
    m = net.zeros_like_params(p)
    v = net.zeros_like_params(p)
    net.adam_step(p, [[grad, np.zeros(1)]], m, v, 1, lr=1e-3, eps=1e-8)
    assert np.max(np.abs(w1 - p[0][0])) <= 1e-6 * max(1.0, np.max(np.abs(w0)))
    ctx.close()


def test_pairs_follow_the_fine_trajectories():
    cfg = learned_cfg(n=16, N=3)
    ctx = native.Parareal(cfg)
    ics = np.stack([inputs.spectral_ic(16, seed=40 + i, kmax=4) for i in range(2)]).astype(np.float32)
    pu = torch.empty((6, 16, 16, 16), dtype=torch.float32, device="cuda")
    pf = torch.empty_like(pu)
    sl = ctx.make_pairs(torch.from_numpy(ics).cuda(), pu, pf)
    assert list(sl) == [0, 1, 2, 0, 1, 2]
    F = oracle_F(cfg)
    for i in range(2):
        x = ics[i].astype(np.float64)
        for n in range(3):
            assert rel_l2(pu[i * 3 + n].double().cpu().numpy(), x) < 1e-5
            x = F(x, n)
            assert rel_l2(pf[i * 3 + n].double().cpu().numpy(), x) < 1e-5
    ctx.close()


def test_training_reduces_parareal_iterations():
    """The trained net beats the untrained one (G = S) as Parareal's coarse
    propagator: fewer iterations to the same defect."""
    n, N = 32, 8
    nu_max = 0.015
    m = max(6, math.ceil(math.log2(12.0 * nu_max * n * n / 1.5)))
    dt = 2.0 ** -m
    T = 1.0
    nf = round(T / N / dt)
    def make(kind):
        c = native.Config.make(n, N, T, dt, T / N, 1, fine_dtype=native.F32, coarse_kind=kind,
                               nu0=0.01, nu_amp=0.5, nu_omega=2 * math.pi)
        return c
    ctx = native.Parareal(make(native.COARSE_LEARNED))
    # broadband training fields: the k^-2 spectrum up to Nyquist plus white
    # noise, so the net also learns how F damps the highest modes (a net that
    # never saw them may amplify them, and Parareal then diverges)
    ics = np.stack([inputs.spectral_ic(n, seed=100 + i, kmax=n // 2 - 1)
                    + 0.2 * inputs.random_field(n, seed=200 + i) for i in range(16)]).astype(np.float32)
    pu = torch.empty((16 * N, n, n, n), dtype=torch.float32, device="cuda")
    pf = torch.empty_like(pu)
    sl = ctx.make_pairs(torch.from_numpy(ics).cuda(), pu, pf)
    ctx.set_coarse_model(inputs.initial_weights(seed=0))
    hist = ctx.train_coarse(pu, pf, sl, epochs=40, batch=8, lr=2e-3, seed=1)
    assert hist[-1] < 0.5 * hist[0], hist
    u0 = torch.from_numpy(inputs.spectral_ic(n, seed=7, kmax=6)).cuda()

    def iterations(c):
        c.set_problem(u0)
        c.serial_fine(None, as_reference=True)
        k, h = c.iterate(N, 1e-6, native.STOP_DEFECT)
        return k, h[:, 2]

    k_learned, d_learned = iterations(ctx)
    shift_ctx = native.Parareal(make(native.COARSE_SHIFT))
    k_shift, d_shift = iterations(shift_ctx)
    # both reach the fine solution (at k = N at the latest: Eq. parareal is exact there)
    assert d_learned[-1] <= 1e-6 and d_shift[-1] <= 1e-6
    assert k_learned <= k_shift
    # what the net buys over the same propagator without it (G = S): a far
    # smaller defect at every iteration before the exact one
    for k in range(min(len(d_learned), len(d_shift)) - 1):
        assert d_learned[k] < 0.1 * d_shift[k], (k, d_learned, d_shift)
    assert d_learned[0] < 0.1, d_learned
    ctx.close()
    shift_ctx.close()


def test_stencil_skip_forward_matches_oracle():
    """G(u) = Gs(u) + Net([Gs(u), nu/nu0]) with Gs the coarsened stencil propagator."""
    base, _ = configs.small(n=32, n_slices=4, dtype=native.F32, r=2, nf=8, nc=4)
    base.coarse_kind = native.COARSE_LEARNED
    base.learned_skip = native.SKIP_STENCIL
    ctx = native.Parareal(base)
    params = net.init_params(seed=5, scale=0.15)
    w = to_master(params)
    ctx.set_coarse_model(w)
    params = from_master(w)
    u = inputs.spectral_ic(32, seed=9, kmax=6)
    src = torch.from_numpy(u).cuda().contiguous()
    dst = torch.empty_like(src)
    s = 1
    ctx.propagate(1, src, dst, s, 1)
    got = dst.cpu().numpy()
    gs = oracle_G_stencil(base)(u, s)
    ref, _ = net.forward(gs, nu_hat(base, s), params, (0, 0, 0), bf16_emul=True)
    assert np.max(np.abs(ref - gs)) > 1e-2
    err = rel_l2(got - gs, ref - gs)
    assert err < NET_TOL, err
    ctx.close()


def oracle_G_stencil(cfg):
    from tests.helpers import steps, oracle_problem
    _, nc = steps(cfg)
    return opr.coarsened_rk4_propagator(oracle_problem(cfg), cfg.coarse_factor, cfg.dt_coarse, nc)


def test_stencil_skip_training_improves_the_early_iterates():
    """The net trained on F - Gs improves the one-slice prediction of the stencil
    propagator Gs: the start-up chain and the first Parareal iterates have a
    defect several times smaller than with Gs alone.  Later iterates are not
    asserted: the net is nonlinear, the correction G(U^{k+1}) - G(U^k) sees its
    Jacobian, which training does not fit, and the defect levels off near 2e-3
    while Gs keeps contracting.  k = N is exact for every G (Eq. parareal)."""
    n, N = 32, 8
    m = max(6, math.ceil(math.log2(12.0 * 0.015 * n * n / 1.5)))
    dt = 2.0 ** -m
    T = 1.0

    def make(kind):
        return native.Config.make(n, N, T, dt, T / N / 4, 2, fine_dtype=native.F32,
                                  coarse_kind=kind, learned_skip=native.SKIP_STENCIL,
                                  nu0=0.01, nu_amp=0.5, nu_omega=2 * math.pi)
    ctx = native.Parareal(make(native.COARSE_LEARNED))
    ics = np.stack([inputs.spectral_ic(n, seed=100 + i, kmax=n // 2 - 1)
                    + 0.2 * inputs.random_field(n, seed=200 + i) for i in range(16)]).astype(np.float32)
    pu = torch.empty((16 * N, n, n, n), dtype=torch.float32, device="cuda")
    pf = torch.empty_like(pu)
    sl = ctx.make_pairs(torch.from_numpy(ics).cuda(), pu, pf)
    w0 = inputs.initial_weights(seed=0)
    ctx.set_coarse_model(w0)
    hist = ctx.train_coarse(pu, pf, sl, epochs=40, batch=8, lr=2e-3, seed=1)
    assert hist[-1] < 0.2 * hist[0], hist
    u0 = torch.from_numpy(inputs.spectral_ic(n, seed=7, kmax=6)).cuda()

    def iterations(c):
        c.set_problem(u0)
        c.serial_fine(None, as_reference=True)
        k, h = c.iterate(N, 0.0, native.STOP_NONE)
        return k, h[:, 2]

    k_learned, d_learned = iterations(ctx)
    st = native.Parareal(make(native.COARSE_STENCIL))
    k_st, d_st = iterations(st)
    assert k_learned == k_st == N
    assert d_learned[-1] == 0.0 and d_st[-1] == 0.0
    for k in range(3):
        assert d_learned[k] < 0.5 * d_st[k], (k, d_learned, d_st)
    assert np.all(np.isfinite(d_learned)) and np.max(d_learned) < 1.0
    ctx.close()
    st.close()


# ------------------------------------------------- linear learned propagator

@pytest.mark.parametrize("skip", [native.SKIP_SHIFT, native.SKIP_STENCIL])
def test_linear_forward_matches_oracle(skip):
    base, _ = configs.small(n=16, n_slices=4, dtype=native.F32, r=2, nf=8, nc=4)
    base.coarse_kind = native.COARSE_LEARNED
    base.learned_skip = skip
    base.learned_act = native.ACT_LINEAR
    if skip == native.SKIP_SHIFT:
        base.coarse_factor = 1
    ctx = native.Parareal(base)
    params = net.init_params(seed=8, scale=0.15)
    for W, b in params:
        b += 0.25                      # ignored in linear mode
    w = to_master(params)
    ctx.set_coarse_model(w)
    params = from_master(w)
    u = inputs.spectral_ic(16, seed=12, kmax=4)
    src = torch.from_numpy(u).cuda().contiguous()
    dst = torch.empty_like(src)
    s = 3
    ctx.propagate(1, src, dst, s, 1)
    got = dst.cpu().numpy()
    if skip == native.SKIP_STENCIL:
        sk, shift = oracle_G_stencil(base)(u, s), (0, 0, 0)
    else:
        sk, shift = u, shift_of(base)
    ref, _ = net.forward(sk, nu_hat(base, s), params, shift, bf16_emul=True, linear=True)
    base_out = core.shift(sk, shift)
    assert np.max(np.abs(ref - base_out)) > 1e-2
    err = rel_l2(got - base_out, ref - base_out)
    assert err < NET_TOL, err
    # linear: G(2u) = 2 G(u) up to the bf16 rounding of the network input
    ctx.propagate(1, 2 * src, dst, s, 1)
    assert rel_l2(dst.cpu().numpy() - 2 * base_out, 2 * (got - base_out)) < NET_TOL
    ctx.close()


def test_linear_gradients_match_oracle():
    cfg = learned_cfg()
    cfg.learned_act = native.ACT_LINEAR
    ctx = native.Parareal(cfg)
    params = net.init_params(seed=9, scale=0.15)
    w = to_master(params)
    ctx.set_coarse_model(w)
    params = from_master(w)
    us = [inputs.spectral_ic(16, seed=40 + i, kmax=4) for i in range(2)]
    tg = [core.shift(x, shift_of(cfg)) * 0.9 + 0.05 * inputs.spectral_ic(16, seed=50 + i, kmax=6)
          for i, x in enumerate(us)]
    us32 = [x.astype(np.float32) for x in us]
    tg32 = [x.astype(np.float32) for x in tg]
    slices = [0, 2]
    U = torch.from_numpy(np.stack(us32)).cuda()
    Tg = torch.from_numpy(np.stack(tg32)).cuda()
    g = torch.empty(native.MODEL_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctx.coarse_model_grad(U, Tg, slices, g)
    ref_loss, ref_g = net.loss_and_grads([x.astype(np.float64) for x in us32],
                                         [nu_hat(cfg, s) for s in slices],
                                         [x.astype(np.float64) for x in tg32], params,
                                         shift_of(cfg), bf16_emul=True, linear=True)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss, (loss, ref_loss)
    got = from_master(g.cpu().numpy())
    for li in range(4):
        e = rel_l2(got[li][0], ref_g[li][0])
        assert e < 2 * NET_TOL, (li, e)
        assert not np.any(got[li][1])          # no biases in linear mode
    ctx.close()


def test_difference_form_needs_a_linear_propagator():
    cfg = learned_cfg()
    cfg.correction_form = native.CORRECTION_DIFFERENCE
    with pytest.raises(native.PararealError):
        native.Parareal(cfg)
    cfg.learned_act = native.ACT_LINEAR
    native.Parareal(cfg).close()


def _linear_pair_cfg(kind, form):
    n, N = 32, 8
    m = max(6, math.ceil(math.log2(12.0 * 0.015 * n * n / 1.5)))
    dt = 2.0 ** -m
    return native.Config.make(n, N, 1.0, dt, 1.0 / N / 4, 2, fine_dtype=native.F32,
                              coarse_kind=kind, learned_skip=native.SKIP_STENCIL,
                              learned_act=native.ACT_LINEAR, correction_form=form,
                              nu0=0.01, nu_amp=0.5, nu_omega=2 * math.pi)


def test_linear_learned_propagator_beats_the_stencil_propagator():
    """The linear learned G (stencil skip, nu as a factor) trained on F - Gs,
    with the correction applied to U^{k+1}[n] - U^k[n]: a smaller defect than
    the stencil G at every iteration before k = N.  (With the standard form
    the bf16 rounding of the network input puts a floor under the defect.)"""
    N = 8
    ctx = native.Parareal(_linear_pair_cfg(native.COARSE_LEARNED, native.CORRECTION_DIFFERENCE))
    n = 32
    ics = np.stack([inputs.spectral_ic(n, seed=100 + i, kmax=n // 2 - 1)
                    + 0.2 * inputs.random_field(n, seed=200 + i) for i in range(16)]).astype(np.float32)
    pu = torch.empty((16 * N, n, n, n), dtype=torch.float32, device="cuda")
    pf = torch.empty_like(pu)
    sl = ctx.make_pairs(torch.from_numpy(ics).cuda(), pu, pf)
    ctx.set_coarse_model(inputs.initial_weights(seed=0))
    hist = ctx.train_coarse(pu, pf, sl, epochs=40, batch=8, lr=2e-3, seed=1)
    assert hist[-1] < 0.2 * hist[0], hist
    u0 = torch.from_numpy(inputs.spectral_ic(n, seed=7, kmax=6)).cuda()

    def defects(c):
        c.set_problem(u0)
        c.serial_fine(None, as_reference=True)
        k, h = c.iterate(N, 0.0, native.STOP_NONE)
        return h[:, 2]

    d_lin = defects(ctx)
    st = native.Parareal(_linear_pair_cfg(native.COARSE_STENCIL, native.CORRECTION_STANDARD))
    d_st = defects(st)
    assert d_lin[-1] == 0.0 and d_st[-1] == 0.0
    for k in range(N - 1):
        assert d_lin[k] < d_st[k], (k, d_lin, d_st)
    ctx.close()
    st.close()
