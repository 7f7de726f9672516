"""GPU parity of the phase-kernel evaluation of the LINEAR learned propagator
(learned_eval POLYPHASE) through the C ABI.

With the stencil skip, G(u) = x + K * x with x the stencil propagator's
coarse result prolonged (trilinear) to the fine grid; POLYPHASE folds
(delta + K) and the prolongation into r^3 phase kernels on the coarse grid
and applies them to the change of G's coarse output inside the correction.
It is the operator of the COMPOSED evaluation, computed in another order.

Tolerances: G's output against the FP64 oracle network (applied to the FP64
oracle stencil propagator) at the FP32 stencil tolerance 1e-5 relative L2;
its network part (G - x) at 5e-5 (FP32 rounding of the folded weights and of
the 64-216 term sums, relative to a network part 10-100 times smaller than
x).  Parareal iterates against the oracle's Parareal with the same G at
1e-5.
"""
import numpy as np
import pytest

from oracle import net
from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, rel_l2
from tests.test_gpu_composed import from_master, linear_cfg, nu_hat, oracle_G_stencil, to_master

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NET_TOL = 5e-5


def oracle_learned_G(cfg, params):
    Gs = oracle_G_stencil(cfg)

    def G(x, s):
        out, _ = net.forward(Gs(x, s), nu_hat(cfg, s), params, (0, 0, 0), linear=True)
        return out
    return G


@pytest.mark.parametrize("n,r", [(32, 2), (32, 4), (64, 4), (64, 8)])
def test_polyphase_G_matches_oracle_and_composed(n, r):
    N = 3
    cfgs = {e: linear_cfg(n, N, native.SKIP_STENCIL, e, r)
            for e in (native.EVAL_POLYPHASE, native.EVAL_COMPOSED)}
    ctxs = {e: native.Parareal(c) for e, c in cfgs.items()}
    w = to_master(net.init_params(seed=23, scale=0.12))
    for c in ctxs.values():
        c.set_coarse_model(w)
    params = from_master(w)
    cfg = cfgs[native.EVAL_POLYPHASE]
    us = np.stack([inputs.spectral_ic(n, seed=40 + s, kmax=max(2, n // 4)) for s in range(N)])
    src = torch.from_numpy(us).cuda().contiguous()
    got = {}
    for e, c in ctxs.items():
        dst = torch.empty_like(src)
        c.propagate(1, src, dst, 0, N)
        got[e] = dst.cpu().numpy()
    G = oracle_learned_G(cfg, params)
    Gs = oracle_G_stencil(cfg)
    for s in range(N):
        ref, base = G(us[s], s), Gs(us[s], s)
        assert np.max(np.abs(ref - base)) > 1e-2 * np.max(np.abs(base))
        assert rel_l2(got[native.EVAL_POLYPHASE][s], ref) < TOL[native.F32], s
        e_p = rel_l2(got[native.EVAL_POLYPHASE][s] - base, ref - base)
        assert e_p < NET_TOL, (s, e_p)
        e_c = rel_l2(got[native.EVAL_POLYPHASE][s], got[native.EVAL_COMPOSED][s])
        assert e_c < TOL[native.F32], (s, e_c)
    for c in ctxs.values():
        c.close()


@pytest.mark.parametrize("form", [native.CORRECTION_STANDARD, native.CORRECTION_DIFFERENCE])
def test_polyphase_parareal_matches_oracle(form):
    n, N, r = 32, 4, 4
    cfg = linear_cfg(n, N, native.SKIP_STENCIL, native.EVAL_POLYPHASE, r)
    cfg.correction_form = form
    w = to_master(net.init_params(seed=31, scale=0.08))
    params = from_master(w)
    u0 = inputs.spectral_ic(n, seed=9, kmax=6)
    ctx = native.Parareal(cfg)
    ctx.set_coarse_model(w)
    ctx.set_problem(torch.from_numpy(u0).cuda())
    hist = opr.parareal(oracle_F(cfg), oracle_learned_G(cfg, params), u0, N, 2,
                        form="difference" if form == native.CORRECTION_DIFFERENCE else "standard")
    buf = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    for k in range(3):
        if k:
            assert ctx.iterate(1, 0.0, native.STOP_NONE)[0] == 1
        else:
            ctx.iterate(0, 0.0, native.STOP_NONE)
        for s in range(1, N + 1):
            ctx.get_slice(s, buf)
            e = rel_l2(buf.cpu().numpy(), hist[k][s])
            assert e < TOL[native.F32], (k, s, e)
    ctx.close()


def test_polyphase_reaches_serial_fine_exactly_and_follows_model_changes():
    n, N, r = 32, 4, 2
    cfg = linear_cfg(n, N, native.SKIP_STENCIL, native.EVAL_POLYPHASE, r)
    ctx = native.Parareal(cfg)
    u0 = torch.from_numpy(inputs.spectral_ic(n, seed=8, kmax=6)).cuda()
    # no model: the network is zero and G is the stencil propagator
    src = u0.unsqueeze(0).contiguous()
    a, b = torch.empty_like(src), torch.empty_like(src)
    ctx.propagate(1, src, a, 1, 1)
    Gs = oracle_G_stencil(cfg)(u0.cpu().numpy(), 1)
    assert rel_l2(a[0].cpu().numpy(), Gs) < TOL[native.F32]
    ctx.set_coarse_model(to_master(net.init_params(seed=6, scale=0.05)))
    ctx.propagate(1, src, b, 1, 1)
    assert not torch.equal(a, b)
    ctx.set_problem(u0)
    fine = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(fine, as_reference=True)
    k, h = ctx.iterate(N, 0.0, native.STOP_NONE, device=True)
    assert k == N and h[-1, 2] == 0.0
    last = torch.empty_like(fine)
    ctx.get_slice(N, last)
    assert torch.equal(last, fine)
    ctx.close()


def test_polyphase_configuration_is_checked():
    bad = [lambda c: setattr(c, "learned_skip", native.SKIP_SHIFT),
           lambda c: setattr(c, "coarse_factor", 1),
           lambda c: setattr(c, "coarse_transfer", native.TRANSFER_SPECTRAL),
           lambda c: setattr(c, "learned_act", native.ACT_GELU)]
    for mutate in bad:
        cfg = linear_cfg(32, 2, native.SKIP_STENCIL, native.EVAL_POLYPHASE, 2)
        mutate(cfg)
        with pytest.raises(native.PararealError) as e:
            native.Parareal(cfg)
        assert e.value.status == native.E_INVALID
