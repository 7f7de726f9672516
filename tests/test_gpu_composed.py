"""GPU parity of the composed evaluation of the LINEAR learned propagator
(learned_eval COMPOSED: the four linear layers as one 9^3 cross-correlation
per slice) through the C ABI.

Tolerances: the composed path has no bfloat16 rounding (FP64 composition of
the FP32 master weights, FP32 application), so its network part is held to
1e-5 relative L2 against the FP64 oracle network evaluated layer by layer
without rounding; against the GPU's own layer-by-layer path (bfloat16
weights and activations) to the learned-propagator tolerance 1e-2.
"""
import math

import numpy as np
import pytest

from oracle import core, net
from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import oracle_problem, rel_l2, steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

COMPOSED_TOL = 1e-5
LAYERS_TOL = 1e-2


def to_master(params):
    flat = []
    for W, b in params:
        flat.append(W.ravel())
        flat.append(b.ravel())
    return np.concatenate(flat).astype(np.float32)


def from_master(v):
    params, off = [], 0
    for ci, co in net.LAYERS:
        W = v[off:off + co * ci * 27].reshape(co, ci, 3, 3, 3).astype(np.float64)
        off += co * ci * 27
        b = v[off:off + co].astype(np.float64)
        off += co
        params.append([W, b])
    return params


def nu_hat(cfg, s):
    t = s * cfg.T / cfg.n_slices
    return float(np.float32(1 + cfg.nu_amp * math.sin(cfg.nu_omega * t)))


def shift_of(cfg):
    m = cfg.n // cfg.coarse_factor
    sl = cfg.T / cfg.n_slices
    return tuple(int(round(cfg.a[d] * sl * m)) % m for d in range(3))


def linear_cfg(n, N, skip, evaluation, r=1):
    base, _ = configs.small(n=n, n_slices=N, dtype=native.F32, r=max(r, 1), nf=8, nc=4)
    base.coarse_kind = native.COARSE_LEARNED
    base.learned_skip = skip
    base.learned_act = native.ACT_LINEAR
    base.learned_eval = evaluation
    base.coarse_factor = r
    return base


def oracle_G_stencil(cfg):
    _, nc = steps(cfg)
    return opr.coarsened_rk4_propagator(oracle_problem(cfg), cfg.coarse_factor, cfg.dt_coarse, nc)


def test_composed_eval_needs_the_linear_network():
    cfg = linear_cfg(16, 2, native.SKIP_SHIFT, native.EVAL_COMPOSED)
    cfg.learned_act = native.ACT_GELU
    with pytest.raises(native.PararealError):
        native.Parareal(cfg)


@pytest.mark.parametrize("skip,n,r", [(native.SKIP_SHIFT, 16, 1), (native.SKIP_SHIFT, 48, 1),
                                      (native.SKIP_STENCIL, 32, 2)])
def test_composed_forward_matches_oracle(skip, n, r):
    """Every slice's G against the oracle network (FP64, no rounding), and
    against the GPU's layer-by-layer evaluation of the same weights."""
    N = 3
    cfgs = {e: linear_cfg(n, N, skip, e, r) for e in (native.EVAL_COMPOSED, native.EVAL_LAYERS)}
    ctxs = {e: native.Parareal(c) for e, c in cfgs.items()}
    params = net.init_params(seed=21, scale=0.15)
    w = to_master(params)
    for c in ctxs.values():
        c.set_coarse_model(w)
    params = from_master(w)
    cfg = cfgs[native.EVAL_COMPOSED]
    us = np.stack([inputs.spectral_ic(n, seed=70 + s, kmax=max(2, n // 4)) for s in range(N)])
    src = torch.from_numpy(us).cuda().contiguous()
    got = {}
    for e, c in ctxs.items():
        dst = torch.empty_like(src)
        c.propagate(1, src, dst, 0, N)
        got[e] = dst.cpu().numpy()
    for s in range(N):
        if skip == native.SKIP_STENCIL:
            sk, shift = oracle_G_stencil(cfg)(us[s], s), (0, 0, 0)
        else:
            sk, shift = us[s], shift_of(cfg)
        ref, _ = net.forward(sk, nu_hat(cfg, s), params, shift, linear=True)
        base = core.shift(sk, shift)
        assert np.max(np.abs(ref - base)) > 1e-2
        e_c = rel_l2(got[native.EVAL_COMPOSED][s] - base, ref - base)
        assert e_c < COMPOSED_TOL, (s, e_c)
        e_l = rel_l2(got[native.EVAL_COMPOSED][s] - base, got[native.EVAL_LAYERS][s] - base)
        assert e_l < LAYERS_TOL, (s, e_l)
    for c in ctxs.values():
        c.close()


def test_composed_eval_follows_model_changes():
    """The per-slice kernels are rebuilt when the model changes: a zero model
    gives G = S exactly, a new model the oracle's G."""
    n, N = 16, 2
    cfg = linear_cfg(n, N, native.SKIP_SHIFT, native.EVAL_COMPOSED)
    ctx = native.Parareal(cfg)
    u = inputs.spectral_ic(n, seed=3, kmax=4)
    src = torch.from_numpy(u).cuda().contiguous()
    dst = torch.empty_like(src)
    ctx.propagate(1, src, dst, 1, 1)
    assert np.array_equal(dst.cpu().numpy(), core.shift(u, shift_of(cfg)))
    params = net.init_params(seed=4, scale=0.2)
    w = to_master(params)
    ctx.set_coarse_model(w)
    ctx.propagate(1, src, dst, 1, 1)
    ref, _ = net.forward(u, nu_hat(cfg, 1), from_master(w), shift_of(cfg), linear=True)
    base = core.shift(u, shift_of(cfg))
    assert rel_l2(dst.cpu().numpy() - base, ref - base) < COMPOSED_TOL
    ctx.close()


def test_composed_parareal_reaches_serial_fine_exactly():
    """Eq. (parareal) with the composed G: the iterate equals the serial fine
    solution bitwise at k = N (standard form)."""
    n, N = 32, 4
    cfg = linear_cfg(n, N, native.SKIP_STENCIL, native.EVAL_COMPOSED, r=2)
    ctx = native.Parareal(cfg)
    ctx.set_coarse_model(to_master(net.init_params(seed=6, scale=0.05)))
    u0 = torch.from_numpy(inputs.spectral_ic(n, seed=8, kmax=6)).cuda()
    ctx.set_problem(u0)
    fine = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(fine, as_reference=True)
    k, h = ctx.iterate(N, 0.0, native.STOP_NONE)
    assert k == N and h[-1, 2] == 0.0
    last = torch.empty_like(fine)
    ctx.get_slice(N, last)
    assert torch.equal(last, fine)
    ctx.close()
