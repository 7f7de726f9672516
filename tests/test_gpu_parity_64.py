"""GPU parity at sizes where the launch configuration of the production runs
differs from the small parity cases:

* the learned propagator's tensor-core 16 -> 16 layers at m = 64, where the
  persistent grid (three CTAs per SM) is smaller than the 1024 tiles, so
  every CTA takes a second tile (double-buffered halo, mbarrier phase flip,
  prefetch of the next tile), in both network modes;
* the stencil coarse propagator with coarsening factor 8, the factor of the
  256^3 configuration (here 64^3 -> 8^3);
* one Parareal iteration at 64^3 with the learned propagator as the 128^3
  workload runs it (stencil skip, linear network, composed evaluation,
  difference-form correction), through parareal_iterate, against the
  oracle's serial Parareal (Eq. parareal, standard form: for a linear G the
  two forms are the same iteration).

Tolerances as in the other parity tests: 1e-2 on the network part of a
bfloat16 layer-by-layer G, 1e-5 for FP32 paths without bfloat16 rounding.
"""
import math

import numpy as np
import pytest

from oracle import core, net
from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, oracle_G, oracle_problem, rel_l2, steps, tile_env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

NET_TOL = 1e-2
COMPOSED_TOL = 1e-5


def to_master(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)


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


@pytest.mark.parametrize("act", [native.ACT_GELU, native.ACT_LINEAR])
def test_tensor_core_layers_take_several_tiles_per_cta(act):
    n = 64
    tiles = (n // 8) * (n // 16) * (n // 2)
    assert tiles > 3 * torch.cuda.get_device_properties(0).multi_processor_count
    cfg, _ = configs.small(n=n, n_slices=4, dtype=native.F32, nf=8, nc=2)
    cfg.coarse_kind = native.COARSE_LEARNED
    cfg.learned_act = act
    lin = act == native.ACT_LINEAR
    ctx = native.Parareal(cfg)
    w = to_master(net.init_params(seed=31, scale=0.12))
    ctx.set_coarse_model(w)
    params = from_master(w)
    u = inputs.spectral_ic(n, seed=32, kmax=12)
    src = torch.from_numpy(u).float().cuda().contiguous()
    dst = torch.empty_like(src)
    s = 1
    ctx.propagate(1, src, dst, s, 1)
    got = dst.double().cpu().numpy()
    u32 = u.astype(np.float32).astype(np.float64)
    ref, _ = net.forward(u32, nu_hat(cfg, s), params, shift_of(cfg), bf16_emul=True, linear=lin)
    base = core.shift(u32, shift_of(cfg))
    assert np.max(np.abs(ref - base)) > 1e-2          # the network contributes
    err = rel_l2(got - base, ref - base)
    assert err < NET_TOL, err
    ctx.close()


@pytest.mark.parametrize("dtype", [native.F32, native.F64])
def test_coarse_factor_8_matches_oracle(monkeypatch, dtype):
    tile_env(monkeypatch)
    n, r = 64, 8
    cfg, _ = configs.small(n=n, n_slices=2, dtype=dtype, r=r, nf=8, nc=3)
    assert cfg.coarse_factor == 8
    ctx = native.Parareal(cfg)
    src = np.stack([inputs.spectral_ic(n, seed=40 + s, kmax=4) for s in range(2)])
    dsrc = torch.from_numpy(src).to("cuda", torch.float64 if dtype == native.F64 else torch.float32)
    ddst = torch.empty_like(dsrc)
    ctx.propagate(1, dsrc, ddst, 0, 2)
    got = ddst.double().cpu().numpy()
    G = oracle_G(cfg)
    for s in range(2):
        ref = G(src[s], s)
        assert rel_l2(got[s], ref) < TOL[dtype], (s, rel_l2(got[s], ref))
    ctx.close()


def test_learned_parareal_iteration_at_64_matches_oracle(monkeypatch):
    tile_env(monkeypatch)
    n, N, r = 64, 3, 2
    cfg, _ = configs.small(n=n, n_slices=N, dtype=native.F32, r=r, nf=8, nc=4)
    cfg.coarse_kind = native.COARSE_LEARNED
    cfg.learned_skip = native.SKIP_STENCIL
    cfg.learned_act = native.ACT_LINEAR
    cfg.learned_eval = native.EVAL_COMPOSED
    cfg.correction_form = native.CORRECTION_DIFFERENCE
    ctx = native.Parareal(cfg)
    w = to_master(net.init_params(seed=33, scale=0.05))
    ctx.set_coarse_model(w)
    params = from_master(w)
    u0 = inputs.spectral_ic(n, seed=34, kmax=8)
    ctx.set_problem(torch.from_numpy(u0).cuda())

    _, nc = steps(cfg)
    Gs = opr.coarsened_rk4_propagator(oracle_problem(cfg), r, cfg.dt_coarse, nc)

    def G(u, s):
        # the linear network on the stencil propagator's output, as one 9^3
        # kernel (the oracle's composition of its four layers)
        g = Gs(u, s)
        return g + net.apply_kernel(g, net.compose_linear(params, nu_hat(cfg, s)))

    hist = opr.parareal(oracle_F(cfg), G, u0, N, 1)
    buf = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    for k in range(2):
        if k == 0:
            ctx.iterate(0, 0.0, native.STOP_NONE)       # the coarse start-up only
        else:
            kd, _ = ctx.iterate(1, 0.0, native.STOP_NONE)
            assert kd == 1
        for s in range(1, N + 1):
            ctx.get_slice(s, buf)
            e = rel_l2(buf.cpu().numpy(), hist[k][s])
            assert e < COMPOSED_TOL, (k, s, e)
    ctx.close()
