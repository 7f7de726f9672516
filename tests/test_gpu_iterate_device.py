"""parareal_iterate_device -- the iterations as one CUDA graph launch with the
stopping test on the device -- against parareal_iterate (one host round
trip per iteration) through the C ABI: the iterates, the iteration counts and
the norms must be the same bit for bit, for every stopping rule, both
correction forms, FP32 and FP64, the learned and the spectral coarse
propagators, and for solves split across calls of either kind."""
import numpy as np
import pytest

from oracle import net
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import tile_env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = native.F32, native.F64


def read_all(ctx, cfg):
    buf = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    out = []
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, buf)
        out.append(buf.cpu().numpy().copy())
    return out


def twin(cfg, u0, model=None, reference=True):
    ctxs = []
    for _ in range(2):
        c = native.Parareal(cfg)
        if model is not None:
            c.set_coarse_model(model)
        c.set_problem(torch.from_numpy(u0).cuda())
        if reference:
            c.serial_fine(None, as_reference=True)
        ctxs.append(c)
    return ctxs


def same_state(a, b, cfg):
    for s, (x, y) in enumerate(zip(read_all(a, cfg), read_all(b, cfg))):
        assert np.array_equal(x, y), s
    for kind in (native.RES_DIFF_INF, native.RES_DIFF_L2, native.RES_DEFECT):
        assert np.array_equal(a.residual(kind), b.residual(kind)), kind


CASES = [
    ("f32_r2_standard", dict(n=32, n_slices=5, dtype=F32, r=2, nf=8, nc=2), native.CORRECTION_STANDARD),
    ("f32_r2_difference", dict(n=32, n_slices=6, dtype=F32, r=2, nf=8, nc=2), native.CORRECTION_DIFFERENCE),
    ("f64_same_grid", dict(n=16, n_slices=4, dtype=F64, r=1, nf=8, nc=2), native.CORRECTION_STANDARD),
]


@pytest.mark.parametrize("name,kw,form", CASES)
def test_device_loop_equals_host_loop_bitwise(monkeypatch, name, kw, form):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(**kw)
    cfg.correction_form = form
    host, dev = twin(cfg, u0)
    N = cfg.n_slices
    # in two calls each: 2 iterations, then the rest
    for k in (2, N - 2):
        kh, hh = host.iterate(k, 0.0, native.STOP_NONE)
        kd, hd = dev.iterate(k, 0.0, native.STOP_NONE, device=True)
        assert kh == kd == k
        assert np.array_equal(hh[:, :3], hd[:, :3])
        same_state(host, dev, cfg)
    assert hd[-1, 2] == 0.0          # k = N: the serial fine solution, exactly
    host.close()
    dev.close()


@pytest.mark.parametrize("rule,tol", [(native.STOP_DEFECT, 1e-4), (native.STOP_DIFF, 1e-3)])
def test_device_stopping_rules(monkeypatch, rule, tol):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=8, dtype=F32, r=2, nf=16, nc=2)
    cfg.correction_form = native.CORRECTION_DIFFERENCE
    host, dev = twin(cfg, u0)
    kh, hh = host.iterate(8, tol, rule)
    kd, hd = dev.iterate(8, tol, rule, device=True)
    assert kh == kd >= 1
    assert np.array_equal(hh[:, :3], hd[:, :3])
    assert np.all(np.diff(hd[:, 3]) >= 0.0) and hd[0, 3] > 0.0     # device times, increasing
    same_state(host, dev, cfg)
    # a new problem on the same context reuses the graph
    for c in (host, dev):
        c.set_problem(torch.from_numpy(u0 * 0.5).cuda())
        c.serial_fine(None, as_reference=True)
    kh, hh = host.iterate(8, tol, rule)
    kd, hd = dev.iterate(8, tol, rule, device=True)
    assert kh == kd and np.array_equal(hh[:, :3], hd[:, :3])
    same_state(host, dev, cfg)
    host.close()
    dev.close()


def test_mixed_host_and_device_calls(monkeypatch):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=6, dtype=F32, r=2, nf=8, nc=2)
    host, mixed = twin(cfg, u0)
    host.iterate(5, 0.0, native.STOP_NONE)
    mixed.iterate(1, 0.0, native.STOP_NONE)
    mixed.iterate(2, 0.0, native.STOP_NONE, device=True)
    mixed.iterate(1, 0.0, native.STOP_NONE)
    mixed.iterate(1, 0.0, native.STOP_NONE, device=True)
    same_state(host, mixed, cfg)
    host.close()
    mixed.close()


def test_device_loop_learned_and_spectral(monkeypatch):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=5, dtype=F32, r=2, nf=8, nc=4)
    cfg.coarse_kind = native.COARSE_LEARNED
    cfg.learned_skip = native.SKIP_STENCIL
    cfg.learned_act = native.ACT_LINEAR
    cfg.learned_eval = native.EVAL_COMPOSED
    cfg.correction_form = native.CORRECTION_DIFFERENCE
    params = net.init_params(seed=41, scale=0.05)
    w = np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)
    host, dev = twin(cfg, u0, model=w)
    assert host.iterate(4, 0.0, native.STOP_NONE)[0] == dev.iterate(4, 0.0, native.STOP_NONE, device=True)[0]
    same_state(host, dev, cfg)
    # another model on the same contexts: the graph reads the new weights
    w2 = (w * 0.5).astype(np.float32)
    for c in (host, dev):
        c.set_coarse_model(w2)
        c.set_problem(torch.from_numpy(u0).cuda())
    host.iterate(3, 0.0, native.STOP_NONE)
    dev.iterate(3, 0.0, native.STOP_NONE, device=True)
    same_state(host, dev, cfg)
    host.close()
    dev.close()

    cfg, u0 = configs.small(n=32, n_slices=4, dtype=F32, r=4, nf=8, nc=2)
    cfg.coarse_transfer = native.TRANSFER_SPECTRAL
    host, dev = twin(cfg, u0)
    host.iterate(4, 0.0, native.STOP_NONE)
    dev.iterate(4, 0.0, native.STOP_NONE, device=True)
    same_state(host, dev, cfg)
    host.close()
    dev.close()


def test_device_loop_reports_divergence_and_stays_usable():
    cfg, u0 = configs.small(n=16, n_slices=2, dtype=F64)
    ctx = native.Parareal(cfg)
    bad = u0.copy()
    bad[3, 2, 1] = np.nan
    ctx.set_problem(torch.from_numpy(bad).cuda())
    with pytest.raises(native.PararealError) as e:
        ctx.iterate(2, 0.0, native.STOP_NONE, device=True)
    assert e.value.status == native.E_DIVERGED
    ctx.set_problem(torch.from_numpy(u0).cuda())
    kd, _ = ctx.iterate(2, 0.0, native.STOP_NONE, device=True)
    assert kd == 2
    ctx.close()
