"""GPU parity of the persistent RK4 path (launch path 3: every step of a
sweep in one cooperative launch, grid barriers between the stages) through
the C ABI.  Per point it performs the per-stage kernels' operations in the
same order, so the two paths agree bitwise; both are checked against the
FP64 oracle (relative L2 1e-12 for FP64, 1e-5 for FP32)."""
import numpy as np
import pytest

from oracle import core
from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, oracle_G, oracle_problem, rel_l2, steps, tile_env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = native.F32, native.F64
STAGED, PERSIST = 1, 3


def read_all(ctx, cfg):
    buf = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    out = []
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, buf)
        out.append(buf.cpu().numpy().copy())
    return out


def run_paths(monkeypatch, cfg, u0, k, device=False):
    res = []
    for path in (STAGED, PERSIST):
        shape = (path, 16, 8, cfg.n)
        tile_env(monkeypatch, fine=shape, coarse=(path, 16, 8, cfg.n // cfg.coarse_factor))
        monkeypatch.setenv("PARAREAL_SERIAL_TILE", ",".join(map(str, shape)))
        ctx = native.Parareal(cfg)
        assert ctx.launch_shape()[0][0] == path
        ctx.set_problem(torch.from_numpy(u0).cuda())
        fine = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
        ctx.serial_fine(fine, as_reference=True)
        kd, h = ctx.iterate(k, 0.0, native.STOP_NONE, device=device and path == PERSIST)
        res.append((read_all(ctx, cfg), fine.cpu().numpy(), h))
        ctx.close()
    return res


@pytest.mark.parametrize("n,dtype,r,N", [(32, F64, 1, 8), (32, F32, 2, 4), (16, F64, 2, 5)])
def test_persistent_path_bitwise_equals_staged(monkeypatch, n, dtype, r, N):
    cfg, u0 = configs.small(n=n, n_slices=N, dtype=dtype, r=r, nf=16, nc=4)
    (a, fa, ha), (b, fb, hb) = run_paths(monkeypatch, cfg, u0, 3)
    assert np.array_equal(fa, fb)
    assert np.array_equal(ha[:, :3], hb[:, :3])
    for s in range(N + 1):
        assert np.array_equal(a[s], b[s]), s
    # and against the oracle: the serial fine run
    ref = u0
    F = oracle_F(cfg)
    for s in range(N):
        ref = F(ref, s)
    assert rel_l2(fb, ref) < TOL[dtype]


def test_persistent_path_fourth_order_operator(monkeypatch):
    """The paper's fourth-order fine operator (radius 2) on the persistent path."""
    cfg, u0 = configs.small(n=16, n_slices=3, dtype=F64, nf=8, nc=2)
    cfg.fine_scheme = native.SCHEME_C4
    (a, fa, _), (b, fb, _) = run_paths(monkeypatch, cfg, u0, 2)
    assert np.array_equal(fa, fb)
    for s in range(cfg.n_slices + 1):
        assert np.array_equal(a[s], b[s]), s
    ref = u0
    F = oracle_F(cfg)
    for s in range(cfg.n_slices):
        ref = F(ref, s)
    assert rel_l2(fb, ref) < TOL[F64]


def test_persistent_path_more_fields_than_one_launch_holds(monkeypatch):
    """70 slices: the batched sweep runs as launches of at most 64 fields."""
    cfg, u0 = configs.small(n=8, n_slices=70, dtype=F64, nf=4, nc=1)
    (a, fa, _), (b, fb, _) = run_paths(monkeypatch, cfg, u0, 1)
    assert np.array_equal(fa, fb)
    for s in range(cfg.n_slices + 1):
        assert np.array_equal(a[s], b[s]), s


def test_persistent_path_inside_the_device_loop(monkeypatch):
    """Cooperative launches inside the conditional graph of
    parareal_iterate_device: the same iterates as the staged host loop."""
    cfg, u0 = configs.small(n=32, n_slices=6, dtype=F64, nf=16, nc=4)
    (a, fa, ha), (b, fb, hb) = run_paths(monkeypatch, cfg, u0, 4, device=True)
    assert np.array_equal(ha[:, :3], hb[:, :3])
    for s in range(cfg.n_slices + 1):
        assert np.array_equal(a[s], b[s]), s


def test_default_fp64_small_grid_uses_the_persistent_path(monkeypatch):
    tile_env(monkeypatch)
    monkeypatch.delenv("PARAREAL_SERIAL_TILE", raising=False)
    cfg, u0 = configs.plain_fp64_32()
    ctx = native.Parareal(cfg)
    f4, c4, s4 = ctx.launch_shape()
    assert f4[0] == c4[0] == s4[0] == PERSIST
    ctx.close()
