"""GPU parity of the fused RK4 kernel with two region rows per thread
(launch path 2) through the C ABI.

Per point the two-row kernel performs the same FP32 operations in the same
order as the one-row kernel (same weights, the seven stencil terms summed
in the same order, the same step formula), so the two agree bitwise; both
are checked against the FP64 oracle at the FP32 tolerance (relative L2
1e-5).
"""
import numpy as np
import pytest

from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, oracle_G, rel_l2, tile_env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32 = native.F32
ROWS2 = 2


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", torch.float64)


def read_all(ctx, cfg):
    out = []
    buf = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, buf)
        out.append(buf.cpu().numpy().copy())
    return out


# (n, slices, fine launch shape "path,tile_x,tile_y,zchunk")
ROWS2_CASES = [
    (64, 3, (ROWS2, 64, 32, 64)),   # the large-grid shape, 1 x 2 tiles
    (64, 4, (ROWS2, 64, 16, 24)),   # ragged z chunks 24 + 24 + 16
    (32, 3, (ROWS2, 32, 32, 8)),    # region wider than the grid (the halo wraps), four z chunks
    (32, 5, (ROWS2, 32, 16, 32)),   # two CTAs per SM
]


@pytest.mark.parametrize("n,N,shape", ROWS2_CASES)
def test_two_row_sweep_iterates_match_oracle(monkeypatch, n, N, shape):
    tile_env(monkeypatch, fine=shape)
    cfg, u0 = configs.small(n=n, n_slices=N, dtype=F32, r=2, nf=8, nc=2)
    ctx = native.Parareal(cfg)
    assert ctx.launch_shape()[0] == shape
    ctx.set_problem(dev(u0))
    hist = opr.parareal(oracle_F(cfg), oracle_G(cfg), u0, N, N)
    for k in range(N + 1):
        if k > 0:
            kd, _ = ctx.iterate(1, 0.0, native.STOP_NONE)
            assert kd == 1
        else:
            ctx.iterate(0, 0.0, native.STOP_NONE)
        got = read_all(ctx, cfg)
        for s in range(1, N + 1):
            e = rel_l2(got[s], hist[k][s])
            assert e < TOL[F32], (k, s, e)
    ctx.close()


@pytest.mark.parametrize("tile", [(64, 32), (64, 16), (32, 16)])
def test_two_row_sweep_bitwise_equals_one_row_kernel(monkeypatch, tile):
    n, N = 64, 4
    cfg, u0 = configs.small(n=n, n_slices=N, dtype=F32, r=2, nf=6, nc=2)
    outs = []
    for path, zc in ((0, n), (ROWS2, 24)):
        tile_env(monkeypatch, fine=(path, tile[0], tile[1], zc))
        ctx = native.Parareal(cfg)
        ctx.set_problem(dev(u0))
        ctx.iterate(2, 0.0, native.STOP_NONE)
        outs.append(read_all(ctx, cfg))
        ctx.close()
    for s in range(N + 1):
        assert np.array_equal(outs[0][s], outs[1][s]), s


def test_two_row_serial_and_coarse_paths(monkeypatch):
    """The single-field launches (serial fine run, coarse steps on 32^3) on
    the two-row kernel: U^N[N] equals the serial fine solution bitwise and
    both match the oracle."""
    n, N = 64, 4
    tile_env(monkeypatch, fine=(ROWS2, 64, 16, n), coarse=(ROWS2, 32, 16, 32))
    monkeypatch.setenv("PARAREAL_SERIAL_TILE", f"{ROWS2},64,32,32")
    cfg, u0 = configs.small(n=n, n_slices=N, dtype=F32, r=2, nf=8, nc=2)
    ctx = native.Parareal(cfg)
    f4, c4, s4 = ctx.launch_shape()
    assert f4[0] == c4[0] == s4[0] == ROWS2
    ctx.set_problem(dev(u0))
    fine = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(fine, as_reference=True)
    ref = u0
    F = oracle_F(cfg)
    for s in range(N):
        ref = F(ref, s)
    assert rel_l2(fine.cpu().numpy(), ref) < TOL[F32]
    kd, h = ctx.iterate(N, 0.0, native.STOP_NONE)
    assert kd == N and h[-1, 2] == 0.0
    last = torch.empty_like(fine)
    ctx.get_slice(N, last)
    assert torch.equal(last, fine)
    ctx.close()


def test_two_row_pair_generation_equals_one_row_kernel(monkeypatch):
    """Training-pair generation advances all initial fields at one slice time
    (slice stride 0) through the batched sweep."""
    n, N = 32, 3
    base, _ = configs.small(n=n, n_slices=N, dtype=F32, nf=8, nc=2)
    base.coarse_kind = native.COARSE_LEARNED
    ics = np.stack([inputs.spectral_ic(n, seed=60 + i, kmax=4) for i in range(3)]).astype(np.float32)
    res = []
    for path in (0, ROWS2):
        tile_env(monkeypatch, fine=(path, 32, 16, n))
        ctx = native.Parareal(base)
        pu = torch.empty((3 * N, n, n, n), dtype=torch.float32, device="cuda")
        pf = torch.empty_like(pu)
        ctx.make_pairs(torch.from_numpy(ics).cuda(), pu, pf)
        torch.cuda.synchronize()
        res.append((pu.cpu().numpy(), pf.cpu().numpy()))
        ctx.close()
    assert np.array_equal(res[0][0], res[1][0])
    assert np.array_equal(res[0][1], res[1][1])
