"""GPU parity of the CUDA path (through the C ABI) against the FP64 oracle.

Tolerances (relative L2 over the whole field, stated by the method's
precision split): 1e-5 for FP32 stencil paths, 1e-12 for FP64 paths.
"""
import numpy as np
import pytest

from oracle import modal
from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, oracle_G, rel_l2, steps, tile_env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = native.F32, native.F64


def dev(x, dtype):
    t = torch.float64 if dtype == F64 else torch.float32
    return torch.from_numpy(np.ascontiguousarray(x)).to("cuda", t)


def host(t):
    return t.double().cpu().numpy()


# (n, dtype, fine launch shape override "path,tile_x,tile_y,zchunk")
FINE_CASES = [
    (16, F64, (1, 16, 8, 16)),     # staged FP64
    (16, F64, (0, 16, 8, 16)),     # fused FP64, 1 x 2 tiles
    (48, F32, (0, 16, 16, 32)),    # fused FP32, 3 x 3 tiles, ragged z chunks 32 + 16
    (64, F32, (0, 64, 16, 64)),    # the large-grid shape
    (64, F32, (0, 32, 8, 24)),     # ragged z chunks 24 + 24 + 16
    (32, F32, (1, 16, 8, 32)),     # staged FP32
    (24, F64, None),               # no fused shape divides 24: staged default
]


@pytest.mark.parametrize("n,dtype,shape", FINE_CASES)
def test_fine_propagator_matches_oracle(monkeypatch, n, dtype, shape):
    tile_env(monkeypatch, fine=shape)
    cfg, _ = configs.small(n=n, n_slices=3, dtype=dtype, nf=6, nc=2)
    ctx = native.Parareal(cfg)
    src = np.stack([inputs.spectral_ic(n, seed=10 + s, kmax=max(2, n // 4)) for s in range(3)])
    dsrc = dev(src, dtype)
    ddst = torch.empty_like(dsrc)
    ctx.propagate(0, dsrc, ddst, 0, 3)
    got = host(ddst)
    F = oracle_F(cfg)
    for s in range(3):
        ref = F(src[s], s)
        assert rel_l2(got[s], ref) < TOL[dtype], (s, rel_l2(got[s], ref))
    ctx.close()


@pytest.mark.parametrize("n,dtype,r", [(16, F64, 1), (32, F32, 2), (64, F32, 4), (32, F64, 2),
                                       (48, F32, 4)])
def test_coarse_propagator_matches_oracle(monkeypatch, n, dtype, r):
    tile_env(monkeypatch)
    cfg, _ = configs.small(n=n, n_slices=2, dtype=dtype, r=r, nf=8, nc=3)
    ctx = native.Parareal(cfg)
    src = np.stack([inputs.spectral_ic(n, seed=20 + s, kmax=max(2, n // 8)) for s in range(2)])
    dsrc = dev(src, dtype)
    ddst = torch.empty_like(dsrc)
    ctx.propagate(1, dsrc, ddst, 0, 2)
    got = host(ddst)
    G = oracle_G(cfg)
    for s in range(2):
        ref = G(src[s], s)
        assert rel_l2(got[s], ref) < TOL[dtype], (s, rel_l2(got[s], ref))
    ctx.close()


def read_all(ctx, cfg):
    out = []
    buf = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, buf)
        out.append(host(buf))
    return out


@pytest.mark.parametrize("n,dtype,r,N", [(16, F64, 1, 4), (32, F32, 2, 4), (16, F64, 2, 3)])
def test_parareal_iterates_match_oracle(monkeypatch, n, dtype, r, N):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=n, n_slices=N, dtype=dtype, r=r, nf=16, nc=4)
    ctx = native.Parareal(cfg)
    ctx.set_problem(dev(u0, F64))
    hist = opr.parareal(oracle_F(cfg), oracle_G(cfg), u0, N, N)
    for k in range(N + 1):
        if k > 0:
            kd, _ = ctx.iterate(1, 0.0, native.STOP_NONE)
            assert kd == 1
        else:
            ctx.iterate(0, 0.0, native.STOP_NONE)      # runs the coarse start-up only
        got = read_all(ctx, cfg)
        for s in range(1, N + 1):
            assert rel_l2(got[s], hist[k][s]) < TOL[dtype], (k, s, rel_l2(got[s], hist[k][s]))
    ctx.close()


@pytest.mark.parametrize("n,dtype,r,N", [(16, F64, 1, 4), (32, F32, 2, 5)])
def test_parareal_reaches_serial_fine_exactly_at_k_equals_n(monkeypatch, n, dtype, r, N):
    """U^k[n] is the serial fine solution for n <= k, bitwise, and the defect
    d^N is exactly zero (Eq. parareal with F + (G_new - G_old))."""
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=n, n_slices=N, dtype=dtype, r=r, nf=8, nc=2)
    ctx = native.Parareal(cfg)
    ctx.set_problem(dev(u0, F64))
    fine = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(fine, as_reference=True)
    kd, h = ctx.iterate(N, 0.0, native.STOP_NONE)
    assert kd == N
    assert h[-1, 2] == 0.0
    assert np.all(np.diff(h[:, 2]) <= 0) or h[0, 2] > h[-1, 2]
    res = ctx.residual(native.RES_DEFECT)
    assert res[N] == 0.0
    last = torch.empty_like(fine)
    ctx.get_slice(N, last)
    assert torch.equal(last, fine)
    # stop rule on the defect: stops as soon as d^k <= tol
    ctx.set_problem(dev(u0, F64))
    kd2, h2 = ctx.iterate(N, 1e-300, native.STOP_DEFECT)
    assert kd2 == N and h2[-1, 2] == 0.0
    ctx.close()


def test_plain_fp64_32_configuration_matches_oracle():
    """The 32^3 FP64 configuration in full: T = 1, N = 8, 1024 fine steps."""
    cfg, u0 = configs.plain_fp64_32()
    ctx = native.Parareal(cfg)
    assert ctx.status == native.W_MARGINAL
    ctx.set_problem(dev(u0, F64))
    fine = torch.empty((32,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(fine, as_reference=True)
    F, G = oracle_F(cfg), oracle_G(cfg)
    ref_fine = opr.serial_fine(F, u0, 8)
    assert rel_l2(host(fine), ref_fine[8]) < 1e-12
    hist = opr.parareal(F, G, u0, 8, 3)
    kd, h = ctx.iterate(3, 0.0, native.STOP_NONE)
    got = read_all(ctx, cfg)
    for s in range(9):
        assert rel_l2(got[s], hist[3][s]) < 1e-12, s
    for k in range(3):
        d_or = opr.defect(hist[k + 1][8], ref_fine[8])
        assert abs(h[k, 2] - d_or) <= 1e-9 * d_or + 1e-15, (k, h[k, 2], d_or)
    ctx.close()


@pytest.mark.parametrize("shape", [(0, 64, 32, 256), (2, 64, 32, 256)])
def test_fp32_256_fine_sweep_full_size_against_modal_solution(monkeypatch, shape):
    """Full 256^3, 32-slice batched fine sweep in the launch shapes the
    benchmark's autotuner chooses between (64 x 32 tiles, one or two rows per
    thread, whole z columns): U[2m+1] is set to the exact discrete F(U[2m])
    (modal oracle), so the fine residual of odd slices is the relative L2
    error of the GPU sweep."""
    tile_env(monkeypatch, fine=shape)
    cfg, _ = configs.fp32_256()
    ctx = native.Parareal(cfg)
    assert ctx.launch_shape()[0] == shape
    nf, _ = steps(cfg)
    n = cfg.n
    nu = (cfg.nu0, cfg.nu_amp, cfg.nu_omega)
    fields = {}
    for m in range(0, cfg.n_slices, 2):
        u = inputs.spectral_ic(n, seed=100 + m, kmax=8)
        fields[m] = u
        fields[m + 1] = modal.evolve_field(u, tuple(cfg.a), modal.C2, m * nf, cfg.dt_fine, nf, nu,
                                           min_abs=1e-9)
    fields[cfg.n_slices] = fields[cfg.n_slices - 1]
    ctx.set_problem(dev(fields[0], F64))
    for s in range(1, cfg.n_slices + 1):
        ctx.set_slice(s, dev(fields[s], F64))
    res = ctx.residual(native.RES_FINE_L2)
    odd = [res[s] for s in range(1, cfg.n_slices + 1, 2)]
    assert max(odd) < 1e-5, odd
    ctx.close()


def test_fp32_256_parareal_invariants_full_size():
    """Two full-size iterations: the exact slices equal the serial fine
    solution bitwise and the mean is conserved."""
    cfg, u0 = configs.fp32_256()
    ctx = native.Parareal(cfg)
    ctx.set_problem(dev(u0, F64))
    kd, h = ctx.iterate(2, 0.0, native.STOP_NONE)
    assert kd == 2 and h[1, 0] < h[0, 0]
    got = [torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda") for _ in range(3)]
    for s in range(3):
        ctx.get_slice(s, got[s])
    # serial fine over slices 0 and 1 through the same F
    a = dev(u0, F32).contiguous()
    b = torch.empty_like(a)
    ctx.propagate(0, a, b, 0, 1)
    c = torch.empty_like(a)
    ctx.propagate(0, b, c, 1, 1)
    assert torch.equal(got[1].float(), b) and torch.equal(got[2].float(), c)
    for s in range(3):
        assert abs(got[s].mean().item()) < 1e-6
    ctx.close()


def test_error_paths_on_device():
    cfg, u0 = configs.small(n=16, n_slices=2, dtype=F64)
    ctx = native.Parareal(cfg)
    with pytest.raises(native.PararealError) as e:
        ctx.iterate(1)
    assert e.value.status == native.E_STATE
    with pytest.raises(native.PararealError) as e:
        ctx.get_slice(5, torch.empty((16,) * 3, dtype=torch.float64, device="cuda"))
    assert e.value.status == native.E_INVALID
    bad = u0.copy()
    bad[3, 2, 1] = np.nan
    ctx.set_problem(dev(bad, F64))
    with pytest.raises(native.PararealError) as e:
        ctx.iterate(1)
    assert e.value.status == native.E_DIVERGED
    # the context stays usable after a non-CUDA error
    ctx.set_problem(dev(u0, F64))
    kd, _ = ctx.iterate(2)
    assert kd == 2
    ctx.close()


def test_host_buffers_round_trip():
    cfg, u0 = configs.small(n=16, n_slices=2, dtype=F32, r=2)
    ctx = native.Parareal(cfg)
    ctx.set_problem(np.ascontiguousarray(u0))           # host FP64
    out = np.empty_like(u0, dtype=np.float32)
    ctx.get_slice(0, out)                               # host FP32
    assert np.array_equal(out, u0.astype(np.float32))
    ctx.iterate(2)
    fine = np.empty_like(u0)
    ctx.serial_fine(fine, as_reference=True)
    ref = opr.serial_fine(oracle_F(cfg), u0, 2)[2]
    assert rel_l2(fine, ref) < TOL[F32]
    ctx.close()


def test_single_slice_parareal_is_exact_after_one_iteration():
    cfg, u0 = configs.small(n=16, n_slices=1, dtype=F64, nf=8, nc=2)
    ctx = native.Parareal(cfg)
    ctx.set_problem(dev(u0, F64))
    ctx.serial_fine(None, as_reference=True)
    kd, h = ctx.iterate(5, 0.0, native.STOP_NONE)
    assert kd == 1 and h[0, 2] == 0.0
    ctx.close()


@pytest.mark.parametrize("dtype,r", [(F64, 1), (F64, 2), (F32, 2), (F32, 4)])
def test_difference_form_matches_oracle(monkeypatch, dtype, r):
    """F(U^k[n]) + G(U^{k+1}[n] - U^k[n]) on the GPU against Eq. (parareal) as
    printed in the oracle (equal for the linear stencil G), and exact at k = N."""
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=4, dtype=dtype, r=r, nf=8, nc=2)
    cfg.correction_form = native.CORRECTION_DIFFERENCE
    K = 2
    ctx = native.Parareal(cfg)
    ctx.set_problem(dev(u0, F64))
    ctx.iterate(K, 0.0, native.STOP_NONE)
    got = read_all(ctx, cfg)
    hist = opr.parareal(oracle_F(cfg), oracle_G(cfg), u0, cfg.n_slices, K)
    for s in range(1, cfg.n_slices + 1):
        e = rel_l2(got[s], hist[K][s])
        assert e < TOL[dtype], (s, e)
    ctx.set_problem(dev(u0, F64))
    ctx.iterate(cfg.n_slices, 0.0, native.STOP_NONE)
    last = read_all(ctx, cfg)[cfg.n_slices]
    ref = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(ref, as_reference=False)
    assert np.array_equal(last, host(ref))
    ctx.close()
