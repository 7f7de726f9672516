"""The cluster-resident RK4 path (launch path 4) through the C ABI.

A small field lives in the distributed shared memory of one thread-block
cluster for a whole sweep; its per-point arithmetic is the per-stage
kernel's, so every result must equal the per-stage path (launch path 1) bit
for bit: one coarse propagator application, one serial fine propagation,
batched fine sweeps of several slices, and whole Parareal iterations, FP32
and FP64, with classical and frozen nu(t), on grids split over 1 to 8 CTAs.
The oracle pins the path once more at relative L2 1e-5 / 1e-12."""
import numpy as np
import pytest

from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, oracle_G, rel_l2, steps

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = native.F32, native.F64
STAGED, CLUSTER = 1, 4


def shapes(monkeypatch, fine, serial, coarse, n, m):
    """Launch paths of the batched fine sweep, the serial fine run and the
    coarse propagator (1 = per-stage, 4 = cluster)."""
    for var, path, size in (("PARAREAL_FINE_TILE", fine, n), ("PARAREAL_SERIAL_TILE", serial, n),
                            ("PARAREAL_COARSE_TILE", coarse, m)):
        monkeypatch.setenv(var, f"{path},16,8,{size}" if path == STAGED else f"{path},0,0,{size}")


def fields(n, count, seed):
    return np.stack([inputs.random_field(n, seed=seed + s) + inputs.spectral_ic(n, seed=seed + 50 + s, kmax=3)
                     for s in range(count)])


@pytest.mark.parametrize("n,r,dtype", [(32, 4, F32), (32, 1, F32), (48, 4, F32), (16, 2, F32),
                                       (24, 2, F32), (32, 2, F64), (16, 1, F64)])
@pytest.mark.parametrize("frozen", [False, True])
def test_propagators_equal_the_per_stage_path_bitwise(monkeypatch, n, r, dtype, frozen):
    m = n // r
    cfg, _ = configs.small(n=n, n_slices=3, dtype=dtype, r=r, nf=8, nc=2)
    if frozen:
        cfg.nu_mode = native.NU_FROZEN
    out = {}
    src = fields(n, 3, seed=7)
    t = torch.float64 if dtype == F64 else torch.float32
    dsrc = torch.from_numpy(src).to("cuda", t)
    for path in (STAGED, CLUSTER):
        coarse = path if native.cluster_size(dtype, m) else STAGED
        serial = path if native.cluster_size(dtype, n) else STAGED
        shapes(monkeypatch, STAGED, serial, coarse, n, m)
        ctx = native.Parareal(cfg)
        res = []
        for which in (0, 1):
            dst = torch.empty_like(dsrc)
            ctx.propagate(which, dsrc, dst, 0, 3)
            res.append(dst.cpu().numpy())
        out[path] = res
        ctx.close()
    for which in (0, 1):
        assert np.array_equal(out[STAGED][which], out[CLUSTER][which]), which
    # and the oracle: F and G of slice s on the field as the GPU saw it
    F, G = oracle_F(cfg), oracle_G(cfg)
    for s in range(3):
        x = src[s].astype(np.float32).astype(np.float64) if dtype == F32 else src[s]
        assert rel_l2(out[CLUSTER][0][s], F(x, s)) < TOL[dtype]
        assert rel_l2(out[CLUSTER][1][s], G(x, s)) < TOL[dtype]


def read_all(ctx, cfg):
    buf = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    out = []
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, buf)
        out.append(buf.cpu().numpy().copy())
    return out


@pytest.mark.parametrize("n,r,dtype,form", [(32, 4, F32, native.CORRECTION_DIFFERENCE),
                                            (24, 2, F32, native.CORRECTION_STANDARD),
                                            (16, 1, F64, native.CORRECTION_STANDARD)])
def test_parareal_iterations_equal_the_per_stage_path_bitwise(monkeypatch, n, r, dtype, form):
    # batched fine sweeps of N slices (N clusters per launch), the serial fine
    # reference and the coarse chain all on the cluster path
    m = n // r
    cfg, u0 = configs.small(n=n, n_slices=5, dtype=dtype, r=r, nf=8, nc=2)
    cfg.correction_form = form
    assert native.cluster_size(dtype, n) > 0 and native.cluster_size(dtype, m) > 0
    runs = {}
    for path in (STAGED, CLUSTER):
        shapes(monkeypatch, path, path, path, n, m)
        ctx = native.Parareal(cfg)
        assert [sh[0] for sh in ctx.launch_shape()] == [path] * 3
        ctx.set_problem(torch.from_numpy(u0).cuda())
        ctx.serial_fine(None, as_reference=True)
        k, h = ctx.iterate(3, 0.0, native.STOP_NONE)
        k2, h2 = ctx.iterate(2, 0.0, native.STOP_NONE, device=True)
        runs[path] = (read_all(ctx, cfg), np.vstack([h, h2]))
        ctx.close()
    for s in range(cfg.n_slices + 1):
        assert np.array_equal(runs[STAGED][0][s], runs[CLUSTER][0][s]), s
    assert np.array_equal(runs[STAGED][1][:, :3], runs[CLUSTER][1][:, :3])
    assert runs[CLUSTER][1][-1, 2] == 0.0          # k = N: the serial fine run, exactly
    # three iterations against the oracle's Parareal
    hist = opr.parareal(oracle_F(cfg), oracle_G(cfg), u0, cfg.n_slices, 3,
                        form="difference" if form == native.CORRECTION_DIFFERENCE else "standard")
    for path in (CLUSTER,):
        shapes(monkeypatch, path, path, path, n, m)
        ctx = native.Parareal(cfg)
        ctx.set_problem(torch.from_numpy(u0).cuda())
        ctx.iterate(3, 0.0, native.STOP_NONE)
        got = read_all(ctx, cfg)
        for s in range(1, cfg.n_slices + 1):
            assert rel_l2(got[s], hist[3][s]) < TOL[dtype], s
        ctx.close()


def test_cluster_sizes_and_unsupported_shapes(monkeypatch):
    c32 = native.cluster_size(F32, 32)
    assert c32 in (8, 16)                              # 16 where the device schedules it
    assert native.cluster_size(F64, 32) == c32
    assert native.cluster_size(F32, 12) == 4
    # 48^3: fits 16 CTAs, not 8; 64^3 fits neither
    assert native.cluster_size(F32, 48) == (16 if c32 == 16 else 0)
    assert native.cluster_size(F32, 64) == 0
    cfg, _ = configs.small(n=64, n_slices=2, dtype=F32)
    monkeypatch.setenv("PARAREAL_FINE_TILE", "4,0,0,64")
    with pytest.raises(native.PararealError) as e:
        native.Parareal(cfg)
    assert e.value.status == native.E_INVALID
