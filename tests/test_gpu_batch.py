"""Batched uneven problems (one CUDA graph per round, instances as parallel
branches) and the autotuner: every instance of a batch must give bitwise the
same iterates as the same problem run alone with the same launch shapes, and
the oracle's iterates within the FP32 tolerance."""
import json
import os

import numpy as np
import pytest

from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, oracle_G, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def small_batch():
    # uneven sizes and viscosities, N = 4 slices, T = 1/16, dt_F = 2^-m from the
    # batch rule, coarse step 4 dt_F on n / r
    specs = [(16, 0.004, 2), (24, 0.01, 2), (32, 0.02, 4), (48, 0.006, 4), (16, 0.015, 1)]
    cfgs, u0s = [], []
    for k, (n, nu0, r) in enumerate(specs):
        m = configs.batch_dt_exponent(n, nu0)
        cfg = native.Config.make(n, 4, 1.0 / 16, 2.0 ** -m, 4 * 2.0 ** -m, r,
                                 fine_dtype=native.F32, nu0=nu0)
        assert native.stability(cfg)[0] == native.OK
        cfgs.append(cfg)
        u0s.append(inputs.spectral_ic(n, seed=k, kmax=max(2, n // 8)))
    return cfgs, u0s


def test_batch_matches_single_contexts_bitwise_and_the_oracle():
    cfgs, u0s = small_batch()
    b = native.Batch(cfgs)
    for i, u0 in enumerate(u0s):
        b.set_problem(i, torch.from_numpy(u0).cuda())
    b.serial_fine(as_reference=True)
    k, d = b.iterate(2, 0.0, native.STOP_NONE)
    assert list(k) == [2] * len(cfgs)
    assert b.graph_launches() == 3            # start-up + two iterations
    for i, (cfg, u0) in enumerate(zip(cfgs, u0s)):
        solo = native.Parareal(cfg)
        solo.set_problem(torch.from_numpy(u0).cuda())
        solo.iterate(2, 0.0, native.STOP_NONE)
        view = b.context(i)
        a = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
        c = torch.empty_like(a)
        hist = opr.parareal(oracle_F(cfg), oracle_G(cfg), u0, cfg.n_slices, 2)
        for s in range(cfg.n_slices + 1):
            view.get_slice(s, a)
            solo.get_slice(s, c)
            assert torch.equal(a, c), (i, s)
            assert rel_l2(a.cpu().numpy(), hist[2][s]) < TOL[native.F32] or s == 0
        solo.close()
    b.close()


def test_batch_stops_each_instance_on_its_own_rule():
    cfgs, u0s = small_batch()
    b = native.Batch(cfgs)
    for i, u0 in enumerate(u0s):
        b.set_problem(i, torch.from_numpy(u0).cuda())
    b.serial_fine(as_reference=True)
    k, d = b.iterate(4, 1e-6, native.STOP_DEFECT)
    assert np.all(d <= 1e-6) and np.all(k >= 1) and np.all(k <= 4)
    b.close()


def test_autotune_picks_a_valid_shape_and_caches_it(tmp_path):
    cfg, u0 = configs.small(n=64, n_slices=4, dtype=native.F32, r=4, nf=8, nc=2)
    cache = str(tmp_path / "tune.jsonl")
    ctx = native.Parareal(cfg)
    fms, cms = ctx.autotune(cache)
    assert fms > 0
    fine, coarse, serial = ctx.launch_shape()
    lines = [json.loads(l) for l in open(cache)]
    assert any(l["shape"] == list(fine) for l in lines)
    # results with the tuned shape still match the oracle
    ctx.set_problem(torch.from_numpy(u0).cuda())
    ctx.iterate(1, 0.0, native.STOP_NONE)
    hist = opr.parareal(oracle_F(cfg), oracle_G(cfg), u0, 4, 1)
    a = torch.empty((64,) * 3, dtype=torch.float64, device="cuda")
    ctx.get_slice(4, a)
    assert rel_l2(a.cpu().numpy(), hist[1][4]) < TOL[native.F32]
    # a second context takes the cached shape without timing
    ctx2 = native.Parareal(cfg)
    fms2, _ = ctx2.autotune(cache)
    assert fms2 == -1.0 and ctx2.launch_shape()[0] == fine
    ctx.close()
    ctx2.close()


def test_uneven_batch_of_64_instances_converges():
    """The 64-instance workload (sizes from {32,48,64,96,128}, nu0 in
    [0.002, 0.02], N = 8) with shortened horizons T = 1/8 so the test stays
    short; every instance reaches d^k <= 1e-6."""
    ns, nus = inputs.batch_instances(seed=0)
    cfgs, u0s = [], []
    for i, (n, nu0) in enumerate(zip(ns, nus)):
        m = configs.batch_dt_exponent(n, nu0)
        T = 1.0 / 8
        cfg = native.Config.make(n, 8, T, 2.0 ** -m, 16 * 2.0 ** -m, 4, fine_dtype=native.F32,
                                 nu0=nu0)
        cfgs.append(cfg)
        u0s.append(inputs.spectral_ic(n, seed=i, kmax=n // 8))
    b = native.Batch(cfgs)
    b.autotune(None)
    for i, u0 in enumerate(u0s):
        b.set_problem(i, torch.from_numpy(u0).cuda())
    b.serial_fine(as_reference=True)
    k, d = b.iterate(8, 1e-6, native.STOP_DEFECT)
    assert np.all(d <= 1e-6), d
    assert np.all(k <= 8)
    b.close()


def _all_slices(ctx, cfg):
    a = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    out = []
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, a)
        out.append(a.cpu().numpy().copy())
    return out


@pytest.mark.parametrize("shape", [(64, 32, 1), (32, 16, 1), (64, 32, 2), (64, 16, 1)])
def test_queue_round_matches_graph_round_bitwise(shape):
    """Fine sweeps of a round as one persistent launch over the queue of every
    instance's tile steps (uneven sizes, so uneven step counts and tiles
    that wrap past the grid's edge): each instance's iterates equal those of
    the per-instance graph branches, bit for bit, and the oracle's."""
    cfgs, u0s = small_batch()
    runs = []
    for mode in (0, 1):
        b = native.Batch(cfgs)
        if mode:
            b.set_fine_mode(1, *shape)
            assert b.fine_mode() == (1,) + tuple(shape)
        else:
            fused = [b.context(i).launch_shape()[0][0] in (0, 2) for i in range(len(cfgs))]
        for i, u0 in enumerate(u0s):
            b.set_problem(i, torch.from_numpy(u0).cuda())
        b.serial_fine(as_reference=True)
        k, d = b.iterate(3, 0.0, native.STOP_NONE)
        assert list(k) == [3] * len(cfgs)
        runs.append(([_all_slices(b.context(i), c) for i, c in enumerate(cfgs)], d))
        b.close()
    (g, dg), (q, dq) = runs
    # an instance that no fused tile divides (24^3) runs the per-stage kernels
    # in the graph branches and the fused arithmetic in the queue: the same
    # iteration within FP32 rounding; the others bit for bit
    assert sum(fused) >= 3
    for i, cfg in enumerate(cfgs):
        if fused[i]:
            assert dg[i] == dq[i], i
        for s in range(cfg.n_slices + 1):
            if fused[i]:
                assert np.array_equal(g[i][s], q[i][s]), (i, s)
            elif s > 0:
                assert rel_l2(q[i][s], g[i][s]) < TOL[native.F32], (i, s)
    i = 3                                      # the 48^3 instance: tiles wrap in x and y
    hist = opr.parareal(oracle_F(cfgs[i]), oracle_G(cfgs[i]), u0s[i], cfgs[i].n_slices, 3)
    for s in range(1, cfgs[i].n_slices + 1):
        assert rel_l2(q[i][s], hist[3][s]) < TOL[native.F32], s


def test_queue_autotune_and_stopping(monkeypatch):
    cfgs, u0s = small_batch()
    b = native.Batch(cfgs)
    b.set_fine_mode(1)
    b.autotune(None)
    mode = b.fine_mode()
    assert mode[0] == 1 and mode[1:] in [(64, 32, 1), (64, 16, 1), (32, 16, 1), (64, 32, 2)]
    for i, u0 in enumerate(u0s):
        b.set_problem(i, torch.from_numpy(u0).cuda())
    b.serial_fine(as_reference=True)
    k, d = b.iterate(4, 1e-5, native.STOP_DEFECT)
    for i, cfg in enumerate(cfgs):
        # the instance alone, with the launch shapes the batch's autotuner gave it
        fine4, coarse4, serial4 = b.context(i).launch_shape()
        for var, sh in (("PARAREAL_FINE_TILE", fine4), ("PARAREAL_COARSE_TILE", coarse4),
                        ("PARAREAL_SERIAL_TILE", serial4)):
            monkeypatch.setenv(var, ",".join(map(str, sh)))
        solo = native.Parareal(cfg)
        solo.set_problem(torch.from_numpy(u0s[i]).cuda())
        solo.serial_fine(None, as_reference=True)
        ks, hs = solo.iterate(4, 1e-5, native.STOP_DEFECT)
        assert ks == k[i] and hs[-1, 2] == d[i], i
        got = _all_slices(b.context(i), cfg)
        want = _all_slices(solo, cfg)
        for s in range(cfg.n_slices + 1):
            assert np.array_equal(got[s], want[s]), (i, s)
        solo.close()
    b.close()


def test_queue_mode_is_checked():
    cfgs, _ = small_batch()
    b = native.Batch(cfgs)
    with pytest.raises(native.PararealError):
        b.set_fine_mode(1, 16, 16, 1)           # not a compiled queue shape
    b.close()
    cfg64, _ = configs.small(n=16, n_slices=2, dtype=native.F64)
    b = native.Batch([cfg64, cfg64])
    with pytest.raises(native.PararealError):
        b.set_fine_mode(1)                       # FP64 instances
    b.close()
