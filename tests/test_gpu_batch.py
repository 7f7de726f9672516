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
