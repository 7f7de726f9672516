"""Failure detection on the GPU without a GPU fault: the bounded device-side
wait of the tensor-core layers gives up on a barrier that nothing arrives
on, the host reads PARAREAL_E_TIMEOUT, and the device stays usable.  (A
non-finite iterate giving PARAREAL_E_DIVERGED is in test_gpu_parity.py.)"""
import time

import numpy as np
import pytest

from paper_1409_8563_gb300 import configs, native
from tests.helpers import TOL, oracle_F, rel_l2

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def test_bounded_wait_gives_up_and_the_device_stays_usable():
    t0 = time.perf_counter()
    st = native.selftest_timeout()
    took = time.perf_counter() - t0
    assert st == native.E_TIMEOUT, st
    assert "self-test" in native.lib().parareal_last_error(None).decode()
    assert took < 30.0, took
    # the device still computes: one fine propagation against the oracle
    cfg, u0 = configs.small(n=16, n_slices=2, dtype=native.F32, nf=4, nc=2)
    ctx = native.Parareal(cfg)
    src = torch.from_numpy(np.ascontiguousarray(u0[None])).cuda()
    dst = torch.empty_like(src)
    ctx.propagate(0, src, dst, 0, 1)
    assert rel_l2(dst[0].cpu().numpy(), oracle_F(cfg)(u0, 0)) < TOL[native.F32]
    ctx.close()
    # and the self-test is repeatable on the same device
    assert native.selftest_timeout() == native.E_TIMEOUT


def test_grid_barrier_gives_up_and_the_device_stays_usable():
    """The persistent RK4 path's grid barrier with one block that never
    arrives: the other blocks' bounded waits give up, the host reads
    PARAREAL_E_TIMEOUT, and an FP64 context on the persistent path still
    matches the oracle afterwards."""
    t0 = time.perf_counter()
    st = native.selftest_grid_barrier()
    took = time.perf_counter() - t0
    assert st == native.E_TIMEOUT, st
    assert "self-test" in native.lib().parareal_last_error(None).decode()
    assert took < 30.0, took
    cfg, u0 = configs.small(n=16, n_slices=2, dtype=native.F64, nf=4, nc=2)
    ctx = native.Parareal(cfg)
    assert ctx.launch_shape()[0][0] == 3          # the persistent path
    src = torch.from_numpy(np.ascontiguousarray(u0[None])).cuda()
    dst = torch.empty_like(src)
    ctx.propagate(0, src, dst, 0, 1)
    assert rel_l2(dst[0].cpu().numpy(), oracle_F(cfg)(u0, 0)) < TOL[native.F64]
    ctx.close()
    assert native.selftest_grid_barrier() == native.E_TIMEOUT
