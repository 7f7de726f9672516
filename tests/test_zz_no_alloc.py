"""The allocation-free defect-norm entry point.

parareal_diff_norms_noalloc serves callers that cannot call cudaMalloc --
code recording into a CUDA graph during stream capture, code whose device
memory belongs to a framework's caching allocator, latency-critical loops --
by keeping its per-block partial sums in a fixed scratch array inside the
library.  These tests call it through the C ABI and check it against the
defect the context computes with its own (allocated) workspace, on two calls
in a row.  The file is named to be collected last, and passes alone in a
fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest

from paper_1409_8563_gb300 import configs, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def noalloc(a, b, out, count=None):
    return native.lib().parareal_diff_norms_noalloc(
        ctypes.c_void_p(a.data_ptr()), ctypes.c_void_p(b.data_ptr()),
        a.numel() if count is None else count, ctypes.c_void_p(out.data_ptr()), None)


def test_noalloc_defect_matches_the_context_defect_twice():
    cfg, u0 = configs.small(n=32, n_slices=4, dtype=native.F32, r=2, nf=16, nc=4)
    ctx = native.Parareal(cfg)
    ctx.set_problem(torch.from_numpy(u0).cuda())
    fine = torch.empty((32,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(fine, as_reference=True)
    last = torch.empty_like(fine)
    out = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        ctx.iterate(1, 0.0, native.STOP_NONE)             # changes U[N] every time
        d_ctx = ctx.residual(native.RES_DEFECT)[cfg.n_slices]
        ctx.get_slice(cfg.n_slices, last)
        assert noalloc(last, fine, out) == native.OK
        torch.cuda.synchronize()
        o = out.cpu().numpy()
        a, b = last.cpu().numpy(), fine.cpu().numpy()
        assert d_ctx > 0.0
        assert abs(o[0] / o[1] - d_ctx) <= 1e-12 * d_ctx, (call, o, d_ctx)
        assert o[0] == np.max(np.abs(a - b)) and o[1] == np.max(np.abs(b))
        assert abs(o[2] - np.sum((a - b) ** 2)) <= 1e-12 * np.sum((a - b) ** 2)
        assert abs(o[3] - np.sum(b * b)) <= 1e-12 * np.sum(b * b)
        assert o[4] == 0.0
    ctx.close()


def test_noalloc_rejects_counts_beyond_its_scratch():
    a = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    st = noalloc(a, a, out, count=(1 << 26) + 1)   # rejected on the host, nothing launched
    assert st == native.E_INVALID
    assert b"exceeds the maximum" in native.lib().parareal_noalloc_last_error()


def _check_against_numpy(a, b, o):
    d = a - b
    assert o[0] == np.max(np.abs(d)) and o[1] == np.max(np.abs(b))
    assert abs(o[2] - np.sum(d * d)) <= 1e-11 * np.sum(d * d)
    assert abs(o[3] - np.sum(b * b)) <= 1e-11 * np.sum(b * b)
    assert o[4] == 0.0


@pytest.mark.parametrize("count", [1_000_003, native.NOALLOC_MAX_COUNT - 3])
def test_noalloc_ragged_and_near_maximal_counts(count):
    """A count that is not a multiple of the per-block chunk, and one that
    fills the scratch array up to its last block (about 0.5 GB of FP64 per
    input), on two calls in a row with different data."""
    rng = np.random.default_rng(count % 1000)
    out = torch.full((5,), -1.0, dtype=torch.float64, device="cuda")
    for call in range(2):
        a = rng.standard_normal(count)
        b = rng.standard_normal(count) * (call + 1)
        assert noalloc(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), out) == native.OK
        torch.cuda.synchronize()
        _check_against_numpy(a, b, out.cpu().numpy())


@pytest.mark.parametrize("bad", [np.nan, np.inf])
def test_noalloc_flags_a_non_finite_value(bad):
    count = 1_000_003
    rng = np.random.default_rng(7)
    a = rng.standard_normal(count)
    b = rng.standard_normal(count)
    a[count // 3] = bad
    out = torch.zeros(5, dtype=torch.float64, device="cuda")
    assert noalloc(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), out) == native.OK
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert o[4] == 1.0
    assert not np.isfinite(o[0]) and not np.isfinite(o[2])
    assert o[1] == np.max(np.abs(b)) and abs(o[3] - np.sum(b * b)) <= 1e-11 * np.sum(b * b)
    # a later call on finite data clears the flag (the scratch keeps no state)
    a[count // 3] = 0.0
    assert noalloc(torch.from_numpy(a).cuda(), torch.from_numpy(b).cuda(), out) == native.OK
    torch.cuda.synchronize()
    _check_against_numpy(a, b, out.cpu().numpy())
