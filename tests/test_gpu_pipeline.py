"""Pipelined iterations (pipeline_blocks = B > 0) through the C ABI.

The next iteration's fine sweep F(U^{k+1}[n]) runs on a second stream in B
blocks of slices, each started as soon as the serial coarse chain has made
its slices final (the pipelining Sec. 2.2 notes for the fine propagations).
The F values go to a second buffer and the chain waits for the block it
reads, so the iterates, iteration counts and norms must be the same, bit for
bit, as those of the same context without pipelining: in the host loop and
the device loop, for both correction forms, for the learned and the spectral
coarse propagators, when a stopping rule cancels the speculative sweep and
the solve then goes on, and across calls of either kind."""
import numpy as np
import pytest

from oracle import net
from paper_1409_8563_gb300 import configs, native
from tests.helpers import TOL, oracle_F, oracle_G, rel_l2, tile_env
from oracle import parareal as opr

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


def with_blocks(cfg, blocks):
    c = native.Config.from_buffer_copy(cfg)
    c.pipeline_blocks = blocks
    return c


def pair(cfg, u0, blocks, model=None):
    """(plain, pipelined) contexts on the same problem, each with its serial
    fine reference."""
    out = []
    for b in (0, blocks):
        c = native.Parareal(with_blocks(cfg, b))
        if model is not None:
            c.set_coarse_model(model)
        c.set_problem(torch.from_numpy(u0).cuda())
        c.serial_fine(None, as_reference=True)
        out.append(c)
    return out


def same_state(a, b, cfg):
    for s, (x, y) in enumerate(zip(read_all(a, cfg), read_all(b, cfg))):
        assert np.array_equal(x, y), s
    for kind in (native.RES_DIFF_INF, native.RES_DIFF_L2, native.RES_DEFECT):
        assert np.array_equal(a.residual(kind), b.residual(kind)), kind


@pytest.mark.parametrize("form", [native.CORRECTION_STANDARD, native.CORRECTION_DIFFERENCE])
@pytest.mark.parametrize("blocks", [1, 2, 3, 5])
@pytest.mark.parametrize("device", [False, True])
def test_pipelined_iterates_equal_plain_bitwise(monkeypatch, form, blocks, device):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=6, dtype=F32, r=2, nf=8, nc=2)
    cfg.correction_form = form
    plain, pipe = pair(cfg, u0, blocks)
    N = cfg.n_slices
    for k in (1, 2, N - 3):          # three calls: the speculative sweep crosses calls
        kp, hp = plain.iterate(k, 0.0, native.STOP_NONE, device=device)
        kq, hq = pipe.iterate(k, 0.0, native.STOP_NONE, device=device)
        assert kp == kq == k
        assert np.array_equal(hp[:, :3], hq[:, :3])
        same_state(plain, pipe, cfg)
    assert hq[-1, 2] == 0.0          # k = N: the serial fine solution, exactly
    plain.close()
    pipe.close()


@pytest.mark.parametrize("rule,tol", [(native.STOP_DEFECT, 1e-4), (native.STOP_DIFF, 1e-3)])
@pytest.mark.parametrize("device", [False, True])
def test_stopping_cancels_the_speculative_sweep_and_the_solve_goes_on(monkeypatch, rule, tol,
                                                                      device):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=8, dtype=F32, r=2, nf=16, nc=2)
    cfg.correction_form = native.CORRECTION_DIFFERENCE
    plain, pipe = pair(cfg, u0, 3)
    kp, hp = plain.iterate(8, tol, rule, device=device)
    kq, hq = pipe.iterate(8, tol, rule, device=device)
    assert kp == kq and 1 <= kq < cfg.n_slices
    assert np.array_equal(hp[:, :3], hq[:, :3])
    same_state(plain, pipe, cfg)
    # the cancelled sweep is not used: the next iterations recompute F
    for c in (plain, pipe):
        c.iterate(2, 0.0, native.STOP_NONE, device=not device)
    same_state(plain, pipe, cfg)
    # a new problem on the same contexts
    for c in (plain, pipe):
        c.set_problem(torch.from_numpy(u0 * 0.5).cuda())
        c.serial_fine(None, as_reference=True)
    kp, hp = plain.iterate(8, tol, rule, device=device)
    kq, hq = pipe.iterate(8, tol, rule, device=device)
    assert kp == kq and np.array_equal(hp[:, :3], hq[:, :3])
    same_state(plain, pipe, cfg)
    plain.close()
    pipe.close()


def test_mixed_host_and_device_calls(monkeypatch):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=7, dtype=F32, r=2, nf=8, nc=2)
    plain, pipe = pair(cfg, u0, 2)
    plain.iterate(6, 0.0, native.STOP_NONE)
    for k, dev in ((1, False), (2, True), (1, False), (2, True)):
        pipe.iterate(k, 0.0, native.STOP_NONE, device=dev)
    same_state(plain, pipe, cfg)
    plain.close()
    pipe.close()


def test_pipelined_learned_and_spectral(monkeypatch):
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=32, n_slices=5, dtype=F32, r=2, nf=8, nc=4)
    cfg.coarse_kind = native.COARSE_LEARNED
    cfg.learned_skip = native.SKIP_STENCIL
    cfg.learned_act = native.ACT_LINEAR
    cfg.learned_eval = native.EVAL_COMPOSED
    cfg.correction_form = native.CORRECTION_DIFFERENCE
    params = net.init_params(seed=41, scale=0.05)
    w = np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params]).astype(np.float32)
    for dev in (False, True):
        plain, pipe = pair(cfg, u0, 2, model=w)
        assert plain.iterate(4, 0.0, native.STOP_NONE, device=dev)[0] == \
            pipe.iterate(4, 0.0, native.STOP_NONE, device=dev)[0]
        same_state(plain, pipe, cfg)
        plain.close()
        pipe.close()

    cfg, u0 = configs.small(n=32, n_slices=4, dtype=F32, r=4, nf=8, nc=2)
    cfg.coarse_transfer = native.TRANSFER_SPECTRAL
    plain, pipe = pair(cfg, u0, 2)
    plain.iterate(4, 0.0, native.STOP_NONE)
    pipe.iterate(4, 0.0, native.STOP_NONE, device=True)
    same_state(plain, pipe, cfg)
    plain.close()
    pipe.close()


def test_pipelined_iterates_match_the_oracle_over_several_tiles(monkeypatch):
    # 64^3 spans several fused tiles per field; every block of the
    # speculative sweep holds several slices
    tile_env(monkeypatch)
    cfg, u0 = configs.small(n=64, n_slices=8, dtype=F32, r=4, nf=8, nc=2)
    cfg.pipeline_blocks = 3
    ctx = native.Parareal(cfg)
    ctx.set_problem(torch.from_numpy(u0).cuda())
    k, _ = ctx.iterate(3, 0.0, native.STOP_NONE, device=True)
    assert k == 3
    hist = opr.parareal(oracle_F(cfg), oracle_G(cfg), u0, cfg.n_slices, 3)
    got = read_all(ctx, cfg)
    for s in range(1, cfg.n_slices + 1):
        assert rel_l2(got[s], hist[3][s]) < TOL[F32], s
    ctx.close()


def test_pipeline_configuration_is_checked():
    cfg, _ = configs.small(n=16, n_slices=4, dtype=F64)
    cfg.pipeline_blocks = 2
    with pytest.raises(native.PararealError) as e:
        native.Parareal(cfg)                     # FP64: no fused fine sweep
    assert e.value.status == native.E_INVALID
    cfg, _ = configs.small(n=16, n_slices=1, dtype=F32)
    cfg.pipeline_blocks = 1
    with pytest.raises(native.PararealError):
        native.Parareal(cfg)                     # one slice: nothing to pipeline
    cfg, _ = configs.small(n=16, n_slices=4, dtype=F32)
    cfg.pipeline_blocks = -1
    with pytest.raises(native.PararealError):
        native.Parareal(cfg)
    cfg.pipeline_blocks = 2
    with pytest.raises(native.PararealError):
        native.Batch([cfg, cfg])                 # not for batch instances
