"""Training kernels on the 5th-generation tensor cores at sizes where every
persistent CTA takes several tiles: the forward pass that keeps the FP32
pre-activations, the input gradient through the mirrored taps and the
weight gradient (MN-major operands read straight from the [point][16]
layouts, nine accumulators per CTA held in tensor memory across its tiles)
against the FP64 oracle network.

Tolerances as in test_gpu_learned: the oracle rounds to bfloat16 at the same
points as the GPU, so the two differ by one bf16 ulp (2^-8 relative) on the
elements whose FP32 and FP64 sums round differently; per-layer gradients are
held to 2e-2 relative L2.
"""
import numpy as np
import pytest

from oracle import core, net
from paper_1409_8563_gb300 import inputs, native
from tests.helpers import rel_l2
from tests.test_gpu_learned import NET_TOL, from_master, learned_cfg, nu_hat, shift_of, to_master

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _grads(cfg, params, us, tg, slices, linear):
    ctx = native.Parareal(cfg)
    w = to_master(params)
    ctx.set_coarse_model(w)
    params = from_master(w)
    us32 = [x.astype(np.float32) for x in us]
    tg32 = [x.astype(np.float32) for x in tg]
    U = torch.from_numpy(np.stack(us32)).cuda()
    Tg = torch.from_numpy(np.stack(tg32)).cuda()
    g = torch.empty(native.MODEL_PARAMS, dtype=torch.float32, device="cuda")
    loss = ctx.coarse_model_grad(U, Tg, slices, g)
    got = from_master(g.cpu().numpy())
    # a second call on the same context reuses the partial-sum slots: same result
    g2 = torch.empty_like(g)
    ctx.coarse_model_grad(U, Tg, slices, g2)
    assert torch.equal(g, g2)
    ctx.close()
    ref_loss, ref_g = net.loss_and_grads([x.astype(np.float64) for x in us32],
                                         [nu_hat(cfg, s) for s in slices],
                                         [x.astype(np.float64) for x in tg32], params,
                                         shift_of(cfg), bf16_emul=True, linear=linear)
    return loss, got, ref_loss, ref_g


def test_gelu_gradients_at_32_cubed_batch_3():
    """m = 32, three samples: 384 weight-gradient tiles over 192 CTAs (two
    tiles each, the second through the other halo buffer and the next
    mbarrier phase), all three samples in one launch of each layer."""
    cfg = learned_cfg(n=32, N=4)
    params = net.init_params(seed=14, scale=0.15)
    us = [inputs.spectral_ic(32, seed=60 + i, kmax=6) for i in range(3)]
    tg = [core.shift(x, shift_of(cfg)) * 0.9 + 0.05 * inputs.spectral_ic(32, seed=70 + i, kmax=8)
          for i, x in enumerate(us)]
    loss, got, ref_loss, ref_g = _grads(cfg, params, us, tg, [0, 1, 3], linear=False)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss, (loss, ref_loss)
    for li in range(4):
        for k in range(2):
            e = rel_l2(got[li][k], ref_g[li][k])
            assert e < 2 * NET_TOL, (li, k, e)


def test_linear_gradients_at_32_cubed():
    cfg = learned_cfg(n=32, N=4)
    cfg.learned_act = native.ACT_LINEAR
    params = net.init_params(seed=15, scale=0.15)
    us = [inputs.spectral_ic(32, seed=80 + i, kmax=6) for i in range(2)]
    tg = [core.shift(x, shift_of(cfg)) * 0.9 + 0.05 * inputs.spectral_ic(32, seed=90 + i, kmax=8)
          for i, x in enumerate(us)]
    loss, got, ref_loss, ref_g = _grads(cfg, params, us, tg, [2, 3], linear=True)
    assert abs(loss - ref_loss) <= 1e-3 * ref_loss, (loss, ref_loss)
    for li in range(4):
        assert rel_l2(got[li][0], ref_g[li][0]) < 2 * NET_TOL, li
        assert not np.any(got[li][1])
