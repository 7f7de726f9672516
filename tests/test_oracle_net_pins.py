"""Pins of the learned-propagator oracle: finite differences of the loss,
the zero-net identity G = S, bfloat16 rounding against torch's conversion,
and the first Adam step's closed form."""
import numpy as np
import pytest

from oracle import core, net
from paper_1409_8563_gb300 import inputs


def small_problem(n=5, seed=0):
    u = inputs.random_field(n, seed=seed)
    tgt = core.shift(u, (1, 0, 2)) + 0.1 * inputs.random_field(n, seed=seed + 1)
    return u, tgt


def test_zero_last_layer_gives_pure_shift():
    u, _ = small_problem()
    params = net.init_params(seed=1)
    out, _ = net.forward(u, 0.7, params, (1, 0, 2))
    assert np.array_equal(out, core.shift(u, (1, 0, 2)))


@pytest.mark.parametrize("layer,idx", [(0, (3, 1, 0, 2, 1)), (1, (5, 7, 2, 2, 0)),
                                       (2, (0, 15, 1, 1, 1)), (3, (0, 4, 0, 1, 2))])
def test_loss_gradient_matches_central_differences(layer, idx):
    u, tgt = small_problem()
    params = net.init_params(seed=2, scale=0.2)
    _, grads = net.loss_and_grads([u], [0.8], [tgt], params, (1, 0, 2))
    eps = 1e-5
    vals = []
    for sgn in (+1, -1):
        p = [[W.copy(), b.copy()] for W, b in params]
        p[layer][0][idx] += sgn * eps
        vals.append(net.loss_and_grads([u], [0.8], [tgt], p, (1, 0, 2))[0])
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert abs(fd - grads[layer][0][idx]) < 1e-7 * max(1.0, abs(fd)), (fd, grads[layer][0][idx])
    # bias of the same layer
    vals = []
    for sgn in (+1, -1):
        p = [[W.copy(), b.copy()] for W, b in params]
        p[layer][1][0] += sgn * eps
        vals.append(net.loss_and_grads([u], [0.8], [tgt], p, (1, 0, 2))[0])
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert abs(fd - grads[layer][1][0]) < 1e-7 * max(1.0, abs(fd))


def test_bf16_rounding_matches_torch_and_ties_to_even():
    torch = pytest.importorskip("torch")
    x = np.array([1.0, 1 + 2 ** -8, 1 + 3 * 2 ** -8, -2.71828, 3.14159e-3, 65504.0, 1e-30,
                  0.1, -0.3333333])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(net.bf16(x), ref)
    assert net.bf16(1 + 2 ** -8) == 1.0 and net.bf16(1 + 3 * 2 ** -8) == 1.015625
    r = inputs.random_field(8, seed=3).ravel() * 10
    ref = torch.tensor(r, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(net.bf16(r), ref)


def test_first_adam_step_moves_by_lr_times_sign():
    params = [[np.array([[0.5, -1.0]]), np.array([0.0])]]
    grads = [[np.array([[2.0, -3.0]]), np.array([1e-3])]]
    m = net.zeros_like_params(params)
    v = net.zeros_like_params(params)
    net.adam_step(params, grads, m, v, 1, lr=0.01, eps=0.0)
    assert np.allclose(params[0][0], [[0.49, -0.99]], atol=1e-15, rtol=0)
    assert np.allclose(params[0][1], [-0.01], atol=1e-15, rtol=0)


@pytest.mark.parametrize("layer,idx", [(0, (3, 1, 0, 2, 1)), (0, (9, 0, 1, 1, 2)),
                                       (1, (5, 7, 2, 2, 0)), (3, (0, 4, 0, 1, 2))])
def test_linear_mode_gradient_matches_central_differences(layer, idx):
    """Linear mode: backprop through identity activations and the nu-weighted
    second channel (index (co, 1, ...) of layer 0) against central differences;
    the unused biases get zero gradient."""
    u, tgt = small_problem()
    params = net.init_params(seed=2, scale=0.2)
    _, grads = net.loss_and_grads([u], [0.8], [tgt], params, (1, 0, 2), linear=True)
    eps = 1e-5
    vals = []
    for sgn in (+1, -1):
        p = [[W.copy(), b.copy()] for W, b in params]
        p[layer][0][idx] += sgn * eps
        vals.append(net.loss_and_grads([u], [0.8], [tgt], p, (1, 0, 2), linear=True)[0])
    fd = (vals[0] - vals[1]) / (2 * eps)
    assert abs(fd - grads[layer][0][idx]) < 1e-7 * max(1.0, abs(fd)), (fd, grads[layer][0][idx])
    assert not np.any(grads[layer][1])


def test_linear_mode_is_linear_in_u_with_a_nu_dependent_kernel():
    """G(a u + b v) = a G(u) + b G(v) and G(0) = 0, even with nonzero biases;
    the map changes with nu_hat (nu enters as a factor, not as an offset)."""
    u, _ = small_problem(seed=4)
    v, _ = small_problem(seed=7)
    params = net.init_params(seed=5, scale=0.2)
    for W, b in params:
        b += 0.3
    G = lambda x, nu=0.9: net.forward(x, nu, params, (1, 0, 2), linear=True)[0]
    assert np.allclose(G(2.0 * u - 0.5 * v), 2.0 * G(u) - 0.5 * G(v), atol=1e-12, rtol=0)
    assert not np.any(G(np.zeros_like(u)))
    assert np.max(np.abs(G(u, 0.9) - G(u, 1.3))) > 1e-3
