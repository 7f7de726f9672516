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


def test_composed_kernel_of_single_tap_layers_is_one_shifted_tap():
    """Four layers that each copy channel 0 one cell along a fixed offset
    compose into a single tap at the sum of the offsets, scaled by the product
    of the weights (offsets add under composition of cross-correlations)."""
    params = [[np.zeros((co, ci, 3, 3, 3)), np.zeros(co)] for ci, co in net.LAYERS]
    offs = [(1, 0, 2), (2, 1, 1), (0, 2, 2), (2, 2, 0)]       # (kz, ky, kx) = offset + 1
    scale = [0.5, -2.0, 3.0, 0.25]
    for (W, _), o, a in zip(params, offs, scale):
        W[0, 0][o] = a
    params[0][0][0, 1][1, 1, 1] = 7.0      # channel 1: centre tap, then the same path
    K = net.compose_linear(params, 0.3)
    e = tuple(sum(o[i] - 1 for o in offs) + 4 for i in range(3))
    want = np.zeros((9, 9, 9))
    want[e] += 0.5 * -2.0 * 3.0 * 0.25
    e1 = tuple(sum(o[i] - 1 for o in offs[1:]) + 4 for i in range(3))
    want[e1] += 0.3 * 7.0 * -2.0 * 3.0 * 0.25
    assert np.array_equal(K != 0, want != 0)
    assert np.allclose(K, want, rtol=1e-15, atol=0)


def test_linear_network_equals_its_composed_kernel():
    """Net(S(u)) of the linear network, layer by layer, equals one 9^3
    cross-correlation with the composed kernel (associativity of convolution)."""
    n, s = 11, (2, 0, 1)
    u = inputs.random_field(n, seed=5)
    params = net.init_params(seed=3, scale=0.15)
    for nu_hat in (0.6, 1.4):
        g, _ = net.forward(u, nu_hat, params, s, linear=True)
        su = core.shift(u, s)
        K = net.compose_linear(params, nu_hat)
        got = su + net.apply_kernel(su, K)
        assert np.max(np.abs(got - g)) <= 1e-12 * np.max(np.abs(g)), np.max(np.abs(got - g))
