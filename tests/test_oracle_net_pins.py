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


@pytest.mark.parametrize("b1,b2,want", [(0.5, 0.5, 1.0 / np.sqrt(3.0)),
                                         (0.5, 0.75, np.sqrt(7.0 / 27.0)),
                                         (0.9, 0.999, (0.9 / 1.9) * np.sqrt(1.999 / 0.999))])
def test_second_adam_step_closed_form(b1, b2, want):
    """Two Adam steps with gradients g, then 0.  Unrolling the moment
    recurrences with their bias corrections gives, at step 2,
    m_hat = b1 g / (1 + b1) and v_hat = b2 g^2 / (1 + b2), so the second step
    moves the parameter by lr (b1 / (1 + b1)) sqrt((1 + b2) / b2) sign(g).
    A swapped decay, a wrong bias-correction exponent or a missing square
    root changes it."""
    lr = 0.01
    for g in (3.0, -0.25):
        params = [[np.array([[1.0]]), np.array([0.0])]]
        m = net.zeros_like_params(params)
        v = net.zeros_like_params(params)
        net.adam_step(params, [[np.array([[g]]), np.array([1.0])]], m, v, 1, lr=lr, b1=b1, b2=b2,
                      eps=0.0)
        p1 = params[0][0][0, 0]
        assert abs(p1 - (1.0 - lr * np.sign(g))) < 1e-15
        net.adam_step(params, [[np.array([[0.0]]), np.array([1.0])]], m, v, 2, lr=lr, b1=b1, b2=b2,
                      eps=0.0)
        step = p1 - params[0][0][0, 0]
        assert abs(step - lr * want * np.sign(g)) < 1e-14, (step, lr * want)


def test_constant_gradient_adam_steps_by_lr():
    """With a constant gradient the bias-corrected moments are exactly g and
    g^2 at every step, so each step is lr sign(g)."""
    params = [[np.array([[0.0, 0.0]]), np.array([0.0])]]
    m = net.zeros_like_params(params)
    v = net.zeros_like_params(params)
    g = [[np.array([[0.7, -5.0]]), np.array([1.0])]]
    for step in range(1, 6):
        net.adam_step(params, g, m, v, step, lr=0.1, eps=0.0)
        assert np.allclose(params[0][0], [[-0.1 * step, 0.1 * step]], atol=1e-12, rtol=0)


def _one_path_params(a, c1, b, c, d, e, a_nu=0.0):
    """Network whose only nonzero path is channel 0 through the centre taps:
    layer 1 weight a on input channel 0 (a_nu on channel 1) and bias c1,
    layers 2 and 3 weights b and c, layer 4 weight d and bias e."""
    params = [[np.zeros((co, ci, 3, 3, 3)), np.zeros(co)] for ci, co in net.LAYERS]
    params[0][0][0, 0, 1, 1, 1] = a
    params[0][0][0, 1, 1, 1, 1] = a_nu
    params[0][1][0] = c1
    params[1][0][0, 0, 1, 1, 1] = b
    params[2][0][0, 0, 1, 1, 1] = c
    params[3][0][0, 0, 1, 1, 1] = d
    params[3][1][0] = e
    return params


def test_gelu_follows_the_first_three_layers_only():
    """G(u) = S(u) + d gelu(c gelu(b gelu(a S(u) + c1))) + e, written out with
    the error function: GELU after layers 1-3 and none after layer 4.  An
    activation moved, added or dropped changes the value."""
    import math
    u, _ = small_problem(n=4, seed=5)
    shift = (1, 0, 2)
    a, c1, b, c, d, e = 1.3, 0.2, -0.8, 1.7, 0.9, -0.05
    out, _ = net.forward(u, 0.6, _one_path_params(a, c1, b, c, d, e), shift)
    gelu = np.vectorize(lambda x: 0.5 * x * (1.0 + math.erf(x / math.sqrt(2.0))))
    su = core.shift(u, shift)
    want = su + d * gelu(c * gelu(b * gelu(a * su + c1))) + e
    assert np.allclose(out, want, atol=1e-13, rtol=0)
    # GELU after layer 4 as well would give a different value
    assert np.max(np.abs(out - (su + gelu(d * gelu(c * gelu(b * gelu(a * su + c1))) + e)))) > 1e-3


def test_linear_mode_is_the_product_of_the_path_weights():
    """Linear mode: identity activations, biases unused, second input channel
    nu_hat S(u): G(u) = S(u) + d c b (a + a_nu nu_hat) S(u)."""
    u, _ = small_problem(n=4, seed=6)
    shift = (0, 1, 1)
    a, a_nu, b, c, d, nu_hat = 0.7, -0.4, 1.1, -0.6, 0.5, 0.8
    out, _ = net.forward(u, nu_hat, _one_path_params(a, 0.3, b, c, d, 0.2, a_nu=a_nu), shift,
                         linear=True)
    su = core.shift(u, shift)
    assert np.allclose(out, su * (1.0 + d * c * b * (a + a_nu * nu_hat)), atol=1e-14, rtol=0)
