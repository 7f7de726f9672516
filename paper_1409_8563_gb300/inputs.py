"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the oracle.

This module holds none of the method's arithmetic: it only draws random
numbers and samples initial fields on the grid x_i = i / n (i = 0..n-1 per
axis, arrays indexed [z][y][x]).  All generators use
``numpy.random.default_rng(seed)`` and return float64 arrays.
"""
import numpy as np


def paper_ic(n):
    """u0 = sin(2 pi x) sin(2 pi y) sin(2 pi z), the initial value of Sec. 3."""
    s = np.sin(2 * np.pi * np.arange(n) / n)
    return s[:, None, None] * s[None, :, None] * s[None, None, :]


def modes_ic(n, seed=0, n_modes=8, kmin=1, kmax=4):
    """Sum of n_modes Fourier modes A cos(2 pi k.x) + B sin(2 pi k.x).

    Per mode the draws are, in this order: the wavevector k (three integers,
    uniform in kmin..kmax), then A ~ N(0,1), then B ~ N(0,1)."""
    rng = np.random.default_rng(seed)
    x = np.arange(n) / n
    u = np.zeros((n, n, n))
    for _ in range(n_modes):
        k = rng.integers(kmin, kmax + 1, size=3)
        A = rng.standard_normal()
        B = rng.standard_normal()
        ph = 2 * np.pi * (k[0] * x[None, None, :] + k[1] * x[None, :, None] + k[2] * x[:, None, None])
        u += A * np.cos(ph) + B * np.sin(ph)
    return u


def spectral_ic(n, seed=0, kmax=32, slope=-2.0):
    """Gaussian random field with energy per mode |u_k|^2 ~ |k|^slope for
    integer wavevectors 1 <= |k| <= kmax, zero mean, unit RMS.

    The random coefficients are drawn on the fixed block kz, ky in
    [-kmax, kmax], kx in [0, kmax] (real part, then imaginary part, each
    standard normal), so the same seed gives the same field at every n."""
    if 2 * kmax >= n:
        raise ValueError("kmax must be below n/2")
    rng = np.random.default_rng(seed)
    m = 2 * kmax + 1
    re = rng.standard_normal((m, m, kmax + 1))
    im = rng.standard_normal((m, m, kmax + 1))
    kk = np.arange(-kmax, kmax + 1)
    KZ, KY, KX = np.meshgrid(kk, kk, np.arange(kmax + 1), indexing="ij")
    kabs = np.sqrt(KX ** 2 + KY ** 2 + KZ ** 2)
    keep = (kabs >= 1) & (kabs <= kmax)
    amp = np.where(keep, np.maximum(kabs, 1.0) ** (slope / 2.0), 0.0)
    spec = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    spec[np.mod(KZ, n), np.mod(KY, n), KX] = (re + 1j * im) * amp
    u = np.fft.irfftn(spec, s=(n, n, n), axes=(0, 1, 2))
    u -= u.mean()
    return u / np.sqrt(np.mean(u * u))


def batch_instances(seed=0, count=64, sizes=(32, 48, 64, 96, 128), nu0_range=(0.002, 0.02)):
    """Edge sizes and nu0 values of a batch of independent problems.

    Draws: ``count`` sizes uniformly from ``sizes``, then ``count`` values of
    nu0 uniform in ``nu0_range``."""
    rng = np.random.default_rng(seed)
    ns = rng.choice(np.asarray(sizes), size=count)
    nu0 = rng.uniform(nu0_range[0], nu0_range[1], size=count)
    return [int(v) for v in ns], [float(v) for v in nu0]


def initial_weights(seed=0):
    """Starting weights of the learned coarse propagator, flattened in the
    library's order W1[16][2][27] b1 W2[16][16][27] b2 W3 b3 W4[1][16][27] b4:
    normal with standard deviation sqrt(2 / (27 cin)) for the first three
    layers (He et al. 2015), zero for the last layer and all biases, so the
    untrained propagator is the plain shift.  float32."""
    rng = np.random.default_rng(seed)
    out = []
    for li, (ci, co) in enumerate(((2, 16), (16, 16), (16, 16), (16, 1))):
        W = rng.standard_normal((co, ci, 3, 3, 3)) * np.sqrt(2.0 / (27 * ci))
        if li == 3:
            W[:] = 0.0
        out += [W.ravel(), np.zeros(co)]
    return np.concatenate(out).astype(np.float32)


def random_field(n, seed=0):
    """Standard-normal white noise on the n^3 grid (test inputs)."""
    return np.random.default_rng(seed).standard_normal((n, n, n))


def random_weights(shape, seed=0, scale=1.0):
    """Normal weights of a given shape (learned-propagator tests)."""
    return scale * np.random.default_rng(seed).standard_normal(shape)
