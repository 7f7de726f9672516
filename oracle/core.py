"""ctypes wrappers for the plain-C FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY (see the package docstring).  Every wrapper copies
its inputs to contiguous float64 arrays and returns new arrays.
"""
import ctypes
import os

import numpy as np

from . import build as _build

C2, C4, UPWIND = 0, 1, 2

_lib = None


class _Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("scheme", ctypes.c_int),
                ("a", ctypes.c_double * 3), ("nu0", ctypes.c_double),
                ("nu_amp", ctypes.c_double), ("nu_omega", ctypes.c_double)]


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        pp = ctypes.POINTER(_Problem)
        L.orc_nu.argtypes = [pp, ctypes.c_double]
        L.orc_nu.restype = ctypes.c_double
        L.orc_apply_A.argtypes = [pp, ctypes.c_double, dp, dp]
        L.orc_rk4.argtypes = [pp, dp, ctypes.c_long, ctypes.c_double, ctypes.c_int, ctypes.c_int]
        L.orc_euler.argtypes = [pp, dp, ctypes.c_long, ctypes.c_double, ctypes.c_int]
        L.orc_restrict_box.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        L.orc_prolong_trilinear.argtypes = [dp, ctypes.c_int, ctypes.c_int, dp]
        L.orc_shift.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp]
        L.orc_conv3d_fwd.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, dp]
        L.orc_conv3d_dgrad.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_conv3d_wgrad.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp]
        L.orc_gelu.argtypes = [dp, ctypes.c_long, dp]
        L.orc_gelu_grad.argtypes = [dp, ctypes.c_long, dp]
        _lib = L
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Problem:
    """Periodic n^3 advection-diffusion problem u_t = -a.grad u + nu(t) Lap u.

    nu(t) = nu0 * (1 + nu_amp * sin(nu_omega * t)) (Sec. 3); ``scheme`` is one
    of C2 (7-point Laplacian + centred advection), C4 (fourth-order centred)
    or UPWIND (7-point Laplacian + first-order upwind, Algorithm 2).
    """

    def __init__(self, n, a=(1.0, 1.0, 1.0), nu0=0.01, nu_amp=0.5,
                 nu_omega=2.0 * np.pi, scheme=C2):
        self.n = int(n)
        self.a = tuple(float(x) for x in a)
        self.nu0, self.nu_amp, self.nu_omega = float(nu0), float(nu_amp), float(nu_omega)
        self.scheme = int(scheme)
        self._c = _Problem(self.n, self.scheme, (ctypes.c_double * 3)(*self.a),
                           self.nu0, self.nu_amp, self.nu_omega)

    def with_n(self, n, scheme=None):
        return Problem(n, self.a, self.nu0, self.nu_amp, self.nu_omega,
                       self.scheme if scheme is None else scheme)

    def nu(self, t):
        return lib().orc_nu(ctypes.byref(self._c), float(t))

    def apply_A(self, u, nu):
        u = _f64(u)
        out = np.empty_like(u)
        lib().orc_apply_A(ctypes.byref(self._c), float(nu), _dp(u), _dp(out))
        return out

    def rk4(self, u, s0, dt, nsteps, frozen=False):
        """Classical RK4 over nsteps steps starting at time s0*dt."""
        u = _f64(u).copy()
        assert u.shape == (self.n,) * 3
        lib().orc_rk4(ctypes.byref(self._c), _dp(u), int(s0), float(dt), int(nsteps),
                      1 if frozen else 0)
        return u

    def euler(self, u, s0, dt, nsteps):
        u = _f64(u).copy()
        lib().orc_euler(ctypes.byref(self._c), _dp(u), int(s0), float(dt), int(nsteps))
        return u


def restrict_box(f, r):
    f = _f64(f)
    n = f.shape[0]
    c = np.empty((n // r,) * 3)
    lib().orc_restrict_box(_dp(f), n, int(r), _dp(c))
    return c


def prolong_trilinear(c, r):
    c = _f64(c)
    nc = c.shape[0]
    f = np.empty((nc * r,) * 3)
    lib().orc_prolong_trilinear(_dp(c), nc, int(r), _dp(f))
    return f


def shift(u, s):
    """out[z, y, x] = u[z - s_z, y - s_y, x - s_x] (periodic); s = (s_x, s_y, s_z)."""
    u = _f64(u)
    out = np.empty_like(u)
    lib().orc_shift(_dp(u), u.shape[0], int(s[0]), int(s[1]), int(s[2]), _dp(out))
    return out


def conv3d_fwd(x, W, b=None):
    """x: [cin, n, n, n], W: [cout, cin, 3, 3, 3], b: [cout] -> [cout, n, n, n]."""
    x, W = _f64(x), _f64(W)
    cout, cin = W.shape[0], W.shape[1]
    n = x.shape[1]
    out = np.empty((cout, n, n, n))
    bb = _f64(b) if b is not None else None
    lib().orc_conv3d_fwd(_dp(x), n, cin, cout, _dp(W), _dp(bb) if bb is not None else None,
                         _dp(out))
    return out


def conv3d_dgrad(dout, W):
    dout, W = _f64(dout), _f64(W)
    cout, cin = W.shape[0], W.shape[1]
    n = dout.shape[1]
    din = np.empty((cin, n, n, n))
    lib().orc_conv3d_dgrad(_dp(dout), n, cin, cout, _dp(W), _dp(din))
    return din


def conv3d_wgrad(x, dout):
    x, dout = _f64(x), _f64(dout)
    cin, cout, n = x.shape[0], dout.shape[0], x.shape[1]
    dW = np.empty((cout, cin, 3, 3, 3))
    db = np.empty(cout)
    lib().orc_conv3d_wgrad(_dp(x), _dp(dout), n, cin, cout, _dp(dW), _dp(db))
    return dW, db


def gelu(x):
    x = _f64(x)
    y = np.empty_like(x)
    lib().orc_gelu(_dp(x), x.size, _dp(y))
    return y


def gelu_grad(x):
    x = _f64(x)
    g = np.empty_like(x)
    lib().orc_gelu_grad(_dp(x), x.size, _dp(g))
    return g
