"""Exact discrete solutions per Fourier mode, the analytic solution, and the
speedup model -- numpy, FP64.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Every discrete operator of the benchmark problem (Sec. 3, Eq. adv_diff_eq) is
a constant-coefficient periodic difference operator, so each Fourier mode
exp(2 pi i k.x) is an eigenvector.  For nu given, its eigenvalue ("symbol")
is nu * L(k) + D(k) with

  C2      L = sum_d (2 cos th_d - 2) / h^2,       D = -i sum_d a_d sin(th_d) / h
  C4      L = sum_d (-2 cos 2th_d + 32 cos th_d - 30) / (12 h^2),
          D = -i sum_d a_d (16 sin th_d - 2 sin 2th_d) / (12 h)
  UPWIND  L as C2,  D = -sum_d a_d (1 - exp(-i th_d)) / h   (a_d > 0)
                         -sum_d a_d (exp(i th_d) - 1) / h   (a_d <= 0)

where th_d = 2 pi k_d / n.  A time-stepping scheme applied to the field acts
on each mode as the same scheme applied to the scalar ODE y' = lambda(t) y.
"""
import numpy as np

C2, C4, UPWIND = 0, 1, 2


def nu_of_t(t, nu0, nu_amp, nu_omega):
    """nu(t) = nu0 (1 + nu_amp sin(omega t)), Sec. 3."""
    return nu0 * (1.0 + nu_amp * np.sin(nu_omega * t))


def symbol_parts(n, a, scheme, k):
    """(L, D) for integer wavevectors k of shape [..., 3] (x, y, z order)."""
    k = np.asarray(k, dtype=np.float64)
    h = 1.0 / n
    th = 2.0 * np.pi * k / n
    if scheme == C4:
        L = np.sum((-2.0 * np.cos(2 * th) + 32.0 * np.cos(th) - 30.0) / (12.0 * h * h), axis=-1)
        D = -1j * np.sum(np.asarray(a) * (16.0 * np.sin(th) - 2.0 * np.sin(2 * th)) / (12.0 * h),
                         axis=-1)
    else:
        L = np.sum((2.0 * np.cos(th) - 2.0) / (h * h), axis=-1)
        if scheme == C2:
            D = -1j * np.sum(np.asarray(a) * np.sin(th) / h, axis=-1)
        else:
            D = np.zeros(L.shape, dtype=np.complex128)
            for d in range(3):
                if a[d] > 0:
                    D = D - a[d] * (1.0 - np.exp(-1j * th[..., d])) / h
                else:
                    D = D - a[d] * (np.exp(1j * th[..., d]) - 1.0) / h
    return L, D + 0j


def rk4_multiplier(L, D, s0, dt, nsteps, nu_params, frozen=False):
    """Product over nsteps classical RK4 steps of the scalar map y -> y'.

    Step j starts at t = (s0 + j) dt; stage eigenvalues lambda_s = nu(t_s) L + D
    at t, t+dt/2, t+dt/2, t+dt (all t when frozen)."""
    R = np.ones(np.shape(L), dtype=np.complex128)
    for j in range(nsteps):
        t = (s0 + j) * dt
        nu1 = nu_of_t(t, *nu_params)
        nu2 = nu1 if frozen else nu_of_t(t + 0.5 * dt, *nu_params)
        nu4 = nu1 if frozen else nu_of_t(t + dt, *nu_params)
        l1 = nu1 * L + D
        l2 = nu2 * L + D
        l4 = nu4 * L + D
        y = np.ones_like(R)
        k1 = l1 * y
        k2 = l2 * (y + 0.5 * dt * k1)
        k3 = l2 * (y + 0.5 * dt * k2)
        k4 = l4 * (y + dt * k3)
        R = R * (y + dt / 6.0 * (k1 + 2.0 * k2 + 2.0 * k3 + k4))
    return R


def euler_multiplier(L, D, s0, dt, nsteps, nu_params):
    """Product over nsteps forward-Euler steps of y -> (1 + dt lambda(t_j)) y."""
    R = np.ones(np.shape(L), dtype=np.complex128)
    for j in range(nsteps):
        t = (s0 + j) * dt
        R = R * (1.0 + dt * (nu_of_t(t, *nu_params) * L + D))
    return R


def rk4_polynomial(z):
    """Stability function of classical RK4: 1 + z + z^2/2 + z^3/6 + z^4/24."""
    return 1.0 + z + z * z / 2.0 + z ** 3 / 6.0 + z ** 4 / 24.0


def fft_wavevectors(n):
    """Integer wavevectors (x, y, z) matching numpy.fft.fftn of a [z][y][x] array."""
    f = np.fft.fftfreq(n, d=1.0 / n)
    kz, ky, kx = np.meshgrid(f, f, f, indexing="ij")
    return np.stack([kx, ky, kz], axis=-1)


def evolve_field(u0, a, scheme, s0, dt, nsteps, nu_params, frozen=False, method="rk4",
                 min_abs=0.0):
    """Exact discrete evolution of a real [z][y][x] field by FFT: every mode with
    |coefficient| > min_abs is multiplied by its scheme multiplier."""
    n = u0.shape[0]
    U = np.fft.fftn(np.asarray(u0, dtype=np.float64))
    k = fft_wavevectors(n)
    mask = np.abs(U) > min_abs
    L, D = symbol_parts(n, a, scheme, k[mask])
    if method == "rk4":
        R = rk4_multiplier(L, D, s0, dt, nsteps, nu_params, frozen)
    else:
        R = euler_multiplier(L, D, s0, dt, nsteps, nu_params)
    V = np.zeros_like(U)
    V[mask] = U[mask] * R
    return np.real(np.fft.ifftn(V))


def field_from_modes(n, k, c):
    """Real part of sum_m c_m exp(2 pi i k_m . x) on the n^3 grid ([z][y][x])."""
    x = np.arange(n) / n
    out = np.zeros((n, n, n), dtype=np.complex128)
    for km, cm in zip(np.asarray(k), np.asarray(c)):
        ex = np.exp(2j * np.pi * km[0] * x)
        ey = np.exp(2j * np.pi * km[1] * x)
        ez = np.exp(2j * np.pi * km[2] * x)
        out += cm * ez[:, None, None] * ey[None, :, None] * ex[None, None, :]
    return np.real(out)


# ----------------------------------------------------------- paper's problem

def paper_modes():
    """u0 = sin(2 pi x) sin(2 pi y) sin(2 pi z) (Sec. 3) as 8 Fourier modes."""
    ks, cs = [], []
    for sx in (-1, 1):
        for sy in (-1, 1):
            for sz in (-1, 1):
                ks.append((sx, sy, sz))
                # sin(th) = (e^{i th} - e^{-i th}) / (2i), one factor per axis
                cs.append((sx / 2j) * (sy / 2j) * (sz / 2j))
    return np.array(ks, dtype=np.float64), np.array(cs)


def analytic_amplitude(t, nu0, nu_amp, nu_omega):
    """a(t) = exp(-12 pi^2 int_0^t nu(s) ds) for nu = nu0 (1 + amp sin(omega s)),
    Sec. 3; the omega -> 0 limit is exp(-12 pi^2 nu0 t)."""
    if nu_omega == 0.0:
        integral = nu0 * t
    else:
        integral = nu0 * t + nu0 * nu_amp * (1.0 - np.cos(nu_omega * t)) / nu_omega
    return np.exp(-12.0 * np.pi ** 2 * integral)


def analytic_paper_field(n, t, nu0, nu_amp, nu_omega, c=(1.0, 1.0, 1.0)):
    """u(x, t) = a(t) u0(x - c t) on the n^3 grid, Sec. 3."""
    x = np.arange(n) / n
    sx = np.sin(2 * np.pi * (x - c[0] * t))
    sy = np.sin(2 * np.pi * (x - c[1] * t))
    sz = np.sin(2 * np.pi * (x - c[2] * t))
    return analytic_amplitude(t, nu0, nu_amp, nu_omega) * (
        sz[:, None, None] * sy[None, :, None] * sx[None, None, :])


def modal_parareal(F_mult, G_mult, c0, k_max):
    """Parareal per mode (Eq. parareal) for slice multipliers F_mult[n], G_mult[n]
    (arrays over modes).  Returns U[k][n] (arrays over modes)."""
    N = len(F_mult)
    U = [c0]
    for n in range(N):
        U.append(G_mult[n] * U[n])
    hist = [list(U)]
    for _ in range(k_max):
        new = [c0]
        for n in range(N):
            new.append(F_mult[n] * U[n] + (G_mult[n] * new[n] - G_mult[n] * U[n]))
        U = new
        hist.append(list(U))
    return hist


# ------------------------------------------------------------- speedup model

def s_bound(n_p, K, nc_over_nf, tauc_over_tauf):
    """Eq. (speedup): 1 / ((1 + K/N_p) (N_c/N_f)(tau_c/tau_f) + K/N_p)."""
    return 1.0 / ((1.0 + K / n_p) * nc_over_nf * tauc_over_tauf + K / n_p)
