"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

Each test ties an oracle routine to something other than itself: the RK4
stability polynomial at the discrete Fourier symbol, conservation laws,
convergence orders against the analytic solution of Sec. 3, the errors the
paper prints (Sec. 3.1), the convergence statement of Sec. 3.4.1, Table 1,
and exact identities of restriction/prolongation/shift/convolution.
"""
import numpy as np
import pytest

from oracle import core, modal
from oracle import parareal as opr
from paper_1409_8563_gb300 import inputs

TWO_PI = 2.0 * np.pi


def cos_mode(n, k):
    x = np.arange(n) / n
    ph = TWO_PI * (k[0] * x[None, None, :] + k[1] * x[None, :, None] + k[2] * x[:, None, None])
    return ph


# ------------------------------------------------------- operator and RK4 pins

@pytest.mark.parametrize("k", [(1, 0, 0), (2, 3, 1), (5, 5, 5), (6, 1, 4)])
def test_single_mode_decays_by_rk4_polynomial_at_discrete_symbol(k):
    """A Fourier mode of the 7-point/centred operator evolves, per RK4 step,
    by R(z) = 1 + z + z^2/2 + z^3/6 + z^4/24 at z = dt * symbol (constant nu).
    The symbol is derived analytically (Fourier transform of the stencil):
    lambda = nu sum (2cos th - 2)/h^2 - i sum a_d sin th_d / h."""
    n, dt, steps, nu = 12, 2e-3, 3, 0.03
    a = (1.0, -0.5, 0.25)
    P = core.Problem(n, a=a, nu0=nu, nu_amp=0.0, scheme=core.C2)
    ph = cos_mode(n, k)
    u1 = P.rk4(np.cos(ph), 0, dt, steps)
    h = 1.0 / n
    th = TWO_PI * np.array(k) / n
    lam = nu * np.sum((2 * np.cos(th) - 2) / h ** 2) - 1j * np.sum(np.array(a) * np.sin(th) / h)
    R = modal.rk4_polynomial(dt * lam) ** steps
    expected = np.real(R * np.exp(1j * ph))
    assert np.max(np.abs(u1 - expected)) < 1e-13


@pytest.mark.parametrize("scheme", [core.C2, core.C4, core.UPWIND])
def test_mean_is_conserved(scheme):
    n = 10
    P = core.Problem(n, a=(1.0, 0.7, -0.3), nu0=0.02, nu_amp=0.5, nu_omega=TWO_PI, scheme=scheme)
    u = inputs.random_field(n, seed=3) + 0.37
    v = P.rk4(u, 5, 1e-3, 7)
    w = P.euler(u, 5, 1e-3, 7)
    assert abs(v.mean() - u.mean()) < 1e-14
    assert abs(w.mean() - u.mean()) < 1e-14


@pytest.mark.parametrize("scheme", [core.C2, core.C4, core.UPWIND])
@pytest.mark.parametrize("frozen", [False, True])
def test_stepper_equals_modal_exact_discrete_solution(scheme, frozen):
    """Real-space C stepper vs FFT-diagonalised scalar recurrence."""
    n = 12
    a = (1.0, -0.6, 0.35)
    nu = (0.02, 0.5, 7.0)
    P = core.Problem(n, a=a, nu0=nu[0], nu_amp=nu[1], nu_omega=nu[2], scheme=scheme)
    u = inputs.random_field(n, seed=11)
    got = P.rk4(u, 13, 1.5e-3, 9, frozen=frozen)
    ref = modal.evolve_field(u, a, scheme, 13, 1.5e-3, 9, nu, frozen=frozen)
    assert np.max(np.abs(got - ref)) < 1e-12 * np.max(np.abs(u))
    got_e = P.euler(u, 13, 1.5e-3, 9)
    ref_e = modal.evolve_field(u, a, scheme, 13, 1.5e-3, 9, nu, method="euler")
    assert np.max(np.abs(got_e - ref_e)) < 1e-12 * np.max(np.abs(u))


def test_rk4_stage_times_give_fourth_order_frozen_nu_first_order():
    """For y' = (nu(t) L + D) y the exact solution is exp(L int nu + D t).
    Classical stage times make RK4 fourth order; nu frozen at the step start
    drops it to first order (the reading that reproduces the paper's
    omega = 100 fine error)."""
    L, D = -40.0, -3.0j
    nu = (0.1, 0.5, 100.0)
    T = 0.1
    exact = np.exp(L * (nu[0] * T + nu[0] * nu[1] * (1 - np.cos(nu[2] * T)) / nu[2]) + D * T)
    errs = {False: [], True: []}
    for m in (200, 400, 800):
        for frozen in (False, True):
            R = modal.rk4_multiplier(np.array([L]), np.array([D]), 0, T / m, m, nu, frozen)
            errs[frozen].append(abs(R[0] - exact))
    classical = np.log2(np.array(errs[False][:-1]) / np.array(errs[False][1:]))
    frozen = np.log2(np.array(errs[True][:-1]) / np.array(errs[True][1:]))
    assert np.all(np.abs(classical - 4.0) < 0.2), classical
    assert np.all(np.abs(frozen - 1.0) < 0.2), frozen


@pytest.mark.parametrize("scheme,order", [(core.C2, 2), (core.C4, 4)])
def test_spatial_order_against_analytic_solution(scheme, order):
    """Discretisation error of the semi-discrete operator vs the analytic
    solution a(t) u0(x - c t) of Sec. 3 (nu constant, tiny dt so time error
    is negligible): halving h divides the error by 2^order."""
    nu = (0.1, 0.0, 0.0)
    T = 0.01
    errs = []
    for n in (16, 32):
        k, c = modal.paper_modes()
        L, D = modal.symbol_parts(n, (1.0, 1.0, 1.0), scheme, k)
        R = np.exp((nu[0] * L + D) * T)          # exact time integration
        u = modal.field_from_modes(n, k, c * R)
        ex = modal.analytic_paper_field(n, T, *nu)
        errs.append(np.max(np.abs(u - ex)) / np.max(np.abs(ex)))
    rate = np.log2(errs[0] / errs[1])
    assert abs(rate - order) < 0.15, (errs, rate)


# --------------------------------------------------------- paper's numbers

def _paper_error(scheme, method, m, nu_omega, frozen):
    n, T, nu0 = 128, 0.1, 0.1
    k, c = modal.paper_modes()
    L, D = modal.symbol_parts(n, (1.0, 1.0, 1.0), scheme, k)
    nu = (nu0, 0.5, nu_omega)
    if method == "rk4":
        R = modal.rk4_multiplier(L, D, 0, T / m, m, nu, frozen)
    else:
        R = modal.euler_multiplier(L, D, 0, T / m, m, nu)
    u = modal.field_from_modes(n, k, c * R)
    ex = modal.analytic_paper_field(n, T, *nu)
    return np.max(np.abs(u - ex)) / np.max(np.abs(ex))


@pytest.mark.slow
def test_paper_fine_error_omega0():
    """Sec. 3.1: eps_fine ~ 1.9e-7 for omega = 0 (RK4, 4th-order, 128^3, T/2^15)."""
    e = _paper_error(modal.C4, "rk4", 2 ** 15, 0.0, False)
    assert 1.85e-7 <= e < 1.95e-7, e


@pytest.mark.slow
def test_paper_fine_error_omega100_needs_frozen_nu():
    """Sec. 3.1: eps_fine ~ 4.8e-6 for omega = 100.  Reproduced only with nu
    frozen at the step start; classical stage times give ~1.9e-7."""
    e_frozen = _paper_error(modal.C4, "rk4", 2 ** 15, 100.0, True)
    e_stage = _paper_error(modal.C4, "rk4", 2 ** 15, 100.0, False)
    assert 4.75e-6 <= e_frozen < 4.85e-6, e_frozen
    assert e_stage < 3e-7, e_stage


@pytest.mark.parametrize("omega", [0.0, 100.0])
def test_paper_coarse_error(omega):
    """Sec. 3.1: eps_coarse ~ 4.5e-2 (forward Euler, upwind, T/2^11), both omega."""
    e = _paper_error(modal.UPWIND, "euler", 2 ** 11, omega, False)
    assert 4.45e-2 <= e < 4.55e-2, e


@pytest.mark.slow
@pytest.mark.parametrize("n_p", [8, 32, 128])
def test_paper_parareal_defect_after_three_iterations(n_p):
    """Sec. 3.4.1: after three iterations d^k is far below eps_fine = 4.8e-6
    (omega = 100) and of the order of the fine error 1.9e-7 (omega = 0)."""
    n, T, nu0 = 128, 0.1, 0.1
    k, c = modal.paper_modes()
    Lf, Df = modal.symbol_parts(n, (1.0, 1.0, 1.0), modal.C4, k)
    Lg, Dg = modal.symbol_parts(n, (1.0, 1.0, 1.0), modal.UPWIND, k)
    nf, nc = 2 ** 15 // n_p, 2 ** 11 // n_p
    for omega, lo, hi in ((100.0, 0.0, 4.8e-7), (0.0, 1.9e-8, 1.9e-6)):
        nu = (nu0, 0.5, omega)
        Fm = [modal.rk4_multiplier(Lf, Df, s * nf, T / 2 ** 15, nf, nu, True) for s in range(n_p)]
        Gm = [modal.euler_multiplier(Lg, Dg, s * nc, T / 2 ** 11, nc, nu) for s in range(n_p)]
        hist = modal.modal_parareal(Fm, Gm, c, 3)
        fine = c.copy()
        for s in range(n_p):
            fine = Fm[s] * fine
        u_f = modal.field_from_modes(n, k, fine)
        u_3 = modal.field_from_modes(n, k, hist[3][n_p])
        d3 = np.max(np.abs(u_3 - u_f)) / np.max(np.abs(u_f))
        assert lo < d3 < hi, (omega, d3)


def test_speedup_bound_reproduces_table1():
    """Table 1: S_bound for K = 3, N_c/N_f = 1/16 and one fitted tau_c/tau_f per
    backend reproduces the printed column to its rounding."""
    nodes = np.array([4, 8, 16, 32, 64, 128])
    table = {"cpu": [1.3, 2.6, 5.0, 9.5, 17.4, 29.8], "gpu": [1.3, 2.6, 5.0, 9.4, 16.8, 28.0]}
    for col in table.values():
        col = np.array(col)
        ratios = np.linspace(0.05, 0.4, 3501)
        resid = [np.sum((modal.s_bound(nodes, 3, 1 / 16, r) - col) ** 2) for r in ratios]
        r = ratios[int(np.argmin(resid))]
        got = modal.s_bound(nodes, 3, 1 / 16, r)
        assert np.all(np.abs(got - col) <= 0.1 + 1e-9), (r, got)
        assert 0.1 < r < 0.3


# -------------------------------------------------------------- Parareal pins

def test_parareal_is_exact_on_converged_slices_and_at_k_equals_n():
    """U^k[n] equals the serial fine solution for n <= k, bitwise, and the
    whole iterate does at k = N_p (Eq. parareal with F + (G_new - G_old))."""
    n, N = 8, 4
    P = core.Problem(n, nu0=0.01)
    u0 = inputs.modes_ic(n, seed=0)
    F = opr.rk4_propagator(P, 1.0 / 64, 16)
    G = opr.rk4_propagator(P, 1.0 / 8, 2)
    fine = opr.serial_fine(F, u0, N)
    hist = opr.parareal(F, G, u0, N, N)
    for k in range(N + 1):
        for s in range(k + 1):
            assert np.array_equal(hist[k][s], fine[s]), (k, s)
    assert opr.defect(hist[N][N], fine[N]) == 0.0
    assert opr.defect(hist[1][N], fine[N]) > 0.0


def test_parareal_with_coarsened_propagator_converges():
    n, N = 16, 4
    P = core.Problem(n, nu0=0.01)
    u0 = inputs.spectral_ic(n, seed=1, kmax=4)
    F = opr.rk4_propagator(P, 1.0 / 256, 64)
    G = opr.coarsened_rk4_propagator(P, 2, 1.0 / 32, 8)
    fine = opr.serial_fine(F, u0, N)
    hist = opr.parareal(F, G, u0, N, N)
    d = [opr.defect(h[N], fine[N]) for h in hist]
    assert d[-1] == 0.0
    assert d[1] < d[0] and d[2] < d[1]


# --------------------------------------------- restriction / prolongation / shift

@pytest.mark.parametrize("r", [2, 4])
def test_restriction_prolongation_identities(r):
    nc = 4
    n = nc * r
    f = inputs.random_field(n, seed=5)
    c = inputs.random_field(nc, seed=6)
    # constants are kept
    assert np.allclose(core.restrict_box(np.full((n,) * 3, 2.5), r), 2.5, atol=1e-15, rtol=0)
    assert np.allclose(core.prolong_trilinear(np.full((nc,) * 3, -1.25), r), -1.25, atol=1e-15, rtol=0)
    # means are kept
    assert abs(core.restrict_box(f, r).mean() - f.mean()) < 1e-14
    assert abs(core.prolong_trilinear(c, r).mean() - c.mean()) < 1e-14
    # a field linear in the fine x index restricts to its value at the cell centroid
    lin = np.broadcast_to(np.arange(n, dtype=float)[None, None, :], (n, n, n))
    R = core.restrict_box(lin, r)
    assert np.allclose(R[0, 0, :], np.arange(nc) * r + 0.5 * (r - 1), atol=1e-13, rtol=0)
    # a coarse field linear in I interpolates exactly where no wrap intervenes
    clin = np.broadcast_to(np.arange(nc, dtype=float)[None, None, :], (nc, nc, nc))
    Pf = core.prolong_trilinear(clin, r)
    s = (np.arange(n) - 0.5 * (r - 1)) / r
    inner = (np.floor(s) >= 0) & (np.floor(s) + 1 <= nc - 1)
    assert np.allclose(Pf[1, 2, inner], s[inner], atol=1e-13, rtol=0)


def test_shift_multiplies_modes_by_phase():
    n, sh = 8, (3, -2, 1)
    k = (1, 2, 3)
    ph = cos_mode(n, k)
    out = core.shift(np.cos(ph), sh)
    expected = np.cos(ph - TWO_PI * (k[0] * sh[0] + k[1] * sh[1] + k[2] * sh[2]) / n)
    assert np.max(np.abs(out - expected)) < 1e-13
    back = core.shift(out, (-sh[0], -sh[1], -sh[2]))
    assert np.max(np.abs(back - np.cos(ph))) < 1e-13


# -------------------------------------------------------------- convolution pins

def test_conv_single_tap_is_shift_and_modes_are_eigenvectors():
    n = 6
    x = inputs.random_field(n, seed=7)[None]
    W = np.zeros((1, 1, 3, 3, 3))
    W[0, 0, 2, 0, 1] = 1.0          # tap (dz, dy, dx) = (+1, -1, 0)
    out = core.conv3d_fwd(x, W)[0]
    assert np.array_equal(out, core.shift(x[0], (0, 1, -1)))
    # a Fourier mode is scaled by sum_tap W[tap] exp(2 pi i k.tap / n)
    W = inputs.random_weights((1, 1, 3, 3, 3), seed=8)
    k = (1, 2, 1)
    ph = cos_mode(n, k)
    sym = 0.0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                sym += W[0, 0, dz + 1, dy + 1, dx + 1] * np.exp(
                    2j * np.pi * (k[0] * dx + k[1] * dy + k[2] * dz) / n)
    out = core.conv3d_fwd(np.cos(ph)[None], W, np.array([0.5]))[0]
    assert np.max(np.abs(out - (np.real(sym * np.exp(1j * ph)) + 0.5))) < 1e-12


def test_conv_gradients_adjoint_and_finite_difference():
    n, cin, cout = 4, 2, 3
    x = inputs.random_field(n, seed=9)[None].repeat(cin, 0) * np.array([1.0, -0.5])[:, None, None, None]
    x[1] += inputs.random_field(n, seed=10)
    W = inputs.random_weights((cout, cin, 3, 3, 3), seed=11)
    y = inputs.random_weights((cout, n, n, n), seed=12)
    # adjoint (dot-product) identity: <conv(x), y> = <x, dgrad(y)>
    lhs = np.sum(core.conv3d_fwd(x, W) * y)
    rhs = np.sum(x * core.conv3d_dgrad(y, W))
    assert abs(lhs - rhs) < 1e-10 * abs(lhs)
    # weight gradient against central differences of the scalar <conv(x;W,b), y>
    dW, db = core.conv3d_wgrad(x, y)
    eps = 1e-3
    for idx in [(0, 0, 0, 0, 0), (2, 1, 1, 2, 0), (1, 0, 2, 2, 2)]:
        Wp, Wm = W.copy(), W.copy()
        Wp[idx] += eps
        Wm[idx] -= eps
        fd = (np.sum(core.conv3d_fwd(x, Wp) * y) - np.sum(core.conv3d_fwd(x, Wm) * y)) / (2 * eps)
        assert abs(fd - dW[idx]) < 1e-8 * max(1.0, abs(fd))
    b0 = np.zeros(cout)
    bp = b0.copy(); bp[1] = eps
    fd_b = (np.sum(core.conv3d_fwd(x, W, bp) * y) - np.sum(core.conv3d_fwd(x, W, b0) * y)) / eps
    assert abs(fd_b - db[1]) < 1e-8 * max(1.0, abs(fd_b))


def test_gelu_values_and_derivative():
    x = np.array([-3.0, -1.0, 0.0, 0.5, 1.0, 2.0])
    g = core.gelu(x)
    # x * Phi(x) with Phi(1) = 0.8413447460685429, Phi(2) = 0.9772498680518208
    assert abs(g[2]) == 0.0
    assert abs(g[4] - 0.8413447460685429) < 1e-15
    assert abs(g[1] + (1 - 0.8413447460685429)) < 1e-15
    assert abs(g[5] - 2 * 0.9772498680518208) < 1e-15
    eps = 1e-6
    fd = (core.gelu(x + eps) - core.gelu(x - eps)) / (2 * eps)
    assert np.max(np.abs(fd - core.gelu_grad(x))) < 1e-8


# ------------------------------------------------------------- input recipes

def test_input_generators_are_seeded_and_normalised():
    a = inputs.spectral_ic(32, seed=4, kmax=8)
    b = inputs.spectral_ic(32, seed=4, kmax=8)
    assert np.array_equal(a, b)
    assert abs(a.mean()) < 1e-12 and abs(np.sqrt(np.mean(a * a)) - 1.0) < 1e-12
    spec = np.abs(np.fft.fftn(a))
    kk = modal.fft_wavevectors(32)
    kabs = np.sqrt(np.sum(kk ** 2, axis=-1))
    assert np.max(spec[kabs > 8 + 1e-9]) < 1e-9 * np.max(spec)
    m1 = inputs.modes_ic(16, seed=0)
    assert np.array_equal(m1, inputs.modes_ic(16, seed=0))
    ns, nus = inputs.batch_instances(seed=0)
    assert len(ns) == 64 and set(ns) <= {32, 48, 64, 96, 128}
    assert all(0.002 <= v <= 0.02 for v in nus)


def test_difference_form_equals_standard_form_for_a_linear_coarse_propagator():
    """With a linear G, F(U^k[n]) + G(U^{k+1}[n] - U^k[n]) is Eq. (parareal)
    rearranged: both forms agree to rounding at every iteration, and both are
    exact at k = N."""
    n, N = 8, 4
    P = core.Problem(n, a=(1.0, -0.5, 0.25), nu0=0.01, nu_amp=0.5, nu_omega=2 * np.pi)
    F = opr.rk4_propagator(P, 1 / 256, 8)
    G = opr.coarsened_rk4_propagator(P, 2, 1 / 64, 2)
    u0 = inputs.spectral_ic(n, seed=2, kmax=3)
    hs = opr.parareal(F, G, u0, N, N)
    hd = opr.parareal(F, G, u0, N, N, form="difference")
    scale = np.max(np.abs(u0))
    for k in range(N + 1):
        for s in range(N + 1):
            assert np.max(np.abs(hs[k][s] - hd[k][s])) < 1e-13 * scale, (k, s)
    fine = opr.serial_fine(F, u0, N)
    assert np.max(np.abs(hd[N][N] - fine[N])) < 1e-13 * scale


# ------------------------------------------------ spectral transfers (Sec. 2.2.2)

def _band_limited(n, m, seed, count=6):
    """Real field of `count` random modes, every component |k_d| <= m/2 - 1."""
    rng = np.random.default_rng(seed)
    k = rng.integers(-(m // 2 - 1), m // 2, size=(count, 3)).astype(np.float64)
    c = rng.standard_normal(count) + 1j * rng.standard_normal(count)
    return k, c


@pytest.mark.parametrize("n,r", [(16, 2), (24, 3), (32, 4), (32, 8)])
def test_spectral_restriction_samples_band_limited_fields(n, r):
    """A field made of modes both grids represent is restricted to its exact
    values at the coarse points (coarse point I on fine point I r)."""
    from oracle import spectral
    m = n // r
    k, c = _band_limited(n, m, seed=n + r)
    u = modal.field_from_modes(n, k, c)
    assert np.allclose(spectral.restrict_spectral(u, r), u[::r, ::r, ::r], atol=1e-12, rtol=0)


@pytest.mark.parametrize("m,r", [(8, 2), (6, 4), (8, 4)])
def test_spectral_prolongation_is_the_trigonometric_interpolant(m, r):
    """P c sampled on the fine grid equals the coarse field's Fourier series
    evaluated at the fine points, written out mode by mode."""
    from oracle import spectral
    k, cf = _band_limited(m * r, m, seed=3 * m + r)
    c = modal.field_from_modes(m, k, cf)
    assert np.allclose(spectral.prolong_spectral(c, r), modal.field_from_modes(m * r, k, cf),
                       atol=1e-12, rtol=0)


def test_spectral_transfers_drop_unrepresented_modes_and_keep_the_mean():
    from oracle import spectral
    n, r = 16, 4
    m = n // r
    for kx in (m // 2, m // 2 + 1, n // 2):            # the coarse Nyquist mode and beyond
        u = modal.field_from_modes(n, [(kx, 1, 0)], [1.0 + 0.5j])
        assert np.max(np.abs(spectral.restrict_spectral(u, r))) < 1e-13
    u = inputs.random_field(n, seed=4) + 3.25
    assert abs(spectral.restrict_spectral(u, r).mean() - u.mean()) < 1e-13
    c = inputs.random_field(m, seed=5) - 1.5
    assert abs(spectral.prolong_spectral(c, r).mean() - c.mean()) < 1e-13


def test_spectral_restriction_inverts_prolongation_and_projects():
    """R P = identity on coarse fields without Nyquist content; P R is a
    projection (applying it twice changes nothing)."""
    from oracle import spectral
    n, r = 24, 3
    m = n // r
    k, cf = _band_limited(n, m, seed=11)
    c = modal.field_from_modes(m, k, cf)
    assert np.allclose(spectral.restrict_spectral(spectral.prolong_spectral(c, r), r), c,
                       atol=1e-12, rtol=0)
    u = inputs.random_field(n, seed=12)
    pu = spectral.prolong_spectral(spectral.restrict_spectral(u, r), r)
    assert np.allclose(spectral.prolong_spectral(spectral.restrict_spectral(pu, r), r), pu,
                       atol=1e-12, rtol=0)
    assert np.linalg.norm(pu) < np.linalg.norm(u)       # white noise loses its high modes


def test_spectral_coarse_parareal_equals_the_modal_recurrence():
    """With spectral transfers the coarse propagator acts on each fine mode
    the grids share as the coarse RK4 map at the coarse grid's symbol and
    removes every other mode, so Parareal (Eq. parareal) decouples into one
    scalar recurrence per mode.  The field iteration (C stepper on both grids,
    FFT transfers) must equal that recurrence."""
    from oracle import parareal as opr
    from oracle import spectral
    n, r, N, nf, nc = 16, 2, 3, 6, 2
    m = n // r
    a, nu = (1.0, 1.0, 1.0), (0.01, 0.5, 2 * np.pi)
    dt_f, dt_c = 2.0 ** -9, 3 * 2.0 ** -9
    P = core.Problem(n, a=a, nu0=nu[0], nu_amp=nu[1], nu_omega=nu[2])
    F = opr.rk4_propagator(P, dt_f, nf)
    G = opr.spectral_coarsened_rk4_propagator(P, r, dt_c, nc)
    u0 = inputs.random_field(n, seed=21)
    hist = opr.parareal(F, G, u0, N, N)

    k = modal.fft_wavevectors(n).reshape(-1, 3)
    Lf, Df = modal.symbol_parts(n, a, modal.C2, k)
    Lc, Dc = modal.symbol_parts(m, a, modal.C2, k)
    keep = spectral.kept_mask(n, m).ravel()
    Fm = [modal.rk4_multiplier(Lf, Df, s * nf, dt_f, nf, nu) for s in range(N)]
    Gm = [np.where(keep, modal.rk4_multiplier(Lc, Dc, s * nc, dt_c, nc, nu), 0.0) for s in range(N)]
    c0 = np.fft.fftn(u0).ravel()
    mh = modal.modal_parareal(Fm, Gm, c0, N)
    for kk in range(N + 1):
        for s in range(1, N + 1):
            want = np.real(np.fft.ifftn(mh[kk][s].reshape(n, n, n)))
            assert np.max(np.abs(hist[kk][s] - want)) < 1e-12 * np.max(np.abs(want)), (kk, s)
