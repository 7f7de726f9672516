"""Serial Parareal, written out exactly as the paper states it.

TEST INFRASTRUCTURE ONLY (see the package docstring).

Eq. (parareal), Sec. 2.2:
    u_{n+1}^{k+1} = G(u_n^{k+1}) + F(u_n^k) - G(u_n^k),   n = 0 .. N_p - 1,
with the initial guess u_n^0 from one serial run of G (Sec. 2.2 and the
initialisation of Algorithm 1), and u_0^k = u_0 for every k (Algorithm 1,
p = 0).  The three-field sum of the correction (Algorithm 1, "Correction") is
evaluated as F + (G_new - G_old), so that an unchanged input gives an exactly
zero coarse difference.

Propagators are callables ``P(u, n) -> u'`` advancing a field over time slice
n, [t_n, t_{n+1}]; builders for the fine and coarse propagators used by the
tests follow below.
"""
import numpy as np

from . import core, spectral


def serial_fine(F, u0, n_slices):
    """u_fine(t_n) for n = 0..N_p: F applied slice after slice (Eq. fine)."""
    out = [np.array(u0, dtype=np.float64)]
    for n in range(n_slices):
        out.append(F(out[-1], n))
    return out


def parareal(F, G, u0, n_slices, k_max, form="standard"):
    """Return [U^0, U^1, ..., U^{k_max}], each a list of N_p + 1 fields.

    U^k[n] approximates u(t_n) after k Parareal iterations.  form="standard"
    evaluates Eq. (parareal) as printed, F(U^k[n]) + (G(U^{k+1}[n]) - G(U^k[n]));
    form="difference" evaluates F(U^k[n]) + G(U^{k+1}[n] - U^k[n]), the same
    for a linear G.
    """
    u0 = np.array(u0, dtype=np.float64)
    # Initial guess: one serial run of the coarse propagator.
    U = [u0]
    for n in range(n_slices):
        U.append(G(U[n], n))
    G_old = [None] + [U[n + 1] for n in range(n_slices)]   # G(U^0[n]) for slice n
    history = [list(U)]
    for _k in range(k_max):
        # Fine propagator on every slice from the current iterate (parallel part).
        F_val = [None] + [F(U[n], n) for n in range(n_slices)]
        # Coarse propagator and correction, slice after slice (serial part).
        U_new = [u0]
        for n in range(n_slices):
            if form == "difference":
                U_new.append(F_val[n + 1] + G(U_new[n] - U[n], n))
            else:
                g = G(U_new[n], n)
                U_new.append(F_val[n + 1] + (g - G_old[n + 1]))
                G_old[n + 1] = g
        U = U_new
        history.append(list(U))
    return history


def defect(u_k_last, u_fine_last):
    """Relative infinity-norm defect d^k of Eq. (defect)."""
    return float(np.max(np.abs(u_k_last - u_fine_last)) / np.max(np.abs(u_fine_last)))


# ---------------------------------------------------------------- propagators

def rk4_propagator(problem, dt, steps_per_slice, frozen=False):
    """RK4 over one slice: slice n starts at step index n * steps_per_slice."""
    def P(u, n):
        return problem.rk4(u, n * steps_per_slice, dt, steps_per_slice, frozen)
    return P


def euler_propagator(problem, dt, steps_per_slice):
    """Forward Euler over one slice (Algorithm 2, with N_c steps per call)."""
    def P(u, n):
        return problem.euler(u, n * steps_per_slice, dt, steps_per_slice)
    return P


def spectral_coarsened_rk4_propagator(problem, r, dt, steps_per_slice, frozen=False):
    """RK4 on the grid coarsened by r with the spectral transfers (Sec. 2.2.2):
    Fourier restriction, step, Fourier prolongation."""
    coarse = problem.with_n(problem.n // r)

    def P(u, n):
        c = spectral.restrict_spectral(u, r)
        c = coarse.rk4(c, n * steps_per_slice, dt, steps_per_slice, frozen)
        return spectral.prolong_spectral(c, r)
    return P


def coarsened_rk4_propagator(problem, r, dt, steps_per_slice, frozen=False):
    """RK4 on the grid coarsened by r: restrict, step, prolong (Sec. 2.2.2)."""
    coarse = problem.with_n(problem.n // r)

    def P(u, n):
        c = core.restrict_box(u, r)
        c = coarse.rk4(c, n * steps_per_slice, dt, steps_per_slice, frozen)
        return core.prolong_trilinear(c, r)
    return P
