"""Workload presets: the benchmark configurations with their readings made
explicit (host-side data only; no arithmetic of the method).

Each preset returns ``(config, u0)`` where ``config`` is a native.Config and
``u0`` a float64 [z][y][x] numpy array from ``inputs``.

  plain_fp64_32      32^3, FP64, T = 1, N = 8, dt_F = 1/1024, same-grid
                     RK4 coarse propagator at dt_G = 1/64 (growth 1.15/step
                     for the Nyquist band at nu > 0.0145, kept verbatim and
                     accepted as a warning), 8-mode initial condition.
  fp32_256           256^3, FP32 stencil / FP64 correction, N = 32, T = 1,
                     dt_F = 1/8192 (1/4096 is unstable for nu > 0.0145), coarse
                     propagator = RK4 on 32^3 (box restriction by 8, trilinear
                     prolongation) at dt_G = 1/256, k^-2 random field to k = 32.
  fp32_128           128^3, N = 32, dt_F = 1/2048, coarse RK4 on 32^3 at 1/256.
  fp32_512           512^3, N = 16, dt_F = 1/32768, coarse RK4 on 64^3 at 1/512.
  batch_instance     one of the 64 uneven problems: T = 1, N = 8, dt_F = 2^-m
                     with m = max(10, ceil(log2(12 nu0 n^2))), coarse RK4 on
                     n/4 at 16 dt_F.
  paper_128          the paper's own run (Sec. 3.1) on the 7-point/centred
                     scheme: 128^3, nu0 = 0.1, omega = 100, T = 0.1,
                     dt_F = T/2^15, dt_G = T/2^11 on the same grid, frozen nu.
"""
import math

import numpy as np

from . import inputs
from .native import (COARSE_EULER_UPWIND, COARSE_STENCIL, F32, F64, NU_FROZEN, NU_STAGE, SCHEME_C4,
                     Config, stability)

NU_BASE = dict(nu0=0.01, nu_amp=0.5, nu_omega=2 * math.pi)


def plain_fp64_32(seed=0):
    cfg = Config.make(32, 8, 1.0, 1 / 1024, 1 / 64, 1, fine_dtype=F64, allow_unstable=1, **NU_BASE)
    return cfg, inputs.modes_ic(32, seed=seed)


def fp32_256(seed=0):
    cfg = Config.make(256, 32, 1.0, 1 / 8192, 1 / 256, 8, fine_dtype=F32, **NU_BASE)
    return cfg, inputs.spectral_ic(256, seed=seed, kmax=32)


def fp32_256_literal(seed=0):
    """The literal dt_F = 1/4096 (rejected by the stability pre-check)."""
    cfg = Config.make(256, 32, 1.0, 1 / 4096, 1 / 256, 8, fine_dtype=F32, **NU_BASE)
    return cfg, None


def fp32_128(seed=0):
    cfg = Config.make(128, 32, 1.0, 1 / 2048, 1 / 256, 4, fine_dtype=F32, **NU_BASE)
    return cfg, inputs.spectral_ic(128, seed=seed, kmax=32)


def fp32_512(seed=0):
    cfg = Config.make(512, 16, 1.0, 1 / 32768, 1 / 512, 8, fine_dtype=F32, **NU_BASE)
    return cfg, inputs.spectral_ic(512, seed=seed, kmax=32)


def batch_dt_exponent(n, nu0):
    return max(10, math.ceil(math.log2(12.0 * nu0 * n * n)))


def batch_instance(n, nu0, seed=0):
    m = batch_dt_exponent(n, nu0)
    cfg = Config.make(n, 8, 1.0, 2.0 ** -m, 16 * 2.0 ** -m, 4, fine_dtype=F32,
                      nu0=nu0, nu_amp=0.5, nu_omega=2 * math.pi)
    return cfg, inputs.spectral_ic(n, seed=seed, kmax=n // 8)


def paper_128(omega=100.0):
    T = 0.1
    cfg = Config.make(128, 32, T, T / 2 ** 15, T / 2 ** 11, 1, fine_dtype=F64, nu0=0.1,
                      nu_amp=0.5, nu_omega=omega, nu_mode=NU_FROZEN, allow_unstable=1)
    return cfg, inputs.paper_ic(128)


def paper_faithful(n=128, n_slices=8, omega=0.0, fine_log2=15, coarse_log2=11, dtype=F64,
                   a=(1.0, 1.0, 1.0)):
    """The paper's own configuration (Sec. 3.1): T = 0.1, nu0 = 0.1,
    nu(t) = nu0 (1 + 0.5 sin(omega t)) frozen at the step start, a = (1, 1, 1);
    F = RK4 with fourth-order centred differences at T/2^fine_log2, G = forward
    Euler with upwind advection at T/2^coarse_log2 on the same grid (Algorithm 2);
    u0 = sin(2 pi x) sin(2 pi y) sin(2 pi z)."""
    T = 0.1
    cfg = Config.make(n, n_slices, T, T / 2 ** fine_log2, T / 2 ** coarse_log2, 1, a=a, nu0=0.1,
                      nu_amp=0.5, nu_omega=omega, fine_dtype=dtype, nu_mode=NU_FROZEN,
                      coarse_kind=COARSE_EULER_UPWIND, fine_scheme=SCHEME_C4)
    return cfg, inputs.paper_ic(n)


def small(n=32, n_slices=4, dtype=F64, r=1, nf=32, nc=4, seed=0, ic="spectral"):
    """A small stable configuration for parity tests: N slices of nf fine
    steps with dt_F = 2^-m, z = 12 nu_max n^2 dt_F <= 1.5 on the fine grid;
    nc is raised until the coarse step obeys the same bound on the coarse grid."""
    nu_max = NU_BASE["nu0"] * (1 + NU_BASE["nu_amp"])
    m = max(6, math.ceil(math.log2(12.0 * nu_max * n * n / 1.5)))
    dt_f = 2.0 ** -m
    slice_len = nf * dt_f
    nco = n // r
    need = math.ceil(12.0 * nu_max * nco * nco * slice_len / 1.5 - 1e-9)
    nc = min(max(nc, need, 1), nf)
    while True:
        while nf % nc:      # ends at nc = nf at the latest
            nc += 1
        cfg = Config.make(n, n_slices, n_slices * slice_len, dt_f, slice_len / nc, r,
                          fine_dtype=dtype, **NU_BASE)
        # advection can destabilise a step that diffusion alone allows
        if nc >= nf or stability(cfg)[0] == 0:
            break
        nc += 1
    if ic == "spectral":
        u0 = inputs.spectral_ic(n, seed=seed, kmax=max(2, n // 8))
    else:
        u0 = inputs.modes_ic(n, seed=seed)
    return cfg, u0


def as_dict(cfg):
    return {"n": cfg.n, "n_slices": cfg.n_slices, "T": cfg.T, "dt_fine": cfg.dt_fine,
            "dt_coarse": cfg.dt_coarse, "coarse_factor": cfg.coarse_factor,
            "a": list(cfg.a), "nu0": cfg.nu0, "nu_amp": cfg.nu_amp, "nu_omega": cfg.nu_omega,
            "dtype": "f64" if cfg.fine_dtype == F64 else "f32",
            "nu_mode": "frozen" if cfg.nu_mode == NU_FROZEN else "stage"}


__all__ = ["plain_fp64_32", "fp32_256", "fp32_256_literal", "fp32_128", "fp32_512",
           "batch_instance", "batch_dt_exponent", "paper_128", "small", "as_dict",
           "COARSE_STENCIL", "NU_STAGE", "np"]
