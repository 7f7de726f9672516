"""Shared test helpers: oracle propagators built from a native Config, and
field comparisons.  (Test infrastructure: may import the oracle.)"""
import math
import re
import os

import numpy as np

from oracle import core
from oracle import parareal as opr

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def steps(cfg):
    sl = cfg.T / cfg.n_slices
    return int(round(sl / cfg.dt_fine)), int(round(sl / cfg.dt_coarse))


def oracle_problem(cfg, n=None, scheme=None):
    if scheme is None:
        scheme = core.C4 if getattr(cfg, "fine_scheme", 0) == 1 else core.C2
    return core.Problem(cfg.n if n is None else n, a=tuple(cfg.a), nu0=cfg.nu0,
                        nu_amp=cfg.nu_amp, nu_omega=cfg.nu_omega, scheme=scheme)


def oracle_F(cfg):
    nf, _ = steps(cfg)
    return opr.rk4_propagator(oracle_problem(cfg), cfg.dt_fine, nf, frozen=cfg.nu_mode == 1)


def oracle_G(cfg):
    _, nc = steps(cfg)
    if cfg.coarse_kind == 3:   # forward Euler / upwind on the same grid (Algorithm 2)
        return opr.euler_propagator(oracle_problem(cfg, scheme=core.UPWIND), cfg.dt_coarse, nc)
    P = oracle_problem(cfg, scheme=core.C2)
    if cfg.coarse_factor == 1:
        return opr.rk4_propagator(P, cfg.dt_coarse, nc, frozen=cfg.nu_mode == 1)
    return opr.coarsened_rk4_propagator(P, cfg.coarse_factor, cfg.dt_coarse, nc,
                                        frozen=cfg.nu_mode == 1)


def rel_l2(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((got - ref).ravel()) / np.linalg.norm(ref.ravel()))


def rel_inf(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.max(np.abs(got - ref)) / np.max(np.abs(ref)))


# Tolerances against the FP64 oracle (relative L2 over the whole field).
TOL = {0: 1e-5, 1: 1e-12}   # keyed by fine_dtype: F32 = 0, F64 = 1


def header_symbols():
    """Function names declared in include/*.h."""
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if f.endswith(".h"):
            text = open(os.path.join(inc, f)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(parareal_[a-z0-9_]+)\s*\(", text))
    return names


def tile_env(monkeypatch, fine=None, coarse=None):
    if fine is None:
        monkeypatch.delenv("PARAREAL_FINE_TILE", raising=False)
    else:
        monkeypatch.setenv("PARAREAL_FINE_TILE", ",".join(str(v) for v in fine))
    if coarse is None:
        monkeypatch.delenv("PARAREAL_COARSE_TILE", raising=False)
    else:
        monkeypatch.setenv("PARAREAL_COARSE_TILE", ",".join(str(v) for v in coarse))


__all__ = ["steps", "oracle_problem", "oracle_F", "oracle_G", "rel_l2", "rel_inf", "TOL",
           "header_symbols", "tile_env", "math"]
