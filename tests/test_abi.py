"""CPU-side checks of the C ABI: the library loads, exports every symbol the
headers declare, and its host-only logic (validation, stability pre-check)
behaves as documented.  No CUDA computation is launched here."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

from oracle import modal
from paper_1409_8563_gb300 import configs, native
from tests.helpers import ROOT, header_symbols

HERE = os.path.dirname(os.path.abspath(__file__))


def test_library_exports_every_declared_symbol():
    L = native.lib()
    names = header_symbols()
    assert "parareal_create" in names and "parareal_destroy" in names
    for name in sorted(names):
        assert hasattr(L, name), name


def test_binding_names_match_header():
    assert set(native.SIGNATURES) <= header_symbols()
    missing = header_symbols() - set(native.SIGNATURES)
    assert not missing, missing


def test_config_struct_layout_matches_header(tmp_path):
    # parareal_config: 2 ints, 3 doubles, int (+pad), 3 doubles, 3 doubles, 11 ints
    # (+pad to the struct's 8-byte alignment)
    assert ctypes.sizeof(native.Config) == 4 + 4 + 8 * 3 + 8 + 8 * 3 + 8 * 3 + 4 * 11 + 4
    # every field offset as the C compiler lays the header out
    fields = [f for f, _ in native.Config._fields_]
    src = tmp_path / "layout.c"
    src.write_text('#include <stdio.h>\n#include <stddef.h>\n#include "parareal.h"\nint main(void){\n'
                   'printf("%zu\\n", sizeof(parareal_config));\n'
                   + "".join(f'printf("%zu\\n", offsetof(parareal_config, {f}));\n' for f in fields)
                   + "return 0;}\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = [int(v) for v in subprocess.run([str(exe)], capture_output=True, text=True,
                                          check=True).stdout.split()]
    assert got[0] == ctypes.sizeof(native.Config)
    assert got[1:] == [getattr(native.Config, f).offset for f in fields]


def test_stability_precheck_flags_the_literal_unstable_fine_step():
    cfg, _ = configs.fp32_256_literal()
    st, g = native.stability(cfg)
    assert st == native.E_UNSTABLE
    # 7-point diffusion at nu = 0.015, dt = 1/4096, n = 256: z = -2.88 > 2.785
    assert abs(g[0] - 1.15243264) < 1e-6
    cfg, _ = configs.fp32_256()
    st, g = native.stability(cfg)
    assert st == native.OK and g[0] <= 1.0 + 1e-12 and g[1] <= 1.0 + 1e-12


def test_stability_growth_matches_rk4_polynomial_at_nyquist():
    """Growth of the Nyquist corner mode: z = -12 nu n^2 dt (no advection there)."""
    from oracle import modal
    cfg, _ = configs.plain_fp64_32()
    st, g = native.stability(cfg)
    assert st == native.E_UNSTABLE       # accepted only with allow_unstable
    z = -12 * 0.015 * 32 ** 2 / 64
    assert abs(g[1] - abs(modal.rk4_polynomial(z))) < 1e-9


@pytest.mark.parametrize("field,value", [("n", 30), ("n", 4), ("dt_fine", 1 / 1001.0),
                                         ("coarse_factor", 3), ("n_slices", 0),
                                         ("fine_dtype", 7), ("nu_amp", 1.5)])
def test_create_rejects_invalid_configs_before_touching_the_gpu(field, value):
    cfg, _ = configs.small(n=32, n_slices=4)
    setattr(cfg, field, value)
    h = ctypes.c_void_p()
    st = native.lib().parareal_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == native.E_INVALID
    assert h.value is None
    assert native.lib().parareal_last_error(None)


def test_create_rejects_unstable_without_allocating():
    cfg, _ = configs.fp32_256_literal()
    h = ctypes.c_void_p()
    st = native.lib().parareal_create(ctypes.byref(cfg), None, ctypes.byref(h))
    assert st == native.E_UNSTABLE and h.value is None
    assert b"stability" in native.lib().parareal_last_error(None)


def test_batch_dt_rule_is_stable_at_the_extremes():
    for n in (32, 48, 64, 96, 128):
        for nu0 in (0.002, 0.02):
            m = configs.batch_dt_exponent(n, nu0)
            cfg = native.Config.make(n, 8, 1.0, 2.0 ** -m, 16 * 2.0 ** -m, 4, nu0=nu0)
            st, g = native.stability(cfg)
            assert st == native.OK, (n, nu0, g)


def test_paper_scheme_stability_precheck_matches_modal_symbols():
    """The library's pre-check equals max |R(dt lambda)| over the modes, with
    lambda from the oracle's symbols of the C4 and upwind operators."""
    cfg, _ = configs.paper_faithful(n=32, n_slices=8, omega=0.0, fine_log2=12, coarse_log2=8)
    st, g = native.stability(cfg)
    k = np.stack(np.meshgrid(*[np.arange(32)] * 3, indexing="ij"), -1).reshape(-1, 3)
    nus = cfg.nu0 * np.array([0.5, 0.75, 1.0, 1.25, 1.5])     # nu0 (1 +- 0.5) and between
    Lf, Df = modal.symbol_parts(32, tuple(cfg.a), modal.C4, k)
    Lg, Dg = modal.symbol_parts(32, tuple(cfg.a), modal.UPWIND, k)
    gf = max(np.max(np.abs(modal.rk4_polynomial(cfg.dt_fine * (nu * Lf + Df)))) for nu in nus)
    gc = max(np.max(np.abs(1 + cfg.dt_coarse * (nu * Lg + Dg))) for nu in nus)
    assert st == native.OK
    assert abs(g[0] - gf) < 1e-12 and abs(g[1] - gc) < 1e-12, (g, gf, gc)
    # an Euler step beyond the diffusive limit (dt |lambda| > 2) is rejected
    cfg, _ = configs.paper_faithful(n=32, n_slices=8, omega=0.0, fine_log2=12, coarse_log2=5)
    st, g = native.stability(cfg)
    assert st == native.E_UNSTABLE and g[1] > 1.0
    # C4 and Euler/upwind ask for a same-grid G
    cfg, _ = configs.paper_faithful(n=32, n_slices=8)
    cfg.coarse_factor = 2
    assert native.stability(cfg)[0] == native.E_INVALID
