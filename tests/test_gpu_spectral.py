"""GPU parity of the stencil coarse propagator with spectral transfers
(coarse_transfer SPECTRAL, Sec. 2.2.2) through the C ABI.

With spectral restriction and prolongation the coarse propagator acts on
every Fourier mode both grids share as the coarse RK4 map at the coarse
grid's symbol and removes all other modes, so Parareal decouples into one
scalar recurrence per mode (oracle.modal): the GPU iterates are compared
with the field oracle (C stepper, FFT transfers) and with that recurrence.
Tolerances: relative L2 1e-5 for FP32 paths, 1e-12 for FP64 paths.
"""
import numpy as np
import pytest

from oracle import modal, spectral
from oracle import parareal as opr
from paper_1409_8563_gb300 import configs, inputs, native
from tests.helpers import TOL, oracle_F, oracle_problem, rel_l2, steps, tile_env

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

F32, F64 = native.F32, native.F64


def spectral_cfg(n, N, dtype, r, nf=8, nc=2):
    cfg, u0 = configs.small(n=n, n_slices=N, dtype=dtype, r=r, nf=nf, nc=nc)
    cfg.coarse_transfer = native.TRANSFER_SPECTRAL
    return cfg, u0


def oracle_G_spectral(cfg):
    _, nc = steps(cfg)
    return opr.spectral_coarsened_rk4_propagator(oracle_problem(cfg), cfg.coarse_factor,
                                                 cfg.dt_coarse, nc)


def read_all(ctx, cfg):
    buf = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    out = []
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, buf)
        out.append(buf.cpu().numpy().copy())
    return out


@pytest.mark.parametrize("n,dtype,r", [(32, F32, 2), (64, F32, 4), (64, F32, 8), (48, F32, 4),
                                       (32, F64, 4), (16, F64, 2)])
def test_spectral_coarse_propagator_matches_oracle(monkeypatch, n, dtype, r):
    tile_env(monkeypatch)
    cfg, _ = spectral_cfg(n, 2, dtype, r)
    ctx = native.Parareal(cfg)
    src = np.stack([inputs.random_field(n, seed=80 + s) + inputs.spectral_ic(n, seed=90 + s, kmax=4)
                    for s in range(2)])
    t = torch.float64 if dtype == F64 else torch.float32
    dsrc = torch.from_numpy(src).to("cuda", t)
    ddst = torch.empty_like(dsrc)
    ctx.propagate(1, dsrc, ddst, 0, 2)
    got = ddst.double().cpu().numpy()
    G = oracle_G_spectral(cfg)
    for s in range(2):
        # the oracle sees the field the GPU sees (rounded to G's precision on input)
        x = src[s].astype(np.float32).astype(np.float64) if dtype == F32 else src[s]
        ref = G(x, s)
        assert rel_l2(got[s], ref) < TOL[dtype], (s, rel_l2(got[s], ref))
    ctx.close()


@pytest.mark.parametrize("n,dtype,r,N,form", [(32, F32, 2, 4, native.CORRECTION_STANDARD),
                                              (32, F32, 4, 4, native.CORRECTION_DIFFERENCE),
                                              (16, F64, 2, 3, native.CORRECTION_STANDARD)])
def test_spectral_parareal_iterates_match_oracle_and_modal_recurrence(monkeypatch, n, dtype, r, N,
                                                                      form):
    tile_env(monkeypatch)
    cfg, u0 = spectral_cfg(n, N, dtype, r, nf=8, nc=2)
    cfg.correction_form = form
    nf, nc = steps(cfg)
    ctx = native.Parareal(cfg)
    ctx.set_problem(torch.from_numpy(u0).cuda())
    hist = opr.parareal(oracle_F(cfg), oracle_G_spectral(cfg), u0, N, N)
    # the per-mode recurrence
    m = n // r
    a, nu = tuple(cfg.a), (cfg.nu0, cfg.nu_amp, cfg.nu_omega)
    k = modal.fft_wavevectors(n).reshape(-1, 3)
    Lf, Df = modal.symbol_parts(n, a, modal.C2, k)
    Lc, Dc = modal.symbol_parts(m, a, modal.C2, k)
    keep = spectral.kept_mask(n, m).ravel()
    Fm = [modal.rk4_multiplier(Lf, Df, s * nf, cfg.dt_fine, nf, nu) for s in range(N)]
    Gm = [np.where(keep, modal.rk4_multiplier(Lc, Dc, s * nc, cfg.dt_coarse, nc, nu), 0.0)
          for s in range(N)]
    mh = modal.modal_parareal(Fm, Gm, np.fft.fftn(u0).ravel(), N)
    for kk in range(N + 1):
        if kk > 0:
            kd, _ = ctx.iterate(1, 0.0, native.STOP_NONE)
            assert kd == 1
        else:
            ctx.iterate(0, 0.0, native.STOP_NONE)
        got = read_all(ctx, cfg)
        for s in range(1, N + 1):
            e = rel_l2(got[s], hist[kk][s])
            assert e < TOL[dtype], (kk, s, e)
            want = np.real(np.fft.ifftn(mh[kk][s].reshape(n, n, n)))
            e2 = rel_l2(got[s], want)
            assert e2 < TOL[dtype], (kk, s, e2)
    ctx.close()


def test_spectral_parareal_reaches_serial_fine_exactly_at_k_equals_n(monkeypatch):
    tile_env(monkeypatch)
    n, N = 32, 4
    cfg, u0 = spectral_cfg(n, N, F32, 4)
    ctx = native.Parareal(cfg)
    ctx.set_problem(torch.from_numpy(u0).cuda())
    fine = torch.empty((n,) * 3, dtype=torch.float64, device="cuda")
    ctx.serial_fine(fine, as_reference=True)
    kd, h = ctx.iterate(N, 0.0, native.STOP_NONE)
    assert kd == N and h[-1, 2] == 0.0
    last = torch.empty_like(fine)
    ctx.get_slice(N, last)
    assert torch.equal(last, fine)
    ctx.close()


def test_spectral_transfer_configuration_is_checked():
    for mutate in (lambda c: setattr(c, "coarse_factor", 1),
                   lambda c: setattr(c, "coarse_kind", native.COARSE_LEARNED),
                   lambda c: setattr(c, "coarse_transfer", 2)):
        cfg, _ = spectral_cfg(32, 2, F32, 2)
        mutate(cfg)
        with pytest.raises(native.PararealError) as e:
            native.Parareal(cfg)
        assert e.value.status == native.E_INVALID
