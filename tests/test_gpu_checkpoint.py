"""Checkpoint and resume of the iteration state through the C ABI: a context
restored from a saved state continues bitwise where the saved one would
have; states of another configuration or truncated buffers are rejected."""
import numpy as np
import pytest

from paper_1409_8563_gb300 import configs, native

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def read_all(ctx, cfg):
    buf = torch.empty((cfg.n,) * 3, dtype=torch.float64, device="cuda")
    out = []
    for s in range(cfg.n_slices + 1):
        ctx.get_slice(s, buf)
        out.append(buf.cpu().numpy().copy())
    return out


@pytest.mark.parametrize("r,dtype", [(2, native.F32), (1, native.F64)])
def test_resume_continues_bitwise(r, dtype):
    cfg, u0 = configs.small(n=32, n_slices=5, dtype=dtype, r=r, nf=8, nc=2)
    a = native.Parareal(cfg)
    a.set_problem(torch.from_numpy(u0).cuda())
    a.serial_fine(None, as_reference=True)
    a.iterate(2, 0.0, native.STOP_NONE)
    state = a.save_state()
    ka, ha = a.iterate(2, 0.0, native.STOP_NONE)
    want = read_all(a, cfg)
    b = native.Parareal(cfg)
    b.load_state(state)
    kb, hb = b.iterate(2, 0.0, native.STOP_NONE)
    got = read_all(b, cfg)
    assert ka == kb == 2
    assert np.array_equal(ha[:, :3], hb[:, :3])     # norms and defect (column 3 is wall time)
    for s in range(cfg.n_slices + 1):
        assert np.array_equal(got[s], want[s]), s
    a.close()
    b.close()


def test_foreign_or_truncated_states_are_rejected():
    cfg, u0 = configs.small(n=16, n_slices=3, dtype=native.F32, r=2, nf=8, nc=2)
    a = native.Parareal(cfg)
    with pytest.raises(native.PararealError) as e:
        a.save_state()                       # no problem set yet
    assert e.value.status == native.E_STATE
    a.set_problem(torch.from_numpy(u0).cuda())
    a.iterate(1, 0.0, native.STOP_NONE)
    state = a.save_state()
    other, _ = configs.small(n=16, n_slices=4, dtype=native.F32, r=2, nf=8, nc=2)
    b = native.Parareal(other)
    with pytest.raises(native.PararealError) as e:
        b.load_state(state)
    assert e.value.status == native.E_INVALID
    with pytest.raises(native.PararealError) as e:
        a.load_state(state[: len(state) // 2])
    assert e.value.status == native.E_INVALID
    bad = state.copy()
    bad[0] ^= 0xFF
    with pytest.raises(native.PararealError) as e:
        a.load_state(bad)
    assert e.value.status == native.E_INVALID
    # same sizes, another viscosity history nu(t): a different configuration
    visc, _ = configs.small(n=16, n_slices=3, dtype=native.F32, r=2, nf=8, nc=2)
    visc.nu_omega = 2.0 * visc.nu_omega
    c = native.Parareal(visc)
    with pytest.raises(native.PararealError) as e:
        c.load_state(state)
    assert e.value.status == native.E_INVALID
    c.close()
    a.load_state(state)                      # the context stays usable
    k, _ = a.iterate(1, 0.0, native.STOP_NONE)
    assert k == 1
    a.close()
    b.close()


def test_learned_state_needs_the_weights_it_was_iterated_with():
    """The coarse model's weights are not saved, but their fingerprint is: a
    learned context without a model cannot save or load, and a state iterated
    with other weights is refused."""
    from paper_1409_8563_gb300 import inputs
    cfg, u0 = configs.small(n=16, n_slices=3, dtype=native.F32, nf=8, nc=2)
    cfg.coarse_kind = native.COARSE_LEARNED
    w = inputs.initial_weights(seed=1)
    a = native.Parareal(cfg)
    a.set_problem(torch.from_numpy(u0).cuda())
    with pytest.raises(native.PararealError) as e:
        a.save_state()                       # no model yet
    assert e.value.status == native.E_STATE
    a.set_coarse_model(w)
    a.iterate(1, 0.0, native.STOP_NONE)
    state = a.save_state()
    b = native.Parareal(cfg)
    with pytest.raises(native.PararealError) as e:
        b.load_state(state)                  # no model
    assert e.value.status == native.E_STATE
    w2 = w.copy()
    w2[-1] += 1e-3                           # another model
    b.set_coarse_model(w2)
    with pytest.raises(native.PararealError) as e:
        b.load_state(state)
    assert e.value.status == native.E_STATE
    b.set_coarse_model(w)                    # the same weights: accepted, continues bitwise
    b.load_state(state)
    ka, ha = a.iterate(1, 0.0, native.STOP_NONE)
    kb, hb = b.iterate(1, 0.0, native.STOP_NONE)
    assert ka == kb == 1 and np.array_equal(ha[:, :3], hb[:, :3])
    assert np.array_equal(read_all(a, cfg)[-1], read_all(b, cfg)[-1])
    a.close()
    b.close()
