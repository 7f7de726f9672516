"""Thin ctypes binding of the C ABI in include/parareal.h.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Field arguments may be CUDA torch tensors (passed as device
pointers) or numpy arrays (passed as host pointers; the library copies them).
Loading fails loudly when libparareal.so is missing: there is no fallback.
"""
import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libparareal.so")

OK, W_MARGINAL = 0, 1
E_INVALID, E_UNSTABLE, E_NOMEM, E_CUDA, E_DIVERGED, E_TIMEOUT, E_STATE = -1, -2, -3, -4, -5, -6, -7
F32, F64 = 0, 1
MEM_DEVICE, MEM_HOST = 0, 1
NU_STAGE, NU_FROZEN = 0, 1
COARSE_STENCIL, COARSE_LEARNED, COARSE_SHIFT, COARSE_EULER_UPWIND = 0, 1, 2, 3
SCHEME_C2, SCHEME_C4 = 0, 1
ACT_GELU, ACT_LINEAR = 0, 1
CORRECTION_STANDARD, CORRECTION_DIFFERENCE = 0, 1
EVAL_LAYERS, EVAL_COMPOSED, EVAL_POLYPHASE = 0, 1, 2
SKIP_SHIFT, SKIP_STENCIL = 0, 1
TRANSFER_BOX, TRANSFER_SPECTRAL = 0, 1
STOP_DIFF, STOP_DEFECT, STOP_NONE = 0, 1, 2
RES_DIFF_INF, RES_DIFF_L2, RES_FINE, RES_DEFECT, RES_FINE_L2 = 0, 1, 2, 3, 4

_STATUS = {0: "OK", 1: "W_MARGINAL", -1: "E_INVALID", -2: "E_UNSTABLE", -3: "E_NOMEM",
           -4: "E_CUDA", -5: "E_DIVERGED", -6: "E_TIMEOUT", -7: "E_STATE"}


class PararealError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class Config(ctypes.Structure):
    """Mirror of parareal_config."""
    _fields_ = [("n", ctypes.c_int), ("n_slices", ctypes.c_int), ("T", ctypes.c_double),
                ("dt_fine", ctypes.c_double), ("dt_coarse", ctypes.c_double),
                ("coarse_factor", ctypes.c_int), ("a", ctypes.c_double * 3),
                ("nu0", ctypes.c_double), ("nu_amp", ctypes.c_double),
                ("nu_omega", ctypes.c_double), ("fine_dtype", ctypes.c_int),
                ("nu_mode", ctypes.c_int), ("coarse_kind", ctypes.c_int),
                ("allow_unstable", ctypes.c_int), ("learned_skip", ctypes.c_int),
                ("fine_scheme", ctypes.c_int), ("learned_act", ctypes.c_int),
                ("correction_form", ctypes.c_int), ("learned_eval", ctypes.c_int),
                ("coarse_transfer", ctypes.c_int), ("pipeline_blocks", ctypes.c_int)]

    @classmethod
    def make(cls, n, n_slices, T, dt_fine, dt_coarse, coarse_factor=1, a=(1.0, 1.0, 1.0),
             nu0=0.01, nu_amp=0.5, nu_omega=2 * np.pi, fine_dtype=F32, nu_mode=NU_STAGE,
             coarse_kind=COARSE_STENCIL, allow_unstable=0, learned_skip=0, fine_scheme=SCHEME_C2,
             learned_act=ACT_GELU, correction_form=CORRECTION_STANDARD, learned_eval=EVAL_LAYERS,
             coarse_transfer=0, pipeline_blocks=0):
        return cls(int(n), int(n_slices), float(T), float(dt_fine), float(dt_coarse),
                   int(coarse_factor), (ctypes.c_double * 3)(*a), float(nu0), float(nu_amp),
                   float(nu_omega), int(fine_dtype), int(nu_mode), int(coarse_kind),
                   int(allow_unstable), int(learned_skip), int(fine_scheme), int(learned_act),
                   int(correction_form), int(learned_eval), int(coarse_transfer),
                   int(pipeline_blocks))


MODEL_PARAMS = 15169
NOALLOC_MAX_COUNT = 1 << 26     # PARAREAL_NOALLOC_MAX_COUNT


class TrainConfig(ctypes.Structure):
    """Mirror of parareal_train_config."""
    _fields_ = [("epochs", ctypes.c_int), ("batch", ctypes.c_int), ("lr", ctypes.c_double),
                ("beta1", ctypes.c_double), ("beta2", ctypes.c_double), ("eps", ctypes.c_double),
                ("seed", ctypes.c_ulonglong)]


_lib = None

# name -> (restype, argtypes)
_vp, _cp, _i, _d, _dp, _ip = (ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int, ctypes.c_double,
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int))
SIGNATURES = {
    "parareal_create": (_i, [ctypes.POINTER(Config), _vp, ctypes.POINTER(_vp)]),
    "parareal_cluster_size": (_i, [_i, _i]),
    "parareal_stability": (_i, [ctypes.POINTER(Config), _dp]),
    "parareal_set_problem": (_i, [_vp, _vp, _i, _i]),
    "parareal_fine_sweep": (_i, [_vp, _i, _i]),
    "parareal_coarse_sweep": (_i, [_vp, _i, _i, _i]),
    "parareal_iterate": (_i, [_vp, _i, _d, _i, _ip, _dp]),
    "parareal_iterate_device": (_i, [_vp, _i, _d, _i, _ip, _dp]),
    "parareal_residual": (_i, [_vp, _i, _dp]),
    "parareal_set_reference": (_i, [_vp, _vp, _i, _i]),
    "parareal_serial_fine": (_i, [_vp, _vp, _i, _i, _i]),
    "parareal_get_slice": (_i, [_vp, _i, _vp, _i, _i]),
    "parareal_set_slice": (_i, [_vp, _i, _vp, _i, _i]),
    "parareal_propagate": (_i, [_vp, _i, _vp, _vp, _i, _i, _i]),
    "parareal_set_coarse_model": (_i, [_vp, _vp, _i]),
    "parareal_get_coarse_model": (_i, [_vp, _vp, _i]),
    "parareal_make_pairs": (_i, [_vp, _vp, _i, _vp, _vp, _ip]),
    "parareal_train_coarse": (_i, [_vp, _vp, _vp, _ip, _i, _vp, _dp]),
    "parareal_coarse_model_grad": (_i, [_vp, _vp, _vp, _ip, _i, _vp, _dp]),
    "parareal_autotune": (_i, [_vp, _cp, _dp]),
    "parareal_get_launch_shape": (_i, [_vp, _ip, _ip, _ip]),
    "parareal_batch_create": (_i, [ctypes.POINTER(Config), _i, _vp, ctypes.POINTER(_vp)]),
    "parareal_batch_set_problem": (_i, [_vp, _i, _vp, _i, _i]),
    "parareal_batch_serial_fine": (_i, [_vp, _i]),
    "parareal_batch_iterate": (_i, [_vp, _i, _d, _i, _ip, _dp]),
    "parareal_batch_autotune": (_i, [_vp, _cp]),
    "parareal_batch_set_fine_mode": (_i, [_vp, _i, _i, _i, _i]),
    "parareal_batch_get_fine_mode": (_i, [_vp, _ip]),
    "parareal_batch_context": (_vp, [_vp, _i]),
    "parareal_batch_graph_launches": (ctypes.c_longlong, [_vp]),
    "parareal_batch_last_error": (_cp, [_vp]),
    "parareal_batch_destroy": (None, [_vp]),
    "parareal_diff_norms_noalloc": (_i, [_vp, _vp, ctypes.c_longlong, _vp, _vp]),
    "parareal_noalloc_last_error": (_cp, []),
    "parareal_profile": (_i, [_vp, _i]),
    "parareal_profile_read": (_i, [_vp, _dp, ctypes.POINTER(ctypes.c_longlong), _dp]),
    "parareal_launch_count": (ctypes.c_longlong, [_vp]),
    "parareal_selftest_timeout": (_i, [_vp]),
    "parareal_selftest_grid_barrier": (_i, [_vp]),
    "parareal_save_state": (_i, [_vp, _vp, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]),
    "parareal_load_state": (_i, [_vp, _vp, ctypes.c_size_t]),
    "parareal_last_error": (_cp, [_vp]),
    "parareal_destroy": (None, [_vp]),
}


def lib():
    """Open libparareal.so (once).  Raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: run __graft_entry__.build() (no CPU fallback)")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _field(x):
    """(pointer, dtype code, mem code, keepalive) for a torch tensor or numpy array."""
    if isinstance(x, np.ndarray):
        if not x.flags.c_contiguous:
            raise ValueError("numpy field must be C-contiguous")
        code = {np.dtype(np.float32): F32, np.dtype(np.float64): F64}[x.dtype]
        return ctypes.c_void_p(x.ctypes.data), code, MEM_HOST, x
    import torch
    if not isinstance(x, torch.Tensor):
        raise TypeError("field must be a numpy array or a torch tensor")
    if not x.is_contiguous():
        raise ValueError("tensor must be contiguous")
    code = {torch.float32: F32, torch.float64: F64}[x.dtype]
    mem = MEM_DEVICE if x.is_cuda else MEM_HOST
    return ctypes.c_void_p(x.data_ptr()), code, mem, x


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def selftest_grid_barrier(stream=None):
    """Run the persistent kernel's bounded grid-barrier self-test; returns the status."""
    return int(lib().parareal_selftest_grid_barrier(_stream_ptr(stream)))


def selftest_timeout(stream=None):
    """Run the bounded device-side wait on a barrier nothing arrives on;
    returns its status (E_TIMEOUT when the wait gave up as designed)."""
    return int(lib().parareal_selftest_timeout(_stream_ptr(stream)))


def stability(cfg):
    g = (ctypes.c_double * 2)()
    st = lib().parareal_stability(ctypes.byref(cfg), g)
    return st, (g[0], g[1])


def cluster_size(dtype, n):
    """CTAs of the cluster that holds one n^3 field in launch path 4 (0: does not fit)."""
    return int(lib().parareal_cluster_size(int(dtype), int(n)))


class Parareal:
    """One context of the C library (parareal_create ... parareal_destroy)."""

    def __init__(self, cfg, stream=None):
        self.cfg = cfg
        h = ctypes.c_void_p()
        st = lib().parareal_create(ctypes.byref(cfg), _stream_ptr(stream), ctypes.byref(h))
        if st < 0:
            raise PararealError(st, lib().parareal_last_error(None).decode())
        self.status = st
        self._h = h

    def _check(self, st):
        if st < 0:
            raise PararealError(st, lib().parareal_last_error(self._h).decode())
        return st

    def set_problem(self, u0):
        p, code, mem, _k = _field(u0)
        return self._check(lib().parareal_set_problem(self._h, p, code, mem))

    def set_reference(self, ref):
        p, code, mem, _k = _field(ref)
        return self._check(lib().parareal_set_reference(self._h, p, code, mem))

    def fine_sweep(self, first, count):
        return self._check(lib().parareal_fine_sweep(self._h, first, count))

    def coarse_sweep(self, first, count, chain=1):
        return self._check(lib().parareal_coarse_sweep(self._h, first, count, chain))

    def iterate(self, k_max, tol=0.0, stop_rule=STOP_NONE, device=False):
        """Run up to k_max iterations; device=True runs them as one CUDA graph
        launch with the stopping test on the device (parareal_iterate_device)."""
        k = ctypes.c_int()
        hist = (ctypes.c_double * (4 * max(k_max, 1)))()
        fn = lib().parareal_iterate_device if device else lib().parareal_iterate
        self._check(fn(self._h, k_max, tol, stop_rule, ctypes.byref(k), hist))
        h = np.array(hist[:4 * k.value]).reshape(k.value, 4)
        return k.value, h

    def residual(self, kind):
        out = (ctypes.c_double * (self.cfg.n_slices + 1))()
        self._check(lib().parareal_residual(self._h, kind, out))
        return np.array(out[:])

    def serial_fine(self, dst=None, as_reference=True):
        if dst is None:
            self._check(lib().parareal_serial_fine(self._h, None, F64, MEM_DEVICE, int(as_reference)))
            return None
        p, code, mem, _k = _field(dst)
        return self._check(lib().parareal_serial_fine(self._h, p, code, mem, int(as_reference)))

    def get_slice(self, s, dst):
        p, code, mem, _k = _field(dst)
        return self._check(lib().parareal_get_slice(self._h, s, p, code, mem))

    def set_slice(self, s, src):
        p, code, mem, _k = _field(src)
        return self._check(lib().parareal_set_slice(self._h, s, p, code, mem))

    def propagate(self, which, src, dst, first, count):
        ps, code, mem, _k1 = _field(src)
        pd, code2, mem2, _k2 = _field(dst)
        if code != code2 or mem != MEM_DEVICE or mem2 != MEM_DEVICE:
            raise ValueError("propagate needs device tensors of one dtype")
        return self._check(lib().parareal_propagate(self._h, which, ps, pd, code, first, count))

    # ------------------------------------------------ learned coarse propagator

    def set_coarse_model(self, w):
        """w: MODEL_PARAMS float32 values (numpy host array or CUDA tensor)."""
        p, code, mem, _k = _field(w)
        if code != F32:
            raise ValueError("model weights are float32")
        return self._check(lib().parareal_set_coarse_model(self._h, p, mem))

    def get_coarse_model(self):
        out = np.empty(MODEL_PARAMS, dtype=np.float32)
        self._check(lib().parareal_get_coarse_model(self._h, ctypes.c_void_p(out.ctypes.data), MEM_HOST))
        return out

    def make_pairs(self, ics, pairs_u, pairs_f):
        """ics: [n_ics, n, n, n] float32 CUDA tensor; pairs_*: [n_ics*N, m, m, m]
        float32 CUDA tensors.  Returns the slice index of every pair."""
        n_ics = ics.shape[0]
        sl = (ctypes.c_int * (n_ics * self.cfg.n_slices))()
        self._check(lib().parareal_make_pairs(self._h, ctypes.c_void_p(ics.data_ptr()), n_ics,
                                              ctypes.c_void_p(pairs_u.data_ptr()),
                                              ctypes.c_void_p(pairs_f.data_ptr()), sl))
        return np.array(sl[:], dtype=np.int32)

    def train_coarse(self, pairs_u, pairs_f, pair_slice, epochs, batch, lr=1e-3, beta1=0.9,
                     beta2=0.999, eps=1e-8, seed=0):
        tc = TrainConfig(int(epochs), int(batch), float(lr), float(beta1), float(beta2), float(eps),
                         int(seed))
        n = len(pair_slice)
        sl = (ctypes.c_int * n)(*[int(v) for v in pair_slice])
        hist = (ctypes.c_double * max(1, epochs))()
        self._check(lib().parareal_train_coarse(self._h, ctypes.c_void_p(pairs_u.data_ptr()),
                                                ctypes.c_void_p(pairs_f.data_ptr()), sl, n,
                                                ctypes.byref(tc), hist))
        return np.array(hist[:epochs])

    def coarse_model_grad(self, u, target, slices, grad_out):
        n = len(slices)
        sl = (ctypes.c_int * n)(*[int(v) for v in slices])
        loss = ctypes.c_double()
        self._check(lib().parareal_coarse_model_grad(self._h, ctypes.c_void_p(u.data_ptr()),
                                                     ctypes.c_void_p(target.data_ptr()), sl, n,
                                                     ctypes.c_void_p(grad_out.data_ptr()),
                                                     ctypes.byref(loss)))
        return loss.value

    def save_state(self):
        """The iteration state as a bytes-like numpy uint8 array (host)."""
        need = ctypes.c_size_t()
        self._check(lib().parareal_save_state(self._h, None, 0, ctypes.byref(need)))
        buf = np.empty(need.value, dtype=np.uint8)
        self._check(lib().parareal_save_state(self._h, ctypes.c_void_p(buf.ctypes.data), buf.nbytes,
                                              ctypes.byref(need)))
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        return self._check(lib().parareal_load_state(self._h, ctypes.c_void_p(buf.ctypes.data), buf.nbytes))

    def autotune(self, cache_path=None):
        """Time the launch shapes and keep the fastest (call before set_problem)."""
        ms = (ctypes.c_double * 2)()
        cp = cache_path.encode() if cache_path else None
        self._check(lib().parareal_autotune(self._h, cp, ms))
        return ms[0], ms[1]

    def launch_shape(self):
        """(batched fine sweep, coarse steps, single fine field) launch shapes."""
        f, c, s = (ctypes.c_int * 4)(), (ctypes.c_int * 4)(), (ctypes.c_int * 4)()
        self._check(lib().parareal_get_launch_shape(self._h, f, c, s))
        return tuple(f[:]), tuple(c[:]), tuple(s[:])

    def profile(self, enable=True):
        return self._check(lib().parareal_profile(self._h, int(enable)))

    def profile_read(self):
        """(device ms, launches, algorithmic bytes) of the timed fine-kernel launches."""
        ms, nl, by = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
        self._check(lib().parareal_profile_read(self._h, ctypes.byref(ms), ctypes.byref(nl),
                                                ctypes.byref(by)))
        return ms.value, nl.value, by.value

    def launch_count(self):
        return int(lib().parareal_launch_count(self._h))

    def close(self):
        if self._h:
            lib().parareal_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class _View(Parareal):
    """A context owned by a Batch (not destroyed by this object)."""

    def __init__(self, handle, cfg):  # noqa: D401 - no parareal_create here
        self.cfg = cfg
        self.status = OK
        self._h = ctypes.c_void_p(handle)

    def close(self):
        self._h = None


class Batch:
    """Independent problems of uneven sizes advanced together (parareal_batch_*)."""

    def __init__(self, cfgs, stream=None):
        self.cfgs = list(cfgs)
        arr = (Config * len(self.cfgs))(*self.cfgs)
        h = ctypes.c_void_p()
        st = lib().parareal_batch_create(arr, len(self.cfgs), _stream_ptr(stream), ctypes.byref(h))
        if st < 0:
            raise PararealError(st, lib().parareal_last_error(None).decode())
        self._h = h

    def _check(self, st):
        if st < 0:
            raise PararealError(st, lib().parareal_batch_last_error(self._h).decode())
        return st

    def context(self, i):
        return _View(lib().parareal_batch_context(self._h, i), self.cfgs[i])

    def set_problem(self, i, u0):
        p, code, mem, _k = _field(u0)
        return self._check(lib().parareal_batch_set_problem(self._h, i, p, code, mem))

    def serial_fine(self, as_reference=True):
        return self._check(lib().parareal_batch_serial_fine(self._h, int(as_reference)))

    def iterate(self, k_max, tol=0.0, stop_rule=STOP_NONE):
        M = len(self.cfgs)
        k = (ctypes.c_int * M)()
        d = (ctypes.c_double * M)()
        self._check(lib().parareal_batch_iterate(self._h, k_max, tol, stop_rule, k, d))
        return np.array(k[:]), np.array(d[:])

    def autotune(self, cache_path=None):
        cp = cache_path.encode() if cache_path else None
        return self._check(lib().parareal_batch_autotune(self._h, cp))

    def graph_launches(self):
        return int(lib().parareal_batch_graph_launches(self._h))

    def set_fine_mode(self, mode, tile_x=64, tile_y=32, rows=1):
        """mode 0: per-instance launches in graph branches; 1: one persistent
        launch over a queue of every instance's tile steps."""
        return self._check(lib().parareal_batch_set_fine_mode(self._h, mode, tile_x, tile_y, rows))

    def fine_mode(self):
        m = (ctypes.c_int * 4)()
        self._check(lib().parareal_batch_get_fine_mode(self._h, m))
        return tuple(m[:])

    def close(self):
        if self._h:
            lib().parareal_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
