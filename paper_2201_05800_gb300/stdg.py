"""Thin ctypes binding of libstdg.so (include/stdg.h): argument marshalling only.

Every computation happens in the CUDA library; this module converts Python
arguments (numpy arrays for host memory, torch CUDA tensors for device memory)
to the C ABI and raises ``StdgError`` on a non-OK status.  There is no CPU
fallback: ``load()`` raises if the library has not been built.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libstdg.so")

ADVECTION, EULER, BURGERS = 0, 1, 2
FLUX_RUSANOV = 0
FP64, MIXED_FP32, MIXED_BF16 = 0, 1, 2
JV_FD, JV_EXACT = 0, 1
HOST, DEVICE = 0, 1
PRECOND_NONE, PRECOND_TEMPORAL_MASS, PRECOND_POINT_BLOCK = 0, 1, 2
PREDICTOR_CONSTANT, PREDICTOR_EXTRAPOLATE = 0, 1

STATUS = {0: "STDG_OK", 1: "STDG_ERR_INVALID_ARG", 2: "STDG_ERR_OOM", 3: "STDG_ERR_CUDA",
          4: "STDG_ERR_NOT_CONVERGED", 5: "STDG_ERR_GMRES_BREAKDOWN", 6: "STDG_ERR_NAN",
          7: "STDG_ERR_TIMEOUT", 8: "STDG_ERR_CANCELLED", 9: "STDG_ERR_UNSUPPORTED"}


class stdg_config_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("cells", ctypes.c_int * 3),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3),
                ("N", ctypes.c_int), ("s", ctypes.c_int), ("equation", ctypes.c_int),
                ("adv_vel", ctypes.c_double * 3), ("gamma", ctypes.c_double), ("flux", ctypes.c_int),
                ("dt", ctypes.c_double), ("precision", ctypes.c_int), ("jv_mode", ctypes.c_int),
                ("newton_rtol", ctypes.c_double), ("newton_atol", ctypes.c_double),
                ("newton_maxit", ctypes.c_int), ("gmres_m", ctypes.c_int),
                ("gmres_rtol", ctypes.c_double), ("gmres_maxit", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t), ("precond", ctypes.c_int),
                ("viscosity", ctypes.c_double), ("penalty", ctypes.c_double),
                ("predictor", ctypes.c_int)]


class stdg_slab_stats(ctypes.Structure):
    _fields_ = [("newton_its", ctypes.c_int), ("gmres_its", ctypes.c_int),
                ("residual_evals", ctypes.c_int), ("jv_evals", ctypes.c_int),
                ("res0", ctypes.c_double), ("res_final", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class stdg_profile(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int * 5), ("ms", ctypes.c_double * 5)]


PROFILE_CLASSES = ("residual", "jv", "gram_schmidt", "other", "precond")


class StdgError(RuntimeError):
    def __init__(self, status, msg=""):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


_lib = None

_P = ctypes.c_void_p
_SIGS = {
    "stdg_config_default": (None, [ctypes.POINTER(stdg_config_desc)]),
    "stdg_create": (ctypes.c_int, [ctypes.POINTER(stdg_config_desc), _P, ctypes.POINTER(_P)]),
    "stdg_destroy": (ctypes.c_int, [_P]),
    "stdg_state_len": (ctypes.c_size_t, [_P]),
    "stdg_slab_len": (ctypes.c_size_t, [_P]),
    "stdg_coord_len": (ctypes.c_size_t, [_P]),
    "stdg_device_bytes": (ctypes.c_size_t, [_P]),
    "stdg_node_coordinates": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "stdg_set_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "stdg_get_state": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "stdg_get_slab": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "stdg_advance_slab": (ctypes.c_int, [_P, ctypes.POINTER(stdg_slab_stats)]),
    "stdg_residual": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "stdg_jv": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int]),
    "stdg_slab_norm": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.POINTER(ctypes.c_double)]),
    "stdg_spatial_operator": (ctypes.c_int, [_P, _P, _P, ctypes.c_int]),
    "stdg_jv_fd_apply": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_double, _P]),
    "stdg_jv_fp32": (ctypes.c_int, [_P, _P, _P, _P]),
    "stdg_precond_apply": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int]),
    "stdg_lodg_residual": (ctypes.c_int, [_P, _P, _P, _P, ctypes.c_int, ctypes.c_int]),
    "stdg_profile_enable": (ctypes.c_int, [_P, ctypes.c_int]),
    "stdg_profile_read": (ctypes.c_int, [_P, ctypes.POINTER(stdg_profile), ctypes.c_int]),
    "stdg_last_error": (ctypes.c_char_p, [_P]),
    "stdg_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "stdg_version": (ctypes.c_char_p, []),
    "stdg_predictor_matrix": (ctypes.c_int, [ctypes.c_int, _P]),
    "stdg_fdm_symbol": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_double, _P, _P, _P]),
    "stdg_lgl_constants": (ctypes.c_int, [ctypes.c_int, _P, _P, _P]),
}


def load(path=None):
    """Load libstdg.so (built by paper_2201_05800_gb300.build); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError("libstdg.so not built (%s): run python -m paper_2201_05800_gb300.build" % path)
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def config_default():
    d = stdg_config_desc()
    load().stdg_config_default(ctypes.byref(d))
    return d


def make_config(**kw):
    """stdg_config_desc from defaults overridden by keyword arguments (sequences for arrays)."""
    d = config_default()
    names = {f[0] for f in stdg_config_desc._fields_}
    for k, v in kw.items():
        if k not in names:
            raise KeyError(f"stdg_config_desc has no field {k!r}")
        if k in ("cells", "lo", "hi", "adv_vel"):
            arr = getattr(d, k)
            for i, x in enumerate(v):
                arr[i] = x
        else:
            setattr(d, k, v)
    return d


def _ptr(x, kind):
    """(pointer, kind) for a numpy FP64 array (host) or a torch CUDA FP64 tensor (device)."""
    if isinstance(x, np.ndarray):
        if x.dtype != np.float64 or not x.flags.c_contiguous:
            raise TypeError("host arrays must be C-contiguous float64")
        return ctypes.c_void_p(x.ctypes.data), HOST
    import torch  # device memory comes from torch
    if isinstance(x, torch.Tensor):
        if x.dtype != torch.float64 or not x.is_contiguous() or not x.is_cuda:
            raise TypeError("device tensors must be contiguous float64 CUDA tensors")
        return ctypes.c_void_p(x.data_ptr()), DEVICE
    raise TypeError("expected numpy.ndarray or torch.Tensor, got %r" % type(x))


class Context:
    """Owns one stdg_ctx.  Methods mirror the C entry points (stdg_<name>)."""

    def __init__(self, desc, stream=None):
        lib = load()
        self._lib = lib
        self.desc = desc
        handle = _P()
        sp = ctypes.c_void_p(stream) if stream is not None else None
        st = lib.stdg_create(ctypes.byref(desc), sp, ctypes.byref(handle))
        if st != 0:
            raise StdgError(st, "stdg_create failed")
        self._h = handle

    def _check(self, st):
        if st != 0:
            raise StdgError(st, (self._lib.stdg_last_error(self._h) or b"").decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stdg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    @property
    def state_len(self):
        return self._lib.stdg_state_len(self._h)

    @property
    def slab_len(self):
        return self._lib.stdg_slab_len(self._h)

    @property
    def device_bytes(self):
        return self._lib.stdg_device_bytes(self._h)

    def node_coordinates(self):
        X = np.empty(self._lib.stdg_coord_len(self._h))
        self._check(self._lib.stdg_node_coordinates(self._h, ctypes.c_void_p(X.ctypes.data), HOST))
        return X.reshape(-1, self.desc.dim)

    def set_state(self, u):
        p, kind = _ptr(u, None)
        self._check(self._lib.stdg_set_state(self._h, p, kind))

    def get_state(self, out=None):
        out = np.empty(self.state_len) if out is None else out
        p, kind = _ptr(out, None)
        self._check(self._lib.stdg_get_state(self._h, p, kind))
        return out

    def get_slab(self, out=None):
        out = np.empty(self.slab_len) if out is None else out
        p, kind = _ptr(out, None)
        self._check(self._lib.stdg_get_slab(self._h, p, kind))
        return out

    def advance_slab(self, check=True):
        stats = stdg_slab_stats()
        st = self._lib.stdg_advance_slab(self._h, ctypes.byref(stats))
        if check:
            self._check(st)
        return stats.as_dict() | {"status": st}

    def residual(self, U, u_prev, out=None):
        out = (np.empty(self.slab_len) if isinstance(U, np.ndarray) else U.new_empty(self.slab_len)) \
            if out is None else out
        (pU, k1), (pu, k2), (pR, k3) = _ptr(U, None), _ptr(u_prev, None), _ptr(out, None)
        if not k1 == k2 == k3:
            raise TypeError("all buffers must be on the same side (host or device)")
        self._check(self._lib.stdg_residual(self._h, pU, pu, pR, k1))
        return out

    def jv(self, U, u_prev, v, out=None):
        out = (np.empty(self.slab_len) if isinstance(U, np.ndarray) else U.new_empty(self.slab_len)) \
            if out is None else out
        ptrs = [_ptr(x, None) for x in (U, u_prev, v, out)]
        if len({k for _, k in ptrs}) != 1:
            raise TypeError("all buffers must be on the same side (host or device)")
        self._check(self._lib.stdg_jv(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[3][0], ptrs[0][1]))
        return out

    def jv_fp32(self, U, v, out=None):
        """stdg_jv_fp32: FP32 exact J(U) v on device float32 tensors (slab layout)."""
        import torch
        assert U.dtype == torch.float32 and v.dtype == torch.float32 and U.is_cuda and v.is_cuda
        out = torch.empty_like(U) if out is None else out
        self._check(self._lib.stdg_jv_fp32(self._h, ctypes.c_void_p(U.data_ptr()), ctypes.c_void_p(v.data_ptr()),
                                           ctypes.c_void_p(out.data_ptr())))
        return out

    def spatial_operator(self, U, out=None):
        out = (np.empty(self.slab_len) if isinstance(U, np.ndarray) else U.new_empty(self.slab_len)) \
            if out is None else out
        (pU, k1), (pF, k2) = _ptr(U, None), _ptr(out, None)
        if k1 != k2:
            raise TypeError("all buffers must be on the same side (host or device)")
        self._check(self._lib.stdg_spatial_operator(self._h, pU, pF, k1))
        return out

    def jv_fd_apply(self, U, F0, v, eps, out):
        """One FD Jacobian-vector kernel launch on device tensors (as issued inside GMRES)."""
        ptrs = [_ptr(x, None) for x in (U, F0, v, out)]
        if any(k != DEVICE for _, k in ptrs):
            raise TypeError("jv_fd_apply takes device tensors")
        self._check(self._lib.stdg_jv_fd_apply(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0], float(eps), ptrs[3][0]))
        return out

    def lodg_residual(self, U, u_prev, form=0, out=None):
        """Lobatto IIIC (method-of-lines) slab residual, form 0 (A) or 1 (A^-1)."""
        out = (np.empty(self.slab_len) if isinstance(U, np.ndarray) else U.new_empty(self.slab_len)) \
            if out is None else out
        ptrs = [_ptr(x, None) for x in (U, u_prev, out)]
        if len({k for _, k in ptrs}) != 1:
            raise TypeError("all buffers must be on the same side (host or device)")
        self._check(self._lib.stdg_lodg_residual(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0], int(form), ptrs[0][1]))
        return out

    def precond_apply(self, U, v, out=None):
        """z = P(U)^-1 v with the point-block preconditioner built from the slab U."""
        out = (np.empty(self.slab_len) if isinstance(U, np.ndarray) else U.new_empty(self.slab_len)) \
            if out is None else out
        ptrs = [_ptr(x, None) for x in (U, v, out)]
        if len({k for _, k in ptrs}) != 1:
            raise TypeError("all buffers must be on the same side (host or device)")
        self._check(self._lib.stdg_precond_apply(self._h, ptrs[0][0], ptrs[1][0], ptrs[2][0], ptrs[0][1]))
        return out

    def profile_enable(self, on=True):
        self._check(self._lib.stdg_profile_enable(self._h, 1 if on else 0))

    def profile_read(self, reset=True):
        p = stdg_profile()
        self._check(self._lib.stdg_profile_read(self._h, ctypes.byref(p), 1 if reset else 0))
        return {name: {"launches": p.launches[i], "ms": p.ms[i]} for i, name in enumerate(PROFILE_CLASSES)}

    def slab_norm(self, x):
        p, kind = _ptr(x, None)
        r = ctypes.c_double()
        self._check(self._lib.stdg_slab_norm(self._h, p, kind, ctypes.byref(r)))
        return r.value


class stdg_batch_desc(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("equation", ctypes.c_int), ("max_slots", ctypes.c_int),
                ("hbm_budget_bytes", ctypes.c_size_t)]


_BATCH_SIGS = {
    "stdg_batch_create": (ctypes.c_int, [ctypes.POINTER(stdg_batch_desc), _P, ctypes.POINTER(_P)]),
    "stdg_batch_destroy": (ctypes.c_int, [_P]),
    "stdg_batch_add": (ctypes.c_int, [_P, ctypes.POINTER(stdg_config_desc), _P, ctypes.c_int,
                                      ctypes.POINTER(ctypes.c_int)]),
    "stdg_batch_step": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "stdg_batch_run": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]),
    "stdg_batch_query": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(stdg_slab_stats)]),
    "stdg_batch_get_state": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    "stdg_batch_get_slab": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    "stdg_batch_remove": (ctypes.c_int, [_P, ctypes.c_int]),
    "stdg_batch_slot_bytes": (ctypes.c_size_t, [_P, ctypes.POINTER(stdg_config_desc)]),
    "stdg_batch_free_bytes": (ctypes.c_size_t, [_P]),
    "stdg_batch_last_error": (ctypes.c_char_p, [_P]),
}
_BATCH_SIGS.update({
    "stdg_batch_done_slots": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.c_int]),
    "stdg_batch_configure": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "stdg_server_configure": (ctypes.c_int, [_P, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "stdg_server_cancel": (ctypes.c_int, [_P, ctypes.c_ulonglong]),
    "stdg_server_set_policy": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_double]),
    "stdg_server_set_queue_limit": (ctypes.c_int, [_P, ctypes.c_size_t]),
    "stdg_server_create": (ctypes.c_int, [ctypes.POINTER(stdg_batch_desc), ctypes.c_int, ctypes.POINTER(_P)]),
    "stdg_server_destroy": (ctypes.c_int, [_P]),
    "stdg_server_submit": (ctypes.c_int, [_P, ctypes.POINTER(stdg_config_desc), _P,
                                          ctypes.POINTER(ctypes.c_ulonglong)]),
    "stdg_server_poll": (ctypes.c_int, [_P, ctypes.c_ulonglong, ctypes.c_double, ctypes.POINTER(ctypes.c_int),
                                        ctypes.POINTER(ctypes.c_int), ctypes.POINTER(stdg_slab_stats), _P,
                                        ctypes.POINTER(ctypes.c_double)]),
    "stdg_server_counters": (ctypes.c_int, [_P] + [ctypes.POINTER(ctypes.c_ulonglong)] * 3
                             + [ctypes.POINTER(ctypes.c_int)] * 3),
})
_SIGS.update(_BATCH_SIGS)


class Batch:
    """Owns one stdg_batch (batched device-driven slab solves).  Methods mirror stdg_batch_*."""

    def __init__(self, dim, equation, max_slots, hbm_budget_bytes, stream=None):
        lib = load()
        self._lib = lib
        self.desc = stdg_batch_desc(dim, equation, max_slots, hbm_budget_bytes)
        h = _P()
        st = lib.stdg_batch_create(ctypes.byref(self.desc), ctypes.c_void_p(stream) if stream is not None else None,
                                   ctypes.byref(h))
        if st != 0:
            raise StdgError(st, "stdg_batch_create failed")
        self._h = h
        self._descs = {}

    def _check(self, st):
        if st != 0:
            raise StdgError(st, (self._lib.stdg_batch_last_error(self._h) or b"").decode())

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stdg_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def slot_bytes(self, desc):
        return self._lib.stdg_batch_slot_bytes(self._h, ctypes.byref(desc))

    def free_bytes(self):
        return self._lib.stdg_batch_free_bytes(self._h)

    def add(self, desc, u0):
        """Admit one problem; returns the slot id (raises StdgError STDG_ERR_OOM when full)."""
        p, kind = _ptr(u0, None)
        slot = ctypes.c_int(-1)
        self._check(self._lib.stdg_batch_add(self._h, ctypes.byref(desc), p, kind, ctypes.byref(slot)))
        self._descs[slot.value] = desc
        return slot.value

    def try_add(self, desc, u0):
        """Like add, but returns None when the arena or the slot table is full."""
        try:
            return self.add(desc, u0)
        except StdgError as e:
            if e.status == 2:
                return None
            raise

    def step(self, ticks=1):
        w = ctypes.c_int(0)
        self._check(self._lib.stdg_batch_step(self._h, ticks, ctypes.byref(w)))
        return w.value

    def run(self, max_ticks=100000):
        w = ctypes.c_int(0)
        self._check(self._lib.stdg_batch_run(self._h, max_ticks, ctypes.byref(w)))
        return w.value

    def query(self, slot):
        done, status = ctypes.c_int(0), ctypes.c_int(0)
        stats = stdg_slab_stats()
        self._check(self._lib.stdg_batch_query(self._h, slot, ctypes.byref(done), ctypes.byref(status),
                                               ctypes.byref(stats)))
        return bool(done.value), status.value, stats.as_dict()

    def _len(self, slot, slab):
        d = self._descs[slot]
        r = d.dim + 2 if d.equation == EULER else 1
        n = r
        for a in range(d.dim):
            n *= d.cells[a] * (d.N + 1)
        return n * (d.s if slab else 1)

    def get_state(self, slot, out=None):
        out = np.empty(self._len(slot, False)) if out is None else out
        p, kind = _ptr(out, None)
        self._check(self._lib.stdg_batch_get_state(self._h, slot, p, kind))
        return out

    def get_slab(self, slot, out=None):
        out = np.empty(self._len(slot, True)) if out is None else out
        p, kind = _ptr(out, None)
        self._check(self._lib.stdg_batch_get_slab(self._h, slot, p, kind))
        return out

    def remove(self, slot):
        self._check(self._lib.stdg_batch_remove(self._h, slot))
        self._descs.pop(slot, None)

    def configure(self, share_quantum=0.0, share_max_stride=16, use_graphs=True, autotune=False):
        """stdg_batch_configure: size-aware sharing, CUDA-graph ticks, tile autotuning."""
        self._check(self._lib.stdg_batch_configure(self._h, float(share_quantum), int(share_max_stride),
                                                   1 if use_graphs else 0, 1 if autotune else 0))

    def done_slots(self):
        """Slots that finished as of the last step/run and are not removed yet."""
        n = self._lib.stdg_batch_done_slots(self._h, None, 0)
        buf = (ctypes.c_int * max(n, 1))()
        n = self._lib.stdg_batch_done_slots(self._h, buf, n)
        return list(buf[:n])


def _desc_state_len(d):
    n = d.dim + 2 if d.equation == EULER else 1
    for a in range(d.dim):
        n *= d.cells[a] * (d.N + 1)
    return n


class Server:
    """Owns one stdg_server (continuous batching of slab solves on a worker thread)."""

    def __init__(self, dim, equation, max_slots, hbm_budget_bytes, ticks_per_round=4):
        lib = load()
        self._lib = lib
        self.desc = stdg_batch_desc(dim, equation, max_slots, hbm_budget_bytes)
        h = _P()
        st = lib.stdg_server_create(ctypes.byref(self.desc), ticks_per_round, ctypes.byref(h))
        if st != 0:
            raise StdgError(st, "stdg_server_create failed")
        self._h = h
        self._lens = {}

    def close(self):
        if getattr(self, "_h", None):
            self._lib.stdg_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def submit(self, desc, u0):
        """Queue one request (u0: host FP64 state); returns its ticket."""
        u0 = np.ascontiguousarray(u0, dtype=np.float64).ravel()
        if u0.size != _desc_state_len(desc):
            raise ValueError("u0 has %d values, the problem needs %d" % (u0.size, _desc_state_len(desc)))
        t = ctypes.c_ulonglong(0)
        st = self._lib.stdg_server_submit(self._h, ctypes.byref(desc), ctypes.c_void_p(u0.ctypes.data), ctypes.byref(t))
        if st != 0:
            raise StdgError(st, "stdg_server_submit failed")
        self._lens[t.value] = u0.size
        return t.value

    def poll(self, ticket, wait_s=0.0):
        """None while the request runs; else dict(status, stats, u, queue_s, service_s, latency_s)."""
        done, status = ctypes.c_int(0), ctypes.c_int(0)
        stats = stdg_slab_stats()
        u = np.empty(self._lens[ticket])
        times = (ctypes.c_double * 3)()
        st = self._lib.stdg_server_poll(self._h, ticket, float(wait_s), ctypes.byref(done), ctypes.byref(status),
                                        ctypes.byref(stats), ctypes.c_void_p(u.ctypes.data), times)
        if st != 0:
            raise StdgError(st, "stdg_server_poll failed")
        if not done.value:
            return None
        self._lens.pop(ticket, None)
        return {"status": status.value, "stats": stats.as_dict(), "u": u, "queue_s": times[0],
                "service_s": times[1], "latency_s": times[2]}

    def configure(self, share_quantum=0.0, share_max_stride=16, use_graphs=True, autotune=False):
        st = self._lib.stdg_server_configure(self._h, float(share_quantum), int(share_max_stride),
                                             1 if use_graphs else 0, 1 if autotune else 0)
        if st != 0:
            raise StdgError(st, "stdg_server_configure failed")

    def set_policy(self, order=0, max_running_dof=0.0):
        """stdg_server_set_policy: 0 = arrival order, 1 = smallest first; cap on admitted DOF."""
        st = self._lib.stdg_server_set_policy(self._h, int(order), float(max_running_dof))
        if st != 0:
            raise StdgError(st, "stdg_server_set_policy failed")

    def cancel(self, ticket):
        st = self._lib.stdg_server_cancel(self._h, ticket)
        if st != 0:
            raise StdgError(st, "stdg_server_cancel failed")

    def set_queue_limit(self, max_queued):
        st = self._lib.stdg_server_set_queue_limit(self._h, int(max_queued))
        if st != 0:
            raise StdgError(st, "stdg_server_set_queue_limit failed")

    def counters(self):
        a, c, t = ctypes.c_ulonglong(0), ctypes.c_ulonglong(0), ctypes.c_ulonglong(0)
        q, r, mr = ctypes.c_int(0), ctypes.c_int(0), ctypes.c_int(0)
        st = self._lib.stdg_server_counters(self._h, ctypes.byref(a), ctypes.byref(c), ctypes.byref(t),
                                            ctypes.byref(q), ctypes.byref(r), ctypes.byref(mr))
        return {"admitted": a.value, "completed": c.value, "ticks": t.value, "queued": q.value,
                "running": r.value, "max_running": mr.value, "fatal": st}


def version():
    return load().stdg_version().decode()


def status_string(st):
    return load().stdg_status_string(st).decode()


def lgl_constants(n):
    """stdg_lgl_constants: (x, w, D) of the n-point LGL rule as the CUDA path computes them
    (host computation, no GPU needed)."""
    x, w, D = np.zeros(n), np.zeros(n), np.zeros((n, n))
    st = load().stdg_lgl_constants(n, x.ctypes.data, w.ctypes.data, D.ctypes.data)
    if st != 0:
        raise StdgError(st, status_string(st))
    return x, w, D


def fdm_symbol(N, K, h, nu, eta, lam):
    """stdg_fdm_symbol: eigenvalues (K, N+1) and eigenvector blocks V (K, N+1, N+1) of the periodic
    1D operator the batch engine's global preconditioner diagonalises."""
    n = N + 1
    lam_out = np.empty(K * n)
    vre, vim = np.empty(K * n * n), np.empty(K * n * n)
    st = load().stdg_fdm_symbol(N, K, h, nu, eta, lam, lam_out.ctypes.data, vre.ctypes.data, vim.ctypes.data)
    if st != 0:
        raise StdgError(st, "stdg_fdm_symbol failed")
    return lam_out.reshape(K, n), (vre + 1j * vim).reshape(K, n, n)


def predictor_matrix(s):
    """stdg_predictor_matrix: the s x s matrix E[m, j] = l_j(tau_m + 2) of the extrapolated
    initial iterate (host computation, no GPU needed)."""
    E = np.zeros((s, s))
    st = load().stdg_predictor_matrix(s, E.ctypes.data)
    if st != 0:
        raise StdgError(st, status_string(st))
    return E


def slab_norm_noalloc(x, out, stream=None):
    """stdg_slab_norm_noalloc: ||x||_2 of a device FP64 tensor into the one-element device
    tensor ``out`` without any device allocation (for callers that cannot allocate; the
    partial sums live in a static device array, see include/stdg.h)."""
    lib = load()
    fn = lib.stdg_slab_norm_noalloc
    fn.restype = ctypes.c_int
    fn.argtypes = [_P, ctypes.c_size_t, _P, _P]
    px, kx = _ptr(x, None)
    po, ko = _ptr(out, None)
    if kx != DEVICE or ko != DEVICE:
        raise TypeError("slab_norm_noalloc takes device tensors")
    st = fn(px, x.numel(), po, ctypes.c_void_p(stream) if stream is not None else None)
    if st != 0:
        raise StdgError(st, "stdg_slab_norm_noalloc")
    return out
