"""ctypes binding of ``libbg.so`` (C-ABI in ``include/bg.h``).

Argument marshalling only: torch tensors are passed as raw device pointers
and ``torch.cuda.Stream`` objects as ``cudaStream_t``; every step of the
recursion runs in the library's CUDA kernel.  Importing this module loads the
library and raises ``ImportError`` when it has not been built (there is no CPU
fallback).
"""

from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

BG_OK = 0
BG_ERR_INVALID_ARG = 1
BG_ERR_UNSUPPORTED = 2
BG_ERR_NOMEM = 3
BG_ERR_CUDA = 4
BG_ERR_TIMEOUT = 5
BG_ERR_BUSY = 6

FIELD_C64 = 0
FIELD_FP = 1
FIELD_C64_REAL = 2        # complex values, real momenta (float64 [E][n][d])
MOSTLY_MINUS = 0
ALTERNATING = 1

# bg_plan_create / bg_eval / ... as declared in include/bg.h
EXPORTED = ("bg_plan_create", "bg_plan_create_product", "bg_plan_create_mixed", "bg_cut_trace", "bg_plan_destroy", "bg_workspace_size", "bg_eval",
            "bg_eval_noalloc", "bg_host_staging_size", "bg_eval_host", "bg_batch_workspace_size",
            "bg_batch_create", "bg_batch_launch", "bg_batch_describe", "bg_batch_destroy",
            "bg_batch_autotune", "bg_serve_create", "bg_serve_submit", "bg_serve_wait",
            "bg_serve_stats", "bg_serve_destroy", "bg_plan_describe", "bg_strerror", "bg_last_error",
            "bg_version", "bg_debug_inject_fault", "bg_debug_bounds_report", "bg_debug_in_place_pays")

# BG_LIBRARY selects another build of the same library (the bounds-checked
# one, _build.build(checked=True)); default: the ordinary in-tree build
LIB_PATH = os.environ.get("BG_LIBRARY") or _build.LIB


class BgGroup(ctypes.Structure):
    """bg_group of include/bg.h."""
    _fields_ = [("plan", ctypes.c_void_p), ("E", ctypes.c_int64), ("momenta", ctypes.c_void_p),
                ("eps", ctypes.c_void_p), ("out", ctypes.c_void_p), ("status", ctypes.c_void_p)]


class BgBatchConfig(ctypes.Structure):
    """bg_batch_config of include/bg.h."""
    _fields_ = [("tile_points", ctypes.c_int), ("fp_blocks_per_sm", ctypes.c_int),
                ("c64_blocks_per_sm", ctypes.c_int), ("lanes_max_items", ctypes.c_int)]


def load_library(path=None):
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libbg.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    vp = ctypes.c_void_p
    lib.bg_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                   ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(vp)]
    lib.bg_plan_create.restype = ctypes.c_int
    lib.bg_plan_create_product.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_uint32, ctypes.c_int, ctypes.c_int,
                                           ctypes.POINTER(ctypes.c_uint8), ctypes.POINTER(vp)]
    lib.bg_plan_create_product.restype = ctypes.c_int
    lib.bg_plan_create_mixed.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.c_uint32, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                         ctypes.POINTER(ctypes.c_uint8), ctypes.c_uint32, ctypes.POINTER(vp)]
    lib.bg_plan_create_mixed.restype = ctypes.c_int
    lib.bg_cut_trace.argtypes = [ctypes.c_int, ctypes.c_uint32, ctypes.c_int64, ctypes.c_int, ctypes.c_int,
                                 ctypes.POINTER(vp), vp, vp]
    lib.bg_cut_trace.restype = ctypes.c_int
    lib.bg_plan_destroy.argtypes = [vp]
    lib.bg_plan_destroy.restype = ctypes.c_int
    lib.bg_workspace_size.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    lib.bg_workspace_size.restype = ctypes.c_int
    lib.bg_eval.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp, ctypes.c_size_t, vp]
    lib.bg_eval.restype = ctypes.c_int
    lib.bg_eval_noalloc.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, vp]
    lib.bg_eval_noalloc.restype = ctypes.c_int
    lib.bg_host_staging_size.argtypes = [vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_size_t)]
    lib.bg_host_staging_size.restype = ctypes.c_int
    lib.bg_eval_host.argtypes = [vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.c_int64, vp,
                                 ctypes.c_size_t, vp]
    lib.bg_eval_host.restype = ctypes.c_int
    gp = ctypes.POINTER(BgGroup)
    cp = ctypes.POINTER(BgBatchConfig)
    lib.bg_batch_workspace_size.argtypes = [gp, ctypes.c_int, cp, ctypes.POINTER(ctypes.c_size_t)]
    lib.bg_batch_workspace_size.restype = ctypes.c_int
    lib.bg_batch_create.argtypes = [gp, ctypes.c_int, cp, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
    lib.bg_batch_create.restype = ctypes.c_int
    lib.bg_batch_launch.argtypes = [vp, vp]
    lib.bg_batch_launch.restype = ctypes.c_int
    lib.bg_batch_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.bg_batch_describe.restype = ctypes.c_int
    lib.bg_batch_destroy.argtypes = [vp]
    lib.bg_batch_destroy.restype = ctypes.c_int
    lib.bg_batch_autotune.argtypes = [gp, ctypes.c_int, vp, ctypes.c_size_t, ctypes.c_int, vp, cp,
                                      ctypes.POINTER(ctypes.c_double)]
    lib.bg_batch_autotune.restype = ctypes.c_int
    lib.bg_serve_create.argtypes = [ctypes.c_size_t, ctypes.c_int, ctypes.POINTER(vp)]
    lib.bg_serve_create.restype = ctypes.c_int
    lib.bg_serve_submit.argtypes = [vp, vp, ctypes.c_int64, vp, vp, vp, vp, ctypes.POINTER(ctypes.c_uint64)]
    lib.bg_serve_submit.restype = ctypes.c_int
    lib.bg_serve_wait.argtypes = [vp, ctypes.c_uint64, ctypes.c_int64]
    lib.bg_serve_wait.restype = ctypes.c_int
    u64p = ctypes.POINTER(ctypes.c_uint64)
    szp = ctypes.POINTER(ctypes.c_size_t)
    lib.bg_serve_stats.argtypes = [vp, u64p, u64p, u64p, szp, szp]
    lib.bg_serve_stats.restype = ctypes.c_int
    lib.bg_serve_destroy.argtypes = [vp]
    lib.bg_serve_destroy.restype = ctypes.c_int
    lib.bg_plan_describe.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t]
    lib.bg_plan_describe.restype = ctypes.c_int
    lib.bg_strerror.argtypes = [ctypes.c_int]
    lib.bg_strerror.restype = ctypes.c_char_p
    lib.bg_last_error.argtypes = []
    lib.bg_last_error.restype = ctypes.c_char_p
    lib.bg_debug_bounds_report.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_uint64)]
    lib.bg_debug_bounds_report.restype = ctypes.c_int
    lib.bg_debug_in_place_pays.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                           ctypes.c_int64, ctypes.c_size_t, ctypes.POINTER(ctypes.c_int),
                                           ctypes.POINTER(ctypes.c_double)]
    lib.bg_debug_in_place_pays.restype = ctypes.c_int
    lib.bg_debug_inject_fault.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.bg_debug_inject_fault.restype = ctypes.c_int
    lib.bg_version.argtypes = []
    lib.bg_version.restype = ctypes.c_int
    return lib


_lib = load_library()


class BGError(RuntimeError):
    def __init__(self, status, detail):
        self.status = status
        super().__init__(f"{_lib.bg_strerror(status).decode()}: {detail}")


def _check(status):
    if status != BG_OK:
        raise BGError(status, _lib.bg_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


def _stream_handle(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class Plan:
    """One (n, d, D_s, field, p, metric, states) configuration (bg_plan)."""

    def __init__(self, n, d, Ds, field, p=0, metric=MOSTLY_MINUS, n_states=1, assign=None,
                 states_per_leg=None, four_dim_legs=None):
        """assign: None (every leg takes state 0), an [H][n] table of state
        indices, or "all": every one of the n_states^n assignments, output
        index h = sum_l s_l n_states^l, evaluated with shared sub-currents.
        states_per_leg (instead of assign): the product plan of
        bg_plan_create_product (leg l takes states 0..states_per_leg[l]-1).
        four_dim_legs: bit mask of four-dimensional legs (bg_plan_create_mixed)."""
        self.n, self.d, self.Ds = n, d, Ds
        self.field, self.p, self.metric = field, p, metric
        self.n_states = n_states
        self._ws = None
        if states_per_leg is not None:
            import numpy as np
            r = np.ascontiguousarray(states_per_leg, dtype=np.uint8)
            if r.shape != (n,):
                raise ValueError("states_per_leg must have n entries")
            self._radix = r
            self.n_assign = int(np.prod(r.astype(np.int64)))
            h = ctypes.c_void_p()
            _check(_lib.bg_plan_create_product(n, d, Ds, field, p, metric, n_states,
                                               r.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8)),
                                               ctypes.byref(h)))
            self._h = h
            return
        buf = None
        H = 1
        if isinstance(assign, str):
            if assign != "all":
                raise ValueError('assign must be None, a table or "all"')
            H = n_states ** n
        elif assign is not None:
            import numpy as np
            a = np.ascontiguousarray(assign, dtype=np.uint8)
            if a.ndim != 2 or a.shape[1] != n:
                raise ValueError("assign must have shape [H][n]")
            H = a.shape[0]
            self._assign = a
            buf = a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint8))
        self.n_assign = H
        h = ctypes.c_void_p()
        if four_dim_legs is not None:
            _check(_lib.bg_plan_create_mixed(n, d, Ds, field, p, metric, n_states, H, buf,
                                             int(four_dim_legs), ctypes.byref(h)))
        else:
            _check(_lib.bg_plan_create(n, d, Ds, field, p, metric, n_states, H, buf, ctypes.byref(h)))
        self._h = h
        self._ws = None

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.bg_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def describe(self):
        buf = ctypes.create_string_buffer(512)
        _check(_lib.bg_plan_describe(self._h, buf, 512))
        return buf.value.decode()

    def workspace_size(self, E):
        b = ctypes.c_size_t()
        _check(_lib.bg_workspace_size(self._h, E, ctypes.byref(b)))
        return b.value

    def workspace(self, E, device=None):
        """A cached device workspace of at least workspace_size(E) bytes."""
        need = self.workspace_size(E)
        if need == 0:
            return None
        if self._ws is None or self._ws.numel() < need:
            self._ws = torch.empty(need, dtype=torch.uint8, device=device or "cuda")
        return self._ws

    @property
    def io_dtype(self):
        """dtype of polarisations and amplitudes."""
        return torch.int32 if self.field == FIELD_FP else torch.complex128

    @property
    def momentum_dtype(self):
        """dtype of the momenta (float64 for FIELD_C64_REAL)."""
        return torch.float64 if self.field == FIELD_C64_REAL else self.io_dtype

    def _check_types(self, momenta, eps, out):
        want_k = torch.empty((), dtype=self.momentum_dtype).element_size()
        want_v = torch.empty((), dtype=self.io_dtype).element_size()
        if momenta.element_size() != want_k or eps.element_size() != want_v or out.element_size() != want_v:
            raise TypeError(f"element sizes: momenta {momenta.element_size()} (want {want_k}), "
                            f"eps {eps.element_size()} and out {out.element_size()} (want {want_v})")

    def eval(self, momenta, eps, out=None, status=None, workspace=None, stream=None):
        """Amplitudes of E points.  momenta [E][n][d] and eps [E][n][(S)][D_s]
        as device tensors (int32/uint32 residues for F_p, complex128 for C64;
        momenta float64 for C64_REAL).
        Returns (out [E] or [E][H], status [E] uint8)."""
        E = momenta.shape[0]
        dev = momenta.device
        if out is None:
            shape = (E,) if self.n_assign == 1 else (E, self.n_assign)
            out = torch.empty(shape, dtype=eps.dtype, device=dev)
        if status is None:
            status = torch.empty(E, dtype=torch.uint8, device=dev)
        for t in (momenta, eps, out, status):
            if not t.is_contiguous():
                raise ValueError("tensors must be contiguous")
        if workspace is None:
            workspace = self.workspace(E, dev)
        ws_bytes = workspace.numel() if workspace is not None else 0
        self._check_types(momenta, eps, out)
        _check(_lib.bg_eval(self._h, E, _ptr(momenta), _ptr(eps), _ptr(out), _ptr(status),
                            _ptr(workspace), ws_bytes, _stream_handle(stream)))
        return out, status


    def staging_size(self, chunk):
        b = ctypes.c_size_t()
        _check(_lib.bg_host_staging_size(self._h, chunk, ctypes.byref(b)))
        return b.value

    def eval_host(self, momenta, eps, out=None, status=None, chunk=1 << 18, staging=None,
                  stream=None):
        """bg_eval_host: host (preferably pinned) input tensors in, host results
        out; transfers and kernels of consecutive chunks overlap.  Returns
        (out, status) host tensors, valid after the stream synchronises."""
        E = momenta.shape[0]
        if out is None:
            shape = (E,) if self.n_assign == 1 else (E, self.n_assign)
            out = torch.empty(shape, dtype=eps.dtype, pin_memory=momenta.is_pinned())
        if status is None:
            status = torch.empty(E, dtype=torch.uint8, pin_memory=momenta.is_pinned())
        for t in (momenta, eps, out, status):
            if not t.is_contiguous() or t.is_cuda:
                raise ValueError("eval_host takes contiguous host tensors")
        chunk = max(1, min(chunk, E)) if E else 1
        need = self.staging_size(chunk)
        if staging is None:
            if getattr(self, "_staging", None) is None or self._staging.numel() < need:
                self._staging = torch.empty(need, dtype=torch.uint8, device="cuda")
            staging = self._staging
        self._check_types(momenta, eps, out)
        _check(_lib.bg_eval_host(self._h, E, _ptr(momenta), _ptr(eps), _ptr(out), _ptr(status),
                                 chunk, _ptr(staging), staging.numel(), _stream_handle(stream)))
        return out, status

    def eval_noalloc(self, momenta, eps, out=None, status=None, stream=None):
        """bg_eval_noalloc: the same result as eval() without any device
        allocation by the library (scratch in its static device array).
        ``out``/``status`` are allocated here by torch only when not given."""
        E = momenta.shape[0]
        dev = momenta.device
        if out is None:
            shape = (E,) if self.n_assign == 1 else (E, self.n_assign)
            out = torch.empty(shape, dtype=eps.dtype, device=dev)
        if status is None:
            status = torch.empty(E, dtype=torch.uint8, device=dev)
        self._check_types(momenta, eps, out)
        _check(_lib.bg_eval_noalloc(self._h, E, _ptr(momenta), _ptr(eps), _ptr(out), _ptr(status),
                                    _stream_handle(stream)))
        return out, status


class Batch:
    """An uneven batch (bg_batch): groups = [(plan, momenta, eps, out, status)]
    of device tensors, evaluated by one CUDA-graph launch."""

    def __init__(self, groups, config=None, workspace=None):
        self._keep = groups
        arr = (BgGroup * len(groups))()
        for i, (plan, k, e, out, st) in enumerate(groups):
            plan._check_types(k, e, out)
            arr[i] = BgGroup(plan.handle.value, k.shape[0], k.data_ptr(), e.data_ptr(), out.data_ptr(),
                             st.data_ptr() if st is not None else 0)
        self._arr = arr
        self.config = config
        cfgp = ctypes.byref(config) if config is not None else None
        need = ctypes.c_size_t()
        _check(_lib.bg_batch_workspace_size(arr, len(groups), cfgp, ctypes.byref(need)))
        if workspace is None or workspace.numel() < need.value:
            workspace = torch.empty(max(need.value, 256), dtype=torch.uint8, device="cuda")
        self.workspace = workspace
        h = ctypes.c_void_p()
        _check(_lib.bg_batch_create(arr, len(groups), cfgp, _ptr(workspace), workspace.numel(),
                                    ctypes.byref(h)))
        self._h = h

    def launch(self, stream=None):
        _check(_lib.bg_batch_launch(self._h, _stream_handle(stream)))

    def describe(self):
        buf = ctypes.create_string_buffer(512)
        _check(_lib.bg_batch_describe(self._h, buf, 512))
        return buf.value.decode()

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.bg_batch_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def autotune(groups, reps=2, stream=None):
        """bg_batch_autotune over the library's candidate set; returns
        (BgBatchConfig, ms per launch)."""
        arr = (BgGroup * len(groups))()
        for i, (plan, k, e, out, st) in enumerate(groups):
            plan._check_types(k, e, out)
            arr[i] = BgGroup(plan.handle.value, k.shape[0], k.data_ptr(), e.data_ptr(), out.data_ptr(),
                             st.data_ptr() if st is not None else 0)
        need = ctypes.c_size_t()
        _check(_lib.bg_batch_workspace_size(arr, len(groups), None, ctypes.byref(need)))
        ws = torch.empty(max(need.value, 256), dtype=torch.uint8, device="cuda")
        best = BgBatchConfig()
        ms = ctypes.c_double()
        _check(_lib.bg_batch_autotune(arr, len(groups), _ptr(ws), ws.numel(), reps,
                                      _stream_handle(stream), ctypes.byref(best), ctypes.byref(ms)))
        return best, ms.value


class Server:
    """bg_server: continuous admission of evaluation requests on host buffers.

    submit() returns a ticket; wait(ticket, timeout_ms) returns True when the
    results are in the request's host tensors, False on timeout.  The caller
    keeps the request's tensors alive until its wait succeeds (the server
    also keeps references until then)."""

    def __init__(self, budget_bytes, max_inflight=8):
        h = ctypes.c_void_p()
        _check(_lib.bg_serve_create(budget_bytes, max_inflight, ctypes.byref(h)))
        self._h = h
        self._live = {}

    def submit(self, plan, momenta, eps, out, status=None):
        plan._check_types(momenta, eps, out)
        t = ctypes.c_uint64()
        _check(_lib.bg_serve_submit(self._h, plan.handle, momenta.shape[0], _ptr(momenta), _ptr(eps),
                                    _ptr(out), _ptr(status), ctypes.byref(t)))
        self._live[t.value] = (plan, momenta, eps, out, status)
        return t.value

    def wait(self, ticket, timeout_ms=-1):
        st = _lib.bg_serve_wait(self._h, ticket, timeout_ms)
        if st == BG_ERR_TIMEOUT:
            return False
        self._live.pop(ticket, None)
        _check(st)
        return True

    def stats(self):
        a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        d, e = ctypes.c_size_t(), ctypes.c_size_t()
        _check(_lib.bg_serve_stats(self._h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c),
                                   ctypes.byref(d), ctypes.byref(e)))
        return {"submitted": a.value, "completed": b.value, "pending": c.value,
                "bytes_in_use": d.value, "peak_bytes": e.value}

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.bg_serve_destroy(self._h)
            self._h = ctypes.c_void_p()
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def cut_trace(field, matrices, out=None, p=0, stream=None):
    """bg_cut_trace: out[e] = trace(M_k ... M_1) for device tensors
    matrices[i] of shape [E][S][S] or [E][S*S] (row = outgoing state)."""
    import torch
    k = len(matrices)
    E = matrices[0].shape[0]
    S = int(round((matrices[0][0].numel()) ** 0.5)) if E else 1
    for m in matrices:
        if not m.is_contiguous() or m.shape[0] != E or m[0].numel() != S * S:
            raise ValueError("matrices must be contiguous [E][S][S] tensors")
    if out is None:
        out = torch.empty(E, dtype=matrices[0].dtype, device=matrices[0].device)
    ptrs = (ctypes.c_void_p * k)(*[m.data_ptr() for m in matrices])
    _check(_lib.bg_cut_trace(field, p, E, k, S, ptrs, _ptr(out), _stream_handle(stream)))
    return out


def strerror(status):
    return _lib.bg_strerror(status).decode()


def version():
    return _lib.bg_version()


FAULT_DEVICE_ALLOC = 1
FAULT_LAUNCH = 2
FAULT_COPY = 3


def inject_fault(site, skip=0, count=1):
    """bg_debug_inject_fault: operations skip .. skip+count-1 at `site` fail
    as if the CUDA runtime had refused them (count = 0 disarms)."""
    _check(_lib.bg_debug_inject_fault(site, skip, count))


def in_place_pays(field, n, d, Ds, H, E, host_bytes):
    """bg_debug_in_place_pays: (read page-locked buffers in place?, literal
    multiplications per amplitude of the estimate)."""
    flag, ops = ctypes.c_int(), ctypes.c_double()
    _check(_lib.bg_debug_in_place_pays(field, n, d, Ds, H, E, host_bytes, ctypes.byref(flag), ctypes.byref(ops)))
    return bool(flag.value), ops.value


def bounds_report():
    """bg_debug_bounds_report: (checked build?, first violation or 0); clears it."""
    c, v = ctypes.c_int(), ctypes.c_uint64()
    _check(_lib.bg_debug_bounds_report(ctypes.byref(c), ctypes.byref(v)))
    return bool(c.value), v.value
