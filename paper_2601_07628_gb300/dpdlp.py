"""Python binding of libdpdlp (the C ABI in include/dpdlp.h) by ctypes.

Argument marshalling only: every step of the solve runs in the library's CUDA kernels.
Host arrays are numpy float64/int arrays; device arrays may be given as CUDA torch tensors
(any object with ``data_ptr()`` and ``is_cuda``), in which case the call runs in the
library's device-pointer mode on the tensor's device.

The library must have been built (``paper_2601_07628_gb300.build()``); importing
this module on a machine without it raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdpdlp.so")

CONVERGED, MAX_ITER, NUMERICAL = 0, 1, 2
ERRORS = {-1: "invalid argument", -2: "out of memory", -3: "CUDA error", -4: "not loaded",
          -5: "device timeout", -6: "size beyond the fixed scratch of the no-allocation SpMV"}


class DpdlpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)} ({code}): {msg}")
        self.code = code


class KKT(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("r_primal", "r_dual", "r_gap", "obj_p", "obj_d", "r_fp",
                                          "omega", "eta", "tau", "sigma")] + \
               [("iterations", C.c_int64), ("restarts", C.c_int64), ("checks", C.c_int64),
                ("status", C.c_int32), ("spmv_mode", C.c_int32)]


class Trace(C.Structure):
    _fields_ = [("T", C.c_int64), ("k", C.c_int64)] + \
               [(k, C.c_double) for k in ("r_primal", "r_dual", "r_gap", "obj_p", "obj_d", "r_fp",
                                          "omega")] + \
               [("restart", C.c_int32), ("spmv_mode", C.c_int32), ("inst", C.c_int32),
                ("status", C.c_int32)]


class ScalarState(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("T", "k", "restarts", "checks")] + \
               [(k, C.c_double) for k in ("eta", "omega", "r_anchor", "r_prev", "e_sum", "e_prev")] + \
               [("has_anchor", C.c_int32), ("has_e_prev", C.c_int32),
                ("spmv_mode", C.c_int32), ("stall_checks", C.c_int32), ("best_kkt", C.c_double)]


class Info(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("nnz", C.c_int64),
                ("nnz_padded_csr", C.c_int64), ("nnz_padded_csc", C.c_int64),
                ("tiles_csr", C.c_int32), ("tiles_csc", C.c_int32),
                ("long_rows", C.c_int32), ("long_cols", C.c_int32),
                ("device_bytes", C.c_int64), ("preprocess_ms", C.c_double),
                ("fused_body", C.c_int32), ("reserved", C.c_int32)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)

EXPORTS = {
    "dpdlp_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "dpdlp_destroy": (None, [C.c_void_p]),
    "dpdlp_last_error": (C.c_char_p, [C.c_void_p]),
    "dpdlp_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dpdlp_set_allocator": (C.c_int, [C.c_void_p, ALLOC_FN, RELEASE_FN, C.c_void_p]),
    "dpdlp_load_lp": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_load_batch": (C.c_int, [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32,
                                   C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_set_batch_eta": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "dpdlp_get_batch_kkt": (C.c_int, [C.c_void_p, C.POINTER(KKT), C.c_int32]),
    "dpdlp_set_row_bounds": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_set_objective_diag": (C.c_int, [C.c_void_p, C.c_void_p]),
    "dpdlp_set_param": (C.c_int, [C.c_void_p, C.c_char_p, C.c_double]),
    "dpdlp_get_param": (C.c_int, [C.c_void_p, C.c_char_p, C.POINTER(C.c_double)]),
    "dpdlp_set_start": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_solve": (C.c_int, [C.c_void_p, C.c_double, C.c_int64]),
    "dpdlp_get_solution": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_get_kkt": (C.c_int, [C.c_void_p, C.POINTER(KKT)]),
    "dpdlp_get_trace": (C.c_int, [C.c_void_p, C.POINTER(Trace), C.c_int32, C.POINTER(C.c_int32)]),
    "dpdlp_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(ScalarState)]),
    "dpdlp_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(ScalarState)]),
    "dpdlp_set_schedule": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "dpdlp_apply_A": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_apply_AT": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_time_kernel": (C.c_int, [C.c_void_p, C.c_char_p, C.c_int32, C.POINTER(C.c_double)]),
    "dpdlp_get_info": (C.c_int, [C.c_void_p, C.POINTER(Info)]),
    "dpdlp_csr_spmv_noalloc": (C.c_int, [C.c_int32, C.c_int32, C.c_int64, C.c_void_p, C.c_void_p,
                                         C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
}

_lib = None


def load_library(path: str = LIB_PATH):
    """Load libdpdlp.so and declare every exported signature (no GPU needed)."""
    global _lib
    if _lib is not None and path == LIB_PATH:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2601_07628_gb300.build()")
    lib = C.CDLL(path)
    for name, (res, args) in EXPORTS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path == LIB_PATH:
        _lib = lib
    return lib


def _is_dev(a) -> bool:
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _host_f64(a, n):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.shape != (n,):
        raise ValueError(f"expected shape ({n},), got {a.shape}")
    return a


def _ptr(a):
    if a is None:
        return None
    if _is_dev(a):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


class Solver:
    """One LP on one GPU: ``load``, ``solve``, ``solution``, ``kkt``."""

    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = C.c_void_p()
        rc = self.lib.dpdlp_create(C.byref(h), int(device))
        if rc < 0:
            raise DpdlpError(rc, "dpdlp_create failed (no CUDA device?)")
        self.device = int(device)
        self.h = h
        self.device = int(device)
        self.n = self.m = 0
        self._device_mode = False

    # --------------------------------------------------------------- plumbing
    def _check(self, rc):
        if rc < 0:
            raise DpdlpError(rc, self.lib.dpdlp_last_error(self.h).decode())
        return rc

    def _mode(self, *arrays):
        dev = any(_is_dev(a) for a in arrays if a is not None)
        if dev != self._device_mode:
            self._check(self.lib.dpdlp_set_param(self.h, b"ptr_mode_device", 1.0 if dev else 0.0))
            self._device_mode = dev
        if dev:
            import torch  # device memory and streams only

            self._check(self.lib.dpdlp_set_stream(self.h, C.c_void_p(
                torch.cuda.current_stream(self.device).cuda_stream)))
        return dev

    def close(self):
        if getattr(self, "h", None):
            self.lib.dpdlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # --------------------------------------------------------------- problem
    def load(self, lp=None, *, n=None, m=None, c=None, row_ptr=None, col=None, val=None, b=None,
             ctype=None, lv=None, uv=None, lc=None, uc=None):
        """Load an LP: an ``lpgen.LP`` or keyword arrays.  Row bounds come from (b, ctype)
        or from (lc, uc) (general ranges)."""
        if lp is not None:
            n, m, c, row_ptr, col, val, lv, uv = lp.n, lp.m, lp.c, lp.row_ptr, lp.col, lp.val, lp.lv, lp.uv
            b, ctype, lc, uc = lp.b, lp.ctype, lp.lc, lp.uc
        n, m = int(n), int(m)
        c = _host_f64(c, n)
        lv, uv = _host_f64(lv, n), _host_f64(uv, n)
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        val = np.ascontiguousarray(val, dtype=np.float64)
        if ctype is not None:
            b = _host_f64(b, m)
            ctype = np.ascontiguousarray(ctype, dtype=np.int8)
        self._check(self.lib.dpdlp_load_lp(self.h, n, m, _ptr(c), _ptr(row_ptr), _ptr(col), _ptr(val),
                                           _ptr(b) if ctype is not None else None, _ptr(lv), _ptr(uv),
                                           _ptr(ctype) if ctype is not None else None))
        self.n, self.m = n, m
        self.row_off = np.array([0, m], np.int32)
        self.col_off = np.array([0, n], np.int32)
        if ctype is None:
            self.set_row_bounds(lc, uc)
        if lp is not None and getattr(lp, "q", None) is not None:
            self.set_objective_diag(lp.q)
        return self

    def set_objective_diag(self, q):
        """Diagonal QP: objective 1/2 x^T diag(q) x + c^T x (q = None: the LP again)."""
        if q is None:
            self._check(self.lib.dpdlp_set_objective_diag(self.h, None))
        else:
            self._check(self.lib.dpdlp_set_objective_diag(self.h, _ptr(_host_f64(q, self.n))))
        return self

    def load_batch(self, lps):
        """Load a batch of LPs (a list of ``lpgen.LP``) into one handle: the block-diagonal
        stack of the instances, solved together with per-instance step sizes, weights,
        restarts and statuses.  Row bounds come from (b, ctype) when every instance has
        them, else from the instances' (lc, uc)."""
        lps = list(lps)
        if not lps:
            raise ValueError("empty batch")
        row_off = np.zeros(len(lps) + 1, np.int32)
        col_off = np.zeros(len(lps) + 1, np.int32)
        row_off[1:] = np.cumsum([lp.m for lp in lps])
        col_off[1:] = np.cumsum([lp.n for lp in lps])
        n, m = int(col_off[-1]), int(row_off[-1])
        c = np.ascontiguousarray(np.concatenate([lp.c for lp in lps]), dtype=np.float64)
        lv = np.ascontiguousarray(np.concatenate([lp.lv for lp in lps]), dtype=np.float64)
        uv = np.ascontiguousarray(np.concatenate([lp.uv for lp in lps]), dtype=np.float64)
        nnz_off = np.concatenate([[0], np.cumsum([int(lp.row_ptr[-1]) for lp in lps])])
        row_ptr = np.ascontiguousarray(np.concatenate(
            [[0]] + [np.asarray(lp.row_ptr[1:], np.int64) + nnz_off[i] for i, lp in enumerate(lps)]),
            dtype=np.int64)
        col = np.ascontiguousarray(np.concatenate(
            [np.asarray(lp.col, np.int64) + col_off[i] for i, lp in enumerate(lps)]), dtype=np.int32)
        val = np.ascontiguousarray(np.concatenate([lp.val for lp in lps]), dtype=np.float64)
        typed = all(lp.ctype is not None for lp in lps)
        b = ctype = None
        if typed:
            b = np.ascontiguousarray(np.concatenate([lp.b for lp in lps]), dtype=np.float64)
            ctype = np.ascontiguousarray(np.concatenate([lp.ctype for lp in lps]), dtype=np.int8)
        self._check(self.lib.dpdlp_load_batch(
            self.h, len(lps), _ptr(row_off), _ptr(col_off), n, m, _ptr(c), _ptr(row_ptr), _ptr(col),
            _ptr(val), _ptr(b) if typed else None, _ptr(lv), _ptr(uv), _ptr(ctype) if typed else None))
        self.n, self.m = n, m
        self.row_off, self.col_off = row_off, col_off
        if not typed:
            self.set_row_bounds(np.concatenate([lp.lc for lp in lps]), np.concatenate([lp.uc for lp in lps]))
        if any(getattr(lp, "q", None) is not None for lp in lps):
            self.set_objective_diag(np.concatenate(
                [lp.q if getattr(lp, "q", None) is not None else np.zeros(lp.n) for lp in lps]))
        return self

    def split(self, x, y):
        """Per-instance pieces [(x_i, y_i)] of stacked batch vectors."""
        ro, co = self.row_off, self.col_off
        return [(x[co[i]:co[i + 1]], y[ro[i]:ro[i + 1]]) for i in range(len(ro) - 1)]

    def set_batch_eta(self, eta):
        e = np.ascontiguousarray(eta, dtype=np.float64)
        self._check(self.lib.dpdlp_set_batch_eta(self.h, _ptr(e) if e.size else None, int(e.size)))

    def batch_kkt(self) -> list:
        cnt = len(self.row_off) - 1
        buf = (KKT * cnt)()
        self._check(self.lib.dpdlp_get_batch_kkt(self.h, buf, cnt))
        return [{f: getattr(buf[i], f) for f, _ in KKT._fields_} for i in range(cnt)]

    def use_torch_allocator(self, on: bool = True):
        """Take the device buffers of the LP from torch's caching allocator (on=True) or from
        cudaMalloc (on=False).  Unloads the current LP; call before load / load_batch."""
        if not on:
            self._check(self.lib.dpdlp_set_allocator(self.h, ALLOC_FN(), RELEASE_FN(), None))
            self._alloc_cbs = None
            return self
        import torch

        dev = self.device

        def _alloc(nbytes, ctx):
            try:
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev)
            except Exception:
                return None

        def _release(ptr, nbytes, ctx):
            try:
                torch.cuda.caching_allocator_delete(ptr)
            except Exception:
                pass

        cbs = (ALLOC_FN(_alloc), RELEASE_FN(_release))  # kept alive with the solver
        self._check(self.lib.dpdlp_set_allocator(self.h, cbs[0], cbs[1], None))
        self._alloc_cbs = cbs
        return self

    def set_row_bounds(self, lc, uc):
        lc, uc = _host_f64(lc, self.m), _host_f64(uc, self.m)
        self._check(self.lib.dpdlp_set_row_bounds(self.h, _ptr(lc), _ptr(uc)))

    def set_param(self, key: str, value: float):
        if key == "ptr_mode_device":
            raise ValueError("pointer mode follows the arrays passed to each call")
        self._check(self.lib.dpdlp_set_param(self.h, key.encode(), float(value)))
        return self

    def set_params(self, **kw):
        for k, v in kw.items():
            self.set_param(k, v)
        return self

    def get_param(self, key: str) -> float:
        v = C.c_double()
        self._check(self.lib.dpdlp_get_param(self.h, key.encode(), C.byref(v)))
        return v.value

    def set_start(self, x0=None, y0=None):
        """Start point of every later fresh solve until replaced; ``set_start()`` restores
        the default start (x = proj_X(0), y = 0)."""
        dev = self._mode(x0, y0)
        if not dev:
            x0 = None if x0 is None else _host_f64(x0, self.n)
            y0 = None if y0 is None else _host_f64(y0, self.m)
        self._check(self.lib.dpdlp_set_start(self.h, _ptr(x0), _ptr(y0)))

    # --------------------------------------------------------------- solve
    def solve(self, tol: float = 1e-8, max_iter: int = 1_000_000) -> int:
        return self._check(self.lib.dpdlp_solve(self.h, float(tol), int(max_iter)))

    def solution(self, x_out=None, y_out=None):
        """(x^, y^) at the final check, as numpy arrays (or written into given CUDA tensors)."""
        dev = self._mode(x_out, y_out)
        if not dev:
            x_out = np.empty(self.n) if x_out is None else x_out
            y_out = np.empty(self.m) if y_out is None else y_out
            for a, k in ((x_out, self.n), (y_out, self.m)):
                if a.dtype != np.float64 or a.shape != (k,) or not a.flags.c_contiguous:
                    raise ValueError("output arrays must be contiguous float64 of the LP's sizes")
        self._check(self.lib.dpdlp_get_solution(self.h, _ptr(x_out), _ptr(y_out)))
        return x_out, y_out

    def kkt(self) -> dict:
        k = KKT()
        self._check(self.lib.dpdlp_get_kkt(self.h, C.byref(k)))
        return {f: getattr(k, f) for f, _ in KKT._fields_}

    def trace(self, cap: int = 1 << 16) -> list:
        buf = (Trace * cap)()
        cnt = C.c_int32()
        self._check(self.lib.dpdlp_get_trace(self.h, buf, cap, C.byref(cnt)))
        return [{f: getattr(buf[i], f) for f, _ in Trace._fields_} for i in range(cnt.value)]

    def get_state(self) -> dict:
        self._mode()
        x, y, x0, y0 = np.empty(self.n), np.empty(self.m), np.empty(self.n), np.empty(self.m)
        s = ScalarState()
        self._check(self.lib.dpdlp_get_state(self.h, _ptr(x), _ptr(y), _ptr(x0), _ptr(y0), C.byref(s)))
        return dict(x=x, y=y, x0=x0, y0=y0, scalars={f: getattr(s, f) for f, _ in ScalarState._fields_})

    def set_state(self, st: dict):
        self._mode()
        s = ScalarState(**st["scalars"])
        x, y = _host_f64(st["x"], self.n), _host_f64(st["y"], self.m)
        x0, y0 = _host_f64(st["x0"], self.n), _host_f64(st["y0"], self.m)
        self._check(self.lib.dpdlp_set_state(self.h, _ptr(x), _ptr(y), _ptr(x0), _ptr(y0), C.byref(s)))

    def set_schedule(self, kinds):
        """Forced restart decisions per check.  For a batch: a list with one sequence per
        instance (shorter ones are padded with 0, no restart)."""
        if len(kinds) and not np.isscalar(kinds[0]):
            L = max(len(k) for k in kinds)
            kinds = np.concatenate([np.pad(np.asarray(k, np.int8), (0, L - len(k))) for k in kinds])
        k = np.ascontiguousarray(kinds, dtype=np.int8)
        self._check(self.lib.dpdlp_set_schedule(self.h, _ptr(k) if k.size else None, int(k.size)))

    def apply_A(self, x, out=None):
        dev = self._mode(x, out)
        if not dev:
            x = _host_f64(x, self.n)
            out = np.empty(self.m)
        self._check(self.lib.dpdlp_apply_A(self.h, _ptr(x), _ptr(out)))
        return out

    def apply_AT(self, y, out=None):
        dev = self._mode(y, out)
        if not dev:
            y = _host_f64(y, self.m)
            out = np.empty(self.n)
        self._check(self.lib.dpdlp_apply_AT(self.h, _ptr(y), _ptr(out)))
        return out

    def time_kernel(self, which: str, reps: int = 20) -> float:
        ms = C.c_double()
        self._check(self.lib.dpdlp_time_kernel(self.h, which.encode(), int(reps), C.byref(ms)))
        return ms.value

    def set_stream(self, stream_ptr: int | None):
        self._check(self.lib.dpdlp_set_stream(self.h, C.c_void_p(stream_ptr) if stream_ptr else None))

    def info(self) -> dict:
        i = Info()
        self._check(self.lib.dpdlp_get_info(self.h, C.byref(i)))
        return {f: getattr(i, f) for f, _ in Info._fields_}


def csr_spmv_noalloc(row_ptr, col_idx, val, x, y, n, stream=None) -> int:
    """y = A x through ``dpdlp_csr_spmv_noalloc`` (no device allocation).  All arrays are
    contiguous CUDA tensors on the current device: int32 row_ptr [m+1] and col_idx [nnz],
    float64 val [nnz], x [>= n] and y [>= m]; ``stream`` is a raw cudaStream_t handle
    (default: torch's current stream).  Returns the ABI code; arguments of the wrong type,
    layout, device or length return DPDLP_ERR_INVALID (-1) without calling the library.
    The CSR contents themselves (row_ptr[m] = nnz, indices in range) are the caller's
    guarantee, as in the C ABI."""
    import torch

    lib = load_library()
    dev = torch.device("cuda", torch.cuda.current_device())
    want = ((row_ptr, torch.int32), (col_idx, torch.int32), (val, torch.float64),
            (x, torch.float64), (y, torch.float64))
    for t, dt in want:
        if not isinstance(t, torch.Tensor) or t.dtype != dt or t.device != dev or t.dim() != 1 \
                or not t.is_contiguous():
            return -1
    m = int(row_ptr.numel()) - 1
    nnz = int(col_idx.numel())
    if m < 0 or val.numel() != nnz or x.numel() < int(n) or y.numel() < m:
        return -1
    if stream is None:
        stream = torch.cuda.current_stream().cuda_stream
    return lib.dpdlp_csr_spmv_noalloc(m, int(n), nnz, C.c_void_p(row_ptr.data_ptr()),
                                      C.c_void_p(col_idx.data_ptr()), C.c_void_p(val.data_ptr()),
                                      C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()),
                                      C.c_void_p(stream) if stream else None)
