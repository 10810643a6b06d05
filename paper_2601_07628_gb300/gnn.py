"""Learned warm start: binding of the network's C ABI (include/dpdlp_gnn.h) and the steps
around it (node features, target scaling, training loop, prediction for dpdlp_set_start).

Every forward and backward step runs in the library's CUDA kernels; this module only
marshals arrays and orders the calls.
"""
from __future__ import annotations

import ctypes as C
import math
from dataclasses import dataclass

import numpy as np

from . import dpdlp

H, F, ROUNDS = 64, 8, 4

EXPORTS = {
    "dpdlp_gnn_param_count": (C.c_int64, []),
    "dpdlp_gnn_create": (C.c_int, [C.POINTER(C.c_void_p), C.c_int]),
    "dpdlp_gnn_destroy": (None, [C.c_void_p]),
    "dpdlp_gnn_last_error": (C.c_char_p, [C.c_void_p]),
    "dpdlp_gnn_set_ptr_mode": (C.c_int, [C.c_void_p, C.c_int]),
    "dpdlp_gnn_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "dpdlp_gnn_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "dpdlp_gnn_get_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64]),
    "dpdlp_gnn_zero_grads": (C.c_int, [C.c_void_p]),
    "dpdlp_gnn_set_graph": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_gnn_set_features": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_gnn_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dpdlp_gnn_backward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]),
    "dpdlp_gnn_adam": (C.c_int, [C.c_void_p, C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64]),
    "dpdlp_gnn_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                       C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64,
                                       C.POINTER(C.c_double)]),
}

_declared = set()


def _lib():
    lib = dpdlp.load_library()
    if id(lib) not in _declared:
        for name, (res, args) in EXPORTS.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _declared.add(id(lib))
    return lib


def _ptr(a):
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        return C.c_void_p(a.data_ptr())
    return a.ctypes.data_as(C.c_void_p)


def param_count() -> int:
    return int(_lib().dpdlp_gnn_param_count())


class Network:
    """One network on one GPU.  Arrays are numpy (host) or, after ``device_arrays(True)``,
    CUDA tensors for features, targets and outputs."""

    def __init__(self, device: int = 0):
        self.lib = _lib()
        h = C.c_void_p()
        rc = self.lib.dpdlp_gnn_create(C.byref(h), int(device))
        if rc != 0:
            raise dpdlp.DpdlpError(rc, "dpdlp_gnn_create failed")
        self.h = h
        self.P = param_count()
        self.n = self.m = 0
        self.dev = False

    def close(self):
        if getattr(self, "h", None):
            self.lib.dpdlp_gnn_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, rc):
        if rc < 0:
            raise dpdlp.DpdlpError(rc, self.lib.dpdlp_gnn_last_error(self.h).decode())
        return rc

    def device_arrays(self, on: bool):
        self._check(self.lib.dpdlp_gnn_set_ptr_mode(self.h, 1 if on else 0))
        self.dev = on

    def set_params(self, theta):
        t = np.ascontiguousarray(theta, dtype=np.float32)
        if t.shape != (self.P,):
            raise ValueError(f"expected {self.P} parameters, got shape {t.shape}")
        self._check(self.lib.dpdlp_gnn_set_params(self.h, _ptr(t), self.P))

    def params(self) -> np.ndarray:
        out = np.empty(self.P, np.float32)
        self._check(self.lib.dpdlp_gnn_get_params(self.h, _ptr(out), self.P))
        return out

    def grads(self) -> np.ndarray:
        out = np.empty(self.P, np.float32)
        self._check(self.lib.dpdlp_gnn_get_grads(self.h, _ptr(out), self.P))
        return out

    def zero_grads(self):
        self._check(self.lib.dpdlp_gnn_zero_grads(self.h))

    def set_graph(self, n, m, row_ptr, col, val):
        rp = np.ascontiguousarray(row_ptr, np.int64)
        ci = np.ascontiguousarray(col, np.int32)
        va = np.ascontiguousarray(val, np.float64)
        self._check(self.lib.dpdlp_gnn_set_graph(self.h, int(n), int(m), _ptr(rp), _ptr(ci), _ptr(va)))
        self.n, self.m = int(n), int(m)

    def set_features(self, fv, fc):
        if not self.dev:
            fv = np.ascontiguousarray(fv, np.float32)
            fc = np.ascontiguousarray(fc, np.float32)
        self._check(self.lib.dpdlp_gnn_set_features(self.h, _ptr(fv), _ptr(fc)))

    def forward(self, x_out=None, y_out=None):
        if not self.dev:
            x_out = np.empty(self.n, np.float32) if x_out is None else x_out
            y_out = np.empty(self.m, np.float32) if y_out is None else y_out
        self._check(self.lib.dpdlp_gnn_forward(self.h, _ptr(x_out), _ptr(y_out)))
        return x_out, y_out

    def backward(self, tx, ty) -> float:
        if not self.dev:
            tx = np.ascontiguousarray(tx, np.float32)
            ty = np.ascontiguousarray(ty, np.float32)
        loss = C.c_double()
        self._check(self.lib.dpdlp_gnn_backward(self.h, _ptr(tx), _ptr(ty), C.byref(loss)))
        return loss.value

    def adam(self, lr, step, beta1=0.9, beta2=0.999, eps=1e-8):
        self._check(self.lib.dpdlp_gnn_adam(self.h, float(lr), float(beta1), float(beta2), float(eps), int(step)))

    def train_step(self, fv, fc, tx, ty, lr, step, beta1=0.9, beta2=0.999, eps=1e-8,
                   want_loss=True):
        """Features, forward, backward and one Adam step as one replay of a captured CUDA
        graph (the same kernels in the same order as the separate calls).  Returns the
        step's loss, or None without waiting for the step when ``want_loss`` is False."""
        if not self.dev:
            fv = np.ascontiguousarray(fv, np.float32)
            fc = np.ascontiguousarray(fc, np.float32)
            tx = np.ascontiguousarray(tx, np.float32)
            ty = np.ascontiguousarray(ty, np.float32)
        loss = C.c_double()
        self._check(self.lib.dpdlp_gnn_train_step(
            self.h, _ptr(fv), _ptr(fc), _ptr(tx), _ptr(ty), float(lr), float(beta1), float(beta2),
            float(eps), int(step), C.byref(loss) if want_loss else None))
        return loss.value if want_loss else None


# ---------------------------------------------------------------- features and scales
@dataclass
class Scales:
    """Family-level constants: inputs are divided by c_scale (costs) and b_scale (right-hand
    sides and finite bounds); the network predicts x / x_scale and y / y_scale."""
    c_scale: float
    b_scale: float
    x_scale: float
    y_scale: float


def finite_rhs(lp) -> np.ndarray:
    """The finite side of each row's range (lc for '>=' and '=' rows, uc for '<=' rows)."""
    lc, uc = np.asarray(lp.lc, np.float64), np.asarray(lp.uc, np.float64)
    return np.where(np.isfinite(uc), uc, np.where(np.isfinite(lc), lc, 0.0))


def features(lp, sc: Scales):
    """Fv[n][8] = [c / c_scale, lv finite, uv finite, lv / b_scale, uv / b_scale, 0, 0, 1]
    (infinite bounds enter as 0); Fc[m][8] = [rhs / b_scale, '=', '<=', '>=', 0, 0, 0, 1]."""
    n, m = lp.n, lp.m
    fv = np.zeros((n, F), np.float32)
    lv, uv = np.asarray(lp.lv), np.asarray(lp.uv)
    fv[:, 0] = lp.c / sc.c_scale
    fv[:, 1] = np.isfinite(lv)
    fv[:, 2] = np.isfinite(uv)
    fv[:, 3] = np.where(np.isfinite(lv), lv, 0.0) / sc.b_scale
    fv[:, 4] = np.where(np.isfinite(uv), uv, 0.0) / sc.b_scale
    fv[:, 7] = 1.0
    fc = np.zeros((m, F), np.float32)
    lc, uc = np.asarray(lp.lc), np.asarray(lp.uc)
    eq = np.isfinite(lc) & np.isfinite(uc) & (lc == uc)
    fc[:, 0] = finite_rhs(lp) / sc.b_scale
    fc[:, 1] = eq
    fc[:, 2] = np.isfinite(uc) & ~eq
    fc[:, 3] = np.isfinite(lc) & ~eq
    fc[:, 7] = 1.0
    return fv, fc


def fit_scales(lps, xs, ys) -> Scales:
    """Scales from a training set: mean max |c|, mean max |rhs|, and the RMS of the
    solutions."""
    c_scale = float(np.mean([np.abs(lp.c).max() for lp in lps])) or 1.0
    b_scale = float(np.mean([np.abs(finite_rhs(lp)).max() for lp in lps])) or 1.0
    x_scale = float(np.sqrt(np.mean([np.mean(np.square(x)) for x in xs]))) or 1.0
    y_scale = float(np.sqrt(np.mean([np.mean(np.square(y)) for y in ys]))) or 1.0
    return Scales(c_scale, b_scale, x_scale, y_scale)


def init_params(seed: int = 0) -> np.ndarray:
    """Seeded initial parameters: weights U(-a, a) with a = sqrt(6 / (fan_in + fan_out)),
    biases 0.01 (every unit starts active), heads U(-a, a) with a = sqrt(6 / (H + 1))."""
    rng = np.random.default_rng(seed)
    blocks = []

    def w(rows, cols):
        a = math.sqrt(6.0 / (rows + cols))
        blocks.append(rng.uniform(-a, a, size=rows * cols))

    def b(k, v=0.01):
        blocks.append(np.full(k, v))

    w(H, F), b(H), w(H, F), b(H)
    for _ in range(ROUNDS):
        w(H, H), w(H, H), b(H), w(H, H), w(H, H), b(H)
    w(1, H), b(1, 0.0), w(1, H), b(1, 0.0)
    return np.concatenate(blocks).astype(np.float32)


# ---------------------------------------------------------------- training and prediction
def train(net: Network, data, epochs: int, lr: float = 1e-3, seed: int = 0, log=None) -> list:
    """Adam over the instances of ``data`` (a list of (fv, fc, tx, ty), all on the network's
    side: numpy or CUDA tensors), one instance per step, shuffled each epoch.  Returns the
    mean loss of every epoch."""
    rng = np.random.default_rng(seed)
    step, hist = 0, []
    for ep in range(epochs):
        tot = 0.0
        for i in rng.permutation(len(data)):
            fv, fc, tx, ty = data[i]
            step += 1
            tot += net.train_step(fv, fc, tx, ty, lr, step)
        hist.append(tot / len(data))
        if log:
            log(ep, hist[-1])
    return hist


def project_dual(lp, y):
    """y projected onto the dual set Y of Section 2.1: a row with only an upper bound
    (lc = -inf) has y <= 0, a row with only a lower bound (uc = +inf) has y >= 0, a free row
    has y = 0, an equality or ranged row any sign."""
    lc, uc = np.asarray(lp.lc, np.float64), np.asarray(lp.uc, np.float64)
    y = np.where(np.isfinite(lc), y, np.minimum(y, 0.0))
    return np.where(np.isfinite(uc), y, np.maximum(y, 0.0))


def predict(net: Network, lp, sc: Scales):
    """Start point for ``lp``: the network's (x, y), rescaled, x clipped into its bounds and
    y projected onto the dual set."""
    fv, fc = features(lp, sc)
    was = net.dev
    if was:
        net.device_arrays(False)
    net.set_features(fv, fc)
    xh, yh = net.forward()
    if was:
        net.device_arrays(True)
    x = np.clip(xh.astype(np.float64) * sc.x_scale, lp.lv, lp.uv)
    y = project_dual(lp, yh.astype(np.float64) * sc.y_scale)
    return x, y


def cold_start(lp):
    """The solver's own start point: x = proj_X(0), y = 0."""
    return np.clip(np.zeros(lp.n), lp.lv, lp.uv), np.zeros(lp.m)


def _max_kkt(k):
    return max(k["r_primal"], k["r_dual"], k["r_gap"])


def guard_starts(solver, lps, starts, probe_iters: int = 64):
    """Keep each predicted start only where it is no worse than the cold start.

    ``solver`` holds ``lps`` as a batch (``load_batch``).  Both start sets are run for
    ``probe_iters`` iterations on that handle; an instance keeps its predicted start when
    its relative KKT error after them is at most that of the cold start, else it falls back
    to the cold start (plain PDHG from zero stays the fallback and the yardstick for the
    prediction).  The handle is left with the chosen start set and ``resume`` = 0, so the
    next solve starts from the chosen starts.  Returns (chosen starts, kept mask, KKT from
    the prediction, KKT cold)."""
    cold = [cold_start(lp) for lp in lps]
    solver.set_param("resume", 0)
    errs = []
    for st in (starts, cold):
        solver.set_start(np.concatenate([x for x, _ in st]), np.concatenate([y for _, y in st]))
        solver.solve(0.0, probe_iters)
        errs.append([_max_kkt(k) for k in solver.batch_kkt()])
    keep = [w <= c for w, c in zip(*errs)]
    chosen = [s if k else c for s, k, c in zip(starts, keep, cold)]
    solver.set_start(np.concatenate([x for x, _ in chosen]), np.concatenate([y for _, y in chosen]))
    return chosen, keep, errs[0], errs[1]
