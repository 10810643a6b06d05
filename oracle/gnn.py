"""FP64 reference of the warm-start network (test infrastructure only).

Plain numpy, written from the network's definition (the bipartite message-passing model
declared in include/dpdlp_gnn.h): forward pass, loss and the gradient of the loss by
hand-written backpropagation.  It is pinned by finite differences and closed forms in
tests/test_gnn_oracle.py and is the reference the GPU forward and backward kernels are
compared with.  Imported only by tests and the benchmark's checks.

Weights enter as given (the GPU side rounds its weight matrices to BF16; a comparison
passes the rounded values here, as float64).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

H = 64  # hidden units
F = 8   # input features per node
L = 4   # message-passing rounds


def param_layout() -> list:
    """(name, shape) of every parameter block, in the order of the flat vector."""
    blocks = [("Ev", (H, F)), ("ev", (H,)), ("Ec", (H, F)), ("ec", (H,))]
    for l in range(L):
        blocks += [(f"Uc{l}", (H, H)), (f"Vc{l}", (H, H)), (f"bc{l}", (H,)),
                   (f"Uv{l}", (H, H)), (f"Vv{l}", (H, H)), (f"bv{l}", (H,))]
    blocks += [("wx", (H,)), ("bx", ()), ("wy", (H,)), ("by", ())]
    return blocks


def param_count() -> int:
    return int(sum(int(np.prod(s)) for _, s in param_layout()))


def unpack(theta: np.ndarray) -> dict:
    out, o = {}, 0
    for name, shape in param_layout():
        k = int(np.prod(shape))
        out[name] = theta[o:o + k].reshape(shape) if shape else theta[o]
        o += k
    return out


def pack(P: dict) -> np.ndarray:
    return np.concatenate([np.atleast_1d(np.asarray(P[name], dtype=np.float64)).reshape(-1)
                           for name, _ in param_layout()])


def is_weight(name: str) -> bool:
    """Blocks used in BF16 on the GPU (matrices and head vectors; biases stay FP32)."""
    return name[0] in "EUVw"


def aggregation(n: int, m: int, row_ptr, col, val):
    """R = diag(1/max(1, sum_j |a_ij|)) A (m x n) and C = diag(1/max(1, sum_i |a_ij|)) A^T."""
    A = sp.csr_matrix((np.asarray(val, np.float64), np.asarray(col), np.asarray(row_ptr)),
                      shape=(m, n))
    rs = np.maximum(1.0, np.asarray(abs(A).sum(axis=1)).ravel())
    cs = np.maximum(1.0, np.asarray(abs(A).sum(axis=0)).ravel())
    R = sp.diags(1.0 / rs) @ A
    C = sp.diags(1.0 / cs) @ A.T
    return R.tocsr(), C.tocsr()


def relu(z):
    return np.maximum(z, 0.0)


def forward(theta, R, C, Fv, Fc):
    """Returns (x_hat, y_hat, cache) for the backward pass."""
    P = unpack(np.asarray(theta, np.float64))
    hv = relu(Fv @ P["Ev"].T + P["ev"])
    hc = relu(Fc @ P["Ec"].T + P["ec"])
    cache = {"hv": [hv], "hc": [hc], "gv": [], "gc": []}
    for l in range(L):
        gc = R @ hv
        hc = relu(hc @ P[f"Uc{l}"].T + gc @ P[f"Vc{l}"].T + P[f"bc{l}"])
        gv = C @ hc
        hv = relu(hv @ P[f"Uv{l}"].T + gv @ P[f"Vv{l}"].T + P[f"bv{l}"])
        cache["gc"].append(gc)
        cache["hc"].append(hc)
        cache["gv"].append(gv)
        cache["hv"].append(hv)
    x_hat = hv @ P["wx"] + P["bx"]
    y_hat = hc @ P["wy"] + P["by"]
    return x_hat, y_hat, cache


def loss(x_hat, y_hat, tx, ty) -> float:
    return float(np.mean((x_hat - tx) ** 2) + np.mean((y_hat - ty) ** 2))


def backward(theta, R, C, Fv, Fc, tx, ty):
    """Loss and its gradient with respect to the flat parameter vector."""
    P = unpack(np.asarray(theta, np.float64))
    x_hat, y_hat, K = forward(theta, R, C, Fv, Fc)
    n, m = x_hat.shape[0], y_hat.shape[0]
    G = {name: np.zeros(shape) if shape else 0.0 for name, shape in param_layout()}
    dx = 2.0 * (x_hat - tx) / n
    dy = 2.0 * (y_hat - ty) / m
    hv, hc = K["hv"][L], K["hc"][L]
    G["wx"] = hv.T @ dx
    G["bx"] = dx.sum()
    G["wy"] = hc.T @ dy
    G["by"] = dy.sum()
    dhv = np.outer(dx, P["wx"])
    dhc = np.outer(dy, P["wy"])
    for l in reversed(range(L)):
        # variable update of round l: hv_{l+1} = relu(hv_l Uv^T + gv Vv^T + bv)
        dz = dhv * (K["hv"][l + 1] > 0)
        G[f"Uv{l}"] = dz.T @ K["hv"][l]
        G[f"Vv{l}"] = dz.T @ K["gv"][l]
        G[f"bv{l}"] = dz.sum(axis=0)
        dhv = dz @ P[f"Uv{l}"]
        dgv = dz @ P[f"Vv{l}"]
        dhc = dhc + C.T @ dgv          # gv = C hc_{l+1}
        # constraint update of round l: hc_{l+1} = relu(hc_l Uc^T + gc Vc^T + bc)
        dz = dhc * (K["hc"][l + 1] > 0)
        G[f"Uc{l}"] = dz.T @ K["hc"][l]
        G[f"Vc{l}"] = dz.T @ K["gc"][l]
        G[f"bc{l}"] = dz.sum(axis=0)
        dhc = dz @ P[f"Uc{l}"]
        dgc = dz @ P[f"Vc{l}"]
        dhv = dhv + R.T @ dgc          # gc = R hv_l
    dz = dhv * (K["hv"][0] > 0)
    G["Ev"] = dz.T @ Fv
    G["ev"] = dz.sum(axis=0)
    dz = dhc * (K["hc"][0] > 0)
    G["Ec"] = dz.T @ Fc
    G["ec"] = dz.sum(axis=0)
    return loss(x_hat, y_hat, tx, ty), pack(G)


def round_weights_bf16(theta: np.ndarray) -> np.ndarray:
    """The parameters as the GPU uses them: weight blocks rounded to BF16 (round to nearest
    even from FP32), biases rounded to FP32."""
    out = np.asarray(theta, np.float64).astype(np.float32)
    o = 0
    for name, shape in param_layout():
        k = int(np.prod(shape))
        if is_weight(name):
            bits = out[o:o + k].view(np.uint32).astype(np.uint64)
            lsb = (bits >> 16) & 1
            bits = ((bits + 0x7FFF + lsb) >> 16) << 16
            out[o:o + k] = bits.astype(np.uint32).view(np.float32)
        o += k
    return out.astype(np.float64)
