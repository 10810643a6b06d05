"""Pins of the FP64 warm-start network reference (oracle/gnn.py), on the CPU.

The backward pass is pinned by central finite differences of the forward pass; the forward
pass by closed forms and invariants that any slip in it (a swapped aggregation matrix, a
dropped term, a wrong index) breaks: all-zero weights, permutation equivariance, independent
graph components, no-message locality, hand-computed aggregation matrices.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import gnn as G


def random_graph(rng, n, m, density=0.4):
    A = sp.random(m, n, density=density, random_state=np.random.RandomState(rng.integers(1 << 30)),
                  data_rvs=lambda k: rng.uniform(0.5, 2.0, k) * rng.choice([-1, 1], k)).tocsr()
    A.sort_indices()
    return A


def random_theta(rng, scale=0.1):
    t = rng.standard_normal(G.param_count()) * scale
    P = G.unpack(t)
    for l in range(G.L):  # positive biases keep most units away from the ReLU kink
        P[f"bc{l}"] = np.abs(P[f"bc{l}"]) + 0.2
        P[f"bv{l}"] = np.abs(P[f"bv{l}"]) + 0.2
    P["ev"] = np.abs(P["ev"]) + 0.2
    P["ec"] = np.abs(P["ec"]) + 0.2
    return G.pack(P)


def setup(seed=0, n=7, m=5):
    rng = np.random.default_rng(seed)
    A = random_graph(rng, n, m)
    R, C = G.aggregation(n, m, A.indptr, A.indices, A.data)
    Fv = rng.standard_normal((n, G.F))
    Fc = rng.standard_normal((m, G.F))
    tx = rng.standard_normal(n)
    ty = rng.standard_normal(m)
    return rng, A, R, C, Fv, Fc, tx, ty


def test_layout_and_count():
    assert G.param_count() == 2 * (G.H * G.F + G.H) + G.L * (4 * G.H * G.H + 2 * G.H) + 2 * (G.H + 1)
    t = np.arange(G.param_count(), dtype=np.float64)
    assert np.array_equal(G.pack(G.unpack(t)), t)


def test_aggregation_by_hand():
    # A = [[2, 0, -1], [0, 0, 0], [1, 3, 0]]
    A = sp.csr_matrix(np.array([[2.0, 0, -1], [0, 0, 0], [1, 3, 0]]))
    R, C = G.aggregation(3, 3, A.indptr, A.indices, A.data)
    assert np.allclose(R.toarray(), [[2 / 3, 0, -1 / 3], [0, 0, 0], [1 / 4, 3 / 4, 0]])
    # column sums of |A|: 3, 3, 1 -> C = diag(1/3, 1/3, 1) A^T
    assert np.allclose(C.toarray(), [[2 / 3, 0, 1 / 3], [0, 0, 1], [-1, 0, 0]])


def test_zero_weights_closed_form():
    _, A, R, C, Fv, Fc, tx, ty = setup(1)
    P = G.unpack(np.zeros(G.param_count()))
    P["bx"], P["by"] = 3.0, -2.0
    th = G.pack(P)
    x, y, _ = G.forward(th, R, C, Fv, Fc)
    assert np.all(x == 3.0) and np.all(y == -2.0)
    loss, g = G.backward(th, R, C, Fv, Fc, tx, ty)
    assert loss == pytest.approx(np.mean((3 - tx) ** 2) + np.mean((-2 - ty) ** 2))
    Q = G.unpack(g)
    assert Q["bx"] == pytest.approx(2 * np.mean(3 - tx))
    assert Q["by"] == pytest.approx(2 * np.mean(-2 - ty))
    assert np.all(Q["Uv0"] == 0) and np.all(Q["wx"] == 0)


@pytest.mark.parametrize("seed", [0, 1])
def test_gradient_matches_finite_differences(seed):
    rng, A, R, C, Fv, Fc, tx, ty = setup(seed)
    th = random_theta(rng)
    _, g = G.backward(th, R, C, Fv, Fc, tx, ty)
    # every bias and head entry, and 24 random entries of every weight matrix (so a slip in
    # any one block of the backward pass meets the check)
    names = [nm for nm, _ in G.param_layout()]
    offs = np.cumsum([0] + [int(np.prod(s)) for _, s in G.param_layout()])
    idx = []
    for k, nm in enumerate(names):
        if not nm[0] in "EUV":
            idx += list(range(offs[k], offs[k + 1]))
        else:
            idx += list(offs[k] + rng.choice(offs[k + 1] - offs[k], size=24, replace=False))
    loss0 = G.loss(*G.forward(th, R, C, Fv, Fc)[:2], tx, ty)
    h = 1e-6  # central differences: roundoff ~1e-16 * loss / h, and a step too small to cross a ReLU kink
    gscale = np.abs(g).max()
    worst = 0.0
    for i in idx:
        tp, tm = th.copy(), th.copy()
        tp[i] += h
        tm[i] -= h
        xp, yp, _ = G.forward(tp, R, C, Fv, Fc)
        xm, ym, _ = G.forward(tm, R, C, Fv, Fc)
        fd = (G.loss(xp, yp, tx, ty) - G.loss(xm, ym, tx, ty)) / (2 * h)
        worst = max(worst, abs(fd - g[i]) / (abs(g[i]) + 1e-4 * gscale))
    assert loss0 < 1e3 and worst < 1e-5, (loss0, worst)


def test_permutation_equivariance():
    rng, A, R, C, Fv, Fc, tx, ty = setup(2, n=9, m=6)
    th = random_theta(rng)
    pc = rng.permutation(9)
    pr = rng.permutation(6)
    A2 = A[pr][:, pc].tocsr()
    A2.sort_indices()
    R2, C2 = G.aggregation(9, 6, A2.indptr, A2.indices, A2.data)
    x, y, _ = G.forward(th, R, C, Fv, Fc)
    x2, y2, _ = G.forward(th, R2, C2, Fv[pc], Fc[pr])
    assert np.allclose(x2, x[pc], rtol=1e-12, atol=1e-12)
    assert np.allclose(y2, y[pr], rtol=1e-12, atol=1e-12)


def test_components_are_independent():
    rng, A, R, C, Fv, Fc, tx, ty = setup(3, n=6, m=4)
    th = random_theta(rng)
    B = random_graph(rng, 5, 3)
    D = sp.block_diag([A, B]).tocsr()
    D.sort_indices()
    Rd, Cd = G.aggregation(11, 7, D.indptr, D.indices, D.data)
    Fv2 = np.vstack([Fv, rng.standard_normal((5, G.F))])
    Fc2 = np.vstack([Fc, rng.standard_normal((3, G.F))])
    x, y, _ = G.forward(th, R, C, Fv, Fc)
    xd, yd, _ = G.forward(th, Rd, Cd, Fv2, Fc2)
    assert np.allclose(xd[:6], x, rtol=1e-12, atol=1e-12) and np.allclose(yd[:4], y, rtol=1e-12, atol=1e-12)


def test_no_messages_is_node_local():
    """With Vc = Vv = 0 every output depends on its own node's features only."""
    rng, A, R, C, Fv, Fc, tx, ty = setup(4)
    P = G.unpack(random_theta(rng))
    for l in range(G.L):
        P[f"Vc{l}"][:] = 0
        P[f"Vv{l}"][:] = 0
    th = G.pack(P)
    x, y, _ = G.forward(th, R, C, Fv, Fc)
    E = sp.csr_matrix(A.shape)
    Re, Ce = G.aggregation(A.shape[1], A.shape[0], E.indptr, E.indices, E.data)
    x0, y0, _ = G.forward(th, Re, Ce, Fv, Fc)
    assert np.allclose(x, x0) and np.allclose(y, y0)
    # but with messages the graph matters
    x1, _, _ = G.forward(random_theta(rng), R, C, Fv, Fc)
    x1e, _, _ = G.forward(random_theta(np.random.default_rng(4 + 1000)), Re, Ce, Fv, Fc)
    assert not np.allclose(x1, x1e)


def test_bf16_rounding():
    """BF16 keeps 7 fraction bits: near 1 the spacing is 2^-7 and ties go to the even value."""
    P = G.unpack(np.zeros(G.param_count()))
    P["Ev"][0, 0] = 1.0 + 2.0 ** -8                # tie between 1 and 1 + 2^-7: to 1 (even)
    P["Ev"][0, 1] = 1.0 + 3 * 2.0 ** -8            # tie between 1 + 2^-7 and 1 + 2^-6: to 1 + 2^-6
    P["Ev"][0, 2] = 1.0 + 2.0 ** -8 + 2.0 ** -20   # above the tie: up to 1 + 2^-7
    P["Ev"][0, 3] = -(1.0 + 2.0 ** -8 + 2.0 ** -20)
    P["ev"][0] = 1.0 + 2.0 ** -9                   # a bias: FP32, unchanged
    r = G.unpack(G.round_weights_bf16(G.pack(P)))
    assert r["Ev"][0, 0] == 1.0
    assert r["Ev"][0, 1] == 1.0 + 2.0 ** -6
    assert r["Ev"][0, 2] == 1.0 + 2.0 ** -7
    assert r["Ev"][0, 3] == -(1.0 + 2.0 ** -7)
    assert r["ev"][0] == 1.0 + 2.0 ** -9


def _routing_theta(block_constraints=False):
    """Weights that route one channel: hv0 = Fv[:, 0], then per round c = R v (channel 0 of
    the constraint update) and v = v + C c (channel 0 of the variable update), heads read
    channel 0.  With block_constraints a bias of -1e6 zeroes every constraint state."""
    P = G.unpack(np.zeros(G.param_count()))
    P["Ev"][0, 0] = 1.0
    for l in range(G.L):
        P[f"Vc{l}"][0, 0] = 1.0
        if block_constraints:
            P[f"bc{l}"][0] = -1e6
        P[f"Uv{l}"][0, 0] = 1.0
        P[f"Vv{l}"][0, 0] = 1.0
    P["wx"][0] = 1.0
    P["wy"][0] = 1.0
    return G.pack(P)


def test_routed_channel_closed_form():
    """With non-negative entries and inputs every ReLU passes its argument, and the network
    reduces to the linear recurrence c <- R v, v <- v + C c over its L rounds: x_hat =
    (I + C R)^L v0 and y_hat = R (I + C R)^(L-1) v0.  A variable update that read the
    constraint state from before the round, an aggregation applied the wrong way, a round
    too many or too few, or heads on the wrong state would each change these."""
    rng = np.random.default_rng(11)
    n, m = 7, 5
    A = abs(random_graph(rng, n, m))
    R, C = G.aggregation(n, m, A.indptr, A.indices, A.data)
    Fv = np.abs(rng.standard_normal((n, G.F)))
    Fc = rng.standard_normal((m, G.F))
    v0 = Fv[:, 0]
    M = np.eye(n) + (C @ R).toarray()
    x, y, _ = G.forward(_routing_theta(), R, C, Fv, Fc)
    np.testing.assert_allclose(x, np.linalg.matrix_power(M, G.L) @ v0, rtol=1e-13)
    np.testing.assert_allclose(y, R @ (np.linalg.matrix_power(M, G.L - 1) @ v0), rtol=1e-13)
    # a large negative bias in the constraint update: its ReLU stops every message
    x, y, _ = G.forward(_routing_theta(block_constraints=True), R, C, Fv, Fc)
    assert np.array_equal(x, v0) and np.all(y == 0.0)
