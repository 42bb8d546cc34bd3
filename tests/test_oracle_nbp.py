"""Pins of the FP64 unrolled normalised-BP reference (oracle/nbp.py), on the CPU.

  * alpha = 1, beta = 0 is the plain decoder: L^t equals the C oracle's posterior after t
    iterations (no early exit) for every t.
  * A row-by-row unrolled evaluation that calls the C oracle's check-node routine (eq. 6) and
    applies the normalisation in plain Python gives the same L^t for random alpha, beta.
  * Closed forms: alpha = 0, or beta >= L_max, leaves every posterior at L_P.
  * The autograd gradient matches central finite differences of the forward.
"""
import numpy as np
import pytest

import mbp_inputs as mi
import oracle as orc
from oracle import nbp

torch = pytest.importorskip("torch")


def small(n=60, m=24, u=2, seed=3, F=3, qber=0.06, dist=None):
    dist = dist or {2: 0.3, 3: 0.4, 8: 0.3}
    H = mi.make_codes(n, m, dist, u, seed)
    x, y, e = mi.bsc_frames(n, F, qber, seed=seed + 100)
    return H, x, y, orc.bsc_llr(y, n, e), orc.syndrome(H, x)


def test_plain_parameters_equal_plain_decoder():
    H, x, y, LP, z = small()
    T = 6
    L = nbp.forward_np(H, LP, z, np.ones((T, 2)), np.zeros((T, 2)))
    for t in range(1, T + 1):
        ref = orc.decode(H, LP, z, t, early_exit=False, want_lv=True)["L_V"]
        assert np.max(np.abs(L[t - 1] - ref)) <= 1e-9, t


def unrolled_by_rows(H, LP, z, alpha, beta, l_max=20.0):
    """Independent evaluation: per frame, per iteration, per stacked row, the C oracle's check-node routine on
    the row's V2C, then the normalisation of the row's matrix and iteration, then eq. (2)."""
    n = H[0].n
    F, T = LP.shape[0], alpha.shape[0]
    rows = []
    for l, h in enumerate(H):
        for j in range(h.m):
            rows.append((l, j, [int(c) for c in h.col_idx[h.row_ptr[j]:h.row_ptr[j + 1]]]))
    out = np.zeros((T, F, n))
    for f in range(F):
        C = [np.zeros(len(cols)) for _, _, cols in rows]
        Lf = LP[f].copy()
        for t in range(T):
            newC = []
            for q, (l, j, cols) in enumerate(rows):
                V = np.clip(Lf[cols] - C[q], -l_max, l_max)
                zj = int((z[l][f, j >> 5] >> np.uint32(j & 31)) & 1)
                c = orc.check_node(V, zj, l_max)
                # sign factor of c: (-1)^z times the signs of the other V (a zero V counts as +)
                sg = np.where(V < 0, -1.0, 1.0)
                s = (-1.0 if zj else 1.0) * np.prod(sg) * sg
                newC.append(alpha[t, l] * s * np.maximum(np.abs(c) - beta[t, l], 0.0))
            C = newC
            Lf = LP[f].copy()
            for q, (_, _, cols) in enumerate(rows):
                for k, col in enumerate(cols):
                    Lf[col] += C[q][k]
            out[t, f] = Lf
    return out


def test_row_by_row_unrolled_evaluation():
    H, x, y, LP, z = small(n=40, m=16, F=2, seed=5)
    rng = np.random.default_rng(0)
    T = 4
    alpha = rng.uniform(0.5, 1.2, size=(T, 2))
    beta = rng.uniform(0.0, 0.8, size=(T, 2))
    L = nbp.forward_np(H, LP, z, alpha, beta)
    ref = unrolled_by_rows(H, LP, z, alpha, beta)
    assert np.max(np.abs(L - ref)) <= 1e-9


def test_closed_forms():
    H, x, y, LP, z = small()
    T = 3
    L0 = nbp.forward_np(H, LP, z, np.zeros((T, 2)), np.zeros((T, 2)))
    assert np.array_equal(L0, np.broadcast_to(LP, L0.shape))
    Lb = nbp.forward_np(H, LP, z, np.ones((T, 2)), np.full((T, 2), 20.0))
    assert np.array_equal(Lb, np.broadcast_to(LP, Lb.shape))


def test_per_matrix_parameters_act_on_their_matrix():
    """Switching off matrix 2's messages (alpha[:, 1] = 0) equals decoding with H_1 alone."""
    H, x, y, LP, z = small(seed=8)
    T = 4
    a = np.ones((T, 2))
    a[:, 1] = 0.0
    L = nbp.forward_np(H, LP, z, a, np.zeros((T, 2)))
    L1 = nbp.forward_np(H[:1], LP, z[:1], np.ones((T, 1)), np.zeros((T, 1)))
    assert np.max(np.abs(L - L1)) <= 1e-12


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_central_differences(seed):
    H, x, y, LP, z = small(n=40, m=16, F=2, seed=seed, qber=0.08)
    rng = np.random.default_rng(seed)
    T = 3
    alpha = rng.uniform(0.6, 1.1, size=(T, 2))
    beta = rng.uniform(0.05, 0.5, size=(T, 2))
    G = rng.normal(size=(T,) + LP.shape)
    _, ga, gb, gl = nbp.gradient(H, LP, z, alpha, beta, G)

    def J(a, b, lp):
        return float(np.sum(G * nbp.forward_np(H, lp, z, a, b)))

    eps = 1e-6
    for (t, l) in [(0, 0), (1, 1), (2, 0)]:
        d = np.zeros_like(alpha)
        d[t, l] = eps
        fd_a = (J(alpha + d, beta, LP) - J(alpha - d, beta, LP)) / (2 * eps)
        fd_b = (J(alpha, beta + d, LP) - J(alpha, beta - d, LP)) / (2 * eps)
        assert abs(fd_a - ga[t, l]) <= 1e-5 * max(1.0, abs(fd_a))
        assert abs(fd_b - gb[t, l]) <= 1e-5 * max(1.0, abs(fd_b))
    for (f, i) in [(0, 3), (1, 17)]:
        d = np.zeros_like(LP)
        d[f, i] = eps
        fd = (J(alpha, beta, LP + d) - J(alpha, beta, LP - d)) / (2 * eps)
        assert abs(fd - gl[f, i]) <= 1e-5 * max(1.0, abs(fd))


def test_bce_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    L = rng.normal(scale=3.0, size=(3, 7))
    x = rng.integers(0, 2, size=(3, 7))
    loss, g = nbp.bce_grad(L, x)
    eps = 1e-6
    for idx in [(0, 0), (2, 5)]:
        d = np.zeros_like(L)
        d[idx] = eps
        fd = (nbp.bce_grad(L + d, x)[0] - nbp.bce_grad(L - d, x)[0]) / (2 * eps)
        assert abs(fd - g[idx]) <= 1e-8
    # P(bit = 1) = sigmoid(-L): a confident correct posterior has a small loss
    assert nbp.bce_grad(np.array([[30.0, -30.0]]), np.array([[0, 1]]))[0] < 1e-12
