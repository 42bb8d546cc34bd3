"""Pins of the FP64 oracle against things other than itself.

Each test ties one part of the oracle to a fact fixed by the paper or by the
mathematics: the probabilistic definition of eq. (6) by enumeration, exact
bitwise-MAP posteriors of tree codes by enumeration (eqs. 2, 5, 6 and
Algorithm 1 together), dense GF(2) products (eq. 1), GF(2) elimination,
invariants of the stopping rule (Section 2) and equivariances.
"""
import itertools
import math

import numpy as np
import pytest

import mbp_inputs as mi
import oracle as orc


# ----------------------------------------------------------------- helpers

def dense_syndrome(codes, x_bits, n):
    x = mi.unpack_bits(x_bits, n).astype(np.int64)
    return [(h.dense().astype(np.int64) @ x.T % 2).T.astype(np.uint8) for h in codes]


def csr_from_dense(h):
    m, n = h.shape
    rp = np.zeros(m + 1, np.int32)
    cols = []
    for j in range(m):
        c = np.nonzero(h[j])[0]
        cols.extend(c.tolist())
        rp[j + 1] = rp[j] + len(c)
    return mi.CSR(n, m, rp, np.asarray(cols, np.int32))


def random_tree_codes(n_target, u, rng, max_new=3):
    """u matrices whose stacked Tanner graph is a tree (checks of degree 2..4)."""
    nvar, checks = 1, []
    while nvar < n_target:
        k = int(rng.integers(1, max_new + 1))
        k = min(k, n_target - nvar)
        anchor = int(rng.integers(0, nvar))
        checks.append((int(rng.integers(0, u)), [anchor] + list(range(nvar, nvar + k))))
        nvar += k
    n = nvar
    dens = []
    for l in range(u):
        rows = [c for (ll, c) in checks if ll == l]
        h = np.zeros((max(len(rows), 1), n), np.uint8)
        for j, c in enumerate(rows):
            h[j, c] = 1
        if not rows:  # keep every matrix non-empty: give it one degree-2 check on a fresh edge pair
            raise ValueError("empty matrix")
        dens.append(h)
    return n, [csr_from_dense(h) for h in dens], dens


def exact_map_llr(dens, z_list, y_bits_row, e, n):
    """Bitwise-MAP LLR ln P(x_i=0|y,z)/P(x_i=1|y,z) by enumeration of all 2^n keys."""
    X = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    ok = np.ones(2 ** n, bool)
    for h, z in zip(dens, z_list):
        ok &= np.all((X.astype(np.int64) @ h.T.astype(np.int64)) % 2 == z[None, :], axis=1)
    d = (X[ok] ^ y_bits_row[None, :]).sum(axis=1)
    logw = d * math.log(e) + (n - d) * math.log(1 - e)  # BSC likelihood P(y|x)
    w = np.exp(logw - logw.max())
    Xo = X[ok]
    out = np.empty(n)
    for i in range(n):
        out[i] = math.log(w[Xo[:, i] == 0].sum() / w[Xo[:, i] == 1].sum())
    return out


def z_bits_from_dense(zs, F=1):
    return [mi.pack_bits(z.reshape(F, -1)) for z in zs]


# -------------------------------------------------------------- eq. (5)

@pytest.mark.parametrize("e", [0.001, 0.02, 0.03, 0.1, 0.3])
def test_bsc_llr_is_channel_likelihood_ratio(e):
    # L_P = ln P(y|x=0) / P(y|x=1) for the binary symmetric channel with crossover e
    y = np.array([[0, 1, 1, 0, 1]], np.uint8)
    L = orc.bsc_llr(mi.pack_bits(y), 5, e)[0]
    for yi, li in zip(y[0], L):
        p_y_given_0 = (1 - e) if yi == 0 else e
        p_y_given_1 = e if yi == 0 else (1 - e)
        assert li == pytest.approx(math.log(p_y_given_0 / p_y_given_1), abs=1e-13)


def test_bsc_llr_named_values():
    # e = 0.02 -> ln 49, e = 0.03 -> ln(97/3): the magnitudes quoted for the benchmark workloads
    L = orc.bsc_llr(mi.pack_bits(np.array([[0, 1]], np.uint8)), 2, 0.02)[0]
    assert L[0] == pytest.approx(3.891820298110627, abs=1e-12) and L[1] == pytest.approx(-3.891820298110627)
    L = orc.bsc_llr(mi.pack_bits(np.array([[0]], np.uint8)), 1, 0.03)[0]
    assert L[0] == pytest.approx(3.4760986898352733, abs=1e-12)


# -------------------------------------------------------------- eq. (6)

def xor_llr_enumerated(llrs):
    """LLR of the XOR of independent bits with the given LLRs, by enumeration."""
    p0 = [1.0 / (1.0 + math.exp(-a)) for a in llrs]
    P = [0.0, 0.0]
    for bits in itertools.product([0, 1], repeat=len(llrs)):
        pr = 1.0
        for b, q in zip(bits, p0):
            pr *= q if b == 0 else 1 - q
        P[sum(bits) % 2] += pr
    return math.log(P[0] / P[1])


@pytest.mark.parametrize("d", [2, 3, 4, 6])
@pytest.mark.parametrize("z", [0, 1])
def test_check_node_is_parity_posterior(d, z):
    rng = np.random.default_rng(100 + d + 10 * z)
    for _ in range(20):
        v = rng.normal(0, 3, size=d)
        c = orc.check_node(v, z)
        for k in range(d):
            ref = xor_llr_enumerated([v[r] for r in range(d) if r != k])
            assert c[k] == pytest.approx((-1) ** z * ref, abs=1e-10)


def test_check_node_degree2_passes_the_other_message():
    for z in (0, 1):
        c = orc.check_node([1.25, -7.5], z)
        assert c[0] == (-1) ** z * -7.5 and c[1] == (-1) ** z * 1.25


def test_check_node_degree1_is_clipped_infinity():
    assert orc.check_node([0.3], 0, 20.0)[0] == 20.0
    assert orc.check_node([0.3], 1, 20.0)[0] == -20.0


def test_check_node_forms_agree_and_symmetries():
    rng = np.random.default_rng(5)
    for _ in range(50):
        d = int(rng.integers(2, 15))
        v = rng.normal(0, 4, size=d)
        a = orc.check_node(v, 0)
        mask = np.abs(a) < 15
        assert np.allclose(a[mask], orc.check_node_tanh(v, 0)[mask], atol=1e-9)
        assert np.allclose(orc.check_node(v, 1), -a, atol=0)
        p = rng.permutation(d)
        assert np.allclose(orc.check_node(v[p], 0), a[p], atol=1e-12)


def test_check_node_saturation_against_high_precision():
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    for v in ([20.0, 20.0, 20.0], [20.0, -19.5, 20.0, 18.0], [20.0] * 14, [20.0, 1e-6, 20.0]):
        c = orc.check_node(v, 0)
        for k in range(len(v)):
            p = mpmath.mpf(1)
            for r in range(len(v)):
                if r != k:
                    p *= mpmath.tanh(mpmath.mpf(v[r]) / 2)
            ref = float(2 * mpmath.atanh(p))
            assert c[k] == pytest.approx(max(min(ref, 20.0), -20.0), abs=1e-9)


def test_boxplus_identities():
    assert orc.boxplus(3.0, 0.0) == pytest.approx(0.0, abs=1e-15)
    assert orc.boxplus(-2.0, 5.0) == pytest.approx(orc.boxplus(5.0, -2.0), abs=1e-15)
    assert orc.boxplus(40.0, 1.5) == pytest.approx(1.5, abs=1e-15)


# -------------------------------------------------------------- eq. (1)

def test_syndrome_against_dense_gf2_and_linearity():
    H = mi.make_codes(300, 120, {2: 0.4, 3: 0.6}, 3, 4)
    rng = np.random.default_rng(1)
    a = mi.pack_bits(rng.integers(0, 2, (5, 300), dtype=np.uint8))
    b = mi.pack_bits(rng.integers(0, 2, (5, 300), dtype=np.uint8))
    za, zb, zab = orc.syndrome(H, a), orc.syndrome(H, b), orc.syndrome(H, a ^ b)
    dense = dense_syndrome(H, a, 300)
    for l in range(3):
        assert np.array_equal(mi.unpack_bits(za[l], 120), dense[l])
        assert np.array_equal(za[l] ^ zb[l], zab[l])


# ---------------------------------------------- Algorithm 1, whole decoder

@pytest.mark.parametrize("u", [1, 2, 3])
@pytest.mark.parametrize("trial", range(4))
def test_tree_codes_reach_exact_map(u, trial):
    rng = np.random.default_rng(1000 * u + trial)
    while True:
        try:
            n, H, dens = random_tree_codes(int(rng.integers(8, 15)), u, rng)
            break
        except ValueError:
            continue
    e = 0.25
    x = rng.integers(0, 2, size=(1, n), dtype=np.uint8)
    noise = (rng.random((1, n)) < e).astype(np.uint8)
    y = x ^ noise
    zs = [(h.astype(np.int64) @ x[0].astype(np.int64)) % 2 for h in dens]
    LP = orc.bsc_llr(mi.pack_bits(y), n, e)
    out = orc.decode(H, LP, z_bits_from_dense([z.astype(np.uint8) for z in zs]), max_iter=2 * n,
                     early_exit=False, want_lv=True)
    ref = exact_map_llr(dens, zs, y[0], e, n)
    assert np.max(np.abs(ref)) < 19.0, "case must stay inside the clip"
    assert np.allclose(out["L_V"][0], ref, atol=1e-9), (out["L_V"][0], ref)


def gf2_solve(A, b):
    """Solve A x = b over GF(2) for full-column-rank A; returns (x, rank)."""
    A = A.copy().astype(np.uint8)
    b = b.copy().astype(np.uint8)
    m, n = A.shape
    row, piv = 0, []
    for col in range(n):
        r = np.nonzero(A[row:, col])[0]
        if r.size == 0:
            continue
        r = row + r[0]
        if r != row:
            A[[row, r]] = A[[r, row]]
            b[[row, r]] = b[[r, row]]
        hit = np.nonzero(A[:, col])[0]
        hit = hit[hit != row]
        A[hit] ^= A[row]
        b[hit] ^= b[row]
        piv.append(col)
        row += 1
        if row == m:
            break
    x = np.zeros(n, np.uint8)
    for i, col in enumerate(piv):
        x[col] = b[i]
    return x, len(piv)


def test_small_code_converged_frames_are_the_unique_solution():
    """Rate-0.5 n=1024 code, u=2: u*m = n, so the stacked H is square."""
    H = mi.make_codes(1024, 512, {3: 1.0}, 2, 0)
    x, y, e = mi.bsc_frames(1024, 64, 0.03, seed=0)
    z = orc.syndrome(H, x)
    out = orc.decode(H, orc.bsc_llr(y, 1024, e), z, 50, threads=4, want_synd=True)
    stacked = np.concatenate([h.dense() for h in H])
    _, rank = gf2_solve(stacked, np.zeros(1024, np.uint8))
    dense_ok = dense_syndrome(H, out["x_hat_bits"], 1024)
    zd = [mi.unpack_bits(zl, 512) for zl in z]
    for f in range(64):
        sat = all(np.array_equal(dense_ok[l][f], zd[l][f]) for l in range(2))
        assert bool(out["success"][f]) == sat
        assert out["synd_ok"][f].tolist() == [int(np.array_equal(dense_ok[l][f], zd[l][f])) for l in range(2)]
        if out["success"][f] and rank == 1024:
            sol, _ = gf2_solve(stacked, np.concatenate([zd[0][f], zd[1][f]]))
            assert np.array_equal(mi.unpack_bits(out["x_hat_bits"][f], 1024), sol)
    assert out["success"].all() and np.array_equal(out["x_hat_bits"], x)


def test_noise_free_frame_stops_before_iterating():
    H = mi.make_codes(512, 200, {3: 1.0}, 2, 3)
    x, _, _ = mi.bsc_frames(512, 3, 0.0, seed=2)
    out = orc.decode(H, orc.bsc_llr(x, 512, 0.02), orc.syndrome(H, x), 10)
    assert out["iters"].tolist() == [0, 0, 0] and out["success"].all()
    assert np.array_equal(out["x_hat_bits"], x)


def test_stacked_matrices_equal_single_matrix_bp():
    """MBP(H_1..H_u) equals single-matrix BP on [H_1; ...; H_u] with stacked syndromes."""
    H = mi.make_codes(400, 150, {2: 0.3, 3: 0.7}, 2, 9)
    x, y, e = mi.bsc_frames(400, 6, 0.06, seed=3)
    z = orc.syndrome(H, x)
    LP = orc.bsc_llr(y, 400, e)
    a = orc.decode(H, LP, z, 30, want_lv=True)
    stacked = csr_from_dense(np.concatenate([h.dense() for h in H]))
    zs = [mi.pack_bits(np.concatenate([mi.unpack_bits(z[0], 150), mi.unpack_bits(z[1], 150)], axis=1))]
    b = orc.decode([stacked], LP, zs, 30, want_lv=True)
    assert np.array_equal(a["iters"], b["iters"]) and np.array_equal(a["x_hat_bits"], b["x_hat_bits"])
    assert np.allclose(a["L_V"], b["L_V"], atol=1e-12)


def test_column_and_row_permutation_equivariance():
    H = mi.make_codes(300, 120, {2: 0.3, 3: 0.7}, 2, 12)
    x, y, e = mi.bsc_frames(300, 4, 0.07, seed=5)
    z = orc.syndrome(H, x)
    LP = orc.bsc_llr(y, 300, e)
    base = orc.decode(H, LP, z, 8, early_exit=False, want_lv=True)
    rng = np.random.default_rng(0)
    p = rng.permutation(300)  # new column c holds old column p[c]
    Hp = [csr_from_dense(h.dense()[:, p]) for h in H]
    out = orc.decode(Hp, LP[:, p], z, 8, early_exit=False, want_lv=True)
    assert np.allclose(out["L_V"], base["L_V"][:, p], atol=1e-12)
    # row permutation of each matrix with the syndrome bits permuted alike
    q = [rng.permutation(h.m) for h in H]
    Hr = [csr_from_dense(h.dense()[qq]) for h, qq in zip(H, q)]
    zr = [mi.pack_bits(mi.unpack_bits(zl, h.m)[:, qq]) for zl, h, qq in zip(z, H, q)]
    out = orc.decode(Hr, LP, zr, 8, early_exit=False, want_lv=True)
    assert np.allclose(out["L_V"], base["L_V"], atol=1e-12)


def test_loopy_tiny_codes_invariants_and_ml_bound():
    """n = 14 loopy codes: successes satisfy every syndrome; BP never beats ML on average."""
    rng = np.random.default_rng(77)
    n, e = 14, 0.12
    X = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    bp_err = ml_err = trials = 0
    for _ in range(12):
        dens = [(rng.random((5, n)) < 0.3).astype(np.uint8) for _ in range(2)]
        for h in dens:
            for j in range(h.shape[0]):
                if h[j].sum() < 2:
                    h[j, rng.choice(n, 2, replace=False)] = 1
        H = [csr_from_dense(h) for h in dens]
        for _ in range(10):
            x = rng.integers(0, 2, size=(1, n), dtype=np.uint8)
            y = x ^ (rng.random((1, n)) < e).astype(np.uint8)
            zs = [((h.astype(np.int64) @ x[0]) % 2).astype(np.uint8) for h in dens]
            out = orc.decode(H, orc.bsc_llr(mi.pack_bits(y), n, e), z_bits_from_dense(zs), 30)
            xh = mi.unpack_bits(out["x_hat_bits"], n)[0]
            if out["success"][0]:
                for h, z in zip(dens, zs):
                    assert np.array_equal((h.astype(np.int64) @ xh) % 2, z)
            ok = np.ones(2 ** n, bool)
            for h, z in zip(dens, zs):
                ok &= np.all((X.astype(np.int64) @ h.T) % 2 == z[None, :], axis=1)
            cand = X[ok]
            dist = (cand ^ y[0][None, :]).sum(axis=1)
            best = cand[np.argmin(dist)]
            ml_err += int(not np.array_equal(best, x[0]))
            bp_err += int(not (out["success"][0] and np.array_equal(xh, x[0])))
            trials += 1
    assert bp_err >= ml_err - 3 * math.sqrt(trials * 0.25)


# ------------------------------------- message clip inside whole decodes
#
# The paper has no guard against atanh(+-1) or message growth (eq. 6); the
# decoder clips every variable-to-check message to [-L_max, L_max] before eq. (6)
# and every check-to-variable message after it, so that an empty combination
# (a degree-1 check, +inf) becomes +-L_max. These cases pin that reading inside
# whole decodes, on codes where the clip is reached, against enumeration and
# closed forms that do not run the oracle's message passing.

def _star(K, u, deg1_matrix, rng, L, group=(1, 2)):
    """Centre variable 0 and K leaf groups: group k (one or two fresh leaves, sizes cycling through `group`) is
    joined to the centre by one check of matrix k % u (degree 2 or 3), plus one degree-1 check on the centre in
    matrix `deg1_matrix`. Leaf priors reach up to 3 L. Returns n, the dense matrices, syndromes, priors and
    the leaves of each group."""
    n, leaves = 1, []
    for k in range(K):
        g = group[k % len(group)]
        leaves.append(list(range(n, n + g)))
        n += g
    rows = [[] for _ in range(u)]
    for k in range(K):
        rows[k % u].append([0] + leaves[k])
    rows[deg1_matrix].append([0])
    dens = []
    for l in range(u):
        h = np.zeros((len(rows[l]), n), np.uint8)
        for j, c in enumerate(rows[l]):
            h[j, c] = 1
        dens.append(h)
    zs = [rng.integers(0, 2, size=h.shape[0]).astype(np.uint8) for h in dens]
    LP = np.empty(n)
    LP[0] = rng.uniform(-1.0, 1.0)
    LP[1:] = rng.choice([-1.0, 1.0], size=n - 1) * rng.uniform(0.3 * L, 3.0 * L, size=n - 1)
    return n, dens, zs, LP, leaves


def _map_llr_from_priors(dens, zs, LP, i):
    """ln P(x_i = 0 | checks) / P(x_i = 1 | checks) for independent priors of LLR LP, by enumeration."""
    n = len(LP)
    X = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.int64)
    ok = np.ones(2 ** n, bool)
    for h, z in zip(dens, zs):
        if h.shape[0]:
            ok &= np.all((X @ h.T.astype(np.int64)) % 2 == z[None, :].astype(np.int64), axis=1)
    # log P(x) up to a constant: sum over bits of -LP_k x_k (LLR = ln P(0)/P(1))
    logw = -(X[ok] * LP[None, :]).sum(axis=1)
    w = np.exp(logw - logw.max())
    Xo = X[ok]
    return math.log(w[Xo[:, i] == 0].sum() / w[Xo[:, i] == 1].sum())


def _replace_degree1_by_aux(dens, L):
    """A degree-1 check on x_i with syndrome z is, after the clip, the message (-1)^z L_max: the same as a
    degree-2 check (x_i, a) with syndrome z on a fresh variable a of prior +L_max. Returns the extended
    matrices and the number of auxiliary variables (appended after the code's own)."""
    n = dens[0].shape[1]
    n_aux = sum(int((h.sum(axis=1) == 1).sum()) for h in dens)
    out, a = [], n
    for h in dens:
        g = np.zeros((h.shape[0], n + n_aux), np.uint8)
        g[:, :n] = h
        for j in range(h.shape[0]):
            if h[j].sum() == 1:
                g[j, a] = 1
                a += 1
        out.append(g)
    return out, n_aux


@pytest.mark.parametrize("u", [1, 2, 3])
@pytest.mark.parametrize("trial", range(3))
def test_clip_star_centre_is_map_of_clipped_leaves(u, trial):
    """Centre of a star: after any iteration t >= 1 each leaf check sends eq. (6) of its leaves' clipped priors
    (a leaf has no other check) and the degree-1 check (-1)^z L_max, so the centre's posterior is the exact
    bitwise MAP of the same code with every leaf prior clipped to L_max and the degree-1 check replaced by an
    auxiliary variable of prior L_max. On the degree-3 leaf checks the clip before eq. (6) decides the message
    (on degree-2 ones the clip after it would give the same)."""
    rng = np.random.default_rng(7000 + 10 * u + trial)
    L = 4.0
    n, dens, zs, LP, _ = _star(6, u, trial % u, rng, L)
    assert np.max(np.abs(LP)) > L, "case must reach the clip"
    H = [csr_from_dense(h) for h in dens]
    for T in (1, 2, 5):
        out = orc.decode(H, LP[None, :], z_bits_from_dense(zs), T, l_max=L, early_exit=False, want_lv=True)
        ext, n_aux = _replace_degree1_by_aux(dens, L)
        LPc = np.concatenate([[LP[0]], np.clip(LP[1:], -L, L), np.full(n_aux, L)])
        ref = _map_llr_from_priors(ext, zs, LPc, 0)
        assert out["L_V"][0, 0] == pytest.approx(ref, abs=1e-12), (T, out["L_V"][0, 0], ref)


@pytest.mark.parametrize("u", [1, 2])
@pytest.mark.parametrize("trial", range(3))
def test_clip_star_leaves_take_the_clipped_centre_extrinsic(u, trial):
    """A leaf of a star from iteration 2 on: its only check k sends it the LLR of the XOR of the check's other
    bits (eq. 6, by enumeration) given the clipped message of each: clip(E_k, L_max) from the centre, where E_k
    is the MAP LLR of the centre in the code without check k (leaf priors clipped, degree-1 check as an
    auxiliary variable of prior L_max; enumeration), and clip(L_P, L_max) from the other leaf of a degree-3
    check. The centre's message exceeds L_max here, so the clip before eq. (6) decides the result."""
    rng = np.random.default_rng(7100 + 10 * u + trial)
    L = 3.0
    n, dens, zs, LP, leaves = _star(6, u, 0, rng, L)
    H = [csr_from_dense(h) for h in dens]
    out = orc.decode(H, LP[None, :], z_bits_from_dense(zs), 4, l_max=L, early_exit=False, want_lv=True)
    ext, n_aux = _replace_degree1_by_aux(dens, L)
    LPc = np.concatenate([[LP[0]], np.clip(LP[1:], -L, L), np.full(n_aux, L)])
    reached = 0
    for k, grp in enumerate(leaves):
        l = k % u
        j = int(np.nonzero(dens[l][:, grp[0]])[0][0])
        without = [g if q != l else np.delete(g, j, axis=0) for q, g in enumerate(ext)]
        zw = [z if q != l else np.delete(z, j) for q, z in enumerate(zs)]
        E = _map_llr_from_priors(without, zw, LPc, 0)
        reached += abs(E) > L
        for a in grp:
            others = [float(np.clip(E, -L, L))] + [float(np.clip(LP[b], -L, L)) for b in grp if b != a]
            ref = LP[a] + (-1) ** int(zs[l][j]) * xor_llr_enumerated(others)
            assert out["L_V"][0, a] == pytest.approx(ref, abs=1e-12), (a, out["L_V"][0, a], ref)
    assert reached >= 1, "case must reach the variable-to-check clip"


def _chain(K, u, rng, L):
    """Path x_0 - x_1 - ... - x_{K-1}: check j joins (x_j, x_{j+1}) in matrix j % u; a degree-1 check on x_0
    in matrix 0."""
    rows = [[] for _ in range(u)]
    for j in range(K - 1):
        rows[j % u].append((j, [j, j + 1]))
    rows[0].append((-1, [0]))
    dens, where = [], {}
    for l in range(u):
        h = np.zeros((len(rows[l]), K), np.uint8)
        for r, (j, c) in enumerate(rows[l]):
            h[r, c] = 1
            where[j] = (l, r)
        dens.append(h)
    zs = [rng.integers(0, 2, size=h.shape[0]).astype(np.uint8) for h in dens]
    LP = rng.choice([-1.0, 1.0], size=K) * rng.uniform(0.2 * L, 2.5 * L, size=K)
    return dens, zs, LP, where


@pytest.mark.parametrize("u", [1, 2, 3])
@pytest.mark.parametrize("trial", range(3))
def test_clip_chain_closed_form(u, trial):
    """On a path every check has degree 2 (it passes the other side's message with the sign of its syndrome
    bit) and every variable at most two checks, so the message entering x_i from the left is
    a_i = s_{i-1} clip(L_P,{i-1} + a_{i-1}, L_max) with a_0 the degree-1 check's s L_max, the one from the
    right b_i = s_i clip(L_P,{i+1} + b_{i+1}, L_max) with b_{K-1} = 0, and after K iterations (the flooding
    messages have then crossed the whole path) the posterior is L_P,i + a_i + b_i."""
    rng = np.random.default_rng(7200 + 10 * u + trial)
    L, K = 3.0, 10
    dens, zs, LP, where = _chain(K, u, rng, L)
    H = [csr_from_dense(h) for h in dens]
    out = orc.decode(H, LP[None, :], z_bits_from_dense(zs), K + 2, l_max=L, early_exit=False, want_lv=True)

    def sign(j):
        l, r = where[j]
        return -1.0 if zs[l][r] else 1.0

    a = np.zeros(K)
    a[0] = sign(-1) * L
    for i in range(1, K):
        a[i] = sign(i - 1) * min(max(LP[i - 1] + a[i - 1], -L), L)
    b = np.zeros(K)
    for i in range(K - 2, -1, -1):
        b[i] = sign(i) * min(max(LP[i + 1] + b[i + 1], -L), L)
    assert np.any(np.abs(LP[:-1] + a[:-1]) > L) and np.any(np.abs(LP[1:] + b[1:]) > L), "case must reach the clip"
    assert np.allclose(out["L_V"][0], LP + a + b, atol=1e-12, rtol=0), (out["L_V"][0], LP + a + b)


@pytest.mark.parametrize("u", [1, 2])
@pytest.mark.parametrize("trial", range(3))
def test_clip_far_away_star_posteriors_exact(u, trial):
    """The clip is only a bound: on a star (a tree) whose exact MAP posteriors exceed 20 in magnitude, a decode
    with L_max far above every message gives the exact bitwise MAP posterior of every variable (enumeration of
    the unclipped problem), as a decode inside the clip does."""
    rng = np.random.default_rng(7300 + 10 * u + trial)
    n, dens, zs, LP, _ = _star(6, u, 0, rng, 5.0, group=(1,))
    dens = [h[h.sum(axis=1) > 1] for h in dens]  # no degree-1 check: its unclipped message is infinite
    x = rng.integers(0, 2, size=n)  # priors that mostly agree with a word of the code, as a channel's do
    zs = [((h.astype(np.int64) @ x) % 2).astype(np.uint8) for h in dens]
    LP = (1.0 - 2.0 * x) * np.abs(LP)
    LP[1] = -LP[1]
    ref = np.array([_map_llr_from_priors(dens, zs, LP, i) for i in range(n)])
    assert np.max(np.abs(ref)) > 20.0, "case must leave the default clip"
    H = [csr_from_dense(h) for h in dens]
    out = orc.decode(H, LP[None, :], z_bits_from_dense(zs), 3, l_max=1e4, early_exit=False, want_lv=True)
    assert np.allclose(out["L_V"][0], ref, atol=1e-9, rtol=1e-12), (out["L_V"][0], ref)
