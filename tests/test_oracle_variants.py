"""Pins of the oracle's algorithm variants (CPU): the min-sum check rule and the matrix-serial schedule.

  * min-sum check rule: equal to eq. (6) on degree-2 checks; same sign as eq. (6) and a magnitude
    bracketed by |eq. (6)| <= |min-sum| <= |eq. (6)| + ln(d - 1); equivariant under edge permutations;
    a syndrome bit of 1 negates every output.
  * min-sum decoding of tree codes reaches the exact max-log posteriors (brute-force minimum costs).
  * matrix-serial schedule: identical to flooding for u = 1; reaches the exact bitwise-MAP posteriors on
    tree codes (any schedule does on a tree); differs from flooding after one iteration for u = 2; every
    reported success satisfies all syndromes.
"""
import math

import numpy as np
import pytest

import mbp_inputs as mi
import oracle as orc
import test_oracle_pins as pins


@pytest.mark.parametrize("z", [0, 1])
def test_minsum_equals_sum_product_on_degree_two(z):
    rng = np.random.default_rng(z)
    for _ in range(20):
        v = rng.normal(scale=6.0, size=2)
        assert np.array_equal(orc.check_node_minsum(v, z), orc.check_node(v, z))


@pytest.mark.parametrize("d", [3, 4, 6, 8])
def test_minsum_bracketed_by_sum_product(d):
    rng = np.random.default_rng(d)
    for _ in range(50):
        v = rng.normal(scale=4.0, size=d)
        z = int(rng.integers(0, 2))
        ms, sp = orc.check_node_minsum(v, z), orc.check_node(v, z)
        assert np.all(np.sign(ms) == np.sign(sp))
        assert np.all(np.abs(ms) >= np.abs(sp) - 1e-12)
        assert np.all(np.abs(ms) <= np.abs(sp) + math.log(d - 1) + 1e-12)
        perm = rng.permutation(d)
        assert np.array_equal(orc.check_node_minsum(v[perm], z), ms[perm])
        assert np.array_equal(orc.check_node_minsum(v, 1 - z), -ms)


def exact_maxlog_llr(dens, z_list, LP, n):
    """min over valid keys with x_i = 1 of sum_j x_j L_P,j minus the same with x_i = 0 (max-log posterior)."""
    X = ((np.arange(2 ** n)[:, None] >> np.arange(n)[None, :]) & 1).astype(np.uint8)
    ok = np.ones(2 ** n, bool)
    for h, z in zip(dens, z_list):
        ok &= np.all((X.astype(np.int64) @ h.T.astype(np.int64)) % 2 == z[None, :], axis=1)
    Xo = X[ok]
    cost = Xo.astype(np.float64) @ LP
    return np.array([cost[Xo[:, i] == 1].min() - cost[Xo[:, i] == 0].min() for i in range(n)])


def tree_case(u, trial):
    rng = np.random.default_rng(7000 + 100 * u + trial)
    while True:
        try:
            n, H, dens = pins.random_tree_codes(int(rng.integers(8, 14)), u, rng)
            break
        except ValueError:
            continue
    e = 0.25
    x = rng.integers(0, 2, size=(1, n), dtype=np.uint8)
    y = x ^ (rng.random((1, n)) < e).astype(np.uint8)
    zs = [((h.astype(np.int64) @ x[0].astype(np.int64)) % 2).astype(np.uint8) for h in dens]
    LP = orc.bsc_llr(mi.pack_bits(y), n, e)
    return n, H, dens, zs, y, e, LP


@pytest.mark.parametrize("u", [1, 2, 3])
@pytest.mark.parametrize("trial", range(3))
def test_minsum_tree_codes_reach_max_log_posteriors(u, trial):
    n, H, dens, zs, y, e, LP = tree_case(u, trial)
    for update in ("flooding", "matrix-serial"):
        out = orc.decode(H, LP, pins.z_bits_from_dense(zs), max_iter=2 * n, early_exit=False, want_lv=True,
                         rule="min-sum", update=update)
        ref = exact_maxlog_llr(dens, zs, LP[0], n)
        assert np.max(np.abs(ref)) < 19.0
        assert np.allclose(out["L_V"][0], ref, atol=1e-9), (update, out["L_V"][0], ref)


@pytest.mark.parametrize("u", [2, 3])
@pytest.mark.parametrize("trial", range(3))
def test_serial_tree_codes_reach_exact_map(u, trial):
    n, H, dens, zs, y, e, LP = tree_case(u, trial)
    out = orc.decode(H, LP, pins.z_bits_from_dense(zs), max_iter=2 * n, early_exit=False, want_lv=True,
                     update="matrix-serial")
    ref = pins.exact_map_llr(dens, zs, y[0], e, n)
    assert np.allclose(out["L_V"][0], ref, atol=1e-9)


def small_code(u, seed=3, n=300, m=120, F=12, qber=0.07):
    H = mi.make_codes(n, m, {2: 0.3, 3: 0.4, 8: 0.3}, u, seed)
    x, y, e = mi.bsc_frames(n, F, qber, seed=seed + 1)
    return H, x, orc.bsc_llr(y, n, e), orc.syndrome(H, x)


def test_serial_equals_flooding_for_one_matrix():
    H, x, LP, z = small_code(1)
    for rule in ("sum-product", "min-sum"):
        a = orc.decode(H, LP, z, 15, want_lv=True, rule=rule)
        b = orc.decode(H, LP, z, 15, want_lv=True, rule=rule, update="matrix-serial")
        for k in ("x_hat_bits", "iters", "success", "L_V"):
            assert np.array_equal(a[k], b[k]), (rule, k)


def test_serial_differs_from_flooding_for_two_matrices_and_successes_are_valid():
    H, x, LP, z = small_code(2)
    a = orc.decode(H, LP, z, 1, early_exit=False, want_lv=True)
    b = orc.decode(H, LP, z, 1, early_exit=False, want_lv=True, update="matrix-serial")
    assert not np.allclose(a["L_V"], b["L_V"])
    H, x, LP, z = small_code(2, qber=0.04)
    for rule in ("sum-product", "min-sum"):
        out = orc.decode(H, LP, z, 30, rule=rule, update="matrix-serial")
        ok = out["success"].astype(bool)
        assert ok.sum() >= 1
        zz = orc.syndrome(H, out["x_hat_bits"][ok])
        for l in range(2):
            assert np.array_equal(zz[l], z[l][ok])
