"""Seeded input generators: PRNG, PEG matrices, BSC frames, bit packing."""
import numpy as np
import pytest
import scipy.sparse as sp

import mbp_inputs as mi

M64 = (1 << 64) - 1


def _splitmix64(state):
    state = (state + 0x9E3779B97F4A7C15) & M64
    z = state
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
    return state, z ^ (z >> 31)


def _rotl(x, k):
    return ((x << k) | (x >> (64 - k))) & M64


def _xoshiro_ref(seed, count):
    # xoshiro256** (Blackman & Vigna 2018) seeded by splitmix64, from the published definition
    st, s = seed & M64, []
    for _ in range(4):
        st, v = _splitmix64(st)
        s.append(v)
    out = []
    for _ in range(count):
        out.append((_rotl((s[1] * 5) & M64, 7) * 9) & M64)
        t = (s[1] << 17) & M64
        s[2] ^= s[0]
        s[3] ^= s[1]
        s[1] ^= s[2]
        s[0] ^= s[3]
        s[2] ^= t
        s[3] = _rotl(s[3], 45)
    return out


def test_splitmix64_known_answer():
    # first output of splitmix64 from state 0 (Vigna's reference implementation)
    assert _splitmix64(0)[1] == 0xE220A8397B1DCDAF


@pytest.mark.parametrize("seed", [0, 1, 12345, 2**63 + 7])
def test_xoshiro_matches_definition(seed):
    got = mi.xoshiro_stream(seed, 64)
    assert [int(v) for v in got] == _xoshiro_ref(seed, 64)


def test_pack_unpack_roundtrip():
    rng = np.random.default_rng(3)
    for nb in [1, 31, 32, 33, 100, 1024]:
        bits = rng.integers(0, 2, size=(3, nb), dtype=np.uint8)
        w = mi.pack_bits(bits)
        assert w.shape == (3, (nb + 31) // 32) and w.dtype == np.uint32
        assert np.array_equal(mi.unpack_bits(w, nb), bits)
        # LSB-first layout: bit i in word i >> 5 at position i & 31
        i = nb - 1
        assert ((w[:, i >> 5] >> np.uint32(i & 31)) & 1).tolist() == bits[:, i].tolist()


def test_degree_sequence_rounding():
    d = mi.degree_sequence(65536, {2: 0.3, 3: 0.4, 8: 0.3})
    assert np.bincount(d).tolist()[2:] == [19661, 26214, 0, 0, 0, 0, 19661]
    assert int(d.sum()) == 275252
    assert np.all(np.diff(d) >= 0)
    assert mi.checks_for_rate(65536, 0.7) == 19661


def _check_csr(h: mi.CSR, var_deg):
    assert h.row_ptr[0] == 0 and np.all(np.diff(h.row_ptr) >= 0)
    assert np.all((h.col_idx >= 0) & (h.col_idx < h.n))
    assert np.array_equal(h.col_degrees(), var_deg)
    for j in range(h.m):
        row = h.col_idx[h.row_ptr[j]:h.row_ptr[j + 1]]
        assert np.all(np.diff(row) > 0), "columns ascending, no duplicate edge"


def _has_4cycle(h: mi.CSR) -> bool:
    A = sp.csr_matrix((np.ones(h.nnz, np.int32), h.col_idx, h.row_ptr), shape=(h.m, h.n))
    G = (A @ A.T).tocoo()
    off = G.row != G.col
    return bool(np.any(G.data[off] > 1))


def test_peg_small_regular():
    var_deg = mi.degree_sequence(1024, {3: 1.0})
    H = mi.make_codes(1024, 512, {3: 1.0}, 2, 0)
    for h in H:
        _check_csr(h, var_deg)
        rd = h.row_degrees()
        assert rd.sum() == 3072 and rd.max() - rd.min() <= 2
        assert not _has_4cycle(h)
    assert not np.array_equal(H[0].col_idx, H[1].col_idx), "the u matrices differ"


def test_peg_deterministic_and_seeded():
    a = mi.make_codes(256, 128, {2: 0.5, 3: 0.5}, 2, 7)
    b = mi.make_codes(256, 128, {2: 0.5, 3: 0.5}, 2, 7)
    c = mi.make_codes(256, 128, {2: 0.5, 3: 0.5}, 2, 8)
    for x, y in zip(a, b):
        assert np.array_equal(x.row_ptr, y.row_ptr) and np.array_equal(x.col_idx, y.col_idx)
    assert not np.array_equal(a[0].col_idx, c[0].col_idx)


@pytest.mark.slow
def test_peg_large_irregular_no_4cycles():
    dist = {2: 0.3, 3: 0.4, 8: 0.3}
    H = mi.make_codes(65536, 19661, dist, 2, 1)
    var_deg = mi.degree_sequence(65536, dist)
    for h in H:
        _check_csr(h, var_deg)
        rd = h.row_degrees()
        assert h.nnz == 275252 and rd.min() >= 13 and rd.max() <= 15
        assert not _has_4cycle(h)


def test_peg_rejects_impossible():
    with pytest.raises(RuntimeError):
        mi.peg_matrix(4, 2, np.array([3, 1, 1, 1], np.int32), 0)


def test_bsc_frames_statistics():
    x, y, e = mi.bsc_frames(4096, 16, 0.05, seed=11)
    xb, yb = mi.unpack_bits(x, 4096), mi.unpack_bits(y, 4096)
    rate = (xb ^ yb).mean()
    assert abs(rate - 0.05) < 4 * np.sqrt(0.05 * 0.95 / xb.size)
    assert abs(xb.mean() - 0.5) < 4 * np.sqrt(0.25 / xb.size)
    x2, y2, _ = mi.bsc_frames(4096, 16, 0.05, seed=11)
    assert np.array_equal(x, x2) and np.array_equal(y, y2)
    _, _, ev = mi.bsc_frames(64, 3, [0.01, 0.02, 0.03], seed=1)
    assert ev.tolist() == [0.01, 0.02, 0.03]
