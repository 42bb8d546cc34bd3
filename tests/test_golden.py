"""The FP64 oracle against tests/golden/oracle_small_decode.json (written by tests/golden/make_golden.py from
the oracle itself): a regression guard, so that any change to the oracle's arithmetic fails here and has to be
justified by the passage of the paper it follows. The oracle's pins are in tests/test_oracle_*.py.

The fixture's own outputs are also checked by plain GF(2) arithmetic written here: every frame the oracle
declares decoded satisfies both matrices' syndromes (eq. 1), and the low-QBER frames decode to Alice's key.
"""
import json
import os
from types import SimpleNamespace

import numpy as np
import pytest

import oracle as orc

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module")
def fx():
    with open(os.path.join(HERE, "oracle_small_decode.json")) as fh:
        d = json.load(fh)
    n = d["n"]
    d["H"] = [SimpleNamespace(n=n, m=h["m"], row_ptr=np.asarray(h["row_ptr"], np.int32),
                              col_idx=np.asarray(h["col_idx"], np.int32)) for h in d["matrices"]]
    for k in ("x_bits", "y_bits"):
        d[k] = np.asarray(d[k], np.uint32)
    d["z_bits"] = [np.asarray(a, np.uint32) for a in d["z_bits"]]
    return d


def bits(words, n):
    w = np.asarray(words, np.uint32)
    return ((w[:, :, None] >> np.arange(32, dtype=np.uint32)) & 1).reshape(w.shape[0], -1)[:, :n]


def test_syndrome_and_channel_reproduce(fx):
    z = orc.syndrome(fx["H"], fx["x_bits"])
    for a, b in zip(z, fx["z_bits"]):
        assert np.array_equal(np.asarray(a, np.uint32), b)


def test_decode_reproduces_fixture(fx):
    n, H = fx["n"], fx["H"]
    LP = orc.bsc_llr(fx["y_bits"], n, np.asarray(fx["qber"]))
    ref = fx["early_exit_20"]
    out = orc.decode(H, LP, fx["z_bits"], 20, l_max=fx["l_max"], want_lv=True, want_synd=True)
    assert out["iters"].tolist() == ref["iters"]
    assert out["success"].tolist() == ref["success"]
    assert out["synd_ok"].tolist() == ref["synd_ok"]
    assert np.array_equal(out["x_hat_bits"], np.asarray(ref["x_hat_bits"], np.uint32))
    assert np.allclose(out["L_V"], np.asarray(ref["L_V"]), rtol=1e-12, atol=1e-9)
    ref2 = fx["fixed_2"]
    out2 = orc.decode(H, LP, fx["z_bits"], 2, l_max=fx["l_max"], early_exit=False, want_lv=True, want_c2v=True)
    assert out2["iters"].tolist() == ref2["iters"]
    assert np.array_equal(out2["x_hat_bits"], np.asarray(ref2["x_hat_bits"], np.uint32))
    assert np.allclose(out2["L_V"], np.asarray(ref2["L_V"]), rtol=1e-12, atol=1e-9)
    assert np.allclose(out2["c2v"][ref2["c2v_frames"]], np.asarray(ref2["c2v"]), rtol=1e-12, atol=1e-9)


def test_fixture_outputs_satisfy_the_syndromes(fx):
    n = fx["n"]
    xh = bits(fx["early_exit_20"]["x_hat_bits"], n)
    x = bits(fx["x_bits"], n)
    ok = np.asarray(fx["early_exit_20"]["success"], bool)
    assert ok.sum() >= 4
    for h, zw in zip(fx["H"], fx["z_bits"]):
        z = bits(zw, h.m)
        for f in np.flatnonzero(ok):
            par = np.array([xh[f, h.col_idx[h.row_ptr[j]:h.row_ptr[j + 1]]].sum() & 1 for j in range(h.m)])
            assert np.array_equal(par, z[f]), f
    q = np.asarray(fx["qber"])
    assert np.array_equal(xh[(q <= 0.05) & ok], x[(q <= 0.05) & ok])
