"""Write oracle_small_decode.json: a regression fixture of the FP64 oracle on a small two-matrix code.

The paper prints no worked decoding example, so no fixture here holds the paper's own values. This one records
what the oracle computes, so that a later change to the oracle's arithmetic shows up as a failing test
(tests/test_golden.py) and has to be justified by the passage of the paper it follows. It is not a pin: the
oracle's pins are the closed forms, enumerations and invariants of tests/test_oracle_*.py.

It calls only oracle/ (the decoder) and mbp_inputs/ (the seeded PEG code and BSC frames, stored in the fixture
so that the test does not depend on the generators):

    python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import mbp_inputs as mi  # noqa: E402
import oracle as orc  # noqa: E402

N, M, U, SEED = 96, 48, 2, 7
DIST = {2: 0.3, 3: 0.4, 8: 0.3}
QBER = [0.02, 0.05, 0.08, 0.10, 0.12, 0.15]
C2V_FRAMES = [0, 4]  # messages (stacked CSR edge order) kept for two frames, to keep the file small


def main():
    H = mi.make_codes(N, M, DIST, U, SEED)
    x, y, e = mi.bsc_frames(N, len(QBER), np.asarray(QBER), seed=SEED + 1)
    z = orc.syndrome(H, x)
    LP = orc.bsc_llr(y, N, e)
    full = orc.decode(H, LP, z, 20, want_lv=True, want_synd=True)
    two = orc.decode(H, LP, z, 2, early_exit=False, want_lv=True, want_c2v=True)
    w = lambda a: [[int(v) for v in row] for row in np.asarray(a, np.uint32)]
    f = lambda a: [[float(v) for v in row] for row in np.asarray(a, np.float64)]
    fixture = {
        "about": "FP64 oracle outputs on a small two-matrix PEG code (regression fixture, not a pin); written by "
                 "tests/golden/make_golden.py",
        "n": N, "l_max": orc.L_MAX_DEFAULT,
        "matrices": [{"m": h.m, "row_ptr": h.row_ptr.tolist(), "col_idx": h.col_idx.tolist()} for h in H],
        "qber": [float(v) for v in e], "x_bits": w(x), "y_bits": w(y), "z_bits": [w(a) for a in z],
        "early_exit_20": {"iters": full["iters"].tolist(), "success": full["success"].tolist(),
                          "synd_ok": full["synd_ok"].tolist(), "x_hat_bits": w(full["x_hat_bits"]),
                          "L_V": f(full["L_V"])},
        "fixed_2": {"iters": two["iters"].tolist(), "x_hat_bits": w(two["x_hat_bits"]), "L_V": f(two["L_V"]),
                    "c2v_frames": C2V_FRAMES, "c2v": f(two["c2v"][C2V_FRAMES])},
    }
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "oracle_small_decode.json")
    with open(out, "w") as fh:
        json.dump(fixture, fh, indent=None, separators=(",", ":"))
        fh.write("\n")
    print(out, "iters", full["iters"].tolist(), "success", full["success"].tolist())


if __name__ == "__main__":
    main()
