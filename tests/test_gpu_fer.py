"""Frame error rate of the n = 65536 rate-0.7 two-matrix code against QBER (needs a GB300).

The throughput metric is quoted at a frame error rate of at most 1e-3, so the
frame error rate at the workload's QBER has to be measured on enough frames to
bound it there: 8192 distinct frames per point at QBER 2%, 3% and 4% (FP32,
FP16 and BF16 message storage, default options), and 2048 frames per point from
5% up to the first QBER where frames fail (the waterfall; the paper's Fig. 2
plots success rate against QBER the same way). A frame is in error if it
reports failure or if its output differs from Alice's key (an undetected
error). The one-sided 95% upper bound of the error rate is the Clopper-Pearson
bound (3/N, about, when nothing fails). A sample of frames at every point,
failing ones first, is compared with the FP64 oracle.
"""
import json
import math
import os

import numpy as np
import pytest
import torch

import mbp_inputs as mi
import oracle as orc

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

N, M, DIST, U, SEED = 65536, 19661, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 1
MAX_ITER = 60


@pytest.fixture(scope="module")
def mbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07979_gb300 as m
    m.build()
    return m


def upper95(k, n):
    """One-sided 95% Clopper-Pearson upper bound of a rate with k events in n trials."""
    if k >= n:
        return 1.0
    if k == 0:
        return 1.0 - 0.05 ** (1.0 / n)
    from scipy.stats import beta
    return float(beta.ppf(0.95, k + 1, n - k))


def run_point(mbp, H, codes, q, frames, msg, seed):
    x, y, e = mi.bsc_frames(N, frames, q, seed=seed, stream=int(round(q * 1000)))
    yd = torch.from_numpy(y.view(np.int32)).cuda()
    ed = torch.from_numpy(e).cuda()
    zd = mbp.mbp_syndrome(codes, torch.from_numpy(x.view(np.int32)).cuda())
    out = mbp.mbp_decode_bsc(codes, yd, ed, zd, MAX_ITER, msg_dtype=msg)
    xh = out["x_hat_bits"].cpu().numpy().view(np.uint32)
    ok = out["success"].cpu().numpy().astype(bool)
    it = out["iters"].cpu().numpy()
    wrong = ~np.all(xh == x, axis=1)
    fail = ~ok
    undetected = ok & wrong
    err = fail | undetected
    # oracle on a sample: every failing frame (up to 4) and 4 spread over the batch
    sample = np.unique(np.concatenate([np.nonzero(err)[0][:4], np.linspace(0, frames - 1, 4).astype(int)]))
    ref = orc.decode(H, orc.bsc_llr(y[sample], N, e[sample]), orc.syndrome(H, x[sample]), MAX_ITER, threads=8)
    conv = ref["success"].astype(bool)
    assert np.array_equal(ref["x_hat_bits"][conv], xh[sample][conv]), "outputs differ where the oracle converged"
    assert np.array_equal(ok[sample][conv], ref["success"][conv])
    k = int(err.sum())
    return {"qber": q, "frames": frames, "failures": int(fail.sum()), "undetected": int(undetected.sum()),
            "fer": k / frames, "fer_upper95": upper95(k, frames), "mean_iterations": float(it.mean()),
            "max_iterations": int(it.max()), "oracle_sample": len(sample),
            "oracle_failures_in_sample": int((~conv).sum()), "gpu_failures_in_sample": int((~ok[sample]).sum())}


def test_fer_against_qber_headline_code(mbp):
    H = mi.make_codes(N, M, DIST, U, SEED)
    codes = mbp.mbp_create_codes(H)
    rows = []
    for name, msg in (("f32", mbp.MSG_F32), ("f16", mbp.MSG_F16), ("bf16", mbp.MSG_BF16)):
        for q in (0.02, 0.03, 0.04):
            r = run_point(mbp, H, codes, q, 8192, msg, seed=51)
            r["msg"] = name
            rows.append(r)
            print(json.dumps(r))
            if q == 0.02:
                assert r["fer_upper95"] < 1e-3, r
    waterfall = None
    for q in (0.05, 0.06, 0.065, 0.07, 0.08, 0.09, 0.10, 0.11, 0.12):
        r = run_point(mbp, H, codes, q, 2048, mbp.MSG_F32, seed=52)
        r["msg"] = "f32"
        rows.append(r)
        print(json.dumps(r))
        if r["fer"] > 0:
            waterfall = q
            if r["fer"] > 0.5:
                break
    assert waterfall is not None, "no QBER up to 12% made a frame fail"
    out_dir = os.environ.get("MBP_RESULTS_DIR")  # where to keep the table as JSON, if anywhere
    if out_dir:
        os.makedirs(out_dir, exist_ok=True)
        with open(os.path.join(out_dir, "fer_vs_qber.json"), "w") as f:
            json.dump(rows, f, indent=1)
