"""The default decode is asynchronous and stream-ordered (needs a GB300).

With default options a single-code decode of FP32 messages runs the graph
schedule: the iteration loop is one CUDA graph, so the call returns once the
work is queued on the stream, before the GPU has finished it. The outputs, read
after the stream is synchronised, still match the FP64 oracle.
"""
import time

import numpy as np
import pytest
import torch

import mbp_inputs as mi
import oracle as orc

pytestmark = pytest.mark.gpu

N, M, DIST, U, SEED, F, QBER = 65536, 19661, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 1, 1024, 0.02


@pytest.fixture(scope="module")
def mbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07979_gb300 as m
    m.build()
    return m


def test_default_decode_returns_before_the_work_finishes(mbp):
    H = mi.make_codes(N, M, DIST, U, SEED)
    x, y, e = mi.bsc_frames(N, F, QBER, seed=SEED)
    codes = mbp.mbp_create_codes(H)
    yd = torch.from_numpy(y.view(np.int32)).cuda()
    ed = torch.from_numpy(e).cuda()
    zd = mbp.mbp_syndrome(codes, torch.from_numpy(x.view(np.int32)).cuda())
    ws = torch.empty(mbp.mbp_decode_workspace_size(codes, F), dtype=torch.uint8, device="cuda")
    mbp.mbp_decode_bsc(codes, yd, ed, zd, 60, workspace=ws)  # first call: builds and caches the graph
    torch.cuda.synchronize()
    pending = []
    for _ in range(3):
        done = torch.cuda.Event()
        t0 = time.perf_counter()
        out = mbp.mbp_decode_bsc(codes, yd, ed, zd, 60, workspace=ws)
        host_ms = 1e3 * (time.perf_counter() - t0)
        done.record()
        pending.append(not done.query())
        torch.cuda.synchronize()
        print(f"host time of the call {host_ms:.3f} ms, still running on return: {pending[-1]}")
    assert all(pending), "the default decode waited for the GPU"
    torch.cuda.synchronize()
    xh = out["x_hat_bits"].cpu().numpy().view(np.uint32)
    ok = out["success"].cpu().numpy().astype(bool)
    assert ok.all() and np.array_equal(xh, x)
    sample = np.arange(0, F, 131)
    z_orc = orc.syndrome(H, x[sample])
    ref = orc.decode(H, orc.bsc_llr(y[sample], N, e[sample]), z_orc, 60, threads=8)
    assert np.array_equal(ref["x_hat_bits"], xh[sample])
    # iteration counts are a diagnostic (FP32 may cross a decision boundary one iteration apart)
    assert int(np.sum(ref["iters"] != out["iters"].cpu().numpy()[sample])) <= 1
