"""Iteration 1 in row form (BSC inputs: one sign word per check and one magnitude per check degree and frame)
against the per-edge form, through the C ABI.

Single-code streaming decodes of BSC frames keep iteration 1 in row form when the code allows it; the
persistent kernels of the grouped decode always keep per-edge messages. The two are separate
implementations of the same per-frame arithmetic, so their outputs (bits, iterations, success flags,
posteriors) must be equal bit for bit. The codes cover the three variable-node paths of the row form: check
degrees within four values (the bit-transpose kernel), a wide check-degree spread (the shuffle kernel), and a
check of more than 32 edges (row form off). Converged frames also equal the FP64 oracle's bits.
"""
import numpy as np
import pytest
import torch

import mbp_inputs as mi
import oracle as orc

pytestmark = pytest.mark.gpu

DIST = {2: 0.3, 3: 0.4, 8: 0.3}
KEYS = ("x_hat_bits", "iters", "success", "soft")


@pytest.fixture(scope="module")
def mbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07979_gb300 as m
    m.build()
    return m


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def i32(a):
    return np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)


def row_degrees(H):
    return np.concatenate([np.diff(np.asarray(h.row_ptr)) for h in H])


def code(kind, n=3000):
    if kind == "narrow":  # PEG rows: a degree or two around the mean
        return mi.make_codes(n, 1000, DIST, 2, 81), 0.035
    if kind == "wide":  # two matrices of different rates: check degrees about 5 and 16
        return mi.make_codes(n, 2400, DIST, 1, 82) + mi.make_codes(n, 800, DIST, 1, 83), 0.03
    return mi.make_codes(n, 300, DIST, 2, 84), 0.004  # checks of about 42 edges


@pytest.mark.parametrize("kind", ["narrow", "wide", "long"])
@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_row_form_equals_per_edge_form(mbp, kind, msg):
    H, qber = code(kind)
    deg = row_degrees(H)
    spread, dmax = int(deg.max() - deg[deg > 0].min()), int(deg.max())
    if kind == "narrow":
        assert spread <= 3 and dmax <= 32
    elif kind == "wide":
        assert spread > 3 and dmax <= 32
    else:
        assert dmax > 32
    n, F = H[0].n, 70  # 3 tiles, the last one ragged (and unpaired for 2-byte messages)
    x, y, e = mi.bsc_frames(n, F, qber, seed=90)
    codes = mbp.mbp_create_codes(H)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    dt = {"f32": mbp.MSG_F32, "f16": mbp.MSG_F16, "bf16": mbp.MSG_BF16}[msg]
    yd, ed = dev(i32(y)), dev(e)
    a = mbp.mbp_decode_bsc(codes, yd, ed, z, 30, msg_dtype=dt, want_soft=True, schedule=mbp.SCHED_STREAMING)
    g = [dict(codes=codes, z_bits=z, F=F, y_bits=yd, qber=ed)]
    mbp.mbp_multi_set_tuning(g, dict(grid_kernels=0, cn_warps=8, cn_waves=1, vn_warps=8, syn_warps=8), msg_dtype=dt)
    b = mbp.mbp_decode_multi(g, 30, msg_dtype=dt, want_soft=True)[0]
    torch.cuda.synchronize()
    for k in KEYS:
        assert torch.equal(a[k], b[k]), (kind, msg, k)
    ref = orc.decode(H, orc.bsc_llr(y, n, e), orc.syndrome(H, x), 30, threads=8)
    conv = ref["success"].astype(bool) & a["success"].cpu().numpy().astype(bool)
    assert conv.sum() >= 60
    assert np.array_equal(a["x_hat_bits"].cpu().numpy().view(np.uint32)[conv], ref["x_hat_bits"][conv])


def test_row_form_export_after_one_and_two_iterations(mbp):
    """The message export after a one-iteration decode rebuilds the row form; after two it reads per-edge
    messages; both equal the oracle's C2V within the FP32 tolerance."""
    H, qber = code("wide")
    n, F = H[0].n, 40
    x, y, e = mi.bsc_frames(n, F, 0.05, seed=91)
    codes = mbp.mbp_create_codes(H)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    for t in (1, 2):
        out = mbp.mbp_decode_bsc(codes, dev(i32(y)), dev(e), z, t, early_exit=False,
                                 schedule=mbp.SCHED_STREAMING)
        ref = orc.decode(H, orc.bsc_llr(y, n, e), orc.syndrome(H, x), t, early_exit=False, want_c2v=True)["c2v"]
        for f in (0, 17, 39):
            c = mbp.mbp_export_c2v(codes, F, out["workspace"], f, schedule=mbp.SCHED_STREAMING).cpu().numpy()
            assert np.max(np.abs(c - ref[f])) <= 1e-3, (t, f)


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_more_than_32_tiles(mbp, msg):
    """1115 frames = 35 tiles: the kernels that take one tile per lane (stopping test, iteration-1 row signs)
    run a second, ragged chunk of 3 tiles. Streaming (row form) equals the persistent per-edge kernels, and a
    sample of frames from both chunks equals the oracle's bits where it converges."""
    H, qber = code("narrow", n=2000)
    n, F = H[0].n, 35 * 32 - 5
    x, y, e = mi.bsc_frames(n, F, 0.04, seed=92)
    codes = mbp.mbp_create_codes(H)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    dt = {"f32": mbp.MSG_F32, "f16": mbp.MSG_F16}[msg]
    yd, ed = dev(i32(y)), dev(e)
    a = mbp.mbp_decode_bsc(codes, yd, ed, z, 30, msg_dtype=dt, want_soft=True, schedule=mbp.SCHED_STREAMING)
    g = [dict(codes=codes, z_bits=z, F=F, y_bits=yd, qber=ed)]
    mbp.mbp_multi_set_tuning(g, dict(grid_kernels=0, cn_warps=8, cn_waves=1, vn_warps=8, syn_warps=8), msg_dtype=dt)
    b = mbp.mbp_decode_multi(g, 30, msg_dtype=dt, want_soft=True)[0]
    torch.cuda.synchronize()
    for k in KEYS:
        assert torch.equal(a[k], b[k]), (msg, k)
    idx = np.r_[0:24, 1020:1060, F - 24:F]
    ref = orc.decode(H, orc.bsc_llr(y[idx], n, e[idx]), orc.syndrome(H, x[idx]), 30, threads=8)
    conv = ref["success"].astype(bool) & a["success"].cpu().numpy()[idx].astype(bool)
    assert conv.sum() >= 70
    assert np.array_equal(a["x_hat_bits"].cpu().numpy().view(np.uint32)[idx][conv], ref["x_hat_bits"][conv])
