"""Algorithm variants on the GPU against the FP64 oracle, through the C ABI: the min-sum check rule and the
matrix-serial update order (Algorithm 1's loop nesting), alone and combined.

Same acceptance as the plain decoder: output bits, success flags and per-matrix syndrome passes bit-exact on
every frame where the oracle converges; posteriors within 1e-3 of FP64 over iterations 1..5 (FP32 storage).
"""
import numpy as np
import pytest
import torch

import mbp_inputs as mi
import oracle as orc

pytestmark = pytest.mark.gpu


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


VARIANTS = [("min-sum", "flooding"), ("sum-product", "matrix-serial"), ("min-sum", "matrix-serial")]


def args(mbp, rule, update):
    return dict(rule=mbp.RULE_MIN_SUM if rule == "min-sum" else mbp.RULE_SUM_PRODUCT,
                update=mbp.UPDATE_MATRIX_SERIAL if update == "matrix-serial" else mbp.UPDATE_FLOODING)


class Case:
    def __init__(self, mbp, n, m, u, seed, F, qber):
        self.n, self.F = n, F
        self.H = mi.make_codes(n, m, {2: 0.3, 3: 0.4, 8: 0.3}, u, seed)
        self.x, self.y, self.e = mi.bsc_frames(n, F, qber, seed=seed + 50)
        self.LP = orc.bsc_llr(self.y, n, self.e)
        self.z_orc = orc.syndrome(self.H, self.x)
        self.codes = mbp.mbp_create_codes(self.H)
        self.z = mbp.mbp_syndrome(self.codes, dev(i32(self.x)))
        self.yd, self.ed = dev(i32(self.y)), dev(self.e)


@pytest.mark.parametrize("rule,update", VARIANTS)
@pytest.mark.parametrize("u", [2, 3])
def test_variant_outputs_match_oracle(mbp, rule, update, u):
    # min-sum decodes fewer frames than eq. (6) at equal noise: it is run at a lower QBER
    c = Case(mbp, 4000, 1200 if u == 2 else 900, u, 30 + u, 45, 0.012 if rule == "min-sum" else 0.03)
    out = mbp.mbp_decode_bsc(c.codes, c.yd, c.ed, c.z, 40, want_synd=True, **args(mbp, rule, update))
    ref = orc.decode(c.H, c.LP, c.z_orc, 40, threads=8, want_synd=True, rule=rule, update=update)
    conv = ref["success"].astype(bool)
    assert conv.sum() >= 30
    xh = out["x_hat_bits"].cpu().numpy().view(np.uint32)
    assert np.array_equal(out["success"].cpu().numpy()[conv], ref["success"][conv])
    assert np.array_equal(xh[conv], ref["x_hat_bits"][conv])
    assert np.array_equal(out["synd_ok"].cpu().numpy()[conv], ref["synd_ok"][conv])
    mism = int(np.sum(out["iters"].cpu().numpy()[conv] != ref["iters"][conv]))
    print(f"{rule}/{update} u={u}: {int(conv.sum())} converged, mean iterations "
          f"{ref['iters'][conv].mean():.2f}, iteration-count mismatches {mism}")
    # near a decision FP32 and FP64 can take different iteration counts (more often with min-sum)
    assert mism <= max(2, int(conv.sum()) // 8)


@pytest.mark.parametrize("rule,update", VARIANTS)
@pytest.mark.parametrize("t", [1, 2, 3, 5])
def test_variant_posteriors_within_tolerance(mbp, rule, update, t):
    c = Case(mbp, 2000, 700, 2, 41, 40, 0.05)
    out = mbp.mbp_decode_bsc(c.codes, c.yd, c.ed, c.z, t, early_exit=False, want_soft=True, **args(mbp, rule, update))
    ref = orc.decode(c.H, c.LP, c.z_orc, t, early_exit=False, want_lv=True, threads=8, rule=rule, update=update)
    err = float(np.max(np.abs(out["soft"].cpu().numpy() - ref["L_V"])))
    print(f"{rule}/{update} t={t}: max |dL_V| = {err:.3g}")
    assert err <= 1e-3


@pytest.mark.parametrize("msg", ["f16", "bf16"])
def test_minsum_with_half_storage_runs(mbp, msg):
    """Min-sum with FP16/BF16 message storage: converged frames agree with the oracle's bits."""
    c = Case(mbp, 4000, 1200, 2, 47, 40, 0.012)
    dt = mbp.MSG_F16 if msg == "f16" else mbp.MSG_BF16
    out = mbp.mbp_decode_bsc(c.codes, c.yd, c.ed, c.z, 40, msg_dtype=dt, rule=mbp.RULE_MIN_SUM)
    ref = orc.decode(c.H, c.LP, c.z_orc, 40, threads=8, rule="min-sum")
    conv = ref["success"].astype(bool) & out["success"].cpu().numpy().astype(bool)
    assert conv.sum() >= 30
    assert np.array_equal(out["x_hat_bits"].cpu().numpy().view(np.uint32)[conv], ref["x_hat_bits"][conv])


def test_serial_single_matrix_equals_flooding(mbp):
    c = Case(mbp, 2000, 900, 1, 51, 33, 0.04)
    a = mbp.mbp_decode_bsc(c.codes, c.yd, c.ed, c.z, 30, want_soft=True)
    b = mbp.mbp_decode_bsc(c.codes, c.yd, c.ed, c.z, 30, want_soft=True, update=mbp.UPDATE_MATRIX_SERIAL)
    for k in ("x_hat_bits", "iters", "success", "soft"):
        assert torch.equal(a[k], b[k]), k


def test_variants_refused_where_unsupported(mbp):
    c = Case(mbp, 1000, 400, 2, 52, 8, 0.03)
    for kw in (dict(rule=mbp.RULE_MIN_SUM, schedule=mbp.SCHED_RESIDENT),
               dict(update=mbp.UPDATE_MATRIX_SERIAL, accumulate=mbp.ACC_FIXED),
               dict(rule=mbp.RULE_MIN_SUM, schedule=mbp.SCHED_GRAPH)):
        with pytest.raises(mbp.MBPError) as ei:
            mbp.mbp_decode_bsc(c.codes, c.yd, c.ed, c.z, 10, **kw)
        assert ei.value.status == 5
    llr = dev(c.LP)
    with pytest.raises(mbp.MBPError) as ei:
        mbp.mbp_decode_batch(c.codes, llr, c.z, 10, rule=mbp.RULE_MIN_SUM)
    assert ei.value.status == 5
