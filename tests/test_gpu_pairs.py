"""Message storage in tile pairs (tiles 2q and 2q + 1 store an edge's messages together: one 32-bit word
per lane for FP16 / BF16, two adjacent 128-byte lines for FP32), through the C ABI.

Each frame's arithmetic is independent of the other frames: the per-frame outputs of a decode (bits,
iterations, success, posteriors) must not change, bit for bit, with the batch the frame is decoded in. The
batches here put a frame alone in a tile (no partner tile), beside a partner tile that retires iterations
earlier, in an odd tile count and in a ragged last tile. Converged frames must also equal the FP64
oracle's bits, for BSC and LLR inputs and the matrix-serial order.
"""
import numpy as np
import pytest
import torch

import mbp_inputs as mi
import oracle as orc

pytestmark = pytest.mark.gpu

KEYS = ("x_hat_bits", "iters", "success", "soft")


@pytest.fixture(scope="module")
def mbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07979_gb300 as m
    m.build()
    return m


MSG = {"f32": lambda m: m.MSG_F32, "f16": lambda m: m.MSG_F16, "bf16": lambda m: m.MSG_BF16}


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def i32(a):
    return np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)


class Mixed:
    """80 frames = 3 tiles (the last one ragged): the first 32 at QBER 0.5% (they retire after one or two
    iterations), the rest at 4%."""

    def __init__(self, mbp, n=4000, m=1400, u=2, seed=61):
        self.n = n
        self.H = mi.make_codes(n, m, {2: 0.3, 3: 0.4, 8: 0.3}, u, seed)
        self.e = np.concatenate([np.full(32, 0.005), np.full(48, 0.04)])
        self.F = len(self.e)
        self.x, self.y, _ = mi.bsc_frames(n, self.F, self.e, seed=seed + 1)
        self.codes = mbp.mbp_create_codes(self.H)

    def decode(self, mbp, idx, dt, **kw):
        idx = np.asarray(idx)
        z = mbp.mbp_syndrome(self.codes, dev(i32(self.x[idx])))
        out = mbp.mbp_decode_bsc(self.codes, dev(i32(self.y[idx])), dev(self.e[idx]), z, 40, msg_dtype=dt,
                                 want_soft=True, **kw)
        return {k: out[k].cpu().numpy() for k in KEYS}


@pytest.fixture(scope="module")
def mixed(mbp):
    return Mixed(mbp)


@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_pair_storage_frames_independent_of_batch(mbp, mixed, msg):
    dt = MSG[msg](mbp)
    full = mixed.decode(mbp, np.arange(mixed.F), dt)
    its = full["iters"]
    assert its[:32].max() < its[32:].max()  # the first tile retires before its partner
    subsets = [np.arange(32), np.arange(32, 80), np.array([40]), np.arange(0, 80, 3), np.arange(79, -1, -1)]
    for idx in subsets:
        part = mixed.decode(mbp, idx, dt)
        for k in KEYS:
            assert np.array_equal(part[k], full[k][idx]), (msg, k, idx[:4])
    graph = mixed.decode(mbp, np.arange(mixed.F), dt, schedule=mbp.SCHED_GRAPH)
    for k in KEYS:
        assert np.array_equal(graph[k], full[k]), (msg, k)


@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_pair_storage_converged_frames_match_oracle(mbp, mixed, msg):
    dt = MSG[msg](mbp)
    out = mixed.decode(mbp, np.arange(mixed.F), dt)
    LP = orc.bsc_llr(mixed.y, mixed.n, mixed.e)
    ref = orc.decode(mixed.H, LP, orc.syndrome(mixed.H, mixed.x), 40, threads=8)
    conv = ref["success"].astype(bool) & out["success"].astype(bool)
    assert conv.sum() >= 75
    assert np.array_equal(out["x_hat_bits"].view(np.uint32)[conv], ref["x_hat_bits"][conv])


@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_pair_storage_llr_inputs_and_serial_order(mbp, mixed, msg):
    """General LLR inputs (the first iteration reads L_P through the pair kernel) and the matrix-serial order
    (row ranges per matrix, messages cleared to 0 first): converged frames equal the oracle's bits."""
    dt = MSG[msg](mbp)
    LP = orc.bsc_llr(mixed.y, mixed.n, mixed.e)
    z_orc = orc.syndrome(mixed.H, mixed.x)
    z = mbp.mbp_syndrome(mixed.codes, dev(i32(mixed.x)))
    out = mbp.mbp_decode_batch(mixed.codes, dev(LP.astype(np.float32)), z, 40, msg_dtype=dt)
    ref = orc.decode(mixed.H, LP, z_orc, 40, threads=8)
    conv = ref["success"].astype(bool) & out["success"].cpu().numpy().astype(bool)
    assert conv.sum() >= 75
    assert np.array_equal(out["x_hat_bits"].cpu().numpy().view(np.uint32)[conv], ref["x_hat_bits"][conv])
    ser = mbp.mbp_decode_bsc(mixed.codes, dev(i32(mixed.y)), dev(mixed.e), z, 40, msg_dtype=dt,
                             update=mbp.UPDATE_MATRIX_SERIAL)
    ref_s = orc.decode(mixed.H, LP, z_orc, 40, threads=8, update="matrix-serial")
    conv = ref_s["success"].astype(bool) & ser["success"].cpu().numpy().astype(bool)
    assert conv.sum() >= 75
    assert np.array_equal(ser["x_hat_bits"].cpu().numpy().view(np.uint32)[conv], ref_s["x_hat_bits"][conv])


def test_half_storage_first_iteration_messages_odd_tiles(mbp):
    """After one iteration every exported FP16 message of 70 frames (3 tiles, the third without a partner)
    is the oracle's C2V rounded to FP16 storage: within half an FP16 unit of the largest clipped message."""
    n, F = 2000, 70
    H = mi.make_codes(n, 800, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 62)
    x, y, e = mi.bsc_frames(n, F, 0.05, seed=63)
    codes = mbp.mbp_create_codes(H)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    out = mbp.mbp_decode_bsc(codes, dev(i32(y)), dev(e), z, 1, early_exit=False, msg_dtype=mbp.MSG_F16)
    ref = orc.decode(H, orc.bsc_llr(y, n, e), orc.syndrome(H, x), 1, early_exit=False, want_c2v=True)["c2v"]
    for f in (0, 31, 32, 63, 64, 69):
        c = mbp.mbp_export_c2v(codes, F, out["workspace"], f, mbp.MSG_F16).cpu().numpy()
        # |C2V| <= l_max = 20 < 32: FP16 spacing <= 2^-6 there, rounding error <= 2^-7, plus FP32 arithmetic
        assert np.max(np.abs(c - ref[f])) <= 2.0 ** -7 + 1e-3, f


def test_f32_pair_messages_odd_tiles(mbp):
    """FP32 messages of 70 frames (3 tiles, the third without a partner) after one iteration on LLR inputs
    (the pair kernel's first iteration) and after two (old messages read back from the pair's two lines):
    every exported C2V within 1e-3 of the oracle's."""
    n, F = 2000, 70
    H = mi.make_codes(n, 800, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 64)
    x, y, e = mi.bsc_frames(n, F, 0.05, seed=65)
    codes = mbp.mbp_create_codes(H)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    LP = orc.bsc_llr(y, n, e)
    for t in (1, 2):
        out = mbp.mbp_decode_batch(codes, dev(LP.astype(np.float32)), z, t, early_exit=False,
                                   schedule=mbp.SCHED_STREAMING)
        ref = orc.decode(H, LP, orc.syndrome(H, x), t, early_exit=False, want_c2v=True)["c2v"]
        for f in (0, 31, 32, 63, 64, 69):
            c = mbp.mbp_export_c2v(codes, F, out["workspace"], f, schedule=mbp.SCHED_STREAMING).cpu().numpy()
            assert np.max(np.abs(c - ref[f])) <= 1e-3, (t, f)


@pytest.mark.parametrize("msg", ["f32", "f16"])
def test_pair_kernels_on_long_rows(mbp, msg):
    """A rate-0.8 code (check rows of about 21 edges: the pair check kernel's longest unroll bounds, 22 and 24),
    70 frames (3 tiles, the last ragged and unpaired): streaming decodes through the pair kernels equal the
    persistent per-edge kernels bit for bit, and converged frames equal the oracle's bits."""
    n = 3000
    H = mi.make_codes(n, 600, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 66)
    deg = np.concatenate([np.diff(np.asarray(h.row_ptr)) for h in H])
    assert 18 < deg.max() <= 24
    F = 70
    x, y, e = mi.bsc_frames(n, F, 0.02, seed=67)  # 3 to 5 iterations per frame
    codes = mbp.mbp_create_codes(H)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    dt = MSG[msg](mbp)
    yd, ed = dev(i32(y)), dev(e)
    a = mbp.mbp_decode_bsc(codes, yd, ed, z, 40, msg_dtype=dt, want_soft=True, schedule=mbp.SCHED_STREAMING)
    g = [dict(codes=codes, z_bits=z, F=F, y_bits=yd, qber=ed)]
    mbp.mbp_multi_set_tuning(g, dict(grid_kernels=0, cn_warps=8, cn_waves=1, vn_warps=8, syn_warps=8), msg_dtype=dt)
    b = mbp.mbp_decode_multi(g, 40, msg_dtype=dt, want_soft=True)[0]
    torch.cuda.synchronize()
    for k in KEYS:
        assert torch.equal(a[k], b[k]), (msg, k)
    ref = orc.decode(H, orc.bsc_llr(y, n, e), orc.syndrome(H, x), 40, threads=8)
    conv = ref["success"].astype(bool) & a["success"].cpu().numpy().astype(bool)
    assert conv.sum() >= 60
    assert np.array_equal(a["x_hat_bits"].cpu().numpy().view(np.uint32)[conv], ref["x_hat_bits"][conv])


def test_frames_ordered_by_qber_keep_the_callers_order(mbp):
    """BSC frames are placed in the decoder's tiles in order of QBER (ties by index) and the outputs go back to
    the caller's order. 100 frames with QBERs from 0.5% to 12% in shuffled order (so every tile holds frames of
    other positions, and some frames fail): FP64 outputs, iteration counts, success and per-matrix flags equal
    the oracle's frame by frame, the soft output equals the oracle's posterior and mbp_export_c2v of a frame
    returns that frame's messages (after two iterations without early exit); FP32 decodes of the shuffled
    batch (graph and streaming schedules) equal those of the same frames in another order, frame by frame."""
    n, F = 2000, 100
    H = mi.make_codes(n, 800, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 68)
    rng = np.random.default_rng(69)
    e = rng.permutation(np.linspace(0.005, 0.12, F))
    x, y, _ = mi.bsc_frames(n, F, e, seed=70)
    codes = mbp.mbp_create_codes(H)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    LP = orc.bsc_llr(y, n, e)
    z_orc = orc.syndrome(H, x)
    yd, ed = dev(i32(y)), dev(e)
    ref = orc.decode(H, LP, z_orc, 30, threads=8, want_lv=True, want_synd=True)
    ok = ref["success"].astype(bool)
    assert F // 2 < ok.sum() < F  # frames that decode and frames that do not
    out = mbp.mbp_decode_bsc(codes, yd, ed, z, 30, msg_dtype=mbp.MSG_F64, want_soft=True, want_synd=True)
    # the decoded frames' outputs (a frame still failing after 30 iterations may wander at the last bits); a
    # frame's outputs written to another frame's place would show on the decoded frames
    assert np.array_equal(out["iters"].cpu().numpy()[ok], ref["iters"][ok])
    assert np.array_equal(out["success"].cpu().numpy()[ok], ref["success"][ok])
    assert abs(int(out["success"].sum()) - int(ok.sum())) <= 2
    assert np.array_equal(out["x_hat_bits"].cpu().numpy().view(np.uint32)[ok], ref["x_hat_bits"][ok])
    assert np.array_equal(out["synd_ok"].cpu().numpy()[ok], ref["synd_ok"][ok])
    assert np.max(np.abs(out["soft"].cpu().numpy()[ok] - ref["L_V"][ok])) <= 1e-9
    two = mbp.mbp_decode_bsc(codes, yd, ed, z, 2, early_exit=False, msg_dtype=mbp.MSG_F64)
    ref2 = orc.decode(H, LP, z_orc, 2, early_exit=False, want_c2v=True)["c2v"]
    order = np.argsort(e, kind="stable")
    for f in (int(order[0]), int(order[-1]), int(order[33]), 0, F - 1):
        c = mbp.mbp_export_c2v(codes, F, two["workspace"], f, mbp.MSG_F64).cpu().numpy()
        assert np.max(np.abs(c - ref2[f])) <= 1e-9, f
    perm = rng.permutation(F)
    for sched in (mbp.SCHED_GRAPH, mbp.SCHED_STREAMING):
        a = mbp.mbp_decode_bsc(codes, yd, ed, z, 30, want_soft=True, schedule=sched)
        zp = mbp.mbp_syndrome(codes, dev(i32(x[perm])))
        b = mbp.mbp_decode_bsc(codes, dev(i32(y[perm])), dev(e[perm]), zp, 30, want_soft=True, schedule=sched)
        for k in KEYS:
            assert torch.equal(a[k][perm], b[k]), (sched, k)
