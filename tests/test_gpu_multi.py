"""Grouped decode of uneven frames (mbp_decode_multi, mbp_autotune_multi, MBP_SCHED_GRAPH), through the C ABI.

A batch mixes codes of different n, rate and u, per-frame QBERs and ragged
group sizes. Each group's results must equal, bit for bit, a single-code
decode of the same frames with the streaming schedule (the per-row and per-node
arithmetic is the same), and agree with the FP64 oracle on every frame the
oracle decodes (output bits and success flags where it converges).
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


# (n, m per matrix, column-degree distribution, u, code seed, frames, QBER range)
SPECS = [
    (1024, 512, {3: 1.0}, 2, 0, 45, (0.01, 0.04)),
    (2048, 614, {2: 0.3, 3: 0.4, 8: 0.3}, 3, 11, 33, (0.01, 0.03)),
    (4096, 819, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 12, 5, (0.005, 0.02)),
    (1000, 400, {2: 0.5, 3: 0.5}, 1, 13, 70, (0.01, 0.04)),
    (2048, 614, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 14, 0, (0.01, 0.04)),
]


class Group:
    def __init__(self, mbp, spec, fseed):
        n, m, dist, u, seed, F, (lo, hi) = spec
        self.n, self.F = n, F
        self.H = mi.make_codes(n, m, dist, u, seed)
        rng = np.random.default_rng(seed * 7 + fseed)
        self.e = rng.uniform(lo, hi, size=F)
        self.x, self.y, _ = mi.bsc_frames(n, F, self.e, seed=seed * 1000 + fseed)
        self.codes = mbp.mbp_create_codes(self.H)
        self.z = mbp.mbp_syndrome(self.codes, dev(i32(self.x))) if F else torch.zeros(0, dtype=torch.int32,
                                                                                         device="cuda")
        self.yd, self.ed = dev(i32(self.y)), dev(self.e)

    def arg(self, llr=False):
        g = dict(codes=self.codes, z_bits=self.z, F=self.F)
        if llr:
            g["llr"] = dev(orc.bsc_llr(self.y, self.n, self.e).astype(np.float32))
        else:
            g.update(y_bits=self.yd, qber=self.ed)
        return g


@pytest.fixture(scope="module")
def batch(mbp):
    return [Group(mbp, s, i) for i, s in enumerate(SPECS)]


def single(mbp, g, max_iter, early_exit=True, msg_dtype=None, schedule=None):
    msg_dtype = mbp.MSG_F32 if msg_dtype is None else msg_dtype
    schedule = mbp.SCHED_STREAMING if schedule is None else schedule
    return mbp.mbp_decode_bsc(g.codes, g.yd, g.ed, g.z, max_iter, early_exit=early_exit, want_soft=True,
                              want_synd=True, msg_dtype=msg_dtype, schedule=schedule)


KEYS = ("x_hat_bits", "iters", "success", "synd_ok", "soft")


@pytest.mark.parametrize("early_exit", [True, False])
@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_multi_equals_single_code_decodes(mbp, batch, early_exit, msg):
    dt = {"f32": mbp.MSG_F32, "f16": mbp.MSG_F16, "bf16": mbp.MSG_BF16}[msg]
    max_iter = 30 if early_exit else 7
    outs = mbp.mbp_decode_multi([g.arg() for g in batch], max_iter, msg_dtype=dt, early_exit=early_exit,
                                want_soft=True, want_synd=True)
    torch.cuda.synchronize()
    for g, o in zip(batch, outs):
        if g.F == 0:
            assert o["iters"].numel() == 0
            continue
        ref = single(mbp, g, max_iter, early_exit, dt)
        for k in KEYS:
            assert torch.equal(o[k], ref[k]), (g.n, k)


def test_multi_matches_oracle(mbp, batch):
    outs = mbp.mbp_decode_multi([g.arg() for g in batch], 40, want_soft=False, want_synd=True)
    torch.cuda.synchronize()
    converged = 0
    for g, o in zip(batch, outs):
        if g.F == 0:
            continue
        ref = orc.decode(g.H, orc.bsc_llr(g.y, g.n, g.e), orc.syndrome(g.H, g.x), 40, threads=8, want_synd=True)
        conv = ref["success"].astype(bool)
        converged += int(conv.sum())
        xh = o["x_hat_bits"].cpu().numpy().view(np.uint32)
        assert np.array_equal(o["success"].cpu().numpy()[conv], ref["success"][conv])
        assert np.array_equal(xh[conv], ref["x_hat_bits"][conv])
        assert np.array_equal(o["synd_ok"].cpu().numpy()[conv], ref["synd_ok"][conv])
        # every reported success satisfies all of its syndromes
        ok = o["success"].cpu().numpy().astype(bool)
        z = orc.syndrome(g.H, xh[ok])
        for l, zl in enumerate(z):
            assert np.array_equal(zl, orc.syndrome(g.H, g.x[ok])[l])
    assert converged >= 100


def test_llr_groups_equal_bsc_groups(mbp, batch):
    a = mbp.mbp_decode_multi([g.arg() for g in batch], 30, want_soft=True)
    b = mbp.mbp_decode_multi([g.arg(llr=True) for g in batch], 30, want_soft=True)
    torch.cuda.synchronize()
    for g, oa, ob in zip(batch, a, b):
        for k in ("x_hat_bits", "iters", "success"):
            assert torch.equal(oa[k], ob[k]), (g.n, k)
        if g.F:  # L_P rounds differently (LLR input x log2 e vs the BSC magnitude): FP32 relative agreement
            assert torch.allclose(oa["soft"], ob["soft"], rtol=1e-5, atol=1e-4)


def test_host_driven_loop_equals_graph(mbp, batch):
    """Kernel accounting drives the same kernels from the host; results are the same."""
    a = mbp.mbp_decode_multi([g.arg() for g in batch], 30, want_soft=True, want_synd=True)
    torch.cuda.synchronize()
    mbp.mbp_profile_enable(True)
    try:
        b = mbp.mbp_decode_multi([g.arg() for g in batch], 30, want_soft=True, want_synd=True)
        prof = mbp.mbp_profile_get()
    finally:
        mbp.mbp_profile_enable(False)
    for oa, ob in zip(a, b):
        for k in KEYS:
            assert torch.equal(oa[k], ob[k]), k
    assert prof["check"][0] > 0 and prof["variable"][0] > 0 and prof["retire"][0] > 0


def test_autotune_picks_a_candidate_and_keeps_results(mbp, batch):
    ref = mbp.mbp_decode_multi([g.arg() for g in batch], 30)
    torch.cuda.synchronize()
    outs, tu = mbp.mbp_autotune_multi([g.arg() for g in batch], 30)
    assert tu["cn_warps"] in (2, 4, 8) and tu["cn_waves"] in (1, 2) and tu["vn_warps"] in (2, 4, 8)
    assert tu["ms"] > 0
    for oa, ob in zip(ref, outs):
        for k in ("x_hat_bits", "iters", "success"):
            assert torch.equal(oa[k], ob[k]), k
    again = mbp.mbp_decode_multi([g.arg() for g in batch], 30)  # uses the tuned shape
    torch.cuda.synchronize()
    for oa, ob in zip(ref, again):
        assert torch.equal(oa["x_hat_bits"], ob["x_hat_bits"])


def test_edge_cases(mbp, batch):
    # max_iter = 0: the hard decision of the channel LLRs, success where it already satisfies every syndrome
    outs = mbp.mbp_decode_multi([g.arg() for g in batch], 0)
    torch.cuda.synchronize()
    for g, o in zip(batch, outs):
        if g.F:
            ref = single(mbp, g, 0)
            for k in ("x_hat_bits", "iters", "success"):
                assert torch.equal(o[k], ref[k])
            assert int(o["iters"].max()) == 0
    # noise-free frames stop before iteration 1 (the loop body never runs)
    g = batch[0]
    clean = dict(codes=g.codes, z_bits=g.z, y_bits=dev(i32(g.x)), qber=g.ed)
    o = mbp.mbp_decode_multi([clean], 20)[0]
    torch.cuda.synchronize()
    assert int(o["iters"].max()) == 0 and bool(o["success"].all())
    assert np.array_equal(o["x_hat_bits"].cpu().numpy().view(np.uint32), g.x)
    # only empty groups, and no groups
    assert mbp.mbp_decode_multi([batch[-1].arg()], 10)[0]["iters"].numel() == 0
    assert mbp.mbp_decode_multi([], 10) == []


def test_single_frame_groups(mbp, batch):
    """Groups of one frame each (32-lane tiles holding a single frame)."""
    args = []
    for g in batch[:4]:
        a = g.arg()
        a["y_bits"], a["qber"], a["F"] = g.yd[:1], g.ed[:1], 1
        a["z_bits"] = mbp.mbp_syndrome(g.codes, dev(i32(g.x[:1])))
        args.append(a)
    outs = mbp.mbp_decode_multi(args, 30)
    torch.cuda.synchronize()
    for g, o in zip(batch, outs):
        ref = mbp.mbp_decode_bsc(g.codes, g.yd[:1], g.ed[:1], mbp.mbp_syndrome(g.codes, dev(i32(g.x[:1]))), 30,
                                 schedule=mbp.SCHED_STREAMING)
        for k in ("x_hat_bits", "iters", "success"):
            assert torch.equal(o[k], ref[k])


def test_graph_schedule_single_code_entries(mbp, batch):
    """MBP_SCHED_GRAPH through the single-code entry points: device, host-memory and LLR inputs, and the
    message export, equal the streaming schedule."""
    g = batch[1]
    a = single(mbp, g, 25, early_exit=False)
    b = single(mbp, g, 25, early_exit=False, schedule=mbp.SCHED_GRAPH)
    for k in KEYS:
        assert torch.equal(a[k], b[k]), k
    for f in (0, g.F - 1):
        ca = mbp.mbp_export_c2v(g.codes, g.F, a["workspace"], f, schedule=mbp.SCHED_STREAMING)
        cb = mbp.mbp_export_c2v(g.codes, g.F, b["workspace"], f, schedule=mbp.SCHED_GRAPH)
        assert torch.equal(ca, cb)
    z_host = g.z.cpu().numpy().view(np.uint32)
    h = mbp.mbp_decode_bsc_host(g.codes, g.y, g.e, z_host, 25, schedule=mbp.SCHED_GRAPH)
    s = single(mbp, g, 25)
    assert np.array_equal(h["x_hat_bits"], s["x_hat_bits"].cpu().numpy().view(np.uint32))
    assert np.array_equal(h["iters"], s["iters"].cpu().numpy())
    llr = dev(orc.bsc_llr(g.y, g.n, g.e).astype(np.float32))
    c = mbp.mbp_decode_batch(g.codes, llr, g.z, 25, schedule=mbp.SCHED_GRAPH)
    torch.cuda.synchronize()
    assert torch.equal(c["x_hat_bits"], s["x_hat_bits"]) and torch.equal(c["success"], s["success"])


def test_multi_rejects_bad_arguments(mbp, batch):
    g = batch[0]
    with pytest.raises(mbp.MBPError) as ei:
        mbp.mbp_decode_multi([g.arg()], 10, msg_dtype=mbp.MSG_F64)
    assert ei.value.status == 5
    bad = g.arg()
    bad["F"] = -1
    with pytest.raises(mbp.MBPError) as ei:
        mbp.mbp_multi_workspace_size([bad])
    assert ei.value.status == 1
    host = g.arg()
    host["z_bits"] = g.z.cpu()
    with pytest.raises(mbp.MBPError) as ei:
        mbp.mbp_decode_multi([host], 10)
    assert ei.value.status == 1


def test_uneven_batch_recipe_small(mbp):
    """The uneven-batch recipe at reduced sizes (n in {1024, 2048, 4096}): all 24 classes in one call, every
    frame equal to its single-code decode."""
    specs = mi.uneven_batch(384, 5, sizes=(1024, 2048, 4096))
    groups, args = [], []
    for s in specs:
        H = mi.make_codes(s["n"], s["m"], s["dist"], s["u"], s["cfg_seed"])
        x, y, e = mi.bsc_frames(s["n"], s["frames"], s["qber"], seed=s["cfg_seed"])
        codes = mbp.mbp_create_codes(H)
        z = mbp.mbp_syndrome(codes, dev(i32(x)))
        groups.append((codes, dev(i32(y)), dev(e), z, x))
        args.append(dict(codes=codes, y_bits=groups[-1][1], qber=groups[-1][2], z_bits=z))
    outs = mbp.mbp_decode_multi(args, 40)
    torch.cuda.synchronize()
    ok = 0
    for (codes, y, e, z, x), o in zip(groups, outs):
        ref = mbp.mbp_decode_bsc(codes, y, e, z, 40, schedule=mbp.SCHED_STREAMING)
        for k in ("x_hat_bits", "iters", "success"):
            assert torch.equal(o[k], ref[k])
        s = o["success"].cpu().numpy().astype(bool)
        ok += int(s.sum())
        assert np.array_equal(o["x_hat_bits"].cpu().numpy().view(np.uint32)[s], x[s])
    assert ok >= 200


@pytest.mark.parametrize("msg", ["f32", "f16", "bf16"])
def test_set_tuning_selects_kernels_without_changing_results(mbp, batch, msg):
    """Persistent list kernels (one tile per warp) and grid kernels (for FP16/BF16 the tile-pair kernels, two
    frames per lane, mixed-precision adds) are separate implementations of the same per-frame arithmetic:
    equal outputs, bit for bit."""
    dt = {"f32": mbp.MSG_F32, "f16": mbp.MSG_F16, "bf16": mbp.MSG_BF16}[msg]
    ref = mbp.mbp_decode_multi([g.arg() for g in batch], 30, want_soft=True, msg_dtype=dt)
    torch.cuda.synchronize()
    for tu in (dict(grid_kernels=0, cn_warps=2, cn_waves=2, vn_warps=4, syn_warps=8),
               dict(grid_kernels=1, cn_warps=8, cn_waves=1, vn_warps=8, syn_warps=8)):
        mbp.mbp_multi_set_tuning([g.arg() for g in batch], tu, msg_dtype=dt)
        out = mbp.mbp_decode_multi([g.arg() for g in batch], 30, want_soft=True, msg_dtype=dt)
        torch.cuda.synchronize()
        for a, b in zip(ref, out):
            for k in ("x_hat_bits", "iters", "success", "soft"):
                assert torch.equal(a[k], b[k]), (tu, k)
    with pytest.raises(mbp.MBPError) as ei:
        mbp.mbp_multi_set_tuning([g.arg() for g in batch], dict(cn_warps=16))
    assert ei.value.status == 1


def test_graph_cache_keys_on_inputs_and_forgets_freed_codes(mbp, batch):
    """The cached graph of a batch bakes in every group's state: BSC then LLR inputs on one workspace must
    each get their own graph, and a code freed and replaced by another (whose handle may reuse the address)
    must not meet the old code's graph."""
    arg_b = [g.arg() for g in batch]
    arg_l = [g.arg(llr=True) for g in batch]
    ws = torch.empty(mbp.mbp_multi_workspace_size(arg_b, mbp.MSG_F32), dtype=torch.uint8, device="cuda")
    a = mbp.mbp_decode_multi(arg_b, 30, want_soft=True, workspace=ws)
    b = mbp.mbp_decode_multi(arg_l, 30, want_soft=True, workspace=ws)
    fresh = mbp.mbp_decode_multi(arg_l, 30, want_soft=True)
    torch.cuda.synchronize()
    for g, oa, ob, of in zip(batch, a, b, fresh):
        for k in ("x_hat_bits", "iters", "success", "soft"):
            assert torch.equal(ob[k], of[k]), (g.n, k)
        for k in ("x_hat_bits", "iters", "success"):
            assert torch.equal(oa[k], ob[k]), (g.n, k)
    n, F = 1024, 40
    ws1 = None
    for seed in range(4):
        H = mi.make_codes(n, 512, {3: 1.0}, 2, 100 + seed)
        codes = mbp.mbp_create_codes(H)
        x, y, e = mi.bsc_frames(n, F, 0.03, seed=200 + seed)
        z = mbp.mbp_syndrome(codes, dev(i32(x)))
        if ws1 is None:
            ws1 = torch.empty(mbp.mbp_decode_workspace_size(codes, F, mbp.MSG_F32, schedule=mbp.SCHED_GRAPH),
                              dtype=torch.uint8, device="cuda")
        og = mbp.mbp_decode_bsc(codes, dev(i32(y)), dev(e), z, 30, schedule=mbp.SCHED_GRAPH, workspace=ws1)
        os_ = mbp.mbp_decode_bsc(codes, dev(i32(y)), dev(e), z, 30, schedule=mbp.SCHED_STREAMING)
        for k in ("x_hat_bits", "iters", "success"):
            assert torch.equal(og[k], os_[k]), (seed, k)
        del codes, og, os_


@pytest.mark.slow
def test_multi_config4_sizes_match_oracle(mbp):
    """Codes of the 4096-frame uneven workload at full size (n = 2^14, 2^16, 2^18; rates 0.5 and 0.8; u = 2
    and 3), five frames of each with the workload's own QBERs, decoded in one grouped call (default launch
    shapes, after autotuning, and with the persistent list kernels): output bits, success flags and per-matrix
    syndrome flags equal the FP64
    oracle's on every frame the oracle decodes, and every reported success satisfies all syndromes."""
    specs = mi.uneven_batch(4096, 4)
    pick = [(65536, 0.5, 3), (65536, 0.8, 2), (262144, 0.5, 2), (262144, 0.8, 3), (16384, 0.8, 2)]
    groups = []
    for key in pick:
        sp = next(s for s in specs if (s["n"], s["rate"], s["u"]) == key)
        H = mi.make_codes(sp["n"], sp["m"], sp["dist"], sp["u"], sp["cfg_seed"])
        x, y, e = mi.bsc_frames(sp["n"], sp["frames"], sp["qber"], seed=sp["cfg_seed"])
        x, y, e = x[:5], y[:5], e[:5]
        codes = mbp.mbp_create_codes(H)
        groups.append(dict(H=H, x=x, y=y, e=e, n=sp["n"],
                           arg=dict(codes=codes, y_bits=dev(i32(y)), qber=dev(e),
                                    z_bits=mbp.mbp_syndrome(codes, dev(i32(x))))))
    args = [g["arg"] for g in groups]
    runs = [mbp.mbp_decode_multi(args, 60, want_synd=True)]
    runs.append(mbp.mbp_autotune_multi(args, 60)[0])
    # and the persistent list kernels over the frames of all groups, whichever shape the autotuner kept
    mbp.mbp_multi_set_tuning(args, dict(grid_kernels=0, cn_warps=8, cn_waves=1, vn_warps=8, syn_warps=8))
    runs.append(mbp.mbp_decode_multi(args, 60, want_synd=True))
    torch.cuda.synchronize()
    converged = 0
    for gi, g in enumerate(groups):
        ref = orc.decode(g["H"], orc.bsc_llr(g["y"], g["n"], g["e"]), orc.syndrome(g["H"], g["x"]), 60, threads=8,
                         want_synd=True)
        conv = ref["success"].astype(bool)
        converged += int(conv.sum())
        for o in runs:
            xh = o[gi]["x_hat_bits"].cpu().numpy().view(np.uint32)
            ok = o[gi]["success"].cpu().numpy().astype(bool)
            assert np.array_equal(ok[conv], ref["success"][conv]), pick[gi]
            assert np.array_equal(xh[conv], ref["x_hat_bits"][conv]), pick[gi]
            if "synd_ok" in o[gi]:
                assert np.array_equal(o[gi]["synd_ok"].cpu().numpy()[conv], ref["synd_ok"][conv])
            for l, zl in enumerate(orc.syndrome(g["H"], xh[ok])):
                assert np.array_equal(zl, orc.syndrome(g["H"], g["x"][ok])[l])
        it = runs[0][gi]["iters"].cpu().numpy()
        print(pick[gi], "oracle iterations", ref["iters"].tolist(), "GPU", it.tolist())
    assert converged >= 20


@pytest.mark.slow
def test_uneven_weakest_group_failures_are_the_oracles(mbp):
    """The n = 2^14, rate-0.8, u = 2 group of the 4096-frame uneven workload (its QBERs reach 4%, near this
    short code's decoding threshold): all of its frames through the grouped decode and the FP64 oracle. Bits
    and flags agree where the oracle converges, and every frame the GPU fails to decode fails in the oracle
    too (a frame that runs to max_iter is the code's failure, not the kernels')."""
    sp = next(s for s in mi.uneven_batch(4096, 4) if (s["n"], s["rate"], s["u"]) == (16384, 0.8, 2))
    H = mi.make_codes(sp["n"], sp["m"], sp["dist"], sp["u"], sp["cfg_seed"])
    x, y, e = mi.bsc_frames(sp["n"], sp["frames"], sp["qber"], seed=sp["cfg_seed"])
    codes = mbp.mbp_create_codes(H)
    arg = dict(codes=codes, y_bits=dev(i32(y)), qber=dev(e), z_bits=mbp.mbp_syndrome(codes, dev(i32(x))))
    o = mbp.mbp_decode_multi([arg], 60)[0]
    torch.cuda.synchronize()
    ref = orc.decode(H, orc.bsc_llr(y, sp["n"], e), orc.syndrome(H, x), 60, threads=8)
    conv = ref["success"].astype(bool)
    ok = o["success"].cpu().numpy().astype(bool)
    xh = o["x_hat_bits"].cpu().numpy().view(np.uint32)
    assert np.array_equal(ok[conv], ref["success"][conv]) and np.array_equal(xh[conv], ref["x_hat_bits"][conv])
    assert not np.any(~ok & conv), "a frame the oracle decodes failed on the GPU"
    print(f"{sp['frames']} frames: GPU failures {int((~ok).sum())}, oracle failures {int((~conv).sum())}, "
          f"QBER of the failures {e[~ok].round(4).tolist()}")
