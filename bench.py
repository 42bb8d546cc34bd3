#!/usr/bin/env python
"""Throughput of batched multi-matrix BP reconciliation on GB300.

One step = one mbp_decode_bsc call with default options (the graph schedule:
the iteration loop inside one CUDA graph) that reconciles a batch of BSC frames:
n = 65536 bits per frame, u = 2 PEG matrices of rate 0.7 (m = 19661 each),
variable degrees {2: 30%, 3: 40%, 8: 30%}, QBER 2%, 1024 frames, at most 60
flooding iterations, FP32 messages. Frames are synthetic (seeded), the codes
are built by the seeded PEG generator. The timed steps cycle through 8 distinct
batches, so the frame error rate is counted over 8192 distinct frames, and
alternate over four CUDA streams (a workspace each), so that independent
batches are in flight together as in a server; the one-stream figure is
reported beside it.

The metric is corrected sifted key per second: sum over frames of n divided by
the decode time, all frames counted (the frame error rate is reported beside
it, with its one-sided 95% upper bound). ``value`` is timed with CUDA events on
the decode stream with every input already in HBM; ``e2e`` times the
host-memory entry point, which copies Bob's bits, the QBERs and Alice's
syndromes in and the corrected bits, iteration counts and success flags out.
The per-step decoder state (about 2.8 GB) is far larger than the 129 MB L2, so
no flush is needed between steps. Beside the headline: the same code at QBER
4% (more iterations, most of them with per-edge messages) and FP16/BF16
message storage at QBER 2%.

``--impl reference`` times the FP64 CPU oracle on the host cores instead (a
bounded sample of the same workload per step).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import mbp_inputs as mi  # noqa: E402

N, M, DIST, U, SEED = 65536, 19661, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 1
QBER, MAX_ITER, FRAMES = 0.02, 60, 1024
WORKLOAD = "MBP decode, n=65536, R=0.7 (m=19661 x u=2 PEG), dv {2:.3,3:.4,8:.3}, BSC QBER 2%, 1024 frames, max 60 it"
METRIC = "corrected-key Mbps per GB300 at FER<=1e-3 (and % of HBM roofline) vs plain FP32 MBP"
L_MAX = 20.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=300)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    p.add_argument("--frames", type=int, default=FRAMES)
    p.add_argument("--batches", type=int, default=8, help="distinct frame batches cycled through the timed steps")
    p.add_argument("--streams", type=int, default=4, help="streams the steps' decodes alternate over")
    p.add_argument("--no-extras", action="store_true", help="skip the QBER-4%% and FP16/BF16 side measurements")
    p.add_argument("--cpu-sample", type=int, default=256, help="frames in the oracle's timed sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--accumulate", default="auto", choices=["auto", "float", "fixed"],
                   help="eq. (2) accumulation: fixed-point single pass or float second pass")
    p.add_argument("--schedule", default="auto", choices=["auto", "streaming", "resident", "graph"],
                   help="auto (the library default: graph where it applies), kernels per iteration, one "
                        "cooperative launch keeping tile groups in L2, or the iteration loop in a CUDA graph")
    p.add_argument("--rule", default="sum-product", choices=["sum-product", "min-sum"],
                   help="check-node rule: eq. (6) or the min-sum approximation (variant)")
    p.add_argument("--update", default="flooding", choices=["flooding", "matrix-serial"],
                   help="update order: flooding over all matrices, or matrix by matrix (variant)")
    p.add_argument("--workload", default="n65536", choices=["n65536", "uneven"],
                   help="n65536: the rate-0.7 n=65536 batch; uneven: 4096 frames of 24 codes "
                        "(n 2^14..2^18, R 0.5..0.8, u 2..3, QBER U[1%%, 4%%]) in one grouped call")
    p.add_argument("--msg-dtype", default="f32", choices=["f32", "f16", "bf16"],
                   help="message storage: FP32, or FP16/BF16 with FP32 arithmetic")
    return p.parse_args()


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def algorithmic_bytes(iters, n, e_tot, msg_bytes=4, rows=False):
    """Floor bytes of the frame-iterations run, for the per-edge check kernel and for the whole path.

    A per-edge check iteration writes each message once and reads the posterior
    once (s E + 4 n), and after a frame's first iteration also reads the previous
    messages (s E). With the row form (BSC inputs) iterations 1 and 2 run as
    row-form check work of their own (their bytes are not the per-edge kernel's),
    and the per-edge kernel runs from iteration 3 on: 2 s E + 4 n each. The
    whole path adds the variable-node pass, which reads the messages and writes
    the posterior: per frame, 4 n in iteration 1 (row form) or 2 s E + 8 n
    (per edge), 2 s E + 8 n in iteration 2 (row form) and 3 s E + 8 n later.
    """
    it = np.asarray(iters, dtype=np.int64)
    sE = msg_bytes * e_tot
    if rows:
        check = int(np.sum(np.maximum(it - 2, 0) * (2 * sE + 4 * n)))
        path = int(np.sum((it >= 1) * 4 * n + (it >= 2) * (2 * sE + 8 * n) + np.maximum(it - 2, 0) * (3 * sE + 8 * n)))
    else:
        later = np.maximum(it - 1, 0)
        check = int(np.sum(it * (sE + 4 * n) + later * sE))
        path = int(np.sum((it >= 1) * (2 * sE + 8 * n) + later * (3 * sE + 8 * n)))
    return check, path


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index, self.rows, self.proc = index, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(sm)}


def rank_inputs(frames, rank, batch=0, qber=QBER):
    """Weak scaling: every rank reconciles its own `frames` frames per batch (frame stream = 1024 rank + batch)."""
    return mi.bsc_frames(N, frames, qber, seed=SEED, stream=1024 * rank + batch)


def fer_upper95(k, n):
    """One-sided 95% Clopper-Pearson upper bound of a frame error rate with k errors in n frames."""
    if n == 0 or k >= n:
        return 1.0
    if k == 0:
        return 1.0 - 0.05 ** (1.0 / n)
    try:
        from scipy.stats import beta
        return float(beta.ppf(0.95, k + 1, n - k))
    except ImportError:
        return None


def reduce_over_ranks(dist, device, ms, ms_e2e, fails, undetected):
    """Slowest rank's times (MAX) and the job's failure counts (SUM); identity for one process."""
    if dist is None or not dist.is_initialized() or dist.get_world_size() == 1:
        return ms, ms_e2e, fails, undetected
    import torch
    t = torch.tensor([ms, ms_e2e], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    c = torch.tensor([fails, undetected], dtype=torch.int64, device=device)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t[0]), float(t[1]), int(c[0]), int(c[1])


def job_mbps(frames_per_rank, world, ms):
    """Whole-job throughput: bits of every rank's frames over the slowest rank's time."""
    return frames_per_rank * N * world / (ms / 1e3) / 1e6


def cpu_count():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_time(H, x, y, e, frames, threads):
    import oracle as orc
    z = orc.syndrome(H, x[:frames])
    LP = orc.bsc_llr(y[:frames], N, e[:frames])
    t0 = time.perf_counter()
    out = orc.decode(H, LP, z, MAX_ITER, l_max=L_MAX, threads=threads)
    dt = time.perf_counter() - t0
    return dt, out


NOMINAL_HBM_GBS = 8000.0  # GB300 HBM3e, nominal (the roofline's "frac" uses the measured copy bandwidth)

KERNEL_SOURCES = ("mbp_internal.h", "mbp_device.cuh", "mbp_stream.cuh", "mbp_pair.cuh", "mbp_stream_f32.cu",
                  "mbp_resident.cuh")


def source_code_only(text):
    """C++ source without its comments and blank lines, each remaining line stripped of trailing blanks (the
    sources have no comment markers inside string or character literals)."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*", "", line).rstrip() for line in text.splitlines())
    return "\n".join(line for line in lines if line.strip())


def kernel_source_digest():
    """First 16 hex digits of the SHA-256 of the code (comments left out) of the sources that define the decoder
    kernels: the key a committed ncu summary records, so that its DRAM figures are used only for the kernels
    they were measured on."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(source_code_only(open(os.path.join(ROOT, "paper_2001_07979_gb300", "csrc", f)).read()).encode())
    return h.hexdigest()[:16]


def kernel_traffic(iters, launches, summary, msg_dtype, rows=False):
    """Mean DRAM bytes per launch of the dominant kernel, from the committed full-size ncu capture (bytes per
    frame in a frame's first iteration and in a later one), if that capture was taken on the current source
    with the same message type."""
    path = os.path.join(ROOT, "profiles", summary)
    try:
        text = open(path).read()
        kv = dict(line.split("=", 1) for line in text.splitlines() if "=" in line and not line.startswith("#"))
        kv = {k.strip(): v.strip() for k, v in kv.items()}
        if kv.get("kernel_source_sha256_16") != kernel_source_digest() or not launches:
            return None
        if kv.get("msg_dtype", "f32") != msg_dtype:
            return None
        it = np.asarray(iters, dtype=np.int64)
        if rows:  # the per-edge kernel runs the iterations after the second
            total = int(np.sum(np.maximum(it - 2, 0))) * float(kv["dram_bytes_per_frame_later_iteration"])
        else:
            first, later = int(np.sum(it >= 1)), int(np.sum(np.maximum(it - 1, 0)))
            total = first * float(kv["dram_bytes_per_frame_first_iteration"]) + \
                later * float(kv["dram_bytes_per_frame_later_iteration"])
        return total / launches
    except Exception:
        return None


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    H = mi.make_codes(N, M, DIST, U, SEED)
    sample = 32
    x, y, e = mi.bsc_frames(N, sample, QBER, seed=SEED)
    threads = cpu_count()
    for _ in range(args.warmup):
        oracle_time(H, x, y, e, sample, threads)
    times, fails = [], 0
    for _ in range(args.steps):
        dt, out = oracle_time(H, x, y, e, sample, threads)
        times.append(dt)
        fails = int((out["success"] == 0).sum())
    ms = 1e3 * sum(times) / len(times)
    value = sample * N / (ms / 1e3) / 1e6
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "Mbps", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD, "frames_per_step": sample, "fer": fails / sample},
        "cpu_baseline": {"value": value, "unit": "Mbps", "cores": threads, "kind": "oracle",
                         "sample": f"{sample} frames of the workload per step, FP64 oracle, {threads} threads"},
        "e2e": {"value": value, "unit": "Mbps", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    import torch
    import torch.distributed as dist

    import paper_2001_07979_gb300 as mbp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    if rank == 0:
        mbp.build()
    if world > 1:
        dist.barrier()
    mbp._load()

    F, B = args.frames, max(1, args.batches)
    H = mi.make_codes(N, M, DIST, U, SEED)
    codes = mbp.mbp_create_codes(H)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream()

    def device_batch(x, y, e):
        yd = torch.from_numpy(y.view(np.int32)).to(dev)
        ed = torch.from_numpy(e).to(dev)
        zd = mbp.mbp_syndrome(codes, torch.from_numpy(x.view(np.int32)).to(dev))  # Alice's side, untimed
        return yd, ed, zd

    host = [rank_inputs(F, rank, b) for b in range(B)]  # (x, y, e) per batch
    batches = [device_batch(*h) for h in host]
    msg = {"f32": mbp.MSG_F32, "f16": mbp.MSG_F16, "bf16": mbp.MSG_BF16}[args.msg_dtype]
    msg_bytes = {"f32": 4, "f16": 2, "bf16": 2}[args.msg_dtype]
    acc = {"auto": mbp.ACC_AUTO, "float": mbp.ACC_FLOAT, "fixed": mbp.ACC_FIXED}[args.accumulate]
    sched = {"auto": mbp.SCHED_AUTO, "streaming": mbp.SCHED_STREAMING, "resident": mbp.SCHED_RESIDENT,
             "graph": mbp.SCHED_GRAPH}[args.schedule]
    variant = dict(rule=mbp.RULE_MIN_SUM if args.rule == "min-sum" else mbp.RULE_SUM_PRODUCT,
                   update=mbp.UPDATE_MATRIX_SERIAL if args.update == "matrix-serial" else mbp.UPDATE_FLOODING)

    # Decodes of independent batches are issued on `lanes` streams in turn, each with a workspace of its own, so
    # that one batch's small kernels and kernel tails overlap another batch's work (a server keeps several
    # batches in flight the same way); the per-kernel accounting pass uses one stream.
    lanes = [torch.cuda.Stream(device=dev) for _ in range(max(1, args.streams))]

    def make_step(msg_code, bats, schedule=sched, n_lanes=len(lanes)):
        ws = [torch.empty(mbp.mbp_decode_workspace_size(codes, F, msg_code, schedule=schedule), dtype=torch.uint8,
                          device=dev) for _ in range(n_lanes)]

        def step(s):
            yd, ed, zd = bats[s % len(bats)]
            k = s % n_lanes
            with torch.cuda.stream(lanes[k]):  # the outputs are allocated on, and written by, this stream
                return mbp.mbp_decode_bsc(codes, yd, ed, zd, MAX_ITER, msg_dtype=msg_code, l_max=L_MAX,
                                          workspace=ws[k], accumulate=acc, schedule=schedule, **variant)
        return step

    def timed(step, steps, warmup, outs=None):
        """Mean device time per step of `steps` steps after `warmup` untimed ones: CUDA events on the main
        stream, which the decode streams wait for at the start and which waits for them at the end; outs[b]
        keeps the last output of batch b."""
        for s in range(max(warmup, 3)):
            r = step(s)
            if outs is not None:
                outs[s % len(outs)] = r
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for ln in lanes:
            ln.wait_event(a)
        for s in range(steps):
            r = step(s)
            if outs is not None:
                outs[s % len(outs)] = r
        for ln in lanes:
            done = torch.cuda.Event()
            done.record(ln)
            stream.wait_event(done)
        b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return a.elapsed_time(b) / steps

    step = make_step(msg, batches)
    outs = [None] * B
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms = timed(step, args.steps, args.warmup, outs)
    clk = clocks.stop()
    for b in range(B):  # batches the timed steps did not reach (steps < batches)
        if outs[b] is None:
            outs[b] = step(b)
    step1 = make_step(msg, batches, n_lanes=1)
    ms_one = timed(step1, args.steps, args.warmup) if len(lanes) > 1 else ms
    # per-kernel device times: the same steps again, on one stream, with a CUDA event pair around every kernel
    # launch (the graph schedule's kernels are then launched from the host, one per event pair)
    mbp.mbp_profile_enable(True)
    for s in range(args.steps):
        step1(s)
    torch.cuda.synchronize()
    prof = mbp.mbp_profile_get()
    mbp.mbp_profile_enable(False)

    iters_b = [o["iters"].cpu().numpy() for o in outs]
    fails = undetected = 0
    for o, (x, _, _) in zip(outs, host):
        ok = o["success"].cpu().numpy().astype(bool)
        xh = o["x_hat_bits"].cpu().numpy().view(np.uint32)
        fails += int((~ok).sum())
        undetected += int(np.sum(ok & ~np.all(xh == x, axis=1)))
    xh0 = outs[0]["x_hat_bits"].cpu().numpy().view(np.uint32)

    # end to end through the host-memory entry point: every step copies its batch's Bob bits, QBERs and Alice
    # syndromes from pinned host memory and its corrected bits, iteration counts and success flags back, inside
    # the timed region. The asynchronous form of the entry point lets consecutive steps overlap on two streams
    # (each with a workspace and output buffers of its own): the copies of one batch run beside the decode of
    # the other, and the host prepares the next call while the GPU works.
    Wn = (N + 31) // 32
    host_in = [(torch.from_numpy(y.view(np.int32)).pin_memory(), torch.from_numpy(e).pin_memory(),
                zd.cpu().pin_memory()) for (_, y, e), (_, _, zd) in zip(host, batches)]
    outh = [dict(x_hat_bits=torch.empty((F, Wn), dtype=torch.int32).pin_memory(),
                 iters=torch.empty(F, dtype=torch.int32).pin_memory(),
                 success=torch.empty(F, dtype=torch.uint8).pin_memory()) for _ in lanes]
    wsh = [torch.empty(mbp.mbp_decode_workspace_size(codes, F, msg, host_io=True, schedule=sched), dtype=torch.uint8,
                       device=dev) for _ in lanes]

    def step_e2e(s):
        k = s % len(lanes)
        yh, eh, zh = host_in[s % B]
        mbp.mbp_decode_bsc_host(codes, yh, eh, zh, MAX_ITER, msg_dtype=msg, l_max=L_MAX, workspace=wsh[k],
                                out=outh[k], stream=lanes[k], accumulate=acc, schedule=sched, sync=False, **variant)

    def timed_e2e(steps, warmup):
        for s in range(warmup):
            step_e2e(s)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for ln in lanes:
            ln.wait_event(a)
        for s in range(steps):
            step_e2e(s)
        for ln in lanes:
            done = torch.cuda.Event()
            done.record(ln)
            stream.wait_event(done)
        b.record(stream)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        return a.elapsed_time(b) / steps

    ms_e2e = timed_e2e(args.steps, 3)
    last = args.steps - 1  # the outputs left in the host buffers are those of the last step
    assert np.array_equal(outh[last % len(lanes)]["x_hat_bits"].numpy().view(np.uint32),
                          outs[last % B]["x_hat_bits"].cpu().numpy().view(np.uint32))
    yh, eh, zh = host_in[0]
    h2d = yh.numel() * 4 + eh.numel() * 8 + zh.numel() * 4
    d2h = outh[0]["x_hat_bits"].numel() * 4 + F * 4 + F

    ms, ms_e2e, fails, undetected = reduce_over_ranks(dist if world > 1 else None, dev, ms, ms_e2e, fails,
                                                      undetected)
    value = job_mbps(F, world, ms)
    value_e2e = job_mbps(F, world, ms_e2e)

    # roofline of the dominant kernel: algorithmic bytes of the frame-iterations it ran / its event time; the
    # timed steps cycle through the batches, so the bytes of a step are averaged over the steps run
    e_tot = codes.edges
    rows = prof.get("check_rows", (0, 0.0))[0] > 0  # iterations 1 and 2 ran in row form
    per_batch = [algorithmic_bytes(it, N, e_tot, msg_bytes, rows) for it in iters_b]
    b_check = sum(per_batch[s % B][0] for s in range(args.steps)) / args.steps
    b_path = sum(per_batch[s % B][1] for s in range(args.steps)) / args.steps
    iters_steps = np.concatenate([iters_b[s % B] for s in range(args.steps)])
    peak, peak_src = load_peaks()
    # the floor of one frame-iteration, B_it = 2 s E + 12 n (every message read and written once, the posterior
    # read, written and gathered once), times the frame-iterations the timed steps ran
    b_it = (2 * msg_bytes * e_tot + 12 * N) * float(iters_steps.sum()) / args.steps
    dominant = "persistent" if prof.get("persistent", (0, 0.0))[0] > 0 else "check"
    launches = int(sum(v[0] for v in prof.values()))
    path_gbs = b_path / (ms / 1e3) / 1e9
    if dominant == "persistent":
        # one cooperative launch runs every step of every iteration: its algorithmic bytes are the path's
        n_dom, ms_dom = prof["persistent"]
        kernel_name = "resident_kernel (all steps of eq. 6, eq. 2 and the stopping rule, tile groups in L2)"
        b_dom, rule = b_path, "2*s*E+12n per frame-iteration (s*E less in a frame's first)"
        traffic = kernel_traffic(iters_steps, n_dom if n_dom else 0, "resident_kernel_n65536.txt", args.msg_dtype)
    else:
        n_dom, ms_dom = prof["check"]
        kernel_name = ("check-node update of eq. 6 on per-edge messages (cn_pair_kernel: one warp per tile pair "
                       "and row for rows of up to 24 edges, else cn_kernel)")
        rule = ("per frame: 2*s*E+4n per iteration after the second (iterations 1 and 2 run in row form)" if rows
                else "per frame: s*E+4n per iteration, plus s*E per iteration after the first")
        b_dom = b_check
        traffic = kernel_traffic(iters_steps, n_dom if n_dom else 0, "check_node_kernel_n65536.txt",
                                 args.msg_dtype, rows)
    achieved = b_dom * args.steps / (ms_dom / 1e3) / 1e9 if ms_dom > 0 else None

    # side measurements on the same code (not the headline): QBER 4%, and FP16/BF16 message storage at 2%
    extras = {}
    if rank == 0 and world == 1 and not args.no_extras and args.msg_dtype == "f32" and args.rule == "sum-product" \
            and args.update == "flooding":
        side_steps = max(3, min(args.steps, 100))
        h4 = [rank_inputs(F, rank, 100 + b, qber=0.04) for b in range(2)]
        b4 = [device_batch(*h) for h in h4]
        outs4 = [None, None]
        ms4 = timed(make_step(msg, b4), side_steps, 3, outs4)
        it4 = [o["iters"].cpu().numpy() for o in outs4]
        f4 = sum(int((o["success"] == 0).sum().item()) for o in outs4)
        bp4 = sum(algorithmic_bytes(it, N, e_tot, msg_bytes, rows)[1] for it in it4) / 2
        extras["qber_4pct"] = {"value": F * N / (ms4 / 1e3) / 1e6, "unit": "Mbps", "ms_per_step": ms4,
                               "mean_iterations": float(np.mean(np.concatenate(it4))), "frames": 2 * F,
                               "fer": f4 / (2 * F), "steps": side_steps,
                               "path_gbs": bp4 / (ms4 / 1e3) / 1e9, "path_frac": bp4 / (ms4 / 1e3) / 1e9 / peak}
        for name, code in (("f16", mbp.MSG_F16), ("bf16", mbp.MSG_BF16)):
            o16 = [None] * B
            ms16 = timed(make_step(code, batches), side_steps, 3, o16)
            for b in range(B):
                if o16[b] is None:
                    o16[b] = make_step(code, batches)(b)
            err16 = 0
            for o, (x, _, _) in zip(o16, host):
                ok = o["success"].cpu().numpy().astype(bool)
                xh = o["x_hat_bits"].cpu().numpy().view(np.uint32)
                err16 += int((~ok | ~np.all(xh == x, axis=1)).sum())
            extras[name] = {"value": F * N / (ms16 / 1e3) / 1e6, "unit": "Mbps", "ms_per_step": ms16,
                            "vs_f32": ms / ms16, "frames": B * F, "fer": err16 / (B * F),
                            "fer_upper95": fer_upper95(err16, B * F), "steps": side_steps}

    result = None
    if rank == 0:
        n_frames = B * F * world
        result = {
            "metric": METRIC, "value": value, "unit": "Mbps", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": args.msg_dtype if args.msg_dtype == "f32" else f"{args.msg_dtype}+f32",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "frames_per_gpu": F, "n": N, "m_per_matrix": M, "u": U,
                       "edges": e_tot, "qber": QBER, "max_iter": MAX_ITER, "l_max": L_MAX,
                       "distinct_batches": B, "distinct_frames": n_frames, "streams": len(lanes),
                       "mean_iterations": float(iters_steps.mean()), "max_iterations": int(iters_steps.max()),
                       "fer": (fails + undetected) / n_frames, "failures": fails, "undetected_errors": undetected,
                       "fer_upper95": fer_upper95(fails + undetected, n_frames),
                       "l2": "per-step decoder state ~2.8 GB > 129 MB L2 (no flush)",
                       "accumulate": args.accumulate, "schedule": args.schedule, "rule": args.rule,
                       "update": args.update,
                       "parallelism": f"replicas x{world} (frames sharded, no collective on the path)"},
            "roofline": {"bound": "hbm", "kernel": kernel_name,
                         "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                         "peak_source": f"{peak_src} HBM copy bandwidth",
                         "nominal_peak": NOMINAL_HBM_GBS,
                         "frac_nominal": (achieved / NOMINAL_HBM_GBS) if achieved else None,
                         "algorithmic_bytes_per_step": b_dom, "bytes_rule": rule,
                         "launches": n_dom,
                         "mean_launch_ms": ms_dom / n_dom if n_dom else None,
                         "dominant_family": dominant,
                         "path_gbs": path_gbs, "path_frac": path_gbs / peak,
                         "path_bytes_rule": ("per frame: 4n (iteration 1, row form), 2*s*E+8n (iteration 2), "
                                             "3*s*E+8n later" if rows else
                                             "per frame: 2*s*E+8n (iteration 1), 3*s*E+8n later"),
                         "row_form": rows,
                         "b_it_gbs": b_it / (ms / 1e3) / 1e9, "b_it_frac": b_it / (ms / 1e3) / 1e9 / peak,
                         "b_it_rule": "B_it = 2*s*E + 12n per executed frame-iteration (the method's floor), "
                                      "times the frame-iterations of a step, over the step time"},
            "kernel_ms": {k: v[1] / args.steps for k, v in prof.items()},
            "kernel_ms_source": "a second pass of the same steps with a CUDA event pair around every kernel launch",
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": {"value": value_e2e, "unit": "Mbps", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "ms_per_step": ms_e2e,
                    "how": f"mbp_decode_bsc_host_async from pinned host buffers, steps alternating over "
                           f"{len(lanes)} streams, each step's copies in and out inside the timed region"},
            "one_stream": {"value": job_mbps(F, world, ms_one), "unit": "Mbps", "ms_per_step": ms_one},
            "side": extras,
            "context": "paper: 85.67 Mbps average / 102.084 Mbps maximum on TitanV (other codes, other hardware)",
        }
        if world == 1 and not args.no_cpu_baseline:
            threads = cpu_count()
            sample = min(args.cpu_sample, F)
            x, y, e = host[0]
            dt, ref = oracle_time(H, x, y, e, sample, threads)
            agree = bool(np.array_equal(ref["x_hat_bits"], xh0[:sample]))
            result["cpu_baseline"] = {"value": sample * N / dt / 1e6, "unit": "Mbps", "cores": threads,
                                      "kind": "oracle",
                                      "sample": f"first {sample} of the {F} frames, FP64 oracle, {dt:.1f} s",
                                      "outputs_agree": agree}
        print(json.dumps(result), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()
    return 0


UNEVEN_FRAMES, UNEVEN_SEED = 4096, 4
UNEVEN_WORKLOAD = ("MBP grouped decode of uneven frames: 4096 frames, each of a code drawn from n in {2^14, 2^16, "
                   "2^18} x R in {0.5, 0.6, 0.7, 0.8} x u in {2, 3} (24 PEG codes, dv {2:.3,3:.4,8:.3}), QBER "
                   "uniform in [1%, 4%] per frame, max 60 it")


def run_uneven(args):
    """One step = one mbp_decode_multi call over the whole uneven batch (launch shapes from the autotuner,
    untimed); beside it, the same frames decoded by one single-code streaming call per code."""
    import torch

    import paper_2001_07979_gb300 as mbp

    torch.cuda.set_device(0)
    mbp.build()
    mbp._load()
    dev = torch.device("cuda", 0)
    frames = UNEVEN_FRAMES if args.frames == FRAMES else args.frames
    specs = mi.uneven_batch(frames, UNEVEN_SEED)
    msg = {"f32": mbp.MSG_F32, "f16": mbp.MSG_F16, "bf16": mbp.MSG_BF16}[args.msg_dtype]
    groups, xs, bits = [], [], 0
    for sp in specs:
        H = mi.make_codes(sp["n"], sp["m"], sp["dist"], sp["u"], sp["cfg_seed"])
        x, y, e = mi.bsc_frames(sp["n"], sp["frames"], sp["qber"], seed=sp["cfg_seed"])
        codes = mbp.mbp_create_codes(H)
        xd = torch.from_numpy(x.view(np.int32)).to(dev)
        groups.append(dict(codes=codes, y_bits=torch.from_numpy(y.view(np.int32)).to(dev),
                           qber=torch.from_numpy(e).to(dev), z_bits=mbp.mbp_syndrome(codes, xd)))
        xs.append(x)
        bits += sp["n"] * sp["frames"]
    stream = torch.cuda.current_stream()
    # as in the headline bench, consecutive steps alternate over streams with a workspace each, so that one
    # batch's tail of iterations (a few groups still decoding) overlaps the next batch's work
    lanes = [torch.cuda.Stream(device=dev) for _ in range(max(1, min(args.streams, 2)))]
    wss_m = [torch.empty(mbp.mbp_multi_workspace_size(groups, msg), dtype=torch.uint8, device=dev) for _ in lanes]
    _, tuning = mbp.mbp_autotune_multi(groups, MAX_ITER, msg_dtype=msg, l_max=L_MAX, workspace=wss_m[0])
    count = [0]

    def step(k=None):
        k = count[0] % len(lanes) if k is None else k
        count[0] += 1
        with torch.cuda.stream(lanes[k]):
            return mbp.mbp_decode_multi(groups, MAX_ITER, msg_dtype=msg, l_max=L_MAX, workspace=wss_m[k])

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            r = fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for ln in lanes:
            ln.wait_event(a)
        for _ in range(args.steps):
            r = fn()
        for ln in lanes:
            done = torch.cuda.Event()
            done.record(ln)
            stream.wait_event(done)
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / args.steps, r

    clocks = ClockSampler(0)
    clocks.start()
    time.sleep(0.3)
    ms, outs = timed(step)
    clk = clocks.stop()
    ms_one, _ = timed(lambda: step(0)) if len(lanes) > 1 else (ms, None)
    # the same frames, one single-code call (streaming schedule) per code
    wss = [torch.empty(mbp.mbp_decode_workspace_size(g["codes"], g["y_bits"].shape[0], msg), dtype=torch.uint8,
                       device=dev) for g in groups]

    def step_single():
        return [mbp.mbp_decode_bsc(g["codes"], g["y_bits"], g["qber"], g["z_bits"], MAX_ITER, msg_dtype=msg,
                                   l_max=L_MAX, workspace=w, schedule=mbp.SCHED_STREAMING)
                for g, w in zip(groups, wss)]

    ms_single, outs_single = timed(step_single)
    same = all(torch.equal(a[k], b[k]) for a, b in zip(outs, outs_single) for k in ("x_hat_bits", "iters", "success"))
    # per-family device times of one grouped decode (kernel accounting drives the same kernels from the host)
    mbp.mbp_profile_enable(True)
    step(0)
    torch.cuda.synchronize()
    prof = mbp.mbp_profile_get()
    mbp.mbp_profile_enable(False)
    fails = undetected = 0
    it_sum = 0
    failing, per_group = [], []
    for sp, o, x, g in zip(specs, outs, xs, groups):
        ok = o["success"].cpu().numpy().astype(bool)
        xh = o["x_hat_bits"].cpu().numpy().view(np.uint32)
        it = o["iters"].cpu().numpy()
        fails += int((~ok).sum())
        undetected += int(np.sum(ok & ~np.all(xh == x, axis=1)))
        it_sum += int(it.sum())
        h = lambda q: -q * np.log2(q) - (1 - q) * np.log2(1 - q)
        for f in np.flatnonzero(~ok):
            q = float(sp["qber"][f])
            failing.append({"n": sp["n"], "rate": sp["rate"], "u": sp["u"], "qber": q, "iters": int(it[f]),
                            "f": sp["m"] / (sp["n"] * h(q)), "f_leak": sp["u"] * sp["m"] / (sp["n"] * h(q))})
        if sp["frames"]:
            # work in edge x frame x iteration units: per frame as run, and as a tile pair (64 frames) costs,
            # since the kernels move a pair's messages until its last frame has stopped; the decoder places a
            # group's frames in its tiles in order of QBER (ties by index), so the pairs are formed that way
            e_tot = g["codes"].edges
            its = it[np.argsort(sp["qber"], kind="stable")]
            pair_max = [int(its[q:q + 64].max()) for q in range(0, its.size, 64)]
            per_group.append({"n": sp["n"], "rate": sp["rate"], "u": sp["u"], "frames": sp["frames"],
                              "mean_iterations": float(it.mean()), "max_iterations": int(it.max()),
                              "edge_frame_iterations": int(e_tot) * int(it.sum()),
                              "edge_frame_iterations_per_pair": int(e_tot) * 64 * int(sum(pair_max))})
    line = {
        "metric": METRIC, "value": bits / (ms / 1e3) / 1e6, "unit": "Mbps", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": args.msg_dtype if args.msg_dtype == "f32" else f"{args.msg_dtype}+f32", "data": "synthetic",
        "config": {"workload": UNEVEN_WORKLOAD, "frames": frames, "codes": len(groups), "bits_per_step": bits,
                   "fer": fails / frames, "undetected_errors": undetected, "mean_iterations": it_sum / frames,
                   "tuning": tuning, "l2": "per-step decoder state of several GB > 129 MB L2 (no flush)"},
        "single_code_calls": {"ms_per_step": ms_single, "value": bits / (ms_single / 1e3) / 1e6,
                              "outputs_identical": same},
        "streams": len(lanes),
        "one_stream": {"value": bits / (ms_one / 1e3) / 1e6, "unit": "Mbps", "ms_per_step": ms_one},
        "failing_frames": failing, "groups": per_group,
        "work_rate": {"edge_frame_iterations_per_s": sum(g["edge_frame_iterations"] for g in per_group) / (ms / 1e3),
                      "pair_granularity_per_s": sum(g["edge_frame_iterations_per_pair"] for g in per_group)
                      / (ms / 1e3)},
        "kernel_ms": {k: v[1] for k, v in prof.items()},
        "kernel_ms_source": "one grouped decode with a CUDA event pair around every kernel launch (host-driven loop)",
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "uneven":
        return run_uneven(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
