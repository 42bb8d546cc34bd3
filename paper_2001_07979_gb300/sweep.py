"""Throughput, frame error rate and iterations across QBER, number of matrices and rate.

The analogue of the paper's Fig. 2 (throughput against the error rate e for
single-, two- and three-matrix decoding at rate 0.5) and Table 3 (efficiency
and throughput at rates 0.5..0.8), on synthetic PEG codes and BSC frames:

    python -m paper_2001_07979_gb300.sweep --out sweep.json
    python -m paper_2001_07979_gb300.sweep --table fig2 --n 16384 --frames 256

Each point decodes F frames with every input resident on the GPU and times
the decode with CUDA events (after a warm-up decode). It reports the
corrected-key throughput (n F / time, every frame counted), the frame error
rate (failures and undetected errors), the mean number of iterations, and two
efficiencies: f = m / (n h(e)) with m the rows of one matrix (the paper's
definition), and f_leak = u m / (n h(e)), counting every syndrome bit sent.
"""
from __future__ import annotations

import argparse
import json
import math
import sys

import numpy as np
import torch

import mbp_inputs as mi

from . import (MSG_F32, RULE_MIN_SUM, RULE_SUM_PRODUCT, UPDATE_FLOODING, UPDATE_MATRIX_SERIAL, mbp_create_codes,
               mbp_decode_bsc, mbp_decode_workspace_size, mbp_syndrome)

DIST = {2: 0.3, 3: 0.4, 8: 0.3}


def h2(e: float) -> float:
    return -e * math.log2(e) - (1 - e) * math.log2(1 - e)


def point(codes, n, m, u, e, frames, max_iter, seed, rule=RULE_SUM_PRODUCT, update=UPDATE_FLOODING, reps=3):
    x, y, q = mi.bsc_frames(n, frames, e, seed=seed)
    dev = torch.device("cuda")
    xd = torch.from_numpy(x.view(np.int32)).to(dev)
    yd = torch.from_numpy(y.view(np.int32)).to(dev)
    qd = torch.from_numpy(q).to(dev)
    zd = mbp_syndrome(codes, xd)
    ws = torch.empty(mbp_decode_workspace_size(codes, frames, MSG_F32), dtype=torch.uint8, device=dev)
    out = mbp_decode_bsc(codes, yd, qd, zd, max_iter, workspace=ws, rule=rule, update=update)  # warm-up
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        out = mbp_decode_bsc(codes, yd, qd, zd, max_iter, workspace=ws, rule=rule, update=update)
    b.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(b) / reps
    ok = out["success"].cpu().numpy().astype(bool)
    xh = out["x_hat_bits"].cpu().numpy().view(np.uint32)
    undetected = int(np.sum(ok & ~np.all(xh == x, axis=1)))
    it = out["iters"].cpu().numpy()
    return {"n": n, "m": m, "u": u, "rate": 1 - m / n, "qber": e, "frames": frames,
            "mbps": n * frames / (ms / 1e3) / 1e6, "ms": ms,
            "fer": (int((~ok).sum()) + undetected) / frames, "undetected": undetected,
            "mean_iterations": float(it.mean()), "f": m / (n * h2(e)), "f_leak": u * m / (n * h2(e))}


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--table", choices=["fig2", "table3", "all"], default="all")
    p.add_argument("--n", type=int, default=65536)
    p.add_argument("--frames", type=int, default=512)
    p.add_argument("--max-iter", type=int, default=60)
    p.add_argument("--variants", action="store_true", help="also the min-sum rule and the matrix-serial order")
    p.add_argument("--out", default=None, help="write the points as JSON here (default: stdout)")
    args = p.parse_args(argv)
    if not torch.cuda.is_available():
        print("a CUDA device is required", file=sys.stderr)
        return 1
    n, F = args.n, args.frames
    modes = [("sum-product", "flooding", RULE_SUM_PRODUCT, UPDATE_FLOODING)]
    if args.variants:
        modes += [("min-sum", "flooding", RULE_MIN_SUM, UPDATE_FLOODING),
                  ("sum-product", "matrix-serial", RULE_SUM_PRODUCT, UPDATE_MATRIX_SERIAL)]
    grid = []
    if args.table in ("fig2", "all"):  # rate 0.5 per matrix, u = 1, 2, 3, e = 3% .. 10%
        for u in (1, 2, 3):
            grid += [("fig2", 0.5, u, e) for e in (0.03, 0.04, 0.05, 0.06, 0.07, 0.08, 0.09, 0.10)]
    if args.table in ("table3", "all"):  # rates 0.5 .. 0.8, u = 2
        for r, es in ((0.5, (0.06, 0.08, 0.10)), (0.6, (0.04, 0.06, 0.08)), (0.7, (0.03, 0.04, 0.05)),
                      (0.8, (0.02, 0.03, 0.04))):
            grid += [("table3", r, 2, e) for e in es]
    cache, points = {}, []
    for k, (tab, r, u, e) in enumerate(grid):
        m = int(round(n * (1 - r)))
        key = (m, u)
        if key not in cache:
            cache[key] = mbp_create_codes(mi.make_codes(n, m, DIST, u, 70 + u))
        for name, upd, rule, update in modes:
            pt = point(cache[key], n, m, u, e, F, args.max_iter, seed=1000 + k, rule=rule, update=update)
            pt.update(table=tab, rule=name, update=upd)
            points.append(pt)
            print(f"{tab} R={r:.1f} u={u} e={e:.2f} {name}/{upd}: {pt['mbps']:9.1f} Mbps  FER {pt['fer']:.4f}  "
                  f"iters {pt['mean_iterations']:5.2f}  f {pt['f']:.3f}  f_leak {pt['f_leak']:.3f}",
                  file=sys.stderr, flush=True)
    text = json.dumps(points, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    else:
        print(text)
    return 0


if __name__ == "__main__":
    sys.exit(main())
