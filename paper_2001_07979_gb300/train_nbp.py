"""Train the unrolled normalised BP and compare it with the plain decoder.

    python -m paper_2001_07979_gb300.train_nbp --steps 200 --out nbp.json
    python -m paper_2001_07979_gb300.train_nbp --time        # forward / adjoint pass times only

The learned form (mbp_nbp_forward / mbp_nbp_backward behind NormalizedBP)
rescales every check-to-variable message of matrix l at iteration t by a
learnable scale alpha[t][l] and offset beta[t][l]. Training uses fresh BSC
frames every step (seeded), the loss is the mean over the T iterations of the
binary cross-entropy of sigmoid(-L^t) against Alice's bits, optimised with
Adam. Evaluation decodes other frames with the learned parameters and with
alpha = 1, beta = 0 (the plain decoder) and reports, per iteration t, the
fraction of frames whose hard decision satisfies every syndrome, and the mean
iteration at which a frame first does (frames that never do count as T).
"""
from __future__ import annotations

import argparse
import json
import sys
import time

import numpy as np
import torch

import mbp_inputs as mi

from . import (NBPDecoder, mbp_bsc_llr, mbp_create_codes, mbp_nbp_backward, mbp_nbp_forward,
               mbp_nbp_workspace_size, mbp_syndrome)


def frames(codes, n, F, qber, seed):
    x, y, e = mi.bsc_frames(n, F, qber, seed=seed)
    dev = torch.device("cuda")
    llr = mbp_bsc_llr(torch.from_numpy(y.view(np.int32)).to(dev), torch.from_numpy(e).to(dev), n, torch.float32)
    z = mbp_syndrome(codes, torch.from_numpy(x.view(np.int32)).to(dev))
    xb = torch.from_numpy(np.stack([mi.unpack_bits(x[f], n) for f in range(F)]).astype(np.float32)).to(dev)
    return llr, z, xb


def pack(bits: torch.Tensor) -> torch.Tensor:
    """[F, n] 0/1 -> [F, ceil(n/32)] int32 words, bit i of a frame at word i >> 5, position i & 31."""
    F, n = bits.shape
    w = (n + 31) // 32
    b = torch.zeros((F, w * 32), dtype=torch.int64, device=bits.device)
    b[:, :n] = bits.to(torch.int64)
    words = (b.view(F, w, 32) << torch.arange(32, device=bits.device)).sum(dim=2)  # in [0, 2^32)
    return torch.where(words >= 2 ** 31, words - 2 ** 32, words).to(torch.int32)


def main(argv=None):
    p = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--rate", type=float, default=0.6)
    p.add_argument("--u", type=int, default=2)
    p.add_argument("--T", type=int, default=20)
    p.add_argument("--frames", type=int, default=256)
    p.add_argument("--qber", type=float, default=0.03)
    p.add_argument("--steps", type=int, default=100)
    p.add_argument("--lr", type=float, default=0.01)
    p.add_argument("--eval-frames", type=int, default=1024)
    p.add_argument("--out", default=None)
    p.add_argument("--time", action="store_true",
                   help="only time one forward pass (T iterations, checkpoints kept) and one adjoint pass")
    args = p.parse_args(argv)
    n, m = args.n, int(round(args.n * (1 - args.rate)))
    codes = mbp_create_codes(mi.make_codes(n, m, {2: 0.3, 3: 0.4, 8: 0.3}, args.u, 4))
    if args.time:
        print(json.dumps(time_passes(codes, n, m, args), indent=1))
        return 0
    dec = NBPDecoder(codes, args.T, device="cuda")
    opt = torch.optim.Adam(dec.parameters(), lr=args.lr)
    losses = []
    t0 = time.time()
    for step in range(args.steps):
        llr, z, xb = frames(codes, n, args.frames, args.qber, seed=10_000 + step)
        L = dec(llr, z)
        loss = torch.nn.functional.binary_cross_entropy_with_logits(-L, xb.expand_as(L))
        opt.zero_grad()
        loss.backward()
        opt.step()
        losses.append(float(loss))
    train_s = time.time() - t0
    res = {"n": n, "m": m, "u": args.u, "T": args.T, "qber": args.qber, "frames": args.frames, "steps": args.steps,
           "train_seconds": train_s, "loss_first": losses[0], "loss_last": losses[-1],
           "alpha": dec.alpha.detach().cpu().numpy().tolist(), "beta": dec.beta.detach().cpu().numpy().tolist()}
    llr, z, _ = frames(codes, n, args.eval_frames, args.qber, seed=99_999)
    ones = torch.ones_like(dec.alpha)
    zeros = torch.zeros_like(dec.beta)
    with torch.no_grad():
        L_plain, _ = mbp_nbp_forward(codes, llr, z, ones, zeros)
        L_learn, _ = mbp_nbp_forward(codes, llr, z, dec.alpha, dec.beta)
    for name, L in (("plain", L_plain), ("learned", L_learn)):
        frac, mean_first = evaluate_frames(codes, L, z, args.eval_frames)
        res[name] = {"solved_fraction_by_iteration": frac.tolist(), "fer_at_T": float(1 - frac[-1]),
                     "mean_first_iteration": mean_first}
    text = json.dumps(res, indent=1)
    if args.out:
        with open(args.out, "w") as f:
            f.write(text)
    print(text)
    return 0


def time_passes(codes, n, m, args, reps=10, warmup=3):
    """CUDA-event times of the forward pass (posteriors of all T iterations and the per-iteration message
    checkpoints) and of the adjoint pass (gradients for alpha, beta and the LLRs) on one batch, inputs resident
    on the GPU, after warm-up passes."""
    llr, z, _ = frames(codes, n, args.frames, args.qber, seed=7)
    T, u = args.T, args.u
    alpha = torch.full((T, u), 0.9, device="cuda")
    beta = torch.full((T, u), 0.1, device="cuda")
    ws = torch.empty(mbp_nbp_workspace_size(codes, args.frames, T), dtype=torch.uint8, device="cuda")
    grad = torch.randn((T, args.frames, n), device="cuda", generator=torch.Generator("cuda").manual_seed(1))
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd, bwd = [], []
    for r in range(warmup + reps):
        ev[0].record()
        mbp_nbp_forward(codes, llr, z, alpha, beta, workspace=ws)
        ev[1].record()
        mbp_nbp_backward(codes, args.frames, alpha, beta, grad, ws, want_grad_llr=True)
        ev[2].record()
        torch.cuda.synchronize()
        if r >= warmup:
            fwd.append(ev[0].elapsed_time(ev[1]))
            bwd.append(ev[1].elapsed_time(ev[2]))
    f_ms, b_ms = float(np.median(fwd)), float(np.median(bwd))
    return {"n": n, "m": m, "u": u, "T": T, "frames": args.frames, "workspace_bytes": ws.numel(),
            "forward_ms": f_ms, "adjoint_ms": b_ms,
            "forward_frame_iterations_per_s": args.frames * T / (f_ms / 1e3),
            "note": "median of %d passes after %d warm-up passes, CUDA events, inputs on the GPU" % (reps, warmup)}


def evaluate_frames(codes, L: torch.Tensor, z: torch.Tensor, F: int):
    """Per iteration: the fraction of frames whose hard decision satisfies every syndrome (mbp_syndrome of the
    packed decision against Alice's words, matrix by matrix), and the mean first such iteration."""
    T = L.shape[0]
    m_words = [(mm + 31) // 32 for mm in codes.m]
    ok = torch.zeros((T, F), dtype=torch.bool, device=L.device)
    zf = z.view(-1)
    for t in range(T):
        zt = mbp_syndrome(codes, pack((L[t] < 0).to(torch.int32))).view(-1)
        good = torch.ones(F, dtype=torch.bool, device=L.device)
        off = 0
        for w in m_words:
            blk = F * w
            good &= torch.all((zt[off:off + blk] == zf[off:off + blk]).view(F, w), dim=1)
            off += blk
        ok[t] = good
    first = torch.where(ok.any(dim=0), ok.int().argmax(dim=0) + 1, torch.full((F,), T, device=L.device))
    return ok.float().mean(dim=1).cpu().numpy(), float(first.float().mean())


if __name__ == "__main__":
    sys.exit(main())
