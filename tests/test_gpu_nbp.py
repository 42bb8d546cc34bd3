"""Unrolled normalised BP on the GPU (mbp_nbp_forward / mbp_nbp_backward / NormalizedBP), through the C ABI.

  * alpha = 1, beta = 0 reproduces the plain decoder's posteriors bit for bit, every iteration;
  * the forward posteriors agree with the FP64 reference (oracle/nbp.py) for random alpha, beta;
  * the hand-written adjoint agrees with the FP64 reference gradient (autograd) and with central finite
    differences (eps = 1e-3) of the GPU forward;
  * the gradient is deterministic, and a few optimiser steps on decoder-generated frames lower the loss
    at the n=16384 rate-0.6 u=2 size with 20 iterations.
"""
import numpy as np
import pytest
import torch

import mbp_inputs as mi
import oracle as orc
from oracle import nbp as onbp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def mbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07979_gb300 as m
    m.build()
    return m


def dev(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a))
    return (t.to(dtype) if dtype is not None else t).cuda()


def i32(a):
    return np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)


class Case:
    def __init__(self, mbp, n, m, u, seed, F, qber, dist=None):
        dist = dist or {2: 0.3, 3: 0.4, 8: 0.3}
        self.n, self.F, self.u = n, F, u
        self.H = mi.make_codes(n, m, dist, u, seed)
        self.x, self.y, self.e = mi.bsc_frames(n, F, qber, seed=seed + 500)
        self.LP = orc.bsc_llr(self.y, n, self.e)
        self.z_orc = orc.syndrome(self.H, self.x)
        self.codes = mbp.mbp_create_codes(self.H)
        self.z = mbp.mbp_syndrome(self.codes, dev(i32(self.x)))
        self.llr = dev(self.LP.astype(np.float32))


def test_plain_parameters_bit_exact_with_plain_decoder(mbp):
    c = Case(mbp, 4000, 1600, 2, 3, 45, 0.05)
    T = 5
    lv, _ = mbp.mbp_nbp_forward(c.codes, c.llr, c.z, torch.ones((T, 2), device="cuda"),
                                torch.zeros((T, 2), device="cuda"))
    for t in range(1, T + 1):
        ref = mbp.mbp_decode_batch(c.codes, c.llr, c.z, t, early_exit=False, want_soft=True,
                                   schedule=mbp.SCHED_STREAMING)
        assert torch.equal(lv[t - 1], ref["soft"]), t


def params(T, u, seed):
    rng = np.random.default_rng(seed)
    return rng.uniform(0.6, 1.1, size=(T, u)), rng.uniform(0.0, 0.6, size=(T, u))


def test_forward_matches_oracle(mbp):
    c = Case(mbp, 1000, 400, 2, 7, 9, 0.05)
    T = 6
    a, b = params(T, 2, 1)
    lv, _ = mbp.mbp_nbp_forward(c.codes, c.llr, c.z, dev(a, torch.float32), dev(b, torch.float32))
    ref = onbp.forward_np(c.H, c.LP, c.z_orc, a.astype(np.float32).astype(np.float64),
                          b.astype(np.float32).astype(np.float64))
    err = np.max(np.abs(lv.cpu().numpy() - ref))
    print(f"max |dL| over {T} iterations: {err:.3g}")
    assert err <= 1e-3


def grads_gpu(mbp, c, a, b, G, want_llr=True):
    at, bt = dev(a, torch.float32), dev(b, torch.float32)
    lv, ws = mbp.mbp_nbp_forward(c.codes, c.llr, c.z, at, bt)
    ga, gb, gl = mbp.mbp_nbp_backward(c.codes, c.F, at, bt, dev(G, torch.float32), ws, want_grad_llr=want_llr)
    return lv, ga.cpu().numpy(), gb.cpu().numpy(), (gl.cpu().numpy() if gl is not None else None)


def rel_err(x, y):
    return float(np.linalg.norm(x - y) / max(np.linalg.norm(y), 1e-30))


@pytest.mark.parametrize("seed", [1, 2])
def test_gradient_matches_fp64_reference(mbp, seed):
    c = Case(mbp, 1000, 400, 2, 10 + seed, 6, 0.06)
    T = 5
    a, b = params(T, 2, seed)
    a32, b32 = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(seed + 9)
    G = rng.normal(size=(T, c.F, c.n)) / (c.F * c.n)
    _, ga, gb, gl = grads_gpu(mbp, c, a32, b32, G)
    _, ra, rb, rl = onbp.gradient(c.H, c.LP, c.z_orc, a32, b32, G)
    print(f"relative errors: alpha {rel_err(ga, ra):.2e}, beta {rel_err(gb, rb):.2e}, llr {rel_err(gl, rl):.2e}")
    assert rel_err(ga, ra) <= 2e-3 and rel_err(gb, rb) <= 2e-3 and rel_err(gl, rl) <= 2e-3


@pytest.mark.slow
def test_gradient_matches_fp64_reference_config5(mbp):
    """The normalised-BP size: n = 16384, rate 0.6, u = 2, 20 unrolled iterations, on 2 frames at QBER 3%:
    the hand-written adjoint against the FP64 autograd gradient (relative 2e-3 in the norm, as above)."""
    c = Case(mbp, 16384, 6554, 2, 4, 2, 0.03)
    T = 20
    a, b = params(T, 2, 3)
    a32, b32 = a.astype(np.float32).astype(np.float64), b.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(17)
    G = rng.normal(size=(T, c.F, c.n)) / (c.F * c.n)
    lv, ga, gb, gl = grads_gpu(mbp, c, a32, b32, G)
    ref_lv = onbp.forward_np(c.H, c.LP, c.z_orc, a32, b32)
    _, ra, rb, rl = onbp.gradient(c.H, c.LP, c.z_orc, a32, b32, G)
    print(f"T={T}: max |dL| {np.max(np.abs(lv.cpu().numpy() - ref_lv)):.3g}; relative errors: alpha "
          f"{rel_err(ga, ra):.2e}, beta {rel_err(gb, rb):.2e}, llr {rel_err(gl, rl):.2e}")
    assert rel_err(ga, ra) <= 2e-3 and rel_err(gb, rb) <= 2e-3 and rel_err(gl, rl) <= 2e-3


def test_gradient_matches_central_differences(mbp):
    """J = BCE of sigmoid(-L^T) against the true bits; central differences of the GPU forward, eps = 1e-3."""
    c = Case(mbp, 1000, 400, 2, 21, 32, 0.06)
    T = 4
    a, b = params(T, 2, 5)
    xb = np.stack([mi.unpack_bits(c.x[f], c.n) for f in range(c.F)]).astype(np.float64)

    def loss_and_grad(a_, b_):
        lv, _ = mbp.mbp_nbp_forward(c.codes, c.llr, c.z, dev(a_, torch.float32), dev(b_, torch.float32))
        L = lv.cpu().numpy().astype(np.float64)
        loss, gT = onbp.bce_grad(L[-1], xb)
        return loss, gT

    _, gT = loss_and_grad(a, b)
    G = np.zeros((T, c.F, c.n))
    G[-1] = gT
    _, ga, gb, _ = grads_gpu(mbp, c, a, b, G, want_llr=False)
    eps = 1e-3
    checked = 0
    for (t, l) in [(0, 0), (1, 1), (2, 0), (3, 1)]:
        for which, g in (("alpha", ga), ("beta", gb)):
            d = np.zeros_like(a)
            d[t, l] = eps
            if which == "alpha":
                fd = (loss_and_grad(a + d, b)[0] - loss_and_grad(a - d, b)[0]) / (2 * eps)
            else:
                fd = (loss_and_grad(a, b + d)[0] - loss_and_grad(a, b - d)[0]) / (2 * eps)
            print(f"{which}[{t},{l}]: adjoint {g[t, l]:.6g}, central difference {fd:.6g}")
            assert abs(fd - g[t, l]) <= 0.02 * abs(fd) + 2e-5
            checked += 1
    assert checked == 8


def test_backward_is_deterministic(mbp):
    c = Case(mbp, 2000, 800, 2, 4, 40, 0.05)
    T = 6
    a, b = params(T, 2, 3)
    G = np.random.default_rng(0).normal(size=(T, c.F, c.n))
    r1 = grads_gpu(mbp, c, a, b, G)
    r2 = grads_gpu(mbp, c, a, b, G)
    for x, y in zip(r1[1:], r2[1:]):
        assert np.array_equal(x, y)


def test_autograd_function_and_training_steps(mbp):
    """The n=16384, rate-0.6, u=2 code, 20 unrolled iterations, 64 frames generated at QBER 3%: NormalizedBP's
    gradients equal mbp_nbp_backward's, and Adam steps from a poor start (alpha = 0.5, beta = 0.5: messages
    halved and offset) lower the loss (mean over the iterations of the BCE of sigmoid(-L^t) against the true
    bits) on the training batch."""
    n, m, T, F = 16384, 6554, 20, 64
    H = mi.make_codes(n, m, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 4)
    codes = mbp.mbp_create_codes(H)
    dec = mbp.NBPDecoder(codes, T, device="cuda")
    with torch.no_grad():
        dec.alpha.fill_(0.5)
        dec.beta.fill_(0.5)
    opt = torch.optim.Adam(dec.parameters(), lr=0.05)
    x, y, e = mi.bsc_frames(n, F, 0.03, seed=100)
    llr = mbp.mbp_bsc_llr(dev(i32(y)), dev(e), n, torch.float32)
    z = mbp.mbp_syndrome(codes, dev(i32(x)))
    xb = torch.from_numpy(np.stack([mi.unpack_bits(x[f], n) for f in range(F)]).astype(np.float32)).cuda()

    def multiloss(L):
        return torch.nn.functional.binary_cross_entropy_with_logits(-L, xb.expand_as(L))

    losses = []
    for step in range(10):
        L = dec(llr, z)
        loss = multiloss(L)
        opt.zero_grad()
        loss.backward()
        if step == 0:
            Ld = L.detach().requires_grad_(True)
            (G,) = torch.autograd.grad(multiloss(Ld), [Ld])
            _, ws = mbp.mbp_nbp_forward(codes, llr, z, dec.alpha, dec.beta, want_lv=False)
            ga, gb, _ = mbp.mbp_nbp_backward(codes, F, dec.alpha, dec.beta, G, ws)
            assert torch.equal(ga, dec.alpha.grad) and torch.equal(gb, dec.beta.grad)
        opt.step()
        losses.append(float(loss))
    print("losses:", [round(v, 6) for v in losses])
    assert np.isfinite(losses).all()
    assert losses[-1] < 0.8 * losses[0]
