"""CUDA path against the FP64 oracle where the message clip decides the result (needs a GB300).

The decoder clips variable-to-check messages to [-L_max, L_max] before eq. (6)
and check-to-variable messages after it (a degree-1 check sends +-L_max). The
oracle's clip is pinned in ``test_oracle_pins`` on star and chain codes whose
messages exceed L_max; here the same codes, with L_max = 3 or 4 and every frame
drawing its own priors and syndromes, go through the C ABI (LLR inputs, no
early exit) and the posteriors of eq. (2) are compared with the oracle's after
1 to 6 iterations: within 1e-9 for FP64 messages, 1e-3 for FP32.
"""
import numpy as np
import pytest
import torch

import mbp_inputs as mi
import oracle as orc
import test_oracle_pins as pins

pytestmark = pytest.mark.gpu

F = 45  # two tiles of 32 frames, the second ragged


@pytest.fixture(scope="module")
def mbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07979_gb300 as m
    m.build()
    return m


def _frames(dens, L, rng, draw):
    """F frames on one code: per-frame priors from `draw` and uniform random syndromes."""
    n = dens[0].shape[1]
    LP = np.stack([draw(rng) for _ in range(F)])
    zs = [rng.integers(0, 2, size=(F, h.shape[0])).astype(np.uint8) for h in dens]
    return n, LP, [mi.pack_bits(z) for z in zs]


def _cases(seed):
    rng = np.random.default_rng(seed)
    out = []
    for u in (1, 2, 3):
        L = 4.0
        n, dens, _, _, _ = pins._star(6, u, u - 1, rng, L)
        draw = lambda r, n=n, L=L: np.concatenate(
            [[r.uniform(-1, 1)], r.choice([-1.0, 1.0], size=n - 1) * r.uniform(0.3 * L, 3 * L, size=n - 1)])
        out.append(("star", u, L, dens, draw))
        L = 3.0
        dens, _, _, _ = pins._chain(10, u, rng, L)
        draw = lambda r, L=L: r.choice([-1.0, 1.0], size=10) * r.uniform(0.2 * L, 2.5 * L, size=10)
        out.append(("chain", u, L, dens, draw))
    return out


CASES = _cases(9100)


@pytest.mark.parametrize("case", range(len(CASES)), ids=[f"{c[0]}-u{c[1]}" for c in CASES])
@pytest.mark.parametrize("mode", ["f64", "f32-streaming", "f32-default"])
def test_clipped_posteriors_match_oracle(mbp, case, mode):
    kind, u, L, dens, draw = CASES[case]
    rng = np.random.default_rng(9200 + case)
    n, LP, zb = _frames(dens, L, rng, draw)
    H = [pins.csr_from_dense(h) for h in dens]
    codes = mbp.mbp_create_codes(H)
    zg = torch.from_numpy(np.concatenate([z.reshape(-1) for z in zb]).view(np.int32)).cuda()
    fp64 = mode == "f64"
    llr = torch.from_numpy(LP if fp64 else LP.astype(np.float32)).cuda()
    kw = dict(schedule=mbp.SCHED_STREAMING) if mode != "f32-default" else {}
    tol = 1e-9 if fp64 else 1e-3
    saturated = 0
    for T in (1, 2, 3, 6):
        ref = orc.decode(H, LP, zb, T, l_max=L, early_exit=False, want_lv=True, want_synd=True)
        out = mbp.mbp_decode_batch(codes, llr, zg, T, l_max=L, early_exit=False, want_soft=True, want_synd=True,
                                   **kw)
        lv = out["soft"].cpu().numpy()
        err = np.max(np.abs(lv - ref["L_V"]))
        assert err <= tol, (kind, u, T, err)
        assert np.array_equal(out["iters"].cpu().numpy(), np.full(F, T))
        xh = out["x_hat_bits"].cpu().numpy().view(np.uint32)
        sure = np.all(np.abs(ref["L_V"]) > 10 * tol, axis=1)  # frames with no posterior at a decision boundary
        assert np.array_equal(xh[sure], ref["x_hat_bits"][sure])
        assert np.array_equal(out["success"].cpu().numpy()[sure], ref["success"][sure])
        saturated += int(np.sum(np.abs(LP) > L))
    assert saturated > 0
