"""FP64 reference of the unrolled, normalised multi-matrix BP and of its gradient.

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT: only the test suite may import
this module. It shares no code with the CUDA library. It is written with plain
PyTorch CPU operations in float64 so that the reference gradient comes from
autograd (a library primitive) and not from a hand derivation.

What it computes. The paper's decoder (Algorithm 1 with eq. 6 and eq. 2,
flooding over the u matrices) is unrolled for T iterations and every
check-to-variable message is rescaled by learnable per-iteration, per-matrix
scalars (the paper has no learned form; this is the reading used here):

    V_e^t  = clip(L^{t-1}[i(e)] - C_e^{t-1}, +-L_max)          (L^0 = L_P, C^0 = 0)
    c_e^t  = (-1)^{z_j} prod_{e' != e} sgn(V_e'^t)
             * min(2 atanh(prod_{e' != e} tanh(|V_e'^t| / 2)), L_max)      (eq. 6, clipped;
             evaluated in the complement form ln((1 - D) / D), see forward())
    C_e^t  = alpha[t, l] * s_e^t * max(|c_e^t| - beta[t, l], 0)   (l = matrix of the row of e,
                                                                   s_e^t = the sign factor of c_e^t)
    L^t[i] = L_P[i] + sum over the edges e of node i (all matrices) of C_e^t   (eq. 2)

With alpha = 1 and beta = 0 this is the plain decoder without early exit. The
exclusions e' != e use prefix and suffix combinations, never a division. The sign
of a zero message is +. clip and min pass the gradient on their closed
interval (torch.clamp); max(. , 0) passes it where its argument is > 0.

Parity status: pinned by tests/test_oracle_nbp.py (alpha = 1, beta = 0 against
the C oracle's plain decoder; a row-by-row unrolled evaluation through the C
oracle's check-node routine; closed forms at alpha = 0 and large beta; central
finite differences of the gradient).
"""
from __future__ import annotations

import numpy as np
import torch

DT = torch.float64


class Graph:
    """Index tensors of the stacked code [H_1; ...; H_u] in stacked CSR edge order."""

    def __init__(self, codes):
        self.n = int(codes[0].n)
        self.u = len(codes)
        cols, rows, row_mat, row_local, deg = [], [], [], [], []
        r = 0
        for l, h in enumerate(codes):
            rp = np.asarray(h.row_ptr, np.int64)
            ci = np.asarray(h.col_idx, np.int64)
            for j in range(int(h.m)):
                a, b = int(rp[j]), int(rp[j + 1])
                cols.extend(ci[a:b].tolist())
                rows.extend([r] * (b - a))
                row_mat.append(l)
                row_local.append(j)
                deg.append(b - a)
                r += 1
        self.m_tot = r
        self.E = len(cols)
        self.col = torch.tensor(cols, dtype=torch.int64)
        self.row = torch.tensor(rows, dtype=torch.int64)
        self.row_mat = torch.tensor(row_mat, dtype=torch.int64)
        self.row_local = np.asarray(row_local, np.int64)
        self.deg = np.asarray(deg, np.int64)
        self.dmax = int(self.deg.max()) if r else 0
        # padded [m_tot, dmax] table of edge indices (E = padding) and the slot of every edge in it
        pad = np.full((r, max(self.dmax, 1)), self.E, np.int64)
        starts = np.concatenate([[0], np.cumsum(self.deg)])
        for q in range(r):
            pad[q, :self.deg[q]] = np.arange(starts[q], starts[q + 1])
        self.pad = torch.tensor(pad)
        self.valid = self.pad < self.E
        self.edge_mat = self.row_mat[self.row]


def syndrome_signs(g: Graph, codes, z_bits, F: int) -> torch.Tensor:
    """(-1)^{z_j} per frame and stacked row: [F, m_tot] float64."""
    s = np.ones((F, g.m_tot))
    r0 = 0
    for l, h in enumerate(codes):
        z = np.asarray(z_bits[l], np.uint32).reshape(F, -1)
        for j in range(int(h.m)):
            bit = (z[:, j >> 5] >> np.uint32(j & 31)) & np.uint32(1)
            s[:, r0 + j] = np.where(bit == 1, -1.0, 1.0)
        r0 += int(h.m)
    return torch.tensor(s, dtype=DT)


def forward(g: Graph, L_P: torch.Tensor, signs: torch.Tensor, alpha: torch.Tensor, beta: torch.Tensor,
            l_max: float = 20.0) -> torch.Tensor:
    """Posteriors L^1..L^T of the unrolled normalised BP: [T, F, n] (differentiable in L_P, alpha, beta)."""
    T = alpha.shape[0]
    F = L_P.shape[0]
    L = L_P
    C = torch.zeros((F, g.E), dtype=DT)
    out = []
    for t in range(T):
        V = torch.clamp(L[:, g.col] - C, -l_max, l_max)                       # [F, E]
        Vp = torch.cat([V, torch.zeros((F, 1), dtype=DT)], dim=1)[:, g.pad]    # [F, m_tot, dmax], padding 0
        # eq. (6) in the complement form: with delta = (1 - tanh(|V|/2)) / 2 = 1 / (1 + e^|V|), the product of
        # tanh over a set is 1 - 2 D with D the (+)-combination of the deltas, x (+) y = x + y - 2 x y, and
        # 2 atanh(1 - 2 D) = ln((1 - D) / D). Padding has delta = 0, the neutral element of (+).
        delta = torch.where(g.valid, torch.sigmoid(-torch.abs(Vp)), torch.zeros((), dtype=DT))
        sg = torch.where(Vp < 0, -1.0, 1.0).to(DT)
        zero = torch.zeros_like(delta[..., 0])
        pre, acc = [], zero
        for k in range(delta.shape[-1]):                                  # combination of r < k
            pre.append(acc)
            acc = acc + delta[..., k] - 2.0 * acc * delta[..., k]
        suf, acc = [None] * delta.shape[-1], zero
        for k in reversed(range(delta.shape[-1])):                        # combination of r > k
            suf[k] = acc
            acc = acc + delta[..., k] - 2.0 * acc * delta[..., k]
        D = torch.stack([p_ + s_ - 2.0 * p_ * s_ for p_, s_ in zip(pre, suf)], dim=-1)   # r != k
        s_all = torch.prod(sg, dim=-1, keepdim=True) * signs[:, :, None]
        s_ex = s_all * sg                                                                 # sign of the others
        Dc = torch.clamp(D, min=1e-300)
        g_ex = torch.where(D > 0, torch.log1p(-Dc) - torch.log(Dc), torch.full_like(D, float("inf")))
        c_mag = torch.clamp(g_ex, max=l_max)
        a = alpha[t][g.row_mat][None, :, None]
        b = beta[t][g.row_mat][None, :, None]
        Cp = a * s_ex * torch.relu(c_mag - b)                                             # [F, m_tot, dmax]
        C = Cp[:, g.valid]                                                                # stacked CSR order
        L = L_P.index_add(1, g.col, C)
        out.append(L)
    return torch.stack(out)


def forward_np(codes, L_P: np.ndarray, z_bits, alpha: np.ndarray, beta: np.ndarray, l_max: float = 20.0):
    g = Graph(codes)
    F = L_P.shape[0]
    with torch.no_grad():
        return forward(g, torch.tensor(L_P, dtype=DT), syndrome_signs(g, codes, z_bits, F),
                       torch.tensor(alpha, dtype=DT), torch.tensor(beta, dtype=DT), l_max).numpy()


def gradient(codes, L_P: np.ndarray, z_bits, alpha: np.ndarray, beta: np.ndarray, grad_L: np.ndarray,
             l_max: float = 20.0):
    """Reference gradient of J = sum(grad_L * L) (grad_L: [T, F, n]) with respect to alpha, beta and L_P,
    by autograd through forward(); returns (L [T, F, n], d alpha [T, u], d beta [T, u], d L_P [F, n])."""
    g = Graph(codes)
    F = L_P.shape[0]
    lp = torch.tensor(L_P, dtype=DT, requires_grad=True)
    a = torch.tensor(alpha, dtype=DT, requires_grad=True)
    b = torch.tensor(beta, dtype=DT, requires_grad=True)
    L = forward(g, lp, syndrome_signs(g, codes, z_bits, F), a, b, l_max)
    J = torch.sum(L * torch.tensor(grad_L, dtype=DT))
    J.backward()
    return L.detach().numpy(), a.grad.numpy(), b.grad.numpy(), lp.grad.numpy()


def bce_grad(L: np.ndarray, x_bits_dense: np.ndarray) -> tuple[float, np.ndarray]:
    """Binary cross-entropy of P(bit = 1) = sigmoid(-L) against the true bits, averaged over entries, and its
    derivative with respect to L: mean(x softplus(L) + (1 - x) softplus(-L)), d/dL = (sigmoid(L) - (1 - x)) / N."""
    x = x_bits_dense.astype(np.float64)
    N = L.size
    loss = float(np.mean(x * np.logaddexp(0.0, L) + (1 - x) * np.logaddexp(0.0, -L)))
    return loss, (1.0 / (1.0 + np.exp(-L)) - (1.0 - x)) / N
