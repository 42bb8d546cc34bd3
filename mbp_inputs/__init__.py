"""Seeded synthetic inputs for multi-matrix BP reconciliation.

This module is shared by the CUDA path's tests and benchmark and by the oracle's
tests. It holds none of the decoding arithmetic:

* ``make_codes`` builds the u PEG parity-check matrices H_1..H_u (Section 2 of the
  paper assumes u > 1 matrices "generated by PEG"); the construction is in
  ``peg.c``.
* ``bsc_frames`` draws Alice's sifted key x (uniform bits) and Bob's key
  y = x XOR Bernoulli(e) noise, i.e. a binary symmetric channel with QBER e.
* ``pack_bits`` / ``unpack_bits`` convert between 0/1 arrays and the packed
  layout used at the library boundary: uint32 words, LSB first, bit i of a frame
  in word i >> 5 at position i & 31.

Syndromes (eq. 1) and channel LLRs (eq. 5) are method arithmetic and are
computed by each side on its own.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_peg.so")
_SRC = os.path.join(_HERE, "peg.c")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile ``peg.c`` into ``_peg.so`` next to it (host C, any architecture)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.mbpin_peg.restype = ctypes.c_int
            lib.mbpin_peg.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_void_p, ctypes.c_int,
                                      ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p]
            lib.mbpin_xoshiro_stream.restype = None
            lib.mbpin_xoshiro_stream.argtypes = [ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p]
            _lib = lib
    return _lib


def xoshiro_stream(seed: int, count: int) -> np.ndarray:
    """Raw xoshiro256** outputs (seeded through splitmix64), for tests of the generator."""
    out = np.zeros(count, dtype=np.uint64)
    _load().mbpin_xoshiro_stream(ctypes.c_uint64(seed & (2**64 - 1)), count, out.ctypes.data)
    return out


class CSR:
    """One m x n binary matrix: row_ptr[m+1], col_idx[nnz] (int32, ascending columns per row)."""

    def __init__(self, n: int, m: int, row_ptr: np.ndarray, col_idx: np.ndarray):
        self.n, self.m = int(n), int(m)
        self.row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int32)
        self.col_idx = np.ascontiguousarray(col_idx, dtype=np.int32)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def dense(self) -> np.ndarray:
        h = np.zeros((self.m, self.n), dtype=np.uint8)
        rows = np.repeat(np.arange(self.m), np.diff(self.row_ptr))
        h[rows, self.col_idx] = 1
        return h

    def row_degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def col_degrees(self) -> np.ndarray:
        return np.bincount(self.col_idx, minlength=self.n)


def degree_sequence(n: int, dist: dict[int, float]) -> np.ndarray:
    """Column degrees from a node-perspective distribution {degree: fraction}.

    Class counts are round(p * n) for every class but the last, which takes the
    remainder; the sequence is sorted by non-decreasing degree (PEG's order).
    """
    degs = sorted(dist)
    counts = [int(round(dist[d] * n)) for d in degs[:-1]]
    counts.append(n - sum(counts))
    if min(counts) < 0:
        raise ValueError("degree distribution does not fit n")
    return np.repeat(np.asarray(degs, dtype=np.int32), counts)


def checks_for_rate(n: int, rate: float) -> int:
    """m = round(n (1 - R)), the code rate R = 1 - m/n of Section 4."""
    return int(round(n * (1.0 - rate)))


def matrix_seed(cfg_seed: int, l: int) -> int:
    """PEG seed of matrix l (0-based) for a configuration seed."""
    return (((cfg_seed & 0xFFFFFFFF) << 32) | (((l + 1) * 0x9E3779B1) & 0xFFFFFFFF)) & (2**64 - 1)


def peg_matrix(n: int, m: int, var_deg: np.ndarray, seed: int, depth_cap: int = -1) -> CSR:
    var_deg = np.ascontiguousarray(var_deg, dtype=np.int32)
    if var_deg.shape != (n,):
        raise ValueError("var_deg must have n entries")
    nnz = int(var_deg.sum())
    row_ptr = np.zeros(m + 1, dtype=np.int32)
    col_idx = np.zeros(max(nnz, 1), dtype=np.int32)
    rc = _load().mbpin_peg(n, m, var_deg.ctypes.data, depth_cap, ctypes.c_uint64(seed & (2**64 - 1)),
                           row_ptr.ctypes.data, col_idx.ctypes.data)
    if rc != 0:
        raise RuntimeError(f"PEG construction failed (rc={rc}) for n={n} m={m}")
    return CSR(n, m, row_ptr, col_idx[:nnz])


def default_depth_cap(n: int) -> int:
    """Unlimited search for small codes; 1 (no 4-cycles) for large ones to bound the cost."""
    return -1 if n <= 8192 else 1


def make_codes(n: int, m: int, dist: dict[int, float], u: int, cfg_seed: int,
               depth_cap: int | None = None) -> list[CSR]:
    """u PEG matrices sharing n and the column degree sequence, seeds (cfg_seed, l)."""
    var_deg = degree_sequence(n, dist)
    cap = default_depth_cap(n) if depth_cap is None else depth_cap
    return [peg_matrix(n, m, var_deg, matrix_seed(cfg_seed, l), cap) for l in range(u)]


def words(nbits: int) -> int:
    return (nbits + 31) // 32


def pack_bits(bits: np.ndarray) -> np.ndarray:
    """0/1 array [..., nbits] -> uint32 [..., ceil(nbits/32)], LSB first."""
    bits = np.asarray(bits, dtype=np.uint8)
    nb = bits.shape[-1]
    pad = words(nb) * 32 - nb
    if pad:
        bits = np.concatenate([bits, np.zeros(bits.shape[:-1] + (pad,), dtype=np.uint8)], axis=-1)
    by = np.packbits(bits, axis=-1, bitorder="little")
    return np.ascontiguousarray(by).view("<u4").astype(np.uint32)


def unpack_bits(w: np.ndarray, nbits: int) -> np.ndarray:
    w = np.ascontiguousarray(np.asarray(w, dtype=np.uint32)).astype("<u4")
    by = w.view(np.uint8)
    return np.unpackbits(by, axis=-1, bitorder="little")[..., :nbits]


def bsc_frames(n: int, frames: int, qber, seed: int, stream: int = 0):
    """Alice's keys x and Bob's keys y = x XOR Bernoulli(e) noise, packed.

    ``qber`` is a scalar or a per-frame array. Returns (x_bits, y_bits, e) with
    x_bits, y_bits uint32 [frames, ceil(n/32)] and e float64 [frames].
    """
    e = np.broadcast_to(np.asarray(qber, dtype=np.float64), (frames,)).copy()
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), int(stream), 0x51D])))
    W = words(n)
    x = np.empty((frames, W), dtype=np.uint32)
    y = np.empty((frames, W), dtype=np.uint32)
    for f in range(frames):
        xb = rng.integers(0, 2, size=n, dtype=np.uint8)
        noise = (rng.random(n) < e[f]).astype(np.uint8)
        x[f] = pack_bits(xb)
        y[f] = pack_bits(xb ^ noise)
    return x, y, e


# Workloads of the benchmark and the parity tests, named by what they are.
CODE_N1024_RATE05_DV3 = dict(n=1024, m=512, dist={3: 1.0}, u=2, seed=0)
CODE_N65536_RATE07_DV238 = dict(n=65536, m=19661, dist={2: 0.3, 3: 0.4, 8: 0.3}, u=2, seed=1)


# Uneven batches: frames of several codes in one decode call. Each frame draws its code class (n, R, u)
# uniformly from the grid below and its QBER from U[qber_lo, qber_hi]; the column degrees follow the n=65536
# rate-0.7 workload's distribution at every size and rate, m = round(n (1 - R)) per matrix.
UNEVEN_SIZES = (1 << 14, 1 << 16, 1 << 18)
UNEVEN_RATES = (0.5, 0.6, 0.7, 0.8)
UNEVEN_US = (2, 3)
UNEVEN_DIST = {2: 0.3, 3: 0.4, 8: 0.3}


def uneven_batch(frames: int, seed: int, sizes=UNEVEN_SIZES, rates=UNEVEN_RATES, us=UNEVEN_US,
                 qber=(0.01, 0.04)) -> list[dict]:
    """Group specs of an uneven batch: one dict per (n, R, u) class with its code parameters
    (n, m, dist, u, cfg_seed), the number of frames that drew it and their QBERs (float64 array)."""
    classes = [(n, r, u) for n in sizes for r in rates for u in us]
    rng = np.random.Generator(np.random.PCG64(np.random.SeedSequence([int(seed), 0xBA7C])))
    cls = rng.integers(0, len(classes), size=frames)
    e = rng.uniform(qber[0], qber[1], size=frames)
    groups = []
    for k, (n, r, u) in enumerate(classes):
        idx = np.flatnonzero(cls == k)
        groups.append(dict(n=n, m=int(round(n * (1.0 - r))), dist=dict(UNEVEN_DIST), u=u, rate=r,
                           cfg_seed=int(seed) * 100 + k, frames=int(idx.size), qber=e[idx].copy()))
    return groups
