"""FP64 CPU oracle for multi-matrix BP reconciliation (MBP).

TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT: only the test suite, the smoke
check and the benchmark's CPU-baseline leg may import this package. It shares
no code with the CUDA library (``paper_2001_07979_gb300``) and never imports it.

The arithmetic lives in ``mbp_oracle.c`` (plain C, double precision), loaded
with ctypes; this file only marshals arguments. See that file's header for the
equations it follows and the readings of the paper it takes.

``nbp.py`` (plain PyTorch CPU float64) is the reference of the unrolled,
normalised BP with learnable scale and offset and of its gradient (autograd).

Parity status: every function here is pinned by ``tests/test_oracle_*.py``
against closed forms, brute-force enumeration, GF(2) elimination and
invariants; none is "parity unpinned".
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "mbp_oracle.c")
_SO = os.path.join(_HERE, "_mbp_oracle.so")
_lock = threading.Lock()
_lib = None

L_MAX_DEFAULT = 20.0


def build(force: bool = False) -> str:
    """Compile the oracle with gcc -O2 (host C; x86_64 or aarch64)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-D_POSIX_C_SOURCE=200809L", "-shared", "-fPIC",
                               "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _SO)
    return _SO


def _configure(lib):
    P, I, D = ctypes.c_void_p, ctypes.c_int, ctypes.c_double
    lib.orc_syndrome.restype = I
    lib.orc_syndrome.argtypes = [I, I, P, P, P, I, P, P]
    lib.orc_bsc_llr.restype = None
    lib.orc_bsc_llr.argtypes = [I, P, D, P]
    lib.orc_boxplus.restype = D
    lib.orc_boxplus.argtypes = [D, D]
    lib.orc_check_node.restype = I
    lib.orc_check_node.argtypes = [I, P, I, D, P]
    lib.orc_check_node_tanh.restype = I
    lib.orc_check_node_tanh.argtypes = [I, P, I, D, P]
    lib.orc_decode.restype = I
    lib.orc_decode.argtypes = [I, I, P, P, P, I, P, P, I, D, I, I, P, P, P, P, P, P]
    lib.orc_decode_ex.restype = I
    lib.orc_decode_ex.argtypes = [I, I, P, P, P, I, P, P, I, D, I, I, I, I, P, P, P, P, P, P]
    lib.orc_check_node_minsum.restype = I
    lib.orc_check_node_minsum.argtypes = [I, P, I, D, P]
    return lib


def _load():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _configure(ctypes.CDLL(build()))
    return _lib


@contextlib.contextmanager
def library_override(so_path: str):
    """Run the wrappers against another build of the oracle source (mutation tests only)."""
    global _lib
    _load()
    with _lock:
        saved, _lib = _lib, _configure(ctypes.CDLL(so_path))
    try:
        yield
    finally:
        with _lock:
            _lib = saved


def _words(nbits: int) -> int:
    return (nbits + 31) // 32


def _cat(codes):
    n = codes[0].n
    if any(h.n != n for h in codes):
        raise ValueError("all matrices must share n")
    m = np.asarray([h.m for h in codes], dtype=np.int32)
    rp = np.ascontiguousarray(np.concatenate([np.asarray(h.row_ptr, np.int32) for h in codes]))
    ci = np.ascontiguousarray(np.concatenate([np.asarray(h.col_idx, np.int32) for h in codes]))
    return n, m, rp, ci


def _u32(a):
    return np.ascontiguousarray(a, dtype=np.uint32)


def syndrome(codes, x_bits: np.ndarray) -> list[np.ndarray]:
    """eq. (1): z^l = H_l x mod 2 for each matrix; returns u arrays [F, ceil(m_l/32)]."""
    n, m, rp, ci = _cat(codes)
    x = _u32(x_bits).reshape(-1, _words(n))
    F = x.shape[0]
    z = np.zeros(int(sum(F * _words(int(ml)) for ml in m)), dtype=np.uint32)
    rc = _load().orc_syndrome(len(codes), n, m.ctypes.data, rp.ctypes.data, ci.ctypes.data, F,
                              x.ctypes.data, z.ctypes.data)
    if rc:
        raise RuntimeError(f"orc_syndrome rc={rc}")
    out, off = [], 0
    for ml in m:
        w = F * _words(int(ml))
        out.append(z[off:off + w].reshape(F, _words(int(ml))))
        off += w
    return out


def bsc_llr(y_bits: np.ndarray, n: int, qber) -> np.ndarray:
    """eq. (5) priors -> channel LLR L_P [F, n] (float64)."""
    y = _u32(y_bits).reshape(-1, _words(n))
    F = y.shape[0]
    e = np.broadcast_to(np.asarray(qber, dtype=np.float64), (F,))
    out = np.zeros((F, n), dtype=np.float64)
    lib = _load()
    for f in range(F):
        lib.orc_bsc_llr(n, y[f].ctypes.data, float(e[f]), out[f].ctypes.data)
    return out


def boxplus(a: float, b: float) -> float:
    return _load().orc_boxplus(float(a), float(b))


def check_node(v2c, z: int, l_max: float = L_MAX_DEFAULT) -> np.ndarray:
    """eq. (6) for one check (Jacobian-log form with prefix/suffix extrinsics)."""
    v = np.ascontiguousarray(v2c, dtype=np.float64)
    out = np.zeros_like(v)
    rc = _load().orc_check_node(len(v), v.ctypes.data, int(z), float(l_max), out.ctypes.data)
    if rc:
        raise RuntimeError(f"orc_check_node rc={rc}")
    return out


def check_node_tanh(v2c, z: int, l_max: float = L_MAX_DEFAULT) -> np.ndarray:
    """eq. (6) as printed, tanh/atanh product (cross-check form)."""
    v = np.ascontiguousarray(v2c, dtype=np.float64)
    out = np.zeros_like(v)
    _load().orc_check_node_tanh(len(v), v.ctypes.data, int(z), float(l_max), out.ctypes.data)
    return out


def check_node_minsum(v2c, z: int, l_max: float = L_MAX_DEFAULT) -> np.ndarray:
    """The min-sum check rule (variant): sign of the others and z, smallest other magnitude."""
    v = np.ascontiguousarray(v2c, dtype=np.float64)
    out = np.zeros_like(v)
    _load().orc_check_node_minsum(len(v), v.ctypes.data, int(z), float(l_max), out.ctypes.data)
    return out


RULES = {"sum-product": 0, "min-sum": 1}
UPDATES = {"flooding": 0, "matrix-serial": 1}


def decode(codes, L_P: np.ndarray, z_bits, max_iter: int, l_max: float = L_MAX_DEFAULT,
           early_exit: bool = True, threads: int = 1, want_lv: bool = False, want_c2v: bool = False,
           want_synd: bool = False, rule: str = "sum-product", update: str = "flooding") -> dict:
    """Algorithm 1 (flooding MBP) on F frames; rule="min-sum" and update="matrix-serial" select the variants.

    L_P [F, n] float64; z_bits: list of u arrays [F, ceil(m_l/32)] (or one flat
    array in the [u][F][words] layout). Returns a dict with x_hat_bits, iters,
    success and, on request, synd_ok [F, u], L_V [F, n], c2v [F, E_tot]
    (stacked CSR edge order).
    """
    n, m, rp, ci = _cat(codes)
    LP = np.ascontiguousarray(L_P, dtype=np.float64).reshape(-1, n)
    F = LP.shape[0]
    if isinstance(z_bits, (list, tuple)):
        z = _u32(np.concatenate([np.asarray(a, np.uint32).reshape(-1) for a in z_bits]))
    else:
        z = _u32(z_bits).reshape(-1)
    if z.size != sum(F * _words(int(ml)) for ml in m):
        raise ValueError("z_bits has the wrong size")
    e_tot = int(rp_total(codes))
    xh = np.zeros((F, _words(n)), dtype=np.uint32)
    it = np.zeros(F, dtype=np.int32)
    ok = np.zeros(F, dtype=np.uint8)
    so = np.zeros((F, len(codes)), dtype=np.uint8) if want_synd else None
    lv = np.zeros((F, n), dtype=np.float64) if want_lv else None
    cv = np.zeros((F, e_tot), dtype=np.float64) if want_c2v else None
    ptr = lambda a: a.ctypes.data if a is not None else None
    rc = _load().orc_decode_ex(len(codes), n, m.ctypes.data, rp.ctypes.data, ci.ctypes.data, F, LP.ctypes.data,
                               z.ctypes.data, int(max_iter), float(l_max), int(bool(early_exit)), RULES[rule],
                               UPDATES[update], int(threads), xh.ctypes.data, it.ctypes.data, ok.ctypes.data,
                               ptr(so), ptr(lv), ptr(cv))
    if rc:
        raise RuntimeError(f"orc_decode rc={rc}")
    out = dict(x_hat_bits=xh, iters=it, success=ok)
    if want_synd:
        out["synd_ok"] = so
    if want_lv:
        out["L_V"] = lv
    if want_c2v:
        out["c2v"] = cv
    return out


def rp_total(codes) -> int:
    return int(sum(int(h.row_ptr[-1]) - int(h.row_ptr[0]) for h in codes))
