"""GB300 multi-matrix belief-propagation (MBP) reconciliation — Python binding.

A thin ctypes layer over ``libmbp.so`` (the C ABI in ``include/mbp.h``). It
marshals arguments only: every step of decoding runs in the library's CUDA
kernels. PyTorch provides device memory and streams. There is no CPU fallback:
if the library is not built, every entry point raises.

Function names follow the C ABI (``mbp_create_codes``, ``mbp_syndrome``,
``mbp_bsc_llr``, ``mbp_decode_batch``, ``mbp_decode_bsc``,
``mbp_decode_bsc_host``, ``mbp_export_c2v``, ``mbp_decode_multi``,
``mbp_autotune_multi``, ...). Bit vectors are int32
tensors holding the packed uint32 words of the ABI (bit i of a frame in word
i >> 5 at position i & 31).
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np
import torch

from ._build import LIB, build, up_to_date

__all__ = [
    "build", "library_path", "MBPError", "Codes", "MSG_F32", "MSG_F64", "MSG_F16", "MSG_BF16", "ACC_AUTO", "ACC_FLOAT", "ACC_FIXED",
    "SCHED_AUTO", "SCHED_STREAMING", "SCHED_RESIDENT", "SCHED_GRAPH", "RULE_SUM_PRODUCT", "RULE_MIN_SUM",
    "UPDATE_FLOODING", "UPDATE_MATRIX_SERIAL",
    "mbp_create_codes", "mbp_destroy_codes", "mbp_syndrome", "mbp_bsc_llr", "mbp_decode_workspace_size",
    "mbp_decode_batch", "mbp_decode_bsc", "mbp_decode_bsc_host", "mbp_export_c2v", "mbp_version",
    "split_syndromes", "join_syndromes", "mbp_profile_enable", "mbp_profile_get", "KERNEL_FAMILIES",
    "mbp_multi_workspace_size", "mbp_decode_multi", "mbp_autotune_multi", "mbp_release_cached",
    "mbp_multi_set_tuning",
    "mbp_nbp_workspace_size", "mbp_nbp_forward", "mbp_nbp_backward", "NormalizedBP", "NBPDecoder",
]

MSG_F32, MSG_F64, MSG_F16, MSG_BF16 = 0, 1, 2, 3
ACC_AUTO, ACC_FLOAT, ACC_FIXED = 0, 1, 2
SCHED_AUTO, SCHED_STREAMING, SCHED_RESIDENT, SCHED_GRAPH = 0, 1, 2, 3
RULE_SUM_PRODUCT, RULE_MIN_SUM = 0, 1
UPDATE_FLOODING, UPDATE_MATRIX_SERIAL = 0, 1
_STATUS = {0: "MBP_OK", 1: "MBP_EINVAL", 2: "MBP_ENOMEM", 3: "MBP_ECUDA", 4: "MBP_ETIMEOUT", 5: "MBP_EUNSUPPORTED"}


class MBPError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class _Csr(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("m", ctypes.c_int32), ("nnz", ctypes.c_int32),
                ("row_ptr", ctypes.c_void_p), ("col_idx", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("msg_dtype", ctypes.c_int32), ("early_exit", ctypes.c_int32), ("validate", ctypes.c_int32),
                ("host_io", ctypes.c_int32), ("l_max", ctypes.c_double), ("workspace", ctypes.c_void_p),
                ("workspace_bytes", ctypes.c_size_t), ("soft_out", ctypes.c_void_p), ("synd_ok", ctypes.c_void_p),
                ("accumulate", ctypes.c_int32), ("schedule", ctypes.c_int32), ("rule", ctypes.c_int32),
                ("update", ctypes.c_int32)]


class _Group(ctypes.Structure):
    _fields_ = [("codes", ctypes.c_void_p), ("F", ctypes.c_int32), ("llr", ctypes.c_void_p),
                ("y_bits", ctypes.c_void_p), ("qber", ctypes.c_void_p), ("z_bits", ctypes.c_void_p),
                ("x_hat_bits", ctypes.c_void_p), ("iters", ctypes.c_void_p), ("success", ctypes.c_void_p),
                ("synd_ok", ctypes.c_void_p), ("soft_out", ctypes.c_void_p)]


class _Tuning(ctypes.Structure):
    _fields_ = [("grid_kernels", ctypes.c_int32), ("cn_warps", ctypes.c_int32), ("cn_waves", ctypes.c_int32), ("vn_warps", ctypes.c_int32),
                ("syn_warps", ctypes.c_int32), ("ms", ctypes.c_double)]


_lock = threading.Lock()
_lib = None


def library_path() -> str:
    return LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(LIB):
            raise MBPError(3, f"{LIB} is not built; call paper_2001_07979_gb300.build() (needs nvcc)")
        lib = ctypes.CDLL(LIB)
        P, I, I64, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_size_t
        sig = {
            "mbp_last_error_string": (ctypes.c_char_p, []),
            "mbp_version": (I, []),
            "mbp_default_opts": (None, [P]),
            "mbp_create_codes": (I, [P, I, P]),
            "mbp_destroy_codes": (I, [P]),
            "mbp_codes_info": (I, [P, P, P, P, P, P]),
            "mbp_syndrome": (I, [P, P, I, P, P]),
            "mbp_bsc_llr": (I, [P, P, I, I, I, P, P]),
            "mbp_decode_workspace_size": (I, [P, I, P, P]),
            "mbp_decode_batch": (I, [P, I, P, P, I, P, P, P, P, P]),
            "mbp_decode_bsc": (I, [P, I, P, P, P, I, P, P, P, P, P]),
            "mbp_decode_bsc_host": (I, [P, I, P, P, P, I, P, P, P, P, P]),
            "mbp_decode_bsc_host_async": (I, [P, I, P, P, P, I, P, P, P, P, P]),
            "mbp_export_c2v": (I, [P, I, P, I, P, P]),
            "mbp_multi_workspace_size": (I, [P, I, P, P]),
            "mbp_decode_multi": (I, [P, I, I, P, P]),
            "mbp_autotune_multi": (I, [P, I, I, P, P, P]),
            "mbp_release_cached": (I, []),
            "mbp_multi_set_tuning": (I, [P, I, P, P]),
            "mbp_nbp_workspace_size": (I, [P, I, I, P]),
            "mbp_nbp_forward": (I, [P, I, I, P, P, P, P, ctypes.c_double, P, S, P, P]),
            "mbp_nbp_backward": (I, [P, I, I, P, P, ctypes.c_double, P, P, S, P, P, P, P]),
            "mbp_profile_enable": (I, [I]),
            "mbp_profile_get": (I, [I, P, P]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        del I64, S
        _lib = lib
        return lib


def _check(rc: int):
    if rc != 0:
        msg = _load().mbp_last_error_string().decode(errors="replace")
        raise MBPError(rc, msg)


def mbp_version() -> int:
    return _load().mbp_version()


def _stream_ptr(stream) -> int | None:
    if stream is None:
        stream = torch.cuda.current_stream()
    return stream.cuda_stream or None


def _ptr(t):
    if t is None:
        return None
    if isinstance(t, torch.Tensor):
        return t.data_ptr()
    if isinstance(t, np.ndarray):
        return t.ctypes.data
    raise TypeError(type(t))


def _words(nbits: int) -> int:
    return (nbits + 31) // 32


class Codes:
    """Handle of u matrices uploaded with ``mbp_create_codes``."""

    def __init__(self, handle: int, n: int, m: list[int], edges: int, max_deg: int):
        self._h = handle
        self.n, self.m, self.u, self.edges, self.max_check_degree = n, m, len(m), edges, max_deg

    @property
    def handle(self) -> int:
        if not self._h:
            raise MBPError(1, "codes handle was destroyed")
        return self._h

    def syndrome_words(self) -> list[int]:
        return [_words(ml) for ml in self.m]

    def destroy(self):
        if self._h:
            h, self._h = self._h, None
            _check(_load().mbp_destroy_codes(h))

    def __del__(self):
        try:
            if self._h and _lib is not None:
                _lib.mbp_destroy_codes(self._h)
                self._h = None
        except Exception:
            pass


def mbp_create_codes(matrices) -> Codes:
    """Upload u CSR matrices (objects with n, m, row_ptr, col_idx) to the current device."""
    lib = _load()
    u = len(matrices)
    keep, arr = [], (_Csr * max(u, 1))()
    for l, h in enumerate(matrices):
        rp = np.ascontiguousarray(h.row_ptr, dtype=np.int32)
        ci = np.ascontiguousarray(h.col_idx, dtype=np.int32)
        keep += [rp, ci]
        arr[l] = _Csr(int(h.n), int(h.m), int(rp[-1]) if rp.size else 0, rp.ctypes.data,
                      ci.ctypes.data if ci.size else None)
    out = ctypes.c_void_p()
    _check(lib.mbp_create_codes(ctypes.addressof(arr), u, ctypes.byref(out)))
    n = ctypes.c_int32()
    e = ctypes.c_int64()
    d = ctypes.c_int32()
    _check(lib.mbp_codes_info(out, None, ctypes.byref(n), None, ctypes.byref(e), ctypes.byref(d)))
    return Codes(out.value, n.value, [int(h.m) for h in matrices], e.value, d.value)


def mbp_destroy_codes(codes: Codes):
    codes.destroy()


def mbp_syndrome(codes: Codes, x_bits: torch.Tensor, stream=None) -> torch.Tensor:
    """eq. (1) on the device: x_bits int32 [F, ceil(n/32)] -> z int32 [sum_l F*ceil(m_l/32)] ([u][F][W_l])."""
    x = x_bits.contiguous()
    F = x.shape[0]
    z = torch.empty(F * sum(codes.syndrome_words()), dtype=torch.int32, device=x.device)
    _check(_load().mbp_syndrome(codes.handle, _ptr(x), F, _ptr(z), _stream_ptr(stream)))
    return z


def split_syndromes(codes: Codes, z_flat, F: int):
    """Flat [u][F][W_l] syndromes -> list of u arrays/tensors [F, W_l]."""
    out, off = [], 0
    for w in codes.syndrome_words():
        out.append(z_flat[off:off + F * w].reshape(F, w))
        off += F * w
    return out


def join_syndromes(parts):
    if isinstance(parts[0], torch.Tensor):
        return torch.cat([p.reshape(-1) for p in parts]).contiguous()
    return np.ascontiguousarray(np.concatenate([np.asarray(p).reshape(-1) for p in parts]))


def mbp_bsc_llr(y_bits: torch.Tensor, qber: torch.Tensor, n: int, dtype=torch.float32, stream=None) -> torch.Tensor:
    """eq. (5) on the device: y_bits int32 [F, W], qber float64 [F] -> LLR [F, n]."""
    y = y_bits.contiguous()
    q = qber.to(torch.float64).contiguous()
    F = y.shape[0]
    code = MSG_F64 if dtype == torch.float64 else MSG_F32
    out = torch.empty((F, n), dtype=torch.float64 if code == MSG_F64 else torch.float32, device=y.device)
    _check(_load().mbp_bsc_llr(_ptr(y), _ptr(q), F, n, code, _ptr(out), _stream_ptr(stream)))
    return out


def _opts(msg_dtype, l_max, early_exit, validate, host_io, workspace=None, soft=None, synd=None,
          accumulate=ACC_AUTO, schedule=SCHED_AUTO, rule=RULE_SUM_PRODUCT, update=UPDATE_FLOODING) -> _Opts:
    o = _Opts()
    _load().mbp_default_opts(ctypes.byref(o))
    o.msg_dtype = msg_dtype
    o.accumulate = int(accumulate)
    o.schedule = int(schedule)
    o.rule = int(rule)
    o.update = int(update)
    o.l_max = float(l_max)
    o.early_exit = int(bool(early_exit))
    o.validate = int(bool(validate))
    o.host_io = int(bool(host_io))
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel()
    o.soft_out = _ptr(soft)
    o.synd_ok = _ptr(synd)
    return o


def mbp_decode_workspace_size(codes: Codes, F: int, msg_dtype: int = MSG_F32, host_io: bool = False,
                              schedule: int = SCHED_AUTO) -> int:
    o = _opts(msg_dtype, 20.0, True, False, host_io, schedule=schedule)
    b = ctypes.c_size_t()
    _check(_load().mbp_decode_workspace_size(codes.handle, F, ctypes.byref(o), ctypes.byref(b)))
    return b.value


def _workspace(codes, F, msg_dtype, host_io, workspace, device, schedule=SCHED_AUTO):
    need = mbp_decode_workspace_size(codes, F, msg_dtype, host_io, schedule)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
    return workspace


def _decode(entry, codes, F, inputs, z_bits, max_iter, msg_dtype, l_max, early_exit, validate, want_soft,
            want_synd, workspace, device, stream, accumulate=ACC_AUTO, schedule=SCHED_AUTO, rule=RULE_SUM_PRODUCT,
            update=UPDATE_FLOODING):
    workspace = _workspace(codes, F, msg_dtype, False, workspace, device, schedule)
    fdt = torch.float64 if msg_dtype == MSG_F64 else torch.float32
    xh = torch.empty((F, _words(codes.n)), dtype=torch.int32, device=device)
    it = torch.empty(F, dtype=torch.int32, device=device)
    ok = torch.empty(F, dtype=torch.uint8, device=device)
    soft = torch.empty((F, codes.n), dtype=fdt, device=device) if want_soft else None
    synd = torch.empty((F, codes.u), dtype=torch.uint8, device=device) if want_synd else None
    o = _opts(msg_dtype, l_max, early_exit, validate, False, workspace, soft, synd, accumulate, schedule, rule, update)
    z = z_bits.contiguous()
    _check(entry(codes.handle, F, *[_ptr(t) for t in inputs], _ptr(z), int(max_iter), ctypes.byref(o),
                 _ptr(xh), _ptr(it), _ptr(ok), _stream_ptr(stream)))
    out = dict(x_hat_bits=xh, iters=it, success=ok, workspace=workspace)
    if want_soft:
        out["soft"] = soft
    if want_synd:
        out["synd_ok"] = synd
    return out


def mbp_decode_batch(codes: Codes, llr: torch.Tensor, z_bits: torch.Tensor, max_iter: int, *, l_max: float = 20.0,
                     early_exit: bool = True, validate: bool = False, want_soft: bool = False,
                     want_synd: bool = False, workspace: torch.Tensor | None = None, stream=None,
                     accumulate: int = ACC_AUTO, schedule: int = SCHED_AUTO, msg_dtype: int | None = None,
                     rule: int = RULE_SUM_PRODUCT, update: int = UPDATE_FLOODING) -> dict:
    """Decode F frames from channel LLRs: float64 LLRs decode with FP64 messages, float32 LLRs with FP32
    messages unless msg_dtype asks for MSG_F16 or MSG_BF16 storage."""
    x = llr.contiguous()
    if x.dtype not in (torch.float32, torch.float64):
        raise TypeError("llr must be float32 or float64")
    msg = MSG_F64 if x.dtype == torch.float64 else (MSG_F32 if msg_dtype is None else msg_dtype)
    if (msg == MSG_F64) != (x.dtype == torch.float64):
        raise TypeError("FP64 messages take float64 LLRs; the other storage types take float32")
    return _decode(_load().mbp_decode_batch, codes, x.shape[0], [x], z_bits, max_iter, msg, l_max, early_exit,
                   validate, want_soft, want_synd, workspace, x.device, stream, accumulate, schedule, rule, update)


def mbp_decode_bsc(codes: Codes, y_bits: torch.Tensor, qber: torch.Tensor, z_bits: torch.Tensor, max_iter: int, *,
                   msg_dtype: int = MSG_F32, l_max: float = 20.0, early_exit: bool = True, want_soft: bool = False,
                   want_synd: bool = False, workspace: torch.Tensor | None = None, stream=None,
                   accumulate: int = ACC_AUTO, schedule: int = SCHED_AUTO, rule: int = RULE_SUM_PRODUCT,
                   update: int = UPDATE_FLOODING) -> dict:
    """Decode F BSC frames from Bob's bits and per-frame QBER (eq. 5 formed on the device)."""
    y = y_bits.contiguous()
    q = qber.to(torch.float64).contiguous()
    return _decode(_load().mbp_decode_bsc, codes, y.shape[0], [y, q], z_bits, max_iter, msg_dtype, l_max,
                   early_exit, False, want_soft, want_synd, workspace, y.device, stream, accumulate, schedule, rule,
                   update)


def mbp_decode_bsc_host(codes: Codes, y_bits: np.ndarray, qber: np.ndarray, z_bits: np.ndarray, max_iter: int, *,
                        msg_dtype: int = MSG_F32, l_max: float = 20.0, early_exit: bool = True,
                        workspace: torch.Tensor | None = None, out: dict | None = None, stream=None,
                        device=None, accumulate: int = ACC_AUTO, schedule: int = SCHED_AUTO,
                        rule: int = RULE_SUM_PRODUCT, update: int = UPDATE_FLOODING, sync: bool = True) -> dict:
    """Host-memory variant: inputs and outputs are numpy arrays (or pinned CPU tensors). sync=False calls
    mbp_decode_bsc_host_async: the call returns once everything is queued on the stream, and the outputs are
    valid (and the inputs free to change) only after the stream has been synchronised."""
    y = y_bits if isinstance(y_bits, torch.Tensor) else np.ascontiguousarray(y_bits, dtype=np.uint32)
    q = qber if isinstance(qber, torch.Tensor) else np.ascontiguousarray(qber, dtype=np.float64)
    z = z_bits if isinstance(z_bits, torch.Tensor) else np.ascontiguousarray(z_bits, dtype=np.uint32)
    F = y.shape[0]
    device = device or torch.device("cuda", torch.cuda.current_device())
    need = mbp_decode_workspace_size(codes, F, msg_dtype, True, schedule)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=device)
    if out is None:
        out = dict(x_hat_bits=np.zeros((F, _words(codes.n)), np.uint32), iters=np.zeros(F, np.int32),
                   success=np.zeros(F, np.uint8))
    o = _opts(msg_dtype, l_max, early_exit, False, True, workspace, accumulate=accumulate, schedule=schedule,
              rule=rule, update=update)
    entry = _load().mbp_decode_bsc_host if sync else _load().mbp_decode_bsc_host_async
    _check(entry(codes.handle, F, _ptr(y), _ptr(q), _ptr(z), int(max_iter), ctypes.byref(o), _ptr(out["x_hat_bits"]),
                 _ptr(out["iters"]), _ptr(out["success"]), _stream_ptr(stream)))
    out["workspace"] = workspace
    return out


def mbp_export_c2v(codes: Codes, F: int, workspace: torch.Tensor, frame: int, msg_dtype: int = MSG_F32,
                   stream=None, schedule: int = SCHED_AUTO) -> torch.Tensor:
    """Check-to-variable messages of one frame after a decode, in stacked CSR edge order."""
    fdt = torch.float64 if msg_dtype == MSG_F64 else torch.float32
    out = torch.empty(codes.edges, dtype=fdt, device=workspace.device)
    o = _opts(msg_dtype, 20.0, True, False, False, workspace, schedule=schedule)
    _check(_load().mbp_export_c2v(codes.handle, F, ctypes.byref(o), int(frame), _ptr(out), _stream_ptr(stream)))
    return out


def _groups(groups, want_soft, want_synd, alloc=True):
    """ctypes array of mbp_group from dicts {codes, z_bits, and llr or (y_bits, qber)}; allocates the outputs."""
    arr = (_Group * max(len(groups), 1))()
    outs, keep = [], []
    for i, g in enumerate(groups):
        codes, F = g["codes"], int(g.get("F", (g["llr"] if "llr" in g else g["y_bits"]).shape[0]))
        o = {}
        if alloc:
            dev = (g["llr"] if "llr" in g else g["y_bits"]).device
            o = dict(x_hat_bits=torch.empty((F, _words(codes.n)), dtype=torch.int32, device=dev),
                     iters=torch.empty(F, dtype=torch.int32, device=dev),
                     success=torch.empty(F, dtype=torch.uint8, device=dev))
            if want_soft:
                o["soft"] = torch.empty((F, codes.n), dtype=torch.float32, device=dev)
            if want_synd:
                o["synd_ok"] = torch.empty((F, codes.u), dtype=torch.uint8, device=dev)
        ins = {k: g[k].contiguous() for k in ("llr", "y_bits", "z_bits") if k in g}
        if "qber" in g:
            ins["qber"] = g["qber"].to(torch.float64).contiguous()
        keep.append(ins)
        arr[i].codes = codes.handle
        arr[i].F = F
        arr[i].llr = _ptr(ins.get("llr"))
        arr[i].y_bits = _ptr(ins.get("y_bits"))
        arr[i].qber = _ptr(ins.get("qber"))
        arr[i].z_bits = _ptr(ins.get("z_bits"))
        arr[i].x_hat_bits = _ptr(o.get("x_hat_bits"))
        arr[i].iters = _ptr(o.get("iters"))
        arr[i].success = _ptr(o.get("success"))
        arr[i].synd_ok = _ptr(o.get("synd_ok"))
        arr[i].soft_out = _ptr(o.get("soft"))
        outs.append(o)
    return arr, outs, keep


def mbp_multi_workspace_size(groups, msg_dtype: int = MSG_F32) -> int:
    arr, _, _ = _groups(groups, False, False, alloc=False)
    o = _opts(msg_dtype, 20.0, True, False, False)
    b = ctypes.c_size_t()
    _check(_load().mbp_multi_workspace_size(arr, len(groups), ctypes.byref(o), ctypes.byref(b)))
    return b.value


def _multi(entry, groups, max_iter, msg_dtype, l_max, early_exit, validate, want_soft, want_synd, workspace,
           stream, extra=()):
    arr, outs, keep = _groups(groups, want_soft, want_synd)
    need = mbp_multi_workspace_size(groups, msg_dtype)
    if workspace is None or workspace.numel() < need:
        dev = outs[0]["iters"].device if outs else torch.device("cuda", torch.cuda.current_device())
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=dev)
    o = _opts(msg_dtype, l_max, early_exit, validate, False, workspace)
    _check(entry(arr, len(groups), int(max_iter), ctypes.byref(o), *extra, _stream_ptr(stream)))
    for out in outs:
        out["workspace"] = workspace
    del keep  # inputs were only read by work already queued on the stream, which owns their memory
    return outs


def mbp_decode_multi(groups, max_iter: int, *, msg_dtype: int = MSG_F32, l_max: float = 20.0,
                     early_exit: bool = True, validate: bool = False, want_soft: bool = False,
                     want_synd: bool = False, workspace: torch.Tensor | None = None, stream=None) -> list:
    """Decode groups of frames of different codes in one call. groups: dicts with "codes", "z_bits" and either
    "llr" (float32 [F][n]) or "y_bits" and "qber". Returns one output dict per group. Asynchronous on the
    stream (the iteration loop is a CUDA graph)."""
    return _multi(_load().mbp_decode_multi, groups, max_iter, msg_dtype, l_max, early_exit, validate, want_soft,
                  want_synd, workspace, stream)


def mbp_autotune_multi(groups, max_iter: int, *, msg_dtype: int = MSG_F32, l_max: float = 20.0,
                       early_exit: bool = True, workspace: torch.Tensor | None = None, stream=None):
    """Pick the launch shapes of mbp_decode_multi for this batch by timing candidates; returns
    (outputs of a decode with the chosen shape, {cn_warps, cn_waves, vn_warps, syn_warps, ms})."""
    best = _Tuning()
    outs = _multi(_load().mbp_autotune_multi, groups, max_iter, msg_dtype, l_max, early_exit, False, False, False,
                  workspace, stream, extra=(ctypes.byref(best),))
    return outs, dict(grid_kernels=best.grid_kernels, cn_warps=best.cn_warps, cn_waves=best.cn_waves, vn_warps=best.vn_warps,
                      syn_warps=best.syn_warps, ms=best.ms)


def mbp_multi_set_tuning(groups, tuning: dict, msg_dtype: int = MSG_F32):
    """Use this launch shape ({grid_kernels, cn_warps, cn_waves, vn_warps, syn_warps}) for later
    mbp_decode_multi calls on these codes and frame counts."""
    arr, _, _ = _groups(groups, False, False, alloc=False)
    o = _opts(msg_dtype, 20.0, True, False, False)
    t = _Tuning(int(tuning.get("grid_kernels", 1)), int(tuning.get("cn_warps", 8)), int(tuning.get("cn_waves", 1)),
                int(tuning.get("vn_warps", 8)), int(tuning.get("syn_warps", 8)), 0.0)
    _check(_load().mbp_multi_set_tuning(arr, len(groups), ctypes.byref(o), ctypes.byref(t)))


def mbp_release_cached():
    """Free the library's cached CUDA graphs and tuned launch shapes."""
    _check(_load().mbp_release_cached())


def mbp_nbp_workspace_size(codes: Codes, F: int, T: int) -> int:
    b = ctypes.c_size_t()
    _check(_load().mbp_nbp_workspace_size(codes.handle, int(F), int(T), ctypes.byref(b)))
    return b.value


def mbp_nbp_forward(codes: Codes, llr: torch.Tensor, z_bits: torch.Tensor, alpha: torch.Tensor,
                    beta: torch.Tensor, *, l_max: float = 20.0, workspace: torch.Tensor | None = None,
                    want_lv: bool = True, stream=None):
    """Unrolled normalised BP: posteriors after each of the T = alpha.shape[0] iterations, [T, F, n] float32
    (or None), and the workspace holding the checkpoints for mbp_nbp_backward."""
    x = llr.contiguous()
    if x.dtype != torch.float32:
        raise TypeError("llr must be float32")
    F, T = x.shape[0], alpha.shape[0]
    a = alpha.detach().to(torch.float32).contiguous()
    b = beta.detach().to(torch.float32).contiguous()
    need = mbp_nbp_workspace_size(codes, F, T)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 256), dtype=torch.uint8, device=x.device)
    lv = torch.empty((T, F, codes.n), dtype=torch.float32, device=x.device) if want_lv else None
    z = z_bits.contiguous()
    _check(_load().mbp_nbp_forward(codes.handle, F, T, _ptr(x), _ptr(z), _ptr(a), _ptr(b), float(l_max),
                                   _ptr(workspace), workspace.numel(), _ptr(lv), _stream_ptr(stream)))
    return lv, workspace


def mbp_nbp_backward(codes: Codes, F: int, alpha: torch.Tensor, beta: torch.Tensor, grad_lv: torch.Tensor,
                     workspace: torch.Tensor, *, l_max: float = 20.0, want_grad_llr: bool = False, stream=None):
    """Gradients of sum(grad_lv * L) with respect to alpha, beta ([T, u] each) and, on request, the LLRs."""
    T = alpha.shape[0]
    a = alpha.detach().to(torch.float32).contiguous()
    b = beta.detach().to(torch.float32).contiguous()
    g = grad_lv.to(torch.float32).contiguous()
    ga = torch.empty_like(a)
    gb = torch.empty_like(b)
    gl = torch.empty((F, codes.n), dtype=torch.float32, device=a.device) if want_grad_llr else None
    _check(_load().mbp_nbp_backward(codes.handle, int(F), T, _ptr(a), _ptr(b), float(l_max), _ptr(g),
                                    _ptr(workspace), workspace.numel(), _ptr(ga), _ptr(gb), _ptr(gl),
                                    _stream_ptr(stream)))
    return ga, gb, gl


class NormalizedBP(torch.autograd.Function):
    """L = NormalizedBP.apply(llr, alpha, beta, codes, z_bits, l_max): posteriors [T, F, n] of the unrolled
    normalised BP; backward runs the library's adjoint kernels (gradients for llr, alpha and beta)."""

    @staticmethod
    def forward(ctx, llr, alpha, beta, codes, z_bits, l_max=20.0):
        lv, ws = mbp_nbp_forward(codes, llr, z_bits, alpha, beta, l_max=l_max)
        ctx.codes, ctx.l_max, ctx.ws, ctx.F = codes, l_max, ws, llr.shape[0]
        ctx.save_for_backward(alpha, beta)
        ctx.llr_grad = llr.requires_grad
        return lv

    @staticmethod
    def backward(ctx, grad_lv):
        alpha, beta = ctx.saved_tensors
        ga, gb, gl = mbp_nbp_backward(ctx.codes, ctx.F, alpha, beta, grad_lv, ctx.ws, l_max=ctx.l_max,
                                      want_grad_llr=ctx.llr_grad)
        return gl, ga.to(alpha.dtype), gb.to(beta.dtype), None, None, None


class NBPDecoder(torch.nn.Module):
    """T unrolled iterations over the u matrices of `codes` with learnable scale alpha[t][l] (initially 1)
    and offset beta[t][l] (initially 0): plain BP at initialisation."""

    def __init__(self, codes: Codes, T: int, l_max: float = 20.0, device=None):
        super().__init__()
        self.codes, self.l_max = codes, l_max
        self.alpha = torch.nn.Parameter(torch.ones((T, codes.u), dtype=torch.float32, device=device))
        self.beta = torch.nn.Parameter(torch.zeros((T, codes.u), dtype=torch.float32, device=device))

    def forward(self, llr: torch.Tensor, z_bits: torch.Tensor) -> torch.Tensor:
        return NormalizedBP.apply(llr, self.alpha, self.beta, self.codes, z_bits, self.l_max)


KERNEL_FAMILIES = ("check", "variable", "syndrome", "retire", "setup", "output", "persistent", "check_rows")


def mbp_profile_enable(on: bool = True):
    """Start (and clear) or stop per-kernel CUDA-event accounting of this thread's decode calls."""
    _check(_load().mbp_profile_enable(int(bool(on))))


def mbp_profile_get() -> dict:
    """{family: (launches, milliseconds)} accumulated since mbp_profile_enable(True)."""
    out = {}
    for k, name in enumerate(KERNEL_FAMILIES):
        n = ctypes.c_int64()
        ms = ctypes.c_double()
        _check(_load().mbp_profile_get(k, ctypes.byref(n), ctypes.byref(ms)))
        out[name] = (n.value, ms.value)
    return out
