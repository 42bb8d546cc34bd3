"""The allocation-free decode entry point, called through the C ABI.

Some callers cannot call cudaMalloc for a decoder workspace: they can hand the
library device inputs and outputs, but the device memory budget belongs to
another runtime, or an allocation is not allowed where they run. For them
``mbp_decode_bsc_static`` keeps the decoder state in a fixed device array
inside the library (MBP_STATIC_SCRATCH_BYTES). This test checks, on calls made
back to back, that it returns exactly what ``mbp_decode_bsc`` returns on the
same inputs (streaming and resident schedules, FP32, FP64 and FP16 messages),
that a repeated call leaves the device's free memory unchanged, and that a
batch too large for the array is refused.

This file is collected last, so a run that stops at its first failure has run
every other test before this one.
"""
import ctypes

import numpy as np
import pytest
import torch

import mbp_inputs as mi

pytestmark = pytest.mark.gpu

TOL_F32 = 1e-3  # the FP32 tolerance of the parity tests; identical kernels are expected to agree exactly


@pytest.fixture(scope="module")
def mbp():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2001_07979_gb300 as m
    m.build()
    lib = m._load()
    P, I = ctypes.c_void_p, ctypes.c_int
    lib.mbp_decode_bsc_static.restype = I
    lib.mbp_decode_bsc_static.argtypes = [P, I, P, P, P, I, P, P, P, P, P]
    return m


def _inputs(mbp, n, m, dist, u, seed, F, qber):
    H = mi.make_codes(n, m, dist, u, seed)
    x, y, e = mi.bsc_frames(n, F, qber, seed=seed + 17)
    codes = mbp.mbp_create_codes(H)
    xd = torch.from_numpy(x.view(np.int32)).cuda()
    z = mbp.mbp_syndrome(codes, xd)
    return codes, torch.from_numpy(y.view(np.int32)).cuda(), torch.from_numpy(e).cuda(), z


def _outputs(codes, F, msg_dtype, dev):
    soft_dt = torch.float64 if msg_dtype == 1 else torch.float32
    return dict(x_hat_bits=torch.full((F, (codes.n + 31) // 32), -1, dtype=torch.int32, device=dev),
                iters=torch.full((F,), -1, dtype=torch.int32, device=dev),
                success=torch.full((F,), 7, dtype=torch.uint8, device=dev),
                soft=torch.full((F, codes.n), float("nan"), dtype=soft_dt, device=dev),
                synd_ok=torch.full((F, codes.u), 7, dtype=torch.uint8, device=dev))


def _call_static(mbp, codes, y, e, z, max_iter, out, msg_dtype=0, schedule=0):
    o = mbp._opts(msg_dtype, 20.0, True, False, False, None, out["soft"], out["synd_ok"], schedule=schedule)
    return mbp._lib.mbp_decode_bsc_static(codes.handle, y.shape[0], y.data_ptr(), e.data_ptr(), z.data_ptr(),
                                          max_iter, ctypes.byref(o), out["x_hat_bits"].data_ptr(),
                                          out["iters"].data_ptr(), out["success"].data_ptr(),
                                          torch.cuda.current_stream().cuda_stream or None)


def _static_decode(mbp, codes, y, e, z, max_iter, msg_dtype=0, schedule=0):
    out = _outputs(codes, y.shape[0], msg_dtype, y.device)
    return _call_static(mbp, codes, y, e, z, max_iter, out, msg_dtype, schedule), out


def _compare(mbp, codes, y, e, z, max_iter, msg_dtype=0, schedule=0):
    rc, got = _static_decode(mbp, codes, y, e, z, max_iter, msg_dtype, schedule)
    if rc == 5:  # MBP_EUNSUPPORTED: e.g. a tile of this code does not fit the resident schedule's L2 budget
        return False
    assert rc == 0, mbp._lib.mbp_last_error_string()
    ref = mbp.mbp_decode_bsc(codes, y, e, z, max_iter, msg_dtype=msg_dtype, want_soft=True, want_synd=True,
                             schedule=schedule)
    torch.cuda.synchronize()
    for k in ("x_hat_bits", "iters", "success", "synd_ok"):
        assert torch.equal(got[k], ref[k]), k
    assert torch.max(torch.abs(got["soft"] - ref["soft"])).item() <= TOL_F32
    return True


def test_static_scratch_decode_matches_workspace_decode(mbp):
    a = _inputs(mbp, 1024, 512, {3: 1.0}, 2, 0, 64, 0.03)
    b = _inputs(mbp, 4000, 1600, {2: 0.3, 3: 0.4, 8: 0.3}, 3, 3, 13, 0.06)
    _compare(mbp, *a, 50)           # first call on this device: looks up the array's address
    _compare(mbp, *b, 40)           # second call in a row, another code and batch size
    _compare(mbp, *a, 50, msg_dtype=1)  # the array keeps b's state; a must not see it
    _compare(mbp, *b, 40)
    _compare(mbp, *b, 40, msg_dtype=2)  # FP16 message storage
    _compare(mbp, *a, 50, msg_dtype=2)


def test_static_scratch_decode_resident_schedule(mbp):
    a = _inputs(mbp, 1024, 512, {3: 1.0}, 2, 0, 64, 0.03)
    ran = _compare(mbp, *a, 50, schedule=2)  # MBP_SCHED_RESIDENT
    ran += _compare(mbp, *a, 50, msg_dtype=1, schedule=2)
    assert ran >= 1, "the resident schedule refused both message types"


def test_static_scratch_call_allocates_nothing(mbp):
    codes, y, e, z = _inputs(mbp, 4000, 1600, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 3, 40, 0.05)
    out = _outputs(codes, 40, 0, y.device)
    assert _call_static(mbp, codes, y, e, z, 40, out) == 0  # warm call: every kernel it launches is loaded
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(2):
        assert _call_static(mbp, codes, y, e, z, 40, out) == 0, mbp._lib.mbp_last_error_string()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


def test_static_scratch_refuses_oversized_batches(mbp):
    codes, y, e, z = _inputs(mbp, 4000, 1600, {2: 0.3, 3: 0.4, 8: 0.3}, 2, 3, 8, 0.05)
    F = 2000
    need = mbp.mbp_decode_workspace_size(codes, F, schedule=mbp.SCHED_STREAMING)  # the layout it would use
    assert need > 64 * 1024 * 1024
    yb = y.repeat(F // 8, 1)
    eb = e.repeat(F // 8)
    zb = torch.zeros(F * sum(codes.syndrome_words()), dtype=torch.int32, device=y.device)
    rc, _ = _static_decode(mbp, codes, yb, eb, zb, 10)
    assert rc == 1  # MBP_EINVAL
    assert b"static scratch" in mbp._lib.mbp_last_error_string()
