"""The C-ABI library builds for sm_103a, loads, exports every declared symbol,
and rejects malformed input on the host (no GPU needed for any of this)."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2001_07979_gb300 as mbp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADERS = [os.path.join(ROOT, "include", f) for f in os.listdir(os.path.join(ROOT, "include")) if f.endswith(".h")]


def declared_functions():
    names = set()
    for h in HEADERS:
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(mbp_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    path = mbp.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("mbp_create_codes", "mbp_destroy_codes", "mbp_syndrome", "mbp_bsc_llr",
                     "mbp_decode_workspace_size", "mbp_decode_batch", "mbp_decode_bsc", "mbp_decode_bsc_host",
                     "mbp_export_c2v", "mbp_last_error_string", "mbp_default_opts"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def _csr_array(mats):
    arr = (mbp._Csr * len(mats))()
    keep = []
    for l, (n, m, rp, ci) in enumerate(mats):
        rp = np.ascontiguousarray(rp, np.int32)
        ci = np.ascontiguousarray(ci, np.int32)
        keep += [rp, ci]
        arr[l] = mbp._Csr(n, m, int(rp[-1]), rp.ctypes.data, ci.ctypes.data if ci.size else None)
    return arr, keep


@pytest.mark.parametrize("case", ["col_out_of_range", "repeated_col", "bad_row_ptr", "n_mismatch", "u_zero",
                                  "nnz_mismatch"])
def test_create_codes_rejects_malformed(lib, case):
    mbp._load()
    rp, ci = [0, 2, 4], [0, 1, 1, 2]
    mats = [(3, 2, rp, ci), (3, 2, rp, ci)]
    u = 2
    if case == "col_out_of_range":
        mats[1] = (3, 2, rp, [0, 1, 1, 3])
    elif case == "repeated_col":
        mats[0] = (3, 2, rp, [0, 0, 1, 2])
    elif case == "bad_row_ptr":
        mats[0] = (3, 2, [0, 3, 2], [0, 1, 2, 2])
    elif case == "n_mismatch":
        mats[1] = (4, 2, rp, ci)
    elif case == "u_zero":
        u = 0
    arr, keep = _csr_array(mats)
    if case == "nnz_mismatch":
        arr[0].nnz = 3
    out = ctypes.c_void_p(123)
    rc = mbp._lib.mbp_create_codes(ctypes.addressof(arr), u, ctypes.byref(out))
    assert rc == 1  # MBP_EINVAL
    assert out.value is None
    assert mbp._lib.mbp_last_error_string()


def test_create_codes_rejects_long_rows(lib):
    mbp._load()
    n = 100
    arr, keep = _csr_array([(n, 1, [0, 65], list(range(65)))])
    out = ctypes.c_void_p()
    assert mbp._lib.mbp_create_codes(ctypes.addressof(arr), 1, ctypes.byref(out)) == 5  # MBP_EUNSUPPORTED


def test_null_arguments_are_rejected(lib):
    mbp._load()
    L = mbp._lib
    assert L.mbp_create_codes(None, 2, None) == 1
    assert L.mbp_syndrome(None, None, 1, None, None) == 1
    assert L.mbp_decode_batch(None, 1, None, None, 10, None, None, None, None, None) == 1
    assert L.mbp_decode_workspace_size(None, 1, None, None) == 1
    assert L.mbp_destroy_codes(None) == 0
    o = mbp._Opts()
    L.mbp_default_opts(ctypes.byref(o))
    assert o.msg_dtype == 0 and o.early_exit == 1 and o.l_max == 20.0


def test_python_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    monkeypatch.setattr(mbp, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(mbp, "_lib", None)
    with pytest.raises(mbp.MBPError):
        mbp.mbp_version()
