"""The C-ABI library without a GPU: it builds, loads, exports every symbol
include/cg.h declares, and rejects malformed input before touching CUDA."""
import os
import re
import subprocess

import pytest

import fe_inputs as fi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cg.h")


@pytest.fixture(scope="module")
def built():
    import __graft_entry__
    return __graft_entry__._cuda_build_module().build()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:int|void|const char\s*\*)\s*(cg_\w+)\s*\(", text, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["cg_create", "cg_destroy", "cg_spmv", "cg_dot", "cg_axpy", "cg_ewmul", "cg_solve",
                     "cg_last_error"]:
        assert required in names


def test_library_exports_every_declared_symbol(built):
    out = subprocess.run(["nm", "-D", "--defined-only", built], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT\s+(cg_\w+)", out))
    missing = [n for n in declared_functions() if n not in exported]
    assert not missing, missing
    import ctypes
    lib = ctypes.CDLL(built)
    for n in declared_functions():
        assert hasattr(lib, n)


def test_header_compiles_as_c(tmp_path):
    c = tmp_path / "t.c"
    c.write_text('#include "cg.h"\nint main(void){cg_opts o; cg_opts_default(&o); return o.validate == 1 ? 0 : 1;}\n')
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-fsyntax-only", f"-I{os.path.dirname(HEADER)}", str(c)],
                   check=True)


def _bad(kind):
    A = fi.laplace7(3)
    rp, ci, va = A.row_ptr.copy(), A.col_idx.copy(), A.val.copy()
    if kind == "col_range":
        ci[4] = A.n
    elif kind == "col_negative":
        ci[0] = -1
    elif kind == "row_ptr_decreasing":
        rp[5], rp[6] = rp[6], rp[5]
    elif kind == "row_ptr_start":
        rp = rp + 1
    elif kind == "nnz_mismatch":
        rp[-1] -= 1
    return rp, ci, va, A.n


@pytest.mark.parametrize("kind", ["col_range", "col_negative", "row_ptr_decreasing", "row_ptr_start",
                                  "nnz_mismatch"])
def test_malformed_csr_rejected_without_gpu(built, kind):
    import paper_2112_10823_gb300 as cg
    rp, ci, va, n = _bad(kind)
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(rp, ci, va, n=n, nnz=len(ci))
    assert e.value.status == cg.CG_EINVAL
    assert "invalid CSR" in str(e.value)


def test_bad_arguments_rejected(built):
    import paper_2112_10823_gb300 as cg
    A = fi.laplace7(2)
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(A.row_ptr, A.col_idx, A.val, index_base=2)
    assert e.value.status == cg.CG_EINVAL
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(A.row_ptr, A.col_idx, A.val, precision=7)
    assert e.value.status == cg.CG_EINVAL
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(A.row_ptr, A.col_idx, A.val, preconditioner=7)
    assert e.value.status == cg.CG_EINVAL
    with pytest.raises(cg.CGError) as e:
        cg.Batch(precision=7)
    assert e.value.status == cg.CG_EINVAL
    # one-based input validated as one-based
    B = fi.to_one_based(A)
    with pytest.raises(cg.CGError):
        cg.cg_create(B.row_ptr, B.col_idx, B.val, index_base=0)


def test_no_gpu_fails_loudly(built):
    """Without a usable GPU a valid matrix is refused with CG_ECUDA: there is no CPU path."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2112_10823_gb300 as cg
    A = fi.laplace7(3)
    with pytest.raises(cg.CGError) as e:
        cg.cg_create(A.row_ptr, A.col_idx, A.val)
    assert e.value.status in (cg.CG_ECUDA, cg.CG_ENOMEM)


def test_batch_without_gpu_fails_loudly(built):
    """The batched interface has no CPU path either."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import paper_2112_10823_gb300 as cg
    with pytest.raises(cg.CGError) as e:
        cg.Batch()
    assert e.value.status in (cg.CG_ECUDA, cg.CG_ENOMEM)


def test_null_handle_queries_rejected(built):
    """The handle queries refuse a NULL handle with CG_EINVAL (no GPU involved)."""
    import ctypes
    import paper_2112_10823_gb300 as cg
    lib = cg.lib
    i32, i64 = ctypes.c_int32(0), ctypes.c_int64(0)
    assert lib.cg_info(None, ctypes.byref(i64), None, None) == cg.CG_EINVAL
    assert lib.cg_partition_info(None, ctypes.byref(i32), ctypes.byref(i32)) == cg.CG_EINVAL
    assert b"NULL handle" in lib.cg_last_error(None)
    assert lib.cg_selftest_wait_timeout(0, ctypes.byref(i32)) == cg.CG_EINVAL
    d = ctypes.c_double(0.0)
    assert lib.cg_dot_host(-1, None, None, ctypes.byref(d), None) == cg.CG_EINVAL
    assert lib.cg_dot_host(5, None, None, ctypes.byref(d), None) == cg.CG_EINVAL
    assert lib.cg_dot(3, None, None, None, None) == cg.CG_EINVAL
    assert lib.cg_axpy(-2, 1.0, None, None, None) == cg.CG_EINVAL
    assert lib.cg_ewmul(4, None, None, None, None) == cg.CG_EINVAL
    assert lib.cg_probe_fp64_peak(0, None) == cg.CG_EINVAL
    assert lib.cg_blas_release() == cg.CG_OK
