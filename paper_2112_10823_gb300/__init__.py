"""GB300-native conjugate gradient for sparse SPD finite-element systems.

The hot path of "Fast and Green Computing with Graphics Processing Units for
solving Sparse Linear Systems" — the CSR matrix-vector product, dot product,
vector addition, element-wise product and the classical CG solver built from
them — as hand-written sm_103a CUDA kernels behind a C ABI (``include/cg.h``,
``_build/libcg.so``).  This package is its thin Python binding: argument
marshalling only.  Importing it fails if the library is not built.
"""
from ._binding import (  # noqa: F401
    CG_EBREAKDOWN, CG_EBUSY, CG_ECUDA, CG_EINVAL, CG_ENOMEM, CG_ENOTCONV, CG_ETIMEOUT, CG_OK,
    CG_PREC_FP64, CG_PREC_MIXED, CG_PRECOND_JACOBI, CG_PRECOND_NONE, CG_SOLVE_KERNEL_CLUSTER,
    CG_SOLVE_KERNEL_LARGE_SHARE, CG_SOLVE_KERNEL_SMALL_SHARE, LIB_PATH, Batch, BatchResult, CGError, Handle, Request, SolveResult, cg_axpy,
    cg_create,
    cg_blas_release, cg_destroy, cg_dot, cg_dot_host, cg_dot_noalloc, cg_ewmul, cg_probe_fp64_peak,
    cg_probe_group_sync, cg_selftest_wait_timeout, cg_solve, cg_spmv, last_error, lib,
)
