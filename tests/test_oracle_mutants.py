"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one of them (CPU only; the oracle's own source is not touched)."""
import os
import shutil
import subprocess
import tempfile

import pytest

import oracle
import pins

SRC = os.path.join(os.path.dirname(oracle.__file__), "cg_oracle.c")

# (name, exact text in cg_oracle.c, replacement)
MUTANTS = [
    ("spmv_transposed_index", "s = s + AA[k] * x[JA[k] - base];\n        y[i] = s;",
     "s = s + AA[k] * x[i];\n        y[i] = s;"),
    ("spmv_drops_last_entry", "for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)\n            s = s + AA[k] * x[JA[k] - base];\n        y[i] = s;",
     "for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base - 1; ++k)\n            s = s + AA[k] * x[JA[k] - base];\n        y[i] = s;"),
    ("spmv_ignores_base", "s = s + AA[k] * x[JA[k] - base];\n        y[i] = s;",
     "s = s + AA[k] * x[JA[k]];\n        y[i] = s;"),
    ("dot_skips_first", "for (int64_t i = 0; i < n; ++i) s = s + x[i] * y[i];",
     "for (int64_t i = 1; i < n; ++i) s = s + x[i] * y[i];"),
    ("axpy_wrong_operand", "y[i] = a * x[i] + y[i];", "y[i] = a * y[i] + x[i];"),
    ("ewmul_adds", "z[i] = x[i] * y[i];", "z[i] = x[i] + y[i];"),
    ("cg_residual_sign", "for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];\n        double rho_new = oracle_dot(n, r, r);\n        k = k + 1;\n        if (alpha_h",
     "for (int64_t i = 0; i < n; ++i) r[i] = r[i] + alpha * q[i];\n        double rho_new = oracle_dot(n, r, r);\n        k = k + 1;\n        if (alpha_h"),
    ("cg_beta_inverted", "double beta = rho_new / rho;\n        if (beta_h",
     "double beta = rho / rho_new;\n        if (beta_h"),
    ("cg_direction_drops_beta", "for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];\n        rho = rho_new;\n    }\n    *iters = k;\n    *relres_rec = sqrt(rho) / bnorm;\n    if (status == ORC_OK && force_iters",
     "for (int64_t i = 0; i < n; ++i) p[i] = r[i];\n        rho = rho_new;\n    }\n    *iters = k;\n    *relres_rec = sqrt(rho) / bnorm;\n    if (status == ORC_OK && force_iters"),
    ("cg_alpha_uses_old_gamma_sign", "double alpha = rho / gamma;\n        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];\n        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];\n        double rho_new = oracle_dot(n, r, r);\n        k = k + 1;\n        if (alpha_h",
     "double alpha = rho / gamma;\n        for (int64_t i = 0; i < n; ++i) x[i] = x[i] - alpha * p[i];\n        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];\n        double rho_new = oracle_dot(n, r, r);\n        k = k + 1;\n        if (alpha_h"),
    ("cg_stop_test_squared", "if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm)",
     "if (force_iters < 0 && rho_new <= tol * bnorm)"),
    ("mixed_never_replaces", "int replace = (replace_every > 0 && k % replace_every == 0) || sqrt(rho_new) <= tol * bnorm;",
     "int replace = 0; if (sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }"),
    ("mixed_beta_from_true_residual",
     "            if (sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        }",
     "            if (sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n            beta = rho_new / rho;\n        }"),
    ("pcg_no_preconditioner", "oracle_ewmul(n, dinv, r, z);\n        double rho_new = oracle_dot(n, r, z);",
     "for (int64_t i = 0; i < n; ++i) z[i] = r[i];\n        double rho_new = oracle_dot(n, r, z);"),
    ("pcg_rho_uses_r_r", "double rho_new = oracle_dot(n, r, z);", "double rho_new = oracle_dot(n, r, r);"),
    ("pcg_direction_from_r", "for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];",
     "for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];"),
    ("jacobi_diag_from_first_entry", "if ((int64_t)JA[k] - base == i) d = d + AA[k];",
     "if (k == (int64_t)IA[i] - base) d = d + AA[k];"),
    ("stats_bandwidth_off_by_one", "int64_t d = (int64_t)(JA[k] - base) - i;", "int64_t d = (int64_t)(JA[k] - base) - i + 1;"),
]


@pytest.fixture(scope="module")
def src_text():
    with open(SRC) as f:
        return f.read()


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, src_text, tmp_path):
    assert src_text.count(old) == 1, f"mutation site for {name} not unique/found"
    mutated = src_text.replace(old, new)
    c = tmp_path / "mut.c"
    c.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", str(so), str(c), "-lm"])
    caught = []
    with oracle.using(str(so)):
        for pin in pins.ALL_PINS:
            try:
                pin()
            except (AssertionError, FloatingPointError, ValueError, IndexError, OverflowError) as e:
                caught.append(pin.__name__)
    assert caught, f"no pin caught mutant {name}"
