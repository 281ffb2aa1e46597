"""Plant plausible mistakes in copies of the oracle and check that the pins
catch every one of them (CPU only; the oracle's own source is not touched)."""
import os
import subprocess
import sys

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
    ("cg_direction_drops_beta",
     "beta_h[k - 1] = beta;\n        for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];",
     "beta_h[k - 1] = beta;\n        for (int64_t i = 0; i < n; ++i) p[i] = r[i];"),
    ("cg_alpha_uses_old_gamma_sign", "double alpha = rho / gamma;\n        for (int64_t i = 0; i < n; ++i) x[i] = x[i] + alpha * p[i];\n        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];\n        double rho_new = oracle_dot(n, r, r);\n        k = k + 1;\n        if (alpha_h",
     "double alpha = rho / gamma;\n        for (int64_t i = 0; i < n; ++i) x[i] = x[i] - alpha * p[i];\n        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];\n        double rho_new = oracle_dot(n, r, r);\n        k = k + 1;\n        if (alpha_h"),
    ("cg_stop_test_squared",
     "if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        double beta",
     "if (force_iters < 0 && rho_new <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        double beta"),
    ("mixed_never_replaces", "int replace = (replace_every > 0 && k % replace_every == 0) || sqrt(rho_new) <= tol * bnorm;",
     "int replace = 0; if (sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }"),
    ("mixed_beta_from_true_residual",
     "            if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        }",
     "            if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n"
     "            beta = rho_new / rho;\n        }"),
    ("mixed_forced_run_stops_at_tolerance",
     "            if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        }",
     "            if (sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        }"),
    ("mixed_forced_one_extra_step",
     "int64_t limit = force_iters >= 0 ? force_iters : maxit;\n    while (!done && k < limit) {\n        for (int64_t i = 0; i < n; ++i) p32[i]",
     "int64_t limit = force_iters >= 0 ? force_iters + 1 : maxit;\n    while (!done && k < limit) {\n        for (int64_t i = 0; i < n; ++i) p32[i]"),
    ("mixed_replacement_schedule_offset", "k % replace_every == 0", "k % replace_every == 1"),
    ("spmv_rows_row_is_list_position", "int64_t i = rows[t];", "int64_t i = t;"),
    ("spmv_rows_ignores_base", "s = s + AA[k] * x[JA[k] - base];\n        y_sel[t] = s;",
     "s = s + AA[k] * x[JA[k]];\n        y_sel[t] = s;"),
    ("pcg_no_preconditioner", "oracle_ewmul(n, dinv, r, z);\n        double rho_new = oracle_dot(n, r, z);",
     "for (int64_t i = 0; i < n; ++i) z[i] = r[i];\n        double rho_new = oracle_dot(n, r, z);"),
    ("pcg_rho_uses_r_r", "double rho_new = oracle_dot(n, r, z);", "double rho_new = oracle_dot(n, r, r);"),
    ("pcg_direction_from_r", "for (int64_t i = 0; i < n; ++i) p[i] = z[i] + beta * p[i];",
     "for (int64_t i = 0; i < n; ++i) p[i] = r[i] + beta * p[i];"),
    ("jacobi_diag_from_first_entry", "if ((int64_t)JA[k] - base == i) d = d + AA[k];",
     "if (k == (int64_t)IA[i] - base) d = d + AA[k];"),
    ("stats_bandwidth_off_by_one", "int64_t d = (int64_t)(JA[k] - base) - i;", "int64_t d = (int64_t)(JA[k] - base) - i + 1;"),
    ("cg_true_residual_sign",
     "    for (int64_t i = 0; i < n; ++i) { double d = b[i] - q[i]; t = t + d * d; }\n"
     "    *relres_true = sqrt(t) / bnorm;\n    free(r); free(p); free(q);\n    return status;",
     "    for (int64_t i = 0; i < n; ++i) { double d = b[i] + q[i]; t = t + d * d; }\n"
     "    *relres_true = sqrt(t) / bnorm;\n    free(r); free(p); free(q);\n    return status;"),
    ("cg_ignores_initial_guess",
     "for (int64_t i = 0; i < n; ++i) { r[i] = b[i] - q[i]; p[i] = r[i]; }\n"
     "    double rho = oracle_dot(n, r, r);\n    if (res_h && hist_len > 0) res_h[0] = sqrt(rho);",
     "for (int64_t i = 0; i < n; ++i) { r[i] = b[i]; p[i] = r[i]; }\n"
     "    double rho = oracle_dot(n, r, r);\n    if (res_h && hist_len > 0) res_h[0] = sqrt(rho);"),
    ("pcg_setup_rho_uses_r_r", "double rho = oracle_dot(n, r, z);\n    double rr = oracle_dot(n, r, r);",
     "double rho = oracle_dot(n, r, r);\n    double rr = oracle_dot(n, r, r);"),
    ("pcg_stop_test_on_z", "rr = oracle_dot(n, r, r);\n        k = k + 1;\n        if (force_iters < 0 && sqrt(rr) <= tol * bnorm) { done = 1; break; }",
     "rr = oracle_dot(n, z, z);\n        k = k + 1;\n        if (force_iters < 0 && sqrt(rr) <= tol * bnorm) { done = 1; break; }"),
    ("mixed_fp32_product_summed_in_fp64", "float s = 0.0f;\n        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)\n            s = s + AA32[k] * x32[JA[k] - base];",
     "double s = 0.0;\n        for (int64_t k = (int64_t)IA[i] - base; k < (int64_t)IA[i + 1] - base; ++k)\n            s = s + (double)AA32[k] * (double)x32[JA[k] - base];"),
]


# Mistakes planted in the OpenMP timing variant (cg_oracle_omp.c).
OMP_SRC = os.path.join(os.path.dirname(oracle.__file__), "cg_oracle_omp.c")
OMP_MUTANTS = [
    ("omp_dot_drops_last_block", "for (int t = 0; t < T; ++t) s = s + part[t];",
     "for (int t = 0; t + 1 < T; ++t) s = s + part[t];"),
    ("omp_blocks_overlap", "*hi = (n * (t + 1)) / T;", "*hi = (n * (t + 1)) / T + (t + 1 < T);"),
    ("omp_spmv_drops_last_entry", "k < (int64_t)IA[i + 1] - base; ++k)", "k < (int64_t)IA[i + 1] - base - 1; ++k)"),
    ("omp_beta_inverted", "{ rho = rho_new; done = 1; break; }\n        double beta = rho_new / rho;",
     "{ rho = rho_new; done = 1; break; }\n        double beta = rho / rho_new;"),
    ("omp_x_update_sign", "x[i] = x[i] + alpha * p[i];\n#pragma omp parallel for schedule(static)\n        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];\n        double rho_new = omp_dot(n, r, r, part, T);\n        k = k + 1;",
     "x[i] = x[i] - alpha * p[i];\n#pragma omp parallel for schedule(static)\n        for (int64_t i = 0; i < n; ++i) r[i] = r[i] - alpha * q[i];\n        double rho_new = omp_dot(n, r, r, part, T);\n        k = k + 1;"),
    ("omp_true_residual_sign", "    for (int64_t i = 0; i < n; ++i) q[i] = b[i] - q[i];\n    *relres_true = sqrt(omp_dot(n, q, q, part, T)) / bnorm;\n    free(r); free(p); free(q); free(part);",
     "    for (int64_t i = 0; i < n; ++i) q[i] = b[i] + q[i];\n    *relres_true = sqrt(omp_dot(n, q, q, part, T)) / bnorm;\n    free(r); free(p); free(q); free(part);"),
    ("omp_mixed_replacement_offset", "k % replace_every == 0", "k % replace_every == 1"),
    ("omp_mixed_fp32_sum_in_fp64", "float s = 0.0f;", "double s = 0.0;"),
    ("omp_mixed_forced_run_stops", "if (force_iters < 0 && sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        }",
     "if (sqrt(rho_new) <= tol * bnorm) { rho = rho_new; done = 1; break; }\n        }"),
]


@pytest.fixture(scope="module")
def src_text():
    with open(SRC) as f:
        return f.read()


# Runs every pin against one compiled mutant and prints the names of the pins
# that failed.  It runs in a child process: a mutant may also read out of
# bounds and crash, which counts as caught.
_CHILD = r"""
import sys
sys.path[:0] = [sys.argv[2], sys.argv[3]]
import oracle, pins
caught = []
with oracle.using(sys.argv[1]):
    for pin in pins.ALL_PINS:
        try:
            pin()
        except (AssertionError, FloatingPointError, ValueError, IndexError, OverflowError):
            caught.append(pin.__name__)
print("CAUGHT " + " ".join(caught))
"""

_CHILD_OMP = _CHILD.replace("oracle.using(sys.argv[1])", "oracle.using_omp(sys.argv[1])")


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_mutant(name, old, new, src_text, tmp_path):
    assert src_text.count(old) == 1, f"mutation site for {name} not unique/found"
    mutated = src_text.replace(old, new)
    c = tmp_path / "mut.c"
    c.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11",
                           "-o", str(so), str(c), "-lm"])
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", _CHILD, str(so), root, os.path.join(root, "tests")],
                         capture_output=True, text=True, timeout=600)
    if res.returncode < 0:  # killed by a signal: the mutant crashed on a pin's input
        return
    assert res.returncode == 0, res.stderr[-2000:]
    line = [ln for ln in res.stdout.splitlines() if ln.startswith("CAUGHT")][-1]
    assert line.split()[1:], f"no pin caught mutant {name}"


@pytest.mark.parametrize("name,old,new", OMP_MUTANTS, ids=[m[0] for m in OMP_MUTANTS])
def test_pins_catch_omp_mutant(name, old, new, tmp_path):
    import oracle as orc
    if not orc.omp_available():
        pytest.skip("no OpenMP on this host compiler")
    with open(OMP_SRC) as f:
        text = f.read()
    assert text.count(old) == 1, f"mutation site for {name} not unique/found"
    c = tmp_path / "mut_omp.c"
    c.write_text(text.replace(old, new))
    so = tmp_path / "libmut_omp.so"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-std=c11",
                           "-o", str(so), str(c), "-lm"])
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    res = subprocess.run([sys.executable, "-c", _CHILD_OMP, str(so), root, os.path.join(root, "tests")],
                         capture_output=True, text=True, timeout=600)
    if res.returncode < 0:
        return
    assert res.returncode == 0, res.stderr[-2000:]
    line = [ln for ln in res.stdout.splitlines() if ln.startswith("CAUGHT")][-1]
    assert "pin_omp_variant" in line.split()[1:], f"the OpenMP pin did not catch mutant {name}"
