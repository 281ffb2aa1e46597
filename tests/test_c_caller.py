"""The library from a plain C99 program (tests/c_caller.c), host buffers only:
it compiles and links against libcg.so on any machine, and on a GPU it
solves one system through a handle and three through the batch API."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "tests", "c_caller.c")
LIB_DIR = os.path.join(ROOT, "paper_2112_10823_gb300", "_build")


def _build(tmp_path):
    lib = os.path.join(LIB_DIR, "libcg.so")
    if not os.path.exists(lib):
        import paper_2112_10823_gb300.build as b
        b.build()
    exe = tmp_path / "c_caller"
    subprocess.run(["gcc", "-std=c99", "-O2", "-Wall", "-Werror", f"-I{os.path.join(ROOT, 'include')}", SRC,
                    "-o", str(exe), f"-L{LIB_DIR}", "-lcg", f"-Wl,-rpath,{LIB_DIR}", "-lm"], check=True)
    return exe


def test_c_caller_builds(tmp_path):
    assert os.access(_build(tmp_path), os.X_OK)


@pytest.mark.gpu
def test_c_caller_runs(tmp_path):
    exe = _build(tmp_path)
    res = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert "c caller ok" in res.stdout, res.stdout
