"""The benchmark's reference arm (the oracle timed on the host) and its JSON
line, on CPU: the contract keys a driver reads, for a small workload; and the
launcher that starts one rank per GPU when `--gpus N` is given without
torchrun (exercised here with the CPU-only reference arm and gloo)."""
import json
import os
import subprocess
import sys


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _json_lines(out):
    return [json.loads(ln) for ln in out.splitlines() if ln.strip().startswith("{")]


def test_reference_arm_prints_one_contract_line():
    import oracle
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--matrix", "lap7",
                          "--grid", "8", "--steps", "2", "--warmup", "1"],
                         capture_output=True, text=True, check=True, cwd=ROOT, timeout=600).stdout
    lines = _json_lines(out)
    assert len(lines) == 1, out
    d = lines[0]
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["value"] > 0
    assert d["steps"] == 2 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["config"]["n"] == 8 ** 3 and d["solve"]["iters"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"
    assert d["cpu_baseline"]["cores"] == (oracle.omp_threads() if oracle.omp_available() else 1)
    assert d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
    assert abs(d["ms_per_step"] - 1000.0 / d["value"]) <= 1e-6 * d["ms_per_step"]
    # the workload keys are the GPU arm's for the same command line
    import bench
    args = bench.parse(["--matrix", "lap7", "--grid", "8"])
    assert d["config"] == bench.common_config(args, 8 ** 3, d["config"]["nnz"], 1)


def test_launch_ranks_starts_n_gloo_ranks(tmp_path):
    """launch_ranks runs a script as N torchrun ranks that meet in a process group."""
    import bench
    script = tmp_path / "rank.py"
    script.write_text(
        "import os, sys, torch, torch.distributed as dist\n"
        "dist.init_process_group('gloo')\n"
        "r, w = dist.get_rank(), dist.get_world_size()\n"
        "t = torch.tensor([r + 1])\n"
        "dist.all_reduce(t)\n"
        "open(os.path.join(sys.argv[1], f'rank{r}.txt'), 'w').write(f'{r} {w} {int(t)} {os.environ[\"LOCAL_RANK\"]}')\n"
        "dist.destroy_process_group()\n")
    assert bench.launch_ranks(3, str(script), [str(tmp_path)]) == 0
    got = sorted((tmp_path / f"rank{r}.txt").read_text().split() for r in range(3))
    assert got == [[str(r), "3", "6", str(r)] for r in range(3)]
    cmd = bench.torchrun_command(8, "bench.py", ["--gpus", "8"], 29500)
    assert "--nproc-per-node=8" in cmd and "127.0.0.1" in cmd and cmd[-3:] == ["bench.py", "--gpus", "8"]


def test_gpus_flag_without_torchrun_starts_the_ranks():
    """`bench.py --gpus 2` outside torchrun re-runs itself as two ranks; rank 0
    alone prints the (reference arm's) line, with n_gpus = 2."""
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--gpus", "2", "--impl", "reference",
                          "--matrix", "lap7", "--grid", "6", "--steps", "1", "--warmup", "1"],
                         capture_output=True, text=True, cwd=ROOT, timeout=600, env=env)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = _json_lines(out.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2, out.stdout
