"""bench.py host logic on the CPU: the reference arm (the CPU oracle) as one
process and as two gloo ranks launched like the multi-GPU bench (rank 0 prints
the single JSON line, the other rank exits 0 without work)."""
import json
import os
import socket
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


ARGS = ["--impl", "reference", "--scale", "0.01", "--steps", "1", "--warmup", "0", "--ref-budget", "0.5",
        "--ref-restarts", "2"]


def _json_lines(out):
    return [json.loads(l) for l in out.splitlines() if l.startswith("{")]


def test_reference_arm_single_process():
    r = subprocess.run([sys.executable, "bench.py", *ARGS], cwd=ROOT, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr
    lines = _json_lines(r.stdout)
    assert len(lines) == 1
    d = lines[0]
    assert d["impl"] == "reference" and d["higher_is_better"] is False and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert d["e2e"]["h2d_bytes_per_step"] == 0
    # the same config object the GPU arm prints for this workload
    for key in ("workload", "m", "n", "k", "p", "tol", "precision", "nnz", "l2", "maxit", "reorth",
                "parallelism"):
        assert key in d["config"], key
    assert d["config"]["parallelism"] == "single-gpu" and d["config"]["reorth"] == "full"


def test_reference_arm_two_gloo_ranks():
    env = dict(os.environ, CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), "bench.py", "--gpus", "2", *ARGS]
    r = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=900, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = _json_lines(r.stdout)
    assert len(lines) == 1 and lines[0]["n_gpus"] == 2


def test_dist_helpers_gloo_two_ranks(tmp_path):
    """barrier and the max-over-ranks reduction bench.py uses, on two gloo ranks."""
    script = tmp_path / "w.py"
    script.write_text(
        "import os, sys\n"
        f"sys.path.insert(0, {ROOT!r})\n"
        "import torch.distributed as dist\n"
        "import bench\n"
        "dist.init_process_group('gloo', init_method='env://')\n"
        "r = dist.get_rank()\n"
        "bench.barrier(2)\n"
        "m = bench.allreduce_max(float(r + 1), 2)\n"
        "assert m == 2.0, m\n"
        "print('ok', r, m)\n"
        "dist.destroy_process_group()\n")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()), str(script)]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    assert r.stdout.count("ok") == 2
