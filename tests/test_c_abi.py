"""The C-ABI used from plain C: tests/c/abi_solve.c compiled against the
public header and linked to the library, run as its own process."""
import os
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _compile(tmp_path):
    from paper_2405_18966_gb300 import build
    lib = build.build()
    exe = tmp_path / "abi_solve"
    subprocess.run(["gcc", "-std=c99", "-O1", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c", "abi_solve.c"), "-o", str(exe), lib,
                    "-Wl,-rpath," + os.path.dirname(lib), "-lm"], check=True)
    return exe


def test_c_program_compiles_and_links(tmp_path):
    assert _compile(tmp_path).exists()


@pytest.mark.gpu
def test_c_program_solves(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    exe = _compile(tmp_path)
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stdout + r.stderr
    assert "OK (0 problems)" in r.stdout
