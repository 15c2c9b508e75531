"""Writes the stored expected values under tests/golden/.

Every value here comes from the oracle's brute-force one-sided Jacobi dense
SVD (oracle.jacobi_svd) applied to a seeded synthetic input; nothing comes from
the CUDA solver.  Run:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
import synth   # noqa: E402


def sparse_2000x1000():
    a = synth.workload_sparse_small()
    _, s, _, sweeps = oracle.jacobi_svd(a.to_dense())
    assert sweeps > 0, "Jacobi did not converge"
    path = os.path.join(HERE, "sparse_2000x1000_jacobi_sigma.txt")
    with open(path, "w") as f:
        f.write("# Singular values 1..40 (descending) of the seeded 2,000 x 1,000 CSR\n")
        f.write("# matrix synth.workload_sparse_small() (1 % uniform density, N(0,1)),\n")
        f.write("# by brute-force one-sided Jacobi on the dense matrix (oracle.jacobi_svd,\n")
        f.write(f"# {sweeps} sweeps).  Pins the rank-k problem of Eq. (1), Sec. 2.1.\n")
        for v in s[:40]:
            f.write(f"{v:.17e}\n")
    print("wrote", path)


def small_fp32_exact():
    a = synth.workload_sparse_small_fp32()
    _, s, _, sweeps = oracle.jacobi_svd(a.to_dense())
    assert sweeps > 0
    path = os.path.join(HERE, "sparse_2000x1000_fp32exact_jacobi_sigma.txt")
    with open(path, "w") as f:
        f.write("# Singular values 1..120 (descending) of synth.workload_sparse_small_fp32()\n")
        f.write("# (the 2,000 x 1,000 matrix with values rounded to FP32), by brute-force\n")
        f.write(f"# one-sided Jacobi (oracle.jacobi_svd, {sweeps} sweeps).  Eq. (1), Sec. 2.1.\n")
        for v in s[:120]:
            f.write(f"{v:.17e}\n")
    print("wrote", path)


if __name__ == "__main__":
    oracle.build()
    oracle.set_threads(os.cpu_count() or 1)
    sparse_2000x1000()
    small_fp32_exact()
