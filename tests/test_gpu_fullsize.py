"""Parity at the benchmark sizes, in the launch configuration bench.py times.

The oracle cannot run these solves to completion in test time, so the checks
are (a) sampled outputs the oracle computes one by one (products with A and
A^T of returned vectors, by the oracle's own CSR loops), (b) properties that
hold at any size (orthonormality, ordering, the Eq. (4) residual bound), (c) a
closed form (the dense workload's exact singular values), and (d) the first
Lanczos pass (maxit = 1, same start vector) against the oracle's."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_18966_gb300 as p
    from paper_2405_18966_gb300 import build
    build.build()
    return p


@pytest.fixture(scope="module")
def zipf():
    return synth.workload_sparse_zipf(1.0)


def test_zipf_full_size_solution_properties(pkg, orc, zipf):
    """1,000,000 x 500,000 Zipf CSR, k = p = 100, tol = 1e-10, FP64 (the bench workload)."""
    A = zipf
    v0 = synth.start_vector(A.n, 1)
    r = pkg.svds(A, 100, 100, 1e-10, 1000, v0=v0)
    assert r.status == pkg.OK and r.info["converged"] == 1
    S, U, V = r.S, r.U, r.V
    assert np.all(np.diff(S) <= 0) and S[-1] > 0
    # orthonormality (Gram matrices in FP64 on the host)
    assert np.abs(U.T @ U - np.eye(100)).max() < 1e-12
    assert np.abs(V.T @ V - np.eye(100)).max() < 1e-12
    # sampled triplets: A v_j = sigma_j u_j (Prop. 1) and the Eq. (4) residual, by the oracle's loops
    for j in (0, 1, 37, 98, 99):
        Av = orc.matvec(A, V[:, j])
        assert np.linalg.norm(Av - S[j] * U[:, j]) <= 1e-11 * S[0]
        Atu = orc.matvec_t(A, U[:, j])
        assert np.linalg.norm(Atu - S[j] * V[:, j]) / S[j] <= 2e-10
    # the largest singular value dominates every row norm (a property of any A)
    rn = np.sqrt(np.add.reduceat(A.values ** 2, A.row_ptr[:-1])[np.diff(A.row_ptr) > 0])
    assert S[0] >= rn.max() * (1 - 1e-12)


def test_zipf_full_size_first_pass_matches_oracle(pkg, orc, zipf):
    """maxit = 1: the Ritz values of the initial LBP(A, t+1) with the same v_1."""
    A = zipf
    v0 = synth.start_vector(A.n, 1)
    r = pkg.svds(A, 100, 100, 1e-10, 1, v0=v0)
    ref = orc.svds(A, 100, 100, 1e-10, 1, v0=v0)
    assert r.status == pkg.NOT_CONVERGED or r.info["converged"] == ref["info"]["converged"]
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-11)
    np.testing.assert_allclose(r.info["beta_t"], ref["info"]["beta_t"], rtol=1e-9)


def test_dense_full_size_exact_sigma(pkg):
    """50,000 x 5,000 dense Q1 diag(0.95^i) Q2^T, k = p = 50, tol = 1e-12."""
    d = synth.workload_dense(1.0)
    r = pkg.svds(d.a, 50, 50, 1e-12, 1000, seed=3)
    assert r.info["converged"] == 1
    np.testing.assert_allclose(r.S, d.s[:50], rtol=1e-12)
    Q2 = synth.apply_reflectors(d.right_reflectors, np.eye(d.n)[:, :5])
    c = np.sum(r.V[:, :5] * Q2, axis=0)
    assert np.all(np.linalg.norm(Q2 - r.V[:, :5] * c, axis=0) < 1e-9)


def test_mixed_k100_sigma_errors_reported_per_triplet(pkg, orc):
    """Mixed form on the FP32-exact 2,000 x 1,000 matrix, k = 100: every sigma and
    every vector against the FP64 oracle."""
    a = synth.workload_sparse_small_fp32()
    v0 = synth.start_vector(a.n, 4)
    ref = orc.svds(a, 100, 100, 1e-10, 100, v0=v0)
    a32 = synth.CSR(a.m, a.n, a.row_ptr, a.col_idx, a.values.astype(np.float32))
    r = pkg.svds(a32, 100, 100, 1e-10, 100, precision="mixed", v0=v0)
    rel = np.abs(r.S - ref["S"]) / ref["S"]
    assert rel.max() <= 1e-6
    # vectors: sin(angle) within (perturbation size) / (gap to the neighbours),
    # for the first 95 (the gaps of the last ones to the unreturned sigma_101.. are unknown)
    s = ref["S"]
    gaps = np.minimum(np.r_[np.inf, s[:-1] - s[1:]], np.r_[s[:-1] - s[1:], np.inf])[:95]
    c = np.sum(r.V[:, :95] * ref["V"][:, :95], axis=0)
    sin = np.linalg.norm(ref["V"][:, :95] - r.V[:, :95] * c, axis=0)
    assert np.all(sin <= 1e-6 * s[0] / np.maximum(gaps, 1e-12) + 1e-7), (sin / (s[0] / gaps)).max()


def test_batch_full_size_sampled(pkg, orc):
    """The 256-matrix batch (one persistent launch): all converge; five matrices
    sampled across the batch's sizes (the smallest, the quartiles and the
    largest by nonzeros) against the FP64 oracle: sigma within 1e-6, every
    vector within its gap-scaled angle, every triplet's residual."""
    from test_gpu_batched import check_vs_oracle
    items = synth.workload_batch()
    b = pkg.Batch([it.a for it in items], [it.k for it in items], seed=1)
    out = b.solve(1e-10, 1000)
    assert sum(i["converged"] for i in out["infos"]) == len(items)
    by_nnz = sorted(range(len(items)), key=lambda i: items[i].a.nnz)
    sample = [by_nnz[int(q * (len(items) - 1))] for q in (0.0, 0.25, 0.5, 0.75, 1.0)]
    for i in sample:
        it = items[i]
        check_vs_oracle(orc, it.a, it.k, out["S"][i], out["U"][i], out["V"][i])
    b.close()
