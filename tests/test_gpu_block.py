"""Block form on the GPU (block Lanczos bidiagonalization, b = 2, 4, 8, 16)
against the oracle's block form on the same start block: Ritz values of the
first pass, converged singular values (1e-10 relative, the FP64 requirement),
singular vectors (sin-angle 1e-8), restart and product counts; the mixed
block form within 1e-6; closed forms; a value of multiplicity b found b times;
a rank-deficient matrix (the column-by-column repair of a flagged block)."""
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


def _sin(X, Y):
    c = np.sum(X * Y, axis=0)
    return np.linalg.norm(Y - X * c, axis=0)


def _start_block(n, b, seed=100):
    return np.column_stack([synth.start_vector(n, seed + l) for l in range(b)])


def _dense_as_csr(a):
    m, n = a.shape
    rows, cols = np.nonzero(a)
    rp = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=rp[1:])
    return synth.CSR(m, n, rp, cols.astype(np.int32), np.ascontiguousarray(a[rows, cols]))


@pytest.mark.parametrize("b", [2, 4, 8])
def test_block_first_pass_matches_oracle(pkg, orc, b):
    """maxit = 1: the Ritz values of the first block Lanczos pass with the same start block."""
    a = synth.workload_sparse_small()
    V0 = _start_block(a.n, b)
    r = pkg.svds(a, 10, 10, 1e-10, 1, v0=V0, block=b)
    ref = orc.svds_block(a, 10, 10, b, 1e-10, 1, V0=V0)
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-11)
    np.testing.assert_allclose(r.res, ref["res"], rtol=1e-6, atol=1e-14)
    np.testing.assert_allclose(r.info["beta_t"], ref["info"]["beta_t"], rtol=1e-9)
    assert r.info["t"] == ref["t_last"]
    assert r.info["n_matvec"] == ref["info"]["n_matvec"]


@pytest.mark.parametrize("b,k,p", [(2, 10, 10), (4, 10, 10), (8, 10, 10), (16, 10, 22)])
def test_block_solve_matches_oracle(pkg, orc, b, k, p):
    """Converged block solves: sigma to 1e-10 relative, vectors to sin-angle 1e-8,
    restarts within one of the oracle's, the block product count."""
    a = synth.workload_sparse_small()
    V0 = _start_block(a.n, b)
    ref = orc.svds_block(a, k, p, b, 1e-10, 2000, V0=V0)
    r = pkg.svds(a, k, p, 1e-10, 2000, v0=V0, block=b)
    assert r.status == pkg.OK and r.info["converged"] == 1 and ref["info"]["converged"] == 1
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-10)
    assert np.all(_sin(r.U, ref["U"]) < 1e-8)
    assert np.all(_sin(r.V, ref["V"]) < 1e-8)
    assert abs(r.info["restarts"] - ref["info"]["restarts"]) <= 1
    t0, t1 = orc.block_sizes(k, p, b)
    assert r.info["n_matvec"] == 2 * t0 + 2 * r.info["restarts"] * (t1 - k)
    assert np.abs(r.U.T @ r.U - np.eye(k)).max() < 1e-12
    assert np.abs(r.V.T @ r.V - np.eye(k)).max() < 1e-12
    idx = np.argmax(np.abs(r.V), axis=0)
    assert np.all(r.V[idx, np.arange(k)] > 0)


def test_block_closed_form(pkg):
    """A = Q1 diag(s) Q2^T (as CSR): exact singular values and vectors."""
    s = np.linspace(2.0, 1.0, 200) ** 3
    d = synth.dense_prescribed(300, 200, s, 11)
    Q1 = synth.apply_reflectors(d.left_reflectors, np.eye(300)[:, :8])
    Q2 = synth.apply_reflectors(d.right_reflectors, np.eye(200)[:, :8])
    r = pkg.svds(_dense_as_csr(d.a), 8, 12, 1e-12, 400, block=4, seed=2)
    assert r.info["converged"] == 1
    np.testing.assert_allclose(r.S, s[:8], rtol=1e-12)
    assert np.all(_sin(r.U, Q1) < 1e-9) and np.all(_sin(r.V, Q2) < 1e-9)


def test_block_finds_every_copy_of_a_repeated_value(pkg):
    """sigma = 3 with multiplicity 4 and b = 4: all four copies, spanning the eigenspace."""
    s = np.r_[3.0, 3.0, 3.0, 3.0, 2.0, 1.9, 0.9 ** np.arange(194)]
    d = synth.dense_prescribed(300, 200, s, 21)
    Q1 = synth.apply_reflectors(d.left_reflectors, np.eye(300)[:, :4])
    r = pkg.svds(_dense_as_csr(d.a), 6, 10, 1e-12, 400, block=4, seed=5)
    assert r.info["converged"] == 1
    np.testing.assert_allclose(r.S, s[:6], rtol=1e-12)
    assert np.linalg.norm(r.U[:, :4] - Q1 @ (Q1.T @ r.U[:, :4])) < 1e-9


def test_block_rank_deficient_repair(pkg, orc):
    """Rank 2 with b = 4: the first U block is numerically rank 2; the flagged
    block is orthonormalized column by column (zero diagonal entries, random
    replacements), as in the oracle."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((90, 2))
    y = rng.standard_normal((70, 2))
    a = x @ np.diag([5.0, 2.0]) @ y.T
    sv = np.linalg.svd(a, compute_uv=False)
    r = pkg.svds(_dense_as_csr(a), 3, 9, 1e-10, 20, block=4, seed=6)
    assert r.status in (pkg.OK, pkg.NOT_CONVERGED)
    assert r.info["breakdowns"] >= 2
    np.testing.assert_allclose(r.S[:2], sv[:2], rtol=1e-12)
    assert r.S[2] < 1e-12 * sv[0]
    assert np.abs(a @ r.V[:, :2] - r.U[:, :2] * r.S[:2]).max() < 1e-12 * sv[0]
    ref = orc.svds_block(a, 3, 9, 4, 1e-10, 20, seed=6)
    np.testing.assert_allclose(r.S[:2], ref["S"][:2], rtol=1e-12)


@pytest.mark.parametrize("b", [4, 8])
def test_block_mixed_vs_fp64_oracle(pkg, orc, b):
    """Mixed block form on the FP32-exact 2,000 x 1,000 matrix: sigma within 1e-6 of
    the FP64 block oracle's."""
    a = synth.workload_sparse_small_fp32()
    V0 = _start_block(a.n, b)
    ref = orc.svds_block(a, 10, 10, b, 1e-10, 2000, V0=V0)
    a32 = synth.CSR(a.m, a.n, a.row_ptr, a.col_idx, a.values.astype(np.float32))
    r = pkg.svds(a32, 10, 10, 1e-10, 2000, precision="mixed", v0=V0, block=b)
    assert r.info["converged"] == 1
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-6)


def test_block_zipf_sample_vs_oracle(pkg, orc):
    """The Zipf workload at 2 % scale (20,000 x 10,000, long rows in the warp and
    CTA bins of the block product), b = 8: first-pass Ritz values against the oracle."""
    a = synth.workload_sparse_zipf(0.02)
    V0 = _start_block(a.n, 8)
    r = pkg.svds(a, 40, 40, 1e-10, 1, v0=V0, block=8)
    ref = orc.svds_block(a, 40, 40, 8, 1e-10, 1, V0=V0)
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-11)


def test_block_limits(pkg):
    a = synth.workload_sparse_small()
    with pytest.raises(pkg.SvdscError):
        pkg.Solver(a, block=3)
    with pytest.raises(pkg.SvdscError):
        pkg.Solver(a, block=4, which="smallest")
    with pytest.raises(pkg.SvdscError) as e:
        pkg.svds(a, 10, 0, 1e-10, 10, block=4)  # p = 0: t1 = k < k + b
    assert e.value.status == pkg.ERR_SIZE
