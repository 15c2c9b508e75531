"""The k smallest singular triplets with the same machinery (the projected
matrix's Ritz values approximate both ends of the spectrum, Sec. 2): the
restart keeps the k smallest Ritz triplets instead of the k largest.

Pins of the oracle: a closed-form spectrum with separated small values (exact
singular values and vectors of A = H diag(s) G^T), and LAPACK's SVD of the
2,000 x 1,000 sparse matrix (a library routine, used only here as a check).
GPU tests hold the CUDA path to the same answers and to the oracle.
"""
import numpy as np
import pytest

import synth


def _sin_angles(X, Y):
    c = np.sum(X * Y, axis=0)
    return np.linalg.norm(Y - X * c, axis=0)


def _separated():
    s = np.linspace(2.0, 1.0, 200)
    s[-5:] = [0.3, 0.2, 0.1, 0.05, 0.01]
    return synth.dense_prescribed(300, 200, s, 11)


def _exact_smallest(d, k):
    order = np.argsort(d.s, kind="stable")[:k]
    E1 = np.zeros((d.m, k))
    E2 = np.zeros((d.n, k))
    E1[order, np.arange(k)] = 1.0
    E2[order, np.arange(k)] = 1.0
    return (d.s[order], synth.apply_reflectors(d.left_reflectors, E1),
            synth.apply_reflectors(d.right_reflectors, E2))


# ------------------------------------------------------------------ CPU pins

@pytest.mark.parametrize("k,p", [(5, 25), (3, 30)])
def test_oracle_smallest_closed_form(orc, k, p):
    d = _separated()
    r = orc.svds(d.a, k, p, 1e-10, 500, which="smallest", v0=synth.start_vector(200, 1))
    assert r["info"]["converged"] == 1
    s_ex, Q1, Q2 = _exact_smallest(d, k)
    np.testing.assert_allclose(r["S"], s_ex, rtol=0, atol=1e-13)
    assert np.all(np.diff(r["S"]) > 0)                       # ascending
    assert np.all(_sin_angles(r["U"], Q1) < 1e-9)
    assert np.all(_sin_angles(r["V"], Q2) < 1e-9)
    # Eq. (4) residual equals the true one: ||A^T u - sigma v|| <= tol sigma
    assert np.all(np.linalg.norm(d.a.T @ r["U"] - r["V"] * r["S"], axis=0) <= 1e-10 * r["S"] + 1e-13)


def test_oracle_smallest_sparse_vs_lapack(orc):
    a = synth.workload_sparse_small()
    s = np.linalg.svd(a.to_dense(), compute_uv=False)
    r = orc.svds(a, 5, 45, 1e-10, 2000, which="smallest", v0=synth.start_vector(a.n, 1))
    assert r["info"]["converged"] == 1 and r["info"]["restarts"] > 0
    np.testing.assert_allclose(r["S"], np.sort(s)[:5], rtol=1e-12)


def test_oracle_smallest_needs_tall(orc):
    a = np.random.default_rng(0).standard_normal((40, 60))
    with pytest.raises(ValueError):
        orc.svds(a, 2, 10, 1e-10, 10, which="smallest")


def test_oracle_largest_unchanged_by_the_option(orc):
    d = _separated()
    v0 = synth.start_vector(200, 1)
    r1 = orc.svds(d.a, 5, 25, 1e-10, 100, v0=v0)
    r2 = orc.svds(d.a, 5, 25, 1e-10, 100, v0=v0, which="largest")
    assert np.array_equal(r1["S"], r2["S"]) and np.array_equal(r1["U"], r2["U"])
    np.testing.assert_allclose(r1["S"], d.s[:5], rtol=0, atol=1e-13)


# ------------------------------------------------------------------ GPU

@pytest.fixture(scope="module")
def pkg():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_18966_gb300 as p
    from paper_2405_18966_gb300 import build
    build.build()
    return p


@pytest.mark.gpu
@pytest.mark.parametrize("gemm", ["tensor", "fma"])
def test_gpu_smallest_closed_form(pkg, orc, gemm):
    d = _separated()
    v0 = synth.start_vector(200, 1)
    r = pkg.svds(d.a, 5, 25, 1e-10, 500, v0=v0, which="smallest", restart_gemm=gemm)
    ref = orc.svds(d.a, 5, 25, 1e-10, 500, v0=v0, which="smallest")
    assert r.info["converged"] == 1
    assert abs(r.info["restarts"] - ref["info"]["restarts"]) <= 1
    s_ex, Q1, Q2 = _exact_smallest(d, 5)
    np.testing.assert_allclose(r.S, s_ex, rtol=0, atol=1e-13)
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-10)
    assert np.all(_sin_angles(r.U, Q1) < 1e-9)
    assert np.all(_sin_angles(r.V, Q2) < 1e-9)
    assert np.all(r.res < 1e-10)


@pytest.mark.gpu
def test_gpu_smallest_sparse_vs_oracle(pkg, orc):
    a = synth.workload_sparse_small()
    v0 = synth.start_vector(a.n, 1)
    r = pkg.svds(a, 5, 45, 1e-10, 2000, v0=v0, which="smallest")
    ref = orc.svds(a, 5, 45, 1e-10, 2000, v0=v0, which="smallest")
    assert r.info["converged"] == 1
    assert abs(r.info["restarts"] - ref["info"]["restarts"]) <= 2
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-10)
    # smallest values of a random matrix are clustered (gaps ~1e-2): Wedin bound
    assert np.all(_sin_angles(r.V, ref["V"]) < 1e-7)
    assert np.all(_sin_angles(r.U, ref["U"]) < 1e-7)


@pytest.mark.gpu
def test_gpu_smallest_rejects_wide(pkg):
    a = np.random.default_rng(0).standard_normal((40, 60))
    with pytest.raises(pkg.SvdscError):
        pkg.Solver(a, which="smallest")
