"""Pins of the oracle's block form (block Lanczos bidiagonalization with full
re-orthogonalization and augmented restart, block size b) against facts fixed
by the paper's single-vector method and by mathematics:

- b = 1 is the single-vector Alg. 2 itself (bit for bit, the pinned oracle);
- closed forms Q1 diag(s) Q2^T (exact singular values and vectors), and the
  brute-force Jacobi singular values of the 2,000 x 1,000 workload;
- the block Lanczos relations A V = U T and A^T U = V T^T + V_res F^T E^T
  (T upper triangular with bandwidth b), orthonormal bases;
- the block form of the Eq. (4) residual, ||F^T Uh(t-b:t, j)||, equal to the
  true residual ||A^T u_j - sigma_j v_j||;
- the product count of Eq. (8) with blocks;
- a singular value of multiplicity 3 found three times with b = 3 (a block
  Krylov space holds up to b copies), and a rank-deficient matrix (block
  breakdown: a zero diagonal entry and a random replacement column).
No value here comes from the CUDA solver."""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _sin(X, Y):
    c = np.sum(X * Y, axis=0)
    return np.linalg.norm(Y - X * c, axis=0)


def _closed_form(m, n, s, seed):
    d = synth.dense_prescribed(m, n, np.asarray(s, dtype=np.float64), seed)
    Q1 = synth.apply_reflectors(d.left_reflectors, np.eye(m)[:, :n])
    Q2 = synth.apply_reflectors(d.right_reflectors, np.eye(n))
    return d, Q1, Q2


def test_block_size_one_is_the_single_vector_method(orc):
    a = synth.workload_sparse_small()
    v0 = synth.start_vector(a.n, 1)
    r1 = orc.svds(a, 10, 10, 1e-10, 100, v0=v0)
    rb = orc.svds_block(a, 10, 10, 1, 1e-10, 100, V0=v0)
    for key in ("S", "U", "V", "res"):
        np.testing.assert_array_equal(rb[key], r1[key])
    for key in ("restarts", "n_matvec", "n_steps", "converged", "n_reorth"):
        assert rb["info"][key] == r1["info"][key], key
    # and on a dense matrix with restarts, from the seeded draw
    d, _, _ = _closed_form(120, 90, 0.9 ** np.arange(90), 5)
    r1 = orc.svds(d.a, 6, 6, 1e-12, 50, seed=4)
    rb = orc.svds_block(d.a, 6, 6, 1, 1e-12, 50, seed=4)
    np.testing.assert_array_equal(rb["S"], r1["S"])
    np.testing.assert_array_equal(rb["V"], r1["V"])
    assert rb["info"]["restarts"] == r1["info"]["restarts"] > 0


@pytest.mark.parametrize("b", [2, 3, 4])
def test_block_closed_form(orc, b):
    """A = Q1 diag(s) Q2^T: sigma_i = s_i, u_i = +-Q1 e_i, v_i = +-Q2 e_i."""
    s = np.linspace(2.0, 1.0, 200) ** 3
    d, Q1, Q2 = _closed_form(300, 200, s, 11)
    k = 8
    r = orc.svds_block(d.a, k, 12, b, 1e-12, 200, seed=2)
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], s[:k], rtol=1e-12)
    assert np.all(_sin(r["U"], Q1[:, :k]) < 1e-9)
    assert np.all(_sin(r["V"], Q2[:, :k]) < 1e-9)
    assert np.abs(r["U"].T @ r["U"] - np.eye(k)).max() < 1e-12   # the invariant's 1e-12
    assert np.abs(r["V"].T @ r["V"] - np.eye(k)).max() < 1e-12
    idx = np.argmax(np.abs(r["V"]), axis=0)
    assert np.all(r["V"][idx, np.arange(k)] > 0)  # sign rule


@pytest.mark.parametrize("b", [2, 4])
def test_block_matches_brute_force_on_sparse_workload(orc, b):
    """The 2,000 x 1,000 sparse workload against its brute-force Jacobi singular values."""
    a = synth.workload_sparse_small()
    gold = np.loadtxt(os.path.join(GOLDEN, "sparse_2000x1000_jacobi_sigma.txt"), comments="#")
    r = orc.svds_block(a, 10, 10, b, 1e-10, 400, seed=3)
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], gold[:10], rtol=1e-12)


@pytest.mark.parametrize("b,k,p,maxit", [(3, 5, 10, 1), (3, 5, 10, 3), (2, 6, 7, 2)])
def test_block_lanczos_relations(orc, b, k, p, maxit):
    """A V(:,0:t) = U(:,0:t) T(0:t,0:t) and A^T U(:,0:t) = V(:,0:t) T^T + V(:,t:t+b) F^T E^T
    with F = T(t-b:t, t:t+b); T upper triangular with bandwidth b (maxit = 1: the
    first pass; later: after augmented restarts, whose T has the rho columns)."""
    a, _ = _dense_random(160, 120, 7)
    r = orc.svds_block(a, k, p, b, 1e-14, maxit, seed=9, return_basis=True)
    t = r["t_last"]
    U, V, T = r["Ub"][:, :t], r["Vb"][:, :t + b], r["T"]
    Tt = T[:t, :t]
    F = T[t - b:t, t:t + b]
    nrm = np.linalg.norm(a, 2)
    assert np.abs(a @ V[:, :t] - U @ Tt).max() < 1e-12 * nrm
    E = np.zeros((t, b))
    E[t - b:, :] = np.eye(b)
    assert np.abs(a.T @ U - V[:, :t] @ Tt.T - V[:, t:] @ F.T @ E.T).max() < 1e-12 * nrm
    assert np.abs(U.T @ U - np.eye(t)).max() < 1e-13
    assert np.abs(V.T @ V - np.eye(t + b)).max() < 1e-13
    if maxit == 1:  # first pass: block upper triangular with bandwidth b
        assert np.all(np.tril(Tt, -1) == 0.0)
        assert np.all(np.triu(Tt, b + 1) == 0.0)


def _dense_random(m, n, seed):
    rng = np.random.default_rng(seed)
    a = np.asfortranarray(rng.standard_normal((m, n)))
    return a, np.linalg.svd(a, compute_uv=False)


@pytest.mark.parametrize("b", [2, 3])
def test_block_residual_formula_equals_true_residual(orc, b):
    """Block Eq. (4): ||A^T u_j - sigma_j v_j|| = ||F^T Uh(t-b:t, j)|| (= res_j sigma_j),
    and ||A v_j - sigma_j u_j|| = 0, on an unconverged first pass."""
    a, _ = _dense_random(150, 110, 3)
    k = 4
    r = orc.svds_block(a, k, 8, b, 1e-14, 1, seed=1)
    S, U, V, res = r["S"], r["U"], r["V"], r["res"]
    true = np.linalg.norm(a.T @ U - V * S, axis=0)
    assert np.all(res > 1e-6)  # not converged: the comparison is meaningful
    np.testing.assert_allclose(true, res * S, rtol=1e-8)
    assert np.abs(a @ V - U * S).max() < 1e-12 * S[0]


@pytest.mark.parametrize("b,k,p", [(2, 6, 10), (3, 5, 7), (4, 4, 9)])
def test_block_product_count(orc, b, k, p):
    """Products with A and A^T: 2 t0 for the first pass and 2 (t1 - k) per restart
    (Eq. 8 with u_{t+1} not formed), with t0, t1 the block-rounded sizes."""
    a, _ = _dense_random(140, 100, 5)
    r = orc.svds_block(a, k, p, b, 1e-14, 4, seed=1)
    t0, t1 = orc.block_sizes(k, p, b)
    R = r["info"]["restarts"]
    assert R == 3
    assert r["info"]["n_matvec"] == 2 * t0 + 2 * R * (t1 - k)
    assert r["t_last"] == t1


def test_block_finds_every_copy_of_a_repeated_value(orc):
    """sigma = 3 with multiplicity 3: a single-vector Krylov space holds one
    direction of the eigenspace in exact arithmetic, a block of 3 holds all."""
    s = np.r_[3.0, 3.0, 3.0, 2.0, 1.9, 1.8, 0.9 ** np.arange(194)]
    d, Q1, _ = _closed_form(300, 200, s, 21)
    r = orc.svds_block(d.a, 5, 10, 3, 1e-12, 200, seed=5)
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], s[:5], rtol=1e-12)
    # the three returned vectors for sigma = 3 span the exact eigenspace
    P = Q1[:, :3] @ Q1[:, :3].T
    assert np.linalg.norm(r["U"][:, :3] - P @ r["U"][:, :3]) < 1e-9


def test_block_rank_deficient_breakdown(orc):
    """Rank 2 with b = 4: the first U block has two (numerically) zero columns;
    they get zero diagonal entries and random replacements, and the result is
    the two nonzero singular values followed by zeros."""
    rng = np.random.default_rng(4)
    x = rng.standard_normal((90, 2))
    y = rng.standard_normal((70, 2))
    a = np.asfortranarray(x @ np.diag([5.0, 2.0]) @ y.T)
    sv = np.linalg.svd(a, compute_uv=False)
    r = orc.svds_block(a, 3, 9, 4, 1e-10, 20, seed=6)
    assert r["info"]["breakdowns"] >= 2
    np.testing.assert_allclose(r["S"][:2], sv[:2], rtol=1e-12)
    assert r["S"][2] < 1e-12 * sv[0]
    assert np.abs(a @ r["V"][:, :2] - r["U"][:, :2] * r["S"][:2]).max() < 1e-12 * sv[0]


def test_block_arguments(orc):
    a, _ = _dense_random(40, 30, 1)
    with pytest.raises(ValueError):
        orc.svds_block(a, 5, 0, 4, 1e-10, 10)     # p = 0: t1 = k < k + b
    with pytest.raises(ValueError):
        orc.svds_block(a, 5, 20, 4, 1e-10, 10)    # tmax + b > n
    with pytest.raises(ValueError):
        orc.svds_block(a, 5, 5, 0, 1e-10, 10)     # b < 1
