"""Pins of the CPU oracle against facts fixed by the paper and by mathematics.

The oracle (oracle/) restates Alg. 1 and Alg. 2 of the svds-C paper.  These
tests check it against closed forms, brute force, library routines used as
independent cross-checks, and the identities of Proposition 1 / Eq. (2)-(7),
so that a dropped term, a wrong index or a transposed operand fails one of
them.  No value here comes from the CUDA solver.
"""
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _load_golden(name):
    return np.loadtxt(os.path.join(GOLDEN, name), comments="#")


def _rand_csr(m, n, density, seed, long_row=None):
    rng = np.random.default_rng(seed)
    a = (rng.random((m, n)) < density) * rng.standard_normal((m, n))
    if long_row is not None:
        a[long_row, :] = rng.standard_normal(n)
    a[min(3, m - 1), :] = 0.0  # an empty row
    rows, cols = np.nonzero(a)
    row_ptr = np.zeros(m + 1, dtype=np.int64)
    np.cumsum(np.bincount(rows, minlength=m), out=row_ptr[1:])
    return synth.CSR(m, n, row_ptr, cols.astype(np.int32), a[rows, cols]), a


def _angles_ok(X, Y, tol):
    """Columnwise sin(angle) between matched unit vectors (sign-free), computed
    as the norm of Y_j minus its projection on X_j (accurate for tiny angles)."""
    c = np.sum(X * Y, axis=0)
    sin = np.linalg.norm(Y - X * c, axis=0)
    return np.all(sin <= tol)


# --------------------------------------------------------------- random draws

def test_splitmix64_published_sequence(orc):
    # SplitMix64 (Steele, Lea, Flood 2014) from state 0: the first three outputs.
    assert orc.splitmix64(0) == 0xE220A8397B1DCDAF
    assert orc.splitmix64(0x9E3779B97F4A7C15) == 0x6E789E6AA1B965F4
    assert orc.splitmix64((2 * 0x9E3779B97F4A7C15) % 2**64) == 0x06C45D188009454F


def test_rng_normal_distribution(orc):
    from scipy import stats
    x = orc.rng_normal(7, 0, 200_000)
    assert abs(x.mean()) < 0.01 and abs(x.std() - 1.0) < 0.01
    assert stats.kstest(x, "norm").pvalue > 1e-3
    y = orc.rng_normal(7, 1, 1000)
    z = orc.rng_normal(8, 0, 1000)
    assert abs(np.corrcoef(x[:1000], y)[0, 1]) < 0.15
    assert abs(np.corrcoef(x[:1000], z)[0, 1]) < 0.15
    np.testing.assert_array_equal(orc.rng_normal(7, 0, 10), x[:10])


# ------------------------------------------------------------------ products

def test_matvec_tiny_by_hand(orc):
    # A = [[1,0,2,0],[0,0,0,0],[0,3,0,-1]] (row 1 empty)
    A = synth.CSR(3, 4, np.array([0, 2, 2, 4], np.int64), np.array([0, 2, 1, 3], np.int32),
                  np.array([1.0, 2.0, 3.0, -1.0]))
    x = np.array([1.0, 2.0, 3.0, 4.0])
    np.testing.assert_array_equal(orc.matvec(A, x), [7.0, 0.0, 2.0])
    np.testing.assert_array_equal(orc.matvec_t(A, np.array([1.0, 5.0, 2.0])), [1.0, 6.0, 2.0, -2.0])


@pytest.mark.parametrize("m,n", [(300, 170), (64, 400)])
def test_matvec_against_dense(orc, m, n):
    A, ad = _rand_csr(m, n, 0.05, m + n, long_row=5)
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(n), rng.standard_normal(m)
    np.testing.assert_allclose(orc.matvec(A, x), ad @ x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.matvec_t(A, y), ad.T @ y, rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.matvec(ad, x), ad @ x, rtol=0, atol=1e-12)
    np.testing.assert_allclose(orc.matvec_t(ad, y), ad.T @ y, rtol=0, atol=1e-12)


# -------------------------------------------------------- re-orthogonalization

def test_cgs2_projects_out_span(orc):
    rng = np.random.default_rng(3)
    W, _ = np.linalg.qr(rng.standard_normal((500, 40)))
    w = rng.standard_normal(500)
    out = orc.cgs2(W, w)
    ref = w - W @ (W.T @ w)
    np.testing.assert_allclose(out, ref, atol=1e-13)
    assert np.linalg.norm(W.T @ out) < 1e-14 * np.linalg.norm(w)


def test_cgs2_second_pass_matters(orc):
    # w nearly inside span(W): one projection leaves ~eps/1e-10 relative
    # components along W; the second pass of Sec. 2.1's projection removes them.
    rng = np.random.default_rng(4)
    W, _ = np.linalg.qr(rng.standard_normal((2000, 30)))
    w = W @ rng.standard_normal(30) + 1e-10 * rng.standard_normal(2000)
    out = orc.cgs2(W, w)
    assert np.linalg.norm(W.T @ out) <= 1e-13 * np.linalg.norm(out)
    once = orc.gemv_n_sub(W, orc.gemv_t(W, w), w)
    assert np.linalg.norm(W.T @ once) > 1e-9 * np.linalg.norm(once)


def test_gemm_against_numpy(orc):
    rng = np.random.default_rng(5)
    W, Q = rng.standard_normal((333, 21)), rng.standard_normal((21, 7))
    np.testing.assert_allclose(orc.gemm(W, Q), W @ Q, atol=1e-12)


# ---------------------------------------------------------- dense Jacobi SVD

def test_jacobi_diagonal_closed_form(orc):
    d = np.array([3.0, -7.0, 0.5, 7.0 - 1e-9, 2.0])
    U, S, V, sw = orc.jacobi_svd(np.diag(d))
    np.testing.assert_allclose(S, np.sort(np.abs(d))[::-1], rtol=1e-15)
    assert sw > 0
    np.testing.assert_allclose(np.abs(U), np.abs(V), atol=0)
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, np.diag(d), atol=1e-15)


@pytest.mark.parametrize("m,n", [(60, 60), (90, 40), (7, 1), (1, 1)])
def test_jacobi_random_matches_library(orc, m, n):
    rng = np.random.default_rng(m * 100 + n)
    A = rng.standard_normal((m, n))
    U, S, V, sw = orc.jacobi_svd(A)
    assert sw > 0
    np.testing.assert_allclose(S, np.linalg.svd(A, compute_uv=False), rtol=1e-13, atol=1e-14)
    np.testing.assert_allclose(U @ np.diag(S) @ V.T, A, atol=1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(n), atol=1e-13)
    np.testing.assert_allclose(V.T @ V, np.eye(n), atol=1e-13)


def test_jacobi_prescribed_singular_values(orc):
    s = np.array([5.0, 4.0, 1.0, 1e-3, 1e-8, 0.0])
    d = synth.dense_prescribed(40, 6, s, 11, nrefl=3)
    U, S, V, sw = orc.jacobi_svd(d.a)
    # the construction itself rounds at eps*||A||: absolute tolerance there
    np.testing.assert_allclose(S[:5], s[:5], rtol=1e-13, atol=1e-14 * s[0])
    assert S[5] < 1e-14 * s[0]
    # rank-deficient: completed U stays orthonormal
    np.testing.assert_allclose(U.T @ U, np.eye(6), atol=1e-13)
    Q1 = synth.apply_reflectors(d.left_reflectors, np.eye(40)[:, :6])
    # Wedin: angle <= eps*||A|| / gap; the sigma = 1e-8 vector has gap 1e-8
    assert _angles_ok(U[:, :4], Q1[:, :4], 1e-9)
    assert _angles_ok(U[:, 4:5], Q1[:, 4:5], 1e-6)


# ------------------------------------------------------------ Alg. 2 (svds)

def test_svds_closed_form_dense(orc):
    """A = Q1 diag(0.95^i) Q2^T: sigma known exactly, vectors +-Q1 e_i, +-Q2 e_i."""
    d = synth.dense_prescribed(3000, 300, synth.decay_095(300), 21)
    k = 12
    r = orc.svds(d, k, k, 1e-12, 100, seed=5)
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], d.s[:k], rtol=1e-12)
    E = np.eye(3000)[:, :k]
    Q1 = synth.apply_reflectors(d.left_reflectors, E)
    Q2 = synth.apply_reflectors(d.right_reflectors, np.eye(300)[:, :k])
    assert _angles_ok(r["U"], Q1, 1e-8)
    assert _angles_ok(r["V"], Q2, 1e-8)


def test_svds_diagonal_matrix(orc):
    n = 120
    d = np.linspace(1.0, 3.0, n) * np.where(np.arange(n) % 2, -1.0, 1.0)
    A = synth.CSR(n + 30, n, np.concatenate([np.arange(n + 1), np.full(30, n)]).astype(np.int64),
                  np.arange(n, dtype=np.int32), d)
    k = 6
    r = orc.svds(A, k, 14, 1e-10, 200, seed=2)
    assert r["info"]["converged"] == 1
    order = np.argsort(-np.abs(d))[:k]
    np.testing.assert_allclose(r["S"], np.abs(d[order]), rtol=1e-10)
    for j, idx in enumerate(order):
        assert abs(abs(r["V"][idx, j]) - 1.0) < 1e-8
        assert abs(abs(r["U"][idx, j]) - 1.0) < 1e-8


def test_svds_sparse_2000x1000_against_jacobi_golden(orc):
    """The 2,000 x 1,000 1 % workload, k=10, p=10, tol=1e-10 vs brute-force Jacobi."""
    a = synth.workload_sparse_small()
    gold = _load_golden("sparse_2000x1000_jacobi_sigma.txt")
    r = orc.svds(a, 10, 10, 1e-10, 200, seed=1)
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], gold[:10], rtol=1e-10)
    # Prop. 1 / Eq. (2): A v_j = sigma_j u_j, and Eq. (4): the cheap residual
    # equals the true one ||A^T u_j - sigma_j v_j|| / sigma_j.
    ad = a.to_dense()
    lhs = ad @ r["V"] - r["U"] * r["S"]
    assert np.max(np.linalg.norm(lhs, axis=0)) < 1e-12 * gold[0]
    true_res = np.linalg.norm(ad.T @ r["U"] - r["V"] * r["S"], axis=0) / r["S"]
    assert np.all(true_res < 1e-10)
    # equal above the rounding floor eps*||A||/sigma_j (~1e-13 here)
    np.testing.assert_allclose(true_res, r["res"], rtol=1e-2, atol=1e-12)


def test_svds_fp32_exact_k100_against_jacobi_golden(orc):
    a = synth.workload_sparse_small_fp32()
    gold = _load_golden("sparse_2000x1000_fp32exact_jacobi_sigma.txt")
    r = orc.svds(a, 100, 100, 1e-10, 100, seed=4)
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], gold[:100], rtol=1e-10)


@pytest.mark.parametrize("m,n,k,p", [(200, 100, 5, 10), (150, 300, 4, 8), (60, 40, 1, 38)])
def test_svds_small_random_vs_jacobi(orc, m, n, k, p):
    A, ad = _rand_csr(m, n, 0.1, 7 * m + n)
    _, s, _, _ = orc.jacobi_svd(ad)
    r = orc.svds(A, k, p, 1e-10, 300, seed=9)
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], s[:k], rtol=1e-10)
    np.testing.assert_allclose(r["U"].T @ r["U"], np.eye(k), atol=1e-12)
    np.testing.assert_allclose(r["V"].T @ r["V"], np.eye(k), atol=1e-12)


def test_lanczos_relations_and_counts(orc):
    """A V_t = U_t T_t and A^T U_t = V_t T_t^T + beta_t v_{t+1} e_t^T (Prop. 1
    setting), orthonormal bases, and the product count of Eq. (8) with
    u_{t+1} skipped: 2t + 2R(t-k)."""
    a = synth.workload_sparse_small()
    ad = a.to_dense()
    k, p = 8, 12
    for maxit in (1, 3):
        r = orc.svds(a, k, p, 1e-30, maxit, seed=3, return_basis=True)
        t = r["t"]
        Ub, Vb, T = r["Ub"], r["Vb"], r["T"]
        Tt = T[:t, :t]
        beta_t = T[t - 1, t]
        assert np.linalg.norm(Ub.T @ Ub - np.eye(t)) < 1e-12
        assert np.linalg.norm(Vb.T @ Vb - np.eye(t + 1)) < 1e-12
        scale = np.linalg.norm(ad, 2)
        assert np.linalg.norm(ad @ Vb[:, :t] - Ub @ Tt) < 1e-13 * scale
        rhs = Vb[:, :t] @ Tt.T
        rhs[:, t - 1] += beta_t * Vb[:, t]
        assert np.linalg.norm(ad.T @ Ub - rhs) < 1e-13 * scale
        # T is upper triangular: bidiagonal before a restart, spiked after
        assert np.all(np.tril(Tt, -1) == 0)
        if maxit == 1:
            assert np.all(np.triu(Tt, 2) == 0)
        R = r["info"]["restarts"]
        assert R == maxit - 1
        assert r["info"]["n_matvec"] == 2 * t + 2 * R * (t - k)


def test_restart_coefficients_eq6(orc):
    """Eq. (6): u~_j^T A v_{t+1} = beta_t Uh(t,j) for the Ritz vectors of a fresh LBP."""
    a = synth.workload_sparse_small()
    ad = a.to_dense()
    k, p = 5, 10
    r = orc.svds(a, k, p, 1e-30, 1, seed=6, return_basis=True)
    t = r["t"]
    Uh, Sh, Vh, _ = orc.jacobi_svd(r["T"][:t, :t])
    beta_t = r["T"][t - 1, t]
    Ut = r["Ub"] @ Uh[:, :k]
    lhs = Ut.T @ (ad @ r["Vb"][:, t])
    np.testing.assert_allclose(lhs, beta_t * Uh[t - 1, :k], atol=1e-12 * Sh[0])


def test_rank_one_breakdown(orc):
    rng = np.random.default_rng(12)
    x, y = rng.standard_normal(80), rng.standard_normal(50)
    A = np.outer(x, y)
    r = orc.svds(A, 2, 8, 1e-10, 20, seed=1)
    assert r["info"]["breakdowns"] > 0
    np.testing.assert_allclose(r["S"][0], np.linalg.norm(x) * np.linalg.norm(y), rtol=1e-12)
    assert r["S"][1] < 1e-12 * r["S"][0]
    assert _angles_ok(r["U"][:, :1], (x / np.linalg.norm(x))[:, None], 1e-10)


def test_zero_matrix(orc):
    r = orc.svds(np.zeros((30, 20)), 3, 5, 1e-10, 5, seed=1)
    np.testing.assert_array_equal(r["S"], 0.0)
    assert r["info"]["converged"] == 1


def test_repeated_singular_values_subspace(orc):
    # sigma = (2,2,2,1,...): any orthonormal basis of the 3-dim top cluster is right
    s = np.concatenate([[2.0, 2.0, 2.0], np.linspace(1.0, 0.1, 37)])
    d = synth.dense_prescribed(200, 40, s, 31, nrefl=2)
    r = orc.svds(d, 3, 10, 1e-10, 100, seed=2)
    np.testing.assert_allclose(r["S"], 2.0, rtol=1e-10)
    Q2 = synth.apply_reflectors(d.right_reflectors, np.eye(40)[:, :3])
    sv = np.linalg.svd(Q2.T @ r["V"], compute_uv=False)
    assert np.all(sv > 1 - 1e-10)


def test_max_size_and_bad_args(orc):
    A, _ = _rand_csr(40, 21, 0.3, 5)
    r = orc.svds(A, 5, 15, 1e-10, 200, seed=1)  # t + 1 = n exactly
    assert r["S"].shape == (5,)
    for bad in [dict(k=0, p=5), dict(k=5, p=16), dict(k=30, p=0)]:
        with pytest.raises(ValueError):
            orc.svds(A, bad["k"], bad["p"], 1e-10, 10)
    with pytest.raises(ValueError):
        orc.svds(A, 2, 2, 0.0, 10)
    # default subspace dimension of Alg. 2
    assert orc.subspace_dim(3, -1) == 15 and orc.subspace_dim(10, -1) == 30


def test_start_vector_and_thread_independence(orc):
    a = synth.workload_sparse_small()
    v0 = synth.start_vector(a.n, 1)
    orc.set_threads(1)
    r1 = orc.svds(a, 4, 6, 1e-10, 50, v0=v0)
    orc.set_threads(4)
    r4 = orc.svds(a, 4, 6, 1e-10, 50, v0=v0)
    np.testing.assert_array_equal(r1["S"], r4["S"])
    np.testing.assert_array_equal(r1["U"], r4["U"])
    # scaling v0 does not change the normalised v_1, hence nothing else
    r5 = orc.svds(a, 4, 6, 1e-10, 50, v0=3.0 * v0)
    np.testing.assert_allclose(r5["S"], r1["S"], rtol=1e-14)
    orc.set_threads(os.cpu_count() or 1)


def test_sign_rule(orc):
    U = np.array([[1.0, 2.0], [3.0, 4.0]])
    V = np.array([[0.1, -0.9], [-0.5, 0.2]])
    U2, V2 = orc.sign_normalize(U, V)
    np.testing.assert_array_equal(V2[:, 0], [-0.1, 0.5])
    np.testing.assert_array_equal(U2[:, 0], [-1.0, -3.0])
    np.testing.assert_array_equal(V2[:, 1], [0.9, -0.2])


def test_oracle_dense_and_csr_forms_agree(orc):
    """The same matrix as dense column-major and as CSR: same restarts and
    singular values to rounding (the two product loops differ only in order)."""
    a = synth.workload_sparse_small()
    d = a.to_dense()
    v0 = synth.start_vector(a.n, 1)
    r1 = orc.svds(a, 8, 12, 1e-10, 100, v0=v0)
    r2 = orc.svds(d, 8, 12, 1e-10, 100, v0=v0)
    assert r1["info"]["restarts"] == r2["info"]["restarts"]
    np.testing.assert_allclose(r1["S"], r2["S"], rtol=1e-13)
    assert np.all(np.abs(np.sum(r1["V"] * r2["V"], axis=0)) > 1 - 1e-10)


def test_oracle_transpose_swaps_the_factors(orc):
    """svds(A^T) gives the singular values of svds(A), with U and V swapped
    (A^T has the same singular values; its products are A's, exchanged)."""
    a = synth.workload_sparse_small()
    d = a.to_dense()
    r = orc.svds(d, 6, 14, 1e-12, 200, seed=3)
    rt = orc.svds(np.ascontiguousarray(d.T), 6, 14, 1e-12, 200, seed=3)
    assert r["info"]["converged"] == 1 and rt["info"]["converged"] == 1
    np.testing.assert_allclose(rt["S"], r["S"], rtol=1e-12)
    assert np.all(np.abs(np.sum(rt["U"] * r["V"], axis=0)) > 1 - 1e-9)
    assert np.all(np.abs(np.sum(rt["V"] * r["U"], axis=0)) > 1 - 1e-9)


@pytest.mark.parametrize("k,p", [(20, 20), (10, 30)])
def test_oracle_zipf_structure_vs_lapack(orc, k, p):
    """The Zipf workload's structure (Zipf(1.5) row lengths, 39 % one-entry
    rows, heavy rows near the cap) at 0.5 % scale, 5,000 x 2,500: the k
    largest singular values against LAPACK's dense SVD (a library routine, a
    check only) and the vectors within the Wedin bound of their gaps."""
    a = synth.workload_sparse_zipf(0.005)
    ad = a.to_dense()
    Ul, s, Vlt = np.linalg.svd(ad, full_matrices=False)
    r = orc.svds(a, k, p, 1e-10, 500, v0=synth.start_vector(a.n, 1))
    assert r["info"]["converged"] == 1 and r["info"]["restarts"] > 0
    np.testing.assert_allclose(r["S"], s[:k], rtol=1e-13)
    gaps = np.minimum(np.abs(s[:k] - s[1:k + 1]), np.abs(s[:k] - np.r_[np.inf, s[:k - 1]]))
    bound = 10 * 1e-10 * s[:k] / gaps + 1e-12  # Wedin: residual / gap, with slack

    def sines(X, Y):  # sine of the angle between matching columns, sign-free
        c = np.sum(X * Y, axis=0)
        return np.linalg.norm(Y - X * c, axis=0)

    assert np.all(sines(Vlt[:k].T, r["V"]) <= bound)
    assert np.all(sines(Ul[:, :k], r["U"]) <= bound)
