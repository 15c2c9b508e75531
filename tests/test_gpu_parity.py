"""GPU parity: the CUDA path (through the C-ABI) against the CPU oracle.

Tolerances (FP64 form): products and CGS2 agree to ~1e-13 relative (only the
summation order differs); singular values to 1e-10 relative (the requirement
for the FP64 form) and singular vectors to sin(angle) <= 1e-8, both far above
the rounding floor of a converged run (residuals < 1e-10 bound the sigma error
by ~res^2 sigma/gap and the angle by ~res sigma_1/gap).
"""
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
def torch_mod():
    import torch
    return torch


def _sin_angles(X, Y):
    c = np.sum(X * Y, axis=0)
    return np.linalg.norm(Y - X * c, axis=0)


def _rand_csr(m, n, seed, long_rows=(), density=0.01):
    """Random CSR covering every row-length bin: empty rows, 1..32-long rows,
    warp rows and (long_rows) CTA rows."""
    rng = np.random.default_rng(seed)
    lens = rng.integers(0, 40, size=m)
    short = rng.random(m) < 0.3
    lens[short] = rng.integers(0, 3, size=int(short.sum()))
    lens[::7] = 0
    lens[5::11] = rng.integers(33, 300, size=len(lens[5::11]))
    for r in long_rows:
        lens[r] = min(n, 5000)
    lens = np.minimum(lens, n)
    row_ptr, col = synth._fill_rows(rng, m, n, lens)
    vals = rng.standard_normal(int(row_ptr[-1]))
    return synth.CSR(m, n, row_ptr, col, vals)


# ------------------------------------------------------------------ products

@pytest.mark.parametrize("shape", [(3001, 6000), (7000, 1500)])
def test_spmv_and_transpose_vs_oracle(pkg, orc, torch_mod, shape):
    torch = torch_mod
    m, n = shape
    A = _rand_csr(m, n, m + n, long_rows=(17, m - 3))
    rng = np.random.default_rng(0)
    x, y, z = rng.standard_normal(n), rng.standard_normal(m), rng.standard_normal(m)
    with pkg.Solver(A) as s:
        gx = torch.tensor(x, device="cuda")
        gy = torch.tensor(y, device="cuda")
        gz = torch.tensor(z, device="cuda")
        ax = s.matvec(gx).cpu().numpy()
        aty = s.matvec(gy, trans=True).cpu().numpy()
        axz = s.matvec(gx, z=gz, coef=0.75).cpu().numpy()
    ref_ax = orc.matvec(A, x)
    ref_aty = orc.matvec_t(A, y)
    scale = np.abs(A.values).max() * np.sqrt(np.diff(A.row_ptr).max()) * np.abs(x).max()
    np.testing.assert_allclose(ax, ref_ax, rtol=0, atol=1e-13 * scale)
    np.testing.assert_allclose(aty, ref_aty, rtol=0, atol=1e-12 * scale)
    np.testing.assert_allclose(axz, ref_ax - 0.75 * z, rtol=0, atol=1e-13 * scale)


def test_spmv_one_based_and_four_array(pkg, orc, torch_mod):
    torch = torch_mod
    A = _rand_csr(500, 300, 9)
    B = synth.CSR(A.m, A.n, A.row_ptr + 1, (A.col_idx + 1).astype(np.int32), A.values)
    B.index_base = 1
    x = np.random.default_rng(1).standard_normal(A.n)
    with pkg.Solver(B) as s:
        got = s.matvec(torch.tensor(x, device="cuda")).cpu().numpy()
    np.testing.assert_allclose(got, orc.matvec(A, x), atol=1e-12)


def test_dense_gemv_vs_oracle(pkg, orc, torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(2)
    a = rng.standard_normal((3333, 517))
    x, y = rng.standard_normal(517), rng.standard_normal(3333)
    with pkg.Solver(a) as s:
        ax = s.matvec(torch.tensor(x, device="cuda")).cpu().numpy()
        aty = s.matvec(torch.tensor(y, device="cuda"), trans=True).cpu().numpy()
    np.testing.assert_allclose(ax, orc.matvec(a, x), atol=1e-11)
    np.testing.assert_allclose(aty, orc.matvec_t(a, y), atol=1e-11)


# -------------------------------------------------------------------- CGS2

@pytest.mark.parametrize("ncols", [1, 7, 64, 201])
def test_cgs2_vs_oracle(pkg, orc, torch_mod, ncols):
    torch = torch_mod
    m = 90_001  # several chunks and a ragged tail
    A = synth.csr_uniform(m, 300, 0.001, 3)
    rng = np.random.default_rng(ncols)
    W, _ = np.linalg.qr(rng.standard_normal((m, ncols)))
    w = W @ rng.standard_normal(ncols) + 1e-3 * rng.standard_normal(m)
    ref = orc.cgs2(W, w)
    ldw = m + 1  # even leading dimension
    Wt = torch.zeros((ncols, ldw), dtype=torch.float64, device="cuda")
    Wt[:, :m] = torch.tensor(W.T, device="cuda")
    with pkg.Solver(A) as s:
        s.reserve(max(ncols, 2))
        got, nrm = s.cgs2(Wt, torch.tensor(w, device="cuda"))
    got = got.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.linalg.norm(w))
    assert abs(nrm - np.linalg.norm(ref)) <= 1e-13 * np.linalg.norm(ref)


@pytest.mark.parametrize("ncols", [1, 33])
def test_cgs2_vs_oracle_small_cta_layout(pkg, orc, torch_mod, ncols):
    """From 684,032 rows on, the FP64 GEMV-N runs as one 512-row pass per
    256-thread CTA and the norm partials follow that layout: 700,001 rows
    (1,368 CTAs, the last one with a single odd row)."""
    torch = torch_mod
    m = 700_001
    A = synth.csr_uniform(m, 300, 0.0002, 4)
    rng = np.random.default_rng(100 + ncols)
    W, _ = np.linalg.qr(rng.standard_normal((m, ncols)))
    w = W @ rng.standard_normal(ncols) + 1e-3 * rng.standard_normal(m)
    ref = orc.cgs2(W, w)
    Wt = torch.zeros((ncols, m + 1), dtype=torch.float64, device="cuda")
    Wt[:, :m] = torch.tensor(W.T, device="cuda")
    with pkg.Solver(A) as s:
        s.reserve(max(ncols, 2))
        got, nrm = s.cgs2(Wt, torch.tensor(w, device="cuda"))
    got = got.cpu().numpy()
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * np.linalg.norm(w))
    assert abs(nrm - np.linalg.norm(ref)) <= 1e-13 * np.linalg.norm(ref)


# ---------------------------------------------------------- projected SVD

@pytest.mark.parametrize("t", [1, 2, 20, 63, 64, 65, 128, 201, 224, 225])
def test_small_svd_vs_oracle(pkg, orc, torch_mod, t):
    torch = torch_mod
    rng = np.random.default_rng(t)
    T = np.triu(rng.standard_normal((t, t)))
    if t > 4:
        T[2, :] *= 1e-6  # a spread of scales
    _, s_ref, _, _ = orc.jacobi_svd(T)
    A = synth.csr_uniform(max(2 * t + 2, 400), max(2 * t + 2, 400), 0.01, 1)
    with pkg.Solver(A) as s:
        s.reserve(t)
        S, Uh, Vh = s.small_svd(torch.tensor(T, device="cuda"))
    S, Uh, Vh = S.cpu().numpy(), Uh.cpu().numpy(), Vh.cpu().numpy()
    np.testing.assert_allclose(S, s_ref, rtol=1e-13, atol=1e-14 * s_ref[0])
    np.testing.assert_allclose(Uh @ np.diag(S) @ Vh.T, T, atol=1e-13 * s_ref[0])
    np.testing.assert_allclose(Vh.T @ Vh, np.eye(t), atol=1e-13)
    assert np.all(np.diff(S) <= 0)


def test_small_svd_rank_deficient(pkg, orc, torch_mod):
    torch = torch_mod
    t = 30
    T = np.triu(np.random.default_rng(5).standard_normal((t, t)))
    T[:, 4] = 0.0
    T[:, 11] = 0.0
    A = synth.csr_uniform(400, 400, 0.01, 1)
    with pkg.Solver(A) as s:
        s.reserve(t)
        S, Uh, Vh = s.small_svd(torch.tensor(T, device="cuda"))
    Uh = Uh.cpu().numpy()
    np.testing.assert_allclose(Uh.T @ Uh, np.eye(t), atol=1e-12)
    assert S.cpu().numpy()[-2:].max() < 1e-14


@pytest.mark.parametrize("t,scale", [(150, 1.0), (200, 1e60), (200, 1e-60)])
def test_small_svd_multi_cta_rank_deficient_and_scaled(pkg, orc, torch_mod, t, scale):
    """The multi-CTA Jacobi (t > 64) with zero columns (rank deficiency) and
    with entries far outside FP32's range, against the oracle's Jacobi."""
    torch = torch_mod
    rng = np.random.default_rng(t)
    T = np.triu(rng.standard_normal((t, t))) * scale
    T[:, 7] = 0.0
    T[:, 90] = 0.0
    _, s_ref, _, _ = orc.jacobi_svd(T)
    A = synth.csr_uniform(2 * t + 2, 2 * t + 2, 0.01, 1)
    with pkg.Solver(A) as s:
        s.reserve(t)
        S, Uh, Vh = s.small_svd(torch.tensor(T, device="cuda"))
    S, Uh, Vh = S.cpu().numpy(), Uh.cpu().numpy(), Vh.cpu().numpy()
    np.testing.assert_allclose(S, s_ref, rtol=1e-13, atol=1e-14 * s_ref[0])
    assert S[-2:].max() < 1e-14 * s_ref[0]
    np.testing.assert_allclose(Uh @ np.diag(S) @ Vh.T, T, atol=1e-13 * s_ref[0])
    np.testing.assert_allclose(Vh.T @ Vh, np.eye(t), atol=1e-13)
    np.testing.assert_allclose(Uh.T @ Uh, np.eye(t), atol=1e-12)


# ------------------------------------------------------------ full solves

def _compare(r, ref, k, sig_tol=1e-10, ang_tol=1e-8):
    np.testing.assert_allclose(r.S, ref["S"], rtol=sig_tol)
    assert np.all(_sin_angles(r.U, ref["U"]) <= ang_tol)
    assert np.all(_sin_angles(r.V, ref["V"]) <= ang_tol)


def test_solve_sparse_2000x1000(pkg, orc):
    """2,000 x 1,000 1 % sparse, k=10, p=10, tol=1e-10 (FP64 throughout)."""
    a = synth.workload_sparse_small()
    v0 = synth.start_vector(a.n, 1)
    r = pkg.svds(a, 10, 10, 1e-10, 100, v0=v0)
    ref = orc.svds(a, 10, 10, 1e-10, 100, v0=v0)
    assert r.status == pkg.OK and r.info["converged"] == 1
    _compare(r, ref, 10)
    gold = np.loadtxt(__file__.replace("test_gpu_parity.py", "golden/sparse_2000x1000_jacobi_sigma.txt"))
    np.testing.assert_allclose(r.S, gold[:10], rtol=1e-10)
    assert r.info["n_matvec"] == 2 * 20 + 2 * r.info["restarts"] * 10
    assert abs(r.info["restarts"] - ref["info"]["restarts"]) <= 1
    assert np.all(r.res < 1e-10)


@pytest.mark.parametrize("k,p", [(20, 20), (10, 30)])
def test_solve_zipf_structure_vs_lapack(pkg, orc, k, p):
    """The Zipf workload at 0.5 % scale (5,000 x 2,500): sigma against
    LAPACK's dense SVD (a check only) and the oracle; vectors within the
    Wedin bound of their gaps."""
    a = synth.workload_sparse_zipf(0.005)
    Ul, s, Vlt = np.linalg.svd(a.to_dense(), full_matrices=False)
    v0 = synth.start_vector(a.n, 1)
    r = pkg.svds(a, k, p, 1e-10, 500, v0=v0)
    ref = orc.svds(a, k, p, 1e-10, 500, v0=v0)
    assert r.status == pkg.OK and r.info["converged"] == 1
    assert abs(r.info["restarts"] - ref["info"]["restarts"]) <= 1
    np.testing.assert_allclose(r.S, s[:k], rtol=1e-12)
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-12)
    gaps = np.minimum(np.abs(s[:k] - s[1:k + 1]), np.abs(s[:k] - np.r_[np.inf, s[:k - 1]]))
    bound = 10 * 1e-10 * s[:k] / gaps + 1e-12
    assert np.all(_sin_angles(r.V, Vlt[:k].T) <= bound)
    assert np.all(_sin_angles(r.U, Ul[:, :k]) <= bound)


def test_solve_random_start_matches_oracle_rng(pkg, orc):
    """No v0: both sides draw v_1 from the same counter-based generator."""
    a = synth.workload_sparse_small()
    r = pkg.svds(a, 5, 10, 1e-10, 100, seed=77)
    ref = orc.svds(a, 5, 10, 1e-10, 100, seed=77)
    _compare(r, ref, 5)
    assert r.info["restarts"] == ref["info"]["restarts"]


def test_solve_dense_closed_form(pkg):
    """Dense A = Q1 diag(0.95^i) Q2^T (scaled to 5,000 x 500), k=10, p=10, tol=1e-12."""
    d = synth.workload_dense(0.1)
    r = pkg.svds(d.a, 10, 10, 1e-12, 100, seed=3)
    assert r.info["converged"] == 1
    np.testing.assert_allclose(r.S, d.s[:10], rtol=1e-12)
    Q1 = synth.apply_reflectors(d.left_reflectors, np.eye(d.m)[:, :10])
    Q2 = synth.apply_reflectors(d.right_reflectors, np.eye(d.n)[:, :10])
    assert np.all(_sin_angles(r.U, Q1) < 1e-9)
    assert np.all(_sin_angles(r.V, Q2) < 1e-9)


def test_solve_zipf_scaled(pkg, orc):
    """The Zipf-row workload at 2 % scale (20,000 x 10,000), k=20, p=20."""
    a = synth.workload_sparse_zipf(0.02)
    v0 = synth.start_vector(a.n, 2)
    r = pkg.svds(a, 20, 20, 1e-10, 100, v0=v0)
    ref = orc.svds(a, 20, 20, 1e-10, 100, v0=v0)
    assert r.info["converged"] == 1
    _compare(r, ref, 20)


def test_solve_device_outputs_and_one_based(pkg, orc, torch_mod):
    a = synth.workload_sparse_small()
    b = synth.CSR(a.m, a.n, a.row_ptr + 1, (a.col_idx + 1).astype(np.int32), a.values)
    b.index_base = 1
    v0 = synth.start_vector(a.n, 1)
    r = pkg.svds(b, 4, 8, 1e-10, 100, v0=v0, out="device")
    ref = orc.svds(a, 4, 8, 1e-10, 100, v0=v0)
    np.testing.assert_allclose(r.S.cpu().numpy(), ref["S"], rtol=1e-10)
    assert np.all(_sin_angles(r.V.cpu().numpy(), ref["V"]) < 1e-8)


def test_solve_rank_one_breakdown(pkg, orc):
    rng = np.random.default_rng(12)
    x, y = rng.standard_normal(80), rng.standard_normal(50)
    A = np.outer(x, y)
    r = pkg.svds(A, 2, 8, 1e-10, 20, seed=1)
    ref = orc.svds(A, 2, 8, 1e-10, 20, seed=1)
    assert r.info["breakdowns"] > 0
    np.testing.assert_allclose(r.S[0], np.linalg.norm(x) * np.linalg.norm(y), rtol=1e-12)
    assert r.S[1] < 1e-12 * r.S[0]
    np.testing.assert_allclose(r.S[0], ref["S"][0], rtol=1e-12)


def test_solve_max_size_and_k1(pkg, orc):
    a = synth.csr_uniform(60, 31, 0.3, 8)
    v0 = synth.start_vector(31, 3)
    r = pkg.svds(a, 1, 29, 1e-10, 50, v0=v0)  # t + 1 = n
    ref = orc.svds(a, 1, 29, 1e-10, 50, v0=v0)
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-12)


def test_solve_errors(pkg):
    a = synth.workload_sparse_small()
    with pkg.Solver(a) as s:
        with pytest.raises(pkg.SvdscError) as e:
            s.solve(10, 995)  # t + 1 > n
        assert e.value.status == pkg.ERR_SIZE
        with pytest.raises(pkg.SvdscError):
            s.solve(0, 5)
    bad = synth.CSR(a.m, a.n, a.row_ptr.copy(), a.col_idx.copy(), a.values.copy())
    bad.col_idx[7] = a.n + 3
    with pytest.raises(pkg.SvdscError) as e:
        pkg.Solver(bad)
    assert e.value.status == pkg.ERR_CSR
    nanm = synth.CSR(a.m, a.n, a.row_ptr, a.col_idx, a.values.copy())
    nanm.values[100] = np.nan
    with pytest.raises(pkg.SvdscError) as e:
        pkg.Solver(nanm)
    assert e.value.status == pkg.ERR_NONFINITE


def test_not_converged_status(pkg):
    a = synth.workload_sparse_small()
    r = pkg.svds(a, 10, 10, 1e-14, 2, seed=1)
    assert r.status == pkg.NOT_CONVERGED and r.info["converged"] == 0
    assert r.info["restarts"] == 1


def test_repeat_solve_is_deterministic(pkg):
    a = synth.workload_sparse_zipf(0.01)
    with pkg.Solver(a, seed=5) as s:
        r1 = s.solve(8, 8, 1e-10, 50)
        r2 = s.solve(8, 8, 1e-10, 50)
    np.testing.assert_array_equal(r1.S, r2.S)
    np.testing.assert_array_equal(r1.U, r2.U)


# ------------------------------------------------------------ mixed precision

def test_mixed_precision_k100_vs_fp64_oracle(pkg, orc):
    """FP32 products and first CGS pass, FP64 second pass / norms / small SVD,
    on the FP32-exact 2,000 x 1,000 matrix with k=100, p=100: sigma error vs
    the FP64 oracle <= 1e-6 relative for every returned triplet."""
    a = synth.workload_sparse_small_fp32()
    v0 = synth.start_vector(a.n, 4)
    ref = orc.svds(a, 100, 100, 1e-10, 100, v0=v0)
    r = pkg.svds(synth.CSR(a.m, a.n, a.row_ptr, a.col_idx, a.values.astype(np.float32)), 100, 100,
                 1e-10, 100, precision="mixed", v0=v0)
    rel = np.abs(r.S - ref["S"]) / ref["S"]
    assert rel.max() <= 1e-6, rel.max()


# ------------------------------------------------- tensor-core restart GEMM

@pytest.mark.parametrize("rows,t,k", [(1, 1, 1), (127, 16, 10), (128, 20, 10), (1000, 33, 49),
                                      (50_001, 200, 100), (3000, 448, 48), (4096, 64, 64),
                                      # 64 < k <= 128: the row-tile form (each W entry cut once)
                                      (1000, 80, 65), (65, 128, 128), (129, 448, 128), (63, 100, 97)])
def test_tc_gemm_fp64_digits_vs_oracle(pkg, orc, torch_mod, rows, t, k):
    """Mode 0 (Ozaki-style digits on BF16 tcgen05 MMAs) against the oracle's FP64
    loop: error within 8 eps sum_c |W_rc| |Q_cj| (an FP64 GEMM's bound) plus
    the digit split's own bound 2^-47 max|W_r| max|Q_j|."""
    torch = torch_mod
    rng = np.random.default_rng(rows + t + k)
    W = rng.standard_normal((rows, t)) / np.sqrt(rows)
    W[0, :] *= 1e-300 if rows > 2 else 1.0        # tiny row
    if rows > 3:
        W[2, :] = 0.0                                # zero row
        W[3, ::2] *= 1e-12                           # wide range inside one row
    Q = np.linalg.qr(rng.standard_normal((t, t)))[0][:, :k]
    ref = orc.gemm(W, Q)
    bound = (8 * 2.0**-53 * (np.abs(W) @ np.abs(Q))
             + 2.0**-47 * np.outer(np.abs(W).max(axis=1), np.abs(Q).max(axis=0)) + 1e-320)
    A = synth.csr_uniform(600, 600, 0.01, 1)
    with pkg.Solver(A) as s:
        s.reserve(max(t, 2))
        C = s.gemm(torch.tensor(W, device="cuda"), torch.tensor(Q, device="cuda"), mode=0).cpu().numpy()
    err = np.abs(C - ref)
    assert np.all(err <= bound), (err / bound).max()


def test_tc_gemm_mixed_pieces(pkg, orc, torch_mod):
    torch = torch_mod
    rng = np.random.default_rng(3)
    W = rng.standard_normal((20_000, 200)) / 140.0
    Q = np.linalg.qr(rng.standard_normal((200, 200)))[0][:, :100]
    ref = orc.gemm(W.astype(np.float32).astype(np.float64), Q)
    A = synth.csr_uniform(600, 600, 0.01, 1)
    with pkg.Solver(A) as s:
        s.reserve(200)
        C = s.gemm(torch.tensor(W, device="cuda"), torch.tensor(Q, device="cuda"), mode=1).cpu().numpy()
    scale = np.abs(W) @ np.abs(Q)
    assert np.max(np.abs(C - ref) / scale) < 2e-6


@pytest.mark.parametrize("gemm", ["tensor", "fma"])
def test_solve_both_restart_gemms(pkg, orc, gemm):
    a = synth.workload_sparse_zipf(0.01)
    v0 = synth.start_vector(a.n, 5)
    r = pkg.svds(a, 12, 12, 1e-10, 100, v0=v0, restart_gemm=gemm)
    ref = orc.svds(a, 12, 12, 1e-10, 100, v0=v0)
    assert r.info["converged"] == 1
    _compare(r, ref, 12)


@pytest.mark.parametrize("t,k,gemm", [(448, 224, "tensor"), (512, 256, "fma")])
def test_solve_at_the_size_limits(pkg, orc, t, k, gemm):
    """The documented limits: t = 448 with the tensor-core restart GEMM (its
    exactness bound), t = 512 and k = 256 with the FP64-FMA GEMM; one round
    and one restart, against the oracle (singular values of the projected
    matrix after the restart)."""
    a = synth.csr_uniform(3000, 1200, 0.01, 17)
    v0 = synth.start_vector(a.n, 6)
    r = pkg.svds(a, k, t - k, 1e-10, 2, v0=v0, restart_gemm=gemm)
    ref = orc.svds(a, k, t - k, 1e-10, 2, v0=v0)
    assert r.info["t"] == t and r.info["restarts"] == ref["info"]["restarts"] == 1
    # after two rounds the trailing Ritz values are not converged; a Ritz
    # value's error is of order res^2 sigma_1 / gap, so two runs that differ
    # by rounding agree to that, and to 1e-9 where the residual is small
    res = np.maximum(r.res, ref["res"])
    tol = 1e-9 * ref["S"] + 10.0 * res ** 2 * ref["S"][0]
    assert np.all(np.abs(r.S - ref["S"]) <= tol), np.max(np.abs(r.S - ref["S"]) / tol)
    conv = res < 1e-8
    assert conv.sum() >= k // 2
    np.testing.assert_allclose(r.S[conv], ref["S"][conv], rtol=1e-9)
    np.testing.assert_allclose(r.V.T @ r.V, np.eye(k), atol=1e-11)


def test_solve_rejects_beyond_the_limits(pkg):
    a = synth.csr_uniform(3000, 1200, 0.01, 17)
    with pytest.raises(pkg.SvdscError):
        pkg.svds(a, 100, 349, 1e-10, 2)                      # t = 449 > 448 with the tensor GEMM
    with pytest.raises(pkg.SvdscError):
        pkg.svds(a, 100, 413, 1e-10, 2, restart_gemm="fma")  # t = 513 > 512
    with pytest.raises(pkg.SvdscError):
        pkg.svds(a, 257, 100, 1e-10, 2, restart_gemm="fma")  # k = 257 > 256
