"""The paper's synthetic dense suite (Dense1-3: Sec. 5, spectra Decay1-3 of
Eq. 16) and a spectrum with exactly repeated singular values (the property of
LargeRegFile on which Sec. 5 reports other solvers going wrong).

CPU tests pin the input recipe and the oracle against the exact singular
values and vectors of the construction A = H diag(s) G^T; GPU tests hold the
CUDA path to the same exact answers and to the oracle, at the paper's settings
(k = 100, t = max(15, 3k) = 300, tol = 1e-10, at most r = 10 rounds) on a
3,000 x 3,000 scaled copy.

Repeated values: started from one vector, a Krylov method sees one direction
per repeated singular value in exact arithmetic; in floating point the
restarts recover further copies from rounding, but not in every run (the
300 x 200 case with p = 40 below converges with one copy of 1.5 missing).
What holds in every run, and is checked, is that each returned triplet is a
true one and that no value comes back more often than its multiplicity.
"""
import numpy as np
import pytest

import synth


def _cluster_sines(X, Y, s):
    """Largest principal-angle sine between span(X[:, g]) and span(Y[:, g]) for
    each group g of equal exact values s (Decay1 repeats 1e-4 at i = 20, 21:
    any rotation within the pair is a correct answer)."""
    out = np.zeros(X.shape[1])
    j = 0
    while j < X.shape[1]:
        g = j + 1
        while g < X.shape[1] and abs(s[g] - s[j]) <= 1e-15 * s[0]:
            g += 1
        Xg, Yg = X[:, j:g], Y[:, j:g]
        out[j:g] = np.linalg.norm(Yg - Xg @ (Xg.T @ Yg), 2)
        j = g
    return out


def _exact_vectors(d, k):
    Q1 = synth.apply_reflectors(d.left_reflectors, np.eye(d.m)[:, :k])
    Q2 = synth.apply_reflectors(d.right_reflectors, np.eye(d.n)[:, :k])
    return Q1, Q2


def _check_repeated(S, U, V, a, s_exact, tol_val=1e-12):
    """Every triplet true; multiplicities not exceeded; the distinct values
    found are the largest distinct ones."""
    k = len(S)
    distinct = np.unique(s_exact)[::-1]
    idx = [int(np.argmin(np.abs(distinct - x))) for x in S]
    assert np.max(np.abs(distinct[idx] - S)) <= tol_val
    mult = {i: int(np.sum(np.abs(s_exact - distinct[i]) <= 1e-14)) for i in set(idx)}
    for i in set(idx):
        assert idx.count(i) <= mult[i]
    assert sorted(set(idx)) == list(range(len(set(idx))))
    assert np.all(np.diff(S) <= 1e-13)
    np.testing.assert_allclose(U.T @ U, np.eye(k), atol=1e-12)
    np.testing.assert_allclose(V.T @ V, np.eye(k), atol=1e-12)
    assert np.max(np.linalg.norm(a @ V - U * S, axis=0)) <= 1e-9
    assert np.max(np.linalg.norm(a.T @ U - V * S, axis=0)) <= 1e-9


# ------------------------------------------------------------------ CPU pins

def test_decay_spectra_eq16():
    d1 = synth.decay1(60)
    assert d1[0] == 1.0
    np.testing.assert_allclose(d1[:20], 10.0 ** (-4.0 * np.arange(20) / 19.0), rtol=1e-15)
    np.testing.assert_allclose(d1[19], 1e-4, rtol=1e-14)      # the two pieces meet at i = 20, 21
    np.testing.assert_allclose(d1[20], 1e-4, rtol=1e-15)
    np.testing.assert_allclose(d1[39], 1e-4 / 20.0 ** 0.1, rtol=1e-15)
    np.testing.assert_allclose(synth.decay2(4), [1.0, 0.25, 1.0 / 9.0, 1.0 / 16.0], rtol=1e-15)
    np.testing.assert_allclose(synth.decay3(3), [1.0, 0.125, 1.0 / 27.0], rtol=1e-15)
    for f in synth.DECAYS.values():
        assert np.all(np.diff(f(10_000)) <= 0.0)


def test_dense_decay_construction_has_the_prescribed_spectrum():
    d = synth.workload_dense_decay(1, 0.02)                     # 200 x 200
    s = np.linalg.svd(d.a, compute_uv=False)
    np.testing.assert_allclose(s, d.s, rtol=0, atol=1e-14)
    assert d.m == d.n == 200 and d.a.flags["F_CONTIGUOUS"]


@pytest.mark.parametrize("which", [1, 2, 3])
def test_oracle_dense_decay_exact(orc, which):
    """Oracle on a 300 x 300 DenseN: sigma and vectors of the construction."""
    d = synth.workload_dense_decay(which, 0.03)
    r = orc.svds(d.a, 10, 20, 1e-10, 100, v0=synth.start_vector(d.n, 1))
    assert r["info"]["converged"] == 1
    np.testing.assert_allclose(r["S"], d.s[:10], rtol=0, atol=1e-13)
    Q1, Q2 = _exact_vectors(d, 10)
    assert np.all(_cluster_sines(r["U"], Q1, d.s) < 1e-8)
    assert np.all(_cluster_sines(r["V"], Q2, d.s) < 1e-8)


@pytest.mark.parametrize("p", [20, 40])
def test_oracle_repeated_values(orc, p):
    s = synth.repeated_spectrum(200)
    d = synth.dense_prescribed(300, 200, s, 7)
    r = orc.svds(d.a, 11, p, 1e-10, 100)
    assert r["info"]["converged"] == 1
    _check_repeated(r["S"], r["U"], r["V"], d.a, s)


def test_oracle_repeated_values_all_copies_found(orc):
    """With p = 20 the restarts pick up every copy: the exact multiset."""
    s = synth.repeated_spectrum(200)
    d = synth.dense_prescribed(300, 200, s, 7)
    r = orc.svds(d.a, 11, 20, 1e-10, 100)
    np.testing.assert_allclose(r["S"], s[:11], rtol=0, atol=1e-12)


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
@pytest.mark.parametrize("which", [1, 2, 3])
def test_gpu_dense_decay_paper_settings(pkg, orc, which):
    """DenseN at 0.3 scale (3,000 x 3,000), k = 100, p = 200, tol = 1e-10, maxit = 10."""
    d = synth.workload_dense_decay(which, 0.3)
    v0 = synth.start_vector(d.n, 1)
    r = pkg.svds(d.a, 100, 200, 1e-10, 10, v0=v0)
    ref = orc.svds(d.a, 100, 200, 1e-10, 10, v0=v0)
    assert abs(r.info["restarts"] - ref["info"]["restarts"]) <= 1
    assert r.info["converged"] == ref["info"]["converged"] == 1
    np.testing.assert_allclose(r.S, d.s[:100], rtol=0, atol=1e-13)
    np.testing.assert_allclose(r.S, ref["S"], rtol=1e-10)
    Q1, Q2 = _exact_vectors(d, 100)
    # Wedin: sin(angle) <= res sigma_j / gap_j; Decay1's tail gaps are ~1e-3 relative
    assert np.all(_cluster_sines(r.U, Q1, d.s) < 1e-6)
    assert np.all(_cluster_sines(r.V, Q2, d.s) < 1e-6)
    assert np.all(_cluster_sines(r.U, ref["U"], d.s) < 1e-6)


@pytest.mark.gpu
@pytest.mark.parametrize("p", [20, 40])
def test_gpu_repeated_values(pkg, p):
    s = synth.repeated_spectrum(200)
    d = synth.dense_prescribed(300, 200, s, 7)
    r = pkg.svds(d.a, 11, p, 1e-10, 100)
    assert r.info["converged"] == 1
    _check_repeated(r.S, r.U, r.V, d.a, s)
