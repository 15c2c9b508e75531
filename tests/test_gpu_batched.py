"""Batched form (one persistent launch over many matrices, mixed precision)
against the FP64 oracle, matrix by matrix: every returned sigma within 1e-6
relative (the mixed-form tolerance), every singular vector within a
gap-scaled angle of the oracle's (sign-free), the per-triplet residuals
||A v_j - sigma_j u_j|| and ||A^T u_j - sigma_j v_j|| (by the oracle's own
products), orthonormal outputs, per-matrix convergence."""
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


def _fp64_copy(a):
    return synth.CSR(a.m, a.n, a.row_ptr, a.col_idx, a.values.astype(np.float64))


def _sin_angles(X, Y):
    """sin of the angle between matching columns of X and Y (unit vectors, either sign)."""
    c = np.sum(X * Y, axis=0)
    return np.linalg.norm(Y - X * c, axis=0)


# Mixed-form error budget, shared with the mixed full-size test: the FP32
# products, the FP32 first CGS pass and the FP32 restart GEMM perturb the
# Lanczos relations by a few FP32 roundings of ||A|| (2^-24 = 6e-8, times
# sqrt(t) <= 9 for t <= 80), so each singular vector moves by at most about
# 1e-6 sigma_1 / gap_j (Wedin) and each triplet's residual stays below
# ~1e-6 sigma_1; the bounds below allow a factor of ten on the residual.
SIN_SCALE = 1e-6
RES_BOUND = 1e-5


def check_vs_oracle(orc, a32, k, S, U, V, ref=None, maxit=1000):
    """One batched result against the FP64 oracle on the FP64 copy of the matrix;
    returns the per-triplet errors."""
    a64 = _fp64_copy(a32)
    if ref is None:
        ref = orc.svds(a64, k, k, 1e-10, maxit, seed=1)
    s = ref["S"]
    rel = np.abs(S - s) / s
    assert rel.max() <= 1e-6, rel.max()
    # vectors: sin(angle) to the oracle's, within the Wedin bound of the gaps to
    # the neighbouring singular values (the last one's lower neighbour, sigma_{k+1},
    # is not returned, so it is checked through its residual only)
    gaps = np.minimum(np.r_[np.inf, s[:-1] - s[1:]], np.r_[s[:-1] - s[1:], np.inf])[:k - 1]
    bound = SIN_SCALE * s[0] / np.maximum(gaps, 1e-300) + 1e-7
    sin_u = _sin_angles(U, ref["U"])
    sin_v = _sin_angles(V, ref["V"])
    assert np.all(sin_u[:k - 1] <= bound), (sin_u[:k - 1] / bound).max()
    assert np.all(sin_v[:k - 1] <= bound), (sin_v[:k - 1] / bound).max()
    # residuals of every returned triplet, by the oracle's products
    r1 = np.array([np.linalg.norm(orc.matvec(a64, V[:, j]) - S[j] * U[:, j]) for j in range(k)])
    r2 = np.array([np.linalg.norm(orc.matvec_t(a64, U[:, j]) - S[j] * V[:, j]) for j in range(k)])
    assert r1.max() <= RES_BOUND * s[0] and r2.max() <= RES_BOUND * s[0], (r1.max() / s[0], r2.max() / s[0])
    # the sign rule of the outputs: v_j's largest-magnitude entry is positive
    idx = np.argmax(np.abs(V), axis=0)
    assert np.all(V[idx, np.arange(k)] > 0)
    return {"sigma_rel": rel, "sin_u": sin_u, "sin_v": sin_v, "res_av": r1 / s[0], "res_atu": r2 / s[0]}


@pytest.mark.parametrize("cluster", [0, 1, 2, 8])
def test_batched_uneven_shapes_vs_oracle(pkg, orc, cluster):
    """cluster = CTAs per matrix (0: automatic); rows split across the cluster."""
    items = synth.workload_batch(count=10, size_scale=0.08, seed=7)
    mats = [it.a for it in items]
    ks = [it.k for it in items]
    b = pkg.Batch(mats, ks, ks, seed=3, cluster=cluster)
    if cluster:
        assert b.layout()["cluster_size"] == cluster
    out = b.solve(1e-10, 200)
    for i, it in enumerate(items):
        info = out["infos"][i]
        assert info["err"] == 0, info
        assert info["converged"] == 1, (i, info)
        U, V = out["U"][i], out["V"][i]
        check_vs_oracle(orc, it.a, it.k, out["S"][i], U, V, maxit=200)
        assert np.abs(U.T @ U - np.eye(it.k)).max() < 1e-5
        assert np.abs(V.T @ V - np.eye(it.k)).max() < 1e-5
        assert np.all(np.diff(out["S"][i]) <= 0)
        assert info["n_matvec"] == 2 * info["t"] + 2 * info["restarts"] * (info["t"] - it.k)
    tun = b.tuning(0)
    assert tun["lanes_A"] in (1, 2, 4, 8, 16, 32) and tun["gemv_cols"] in (1, 2, 4)
    b.close()


@pytest.mark.parametrize("cluster", [1, 2])
def test_batched_handoff_vs_oracle(pkg, orc, cluster):
    """Hand-off forced at the first idle cluster: the matrices still running
    stop at a restart boundary and a second launch of 8-CTA clusters resumes
    them.  Every result against the oracle as above; the counters carry over
    (the product count of Eq. 8 still holds); solved twice from the graph."""
    items = synth.workload_batch(count=10, size_scale=0.08, seed=7)
    b = pkg.Batch([it.a for it in items], [it.k for it in items], [it.k for it in items], seed=3,
                  cluster=cluster, handoff=1)
    h = b.handoff()
    assert h["idle_threshold"] == 1 and h["cluster_size"] == 8 and h["clusters"] >= 1
    for rep in range(2):
        out = b.solve(1e-10, 200)
        h = b.handoff()
        cl = b.profile()["cluster"]
        assert h["handed_off"] >= 1, h
        assert int(np.sum(cl >= 100000)) == h["handed_off"]
        for i, it in enumerate(items):
            info = out["infos"][i]
            assert info["err"] == 0 and info["converged"] == 1, (i, info)
            check_vs_oracle(orc, it.a, it.k, out["S"][i], out["U"][i], out["V"][i], maxit=200)
            assert info["n_matvec"] == 2 * info["t"] + 2 * info["restarts"] * (info["t"] - it.k)
    b.close()


@pytest.mark.parametrize("cluster", [1, 2])
def test_batched_lead_clusters_vs_oracle(pkg, orc, cluster):
    """A lead launch of one 8-CTA cluster beside clusters of 1 or 2 CTAs (and
    the hand-off after them): the lead cluster takes the first queue position
    and then shares the queue; every result against the oracle, twice (the
    second solve queued by the first one's cycles)."""
    items = synth.workload_batch(count=10, size_scale=0.08, seed=7)
    b = pkg.Batch([it.a for it in items], [it.k for it in items], [it.k for it in items], seed=3,
                  cluster=cluster, handoff=1, lead=1)
    assert b.lead() == {"cluster_size": 8, "clusters": 1}
    for rep in range(2):
        out = b.solve(1e-10, 200)
        cl = b.profile()["cluster"]
        assert int(np.sum(cl >= 200000)) >= 1
        for i, it in enumerate(items):
            info = out["infos"][i]
            assert info["err"] == 0 and info["converged"] == 1, (i, info)
            check_vs_oracle(orc, it.a, it.k, out["S"][i], out["U"][i], out["V"][i], maxit=200)
            assert info["n_matvec"] == 2 * info["t"] + 2 * info["restarts"] * (info["t"] - it.k)
    b.close()
    with pytest.raises(pkg.SvdscError):
        pkg.Batch([it.a for it in items], [it.k for it in items], lead=-2)


def test_batched_handoff_off(pkg):
    items = synth.workload_batch(count=4, size_scale=0.05, seed=11)
    b = pkg.Batch([it.a for it in items], [it.k for it in items], seed=5, cluster=1, handoff=-1)
    assert b.handoff()["idle_threshold"] == 0 and b.handoff()["cluster_size"] == 0
    out = b.solve(1e-10, 100)
    assert b.handoff()["handed_off"] == 0
    assert all(i["converged"] == 1 for i in out["infos"])
    b.close()


def test_batched_graph_replay_is_deterministic_and_device_outputs(pkg):
    items = synth.workload_batch(count=6, size_scale=0.05, seed=11)
    b = pkg.Batch([it.a for it in items], [it.k for it in items], seed=5)
    r1 = b.solve(1e-10, 100)
    r2 = b.solve(1e-10, 100, out="device")
    for i in range(len(items)):
        np.testing.assert_array_equal(r1["S"][i], r2["S"][i].cpu().numpy())
        np.testing.assert_array_equal(r1["U"][i], r2["U"][i].cpu().numpy())
    b.close()


def test_batched_queue_order_from_measured_cycles(pkg):
    """Repeated solves of one batch: the queue follows the previous solve's
    measured cycles (order=0) or the size estimate (order=1); with one cluster
    size and no hand-off the results are the same either way, bit for bit."""
    items = synth.workload_batch(count=8, size_scale=0.05, seed=13)
    mats, ks = [it.a for it in items], [it.k for it in items]
    b0 = pkg.Batch(mats, ks, seed=5, cluster=2, handoff=-1, order=0)
    b1 = pkg.Batch(mats, ks, seed=5, cluster=2, handoff=-1, order=1)
    runs = [b0.solve(1e-10, 200) for _ in range(3)] + [b1.solve(1e-10, 200)]
    for r in runs[1:]:
        for i in range(len(items)):
            np.testing.assert_array_equal(r["S"][i], runs[0]["S"][i])
            np.testing.assert_array_equal(r["U"][i], runs[0]["U"][i])
            assert r["infos"][i]["restarts"] == runs[0]["infos"][i]["restarts"]
    b0.close()
    b1.close()
    with pytest.raises(pkg.SvdscError):
        pkg.Batch(mats, ks, order=2)


def test_batched_limits(pkg):
    a = synth.csr_uniform_rows(500, 400, 5, 10, 1)
    with pytest.raises(pkg.SvdscError) as e:
        pkg.Batch([a], [50], [50])
    assert e.value.status == pkg.ERR_SIZE
