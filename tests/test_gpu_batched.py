"""Batched form (one persistent launch over many matrices, mixed precision)
against the FP64 oracle: every returned sigma within 1e-6 relative (the
mixed-form tolerance), orthonormal outputs, per-matrix convergence."""
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
        ref = orc.svds(_fp64_copy(it.a), it.k, it.k, 1e-10, 200, seed=1)
        rel = np.abs(out["S"][i] - ref["S"]) / ref["S"]
        assert rel.max() <= 1e-6, (i, rel.max())
        U, V = out["U"][i], out["V"][i]
        assert np.abs(U.T @ U - np.eye(it.k)).max() < 1e-5
        assert np.abs(V.T @ V - np.eye(it.k)).max() < 1e-5
        assert np.all(np.diff(out["S"][i]) <= 0)
        assert info["n_matvec"] == 2 * info["t"] + 2 * info["restarts"] * (info["t"] - it.k)
    tun = b.tuning(0)
    assert tun["lanes_A"] in (1, 2, 4, 8, 16, 32) and tun["gemv_cols"] in (1, 2, 4)
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


def test_batched_limits(pkg):
    a = synth.csr_uniform_rows(500, 400, 5, 10, 1)
    with pytest.raises(pkg.SvdscError) as e:
        pkg.Batch([a], [50], [50])
    assert e.value.status == pkg.ERR_SIZE
