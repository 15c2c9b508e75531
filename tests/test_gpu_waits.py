"""Bounded device-side waits: a wait that nothing will satisfy runs out, the
call reports SVDSC_ERR_TIMEOUT through the status block, and the context
stays usable.  The waits are the library's own (the grid barrier of the
multi-CTA Jacobi SVD and the mbarrier wait of the tensor-core GEMM); nothing
faults, traps or hangs."""
import time

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


@pytest.mark.parametrize("kind", [0, 1])
def test_wait_runs_out_and_context_survives(pkg, kind):
    a = synth.workload_sparse_small()
    with pkg.Solver(a) as s:
        t0 = time.perf_counter()
        rc = s.selftest_wait(kind)
        dt = time.perf_counter() - t0
        assert rc == pkg.ERR_TIMEOUT, rc
        assert dt < 120.0
        r = s.solve(5, 10, 1e-10, 100)               # the same context still solves
        assert r.status == pkg.OK and r.info["converged"] == 1
        ref = np.linalg.svd(a.to_dense(), compute_uv=False)[:5]
        np.testing.assert_allclose(r.S, ref, rtol=1e-10)


def test_selftest_rejects_unknown_kind(pkg):
    with pkg.Solver(synth.workload_sparse_small()) as s:
        assert s.selftest_wait(7) == pkg.ERR_ARG
