"""svdsc_cgs2_noalloc: the CGS2 entry point for callers that cannot allocate
device memory (its scratch is a fixed file-scope device array).  Checked
against the allocating entry point svdsc_cgs2 on the same inputs, on two
calls in a row, and against the oracle's CGS2 at the edges of the fixed
scratch (512 columns; 4,194,304 rows, where the row chunks and the GEMV-N
partial norms fill their regions exactly).  Collected last on purpose."""
import ctypes as C

import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2405_18966_gb300 as pkg
    from paper_2405_18966_gb300 import build
    build.build()
    return torch, pkg


def _case(torch, m, ncols, seed):
    rng = np.random.default_rng(seed)
    W, _ = np.linalg.qr(rng.standard_normal((m, ncols)))
    w = W @ rng.standard_normal(ncols) + 1e-3 * rng.standard_normal(m)
    ldw = m + (m & 1)
    Wt = torch.zeros((ncols, ldw), dtype=torch.float64, device="cuda")
    Wt[:, :m] = torch.tensor(W.T, device="cuda")
    return Wt, torch.tensor(w, device="cuda"), np.linalg.norm(w)


@pytest.mark.parametrize("m", [90_001, 700_001])  # ragged tails; the second in the small-CTA GEMV-N layout
def test_noalloc_cgs2_matches_allocating_entry_point(m):
    torch, pkg = _setup()
    L = pkg.lib()
    A = synth.csr_uniform(m, 300, 0.0002, 3)
    with pkg.Solver(A) as s:
        s.reserve(64)
        for call, (ncols, seed) in enumerate([(37, 1), (64, 2)]):  # two calls in a row
            Wt, w, wnorm = _case(torch, m, ncols, seed)
            ref, ref_norm = s.cgs2(Wt, w)
            got = w.clone()
            nrm = torch.empty(1, dtype=torch.float64, device="cuda")
            rc = L.svdsc_cgs2_noalloc(m, ncols, C.c_void_p(Wt.data_ptr()), Wt.shape[1],
                                      C.c_void_p(got.data_ptr()), C.c_void_p(nrm.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
            assert rc == pkg.OK, (call, rc)
            torch.cuda.synchronize()
            np.testing.assert_allclose(got.cpu().numpy(), ref.cpu().numpy(), rtol=0,
                                       atol=1e-13 * wnorm)
            assert abs(nrm.item() - ref_norm) <= 1e-13 * ref_norm


def _noalloc(torch, pkg, Wt, w, m, ncols):
    got = w.clone()
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    rc = pkg.lib().svdsc_cgs2_noalloc(m, ncols, C.c_void_p(Wt.data_ptr()), Wt.shape[1],
                                      C.c_void_p(got.data_ptr()), C.c_void_p(nrm.data_ptr()),
                                      C.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    return rc, got.cpu().numpy(), nrm.item()


@pytest.mark.parametrize("m,ncols", [(5_001, 512), (4_194_304, 1)])
def test_noalloc_cgs2_at_its_size_limits_vs_oracle(orc, m, ncols):
    """The largest column count (the P and h regions full) and the largest
    length (1,024 row chunks and 8,192 GEMV-N partial norms: the P and Pn
    regions full), each against the oracle's CGS2 and norm."""
    torch, pkg = _setup()
    for call, seed in enumerate((5, 6)):  # two calls in a row
        Wt, w, wnorm = _case(torch, m, ncols, seed)
        W = Wt[:, :m].cpu().numpy().T
        ref = orc.cgs2(W, w.cpu().numpy())
        rc, got, nrm = _noalloc(torch, pkg, Wt, w, m, ncols)
        assert rc == pkg.OK, (call, rc)
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-13 * wnorm)
        ref_norm = orc.norm2(ref)
        assert abs(nrm - ref_norm) <= 1e-13 * ref_norm


def test_noalloc_cgs2_rejects_sizes_beyond_its_scratch():
    torch, pkg = _setup()
    L = pkg.lib()
    w = torch.zeros(1000, dtype=torch.float64, device="cuda")
    nrm = torch.empty(1, dtype=torch.float64, device="cuda")
    Wt = torch.zeros((513, 1000), dtype=torch.float64, device="cuda")
    rc = L.svdsc_cgs2_noalloc(1000, 513, C.c_void_p(Wt.data_ptr()), 1000, C.c_void_p(w.data_ptr()),
                              C.c_void_p(nrm.data_ptr()), None)
    assert rc == pkg.ERR_SIZE
    # one row beyond the limit: 1,025 row chunks (rejected before any GPU work,
    # so the small buffers here are never touched)
    for length in (4_194_305, 5_000_000):
        rc = L.svdsc_cgs2_noalloc(length, 1, C.c_void_p(Wt.data_ptr()), length + (length & 1),
                                  C.c_void_p(w.data_ptr()), C.c_void_p(nrm.data_ptr()), None)
        assert rc == pkg.ERR_SIZE, length
