"""svdsc: truncated SVD on one GB300 GPU — Python binding of libsvdsc.so.

This module only marshals arguments to the C-ABI declared in include/svdsc.h
(ctypes); every step of the solver runs in the library's CUDA kernels.  The
library must have been built (``python -c "import __graft_entry__ as g;
g.build()"`` or ``paper_2405_18966_gb300.build.build()``); importing the
binding without it raises, there is no fallback.

Matrices are given as objects with ``m, n, row_ptr, col_idx, values`` (CSR,
0- or 1-based, numpy arrays on the host or torch CUDA tensors on the device)
or as a 2-D numpy array / torch CUDA tensor (dense, column-major copies are
made as needed).
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsvdsc.so")

OK = 0
NOT_CONVERGED = 1
ERR_ARG, ERR_SIZE, ERR_CSR, ERR_NOMEM, ERR_CUDA, ERR_TIMEOUT, ERR_NONFINITE = -1, -2, -3, -4, -5, -6, -7
CSR_FORMAT, DENSE_FORMAT = 0, 1
FP64, MIXED = 0, 1
F64, F32 = 0, 1

# Every symbol include/svdsc.h declares.
EXPORTS = ("svdsc_create", "svdsc_solve", "svdsc_destroy", "svdsc_strerror", "svdsc_matvec",
           "svdsc_cgs2", "svdsc_small_svd", "svdsc_reserve", "svdsc_cgs2_noalloc",
           "svdsc_gemm", "svdsc_batch_create", "svdsc_batch_solve", "svdsc_batch_tuning",
           "svdsc_batch_destroy", "svdsc_solve_batched", "svdsc_batch_layout", "svdsc_batch_profile",
           "svdsc_batch_phase_cycles", "svdsc_batch_handoff", "svdsc_batch_lead",
           "svdsc_selftest_wait")


class SvdscMatrix(C.Structure):
    _fields_ = [("format", C.c_int32), ("index_base", C.c_int32), ("m", C.c_int64),
                ("n", C.c_int64), ("nnz", C.c_int64), ("row_ptr", C.c_void_p),
                ("row_begin", C.c_void_p), ("row_end", C.c_void_p), ("col_idx", C.c_void_p),
                ("values", C.c_void_p), ("value_type", C.c_int32), ("on_device", C.c_int32),
                ("dense", C.c_void_p), ("ld", C.c_int64)]


class SvdscOptions(C.Structure):
    _fields_ = [("precision", C.c_int32), ("timing", C.c_int32), ("seed", C.c_uint64),
                ("restart_gemm", C.c_int32), ("batch_cluster", C.c_int32), ("which", C.c_int32),
                ("reorth", C.c_int32), ("block", C.c_int32), ("batch_handoff", C.c_int32),
                ("batch_order", C.c_int32), ("batch_lead", C.c_int32)]


NUM_PHASES = 8
PHASES = ("spmv", "gemv_t", "gemv_n", "vec", "svd", "gemm", "other", "unused")


class SvdscInfo(C.Structure):
    _fields_ = [("converged", C.c_int32), ("nconv", C.c_int32), ("restarts", C.c_int32),
                ("breakdowns", C.c_int32), ("n_matvec", C.c_int64), ("n_steps", C.c_int64),
                ("n_launches", C.c_int64), ("anorm_est", C.c_double), ("beta_t", C.c_double),
                ("t", C.c_int32), ("reserved", C.c_int32),
                ("ms", C.c_double * NUM_PHASES), ("launches", C.c_int64 * NUM_PHASES),
                ("bytes", C.c_double * NUM_PHASES), ("flops", C.c_double * NUM_PHASES),
                ("n_reorth", C.c_int64)]

    def as_dict(self):
        d = {f: getattr(self, f) for f, _ in self._fields_
             if f not in ("reserved", "ms", "launches", "bytes", "flops")}
        for f in ("ms", "launches", "bytes", "flops"):
            arr = getattr(self, f)
            d[f] = {PHASES[i]: arr[i] for i in range(NUM_PHASES - 1)}
        return d


_lib = None


def lib():
    """Loads libsvdsc.so; raises if it was not built (no CPU fallback exists)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsvdsc.so not built ({LIB_PATH}); run paper_2405_18966_gb300.build.build()")
        L = C.CDLL(LIB_PATH)
        vp, i64, dbl, i32 = C.c_void_p, C.c_int64, C.c_double, C.c_int
        L.svdsc_create.argtypes = [C.POINTER(vp), C.POINTER(SvdscMatrix), C.POINTER(SvdscOptions), vp]
        L.svdsc_solve.argtypes = [vp, i32, i32, dbl, i32, vp, i32, vp, vp, i64, vp, i64, vp, i32,
                                  C.POINTER(SvdscInfo)]
        L.svdsc_destroy.argtypes = [vp]
        L.svdsc_strerror.argtypes = [i32]
        L.svdsc_strerror.restype = C.c_char_p
        L.svdsc_matvec.argtypes = [vp, i32, vp, vp, dbl, vp]
        L.svdsc_cgs2.argtypes = [vp, i64, i64, vp, i64, vp, vp]
        L.svdsc_small_svd.argtypes = [vp, i32, vp, i64, vp, vp, vp]
        L.svdsc_reserve.argtypes = [vp, i32]
        L.svdsc_cgs2_noalloc.argtypes = [i64, i64, vp, i64, vp, vp, vp]
        L.svdsc_gemm.argtypes = [vp, i32, i64, i32, i32, vp, i64, vp, i64, vp, i64]
        L.svdsc_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(SvdscMatrix), vp, vp,
                                         C.POINTER(SvdscOptions), vp]
        L.svdsc_batch_solve.argtypes = [vp, dbl, i32, vp, vp, vp, vp, i32, C.POINTER(SvdscInfo)]
        L.svdsc_batch_tuning.argtypes = [vp, i32, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                         C.POINTER(dbl)]
        L.svdsc_batch_destroy.argtypes = [vp]
        L.svdsc_batch_layout.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.svdsc_batch_profile.argtypes = [vp, vp, vp, vp, vp]
        L.svdsc_batch_phase_cycles.argtypes = [vp, vp]
        L.svdsc_batch_handoff.argtypes = [vp, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32)]
        L.svdsc_batch_lead.argtypes = [vp, C.POINTER(i32), C.POINTER(i32)]
        L.svdsc_selftest_wait.argtypes = [vp, i32]
        L.svdsc_solve_batched.argtypes = [i32, C.POINTER(SvdscMatrix), vp, vp, dbl, i32, vp, vp, vp, vp,
                                          i32, C.POINTER(SvdscOptions), C.POINTER(SvdscInfo)]
        for name in EXPORTS:
            getattr(L, name).restype = getattr(L, name).restype or C.c_int
        L.svdsc_strerror.restype = C.c_char_p
        _lib = L
    return _lib


class SvdscError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().svdsc_strerror(status).decode()
        super().__init__(f"{where}: {msg} (status {status})")
        self.status = status


def _check(status: int, where: str) -> int:
    if status < 0:
        raise SvdscError(status, where)
    return status


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    if x is None:
        return None
    if _is_torch(x):
        return C.c_void_p(x.data_ptr())
    return x.ctypes.data_as(C.c_void_p)


@dataclass
class Result:
    S: object
    U: object
    V: object
    res: object
    info: dict
    status: int


class Solver:
    """A matrix prepared on the device (svdsc_create) that can be solved many times."""

    def __init__(self, A, precision: str = "fp64", seed: int = 0, stream=None, timing: bool = False,
                 restart_gemm: str = "tensor", which: str = "largest", reorth: str = "full",
                 block: int = 1):
        self._keep = []
        self.handle = C.c_void_p()
        prec = {"fp64": FP64, "mixed": MIXED}[precision]
        mat = SvdscMatrix()
        if hasattr(A, "row_ptr"):
            on_dev = _is_torch(A.row_ptr) and A.row_ptr.is_cuda
            rp, ci, va = A.row_ptr, A.col_idx, A.values
            if not on_dev:
                rp = np.ascontiguousarray(rp, dtype=np.int64)
                ci = np.ascontiguousarray(ci, dtype=np.int32)
                va = np.ascontiguousarray(va)
                if va.dtype not in (np.float64, np.float32):
                    va = va.astype(np.float64)
            vt = F32 if str(va.dtype).endswith("float32") else F64
            self._keep += [rp, ci, va]
            mat.format, mat.index_base = CSR_FORMAT, int(getattr(A, "index_base", 0))
            mat.m, mat.n = int(A.m), int(A.n)
            mat.nnz = int(getattr(A, "nnz", 0))
            mat.row_ptr, mat.col_idx, mat.values = _ptr(rp), _ptr(ci), _ptr(va)
            mat.value_type, mat.on_device = vt, int(on_dev)
            self.m, self.n = int(A.m), int(A.n)
        else:
            a = A.a if hasattr(A, "a") else A
            on_dev = _is_torch(a) and a.is_cuda
            if on_dev:
                at = a.t().contiguous()  # column-major storage of a
                self._keep.append(at)
                mat.dense, mat.ld = _ptr(at), a.shape[0]
            else:
                at = np.asfortranarray(a, dtype=np.float64)
                self._keep.append(at)
                mat.dense, mat.ld = _ptr(at), at.shape[0]
            mat.format, mat.on_device = DENSE_FORMAT, int(on_dev)
            mat.m, mat.n = a.shape[0], a.shape[1]
            mat.value_type = F64
            self.m, self.n = int(a.shape[0]), int(a.shape[1])
        opt = SvdscOptions(prec, int(timing), seed, {"tensor": 0, "fma": 1}[restart_gemm], 0,
                           {"largest": 0, "smallest": 1}[which], {"full": 0, "partial": 1}[reorth],
                           int(block))
        self.block = int(block)
        st = None if stream is None else C.c_void_p(int(stream))
        self.stream = stream
        _check(lib().svdsc_create(C.byref(self.handle), C.byref(mat), C.byref(opt), st), "svdsc_create")
        self._keep = []  # create copied everything

    def close(self):
        if self.handle:
            lib().svdsc_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def solve(self, k: int, p: int = -1, tol: float = 1e-10, maxit: int = 100, v0=None,
              out: str = "host", outputs=None) -> Result:
        """Alg. 2: k largest (or, for which='smallest', k smallest, S ascending)
        singular triplets.  out='host' returns numpy arrays,
        out='device' torch CUDA tensors (or writes into `outputs` = (S, U, V, res)
        preallocated with the matching placement, U/V column-major)."""
        info = SvdscInfo()
        if outputs is not None:
            S, U, V, res = outputs
            on_dev = _is_torch(S)
        elif out == "host":
            S, res = np.zeros(k), np.zeros(k)
            U = np.zeros((self.m, k), order="F")
            V = np.zeros((self.n, k), order="F")
            on_dev = False
        else:
            import torch
            dev = torch.device("cuda", torch.cuda.current_device())
            S = torch.zeros(k, dtype=torch.float64, device=dev)
            res = torch.zeros(k, dtype=torch.float64, device=dev)
            U = torch.zeros((k, self.m), dtype=torch.float64, device=dev)  # column-major m x k
            V = torch.zeros((k, self.n), dtype=torch.float64, device=dev)
            on_dev = True
        v0p, v0dev = None, 0
        if v0 is not None:
            # block form: an n x b start block, passed column-major
            if _is_torch(v0):
                if v0.dim() == 2:
                    v0 = v0.t().contiguous()
                v0p, v0dev = _ptr(v0), int(v0.is_cuda)
            else:
                v0 = np.asfortranarray(v0, dtype=np.float64)
                v0p = _ptr(v0)
        status = _check(lib().svdsc_solve(self.handle, k, p, tol, maxit, v0p, v0dev, _ptr(S), _ptr(U),
                                          self.m, _ptr(V), self.n, _ptr(res), int(on_dev),
                                          C.byref(info)), "svdsc_solve")
        if on_dev and outputs is None:
            U, V = U.t(), V.t()  # views: m x k and n x k
        return Result(S, U, V, res, info.as_dict(), status)

    # -- component entry points (device tensors)
    def matvec(self, x, trans: bool = False, z=None, coef: float = 0.0):
        import torch
        y = torch.empty(self.n if trans else self.m, dtype=torch.float64, device=x.device)
        _check(lib().svdsc_matvec(self.handle, int(trans), _ptr(x), _ptr(z), coef, _ptr(y)), "svdsc_matvec")
        return y

    def reserve(self, t: int):
        _check(lib().svdsc_reserve(self.handle, t), "svdsc_reserve")

    def cgs2(self, Wt, w):
        """Wt: (ncols, ldw) torch tensor = column-major basis; w: length-len vector (modified copy)."""
        import torch
        w = w.clone()
        nrm = torch.empty(1, dtype=torch.float64, device=w.device)
        ncols, ldw = Wt.shape
        _check(lib().svdsc_cgs2(self.handle, w.numel(), ncols, _ptr(Wt), ldw, _ptr(w), _ptr(nrm)),
               "svdsc_cgs2")
        return w, float(nrm.item())

    def gemm(self, W, Q, mode: int = 0):
        """C = W Q on the tensor cores (W: rows x t, Q: t x k torch CUDA float64)."""
        import torch
        rows, t = W.shape
        k = Q.shape[1]
        Wc = W.t().contiguous()  # column-major storage
        Qc = Q.t().contiguous()
        Ct = torch.empty((k, rows), dtype=torch.float64, device=W.device)
        _check(lib().svdsc_gemm(self.handle, mode, rows, t, k, _ptr(Wc), rows, _ptr(Qc), t, _ptr(Ct), rows),
               "svdsc_gemm")
        return Ct.t()

    def selftest_wait(self, kind: int) -> int:
        """Makes one bounded device wait run out on purpose (0: grid barrier,
        1: mbarrier); returns the status code (TIMEOUT is the designed outcome)."""
        return lib().svdsc_selftest_wait(self.handle, int(kind))

    def small_svd(self, T):
        """T: t x t torch CUDA float64 tensor; returns (S, Uh, Vh) with T = Uh diag(S) Vh^T."""
        import torch
        t = T.shape[0]
        Tc = T.t().contiguous()  # column-major
        S = torch.empty(t, dtype=torch.float64, device=T.device)
        Uh = torch.empty((t, t), dtype=torch.float64, device=T.device)
        Vh = torch.empty((t, t), dtype=torch.float64, device=T.device)
        _check(lib().svdsc_small_svd(self.handle, t, _ptr(Tc), t, _ptr(S), _ptr(Uh), _ptr(Vh)),
               "svdsc_small_svd")
        return S, Uh.t(), Vh.t()


def _csr_struct(A, keep):
    """SvdscMatrix for a host CSR object (values kept as float32 or float64)."""
    rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
    ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
    va = np.ascontiguousarray(A.values)
    if va.dtype not in (np.float64, np.float32):
        va = va.astype(np.float64)
    keep += [rp, ci, va]
    mat = SvdscMatrix()
    mat.format, mat.index_base = CSR_FORMAT, int(getattr(A, "index_base", 0))
    mat.m, mat.n = int(A.m), int(A.n)
    mat.row_ptr, mat.col_idx, mat.values = _ptr(rp), _ptr(ci), _ptr(va)
    mat.value_type = F32 if va.dtype == np.float32 else F64
    return mat


class Batch:
    """Many truncated SVDs in one persistent launch (svdsc_batch_*), mixed precision.
    handoff: 0 automatic, -1 never, h > 0 hand the running matrices to a second
    launch of 8-CTA clusters once h clusters of the first are idle.
    order: 0 queue by the previous solve's measured cycles (the size estimate
    for the first solve), 1 by the estimate always.
    lead: 0 automatic, -1 none, n > 0 lead clusters of 8 CTAs beside the main launch."""

    def __init__(self, mats, k, p=None, seed: int = 0, cluster: int = 0, handoff: int = 0, order: int = 0,
                 lead: int = 0):
        keep = []
        nb = len(mats)
        arr = (SvdscMatrix * nb)(*[_csr_struct(a, keep) for a in mats])
        self.k = np.ascontiguousarray(k, dtype=np.int32)
        self.p = np.ascontiguousarray(p if p is not None else self.k, dtype=np.int32)
        self.shapes = [(int(a.m), int(a.n)) for a in mats]
        opt = SvdscOptions(MIXED, 0, seed, 0, cluster, 0, 0, 0, handoff, order, lead)
        self.handle = C.c_void_p()
        _check(lib().svdsc_batch_create(C.byref(self.handle), nb, arr, _ptr(self.k), _ptr(self.p),
                                        C.byref(opt), None), "svdsc_batch_create")

    def layout(self):
        a, b = C.c_int(), C.c_int()
        _check(lib().svdsc_batch_layout(self.handle, C.byref(a), C.byref(b)), "svdsc_batch_layout")
        return {"cluster_size": a.value, "clusters": b.value}

    def lead(self):
        """The lead launch: cluster size and cluster count (0: none)."""
        a, b = C.c_int(), C.c_int()
        _check(lib().svdsc_batch_lead(self.handle, C.byref(a), C.byref(b)), "svdsc_batch_lead")
        return {"cluster_size": a.value, "clusters": b.value}

    def handoff(self):
        """Hand-off set-up and the number of matrices handed off in the last solve."""
        a, b, c, d = C.c_int(), C.c_int(), C.c_int(), C.c_int()
        _check(lib().svdsc_batch_handoff(self.handle, C.byref(a), C.byref(b), C.byref(c), C.byref(d)),
               "svdsc_batch_handoff")
        return {"idle_threshold": a.value, "cluster_size": b.value, "clusters": c.value,
                "handed_off": d.value}

    def profile(self):
        nb = len(self.shapes)
        tot, svd, lbp = (np.zeros(nb, dtype=np.int64) for _ in range(3))
        cl = np.zeros(nb, dtype=np.int32)
        _check(lib().svdsc_batch_profile(self.handle, _ptr(tot), _ptr(svd), _ptr(lbp), _ptr(cl)),
               "svdsc_batch_profile")
        ph = np.zeros((nb, 5), dtype=np.int64)
        _check(lib().svdsc_batch_phase_cycles(self.handle, _ptr(ph)), "svdsc_batch_phase_cycles")
        return {"cycles_total": tot, "cycles_svd": svd, "cycles_lbp": lbp, "cluster": cl,
                "cycles_phase": ph}

    def tuning(self, i):
        a, b, c, ms = C.c_int(), C.c_int(), C.c_int(), C.c_double()
        _check(lib().svdsc_batch_tuning(self.handle, i, C.byref(a), C.byref(b), C.byref(c), C.byref(ms)),
               "svdsc_batch_tuning")
        return {"lanes_A": a.value, "lanes_AT": b.value, "gemv_cols": c.value, "tune_ms": ms.value}

    def solve(self, tol: float = 1e-10, maxit: int = 100, out: str = "host"):
        nb = len(self.shapes)
        infos = (SvdscInfo * nb)()
        if out == "host":
            S = [np.zeros(int(k)) for k in self.k]
            R = [np.zeros(int(k)) for k in self.k]
            U = [np.zeros((m, int(k)), order="F") for (m, n), k in zip(self.shapes, self.k)]
            V = [np.zeros((n, int(k)), order="F") for (m, n), k in zip(self.shapes, self.k)]
            on_dev = 0
        else:
            import torch
            S = [torch.zeros(int(k), dtype=torch.float64, device="cuda") for k in self.k]
            R = [torch.zeros(int(k), dtype=torch.float64, device="cuda") for k in self.k]
            U = [torch.zeros((int(k), m), dtype=torch.float64, device="cuda") for (m, n), k in zip(self.shapes, self.k)]
            V = [torch.zeros((int(k), n), dtype=torch.float64, device="cuda") for (m, n), k in zip(self.shapes, self.k)]
            on_dev = 1
        ptrs = lambda xs: (C.c_void_p * nb)(*[_ptr(x).value for x in xs])
        status = _check(lib().svdsc_batch_solve(self.handle, tol, maxit, ptrs(S), ptrs(U), ptrs(V), ptrs(R),
                                                on_dev, infos), "svdsc_batch_solve")
        if on_dev:
            U = [u.t() for u in U]
            V = [v.t() for v in V]
        infl = []
        for i in range(nb):
            d = infos[i].as_dict()
            d["err"] = infos[i].reserved
            infl.append(d)
        return {"S": S, "U": U, "V": V, "res": R, "infos": infl, "status": status}

    def close(self):
        if self.handle:
            lib().svdsc_batch_destroy(self.handle)
            self.handle = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def svds(A, k: int, p: int = -1, tol: float = 1e-10, maxit: int = 100, precision: str = "fp64",
         seed: int = 0, v0=None, out: str = "host", restart_gemm: str = "tensor",
         which: str = "largest", reorth: str = "full", block: int = 1) -> Result:
    """One-shot convenience: create, solve, destroy.  block = b > 1 runs the
    block form (v0, if given, is an n x b start block)."""
    with Solver(A, precision=precision, seed=seed, restart_gemm=restart_gemm, which=which,
                reorth=reorth, block=block) as s:
        return s.solve(k, p, tol, maxit, v0=v0, out=out)
