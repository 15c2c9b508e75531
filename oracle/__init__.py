"""CPU oracle of the truncated SVD method of the svds-C paper (arXiv 2405.18966).

TEST INFRASTRUCTURE ONLY.  The oracle is a plain, slow FP64 C implementation
(``svds_oracle.c``) of Alg. 1 (Lanczos bidiagonalization), the full
re-orthogonalization of Sec. 2.1 (as two classical Gram-Schmidt passes), the
residual test of Eq. (4) and the augmented restart of Eq. (5)-(7) / Alg. 2,
plus a one-sided Jacobi dense SVD used for the projected matrix and as a
brute-force checker.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA solver and never imports it.

Matrices are passed as any object with ``m, n, row_ptr, col_idx, values``
(0-based CSR, int64 row pointers, int32 column indices) or ``m, n, a``
(column-major float64), or as a 2-D numpy array (treated as dense).
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "svds_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (OpenMP, strict FP64: no contraction into FMA)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
           "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Mat(C.Structure):
    _fields_ = [("kind", C.c_int32), ("pad", C.c_int32), ("m", C.c_int64), ("n", C.c_int64),
                ("row_ptr", C.c_void_p), ("col_idx", C.c_void_p), ("val", C.c_void_p),
                ("a", C.c_void_p), ("lda", C.c_int64)]


class Info(C.Structure):
    _fields_ = [("converged", C.c_int32), ("nconv", C.c_int32), ("restarts", C.c_int32),
                ("breakdowns", C.c_int32), ("n_matvec", C.c_int64), ("n_steps", C.c_int64),
                ("svd_sweeps_max", C.c_int32), ("stopped_early", C.c_int32),
                ("anorm_est", C.c_double), ("beta_t", C.c_double), ("n_reorth", C.c_int64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
            L.orc_matvec.argtypes = [C.POINTER(_Mat), vp, vp]
            L.orc_matvec_t.argtypes = [C.POINTER(_Mat), vp, vp]
            L.orc_gemv_t.argtypes = [i64, i64, vp, i64, vp, vp]
            L.orc_gemv_n_sub.argtypes = [i64, i64, vp, i64, vp, vp]
            L.orc_cgs2.argtypes = [i64, i64, vp, i64, vp, vp]
            L.orc_norm2.argtypes = [i64, vp]
            L.orc_norm2.restype = dbl
            L.orc_gemm_nn.argtypes = [i64, i64, i64, vp, i64, vp, i64, vp, i64]
            L.orc_rng_normal.argtypes = [C.c_uint64, C.c_uint64, C.c_uint64]
            L.orc_rng_normal.restype = dbl
            L.orc_splitmix64.argtypes = [C.c_uint64]
            L.orc_splitmix64.restype = C.c_uint64
            L.orc_rng_vector.argtypes = [C.c_uint64, C.c_uint64, i64, vp]
            L.orc_jacobi_svd.argtypes = [i64, i64, vp, i64, vp, vp, i64, vp, i64, C.c_int]
            L.orc_jacobi_svd.restype = C.c_int
            L.orc_sign_normalize.argtypes = [i64, i64, i64, vp, i64, vp, i64]
            L.orc_svds.argtypes = [C.POINTER(_Mat), i64, i64, dbl, i64, i64, i64, C.c_uint64, vp, i64,
                                   vp, vp, i64, vp, i64, vp, C.POINTER(Info), vp, vp, vp, vp, vp]
            L.orc_svds.restype = C.c_int
            L.orc_svds_block.argtypes = [C.POINTER(_Mat), i64, i64, i64, dbl, i64, C.c_uint64, vp, vp, vp,
                                         i64, vp, i64, vp, C.POINTER(Info), vp, vp, vp, vp]
            L.orc_svds_block.restype = C.c_int
            L.orc_set_threads.argtypes = [C.c_int]
            for f in ("orc_pr_nu_step", "orc_pr_mu_step"):
                getattr(L, f).argtypes = [i64, vp, i64, vp, vp, dbl, dbl]
                getattr(L, f).restype = dbl
            L.orc_get_threads.restype = C.c_int
            _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


class _Bound:
    """Keeps the numpy arrays a _Mat points into alive."""

    def __init__(self, A):
        if isinstance(A, np.ndarray):
            a = np.asfortranarray(A, dtype=np.float64)
            self.keep = [a]
            self.mat = _Mat(1, 0, a.shape[0], a.shape[1], None, None, None,
                            a.ctypes.data, a.shape[0])
        elif hasattr(A, "row_ptr"):
            rp = np.ascontiguousarray(A.row_ptr, dtype=np.int64)
            ci = np.ascontiguousarray(A.col_idx, dtype=np.int32)
            va = np.ascontiguousarray(A.values, dtype=np.float64)
            self.keep = [rp, ci, va]
            self.mat = _Mat(0, 0, int(A.m), int(A.n), rp.ctypes.data, ci.ctypes.data,
                            va.ctypes.data, None, 0)
        else:
            a = np.asfortranarray(A.a, dtype=np.float64)
            self.keep = [a]
            self.mat = _Mat(1, 0, a.shape[0], a.shape[1], None, None, None,
                            a.ctypes.data, a.shape[0])
        self.m, self.n = int(self.mat.m), int(self.mat.n)


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def get_threads() -> int:
    return int(lib().orc_get_threads())


def matvec(A, x):
    """y = A x (Alg. 1)."""
    b = _Bound(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(b.m)
    lib().orc_matvec(C.byref(b.mat), _ptr(x), _ptr(y))
    return y


def matvec_t(A, x):
    """y = A^T x (Alg. 1)."""
    b = _Bound(A)
    x = np.ascontiguousarray(x, dtype=np.float64)
    y = np.empty(b.n)
    lib().orc_matvec_t(C.byref(b.mat), _ptr(x), _ptr(y))
    return y


def gemv_t(W, w):
    W = np.asfortranarray(W, dtype=np.float64)
    w = np.ascontiguousarray(w, dtype=np.float64)
    h = np.empty(W.shape[1])
    lib().orc_gemv_t(W.shape[0], W.shape[1], _ptr(W), W.shape[0], _ptr(w), _ptr(h))
    return h


def gemv_n_sub(W, h, w):
    """w - W h."""
    W = np.asfortranarray(W, dtype=np.float64)
    h = np.ascontiguousarray(h, dtype=np.float64)
    w = np.array(w, dtype=np.float64, copy=True)
    lib().orc_gemv_n_sub(W.shape[0], W.shape[1], _ptr(W), W.shape[0], _ptr(h), _ptr(w))
    return w


def cgs2(W, w):
    """(I - W W^T) applied twice to w (Sec. 2.1 full re-orthogonalization)."""
    W = np.asfortranarray(W, dtype=np.float64)
    w = np.array(w, dtype=np.float64, copy=True)
    h = np.empty(max(1, W.shape[1]))
    lib().orc_cgs2(W.shape[0], W.shape[1], _ptr(W), W.shape[0], _ptr(w), _ptr(h))
    return w


def norm2(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    return float(lib().orc_norm2(x.size, _ptr(x)))


def gemm(W, Q):
    W = np.asfortranarray(W, dtype=np.float64)
    Q = np.asfortranarray(Q, dtype=np.float64)
    out = np.empty((W.shape[0], Q.shape[1]), order="F")
    lib().orc_gemm_nn(W.shape[0], W.shape[1], Q.shape[1], _ptr(W), W.shape[0], _ptr(Q),
                      Q.shape[0], _ptr(out), W.shape[0])
    return out


def splitmix64(x: int) -> int:
    """SplitMix64 output for state x (golden-ratio increment, then finaliser)."""
    return int(lib().orc_splitmix64(C.c_uint64(x)))


def rng_normal(seed: int, draw: int, n: int):
    """The counter-based N(0,1) vector (SplitMix64 + Box-Muller) the method draws."""
    x = np.empty(n)
    lib().orc_rng_vector(C.c_uint64(seed), C.c_uint64(draw), n, _ptr(x))
    return x


def jacobi_svd(A, max_sweeps: int = 100):
    """One-sided Jacobi SVD (m >= n); returns (U thin, S desc, V, sweeps or -1)."""
    A = np.asfortranarray(A, dtype=np.float64)
    m, n = A.shape
    if m < n:
        U, S, V, sw = jacobi_svd(A.T, max_sweeps)
        return V, S, U, sw
    S = np.empty(n)
    U = np.empty((m, n), order="F")
    V = np.empty((n, n), order="F")
    sw = lib().orc_jacobi_svd(m, n, _ptr(A), m, _ptr(S), _ptr(U), m, _ptr(V), n, max_sweeps)
    return U, S, V, sw


def sign_normalize(U, V):
    U = np.array(U, dtype=np.float64, order="F", copy=True)
    V = np.array(V, dtype=np.float64, order="F", copy=True)
    lib().orc_sign_normalize(U.shape[0], V.shape[0], U.shape[1], _ptr(U), U.shape[0],
                             _ptr(V), V.shape[0])
    return U, V


def pr_nu_step(i: int, T, mu, nu, beta: float, anorm: float) -> float:
    """One step of the partial re-orthogonalization recurrence for v_{i+1}
    (updates nu in place; T column-major (t+1) x (t+1)); returns the largest
    new estimate."""
    T = np.asfortranarray(T, dtype=np.float64)
    return lib().orc_pr_nu_step(i, _ptr(T), T.shape[0], _ptr(mu), _ptr(nu), beta, anorm)


def pr_mu_step(i: int, T, mu, nu, alpha: float, anorm: float) -> float:
    """One step of the recurrence for u_{i+1} (updates mu in place)."""
    T = np.asfortranarray(T, dtype=np.float64)
    return lib().orc_pr_mu_step(i, _ptr(T), T.shape[0], _ptr(mu), _ptr(nu), alpha, anorm)


def subspace_dim(k: int, p: int) -> int:
    return max(15, 3 * k) if p < 0 else k + p


def svds(A, k: int, p: int = -1, tol: float = 1e-10, maxit: int = 100, seed: int = 0,
         v0=None, step_budget: int = -1, return_basis: bool = False, which: str = "largest",
         reorth: str = "full"):
    """Alg. 2 of the paper: k largest singular triplets of A (which="largest"),
    or the k smallest (which="smallest", m >= n; S ascending).  reorth="full"
    re-orthogonalizes every Lanczos vector (CGS2), reorth="partial" only where
    the orthogonality estimates ask for it.

    Returns a dict with S (k), U (m x k), V (n x k), res (k), info (dict) and,
    if ``return_basis``, the final Lanczos basis Ub (m x t), Vb (n x (t+1)),
    projected matrix T ((t+1) x (t+1)) and, for reorth="partial", the last
    orthogonality estimates mu (u_t against u_1..u_{t-1}) and nu (v_{t+1}
    against v_1..v_t).  Raises ValueError on bad arguments."""
    b = _Bound(A)
    m, n = b.m, b.n
    t = subspace_dim(k, p)
    S = np.zeros(k)
    U = np.zeros((m, k), order="F")
    V = np.zeros((n, k), order="F")
    res = np.zeros(k)
    info = Info()
    v0a = None if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    Ub = Vb = Tb = mu = nu = None
    if return_basis:
        Ub = np.zeros((m, t), order="F")
        Vb = np.zeros((n, t + 1), order="F")
        Tb = np.zeros((t + 1, t + 1), order="F")
        mu = np.zeros(t + 2)
        nu = np.zeros(t + 2)
    wh = {"largest": 0, "smallest": 1}[which]
    ro = {"full": 0, "partial": 1}[reorth]
    rc = lib().orc_svds(C.byref(b.mat), k, p, tol, maxit, wh, ro, C.c_uint64(seed), _ptr(v0a),
                        step_budget, _ptr(S), _ptr(U), m, _ptr(V), n, _ptr(res),
                        C.byref(info), _ptr(Ub), _ptr(Vb), _ptr(Tb), _ptr(mu), _ptr(nu))
    if rc == -1:
        raise ValueError("bad arguments (need 1 <= k <= t, t <= m, t + 1 <= n, tol > 0, maxit >= 1; "
                         "m >= n for the smallest triplets)")
    if rc != 0:
        raise MemoryError("oracle ran out of memory")
    out = {"S": S, "U": U, "V": V, "res": res, "info": info.as_dict(), "t": t}
    if return_basis:
        out.update(Ub=Ub, Vb=Vb, T=Tb, mu=mu, nu=nu)
    return out


def block_sizes(k: int, p: int, b: int):
    """(t0, t1): projected sizes of the block form's first pass and of every
    pass after a restart (t = k + p rounded up to whole blocks)."""
    t = subspace_dim(k, p)
    return b * (-(-t // b)), k + b * (-(-(t - k) // b))


def svds_block(A, k: int, p: int = -1, b: int = 1, tol: float = 1e-10, maxit: int = 100,
               seed: int = 0, V0=None, return_basis: bool = False):
    """Block form of Alg. 2 (block Lanczos bidiagonalization, block size b, full
    re-orthogonalization, augmented restart); b = 1 is the single-vector form.
    V0: n x b start block or None (draws 0..b-1).  Returns the dict of svds
    (S, U, V, res, info) plus t_last (size of the last projected matrix) and,
    with return_basis, Ub (m x tmax), Vb (n x (tmax + b)) and T
    ((tmax + b) x (tmax + b)) of the last pass."""
    if b < 1:
        raise ValueError("block size b must be >= 1")
    bd = _Bound(A)
    m, n = bd.m, bd.n
    t0, t1 = block_sizes(k, p, b)
    tmax = max(t0, t1)
    S = np.zeros(k)
    U = np.zeros((m, k), order="F")
    V = np.zeros((n, k), order="F")
    res = np.zeros(k)
    info = Info()
    v0a = None if V0 is None else np.asfortranarray(V0, dtype=np.float64).reshape(n, b, order="F")
    Ub = Vb = Tb = None
    if return_basis:
        Ub = np.zeros((m, tmax), order="F")
        Vb = np.zeros((n, tmax + b), order="F")
        Tb = np.zeros((tmax + b, tmax + b), order="F")
    tl = C.c_int64(0)
    rc = lib().orc_svds_block(C.byref(bd.mat), k, p, b, tol, maxit, C.c_uint64(seed), _ptr(v0a),
                              _ptr(S), _ptr(U), m, _ptr(V), n, _ptr(res), C.byref(info),
                              _ptr(Ub), _ptr(Vb), _ptr(Tb), C.byref(tl))
    if rc == -1:
        raise ValueError("bad arguments (need b >= 1, k + b <= t1, max(t0, t1) <= m, "
                         "max(t0, t1) + b <= n, tol > 0, maxit >= 1)")
    if rc != 0:
        raise MemoryError("oracle ran out of memory")
    out = {"S": S, "U": U, "V": V, "res": res, "info": info.as_dict(), "t0": t0, "t1": t1,
           "t_last": int(tl.value), "b": b}
    if return_basis:
        out.update(Ub=Ub, Vb=Vb, T=Tb)
    return out
