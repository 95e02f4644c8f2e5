"""FP64 CPU oracle for the diffusion-map H-matvec Lanczos path (ctypes over oracle.c).

TEST INFRASTRUCTURE ONLY. The tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import this package; the product
(``paper_2311_06115_gb300``) never does, and the two share no code.

Every function takes numpy arrays; points are float32 (N, d) C-contiguous (the
product's storage type), all results are float64. Which passage of the paper
each routine follows is stated in oracle.c.

Parity status: every routine here (including the diffusion coordinates and the
intrinsic dimension d(t)) is pinned by a closed form, an invariant, brute force,
exact arithmetic or a library special case in tests/test_oracle_pins.py, except the
paper's own printed accuracy figures (eigenvalue errors of about 9e-4 and 1e-4
in Section 4.1), whose parameters the paper does not give ("parity unpinned").
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess
import sysconfig

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "_liboracle.so")
_lib = None

_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_u64p = C.POINTER(C.c_uint64)


def build(force: bool = False) -> str:
    """Compile oracle.c into _liboracle.so (gcc, FP64, OpenMP, no FMA contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < max(
        os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "oracle.h"))
    ):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is not None:
        return _lib
    build()
    lib = C.CDLL(_LIB_PATH)
    i64, i32, f64, u64, u32 = C.c_int64, C.c_int32, C.c_double, C.c_uint64, C.c_uint32
    sig = {
        "or_splitmix64_next": (u64, [_u64p]),
        "or_stream_key": (u64, [u64, u32, u64]),
        "or_rng": (u64, [u64, u64]),
        "or_sqdist": (f64, [_f32p, i32, i64, i64]),
        "or_median_sqdist": (f64, [_f32p, i64, i32, u64]),
        "or_kernel_W": (None, [_f32p, i64, i32, f64, _f64p]),
        "or_degrees": (None, [_f32p, i64, i32, f64, f64, _f64p, _f64p, _f64p]),
        "or_q_rows": (None, [_f32p, i64, i32, f64, _i64p, i64, _f64p]),
        "or_S_matvec": (None, [_f32p, i64, i32, f64, _f64p, _f64p, i32, _f64p]),
        "or_S_matvec_rows": (None, [_f32p, i64, i32, f64, _f64p, _f64p, _i64p, i64, _f64p]),
        "or_tree_depth": (i32, [i64, i64]),
        "or_node_range": (None, [i64, i32, C.POINTER(i64), C.POINTER(i64)]),
        "or_tree": (i32, [_f32p, i64, i32, f64, i64, _i32p]),
        "or_skeletonize": (i32, [_f32p, i64, i32, f64, _f64p, _i32p, i32, f64, i32, i32, u64, _i32p, _i32p, _f64p]),
        "or_hmatvec": (None, [_f32p, i64, i32, f64, _f64p, _i32p, i32, i32, i32, _i32p, _i32p, _f64p, _f64p, i32,
                              _f64p]),
        "or_jacobi": (i32, [_f64p, i32, _f64p, _f64p]),
        "or_lanczos_dense": (i32, [_f64p, i64, i32, i32, f64, _f64p, _f64p, _f64p, C.POINTER(i32)]),
        "or_lanczos_S": (i32, [_f32p, i64, i32, f64, _f64p, i32, i32, f64, _f64p, _f64p, _f64p, C.POINTER(i32)]),
        "or_lanczos_hmat": (i32, [_f32p, i64, i32, f64, _f64p, _i32p, i32, i32, i32, _i32p, _i32p, _f64p,
                                  i32, i32, f64, _f64p, _f64p, _f64p, C.POINTER(i32)]),
        "or_start_vector": (None, [i64, u64, _f64p]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _pts(X) -> np.ndarray:
    X = np.ascontiguousarray(X, dtype=np.float32)
    if X.ndim != 2:
        raise ValueError("points must be (N, d)")
    return X


def splitmix64_sequence(state: int, count: int) -> list[int]:
    """Outputs of the sequential SplitMix64 generator started at `state`."""
    st = C.c_uint64(state)
    return [int(_load().or_splitmix64_next(C.byref(st))) for _ in range(count)]


def stream_key(seed: int, tag: int, ident: int) -> int:
    return int(_load().or_stream_key(seed, tag, ident))


def rng(key: int, ctr: int) -> int:
    return int(_load().or_rng(key, ctr))


def sqdist(X, i: int, j: int) -> float:
    X = _pts(X)
    return float(_load().or_sqdist(X, X.shape[1], i, j))


def median_sqdist(X, seed: int = 0) -> float:
    """eps = median squared pairwise distance (all pairs up to 2^20 of them, else 2^20 seeded pairs)."""
    X = _pts(X)
    return float(_load().or_median_sqdist(X, X.shape[0], X.shape[1], seed))


def kernel_W(X, eps: float) -> np.ndarray:
    X = _pts(X)
    n = X.shape[0]
    W = np.empty((n, n), dtype=np.float64)
    _load().or_kernel_W(X, n, X.shape[1], eps, W)
    return W


def degrees(X, eps: float, alpha: float = 1.0):
    """(q, dg, s): q = W 1, dg = W^alpha 1, s = q^-alpha dg^-1/2 (Algorithm 1: similarity matrix and normalisations)."""
    X = _pts(X)
    n = X.shape[0]
    q, dg, s = (np.empty(n, dtype=np.float64) for _ in range(3))
    _load().or_degrees(X, n, X.shape[1], eps, alpha, q, dg, s)
    return q, dg, s


def q_rows(X, eps: float, rows) -> np.ndarray:
    X = _pts(X)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.shape[0], dtype=np.float64)
    _load().or_q_rows(X, X.shape[0], X.shape[1], eps, rows, rows.shape[0], out)
    return out


def S_matvec(X, eps: float, s, x) -> np.ndarray:
    """Exact y = S x on the fly; x is (N,) or (N, nrhs)."""
    X = _pts(X)
    n = X.shape[0]
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    xm = x.reshape(n, -1)
    nrhs = xm.shape[1]
    xc = np.ascontiguousarray(xm.T)  # column-major as contiguous columns
    y = np.empty_like(xc)
    _load().or_S_matvec(X, n, X.shape[1], eps, np.ascontiguousarray(s, dtype=np.float64), xc, nrhs, y)
    y = y.T
    return y[:, 0].copy() if squeeze else np.ascontiguousarray(y)


def S_matvec_rows(X, eps: float, s, x, rows) -> np.ndarray:
    X = _pts(X)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty(rows.shape[0], dtype=np.float64)
    _load().or_S_matvec_rows(X, X.shape[0], X.shape[1], eps, np.ascontiguousarray(s, dtype=np.float64),
                             np.ascontiguousarray(x, dtype=np.float64), rows, rows.shape[0], out)
    return out


def tree_depth(n: int, leaf_size: int) -> int:
    return int(_load().or_tree_depth(n, leaf_size))


def node_range(n: int, node: int) -> tuple[int, int]:
    st, sz = C.c_int64(), C.c_int64()
    _load().or_node_range(n, node, C.byref(st), C.byref(sz))
    return int(st.value), int(sz.value)


def tree(X, eps: float, leaf_size: int):
    """(perm, L): perm[pos] = original index; L the depth of the perfect binary tree."""
    X = _pts(X)
    n = X.shape[0]
    perm = np.empty(n, dtype=np.int32)
    L = _load().or_tree(X, n, X.shape[1], eps, leaf_size, perm)
    return perm, int(L)


class HStructure:
    """The oracle's compressed representation: tree + per-node skeletons and P."""

    def __init__(self, perm, L, max_rank, cmax, ranks, skel, P):
        self.perm, self.L, self.max_rank, self.cmax = perm, L, max_rank, cmax
        self.ranks, self.skel, self.P = ranks, skel, P

    @property
    def nnodes(self) -> int:
        return (1 << (self.L + 1)) - 1


def leaf_max(n: int, L: int) -> int:
    return -(-n // (1 << L))


def skeletonize(X, eps: float, s, perm, L: int, tol: float, max_rank: int, seed: int = 0) -> HStructure:
    X = _pts(X)
    n = X.shape[0]
    cmax = max(leaf_max(n, L), 2 * max_rank)
    nn = (1 << (L + 1)) - 1
    ranks = np.zeros(nn, dtype=np.int32)
    skel = np.full(nn * max_rank, -1, dtype=np.int32)
    P = np.zeros(nn * max_rank * cmax, dtype=np.float64)
    _load().or_skeletonize(X, n, X.shape[1], eps, np.ascontiguousarray(s, dtype=np.float64),
                           np.ascontiguousarray(perm, dtype=np.int32), L, tol, max_rank, cmax, seed, ranks, skel, P)
    return HStructure(np.ascontiguousarray(perm, dtype=np.int32), L, max_rank, cmax, ranks, skel, P)


def compress(X, eps: float, s, leaf_size: int, tol: float, max_rank: int, seed: int = 0) -> HStructure:
    perm, L = tree(X, eps, leaf_size)
    return skeletonize(X, eps, s, perm, L, tol, max_rank, seed)


def hmatvec(X, eps: float, s, H: HStructure, x) -> np.ndarray:
    X = _pts(X)
    n = X.shape[0]
    x = np.asarray(x, dtype=np.float64)
    squeeze = x.ndim == 1
    xm = x.reshape(n, -1)
    nrhs = xm.shape[1]
    xc = np.ascontiguousarray(xm.T)
    y = np.empty_like(xc)
    _load().or_hmatvec(X, n, X.shape[1], eps, np.ascontiguousarray(s, dtype=np.float64), H.perm, H.L, H.max_rank,
                       H.cmax, H.ranks, H.skel, H.P, xc, nrhs, y)
    y = y.T
    return y[:, 0].copy() if squeeze else np.ascontiguousarray(y)


def jacobi(A):
    """(evals descending, evecs as columns) of a dense symmetric matrix by cyclic Jacobi."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    ev = np.empty(n, dtype=np.float64)
    V = np.empty((n, n), dtype=np.float64)
    _load().or_jacobi(A, n, ev, V)
    return ev, V


def start_vector(n: int, seed: int = 0) -> np.ndarray:
    v = np.empty(n, dtype=np.float64)
    _load().or_start_vector(n, seed, v)
    return v


def _lanczos_out(n, k):
    return np.empty(k, dtype=np.float64), np.empty((k, n), dtype=np.float64), C.c_int32()


def lanczos_dense(A, k: int, m_max: int = 300, conv_tol: float = 1e-10, v0=None, seed: int = 0):
    """Top-k eigenpairs of a dense symmetric matrix by full-reorthogonalisation Lanczos.

    Returns (evals, evecs (n, k), iterations, status) with status 0 when converged."""
    A = np.ascontiguousarray(A, dtype=np.float64)
    n = A.shape[0]
    v0 = start_vector(n, seed) if v0 is None else np.ascontiguousarray(v0, dtype=np.float64)
    ev, V, it = _lanczos_out(n, k)
    st = _load().or_lanczos_dense(A, n, k, m_max, conv_tol, v0, ev, V, C.byref(it))
    return ev, np.ascontiguousarray(V.T), int(it.value), int(st)


def lanczos_S(X, eps: float, s, k: int, m_max: int = 300, conv_tol: float = 1e-10, seed: int = 0):
    """Top-k eigenpairs of the exact S (entries on the fly)."""
    X = _pts(X)
    n = X.shape[0]
    v0 = start_vector(n, seed)
    ev, V, it = _lanczos_out(n, k)
    st = _load().or_lanczos_S(X, n, X.shape[1], eps, np.ascontiguousarray(s, dtype=np.float64), k, m_max,
                              conv_tol, v0, ev, V, C.byref(it))
    return ev, np.ascontiguousarray(V.T), int(it.value), int(st)


def lanczos_hmat(X, eps: float, s, H: HStructure, k: int, m_max: int = 300, conv_tol: float = 1e-10,
                 seed: int = 0):
    """Top-k eigenpairs of the oracle's H-matrix approximation of S."""
    X = _pts(X)
    n = X.shape[0]
    v0 = start_vector(n, seed)
    ev, V, it = _lanczos_out(n, k)
    st = _load().or_lanczos_hmat(X, n, X.shape[1], eps, np.ascontiguousarray(s, dtype=np.float64), H.perm, H.L,
                                 H.max_rank, H.cmax, H.ranks, H.skel, H.P, k, m_max, conv_tol, v0, ev, V,
                                 C.byref(it))
    return ev, np.ascontiguousarray(V.T), int(it.value), int(st)


def hmatvec_error_2norm(X, eps: float, s, H: HStructure, iters: int = 60, seed: int = 0) -> float:
    """Estimate of ||S~ - S||_2 for the H-matrix H (Eq. 1.1's error in the operator 2-norm; also
    the relative error, since ||S||_2 = lambda_1 = 1): power iteration on (S~ - S)^2 with the
    exact S on the fly. The estimate |E v| / |v| of a unit iterate v is a lower bound that
    rises towards the largest singular value of E = S~ - S."""
    n = _pts(X).shape[0]
    v = start_vector(n, seed)
    v /= np.linalg.norm(v)
    est = 0.0
    for _ in range(iters):
        ev = hmatvec(X, eps, s, H, v) - S_matvec(X, eps, s, v)
        est = float(np.linalg.norm(ev))
        w = hmatvec(X, eps, s, H, ev) - S_matvec(X, eps, s, ev)
        nw = float(np.linalg.norm(w))
        if nw == 0.0:
            break
        v = w / nw
    return est


def diffusion_coords(evals, phi, dg, t: int = 1) -> np.ndarray:
    """Diffusion coordinates after t steps of the walk (Algorithm 1, P^t and its
    eigendecomposition): P = Dg^-1 W^alpha = Dg^-1/2 S Dg^1/2, so P's right eigenvectors
    are Dg^-1/2 phi for eigenvectors phi of S, with P^t's eigenvalues theta^t;
    psi_i = theta_i^t Dg^-1/2 phi_i. phi: (N, k); returns (N, k) float64."""
    ev = np.asarray(evals, dtype=np.float64)
    return (ev ** t)[None, :] * np.asarray(phi, dtype=np.float64) / np.sqrt(np.asarray(dg, dtype=np.float64))[:, None]


def intrinsic_dim(evals, t: int, delta: float) -> tuple[int, bool]:
    """Intrinsic dimension d(t) of Algorithm 1 (its lower dimension), in Coifman and Lafon's form
    (the printed inequality is garbled and delta is not given): eigenvalues indexed from
    the trivial one, lambda_0 = evals[0]; d(t) = the largest l >= 1 with
    |lambda_l|^t > delta |lambda_1|^t, tested as t log(|lambda_l| / |lambda_1|) > log(delta)
    (the same comparison without the range limits of the t-th powers). Also returns
    whether every eigenvalue given passed (the true d(t) may then be larger)."""
    lam = [float(v) for v in evals]
    l1 = abs(lam[1])
    d = 0
    if l1 > 0.0:
        for l in range(1, len(lam)):
            r = abs(lam[l]) / l1
            if r > 0.0 and t * math.log(r) > math.log(delta):
                d = l
    return d, d == len(lam) - 1


def threads() -> int:
    """OpenMP threads the oracle uses (OMP_NUM_THREADS, else the CPUs this process may run on)."""
    env = os.environ.get("OMP_NUM_THREADS")
    if env:
        return int(env)
    return len(os.sched_getaffinity(0))


__all__ = [n for n in dir() if not n.startswith("_") and n not in ("C", "np", "os", "subprocess", "sysconfig")]
