"""Python binding of the GB300 diffusion-map eigensolver (ctypes over libdmaps.so).

The functions carry the names of the C ABI in include/dmaps.h and only marshal
arguments: every step of the computation runs in the CUDA library. Arrays may
be numpy arrays (host) or torch tensors (host or CUDA); the library tells the
two apart by pointer. Device memory the library needs is taken from torch's
caching allocator through the ABI's allocator hooks.

There is no CPU fallback: importing this package raises ImportError when the
CUDA library is missing or cannot be loaded (build it with
``python -m paper_2311_06115_gb300.build``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

__all__ = [
    "DmError", "DM_OK", "DM_EINVAL", "DM_ENOMEM", "DM_ESTATE", "DM_ENOCONV", "DM_ETIMEOUT", "DM_ECUDA", "DM_EBUSY",
    "DM_NEAR_AUTO", "DM_NEAR_CACHED", "DM_NEAR_ONTHEFLY", "DM_PREC_FP32", "DM_PREC_TF32", "DM_PREC_TF32X3", "dm_config", "dm_stats", "lib_path", "load",
    "dm_config_default", "dm_create", "dm_compress", "dm_matvec", "dm_eigs", "dm_coords", "dm_intrinsic_dim",
    "dm_destroy",
    "dm_status_str", "dm_last_error", "dm_get_stats", "dm_get_eps", "dm_get_degrees", "dm_get_tree",
    "dm_get_hmatrix", "dm_load_hmatrix", "dm_kernel_launches", "dm_degrees_noalloc", "dm_request",
    "dm_result", "dm_serve_config", "dm_request_bytes", "dm_serve_start", "dm_serve_stop", "dm_submit", "dm_poll",
    "dm_release", "dm_tune_leaf", "dm_selftest_wait_timeout", "dm_sfu_peak", "dm_eigs_batch",
]

DM_OK, DM_EINVAL, DM_ENOMEM, DM_ESTATE, DM_ENOCONV, DM_ETIMEOUT, DM_ECUDA, DM_EBUSY = 0, -1, -2, -3, -4, -5, -6, -7
DM_NEAR_AUTO, DM_NEAR_CACHED, DM_NEAR_ONTHEFLY = 0, 1, 2
DM_PREC_FP32, DM_PREC_TF32, DM_PREC_TF32X3 = 0, 1, 2

_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)


class dm_config(C.Structure):
    _fields_ = [("seed", C.c_uint64), ("near_mode", C.c_int32), ("m_max", C.c_int32), ("conv_tol", C.c_double),
                ("check_every", C.c_int32), ("device", C.c_int32), ("stream", C.c_void_p), ("alloc", _ALLOC_FN),
                ("free", _FREE_FN), ("alloc_user", C.c_void_p), ("profile", C.c_int32),
                ("shared_device", C.c_int32), ("block_precision", C.c_int32),
                ("block_size", C.c_int32)]


class dm_stats(C.Structure):
    _fields_ = [("N", C.c_int64), ("d", C.c_int32), ("L", C.c_int32), ("eps", C.c_double), ("alpha", C.c_double),
                ("tol", C.c_double), ("leaf_max", C.c_int32), ("max_rank", C.c_int32), ("rank_min", C.c_int32),
                ("rank_max", C.c_int32), ("rank_mean", C.c_double), ("near_bytes", C.c_int64),
                ("basis_bytes", C.c_int64), ("far_bytes", C.c_int64), ("matvec_bytes", C.c_int64),
                ("near_mode", C.c_int32), ("lanczos_iters", C.c_int32), ("converged", C.c_int32),
                ("ms_create", C.c_float), ("ms_tree", C.c_float), ("ms_skeleton", C.c_float),
                ("ms_pack", C.c_float), ("ms_eigs", C.c_float), ("matvec_calls", C.c_int32),
                ("ms_matvec", C.c_float), ("hmatvec_path", C.c_int32), ("degree_path", C.c_int32),
                ("ms_degrees", C.c_float)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


class dm_request(C.Structure):
    _fields_ = [("points", C.c_void_p), ("N", C.c_int64), ("d", C.c_int32), ("eps", C.c_double),
                ("alpha", C.c_double), ("tol", C.c_double), ("leaf_size", C.c_int32), ("max_rank", C.c_int32),
                ("k", C.c_int32), ("want_vectors", C.c_int32), ("seed", C.c_uint64), ("block_size", C.c_int32)]


class dm_result(C.Structure):
    _fields_ = [("status", C.c_int32), ("k", C.c_int32), ("N", C.c_int64), ("evals", C.POINTER(C.c_double)),
                ("evecs", C.POINTER(C.c_float)), ("submit_ms", C.c_double), ("start_ms", C.c_double),
                ("done_ms", C.c_double), ("lanczos_iters", C.c_int32), ("error", C.c_char_p),
                ("built_ms", C.c_double)]


class dm_serve_config(C.Structure):
    _fields_ = [("device", C.c_int32), ("slots", C.c_int32), ("hbm_budget_bytes", C.c_uint64),
                ("queue_capacity", C.c_int32)]


class DmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{dm_status_str(status)}: {msg}")
        self.status = status


_lib = None


def lib_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True):
    """Load libdmaps.so (building it first if it is missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB_PATH
    if not os.path.exists(path) and build_if_missing:
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"CUDA library {path} is missing; build it with python -m paper_2311_06115_gb300.build")
    lib = C.CDLL(path)
    vp, i32, i64, f64 = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "dm_config_default": (None, [C.POINTER(dm_config)]),
        "dm_create": (i32, [vp, i64, i32, f64, f64, C.POINTER(dm_config), C.POINTER(vp)]),
        "dm_compress": (i32, [vp, f64, i32, i32]),
        "dm_matvec": (i32, [vp, vp, vp, i32]),
        "dm_eigs": (i32, [vp, i32, vp, vp]),
        "dm_coords": (i32, [vp, i32, i32, vp]),
        "dm_intrinsic_dim": (i32, [vp, i32, i32, f64, C.POINTER(i32), C.POINTER(i32)]),
        "dm_destroy": (i32, [vp]),
        "dm_status_str": (C.c_char_p, [i32]),
        "dm_last_error": (C.c_char_p, []),
        "dm_get_stats": (i32, [vp, C.POINTER(dm_stats)]),
        "dm_get_eps": (i32, [vp, C.POINTER(f64)]),
        "dm_get_degrees": (i32, [vp, vp, vp, vp]),
        "dm_get_tree": (i32, [vp, C.POINTER(i32), vp]),
        "dm_get_hmatrix": (i32, [vp, vp, vp, vp]),
        "dm_load_hmatrix": (i32, [vp, i32, i32, vp, vp, vp, vp]),
        "dm_kernel_launches": (i64, []),
        "dm_degrees_noalloc": (i32, [vp, i64, i32, f64, f64, vp, vp, vp, vp]),
        "dm_request_bytes": (C.c_uint64, [C.POINTER(dm_request)]),
        "dm_serve_start": (i32, [C.POINTER(dm_serve_config)]),
        "dm_serve_stop": (i32, []),
        "dm_submit": (i32, [C.POINTER(dm_request), C.POINTER(C.c_uint64)]),
        "dm_poll": (i32, [C.c_uint64, C.POINTER(dm_result), C.POINTER(i32)]),
        "dm_release": (i32, [C.c_uint64]),
        "dm_tune_leaf": (i32, [vp, f64, i32, i32, vp, i32, C.POINTER(i32), vp]),
        "dm_selftest_wait_timeout": (i32, [i32, i32, i64, C.POINTER(i32)]),
        "dm_sfu_peak": (i32, [C.POINTER(i64), C.POINTER(C.c_float)]),
        "dm_eigs_batch": (i32, [vp, i32, i32, vp, vp, vp]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def dm_status_str(status: int) -> str:
    return load().dm_status_str(status).decode()


def dm_last_error() -> str:
    return load().dm_last_error().decode()


def _check(status: int, allow=()):
    if status != DM_OK and status not in allow:
        raise DmError(status, dm_last_error())
    return status


# ------------------------------------------------------------------ marshalling helpers

def _torch():
    try:
        import torch
        return torch
    except ImportError:  # numpy-only callers
        return None


def _ptr(a) -> int:
    """Data pointer of a numpy array or a torch tensor (must be contiguous)."""
    t = _torch()
    if t is not None and isinstance(a, t.Tensor):
        if not (a.is_contiguous() or (a.ndim == 2 and a.t().is_contiguous())):
            raise ValueError("tensor must be contiguous (row-major, or column-major for blocks)")
        return a.data_ptr()
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous and not a.flags.f_contiguous:
            raise ValueError("array must be contiguous")
        return a.ctypes.data
    raise TypeError(f"expected numpy array or torch tensor, got {type(a)}")


def _is_cuda(a) -> bool:
    t = _torch()
    return t is not None and isinstance(a, t.Tensor) and a.is_cuda


class _TorchAllocator:
    """Routes the library's device allocations through torch's caching allocator."""

    def __init__(self, device: int, stream):
        torch = _torch()
        self.device = device
        self.stream = stream
        self.live = {}

        def _alloc(nbytes, _user):
            try:
                p = torch.cuda.caching_allocator_alloc(int(nbytes), device=self.device, stream=self.stream)
            except RuntimeError:
                return None
            self.live[int(p)] = int(nbytes)
            return int(p)

        def _free(p, _nbytes, _user):
            if p and int(p) in self.live:
                del self.live[int(p)]
                torch.cuda.caching_allocator_delete(int(p))

        self.alloc_fn = _ALLOC_FN(_alloc)
        self.free_fn = _FREE_FN(_free)


class Handle:
    """Opaque dm_handle plus the Python objects that must outlive it."""

    def __init__(self, ptr: int, keep):
        self.ptr = ptr
        self._keep = keep
        self.N = 0
        self.d = 0

    @property
    def _as_parameter_(self):
        return C.c_void_p(self.ptr)

    def __del__(self):
        if getattr(self, "ptr", None) and _lib is not None:
            try:
                _lib.dm_destroy(C.c_void_p(self.ptr))
            except Exception:
                pass
            self.ptr = None


# ------------------------------------------------------------------ the ABI calls

def dm_config_default(**overrides) -> dm_config:
    cfg = dm_config()
    load().dm_config_default(C.byref(cfg))
    for k, v in overrides.items():
        setattr(cfg, k, v)
    return cfg


def dm_create(points, eps: float = -1.0, alpha: float = 1.0, cfg: dm_config | None = None,
              use_torch_allocator: bool = False) -> Handle:
    """dm_create: points (N, d) float32, host (numpy/torch) or CUDA tensor.

    By default the library allocates from the device's stream-ordered pool; with
    use_torch_allocator=True it draws its device memory from torch's caching allocator
    instead (one pool shared with torch, at the cost of a Python call per allocation)."""
    lib = load()
    if isinstance(points, np.ndarray):
        points = np.ascontiguousarray(points, dtype=np.float32)
    elif points.dtype != _torch().float32:
        raise TypeError("points must be float32")
    N, d = int(points.shape[0]), int(points.shape[1])
    cfg = cfg if cfg is not None else dm_config_default()
    keep = [points]
    torch = _torch()
    if use_torch_allocator and torch is not None and torch.cuda.is_available() and not cfg.alloc:
        dev = cfg.device if cfg.device >= 0 else torch.cuda.current_device()
        # the library runs on one torch stream and the caching allocator hands out blocks for that
        # stream, so freed blocks are reused under the allocator's own stream semantics
        if cfg.stream:
            stream = torch.cuda.ExternalStream(cfg.stream, device=dev)
        else:
            stream = torch.cuda.Stream(device=dev)
            cfg.stream = stream.cuda_stream
        ta = _TorchAllocator(dev, stream)
        cfg.alloc, cfg.free = ta.alloc_fn, ta.free_fn
        keep += [ta, stream]
    keep.append(cfg)
    h = C.c_void_p()
    _check(lib.dm_create(_ptr(points), N, d, float(eps), float(alpha), C.byref(cfg), C.byref(h)))
    out = Handle(h.value, keep)
    out.N, out.d = N, d
    return out


def dm_compress(h: Handle, tol: float, leaf_size: int, max_rank: int) -> None:
    _check(load().dm_compress(h, float(tol), int(leaf_size), int(max_rank)))


def dm_matvec(h: Handle, x, y=None):
    """y = K~ x for x of shape (N,) or (N, nrhs) (column-major blocks); returns y."""
    nrhs = 1 if x.ndim == 1 else int(x.shape[1])
    if nrhs > 1 and not _colmajor(x):
        raise ValueError("x of shape (N, nrhs) must be column-major (Fortran order / .t().contiguous().t())")
    if y is None:
        y = _like(x)
    _check(load().dm_matvec(h, _ptr(x), _ptr(y), nrhs))
    return y


def _colmajor(a) -> bool:
    if isinstance(a, np.ndarray):
        return a.flags.f_contiguous
    return a.stride(0) == 1


def _like(x):
    if isinstance(x, np.ndarray):
        return np.empty_like(x, order="F")
    torch = _torch()
    if x.ndim == 1:
        return torch.empty_like(x)
    return torch.empty((x.shape[1], x.shape[0]), dtype=x.dtype, device=x.device).t()


def dm_eigs(h: Handle, k: int, evecs: bool = True, device_out: bool = False):
    """Top-k eigenpairs: (evals (k,) float64 numpy, evecs (N, k) float32 column-major or None, converged)."""
    ev = np.empty(k, dtype=np.float64)
    vec = None
    if evecs:
        if device_out:
            torch = _torch()
            vec = torch.empty((k, h.N), dtype=torch.float32, device="cuda")
        else:
            vec = np.empty((k, h.N), dtype=np.float32)
    st = load().dm_eigs(h, int(k), ev.ctypes.data, _ptr(vec) if vec is not None else None)
    _check(st, allow=(DM_ENOCONV,))
    return ev, (vec.T if vec is not None else None), st == DM_OK


def dm_eigs_batch(handles, k: int, evecs: bool = True):
    """dm_eigs_batch: (evals (count, k) float64, [evecs (N_i, k) float32 column-major or None],
    status (count,) int32) for a list of compressed handles solved together."""
    n = len(handles)
    hs = (C.c_void_p * n)(*[h.ptr for h in handles])
    ev = np.empty((n, k), dtype=np.float64)
    vecs = [np.empty((k, h.N), dtype=np.float32) for h in handles] if evecs else None
    vp = (C.c_void_p * n)(*[v.ctypes.data for v in vecs]) if evecs else None
    status = np.empty(n, dtype=np.int32)
    st = load().dm_eigs_batch(hs, n, int(k), ev.ctypes.data, vp, status.ctypes.data)
    _check(st, allow=(DM_ENOCONV,))
    return ev, ([v.T for v in vecs] if evecs else None), status


def dm_coords(h: Handle, k: int, t: int = 1) -> np.ndarray:
    psi = np.empty((k, h.N), dtype=np.float32)
    _check(load().dm_coords(h, int(k), int(t), psi.ctypes.data))
    return psi.T


def dm_intrinsic_dim(evals, t: int, delta: float) -> tuple[int, bool]:
    """dm_intrinsic_dim: (d(t), whether every eigenvalue given passed) for the descending
    eigenvalues of a dm_eigs call, evals[0] the trivial one."""
    ev = np.ascontiguousarray(np.asarray(evals, dtype=np.float64))
    d, at_k = C.c_int32(), C.c_int32()
    _check(load().dm_intrinsic_dim(ev.ctypes.data, int(ev.size), int(t), float(delta), C.byref(d), C.byref(at_k)))
    return int(d.value), bool(at_k.value)


def dm_tune_leaf(h: Handle, tol: float, max_rank: int, k: int, candidates=(64, 128, 256, 512)):
    """Leaf-size autotuner: (best leaf, {leaf: cost in ms}); the handle stays compressed with the best."""
    cand = np.ascontiguousarray(np.asarray(candidates, dtype=np.int32))
    cost = np.zeros(len(cand), dtype=np.float32)
    best = C.c_int32()
    _check(load().dm_tune_leaf(h, float(tol), int(max_rank), int(k), cand.ctypes.data, len(cand), C.byref(best),
                               cost.ctypes.data))
    return int(best.value), {int(c): float(v) for c, v in zip(cand, cost)}


def dm_destroy(h: Handle) -> None:
    if h.ptr:
        _check(load().dm_destroy(h))
        h.ptr = None


def dm_degrees_noalloc(points, eps: float, alpha: float, q, dg, s, stream=None) -> None:
    """dm_degrees_noalloc: CUDA float32 points (N, d) and CUDA float64 outputs q, dg, s (N,).

    Enqueues on `stream` (a torch.cuda.Stream or raw handle; default: torch's current stream)
    and does not synchronise. Raises ValueError unless points is a C-contiguous float32 CUDA
    tensor of shape (N, d) and q, dg, s are contiguous float64 CUDA tensors of N elements, all
    on one device (that of `stream` when it is a torch stream): the library writes N doubles
    through each output pointer and reads the points as row-major."""
    torch = _torch()
    if not (isinstance(points, torch.Tensor) and points.is_cuda and points.dtype == torch.float32
            and points.dim() == 2 and points.is_contiguous()):
        raise ValueError("dm_degrees_noalloc: points must be a C-contiguous float32 CUDA tensor of shape (N, d)")
    N, d = int(points.shape[0]), int(points.shape[1])
    for name, t in (("q", q), ("dg", dg), ("s", s)):
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()
                and t.numel() == N):
            raise ValueError(f"dm_degrees_noalloc: {name} must be a contiguous float64 CUDA tensor of {N} elements")
        if t.device != points.device:
            raise ValueError(f"dm_degrees_noalloc: {name} is on {t.device}, points on {points.device}")
    if stream is None:
        stream = torch.cuda.current_stream(points.device)
    if hasattr(stream, "device") and torch.device(stream.device) != points.device:
        raise ValueError(f"dm_degrees_noalloc: stream is on {stream.device}, the tensors on {points.device}")
    handle = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    _check(load().dm_degrees_noalloc(_ptr(points), N, d, float(eps), float(alpha), _ptr(q), _ptr(dg), _ptr(s),
                                     handle))


def dm_kernel_launches() -> int:
    return int(load().dm_kernel_launches())


def dm_sfu_peak() -> tuple[int, float]:
    """dm_sfu_peak: (exponentials of the timed launch, its duration in ms)."""
    n, ms = C.c_int64(), C.c_float()
    _check(load().dm_sfu_peak(C.byref(n), C.byref(ms)))
    return int(n.value), float(ms.value)


def dm_selftest_wait_timeout(blocks: int, missing: int, spin_limit: int) -> tuple[int, int]:
    """dm_selftest_wait_timeout: (status, blocks that passed); the status is returned, not
    raised, since DM_ETIMEOUT is the expected answer when arrivals are missing."""
    passed = C.c_int32(-1)
    st = int(load().dm_selftest_wait_timeout(int(blocks), int(missing), int(spin_limit), C.byref(passed)))
    if st not in (DM_OK, DM_ETIMEOUT):
        raise DmError(st, dm_last_error())
    return st, int(passed.value)


def dm_get_stats(h: Handle) -> dict:
    st = dm_stats()
    _check(load().dm_get_stats(h, C.byref(st)))
    return st.as_dict()


def dm_get_eps(h: Handle) -> float:
    v = C.c_double()
    _check(load().dm_get_eps(h, C.byref(v)))
    return float(v.value)


def dm_get_degrees(h: Handle):
    q, dg, s = (np.empty(h.N, dtype=np.float64) for _ in range(3))
    _check(load().dm_get_degrees(h, q.ctypes.data, dg.ctypes.data, s.ctypes.data))
    return q, dg, s


def dm_get_tree(h: Handle):
    L = C.c_int32()
    _check(load().dm_get_tree(h, C.byref(L), None))
    perm = np.empty(h.N, dtype=np.int32)
    _check(load().dm_get_tree(h, C.byref(L), perm.ctypes.data))
    return perm, int(L.value)


def dm_get_hmatrix(h: Handle):
    """(ranks, skel, P) in the layout of dm_load_hmatrix (P as float32, ld cmax)."""
    st = dm_get_stats(h)
    L, mr = st["L"], st["max_rank"]
    nn = (1 << (L + 1)) - 1
    cmax = max(st["leaf_max"], 2 * mr)
    ranks = np.empty(nn, dtype=np.int32)
    skel = np.empty(nn * mr, dtype=np.int32)
    P = np.empty(nn * mr * cmax, dtype=np.float32)
    _check(load().dm_get_hmatrix(h, ranks.ctypes.data, skel.ctypes.data, P.ctypes.data))
    return ranks, skel, P


def dm_load_hmatrix(h: Handle, L: int, max_rank: int, perm, ranks, skel, P) -> None:
    perm = np.ascontiguousarray(perm, dtype=np.int32)
    ranks = np.ascontiguousarray(ranks, dtype=np.int32)
    skel = np.ascontiguousarray(skel, dtype=np.int32)
    P = np.ascontiguousarray(P, dtype=np.float32)
    _check(load().dm_load_hmatrix(h, int(L), int(max_rank), perm.ctypes.data, ranks.ctypes.data,
                                  skel.ctypes.data, P.ctypes.data))


# ------------------------------------------------------------------ serving

def _request(points, eps=-1.0, alpha=1.0, tol=1e-5, leaf_size=512, max_rank=128, k=10, want_vectors=True, seed=0,
             block_size=0):
    pts = np.ascontiguousarray(points, dtype=np.float32)
    r = dm_request(points=pts.ctypes.data, N=pts.shape[0], d=pts.shape[1], eps=float(eps), alpha=float(alpha),
                   tol=float(tol), leaf_size=int(leaf_size), max_rank=int(max_rank), k=int(k),
                   want_vectors=1 if want_vectors else 0, seed=int(seed), block_size=int(block_size))
    return r, pts


def dm_request_bytes(points, **kw) -> int:
    """Device bytes one solve of this request allocates at its peak (the admission estimate)."""
    r, _ = _request(points, **kw)
    return int(load().dm_request_bytes(C.byref(r)))


def dm_serve_start(slots: int = 4, hbm_budget_bytes: int = 0, device: int = -1, queue_capacity: int = 0) -> None:
    cfg = dm_serve_config(device=device, slots=slots, hbm_budget_bytes=hbm_budget_bytes,
                          queue_capacity=queue_capacity)
    _check(load().dm_serve_start(C.byref(cfg)))


def dm_serve_stop() -> None:
    _check(load().dm_serve_stop())


def dm_submit(points, **kw) -> int:
    """Queue a solve of `points` (host array); returns its ticket. Keywords as dm_request."""
    r, _keep = _request(points, **kw)
    t = C.c_uint64()
    _check(load().dm_submit(C.byref(r), C.byref(t)))  # the library copies the points before returning
    return int(t.value)


def dm_poll(ticket: int):
    """(done, result dict or None): evals (k,), evecs (N, k) or None, status, times in ms."""
    r = dm_result()
    done = C.c_int32()
    _check(load().dm_poll(C.c_uint64(ticket), C.byref(r), C.byref(done)))
    if not done.value:
        return False, None
    out = {"status": int(r.status), "k": int(r.k), "N": int(r.N), "submit_ms": r.submit_ms, "start_ms": r.start_ms,
           "built_ms": r.built_ms, "done_ms": r.done_ms, "lanczos_iters": int(r.lanczos_iters), "evals": None, "evecs": None,
           "error": (r.error or b"").decode(errors="replace")}
    if r.evals:
        out["evals"] = np.ctypeslib.as_array(r.evals, shape=(r.k,)).copy()
    if r.evecs:
        out["evecs"] = np.ctypeslib.as_array(r.evecs, shape=(r.k, r.N)).T.copy()
    return True, out


def dm_release(ticket: int) -> None:
    _check(load().dm_release(C.c_uint64(ticket)))
