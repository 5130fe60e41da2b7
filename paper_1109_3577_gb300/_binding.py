"""ctypes marshalling for libhjbp (names follow include/hjbp.h)."""
from __future__ import annotations

import ctypes as C
import os
import threading
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB_PATH = os.path.join(_HERE, "libhjbp.so")
_lock = threading.Lock()
_lib = None

HJBP_OK, HJBP_EINVAL, HJBP_ENOMEM, HJBP_ENOCONV, HJBP_ETIMEOUT, HJBP_ECUDA, HJBP_EBUSY, HJBP_ESTATE = range(8)
HJBP_FP64, HJBP_FP32_POLISH64 = 0, 1
HJBP_OUT_UCOARSE, HJBP_OUT_U0, HJBP_OUT_ASTAR, HJBP_OUT_PHI, HJBP_OUT_U32 = range(5)
MAX_CONTROLS, MAX_TARGETS = 256, 64
SPEED_KINDS = {"one": 0, "sincos2d": 1, "sin3d": 2, "fourier2d": 3, "fan": 4}
DYN_KINDS = {"speed": 0, "drift": 1, "brockett": 2}
TARGET_KINDS = {"balls": 0, "sectors": 1, "slab": 2, "orthants": 3}
_STATUS = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ENOCONV", 4: "ETIMEOUT", 5: "ECUDA", 6: "EBUSY", 7: "ESTATE"}


class HjbpError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"hjbp {_STATUS.get(status, status)}: {msg}")
        self.status = status


class Desc(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n", C.c_int * 3),
        ("n_coarse", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("speed", C.c_int),
        ("speed_params", C.c_double * 64),
        ("n_controls", C.c_int),
        ("controls", C.POINTER(C.c_double)),
        ("n_targets", C.c_int),
        ("targets", C.POINTER(C.c_double)),
        ("tol", C.c_double),
        ("tol_coarse", C.c_double),
        ("tol_phi", C.c_double),
        ("precision", C.c_int),
        ("max_sweeps", C.c_int),
        ("flags", C.c_int),
        ("tune", C.c_int * 8),
        ("reduce_r", C.c_double),
        ("dyn", C.c_int),
        ("drift", C.c_double * 4),
        ("target_kind", C.c_int),
        ("n_parts", C.c_int),
        ("n_obstacles", C.c_int),
        ("obstacles", C.POINTER(C.c_double)),
    ]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
RELEASE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)


class Allocator(C.Structure):
    _fields_ = [("alloc", ALLOC_FN), ("release", RELEASE_FN), ("ctx", C.c_void_p)]


class Stats(C.Structure):
    _fields_ = [
        ("n_patches", C.c_int),
        ("sweeps_coarse", C.c_int),
        ("sweeps_phi", C.c_int),
        ("sweeps_reach", C.c_int),
        ("sweeps_fine", C.c_int),
        ("sweeps_polish", C.c_int),
        ("sweeps_patch", C.c_int * MAX_TARGETS),
        ("patch_nodes", C.c_int64 * MAX_TARGETS),
        ("patch_tiles", C.c_int64 * MAX_TARGETS),
        ("residual_fine", C.c_double),
        ("residual_polish", C.c_double),
        ("unreachable", C.c_int64),
        ("uncovered_filled", C.c_int64),
        ("node_updates", C.c_int64),
        ("node_control_updates", C.c_int64),
        ("ms_setup", C.c_double),
        ("ms_coarse", C.c_double),
        ("ms_feedback", C.c_double),
        ("ms_labels", C.c_double),
        ("ms_compact", C.c_double),
        ("ms_fine", C.c_double),
        ("ms_polish", C.c_double),
        ("ms_total", C.c_double),
        ("kernel_launches", C.c_int64),
        ("sweep_kernel_launches", C.c_int64),
        ("sweep_tile_visits", C.c_int64),
        ("ms_sweep_kernel", C.c_double),
        ("phi_refinements", C.c_int),
        ("ms_reach", C.c_double),
        ("residual_patch", C.c_double * MAX_TARGETS),
        ("phi_kernel_launches", C.c_int64),
        ("phi_node_colour_updates", C.c_int64),
        ("ms_phi_kernel", C.c_double),
    ]

    def as_dict(self) -> dict:
        out = {}
        R = max(1, self.n_patches)
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v[:R]) if hasattr(v, "__len__") else v
        return out


def library_path() -> str:
    return _LIB_PATH


def library():
    """Load libhjbp.so (raises if it has not been built)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        if not os.path.exists(_LIB_PATH):
            raise ImportError(f"{_LIB_PATH} is missing: build it with paper_1109_3577_gb300/build.py "
                              "(there is no CPU fallback)")
        lib = C.CDLL(_LIB_PATH)
        P = C.POINTER
        vp = C.c_void_p
        lib.hjbp_create.argtypes = [P(Desc), vp, P(Allocator), P(vp)]
        lib.hjbp_create.restype = C.c_int
        lib.hjbp_solve.argtypes = [vp]
        lib.hjbp_solve.restype = C.c_int
        lib.hjbp_sync.argtypes = [vp]
        lib.hjbp_sync.restype = C.c_int
        lib.hjbp_set_initial.argtypes = [vp, vp]
        lib.hjbp_set_initial.restype = C.c_int
        lib.hjbp_get_values.argtypes = [vp, vp]
        lib.hjbp_get_values.restype = C.c_int
        lib.hjbp_get_labels.argtypes = [vp, vp]
        lib.hjbp_get_labels.restype = C.c_int
        lib.hjbp_get_intermediate.argtypes = [vp, C.c_int, vp, C.c_size_t]
        lib.hjbp_get_intermediate.restype = C.c_int
        lib.hjbp_get_device_views.argtypes = [vp, P(vp), P(vp)]
        lib.hjbp_get_device_views.restype = C.c_int
        lib.hjbp_get_stats.argtypes = [vp, P(Stats)]
        lib.hjbp_get_stats.restype = C.c_int
        lib.hjbp_get_sizes.argtypes = [vp, P(C.c_int64), P(C.c_int64)]
        lib.hjbp_get_sizes.restype = C.c_int
        lib.hjbp_destroy.argtypes = [vp]
        lib.hjbp_destroy.restype = None
        lib.hjbp_last_error.argtypes = []
        lib.hjbp_last_error.restype = C.c_char_p
        lib.hjbp_get_patch_lists.argtypes = [vp, vp, vp, vp, vp, vp]
        lib.hjbp_get_patch_lists.restype = C.c_int
        lib.hjbp_solve_global2d_noalloc.argtypes = [P(Desc), vp, vp, vp]
        lib.hjbp_solve_global2d_noalloc.restype = C.c_int
        lib.hjbp_batch_solve.argtypes = [P(vp), C.c_int, C.c_int, P(C.c_int)]
        lib.hjbp_batch_solve.restype = C.c_int
        lib.hjbp_autotune.argtypes = [P(Desc), vp, C.c_char_p, P(C.c_int), P(C.c_int)]
        lib.hjbp_autotune.restype = C.c_int
        lib.hjbp_server_create.argtypes = [C.c_size_t, C.c_int, P(vp)]
        lib.hjbp_server_create.restype = C.c_int
        lib.hjbp_server_submit.argtypes = [vp, P(Desc), P(C.c_uint64)]
        lib.hjbp_server_submit.restype = C.c_int
        lib.hjbp_server_poll.argtypes = [vp, C.c_uint64, P(vp), P(C.c_double)]
        lib.hjbp_server_poll.restype = C.c_int
        lib.hjbp_server_stats.argtypes = [vp, P(C.c_int), P(C.c_int), P(C.c_size_t)]
        lib.hjbp_server_stats.restype = C.c_int
        lib.hjbp_server_destroy.argtypes = [vp]
        lib.hjbp_server_destroy.restype = None
        lib.hjbp_version.argtypes = []
        lib.hjbp_version.restype = C.c_int
        _lib = lib
        return lib


def _check(status: int):
    if status != HJBP_OK:
        raise HjbpError(status, hjbp_last_error())


# ----------------------------------------------------------- C-ABI names ---

def hjbp_version() -> int:
    return library().hjbp_version()


def hjbp_last_error() -> str:
    m = library().hjbp_last_error()
    return m.decode() if m else ""


def hjbp_create(desc: Desc, stream: int = 0, allocator: Optional[Allocator] = None) -> int:
    plan = C.c_void_p()
    st = library().hjbp_create(C.byref(desc), C.c_void_p(stream), C.byref(allocator) if allocator else None,
                               C.byref(plan))
    _check(st)
    return plan.value


def hjbp_solve(plan: int) -> int:
    """Returns the status (OK or ENOCONV); raises on every other error."""
    st = library().hjbp_solve(C.c_void_p(plan))
    if st not in (HJBP_OK, HJBP_ENOCONV):
        _check(st)
    return st


def hjbp_sync(plan: int) -> int:
    """Status of the plan's last solve (OK or ENOCONV); raises otherwise."""
    st = library().hjbp_sync(C.c_void_p(plan))
    if st not in (HJBP_OK, HJBP_ENOCONV):
        _check(st)
    return st


def hjbp_set_initial(plan: int, u_init: Optional[np.ndarray]) -> None:
    """Start values of the value iteration (N doubles, >= 0 or +inf); None clears."""
    if u_init is None:
        _check(library().hjbp_set_initial(C.c_void_p(plan), None))
        return
    u = np.ascontiguousarray(u_init, dtype=np.float64)
    _check(library().hjbp_set_initial(C.c_void_p(plan), u.ctypes.data_as(C.c_void_p)))


def hjbp_get_values(plan: int, out: np.ndarray) -> None:
    assert out.dtype == np.float64 and out.flags.c_contiguous
    _check(library().hjbp_get_values(C.c_void_p(plan), out.ctypes.data_as(C.c_void_p)))


def hjbp_get_labels(plan: int, out: np.ndarray) -> None:
    assert out.dtype == np.int8 and out.flags.c_contiguous
    _check(library().hjbp_get_labels(C.c_void_p(plan), out.ctypes.data_as(C.c_void_p)))


def hjbp_get_intermediate(plan: int, which: int, out: np.ndarray) -> None:
    assert out.flags.c_contiguous
    _check(library().hjbp_get_intermediate(C.c_void_p(plan), which, out.ctypes.data_as(C.c_void_p), out.nbytes))


def hjbp_get_device_views(plan: int):
    u, lab = C.c_void_p(), C.c_void_p()
    _check(library().hjbp_get_device_views(C.c_void_p(plan), C.byref(u), C.byref(lab)))
    return u.value, lab.value


def hjbp_get_stats(plan: int) -> Stats:
    s = Stats()
    _check(library().hjbp_get_stats(C.c_void_p(plan), C.byref(s)))
    return s


def hjbp_get_sizes(plan: int):
    n, nc = C.c_int64(), C.c_int64()
    _check(library().hjbp_get_sizes(C.c_void_p(plan), C.byref(n), C.byref(nc)))
    return n.value, nc.value


def hjbp_batch_solve(plans, workers: int = 0):
    """Solve plan handles concurrently; returns the per-plan statuses."""
    n = len(plans)
    arr = (C.c_void_p * n)(*plans)
    st = (C.c_int * n)()
    rc = library().hjbp_batch_solve(arr, n, int(workers), st)
    if rc not in (HJBP_OK, HJBP_ENOCONV):
        _check(rc)
    return list(st)


def hjbp_autotune(desc, stream: int = 0, cache_path: Optional[str] = None):
    """The launch shape (tune[0..3]) for problems of desc's class, and
    whether it came from the cache."""
    t = (C.c_int * 4)()
    fc = C.c_int(0)
    path = cache_path.encode() if cache_path else None
    _check(library().hjbp_autotune(C.byref(desc), C.c_void_p(stream), path, t, C.byref(fc)))
    return list(t), bool(fc.value)


def hjbp_server_create(budget_bytes: int = 0, workers: int = 0) -> int:
    s = C.c_void_p()
    _check(library().hjbp_server_create(C.c_size_t(budget_bytes), int(workers), C.byref(s)))
    return s.value


def hjbp_server_submit(server: int, desc: Desc) -> int:
    t = C.c_uint64()
    _check(library().hjbp_server_submit(C.c_void_p(server), C.byref(desc), C.byref(t)))
    return t.value


def hjbp_server_poll(server: int, ticket: int):
    """(status, plan handle or None, latency seconds)."""
    plan = C.c_void_p()
    lat = C.c_double()
    st = library().hjbp_server_poll(C.c_void_p(server), C.c_uint64(ticket), C.byref(plan), C.byref(lat))
    if st not in (HJBP_OK, HJBP_ENOCONV):
        _check(st)
    return st, plan.value, lat.value


def hjbp_server_stats(server: int):
    q, r, b = C.c_int(), C.c_int(), C.c_size_t()
    _check(library().hjbp_server_stats(C.c_void_p(server), C.byref(q), C.byref(r), C.byref(b)))
    return q.value, r.value, b.value


def hjbp_server_destroy(server: int) -> None:
    library().hjbp_server_destroy(C.c_void_p(server))


HJBP_NOALLOC_MAX_NODES = 1 << 20


def hjbp_solve_global2d_noalloc(desc: Desc, stream: int, u_out_ptr: int, labels_out_ptr: int) -> int:
    """Global 2D FP64 solve into caller-owned device arrays, allocating
    nothing (scratch is a fixed array inside the library; calls must not
    overlap on the GPU).  Returns OK or ENOCONV; raises on other errors."""
    st = library().hjbp_solve_global2d_noalloc(C.byref(desc), C.c_void_p(stream), C.c_void_p(u_out_ptr),
                                               C.c_void_p(labels_out_ptr))
    if st not in (HJBP_OK, HJBP_ENOCONV):
        _check(st)
    return st


def hjbp_get_patch_lists(plan: int) -> dict:
    """Per-patch tile and node lists of the last patchy solve (CSR):
    tile_offsets / node_offsets (R + 1), tile_ids, tile_nodes, node_ids."""
    lib = library()
    R = max(1, hjbp_get_stats(plan).n_patches)
    to = np.zeros(R + 1, np.int64)
    no = np.zeros(R + 1, np.int64)
    _check(lib.hjbp_get_patch_lists(C.c_void_p(plan), to.ctypes.data, None, None, no.ctypes.data, None))
    tid = np.zeros(max(1, int(to[-1])), np.int32)
    tn = np.zeros(max(1, int(to[-1])), np.int32)
    nid = np.zeros(max(1, int(no[-1])), np.int32)
    _check(lib.hjbp_get_patch_lists(C.c_void_p(plan), None, tid.ctypes.data, tn.ctypes.data, None,
                                    nid.ctypes.data))
    return {"tile_offsets": to, "tile_ids": tid[: int(to[-1])], "tile_nodes": tn[: int(to[-1])],
            "node_offsets": no, "node_ids": nid[: int(no[-1])]}


def hjbp_destroy(plan: int) -> None:
    library().hjbp_destroy(C.c_void_p(plan))


# ------------------------------------------------------------ conveniences ---

def torch_allocator() -> Allocator:
    """Allocator hooks that draw device memory from PyTorch's caching allocator."""
    import torch

    live = {}

    def _alloc(nbytes, stream, ctx):
        try:
            ptr = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), stream or 0)
        except Exception:
            return None
        live[ptr] = nbytes
        return ptr

    def _release(ptr, nbytes, stream, ctx):
        live.pop(ptr, None)
        torch.cuda.caching_allocator_delete(ptr)

    a = Allocator(ALLOC_FN(_alloc), RELEASE_FN(_release), None)
    a._keep = (_alloc, _release, live)  # keep the callbacks alive
    return a


HJBP_FLAG_TIME_SWEEPS = 1
HJBP_FLAG_DIRICHLET = 2
HJBP_FLAG_WARM_START = 4
HJBP_FLAG_CAUSAL_SWEEPS = 8
HJBP_FLAG_TILE_QUEUE = 16


def desc_from_problem(p, precision: int = HJBP_FP32_POLISH64, max_sweeps: int = 0, flags: int = 0, tune=None,
                      reduce_r: float = 0.0):
    """Build an hjbp_problem_desc from a workloads.Problem.  Returns the
    struct plus the arrays it points into (keep both alive)."""
    controls = np.ascontiguousarray(p.controls, dtype=np.float64)
    targets = np.ascontiguousarray(p.targets, dtype=np.float64)
    d = Desc()
    d.dim = p.dim
    for a in range(3):
        d.n[a] = int(p.n[a]) if a < p.dim else 1
        d.n_coarse[a] = (int(p.n_coarse[a]) if a < p.dim else 1) if p.n_coarse else 0
        d.lo[a] = float(p.lo[a])
        d.hi[a] = float(p.hi[a])
    d.speed = SPEED_KINDS[p.speed]
    for i in range(64):
        d.speed_params[i] = float(p.speed_params[i])
    d.n_controls = controls.shape[0]
    d.controls = controls.ctypes.data_as(C.POINTER(C.c_double))
    d.n_targets = targets.shape[0]
    d.targets = targets.ctypes.data_as(C.POINTER(C.c_double))
    d.tol = float(p.tol)
    d.tol_coarse = float(p.tol_coarse)
    d.tol_phi = float(p.tol_phi)
    d.precision = int(precision)
    d.max_sweeps = int(max_sweeps or 0)
    d.flags = int(flags)
    for i, v in enumerate(tune or ()):
        d.tune[i] = int(v)
    d.reduce_r = float(reduce_r)
    d.dyn = DYN_KINDS[getattr(p, "dyn", "speed")]
    for i, v in enumerate(getattr(p, "drift", (1.0, 0.0, 0.0, 0.0))):
        d.drift[i] = float(v)
    d.target_kind = TARGET_KINDS[getattr(p, "target_kind", "balls")]
    d.n_parts = int(getattr(p, "n_parts", 0))
    obs = getattr(p, "obstacles", None)
    obstacles = np.ascontiguousarray(np.zeros((0, 7)) if obs is None else obs, dtype=np.float64)
    d.n_obstacles = obstacles.shape[0]
    d.obstacles = obstacles.ctypes.data_as(C.POINTER(C.c_double)) if d.n_obstacles else C.POINTER(C.c_double)()
    return d, (controls, targets, obstacles)


class Plan:
    """Owns one hjbp_plan.  ``Plan(problem).solve()`` then ``values()`` /
    ``labels()`` / ``stats()``."""

    def __init__(self, problem, precision: int = HJBP_FP32_POLISH64, stream: Optional[int] = None,
                 use_torch_allocator: bool = False, max_sweeps: int = 0, flags: int = 0, tune=None,
                 reduce_r: float = 0.0):
        self.problem = problem
        self._desc, self._keep = desc_from_problem(problem, precision, max_sweeps, flags, tune, reduce_r)
        if stream is None:
            stream = 0
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except Exception:
                pass
        self._alloc = torch_allocator() if use_torch_allocator else None
        self.handle = hjbp_create(self._desc, stream, self._alloc)
        self.N, self.Nc = hjbp_get_sizes(self.handle)
        self.status = None

    @classmethod
    def adopt(cls, problem, handle: int):
        """Wrap a plan handle produced by the library (e.g. a served request)."""
        self = cls.__new__(cls)
        self.problem = problem
        self._desc, self._keep, self._alloc = None, None, None
        self.handle = handle
        self.N, self.Nc = hjbp_get_sizes(handle)
        self.status = None
        return self

    def solve(self) -> int:
        self.status = hjbp_solve(self.handle)
        return self.status

    def sync(self) -> int:
        return hjbp_sync(self.handle)

    def set_initial(self, u_init: Optional[np.ndarray]) -> None:
        if u_init is not None and np.asarray(u_init).size != self.N:
            raise ValueError("start values need one entry per fine node")
        hjbp_set_initial(self.handle, u_init)

    def values(self) -> np.ndarray:
        out = np.empty(self.N, np.float64)
        hjbp_get_values(self.handle, out)
        return out

    def labels(self) -> np.ndarray:
        out = np.empty(self.N, np.int8)
        hjbp_get_labels(self.handle, out)
        return out

    def intermediate(self, which: int) -> np.ndarray:
        R = self.problem.n_patches
        if which == HJBP_OUT_UCOARSE:
            out = np.empty(self.Nc, np.float64)
        elif which == HJBP_OUT_U0:
            out = np.empty(self.N, np.float64)
        elif which == HJBP_OUT_ASTAR:
            out = np.empty(self.N, np.int32)
        elif which == HJBP_OUT_PHI:
            out = np.empty((R, self.N), np.float64)
        elif which == HJBP_OUT_U32:
            out = np.empty(self.N, np.float32)
        else:
            raise ValueError(which)
        hjbp_get_intermediate(self.handle, which, out)
        return out

    def stats(self) -> dict:
        return hjbp_get_stats(self.handle).as_dict()

    def patch_lists(self) -> dict:
        return hjbp_get_patch_lists(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            hjbp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
