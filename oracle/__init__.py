"""FP64 CPU oracle for the patchy semi-Lagrangian minimum-time scheme.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package; the product path
(the CUDA library and its binding) never does.  The arithmetic lives in plain
C (``hjbp_oracle.c``); this module compiles it with gcc and marshals
arguments through ctypes.

Every function follows the paper (Cacace, Cristiani, Falcone, Picarelli,
"A patchy dynamic programming scheme for a class of HJB equations"):

* ``sl_apply``       -- the operator F of Eq. (SLscheme), one application.
* ``iterate``/``global_solve`` -- Eq. (iterativeSLscheme) to the sup-norm
  stopping test of Sec. 2.2 (Step 4), Gauss-Seidel or Jacobi.
* ``patchy_solve``   -- the patchy algorithm of Sec. 3 (Steps 1-4), with the
  Dirichlet patch boundary of Eq. (dbc) and the add-ons AO1-AO3 of Sec. 6 as
  options.
* ``iterate_reduced`` -- ``iterate`` over the AO3 control cones.
* ``interp``         -- the interpolation operator I of Sec. 2.1.

Pins (tests/test_oracle_*.py): eikonal closed form, Dijkstra on the axis
control set, exact policy iteration on 9x9 grids, exactness of I on
multilinear functions, monotonicity of F, D4 symmetry, absorption
probabilities for phi, the R = 1 identity and patch invariance.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading
from dataclasses import dataclass
from typing import Optional

import numpy as np

from workloads import DYN_KINDS, SPEED_KINDS, TARGET_KINDS, Problem

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hjbp_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

FREE, TARGET, GHOST = 0, 1, 2


class _Problem(C.Structure):
    _fields_ = [
        ("dim", C.c_int),
        ("n", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("k", C.c_double),
        ("speed_kind", C.c_int),
        ("speed_params", C.c_double * 64),
        ("n_controls", C.c_int),
        ("controls", C.POINTER(C.c_double)),
        ("n_targets", C.c_int),
        ("targets", C.POINTER(C.c_double)),
        ("dyn_kind", C.c_int),
        ("drift", C.c_double * 4),
        ("target_kind", C.c_int),
        ("n_parts", C.c_int),
        ("n_obstacles", C.c_int),
        ("obstacles", C.POINTER(C.c_double)),
    ]


class _Addons(C.Structure):
    _fields_ = [
        ("dirichlet", C.c_int),
        ("warm", C.c_int),
        ("causal", C.c_int),
        ("reduce_r", C.c_double),
        ("data", C.POINTER(C.c_double)),
    ]


class _Stats(C.Structure):
    _fields_ = [
        ("sweeps_coarse", C.c_int),
        ("residual_coarse", C.c_double),
        ("sweeps_phi", C.c_int * 64),
        ("residual_phi", C.c_double * 64),
        ("sweeps_patch", C.c_int * 64),
        ("residual_patch", C.c_double * 64),
        ("patch_nodes", C.c_int64 * 64),
        ("unreachable", C.c_int64),
        ("uncovered_filled", C.c_int64),
        ("uncovered_left", C.c_int64),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain C11, -O2, no FMA contraction;
    OpenMP only for og_sl_apply_par, the all-core timing of the CPU baseline)."""
    with _lock:
        if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
            tmp = _LIB + f".{os.getpid()}.tmp"
            subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared",
                                   _SRC, "-o", tmp, "-lm"])
            os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = C.CDLL(_LIB)
        P = C.POINTER
        dp = P(C.c_double)
        lib.og_speed.restype = C.c_double
        lib.og_speed.argtypes = [P(_Problem), dp]
        lib.og_setup.argtypes = [P(_Problem), C.c_double, P(C.c_ubyte), P(C.c_int), dp]
        lib.og_interp_points.argtypes = [P(_Problem), dp, C.c_int64, dp, dp]
        lib.og_sl_apply.argtypes = [P(_Problem), P(C.c_ubyte), dp, dp, dp, C.c_int]
        lib.og_sl_apply_par.argtypes = [P(_Problem), P(C.c_ubyte), dp, dp, dp, C.c_int]
        lib.og_iterate.argtypes = [P(_Problem), P(C.c_ubyte), dp, dp, C.c_double, C.c_int, C.c_int,
                                   P(C.c_int), dp]
        lib.og_iterate_reduced.argtypes = [P(_Problem), P(C.c_ubyte), dp, dp, C.c_double, C.c_int, C.c_int,
                                           P(C.c_int), C.c_double, P(C.c_int), dp]
        lib.og_reachable.argtypes = [P(_Problem), P(C.c_ubyte), dp, P(C.c_ubyte)]
        lib.og_global_solve.argtypes = [P(_Problem), C.c_double, C.c_int, C.c_int, dp, P(C.c_int), dp]
        lib.og_patchy_solve.argtypes = [P(_Problem), P(C.c_int), C.c_double, C.c_double, C.c_double,
                                        C.c_int, C.c_int, dp, P(C.c_byte), dp, dp, P(C.c_int), dp, dp,
                                        P(_Stats)]
        lib.og_patchy_solve_ex.argtypes = [P(_Problem), P(C.c_int), C.c_double, C.c_double, C.c_double,
                                           C.c_int, C.c_int, P(_Addons), dp, P(C.c_byte), dp, dp, P(C.c_int),
                                           dp, dp, P(_Stats)]
        _lib = lib
    return _lib


def _ptr(a: Optional[np.ndarray], ctype):
    if a is None:
        return C.POINTER(ctype)()
    return a.ctypes.data_as(C.POINTER(ctype))


class _Desc:
    """Keeps the ctypes struct and the arrays it points into alive together."""

    def __init__(self, p: Problem, n=None):
        self.controls = np.ascontiguousarray(p.controls, dtype=np.float64)
        self.targets = np.ascontiguousarray(p.targets, dtype=np.float64)
        s = _Problem()
        s.dim = p.dim
        nn = n if n is not None else p.n
        for d in range(3):
            s.n[d] = int(nn[d]) if d < p.dim else 1
            s.lo[d] = float(p.lo[d])
        s.k = (p.hi[0] - p.lo[0]) / (nn[0] - 1)
        s.speed_kind = SPEED_KINDS[p.speed]
        for i in range(64):
            s.speed_params[i] = float(p.speed_params[i])
        s.n_controls = self.controls.shape[0]
        s.controls = _ptr(self.controls, C.c_double)
        s.n_targets = self.targets.shape[0]
        s.targets = _ptr(self.targets, C.c_double)
        s.dyn_kind = DYN_KINDS[p.dyn]
        for i in range(4):
            s.drift[i] = float(p.drift[i])
        s.target_kind = TARGET_KINDS[p.target_kind]
        s.n_parts = int(p.n_parts)
        obs = getattr(p, "obstacles", None)
        self.obstacles = np.ascontiguousarray(np.zeros((0, 7)) if obs is None else obs, dtype=np.float64)
        s.n_obstacles = self.obstacles.shape[0]
        s.obstacles = _ptr(self.obstacles, C.c_double) if s.n_obstacles else C.POINTER(C.c_double)()
        self.s = s
        self.N = int(np.prod([s.n[d] for d in range(p.dim)]))
        self.shape = tuple(int(s.n[d]) for d in reversed(range(p.dim)))  # (n3, n2, n1) / (n2, n1)


def speed(p: Problem, x) -> float:
    d = _Desc(p)
    xx = (C.c_double * 3)(*([float(v) for v in x] + [0.0] * (3 - len(x))))
    return _load().og_speed(C.byref(d.s), xx)


def setup(p: Problem, radius_extra: float = 0.0):
    """Node kinds (FREE/TARGET/GHOST), target parts and h_i = k / c(x_i)."""
    d = _Desc(p)
    kind = np.zeros(d.N, np.uint8)
    part = np.zeros(d.N, np.int32)
    h = np.zeros(d.N, np.float64)
    _load().og_setup(C.byref(d.s), radius_extra, _ptr(kind, C.c_ubyte), _ptr(part, C.c_int), _ptr(h, C.c_double))
    return kind, part, h


def interp(p: Problem, U: np.ndarray, xi: np.ndarray) -> np.ndarray:
    """I[U] at points given in grid-index coordinates xi (npts x dim)."""
    d = _Desc(p)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    xi = np.asarray(xi, dtype=np.float64)
    pts = np.zeros((xi.shape[0], 3))
    pts[:, : xi.shape[1]] = xi
    out = np.zeros(xi.shape[0])
    _load().og_interp_points(C.byref(d.s), _ptr(U, C.c_double), xi.shape[0], _ptr(pts, C.c_double),
                             _ptr(out, C.c_double))
    return out


def sl_apply(p: Problem, U: np.ndarray, upd: Optional[np.ndarray] = None, mode: int = 0) -> np.ndarray:
    """One application of F (Eq. SLscheme, mode 0) or of its node-wise exact
    form (mode 1, the local equation solved for u_i); ``upd`` defaults to the
    free nodes."""
    d = _Desc(p)
    kind, _, h = setup(p)
    if upd is None:
        upd = (kind == FREE)
    upd = np.ascontiguousarray(upd, dtype=np.uint8).reshape(-1)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    out = np.zeros_like(U)
    _load().og_sl_apply(C.byref(d.s), _ptr(upd, C.c_ubyte), _ptr(h, C.c_double), _ptr(U, C.c_double),
                        _ptr(out, C.c_double), mode)
    return out


def sl_apply_par(p: Problem, U: np.ndarray, upd: Optional[np.ndarray] = None, mode: int = 0, setup_out=None):
    """sl_apply with the nodes split over the host's threads (OpenMP; the
    paper's Method 1).  Returns (F(U), threads used)."""
    d = _Desc(p)
    kind, _, h = setup(p) if setup_out is None else setup_out
    if upd is None:
        upd = (kind == FREE)
    upd = np.ascontiguousarray(upd, dtype=np.uint8).reshape(-1)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    out = np.zeros_like(U)
    used = _load().og_sl_apply_par(C.byref(d.s), _ptr(upd, C.c_ubyte), _ptr(h, C.c_double), _ptr(U, C.c_double),
                                   _ptr(out, C.c_double), mode)
    return out, int(used)


def reachable(p: Problem, upd: np.ndarray, U: np.ndarray) -> np.ndarray:
    """S*: nodes (among ``upd``) reaching the target almost surely under some
    admissible feedback; targets are the non-updated nodes with finite U."""
    d = _Desc(p)
    upd = np.ascontiguousarray(upd, dtype=np.uint8).reshape(-1)
    U = np.ascontiguousarray(U, dtype=np.float64).reshape(-1)
    out = np.zeros(d.N, np.uint8)
    _load().og_reachable(C.byref(d.s), _ptr(upd, C.c_ubyte), _ptr(U, C.c_double), _ptr(out, C.c_ubyte))
    return out.astype(bool)


@dataclass
class IterResult:
    u: np.ndarray
    sweeps: int
    residual: float
    converged: bool


def iterate(p: Problem, U0: np.ndarray, upd: np.ndarray, tol: float, max_sweeps: int = 100000,
            order: int = 1) -> IterResult:
    d = _Desc(p)
    _, _, h = setup(p)
    U = np.array(U0, dtype=np.float64).reshape(-1).copy()
    upd = np.ascontiguousarray(upd, dtype=np.uint8).reshape(-1)
    sw = C.c_int(0)
    res = C.c_double(0)
    rc = _load().og_iterate(C.byref(d.s), _ptr(upd, C.c_ubyte), _ptr(h, C.c_double), _ptr(U, C.c_double),
                            tol, max_sweeps, order, C.byref(sw), C.byref(res))
    return IterResult(U, sw.value, res.value, rc == 0)


def iterate_reduced(p: Problem, U0: np.ndarray, upd: np.ndarray, astar: np.ndarray, r: float, tol: float,
                    max_sweeps: int = 100000, order: int = 1) -> IterResult:
    """``iterate`` with the AO3 control cones (Sec. 6): at node i only the
    controls a with a . a_{astar[i]} >= cos(pi / r) (astar[i] = -1: all)."""
    d = _Desc(p)
    _, _, h = setup(p)
    U = np.array(U0, dtype=np.float64).reshape(-1).copy()
    upd = np.ascontiguousarray(upd, dtype=np.uint8).reshape(-1)
    ast = np.ascontiguousarray(astar, dtype=np.int32).reshape(-1)
    sw = C.c_int(0)
    res = C.c_double(0)
    rc = _load().og_iterate_reduced(C.byref(d.s), _ptr(upd, C.c_ubyte), _ptr(h, C.c_double),
                                    _ptr(U, C.c_double), tol, max_sweeps, order, _ptr(ast, C.c_int), float(r),
                                    C.byref(sw), C.byref(res))
    return IterResult(U, sw.value, res.value, rc == 0)


def global_solve(p: Problem, tol: Optional[float] = None, order: int = 1,
                 max_sweeps: Optional[int] = None) -> IterResult:
    """Global SL fixed point (Eq. iterativeSLscheme), U^(0) = 0 / +inf."""
    d = _Desc(p)
    U = np.zeros(d.N)
    sw = C.c_int(0)
    res = C.c_double(0)
    rc = _load().og_global_solve(C.byref(d.s), p.tol if tol is None else tol,
                                 p.max_sweeps if max_sweeps is None else max_sweeps, order,
                                 _ptr(U, C.c_double), C.byref(sw), C.byref(res))
    if rc < 0:
        raise MemoryError("oracle allocation failed")
    return IterResult(U, sw.value, res.value, rc == 0)


@dataclass
class PatchyResult:
    u: np.ndarray
    labels: np.ndarray
    ucoarse: np.ndarray
    u0: np.ndarray
    astar: np.ndarray
    gap: np.ndarray
    phi: Optional[np.ndarray]
    stats: dict
    converged: bool


def patchy_solve(p: Problem, order: int = 1, keep_phi: bool = False, tol: Optional[float] = None,
                 max_sweeps: Optional[int] = None, dirichlet: bool = False, warm: bool = False,
                 causal: bool = False, reduce_r: float = 0.0,
                 bc_data: Optional[np.ndarray] = None) -> PatchyResult:
    """The patchy algorithm of Sec. 3 (Steps 1, 2, 3.1, 3.2, 4).  Patch
    boundaries carry state constraints, or with ``dirichlet`` the data
    U_P^(0) of Eq. (dbc) (``bc_data`` replaces it, for tests).  Add-ons of
    Sec. 6: ``warm`` (AO1, start from U_P^(0)), ``causal`` (AO2, visit nodes
    by increasing U_P^(0)), ``reduce_r`` (AO3, control cones of half-angle
    pi / r around the coarse feedback; 0 = off)."""
    if p.n_coarse is None:
        raise ValueError("patchy_solve needs n_coarse")
    d = _Desc(p)
    dc = _Desc(p, n=p.n_coarse)
    N, R = d.N, p.n_patches
    u = np.zeros(N)
    lab = np.zeros(N, np.int8)
    uc = np.zeros(dc.N)
    u0 = np.zeros(N)
    ast = np.zeros(N, np.int32)
    gap = np.zeros(N)
    phi = np.zeros((R, N)) if keep_phi else None
    st = _Stats()
    ncs = (C.c_int * 3)(*[int(v) for v in p.n_coarse])
    ao = _Addons()
    ao.dirichlet = int(bool(dirichlet))
    ao.warm = int(bool(warm))
    ao.causal = int(bool(causal))
    ao.reduce_r = float(reduce_r)
    data = None
    if bc_data is not None:
        data = np.ascontiguousarray(bc_data, dtype=np.float64).reshape(-1)
        if data.size != N:
            raise ValueError("bc_data must hold one value per fine node")
    ao.data = _ptr(data, C.c_double)
    rc = _load().og_patchy_solve_ex(
        C.byref(d.s), ncs, p.tol if tol is None else tol, p.tol_coarse, p.tol_phi,
        p.max_sweeps if max_sweeps is None else max_sweeps, order, C.byref(ao), _ptr(u, C.c_double),
        _ptr(lab, C.c_byte), _ptr(uc, C.c_double), _ptr(u0, C.c_double), _ptr(ast, C.c_int),
        _ptr(gap, C.c_double), _ptr(phi, C.c_double), C.byref(st))
    if rc < 0:
        raise RuntimeError(f"oracle patchy_solve failed ({rc})")
    stats = {
        "sweeps_coarse": st.sweeps_coarse,
        "residual_coarse": st.residual_coarse,
        "sweeps_phi": list(st.sweeps_phi[:R]),
        "residual_phi": list(st.residual_phi[:R]),
        "sweeps_patch": list(st.sweeps_patch[:R]),
        "residual_patch": list(st.residual_patch[:R]),
        "patch_nodes": list(st.patch_nodes[:R]),
        "unreachable": st.unreachable,
        "uncovered_filled": st.uncovered_filled,
        "uncovered_left": st.uncovered_left,
    }
    return PatchyResult(u, lab, uc, u0, ast, gap, phi, stats, rc == 0)


def patchy_error(u_patchy: np.ndarray, u_global: np.ndarray):
    """E = U_P - U_global with E_1 = mean |E| and E_inf = max |E| over the
    nodes where both are finite (Sec. 4.2)."""
    m = np.isfinite(u_patchy) & np.isfinite(u_global)
    e = np.abs(u_patchy[m] - u_global[m])
    return float(e.mean()) if e.size else 0.0, float(e.max()) if e.size else 0.0


def grid_coords(p: Problem) -> np.ndarray:
    """Node coordinates, shape (N, dim), node index i = i1 + n1 (i2 + n2 i3)."""
    k = p.spacing
    axes = [p.lo[d] + k * np.arange(p.n[d]) for d in range(p.dim)]
    mesh = np.meshgrid(*axes, indexing="ij")
    return np.stack([m.reshape(-1, order="F") for m in mesh], axis=1)
