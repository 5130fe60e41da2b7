"""Seeded synthetic inputs for the minimum-time HJB problems.

This module only *describes* problems: grid sizes, the box Omega, the speed
field menu and its parameters, the discrete control set A and the target
balls Omega_0^j.  It holds none of the scheme's arithmetic (no interpolation,
no time step, no fixed-point iteration); both the CPU oracle and the CUDA
library read the same descriptions and evaluate everything else themselves.

Problem families (dynamics f(x, a) = c(x) a, |a| = 1, unless stated):

* ``eikonal2d``     c = 1, one disk target (closed form u = max(|x| - r, 0)).
* ``sincos2d``      c = 1 + A sin(2 pi x1) cos(2 pi x2).
* ``sin3d``         c = 1 + A sin(pi x1) sin(pi x2) sin(pi x3).
* ``fourier2d``     c = 1 + 0.5 g(x), g a normalised random 4x4 Fourier field.
* the paper's own 2D tests (Table 1), with the target split into R parts:
  ``eikonal_sectors`` (f = a, one disk in R sectors), ``zermelo`` (f = 2.1 a
  + (2, 0), a drift, one disk in R sectors) and ``fan`` (c = |x1 + x2 + 0.1|,
  the line x1 = 0 in R pieces).

Control sets: 2D -- unit vectors at angles 2 pi m / N_c (the paper
discretises A = B_2(0,1) with N_c points, Sec. 2.1 and Table 1); 3D -- a
spherical Fibonacci lattice standing in for the paper's geosphere points
(Sec. 6).  Components with magnitude below 1e-15 are snapped to exactly 0 so
that axis controls land exactly on grid nodes on every implementation.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np

SPEED_KINDS = {"one": 0, "sincos2d": 1, "sin3d": 2, "fourier2d": 3, "fan": 4}
DYN_KINDS = {"speed": 0, "drift": 1, "brockett": 2}
TARGET_KINDS = {"balls": 0, "sectors": 1, "slab": 2, "orthants": 3}
SNAP = 1e-15


@dataclasses.dataclass
class Problem:
    """One minimum-time problem on a box with a structured grid.

    ``n`` holds nodes per side (n nodes, n - 1 cells); spacing is equal on
    every axis.  ``n_coarse`` is None for a plain global solve, else the
    coarse grid of the patchy method (Sec. 3, Step 1).  Target j is patch j.
    """

    dim: int
    n: Tuple[int, int, int]
    lo: Tuple[float, float, float]
    hi: Tuple[float, float, float]
    speed: str
    speed_params: np.ndarray          # float64[64]
    controls: np.ndarray              # float64[n_controls, dim]
    targets: np.ndarray               # float64[n_targets, dim + 1] (centre, radius)
    tol: float = 1e-6
    n_coarse: Optional[Tuple[int, int, int]] = None
    tol_coarse: float = 1e-12
    tol_phi: float = 1e-10
    max_sweeps: int = 100000
    name: str = ""
    # dynamics: "speed" f = c(x) a; "drift" f = s a + w with drift = (s, w1, w2, w3)
    dyn: str = "speed"
    drift: Tuple[float, float, float, float] = (1.0, 0.0, 0.0, 0.0)
    # target: "balls" (row j = ball j = part j), "sectors" (row 0 = one ball in
    # n_parts angular sectors), "slab" (row 0 = (v, ., r): |x1 - v| <= r in
    # n_parts pieces along x2)
    target_kind: str = "balls"
    n_parts: int = 0
    # obstacles: rows (kind, p0..p5), kind 0 = closed ball (centre p0..p2,
    # radius p3), kind 1 = closed box (lower corner p0..p2, upper p3..p5);
    # their nodes are state constraints like the ghost ring
    obstacles: Optional[np.ndarray] = None

    @property
    def spacing(self) -> float:
        return (self.hi[0] - self.lo[0]) / (self.n[0] - 1)

    @property
    def n_nodes(self) -> int:
        return int(np.prod(self.n[: self.dim]))

    @property
    def n_controls(self) -> int:
        return int(self.controls.shape[0])

    @property
    def n_targets(self) -> int:
        return int(self.targets.shape[0])

    @property
    def n_patches(self) -> int:
        """R: one patch per target row, or n_parts for a split target."""
        return self.n_targets if self.target_kind == "balls" else int(self.n_parts)

    def with_(self, **kw) -> "Problem":
        return dataclasses.replace(self, **kw)


def _snap(a: np.ndarray) -> np.ndarray:
    a = np.array(a, dtype=np.float64)
    a[np.abs(a) < SNAP] = 0.0
    return a


def controls_2d(n_c: int, phase: float = 0.0) -> np.ndarray:
    """N_c unit vectors at angles 2 pi m / N_c (+ phase), m = 0..N_c-1."""
    th = 2.0 * math.pi * np.arange(n_c, dtype=np.float64) / n_c + phase
    return _snap(np.stack([np.cos(th), np.sin(th)], axis=1))


def controls_axes(dim: int) -> np.ndarray:
    """The 2d axis directions +-e_d (every foot lands exactly on a node)."""
    out = []
    for d in range(dim):
        for s in (1.0, -1.0):
            v = np.zeros(dim)
            v[d] = s
            out.append(v)
    return np.array(out, dtype=np.float64)


def controls_fibonacci(n_c: int) -> np.ndarray:
    """Spherical Fibonacci lattice with n_c points on S^2.

    z_m = 1 - (2m + 1)/n_c, azimuth m * pi (3 - sqrt 5), m = 0..n_c-1.
    """
    m = np.arange(n_c, dtype=np.float64)
    z = 1.0 - (2.0 * m + 1.0) / n_c
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ang = m * math.pi * (3.0 - math.sqrt(5.0))
    return _snap(np.stack([r * np.cos(ang), r * np.sin(ang), z], axis=1))


def _pad3(t: Sequence, fill) -> Tuple:
    t = list(t)
    while len(t) < 3:
        t.append(fill)
    return tuple(t)


def _params(values: Sequence[float] = ()) -> np.ndarray:
    p = np.zeros(64, dtype=np.float64)
    p[: len(values)] = values
    return p


def place_targets(rng: np.random.Generator, dim: int, count: int, lo: float, hi: float,
                  radius: float, min_sep: float) -> np.ndarray:
    """Centres uniform in [lo + 0.25, hi - 0.25]^dim, rejecting any centre
    closer than ``min_sep`` to an earlier one."""
    centres: List[np.ndarray] = []
    tries = 0
    while len(centres) < count:
        tries += 1
        if tries > 100000:
            raise RuntimeError("target placement failed")
        c = rng.uniform(lo + 0.25, hi - 0.25, size=dim)
        if all(np.linalg.norm(c - o) >= min_sep for o in centres):
            centres.append(c)
    t = np.zeros((count, dim + 1), dtype=np.float64)
    t[:, :dim] = np.array(centres)
    t[:, dim] = radius
    return t


def coarse_side(n: int) -> int:
    """Coarse side used by the batched and served families: 33, or (n-1)/8 + 1
    for large grids, never more than the fine side itself."""
    return min(n, max(33, int(math.ceil((n - 1) / 8)) + 1))


# ---------------------------------------------------------------------------
# Named workloads
# ---------------------------------------------------------------------------

def eikonal2d(n: int = 101, n_c: int = 32, radius: float = 0.1, tol: float = 1e-10,
              box: float = 2.0) -> Problem:
    """Plain global SL, 2D eikonal, FP64: f = a, disk target at the origin,
    Omega = [-box, box]^2; closed form u = max(|x| - r, 0)."""
    return Problem(
        dim=2, n=(n, n, 1), lo=(-box, -box, 0.0), hi=(box, box, 0.0), speed="one",
        speed_params=_params(), controls=controls_2d(n_c),
        targets=np.array([[0.0, 0.0, radius]]), tol=tol, name=f"eikonal2d_n{n}_nc{n_c}")


def sincos2d(seed: int = 0, n: int = 2049, n_coarse: int = 65, n_c: int = 64,
             n_targets: int = 4, radius: float = 0.05, tol: float = 1e-6,
             amplitude: float = 0.5) -> Problem:
    """2D patchy workload: c = 1 + 0.5 sin(2 pi x1) cos(2 pi x2) on [-2,2]^2,
    N_c = 64, four disks r = 0.05 at seeded centres (one patch each)."""
    rng = np.random.default_rng(seed)
    kc = 4.0 / (n_coarse - 1)
    tg = place_targets(rng, 2, n_targets, -2.0, 2.0, radius, 4 * radius + 2 * kc)
    return Problem(
        dim=2, n=(n, n, 1), lo=(-2.0, -2.0, 0.0), hi=(2.0, 2.0, 0.0), speed="sincos2d",
        speed_params=_params([amplitude]), controls=controls_2d(n_c), targets=tg, tol=tol,
        n_coarse=(n_coarse, n_coarse, 1), name=f"sincos2d_n{n}_c{n_coarse}_s{seed}")


def sin3d(seed: int = 0, n: int = 257, n_coarse: int = 33, n_c: int = 98,
          n_targets: int = 8, radius: float = 0.05, tol: float = 1e-6,
          amplitude: float = 0.3) -> Problem:
    """3D patchy workload: c = 1 + 0.3 sin(pi x1) sin(pi x2) sin(pi x3) on
    [-1,1]^3, 98 Fibonacci controls, eight balls r = 0.05 (eight patches)."""
    rng = np.random.default_rng(seed)
    kc = 2.0 / (n_coarse - 1)
    tg = place_targets(rng, 3, n_targets, -1.0, 1.0, radius, 4 * radius + 2 * kc)
    return Problem(
        dim=3, n=(n, n, n), lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0), speed="sin3d",
        speed_params=_params([amplitude]), controls=controls_fibonacci(n_c), targets=tg,
        tol=tol, n_coarse=(n_coarse, n_coarse, n_coarse), name=f"sin3d_n{n}_c{n_coarse}_s{seed}")


def fourier_params(rng: np.random.Generator) -> np.ndarray:
    """a_pq ~ U[-1,1], theta_pq, psi_pq ~ U[0, 2 pi), p, q = 0..3, laid out as
    [a(16), theta(16), psi(16)] row-major in (p, q)."""
    a = rng.uniform(-1.0, 1.0, size=16)
    th = rng.uniform(0.0, 2.0 * math.pi, size=16)
    ps = rng.uniform(0.0, 2.0 * math.pi, size=16)
    return _params(np.concatenate([a, th, ps]))


def fourier2d(rng: np.random.Generator, n: int, n_c: int, n_targets: int,
              radius: float = 0.05, tol: float = 1e-6, name: str = "") -> Problem:
    """One problem of the batched family: [-2,2]^2, Fourier speed field."""
    nc = coarse_side(n)
    kc = 4.0 / (nc - 1)
    tg = place_targets(rng, 2, n_targets, -2.0, 2.0, radius, 4 * radius + 2 * kc)
    return Problem(
        dim=2, n=(n, n, 1), lo=(-2.0, -2.0, 0.0), hi=(2.0, 2.0, 0.0), speed="fourier2d",
        speed_params=fourier_params(rng), controls=controls_2d(n_c), targets=tg, tol=tol,
        n_coarse=(nc, nc, 1), name=name or f"fourier2d_n{n}")


def batched(seed: int = 0, count: int = 512, side=(65, 513), n_c=(32, 64),
            n_targets=(1, 8)) -> List[Problem]:
    """Batched family: ``count`` problems, side ~ U{65..513}, R ~ U{1..8},
    N_c ~ U{32..64}, Fourier speed field, r = 0.05, tol 1e-6."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(side[0], side[1] + 1))
        nc = int(rng.integers(n_c[0], n_c[1] + 1))
        r = int(rng.integers(n_targets[0], n_targets[1] + 1))
        out.append(fourier2d(rng, n, nc, r, name=f"batch{seed}_{i}"))
    return out


def serving_stream(seed: int = 0, count: int = 2000, rate: float = 200.0,
                   side2d=(129, 1025), side3d=(65, 193)) -> List[Tuple[float, Problem]]:
    """Served family: Poisson arrivals (mean ``rate``/s); 80% 2D Fourier
    problems, 20% 3D sin3d-family problems with 1..8 targets."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        if rng.uniform() < 0.8:
            n = int(rng.integers(side2d[0], side2d[1] + 1))
            p = fourier2d(rng, n, int(rng.integers(32, 65)), int(rng.integers(1, 9)),
                          name=f"req{i}")
        else:
            n = int(rng.integers(side3d[0], side3d[1] + 1))
            nc = coarse_side(n)
            r = int(rng.integers(1, 9))
            kc = 2.0 / (nc - 1)
            tg = place_targets(rng, 3, r, -1.0, 1.0, 0.05, 4 * 0.05 + 2 * kc)
            p = Problem(dim=3, n=(n, n, n), lo=(-1.0, -1.0, -1.0), hi=(1.0, 1.0, 1.0),
                        speed="sin3d", speed_params=_params([0.3]),
                        controls=controls_fibonacci(98), targets=tg, tol=1e-6,
                        n_coarse=(nc, nc, nc), name=f"req{i}")
        out.append((t, p))
    return out


def random_speed_problem(seed: int, n: int = 9, n_c: int = 8, dim: int = 2,
                         n_targets: int = 1, box: float = 1.0) -> Problem:
    """Tiny seeded problem with a random Fourier speed field (2D) or the
    sin3d field (3D), used by brute-force pins on 9x9 / 9^3 grids."""
    rng = np.random.default_rng(seed)
    if dim == 2:
        ctl = controls_2d(n_c, phase=float(rng.uniform(0, 2 * math.pi / n_c)))
        k = 2 * box / (n - 1)
        centres = rng.integers(1, n - 1, size=(n_targets, 2)) * k - box
        tg = np.concatenate([centres, np.full((n_targets, 1), 0.01)], axis=1)
        return Problem(dim=2, n=(n, n, 1), lo=(-box, -box, 0.0), hi=(box, box, 0.0),
                       speed="fourier2d", speed_params=fourier_params(rng), controls=ctl,
                       targets=tg, tol=1e-13, name=f"tiny2d_s{seed}")
    ctl = controls_fibonacci(n_c)
    k = 2 * box / (n - 1)
    centres = rng.integers(1, n - 1, size=(n_targets, 3)) * k - box
    tg = np.concatenate([centres, np.full((n_targets, 1), 0.01)], axis=1)
    return Problem(dim=3, n=(n, n, n), lo=(-box,) * 3, hi=(box,) * 3, speed="sin3d",
                   speed_params=_params([0.3]), controls=ctl, targets=tg, tol=1e-13,
                   name=f"tiny3d_s{seed}")


# ------------------------------------------------- the paper's 2D tests --

def eikonal_sectors(n: int = 201, n_coarse: int = 51, n_c: int = 32, parts: int = 16, radius: float = 0.5,
                    tol: float = 1e-6) -> Problem:
    """Table 1, Eikonal: f = a on [-2,2]^2, target B(0, 0.5) split into R equal
    angular sectors (one patch each)."""
    return Problem(dim=2, n=(n, n, 1), lo=(-2.0, -2.0, 0.0), hi=(2.0, 2.0, 0.0), speed="one",
                   speed_params=np.zeros(64), controls=controls_2d(n_c),
                   targets=np.array([[0.0, 0.0, radius]]), tol=tol, n_coarse=(n_coarse, n_coarse, 1),
                   name=f"eikonal_sectors{n}", target_kind="sectors", n_parts=parts)


def zermelo(n: int = 201, n_coarse: int = 51, n_c: int = 32, parts: int = 16, radius: float = 0.5,
            s: float = 2.1, w: Tuple[float, float] = (2.0, 0.0), tol: float = 1e-6) -> Problem:
    """Table 1, Zermelo: f = s a + w (s = 2.1, w = (2, 0)) on [-2,2]^2, target
    B(0, 0.5) split into R sectors."""
    return Problem(dim=2, n=(n, n, 1), lo=(-2.0, -2.0, 0.0), hi=(2.0, 2.0, 0.0), speed="one",
                   speed_params=np.zeros(64), controls=controls_2d(n_c),
                   targets=np.array([[0.0, 0.0, radius]]), tol=tol, n_coarse=(n_coarse, n_coarse, 1),
                   name=f"zermelo{n}", dyn="drift", drift=(s, w[0], w[1], 0.0), target_kind="sectors",
                   n_parts=parts)


# ------------------------------------------------- the paper's 3D tests --

def eikonal3d(n: int = 101, n_coarse: int = 51, n_c: int = 189, parts: int = 8, radius: float = 0.5,
              tol: float = 1e-6, split: str = "orthants") -> Problem:
    """Sec. 7, Eikonal 3D: f = a on [-2,2]^3, target B(0, 0.5) split into its
    8 octants (split="orthants") or into R wedges by the azimuth around the
    x3 axis (split="sectors"); N_c Fibonacci controls (the paper's 189
    geosphere vertices, count kept)."""
    if split == "orthants":
        parts = 8
    return Problem(dim=3, n=(n, n, n), lo=(-2.0,) * 3, hi=(2.0,) * 3, speed="one", speed_params=np.zeros(64),
                   controls=controls_fibonacci(n_c), targets=np.array([[0.0, 0.0, 0.0, radius]]), tol=tol,
                   n_coarse=(n_coarse,) * 3, name=f"eikonal3d_{n}", target_kind=split, n_parts=parts)


def fan3d(n: int = 101, n_coarse: int = 51, n_c: int = 189, parts: int = 8, half_width: float = 1e-9,
          tol: float = 1e-6) -> Problem:
    """Sec. 7, Fan 3D: c(x) = |x1 + x2 + x3 + 0.1| on [-2,2]^3, target the
    plane x1 = 0 (a slab of half-width ``half_width``) split into R strips
    along x2; N_c Fibonacci controls."""
    q = np.zeros(64)
    q[:4] = (0.1, 1.0, 1.0, 1.0)
    return Problem(dim=3, n=(n, n, n), lo=(-2.0,) * 3, hi=(2.0,) * 3, speed="fan", speed_params=q,
                   controls=controls_fibonacci(n_c), targets=np.array([[0.0, 0.0, 0.0, half_width]]), tol=tol,
                   n_coarse=(n_coarse,) * 3, name=f"fan3d_{n}", target_kind="slab", n_parts=parts)


def controls_brockett(amax: float = 5.0) -> np.ndarray:
    """Sec. 7, Brockett: the nine controls {-amax, 0, amax}^2 as rows
    (a1, a2, 0) (the third entry is unused; a = 0 cannot move)."""
    v = (-amax, 0.0, amax)
    return np.array([[a1, a2, 0.0] for a2 in v for a1 in v], dtype=np.float64)


def brockett3d(n: int = 101, n_coarse: int = 51, amax: float = 5.0, radius: float = 0.25,
               tol: float = 1e-6, split: str = "orthants") -> Problem:
    """Sec. 7, Brockett 3D: f = (a1, a2, x1 a2 - x2 a1), a in {-5, 0, 5}^2, on
    [-2,2]^3, target B(0, 0.25) split into its 8 octants."""
    return Problem(dim=3, n=(n, n, n), lo=(-2.0,) * 3, hi=(2.0,) * 3, speed="one", speed_params=np.zeros(64),
                   controls=controls_brockett(amax), targets=np.array([[0.0, 0.0, 0.0, radius]]), tol=tol,
                   n_coarse=(n_coarse,) * 3, name=f"brockett3d_{n}", dyn="brockett", target_kind=split, n_parts=8)


def obstacle_ball(centre, radius) -> List[float]:
    c = list(centre) + [0.0] * (3 - len(centre))
    return [0.0, c[0], c[1], c[2], float(radius), 0.0, 0.0]


def obstacle_box(lo, hi) -> List[float]:
    a = list(lo) + [0.0] * (3 - len(lo))
    b = list(hi) + [0.0] * (3 - len(hi))
    return [1.0, a[0], a[1], a[2], b[0], b[1], b[2]]


def eikonal_obstacles(n: int = 201, n_coarse: int = 51, n_c: int = 32, parts: int = 8, radius: float = 0.5,
                      tol: float = 1e-6) -> Problem:
    """Sec. 4, eikonal with obstacles: f = a on [-2,2]^2, target B(0, 0.5) in R
    sectors, one disk and one rectangle as obstacles (the paper gives no
    sizes: disk B((1.1, 0.9), 0.35), box [-1.6, -0.9] x [-1.3, 0.5])."""
    obs = np.array([obstacle_ball((1.1, 0.9), 0.35), obstacle_box((-1.6, -1.3), (-0.9, 0.5))])
    return eikonal_sectors(n=n, n_coarse=n_coarse, n_c=n_c, parts=parts, radius=radius, tol=tol).with_(
        obstacles=obs, name=f"eikonal_obstacles{n}")


def fan(n: int = 201, n_coarse: int = 51, n_c: int = 32, parts: int = 16, half_width: float = 1e-9,
        tol: float = 1e-6) -> Problem:
    """Table 1, Fan: c(x) = |x1 + x2 + 0.1| on [-2,2]^2, target the line x1 = 0
    (a slab of half-width ``half_width``) split into R pieces along x2."""
    q = np.zeros(64)
    q[:4] = (0.1, 1.0, 1.0, 0.0)
    return Problem(dim=2, n=(n, n, 1), lo=(-2.0, -2.0, 0.0), hi=(2.0, 2.0, 0.0), speed="fan",
                   speed_params=q, controls=controls_2d(n_c), targets=np.array([[0.0, 0.0, half_width]]),
                   tol=tol, n_coarse=(n_coarse, n_coarse, 1), name=f"fan{n}", target_kind="slab",
                   n_parts=parts)
