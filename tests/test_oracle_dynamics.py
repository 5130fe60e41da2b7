"""Pins for the oracle's other dynamics and split targets (Table 1): the
Zermelo drift f = s a + w, the Fan speed c = |x1 + x2 + 0.1| with its
zero-speed line, and targets split into R sectors or pieces.  Each is checked
against something other than the oracle's own arithmetic: a closed form,
exact policy iteration, Dijkstra, the geometry of the eikonal's radial
characteristics, and the paper's printed patchy errors (Tables 2-4).
"""
import math
import os

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

import oracle
import workloads as W
from tests import _indep as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_patchy_errors.txt")


def _zermelo_time(x, s, w, r):
    """Minimum time to the ball B(0, r) under f = s a + w, |a| <= 1, s > |w|:
    the smallest T >= 0 with |x + w T| = s T + r (the reachable set after time
    T is the ball of radius s T around x + w T; a straight path, so the box's
    state constraints never bind)."""
    a = w @ w - s * s
    b = 2.0 * (x @ w - s * r)
    c = x @ x - r * r
    if c <= 0.0:
        return 0.0
    return (-b - math.sqrt(b * b - 4.0 * a * c)) / (2.0 * a)


def _drift_ball(n, n_c=64, s=1.0, w=(0.5, 0.0), r=0.5):
    return W.zermelo(n=n, n_c=n_c, s=s, w=w).with_(n_coarse=None, target_kind="balls", n_parts=0,
                                                   targets=np.array([[0.0, 0.0, r]]), tol=1e-12)


def test_zermelo_closed_form_first_order():
    """Drift dynamics against the closed-form minimum time: the mean error
    halves with the grid step (first order) and the max error stays below 2k."""
    errs = []
    for n in (41, 81, 161):
        p = _drift_ball(n)
        g = oracle.global_solve(p)
        x = oracle.grid_coords(p)
        T = np.array([_zermelo_time(xi, 1.0, np.array([0.5, 0.0]), 0.5) for xi in x])
        fin = np.isfinite(g.u)
        kind, _, _ = I.kinds(p)
        assert np.array_equal(fin, kind != 2)
        e = np.abs(g.u[fin] - T[fin])
        assert e.max() <= 2.0 * p.spacing
        errs.append(e.mean())
    assert errs[1] <= 0.6 * errs[0] and errs[2] <= 0.6 * errs[1]


def test_zero_drift_is_the_eikonal():
    """f = 1 a + 0 is the eikonal: the drift code path (directions a/|a|,
    steps k/|a|, equal to a and k up to the last bit) gives the same global
    and patchy solutions; labels may differ only where the feedback ties."""
    e = W.eikonal_sectors(n=61, n_coarse=16, parts=6).with_(tol=1e-13)
    z = W.zermelo(n=61, n_coarse=16, parts=6, s=1.0, w=(0.0, 0.0)).with_(tol=1e-13)
    ge = oracle.global_solve(e.with_(n_coarse=None))
    gz = oracle.global_solve(z.with_(n_coarse=None))
    fin = np.isfinite(ge.u)
    assert np.array_equal(fin, np.isfinite(gz.u))
    np.testing.assert_allclose(gz.u[fin], ge.u[fin], rtol=0, atol=1e-11)
    a = oracle.patchy_solve(e)
    b = oracle.patchy_solve(z)
    assert np.mean(a.labels == b.labels) >= 0.999
    fin = np.isfinite(a.u) & np.isfinite(b.u)
    assert np.abs(a.u[fin] - b.u[fin]).max() <= 1e-3


def _policy_iteration_steps(p):
    """Exact fixed point of F for per-control directions and time steps, by
    policy iteration with dense linear solves (Q1 weights as transition
    probabilities)."""
    kind, _, h = I.kinds(p)
    idx, x = I.node_grid(p)
    dirs, g = I.control_steps(p)
    free = np.nonzero(kind == 0)[0]
    pos = {int(i): q for q, i in enumerate(free)}
    acts = {}
    for i in free:
        lst = []
        for m in range(dirs.shape[0]):
            cs = I.q1_corners(p, idx[i], dirs[m])
            lst.append(None if any(kind[j] == 2 for j, _ in cs) else (cs, h[i] * g[m]))
        acts[int(i)] = lst
    tgt_x = x[kind == 1]
    dist = lambda j: np.min(np.linalg.norm(tgt_x - x[j], axis=1))
    pol = {}
    for i in free:
        cand = [(sum(w * dist(j) for j, w in a[0]) + a[1], m) for m, a in enumerate(acts[int(i)]) if a]
        pol[int(i)] = min(cand)[1]
    for _ in range(300):
        A = np.eye(len(free))
        b = np.zeros(len(free))
        for i in free:
            cs, hh = acts[int(i)][pol[int(i)]]
            b[pos[int(i)]] = hh
            for j, w in cs:
                if kind[j] == 0:
                    A[pos[int(i)], pos[j]] -= w
        v = np.linalg.solve(A, b)
        full = np.where(kind == 1, 0.0, np.inf)
        full[free] = v
        changed = False
        for i in free:
            q = [np.inf if a is None else a[1] + sum(w * full[j] for j, w in a[0]) for a in acts[int(i)]]
            m = int(np.argmin(q))
            if q[m] < q[pol[int(i)]] - 1e-13:
                pol[int(i)] = m
                changed = True
        if not changed:
            return full
    raise AssertionError("policy iteration did not stop")


@pytest.mark.parametrize("seed", range(3))
def test_drift_policy_iteration_9x9(seed):
    """Brute force on 9x9 with a drift: value iteration equals exact policy
    iteration over the directions f/|f| with steps k/|f|."""
    rng = np.random.default_rng(seed)
    w = rng.uniform(-0.6, 0.6, size=2)
    p = W.random_speed_problem(seed, n=9, n_c=12).with_(dyn="drift", drift=(1.0, w[0], w[1], 0.0),
                                                         speed="one", tol=1e-14)
    ref = _policy_iteration_steps(p)
    r = oracle.global_solve(p, tol=1e-14)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-11)


def test_fan_axis_controls_equal_dijkstra():
    """Fan speed with the four axis controls: every foot lands on a node, so
    the fixed point is Dijkstra on the axis graph with cost h_i = k / c(x_i)
    leaving node i; nodes on the zero-speed line cannot move."""
    p = W.fan(n=41, n_coarse=11, parts=4).with_(n_coarse=None, controls=W.controls_2d(4), tol=1e-14)
    kind, _, h = I.kinds(p)
    idx, _ = I.node_grid(p)
    N = kind.size
    rows, cols, vals = [], [], []
    for i in np.nonzero(kind == 0)[0]:
        for d in ((1, 0), (-1, 0), (0, 1), (0, -1)):
            j = int(I.linear(p, idx[i] + np.array(d))[0])
            if kind[j] != 2:
                rows.append(i)
                cols.append(j)
                vals.append(h[i])
    G = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    # distances from every node to the target: shortest paths on the reversed graph
    dist = dijkstra(G.T, directed=True, indices=np.nonzero(kind == 1)[0], min_only=True)
    ref = np.where(kind == 2, np.inf, dist)
    r = oracle.global_solve(p)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-11)


def test_target_parts_follow_the_definitions():
    """Target parts of the split targets equal the independent restatement
    (sectors by angle, slab pieces along x2), and every part is used."""
    for p in (W.eikonal_sectors(n=81, n_coarse=21, parts=16), W.fan(n=81, n_coarse=21, parts=16)):
        kind, part, _ = oracle.setup(p)
        ik, ipart, _ = I.kinds(p)
        assert np.array_equal(kind, ik)
        assert np.array_equal(part, ipart)
        assert set(part[part >= 0]) == set(range(16))


def test_sector_labels_follow_radial_characteristics():
    """Eikonal with a disk split into sectors: characteristics are radial, so
    a node's patch is the sector of its angle except within a few nodes of a
    sector boundary ray."""
    p = W.eikonal_sectors(n=101, n_coarse=51, parts=16).with_(tol=1e-10)
    r = oracle.patchy_solve(p)
    x = oracle.grid_coords(p)
    th = np.mod(np.arctan2(x[:, 1], x[:, 0]), 2 * math.pi)
    sector = np.floor(16 * th / (2 * math.pi) + 1e-9).astype(int) % 16
    lab = r.labels
    ok = lab >= 0
    agree = np.mean(lab[ok] == sector[ok])
    assert agree >= 0.95
    bnd = np.abs(((16 * th / (2 * math.pi) + 0.5) % 1.0) - 0.5) * (2 * math.pi / 16) * np.hypot(x[:, 0], x[:, 1])
    bad = ok & (lab != sector)
    assert np.all(bnd[bad] <= 4 * p.spacing)


def _golden():
    rows = []
    for line in open(GOLDEN):
        if line.strip() and not line.startswith("#"):
            d, c, f, e1, einf = line.split()
            rows.append((d, int(c), int(f), float(e1), float(einf)))
    return rows


@pytest.mark.parametrize("dyn", ["eikonal", "fan", "zermelo"])
def test_patchy_error_matches_paper_tables(dyn):
    """Sec. 4.2, Tables 2-4: the patchy error E1 at the paper's sizes
    (coarse 50 -> fine 100 cells, R = 16, N_c = 32) is within a factor 10 of
    the printed value.  The paper leaves the grid convention, the sector
    layout and the coarse target unstated (R6, R16, R22), so only the order
    of magnitude is fixed; a wrong drift sign, speed field or part layout
    moves E1 by far more."""
    make = {"eikonal": W.eikonal_sectors, "fan": W.fan, "zermelo": W.zermelo}[dyn]
    row = next(r for r in _golden() if r[0] == dyn and r[1] == 50 and r[2] == 100)
    p = make(n=101, n_coarse=51, parts=16).with_(tol=1e-10)
    r = oracle.patchy_solve(p)
    g = oracle.global_solve(p.with_(n_coarse=None), tol=1e-10)
    e1, einf = oracle.patchy_error(r.u, g.u)
    assert row[3] / 10 <= e1 <= row[3] * 10, (e1, row)
    assert einf >= e1


def test_3d_target_parts_follow_the_definitions():
    """Sec. 7 targets in 3D: the ball in R wedges around the x3 axis or in its
    octants (and a disk in its quadrants) and the plane x1 = 0 in R strips
    along x2 equal the independent restatement;
    every part is used and the Fan speed's zero plane holds no node here."""
    for p in (W.eikonal3d(n=33, n_coarse=9, n_c=14, split="sectors"), W.eikonal3d(n=33, n_coarse=9, n_c=14),
              W.fan3d(n=33, n_coarse=9, n_c=14), W.eikonal_sectors(n=41, n_coarse=11).with_(target_kind="orthants",
                                                                                         n_parts=4)):
        kind, part, _ = oracle.setup(p)
        ik, ipart, _ = I.kinds(p)
        assert np.array_equal(kind, ik)
        assert np.array_equal(part, ipart)
        assert set(part[part >= 0]) == set(range(p.n_parts))


@pytest.mark.parametrize("obstacles", [False, True])
def test_fan3d_axis_controls_equal_dijkstra(obstacles):
    """Fan 3D with the six axis controls: the fixed point is Dijkstra on the
    axis graph with cost h_i = k / c(x_i) leaving node i; with a ball and a
    box as obstacles (R23) their nodes leave the graph."""
    p = W.fan3d(n=21, n_coarse=7).with_(n_coarse=None, controls=W.controls_axes(3), tol=1e-14)
    if obstacles:
        p = p.with_(obstacles=np.array([W.obstacle_ball((0.9, 0.3, -0.2), 0.6),
                                        W.obstacle_box((-1.4, -0.6, -1.0), (-0.5, 0.8, 1.2))]))
        assert (I.kinds(p)[0] == 2).sum() > (I.kinds(p.with_(obstacles=None))[0] == 2).sum() + 100
    kind, _, h = I.kinds(p)
    idx, _ = I.node_grid(p)
    N = kind.size
    rows, cols, vals = [], [], []
    for i in np.nonzero(kind == 0)[0]:
        for d in np.vstack([np.eye(3, dtype=int), -np.eye(3, dtype=int)]):
            j = int(I.linear(p, idx[i] + d)[0])
            if kind[j] != 2:
                rows.append(i)
                cols.append(j)
                vals.append(h[i])
    G = sp.csr_matrix((vals, (rows, cols)), shape=(N, N))
    dist = dijkstra(G.T, directed=True, indices=np.nonzero(kind == 1)[0], min_only=True)
    ref = np.where(kind == 2, np.inf, dist)
    r = oracle.global_solve(p)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-11)


def test_eikonal3d_sector_labels_follow_the_azimuth():
    """Eikonal 3D, ball in 8 wedges: characteristics are radial, so a node's
    patch is the wedge of its azimuth except within a few nodes of a wedge
    boundary plane (the colour transport smears the labels over a band that
    is wider in 3D, with 50 directions, than in 2D)."""
    p = W.eikonal3d(n=33, n_coarse=17, n_c=50, split="sectors").with_(tol=1e-10)
    r = oracle.patchy_solve(p)
    x = oracle.grid_coords(p)
    th = np.mod(np.arctan2(x[:, 1], x[:, 0]), 2 * math.pi)
    wedge = np.floor(8 * th / (2 * math.pi) + 1e-9).astype(int) % 8
    ok = r.labels >= 0
    assert np.mean(r.labels[ok] == wedge[ok]) >= 0.75
    rho = np.hypot(x[:, 0], x[:, 1])
    bnd = np.abs(((8 * th / (2 * math.pi) + 0.5) % 1.0) - 0.5) * (2 * math.pi / 8) * rho
    bad = ok & (r.labels != wedge)
    assert np.all(bnd[bad] <= 7 * p.spacing)


def test_eikonal3d_octant_labels_follow_the_signs():
    """Eikonal 3D, ball in its octants: characteristics are radial, so a
    node's patch is the octant of x itself except within a few nodes of a
    coordinate plane (the band the colour transport smears, as for wedges)."""
    p = W.eikonal3d(n=33, n_coarse=17, n_c=50).with_(tol=1e-10)
    r = oracle.patchy_solve(p)
    x = oracle.grid_coords(p)
    octant = (x[:, 0] >= 0).astype(int) | ((x[:, 1] >= 0).astype(int) << 1) | ((x[:, 2] >= 0).astype(int) << 2)
    ok = r.labels >= 0
    assert np.mean(r.labels[ok] == octant[ok]) >= 0.8
    bad = ok & (r.labels != octant)
    assert np.all(np.abs(x[bad]).min(axis=1) <= 7 * p.spacing)


def _policy_iteration_nodewise(p):
    """Exact fixed point of F with per-(node, control) directions and time
    steps.  S* (R14) is restated as the greatest set S of free nodes from
    which the target is reached with controls whose positive-weight corners
    all lie in S or the target: reach breadth-first from the target, drop
    what was not reached, repeat.  The control that first reached a node
    moves it to an earlier node with positive probability, so that policy is
    proper; policy iteration with dense linear solves then gives the exact
    fixed point on S*, +inf elsewhere."""
    kind, _, _ = I.kinds(p)
    idx, x = I.node_grid(p)
    dirs, hs = I.node_control_steps(p, x)
    free = np.nonzero(kind == 0)[0]
    corners = {int(i): [None if not np.isfinite(hs[i, m]) else I.q1_corners(p, idx[i], dirs[i, m])
                        for m in range(dirs.shape[1])] for i in free}
    S = set(int(i) for i in free)
    while True:
        ok = lambda j: kind[j] == 1 or j in S
        level, first = {}, {}
        frontier = True
        while frontier:
            frontier = False
            for i in sorted(S - set(level)):
                for m, cs in enumerate(corners[i]):
                    if cs is None or not all(ok(j) for j, _ in cs):
                        continue
                    if any(kind[j] == 1 or (j in level and j != i) for j, _ in cs):
                        level[i], first[i] = len(level), m
                        frontier = True
                        break
        if set(level) == S:
            break
        S = set(level)
    Sl = sorted(S)
    pos = {i: q for q, i in enumerate(Sl)}
    usable = lambda i, m: corners[i][m] is not None and all(kind[j] == 1 or j in S for j, _ in corners[i][m])
    pol = dict(first)
    for _ in range(300):
        A = np.eye(len(Sl))
        b = np.zeros(len(Sl))
        for i in Sl:
            m = pol[i]
            b[pos[i]] = hs[i, m]
            for j, w in corners[i][m]:
                if j in pos:
                    A[pos[i], pos[j]] -= w
        v = np.linalg.solve(A, b)
        full = np.where(kind == 1, 0.0, np.inf)
        full[Sl] = v
        changed = False
        for i in Sl:
            q = [hs[i, m] + sum(w * full[j] for j, w in corners[i][m]) if usable(i, m) else np.inf
                 for m in range(dirs.shape[1])]
            m = int(np.argmin(q))
            if q[m] < q[pol[i]] - 1e-13:
                pol[i] = m
                changed = True
        if not changed:
            return full
    raise AssertionError("policy iteration did not stop")


def test_brockett_policy_iteration_9x9x9():
    """Brute force on 9^3 (343 free nodes) for Brockett's integrator: value
    iteration equals exact policy iteration over the per-node directions
    f/|f| and steps k/|f| with f = (a1, a2, x1 a2 - x2 a1)."""
    p = W.brockett3d(n=9, n_coarse=5, radius=0.6).with_(n_coarse=None, tol=1e-14)
    ref = _policy_iteration_nodewise(p)
    r = oracle.global_solve(p, tol=1e-14)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-11)


def test_brockett_symmetries_and_axis():
    """Brockett's f is equivariant under the rotation (x1, x2, x3) ->
    (-x2, x1, x3) (controls rotated alike) and the reflection (x1, x2, x3) ->
    (x2, x1, -x3) (controls swapped), and the control set and target are
    invariant, so the solution is too; a wrong sign in x1 a2 - x2 a1 breaks
    the reflection.  On the x1 axis the fastest motion is straight along it
    at speed 5 (a1 = -5 keeps x2 = x3 = 0), which lands on nodes: there the
    scheme gives the exact time (|x1| - 0.25) / 5."""
    n = 33
    p = W.brockett3d(n=n, n_coarse=17).with_(n_coarse=None)
    U = oracle.global_solve(p, tol=1e-13).u.reshape(n, n, n)   # [x3, x2, x1]
    fin = np.isfinite(U)
    rot = np.stack([U[z].T[:, ::-1] for z in range(n)])
    refl = U[::-1].transpose(0, 2, 1)
    for V in (rot, refl):
        assert np.array_equal(fin, np.isfinite(V))
        assert np.abs(U[fin] - V[fin]).max() <= 1e-12
    x1 = -2.0 + 4.0 * np.arange(n) / (n - 1)
    axis = U[n // 2, n // 2, 1:-1]
    np.testing.assert_allclose(axis, np.maximum(np.abs(x1[1:-1]) - 0.25, 0.0) / 5.0, rtol=0, atol=1e-12)


def _coarse_band(p, r):
    """Coarse nodes in the widened target band of R6 (outside the ball, within
    r + k~ sqrt(d)/2 of its centre, clear of the band's edges), with their
    coordinates, gap to the ball and unit direction towards the centre."""
    q = p.with_(n=p.n_coarse)
    _, x = I.node_grid(q)
    c, rad = p.targets[0][: p.dim], p.targets[0][p.dim]
    dist = np.linalg.norm(x - c, axis=1)
    edge = rad + q.spacing * math.sqrt(p.dim) / 2.0
    band = (dist > rad + 1e-9) & (dist < edge - 1e-9)
    # the grids are chosen so that the band holds nodes farther than half a
    # coarse cell from the ball: the widening is k~ sqrt(d) / 2, not k~ / 2
    assert np.any(dist[band] > rad + q.spacing / 2.0 + 1e-9)
    e = (c - x[band]) / dist[band, None]
    return band, x[band], dist[band] - rad, e, r.ucoarse[band]


def test_coarse_boundary_values_follow_the_approach_speed():
    """R6 and R24: the widened coarse target holds gap / v, v the largest
    speed the dynamics allow towards the target.  Checked by the defining
    property of v, not by its formula: for c(x) a, U c(x) = gap; for the
    drift s a + w, v = gap / U is the largest speed with a unit control
    (|v e - w| = s, and a larger v needs |a| > 1); for Brockett, v is the
    largest |f(x, a)| over the controls."""
    # speed field: sincos2d on the sectors problem
    p = W.eikonal_sectors(n=81, n_coarse=21, parts=4).with_(speed="sincos2d", speed_params=W._params([0.5]))
    band, x, gap, e, U = _coarse_band(p, oracle.patchy_solve(p, tol=1e-10))
    assert band.sum() >= 8
    np.testing.assert_allclose(U * I.speed_np(p, x), gap, rtol=1e-9, atol=0)
    # Zermelo drift
    p = W.zermelo(n=81, n_coarse=21, parts=4)
    band, x, gap, e, U = _coarse_band(p, oracle.patchy_solve(p, tol=1e-10))
    assert band.sum() >= 8
    s, w = p.drift[0], np.array(p.drift[1:3])
    v = gap / U
    np.testing.assert_allclose(np.linalg.norm(v[:, None] * e - w, axis=1), s, rtol=1e-9)
    assert np.all(np.linalg.norm((v + 1e-6)[:, None] * e - w, axis=1) > s)
    # Brockett: the largest |(a1, a2, x1 a2 - x2 a1)|, through nodes off the x3 axis
    p = W.brockett3d(n=21, n_coarse=11)
    band, x, gap, e, U = _coarse_band(p, oracle.patchy_solve(p, tol=1e-10))
    a = np.asarray(p.controls, float)[:, :2]
    f3 = x[:, :1] * a[None, :, 1] - x[:, 1:2] * a[None, :, 0]
    vmax = np.sqrt(a[None, :, 0] ** 2 + a[None, :, 1] ** 2 + f3 ** 2).max(axis=1)
    assert band.sum() >= 6 and np.any(np.abs(x[:, :2]).max(axis=1) > 0)
    np.testing.assert_allclose(U * vmax, gap, rtol=1e-9, atol=0)
