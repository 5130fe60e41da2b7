"""Pins for obstacles (Sec. 4, "Patchy method with obstacles"; reading R23):
nodes inside a closed ball or box are state constraints like the ghost ring.
Checked against an independent restatement of the node kinds, Dijkstra on the
axis graph with the obstacle nodes removed, the geodesic distance around a
box (visibility graph), and the patchy invariants with obstacles present.
"""
import numpy as np
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

import oracle
import workloads as W
from tests import _indep as I


def _box_problem(n, n_c=64):
    lo, hi = (-0.4, -1.0), (0.4, 1.0)
    return W.eikonal_sectors(n=n, n_c=n_c).with_(
        n_coarse=None, target_kind="balls", n_parts=0, targets=np.array([[1.2, 0.0, 0.3]]),
        obstacles=np.array([W.obstacle_box(lo, hi)]), tol=1e-12)


def _seg_hits_open_box(a, b, lo, hi):
    """Does the segment [a, b] pass through the open box (lo, hi)?  Clip it
    to the closed box (Liang-Barsky) and test the clipped piece's midpoint."""
    t0, t1 = 0.0, 1.0
    d = b - a
    for k in range(2):
        for pk, qk in ((-d[k], a[k] - lo[k]), (d[k], hi[k] - a[k])):
            if pk == 0.0:
                if qk < 0.0:
                    return False
            else:
                t = qk / pk
                if pk < 0.0:
                    t0 = max(t0, t)
                else:
                    t1 = min(t1, t)
    if t1 - t0 <= 1e-12:
        return False
    m = a + d * (t0 + t1) / 2.0
    return bool(np.all(m > lo + 1e-12) and np.all(m < hi - 1e-12))


def _geodesic(x, c, lo, hi):
    """Shortest path from x to c around a box: Dijkstra on the visibility
    graph of x, the four corners and c."""
    pts = [x] + [np.array(v) for v in ((lo[0], lo[1]), (hi[0], lo[1]), (hi[0], hi[1]), (lo[0], hi[1]))] + [c]
    D = np.full(len(pts), np.inf)
    D[0] = 0.0
    done = np.zeros(len(pts), bool)
    for _ in pts:
        i = int(np.argmin(np.where(done, np.inf, D)))
        done[i] = True
        for j in range(len(pts)):
            if not done[j] and not _seg_hits_open_box(pts[i], pts[j], lo, hi):
                D[j] = min(D[j], D[i] + np.linalg.norm(pts[i] - pts[j]))
    return D[-1]


def test_obstacle_nodes_follow_the_definition():
    """Node kinds with a disk and a box equal the independent restatement,
    in 2D and 3D; both obstacles hold nodes."""
    p = W.eikonal_obstacles(n=81, n_coarse=21)
    kind, part, _ = oracle.setup(p)
    ik, ipart, _ = I.kinds(p)
    assert np.array_equal(kind, ik) and np.array_equal(part, ipart)
    _, x = I.node_grid(p)
    for row in p.obstacles:
        one = p.with_(obstacles=row[None, :])
        assert I.in_obstacles(one, x).sum() > 20
    q = W.sin3d(0, n=25, n_coarse=7, n_c=14).with_(obstacles=np.array([W.obstacle_ball((0.3, -0.2, 0.1), 0.4),
                                                    W.obstacle_box((-0.9, -0.9, -0.9), (-0.5, 0.2, 0.0))]))
    kind, part, _ = oracle.setup(q)
    ik, ipart, _ = I.kinds(q)
    assert np.array_equal(kind, ik) and np.array_equal(part, ipart)
    assert (ik == 2).sum() > 4 * (q.n[0] - 2) ** 2  # more than the ring


def test_obstacles_axis_controls_equal_dijkstra():
    """With the four axis controls every foot is a node, so the fixed point is
    Dijkstra on the axis graph without the obstacle nodes (cost h_i leaving
    node i, here on a varying speed field)."""
    p = W.eikonal_obstacles(n=41, n_coarse=11).with_(n_coarse=None, controls=W.controls_2d(4), speed="sincos2d",
                                                     speed_params=W._params([0.5]), tol=1e-14)
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
    dist = dijkstra(G.T, directed=True, indices=np.nonzero(kind == 1)[0], min_only=True)
    ref = np.where(kind == 2, np.inf, dist)
    r = oracle.global_solve(p)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-11)


def test_obstacle_geodesic_first_order():
    """Eikonal around a box: the solution approaches the geodesic distance to
    the target ball (visibility graph) at first order in k; the straight-line
    distance is far off in the box's shadow."""
    lo, hi = np.array([-0.4, -1.0]), np.array([0.4, 1.0])
    c, r = np.array([1.2, 0.0]), 0.3
    errs = []
    for n in (41, 81, 161):
        p = _box_problem(n)
        g = oracle.global_solve(p)
        _, x = I.node_grid(p)
        fin = np.isfinite(g.u)
        kind, _, _ = I.kinds(p)
        assert np.array_equal(fin, kind != 2)
        T = np.array([max(_geodesic(xi, c, lo, hi) - r, 0.0) for xi in x[fin]])
        e = np.abs(g.u[fin] - T)
        assert e.max() <= 4.0 * p.spacing, (n, e.max())
        errs.append(e.mean())
        straight = np.maximum(np.linalg.norm(x[fin] - c, axis=1) - r, 0.0)
        assert np.abs(straight - T).max() > 0.5
    assert errs[1] <= 0.65 * errs[0] and errs[2] <= 0.65 * errs[1], errs


def test_patchy_with_obstacles_invariants():
    """Patchy solve with obstacles: obstacle nodes are +inf with label -1;
    with one part (R = 1) the patchy solution is the global one; every label
    is a patch that reaches the target."""
    p = W.eikonal_obstacles(n=61, n_coarse=16, parts=4).with_(tol=1e-12)
    kind, _, _ = I.kinds(p)
    _, x = I.node_grid(p)
    blocked = I.in_obstacles(p, x) & (kind != 1)
    r = oracle.patchy_solve(p)
    assert np.all(np.isinf(r.u[blocked])) and np.all(r.labels[blocked] == -1)
    assert set(r.labels[r.labels >= 0]) == set(range(4))
    one = p.with_(n_parts=1)
    a = oracle.patchy_solve(one)
    g = oracle.global_solve(one.with_(n_coarse=None), tol=1e-12)
    fin = np.isfinite(g.u)
    assert np.array_equal(fin, np.isfinite(a.u))
    np.testing.assert_allclose(a.u[fin], g.u[fin], rtol=0, atol=1e-9)


def test_enclosed_pocket_has_no_feedback():
    """R7 with an unreachable region: a pocket enclosed by a box frame two
    coarse cells thick holds no target, so its coarse values are +inf,
    U_P^(0) = +inf there, no feedback is defined (a* = -1) and its nodes end
    unlabelled at +inf.  The pocket comes from a flood fill over the free
    nodes, independent of the scheme."""
    frame = np.array([W.obstacle_box((-1.6, -1.6), (-1.2, 0.2)), W.obstacle_box((-0.2, -1.6), (0.2, 0.2)),
                      W.obstacle_box((-1.2, -1.6), (-0.2, -1.2)), W.obstacle_box((-1.2, -0.2), (-0.2, 0.2))])
    p = W.eikonal_obstacles(n=81, n_coarse=21, n_c=16).with_(
        target_kind="balls", n_parts=0, targets=np.array([[1.2, 1.2, 0.3]]), obstacles=frame, tol=1e-10)
    kind, _, _ = I.kinds(p)
    n = p.n[0]
    seen = kind == 1
    stack = list(np.nonzero(seen)[0])
    while stack:
        i = stack.pop()
        for j in (i - 1, i + 1, i - n, i + n):
            if 0 <= j < kind.size and not seen[j] and kind[j] == 0:
                seen[j] = True
                stack.append(j)
    pocket = (kind == 0) & ~seen
    assert pocket.sum() >= 300
    r = oracle.patchy_solve(p)
    assert np.all(np.isinf(r.u0[pocket])) and np.all(r.astar[pocket] == -1)
    assert np.all(r.labels[pocket] == -1) and np.all(np.isinf(r.u[pocket]))
    # outside the pocket every free node reaches the target
    assert np.all(np.isfinite(r.u[(kind == 0) & seen]))
