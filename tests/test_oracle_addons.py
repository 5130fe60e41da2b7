"""Pins for the oracle's Dirichlet patch boundary (Eq. dbc) and the add-ons
AO1-AO3 of Sec. 6, each checked against something other than the oracle's own
arithmetic: the global fixed point, a linear program, an exact linear solve,
and the order- and start-independence of the fixed point.
"""
import math

import numpy as np
import pytest
from scipy.optimize import linprog

import oracle
import workloads as W
from tests import _indep as I


def _small(seed=0, n=49, nc=13, R=3, radius=0.2, dim=2):
    if dim == 2:
        return W.sincos2d(seed, n=n, n_coarse=nc, n_targets=R, radius=radius).with_(tol=1e-12)
    return W.sin3d(seed, n=n, n_coarse=nc, n_targets=R, radius=radius).with_(tol=1e-12)


# ------------------------------------------------------------- Dirichlet --

@pytest.mark.parametrize("dim,seed", [(2, 0), (2, 1), (3, 0), ("zermelo", 0), ("brockett", 0)])
def test_dirichlet_with_exact_data_gives_global_solution(dim, seed):
    """With the global fixed point as boundary data, each patch's equation
    (Eq. SLscheme restricted to the patch, data outside) is solved by the
    restriction of that fixed point, and it is the only finite one on S*: the
    patchy result must equal the global solution at every node."""
    if dim == "zermelo":        # per-control steps h = k/|s a + w| (R20)
        p = W.zermelo(n=49, n_coarse=13, n_c=16, parts=4).with_(tol=1e-13)
    elif dim == "brockett":     # per-node feet and steps (R24)
        p = W.brockett3d(n=17, n_coarse=9).with_(tol=1e-13)
    else:
        p = _small(seed) if dim == 2 else _small(seed, n=17, nc=7, R=3, radius=0.15, dim=3)
    g = oracle.global_solve(p.with_(n_coarse=None), tol=1e-13)
    r = oracle.patchy_solve(p, tol=1e-13, dirichlet=True, bc_data=g.u)
    fin = np.isfinite(g.u)
    # nodes Step 2 leaves unreachable are labelled -1 and stay +inf
    lab_ok = r.labels >= 0
    assert np.array_equal(np.isfinite(r.u), fin & lab_ok | (r.u == 0))
    both = fin & np.isfinite(r.u)
    np.testing.assert_allclose(r.u[both], g.u[both], rtol=0, atol=1e-10)
    assert both.sum() > 0.5 * fin.sum()


def test_dirichlet_below_state_constraints():
    """F is monotone in the values it reads, and state constraints read +inf
    where Eq. (dbc) reads U_P^(0): the Dirichlet solution is nowhere larger,
    and reaches every node the state-constrained one reaches."""
    p = _small(2, n=65, nc=17, R=4, radius=0.15)
    sc = oracle.patchy_solve(p, tol=1e-12)
    dr = oracle.patchy_solve(p, tol=1e-12, dirichlet=True)
    fin = np.isfinite(sc.u)
    assert np.all(np.isfinite(dr.u)[fin])
    assert np.all(dr.u[fin] <= sc.u[fin] + 1e-12)
    assert np.array_equal(sc.labels, dr.labels)


def test_dirichlet_data_is_the_literal_interpolation():
    """Eq. (dbc) reads U_P^(0) = I[U~] literally: where a coarse corner of
    positive weight is +inf the data is +inf, never a value mixed with the
    bound the feedback uses near the ghost ring.  So every finite Dirichlet
    value stays within the range of the global solution's values (plus the
    coarse error), in 2D and 3D."""
    for p in (_small(8, n=65, nc=9, R=3, radius=0.2), _small(1, n=25, nc=7, R=3, radius=0.15, dim=3)):
        g = oracle.global_solve(p.with_(n_coarse=None), tol=1e-12)
        dr = oracle.patchy_solve(p, tol=1e-12, dirichlet=True)
        fin = np.isfinite(dr.u)
        assert dr.u[fin].max() <= 2.0 * g.u[np.isfinite(g.u)].max()


def test_dirichlet_single_patch_equals_state_constraints():
    """R = 1: outside the patch there are only the target, the ghost ring and
    unreachable nodes, where U_P^(0) is 0, +inf and +inf, so Eq. (dbc) and
    state constraints coincide."""
    p = _small(3, n=41, nc=11, R=1, radius=0.25)
    a = oracle.patchy_solve(p, tol=1e-12)
    b = oracle.patchy_solve(p, tol=1e-12, dirichlet=True)
    assert np.array_equal(a.u, b.u)


def test_dirichlet_uses_the_data_it_is_given():
    """Raising the data by a constant c outside the patches raises every
    value whose optimal path exits its patch, by at most c, and never lowers
    one (monotone, translation-bounded operator)."""
    p = _small(4, n=49, nc=13, R=3, radius=0.2)
    base = oracle.patchy_solve(p, tol=1e-12, dirichlet=True)
    d = base.u0.copy()
    kind, _, _ = oracle.setup(p)
    d[kind == oracle.FREE] += 0.5
    up = oracle.patchy_solve(p, tol=1e-12, dirichlet=True, bc_data=d)
    fin = np.isfinite(base.u)
    diff = up.u[fin] - base.u[fin]
    assert diff.min() >= -1e-12 and diff.max() <= 0.5 + 1e-12
    assert diff.max() > 1e-3  # some node's optimal path leaves its patch


# -------------------------------------------------------------- AO1, AO2 --

@pytest.mark.parametrize("dirichlet", [False, True])
def test_warm_start_and_causal_order_reach_the_same_fixed_point(dirichlet):
    """AO1 changes the start and AO2 the visiting order; the fixed point on S*
    is unique (R14), so both give the basic result."""
    p = _small(5, n=65, nc=17, R=4, radius=0.15)
    base = oracle.patchy_solve(p, tol=1e-13, dirichlet=dirichlet)
    fin = np.isfinite(base.u)
    for kw in ({"warm": True}, {"causal": True}, {"warm": True, "causal": True}):
        r = oracle.patchy_solve(p, tol=1e-13, dirichlet=dirichlet, **kw)
        assert np.array_equal(np.isfinite(r.u), fin), kw
        np.testing.assert_allclose(r.u[fin], base.u[fin], rtol=0, atol=1e-10, err_msg=str(kw))


def test_causal_order_cuts_sweeps_on_the_eikonal():
    """For the eikonal equation the characteristics follow -grad u, so visiting
    nodes by increasing U_P^(0) (a close approximation of u) needs fewer
    Gauss-Seidel sweeps than one fixed lexicographic order."""
    p = W.eikonal2d(n=81, n_c=32, radius=0.2).with_(n_coarse=(21, 21), tol=1e-12)
    p = p.with_(targets=np.array([[-1.0, -1.0, 0.2], [1.0, 0.5, 0.2]]))
    lex = oracle.patchy_solve(p, order=0)
    cau = oracle.patchy_solve(p, order=0, causal=True)
    assert sum(cau.stats["sweeps_patch"]) < 0.6 * sum(lex.stats["sweeps_patch"])


# ------------------------------------------------------------------- AO3 --

def _cones(p, astar, r):
    a = np.asarray(p.controls)
    cr = math.cos(math.pi / r) - 1e-12
    return lambda i, m: astar[i] < 0 or float(a[m] @ a[astar[i]]) >= cr


def _lp_fixed_point(p, allowed, cap=1e3):
    """The fixed point as the largest v with v_i <= h_i + sum_c w_c(a) v_c for
    every allowed, admissible control a (the linear-programming form of the
    stochastic shortest path problem), solved by HiGHS; values are capped at
    `cap` so that nodes off S* stay bounded."""
    kind, _, h = I.kinds(p)
    idx, _ = I.node_grid(p)
    free = np.nonzero(kind == 0)[0]
    pos = {int(i): q for q, i in enumerate(free)}
    rows, rhs = [], []
    for i in free:
        for m, a in enumerate(p.controls):
            if not allowed(int(i), m):
                continue
            cs = I.q1_corners(p, idx[i], a)
            if any(kind[j] == 2 for j, _ in cs):
                continue
            row = np.zeros(len(free))
            row[pos[int(i)]] += 1.0
            for j, w in cs:
                if kind[j] == 0:
                    row[pos[j]] -= w
            rows.append(row)
            rhs.append(h[i])
    res = linprog(-np.ones(len(free)), A_ub=np.array(rows), b_ub=np.array(rhs), bounds=(0, cap),
                  method="highs", options={"primal_feasibility_tolerance": 1e-10,
                                           "dual_feasibility_tolerance": 1e-10})
    assert res.status == 0
    full = np.where(kind == 1, 0.0, np.inf)
    full[free] = res.x
    return full


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("r", [2.0, 4.0])
def test_reduced_controls_match_linear_program(seed, r):
    """The AO3 operator (cones of half-angle pi / r around a per-node control)
    has the fixed point of the linear program over the same reduced sets."""
    p = W.random_speed_problem(seed, n=9, n_c=16)
    rng = np.random.default_rng(100 + seed)
    astar = rng.integers(0, 16, size=int(np.prod(p.n))).astype(np.int32)
    astar[rng.random(astar.size) < 0.2] = -1
    kind, _, _ = oracle.setup(p)
    U = np.where(kind == oracle.TARGET, 0.0, np.inf)
    it = oracle.iterate_reduced(p, U, kind == oracle.FREE, astar, r, tol=1e-14)
    ref = _lp_fixed_point(p, _cones(p, astar, r), cap=1e3)
    ref2 = _lp_fixed_point(p, _cones(p, astar, r), cap=1e4)
    fin = np.isfinite(it.u)
    assert fin.sum() > 0
    np.testing.assert_allclose(it.u[fin], ref[fin], rtol=0, atol=1e-8)
    np.testing.assert_allclose(it.u[fin], ref2[fin], rtol=0, atol=1e-7)
    # off S* some path reaches a trap with positive probability: the LP value
    # there grows with the cap, while on S* it does not depend on it
    off = (kind == oracle.FREE) & ~fin
    assert np.all(ref2[off] - ref[off] > 1e-3)


def _sure_set(p, allowed):
    """S* (R14) restated: the greatest set S of free nodes from which the
    target is reached with allowed controls whose positive-weight corners all
    lie in S or on the target (reach from the target, drop what was not
    reached, repeat)."""
    kind, _, _ = I.kinds(p)
    idx, _ = I.node_grid(p)
    free = [int(i) for i in np.nonzero(kind == 0)[0]]
    corners = {i: [I.q1_corners(p, idx[i], a) if allowed(i, m) else None for m, a in enumerate(p.controls)]
               for i in free}
    S = set(free)
    while True:
        reached, grew = set(), True
        while grew:
            grew = False
            for i in sorted(S - reached):
                for cs in corners[i]:
                    if cs is None or not all(kind[j] == 1 or j in S for j, _ in cs):
                        continue
                    if any(kind[j] == 1 or (j in reached and j != i) for j, _ in cs):
                        reached.add(i)
                        grew = True
                        break
        if reached == S:
            return S, corners
        S = reached


@pytest.mark.parametrize("r", [2.0, 4.0])
def test_reduced_controls_match_linear_program_3d(r):
    """The same in 3D (trilinear transitions among 26 Fibonacci directions;
    cones around the global solution's minimising control, replaced by a
    random control at a fifth of the nodes and dropped at another fifth).
    Here a control can put a tiny positive weight on a node off S*, so the
    capped LP over all nodes is not the comparison: S* is restated
    independently and the LP runs over the controls that stay in it."""
    p = W.random_speed_problem(5, n=7, n_c=26, dim=3)
    g = oracle.global_solve(p, tol=1e-14)
    kind, _, h = I.kinds(p)
    idx, _ = I.node_grid(p)
    rng = np.random.default_rng(205)
    astar = np.full(g.u.size, -1, np.int32)
    for i in np.nonzero((kind == 0) & np.isfinite(g.u))[0]:
        q = [h[i] + sum(w * g.u[j] for j, w in I.q1_corners(p, idx[i], a)) for a in p.controls]
        astar[i] = int(np.argmin(q))
    u = rng.random(astar.size)
    astar[u < 0.2] = rng.integers(0, 26, size=int((u < 0.2).sum()))
    astar[u > 0.8] = -1
    U = np.where(kind == oracle.TARGET, 0.0, np.inf)
    it = oracle.iterate_reduced(p, U, kind == oracle.FREE, astar, r, tol=1e-14)
    S, corners = _sure_set(p, _cones(p, astar, r))
    fin = np.isfinite(it.u) & (kind == 0)
    assert set(np.nonzero(fin)[0].tolist()) == S and len(S) > 10
    Sl = sorted(S)
    pos = {i: q for q, i in enumerate(Sl)}
    rows, rhs = [], []
    for i in Sl:
        for cs in corners[i]:
            if cs is None or not all(kind[j] == 1 or j in S for j, _ in cs):
                continue
            row = np.zeros(len(Sl))
            row[pos[i]] += 1.0
            for j, w in cs:
                if j in pos:
                    row[pos[j]] -= w
            rows.append(row)
            rhs.append(h[i])
    res = linprog(-np.ones(len(Sl)), A_ub=np.array(rows), b_ub=np.array(rhs), bounds=(0, 1e6), method="highs",
                  options={"primal_feasibility_tolerance": 1e-10, "dual_feasibility_tolerance": 1e-10})
    assert res.status == 0
    np.testing.assert_allclose(it.u[Sl], res.x, rtol=0, atol=1e-8)


def test_single_control_cone_is_policy_evaluation():
    """For r so large that the cone holds only a*, the fixed point is the
    value of the feedback a*: the linear system u_i = h_i + sum_c w_c u_c."""
    p = W.random_speed_problem(7, n=9, n_c=8)
    g = oracle.global_solve(p, tol=1e-14)
    kind, _, h = I.kinds(p)
    idx, _ = I.node_grid(p)
    free = np.nonzero((kind == 0) & np.isfinite(g.u))[0]
    # a proper feedback: the minimiser of the global solution's right-hand side
    astar = np.full(g.u.size, -1, np.int32)
    for i in free:
        q = [h[i] + sum(w * g.u[j] for j, w in I.q1_corners(p, idx[i], a)) for a in p.controls]
        astar[i] = int(np.argmin(q))
    pos = {int(i): q for q, i in enumerate(free)}
    A = np.eye(len(free))
    for i in free:
        for j, w in I.q1_corners(p, idx[i], p.controls[astar[i]]):
            if kind[j] == 0:
                A[pos[int(i)], pos[j]] -= w
    v = np.linalg.solve(A, h[free])
    U = np.where(kind == oracle.TARGET, 0.0, np.inf)
    it = oracle.iterate_reduced(p, U, np.isin(np.arange(g.u.size), free), astar, 1e6, tol=1e-14)
    np.testing.assert_allclose(it.u[free], v, rtol=0, atol=1e-11)
    # and that value is the global one (a* is optimal there)
    np.testing.assert_allclose(v, g.u[free], rtol=0, atol=1e-10)


def test_reduction_factor_one_keeps_every_control():
    """r = 1: cos(pi) = -1, every control is in every cone."""
    p = _small(6, n=41, nc=11, R=3, radius=0.25)
    a = oracle.patchy_solve(p, tol=1e-12)
    b = oracle.patchy_solve(p, tol=1e-12, reduce_r=1.0)
    assert np.array_equal(a.u, b.u)


@pytest.mark.parametrize("dirichlet", [False, True])
def test_reduced_controls_never_lower_the_value(dirichlet):
    """Fewer controls can only raise the minimum (and the fixed point); the
    labels of Step 3.1 do not depend on AO3."""
    p = _small(7, n=65, nc=17, R=4, radius=0.15)
    a = oracle.patchy_solve(p, tol=1e-12, dirichlet=dirichlet)
    b = oracle.patchy_solve(p, tol=1e-12, dirichlet=dirichlet, reduce_r=4.0)
    fa = np.isfinite(a.u)
    fb = np.isfinite(b.u)
    assert np.all(fa[fb])
    assert np.all(b.u[fb] >= a.u[fb] - 1e-12)
    assert np.array_equal(a.labels, b.labels)


def test_addons_in_3d():
    """The add-ons on a 3D problem: r = 1 keeps every control (bitwise), r = 4
    never lowers a value and keeps the labels, AO1 and AO2 reach the basic
    fixed point."""
    p = _small(2, n=21, nc=7, R=2, radius=0.25, dim=3)
    a = oracle.patchy_solve(p, tol=1e-13)
    assert np.array_equal(a.u, oracle.patchy_solve(p, tol=1e-13, reduce_r=1.0).u)
    b = oracle.patchy_solve(p, tol=1e-13, reduce_r=4.0)
    fa, fb = np.isfinite(a.u), np.isfinite(b.u)
    assert np.all(fa[fb]) and np.all(b.u[fb] >= a.u[fb] - 1e-12)
    assert np.array_equal(a.labels, b.labels)
    for kw in ({"warm": True}, {"causal": True}):
        r = oracle.patchy_solve(p, tol=1e-13, **kw)
        assert np.array_equal(np.isfinite(r.u), fa), kw
        np.testing.assert_allclose(r.u[fa], a.u[fa], rtol=0, atol=1e-10, err_msg=str(kw))
