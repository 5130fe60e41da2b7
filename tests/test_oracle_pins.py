"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

Each test checks the oracle with something other than itself: a closed form,
a textbook routine (Dijkstra), an exact alternative algorithm (policy
iteration with dense linear solves, absorption probabilities), exactness of
the interpolation on multilinear functions, or an invariant of the scheme.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import dijkstra

import oracle
import workloads as W
from tests import _indep as I


# --------------------------------------------------------------- set-up ---

@pytest.mark.parametrize("make", [lambda: W.sincos2d(0, n=65, n_coarse=17),
                                  lambda: W.sin3d(1, n=17, n_coarse=9),
                                  lambda: W.random_speed_problem(3)])
def test_setup_matches_definition(make):
    """Node kinds, target parts and h_i = k / c(x_i) (Sec. 2.1, |h f| = k)."""
    p = make()
    kind, part, h = oracle.setup(p)
    k2, p2, h2 = I.kinds(p)
    assert np.array_equal(kind, k2)
    assert np.array_equal(part, p2)
    np.testing.assert_allclose(h, h2, rtol=1e-13)


def test_eikonal_target_count():
    """Disk r = 0.1 on the k = 0.04 grid: the 21 nodes with i^2 + j^2 <= 6.25."""
    kind, part, _ = oracle.setup(W.eikonal2d())
    assert int((kind == oracle.TARGET).sum()) == 21


# ------------------------------------------------------- interpolation ---

@pytest.mark.parametrize("dim", [2, 3])
def test_interp_exact_on_multilinear(dim):
    """Q1 interpolation (Sec. 2.1) reproduces multilinear functions exactly."""
    rng = np.random.default_rng(dim)
    p = W.random_speed_problem(0, n=7, dim=dim)
    idx, _ = I.node_grid(p)
    coef = rng.normal(size=2 ** dim)

    def f(z):
        out = np.zeros(z.shape[0])
        for c in range(2 ** dim):
            term = np.full(z.shape[0], coef[c])
            for d in range(dim):
                if c & (1 << d):
                    term = term * z[:, d]
            out += term
        return out

    U = f(idx.astype(float))
    pts = rng.uniform(0, 6, size=(500, dim))
    np.testing.assert_allclose(oracle.interp(p, U, pts), f(pts), rtol=1e-12, atol=1e-12)
    # at the nodes themselves I[U] = U
    np.testing.assert_allclose(oracle.interp(p, U, idx.astype(float)), U, rtol=1e-13, atol=1e-13)


def test_interp_infinity_rule():
    """+inf propagates only through corners of positive weight (state constraints)."""
    p = W.random_speed_problem(0, n=5)
    U = np.zeros(25)
    U[I.linear(p, [[2, 2]])[0]] = np.inf
    assert np.isinf(oracle.interp(p, U, np.array([[1.5, 1.5]]))[0])
    assert oracle.interp(p, U, np.array([[1.0, 1.5]]))[0] == 0.0      # weight on column 2 is 0
    assert oracle.interp(p, U, np.array([[2.0, 1.0]]))[0] == 0.0      # lands on node (2, 1)
    assert np.isinf(oracle.interp(p, U, np.array([[4.5, 1.0]]))[0])   # outside the box


# ------------------------------------------------------- global scheme ---

def test_eikonal_closed_form_config():
    """f = a, disk r = 0.1, 101x101, N_c = 32: u close to max(|x| - r, 0).

    Bound: first-order SL error (2k) plus the control-discretisation bias
    (sec(pi/N_c) - 1) u <= 0.5% of u."""
    p = W.eikonal2d()
    r = oracle.global_solve(p)
    assert r.converged
    x = oracle.grid_coords(p)
    exact = np.maximum(np.linalg.norm(x, axis=1) - 0.1, 0.0)
    kind, _, _ = oracle.setup(p)
    m = kind != oracle.GHOST
    assert np.isfinite(r.u[m]).all()
    assert np.isinf(r.u[~m]).all()
    err = np.abs(r.u[m] - exact[m]).max()
    assert err <= 2 * p.spacing + 0.005 * exact[m].max()
    # discrete value never below the continuous minimum time (it is an upper bound
    # up to the polygonal target error k)
    assert (r.u[m] >= exact[m] - p.spacing).all()


def test_eikonal_first_order_convergence():
    """Mean error vs the closed form falls with k (first order), N_c = 128.
    (The max error is dominated by the polygonal target, itself O(k).)"""
    errs = []
    for n in (21, 41, 81):
        p = W.eikonal2d(n=n, n_c=128, radius=0.5, tol=1e-12)
        r = oracle.global_solve(p)
        x = oracle.grid_coords(p)
        exact = np.maximum(np.linalg.norm(x, axis=1) - 0.5, 0.0)
        m = np.isfinite(r.u)
        errs.append(np.abs(r.u[m] - exact[m]).mean())
        assert np.abs(r.u[m] - exact[m]).max() <= 1.5 * p.spacing
    assert errs[1] <= 0.75 * errs[0] and errs[2] <= 0.75 * errs[1], errs


@pytest.mark.parametrize("dim,n", [(2, 9), (2, 33), (3, 9)])
def test_axis_controls_equal_dijkstra(dim, n):
    """With the 2d axis controls every foot lands on a node, so the fixed
    point of F is the shortest path on the axis-neighbour graph with cost h_i
    for leaving node i (ghost nodes removed)."""
    p = W.random_speed_problem(5, n=n, dim=dim, n_targets=2)
    p = p.with_(controls=W.controls_axes(dim), tol=1e-14)
    kind, part, h = I.kinds(p)
    idx, _ = I.node_grid(p)
    N = idx.shape[0]
    rows, cols, wts = [], [], []
    for i in np.nonzero(kind == 0)[0]:
        for d in range(dim):
            for s in (-1, 1):
                nb = idx[i].copy()
                nb[d] += s
                j = I.linear(p, nb)[0]
                if kind[j] != 2:
                    rows.append(j)            # reversed edge j -> i, cost h_i
                    cols.append(i)
                    wts.append(h[i])
    g = sp.csr_matrix((wts, (rows, cols)), shape=(N, N))
    dist = dijkstra(g, directed=True, indices=np.nonzero(kind == 1)[0], min_only=True)
    r = oracle.global_solve(p, tol=1e-14)
    ref = np.where(kind == 2, np.inf, dist)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-12)


def _policy_iteration(p):
    """Exact fixed point of F by policy iteration on the stochastic shortest
    path problem whose transition probabilities are the Q1 weights."""
    kind, part, h = I.kinds(p)
    idx, x = I.node_grid(p)
    free = np.nonzero(kind == 0)[0]
    pos = {int(i): q for q, i in enumerate(free)}
    tgt_x = x[kind == 1]
    acts = {}
    for i in free:
        lst = []
        for m, a in enumerate(p.controls):
            cs = I.q1_corners(p, idx[i], a)
            if any(kind[j] == 2 for j, _ in cs):
                lst.append(None)
            else:
                lst.append(cs)
        acts[int(i)] = lst
    dist = lambda j: np.min(np.linalg.norm(tgt_x - x[j], axis=1))
    pol = {}
    for i in free:
        best, bm = np.inf, None
        for m, cs in enumerate(acts[int(i)]):
            if cs is None:
                continue
            v = sum(w * dist(j) for j, w in cs)
            if v < best:
                best, bm = v, m
        pol[int(i)] = bm
    F = len(free)
    for _ in range(200):
        A = np.eye(F)
        for i in free:
            for j, w in acts[int(i)][pol[int(i)]]:
                if kind[j] == 0:
                    A[pos[int(i)], pos[j]] -= w
        v = np.linalg.solve(A, h[free])
        assert np.all(np.isfinite(v)) and v.min() > 0
        full = np.where(kind == 1, 0.0, np.inf)
        full[free] = v
        changed = False
        for i in free:
            q = [np.inf if cs is None else h[i] + sum(w * full[j] for j, w in cs) for cs in acts[int(i)]]
            m = int(np.argmin(q))
            if q[m] < q[pol[int(i)]] - 1e-13:
                pol[int(i)] = m
                changed = True
        if not changed:
            return full
    raise AssertionError("policy iteration did not stop")


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("n_c", [8, 32])
def test_policy_iteration_9x9(seed, n_c):
    """Brute force on 9x9: value iteration matches exact policy iteration."""
    p = W.random_speed_problem(seed, n=9, n_c=n_c)
    ref = _policy_iteration(p)
    r = oracle.global_solve(p, tol=1e-14)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-11)


@pytest.mark.parametrize("seed", range(3))
def test_policy_iteration_3d(seed):
    """Brute force on 7^3 with 26 Fibonacci controls (trilinear weights)."""
    p = W.random_speed_problem(seed, n=7, n_c=26, dim=3)
    ref = _policy_iteration(p)
    r = oracle.global_solve(p, tol=1e-14)
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(r.u))
    np.testing.assert_allclose(r.u[fin], ref[fin], rtol=0, atol=1e-11)


def test_order_independence():
    """Lexicographic Gauss-Seidel, alternating orders and Jacobi reach the same
    fixed point (Sec. 2.2: Gauss-Seidel only speeds the iteration up)."""
    p = W.sincos2d(2, n=41, n_coarse=11).with_(n_coarse=None, tol=1e-13)
    rs = [oracle.global_solve(p, order=o) for o in (0, 1, 2)]
    # every order stops by itself: the ghost ring stays +inf, and an unchanged
    # +inf counts as no change (R9)
    assert all(r.converged for r in rs)
    us = [r.u for r in rs]
    fin = np.isfinite(us[0])
    for u in us[1:]:
        assert np.array_equal(fin, np.isfinite(u))
        np.testing.assert_allclose(u[fin], us[0][fin], atol=1e-11)


@pytest.mark.parametrize("mode", [0, 1])
def test_F_monotone_and_iterates_nonincreasing(mode):
    """F (mode 0) and its node-wise exact form (mode 1) are monotone
    (U <= V => F(U) <= F(V)); the iterates from +inf never increase
    (Eq. iterativeSLscheme)."""
    p = W.random_speed_problem(7, n=17, n_c=16)
    rng = np.random.default_rng(0)
    kind, _, _ = oracle.setup(p)
    for _ in range(5):
        V = rng.uniform(0, 3, size=kind.size)
        V[rng.uniform(size=kind.size) < 0.2] = np.inf
        U = np.minimum(V, rng.uniform(0, 3, size=kind.size))
        FU, FV = oracle.sl_apply(p, U, mode=mode), oracle.sl_apply(p, V, mode=mode)
        assert np.all(FU <= FV)
    U = np.where(kind == oracle.TARGET, 0.0, np.inf)
    for _ in range(40):
        U2 = oracle.sl_apply(p, U, mode=mode)
        assert np.all(U2 <= U)
        U = U2
    assert np.all(U[np.isfinite(U)] >= 0)


def test_plus_infinity_start_is_a_fixed_point_of_literal_F():
    """Why the oracle solves the local equation exactly: with no control
    landing on a node, every foot cell has x_i as a positive-weight corner,
    so U = +inf off the target is a fixed point of F itself."""
    p = W.random_speed_problem(7, n=17, n_c=16)
    kind, _, _ = oracle.setup(p)
    U = np.where(kind == oracle.TARGET, 0.0, np.inf)
    assert np.array_equal(oracle.sl_apply(p, U, mode=0), U)


def test_local_exact_form_has_the_same_fixed_point():
    """Solving the node's own equation for u_i (the self corner of the foot
    cell moved to the left side) changes the iteration, not its fixed point:
    iterating that form from 0 on S* lands on the oracle's solution."""
    p = W.random_speed_problem(2, n=17, n_c=16)
    r = oracle.global_solve(p, tol=1e-14)
    kind, _, _ = oracle.setup(p)
    S = np.isfinite(r.u) & (kind == oracle.FREE)
    U = np.where(kind == oracle.TARGET, 0.0, np.inf)
    U[S] = 0.0
    for _ in range(400):
        U = oracle.sl_apply(p, U, upd=S, mode=1)
    np.testing.assert_allclose(U[S], r.u[S], atol=1e-11)


def test_reachable_set_removes_trapped_nodes():
    """S* (almost-sure reachability): a node whose every control puts
    positive weight outside the candidate set is not in S*, nor is a node
    whose only admissible moves lead to such nodes; every other node is."""
    p = W.random_speed_problem(1, n=11, n_c=8)
    kind, _, _ = oracle.setup(p)
    U = np.where(kind == oracle.TARGET, 0.0, np.inf)
    upd = kind == oracle.FREE
    S = oracle.reachable(p, upd, U)
    assert S[upd].all()                      # box without obstacles: everything reaches
    # wall off one interior node's whole 3x3 ring -> it and the wall vanish
    idx, _ = I.node_grid(p)
    tgt = np.nonzero(kind == oracle.TARGET)[0][0]
    far = np.argmax(np.linalg.norm(idx - idx[tgt], axis=1) * upd)
    ring = (np.abs(idx - idx[far]).max(axis=1) == 1)
    upd2 = upd & ~ring
    S2 = oracle.reachable(p, upd2, U)
    assert not S2[far]
    assert S2[upd2 & (np.abs(idx - idx[far]).max(axis=1) > 1)].all()


@pytest.mark.parametrize("make", [lambda: W.random_speed_problem(2, n=17, n_c=16),
                                  lambda: W.sincos2d(1, n=41, n_coarse=11).with_(n_coarse=None, tol=1e-13),
                                  lambda: W.random_speed_problem(4, n=9, n_c=26, dim=3)])
def test_solution_is_fixed_point_of_literal_F(make):
    """The converged oracle solution satisfies U = F(U) of Eq. (SLscheme)."""
    p = make()
    r = oracle.global_solve(p, tol=1e-13)
    FU = oracle.sl_apply(p, r.u, mode=0)
    fin = np.isfinite(r.u)
    assert np.array_equal(fin, np.isfinite(FU))
    np.testing.assert_allclose(FU[fin], r.u[fin], atol=1e-11)


def test_d4_symmetry():
    """Eikonal, D4-symmetric controls, centred target: u is invariant under
    the eight grid symmetries.  (The radius puts no node on the target
    boundary, where rounding of x = lo + i k would decide membership.)"""
    p = W.eikonal2d(n=41, n_c=32, radius=0.35, tol=1e-13)
    u = oracle.global_solve(p).u.reshape(41, 41)
    for g in (u.T, u[::-1], u[:, ::-1], u[::-1, ::-1], u.T[::-1], u.T[:, ::-1], u.T[::-1, ::-1]):
        np.testing.assert_allclose(np.nan_to_num(g, posinf=-1), np.nan_to_num(u, posinf=-1), atol=1e-12)


# ------------------------------------------------------- patchy method ---

def _small_patchy(seed=0, n=33, nc=9, R=3):
    # r = 0.2 so that every disk holds fine nodes at these small sizes
    return W.sincos2d(seed, n=n, n_coarse=nc, n_targets=R, radius=0.2)


@pytest.mark.parametrize("make", [lambda: _small_patchy(0), lambda: _small_patchy(1),
                                  lambda: W.sin3d(2, n=13, n_coarse=7, n_c=26, n_targets=2, radius=0.3)])
def test_phi_is_absorption_probability(make):
    """Step 3.1: phi^j solves a linear fixed point whose solution is the
    probability that the chain with the Q1 transitions of the coarse feedback
    is absorbed in Omega_0^j.  Checked against a dense linear solve on the
    nodes that can reach the target (phi = 0 elsewhere); phi in [0,1] and
    sum_j phi^j <= 1, with equality unless the chain can be trapped.  2D and
    3D (trilinear transitions)."""
    p = make()
    r = oracle.patchy_solve(p, keep_phi=True)
    kind, part, _ = I.kinds(p)
    idx, _ = I.node_grid(p)
    N = kind.size
    act = np.nonzero((kind == 0) & (r.astar >= 0))[0]
    rows, cols = [], []
    trans = {}
    for i in act:
        trans[int(i)] = I.q1_corners(p, idx[i], p.controls[r.astar[i]])
        for j, w in trans[int(i)]:
            rows.append(j)
            cols.append(int(i))
    g = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(N, N))
    reach = np.isfinite(dijkstra(g, directed=True, indices=np.nonzero(kind == 1)[0], min_only=True))
    live = [int(i) for i in act if reach[i]]
    pos = {i: q for q, i in enumerate(live)}
    A = np.eye(len(live))
    B = np.zeros((len(live), p.n_targets))
    for i in live:
        for j, w in trans[i]:
            if j in pos:
                A[pos[i], pos[j]] -= w
            elif kind[j] == 1:
                B[pos[i], part[j]] += w
    phi = np.linalg.solve(A, B)
    np.testing.assert_allclose(r.phi[:, live].T, phi, atol=1e-8)
    dead = [int(i) for i in act if not reach[i]]
    assert np.all(r.phi[:, dead] == 0)
    assert r.phi.min() >= 0 and r.phi.max() <= 1 + 1e-12
    tot = r.phi.sum(axis=0)
    assert tot[act].max() <= 1 + 1e-9
    # sum_j phi^j = 1 wherever the chain cannot fall into a closed class
    dead_set = np.zeros(N, bool)
    dead_set[dead] = True
    if dead:
        can_trap = np.isfinite(dijkstra(g, directed=True, indices=np.array(dead), min_only=True))
    else:
        can_trap = np.zeros(N, bool)
    sure = np.array([i for i in act if not can_trap[i]], dtype=int)
    np.testing.assert_allclose(tot[sure], 1.0, atol=1e-8)
    assert sure.size > 0.5 * len(act)


def test_labels_are_argmax_of_phi():
    """Eq. (proiezionecolore) with the argmax reading of Remark 3.1."""
    p = _small_patchy(3, R=4)
    r = oracle.patchy_solve(p, keep_phi=True)
    kind, part, _ = I.kinds(p)
    act = (kind == 0) & (r.astar >= 0)
    mx = r.phi.max(axis=0)
    covered = act & (mx > 0)
    assert np.array_equal(r.labels[covered], np.argmax(r.phi[:, covered], axis=0))
    # 1/2-projection agrees wherever some colour reaches 1/2
    half = covered & (mx >= 0.5)
    assert np.array_equal(r.labels[half], np.argmax(r.phi[:, half] >= 0.5, axis=0))
    assert np.array_equal(r.labels[kind == 1], part[kind == 1])
    assert (r.labels[kind == 2] == -1).all()


def test_patchy_single_target_equals_global():
    """R = 1: one patch covering every reachable node gives the global solution."""
    p = W.sincos2d(4, n=49, n_coarse=13, n_targets=1, radius=0.2).with_(tol=1e-12)
    rp = oracle.patchy_solve(p)
    rg = oracle.global_solve(p.with_(n_coarse=None))
    assert np.array_equal(rp.u, rg.u)


@pytest.mark.parametrize("make", [lambda: _small_patchy(5, n=49, nc=13, R=4),
                                  lambda: W.eikonal_sectors(n=49, n_coarse=13, n_c=16, parts=4),
                                  lambda: W.fan(n=49, n_coarse=13, n_c=16, parts=4),
                                  lambda: W.sin3d(2, n=17, n_coarse=9, n_c=26, n_targets=2, radius=0.3)])
def test_patchy_not_below_global_and_invariant(make):
    """State constraints on patch boundaries only remove admissible paths, so
    U_P >= U_global; and every finite patch value is reached through corners
    inside its own patch or its own target part (patch invariance).  With a
    target split into parts (a disk in sectors, Fan's line in pieces) the
    neighbouring parts touch each patch, and they are not terminals of it."""
    p = make().with_(tol=1e-12)
    rp = oracle.patchy_solve(p)
    rg = oracle.global_solve(p.with_(n_coarse=None))
    fin = np.isfinite(rg.u)
    assert np.all(rp.u[fin] >= rg.u[fin] - 1e-12)
    kind, part, h = I.kinds(p)
    idx, _ = I.node_grid(p)
    for i in np.nonzero((kind == 0) & np.isfinite(rp.u))[0]:
        j = rp.labels[i]
        best, bc = np.inf, None
        for a in p.controls:
            cs = I.q1_corners(p, idx[i], a)
            vals = [rp.u[c] if (rp.labels[c] == j) else np.inf for c, _ in cs]
            v = np.inf if any(np.isinf(vals)) else sum(w * v for (c, w), v in zip(cs, vals))
            if v < best:
                best, bc = v, cs
        assert abs(best + h[i] - rp.u[i]) < 1e-10
        assert all(rp.labels[c] == j for c, _ in bc)


def test_patchy_error_concentrates_on_patch_boundaries():
    """Sec. 4.2: E = U_P - U_DD is small on average, E_inf > E_1, and the
    error sits along the patch boundaries instead of spreading inside."""
    from scipy import ndimage
    n = 129
    p = W.sincos2d(1, n=n, n_coarse=33, n_targets=4, radius=0.2).with_(tol=1e-10)
    rp = oracle.patchy_solve(p)
    rg = oracle.global_solve(p.with_(n_coarse=None))
    assert np.array_equal(np.isfinite(rp.u), np.isfinite(rg.u))
    e1, einf = oracle.patchy_error(rp.u, rg.u)
    assert einf > e1 and e1 < 2e-3
    lab = rp.labels.reshape(n, n)
    bnd = np.zeros((n, n), bool)
    d0 = np.diff(lab, axis=0) != 0
    d1 = np.diff(lab, axis=1) != 0
    bnd[1:] |= d0
    bnd[:-1] |= d0
    bnd[:, 1:] |= d1
    bnd[:, :-1] |= d1
    near = ndimage.binary_dilation(bnd, iterations=3).reshape(-1)
    fin = np.isfinite(rg.u)
    E = np.zeros(n * n)
    E[fin] = np.abs(rp.u[fin] - rg.u[fin])
    assert near.mean() < 0.5
    assert E[near].sum() >= 0.95 * E.sum()


def _q1_values(n, lo_idx, U, dim):
    """Q1 interpolation of U (nodes per side n, +inf allowed) at grid-index
    points lo_idx (M, dim): +inf where a positive-weight corner is +inf or
    the point leaves the grid."""
    n = np.asarray(n[:dim])
    inside = np.all((lo_idx >= 0.0) & (lo_idx <= n - 1), axis=1)
    base = np.clip(np.floor(lo_idx).astype(np.int64), 0, n - 2)
    t = lo_idx - base
    val = np.zeros(lo_idx.shape[0])
    bad = ~inside
    for bits in range(1 << dim):
        w = np.ones(lo_idx.shape[0])
        j = np.zeros(lo_idx.shape[0], np.int64)
        mul = 1
        for d in range(dim):
            b = (bits >> d) & 1
            w *= t[:, d] if b else 1.0 - t[:, d]
            j += np.clip(base[:, d] + b, 0, n[d] - 1) * mul
            mul *= n[d]
        pos = w > 0.0
        uj = U[j]
        bad |= pos & np.isinf(uj)
        val += np.where(pos & np.isfinite(uj), w * np.where(np.isfinite(uj), uj, 0.0), 0.0)
    return np.where(bad, np.inf, val)


@pytest.mark.parametrize("make", [lambda: W.sincos2d(3, n=65, n_coarse=17, n_c=16, n_targets=2, radius=0.15),
                                  lambda: W.zermelo(n=65, n_coarse=17, n_c=16, parts=4),
                                  lambda: W.sin3d(1, n=17, n_coarse=9, n_c=26, n_targets=2, radius=0.3)])
def test_step2_u0_and_feedback_follow_their_definitions(make):
    """Step 2 restated with an independent Q1.  U_P^(0) is the Q1 of the
    coarse values at each free fine node, a +inf corner counting as the bound
    M = 1e6 and U_P^(0) >= M meaning unreachable (R7).  a* is the argmin over
    controls of I[U_P^(0)](x_i + k f/|f|) + h_{i,a} (Eq. feedbackcontrol),
    and gap its margin to the second best."""
    p = make()
    r = oracle.patchy_solve(p, tol=1e-10)
    kind, _, _ = I.kinds(p)
    idx, x = I.node_grid(p)
    d = p.dim
    free = np.nonzero(kind == 0)[0]
    scale = (np.array(p.n_coarse[:d]) - 1.0) / (np.array(p.n[:d]) - 1.0)
    M = 1.0e6
    u0 = _q1_values(p.n_coarse, idx[free] * scale, np.where(np.isinf(r.ucoarse), M, r.ucoarse), d)
    u0 = np.where(u0 >= M, np.inf, u0)
    fin = np.isfinite(u0)
    assert fin.mean() > 0.9
    assert np.array_equal(fin, np.isfinite(r.u0[free]))
    np.testing.assert_allclose(r.u0[free][fin], u0[fin], rtol=1e-12, atol=1e-12)
    # the feedback at the free nodes with a finite U_P^(0)
    U0 = np.where(kind == 1, 0.0, np.inf)
    U0[free] = u0
    nodes = free[fin]
    dirs, h = I.node_control_steps(p, x[nodes])
    if h.shape[0] != nodes.size:   # per-control steps come for every node
        h = h[nodes]
    vals = np.stack([_q1_values(p.n, idx[nodes] + dirs[:, m], U0, d) + h[:, m]
                     for m in range(p.n_controls)], axis=1)
    order = np.argsort(vals, axis=1, kind="stable")
    best = np.take_along_axis(vals, order[:, :1], axis=1)[:, 0]
    second = np.take_along_axis(vals, order[:, 1:2], axis=1)[:, 0]
    gap = second - best
    has = np.isfinite(best)
    assert np.array_equal(r.astar[nodes] >= 0, has)
    # the chosen control attains the minimum; where no other control comes
    # within rounding of it, it is the unique argmin (the drift's mirrored
    # control pairs tie at a fifth of the nodes)
    tol = 1e-9 * np.maximum(1.0, best[has])
    chosen = np.take_along_axis(vals[has], r.astar[nodes][has, None].astype(np.int64), axis=1)[:, 0]
    assert np.all(chosen <= best[has] + tol)
    clear = has & (gap > 1e-9 * np.maximum(1.0, best))
    assert clear.mean() > 0.5
    assert np.array_equal(r.astar[nodes][clear], order[clear, 0])
    g = r.gap[nodes][has]
    assert np.array_equal(np.isinf(g), np.isinf(gap[has]))
    ok = np.isfinite(g)
    np.testing.assert_allclose(g[ok], gap[has][ok], rtol=0, atol=1e-9)


def test_uncovered_nodes_join_a_neighbouring_patch():
    """Remark 3.1: a node with a feedback that no colour reaches (every
    phi^j = 0) still joins a patch, one of its axis neighbours'.  A coarse
    grid of 5^2 nodes under the Zermelo drift leaves such nodes."""
    p = W.zermelo(n=65, n_coarse=5, parts=4).with_(tol=1e-10)
    r = oracle.patchy_solve(p, keep_phi=True)
    kind, _, _ = I.kinds(p)
    act = (kind == 0) & (r.astar >= 0)
    bare = act & (r.phi.max(axis=0) == 0.0)
    assert bare.sum() >= 50
    assert np.all(r.labels[act] >= 0)
    n = p.n[0]
    for i in np.nonzero(bare)[0]:
        nb = [j for j in (i - 1, i + 1, i - n, i + n) if 0 <= j < kind.size]
        assert r.labels[i] in r.labels[nb]
    assert r.converged


def test_parallel_application_equals_the_serial_one():
    """The all-core application of F (nodes split over threads, Method 1 of
    Sec. 3) used to time the CPU baseline computes the same values."""
    p = W.sincos2d(0, n=129, n_coarse=17)
    kind, _, _ = oracle.setup(p)
    x = oracle.grid_coords(p)
    U = np.where(kind == oracle.GHOST, np.inf, np.linalg.norm(x, axis=1))
    U[kind == oracle.TARGET] = 0.0
    par, used = oracle.sl_apply_par(p, U)
    assert used >= 1
    assert np.array_equal(par, oracle.sl_apply(p, U))
