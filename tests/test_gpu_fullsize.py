"""Parity at the benchmark's full sizes, in the launch configuration bench.py
times (FP32 sweeps with the FP64 polish, default launch shape).

- 2D, 2049^2 (coarse 65^2, 64 controls, 4 disks, seed 0): against the FP64
  oracle's full patchy and global solves stored by tests/golden/make_golden.py
  (20,000 sampled values, the full label map with its tie mask, the reachable
  count, the per-patch node counts).
- 3D, 129^3 (coarse 33^3, 98 controls, 8 balls, seed 0): against the oracle's
  patchy solve stored the same way (the largest 3D size the oracle finishes
  in about an hour).
- 3D, 257^3 (coarse 33^3, 98 controls, 8 balls): the oracle does not finish
  at this size, so the test checks a property that holds at any size: at
  sampled nodes the GPU values satisfy the fixed-point equation of Eq.
  (SLscheme) with state constraints on the patch boundary, restated here in
  numpy (literal Q1 foot, a corner of another patch or off S* is +inf).
"""
import json
import math
import os

import numpy as np
import pytest

import workloads as W
from tests import _indep as I
from tests._labels import check_labels, grid_shape

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sincos2d_n2049_s0.npz")
GOLDEN3 = os.path.join(os.path.dirname(__file__), "golden", "sin3d_n129_s0.npz")


@pytest.fixture(scope="module")
def pkg():
    import torch

    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as P

    torch.cuda.set_device(0)
    return P


def _solve(pkg, p, stats=False):
    with pkg.Plan(p, precision=pkg.HJBP_FP32_POLISH64) as plan:
        st = plan.solve()
        if stats:
            return st, plan.values(), plan.labels(), plan.stats()
        return st, plan.values(), plan.labels()


def _against_golden(pkg, path, p):
    """Values at the sampled nodes, the reachable count, the labels (tie rule)
    and the per-patch node counts against a stored oracle solve."""
    import oracle

    g = np.load(path)
    meta = json.loads(str(g["meta"]))
    assert list(p.n) == meta["n"] and list(p.n_coarse) == meta["n_coarse"]
    st, u, lab, stats = _solve(pkg, p, stats=True)
    assert st == 0
    bound = 1e-4 * meta["max_u"]
    assert int(np.isfinite(u).sum()) == meta["reachable"]
    idx = g["idx"]
    assert np.abs(u[idx] - g["u"]).max() <= bound
    ref_lab = g["labels"]
    tie = np.unpackbits(g["tie"], count=ref_lab.size).astype(bool)
    check_labels(lab, ref_lab, tie, grid_shape(p))
    # patch compaction: GPU counts move from the oracle's only by label disagreements
    kind, _, _ = oracle.setup(p)
    free = kind == oracle.FREE
    for j in range(p.n_patches):
        gain = int(np.sum(free & (lab == j) & (ref_lab != j)))
        loss = int(np.sum(free & (ref_lab == j) & (lab != j)))
        assert stats["patch_nodes"][j] - meta["stats"]["patch_nodes"][j] == gain - loss
    return g, bound


def test_config2_full_size_matches_oracle(pkg):
    p = W.sincos2d(0)
    g, bound = _against_golden(pkg, GOLDEN, p)
    # the plain global GPU solve (the comparison path) against the oracle's global solve
    st, ug, _ = _solve(pkg, p.with_(n_coarse=None))
    assert st == 0
    assert np.abs(ug[g["idx"]] - g["u_global"]).max() <= bound


def test_3d_129_matches_oracle(pkg):
    _against_golden(pkg, GOLDEN3, W.sin3d(0, n=129, n_coarse=33))


def _residual_3d(p, u, lab, nodes):
    """|u_i - F_i(u)| at the given free nodes, F the literal operator of Eq.
    (SLscheme) on the node's patch: min over controls of h_i + sum_b w_b u_b,
    a positive-weight corner with another label or u = +inf making the control
    inadmissible (target part j carries label j and value 0)."""
    n0, n1, n2 = p.n
    ix, iy, iz = nodes % n0, (nodes // n0) % n1, nodes // (n0 * n1)
    idx = np.stack([ix, iy, iz], axis=1).astype(float)
    x = np.array(p.lo) + idx * p.spacing
    h = p.spacing / I.speed_np(p, x)
    best = np.full(nodes.size, np.inf)
    hi = np.array([n0, n1, n2]) - 2
    for a in np.asarray(p.controls, float):
        xi = idx + a
        base = np.clip(np.floor(xi).astype(int), 0, hi)
        t = xi - base
        v = h.copy()
        ok = np.ones(nodes.size, bool)
        for bits in range(8):
            w = np.ones(nodes.size)
            c = base.copy()
            for d in range(3):
                if (bits >> d) & 1:
                    w *= t[:, d]
                    c[:, d] += 1
                else:
                    w *= 1.0 - t[:, d]
            j = c[:, 0] + n0 * (c[:, 1] + n1 * c[:, 2])
            pos = w > 0
            ok &= ~pos | ((lab[j] == lab[nodes]) & np.isfinite(u[j]))
            v += np.where(pos, w * np.where(np.isfinite(u[j]), u[j], 0.0), 0.0)
        best = np.minimum(best, np.where(ok, v, np.inf))
    return np.abs(u[nodes] - best), best


@pytest.mark.parametrize("patchy", [True, False])
def test_config3_full_size_fixed_point(pkg, patchy):
    p = W.sin3d(0)
    if not patchy:
        p = p.with_(n_coarse=None)
    st, u, lab = _solve(pkg, p)
    assert st == 0
    rng = np.random.default_rng(5)
    fin = np.isfinite(u) & (u > 0.0)   # free nodes of S* (targets hold 0)
    cand = np.nonzero(fin)[0]
    nodes = np.sort(rng.choice(cand, size=4000, replace=False))
    if not patchy:
        lab = np.where(np.isfinite(u), 0, -1).astype(np.int8)
    r, best = _residual_3d(p, u, lab, nodes)
    assert np.all(np.isfinite(best))
    # the polish stops when a FP64 sweep changes no value by 1e-6 or more
    assert r.max() <= 1e-5, (r.max(), nodes[np.argmax(r)])
    # a wrong patch rule or foot would leave residuals of the order of h
    assert math.isfinite(float(u[fin].max()))
