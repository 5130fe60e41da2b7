"""Options together on the CUDA path, against the FP64 oracle: obstacles with
the Dirichlet patch boundary (Eq. dbc) and all three add-ons of Sec. 6 in 2D
and 3D, Brockett's integrator in FP64 and with the add-ons, the tile queue
with obstacles.  AO1 (warm start) and AO2 (causal sweeps) leave the fixed
point unchanged, so the oracle runs with the Dirichlet data and cones only."""
import numpy as np
import pytest

import oracle
import workloads as W
from tests._labels import assert_labels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as P

    torch.cuda.set_device(0)
    return P


def _run(pkg, p, precision=None, **kw):
    prec = pkg.HJBP_FP32_POLISH64 if precision is None else precision
    with pkg.Plan(p, precision=prec, **kw) as plan:
        st = plan.solve()
        return st, plan.values(), plan.labels()


def _assert_values(u, ref, rel=1e-4):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(u)), (np.sum(np.isfinite(u) & ~fin), np.sum(fin & ~np.isfinite(u)))
    assert np.abs(u[fin] - ref[fin]).max() <= rel * ref[fin].max()


def _all_addons(pkg):
    return pkg.HJBP_FLAG_DIRICHLET | pkg.HJBP_FLAG_WARM_START | pkg.HJBP_FLAG_CAUSAL_SWEEPS


def test_2d_obstacles_with_every_addon(pkg):
    p = W.eikonal_obstacles(n=129, n_coarse=33, parts=4)
    st, u, lab = _run(pkg, p, flags=_all_addons(pkg), reduce_r=4.0)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True, dirichlet=True, reduce_r=4.0)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)


def test_3d_fan_obstacles_with_every_addon(pkg):
    p = W.fan3d(n=25, n_coarse=7, n_c=26).with_(
        obstacles=np.array([W.obstacle_ball((1.0, 0.8, -0.6), 0.5), W.obstacle_box((-1.5, -1.2, 0.2), (-0.6, 0.4, 1.1))]))
    st, u, lab = _run(pkg, p, flags=_all_addons(pkg), reduce_r=4.0)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True, dirichlet=True, reduce_r=4.0)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)


def test_brockett_fp64_mode(pkg):
    p = W.brockett3d(n=34, n_coarse=17)
    st, u, lab = _run(pkg, p, precision=pkg.HJBP_FP64, flags=pkg.HJBP_FLAG_DIRICHLET)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True, dirichlet=True)
    _assert_values(u, ref.u)


def test_brockett_with_warm_start_and_causal_sweeps(pkg):
    p = W.brockett3d(n=34, n_coarse=17)
    st, u, lab = _run(pkg, p, flags=_all_addons(pkg))
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True, dirichlet=True)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)


def test_tile_queue_with_obstacles(pkg):
    p = W.eikonal_obstacles(n=161, n_coarse=41).with_(n_coarse=None, tol=1e-8)
    st, u, lab = _run(pkg, p, flags=pkg.HJBP_FLAG_TILE_QUEUE)
    assert st == 0
    ref = oracle.global_solve(p, tol=1e-12)
    _assert_values(u, ref.u)
