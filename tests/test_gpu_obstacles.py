"""GPU parity with obstacles (Sec. 4, "Patchy method with obstacles"): nodes
inside a closed ball or box are state constraints like the ghost ring.  The
CUDA path through the C ABI against the FP64 oracle on the same inputs: equal
reachable sets, max |u_gpu - u_oracle| <= 1e-4 max u, labels agreeing on
>= 99.9 % of the nodes."""
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


def _run(pkg, p, **kw):
    with pkg.Plan(p, precision=pkg.HJBP_FP32_POLISH64, **kw) as plan:
        st = plan.solve()
        return st, plan.values(), plan.labels()


def _assert_values(u, ref, rel=1e-4):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(u)), (
        f"reachable sets differ: gpu-only {np.sum(np.isfinite(u) & ~fin)}, oracle-only {np.sum(fin & ~np.isfinite(u))}")
    err = np.abs(u[fin] - ref[fin]).max()
    assert err <= rel * ref[fin].max(), f"max err {err} vs bound {rel * ref[fin].max()}"


def test_global_with_obstacles(pkg):
    p = W.eikonal_obstacles(n=161, n_coarse=41).with_(n_coarse=None, speed="sincos2d", speed_params=W._params([0.5]),
                                                      tol=1e-8)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.global_solve(p, tol=1e-12)
    _assert_values(u, ref.u)


@pytest.mark.parametrize("dirichlet", [False, True])
@pytest.mark.parametrize("n,nc,parts", [(129, 33, 4), (257, 65, 8)])
def test_patchy_with_obstacles(pkg, dirichlet, n, nc, parts):
    p = W.eikonal_obstacles(n=n, n_coarse=nc, parts=parts)
    st, u, lab = _run(pkg, p, flags=pkg.HJBP_FLAG_DIRICHLET if dirichlet else 0)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True, dirichlet=dirichlet)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)
    kind, _, _ = oracle.setup(p)
    assert np.all(lab[kind == oracle.GHOST] == -1)


def test_3d_with_obstacles(pkg):
    p = W.sin3d(2, n=49, n_coarse=13, n_c=50, n_targets=4, radius=0.1).with_(
        obstacles=np.array([W.obstacle_ball((0.2, -0.1, 0.3), 0.3), W.obstacle_box((-0.8, -0.7, -0.9), (-0.3, 0.4, 0.1))]))
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)


def test_noalloc_with_obstacles(pkg):
    import torch

    # the no-allocation entry point takes ball targets
    p = W.eikonal_obstacles(n=129, n_coarse=33).with_(n_coarse=None, tol=1e-8, target_kind="balls", n_parts=0)
    d, keep = pkg.desc_from_problem(p, precision=pkg.HJBP_FP64)
    u = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    lab = torch.empty(p.n_nodes, dtype=torch.int8, device="cuda")
    st = pkg.hjbp_solve_global2d_noalloc(d, torch.cuda.current_stream().cuda_stream, u.data_ptr(), lab.data_ptr())
    torch.cuda.synchronize()
    assert st == 0
    ref = oracle.global_solve(p, tol=1e-12)
    _assert_values(u.cpu().numpy(), ref.u)
