"""The CUDA path at the limits of the ABI and in degenerate cases, against the
FP64 oracle: the largest control sets (HJBP_MAX_CONTROLS = 256 for the global
solve; 255 for patchy solves, whose feedback a* is one byte) in 2D and 3D,
the largest number of patches (HJBP_MAX_TARGETS = 64: one disk in 64
sectors, eight colour groups of the transport), a target that holds no node
(nothing is reachable) and the smallest 3D grid."""
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
    assert np.array_equal(fin, np.isfinite(u))
    if fin.any():
        assert np.abs(u[fin] - ref[fin]).max() <= rel * ref[fin].max()


@pytest.mark.parametrize("patchy", [False, True])
def test_largest_control_sets_2d(pkg, patchy):
    p = W.sincos2d(4, n=97, n_coarse=25, n_c=255 if patchy else 256, n_targets=3, radius=0.15)
    if not patchy:
        p = p.with_(n_coarse=None)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True) if patchy else oracle.global_solve(p, tol=1e-12)
    _assert_values(u, ref.u)
    if patchy:
        assert_labels(lab, ref, p)


def test_patchy_rejects_256_controls(pkg):
    d, keep = pkg.desc_from_problem(W.sincos2d(4, n=97, n_coarse=25, n_c=256, n_targets=3, radius=0.15))
    with pytest.raises(pkg.HjbpError) as ei:
        pkg.hjbp_create(d, 0, None)
    assert ei.value.status == 1


def test_largest_control_set_3d(pkg):
    p = W.sin3d(1, n=25, n_coarse=9, n_c=255, n_targets=2, radius=0.2)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)


def test_64_patches(pkg):
    p = W.eikonal_sectors(n=129, n_coarse=33, parts=64)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)
    assert len(set(ref.labels[ref.labels >= 0])) == 64


@pytest.mark.parametrize("patchy", [False, True])
def test_target_without_nodes(pkg, patchy):
    """A disk thinner than the grid, between nodes: no target node, so no node
    reaches the target and every value is +inf (label -1)."""
    k = 4.0 / 64
    p = W.eikonal2d(n=65).with_(targets=np.array([[0.5 * k, 0.5 * k, 0.1 * k]]))
    if patchy:
        p = p.with_(n_coarse=(17, 17, 1))
    st, u, lab = _run(pkg, p)
    assert st == 0
    assert np.all(np.isinf(u)) and np.all(lab == -1)
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True) if patchy else oracle.global_solve(p, tol=1e-12)
    assert np.all(np.isinf(ref.u))


def test_smallest_3d_grid(pkg):
    """3 x 3 x 3: one interior node, which is the target."""
    p = W.sin3d(0, n=3, n_coarse=3, n_targets=1, radius=0.1).with_(
        targets=np.array([[0.0, 0.0, 0.0, 0.1]]), n_coarse=None)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.global_solve(p, tol=1e-12)
    _assert_values(u, ref.u)
    assert u[13] == 0.0


def test_256_controls_3d_global(pkg):
    p = W.sin3d(1, n=21, n_coarse=9, n_c=256, n_targets=2, radius=0.2).with_(n_coarse=None)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.global_solve(p, tol=1e-12)
    _assert_values(u, ref.u)


@pytest.mark.parametrize("patchy", [False, True])
def test_non_square_grid_2d(pkg, patchy):
    """Different node counts per axis at equal spacing: [-2, 2] x [-1, 1.5]
    with 129 x 81 nodes (x fastest), targets placed inside."""
    p = W.sincos2d(2, n=129, n_coarse=33, n_targets=2, radius=0.12).with_(
        n=(129, 81, 1), hi=(2.0, 1.5, 0.0), lo=(-2.0, -1.0, 0.0),
        targets=np.array([[1.0, 0.5, 0.12], [-0.8, -0.3, 0.12]]))
    p = p.with_(n_coarse=(33, 21, 1) if patchy else None)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True) if patchy else oracle.global_solve(p, tol=1e-12)
    _assert_values(u, ref.u)
    if patchy:
        assert_labels(lab, ref, p)


@pytest.mark.parametrize("patchy", [False, True])
def test_non_square_grid_3d(pkg, patchy):
    p = W.sin3d(3, n=33, n_coarse=9, n_c=26, n_targets=2, radius=0.15).with_(
        n=(33, 25, 21), lo=(-1.0, -1.0, -1.0), hi=(1.0, 0.5, 0.25),
        targets=np.array([[0.4, -0.3, -0.2, 0.15], [-0.5, 0.1, 0.0, 0.15]]))
    p = p.with_(n_coarse=(9, 7, 6) if patchy else None)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True) if patchy else oracle.global_solve(p, tol=1e-12)
    _assert_values(u, ref.u)
    if patchy:
        assert_labels(lab, ref, p)


def test_64_patches_3d(pkg):
    p = W.eikonal3d(n=33, n_coarse=17, n_c=26, split="sectors", parts=64)
    st, u, lab = _run(pkg, p)
    assert st == 0
    ref = oracle.patchy_solve(p, tol=1e-12, keep_phi=True)
    _assert_values(u, ref.u)
    assert_labels(lab, ref, p)
