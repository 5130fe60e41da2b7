"""GPU checks of kernel variants that must give the same result to the last
bit: the value sweep with 2 or 4 warps per tile (each warp takes a share of
the quadrants, Eq. SLscheme's minimum is exact whatever the order) against
the one-warp sweep, in every mode the multi-warp kernel serves (FP32 and
FP64, the symmetric pair form and the generic control table, state
constraints and Dirichlet data, the monotone and the plain update), and the
pair-form FP64 polish against the per-control polish within the tolerance
of the polish itself.  These comparisons run the deterministic block-Jacobi
launches (tune[7] = 1); the FP32 sweeps that exchange halos inside a launch
(the default) are checked against them for the same fixed point."""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    import torch

    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as P

    torch.cuda.set_device(0)
    return P


def _solve(pkg, p, warps, precision=None, flags=0, tune6=0, tune7=1):
    prec = pkg.HJBP_FP32_POLISH64 if precision is None else precision
    with pkg.Plan(p, precision=prec, flags=flags, tune=[0, 0, 0, warps, 0, 0, tune6, tune7]) as plan:
        st = plan.solve()
        return st, plan.values(), plan.labels()


CASES = {
    "patchy_fp32_pairs": (lambda: W.sincos2d(1, n=257, n_coarse=33, n_targets=4, radius=0.1), None, 0),
    "global_fp64_pairs": (lambda: W.sincos2d(2, n=193, n_coarse=25, radius=0.2).with_(n_coarse=None, tol=1e-10),
                          "fp64", 0),
    "generic_table": (lambda: W.random_speed_problem(3, n=75, n_c=27, box=2.0).with_(tol=1e-10), "fp64", 0),
    "dirichlet": (lambda: W.sincos2d(3, n=193, n_coarse=25, n_targets=3, radius=0.1), None, "dirichlet"),
    "warm_start": (lambda: W.sincos2d(4, n=193, n_coarse=25, n_targets=3, radius=0.1), None, "warm"),
    "obstacles": (lambda: W.eikonal_obstacles(n=161, n_coarse=41, parts=8), None, 0),
}


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("warps", [2, 4])
def test_multi_warp_sweep_equals_one_warp(pkg, case, warps):
    make, prec, mode = CASES[case]
    p = make()
    precision = pkg.HJBP_FP64 if prec == "fp64" else None
    flags = {"dirichlet": pkg.HJBP_FLAG_DIRICHLET, "warm": pkg.HJBP_FLAG_WARM_START}.get(mode, 0)
    s1, u1, l1 = _solve(pkg, p, 1, precision, flags)
    sw, uw, lw = _solve(pkg, p, warps, precision, flags)
    assert s1 == 0 and sw == 0
    assert np.array_equal(l1, lw)
    assert np.array_equal(u1, uw), f"max diff {np.nanmax(np.abs(u1 - uw))}"


def test_pair_form_polish_matches_per_control_polish(pkg):
    p = W.sincos2d(5, n=257, n_coarse=33, n_targets=4, radius=0.05)
    s0, u0, l0 = _solve(pkg, p, 1)
    s1, u1, l1 = _solve(pkg, p, 1, tune6=1)
    assert s0 == 0 and s1 == 0
    assert np.array_equal(l0, l1)
    fin = np.isfinite(u1)
    assert np.array_equal(fin, np.isfinite(u0))
    # both stop at an FP64 sup-norm change below tol = 1e-6 of the same fixed point
    assert np.abs(u0[fin] - u1[fin]).max() <= 1e-5
    ref = oracle.patchy_solve(p, tol=1e-12)
    assert np.abs(u0[fin] - ref.u[fin]).max() <= 1e-4 * ref.u[fin].max()


@pytest.mark.parametrize("case", ["patchy_fp32_pairs", "obstacles", "warm_start"])
def test_packed_pair_update_equals_scalar(pkg, case):
    """The FP32 update with two quadrants per packed FP32x2 operation (the
    default) rounds every operation as the scalar form (tune[6] = 2) does."""
    make, prec, mode = CASES[case]
    p = make()
    flags = {"dirichlet": pkg.HJBP_FLAG_DIRICHLET, "warm": pkg.HJBP_FLAG_WARM_START}.get(mode, 0)
    s0, u0, l0 = _solve(pkg, p, 1, None, flags)
    s2, u2, l2 = _solve(pkg, p, 1, None, flags, tune6=2)
    assert s0 == 0 and s2 == 0
    assert np.array_equal(l0, l2)
    assert np.array_equal(u0, u2)


@pytest.mark.parametrize("family", ["sin3d", "eikonal3d_dirichlet"])
def test_packed_pair_update_3d_equals_scalar(pkg, family):
    """3D: two controls of an octant per packed FP32x2 chain (the default)
    against one at a time (tune[6] = 2), equal to the last bit."""
    if family == "sin3d":
        p, flags = W.sin3d(0, n=41, n_coarse=11, n_targets=4, radius=0.12), 0
    else:
        p, flags = W.eikonal3d(n=41, n_coarse=11, n_c=50), pkg.HJBP_FLAG_DIRICHLET
    s0, u0, l0 = _solve(pkg, p, 1, None, flags)
    s2, u2, l2 = _solve(pkg, p, 1, None, flags, tune6=2)
    assert s0 == 0 and s2 == 0
    assert np.array_equal(l0, l2)
    assert np.array_equal(u0, u2)


@pytest.mark.parametrize("case", ["patchy_fp32_pairs", "dirichlet", "obstacles"])
@pytest.mark.parametrize("tune7", [0, 2])
def test_halo_exchange_reaches_the_same_fixed_point(pkg, case, tune7):
    """The FP32 sweep that publishes its boundary and re-reads its halo
    inside a launch (after every pass: tune[7] = 0, the default; after every
    round: 2) reads a neighbour's older or newer value, both upper bounds of
    the fixed point, so the monotone iteration ends at the same fixed point
    (R8) as the block-Jacobi launches: within the stopping tolerance, and
    within the parity bound of the FP64 oracle."""
    make, prec, mode = CASES[case]
    p = make()
    flags = {"dirichlet": pkg.HJBP_FLAG_DIRICHLET, "warm": pkg.HJBP_FLAG_WARM_START}.get(mode, 0)
    s1, u1, l1 = _solve(pkg, p, 1, None, flags, tune7=1)
    sx, ux, lx = _solve(pkg, p, 1, None, flags, tune7=tune7)
    assert s1 == 0 and sx == 0
    assert np.array_equal(l1, lx)
    fin = np.isfinite(u1)
    assert np.array_equal(fin, np.isfinite(ux))
    assert np.abs(ux[fin] - u1[fin]).max() <= 2e-5 * u1[fin].max()
    ref = oracle.patchy_solve(p, tol=1e-12, dirichlet=mode == "dirichlet")
    assert np.abs(ux[fin] - ref.u[fin]).max() <= 1e-4 * ref.u[fin].max()
