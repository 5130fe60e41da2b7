"""The solve entry point that allocates nothing, against hjbp_solve.

hjbp_solve_global2d_noalloc serves callers that cannot allocate device
memory at solve time (for example a real-time loop that forbids allocation
after start-up, or a host whose device memory pool belongs to another
component).  Its scratch is one fixed array inside the library, shared by
every call, so each call must clear what it relies on: two calls in a row,
on the same and on a different problem, must each reproduce hjbp_solve.

Both paths compute in FP64 and run the same kernels in the same order, so
they are compared at 1e-12 of the largest value, with identical labels; the
solves here run to a 1e-11 sup-norm change and are also compared with the
FP64 oracle at 1e-8 of the largest value.

This file is collected last, so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import oracle
import workloads as W

pytestmark = pytest.mark.gpu

SAME_PATH_TOL = 1e-12   # hjbp_solve and the no-allocation call, both FP64
ORACLE_TOL = 1e-8       # against the FP64 oracle solved to 1e-12


@pytest.fixture(scope="module")
def P():
    import torch

    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as P

    torch.cuda.set_device(0)
    return P


def _reference(P, p, max_sweeps=0):
    with P.Plan(p, precision=P.HJBP_FP64, max_sweeps=max_sweeps) as plan:
        st = plan.solve()
        return st, plan.values(), plan.labels()


def _noalloc(P, p, u, lab, max_sweeps=0):
    import torch

    d, keep = P.desc_from_problem(p, precision=P.HJBP_FP64, max_sweeps=max_sweeps)
    u.fill_(float("nan"))
    lab.fill_(99)
    st = P.hjbp_solve_global2d_noalloc(d, torch.cuda.current_stream().cuda_stream, u.data_ptr(), lab.data_ptr())
    torch.cuda.synchronize()
    return st, u.cpu().numpy(), lab.cpu().numpy()


def _compare(u, ref, tol):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(u)), "reachable sets differ"
    err = np.abs(u[fin] - ref[fin]).max()
    assert err <= tol * ref[fin].max(), f"max |u - ref| = {err:.3e}"


def _buffers(p):
    import torch

    u = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
    lab = torch.empty(p.n_nodes, dtype=torch.int8, device="cuda")
    return u, lab


def test_noalloc_matches_solve_on_two_calls_in_a_row(P):
    problems = [W.sincos2d(1, n=129, n_coarse=17, radius=0.2).with_(n_coarse=None, tol=1e-11),
                W.eikonal2d(tol=1e-11)]
    for p in problems:
        st, uref, lref = _reference(P, p)
        assert st == 0
        orc = oracle.global_solve(p, tol=1e-12)
        u, lab = _buffers(p)
        for _ in range(2):
            st, uh, lh = _noalloc(P, p, u, lab)
            assert st == 0, P.hjbp_last_error()
            _compare(uh, uref, SAME_PATH_TOL)
            assert np.array_equal(lh, lref)
            _compare(uh, orc.u, ORACLE_TOL)


def test_noalloc_with_obstacles_and_a_zero_speed_line(P):
    # Fan's speed |x1 + x2 + 0.1| stops nodes on a line; a disk and a box block others
    p = W.fan(n=129).with_(n_coarse=None, tol=1e-11, target_kind="balls", n_parts=0,
                           targets=np.array([[0.9, -0.4, 0.15]]),
                           obstacles=np.array([W.obstacle_ball((-0.8, 0.9), 0.3),
                                               W.obstacle_box((0.2, 0.5), (0.7, 1.2))]))
    st, uref, lref = _reference(P, p)
    assert st == 0
    u, lab = _buffers(p)
    for _ in range(2):
        st, uh, lh = _noalloc(P, p, u, lab)
        assert st == 0, P.hjbp_last_error()
        _compare(uh, uref, SAME_PATH_TOL)
        assert np.array_equal(lh, lref)
    _compare(uh, oracle.global_solve(p, tol=1e-12).u, ORACLE_TOL)


def test_noalloc_sweep_cap_gives_enoconv_and_the_same_iterate(P):
    p = W.eikonal2d(n=257, tol=1e-11)
    st, uref, lref = _reference(P, p, max_sweeps=3)
    assert st == P.HJBP_ENOCONV
    u, lab = _buffers(p)
    st, uh, lh = _noalloc(P, p, u, lab, max_sweeps=3)
    assert st == P.HJBP_ENOCONV
    _compare(uh, uref, SAME_PATH_TOL)
    assert np.array_equal(lh, lref)
    # a later uncapped call on the same scratch still converges to the fixed point
    st, uh, _ = _noalloc(P, p, u, lab)
    assert st == 0
    _compare(uh, oracle.global_solve(p, tol=1e-12).u, ORACLE_TOL)


def test_noalloc_rejects_what_a_global_solve_rejects(P):
    import torch

    u = torch.empty(1, dtype=torch.float64, device="cuda")
    lab = torch.empty(1, dtype=torch.int8, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    p = W.eikonal2d(n=1025)          # 1,050,625 nodes > HJBP_NOALLOC_MAX_NODES
    assert p.n_nodes > P.HJBP_NOALLOC_MAX_NODES
    d, keep = P.desc_from_problem(p, precision=P.HJBP_FP64)
    with pytest.raises(P.HjbpError) as ei:
        P.hjbp_solve_global2d_noalloc(d, stream, u.data_ptr(), lab.data_ptr())
    assert ei.value.status == P.HJBP_EINVAL
    assert "HJBP_NOALLOC_MAX_NODES" in P.hjbp_last_error()
    # patchy-only options on a global descriptor
    small = W.eikonal2d(n=65)
    for field, value, word in (("flags", P.HJBP_FLAG_DIRICHLET, "patchy"), ("reduce_r", 4.0, "reduce_r")):
        d, keep = P.desc_from_problem(small, precision=P.HJBP_FP64)
        setattr(d, field, value)
        with pytest.raises(P.HjbpError) as ei:
            P.hjbp_solve_global2d_noalloc(d, stream, u.data_ptr(), lab.data_ptr())
        assert ei.value.status == P.HJBP_EINVAL
        assert word in P.hjbp_last_error()
