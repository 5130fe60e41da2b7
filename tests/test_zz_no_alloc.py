"""The solve entry point that allocates nothing, against hjbp_solve.

hjbp_solve_global2d_noalloc serves callers that cannot allocate device
memory at solve time (for example code that runs while a stream is captured
into a CUDA graph, or a real-time loop that forbids allocation after start-up).
Its scratch is one fixed array inside the library, shared by every call, so
each call must clear what it relies on: two calls in a row, on the same and
on a different problem, must each reproduce hjbp_solve.

This file is collected last, so that a run stopping at the first failure has
already run every other test.
"""
import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu

REL_TOL = 1e-4   # the parity tolerance of the other GPU tests


def _reference(P, p):
    with P.Plan(p, precision=P.HJBP_FP64) as plan:
        assert plan.solve() == 0
        return plan.values(), plan.labels()


def _noalloc(P, p, u, lab):
    import torch

    d, keep = P.desc_from_problem(p, precision=P.HJBP_FP64)
    u.fill_(float("nan"))
    lab.fill_(99)
    st = P.hjbp_solve_global2d_noalloc(d, torch.cuda.current_stream().cuda_stream, u.data_ptr(), lab.data_ptr())
    torch.cuda.synchronize()
    return st, u.cpu().numpy(), lab.cpu().numpy()


def _compare(u, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(u))
    assert np.abs(u[fin] - ref[fin]).max() <= REL_TOL * ref[fin].max()


def test_noalloc_matches_solve_on_two_calls_in_a_row():
    import torch

    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as P

    torch.cuda.set_device(0)
    problems = [W.sincos2d(1, n=129, n_coarse=17, radius=0.2).with_(n_coarse=None), W.eikonal2d()]
    refs = [_reference(P, p) for p in problems]
    for p, (uref, lref) in zip(problems, refs):
        u = torch.empty(p.n_nodes, dtype=torch.float64, device="cuda")
        lab = torch.empty(p.n_nodes, dtype=torch.int8, device="cuda")
        for _ in range(2):
            st, uh, lh = _noalloc(P, p, u, lab)
            assert st == 0, P.hjbp_last_error()
            _compare(uh, uref)
            assert np.array_equal(lh, lref)


def test_noalloc_rejects_grids_beyond_its_scratch():
    import torch

    import paper_1109_3577_gb300 as P

    p = W.eikonal2d(n=1025)          # 1,050,625 nodes > HJBP_NOALLOC_MAX_NODES
    assert p.n_nodes > P.HJBP_NOALLOC_MAX_NODES
    u = torch.empty(1, dtype=torch.float64, device="cuda")
    lab = torch.empty(1, dtype=torch.int8, device="cuda")
    d, keep = P.desc_from_problem(p, precision=P.HJBP_FP64)
    with pytest.raises(P.HjbpError) as ei:
        P.hjbp_solve_global2d_noalloc(d, torch.cuda.current_stream().cuda_stream, u.data_ptr(), lab.data_ptr())
    assert ei.value.status == 1
    assert "HJBP_NOALLOC_MAX_NODES" in P.hjbp_last_error()
