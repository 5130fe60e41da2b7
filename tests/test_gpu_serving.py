"""Batched and served solves on the GPU: every result equals the same
problem solved alone, within the parity tolerance of the other tests (the
labels exactly; the FP32 sweeps exchange halos inside a launch, so their
iterates, not their fixed point, depend on timing)."""
import time

import numpy as np
import pytest

import workloads as W
from tests._labels import assert_labels

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    import torch

    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as pkg

    torch.cuda.set_device(0)
    return pkg


def _alone(P, p):
    with P.Plan(p, stream=0) as pl:
        st = pl.solve()
        return st, pl.values(), pl.labels()


def _same(u, ref):
    fin = np.isfinite(ref)
    assert np.array_equal(fin, np.isfinite(u))
    if fin.any():  # a ball thinner than the grid holds no node: nothing is reachable
        assert np.abs(u[fin] - ref[fin]).max() <= 1e-4 * ref[fin].max()


def test_batch_solve_matches_one_at_a_time(P):
    probs = W.batched(seed=3, count=10, side=(65, 161))
    refs = [_alone(P, p) for p in probs]
    plans = [P.Plan(p, stream=0) for p in probs]
    try:
        st = P.hjbp_batch_solve([pl.handle for pl in plans], workers=4)
        assert st == [0] * len(probs)
        for pl, (s0, u0, l0) in zip(plans, refs):
            _same(pl.values(), u0)
            assert np.array_equal(pl.labels(), l0)
        # the batch's Fourier-field problems against the FP64 oracle (the three smallest)
        import oracle

        for k in sorted(range(len(probs)), key=lambda q: probs[q].n_nodes)[:3]:
            ref = oracle.patchy_solve(probs[k], tol=1e-12, keep_phi=True)
            _same(plans[k].values(), ref.u)
            assert_labels(plans[k].labels(), ref, probs[k])
    finally:
        for pl in plans:
            pl.close()


def test_served_result_is_the_same_alone_and_in_the_mix(P):
    stream = W.serving_stream(seed=5, count=12, rate=1000.0, side2d=(65, 161), side3d=(17, 33))
    probs = [p for _, p in stream]
    refs = [_alone(P, p) for p in probs]
    srv = P.hjbp_server_create(budget_bytes=2 << 30, workers=4)
    keep = []
    try:
        tickets = []
        for p in probs:
            d, k = P.desc_from_problem(p)
            keep.append((d, k))
            tickets.append(P.hjbp_server_submit(srv, d))
        done = {}
        t0 = time.time()
        while len(done) < len(tickets) and time.time() - t0 < 300:
            for i, t in enumerate(tickets):
                if i in done:
                    continue
                st, h, lat = P.hjbp_server_poll(srv, t)
                if h:
                    done[i] = (st, P.Plan.adopt(probs[i], h), lat)
            time.sleep(0.002)
        assert len(done) == len(tickets)
        for i, (st, pl, lat) in done.items():
            assert st == refs[i][0] == 0
            _same(pl.values(), refs[i][1])
            assert np.array_equal(pl.labels(), refs[i][2])
            assert lat > 0
            pl.close()
    finally:
        P.hjbp_server_destroy(srv)


def test_autotune_picks_a_shape_and_caches_it(P, tmp_path):
    """The tuner times candidate launch shapes once per problem class, keeps
    the fastest in the process and in the cache file, and the tuned solve
    reaches the oracle's fixed point."""
    import oracle

    p = W.sincos2d(11, n=161, n_coarse=21, n_targets=2, radius=0.1)
    d, keep = P.desc_from_problem(p, flags=P.HJBP_FLAG_DIRICHLET)
    path = str(tmp_path / "tune.txt")
    t, cached = P.hjbp_autotune(d, 0, path)
    assert not cached and t[0] in (2, 3, 4) and t[1] in (2, 3, 4)
    t2, cached2 = P.hjbp_autotune(d, 0, path)
    assert cached2 and t2 == t
    fields = open(path).read().split()
    assert len(fields) == 9 and [int(v) for v in fields[5:9]] == t
    with P.Plan(p, tune=t, flags=P.HJBP_FLAG_DIRICHLET) as pl:
        assert pl.solve() == 0
        u = pl.values()
    ref = oracle.patchy_solve(p, tol=1e-12, dirichlet=True)
    _same(u, ref.u)
