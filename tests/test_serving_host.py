"""Host-side checks of the batched / served API that need no GPU: admission
refuses requests that can never fit the memory budget (EBUSY), malformed
requests are rejected at submit (EINVAL), and a server with nothing running
shuts down cleanly."""
import pytest

import workloads as W


@pytest.fixture(scope="module")
def P():
    from paper_1109_3577_gb300 import build as b

    b.build()
    import paper_1109_3577_gb300 as pkg

    return pkg


def test_admission_refuses_oversized_request(P):
    srv = P.hjbp_server_create(budget_bytes=1 << 20, workers=2)
    try:
        d, keep = P.desc_from_problem(W.sincos2d(0, n=1025, n_coarse=33))
        with pytest.raises(P.HjbpError) as ei:
            P.hjbp_server_submit(srv, d)
        assert ei.value.status == 6          # EBUSY
        assert P.hjbp_server_stats(srv) == (0, 0, 0)
    finally:
        P.hjbp_server_destroy(srv)


def test_malformed_request_is_rejected(P):
    srv = P.hjbp_server_create(budget_bytes=1 << 30, workers=1)
    try:
        for q in (W.sincos2d(0, n=65, n_coarse=17).with_(tol=-1.0),
                  W.zermelo(n=33, n_coarse=9, n_c=8, parts=4, s=2.0)):   # a control that cannot move
            d, keep = P.desc_from_problem(q)
            with pytest.raises(P.HjbpError) as ei:
                P.hjbp_server_submit(srv, d)
            assert ei.value.status == 1      # EINVAL
        assert P.hjbp_server_stats(srv) == (0, 0, 0)
    finally:
        P.hjbp_server_destroy(srv)


def test_batch_rejects_null_plan(P):
    with pytest.raises(P.HjbpError) as ei:
        P.hjbp_batch_solve([0, 0])
    assert ei.value.status == 1


def test_failed_create_finishes_the_request_without_a_plan(P):
    """Submit only validates and copies a request; the admitting worker creates
    the plan.  Without a GPU that create fails, and the request finishes with
    its status (the allocation's ENOMEM or ECUDA) and no plan, the message
    carried to the polling thread."""
    import time

    import torch

    if torch.cuda.is_available():
        pytest.skip("needs a process without a GPU")
    srv = P.hjbp_server_create(budget_bytes=1 << 30, workers=2)
    try:
        d, keep = P.desc_from_problem(W.sincos2d(0, n=65, n_coarse=17))
        t = P.hjbp_server_submit(srv, d)
        del d, keep                              # the server holds its own copy
        t0 = time.time()
        while True:
            try:
                st, h, _ = P.hjbp_server_poll(srv, t)
            except P.HjbpError as e:
                assert e.status in (2, 5)           # ENOMEM / ECUDA
                assert "cudaMalloc" in str(e) or "CUDA" in str(e), str(e)
                break
            assert h is None and st == 0
            assert time.time() - t0 < 60
            time.sleep(0.01)
        assert P.hjbp_server_stats(srv) == (0, 0, 0)
    finally:
        P.hjbp_server_destroy(srv)


def test_admission_waits_for_memory_to_be_collected(P):
    """Continuous batching by device memory: a request that does not fit next
    to the bytes held by earlier ones waits in the queue, holding nothing,
    and is admitted once the earlier request is collected.  Without a GPU
    every admitted request fails at plan creation, which still exercises the
    queue and the accounting."""
    import time

    import torch

    if torch.cuda.is_available():
        pytest.skip("needs a process without a GPU")

    def wait_for(srv, want, limit=30.0):
        t0 = time.time()
        while P.hjbp_server_stats(srv) != want:
            assert time.time() - t0 < limit, P.hjbp_server_stats(srv)
            time.sleep(0.005)

    d, keep = P.desc_from_problem(W.sincos2d(0, n=129, n_coarse=17))
    # the request's footprint, read from a server with room to spare
    srv = P.hjbp_server_create(budget_bytes=1 << 40, workers=1)
    try:
        P.hjbp_server_submit(srv, d)
        t0 = time.time()
        while P.hjbp_server_stats(srv)[2] == 0 or P.hjbp_server_stats(srv)[1] != 0:
            assert time.time() - t0 < 30.0
            time.sleep(0.005)
        fp = P.hjbp_server_stats(srv)[2]
    finally:
        P.hjbp_server_destroy(srv)
    assert fp > 0
    srv = P.hjbp_server_create(budget_bytes=fp + fp // 2, workers=2)
    try:
        a = P.hjbp_server_submit(srv, d)
        b = P.hjbp_server_submit(srv, d)
        wait_for(srv, (1, 0, fp))             # a finished and uncollected, b queued
        time.sleep(0.05)
        assert P.hjbp_server_stats(srv) == (1, 0, fp)
        with pytest.raises(P.HjbpError):      # a's plan could not be created
            P.hjbp_server_poll(srv, a)
        wait_for(srv, (0, 0, fp))             # b admitted and finished
        with pytest.raises(P.HjbpError):
            P.hjbp_server_poll(srv, b)
        assert P.hjbp_server_stats(srv) == (0, 0, 0)
    finally:
        P.hjbp_server_destroy(srv)
