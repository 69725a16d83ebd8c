"""Failure paths, with the failure made on the host: a device allocation that
the library is told to fail (wtheta_inject_alloc_failure) must come back as
WTHETA_ENOMEM from the call that made it, leave nothing half-done, and let the
next calls run normally.  No GPU fault is involved."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ENOMEM = -2


@pytest.fixture(scope="module")
def W():
    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta
    yield wtheta
    wtheta.wtheta_inject_alloc_failure(-1)


def test_count_reports_injected_allocation_failure(W):
    wl = synth.small(n=4000)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    d = torch.from_numpy(wl.data).cuda()
    r = torch.from_numpy(wl.rand).cuda()
    c = torch.zeros((3, len(e) + 1), dtype=torch.int64, device="cuda")
    for after in (0, 1, 2):
        W.wtheta_inject_alloc_failure(after)
        with pytest.raises(W.WthetaError) as ex:
            for _ in range(3):  # enough allocations to reach the failing one
                W.wtheta_count(d, r, e, False, c[1])
        assert ex.value.status == ENOMEM
    W.wtheta_inject_alloc_failure(-1)
    W.wtheta_count_wtheta(d, r, False, e, c)
    torch.cuda.synchronize()
    want = O.wtheta(wl.data, wl.rand, e)[:3]
    for k in range(3):
        assert int(c[k].sum()) == int(np.asarray(want[k]).sum())
    W.wtheta_inject_alloc_failure(0)
    with pytest.raises(W.WthetaError) as ex:
        W.wtheta_count_wtheta(d, r, False, e, c)
    assert ex.value.status == ENOMEM
    W.wtheta_inject_alloc_failure(-1)


def test_server_request_fails_alone(W):
    """The second admission's allocation fails: that request ends with
    WTHETA_ENOMEM, the others complete with their exact counts."""
    e = W.wtheta_edges(1.0 / 60.0, 4.0, 16)
    fp = synth.Patch(40.0, 6.0, 10.0, 16.0)
    reqs = [(synth.clustered(fp, 3000 + 500 * q, 60, 3.0, q, "test", "data"),
             synth.uniform(fp, 3200 + 500 * q, q, "test", "random")) for q in range(3)]
    srv = W.wtheta_server_create(e, 8 << 30)
    W.wtheta_inject_alloc_failure(1)
    ids = [W.wtheta_server_submit(srv, d, r) for d, r in reqs]
    try:
        for q, i in enumerate(ids):
            if q == 1:
                with pytest.raises(W.WthetaError) as ex:
                    W.wtheta_server_wait(srv, i, timeout_ms=60_000)
                assert ex.value.status == ENOMEM
                assert W.wtheta_server_request_info(srv, i)["state"] == W.RS_FAILED
            else:
                done, c, _ = W.wtheta_server_wait(srv, i, timeout_ms=60_000)
                assert done
                d, r = reqs[q]
                want = O.wtheta(d, r, e)[:3]
                for k in range(3):
                    assert np.array_equal(c[k], want[k])
            W.wtheta_server_release(srv, i)
    finally:
        W.wtheta_inject_alloc_failure(-1)
        W.wtheta_server_destroy(srv)


def test_server_cancel_queued_request(W):
    """A request cancelled while it waits for admission ends WTHETA_ECANCELED
    and never runs; one already admitted cannot be cancelled (WTHETA_EBUSY);
    the others complete exactly."""
    e = W.wtheta_edges(1.0 / 60.0, 4.0, 16)
    fp = synth.Patch(80.0, 8.0, -20.0, -12.0)
    big = (synth.clustered(fp, 500_000, 10_000, 3.0, 7, "test", "data"),
           synth.uniform(fp, 500_000, 7, "test", "random"))
    small = [(synth.clustered(fp, 2000 + 300 * q, 40, 3.0, 8 + q, "test", "data"),
              synth.uniform(fp, 2100 + 300 * q, 8 + q, "test", "random")) for q in range(3)]
    # one admitted request at a time: the small ones wait in the queue
    srv = W.wtheta_server_create(e, 8 << 30, max_active=1)
    try:
        i_big = W.wtheta_server_submit(srv, *big)
        ids = [W.wtheta_server_submit(srv, *m) for m in small]
        assert W.wtheta_server_request_info(srv, ids[1])["state"] == W.RS_QUEUED
        W.wtheta_server_cancel(srv, ids[1])
        with pytest.raises(W.WthetaError) as ex:
            W.wtheta_server_wait(srv, ids[1], timeout_ms=60_000)
        assert ex.value.status == -9
        assert W.wtheta_server_request_info(srv, ids[1])["state"] == W.RS_FAILED
        done, _, _ = W.wtheta_server_wait(srv, i_big, timeout_ms=120_000)
        assert done
        with pytest.raises(W.WthetaError) as ex:
            W.wtheta_server_cancel(srv, i_big)
        assert ex.value.status == -8
        for q in (0, 2):
            done, c, _ = W.wtheta_server_wait(srv, ids[q], timeout_ms=120_000)
            assert done
            want = O.wtheta(small[q][0], small[q][1], e)[:3]
            for k in range(3):
                assert np.array_equal(c[k], want[k])
    finally:
        W.wtheta_server_destroy(srv)
