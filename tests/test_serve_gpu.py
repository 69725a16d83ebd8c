"""The continuous-batching server: every request's counts and w(theta) equal
those of the request counted alone, whatever it was mixed with."""
import time

import numpy as np
import pytest

from paper_1208_3658_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ARCMIN = 1.0 / 60.0


@pytest.fixture(scope="module")
def W():
    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta
    return wtheta


def _requests(n, lo, hi, seed):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        m = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        ra0, dec0 = rng.uniform(0, 360), rng.uniform(-60, 45)
        fp = synth.Patch(ra0, 8.0, dec0, dec0 + 8.0)
        d = synth.clustered(fp, m, max(1, m // 50), 3.0, seed, "test", "data", q)
        r = synth.uniform(fp, m + 5, seed, "test", "random", q)
        if q % 3 == 2:
            d2 = synth.clustered(fp, m + 11, max(1, m // 50), 3.0, seed, "test", "data2", q)
            r2 = synth.uniform(fp, m + 17, seed, "test", "random2", q)
            out.append((d, r, d2, r2))
        else:
            out.append((d, r, None, None))
    return out


def _alone(W, e, d, r, d2, r2):
    """The request's counts and w from single-count calls."""
    K = len(e) - 1
    dev = [torch.from_numpy(x).cuda() if x is not None else None for x in (d, r, d2, r2)]
    if d2 is None:
        c = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
        W.wtheta_count(dev[0], None, e, True, c[0])
        W.wtheta_count(dev[0], dev[1], e, False, c[1])
        W.wtheta_count(dev[1], None, e, True, c[2])
        torch.cuda.synchronize()
        c = c.cpu().numpy().astype(np.uint64)
        return c, W.wtheta_ls(c[0], c[1], c[2], len(d) // 2, len(r) // 2)
    c = torch.zeros((4, K + 2), dtype=torch.int64, device="cuda")
    for k, (a, b) in enumerate([(0, 2), (0, 3), (1, 2), (1, 3)]):
        W.wtheta_count(dev[a], dev[b], e, False, c[k])
    torch.cuda.synchronize()
    c = c.cpu().numpy().astype(np.uint64)
    return c, W.wtheta_ls_cross(c[0], c[1], c[2], c[3], len(d) // 2, len(d2) // 2,
                                len(r) // 2, len(r2) // 2)


def _serve(W, e, reqs, budget, stagger_s=0.0):
    srv = W.wtheta_server_create(e, budget)
    ids = []
    for d, r, d2, r2 in reqs:
        ids.append(W.wtheta_server_submit(srv, d, r, d2, r2))
        if stagger_s:
            time.sleep(stagger_s)
    out = []
    for i in ids:
        done, c, w = W.wtheta_server_wait(srv, i, timeout_ms=120_000)
        assert done
        out.append((c.copy(), w.copy(), W.wtheta_server_request_info(srv, i)))
        W.wtheta_server_release(srv, i)
    st = W.wtheta_server_stats(srv)
    W.wtheta_server_destroy(srv)
    return out, st


def test_mixed_requests_equal_alone(W):
    e = W.wtheta_edges(1.0 * ARCMIN, 4.0, 24)
    reqs = _requests(10, 500, 30_000, 41)
    got, st = _serve(W, e, reqs, budget=8 << 30)
    assert st["completed"] == len(reqs) and st["queued"] == 0 and st["active"] == 0
    for q, (c, w, info) in enumerate(got):
        want_c, want_w = _alone(W, e, *reqs[q])
        assert np.array_equal(c, want_c), q
        ok = np.isfinite(want_w)
        assert np.array_equal(np.isfinite(w), ok)
        assert np.all(np.abs(w[ok] - want_w[ok]) <= 1e-12 * np.maximum(np.abs(want_w[ok]), 4.0))
        assert info["state"] == W.RS_DONE and info["t_done"] >= info["t_admit"] >= info["t_submit"]


def test_results_do_not_depend_on_the_mix(W):
    """The same requests, staggered and under a budget that admits only a few
    at a time, give identical counts."""
    e = W.wtheta_edges(1.0 * ARCMIN, 4.0, 24)
    reqs = _requests(8, 2_000, 60_000, 42)
    a, _ = _serve(W, e, reqs, budget=8 << 30)
    b, _ = _serve(W, e, reqs, budget=40 << 20, stagger_s=0.01)
    for (ca, wa, _), (cb, wb, _) in zip(a, b):
        assert np.array_equal(ca, cb)
        assert np.array_equal(wa, wb, equal_nan=True)


def test_budget_and_bounded_wait(W):
    e = W.wtheta_edges(1.0 * ARCMIN, 4.0, 24)
    srv = W.wtheta_server_create(e, 4 << 20)          # 4 MiB: a 300k request cannot fit
    big = _requests(1, 300_000, 300_001, 43)[0]
    with pytest.raises(W.WthetaError) as ex:
        W.wtheta_server_submit(srv, *big)
    assert ex.value.status == -5                       # WTHETA_EBUDGET
    W.wtheta_server_destroy(srv)
    srv = W.wtheta_server_create(e, 8 << 30)
    rid = W.wtheta_server_submit(srv, *big)
    done, _, _ = W.wtheta_server_wait(srv, rid, timeout_ms=0)   # just look
    if not done:
        with pytest.raises(W.WthetaError) as ex:
            W.wtheta_server_wait(srv, rid, timeout_ms=1)
        assert ex.value.status in (-4,)                  # WTHETA_ETIMEOUT
    done, c, _ = W.wtheta_server_wait(srv, rid, timeout_ms=120_000)
    assert done and int(c[0].sum()) == 300_000 * 299_999 // 2
    W.wtheta_server_destroy(srv)
