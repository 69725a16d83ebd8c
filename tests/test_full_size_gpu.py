"""Full-size counts against the oracle's own, stored in golden/full_size.txt by
golden/make_full_size.py (the oracle on its FP64 unit vectors; Sec. 2's pair
sets binned by App. A's separation, Eq. 2 on top):

  - the survey workload, whole (1M + 1M points, 2.0e12 pairs), through
    wtheta_count_wtheta with the library's defaults (far tile pairs skipped,
    spans settled per chunk), fed the oracle's unit vectors: P1, every slot of
    DD, DR and RR bit-identical;
  - 8 batch mocks spanning 20k-400k points, through one batch plan over unit
    vectors (wtheta_batch_plan_ex), graph replayed twice: P1;
  - 2 auto and 2 cross serve requests of 50k-150k points mixed into a stream
    of smaller requests on one server: the server converts RA/Dec itself, so
    this is P2 (bit-identical unless the oracle flagged pairs within a few
    ulps of an edge, then off by at most that many).

The stored counts were made from inputs this machine regenerates from the
same seeds; each line carries a hash of them, checked first (the synthetic
inputs depend on the platform's numpy and libm in their last bits).
"""
import hashlib
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "full_size.txt")


def _load():
    out = {}
    for line in open(GOLDEN):
        if not line.strip() or line.startswith("#"):
            continue
        f = line.split()
        out[(f[0], f[1])] = dict(n_a=int(f[2]), n_b=int(f[3]), sha_rd=f[4], sha_xyz=f[5],
                                 amb=int(f[6]), counts=np.array([int(x) for x in f[7:]],
                                                                np.uint64))
    return out


@pytest.fixture(scope="module")
def G():
    return _load()


@pytest.fixture(scope="module")
def W():
    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta
    return wtheta


def _sha(*arrays):
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:32]


def _same_inputs(g, rd, xyz):
    assert _sha(*rd) == g["sha_rd"] and _sha(*xyz) == g["sha_xyz"], (
        "the regenerated inputs differ from those the stored counts were made on "
        "(platform numpy/libm); rerun tests/golden/make_full_size.py on this platform")


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def test_survey_whole_p1(W, G):
    wl = synth.survey()
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    assert np.array_equal(e, O.edges(wl.lo_deg, wl.hi_deg, wl.n_bins))
    D, R = O.radec_to_xyz(wl.data), O.radec_to_xyz(wl.rand)
    _same_inputs(G[("survey", "DD")], [wl.data], [D])
    _same_inputs(G[("survey", "DR")], [wl.data, wl.rand], [D, R])
    _same_inputs(G[("survey", "RR")], [wl.rand], [R])
    K = wl.n_bins
    c = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
    W.wtheta_count_wtheta(_dev(D), _dev(R), True, e, c)
    torch.cuda.synchronize()
    got = c.cpu().numpy().astype(np.uint64)
    for k, name in enumerate(("DD", "DR", "RR")):
        assert np.array_equal(got[k], G[("survey", name)]["counts"]), name
    w = W.wtheta_ls(got[0], got[1], got[2], wl.n_d, wl.n_r)
    w_o = O.ls(*(G[("survey", n)]["counts"] for n in ("DD", "DR", "RR")), wl.n_d, wl.n_r)
    assert np.array_equal(w, w_o, equal_nan=True)


def _golden_mocks(G):
    return sorted({int(k[0].rsplit("_", 1)[1]) for k in G if k[0].startswith("batch_mock_")})


def test_batch_mocks_p1(W, G):
    ms = _golden_mocks(G)
    assert len(ms) >= 8
    e = O.edges(1.0 * synth.ARCMIN, 5.0, 16)
    K = len(e) - 1
    cats, xyz = [], []
    for m in ms:
        mk = synth.batch_mock(1, m)
        D, R = O.radec_to_xyz(mk.data), O.radec_to_xyz(mk.rand)
        _same_inputs(G[("batch_mock_%d" % m, "DR")], [mk.data, mk.rand], [D, R])
        xyz.append((D, R))
        cats.append((_dev(D), _dev(R)))
    plan = W.wtheta_batch_plan(cats, e, coords_are_xyz=True)
    out = torch.zeros((len(ms), 3, K + 2), dtype=torch.int64, device="cuda")
    for run in range(2):  # the graph replayed: identical counts
        out.zero_()
        W.wtheta_batch_run(plan, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().astype(np.uint64)
        for i, m in enumerate(ms):
            for k, name in enumerate(("DD", "DR", "RR")):
                assert np.array_equal(got[i, k], G[("batch_mock_%d" % m, name)]["counts"]), (
                    run, m, name)
    W.wtheta_batch_free(plan)


def _golden_requests(G):
    return sorted({int(k[0].rsplit("_", 1)[1]) for k in G if k[0].startswith("serve_request_")})


def test_serve_requests_in_a_mix_p2(W, G):
    qs = _golden_requests(G)
    kinds = {q: G.get(("serve_request_%d" % q, "DD")) is not None for q in qs}
    assert sum(kinds.values()) >= 2 and sum(not v for v in kinds.values()) >= 2
    e = O.edges(1.0 * synth.ARCMIN, 10.0, 24)
    reqs = {q: synth.serve_request(1, q) for q in qs}
    for q, rq in reqs.items():
        if rq.kind == "auto":
            _same_inputs(G[("serve_request_%d" % q, "DR")], [rq.data, rq.rand],
                         [O.radec_to_xyz(rq.data), O.radec_to_xyz(rq.rand)])
        else:
            _same_inputs(G[("serve_request_%d" % q, "D1D2")], [rq.data, rq.data2],
                         [O.radec_to_xyz(rq.data), O.radec_to_xyz(rq.data2)])
    # smaller requests of the same stream around them (all under 50k points)
    sizes, _ = synth.serve_sizes()
    fill = [q for q in range(200) if sizes[q] < 50_000 and q not in reqs][:16]
    srv = W.wtheta_server_create(e, 40 << 30)
    ids = {}
    order = sorted(list(reqs) + fill)
    for q in order:
        rq = reqs[q] if q in reqs else synth.serve_request(1, q)
        ids[q] = W.wtheta_server_submit(srv, rq.data, rq.rand, rq.data2, rq.rand2)
    for q in order:
        done, c, w = W.wtheta_server_wait(srv, ids[q], timeout_ms=300_000)
        assert done
        if q not in reqs:
            continue
        rq = reqs[q]
        names = ("DD", "DR", "RR") if rq.kind == "auto" else ("D1D2", "D1R2", "R1D2", "R1R2")
        for k, name in enumerate(names):
            g = G[("serve_request_%d" % q, name)]
            want = g["counts"]
            assert int(c[k].sum()) == int(want.sum())
            if g["amb"] == 0:
                assert np.array_equal(c[k], want), (q, name)
            else:
                print("serve request %d %s: %d pairs within tau of an edge" % (q, name, g["amb"]))
                assert np.abs(c[k].astype(np.int64) - want.astype(np.int64)).sum() <= 2 * g["amb"]
        if all(G[("serve_request_%d" % q, n)]["amb"] == 0 for n in names):
            want = [G[("serve_request_%d" % q, n)]["counts"] for n in names]
            if rq.kind == "auto":
                w_o = O.ls(*want, len(rq.data) // 2, len(rq.rand) // 2)
            else:
                w_o = O.ls_cross(*want, len(rq.data) // 2, len(rq.data2) // 2,
                                 len(rq.rand) // 2, len(rq.rand2) // 2)
            assert np.array_equal(w, w_o, equal_nan=True), q
        W.wtheta_server_release(srv, ids[q])
    W.wtheta_server_destroy(srv)
