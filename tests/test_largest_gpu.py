"""The largest workload: 10M clustered + 10M uniform full-sky points, 64 log
bins 0.2'-30 deg, counted in the library's default configuration (far tile
pairs skipped, spans settled per chunk).

The oracle cannot count 2e14 pairs, so the full-size counts are checked by
what holds at any size and by samples the oracle can compute:
  - exact pair totals;
  - RR of full-sky uniform points against the binomial law of Sec. 2's pair
    counts (a pair's separation falls in [t1, t2) with probability
    (cos t1 - cos t2)/2, independently of the other pairs), within 5 sigma;
  - 400 sampled data rows against all 10M randoms, bit-identical to the
    oracle on its own unit vectors;
  - a seeded 200k + 200k subsample: DD, DR, RR against the oracle, P1 on the
    oracle's unit vectors (zero tolerance) and P2 from RA/Dec (the device
    converts; pairs within a few ulps of an edge may differ).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def W():
    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta
    return wtheta


@pytest.fixture(scope="module")
def wl():
    return synth.largest()


def _count(W, a, b, e, auto, xyz=False):
    c = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
    da = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    db = None if auto else torch.from_numpy(np.ascontiguousarray(b)).cuda()
    if xyz:
        W.wtheta_count_xyz(da, db, e, auto, c)
    else:
        W.wtheta_count(da, db, e, auto, c)
    torch.cuda.synchronize()
    return c.cpu().numpy().astype(np.uint64)


def test_full_size_totals_and_binomial_rr(W, wl):
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    nd, nr = wl.n_d, wl.n_r
    RR = _count(W, wl.rand, None, e, True)
    DD = _count(W, wl.data, None, e, True)
    assert int(RR.sum()) == nr * (nr - 1) // 2
    assert int(DD.sum()) == nd * (nd - 1) // 2
    N = nr * (nr - 1) / 2.0
    t = np.radians(e)
    p = (np.cos(t[:-1]) - np.cos(t[1:])) / 2.0
    mean = N * p
    sigma = np.sqrt(N * p * (1.0 - p))
    z = (RR[1:-1].astype(np.float64) - mean) / sigma
    assert np.all(np.abs(z) <= 5.0), z
    # clustering: DD exceeds the random expectation at small separations
    assert DD[1] > 2 * mean[0] * (nd * (nd - 1) / 2.0) / N


def test_full_size_sampled_rows_against_oracle(W, wl):
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    rows = np.sort(np.random.default_rng(11).choice(wl.n_d, 400, replace=False))
    D = O.radec_to_xyz(wl.data.reshape(-1, 2)[rows].reshape(-1))
    R = O.radec_to_xyz(wl.rand)
    got = _count(W, D, R, e, False, xyz=True)
    want = O.count_xyz(D, R, e, False)
    assert np.array_equal(got, want)


def test_subsample_200k_against_oracle(W, wl):
    """DD, DR and RR of a seeded 200k + 200k subsample: P1 through
    wtheta_count_wtheta on the oracle's own unit vectors (library defaults:
    far tile pairs skipped, spans settled), every slot bit-identical; P2
    through wtheta_count from RA/Dec (the device converts; only pairs within
    a few ulps of an edge may move)."""
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    rng = np.random.default_rng(12)
    sd = np.sort(rng.choice(wl.n_d, 200_000, replace=False))
    sr = np.sort(rng.choice(wl.n_r, 200_000, replace=False))
    d = wl.data.reshape(-1, 2)[sd].reshape(-1)
    r = wl.rand.reshape(-1, 2)[sr].reshape(-1)
    D, R = O.radec_to_xyz(d), O.radec_to_xyz(r)
    K = wl.n_bins
    c = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
    W.wtheta_count_wtheta(torch.from_numpy(D).cuda(), torch.from_numpy(R).cuda(), True, e, c)
    torch.cuda.synchronize()
    p1 = c.cpu().numpy().astype(np.uint64)
    for k, (a, b, A, B, auto) in enumerate([(d, None, D, None, True), (d, r, D, R, False),
                                            (r, None, R, None, True)]):
        want = O.count_xyz(A, B, e, auto)
        assert np.array_equal(p1[k], want), k
        got = _count(W, a, b, e, auto)
        assert int(got.sum()) == int(want.sum())
        if np.array_equal(got, want):
            continue
        # P2: only pairs within a few ulps of an edge may move
        amb = O.count_ambiguous_xyz(A, B, e, auto)
        assert np.abs(got.astype(np.int64) - want.astype(np.int64)).sum() <= 2 * amb
