"""Batched counts (one work queue, one graph replay) against the single-count
entry point and the oracle."""
import numpy as np
import pytest

from oracle import oracle as O
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


def _mocks(n_mocks, lo, hi, seed):
    rng = np.random.default_rng(seed)
    out = []
    for m in range(n_mocks):
        n = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        ra0, dec0 = rng.uniform(0, 360), rng.uniform(-60, 45)
        fp = synth.Patch(ra0, 6.0, dec0, dec0 + 6.0)
        d = synth.clustered(fp, n, max(1, n // 50), 3.0, seed, "test", "data", m)
        r = synth.uniform(fp, 2 * n + 3, seed, "test", "random", m)
        out.append((d, r))
    return out


def _single(W, d, r, e):
    K = len(e) - 1
    c = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
    dd, rr = torch.from_numpy(d).cuda(), torch.from_numpy(r).cuda()
    W.wtheta_count(dd, None, e, True, c[0])
    W.wtheta_count(dd, rr, e, False, c[1])
    W.wtheta_count(rr, None, e, True, c[2])
    torch.cuda.synchronize()
    return c.cpu().numpy().astype(np.uint64)


def test_batch_equals_single_counts_and_replays(W):
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    mocks = _mocks(9, 800, 9000, 31)
    dev = [(torch.from_numpy(d).cuda(), torch.from_numpy(r).cuda()) for d, r in mocks]
    plan = W.wtheta_batch_plan(dev, e)
    info = W.wtheta_batch_info(plan)
    assert info["autotuned"] and info["n_counts"] == 27
    K = len(e) - 1
    out = torch.zeros((len(mocks), 3, K + 2), dtype=torch.int64, device="cuda")
    W.wtheta_batch_run(plan, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.uint64)
    for m, (d, r) in enumerate(mocks):
        want = _single(W, d, r, e)
        assert np.array_equal(got[m], want), m
        nd, nr = len(d) // 2, len(r) // 2
        assert int(got[m, 0].sum()) == nd * (nd - 1) // 2
        assert int(got[m, 1].sum()) == nd * nr
        assert int(got[m, 2].sum()) == nr * (nr - 1) // 2
    # replay: identical
    out2 = torch.zeros_like(out)
    W.wtheta_batch_run(plan, out2)
    torch.cuda.synchronize()
    assert torch.equal(out, out2)
    # the graph re-reads the catalogues: change one in place, rerun
    d0, r0 = dev[0]
    d0[1::2] += 0.01  # shift Dec of mock 0 by 0.01 deg
    W.wtheta_batch_run(plan, out2)
    torch.cuda.synchronize()
    got2 = out2.cpu().numpy().astype(np.uint64)
    want0 = _single(W, d0.cpu().numpy(), r0.cpu().numpy(), e)
    assert np.array_equal(got2[0], want0)
    assert np.array_equal(got2[1:], got[1:])
    W.wtheta_batch_free(plan)


def test_batch_against_oracle(W):
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    mocks = _mocks(3, 1500, 4000, 32)
    dev = [(torch.from_numpy(d).cuda(), torch.from_numpy(r).cuda()) for d, r in mocks]
    plan = W.wtheta_batch_plan(dev, e, tune=dict(threads=128, points_per_thread=8, hist_mode=2))
    K = len(e) - 1
    out = torch.zeros((len(mocks), 3, K + 2), dtype=torch.int64, device="cuda")
    W.wtheta_batch_run(plan, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.uint64)
    for m, (d, r) in enumerate(mocks):
        D, R = O.radec_to_xyz(d), O.radec_to_xyz(r)
        for k, (A, B, auto) in enumerate([(D, None, True), (D, R, False), (R, None, True)]):
            want = O.count_xyz(A, B, e, auto)
            amb = O.count_ambiguous_xyz(A, B, e, auto)
            if amb == 0:
                assert np.array_equal(got[m, k], want), (m, k)
            else:
                assert np.abs(got[m, k].astype(np.int64) - want.astype(np.int64)).sum() <= 2 * amb


@pytest.mark.parametrize("tune", [dict(threads=128, points_per_thread=8, hist_mode=3, deferred=2),
                                  dict(threads=256, points_per_thread=8, hist_mode=2),
                                  dict(threads=64, points_per_thread=16, hist_mode=3, deferred=2)])
def test_batch_shapes_agree(W, tune):
    e = W.wtheta_edges(0.5 * ARCMIN, 3.0, 24)
    mocks = _mocks(5, 500, 6000, 33)
    dev = [(torch.from_numpy(d).cuda(), torch.from_numpy(r).cuda()) for d, r in mocks]
    K = len(e) - 1
    ref = W.wtheta_batch_plan(dev, e, tune=dict(threads=128, points_per_thread=8))
    a = torch.zeros((len(mocks), 3, K + 2), dtype=torch.int64, device="cuda")
    W.wtheta_batch_run(ref, a)
    plan = W.wtheta_batch_plan(dev, e, tune=tune)
    b = torch.zeros_like(a)
    W.wtheta_batch_run(plan, b)
    torch.cuda.synchronize()
    assert torch.equal(a, b)


def test_batch_beyond_2_to_the_24_points(W):
    """Catalogues that start more than 2^24 points into the plan's shared
    arrays (their padding sentinels must stay distinct in FP32) count exactly:
    the last mocks of a plan holding ~19M points equal the oracle."""
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    K = len(e) - 1
    rng = np.random.default_rng(35)
    fill = []
    for m in range(62):  # 62 x 300k uniform points ahead of the checked mocks
        ra0, dec0 = rng.uniform(0, 360), rng.uniform(-60, 45)
        fp = synth.Patch(ra0, 15.0, dec0, dec0 + 15.0)
        fill.append((synth.uniform(fp, 150_001 + m, 35, "test", "data", m),
                     synth.uniform(fp, 149_999, 35, "test", "random", m)))
    tail = _mocks(2, 3000, 9000, 36)
    mocks = fill + tail
    dev = [(torch.from_numpy(d).cuda(), torch.from_numpy(r).cuda()) for d, r in mocks]
    assert sum(len(d) + len(r) for d, r in mocks) // 2 > (1 << 24)
    plan = W.wtheta_batch_plan(dev, e, tune=dict(threads=128, points_per_thread=8))
    out = torch.zeros((len(mocks), 3, K + 2), dtype=torch.int64, device="cuda")
    W.wtheta_batch_run(plan, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.uint64)
    W.wtheta_batch_free(plan)
    for i, (d, r) in enumerate(tail):
        D, R = O.radec_to_xyz(d), O.radec_to_xyz(r)
        for k, (A, B, auto) in enumerate([(D, None, True), (D, R, False), (R, None, True)]):
            want = O.count_xyz(A, B, e, auto)
            amb = O.count_ambiguous_xyz(A, B, e, auto)
            g = got[len(fill) + i, k]
            assert int(g.sum()) == int(want.sum())
            if amb == 0:
                assert np.array_equal(g, want), (i, k)
            else:
                assert np.abs(g.astype(np.int64) - want.astype(np.int64)).sum() <= 2 * amb
