"""GPU counts against the CPU oracle, through the C ABI.

P1 (zero tolerance): wtheta_count_xyz is fed the oracle's own FP64 unit
vectors; counts must be bit-identical.
P2: wtheta_count converts RA/Dec on the device (CUDA sin/cos may differ from
the host's in the last place); counts must be bit-identical when the oracle
finds no pair within a few ulps of an edge, otherwise differ by at most that
many pairs.
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ARCMIN = 1.0 / 60.0
# every instantiated kernel shape: (threads, points per thread, B points per
# screening test, histogram mode, deferred binning)
SHAPES = [(128, 8, 2, 3, 2), (128, 8, 2, 3, 1), (128, 8, 2, 1, 2), (128, 8, 2, 2, 1),
          (128, 8, 1, 3, 2), (64, 16, 2, 3, 2), (64, 16, 2, 2, 1), (128, 16, 2, 3, 2),
          (256, 8, 2, 3, 2), (256, 8, 2, 2, 1), (64, 8, 2, 3, 1), (128, 8, 2, 4, 1),
          (64, 8, 2, 4, 1), (32, 8, 2, 3, 1)]
VARIANTS = [dict(threads=a, points_per_thread=b, j_per_screen=c, hist_mode=d, deferred=f)
            for a, b, c, d, f in SHAPES]


@pytest.fixture(scope="module")
def W():
    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta
    assert torch.cuda.is_available()
    return wtheta


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def gpu_count_xyz(W, A, B, e, is_auto, tune=None, stats=None):
    c = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
    a = dev(A)
    b = None if is_auto else dev(B)
    if tune is None and stats is None:
        W.wtheta_count_xyz(a, b, e, is_auto, c)
    else:
        W.wtheta_count_ex(a, b, True, e, is_auto, c, tune=tune, stats=stats)
    torch.cuda.synchronize()
    return c.cpu().numpy().astype(np.uint64)


def gpu_count(W, rd_a, rd_b, e, is_auto, tune=None, stats=None):
    c = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
    a = dev(rd_a)
    b = None if is_auto else dev(rd_b)
    if tune is None and stats is None:
        W.wtheta_count(a, b, e, is_auto, c)
    else:
        W.wtheta_count_ex(a, b, False, e, is_auto, c, tune=tune, stats=stats)
    torch.cuda.synchronize()
    return c.cpu().numpy().astype(np.uint64)


def test_radec_conversion_within_ulps(W):
    rng = np.random.default_rng(3)
    n = 200_000
    ra = np.concatenate([rng.uniform(-720, 720, n - 8), [0, 90, 180, 270, 359.999999, 360, -0.0, 1e-9]])
    dec = np.concatenate([rng.uniform(-90, 90, n - 8), [90, -90, 0, 45, -45, 89.9999999, -89.9999, 0]])
    rd = synth.interleave(ra, dec)
    want = O.radec_to_xyz(rd)
    x = torch.empty(3 * n, dtype=torch.float64, device="cuda")
    W.wtheta_radec_to_xyz(dev(rd), x)
    torch.cuda.synchronize()
    got = x.cpu().numpy().reshape(3, n)
    ulp = np.spacing(np.maximum(np.abs(want), 2.0 ** -60))
    assert np.max(np.abs(got - want) / ulp) <= 4.0


@pytest.mark.parametrize("tune", VARIANTS, ids=lambda t: "nt%d_r%d_j%d_h%d_d%d" % (
    t["threads"], t["points_per_thread"], t["j_per_screen"], t["hist_mode"], t["deferred"]))
def test_small_workload_bit_exact_p1(W, tune):
    """10k clustered + 10k random in a 10 deg patch, 16 log bins 1'-5 deg."""
    wl = synth.small()
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    D, R = O.radec_to_xyz(wl.data), O.radec_to_xyz(wl.rand)
    for A, B, auto in [(D, None, True), (D, R, False), (R, None, True)]:
        want = O.count_xyz(A, B, e, auto)
        got = gpu_count_xyz(W, A, B, e, auto, tune=tune)
        assert np.array_equal(got, want), (auto, got, want)


def test_small_workload_radec_p2_and_w(W):
    wl = synth.small()
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    D, R = O.radec_to_xyz(wl.data), O.radec_to_xyz(wl.rand)
    got = []
    for a, b, A, B, auto in [(wl.data, None, D, None, True), (wl.data, wl.rand, D, R, False),
                             (wl.rand, None, R, None, True)]:
        want = O.count_xyz(A, B, e, auto)
        amb = O.count_ambiguous_xyz(A, B, e, auto)
        g = gpu_count(W, a, b, e, auto)
        if amb == 0:
            assert np.array_equal(g, want)
        else:
            assert np.sum(np.abs(g.astype(np.int64) - want.astype(np.int64))) <= 2 * amb
        assert int(g.sum()) == int(want.sum())
        got.append(g)
    w = W.wtheta_ls(*got, wl.n_d, wl.n_r)
    DD, DR, RR, w_o = O.wtheta(wl.data, wl.rand, e)
    scale = np.maximum(np.abs(w_o), DD[1:-1] / RR[1:-1] + 2 * DR[1:-1] / RR[1:-1] + 1)
    assert np.all(np.abs(w - w_o) <= 1e-12 * scale)


SIZES = [0, 1, 2, 31, 33, 511, 512, 513, 1023, 1024, 1025, 2047, 2049, 4097]


@pytest.mark.parametrize("n", SIZES)
def test_ragged_sizes_bit_exact(W, n):
    fp = synth.Patch(10.0, 3.0, -5.0, -2.0)
    a = synth.clustered(fp, n, max(1, n // 40), 2.0, 5, "test", "data", n) if n else np.zeros(0)
    b = synth.uniform(fp, n + 7, 6, "test", "random", n)
    e = W.wtheta_edges(0.5 * ARCMIN, 2.0, 20)
    A = O.radec_to_xyz(a) if n else np.zeros((3, 0))
    B = O.radec_to_xyz(b)
    for tune in (VARIANTS[0], VARIANTS[1], VARIANTS[3], VARIANTS[5], VARIANTS[6], VARIANTS[8]):
        got = gpu_count_xyz(W, A, None, e, True, tune=tune)
        want = O.count_xyz(A, None, e, True)
        assert np.array_equal(got, want), ("auto", n, got, want)
        assert int(got.sum()) == n * (n - 1) // 2
        got = gpu_count_xyz(W, A, B, e, False, tune=tune)
        want = O.count_xyz(A, B, e, False)
        assert np.array_equal(got, want), ("cross", n, got, want)


def test_hand_placed_points(W):
    import oracle_pins
    rows = [l.split() for l in open(oracle_pins.GOLDEN + "/hand_placed.txt")
            if l.strip() and not l.startswith("#")]
    for name, (lo, hi, K, mode) in oracle_pins.GOLDEN_EDGES.items():
        e = W.wtheta_edges(lo, hi, K, mode)
        sel = [r for r in rows if r[0] == name]
        for r in sel:
            a = np.array([float(r[1]), float(r[2])])
            b = np.array([float(r[3]), float(r[4])])
            got = gpu_count(W, a, b, e, False)
            want = np.zeros(K + 2, np.uint64)
            want[oracle_pins._slot_by_angle(e, float(r[5]))] = 1
            assert np.array_equal(got, want), (name, r, got)


def test_coincident_points_and_linear_bins_from_zero(W):
    rng = np.random.default_rng(11)
    base = synth.uniform(synth.Patch(0, 20, 0, 20), 700, 9, "test", "random")
    dup = np.concatenate([base, base[: 2 * 300]])  # 300 exact duplicates
    e = W.wtheta_edges(0.0, 180.0, 12, W.BINS_LINEAR)
    A = O.radec_to_xyz(dup)
    got = gpu_count_xyz(W, A, None, e, True)
    want = O.count_xyz(A, None, e, True)
    assert np.array_equal(got, want)
    assert got[0] == 0  # e_0 = 0: nothing below the first edge
    del rng


def test_pathological_edges_take_recheck_path(W):
    """256 linear bins to 180 deg: squared-chord edges crowd together near 4,
    the screening table marks those buckets for FP64 recheck; still exact."""
    e = W.wtheta_edges(0.0, 180.0, 256, W.BINS_LINEAR)
    R = O.radec_to_xyz(synth.uniform(synth.FullSky(), 3000, 10, "test", "random"))
    stats = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
    got = gpu_count_xyz(W, R, None, e, True, tune=dict(hist_mode=2), stats=stats)
    want = O.count_xyz(R, None, e, True)
    assert np.array_equal(got, want)
    assert int(stats[W.STAT_RECHECK]) > 0


def test_pairs_straddling_every_edge(W):
    """Pairs placed at e_k (1 +- delta), delta down to 1e-12: the FP32 value
    is ambiguous and the FP64 recheck must reproduce the oracle exactly."""
    rng = np.random.default_rng(21)
    e = W.wtheta_edges(0.5 * ARCMIN, 20.0, 32)
    A_list, B_list = [], []
    for k in range(len(e)):
        for d in np.concatenate([-np.logspace(-12, -3, 40), np.logspace(-12, -3, 40), [0.0]]):
            th = math.radians(e[k] * (1 + d))
            a = rng.normal(size=3)
            a /= np.linalg.norm(a)
            t = rng.normal(size=3)
            t -= a * (a @ t)
            t /= np.linalg.norm(t)
            A_list.append(a)
            B_list.append(a * math.cos(th) + t * math.sin(th))
    A = np.ascontiguousarray(np.array(A_list).T)
    B = np.ascontiguousarray(np.array(B_list).T)
    # one pair per column: compare pair-by-pair through the cross count of
    # single points, batched as a diagonal: count all pairs, then the
    # aligned subset via separate calls would be slow; instead check the full
    # cross count (contains all aligned pairs) and the aligned pairs alone
    stats = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
    got = gpu_count_xyz(W, A, B, e, False, stats=stats)
    want = O.count_xyz(A, B, e, False)
    assert np.array_equal(got, want)
    assert int(stats[W.STAT_RECHECK]) > 0
    for i in range(0, A.shape[1], 97):
        g = gpu_count_xyz(W, A[:, i:i + 1], B[:, i:i + 1], e, False)
        w = O.count_xyz(A[:, i:i + 1], B[:, i:i + 1], e, False)
        assert np.array_equal(g, w), i


def test_cross_is_symmetric(W):
    wl = synth.small(n=5000)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    ab = gpu_count(W, wl.data, wl.rand, e, False)
    ba = gpu_count(W, wl.rand, wl.data, e, False)
    assert np.array_equal(ab, ba)


def test_device_error_word(W):
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    W.wtheta_get_error()  # clear
    bad = np.array([10.0, 20.0, np.nan, 5.0, 30.0, 40.0])
    gpu_count(W, bad, None, e, True)
    assert W.wtheta_get_error() & W.DERR_NONFINITE
    assert W.wtheta_get_error() == 0  # read clears
    bad = np.array([10.0, 95.0, 11.0, 20.0])
    gpu_count(W, bad, None, e, True)
    assert W.wtheta_get_error() & W.DERR_DEC_RANGE


def test_correlate_host_api(W):
    wl = synth.small(n=4000)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    counts, w = W.wtheta_correlate(wl.data, wl.rand, e)
    DD, DR, RR, w_o = O.wtheta(wl.data, wl.rand, e)
    D, R = O.radec_to_xyz(wl.data), O.radec_to_xyz(wl.rand)
    amb = (O.count_ambiguous_xyz(D, None, e, True) + O.count_ambiguous_xyz(D, R, e, False)
           + O.count_ambiguous_xyz(R, None, e, True))
    if amb == 0:
        assert np.array_equal(counts, np.stack([DD, DR, RR]))
        assert np.all(np.abs(w - w_o) <= 1e-12 * np.maximum(np.abs(w_o), 4.0))


def test_survey_workload_full_size(W):
    """1M clustered + 1M random in a 60 deg cap, 32 log bins 0.5'-20 deg, in
    the benchmark's launch configuration: exact totals, DR = RD, additivity
    DD(A) = DD(A1) + DD(A2) + DR(A1, A2), and a sampled block of rows against
    the oracle."""
    wl = synth.survey()
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    nd, nr = wl.n_d, wl.n_r
    DD = gpu_count(W, wl.data, None, e, True)
    DR = gpu_count(W, wl.data, wl.rand, e, False)
    RR = gpu_count(W, wl.rand, None, e, True)
    assert int(DD.sum()) == nd * (nd - 1) // 2
    assert int(RR.sum()) == nr * (nr - 1) // 2
    assert int(DR.sum()) == nd * nr
    RD = gpu_count(W, wl.rand, wl.data, e, False)
    assert np.array_equal(DR, RD)
    h = 2 * 400_003
    a1, a2 = wl.data[:h], wl.data[h:]
    parts = (gpu_count(W, a1, None, e, True).astype(np.int64)
             + gpu_count(W, a2, None, e, True).astype(np.int64)
             + gpu_count(W, a1, a2, e, False).astype(np.int64))
    assert np.array_equal(parts.astype(np.uint64), DD)
    # sampled rows against the oracle (P1: the oracle's own unit vectors)
    D = O.radec_to_xyz(wl.data)
    R = O.radec_to_xyz(wl.rand)
    rows = np.sort(np.random.default_rng(5).choice(nd, 1500, replace=False))
    As = np.ascontiguousarray(D[:, rows])
    got = gpu_count_xyz(W, As, R, e, False)
    want = O.count_xyz(As, R, e, False)
    assert np.array_equal(got, want)
    w = W.wtheta_ls(DD, DR, RR, nd, nr)
    assert np.all(np.isfinite(w))


@pytest.mark.parametrize("is_auto", [True, False])
def test_shards_sum_to_the_whole_count(W, is_auto):
    """wtheta_count_shard over 1..4 shards adds up to wtheta_count exactly."""
    wl = synth.small(n=20_000)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    a = dev(wl.data)
    b = None if is_auto else dev(wl.rand)
    whole = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
    W.wtheta_count(a, b, e, is_auto, whole)
    for S in (1, 2, 3, 4):
        acc = torch.zeros_like(whole)
        for s in range(S):
            c = torch.zeros_like(whole)
            W.wtheta_count_shard(a, b, e, is_auto, s, S, c)
            acc += c
        torch.cuda.synchronize()
        assert torch.equal(acc, whole), S


def test_wtheta_shards_sum_to_the_oracle_and_balance_work(W):
    """wtheta_count_wtheta_shard: every shard's 3 (K+2) counts are exact for
    the pairs of its tile columns (their slots sum to its pairs), the shards add
    up, slot by slot, to the oracle's whole DD, DR and RR (P1: the oracle's
    unit vectors), and shards of a clustered survey get similar numbers of
    kept tile pairs (the split's weights) -- Sec. 5's division of the data set
    over independent GPUs, one sum-reduction combining them."""
    wl = synth.survey(n=60_000)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    D, R = O.radec_to_xyz(wl.data), O.radec_to_xyz(wl.rand)
    want = [O.count_xyz(D, None, e, True), O.count_xyz(D, R, e, False),
            O.count_xyz(R, None, e, True)]
    d, r = dev(D), dev(R)
    K = wl.n_bins
    for S in (1, 2, 3, 5, 200):
        acc = np.zeros((3, K + 2), np.uint64)
        tiles = []
        for s in range(S):
            c = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
            st = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
            W.wtheta_count_wtheta_shard(d, r, True, e, s, S, c, stats=st)
            torch.cuda.synchronize()
            acc += c.cpu().numpy().astype(np.uint64)
            tiles.append(int(st.cpu().numpy()[W.STAT_TILES]))
        for k in range(3):
            assert np.array_equal(acc[k], want[k]), (S, k)
        if 1 < S <= 5:
            # equal work: each count's share is within one tile row's kept tile
            # pairs (at most a row's tiles, 512-point tiles here) of an even split
            row = -(-max(wl.n_d, wl.n_r) // 512)
            assert max(tiles) - min(tiles) <= 2 * 3 * row, (S, tiles)
            assert min(tiles) > 0.5 * sum(tiles) / S, (S, tiles)
    with pytest.raises(W.WthetaError):
        W.wtheta_count_wtheta_shard(d, r, True, e, 3, 3, torch.zeros((3, K + 2), dtype=torch.int64,
                                                                   device="cuda"))


@pytest.mark.parametrize("case", ["survey_200k", "fullsky_150k", "small"])
def test_skipping_far_tile_pairs_is_exact(W, case):
    """Counts with tile pairs skipped by their bounding caps equal counts with
    every tile pair evaluated, and pairs were in fact skipped."""
    if case == "survey_200k":
        wl = synth.survey(n=200_000)
    elif case == "fullsky_150k":
        wl = synth.largest(n=150_000)
    else:
        wl = synth.small()
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    d, r = dev(wl.data), dev(wl.rand)
    for a, b, auto in [(d, None, True), (d, r, False), (r, None, True)]:
        c_all = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
        c_skip = torch.zeros_like(c_all)
        st = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
        W.wtheta_count_ex(a, b, False, e, auto, c_all, tune=dict(skip_far=2))
        W.wtheta_count_ex(a, b, False, e, auto, c_skip, tune=dict(skip_far=1), stats=st)
        torch.cuda.synchronize()
        assert torch.equal(c_all, c_skip), (case, auto)
        if case != "small":
            assert int(st[W.STAT_SKIPPED]) > 0


@pytest.mark.parametrize("case", ["survey_200k", "fullsky_150k", "small", "patch_120k"])
def test_span_bins_are_exact(W, case):
    """Settling (A group, B chunk) spans in one slot or with one comparison
    per pair gives the same counts as binning every pair through the table,
    and it does settle pairs."""
    if case == "survey_200k":
        wl = synth.survey(n=200_000)
    elif case == "fullsky_150k":
        wl = synth.largest(n=150_000)
    elif case == "small":
        wl = synth.small()
    else:
        fp = synth.Patch(200.0, 15.0, 10.0, 25.0)
        wl = synth.Workload("patch", synth.clustered(fp, 120_000, 2400, 3.0, 5, "test", "data", 0),
                            synth.uniform(fp, 120_000, 5, "test", "random", 0),
                            1.0 * ARCMIN, 5.0, 16)
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    d, r = dev(wl.data), dev(wl.rand)
    for a, b, auto in [(d, None, True), (d, r, False), (r, None, True)]:
        c_pair = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
        c_span = torch.zeros_like(c_pair)
        st = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
        W.wtheta_count_ex(a, b, False, e, auto, c_pair, tune=dict(span_bins=2))
        W.wtheta_count_ex(a, b, False, e, auto, c_span, tune=dict(span_bins=1), stats=st)
        torch.cuda.synchronize()
        assert torch.equal(c_pair, c_span), (case, auto)
        st = st.cpu().numpy().astype(np.uint64)
        assert 0 < st[W.STAT_SPAN] <= st[W.STAT_PAIRS] + st[W.STAT_SPAN], case


def test_span_bins_near_an_edge(W):
    """Two compact clusters whose separation is one bin edge: every chunk span
    straddles that edge, many pairs fall inside its guard band, and the counts
    still equal the oracle's bit for bit (P1)."""
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    k = 10
    rng = np.random.default_rng(17)
    n = 3000
    ra = rng.uniform(-0.02, 0.02, n)
    dec = rng.uniform(-0.02, 0.02, n)
    A = synth.interleave(ra, dec)
    B = synth.interleave(ra + e[k], dec)          # the same points, e_k further in RA
    XA, XB = O.radec_to_xyz(A), O.radec_to_xyz(B)
    st = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
    got = gpu_count_xyz(W, XA, XB, e, False, tune=dict(span_bins=1), stats=st)
    want = O.count_xyz(XA, XB, e, False)
    assert np.array_equal(got, want)
    st = st.cpu().numpy()
    assert st[W.STAT_RECHECK] > 0 and st[W.STAT_SPAN] > 0
    both = np.concatenate([XA, XB], axis=1)
    got = gpu_count_xyz(W, both, None, e, True, tune=dict(span_bins=1))
    want = O.count_xyz(both, None, e, True)
    assert np.array_equal(got, want)


def test_span_bins_three_slots_near_two_edges(W):
    """Group-chunk spans that cover two edges (three slots), with many pairs
    inside both edges' guard bands: counts equal the oracle's bit for bit."""
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    k = 10
    rng = np.random.default_rng(23)
    n = 2500
    ra = rng.uniform(-0.05, 0.05, n)
    dec = rng.uniform(-0.05, 0.05, n)
    A = synth.interleave(ra, dec)
    mid = 0.5 * (e[k] + e[k + 1])
    B = np.concatenate([synth.interleave(ra + e[k], dec), synth.interleave(ra + e[k + 1], dec),
                        synth.interleave(rng.uniform(-0.05, 0.05, n) + mid,
                                         rng.uniform(-0.05, 0.05, n))])
    XA, XB = O.radec_to_xyz(A), O.radec_to_xyz(B)
    st = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
    got = gpu_count_xyz(W, XA, XB, e, False, tune=dict(span_bins=1), stats=st)
    want = O.count_xyz(XA, XB, e, False)
    assert np.array_equal(got, want)
    st = st.cpu().numpy()
    assert st[W.STAT_RECHECK] > 0 and st[W.STAT_SPAN] > 0
    off = gpu_count_xyz(W, XA, XB, e, False, tune=dict(span_bins=2))
    assert np.array_equal(off, want)


def test_shared_atomic_probe(W):
    """The measurement kernel returns a plausible rate: at most one warp-wide
    reduction per SM clock per SM sub-partition, and fewer to one word."""
    own = W.wtheta_probe_shared_atomics(False)
    one = W.wtheta_probe_shared_atomics(True)
    assert 0.01 < own <= 4.0
    assert 0.0 < one <= own


@pytest.mark.parametrize("case", ["small", "survey_200k", "tiny", "empty_rand"])
def test_count_wtheta_equals_three_counts(W, case):
    """DD, DR, RR in one launch (each catalogue prepared once) equal the three
    single counts, slot for slot, and the statistics add up."""
    if case == "small":
        wl = synth.small()
        d, r = wl.data, wl.rand
    elif case == "survey_200k":
        wl = synth.survey(n=200_000)
        d, r = wl.data, wl.rand
    elif case == "tiny":
        wl = synth.small(n=1500)
        d, r = wl.data[:14], wl.rand[:2 * 1100]   # 7 data points, 1100 randoms
    else:
        wl = synth.small(n=1500)
        d, r = wl.data, wl.rand[:0]
    e = W.wtheta_edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    K = len(e) - 1
    dd, rr = dev(d), dev(r)
    one = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
    st1 = torch.zeros(W.NSTATS, dtype=torch.int64, device="cuda")
    W.wtheta_count_wtheta(dd, rr, False, e, one, stats=st1)
    three = torch.zeros_like(one)
    st3 = torch.zeros_like(st1)
    for q, (a, b, auto) in enumerate([(dd, None, True), (dd, rr, False), (rr, None, True)]):
        W.wtheta_count_ex(a, b, False, e, auto, three[q], stats=st3)
    torch.cuda.synchronize()
    assert torch.equal(one, three), case
    s1, s3 = st1.cpu().numpy(), st3.cpu().numpy()
    assert s1[W.STAT_TILES] == s3[W.STAT_TILES] and s1[W.STAT_SKIPPED] == s3[W.STAT_SKIPPED]
    if case == "small":
        want = O.wtheta(d, r, e)[:3]
        got = one.cpu().numpy().astype(np.uint64)
        for k in range(3):
            assert int(got[k].sum()) == int(want[k].sum())


def _random_case(seed):
    """A random catalogue pair, footprint and edge set (seeded)."""
    rng = np.random.default_rng(1000 + seed)
    kind = seed % 4
    if kind == 0:
        w = float(rng.uniform(0.5, 20.0))
        ra0, dec0 = float(rng.uniform(0, 360)), float(rng.uniform(-80, 80 - w))
        fp = synth.Patch(ra0, w, dec0, dec0 + w)
    elif kind == 1:
        fp = synth.Cap(float(rng.uniform(1.0, 90.0)))
    elif kind == 2:
        fp = synth.FullSky()
    else:
        w = float(rng.uniform(0.05, 1.0))  # very compact: many pairs in the small bins
        fp = synth.Patch(float(rng.uniform(0, 360)), w, -w / 2, w / 2)
    nd = int(rng.integers(300, 6000))
    nr = int(rng.integers(300, 6000))
    d = synth.clustered(fp, nd, max(1, nd // int(rng.integers(5, 80))),
                        float(rng.uniform(0.2, 6.0)), seed, "test", "data", seed)
    r = synth.uniform(fp, nr, seed, "test", "random", seed)
    K = int(rng.choice([1, 2, 5, 16, 33, 64, 200]))
    mode = int(rng.integers(0, 3))
    hi = float(rng.choice([0.1, 1.0, 5.0, 30.0, 90.0, 179.0, 180.0]))
    lo = 0.0 if mode == 0 and rng.random() < 0.5 else hi * float(10 ** rng.uniform(-4, -0.5))
    if mode != 0 and lo == 0.0:
        lo = hi * 1e-3
    return d, r, lo, hi, K, mode


@pytest.mark.parametrize("seed", range(24))
def test_random_configurations_bit_exact(W, seed):
    """Random footprints (patches, caps, full sky, sub-degree patches), sizes,
    clustering and edge sets (1 to 200 bins, linear or logarithmic, top edge
    up to 180 deg): DD, DR, RR through the single-launch call, with far tile
    pairs skipped and spans settled, equal the oracle bit for bit (P1)."""
    d, r, lo, hi, K, mode = _random_case(seed)
    e = W.wtheta_edges(lo, hi, K, mode)
    XD, XR = O.radec_to_xyz(d), O.radec_to_xyz(r)
    c = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
    # odd seeds: the 1024-point tiles (the default for these sizes is 512)
    tune = dict(threads=128, points_per_thread=8) if seed % 2 else None
    W.wtheta_count_wtheta(dev(XD), dev(XR), True, e, c, tune=tune)
    torch.cuda.synchronize()
    got = c.cpu().numpy().astype(np.uint64)
    assert np.array_equal(got[0], O.count_xyz(XD, None, e, True)), (seed, lo, hi, K, mode)
    assert np.array_equal(got[1], O.count_xyz(XD, XR, e, False)), (seed, lo, hi, K, mode)
    assert np.array_equal(got[2], O.count_xyz(XR, None, e, True)), (seed, lo, hi, K, mode)
