"""The C-ABI library on the CPU: it loads, exports every declared symbol, and
its host-side arithmetic (edges, squared-chord edges, estimators, argument
validation, guard band) agrees with the oracle and with the FP32 error bound.
No kernel is launched here."""
import ctypes

import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth
from paper_1208_3658_gb300 import wtheta as W

ARCMIN = 1.0 / 60.0
EDGE_SETS = [
    (1.0 * ARCMIN, 5.0, 16, W.BINS_LN),
    (0.5 * ARCMIN, 20.0, 32, W.BINS_LN),
    (1.0 * ARCMIN, 10.0, 24, W.BINS_LOG10),
    (0.2 * ARCMIN, 30.0, 64, W.BINS_LN),
    (0.0, 180.0, 12, W.BINS_LINEAR),
    (0.0, 180.0, 256, W.BINS_LINEAR),
    (1e-4, 179.0, 200, W.BINS_LN),
]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1208_3658_gb300 import build
    build.build()


def test_exports_every_declared_symbol():
    L = W.lib()
    names = W.declared_functions()
    assert len(names) >= 12
    for n in names:
        assert hasattr(L, n), n


@pytest.mark.parametrize("lo,hi,K,mode", EDGE_SETS)
def test_edges_and_chords_bit_equal_to_oracle(lo, hi, K, mode):
    e = W.wtheta_edges(lo, hi, K, mode)
    assert np.array_equal(e, O.edges(lo, hi, K, mode))
    assert np.array_equal(W.wtheta_chord2_edges(e), O.chord2(e))


def test_ls_matches_oracle():
    wl = synth.small(n=1500)
    e = O.edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    DD, DR, RR, w_o = O.wtheta(wl.data, wl.rand, e)
    w = W.wtheta_ls(DD, DR, RR, wl.n_d, wl.n_r)
    scale = np.maximum(np.abs(w_o), DD[1:-1] / RR[1:-1] + 2 * DR[1:-1] / RR[1:-1] + 1)
    ok = RR[1:-1] > 0
    assert np.all(np.abs(w - w_o)[ok] <= 1e-12 * scale[ok])
    wc = W.wtheta_ls_cross(DD, DR, DR, RR, 10, 20, 30, 40)
    wco = O.ls_cross(DD, DR, DR, RR, 10, 20, 30, 40)
    assert np.allclose(wc[ok], wco[ok], rtol=1e-12, atol=0)


def test_ls_empty_random_bins_give_nan():
    """Eq. 2 divides by the bin's random pairs: where RR_k (or R1R2_k) is 0
    the estimate is NaN, whatever DD and DR hold; elsewhere it is the value
    worked out by hand (n_d = n_r = 3: totals 3, 9, 3)."""
    u = lambda *v: np.array((0,) + v + (0,), np.uint64)  # noqa: E731
    w = W.wtheta_ls(u(3, 0, 0, 3, 0), u(0, 9, 0, 9, 5), u(3, 3, 0, 0, 0), 3, 3)
    assert w[0] == 2.0 and w[1] == -1.0
    assert np.all(np.isnan(w[2:])), w
    w = W.wtheta_ls_cross(u(4, 0, 0, 4), u(0, 4, 0, 0), u(0, 4, 0, 0), u(4, 4, 0, 0), 2, 2, 2, 2)
    assert w[0] == 2.0 and w[1] == -1.0
    assert np.all(np.isnan(w[2:])), w


def test_noalloc_rejects_huge_sizes_before_any_device_work():
    """Sizes past the fixed scratch's limit return WTHETA_ESIZE before any
    rounding that could overflow, and before any CUDA call (so this runs
    without a GPU): n near INT64_MAX would otherwise wrap when rounded up to
    a whole tile."""
    L = W.lib()
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    ep = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    c = ctypes.c_void_p(256)
    ESIZE = -7
    big = 2 ** 63 - 1
    for na, nb, auto in [(big, big, 1), (big - 100, 0, 0), (5, big, 0), (big, 5, 0),
                         (W.NOALLOC_MAX_POINTS + 1, 0, 1), (W.NOALLOC_MAX_POINTS, 1, 0)]:
        b = None if auto else c
        nb_ = na if auto else nb
        assert L.wtheta_count_xyz_noalloc(c, na, b, nb_, ep, 16, auto, c, None) == ESIZE, (na, nb)


def test_ls_closed_form_d_equals_r():
    """Counts with R = D give w = 2/n (derivation in oracle_pins)."""
    n = 500
    D = synth.clustered(synth.Patch(0, 5, 0, 5), n, 10, 3.0, 2, "test", "data")
    e = O.edges(1.0 * ARCMIN, 5.0, 16)
    DD = O.count(D, None, e, True)
    DR = O.count(D, D, e, False)
    w = W.wtheta_ls(DD, DR, DD, n, n)
    nz = DD[1:-1] > 0
    assert np.all(np.abs(w[nz] - 2.0 / n) <= 3e-12)


def test_argument_validation_needs_no_gpu():
    L = W.lib()
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    dp = ctypes.POINTER(ctypes.c_double)
    ep = e.ctypes.data_as(dp)
    EINVAL = -1
    # bad edge arrays
    for bad in ([1.0, 1.0], [2.0, 1.0], [-1.0, 1.0], [1.0, 181.0], [0.0, np.nan]):
        b = np.array(bad, np.float64)
        assert L.wtheta_chord2_edges(b.ctypes.data_as(dp), 1, b.ctypes.data_as(dp)) == EINVAL
    assert L.wtheta_edges(1.0, 0.5, 4, 1, ep) == EINVAL
    assert L.wtheta_edges(0.0, 5.0, 4, 1, ep) == EINVAL       # log bins need lo > 0
    assert L.wtheta_edges(1.0, 5.0, 0, 1, ep) == EINVAL
    assert L.wtheta_edges(1.0, 5.0, 257, 0, np.empty(258).ctypes.data_as(dp)) == EINVAL
    # counting: bad sizes and pointers are rejected before any device work
    c = ctypes.c_void_p(16)
    assert L.wtheta_count(None, 5, None, 0, ep, 16, 1, c, None) == EINVAL       # null a, n > 0
    assert L.wtheta_count(c, 5, None, 0, ep, 16, 1, None, None) == EINVAL       # null counts
    assert L.wtheta_count(c, -1, None, 0, ep, 16, 1, c, None) == EINVAL
    assert L.wtheta_count(c, 5, c, 4, ep, 16, 1, c, None) == EINVAL             # auto, n_b != n_a
    assert L.wtheta_count(c, 5, None, 3, ep, 16, 0, c, None) == EINVAL          # cross, null b
    assert L.wtheta_count(c, 5, c, 5, ep, 16, 2, c, None) == EINVAL             # is_auto not 0/1
    assert L.wtheta_count(c, 5, c, 5, ep, 0, 0, c, None) == EINVAL              # K = 0
    u = np.zeros(18, np.uint64).ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
    w = np.zeros(16).ctypes.data_as(dp)
    assert L.wtheta_ls(u, u, u, 1, 5, 16, w) == EINVAL                          # n_d < 2
    assert W.wtheta_strerror(EINVAL) == "invalid argument"


def _emulate_s32(A, B):
    """The kernel's FP32 squared chord: d = fl32(a) - fl32(b) in FP32,
    s = fma(dz, dz, fma(dy, dy, dx*dx)).  Each fma is emulated as an exact FP64
    sum (d^2 is exact in FP64) rounded to FP32; where that FP64 sum itself
    rounds, the emulation can differ from a true fma by one FP32 ulp, which the
    bound's factor-2 margin covers."""
    a = A.astype(np.float32)
    b = B.astype(np.float32)
    d = a - b
    p = d[0] * d[0]
    q = (d[1].astype(np.float64) ** 2 + p.astype(np.float64)).astype(np.float32)
    return (d[2].astype(np.float64) ** 2 + q.astype(np.float64)).astype(np.float32)


def _s64(A, B):
    d = A - B
    return ((d[0] * d[0]) + (d[1] * d[1])) + (d[2] * d[2])


def _pairs_at(theta_deg, rng):
    """Unit-vector pairs (FP64) at angular separation theta (radians from deg)."""
    n = len(theta_deg)
    a = rng.normal(size=(3, n))
    a /= np.linalg.norm(a, axis=0)
    t = rng.normal(size=(3, n))
    t -= a * np.sum(a * t, axis=0)
    t /= np.linalg.norm(t, axis=0)
    th = np.radians(theta_deg)
    b = a * np.cos(th) + t * np.sin(th)
    return a, b


@pytest.mark.parametrize("lo,hi,K,mode", EDGE_SETS)
def test_guard_band_classification_is_sound(lo, hi, K, mode):
    """For pairs near every edge (relative offsets 1e-12..1e-2 either side) and
    at random separations: an FP32 value below the band is below the FP64 edge,
    one above the band at or above it.  No pair is misclassified."""
    rng = np.random.default_rng(12345 + K)
    e = W.wtheta_edges(lo, hi, K, mode)
    c = W.wtheta_chord2_edges(e)
    lo_b, hi_b, g = W.wtheta_guard_band(e)
    assert np.all(g > 0) and np.all(lo_b <= hi_b)
    n_in_band = 0
    total = 0
    for k in range(K + 1):
        if e[k] == 0.0:
            continue
        rel = np.concatenate([-np.logspace(-12, -2, 600), np.logspace(-12, -2, 600)])
        theta = np.clip(e[k] * (1 + rel), 1e-9, 180.0)
        A, B = _pairs_at(theta, rng)
        s32 = _emulate_s32(A, B)
        s64 = _s64(A, B)
        bits = s32.view(np.uint32)
        below = bits < lo_b[k]
        above = bits > hi_b[k]
        assert np.all(s64[below] < c[k]), (k, np.nonzero(s64[below] >= c[k]))
        assert np.all(s64[above] >= c[k]), (k, np.nonzero(s64[above] < c[k]))
        n_in_band += int(np.sum(~below & ~above))
        total += len(theta)
    assert n_in_band < total  # the band is narrow: most offsets >= 1e-5 resolve in FP32


@pytest.mark.parametrize("lo,hi,K,mode", EDGE_SETS)
def test_value_in_a_band_lies_between_the_neighbouring_edges(lo, hi, K, mode):
    """The premise of the recheck's hint: an FP32 value inside edge k's guard
    band has its FP64 squared chord in slot k or k+1, c[k-1] <= s64 < c[k+1]
    (so the FP64 recheck compares with at most three edges)."""
    rng = np.random.default_rng(777 + K)
    e = W.wtheta_edges(lo, hi, K, mode)
    c = W.wtheta_chord2_edges(e)
    lo_b, hi_b, _ = W.wtheta_guard_band(e)
    n_in = 0
    for k in range(K + 1):
        if e[k] == 0.0:
            continue
        rel = np.concatenate([-np.logspace(-12, -4, 400), np.logspace(-12, -4, 400)])
        theta = np.clip(e[k] * (1 + rel), 1e-9, 180.0)
        A, B = _pairs_at(theta, rng)
        s32 = _emulate_s32(A, B)
        s64 = _s64(A, B)
        bits = s32.view(np.uint32)
        inside = (bits >= lo_b[k]) & (bits <= hi_b[k])
        below_edge = -np.inf if k == 0 else c[k - 1]
        above_edge = np.inf if k == K else c[k + 1]
        assert np.all(s64[inside] >= below_edge), k
        assert np.all(s64[inside] < above_edge), k
        n_in += int(inside.sum())
    assert n_in > 0


def test_fp32_error_bound_random_pairs():
    """|s32 - s64| <= g(c)/2 whenever c <= s64 <= 2c, over pairs at all
    scales (the half-width doubles the bound E(s), evaluated at 2c)."""
    rng = np.random.default_rng(7)
    theta = 10 ** rng.uniform(-5, np.log10(180.0), 400_000)
    A, B = _pairs_at(theta, rng)
    s32 = _emulate_s32(A, B).astype(np.float64)
    s64 = _s64(A, B)
    # edges at each pair's own separation scale, c = s64 / 1.5 (so c <= s <= 2c)
    e = np.sort(np.degrees(2 * np.arcsin(np.sqrt(s64 / 1.5) / 2)))
    e = np.unique(e[(e > 0) & (e < 180)])
    idx = np.linspace(0, len(e) - 1, 200).astype(int)
    sub = np.unique(e[idx])
    _, _, g = W.wtheta_guard_band(sub)
    cs = W.wtheta_chord2_edges(sub)
    # each pair: use the edge just below s64/1.5 ... 2c range
    j = np.searchsorted(cs, s64 / 2, side="left")
    ok = (j < len(cs)) & (cs[np.minimum(j, len(cs) - 1)] <= s64)
    jj = np.minimum(j, len(cs) - 1)[ok]
    err = np.abs(s32 - s64)[ok]
    assert ok.sum() > 100_000
    assert np.all(err <= g[jj] / 2), np.max(err / (g[jj] / 2))


def test_batch_plan_validation_needs_no_gpu():
    L = W.lib()
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    ep = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    cats = (W.wtheta_catalog_pair * 2)()
    cats[0] = W.wtheta_catalog_pair(16, 100, 32, 200)
    cats[1] = W.wtheta_catalog_pair(16, 1, 32, 200)      # fewer than 2 data points
    assert L.wtheta_batch_plan(cats, 2, ep, 16, None, None, ctypes.byref(h)) == -1
    assert L.wtheta_batch_plan(cats, 0, ep, 16, None, None, ctypes.byref(h)) == -1
    cats[1] = W.wtheta_catalog_pair(None, 100, 32, 200)   # null data pointer
    assert L.wtheta_batch_plan(cats, 2, ep, 16, None, None, ctypes.byref(h)) == -1
    assert L.wtheta_batch_run(None, None, None) == -1
    assert L.wtheta_batch_free(None) == -1


def test_server_validation_needs_no_gpu():
    L = W.lib()
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    ep = e.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    h = ctypes.c_void_p()
    assert L.wtheta_server_create(ep, 16, 0, 0, None, ctypes.byref(h)) == -1   # zero budget
    assert L.wtheta_server_create(ep, 16, 1 << 30, -1, None, ctypes.byref(h)) == -1
    assert L.wtheta_server_submit(None, None, None) == -1
    assert L.wtheta_server_destroy(None) == -1
    d = ctypes.c_int32()
    assert L.wtheta_server_wait(None, 1, 0, ctypes.byref(d), None, None) == -1


@pytest.mark.parametrize("est,name", [(W.EST_LANDY_SZALAY, "landy_szalay"),
                                      (W.EST_NATURAL, "natural"),
                                      (W.EST_DAVIS_PEEBLES, "davis_peebles"),
                                      (W.EST_HAMILTON, "hamilton")])
def test_estimators_match_oracle(est, name):
    wl = synth.small(n=1200)
    e = O.edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    DD, DR, RR, _ = O.wtheta(wl.data, wl.rand, e)
    DR = DR.copy()
    DR[3] = 0                      # an empty denominator bin for two of them
    got = W.wtheta_estimate(DD, DR, RR, wl.n_d, wl.n_r, est)
    want = O.estimator(DD, DR, RR, wl.n_d, wl.n_r, name)
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.all(np.abs(got[ok] - want[ok]) <= 1e-13 * np.maximum(np.abs(want[ok]), 1.0))
    if est == W.EST_LANDY_SZALAY:
        assert np.array_equal(got, W.wtheta_ls(DD, DR, RR, wl.n_d, wl.n_r), equal_nan=True)
    with pytest.raises(W.WthetaError):
        W.wtheta_estimate(DD, DR, RR, wl.n_d, wl.n_r, 4)


def test_jackknife_matches_oracle():
    """wtheta_jackknife on the oracle's region-pair counts equals the oracle's
    jackknife (which sums the kept region pairs directly)."""
    fp = synth.Patch(120.0, 8.0, 20.0, 28.0)
    D = synth.clustered(fp, 900, 18, 3.0, 6, "test", "data")
    Rn = synth.uniform(fp, 1100, 6, "test", "random")
    e = O.edges(1.0 * ARCMIN, 4.0, 12)
    R = 8
    ld = synth.grid_labels(D, 120.0, 128.0, 20.0, 28.0, 4, 2)
    lr = synth.grid_labels(Rn, 120.0, 128.0, 20.0, 28.0, 4, 2)
    c = O.count_regions(O.radec_to_xyz(D), ld, O.radec_to_xyz(Rn), lr, e, R)
    sizes = np.concatenate([np.bincount(ld, minlength=R), np.bincount(lr, minlength=R)])
    w, w_k, cov = W.wtheta_jackknife(c, sizes, R)
    w_o, w_ko, cov_o = O.jackknife(c, sizes, R)
    scale = np.maximum(np.abs(w_o), 1.0)
    ok = np.isfinite(w_o)
    assert np.all(np.abs(w - w_o)[ok] <= 1e-12 * scale[ok])
    okk = np.isfinite(w_ko)
    assert np.array_equal(np.isfinite(w_k), okk)
    assert np.all(np.abs(w_k - w_ko)[okk] <= 1e-12 * np.maximum(np.abs(w_ko[okk]), 1.0))
    cols = np.all(okk, axis=0)
    m = np.ix_(cols, cols)
    assert np.allclose(cov[m], cov_o[m], rtol=1e-9, atol=1e-18)
    with pytest.raises(W.WthetaError):
        W.wtheta_jackknife(c[:, :1, :1], sizes[[0, R]], 1)


def _emulate_fused_d(A, B, mid):
    """The two-slot chunk's d = fma(dz, dz, fma(dy, dy, fma(dx, dx, -mid))),
    each fma emulated as an FP64 sum rounded to FP32 (dx^2 is exact in FP64;
    where the FP64 sum itself rounds, the emulation can differ from a true fma
    by one FP32 ulp, which the band's factor-2 margin covers)."""
    a = A.astype(np.float32)
    b = B.astype(np.float32)
    d = a - b
    f64 = np.float64
    x1 = (d[0].astype(f64) ** 2 - f64(mid)).astype(np.float32)
    x2 = (d[1].astype(f64) ** 2 + x1.astype(f64)).astype(np.float32)
    return (d[2].astype(f64) ** 2 + x2.astype(f64)).astype(np.float32)


@pytest.mark.parametrize("lo,hi,K,mode", EDGE_SETS)
def test_fused_edge_difference_classifies_exactly(lo, hi, K, mode):
    """The two-slot chunks compare d = s - mid, with the subtraction fused
    into the squared chord; outside |d| <= G (G the half-width of the edge's
    guard band about its middle mid) the sign of d must give the side of the
    FP64 squared chord, for pairs placed around every edge."""
    rng = np.random.default_rng(999 + K)
    e = W.wtheta_edges(lo, hi, K, mode)
    c = W.wtheta_chord2_edges(e)
    lo_b, hi_b, _ = W.wtheta_guard_band(e)
    decided = 0
    for k in range(K + 1):
        if e[k] == 0.0:
            continue
        lo_f = np.array([lo_b[k]], np.uint32).view(np.float32)[0]
        hi_f = np.array([hi_b[k]], np.uint32).view(np.float32)[0]
        mid = np.float32(np.float32(0.5) * (lo_f + hi_f))
        G = max(np.float32(mid - lo_f), np.float32(hi_f - mid))
        rel = np.concatenate([-np.logspace(-12, -1, 500), np.logspace(-12, -1, 500)])
        theta = np.clip(e[k] * (1 + rel), 1e-9, 180.0)
        A, B = _pairs_at(theta, rng)
        d = _emulate_fused_d(A, B, mid)
        s64 = _s64(A, B)
        out = np.abs(d) > G
        assert np.all((d[out] > 0) == (s64[out] >= c[k])), k
        decided += int(out.sum())
    assert decided > 0


@pytest.mark.parametrize("lo,hi,K,mode", EDGE_SETS)
def test_three_slot_difference_classifies_exactly(lo, hi, K, mode):
    """The three-slot jobs compute s as the pair-by-pair path does and then
    d = fl32(s - mid) for each of their two edges; outside |d| <= G the sign of
    d must give the side of the FP64 squared chord, for pairs placed around
    every edge, and for one edge evaluated beside its neighbour."""
    rng = np.random.default_rng(4242 + K)
    e = W.wtheta_edges(lo, hi, K, mode)
    c = W.wtheta_chord2_edges(e)
    lo_b, hi_b, _ = W.wtheta_guard_band(e)
    decided = 0
    for k in range(K + 1):
        if e[k] == 0.0:
            continue
        rel = np.concatenate([-np.logspace(-12, -1, 500), np.logspace(-12, -1, 500)])
        theta = np.clip(e[k] * (1 + rel), 1e-9, 180.0)
        A, B = _pairs_at(theta, rng)
        s32 = _emulate_s32(A, B)
        s64 = _s64(A, B)
        for q in (k, k + 1):  # this edge, and the next one seen from these pairs
            if q > K or e[q] == 0.0:
                continue
            lo_f = np.array([lo_b[q]], np.uint32).view(np.float32)[0]
            hi_f = np.array([hi_b[q]], np.uint32).view(np.float32)[0]
            mid = np.float32(np.float32(0.5) * (lo_f + hi_f))
            G = max(np.float32(mid - lo_f), np.float32(hi_f - mid))
            d = (s32 - mid).astype(np.float32)
            out = np.abs(d) > G
            assert np.all((d[out] > 0) == (s64[out] >= c[q])), (k, q)
            decided += int(out.sum())
    assert decided > 0


def test_binding_refuses_misshapen_coordinates_and_short_outputs():
    """The binding passes the library plain pointers and point counts, so it
    checks layouts itself: unit vectors are read as SoA with stride n (a
    row-major (n, 3) array would give wrong counts), RA/Dec as interleaved
    pairs, and the count buffers must hold every slot the library writes.
    Accepted layouts get as far as the device check (there is no GPU here)."""
    torch = pytest.importorskip("torch")
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    f64 = torch.float64
    soa = torch.zeros((3, 100), dtype=f64)
    rd = torch.zeros(200, dtype=f64)
    c = torch.zeros(18, dtype=torch.int64)
    c3 = torch.zeros((3, 18), dtype=torch.int64)
    with pytest.raises(ValueError, match=r"shape \(3, n\)"):
        W.wtheta_count_xyz(torch.zeros((100, 3), dtype=f64), None, e, True, c)
    with pytest.raises(ValueError, match="float64"):
        W.wtheta_count_xyz(soa.float(), None, e, True, c)
    with pytest.raises(ValueError, match="whole points|shape"):
        W.wtheta_count_xyz(torch.zeros(301, dtype=f64), None, e, True, c)
    with pytest.raises(ValueError, match="at least 18 slots"):
        W.wtheta_count_xyz(soa, None, e, True, torch.zeros(17, dtype=torch.int64))
    with pytest.raises(ValueError, match="interleaved RA/Dec"):
        W.wtheta_count(torch.zeros((2, 100), dtype=f64), None, e, True, c)
    with pytest.raises(ValueError, match="interleaved RA/Dec"):
        W.wtheta_count(rd, torch.zeros(201, dtype=f64), e, False, c)
    with pytest.raises(ValueError, match="at least 54 slots"):
        W.wtheta_count_wtheta(rd, rd, False, e, c)
    with pytest.raises(ValueError, match=r"shape \(3, n\)"):
        W.wtheta_count_wtheta(torch.zeros((100, 3), dtype=f64), soa, True, e, c3)
    with pytest.raises(ValueError, match="stats"):
        W.wtheta_count_ex(rd, None, False, e, True, c, stats=torch.zeros(2, dtype=torch.int64))
    with pytest.raises(ValueError, match="xyz"):
        W.wtheta_radec_to_xyz(rd, torch.zeros(200, dtype=f64))
    # the layouts the library reads are accepted: the next check is the device's
    for call in (lambda: W.wtheta_count_xyz(soa, None, e, True, c),
                 lambda: W.wtheta_count_xyz(soa.reshape(-1), None, e, True, c),
                 lambda: W.wtheta_count(rd.reshape(-1, 2), None, e, True, c),
                 lambda: W.wtheta_count_wtheta(rd, rd, False, e, c3)):
        with pytest.raises(ValueError, match="CUDA"):
            call()


def test_binding_counts_host_points_by_elements():
    """Host catalogues (wtheta_correlate, wtheta_server_submit) may be 1-D
    interleaved RA/Dec or (n, 2): both give n points (the length of an (n, 2)
    array is n, not 2n); other shapes are refused before any call."""
    a = np.zeros(20)
    assert W._host_points(a, "data") == 10
    assert W._host_points(a.reshape(10, 2), "data") == 10
    for bad in (np.zeros(21), np.zeros((10, 3)), np.zeros((2, 10)), np.zeros((2, 5, 2))):
        with pytest.raises(ValueError, match="interleaved RA/Dec"):
            W._host_points(bad, "data")
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    with pytest.raises(ValueError, match="interleaved RA/Dec"):
        W.wtheta_correlate(np.zeros((10, 3)), np.zeros(20), e)
