"""Checks that pin the CPU oracle to facts fixed outside itself.

Each check raises AssertionError on failure.  They are collected by
test_oracle_pins.py and re-run against deliberately broken builds of the
oracle in test_oracle_mutants.py, which asserts that every plausible mistake
(a dropped term, a wrong sign or index, an off-by-one) fails at least one.

Sources of truth, none of them the oracle itself:
  - hand_placed: separations known by construction (golden/hand_placed.txt);
  - totals: n(n-1)/2 auto pairs and n_a n_b cross pairs (Sec. 2);
  - dr_rd: the cross count is symmetric in its arguments;
  - d_equals_r: random catalogue == data gives w = 2/n exactly (Eq. 2 with
    pair totals; derivation in the check);
  - r_is_d_twice: random catalogue == data listed twice gives
    w = (3n - 2) / (2n(n - 1));
  - cross_identity: R1 == D1 gives the cross estimator w = 0;
  - analytic_rr: uniform full-sky pairs fall in [t1, t2) with probability
    (cos t1 - cos t2)/2, and the bin counts have binomial variance;
  - bruteforce_angles: App. A's formula (with atan2) in long double on small
    random catalogues agrees with the oracle's slots;
  - edges_*: the three binning modes of Sec. 2.1;
  - chord_values: chord lengths of 60, 90 and 180 degrees;
  - ls_empty_bins: Eq. 2 on hand-made counts, with its value worked out by
    hand, and no value (NaN) where the bin holds no random pairs;
  - ambiguity_tau: pairs placed around every edge of the workloads' edge
    sets, their unit vectors moved by up to 8 ulps per component (aligned
    with the pair's difference, and at random): every pair whose slot moves is
    one the oracle flags as ambiguous, and the flagged width is no more than
    about twice the largest move the perturbations reach.
"""
from __future__ import annotations

import bisect
import math
import os

import numpy as np

from oracle import oracle as O
from paper_1208_3658_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
ARCMIN = 1.0 / 60.0

GOLDEN_EDGES = {
    "log16_1am_5d": (1.0 * ARCMIN, 5.0, 16, O.LN),
    "log32_halfam_20d": (0.5 * ARCMIN, 20.0, 32, O.LN),
    "lin12_0_180": (0.0, 180.0, 12, O.LINEAR),
}


def _slot_by_angle(edges_deg, theta_deg):
    """Expected slot from the angle itself: number of edges <= theta."""
    return bisect.bisect_right(list(edges_deg), theta_deg)


def check_hand_placed():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "hand_placed.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) > 100
    for name, (lo, hi, K, mode) in GOLDEN_EDGES.items():
        e = O.edges(lo, hi, K, mode)
        sel = [r for r in rows if r[0] == name]
        a = np.array([[float(r[1]), float(r[2])] for r in sel]).reshape(-1)
        b = np.array([[float(r[3]), float(r[4])] for r in sel]).reshape(-1)
        A, B = O.radec_to_xyz(a), O.radec_to_xyz(b)
        for i, r in enumerate(sel):
            got = O.count_xyz(A[:, i:i + 1], B[:, i:i + 1], e, False)
            want = np.zeros(K + 2, np.uint64)
            want[_slot_by_angle(e, float(r[5]))] = 1
            assert np.array_equal(got, want), (name, r, got)


def _patch_cat(n, seed, path):
    return synth.uniform(synth.Patch(0.0, 10.0, 0.0, 10.0), n, seed, "test", path)


def check_totals():
    e = O.edges(1.0 * ARCMIN, 5.0, 16)
    for n_a, n_b in [(0, 0), (1, 0), (1, 1), (2, 3), (31, 33), (257, 100)]:
        A = _patch_cat(n_a, 3, n_a)
        B = _patch_cat(n_b, 4, n_b)
        auto = O.count(A, None, e, True)
        cross = O.count(A, B, e, False)
        assert int(auto.sum()) == n_a * (n_a - 1) // 2, (n_a, auto)
        assert int(cross.sum()) == n_a * n_b, (n_a, n_b, cross)


def check_dr_rd():
    e = O.edges(1.0 * ARCMIN, 5.0, 16)
    A, B = _patch_cat(700, 5, 1), _patch_cat(500, 6, 2)
    assert np.array_equal(O.count(A, B, e, False), O.count(B, A, e, False))


def _clustered(n, seed):
    fp = synth.Patch(0.0, 5.0, 0.0, 5.0)
    return synth.clustered(fp, n, max(1, n // 50), 3.0, seed, "test", "data")


def check_d_equals_r():
    """R = D: DR counts ordered pairs, the n self pairs landing in underflow
    (e_0 > 0), so DR_k = 2 DD_k and RR_k = DD_k for k >= 1.  With the pair
    totals, w_k = [2DD/(n(n-1)) - 2*2DD/n^2 + 2DD/(n(n-1))] / [2DD/(n(n-1))]
    = 2 - 2(n-1)/n = 2/n for every bin with DD_k > 0."""
    n = 800
    e = O.edges(1.0 * ARCMIN, 5.0, 16)
    D = _clustered(n, 7)
    DD = O.count(D, None, e, True)
    DR = O.count(D, D, e, False)
    w = O.ls(DD, DR, DD, n, n)
    nz = DD[1:-1] > 0
    assert nz.sum() >= 10
    assert np.all(np.abs(w[nz] - 2.0 / n) <= 1e-12 * 3.0), w[nz]


def check_r_is_d_twice():
    """R = D listed twice (n_r = 2n): for k >= 1, with P_k = DD_k,
    DR_k = 4 P_k, RR_k = 4 P_k (pairs within each copy plus ordered pairs
    across copies), N_DD = n(n-1)/2, N_DR = 2n^2, N_RR = n(2n-1), so
    w_k = (3n - 2) / (2n(n - 1))."""
    n = 600
    e = O.edges(1.0 * ARCMIN, 5.0, 16)
    D = _clustered(n, 8)
    R = np.concatenate([D, D])
    DD = O.count(D, None, e, True)
    DR = O.count(D, R, e, False)
    RR = O.count(R, None, e, True)
    w = O.ls(DD, DR, RR, n, 2 * n)
    nz = DD[1:-1] > 0
    want = (3 * n - 2) / (2 * n * (n - 1))
    assert nz.sum() >= 10
    assert np.all(np.abs(w[nz] - want) <= 1e-12 * 3.0), (w[nz], want)


def check_estimators_closed_forms():
    """The other estimators on the two closed-form cases above.  R = D
    (n_r = n): dd = rr = 2P/(n(n-1)), dr = 2P/n^2, so natural = 0,
    Davis-Peebles = n/(n-1) - 1 = 1/(n-1), Hamilton = n^2/(n-1)^2 - 1 =
    (2n-1)/(n-1)^2.  R = D twice (n_r = 2n): dd = 2P/(n(n-1)), dr = 2P/n^2,
    rr = 4P/(n(2n-1)), so natural = 1/(2(n-1)), Davis-Peebles = 1/(n-1),
    Hamilton = 2n^2/((n-1)(2n-1)) - 1 = (3n-1)/((n-1)(2n-1))."""
    e = O.edges(1.0 * ARCMIN, 5.0, 16)
    n = 700
    D = _clustered(n, 9)
    DD = O.count(D, None, e, True)
    DR = O.count(D, D, e, False)
    nz = DD[1:-1] > 0
    assert nz.sum() >= 10
    for name, want in [("natural", 0.0), ("davis_peebles", 1.0 / (n - 1)),
                       ("hamilton", (2 * n - 1) / (n - 1) ** 2),
                       ("landy_szalay", 2.0 / n)]:
        w = O.estimator(DD, DR, DD, n, n, name)
        assert np.all(np.abs(w[nz] - want) <= 1e-12 * max(abs(want), 1e-3)), (name, w[nz], want)
    R = np.concatenate([D, D])
    DR2 = O.count(D, R, e, False)
    RR2 = O.count(R, None, e, True)
    for name, want in [("natural", 1.0 / (2 * (n - 1))), ("davis_peebles", 1.0 / (n - 1)),
                       ("hamilton", (3 * n - 1) / ((n - 1) * (2 * n - 1))),
                       ("landy_szalay", (3 * n - 2) / (2 * n * (n - 1)))]:
        w = O.estimator(DD, DR2, RR2, n, 2 * n, name)
        assert np.all(np.abs(w[nz] - want) <= 1e-12 * abs(want)), (name, w[nz], want)
    # empty bins of the denominator give NaN
    z = np.zeros(18, np.uint64)
    assert np.all(np.isnan(O.estimator(z, z, z, 10, 10, "hamilton")))


def check_regions_and_jackknife():
    """Region-pair counts sum to the whole counts; the jackknife sample k has
    exactly the counts of the catalogues recounted without region k (the
    definition of the sample), and its w is Eq. 2 of those; the covariance is
    (R-1) times numpy's biased covariance of the samples."""
    fp = synth.Patch(30.0, 6.0, -10.0, -4.0)
    D = synth.clustered(fp, 700, 14, 3.0, 4, "test", "data")
    Rn = synth.uniform(fp, 900, 4, "test", "random")
    e = O.edges(1.0 * ARCMIN, 3.0, 10)
    R = 6
    ld = synth.grid_labels(D, 30.0, 36.0, -10.0, -4.0, 3, 2)
    lr = synth.grid_labels(Rn, 30.0, 36.0, -10.0, -4.0, 3, 2)
    XD, XR = O.radec_to_xyz(D), O.radec_to_xyz(Rn)
    c = O.count_regions(XD, ld, XR, lr, e, R)
    assert np.array_equal(c[0].sum(axis=(0, 1), dtype=np.uint64), O.count_xyz(XD, None, e, True))
    assert np.array_equal(c[1].sum(axis=(0, 1), dtype=np.uint64), O.count_xyz(XD, XR, e, False))
    assert np.array_equal(c[2].sum(axis=(0, 1), dtype=np.uint64), O.count_xyz(XR, None, e, True))
    assert not c[0][np.tril_indices(R, -1)].any()
    sizes = np.concatenate([np.bincount(ld, minlength=R), np.bincount(lr, minlength=R)])
    w, w_k, cov = O.jackknife(c, sizes, R)
    for k in (0, 3, 5):
        Dk, Rk = XD[:, ld != k], XR[:, lr != k]
        DD = O.count_xyz(np.ascontiguousarray(Dk), None, e, True)
        DR = O.count_xyz(np.ascontiguousarray(Dk), np.ascontiguousarray(Rk), e, False)
        RR = O.count_xyz(np.ascontiguousarray(Rk), None, e, True)
        want = O.ls(DD, DR, RR, Dk.shape[1], Rk.shape[1])
        assert np.array_equal(w_k[k], want, equal_nan=True)
    ok = np.all(np.isfinite(w_k), axis=0)
    ref = (R - 1) * np.cov(w_k[:, ok].T, bias=True)
    assert np.allclose(cov[np.ix_(ok, ok)], ref, rtol=1e-12, atol=1e-15)


def check_cross_identity():
    """Cross estimator with R1 = D1: d1d2 - d1r2 - r1d2 + r1r2 = 0."""
    e = O.edges(1.0 * ARCMIN, 5.0, 16)
    D1, D2 = _clustered(400, 9), _clustered(500, 10)
    R2 = _patch_cat(450, 11, 3)
    D1D2 = O.count(D1, D2, e, False)
    D1R2 = O.count(D1, R2, e, False)
    w = O.ls_cross(D1D2, D1R2, D1D2, D1R2, 400, 500, 400, 450)
    ok = D1R2[1:-1] > 0
    assert ok.sum() >= 10
    assert np.all(np.abs(w[ok]) <= 1e-12 * 4.0), w[ok]


def check_analytic_rr(n: int = 20_000):
    """Uniform full-sky points: a pair falls in [t1, t2) with probability
    p = (cos t1 - cos t2)/2; indicators of pairs sharing a point are
    uncorrelated (isotropy), so Var(RR_k) = N p (1 - p) exactly."""
    e = O.edges(1.0, 120.0, 16)
    R = synth.uniform(synth.FullSky(), n, 12, "test", "random")
    RR = O.count(R, None, e, True).astype(np.float64)
    N = n * (n - 1) / 2
    cosd = np.cos(np.radians(np.concatenate([[0.0], e, [180.0]])))
    p = (cosd[:-1] - cosd[1:]) / 2.0
    sigma = np.sqrt(N * p * (1 - p))
    z = (RR - N * p) / sigma
    assert np.all(np.abs(z) <= 5.0), z


def check_bruteforce_angles(n: int = 400):
    """App. A: theta = atan2(sqrt(A + B^2), C) in long double (atan2 for
    theta > 90 deg), binned by degree edges, against the oracle's slots for
    every pair of a small catalogue pair mixing a patch and the full sky."""
    e = O.edges(0.5 * ARCMIN, 100.0, 24)
    a = np.concatenate([_clustered(n // 2, 13),
                        synth.uniform(synth.FullSky(), n // 2, 14, "test", "random")])
    b = np.concatenate([_patch_cat(n // 2, 15, 4),
                        synth.uniform(synth.FullSky(), n // 2, 16, "test", "random")])
    L = np.longdouble
    ra1 = a[0::2].astype(L)[:, None] * (L(np.pi) / 180)
    de1 = a[1::2].astype(L)[:, None] * (L(np.pi) / 180)
    ra2 = b[0::2].astype(L)[None, :] * (L(np.pi) / 180)
    de2 = b[1::2].astype(L)[None, :] * (L(np.pi) / 180)
    da = ra2 - ra1
    Aq = np.cos(de2) ** 2 * np.sin(da) ** 2
    Bq = np.cos(de1) * np.sin(de2) - np.sin(de1) * np.cos(de2) * np.cos(da)
    Cq = np.sin(de1) * np.sin(de2) + np.cos(de1) * np.cos(de2) * np.cos(da)
    theta = np.arctan2(np.sqrt(Aq + Bq * Bq), Cq) * (L(180) / L(np.pi))
    slots = np.searchsorted(e.astype(L), theta.reshape(-1), side="right")
    want = np.bincount(slots, minlength=len(e) + 1).astype(np.uint64)
    got = O.count(a, b, e, False)
    assert np.array_equal(got, want), (got, want)


def check_edges_modes():
    lo, hi, K = 1.0 * ARCMIN, 5.0, 16
    for mode in (O.LN, O.LOG10):
        e = O.edges(lo, hi, K, mode)
        assert e[0] == lo and e[-1] == hi
        r = e[1:] / e[:-1]
        assert np.allclose(r, (hi / lo) ** (1.0 / K), rtol=1e-13, atol=0), r
    for lo_l, hi_l in [(0.0, 3.0), (1.0, 4.0)]:
        e = O.edges(lo_l, hi_l, 12, O.LINEAR)
        assert np.allclose(np.diff(e), 0.25, rtol=1e-13, atol=0)
        assert e[0] == lo_l and e[-1] == hi_l


def check_chord_values():
    c = O.chord2(np.array([0.0, 60.0, 90.0, 180.0]))
    assert c[0] == 0.0
    assert abs(c[1] - 1.0) <= 4e-16 and abs(c[2] - 2.0) <= 8e-16 and abs(c[3] - 4.0) <= 8e-16
    t = 1e-3  # degrees: small-angle chord^2 ~ (t in radians)^2 (1 - t^2/12)
    cs = O.chord2(np.array([t]))[0]
    tr = math.radians(t)
    assert abs(cs - tr * tr * (1 - tr * tr / 12)) <= 1e-15 * cs


def check_ls_empty_bins():
    """Eq. 2 on hand-made counts with n_d = n_r = 3 (pair totals 3, 9, 3):
    DD = 3, DR = 0, RR = 3 gives (1 - 0 + 1)/1 = 2; DD = 0, DR = 9, RR = 3
    gives (0 - 2 + 1)/1 = -1; a bin with RR = 0 has no estimate (NaN),
    whatever DD and DR hold.  The cross form with all sizes 2 (totals 4):
    (4 - 0 - 0 + 4)/4 = 2, (0 - 4 - 4 + 4)/4 = -1, and NaN where R1R2 = 0."""
    u = lambda *v: np.array((0,) + v + (0,), np.uint64)  # noqa: E731
    w = O.ls(u(3, 0, 0, 3, 0), u(0, 9, 0, 9, 5), u(3, 3, 0, 0, 0), 3, 3)
    assert w[0] == 2.0 and w[1] == -1.0, w
    assert np.all(np.isnan(w[2:])), w
    w = O.ls_cross(u(4, 0, 0, 4), u(0, 4, 0, 0), u(0, 4, 0, 0), u(4, 4, 0, 0), 2, 2, 2, 2)
    assert w[0] == 2.0 and w[1] == -1.0, w
    assert np.all(np.isnan(w[2:])), w


# Edge sets of the workloads (lo, hi, K, mode) whose pairs the P2 tests compare.
TAU_EDGE_SETS = [
    (1.0 * ARCMIN, 5.0, 16, O.LN), (0.5 * ARCMIN, 20.0, 32, O.LN),
    (0.2 * ARCMIN, 30.0, 64, O.LN), (1.0 * ARCMIN, 10.0, 24, O.LN),
    (0.0, 180.0, 12, O.LINEAR),
]


def _ulp_move(x, k):
    """x moved by k ulps (k an integer array, same shape)."""
    out = x.copy()
    for step in range(int(np.max(np.abs(k))) if k.size else 0):
        up, down = k > step, k < -step
        out = np.where(up, np.nextafter(out, np.inf), out)
        out = np.where(down, np.nextafter(out, -np.inf), out)
    return out


def _slot(a, b, e):
    return int(np.argmax(O.count_xyz(a.reshape(3, 1), b.reshape(3, 1), e, False, nthreads=1)))


def _flagged(a, b, e, tau):
    return O.count_ambiguous_xyz(a.reshape(3, 1), b.reshape(3, 1), e, False, nthreads=1,
                                 tau=tau) > 0


def check_ambiguity_tau(scale: float = 1.0):
    """The ambiguity width tau_k of the P2 comparisons (device unit vectors
    within a few ulps of the host's).  For each edge c_k a pair (a, b) is
    placed with s = c_k + f W_k, W_k = 2 sqrt(3 c_k) 2^-49 the largest first-
    order move of s when every component of a and b moves by 8 ulps of 2^-53,
    for f in +-{0.3 ... 1.2} and +-3; a has all components near 1/sqrt(3)
    (ulps of 2^-53) and b lies along the tangent (1, 1, -2) direction, so that
    moving each component by 8 ulps against (or with) the sign of a_i - b_i
    reaches about 94% of W_k.  Checked: (1) every perturbed pair whose oracle
    slot differs from the unperturbed pair's is flagged (|s - c_k| <= tau_k);
    (2) some slot change happens at |s - c_k| > tau_k / 2, so that half the
    width would miss it; (3) pairs at |s - c_k| >= 2.5 W_k are not flagged.
    scale multiplies the width (a test plants scaled widths to see them fail)."""
    rng = np.random.default_rng(11)
    far_flip = False
    n_flips = 0
    for lo, hi, K, mode in TAU_EDGE_SETS:
        e = O.edges(lo, hi, K, mode)
        c = O.chord2(e)
        tau = O.ambiguity_tau(c) * scale
        for k in range(K + 1):
            if not (0.0 < c[k] < 3.9):
                continue
            W = 2.0 * math.sqrt(3.0 * c[k]) * 2.0 ** -49
            for f in (-3.0, -1.2, -0.9, -0.75, -0.6, -0.45, -0.3, 0.3, 0.45, 0.6, 0.75, 0.9, 1.2, 3.0):
                a = np.array([1.0, 1.0, 1.0]) + rng.uniform(-0.02, 0.02, 3)
                a /= np.linalg.norm(a)
                t = np.array([1.0, 1.0, -2.0])
                t -= a * np.dot(a, t)
                t /= np.linalg.norm(t)
                th = 2.0 * math.asin(math.sqrt(c[k] + f * W) / 2.0)
                b = math.cos(th) * a + math.sin(th) * t
                d = a - b
                s0 = ((d[0] * d[0]) + (d[1] * d[1])) + (d[2] * d[2])
                slot0 = _slot(a, b, e)
                flag0 = _flagged(a, b, e, tau)
                if abs(f) >= 3.0 and abs(s0 - c[k]) >= 2.5 * W:
                    assert not flag0, ("flagged far from the edge", k, f, s0 - c[k], tau[k])
                moves = [(8 * np.sign(d), -8 * np.sign(d)), (-8 * np.sign(d), 8 * np.sign(d))]
                moves += [(rng.integers(-8, 9, 3), rng.integers(-8, 9, 3)) for _ in range(3)]
                for ka, kb in moves:
                    a1 = _ulp_move(a, ka.astype(np.int64))
                    b1 = _ulp_move(b, kb.astype(np.int64))
                    if _slot(a1, b1, e) != slot0:
                        n_flips += 1
                        assert flag0, ("slot moved but not flagged", k, f, s0 - c[k], tau[k])
                        far_flip |= abs(s0 - c[k]) > 0.5 * tau[k]
    assert n_flips > 100, n_flips
    assert far_flip, "no slot change beyond half the width: the width is loose"


ALL_CHECKS = [
    check_hand_placed, check_totals, check_dr_rd, check_d_equals_r,
    check_r_is_d_twice, check_estimators_closed_forms, check_regions_and_jackknife,
    check_cross_identity, check_analytic_rr,
    check_bruteforce_angles, check_edges_modes, check_chord_values,
    check_ls_empty_bins, check_ambiguity_tau,
]
