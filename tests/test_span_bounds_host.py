"""Soundness of the span bounds, by host emulation of the pair kernel's FP32
sphere arithmetic (no GPU).

Span binning settles a (group, chunk) pair from two bounding spheres alone:
the group sphere of 8 consecutive FP32 points (`group_cap`), the chunk sphere
of 32 (`k_chunk_caps`), and the interval [s_lo, s_hi] that `span_class`
derives from them with fixed slack (relative 1e-6 on distances and radii,
absolute 1e-6, relative 1e-5 on the squares).  Every pair's FP64 squared chord
must lie inside that interval, or a settled chunk would be miscounted.  These
tests evaluate the same FP32 steps in numpy -- each operation rounded to FP32,
once with separate products and sums and once with the products fused into
the sums, since the compiler may contract either way -- and check every pair
of random and adversarial configurations (tiny and wide spheres, coincident
points, near-antipodal spheres)."""
import numpy as np
import pytest

F = np.float32


def _fma(a, b, c):
    """fl32(a * b + c): the product is exact in FP64; rounding the FP64 sum to
    FP32 can differ from a true fma by one FP32 ulp, far inside the slack."""
    return (a.astype(np.float64) * b.astype(np.float64) + c.astype(np.float64)).astype(F)


def _norm2(dx, dy, dz, fused):
    if fused:
        return _fma(dz, dz, _fma(dy, dy, (dx * dx).astype(F)))
    return ((dx * dx).astype(F) + (dy * dy).astype(F)).astype(F) + (dz * dz).astype(F)


def _group_sphere(P, fused):
    """group_cap: P (3, n_cfg, 8) FP32; centre = sequential sum / 8, radius =
    sqrt(max squared distance) * (1 + 1e-6)."""
    c = np.zeros(P.shape[:2], F)
    for r in range(P.shape[2]):
        c = (c + P[:, :, r]).astype(F)
    c = (c * F(1.0 / P.shape[2])).astype(F)
    m = np.zeros(P.shape[1], F)
    for r in range(P.shape[2]):
        d = (P[:, :, r] - c).astype(F)
        m = np.maximum(m, _norm2(d[0], d[1], d[2], fused))
    return c, (np.sqrt(m) * F(1.0 + F(1e-6))).astype(F)


def _chunk_sphere(P, fused):
    """k_chunk_caps: P (3, n_cfg, 32) FP32; centre = butterfly (xor-shuffle)
    sum / 32, radius = sqrt(max squared distance) * (1 + 1e-6)."""
    s = P.copy()
    o = 16
    while o:
        idx = np.arange(32) ^ o
        s = (s + s[:, :, idx]).astype(F)
        o >>= 1
    c = (s[:, :, 0] * F(1.0 / 32)).astype(F)
    d = (P - c[:, :, None]).astype(F)
    m = _norm2(d[0], d[1], d[2], fused).max(axis=1)
    return c, (np.sqrt(m) * F(1.0 + F(1e-6))).astype(F)


def _span(ca, ra, cb, rb, fused):
    """span_class's [s_lo, s_hi] in FP32."""
    d = (ca - cb).astype(F)
    dc = np.sqrt(_norm2(d[0], d[1], d[2], fused)).astype(F)
    k1, k2 = F(1.0 + F(1e-6)), F(1.0 - F(1e-6))
    w = (ra + rb).astype(F)
    if fused:
        rr = _fma(w, np.full_like(w, k1), np.full_like(w, F(1e-6)))
        lo = _fma(dc, np.full_like(dc, k2), -rr)
        hi = _fma(dc, np.full_like(dc, k1), rr)
    else:
        rr = ((w * k1).astype(F) + F(1e-6)).astype(F)
        lo = ((dc * k2).astype(F) - rr).astype(F)
        hi = ((dc * k1).astype(F) + rr).astype(F)
    slo = np.where(lo > 0, ((lo * lo).astype(F) * F(1.0 - F(1e-5))).astype(F), F(0))
    shi = ((hi * hi).astype(F) * F(1.0 + F(1e-5))).astype(F)
    return slo, shi


def _unit(v):
    return v / np.linalg.norm(v, axis=0)


def _cloud(centre, radius, n, rng):
    """n FP64 unit vectors within about `radius` radians of centre (3, n_cfg)."""
    t = rng.normal(size=(3,) + centre.shape[1:] + (n,)) * radius[None, :, None]
    return _unit(centre[:, :, None] + t)


def _check(A, B, fused):
    """A (3, n_cfg, 8), B (3, n_cfg, 32) FP64 unit vectors: every pair's FP64
    squared chord inside the FP32 span of the two spheres."""
    a32, b32 = A.astype(F), B.astype(F)
    ca, ra = _group_sphere(a32, fused)
    cb, rb = _chunk_sphere(b32, fused)
    slo, shi = _span(ca, ra, cb, rb, fused)
    d = A[:, :, :, None] - B[:, :, None, :]
    s64 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]           # (n_cfg, 8, 32)
    lo_ok = s64 >= slo.astype(np.float64)[:, None, None]
    hi_ok = s64 <= shi.astype(np.float64)[:, None, None]
    bad = ~(lo_ok & hi_ok)
    assert not bad.any(), (np.argwhere(bad)[:5], slo[bad.any(axis=(1, 2))][:3],
                           shi[bad.any(axis=(1, 2))][:3])
    return shi - slo


@pytest.mark.parametrize("fused", [False, True])
@pytest.mark.parametrize("r_group,r_chunk", [(1e-7, 1e-7), (1e-5, 3e-5), (2e-3, 5e-3),
                                             (3e-2, 1e-1), (0.0, 0.0), (1e-4, 0.0)])
def test_every_pair_inside_the_span(r_group, r_chunk, fused):
    rng = np.random.default_rng(int(1e7 * (r_group + 2 * r_chunk)) + fused)
    n = 4000
    ca = _unit(rng.normal(size=(3, n)))
    # separations from coincident to antipodal, log-spread at small angles
    theta = np.concatenate([np.zeros(200), 10.0 ** rng.uniform(-8, np.log10(np.pi), n - 400),
                            np.pi - 10.0 ** rng.uniform(-8, -2, 200)])
    t = _unit(rng.normal(size=(3, n)))
    t = _unit(t - ca * np.sum(ca * t, axis=0))
    cb = ca * np.cos(theta) + t * np.sin(theta)
    A = _cloud(ca, np.full(n, r_group), 8, rng)
    B = _cloud(cb, np.full(n, r_chunk), 32, rng)
    _check(A, B, fused)


@pytest.mark.parametrize("fused", [False, True])
def test_coincident_and_duplicated_points(fused):
    """All 40 points one vector, or the chunk a copy of the group: s = 0 must
    lie inside the span (s_lo clamps to 0)."""
    rng = np.random.default_rng(5)
    n = 500
    c = _unit(rng.normal(size=(3, n)))
    A = np.repeat(c[:, :, None], 8, axis=2)
    B = np.repeat(c[:, :, None], 32, axis=2)
    width = _check(A, B, fused)
    assert np.all(width >= 0)
    g = _cloud(c, np.full(n, 1e-3), 8, rng)
    _check(g, np.concatenate([g, g, g, g], axis=2), fused)


@pytest.mark.parametrize("fused", [False, True])
def test_span_is_tight_enough_to_settle(fused):
    """Not a soundness check: at the survey's scales (group 0.15 deg, chunk
    0.3 deg, separations 1-20 deg) the span is barely wider than the spheres
    allow, so span binning can settle most chunks."""
    rng = np.random.default_rng(9)
    n = 2000
    ca = _unit(rng.normal(size=(3, n)))
    theta = np.radians(rng.uniform(1.0, 20.0, n))
    t = _unit(rng.normal(size=(3, n)))
    t = _unit(t - ca * np.sum(ca * t, axis=0))
    cb = ca * np.cos(theta) + t * np.sin(theta)
    A = _cloud(ca, np.full(n, np.radians(0.15)), 8, rng)
    B = _cloud(cb, np.full(n, np.radians(0.3)), 32, rng)
    width = _check(A, B, fused).astype(np.float64)
    # the exact width of the spheres' span, (d + r)^2 - max(d - r, 0)^2
    a32, b32 = A.astype(F), B.astype(F)
    ca32, ra = _group_sphere(a32, fused)
    cb32, rb = _chunk_sphere(b32, fused)
    dist = np.linalg.norm((ca32 - cb32).astype(np.float64), axis=0)
    r = (ra + rb).astype(np.float64)
    ideal = (dist + r) ** 2 - np.maximum(dist - r, 0.0) ** 2
    assert np.all(width <= ideal * 1.001 + 1e-5)
