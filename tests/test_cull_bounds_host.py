"""Soundness of tile culling, by host emulation of the tile caps (no GPU).

A tile pair is skipped when its caps' centres are more than
theta_top + rho_A + rho_B + 3e-6 rad apart (`caps_may_meet`); every pair it
holds is then counted only through the overflow slot, so a skipped tile pair
holding a pair below the top edge would be miscounted.  The caps are emulated
as `k_tile_caps` computes them (FP64 sum of the FP32 points, normalised;
radius = the largest angle from the centre, 2 asin(|c - p| / 2), plus 1e-6
rad), and tile pairs are placed just around the skipping threshold, where a
missing margin would show first.  Every pair of a skipped tile pair must have
its FP64 squared chord at or above the top edge's."""
import numpy as np
import pytest

from paper_1208_3658_gb300 import wtheta as W


def _unit(v):
    return v / np.linalg.norm(v, axis=0)


def _tile(centre, radius, n, rng):
    t = rng.normal(size=(3, n)) * radius
    return _unit(centre[:, None] + t)


def _cap(P64):
    """k_tile_caps on the FP32 copies of one tile's points."""
    p = P64.astype(np.float32).astype(np.float64)
    s = p.sum(axis=1)
    c = s / np.sqrt(np.sum(s * s))
    m = np.max(np.sum((c[:, None] - p) ** 2, axis=0))
    return c, 2.0 * np.arcsin(min(1.0, 0.5 * np.sqrt(m))) + 1e-6


def _skipped(ca, ra, cb, rb, theta_top):
    chord = np.sqrt(np.sum((ca - cb) ** 2))
    theta_c = 2.0 * np.arcsin(min(1.0, 0.5 * chord))
    return theta_c - ra - rb - 3e-6 > theta_top


@pytest.mark.parametrize("top_deg,r_deg", [(0.5, 0.05), (5.0, 0.5), (20.0, 2.0), (90.0, 1.0),
                                           (1.0 / 60, 1e-4)])
def test_skipped_tile_pairs_hold_no_pair_below_the_top_edge(top_deg, r_deg):
    rng = np.random.default_rng(int(top_deg * 1000 + r_deg * 10))
    e = W.wtheta_edges(top_deg / 10, top_deg, 8)
    c_top = W.wtheta_chord2_edges(e)[-1]
    theta_top = np.radians(top_deg)
    n_skipped = 0
    for it in range(300):
        ca = _unit(rng.normal(size=3))
        A = _tile(ca, np.radians(r_deg), 256, rng)
        B0 = _tile(np.array([0.0, 0.0, 1.0]), np.radians(r_deg) * rng.uniform(0.2, 1.5), 256, rng)
        cap_a, rho_a = _cap(A)
        cap_b0, rho_b = _cap(B0)
        # half the tile pairs within a few micro-radians of the threshold, half
        # up to rho_a + rho_b closer than it (never skipped by a sound rule,
        # while a rule that forgot a radius would skip them)
        if it % 2 == 0:
            off = rng.uniform(-2e-5, 2e-5)
        else:
            off = -rng.uniform(0.0, 1.0) * (rho_a + rho_b)
        target = theta_top + rho_a + rho_b + 3e-6 + off
        # rotate B so that its cap centre sits at angle `target` from A's
        t = _unit(rng.normal(size=3))
        t = _unit(t - cap_a * np.dot(cap_a, t))
        want = cap_a * np.cos(target) + t * np.sin(target)
        # rotation taking cap_b0 to want (Rodrigues)
        k = np.cross(cap_b0, want)
        s, c = np.linalg.norm(k), np.dot(cap_b0, want)
        K = np.array([[0, -k[2], k[1]], [k[2], 0, -k[0]], [-k[1], k[0], 0]]) / max(s, 1e-300)
        Rm = np.eye(3) + s * K + (1 - c) * (K @ K)
        B = _unit(Rm @ B0)
        cap_b, rho_b = _cap(B)
        if not _skipped(cap_a, rho_a, cap_b, rho_b, theta_top):
            continue
        n_skipped += 1
        d = A[:, :, None] - B[:, None, :]
        s64 = (d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]
        assert s64.min() >= c_top, (s64.min(), c_top)
    assert n_skipped > 20  # the placement straddles the threshold
