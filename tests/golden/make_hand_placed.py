"""Writes hand_placed.txt: point pairs whose angular separation is known by
construction, for checking the binning of App. A's separation.

Every pair is placed so that its separation follows from the geometry alone,
with no trigonometry evaluated here:
  - two points on the equator, RA 0 and RA t: separation t;
  - two points on one meridian, Dec d and d + t: separation t;
  - RA wrap: RA 360 - t/2 and RA t/2 on the equator: separation t;
  - both at the north pole with different RA: separation 0 (same point);
  - identical coordinates: separation exactly 0, so the squared chord is
    exactly 0 and, for edges starting at 0, sits exactly on the lower edge
    of bin 1 (bins include their lower edge);
  - (RA, Dec) and (RA + 180, -Dec): antipodal, separation 180.
Separations are placed at the geometric middle of each bin of the named edge
set, and below/above the range, so no case sits near an edge.

Run: python tests/golden/make_hand_placed.py
"""
import math
import os

ARCMIN = 1.0 / 60.0

# edge sets: (name, lo_deg, hi_deg, n_bins, spacing) -- spacing 'log' or 'lin'
EDGE_SETS = [
    ("log16_1am_5d", 1.0 * ARCMIN, 5.0, 16, "log"),
    ("log32_halfam_20d", 0.5 * ARCMIN, 20.0, 32, "log"),
    ("lin12_0_180", 0.0, 180.0, 12, "lin"),
]


def mids(lo, hi, K, spacing):
    out = []
    for k in range(K):
        if spacing == "log":
            r = (hi / lo) ** (1.0 / K)
            out.append(lo * r ** (k + 0.5))
        else:
            out.append(lo + (k + 0.5) * (hi - lo) / K)
    return out


def main():
    lines = ["# name ra1 dec1 ra2 dec2 theta_deg construction",
             "# Separation known by construction (App. A geometry); degrees."]
    for name, lo, hi, K, spacing in EDGE_SETS:
        ts = mids(lo, hi, K, spacing)
        if lo > 0:
            ts = [0.5 * lo] + ts
        if hi < 90:
            ts = ts + [min(2.0 * hi, 170.0)]
        for t in ts:
            lines.append(f"{name} 0.0 0.0 {t!r} 0.0 {t!r} equator")
            if t < 140.0:
                lines.append(f"{name} 200.0 -20.0 200.0 {-20.0 + t!r} {t!r} meridian")
            lines.append(f"{name} {360.0 - t / 2!r} 0.0 {t / 2!r} 0.0 {t!r} ra_wrap")
        lines.append(f"{name} 0.0 90.0 123.4 90.0 0.0 pole")
        lines.append(f"{name} 10.0 20.0 10.0 20.0 0.0 coincident")
        lines.append(f"{name} 10.0 20.0 190.0 -20.0 180.0 antipodal")
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "hand_placed.txt")
    with open(path, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
