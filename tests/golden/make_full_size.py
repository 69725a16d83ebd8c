"""Writes full_size.txt: the oracle's exact DD, DR and RR counts (Sec. 2 pair
sets, App. A separations, Sec. 2.1 bins) for workloads too large to count in
a test run:

  - survey: the whole 1M clustered + 1M uniform polar-cap workload, 32 log
    bins 0.5'-20 deg (2.0e12 pairs);
  - batch: 8 of the 256 batch mocks, chosen so that their data sizes span
    the workload's 20k-400k range, 16 log bins 1'-5 deg (2x randoms);
  - serve: the first two auto and the first two cross requests of the serve
    workload's stream whose catalogues hold 50k-150k points, 24 log bins
    1'-10 deg, with the oracle's ambiguity count (pairs within tau_k of an
    edge, the only ones whose slot may differ when the device converts RA/Dec
    itself) beside each count.

Every count is made by the oracle (oracle/) on its own FP64 unit vectors of
the catalogues that paper_1208_3658_gb300/synth.py draws; nothing here comes
from the CUDA path.  Each line records a SHA-256 of the RA/Dec inputs and of
the oracle's unit vectors, so a test on another machine can tell whether it
regenerated the same inputs before comparing counts.

Line format (whitespace separated):
    case  count  n_a  n_b  sha_radec  sha_xyz  ambiguous  slot_0 ... slot_K+1
with count one of DD, DR, RR (auto workloads) or D1D2, D1R2, R1D2, R1R2
(cross requests), and ambiguous = -1 where it was not computed.

Run: python tests/golden/make_full_size.py [--hashes-only] [--only CASE]
(about an hour on 8 cores; --hashes-only prints the input hashes at once).
"""
from __future__ import annotations

import argparse
import hashlib
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from oracle import oracle as O  # noqa: E402
from paper_1208_3658_gb300 import synth  # noqa: E402

OUT = os.path.join(HERE, "full_size.txt")
N_MOCKS_CHOSEN = 8
SERVE_N_RANGE = (50_000, 150_000)


def sha(*arrays) -> str:
    h = hashlib.sha256()
    for a in arrays:
        h.update(np.ascontiguousarray(a).tobytes())
    return h.hexdigest()[:32]


def chosen_mocks(n_pick: int = N_MOCKS_CHOSEN):
    """Indices of batch mocks whose data sizes are nearest to n_pick
    geometrically spaced sizes between the smallest and the largest."""
    sizes = synth.batch_sizes()
    targets = np.geomspace(sizes.min(), sizes.max(), n_pick)
    picked = []
    for t in targets:
        order = np.argsort(np.abs(np.log(sizes / t)))
        picked.append(int(next(i for i in order if int(i) not in picked)))
    return sorted(picked, key=lambda m: sizes[m])


def chosen_requests():
    """The first two auto and two cross serve requests in SERVE_N_RANGE."""
    sizes, is_auto = synth.serve_sizes()
    lo, hi = SERVE_N_RANGE
    autos = [q for q in range(len(sizes)) if is_auto[q] and lo <= sizes[q] <= hi][:2]
    cross = [q for q in range(len(sizes)) if not is_auto[q] and lo <= sizes[q] <= hi][:2]
    return autos + cross


def cases():
    """(case name, edges, [(count, rd_a, rd_b or None, is_auto)], want_ambiguous)."""
    wl = synth.survey()
    e = O.edges(wl.lo_deg, wl.hi_deg, wl.n_bins)
    yield "survey", e, [("DD", wl.data, None, True), ("DR", wl.data, wl.rand, False),
                        ("RR", wl.rand, None, True)], False
    lo, hi, K = 1.0 * synth.ARCMIN, 5.0, 16
    e = O.edges(lo, hi, K)
    for m in chosen_mocks():
        mk = synth.batch_mock(1, m)
        yield "batch_mock_%d" % m, e, [("DD", mk.data, None, True),
                                       ("DR", mk.data, mk.rand, False),
                                       ("RR", mk.rand, None, True)], False
    e = O.edges(1.0 * synth.ARCMIN, 10.0, 24)
    for q in chosen_requests():
        rq = synth.serve_request(1, q)
        if rq.kind == "auto":
            cs = [("DD", rq.data, None, True), ("DR", rq.data, rq.rand, False),
                  ("RR", rq.rand, None, True)]
        else:
            cs = [("D1D2", rq.data, rq.data2, False), ("D1R2", rq.data, rq.rand2, False),
                  ("R1D2", rq.rand, rq.data2, False), ("R1R2", rq.rand, rq.rand2, False)]
        yield "serve_request_%d" % q, e, cs, True


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--hashes-only", action="store_true")
    ap.add_argument("--only", default="")
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args()
    lines = []
    for name, e, counts, want_amb in cases():
        if args.only and not name.startswith(args.only):
            continue
        for cname, a, b, auto in counts:
            A = O.radec_to_xyz(a)
            B = None if auto else O.radec_to_xyz(b)
            n_a = A.shape[1]
            n_b = n_a if auto else B.shape[1]
            h_rd = sha(a) if auto else sha(a, b)
            h_xyz = sha(A) if auto else sha(A, B)
            if args.hashes_only:
                print(name, cname, n_a, n_b, h_rd, h_xyz, flush=True)
                continue
            t = time.time()
            c = O.count_xyz(A, B, e, auto)
            amb = O.count_ambiguous_xyz(A, B, e, auto) if want_amb else -1
            print("%s %s %d x %d: %.0f s" % (name, cname, n_a, n_b, time.time() - t), flush=True)
            lines.append(" ".join([name, cname, str(n_a), str(n_b), h_rd, h_xyz, str(amb)]
                                  + [str(int(x)) for x in c]))
            # written as it goes, so a long run keeps what it finished
            with open(args.out + ".partial", "w") as f:
                f.write("\n".join(lines) + "\n")
    if args.hashes_only:
        return
    with open(args.out, "w") as f:
        f.write("# Oracle counts at full size; written by tests/golden/make_full_size.py\n")
        f.write("# case count n_a n_b sha256(ra_dec)[:32] sha256(oracle xyz)[:32] ambiguous "
                "slots 0..K+1\n")
        f.write("\n".join(lines) + "\n")
    os.remove(args.out + ".partial")


if __name__ == "__main__":
    main()
