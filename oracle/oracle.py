"""Python wrapper for the CPU oracle (``wtheta_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg
of the benchmark use it to produce expected values.  The library never imports
it.  Every function cites the passage of the paper it follows; see the C file
for the definitions.

Pins (tests/test_oracle_pins.py) check this oracle against values fixed by the
paper's statement of the problem and by mathematics: points at constructed
separations, pair totals (Sec. 2), DR = RD, the exact w = 2/n when the random
catalogue equals the data (Eq. 2 with the pair totals), the analytic pair
fraction for uniform full-sky randoms, and an independent long-double
angle-space evaluation of App. A's formula on small inputs; the other
estimators by their closed forms when the randoms are the data (once or
twice over); the region-pair counts by their sums and the jackknife samples
by recounting the catalogues without each region.
"""
from __future__ import annotations

import contextlib
import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wtheta_oracle.c")
_SO = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

LINEAR, LN, LOG10 = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off: no fused multiply-add)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".%d.tmp" % os.getpid()
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
            "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = _load(build())
    return _lib


@contextlib.contextmanager
def use_library(path: str):
    """Run the wrappers against another build of the oracle source (used by
    the mutation test, which compiles deliberately broken copies)."""
    global _lib
    prev = _lib
    _lib = _load(path)
    try:
        yield
    finally:
        _lib = prev


def _load(path: str):
    L = ctypes.CDLL(path)
    dp = ctypes.POINTER(ctypes.c_double)
    up = ctypes.POINTER(ctypes.c_uint64)
    i64, i32 = ctypes.c_int64, ctypes.c_int
    L.orc_num_threads.restype = i32
    L.orc_edges.argtypes = [ctypes.c_double, ctypes.c_double, i32, i32, dp]
    L.orc_chord2.argtypes = [dp, i32, dp]
    L.orc_chord2.restype = None
    L.orc_radec_to_xyz.argtypes = [dp, i64, dp]
    L.orc_radec_to_xyz.restype = None
    L.orc_count.argtypes = [dp, i64, dp, i64, dp, i32, i32, up, i32]
    L.orc_count_ambiguous.argtypes = [dp, i64, dp, i64, dp, dp, i32, i32, up, i32]
    L.orc_ls.argtypes = [up, up, up, i64, i64, i32, dp]
    L.orc_ls_cross.argtypes = [up, up, up, up, i64, i64, i64, i64, i32, dp]
    return L


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _up(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def num_threads() -> int:
    return lib().orc_num_threads()


def edges(lo_deg: float, hi_deg: float, n_bins: int, mode: int = LN) -> np.ndarray:
    """Bin edges in degrees: linear, natural-log or log10 spacing (Sec. 2.1)."""
    e = np.empty(n_bins + 1, np.float64)
    if lib().orc_edges(lo_deg, hi_deg, n_bins, mode, _dp(e)) != 0:
        raise ValueError("bad bin range")
    return e


def chord2(edges_deg: np.ndarray) -> np.ndarray:
    """Squared chord 4 sin^2(theta/2) of each degree edge (App. A geometry)."""
    e = np.ascontiguousarray(edges_deg, np.float64)
    c = np.empty_like(e)
    lib().orc_chord2(_dp(e), len(e) - 1, _dp(c))
    return c


def radec_to_xyz(ra_dec: np.ndarray) -> np.ndarray:
    """Unit vectors (SoA, shape (3, n)) from interleaved RA/Dec degrees (App. A)."""
    rd = np.ascontiguousarray(ra_dec, np.float64)
    n = len(rd) // 2
    xyz = np.empty(3 * n, np.float64)
    lib().orc_radec_to_xyz(_dp(rd), n, _dp(xyz))
    return xyz.reshape(3, n)


def count_xyz(xyz_a: np.ndarray, xyz_b: np.ndarray | None, edges_deg: np.ndarray,
              is_auto: bool, nthreads: int = 0) -> np.ndarray:
    """Exact DD/RR (auto: pairs i<j, n(n-1)/2 of them) or DR (cross: n_a n_b
    pairs) counts, Sec. 2.  Returns K+2 slots: underflow, bins 1..K, overflow."""
    K = len(edges_deg) - 1
    c = chord2(edges_deg)
    A = np.ascontiguousarray(xyz_a, np.float64)
    B = A if (is_auto or xyz_b is None) else np.ascontiguousarray(xyz_b, np.float64)
    out = np.zeros(K + 2, np.uint64)
    rc = lib().orc_count(_dp(A), A.shape[-1], _dp(B), B.shape[-1], _dp(c), K,
                         1 if is_auto else 0, _up(out), nthreads)
    if rc != 0:
        raise MemoryError("oracle allocation failed")
    return out


def count(ra_dec_a: np.ndarray, ra_dec_b: np.ndarray | None, edges_deg: np.ndarray,
          is_auto: bool, nthreads: int = 0) -> np.ndarray:
    """count_xyz on the oracle's own unit vectors."""
    A = radec_to_xyz(ra_dec_a)
    B = None if (is_auto or ra_dec_b is None) else radec_to_xyz(ra_dec_b)
    return count_xyz(A, B, edges_deg, is_auto, nthreads)


def ambiguity_tau(c: np.ndarray) -> np.ndarray:
    """Width around each squared-chord edge inside which moving every
    component of both unit vectors by up to 8 ulps (the device's RA/Dec
    conversion stays within 4 ulps of the host's) can move a pair across the
    edge.  With every component of magnitude below 1 an ulp is at most 2^-53,
    so the difference vector changes by |D| <= sqrt(3) 16 2^-53 = sqrt(3) 2^-49,
    and s = |d|^2 by at most 2 |d| |D| + |D|^2 = 2 sqrt(3 s) 2^-49 + 3 2^-98,
    plus the FP64 roundings of the two evaluations of s (each of d_i, its
    square and the two sums rounds once: about 5 2^-53 s each, 10 2^-53 s
    together).  Taken as 2^-47 (sqrt(c) + c/4) + 2^-90, which covers those
    terms (2 sqrt(3) 2^-49 < 2^-47 and 10 2^-53 < 2^-47 / 4) with about 13% to
    spare at the sqrt(c) term; the pin in
    tests/oracle_pins.py perturbs pairs placed around every edge and checks
    both that every slot change is flagged and that the width is no more than
    about twice what the perturbations reach."""
    return 2.0 ** -47 * (np.sqrt(c) + 0.25 * c) + 2.0 ** -90


def count_ambiguous_xyz(xyz_a, xyz_b, edges_deg, is_auto, nthreads: int = 0,
                        tau: np.ndarray | None = None) -> int:
    """Pairs whose FP64 squared chord lies within tau_k (default
    ambiguity_tau) of some edge c_k."""
    K = len(edges_deg) - 1
    c = chord2(edges_deg)
    tau = ambiguity_tau(c) if tau is None else np.ascontiguousarray(tau, np.float64)
    A = np.ascontiguousarray(xyz_a, np.float64)
    B = A if (is_auto or xyz_b is None) else np.ascontiguousarray(xyz_b, np.float64)
    out = np.zeros(1, np.uint64)
    lib().orc_count_ambiguous(_dp(A), A.shape[-1], _dp(B), B.shape[-1], _dp(c), _dp(tau),
                              K, 1 if is_auto else 0, _up(out), nthreads)
    return int(out[0])


def ls(DD, DR, RR, n_d: int, n_r: int) -> np.ndarray:
    """Landy-Szalay w(theta), Eq. 2, with normalised counts."""
    DD, DR, RR = (np.ascontiguousarray(x, np.uint64) for x in (DD, DR, RR))
    K = len(DD) - 2
    w = np.empty(K, np.float64)
    if lib().orc_ls(_up(DD), _up(DR), _up(RR), n_d, n_r, K, _dp(w)) != 0:
        raise ValueError("bad sizes")
    return w


def estimator(DD, DR, RR, n_d: int, n_r: int, name: str) -> np.ndarray:
    """Other w(theta) estimators over the same counts (Sec. 2 leaves the choice
    of estimator open), on counts normalised by their pair totals as in Eq. 2:
    natural (Peebles & Hauser 1974) dd/rr - 1; Davis & Peebles (1983) dd/dr - 1;
    Hamilton (1993) dd rr / dr^2 - 1; Landy & Szalay (1993) (dd - 2dr + rr)/rr.
    A bin whose denominator count is 0 gives NaN."""
    DD, DR, RR = (np.asarray(x, np.uint64)[1:-1].astype(np.float64) for x in (DD, DR, RR))
    dd = DD / (n_d * (n_d - 1) / 2.0)
    dr = DR / (float(n_d) * float(n_r))
    rr = RR / (n_r * (n_r - 1) / 2.0)
    with np.errstate(divide="ignore", invalid="ignore"):
        if name == "landy_szalay":
            w = ((dd - 2.0 * dr) + rr) / rr
            den = RR
        elif name == "natural":
            w, den = dd / rr - 1.0, RR
        elif name == "davis_peebles":
            w, den = dd / dr - 1.0, DR
        elif name == "hamilton":
            w, den = (dd * rr) / (dr * dr) - 1.0, DR
        else:
            raise ValueError(name)
    return np.where(den > 0, w, np.nan)


def count_regions(xyz_d, labels_d, xyz_r, labels_r, edges_deg, n_regions: int) -> np.ndarray:
    """DD, DR, RR split by region pair, by the definition: the pairs of Sec. 2
    with one point in region a and the other in region b.  Layout
    [DD, DR, RR][a][b][slot]; DD and RR fill a <= b only (a = b: both points
    in a), DR every (a, b) with the data point in a."""
    K = len(edges_deg) - 1
    R = n_regions
    out = np.zeros((3, R, R, K + 2), np.uint64)
    D = [np.ascontiguousarray(xyz_d[:, labels_d == a]) for a in range(R)]
    Q = [np.ascontiguousarray(xyz_r[:, labels_r == a]) for a in range(R)]
    for a in range(R):
        for b in range(R):
            out[1, a, b] = count_xyz(D[a], Q[b], edges_deg, False)
            if b < a:
                continue
            for kind, S in ((0, D), (2, Q)):
                if a == b:
                    out[kind, a, a] = count_xyz(S[a], None, edges_deg, True)
                else:
                    out[kind, a, b] = count_xyz(S[a], S[b], edges_deg, False)
    return out


def jackknife(region_counts: np.ndarray, sizes: np.ndarray, n_regions: int):
    """Delete-one jackknife of Eq. 2 (the error estimate Sec. 4 points at):
    sample k keeps the region pairs (a, b) with a != k and b != k and the
    points outside region k; returns w (all regions), w_k (R x K) and
    cov = (R-1)/R sum_k (w_k - mean)(w_k - mean)^T."""
    R = n_regions
    c = np.asarray(region_counts, np.uint64)
    nd, nr = np.asarray(sizes[:R], np.int64), np.asarray(sizes[R:], np.int64)
    full = [c[kind].sum(axis=(0, 1), dtype=np.uint64) for kind in range(3)]
    w = ls(full[0], full[1], full[2], int(nd.sum()), int(nr.sum()))
    K = len(w)
    w_k = np.empty((R, K))
    for k in range(R):
        keep = np.ones(R, bool)
        keep[k] = False
        s = [c[kind][np.ix_(keep, keep)].sum(axis=(0, 1), dtype=np.uint64) for kind in range(3)]
        w_k[k] = ls(s[0], s[1], s[2], int(nd.sum() - nd[k]), int(nr.sum() - nr[k]))
    mean = w_k.mean(axis=0)
    dev = w_k - mean
    cov = (R - 1) / R * (dev.T @ dev)
    return w, w_k, cov


def ls_cross(D1D2, D1R2, R1D2, R1R2, n_d1, n_d2, n_r1, n_r2) -> np.ndarray:
    """Cross-correlation form of Eq. 2 between two catalogues."""
    arrs = [np.ascontiguousarray(x, np.uint64) for x in (D1D2, D1R2, R1D2, R1R2)]
    K = len(arrs[0]) - 2
    w = np.empty(K, np.float64)
    if lib().orc_ls_cross(*[_up(a) for a in arrs], n_d1, n_d2, n_r1, n_r2, K, _dp(w)) != 0:
        raise ValueError("bad sizes")
    return w


def wtheta(data: np.ndarray, rand: np.ndarray, edges_deg: np.ndarray, nthreads: int = 0):
    """DD, DR, RR and w for one data/random pair of catalogues."""
    D, R = radec_to_xyz(data), radec_to_xyz(rand)
    DD = count_xyz(D, None, edges_deg, True, nthreads)
    DR = count_xyz(D, R, edges_deg, False, nthreads)
    RR = count_xyz(R, None, edges_deg, True, nthreads)
    return DD, DR, RR, ls(DD, DR, RR, D.shape[1], R.shape[1])
