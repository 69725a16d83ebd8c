"""Thin Python binding of libwtheta (include/wtheta.h), same names as the C ABI.

Argument marshalling only: device arrays are torch CUDA tensors (their
pointers are passed), host arrays are numpy arrays, streams are
``torch.cuda.Stream`` objects, raw ``cudaStream_t`` integers, or ``None`` for
torch's current stream.  Every computation happens in libwtheta's CUDA
kernels; if the library is missing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
import re
import threading

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libwtheta.so")
HEADER = os.path.join(os.path.dirname(_PKG), "include", "wtheta.h")

WTHETA_OK = 0
STATUS = {0: "OK", -1: "EINVAL", -2: "ENOMEM", -3: "ECUDA", -4: "ETIMEOUT", -5: "EBUDGET",
          -8: "EBUSY", -9: "ECANCELED",
          -6: "EDEVICE", -7: "ESIZE"}
NOALLOC_MAX_POINTS, NOALLOC_TILE = 262144, 1024
BINS_LINEAR, BINS_LN, BINS_LOG10 = 0, 1, 2
DERR_NONFINITE, DERR_DEC_RANGE, DERR_NOT_UNIT = 1, 2, 4
STAT_PAIRS, STAT_RECHECK, STAT_TILES, STAT_SKIPPED, STAT_SPAN, NSTATS = 0, 1, 2, 3, 4, 5

_lock = threading.Lock()
_lib = None


class WthetaError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%d)" % (where, STATUS.get(status, "?"), status))


class wtheta_tune(ctypes.Structure):
    _fields_ = [("threads", ctypes.c_int32), ("points_per_thread", ctypes.c_int32),
                ("hist_mode", ctypes.c_int32), ("j_per_screen", ctypes.c_int32),
                ("deferred", ctypes.c_int32), ("blocks_per_sm", ctypes.c_int32),
                ("skip_far", ctypes.c_int32),
                ("span_bins", ctypes.c_int32)]


class wtheta_catalog_pair(ctypes.Structure):
    _fields_ = [("data", ctypes.c_void_p), ("n_data", ctypes.c_int64),
                ("rand", ctypes.c_void_p), ("n_rand", ctypes.c_int64)]


class wtheta_batch_info_t(ctypes.Structure):
    _fields_ = [("tune", wtheta_tune), ("n_items", ctypes.c_int64), ("pairs", ctypes.c_int64),
                ("evaluated_pairs", ctypes.c_int64), ("n_counts", ctypes.c_int32),
                ("graph_kernels", ctypes.c_int32), ("autotune_ms", ctypes.c_float),
                ("autotuned", ctypes.c_int32)]


REQ_AUTO, REQ_CROSS = 0, 1
EST_LANDY_SZALAY, EST_NATURAL, EST_DAVIS_PEEBLES, EST_HAMILTON = 0, 1, 2, 3
RS_QUEUED, RS_UPLOADING, RS_COUNTING, RS_FINISHING, RS_DONE, RS_FAILED = range(6)


class wtheta_request(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("data", ctypes.c_void_p), ("n_data", ctypes.c_int64),
                ("rand", ctypes.c_void_p), ("n_rand", ctypes.c_int64),
                ("data2", ctypes.c_void_p), ("n_data2", ctypes.c_int64),
                ("rand2", ctypes.c_void_p), ("n_rand2", ctypes.c_int64)]


class wtheta_request_info(ctypes.Structure):
    _fields_ = [("state", ctypes.c_int32), ("status", ctypes.c_int32),
                ("t_submit", ctypes.c_double), ("t_admit", ctypes.c_double),
                ("t_done", ctypes.c_double), ("pairs", ctypes.c_int64),
                ("n_counts", ctypes.c_int32)]


class wtheta_server_stats_t(ctypes.Structure):
    _fields_ = [(n, ctypes.c_int64) for n in ("rounds", "completed", "queued", "active", "items",
                                              "resident_bytes", "kernels")]


def declared_functions() -> list:
    """Names of the functions include/wtheta.h declares."""
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(wtheta_[a-z0-9_]+)\s*\(", text)))


def lib() -> ctypes.CDLL:
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    "libwtheta.so is not built (%s); run python -m paper_1208_3658_gb300.build"
                    % LIB_PATH)
            L = ctypes.CDLL(LIB_PATH)
            vp, dp = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)
            i64, i32, u32p = ctypes.c_int64, ctypes.c_int32, ctypes.POINTER(ctypes.c_uint32)
            u64p = ctypes.POINTER(ctypes.c_uint64)
            i64p = ctypes.POINTER(ctypes.c_int64)
            L.wtheta_strerror.restype = ctypes.c_char_p
            L.wtheta_strerror.argtypes = [ctypes.c_int]
            L.wtheta_edges.argtypes = [ctypes.c_double, ctypes.c_double, i32, i32, dp]
            L.wtheta_chord2_edges.argtypes = [dp, i32, dp]
            L.wtheta_guard_band.argtypes = [dp, i32, u32p, u32p, dp]
            L.wtheta_count.argtypes = [vp, i64, vp, i64, dp, i32, i32, vp, vp]
            L.wtheta_count_xyz.argtypes = [vp, i64, vp, i64, dp, i32, i32, vp, vp]
            L.wtheta_count_ex.argtypes = [vp, i64, vp, i64, i32, dp, i32, i32, vp,
                                          ctypes.POINTER(wtheta_tune), vp, vp]
            L.wtheta_radec_to_xyz.argtypes = [vp, i64, vp, vp]
            L.wtheta_get_error.argtypes = [vp, u32p]
            L.wtheta_ls.argtypes = [u64p, u64p, u64p, i64, i64, i32, dp]
            L.wtheta_ls_cross.argtypes = [u64p, u64p, u64p, u64p, i64, i64, i64, i64, i32, dp]
            L.wtheta_estimate.argtypes = [u64p, u64p, u64p, i64, i64, i32, i32, dp]
            L.wtheta_count_regions.argtypes = [vp, i64, vp, vp, i64, vp, i32, dp, i32, i32, vp,
                                               i64p, vp]
            L.wtheta_jackknife.argtypes = [u64p, i64p, i32, i32, dp, dp, dp]
            L.wtheta_probe_shared_atomics.argtypes = [i32, dp]
            L.wtheta_inject_alloc_failure.argtypes = [i32]
            L.wtheta_correlate.argtypes = [dp, i64, dp, i64, dp, i32, u64p, dp, vp]
            L.wtheta_count_xyz_noalloc.argtypes = [vp, i64, vp, i64, dp, i32, i32, vp, vp]
            L.wtheta_count_wtheta.argtypes = [vp, i64, vp, i64, i32, dp, i32, vp,
                                              ctypes.POINTER(wtheta_tune), vp, vp]
            L.wtheta_batch_plan.argtypes = [ctypes.POINTER(wtheta_catalog_pair), i32, dp, i32,
                                            ctypes.POINTER(wtheta_tune), vp,
                                            ctypes.POINTER(ctypes.c_void_p)]
            L.wtheta_batch_plan_ex.argtypes = [ctypes.POINTER(wtheta_catalog_pair), i32, i32, dp,
                                               i32, ctypes.POINTER(wtheta_tune), vp,
                                               ctypes.POINTER(ctypes.c_void_p)]
            L.wtheta_batch_run.argtypes = [vp, vp, vp]
            L.wtheta_batch_info.argtypes = [vp, ctypes.POINTER(wtheta_batch_info_t)]
            L.wtheta_batch_free.argtypes = [vp]
            L.wtheta_server_create.argtypes = [dp, i32, ctypes.c_size_t, i32,
                                               ctypes.POINTER(wtheta_tune),
                                               ctypes.POINTER(ctypes.c_void_p)]
            L.wtheta_server_submit.argtypes = [vp, ctypes.POINTER(wtheta_request),
                                               ctypes.POINTER(ctypes.c_uint64)]
            L.wtheta_server_wait.argtypes = [vp, ctypes.c_uint64, i64,
                                             ctypes.POINTER(ctypes.c_int32), u64p, dp]
            L.wtheta_server_request_info.argtypes = [vp, ctypes.c_uint64,
                                                     ctypes.POINTER(wtheta_request_info)]
            L.wtheta_server_release.argtypes = [vp, ctypes.c_uint64]
            L.wtheta_server_cancel.argtypes = [vp, ctypes.c_uint64]
            L.wtheta_server_stats.argtypes = [vp, ctypes.POINTER(wtheta_server_stats_t)]
            L.wtheta_server_destroy.argtypes = [vp]
            L.wtheta_shard_rows.argtypes = [i64, i64, i32, i32, i32,
                                            ctypes.POINTER(ctypes.c_int64),
                                            ctypes.POINTER(ctypes.c_int64)]
            L.wtheta_count_shard.argtypes = [vp, i64, vp, i64, dp, i32, i32, i32, i32, vp, vp]
            L.wtheta_count_wtheta_shard.argtypes = [vp, i64, vp, i64, i32, dp, i32, i32, i32, vp,
                                                    ctypes.POINTER(wtheta_tune), vp, vp]
            L.wtheta_shard_weights.argtypes = [u64p, i64, i32, i32,
                                               ctypes.POINTER(ctypes.c_int64),
                                               ctypes.POINTER(ctypes.c_int64)]
            L.wtheta_kernel_launches.argtypes = []
            L.wtheta_kernel_launches.restype = ctypes.c_uint64
            _lib = L
    return _lib


# ---------------------------------------------------------------------------
# marshalling helpers
# ---------------------------------------------------------------------------
def _check(rc: int, where: str):
    if rc != WTHETA_OK:
        raise WthetaError(rc, where)


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _dev_ptr(t, dtype_size=8, name="array"):
    """Device pointer of a contiguous CUDA tensor (or None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    if t.element_size() != dtype_size:
        raise ValueError("%s must have %d-byte elements" % (name, dtype_size))
    return t.data_ptr()


def _host_f64(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _host_u64(a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    return a, a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _n_points(t, per_point, name="coordinates"):
    """Points in a coordinate tensor, after checking its layout.  Interleaved
    RA/Dec (per_point 2) is 1-D [ra0, dec0, ra1, ...] or (n, 2); unit vectors
    (per_point 3) are SoA, (3, n) or 1-D [x0.., y0.., z0..].  The library
    reads unit vectors with stride n, so a row-major (n, 3) array would give
    wrong counts: it is refused, as are data that are not float64 and sizes
    that are not whole points."""
    if t is None:
        return 0
    if str(t.dtype) != "torch.float64":
        raise ValueError("%s must be float64, not %s" % (name, t.dtype))
    if per_point == 3:
        ok = t.dim() == 1 or (t.dim() == 2 and t.shape[0] == 3)
        layout = "SoA unit vectors of shape (3, n) or 1-D [x.., y.., z..]"
    else:
        ok = t.dim() == 1 or (t.dim() == 2 and t.shape[1] == 2)
        layout = "interleaved RA/Dec, 1-D [ra0, dec0, ...] or shape (n, 2)"
    if not ok or t.numel() % per_point:
        raise ValueError("%s must be %s, not shape %s" % (name, layout, tuple(t.shape)))
    return t.numel() // per_point


def _slots(t, n, name="counts"):
    """Checks that an output tensor holds at least n 8-byte slots (the library
    writes n of them)."""
    if t is None or isinstance(t, int):
        return
    if t.numel() < n:
        raise ValueError("%s must hold at least %d slots, not %d" % (name, n, t.numel()))


# ---------------------------------------------------------------------------
# entry points
# ---------------------------------------------------------------------------
def wtheta_strerror(status: int) -> str:
    return lib().wtheta_strerror(status).decode()


def wtheta_edges(lo_deg: float, hi_deg: float, n_bins: int, mode: int = BINS_LN) -> np.ndarray:
    e = np.empty(n_bins + 1, np.float64)
    _check(lib().wtheta_edges(lo_deg, hi_deg, n_bins, mode, _host_f64(e)[1]), "wtheta_edges")
    return e


def wtheta_chord2_edges(edges_deg) -> np.ndarray:
    e, ep = _host_f64(edges_deg)
    c = np.empty_like(e)
    _check(lib().wtheta_chord2_edges(ep, len(e) - 1, _host_f64(c)[1]), "wtheta_chord2_edges")
    return c


def wtheta_guard_band(edges_deg):
    e, ep = _host_f64(edges_deg)
    lo = np.empty(len(e), np.uint32)
    hi = np.empty(len(e), np.uint32)
    g = np.empty(len(e), np.float64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    _check(lib().wtheta_guard_band(ep, len(e) - 1, lo.ctypes.data_as(u32p),
                                   hi.ctypes.data_as(u32p), _host_f64(g)[1]),
           "wtheta_guard_band")
    return lo, hi, g


def wtheta_count(ra_dec_a, ra_dec_b, edges_deg, is_auto: bool, counts, stream=None,
                 n_a: int | None = None, n_b: int | None = None):
    """ra_dec_*: CUDA float64 tensors [ra0, dec0, ...] (ra_dec_b None for auto);
    counts: CUDA 8-byte tensor of K+2 slots, overwritten."""
    e, ep = _host_f64(edges_deg)
    na = _n_points(ra_dec_a, 2, "ra_dec_a") if n_a is None else n_a
    nb = (na if is_auto else _n_points(ra_dec_b, 2, "ra_dec_b")) if n_b is None else n_b
    _slots(counts, len(e) + 1)
    _check(lib().wtheta_count(_dev_ptr(ra_dec_a), na, _dev_ptr(ra_dec_b), nb, ep, len(e) - 1,
                              1 if is_auto else 0, _dev_ptr(counts), _stream(stream)),
           "wtheta_count")


def wtheta_count_xyz(xyz_a, xyz_b, edges_deg, is_auto: bool, counts, stream=None,
                     n_a: int | None = None, n_b: int | None = None):
    """xyz_*: CUDA float64 tensors, SoA (3, n) contiguous."""
    e, ep = _host_f64(edges_deg)
    na = _n_points(xyz_a, 3, "xyz_a") if n_a is None else n_a
    nb = (na if is_auto else _n_points(xyz_b, 3, "xyz_b")) if n_b is None else n_b
    _slots(counts, len(e) + 1)
    _check(lib().wtheta_count_xyz(_dev_ptr(xyz_a), na, _dev_ptr(xyz_b), nb, ep, len(e) - 1,
                                  1 if is_auto else 0, _dev_ptr(counts), _stream(stream)),
           "wtheta_count_xyz")


def wtheta_shard_rows(n_a: int, n_b: int, is_auto: bool, shard: int, n_shards: int):
    r0, r1 = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().wtheta_shard_rows(n_a, n_b, 1 if is_auto else 0, shard, n_shards,
                                   ctypes.byref(r0), ctypes.byref(r1)), "wtheta_shard_rows")
    return int(r0.value), int(r1.value)


def wtheta_count_shard(ra_dec_a, ra_dec_b, edges_deg, is_auto: bool, shard: int, n_shards: int,
                       counts, stream=None):
    e, ep = _host_f64(edges_deg)
    na = _n_points(ra_dec_a, 2, "ra_dec_a")
    nb = na if is_auto else _n_points(ra_dec_b, 2, "ra_dec_b")
    _slots(counts, len(e) + 1)
    _check(lib().wtheta_count_shard(_dev_ptr(ra_dec_a), na, _dev_ptr(ra_dec_b), nb, ep,
                                    len(e) - 1, 1 if is_auto else 0, shard, n_shards,
                                    _dev_ptr(counts), _stream(stream)), "wtheta_count_shard")


def wtheta_count_xyz_noalloc(xyz_a, xyz_b, edges_deg, is_auto: bool, counts, stream=None):
    """wtheta_count_xyz without any device allocation: the library's fixed
    scratch array is used instead (see include/wtheta.h for its limit)."""
    e, ep = _host_f64(edges_deg)
    for name, t in (("xyz_a", xyz_a), ("xyz_b", None if is_auto else xyz_b)):
        if t is None:
            continue
        if getattr(t, "dim", lambda: 0)() != 2 or t.shape[0] != 3:
            raise ValueError("%s must have shape (3, n): SoA unit vectors" % name)
        if str(t.dtype) != "torch.float64":
            raise ValueError("%s must be float64" % name)
    if counts is None or counts.numel() != len(e) + 1:
        raise ValueError("counts must have len(edges) + 1 = K + 2 slots")
    na = _n_points(xyz_a, 3)
    nb = na if is_auto else _n_points(xyz_b, 3)
    _check(lib().wtheta_count_xyz_noalloc(_dev_ptr(xyz_a), na, _dev_ptr(xyz_b), nb, ep, len(e) - 1,
                                          1 if is_auto else 0, _dev_ptr(counts), _stream(stream)),
           "wtheta_count_xyz_noalloc")


def _tune_struct(tune):
    if not tune:
        return None
    return wtheta_tune(int(tune.get("threads", 0)), int(tune.get("points_per_thread", 0)),
                       int(tune.get("hist_mode", 0)), int(tune.get("j_per_screen", 0)),
                       int(tune.get("deferred", 0)), int(tune.get("blocks_per_sm", 0)),
                       int(tune.get("skip_far", 0)), int(tune.get("span_bins", 0)))


class BatchPlan:
    """A wtheta_batch_plan handle; keeps the catalogue tensors it borrows alive."""

    def __init__(self, handle, tensors, n_cats, n_bins):
        self.handle = handle
        self._tensors = tensors
        self.n_cats = n_cats
        self.n_bins = n_bins

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().wtheta_batch_free(self.handle)
            except Exception:
                pass
            self.handle = None


def wtheta_batch_plan(cats, edges_deg, tune: dict | None = None, stream=None,
                      coords_are_xyz: bool = False) -> BatchPlan:
    """cats: list of (data, rand) CUDA float64 tensors: interleaved RA/Dec, or
    SoA (3, n) unit vectors when coords_are_xyz (wtheta_batch_plan_ex)."""
    e, ep = _host_f64(edges_deg)
    per = 3 if coords_are_xyz else 2
    arr = (wtheta_catalog_pair * len(cats))()
    keep = []
    for i, (d, r) in enumerate(cats):
        nd, nr = _n_points(d, per, "data %d" % i), _n_points(r, per, "rand %d" % i)
        arr[i] = wtheta_catalog_pair(_dev_ptr(d), nd, _dev_ptr(r), nr)
        keep += [d, r]
    t = _tune_struct(tune)
    h = ctypes.c_void_p()
    tp = ctypes.byref(t) if t is not None else None
    if coords_are_xyz:
        _check(lib().wtheta_batch_plan_ex(arr, len(cats), 1, ep, len(e) - 1, tp, _stream(stream),
                                          ctypes.byref(h)), "wtheta_batch_plan_ex")
    else:
        _check(lib().wtheta_batch_plan(arr, len(cats), ep, len(e) - 1, tp, _stream(stream),
                                       ctypes.byref(h)), "wtheta_batch_plan")
    return BatchPlan(h, keep, len(cats), len(e) - 1)


def wtheta_batch_run(plan: BatchPlan, counts, stream=None):
    """counts: CUDA 8-byte tensor of n_cats x 3 x (K+2) slots."""
    _slots(counts, plan.n_cats * 3 * (plan.n_bins + 2))
    _check(lib().wtheta_batch_run(plan.handle, _dev_ptr(counts), _stream(stream)),
           "wtheta_batch_run")


def wtheta_batch_info(plan: BatchPlan) -> dict:
    info = wtheta_batch_info_t()
    _check(lib().wtheta_batch_info(plan.handle, ctypes.byref(info)), "wtheta_batch_info")
    t = info.tune
    return dict(tune=dict(threads=t.threads, points_per_thread=t.points_per_thread,
                          hist_mode=t.hist_mode, j_per_screen=t.j_per_screen,
                          deferred=t.deferred, blocks_per_sm=t.blocks_per_sm,
                          skip_far=t.skip_far, span_bins=t.span_bins),
                n_items=info.n_items, pairs=info.pairs, evaluated_pairs=info.evaluated_pairs,
                n_counts=info.n_counts, graph_kernels=info.graph_kernels,
                autotune_ms=info.autotune_ms, autotuned=bool(info.autotuned))


def wtheta_batch_free(plan: BatchPlan):
    if plan.handle:
        _check(lib().wtheta_batch_free(plan.handle), "wtheta_batch_free")
        plan.handle = None


class Server:
    """A wtheta_server handle (one edge set)."""

    def __init__(self, handle, n_bins):
        self.handle = handle
        self.n_bins = n_bins

    def __del__(self):
        if getattr(self, "handle", None):
            try:
                lib().wtheta_server_destroy(self.handle)
            except Exception:
                pass
            self.handle = None


def wtheta_server_create(edges_deg, hbm_budget_bytes: int, max_active: int = 0,
                         tune: dict | None = None) -> Server:
    e, ep = _host_f64(edges_deg)
    t = _tune_struct(tune)
    h = ctypes.c_void_p()
    _check(lib().wtheta_server_create(ep, len(e) - 1, int(hbm_budget_bytes), int(max_active),
                                      ctypes.byref(t) if t is not None else None, ctypes.byref(h)),
           "wtheta_server_create")
    return Server(h, len(e) - 1)


def _host_points(a, name):
    """Points of a host array of interleaved RA/Dec, 1-D [ra0, dec0, ...] or
    (n, 2): its elements over 2 (not its length, which is n for (n, 2))."""
    if a.ndim > 2 or (a.ndim == 2 and a.shape[1] != 2) or a.size % 2:
        raise ValueError("%s must be interleaved RA/Dec, 1-D [ra0, dec0, ...] or shape (n, 2), "
                         "not shape %s" % (name, a.shape))
    return a.size // 2


def wtheta_server_submit(srv: Server, data, rand, data2=None, rand2=None) -> int:
    """Host numpy arrays of interleaved RA/Dec; auto if data2 is None, else cross."""
    arrs = [np.ascontiguousarray(x, np.float64) if x is not None else None
            for x in (data, rand, data2, rand2)]
    n = [_host_points(x, nm) if x is not None else 0
         for x, nm in zip(arrs, ("data", "rand", "data2", "rand2"))]
    kind = REQ_AUTO if data2 is None else REQ_CROSS
    q = wtheta_request(kind,
                       arrs[0].ctypes.data, n[0], arrs[1].ctypes.data, n[1],
                       arrs[2].ctypes.data if arrs[2] is not None else None, n[2],
                       arrs[3].ctypes.data if arrs[3] is not None else None, n[3])
    rid = ctypes.c_uint64()
    _check(lib().wtheta_server_submit(srv.handle, ctypes.byref(q), ctypes.byref(rid)),
           "wtheta_server_submit")
    return int(rid.value)


def wtheta_server_wait(srv: Server, req_id: int, timeout_ms: int = -1):
    """Returns (done, counts (n_counts, K+2) uint64 or None, w or None).
    timeout_ms < 0 waits without limit (in 1 s slices)."""
    K = srv.n_bins
    counts = np.zeros(4 * (K + 2), np.uint64)
    w = np.empty(K, np.float64)
    done = ctypes.c_int32(0)
    while True:
        t = 1000 if timeout_ms < 0 else timeout_ms
        rc = lib().wtheta_server_wait(srv.handle, req_id, t, ctypes.byref(done),
                                      _host_u64(counts)[1], _host_f64(w)[1])
        if rc == -4 and timeout_ms < 0:
            continue
        _check(rc, "wtheta_server_wait")
        break
    if not done.value:
        return False, None, None
    n = wtheta_server_request_info(srv, req_id)["n_counts"]
    return True, counts[: n * (K + 2)].reshape(n, K + 2), w


def wtheta_server_request_info(srv: Server, req_id: int) -> dict:
    info = wtheta_request_info()
    _check(lib().wtheta_server_request_info(srv.handle, req_id, ctypes.byref(info)),
           "wtheta_server_request_info")
    return {k: getattr(info, k) for k, _ in wtheta_request_info._fields_}


def wtheta_server_cancel(srv: Server, req_id: int):
    _check(lib().wtheta_server_cancel(srv.handle, req_id), "wtheta_server_cancel")


def wtheta_server_release(srv: Server, req_id: int):
    _check(lib().wtheta_server_release(srv.handle, req_id), "wtheta_server_release")


def wtheta_server_stats(srv: Server) -> dict:
    st = wtheta_server_stats_t()
    _check(lib().wtheta_server_stats(srv.handle, ctypes.byref(st)), "wtheta_server_stats")
    return {k: getattr(st, k) for k, _ in wtheta_server_stats_t._fields_}


def wtheta_server_destroy(srv: Server):
    if srv.handle:
        _check(lib().wtheta_server_destroy(srv.handle), "wtheta_server_destroy")
        srv.handle = None


def wtheta_count_ex(coords_a, coords_b, coords_are_xyz: bool, edges_deg, is_auto: bool, counts,
                    tune: dict | None = None, stats=None, stream=None):
    e, ep = _host_f64(edges_deg)
    per = 3 if coords_are_xyz else 2
    na = _n_points(coords_a, per, "coords_a")
    nb = na if is_auto else _n_points(coords_b, per, "coords_b")
    _slots(counts, len(e) + 1)
    _slots(stats, NSTATS, "stats")
    t = _tune_struct(tune)
    _check(lib().wtheta_count_ex(_dev_ptr(coords_a), na, _dev_ptr(coords_b), nb,
                                 1 if coords_are_xyz else 0, ep, len(e) - 1, 1 if is_auto else 0,
                                 _dev_ptr(counts), ctypes.byref(t) if t is not None else None,
                                 _dev_ptr(stats), _stream(stream)), "wtheta_count_ex")


def wtheta_count_wtheta(coords_d, coords_r, coords_are_xyz: bool, edges_deg, counts,
                        tune: dict | None = None, stats=None, stream=None):
    """DD, DR, RR of one w(theta) into counts (device, 3 x (K+2) int64 viewed
    as uint64), in one persistent launch."""
    e, ep = _host_f64(edges_deg)
    per = 3 if coords_are_xyz else 2
    t = _tune_struct(tune)
    nd, nr = _n_points(coords_d, per, "coords_d"), _n_points(coords_r, per, "coords_r")
    _slots(counts, 3 * (len(e) + 1))
    _slots(stats, NSTATS, "stats")
    _check(lib().wtheta_count_wtheta(_dev_ptr(coords_d), nd, _dev_ptr(coords_r), nr,
                                     1 if coords_are_xyz else 0, ep, len(e) - 1, _dev_ptr(counts),
                                     ctypes.byref(t) if t is not None else None, _dev_ptr(stats),
                                     _stream(stream)), "wtheta_count_wtheta")


def wtheta_count_wtheta_shard(coords_d, coords_r, coords_are_xyz: bool, edges_deg, shard: int,
                              n_shards: int, counts, tune: dict | None = None, stats=None,
                              stream=None):
    """Shard `shard` of n_shards of one w(theta): DD, DR, RR of the pairs whose
    first point lies in the shard's tile rows (balanced by kept tile pairs)."""
    e, ep = _host_f64(edges_deg)
    per = 3 if coords_are_xyz else 2
    t = _tune_struct(tune)
    nd, nr = _n_points(coords_d, per, "coords_d"), _n_points(coords_r, per, "coords_r")
    _slots(counts, 3 * (len(e) + 1))
    _slots(stats, NSTATS, "stats")
    _check(lib().wtheta_count_wtheta_shard(_dev_ptr(coords_d), nd, _dev_ptr(coords_r), nr,
                                           1 if coords_are_xyz else 0, ep, len(e) - 1, shard,
                                           n_shards, _dev_ptr(counts),
                                           ctypes.byref(t) if t is not None else None,
                                           _dev_ptr(stats), _stream(stream)),
           "wtheta_count_wtheta_shard")


def wtheta_shard_weights(weights, shard: int, n_shards: int):
    """[row_begin, row_end) of shard among n_shards contiguous weighted ranges."""
    w, wp = _host_u64(weights)
    r0, r1 = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().wtheta_shard_weights(wp, len(w), shard, n_shards, ctypes.byref(r0),
                                      ctypes.byref(r1)), "wtheta_shard_weights")
    return int(r0.value), int(r1.value)


def wtheta_radec_to_xyz(ra_dec, xyz, stream=None):
    n = _n_points(ra_dec, 2, "ra_dec")
    _n_points(xyz, 3, "xyz")
    _slots(xyz, 3 * n, "xyz")
    _check(lib().wtheta_radec_to_xyz(_dev_ptr(ra_dec), n, _dev_ptr(xyz), _stream(stream)),
           "wtheta_radec_to_xyz")


def wtheta_kernel_launches() -> int:
    return int(lib().wtheta_kernel_launches())


def wtheta_get_error(stream=None) -> int:
    code = ctypes.c_uint32(0)
    _check(lib().wtheta_get_error(_stream(stream), ctypes.byref(code)), "wtheta_get_error")
    return int(code.value)


def wtheta_ls(DD, DR, RR, n_d: int, n_r: int) -> np.ndarray:
    (DD, p1), (DR, p2), (RR, p3) = _host_u64(DD), _host_u64(DR), _host_u64(RR)
    K = len(DD) - 2
    w = np.empty(K, np.float64)
    _check(lib().wtheta_ls(p1, p2, p3, n_d, n_r, K, _host_f64(w)[1]), "wtheta_ls")
    return w


def wtheta_estimate(DD, DR, RR, n_d: int, n_r: int, estimator: int) -> np.ndarray:
    (DD, p1), (DR, p2), (RR, p3) = _host_u64(DD), _host_u64(DR), _host_u64(RR)
    K = len(DD) - 2
    w = np.empty(K, np.float64)
    _check(lib().wtheta_estimate(p1, p2, p3, n_d, n_r, K, estimator, _host_f64(w)[1]),
           "wtheta_estimate")
    return w


def wtheta_count_regions(coords_d, labels_d, coords_r, labels_r, edges, n_regions: int, counts,
                         coords_are_xyz: bool = False, stream=None) -> np.ndarray:
    """Region-pair DD, DR, RR into counts (device tensor, 3 x R x R x (K+2)
    int64 viewed as uint64); returns the region sizes (2 x R int64)."""
    e = np.ascontiguousarray(edges, np.float64)
    K = len(e) - 1
    per = 3 if coords_are_xyz else 2
    n_d = _n_points(coords_d, per, "coords_d")
    n_r = _n_points(coords_r, per, "coords_r")
    _slots(counts, 3 * n_regions * n_regions * (K + 2))
    sizes = np.zeros(2 * n_regions, np.int64)
    _check(lib().wtheta_count_regions(_dev_ptr(coords_d), n_d, _dev_ptr(labels_d, 4, "labels_d"),
                                      _dev_ptr(coords_r), n_r, _dev_ptr(labels_r, 4, "labels_r"),
                                      1 if coords_are_xyz else 0, _host_f64(e)[1], K, n_regions,
                                      _dev_ptr(counts),
                                      sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                                      _stream(stream)),
           "wtheta_count_regions")
    return sizes


def wtheta_jackknife(counts, sizes, n_regions: int):
    """(w, w_jk, cov) from host region-pair counts and region sizes."""
    c = np.ascontiguousarray(counts, np.uint64).reshape(-1)
    sz = np.ascontiguousarray(sizes, np.int64)
    K = c.size // (3 * n_regions * n_regions) - 2
    w = np.empty(K, np.float64)
    w_jk = np.empty((n_regions, K), np.float64)
    cov = np.empty((K, K), np.float64)
    _check(lib().wtheta_jackknife(c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                  sz.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), n_regions, K,
                                  _host_f64(w)[1], _host_f64(w_jk)[1], _host_f64(cov)[1]),
           "wtheta_jackknife")
    return w, w_jk, cov


def wtheta_inject_alloc_failure(after: int):
    """The device allocation after `after` more successful ones fails
    (host-side injection); -1 turns it off."""
    _check(lib().wtheta_inject_alloc_failure(int(after)), "wtheta_inject_alloc_failure")


def wtheta_probe_shared_atomics(same_address: bool) -> float:
    """Warp-wide shared reductions per SM per clock on the current device."""
    v = ctypes.c_double(0.0)
    _check(lib().wtheta_probe_shared_atomics(1 if same_address else 0, ctypes.byref(v)),
           "wtheta_probe_shared_atomics")
    return float(v.value)


def wtheta_ls_cross(D1D2, D1R2, R1D2, R1R2, n_d1, n_d2, n_r1, n_r2) -> np.ndarray:
    arrs = [_host_u64(x) for x in (D1D2, D1R2, R1D2, R1R2)]
    K = len(arrs[0][0]) - 2
    w = np.empty(K, np.float64)
    _check(lib().wtheta_ls_cross(*[p for _, p in arrs], n_d1, n_d2, n_r1, n_r2, K,
                                 _host_f64(w)[1]), "wtheta_ls_cross")
    return w


def wtheta_correlate(data, rand, edges_deg, stream=None):
    """Host catalogues in, (counts (3, K+2) uint64, w (K,)) out, one call."""
    d, dp = _host_f64(data)
    r, rp = _host_f64(rand)
    e, ep = _host_f64(edges_deg)
    K = len(e) - 1
    counts = np.zeros(3 * (K + 2), np.uint64)
    w = np.empty(K, np.float64)
    _check(lib().wtheta_correlate(dp, _host_points(d, "data"), rp, _host_points(r, "rand"), ep, K,
                                  _host_u64(counts)[1],
                                  _host_f64(w)[1], _stream(stream)), "wtheta_correlate")
    return counts.reshape(3, K + 2), w
