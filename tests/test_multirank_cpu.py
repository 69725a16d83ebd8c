"""Sharding one count across ranks, on CPU ranks (gloo): each rank counts its
shard of rows (wtheta_shard_rows) with the oracle, one sum-allreduce of K+2
integers combines them, and the result must equal the whole count.  The same
for a whole w(theta) split by the library's weighted split of tile rows
(wtheta_shard_weights, the split wtheta_count_wtheta_shard makes from the
kept tile pairs per row): DD, DR and RR of each rank's rows, reduced, equal
the oracle's whole counts.  A rank that fails before the collective must be
detected by the others (host-side failure injection: no GPU is involved)."""
import os
import socket

import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth
from paper_1208_3658_gb300 import wtheta as W

torch = pytest.importorskip("torch")
mp = torch.multiprocessing


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_1208_3658_gb300 import build
    build.build()
    O.build()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _catalogues():
    fp = synth.Patch(20.0, 6.0, 5.0, 11.0)
    a = synth.clustered(fp, 2500, 50, 3.0, 7, "test", "data", 77)
    b = synth.uniform(fp, 1800, 7, "test", "random", 77)
    return a, b


def _shard_counts(a, b, e, is_auto, shard, n_shards):
    """The shard's counts with the oracle, through the library's row split."""
    na = len(a) // 2
    r0, r1 = W.wtheta_shard_rows(na, na if is_auto else len(b) // 2, is_auto, shard, n_shards)
    rows = a.reshape(-1, 2)[r0:r1].reshape(-1)
    if not is_auto:
        return O.count(rows, b, e, False)
    inside = O.count(rows, None, e, True)
    later = a.reshape(-1, 2)[r1:].reshape(-1)
    if len(later) == 0 or r1 == r0:
        return inside
    return inside + O.count(rows, later, e, False)


TILE = 256  # points per tile row (the library's rows are 512 or 1024 points)


def _sorted(cat):
    """A spatial order stand-in (by RA, then Dec): rows of consecutive points."""
    rd = cat.reshape(-1, 2)
    return rd[np.lexsort((rd[:, 1], rd[:, 0]))].reshape(-1).copy()


def _row_weights(a, b, e, is_auto):
    """Work of each tile row of a count: its pairs below the top edge."""
    na = len(a) // 2
    w = []
    for r0 in range(0, na, TILE):
        r1 = min(r0 + TILE, na)
        rows = a.reshape(-1, 2)[r0:r1].reshape(-1)
        if is_auto:
            c = O.count(rows, None, e, True)
            later = a.reshape(-1, 2)[r1:].reshape(-1)
            if len(later):
                c = c + O.count(rows, later, e, False)
        else:
            c = O.count(rows, b, e, False)
        w.append(int(c[:-1].sum()))
    return np.array(w, np.uint64)


def _wtheta_shard_counts(d, r, e, shard, n_shards):
    """DD, DR, RR of the pairs whose first point is in the shard's tile rows,
    the rows split by the library by their in-range pairs."""
    out = []
    for a, b, auto in [(d, None, True), (d, r, False), (r, None, True)]:
        i0, i1 = W.wtheta_shard_weights(_row_weights(a, b, e, auto), shard, n_shards)
        na = len(a) // 2
        r0, r1 = min(i0 * TILE, na), min(i1 * TILE, na)
        rows = a.reshape(-1, 2)[r0:r1].reshape(-1)
        if r1 == r0:
            out.append(np.zeros(len(e) + 1, np.uint64))
        elif not auto:
            out.append(O.count(rows, b, e, False))
        else:
            c = O.count(rows, None, e, True)
            later = a.reshape(-1, 2)[r1:].reshape(-1)
            out.append(c + O.count(rows, later, e, False) if len(later) else c)
    return np.concatenate(out)


def _rank_main_wtheta(rank, world, port, out_path):
    import torch.distributed as dist
    from datetime import timedelta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=30))
    a, b = _catalogues()
    e = O.edges(1.0 / 60, 4.0, 16)
    c = _wtheta_shard_counts(_sorted(a), _sorted(b), e, rank, world)
    t = torch.from_numpy(c.astype(np.int64))
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    if rank == 0:
        with open(out_path, "w") as f:
            f.write("ok:" + ",".join(str(int(x)) for x in t.tolist()))
    dist.destroy_process_group()


def _rank_main(rank, world, port, is_auto, fail_rank, out_path):
    import torch.distributed as dist
    from datetime import timedelta
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=timedelta(seconds=6))
    a, b = _catalogues()
    e = O.edges(1.0 / 60, 4.0, 16)
    c = _shard_counts(a, b, e, is_auto, rank, world)
    if rank == fail_rank:
        raise SystemExit(3)  # this rank dies before the collective
    t = torch.from_numpy(c.astype(np.int64))
    try:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        result = "ok:" + ",".join(str(int(x)) for x in t.tolist())
    except Exception as ex:  # noqa: BLE001  (a peer failed: detected here)
        result = "error:" + type(ex).__name__
    if rank == 0:
        with open(out_path, "w") as f:
            f.write(result)
    try:
        dist.destroy_process_group()
    except Exception:  # noqa: BLE001
        pass


def _run(world, is_auto, fail_rank, tmp_path):
    port = _free_port()
    out = str(tmp_path / "rank0.txt")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, is_auto, fail_rank, out))
             for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        if p.is_alive():
            p.kill()
    return open(out).read() if os.path.exists(out) else "missing"


def test_shard_rows_partition_and_balance():
    for n, nb, auto in [(0, 0, True), (1, 1, True), (7, 7, True), (1000, 1000, True),
                        (1000, 300, False), (12345, 12345, True), (5, 1, False)]:
        for S in (1, 2, 3, 4, 7):
            cuts = [W.wtheta_shard_rows(n, nb, auto, s, S) for s in range(S)]
            assert cuts[0][0] == 0 and cuts[-1][1] == n
            assert all(cuts[s][1] == cuts[s + 1][0] for s in range(S - 1))
            pairs = [((r1 * (n - 1) - r1 * (r1 - 1) // 2) - (r0 * (n - 1) - r0 * (r0 - 1) // 2))
                     if auto else (r1 - r0) * nb for r0, r1 in cuts]
            total = n * (n - 1) // 2 if auto else n * nb
            assert sum(pairs) == total
            row_max = (n - 1) if auto else nb
            assert max(pairs) - min(pairs) <= 2 * max(row_max, 1)


@pytest.mark.parametrize("is_auto", [True, False])
def test_two_ranks_sum_to_the_whole_count(tmp_path, is_auto):
    res = _run(2, is_auto, -1, tmp_path)
    assert res.startswith("ok:"), res
    got = np.array([int(x) for x in res[3:].split(",")], dtype=np.uint64)
    a, b = _catalogues()
    e = O.edges(1.0 / 60, 4.0, 16)
    want = O.count(a, None if is_auto else b, e, is_auto)
    assert np.array_equal(got, want)


def test_shard_weights_partition_and_balance():
    rng = np.random.default_rng(5)
    cases = [np.zeros(0, np.uint64), np.zeros(7, np.uint64), np.ones(1, np.uint64),
             rng.integers(0, 1000, 37).astype(np.uint64),
             (rng.pareto(1.2, 500) * 100).astype(np.uint64),
             np.array([0, 0, 10 ** 15, 0, 5, 0], np.uint64)]
    for w in cases:
        for S in (1, 2, 3, 5, 8):
            cuts = [W.wtheta_shard_weights(w, s, S) for s in range(S)]
            assert cuts[0][0] == 0 and cuts[-1][1] == len(w)
            assert all(cuts[s][1] == cuts[s + 1][0] for s in range(S - 1))
            assert all(r0 <= r1 for r0, r1 in cuts)
            tot = int(w.sum())
            if tot == 0:
                sizes = [r1 - r0 for r0, r1 in cuts]
                assert max(sizes) - min(sizes) <= 1
                continue
            wmax = int(w.max())
            for r0, r1 in cuts:  # within one row's weight of an even share
                assert int(w[r0:r1].sum()) <= tot / S + wmax


def test_two_ranks_weighted_rows_sum_to_the_whole_wtheta(tmp_path):
    port = _free_port()
    out = str(tmp_path / "rank0.txt")
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank_main_wtheta, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        if p.is_alive():
            p.kill()
    res = open(out).read() if os.path.exists(out) else "missing"
    assert res.startswith("ok:"), res
    got = np.array([int(x) for x in res[3:].split(",")], dtype=np.uint64).reshape(3, -1)
    a, b = _catalogues()
    e = O.edges(1.0 / 60, 4.0, 16)
    want = [O.count(a, None, e, True), O.count(a, b, e, False), O.count(b, None, e, True)]
    for k in range(3):
        assert np.array_equal(got[k], want[k]), k


def test_rank_failure_is_detected(tmp_path):
    res = _run(2, True, 1, tmp_path)
    assert res.startswith("error:"), res
