"""The allocation-free entry point, wtheta_count_xyz_noalloc.

It exists for callers that cannot let a library allocate device memory (a
framework that owns the device's memory in its own pool, a server with a
fixed memory budget reserved up front, a latency-bound loop that cannot take
an allocation's implicit synchronisation).  It must give exactly the counts of
the allocating entry point, wtheta_count_xyz, call after call, although every
call reuses the same fixed scratch array inside the library.

This file is named to be collected last, so that a run stopping at its first
failure has already run every other test; it also passes on its own in a fresh
process (the first call on the device does the scratch set-up).
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def W():
    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta
    return wtheta


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _both(W, A, B, e, auto):
    """Counts from the allocation-free and the allocating entry point."""
    c_free = torch.full((len(e) + 1,), -1, dtype=torch.int64, device="cuda")
    c_ref = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
    a = _dev(A)
    b = None if auto else _dev(B)
    W.wtheta_count_xyz_noalloc(a, b, e, auto, c_free)
    W.wtheta_count_xyz(a, b, e, auto, c_ref)
    torch.cuda.synchronize()
    return c_free.cpu().numpy(), c_ref.cpu().numpy()


def test_noalloc_matches_allocating_entry_point_on_consecutive_calls(W):
    e = W.wtheta_edges(1.0 / 60.0, 5.0, 16)
    fp = synth.Patch(30.0, 8.0, 10.0, 18.0)
    # two calls in a row on different inputs: a larger cross count, then a
    # smaller auto count that must not see the first call's scratch contents
    D = O.radec_to_xyz(synth.clustered(fp, 60_000, 1200, 3.0, 4, "test", "data", 1))
    R = O.radec_to_xyz(synth.uniform(fp, 70_001, 4, "test", "random", 1))
    free1, ref1 = _both(W, D, R, e, False)
    assert np.array_equal(free1, ref1)
    assert int(free1.sum()) == D.shape[1] * R.shape[1]
    S = np.ascontiguousarray(D[:, :9_999])
    free2, ref2 = _both(W, S, None, e, True)
    assert np.array_equal(free2, ref2)
    assert int(free2.sum()) == 9_999 * 9_998 // 2


def test_noalloc_rejects_inputs_beyond_its_fixed_capacity(W):
    e = W.wtheta_edges(1.0 / 60.0, 5.0, 16)
    n = W.NOALLOC_MAX_POINTS - W.NOALLOC_TILE + 1  # pads to one tile past the limit with b
    A = torch.zeros((3, n), dtype=torch.float64, device="cuda")
    B = torch.zeros((3, W.NOALLOC_TILE), dtype=torch.float64, device="cuda")
    c = torch.zeros(len(e) + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(W.WthetaError) as ex:
        W.wtheta_count_xyz_noalloc(A, B, e, False, c)
    assert ex.value.status == -7  # WTHETA_ESIZE
