"""Region-pair counts on the GPU (the jackknife's input) against the oracle,
bit for bit on the oracle's own unit vectors."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1208_3658_gb300 import synth

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")

ARCMIN = 1.0 / 60.0


@pytest.fixture(scope="module")
def W():
    from paper_1208_3658_gb300 import build
    build.build()
    from paper_1208_3658_gb300 import wtheta
    return wtheta


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _case(nd, nr, seed, nx, ny):
    fp = synth.Patch(210.0, 10.0, 5.0, 15.0)
    D = synth.clustered(fp, nd, max(1, nd // 50), 3.0, seed, "test", "data")
    Rn = synth.uniform(fp, nr, seed, "test", "random")
    ld = synth.grid_labels(D, 210.0, 220.0, 5.0, 15.0, nx, ny)
    lr = synth.grid_labels(Rn, 210.0, 220.0, 5.0, 15.0, nx, ny)
    return D, Rn, ld, lr


@pytest.mark.parametrize("nd,nr,nx,ny", [(6000, 7000, 3, 3), (2500, 3100, 4, 4), (1500, 900, 2, 1)])
def test_region_pair_counts_bit_exact(W, nd, nr, nx, ny):
    D, Rn, ld, lr = _case(nd, nr, nd + nr, nx, ny)
    R = nx * ny
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    XD, XR = O.radec_to_xyz(D), O.radec_to_xyz(Rn)
    K = len(e) - 1
    c = torch.zeros((3, R, R, K + 2), dtype=torch.int64, device="cuda")
    sizes = W.wtheta_count_regions(dev(XD), dev(ld), dev(XR), dev(lr), e, R, c,
                                   coords_are_xyz=True)
    torch.cuda.synchronize()
    got = c.cpu().numpy().astype(np.uint64)
    want = O.count_regions(XD, ld, XR, lr, e, R)
    assert np.array_equal(sizes, np.concatenate([np.bincount(ld, minlength=R),
                                                 np.bincount(lr, minlength=R)]))
    assert np.array_equal(got, want)


def test_regions_from_radec_sum_to_plain_counts_and_jackknife(W):
    D, Rn, ld, lr = _case(20_000, 24_000, 9, 4, 4)
    R = 16
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    K = len(e) - 1
    c = torch.zeros((3, R, R, K + 2), dtype=torch.int64, device="cuda")
    sizes = W.wtheta_count_regions(dev(D), dev(ld), dev(Rn), dev(lr), e, R, c)
    plain = torch.zeros((3, K + 2), dtype=torch.int64, device="cuda")
    d, r = dev(D), dev(Rn)
    W.wtheta_count(d, None, e, True, plain[0])
    W.wtheta_count(d, r, e, False, plain[1])
    W.wtheta_count(r, None, e, True, plain[2])
    torch.cuda.synchronize()
    got = c.cpu().numpy().astype(np.uint64)
    p = plain.cpu().numpy().astype(np.uint64)
    for kind in range(3):
        assert np.array_equal(got[kind].sum(axis=(0, 1), dtype=np.uint64), p[kind])
    w, w_k, cov = W.wtheta_jackknife(got, sizes, R)
    w_plain = W.wtheta_ls(p[0], p[1], p[2], 20_000, 24_000)
    assert np.array_equal(w, w_plain, equal_nan=True)
    w_o, w_ko, cov_o = O.jackknife(got, sizes, R)
    ok = np.isfinite(w_ko)
    assert np.all(np.abs(w_k - w_ko)[ok] <= 1e-12 * np.maximum(np.abs(w_ko[ok]), 1.0))
    assert np.all(np.diag(cov)[np.all(ok, axis=0)] >= 0)


def test_bad_label_sets_error_word(W):
    D, Rn, ld, lr = _case(3000, 3000, 5, 2, 2)
    ld = ld.copy()
    ld[17] = 9                                  # outside [0, 4)
    e = W.wtheta_edges(1.0 * ARCMIN, 5.0, 16)
    c = torch.zeros((3, 4, 4, 18), dtype=torch.int64, device="cuda")
    W.wtheta_get_error()                        # clear
    W.wtheta_count_regions(dev(D), dev(ld), dev(Rn), dev(lr), e, 4, c)
    torch.cuda.synchronize()
    assert W.wtheta_get_error() & 8
