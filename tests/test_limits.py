"""The parameter limits on the GPU: the largest grid (n = 32768) with the widest
kernel (W = 16) and the largest tile (T = 128), and the most w-planes
(n_w = 1024).

The largest grid is too big for the oracle's full image, so it is checked on
what the oracle computes one by one: every bin offset, the stats, and the image
at sampled pixels against the per-visibility evaluation of the w-stacked image
(1e-5 of the centre pixel, where a point source sits).  The 1024-plane case is
small enough for the oracle's full image.
"""
import math

import numpy as np
import pytest

import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_07321_gb300 as P
    return P


def point_source_set(n, fov, W, m, w_max, seed):
    """m visibilities with u, v uniform over the grid (footprints inside) and w
    in [-w_max, w_max]: a unit point source at the phase centre plus noise."""
    r = np.random.default_rng(seed)
    lim = (n / 2 - W - 1) / fov
    uvw = np.stack([r.uniform(-lim, lim, m), r.uniform(-lim, lim, m),
                    r.uniform(-w_max, w_max, m)], 1)
    vis = (1.0 + 0.05 * (r.normal(size=m) + 1j * r.normal(size=m))).astype(np.complex64)
    wt = (0.5 + r.random(m)).astype(np.float32)
    return uvw, vis, wt


def test_largest_grid_widest_kernel_largest_tile(P):
    n, n_w, W, T = 32768, 2, 16, 128
    fov = 0.2
    uvw, vis, wt = point_source_set(n, fov, W, 6000, 300.0, 61)
    dev = torch.device("cuda:0")
    im = P.Imager(n, n_w, fov, kernel="kb", support=W, tile=T, max_vis=len(vis), device=dev)
    img = im.image(torch.from_numpy(uvw).to(dev), torch.from_numpy(vis).to(dev),
                   torch.from_numpy(wt).to(dev))
    torch.cuda.synchronize()
    v = P.rick.rick_bin_layout(im.plan)
    offsets = im.ws[v.offsets:v.offsets + 4 * (v.n_bins + 1)].cpu().numpy().view(np.uint32)
    st = im.stats()
    op = oracle.Params(n=n, n_w=n_w, fov=fov, kernel=oracle.KB, support=W, tile=T)
    ob = oracle.bin(op, uvw)
    assert np.array_equal(offsets.astype(np.int64), ob["offsets"])
    assert st["n_binned"] == len(vis) and (st["w_min"], st["w_max"]) == (ob["w_min"],
                                                                           ob["w_max"])
    assert st["sum_weight"] == pytest.approx(math.fsum(wt.astype(np.float64)), rel=1e-13)
    q = n // 4
    rng = np.random.default_rng(62)
    pix = [(n // 2, n // 2)] + [(int(x), int(y)) for x, y in
                                rng.integers(n // 2 - q, n // 2 + q, size=(7, 2))]
    want = oracle.image_pixels(op, uvw, vis.astype(np.complex128), wt.astype(np.float64), pix)
    got = np.array([img[y, x].item() for x, y in pix], np.float64)
    err = np.abs(got - want).max() / abs(want[0])
    print(f"n=32768 W=16 T=128: sampled-pixel error {err:.2e} of the centre {want[0]:.4g}")
    assert err <= TOL
    im.close()
    del img
    torch.cuda.empty_cache()


def test_most_w_planes(P):
    n, n_w, W = 64, 1024, 7
    fov = 0.05
    uvw, vis, wt = point_source_set(n, fov, W, 30000, 2000.0, 63)
    dev = torch.device("cuda:0")
    im = P.Imager(n, n_w, fov, kernel="kb", support=W, tile=16, max_vis=len(vis), device=dev)
    img = im.image(torch.from_numpy(uvw).to(dev), torch.from_numpy(vis).to(dev),
                   torch.from_numpy(wt).to(dev)).cpu().numpy()
    op = oracle.Params(n=n, n_w=n_w, fov=fov, kernel=oracle.KB, support=W, tile=16)
    ref, st = oracle.image(op, uvw, vis.astype(np.complex128), wt.astype(np.float64))
    c = np.array([oracle.taper(op, (i - n // 2) / n) for i in range(n)])
    cc = np.outer(c, c) / oracle.taper(op, 0.0) ** 2
    d = img.astype(np.float64) - ref
    tap = np.abs(d * cc).max() / np.abs(ref * cc).max()
    print(f"n_w=1024: tapered error {tap:.2e}")
    assert tap <= TOL
    assert im.stats()["n_binned"] == st["n_binned"]
    im.close()
