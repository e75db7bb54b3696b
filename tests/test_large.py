"""Parity at the large configuration: 2e8 visibilities (64 channels), an
8192^2 grid with 32 w-planes, Kaiser-Bessel W=9, uv-tile 64.

The FP64 oracle's full image at this size takes too long for a test, so the
checks are on what it can compute one by one and on what holds at any size:
- the bin offsets of all 1,048,576 bins, the drop counts and the w range bit
  for bit against the oracle's counting sort of the whole set, and the weight
  sum against the correctly rounded sum;
- the image at sampled pixels of the inner region (and the centre) against the
  oracle's per-visibility evaluation of the w-stacked image there, within
  1e-5 of the inner region's peak.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = [pytest.mark.gpu, pytest.mark.slow]

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_07321_gb300 as P
    return P


def test_large_binning_and_sampled_pixels(P):
    wl = synth.WORKLOADS["large"]
    d = synth.generate(wl.obs)
    n = len(d["vis"])
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                  max_vis=n, device=dev)
    img = im.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    v = P.rick.rick_bin_layout(im.plan)
    offsets = im.ws[v.offsets:v.offsets + 4 * (v.n_bins + 1)].cpu().numpy().view(np.uint32)
    st = im.stats()
    im.close()
    del t
    torch.cuda.empty_cache()

    op = oracle.Params(n=wl.n, n_w=wl.n_w, fov=wl.fov, kernel=oracle.KB, support=wl.support,
                       tile=wl.tile)
    ob = oracle.bin(op, d["uvw"])
    assert np.array_equal(offsets.astype(np.int64), ob["offsets"])
    assert st["n_binned"] == int((ob["status"] == 0).sum())
    assert st["n_dropped_uv"] == int((ob["status"] == 1).sum())
    assert st["n_dropped_w"] == int((ob["status"] == 2).sum())
    assert (st["w_min"], st["w_max"]) == (ob["w_min"], ob["w_max"])
    kept = ob["status"] == 0
    exact = math.fsum(d["weight"][kept].astype(np.float64))
    assert st["sum_weight"] == pytest.approx(exact, rel=1e-13)
    del ob

    N = wl.n
    q = N // 4
    rng = np.random.default_rng(21)
    pix = [(N // 2, N // 2)] + [(int(x), int(y)) for x, y in
                                rng.integers(N // 2 - q, N // 2 + q, size=(5, 2))]
    want = oracle.image_pixels(op, d["uvw"], d["vis"], d["weight"], pix)
    got = np.array([img[y, x] for x, y in pix], np.float64)
    peak = np.abs(img[N // 2 - q:N // 2 + q, N // 2 - q:N // 2 + q]).max()
    err = np.abs(got - want).max() / peak
    print(f"large: sampled-pixel error {err:.2e} of the inner peak {peak:.4g}")
    assert err <= TOL
