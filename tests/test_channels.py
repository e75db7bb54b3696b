"""Multi-channel input (rows of n_chan channels, uvw once per row times a
per-channel factor) on the GPU.

The binning of rick_bin_channels must be rick_bin's on the expanded uvw, bit
for bit (bin offsets, stats, and every bin's records matched through their
input index); the streamed multi-channel image (rick_image_host_channels) must
be the FP64 oracle's image of the expanded set within 1e-5 of peak on the
tapered image and the inner region, for a range from the data, a given range,
ragged chunks of whole rows and pageable host memory.  With several
correlations per visibility (rick_bin_rows, rick_image_host_rows) each (row,
channel) is gridded once as the weighted sum of its correlations: the image
must be the oracle's image of the set with every correlation as its own
visibility, and the weight sum that set's, correctly rounded to 1e-13.
"""
import math

import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_07321_gb300 as P
    return P


def rows_data(n_rows, seed_shift=0):
    obs = synth.scaled("lofar", n_keep=16 * n_rows).obs
    obs.seed += seed_shift
    return obs, synth.generate(obs, rows=True)


def sets(b):
    off = b["offsets"].astype(np.int64)
    order = np.empty(len(b["perm"]), np.int64)
    for lo, hi in zip(off[:-1], off[1:]):
        if hi > lo:
            order[lo:hi] = lo + np.argsort(b["perm"][lo:hi], kind="stable")
    return dict(offsets=off, perm=b["perm"][order], rec_val=b["rec_val"][order],
                rec_frac=b["rec_frac"][order], rec_cell=b["rec_cell"][order], stats=b["stats"])


def test_channel_binning_is_the_expanded_binning(P):
    obs, d = rows_data(6000)
    wl = synth.WORKLOADS["lofar"]
    dev = torch.device("cuda:0")
    n = len(d["vis"])
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel="kb", support=7, tile=wl.tile, max_vis=n, device=dev)
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight", "uvw_rows",
                                                      "chan_scale")}
    im.bin(t["uvw"], t["vis"], t["weight"])
    torch.cuda.synchronize()
    ref = sets(im.binned())
    im.bin_channels(t["uvw_rows"], t["chan_scale"], t["vis"], t["weight"])
    torch.cuda.synchronize()
    got = sets(im.binned())
    assert got["stats"] == ref["stats"]
    for k in ("offsets", "perm", "rec_val", "rec_frac", "rec_cell"):
        assert np.array_equal(got[k], ref[k]), k
    op = oracle.Params(n=wl.n, n_w=wl.n_w, fov=wl.fov, kernel=oracle.KB, support=7, tile=wl.tile)
    assert np.array_equal(got["offsets"], oracle.bin(op, d["uvw"])["offsets"])
    im.close()


def taper_errors(img, ref, op):
    c = np.array([oracle.taper(op, (i - op.n // 2) / op.n) for i in range(op.n)])
    c = c / oracle.taper(op, 0.0)
    cc = c[:, None] * c[None, :]
    d = img.astype(np.float64) - ref
    q = op.n // 4
    inner = (slice(op.n // 2 - q, op.n // 2 + q),) * 2
    return (np.abs(d * cc).max() / np.abs(ref * cc).max(),
            np.abs(d[inner]).max() / np.abs(ref[inner]).max())


@pytest.mark.parametrize("chunk,w_range,pinned", [
    (5000, None, True),              # 312 rows per chunk, ragged last chunk, range from the data
    (16 * 700, (-3000.0, 2500.0), True),  # given range (drops), ragged
    (100_000, None, False),          # one chunk, pageable host memory
])
def test_streamed_channel_image_matches_oracle(P, chunk, w_range, pinned):
    obs, d = rows_data(2500, seed_shift=3)
    n, n_w, W = 512, 8, 7
    fov = (n / 2 - W - 1) / 12000.0
    im = P.Imager(n, n_w, fov, kernel="kb", support=W, tile=32, w_range=w_range, max_vis=chunk,
                  device=torch.device("cuda:0"))
    h = {k: torch.from_numpy(d[k]) for k in ("uvw_rows", "chan_scale", "vis", "weight")}
    if pinned:
        h = {k: v.pin_memory() for k, v in h.items()}
    img = im.image_streamed(h["uvw_rows"], h["vis"], h["weight"], chan_scale=h["chan_scale"])
    torch.cuda.synchronize()
    wr = w_range or (math.nan, math.nan)
    op = oracle.Params(n=n, n_w=n_w, fov=fov, kernel=oracle.KB, support=W, tile=32, w_min=wr[0],
                       w_max=wr[1])
    ref, st = oracle.image(op, d["uvw"], d["vis"], d["weight"])
    tap, inner = taper_errors(img.cpu().numpy(), ref, op)
    print(f"channels chunk={chunk}: tapered {tap:.2e} inner {inner:.2e}")
    assert tap <= TOL and inner <= TOL
    got = im.stats()
    assert got["n_binned"] == st["n_binned"]
    assert got["n_dropped_w"] == st["n_dropped_w"]
    assert got["sum_weight"] == pytest.approx(st["sum_weight"], rel=1e-12)
    im.close()


def corr_data(n_rows, n_corr, seed_shift=5, flag_frac=0.05):
    """Rows of 16 channels whose visibilities carry n_corr correlations: the
    generator's visibility plus independent noise per correlation, weights in
    [0.5, 1.5) per correlation with a few correlations flagged (weight 0)."""
    obs, d = rows_data(n_rows, seed_shift)
    n = len(d["vis"])
    r = np.random.default_rng(7)
    noise = 0.05 * (r.normal(size=(n, n_corr)) + 1j * r.normal(size=(n, n_corr)))
    vis = (d["vis"][:, None] + noise).astype(np.complex64)
    wt = (0.5 + r.random((n, n_corr))).astype(np.float32)
    wt[r.random((n, n_corr)) < flag_frac] = 0.0
    return d, vis, wt


def expanded(d, vis, wt):
    """The set with every correlation as its own visibility at the same uvw."""
    n_corr = vis.shape[1]
    return np.repeat(d["uvw"], n_corr, axis=0), vis.reshape(-1), wt.reshape(-1)


@pytest.mark.parametrize("n_corr,weighted", [(2, True), (4, True), (2, False)])
def test_correlations_fold_into_one_record(P, n_corr, weighted):
    d, vis, wt = corr_data(1500, n_corr)
    n, n_w, W = 512, 8, 7
    fov = (n / 2 - W - 1) / 12000.0
    dev = torch.device("cuda:0")
    im = P.Imager(n, n_w, fov, kernel="kb", support=W, tile=32, max_vis=len(d["vis"]), device=dev)
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw_rows", "chan_scale")}
    tv = torch.from_numpy(vis).to(dev)
    tw = torch.from_numpy(wt).to(dev) if weighted else None
    im.bin_channels(t["uvw_rows"], t["chan_scale"], tv, tw, n_corr=n_corr)
    img = im.image_from_binned().cpu().numpy()
    got = im.stats()
    uvw_x, vis_x, wt_x = expanded(d, vis, wt if weighted else np.ones_like(wt))
    op = oracle.Params(n=n, n_w=n_w, fov=fov, kernel=oracle.KB, support=W, tile=32)
    ref, st = oracle.image(op, uvw_x, vis_x, wt_x)
    tap, inner = taper_errors(img, ref, op)
    print(f"correlations {n_corr} weighted={weighted}: tapered {tap:.2e} inner {inner:.2e}")
    assert tap <= TOL and inner <= TOL
    assert got["n_binned"] * n_corr == st["n_binned"]
    kept = np.repeat(oracle.coords(op, d["uvw"])["status"] == 0, n_corr)
    exact = math.fsum(wt_x[kept].astype(np.float64))
    assert got["sum_weight"] == pytest.approx(exact, rel=1e-13)
    with pytest.raises(P.rick.RickError):  # checked on the host before any launch
        P.rick.rick_bin_rows(im.plan, 1500, 16, P.rick.RICK_MAX_CORR + 1,
                             t["uvw_rows"].data_ptr(), t["chan_scale"].data_ptr(), tv.data_ptr(),
                             None, im.ws.data_ptr(), im.ws_bytes, None, None)
    im.close()


def test_streamed_correlations(P):
    n_corr = 2
    d, vis, wt = corr_data(2500, n_corr, seed_shift=9)
    n, n_w, W = 512, 8, 7
    fov = (n / 2 - W - 1) / 12000.0
    im = P.Imager(n, n_w, fov, kernel="kb", support=W, tile=32, max_vis=16 * 600,
                  device=torch.device("cuda:0"))  # 300 rows per chunk, ragged last chunk
    h = {k: torch.from_numpy(d[k]).pin_memory() for k in ("uvw_rows", "chan_scale")}
    hv = torch.from_numpy(vis).pin_memory()
    hw = torch.from_numpy(wt).pin_memory()
    img = im.image_streamed(h["uvw_rows"], hv, hw, chan_scale=h["chan_scale"], n_corr=n_corr)
    torch.cuda.synchronize()
    op = oracle.Params(n=n, n_w=n_w, fov=fov, kernel=oracle.KB, support=W, tile=32)
    ref, st = oracle.image(op, *expanded(d, vis, wt))
    tap, inner = taper_errors(img.cpu().numpy(), ref, op)
    print(f"streamed correlations: tapered {tap:.2e} inner {inner:.2e}")
    assert tap <= TOL and inner <= TOL
    got = im.stats()
    assert got["n_binned"] * n_corr == st["n_binned"]
    assert got["sum_weight"] == pytest.approx(st["sum_weight"], rel=1e-12)
    im.close()
