"""The allocation-free binning entry point, rick_bin_noalloc.

Callers that may not allocate device memory (a host program that hands a
plug-in only the buffers it owns, a real-time loop that forbids allocator
calls) bin through rick_bin_noalloc, which keeps its temporaries in a fixed
array inside the library.  Its result must be rick_bin's: the same bins, the
same records and the same image.  Two calls in a row with different data check
that nothing from the first call leaks into the second (the array keeps its
contents between calls).  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_07321_gb300 as P
    return P


def _binned_sets(b):
    """Bin offsets, stats, and every bin's records keyed by input index."""
    off = b["offsets"].astype(np.int64)
    order = np.empty(len(b["perm"]), np.int64)
    for lo, hi in zip(off[:-1], off[1:]):
        if hi > lo:
            order[lo:hi] = lo + np.argsort(b["perm"][lo:hi], kind="stable")
    return dict(offsets=off, stats=b["stats"], perm=b["perm"][order],
                rec_val=b["rec_val"][order], rec_frac=b["rec_frac"][order],
                rec_cell=b["rec_cell"][order])


def _run(P, im, t, noalloc):
    R = P.rick
    n = t["uvw"].shape[0]
    fn = R.rick_bin_noalloc if noalloc else R.rick_bin
    fn(im.plan, n, t["uvw"].data_ptr(), t["vis"].data_ptr(), t["weight"].data_ptr(),
       im.ws.data_ptr(), im.ws_bytes, im.stats_buf.data_ptr(),
       torch.cuda.current_stream().cuda_stream)
    im.n_vis = n
    torch.cuda.synchronize()
    sets = _binned_sets(im.binned())
    im.grid()
    return sets, im.planes.cpu().numpy()


def test_noalloc_binning_matches_rick_bin_twice(P):
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                  max_vis=65536, device=dev)
    for n_keep, seed_shift in ((65536, 0), (40001, 7)):
        obs = synth.scaled("small", n_keep=n_keep).obs
        obs.seed += seed_shift
        d = synth.generate(obs)
        t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
        ref_sets, ref_planes = _run(P, im, t, noalloc=False)
        got_sets, got_planes = _run(P, im, t, noalloc=True)
        assert got_sets["stats"] == ref_sets["stats"]
        for k in ("offsets", "perm", "rec_val", "rec_frac", "rec_cell"):
            assert np.array_equal(got_sets[k], ref_sets[k]), k
        # the gridded planes agree within the parity tests' tolerance (the order
        # of records inside a bin, hence FP32 rounding, may differ between calls)
        assert np.abs(got_planes - ref_planes).max() <= 1e-5 * np.abs(ref_planes).max()
    im.close()


def test_noalloc_rejects_sizes_beyond_its_array(P):
    R = P.rick
    dev = torch.device("cuda:0")
    im = P.Imager(256, 8, 0.035, kernel="kb", support=7, tile=32, max_vis=300000, device=dev)
    n = 262145
    uvw = torch.zeros((n, 3), dtype=torch.float64, device=dev)
    vis = torch.zeros(n, dtype=torch.complex64, device=dev)
    with pytest.raises(R.RickError) as e:
        R.rick_bin_noalloc(im.plan, n, uvw.data_ptr(), vis.data_ptr(), None, im.ws.data_ptr(),
                           im.ws_bytes, None, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == R.RICK_ERANGE
    im.close()
    big = P.Imager(1024, 5, 0.05, kernel="kb", support=7, tile=8, max_vis=1000, device=dev)
    with pytest.raises(R.RickError) as e:  # 4 * 5 * 128^2 = 327680 bins > 131072
        R.rick_bin_noalloc(big.plan, 10, uvw.data_ptr(), vis.data_ptr(), None, big.ws.data_ptr(),
                           big.ws_bytes, None, torch.cuda.current_stream().cuda_stream)
    assert e.value.status == R.RICK_ERANGE
    big.close()


def test_noalloc_binning_feeds_degrid_and_density_weights(P):
    """Degridding and the density weights read the keys and corner cells a
    binning leaves in the workspace.  A workspace that only ever saw
    rick_bin_noalloc (filled with 0xFF first, so nothing from another binning
    can stand in) must give them what rick_bin gives, including the dropped
    visibilities (some placed off the grid)."""
    R = P.rick
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = synth.generate(synth.scaled("small", n_keep=30000).obs)
    uvw = d["uvw"].copy()
    uvw[::97, 0] = 1.0e6  # far outside the grid: dropped
    t = {"uvw": torch.from_numpy(uvw).to(dev), "vis": torch.from_numpy(d["vis"]).to(dev),
         "weight": torch.from_numpy(d["weight"]).to(dev)}
    n = uvw.shape[0]
    out = {}
    rng = np.random.default_rng(3)
    planes = (rng.normal(size=(wl.n_w, wl.n, wl.n)) +
              1j * rng.normal(size=(wl.n_w, wl.n, wl.n))).astype(np.complex64)
    for noalloc in (False, True):
        im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                      max_vis=n, device=dev)
        im.ws.fill_(0xFF)
        fn = R.rick_bin_noalloc if noalloc else R.rick_bin
        fn(im.plan, n, t["uvw"].data_ptr(), t["vis"].data_ptr(), t["weight"].data_ptr(),
           im.ws.data_ptr(), im.ws_bytes, im.stats_buf.data_ptr(),
           torch.cuda.current_stream().cuda_stream)
        im.n_vis = n
        im.planes.copy_(torch.from_numpy(planes).to(dev))
        out[noalloc] = dict(stats=im.stats(), degrid=im.degrid(t["weight"]).cpu().numpy(),
                            uniform=im.density_weights("uniform", 0.0, t["weight"]).cpu().numpy(),
                            briggs=im.density_weights("briggs", 0.5, t["weight"]).cpu().numpy())
        torch.cuda.synchronize()
        im.close()
    ref, got = out[False], out[True]
    assert ref["stats"]["n_dropped_uv"] > 0
    assert got["stats"] == ref["stats"]
    # each model value comes from one record, whose content is the same
    assert np.array_equal(got["degrid"], ref["degrid"])
    assert np.all(got["degrid"][::97] == 0)
    for k in ("uniform", "briggs"):  # densities summed with float atomics (any order)
        assert np.all(got[k][::97] == 0)
        assert np.allclose(got[k], ref[k], rtol=1e-6, atol=0), k
