"""Streamed imaging from host memory (rick_image_host) on the GPU.

A visibility set in host memory is imaged in chunks of the plan's max_vis:
each chunk is binned and gridded into the same planes (the tiles its records
reach, added into those an earlier chunk reached), then one fused FFT and
w-correction (rick_grid, rick_grid_accumulate and cuFFT for grids outside the
fused transform's sizes).  The image must be the
FP64 oracle's image of the WHOLE set (1e-5 of peak on the tapered image and
the inner region, as in test_gpu_parity), the stats must be the whole set's
(counts exact, weight sum to 1e-12), for a w range from the data and a given
one, unit weights, ragged last chunks, a single chunk, an empty set, pageable
host memory, and back-to-back calls that reuse the staging buffers.
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


def taper_2d(op):
    c = np.array([oracle.taper(op, (i - op.n // 2) / op.n) for i in range(op.n)])
    c = c / oracle.taper(op, 0.0)
    return c[:, None] * c[None, :]


def errors(img, ref, op):
    cc = taper_2d(op)
    d = img.astype(np.float64) - ref
    q = op.n // 4
    inner = (slice(op.n // 2 - q, op.n // 2 + q),) * 2
    return dict(tapered=np.abs(d * cc).max() / np.abs(ref * cc).max(),
                inner=np.abs(d[inner]).max() / np.abs(ref[inner]).max())


def host(d, pinned=True):
    t = {k: torch.from_numpy(np.ascontiguousarray(d[k])) for k in ("uvw", "vis", "weight")}
    return {k: (v.pin_memory() if pinned else v) for k, v in t.items()}


def setup(P, n_keep, chunk, w_range=None, kernel="kb", support=7, tile=32, seed_shift=0):
    wl = synth.WORKLOADS["small"]
    obs = synth.scaled("small", n_keep=n_keep).obs
    obs.seed += seed_shift
    d = synth.generate(obs)
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=kernel, support=support, tile=tile,
                  w_range=w_range, max_vis=chunk, device=torch.device("cuda:0"))
    wr = w_range or (math.nan, math.nan)
    op = oracle.Params(n=wl.n, n_w=wl.n_w, fov=wl.fov,
                       kernel=oracle.KB if kernel == "kb" else oracle.GAUSS, support=support,
                       tile=tile, w_min=wr[0], w_max=wr[1])
    return im, op, d


def check_stats(st, op, d, weighted=True):
    ob = oracle.bin(op, d["uvw"])
    kept = ob["status"] == 0
    assert st["n_binned"] == int(kept.sum())
    assert st["n_dropped_uv"] == int((ob["status"] == 1).sum())
    assert st["n_dropped_w"] == int((ob["status"] == 2).sum())
    assert (st["w_min"], st["w_max"]) == (ob["w_min"], ob["w_max"])
    want = float(d["weight"][kept].astype(np.float64).sum()) if weighted else float(kept.sum())
    assert st["sum_weight"] == pytest.approx(want, rel=1e-12)


@pytest.mark.parametrize("n_keep,chunk,w_range,weighted", [
    (65536, 9000, None, True),             # 8 chunks, ragged last one, range from the data
    (50000, 7777, (-150.0, 120.0), True),  # given range (drops), ragged
    (40000, 40000, None, False),           # one chunk, unit weights
    (30001, 1024, None, True),             # many small chunks
])
def test_streamed_image_matches_oracle(P, n_keep, chunk, w_range, weighted):
    im, op, d = setup(P, n_keep, chunk, w_range)
    h = host(d)
    wt = h["weight"] if weighted else None
    img = im.image_streamed(h["uvw"], h["vis"], wt)
    torch.cuda.synchronize()
    got = img.cpu().numpy()
    ref, _ = oracle.image(op, d["uvw"], d["vis"], d["weight"] if weighted else None)
    e = errors(got, ref, op)
    print(f"streamed n={n_keep} chunk={chunk}: tapered {e['tapered']:.2e} inner {e['inner']:.2e}")
    assert e["tapered"] <= TOL and e["inner"] <= TOL
    check_stats(im.stats(), op, d, weighted)
    im.close()


def test_streamed_deterministic(P):
    """Deterministic mode through the streamed call (each chunk's tile sums in
    fixed point, the chunks added into the planes in chunk order): two calls
    give bitwise equal images, and they match the oracle's image."""
    wl = synth.WORKLOADS["small"]
    d = synth.generate(synth.scaled("small", n_keep=40000).obs)
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel="kb", support=7, tile=32, max_vis=9000,
                  device=torch.device("cuda:0"), deterministic=True)
    h = host(d)
    a = im.image_streamed(h["uvw"], h["vis"], h["weight"]).clone()
    b = im.image_streamed(h["uvw"], h["vis"], h["weight"]).clone()
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    op = oracle.Params(n=wl.n, n_w=wl.n_w, fov=wl.fov, kernel=oracle.KB, support=7, tile=32)
    ref, _ = oracle.image(op, d["uvw"], d["vis"], d["weight"])
    e = errors(a.cpu().numpy(), ref, op)
    assert e["tapered"] <= TOL and e["inner"] <= TOL
    im.close()


def test_streamed_equals_single_pass_and_reuses_staging(P):
    """Two calls in a row with different data (the second reuses the staging
    buffers while nothing waits in between): each equals the single-pass
    device path on the same data."""
    dev = torch.device("cuda:0")
    for shift in (0, 11):
        im, op, d = setup(P, 60000, 16384, seed_shift=shift)
        h = host(d)
        streamed = im.image_streamed(h["uvw"], h["vis"], h["weight"]).clone()
        whole = P.Imager(op.n, op.n_w, op.fov, kernel="kb", support=7, tile=32, max_vis=60000,
                         device=dev)
        t = {k: v.to(dev) for k, v in h.items()}
        single = whole.image(t["uvw"], t["vis"], t["weight"])
        torch.cuda.synchronize()
        ref, _ = oracle.image(op, d["uvw"], d["vis"], d["weight"])
        e1 = errors(streamed.cpu().numpy(), ref, op)
        e2 = errors(single.cpu().numpy(), ref, op)
        assert e1["tapered"] <= TOL and e2["tapered"] <= TOL
        s1, s2 = im.stats(), whole.stats()
        for k in ("n_binned", "n_dropped_uv", "n_dropped_w", "w_min", "w_max"):
            assert s1[k] == s2[k], k
        assert s1["sum_weight"] == pytest.approx(s2["sum_weight"], rel=1e-12)
        whole.close()
        im.close()


def test_streamed_back_to_back_calls_on_one_imager(P):
    """Consecutive calls on one imager share its staging area, so each call's
    copies may run under the previous call's gridding, FFT and w-correction;
    the resident uvw areas alternate.  Sizes change between calls (a smaller
    set keeps the area, a larger one gets a new one)."""
    im, op, d = setup(P, 40000, 6000)
    _, _, d2 = setup(P, 40000, 6000, seed_shift=5)
    h, h2 = host(d), host(d2)
    sets = [(h, d, 40000), (h2, d2, 40000), (h, d, 25000), (h2, d2, 40000), (h, d, 40000)]
    outs = []
    for hh, _, n in sets:
        outs.append(im.image_streamed(hh["uvw"][:n], hh["vis"][:n], hh["weight"][:n]).clone())
    torch.cuda.synchronize()
    for (hh, dd, n), got in zip(sets, outs):
        ref, _ = oracle.image(op, dd["uvw"][:n], dd["vis"][:n], dd["weight"][:n])
        assert errors(got.cpu().numpy(), ref, op)["tapered"] <= TOL, n
    check_stats(im.stats(), op, d)
    im.close()


def test_streamed_pageable_host_memory(P):
    im, op, d = setup(P, 20000, 3000, kernel="gauss")
    h = host(d, pinned=False)
    img = im.image_streamed(h["uvw"], h["vis"], h["weight"])
    torch.cuda.synchronize()
    ref, _ = oracle.image(op, d["uvw"], d["vis"], d["weight"])
    assert errors(img.cpu().numpy(), ref, op)["tapered"] <= TOL
    im.close()


def test_streamed_empty_set(P):
    im, op, d = setup(P, 1000, 500)
    e = {k: torch.empty((0, 3) if k == "uvw" else (0,), dtype=v.dtype) for k, v in host(d).items()}
    img = im.image_streamed(e["uvw"], e["vis"], e["weight"])
    torch.cuda.synchronize()
    assert not img.cpu().numpy().any()
    st = im.stats()
    assert st["n_binned"] == 0 and st["sum_weight"] == 0.0
    im.close()
