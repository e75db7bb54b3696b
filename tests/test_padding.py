"""Grid padding with a crop on the GPU: the grid has n cells a side and the
image is its central image_n x image_n pixels (pixel size fov/n).

The cropped image must be the FP64 oracle's cropped image within 1e-5 of peak
(the crop's taper-weighted error where the crop reaches the grid edge), its
adjoint the oracle's zero-padding adjoint, the streamed path and a re-targeted
plan (rick_plan_set_image_n) the same image; and on a w = 0 field a grid padded
by 2 must meet the brute-force DFT at the FP32 floor where the unpadded grid of
the same pixel size misses it by percents (the aliasing that padding removes).
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


# name -> grid side n, image side m, kernel, support, tile, fov / (small workload's fov)
CASES = {
    "kb7_pad2": (512, 256, "kb", 7, 32, 2.0),
    "gauss7_pad2": (512, 256, "gauss", 7, 32, 2.0),
    "kb8_odd_offset": (256, 222, "kb", 8, 16, 1.0),  # offset 17
    "w1_crop": (256, 128, "kb", 1, 8, 1.0),
}


def setup(P, name, n_keep=40000, max_vis=None):
    n, m, kern, W, tile, fs = CASES[name]
    wl = synth.WORKLOADS["small"]
    d = synth.generate(synth.scaled("small", n_keep=n_keep).obs)
    fov = wl.fov * fs
    im = P.Imager(n, 8, fov, kernel=kern, support=W, tile=tile, max_vis=max_vis or n_keep,
                  device=torch.device("cuda:0"), image_n=m)
    op = oracle.Params(n=n, n_w=8, fov=fov, kernel=oracle.KB if kern == "kb" else oracle.GAUSS,
                       support=W, tile=tile, image_n=m)
    return d, im, op


def crop_taper(op):
    """C(l) C(m) / C(0)^2 over the crop's pixels (grid-frame nu = (p - n/2)/n)."""
    o = (op.n - op.side()) // 2
    c = np.array([oracle.taper(op, (o + i - op.n // 2) / op.n) for i in range(op.side())])
    c = c / oracle.taper(op, 0.0)
    return c[:, None] * c[None, :]


def errors(img, ref, op):
    cc = crop_taper(op)
    d = img.astype(np.float64) - ref
    return (np.abs(d).max() / np.abs(ref).max(),
            np.abs(d * cc).max() / np.abs(ref * cc).max())


@pytest.mark.parametrize("name", list(CASES))
def test_cropped_image_and_adjoint_match_oracle(P, name):
    d, im, op = setup(P, name)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
    img = im.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    assert img.shape == (op.side(), op.side())
    ref, st = oracle.image(op, d["uvw"], d["vis"], d["weight"])
    raw, tap = errors(img, ref, op)
    print(f"{name}: raw {raw:.2e} tapered {tap:.2e}")
    assert tap <= TOL
    if op.n == 2 * op.side():  # the crop stays where the taper is healthy
        assert raw <= TOL
    got = im.stats()
    assert got["n_binned"] == st["n_binned"]
    # adjoint: the m x m image enters zero-padded
    y = (np.random.default_rng(5).normal(size=(op.side(), op.side())) *
         crop_taper(op)).astype(np.float32)
    vg = im.adjoint(torch.from_numpy(y).to(dev), t["weight"]).cpu().numpy()
    vr = oracle.adjoint(op, d["uvw"], y.astype(np.float64), d["weight"].astype(np.float64),
                        w_min=got["w_min"], w_max=got["w_max"], sum_weight=got["sum_weight"])
    assert np.abs(vg - vr).max() <= TOL * np.abs(vr).max()
    im.close()


def test_streamed_cropped_image(P):
    d, im, op = setup(P, "kb7_pad2", n_keep=40000, max_vis=7000)  # 6 chunks, ragged
    h = {k: torch.from_numpy(d[k]).pin_memory() for k in ("uvw", "vis", "weight")}
    out = torch.empty((op.side(), op.side()), dtype=torch.float32).pin_memory()
    im.image_streamed(h["uvw"], h["vis"], h["weight"], out_host=out)
    im.wait_out()
    torch.cuda.synchronize()
    ref, _ = oracle.image(op, d["uvw"], d["vis"], d["weight"])
    raw, _ = errors(out.numpy(), ref, op)
    print(f"streamed crop: raw {raw:.2e}")
    assert raw <= TOL
    im.close()


def test_set_image_n_retargets_a_plan(P):
    d, im, op = setup(P, "kb7_pad2")
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
    for m in (None, 128, 256):
        im.set_image_n(m)
        img = im.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
        q = oracle.Params(**{**op.__dict__, "image_n": m or 0})
        ref, _ = oracle.image(q, d["uvw"], d["vis"], d["weight"])
        _, tap = errors(img, ref, q)
        assert img.shape == (q.side(), q.side()) and tap <= TOL, m
    with pytest.raises(P.rick.RickError):
        im.set_image_n(13)
    assert im.m == 256
    im.close()


def point_sources(m_img, fov_img, M, seed):
    r = np.random.default_rng(seed)
    lim = (m_img / 2 - 5) / fov_img
    uvw = np.stack([r.uniform(-lim, lim, M), r.uniform(-lim, lim, M), np.zeros(M)], 1)
    dl = fov_img / m_img
    vis = np.zeros(M, np.complex128)
    for a, b, S in ((0.44 * m_img, -0.42 * m_img, 1.0), (3.0, -2.0, 0.5),
                    (-0.49 * m_img, 0.46 * m_img, 0.7)):
        l0, m0 = a * dl, b * dl
        n0 = math.sqrt(1 - l0 * l0 - m0 * m0)
        vis += S / n0 * np.exp(-2j * np.pi * (uvw[:, 0] * l0 + uvw[:, 1] * m0 +
                                              uvw[:, 2] * (n0 - 1)))
    return uvw, vis


def test_padding_meets_the_dft_on_the_gpu(P):
    m, fov_img, M = 128, 2.0 ** -4, 20000
    uvw, vis = point_sources(m, fov_img, M, 41)
    ref = oracle.dft(m, fov_img, uvw, vis, None, flags=oracle.N_CORRECT | oracle.NORMALIZE,
                     sum_weight=float(M))
    dev = torch.device("cuda:0")
    tu = torch.from_numpy(uvw).to(dev)
    tv = torch.from_numpy(vis.astype(np.complex64)).to(dev)
    res = {}
    for alpha in (1, 2):
        im = P.Imager(m * alpha, 1, fov_img * alpha, kernel="kb", support=7, tile=16,
                      max_vis=M, device=dev, image_n=m)
        img = im.image(tu, tv, None).cpu().numpy()
        res[alpha] = np.abs(img - ref).max() / np.abs(ref).max()
        im.close()
    print(f"vs DFT: unpadded {res[1]:.2e}, padded by 2 {res[2]:.2e}")
    assert res[2] <= 2e-5 and res[1] >= 1e-2
