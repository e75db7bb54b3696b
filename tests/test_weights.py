"""Imaging weights from the uv-cell density (uniform, Briggs robust) on the GPU.

rick_density_weights must give the oracle's FP64 weights to FP32 accuracy (2e-5
relative), zero for dropped visibilities, after a per-visibility or a
multi-channel binning; an image made with them must be the oracle's image with
the oracle's weights (1e-5 of peak, tapered image and inner region).
"""
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


def setup(P, n, fov, n_keep=65536, W=7):
    d = synth.generate(synth.scaled("small", n_keep=n_keep).obs)
    wt = (0.5 + np.random.default_rng(4).random(len(d["vis"]))).astype(np.float32)
    im = P.Imager(n, 8, fov, kernel="kb", support=W, tile=32 if n >= 32 else 16, max_vis=n_keep,
                  device=torch.device("cuda:0"))
    op = oracle.Params(n=n, n_w=8, fov=fov, kernel=oracle.KB, support=W,
                       tile=32 if n >= 32 else 16)
    return d, wt, im, op


@pytest.mark.parametrize("scheme,robust", [("uniform", 0.0), ("briggs", -1.0), ("briggs", 0.0),
                                           ("briggs", 2.0)])
@pytest.mark.parametrize("n,W", [(256, 7), (128, 6)])  # the 128 grid drops the outer tracks
def test_density_weights_match_oracle(P, scheme, robust, n, W):
    wl = synth.WORKLOADS["small"]
    d, wt, im, op = setup(P, n, wl.fov, W=W)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis")}
    w_dev = torch.from_numpy(wt).to(dev)
    im.bin(t["uvw"], t["vis"], w_dev)
    got = im.density_weights(scheme, robust, w_dev).cpu().numpy().astype(np.float64)
    want = oracle.density_weights(op, d["uvw"], wt, oracle.WEIGHT_UNIFORM if scheme == "uniform"
                                  else oracle.WEIGHT_BRIGGS, robust)
    assert np.array_equal(got == 0.0, want == 0.0)
    if n == 128:
        assert (want == 0.0).any()  # some visibilities were dropped
    nz = want != 0.0
    assert np.abs(got[nz] / want[nz] - 1.0).max() <= 2e-5
    im.close()


def test_briggs_image_matches_oracle(P):
    wl = synth.WORKLOADS["small"]
    d, wt, im, op = setup(P, wl.n, wl.fov)
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis")}
    img = im.image_weighted(t["uvw"], t["vis"], torch.from_numpy(wt).to(dev), "briggs",
                            0.5).cpu().numpy()
    w2 = oracle.density_weights(op, d["uvw"], wt, oracle.WEIGHT_BRIGGS, 0.5)
    ref, st = oracle.image(op, d["uvw"], d["vis"], w2)
    c = np.array([oracle.taper(op, (i - op.n // 2) / op.n) for i in range(op.n)])
    cc = np.outer(c, c) / oracle.taper(op, 0.0) ** 2
    diff = img.astype(np.float64) - ref
    q = op.n // 4
    inner = (slice(op.n // 2 - q, op.n // 2 + q),) * 2
    tap = np.abs(diff * cc).max() / np.abs(ref * cc).max()
    inn = np.abs(diff[inner]).max() / np.abs(ref[inner]).max()
    print(f"briggs image: tapered {tap:.2e} inner {inn:.2e}")
    assert tap <= TOL and inn <= TOL
    assert im.stats()["sum_weight"] == pytest.approx(float(w2.sum()), rel=2e-6)
    im.close()


def test_density_weights_after_channel_binning(P):
    obs = synth.scaled("lofar", n_keep=16 * 3000).obs
    d = synth.generate(obs, rows=True)
    n, fov = 512, (512 / 2 - 8) / 12000.0
    im = P.Imager(n, 8, fov, kernel="kb", support=7, tile=32, max_vis=len(d["vis"]),
                  device=torch.device("cuda:0"))
    dev = torch.device("cuda:0")
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw_rows", "chan_scale", "vis", "weight")}
    im.bin_channels(t["uvw_rows"], t["chan_scale"], t["vis"], t["weight"])
    got = im.density_weights("uniform", 0.0, t["weight"]).cpu().numpy().astype(np.float64)
    op = oracle.Params(n=n, n_w=8, fov=fov, kernel=oracle.KB, support=7, tile=32)
    want = oracle.density_weights(op, d["uvw"], d["weight"], oracle.WEIGHT_UNIFORM)
    nz = want != 0.0
    assert np.array_equal(got == 0.0, ~nz)
    assert np.abs(got[nz] / want[nz] - 1.0).max() <= 2e-5
    im.close()
