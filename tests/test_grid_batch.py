"""One gridding launch for several imaging jobs (rick_grid_sparse_batch).

Each job's planes after the merged launch hold what its own rick_grid_sparse
writes: the same tiles (the record-free ones keep what they held) with the same
sums, added in another order by the float atomics, so they agree to FP32
rounding (1e-5 of the plane peak, the plane tolerance of test_gpu_parity), and
so do the images the fused transform makes of them, compared before the taper
division (which amplifies the planes' FP32 rounding near the image corners by up
to max 1/(C C), as in test_fft_fused).  The jobs differ in grid
size, plane count, kernel and visibility count; they share support and tile,
as the entry point requires, and its host checks reject the rest.
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


@pytest.fixture(scope="module")
def data():
    d = synth.generate(synth.scaled("small", n_keep=65_536).obs)
    dev = torch.device("cuda:0")
    return {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}


SPECS = [(256, 4, "kb", 20_000), (512, 9, "gauss", 65_536), (1024, 3, "kb", 40_000),
         (512, 1, "kb", 0)]


def make(P, data, specs, support=7, tile=32, precision="fp32"):
    ims = []
    for n, n_w, kernel, n_vis in specs:
        fov = 2.0 * math.pi / 180 * n / 256
        im = P.Imager(n, n_w, fov, kernel=kernel, support=support, tile=tile,
                      precision=precision, max_vis=max(n_vis, 1), device=data["uvw"].device)
        im.bin(data["uvw"][:n_vis], data["vis"][:n_vis], data["weight"][:n_vis])
        ims.append(im)
    return ims


def taper_2d(n, kernel, support=7):
    """C(l_p) C(m_q) / C(0)^2 over the n x n pixels, from the oracle."""
    op = oracle.Params(n=n, n_w=1, fov=0.03, kernel=oracle.KB if kernel == "kb" else oracle.GAUSS,
                       support=support, tile=8)
    c = np.array([oracle.taper(op, (i - n // 2) / n) for i in range(n)])
    c = c / oracle.taper(op, 0.0)
    return torch.from_numpy(c[:, None] * c[None, :])


def rel(a, b, cc=None):
    wide = torch.complex128 if a.is_complex() else torch.float64
    a, b = a.cpu().to(wide), b.cpu().to(wide)
    if cc is not None:
        a, b = a * cc, b * cc
    d = torch.where(torch.isnan(b), torch.zeros_like(b), a - b)
    return float(d.abs().max()) / max(float(torch.nan_to_num(b).abs().max()), 1e-30)


def test_batch_equals_per_job_gridding(P, data):
    ims = make(P, data, SPECS)
    tapers = [taper_2d(n, kernel) for n, _, kernel, _ in SPECS]
    ref_planes, ref_img = [], []
    for im in ims:
        im.planes.fill_(float("nan"))
        im.grid_sparse()
        ref_planes.append(im.planes.clone())
        ref_img.append(im.fft_wcorrect(sparse=True).clone())
    for rep in range(2):  # twice in a row: the batch resets its own counter
        for im in ims:
            im.planes.fill_(float("nan"))
        P.grid_sparse_batch(ims)
        torch.cuda.synchronize()
        for j, im in enumerate(ims):
            # the same tiles written (record-free tiles keep the NaN fill)
            assert torch.equal(torch.isnan(im.planes), torch.isnan(ref_planes[j])), (rep, j)
            assert rel(im.planes, ref_planes[j]) <= TOL, (rep, j)
            img = im.fft_wcorrect(sparse=True)
            assert rel(img, ref_img[j], tapers[j]) <= TOL, (rep, j)
    assert int(torch.isnan(ims[-1].planes).sum()) == ims[-1].planes.numel()  # empty job
    for im in ims:
        im.close()


def test_batch_of_one_and_the_limit(P, data):
    ims = make(P, data, SPECS[:1])
    ims[0].planes.fill_(0.0)
    ims[0].grid_sparse()
    ref = ims[0].planes.clone()
    P.grid_sparse_batch(ims)
    assert rel(ims[0].planes, ref) <= TOL
    R = P.rick
    with pytest.raises(R.RickError):  # more jobs than the limit
        R.rick_grid_sparse_batch([ims[0].plan] * (R.RICK_GRID_BATCH_MAX + 1),
                                 [ims[0].ws.data_ptr()] * (R.RICK_GRID_BATCH_MAX + 1),
                                 [ims[0].planes.data_ptr()] * (R.RICK_GRID_BATCH_MAX + 1), None)
    ims[0].close()


@pytest.mark.parametrize("other", [dict(support=5), dict(tile=64),
                                   dict(precision="compensated")])
def test_incompatible_jobs_rejected(P, data, other):
    a = make(P, data, SPECS[:1])[0]
    b = make(P, data, SPECS[1:2], **other)[0]
    with pytest.raises(P.rick.RickError):
        P.grid_sparse_batch([a, b])
    with pytest.raises(P.rick.RickError):  # one workspace for two jobs
        P.rick.rick_grid_sparse_batch([a.plan, a.plan], [a.ws.data_ptr()] * 2,
                                      [a.planes.data_ptr(), b.planes.data_ptr()], None)
    # nothing was enqueued: both plans still work
    a.grid_sparse()
    b.grid_sparse()
    torch.cuda.synchronize()
    a.close()
    b.close()
