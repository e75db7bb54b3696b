"""Gradients through the imaging operator and the degridding predictor.

GridFn's backward must equal the oracle's adjoint of the image operator;
DegridFn's chi^2 gradient must match central finite differences of the FP64
oracle's predictor and the exact gradient -2 Re D^H w (V_obs - D x) computed
by the oracle.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import paper_2411_07321_gb300 as P
    return P


def setup(P, n_keep=30000, n=128, n_w=8, W=7):
    wl = synth.scaled("diff", n_keep=n_keep)
    d = synth.generate(wl.obs)
    # a field of view whose uv cell keeps every footprint on the smaller grid
    fov = 0.9 * (n / 2 - W - 1) / wl.obs.uv_max
    dev = torch.device("cuda:0")
    im = P.Imager(n, n_w, fov, kernel="kb", support=W, tile=16, max_vis=n_keep, device=dev)
    op = oracle.Params(n=n, n_w=n_w, fov=fov, kernel=oracle.KB, support=W, tile=16)
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
    im.bin(t["uvw"], t["vis"], t["weight"])
    torch.cuda.synchronize()
    return im, op, d, t


def taper_2d(op):
    c = np.array([oracle.taper(op, (i - op.n // 2) / op.n) for i in range(op.n)])
    c = c / oracle.taper(op, 0.0)
    return np.outer(c, c)


def test_gridfn_backward_is_oracle_adjoint(P):
    from paper_2411_07321_gb300.autograd import grid_image

    im, op, d, t = setup(P)
    st = im.stats()
    assert st["n_binned"] > 0.9 * len(d["vis"])
    y = (np.random.default_rng(5).normal(size=(op.n, op.n)) * taper_2d(op)).astype(np.float32)
    v = t["vis"].clone().requires_grad_(True)
    img = grid_image(v, im, t["weight"])
    (img * torch.from_numpy(y).to(img.device)).sum().backward()
    g = v.grad.cpu().numpy()
    ref = oracle.adjoint(op, d["uvw"], y.astype(np.float64), d["weight"].astype(np.float64),
                         w_min=st["w_min"], w_max=st["w_max"], sum_weight=st["sum_weight"])
    assert np.abs(g - ref).max() <= 1e-5 * np.abs(ref).max()
    im.close()


def _oracle_chi2(op, d, x, st, vobs, w):
    pred = oracle.adjoint(op, d["uvw"], x, None, flags=oracle.N_DIVIDE, w_min=st["w_min"],
                          w_max=st["w_max"], sum_weight=st["sum_weight"])
    keep = oracle.coords(op, d["uvw"])["status"] == 0
    r = (vobs - pred)[keep]
    return float(np.sum(w[keep] * np.abs(r) ** 2)), pred


def test_chi2_gradient_matches_finite_differences(P):
    from paper_2411_07321_gb300.autograd import chi2

    im, op, d, t = setup(P, n_keep=8000, n=64, n_w=4)
    st = im.stats()
    rng = np.random.default_rng(6)
    # a sparse sky of 50 point sources, as float32 pixels
    x = np.zeros((op.n, op.n))
    idx = rng.choice(op.n * op.n, 50, replace=False)
    x.flat[idx] = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 50))
    x32 = x.astype(np.float32)
    keep = oracle.coords(op, d["uvw"])["status"] == 0
    w = d["weight"].astype(np.float64)
    vobs = d["vis"].astype(np.complex128)

    xt = torch.from_numpy(x32).to("cuda:0").requires_grad_(True)
    wt = t["weight"] * torch.from_numpy(keep.astype(np.float32)).to("cuda:0")
    loss = chi2(xt, im, t["vis"], wt)
    loss.backward()
    g = xt.grad.double().cpu().numpy()

    # exact gradient from the oracle: -2 Re D^H (w (V_obs - D x))
    _, pred = _oracle_chi2(op, d, x32.astype(np.float64), st, vobs, w)
    res = np.where(keep, w * (vobs - pred), 0)
    # D^H of a visibility vector = Re(grid -> inverse FFT -> w-correct) with unit weights
    dh = oracle.image(op, d["uvw"], res, None, flags=oracle.N_DIVIDE)[0]
    exact = -2.0 * dh
    # the gradient ends with the division by C(l) C(m), which amplifies the
    # FP32 rounding of the transform (and its run-to-run variation with the
    # order of the grid kernel's float atomics) by up to max 1/(C C) near the
    # corners: compare before that division, as the image tests do
    cc = taper_2d(op)
    assert np.abs((g - exact) * cc).max() <= 1e-5 * np.abs(exact * cc).max()
    assert np.abs(g - exact).max() <= 1e-3 * np.abs(exact).max()

    # central finite differences of the FP64 oracle at a few pixels
    for p in list(idx[:3]) + [op.n * op.n // 2 + 3]:
        h = 1e-3 * max(abs(x.flat[p]), 1.0)
        xp, xm = x32.astype(np.float64).copy(), x32.astype(np.float64).copy()
        xp.flat[p] += h
        xm.flat[p] -= h
        cp, cm = _oracle_chi2(op, d, xp, st, vobs, w)[0], _oracle_chi2(op, d, xm, st, vobs, w)[0]
        fd = (cp - cm) / (2 * h)
        # chi^2 is quadratic in x: the central difference is exact up to the
        # rounding of the two chi^2 values
        assert abs(fd - exact.flat[p]) <= 1e-6 * abs(exact.flat[p]) + 1e-13 * abs(cp) / h
        assert g.flat[p] == pytest.approx(fd, rel=1e-3, abs=1e-4 * np.abs(exact).max())
    im.close()


@pytest.mark.slow
def test_chi2_gradient_at_full_size(P):
    """The differentiable configuration at its full size: 1e7 visibilities (4
    channels of the LOFAR-like tracks), a 2048^2 grid with 16 w-planes, KB W=7,
    the gradient of chi^2 with respect to a 50-source float32 image -- against
    the oracle's exact gradient -2 Re D^H w (V_obs - D x) and central finite
    differences of the oracle's chi^2 at sampled pixels."""
    from paper_2411_07321_gb300.autograd import chi2

    wl = synth.WORKLOADS["diff"]
    d = synth.generate(wl.obs)
    dev = torch.device("cuda:0")
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                  max_vis=len(d["vis"]), device=dev)
    op = oracle.Params(n=wl.n, n_w=wl.n_w, fov=wl.fov, kernel=oracle.KB, support=wl.support,
                       tile=wl.tile)
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
    im.bin(t["uvw"], t["vis"], t["weight"])
    torch.cuda.synchronize()
    st = im.stats()
    rng = np.random.default_rng(4)
    x = np.zeros((wl.n, wl.n))
    idx = rng.choice(wl.n * wl.n, 50, replace=False)
    x.flat[idx] = np.exp(rng.uniform(np.log(0.1), np.log(10.0), 50))
    x32 = x.astype(np.float32)
    keep = oracle.coords(op, d["uvw"])["status"] == 0
    w = d["weight"].astype(np.float64)
    vobs = d["vis"].astype(np.complex128)
    xt = torch.from_numpy(x32).to(dev).requires_grad_(True)
    wt = t["weight"] * torch.from_numpy(keep.astype(np.float32)).to(dev)
    chi2(xt, im, t["vis"], wt).backward()
    g = xt.grad.double().cpu().numpy()
    im.close()

    _, pred = _oracle_chi2(op, d, x32.astype(np.float64), st, vobs, w)
    res = np.where(keep, w * (vobs - pred), 0)
    exact = -2.0 * oracle.image(op, d["uvw"], res, None, flags=oracle.N_DIVIDE)[0]
    c = oracle.taper_row(op)
    c = c / c[wl.n // 2]
    cc = np.outer(c, c)
    e_tap = np.abs((g - exact) * cc).max() / np.abs(exact * cc).max()
    e_raw = np.abs(g - exact).max() / np.abs(exact).max()
    print(f"full-size chi^2 gradient vs oracle: tapered {e_tap:.2e}, raw {e_raw:.2e}")
    assert e_tap <= 1e-5 and e_raw <= 1e-3
    for p in list(idx[:2]) + [wl.n * wl.n // 2 + 3]:
        h = 1e-3 * max(abs(x.flat[p]), 1.0)
        xp, xm = x32.astype(np.float64).copy(), x32.astype(np.float64).copy()
        xp.flat[p] += h
        xm.flat[p] -= h
        cp, cm = _oracle_chi2(op, d, xp, st, vobs, w)[0], _oracle_chi2(op, d, xm, st, vobs, w)[0]
        fd = (cp - cm) / (2 * h)
        assert abs(fd - exact.flat[p]) <= 1e-6 * abs(exact.flat[p]) + 1e-13 * abs(cp) / h
        assert g.flat[p] == pytest.approx(fd, rel=1e-3, abs=1e-4 * np.abs(exact).max())
