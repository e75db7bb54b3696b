"""Pins of the FP64 oracle against things other than itself.

Each test fixes the oracle to a closed form, a textbook library routine, exact
rational arithmetic, the brute-force transform of Eq. 1, or an invariant the
mathematics guarantees, chosen so that a dropped term, a wrong sign, an
off-by-one shift or a transposed axis fails at least one of them.
"""
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.special as sp

import oracle
import synth

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def rng(seed):
    return np.random.default_rng(seed)


# ---------------------------------------------------------------- kernel / I0 / taper

@pytest.mark.parametrize("x", [0.0, 1e-3, 0.5, 3.75, 9.0, 16.25, 21.0, 30.0])
def test_i0_series_matches_scipy(x):
    assert oracle.i0(x) == pytest.approx(float(sp.i0(x)), rel=1e-13, abs=0)


def test_i0_matches_tabulated_values():
    """I0 against the published table in tests/golden/bessel_i0.txt (10 digits)."""
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "bessel_i0.txt")
    rows = [l.split() for l in open(path) if l.strip() and not l.startswith("#")]
    assert len(rows) >= 5
    for x, v in rows:
        assert oracle.i0(float(x)) == pytest.approx(float(v), rel=5e-10)


@pytest.mark.parametrize("W", [3, 5, 7, 9])
def test_kb_kernel_ends_and_centre(W):
    p = oracle.Params(n=64, n_w=1, fov=0.01, kernel=oracle.KB, support=W, tile=16)
    beta = oracle.kb_beta_default(W)
    assert oracle.kernel(p, 0.0) == pytest.approx(1.0, rel=1e-15)
    assert oracle.kernel(p, W / 2) == pytest.approx(1.0 / sp.i0(beta), rel=1e-13)
    assert oracle.kernel(p, -W / 2) == oracle.kernel(p, W / 2)
    assert oracle.kernel(p, W / 2 + 1e-9) == 0.0
    d = 0.37
    t = 2 * d / W
    assert oracle.kernel(p, d) == pytest.approx(sp.i0(beta * np.sqrt(1 - t * t)) / sp.i0(beta),
                                                rel=1e-13)


def test_gauss_kernel_and_delta():
    p = oracle.Params(n=64, n_w=1, fov=0.01, kernel=oracle.GAUSS, support=7, tile=16)
    s = 7 / 6
    for d in (0.0, 0.3, -1.7, 3.5):
        assert oracle.kernel(p, d) == pytest.approx(np.exp(-d * d / (2 * s * s)), rel=1e-15)
    p1 = oracle.Params(n=64, n_w=1, fov=0.01, kernel=oracle.KB, support=1, tile=16)
    assert oracle.kernel(p1, 0.4) == 1.0 and oracle.taper(p1, 0.3) == 1.0


@pytest.mark.parametrize("W", [2, 3, 5, 7, 9])
def test_taper_kb_closed_form(W):
    """Jackson (1991): integral of I0(beta sqrt(1-(2d/W)^2)) e^{-2 pi i nu d} over
    |d| <= W/2 equals W sinh(sqrt(beta^2 - (pi W nu)^2)) / sqrt(...)."""
    p = oracle.Params(n=64, n_w=1, fov=0.01, kernel=oracle.KB, support=W, tile=16)
    beta = oracle.kb_beta_default(W)
    for nu in (0.0, 0.05, 0.2, 0.37, 0.5):
        z = complex(beta ** 2 - (np.pi * W * nu) ** 2) ** 0.5
        closed = (W * np.sinh(z) / z).real / sp.i0(beta) if abs(z) > 0 else W / sp.i0(beta)
        assert oracle.taper(p, nu) == pytest.approx(closed, rel=1e-12)


@pytest.mark.parametrize("W,sigma", [(7, 7 / 6), (5, 0.9), (9, 1.8)])
def test_taper_gauss_closed_form(W, sigma):
    """Truncated Gaussian: integral_{-a}^{a} e^{-d^2/(2 s^2)} cos(2 pi nu d) dd =
    sqrt(pi/al) e^{-k^2/(4 al)} Re erf(sqrt(al) a + i k / (2 sqrt(al)))."""
    p = oracle.Params(n=64, n_w=1, fov=0.01, kernel=oracle.GAUSS, support=W, gauss_sigma=sigma,
                      tile=16)
    a, al = W / 2, 1 / (2 * sigma ** 2)
    for nu in (0.0, 0.1, 0.25, 0.5):
        k = 2 * np.pi * nu
        closed = np.sqrt(np.pi / al) * np.exp(-k * k / (4 * al)) * \
            sp.erf(np.sqrt(al) * a + 1j * k / (2 * np.sqrt(al))).real
        assert oracle.taper(p, nu) == pytest.approx(closed, rel=1e-12)


# ---------------------------------------------------------------- FFT

@pytest.mark.parametrize("n", [2, 4, 8, 16, 32, 64])
@pytest.mark.parametrize("sign", [+1, -1])
def test_fft1d_matches_naive_dft(n, sign):
    x = rng(n).normal(size=n) + 1j * rng(n + 1).normal(size=n)
    j = np.arange(n)
    naive = np.exp(sign * 2j * np.pi * np.outer(j, j) / n) @ x
    assert np.abs(oracle.fft1d(x, sign) - naive).max() <= 1e-12 * np.abs(naive).max()


def test_fft2d_matches_numpy_and_parseval():
    n = 128
    x = rng(3).normal(size=(n, n)) + 1j * rng(4).normal(size=(n, n))
    inv = oracle.fft2d(x, +1)
    assert np.abs(inv - np.fft.ifft2(x) * n * n).max() <= 1e-11 * np.abs(inv).max()
    fwd = oracle.fft2d(x, -1)
    assert np.abs(fwd - np.fft.fft2(x)).max() <= 1e-11 * np.abs(fwd).max()
    assert (np.abs(fwd) ** 2).sum() == pytest.approx(n * n * (np.abs(x) ** 2).sum(), rel=1e-12)
    # transposed-axis mistakes would break this non-square-symmetric case
    y = np.zeros((n, n), complex)
    y[0, 1] = 1.0
    assert np.allclose(oracle.fft2d(y, +1)[0, :], np.exp(2j * np.pi * np.arange(n) / n))


# ---------------------------------------------------------------- geometry (exact arithmetic)

def _fma_exact(a, b, c):
    return float(Fraction(a) * Fraction(b) + Fraction(c))


def _ref_axis(u, fov, n, W):
    """Footprint of one axis from exact rational arithmetic."""
    x = _fma_exact(u, fov, n / 2)
    X = Fraction(x)
    h = (W - 1) // 2 if W % 2 else W // 2 - 1
    c = int(np.floor(X + Fraction(1, 2))) if W % 2 else int(np.floor(X))
    a = c - h
    ok = a >= 0 and a + W - 1 <= n - 1
    return ok, a, float(X - c)


@pytest.mark.parametrize("W", [1, 4, 7])
def test_coords_match_exact_rational_reference(W):
    n, nw, fov = 64, 5, 0.03125 * 0.7
    r = rng(10 + W)
    m = 400
    u = r.uniform(-1.2, 1.2, m) * (n / 2) / fov
    v = r.uniform(-1.2, 1.2, m) * (n / 2) / fov
    # exact half-cell positions and cell centres exercise the rounding ties
    u[:20] = (np.arange(20) - 10 + 0.5) / fov
    v[20:40] = (np.arange(20) - 10.0) / fov
    w = r.uniform(-300, 200, m)
    uvw = np.stack([u, v, w], 1)
    p = oracle.Params(n=n, n_w=nw, fov=fov, kernel=oracle.KB, support=W, tile=16)
    g = oracle.coords(p, uvw)
    wmin, wmax = w.min(), w.max()
    assert (g["w_min"], g["w_max"]) == (wmin, wmax)
    dw = (wmax - wmin) / nw
    bounds = [_fma_exact(j, dw, wmin) for j in range(1, nw)]
    for i in range(m):
        okx, ax, fx = _ref_axis(u[i], fov, n, W)
        oky, ay, fy = _ref_axis(v[i], fov, n, W)
        if not (okx and oky):
            assert g["status"][i] == 1
            continue
        assert g["status"][i] == 0
        assert (g["ax"][i], g["ay"][i]) == (ax, ay)
        assert (g["fx"][i], g["fy"][i]) == (fx, fy)
        if W % 2:
            assert -0.5 <= fx < 0.5
        k = sum(w[i] >= b for b in bounds)
        assert g["plane"][i] == k


def test_coords_given_w_range_drops_and_degenerate_range():
    n, fov = 32, 0.05
    uvw = np.array([[0.0, 0.0, -5.0], [0.0, 0.0, 0.0], [0.0, 0.0, 5.0], [0.0, 0.0, 10.0],
                    [1e9, 0.0, 0.0]])
    p = oracle.Params(n=n, n_w=4, fov=fov, kernel=oracle.GAUSS, support=3, w_min=0.0, w_max=5.0,
                      tile=16)
    g = oracle.coords(p, uvw)
    assert list(g["status"]) == [2, 0, 0, 2, 1]
    assert list(g["plane"][1:3]) == [0, 3]  # w == w_max lands in the top plane
    p0 = oracle.Params(n=n, n_w=4, fov=fov, kernel=oracle.GAUSS, support=3, tile=16)
    g0 = oracle.coords(p0, np.array([[0.0, 0.0, 7.0], [1.0, 1.0, 7.0]]))
    assert list(g0["plane"]) == [0, 0]  # dw == 0 -> plane 0
    assert oracle.plane_centre(p0, 0, 7.0, 7.0) == 7.0


def test_bin_is_stable_counting_sort_with_edge_classes():
    n, T, W = 128, 16, 5
    p = oracle.Params(n=n, n_w=3, fov=0.02, kernel=oracle.KB, support=W, tile=T)
    r = rng(7)
    m = 3000
    uvw = np.stack([r.normal(0, 1500, m), r.normal(0, 1500, m), r.uniform(-50, 50, m)], 1)
    uvw[::7] = uvw[3]  # many exact repeats: stability is observable
    b = oracle.bin(p, uvw)
    key, perm, off = b["key"], b["perm"], b["offsets"]
    kept = np.flatnonzero(key >= 0)
    assert len(perm) == len(kept) and sorted(perm) == list(kept)
    sk = key[perm]
    assert np.all(np.diff(sk) >= 0)
    same = np.diff(sk) == 0
    assert np.all(np.diff(perm)[same] > 0)  # ties keep input order
    counts = np.bincount(key[kept], minlength=oracle.nbins(p))
    assert np.array_equal(off, np.concatenate([[0], np.cumsum(counts)]))
    nt = n // T
    # the edge class from the footprint itself: enumerate its W x W cells and
    # collect the tiles they fall in, relative to the corner's tile
    by_tiles = {frozenset({(0, 0)}): 0, frozenset({(0, 0), (1, 0)}): 1,
                frozenset({(0, 0), (1, 0), (0, 1), (1, 1)}): 2, frozenset({(0, 0), (0, 1)}): 3}
    classes = set()
    for i in kept:
        ax, ay, k = b["ax"][i], b["ay"][i], b["plane"][i]
        tiles = frozenset(((ax + jx) // T - ax // T, (ay + jy) // T - ay // T)
                          for jx in range(W) for jy in range(W))
        cls = by_tiles[tiles]  # a footprint never reaches west, north or two tiles away
        classes.add(cls)
        assert key[i] == ((k * nt + ay // T) * nt + ax // T) * 4 + cls
    assert classes == {0, 1, 2, 3}  # every class occurs


# ---------------------------------------------------------------- the image vs Eq. 1's DFT

def _grid_node_case(seed, n=64, nw=4, m=300, nodes=True):
    """fov = 2^-4 makes u * fov exact for u on grid nodes (multiples of 1/fov)."""
    fov = 2.0 ** -4
    r = rng(seed)
    if nodes:
        u = (r.integers(-n // 2 + 2, n // 2 - 2, m)) / fov
        v = (r.integers(-n // 2 + 2, n // 2 - 2, m)) / fov
    else:
        u = r.uniform(-n / 2 + 2, n / 2 - 2, m) / fov
        v = r.uniform(-n / 2 + 2, n / 2 - 2, m) / fov
    # w range [-64, 64] in nw planes; plane centres are exact binary fractions
    k = r.integers(0, nw, m)
    dw = 128.0 / nw
    w = -64.0 + (k + 0.5) * dw
    vis = r.normal(size=m) + 1j * r.normal(size=m)
    wt = r.uniform(0.5, 1.5, m)
    p = oracle.Params(n=n, n_w=nw, fov=fov, kernel=oracle.KB, support=1, w_min=-64.0,
                      w_max=64.0, tile=16)
    return p, np.stack([u, v, w], 1), vis, wt


@pytest.mark.parametrize("flags", [0, oracle.N_CORRECT | oracle.NORMALIZE])
def test_exact_special_case_equals_dft(flags):
    """W = 1, u,v on grid nodes, w at plane centres: w-stacking is exact (P1)."""
    p, uvw, vis, wt = _grid_node_case(1)
    img, st = oracle.image(p, uvw, vis, wt, flags=flags)
    assert st["n_binned"] == len(vis)
    ref = oracle.dft(p.n, p.fov, uvw, vis, wt, flags=flags, sum_weight=wt.sum())
    assert np.abs(img - ref).max() <= 1e-12 * np.abs(ref).max()


def test_snapped_dft():
    """W = 1, arbitrary uvw: the image is the DFT at the snapped (u', v', w_k) (P2)."""
    p, uvw, vis, wt = _grid_node_case(2, nodes=False)
    uvw[:, 2] = rng(5).uniform(-64, 64, len(vis))
    img, _ = oracle.image(p, uvw, vis, wt, flags=0)
    g = oracle.coords(p, uvw)
    snapped = np.stack([(g["ax"] - p.n / 2) / p.fov, (g["ay"] - p.n / 2) / p.fov,
                        [oracle.plane_centre(p, k, -64.0, 64.0) for k in g["plane"]]], 1)
    ref = oracle.dft(p.n, p.fov, snapped, vis, wt, flags=0)
    assert np.abs(img - ref).max() <= 1e-12 * np.abs(ref).max()


def _point_source_vis(uvw, l0, m0, flux):
    n0 = np.sqrt(1 - l0 * l0 - m0 * m0)
    ph = -2j * np.pi * (uvw[:, 0] * l0 + uvw[:, 1] * m0 + uvw[:, 2] * (n0 - 1))
    return flux / n0 * np.exp(ph)  # Eq. 1 for a point source


def test_point_source_flux_exact_and_dft_sign():
    """A source of flux S at a pixel centre comes back as S there (P4, W = 1)."""
    p, uvw, _, wt = _grid_node_case(3, m=500)
    p0, q0, S = 40, 21, 3.25
    dl = p.fov / p.n
    vis = _point_source_vis(uvw, (p0 - p.n / 2) * dl, (q0 - p.n / 2) * dl, S)
    f = oracle.N_CORRECT | oracle.NORMALIZE
    img, _ = oracle.image(p, uvw, vis, wt, flags=f)
    assert img[q0, p0] == pytest.approx(S, rel=1e-12)
    assert np.unravel_index(np.argmax(img), img.shape) == (q0, p0)
    ref = oracle.dft(p.n, p.fov, uvw, vis, wt, flags=f, sum_weight=wt.sum())
    assert ref[q0, p0] == pytest.approx(S, rel=1e-12)


@pytest.mark.parametrize("kern,W", [(oracle.KB, 7), (oracle.GAUSS, 7), (oracle.KB, 9)])
def test_point_source_flux_with_taper(kern, W):
    """Tapered kernels recover the flux to the kernel's accuracy (reported, P4/P3)."""
    n, fov = 128, 2.0 ** -4
    r = rng(11)
    m = 4000
    uvw = np.stack([r.uniform(-40, 40, m) / fov, r.uniform(-40, 40, m) / fov,
                    r.uniform(-30, 30, m)], 1)
    p = oracle.Params(n=n, n_w=8, fov=fov, kernel=kern, support=W, tile=16)
    p0, q0, S = 70, 50, 2.0
    dl = fov / n
    vis = _point_source_vis(uvw, (p0 - n / 2) * dl, (q0 - n / 2) * dl, S)
    img, _ = oracle.image(p, uvw, vis, None)
    assert abs(img[q0, p0] - S) / S < 5e-3


def test_hermitian_mirror_gives_real_image():
    """Gridding (u,v,w,V) and (-u,-v,-w,conj V) yields a real sum over planes
    (P5) and the same normalised image as the original data alone."""
    n, fov, W = 64, 0.05, 7
    r = rng(12)
    m = 600
    lim = (n / 2 - W - 2) / fov
    uvw = np.stack([r.uniform(-lim, lim, m), r.uniform(-lim, lim, m), r.uniform(-500, 500, m)], 1)
    vis = r.normal(size=m) + 1j * r.normal(size=m)
    wt = r.uniform(0.5, 1.5, m)
    p = oracle.Params(n=n, n_w=8, fov=fov, kernel=oracle.KB, support=W, w_min=-512.0, w_max=512.0,
                      tile=16)
    both = np.concatenate([uvw, -uvw])
    img2, acc2, _ = oracle.image(p, both, np.concatenate([vis, vis.conj()]),
                                 np.concatenate([wt, wt]), want_acc=True)
    peak = np.abs(acc2).max()
    assert np.abs(acc2.imag).max() <= 1e-12 * peak
    img1, _ = oracle.image(p, uvw, vis, wt)
    assert np.abs(img2 - img1).max() <= 1e-12 * np.abs(img1).max()


def test_weight_sum_identity_and_centre_pixel():
    """Sum over cells of g_k = sum_m w V (sum_j Gx)(sum_j Gy), and the centre
    pixel of the image is that total over C(0)^2 sum w (P6)."""
    n, fov, W = 64, 0.05, 5
    r = rng(13)
    m = 500
    lim = (n / 2 - W) / fov
    uvw = np.stack([r.uniform(-lim, lim, m), r.uniform(-lim, lim, m), r.uniform(-100, 100, m)], 1)
    vis = r.normal(size=m) + 1j * r.normal(size=m)
    wt = r.uniform(0.5, 1.5, m)
    p = oracle.Params(n=n, n_w=4, fov=fov, kernel=oracle.GAUSS, support=W, tile=16)
    planes, st = oracle.grid(p, uvw, vis, wt)
    g = oracle.coords(p, uvw)
    h = (W - 1) // 2
    sx = np.array([sum(oracle.kernel(p, (j - h) - f) for j in range(W)) for f in g["fx"]])
    sy = np.array([sum(oracle.kernel(p, (j - h) - f) for j in range(W)) for f in g["fy"]])
    for k in range(p.n_w):
        sel = (g["plane"] == k)
        want = np.sum(wt[sel] * vis[sel] * sx[sel] * sy[sel])
        assert planes[k].sum() == pytest.approx(want, rel=1e-12)
    img, _ = oracle.image(p, uvw, vis, wt, flags=oracle.NORMALIZE)
    total = sum(planes[k].sum() for k in range(p.n_w)).real
    c0 = oracle.taper(p, 0.0)
    assert img[n // 2, n // 2] == pytest.approx(total / (c0 * c0 * wt.sum()), rel=1e-12)


def test_linearity():
    n, fov = 32, 0.04
    r = rng(14)
    m = 200
    uvw = np.stack([r.uniform(-300, 300, m), r.uniform(-300, 300, m), r.uniform(-80, 80, m)], 1)
    v1 = r.normal(size=m) + 1j * r.normal(size=m)
    v2 = r.normal(size=m) + 1j * r.normal(size=m)
    p = oracle.Params(n=n, n_w=4, fov=fov, kernel=oracle.KB, support=5, tile=16)
    a, b = 0.7, -1.9
    i12, _ = oracle.image(p, uvw, a * v1 + b * v2)
    i1, _ = oracle.image(p, uvw, v1)
    i2, _ = oracle.image(p, uvw, v2)
    assert np.abs(i12 - (a * i1 + b * i2)).max() <= 1e-12 * np.abs(i12).max()


@pytest.mark.parametrize("flags,weighted", [(oracle.N_CORRECT | oracle.NORMALIZE, True),
                                            (oracle.N_DIVIDE, False), (0, True)])
def test_adjoint_dot_product(flags, weighted):
    """<A x, y> = Re <x, A^H y> for the image operator and its transpose (P9)."""
    n, fov, W = 64, 0.06, 7
    r = rng(15)
    m = 700
    lim = (n / 2 - 1) / fov
    uvw = np.stack([r.uniform(-lim, lim, m), r.uniform(-lim, lim, m), r.uniform(-400, 400, m)], 1)
    x = r.normal(size=m) + 1j * r.normal(size=m)
    y = r.normal(size=(n, n))
    wt = r.uniform(0.5, 1.5, m) if weighted else None
    p = oracle.Params(n=n, n_w=6, fov=fov, kernel=oracle.KB, support=W, tile=16)
    ax, st = oracle.image(p, uvw, x, wt, flags=flags)
    aty = oracle.adjoint(p, uvw, y, wt, flags=flags, w_min=st["w_min"], w_max=st["w_max"],
                         sum_weight=st["sum_weight"])
    lhs = np.sum(ax * y)
    rhs = np.real(np.sum(x * np.conj(aty)))
    # both sides are sums of many signed terms: bound the error by their magnitude
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(ax * y))
    dropped = oracle.coords(p, uvw)["status"] != 0
    assert np.all(aty[dropped] == 0)


def test_single_plane_zero_w_is_plain_2d_imaging():
    """n_w = 1 with w == 0: the phase screen is exactly 1 (P11)."""
    p, uvw, vis, wt = _grid_node_case(16)
    uvw[:, 2] = 0.0
    p.w_min, p.w_max = float("nan"), float("nan")
    p1 = oracle.Params(**{**p.__dict__, "n_w": 1})
    img1, st = oracle.image(p1, uvw, vis, wt, flags=0)
    assert st["w_min"] == st["w_max"] == 0.0
    ref = oracle.dft(p.n, p.fov, uvw, vis, wt, flags=0)
    assert np.abs(img1 - ref).max() <= 1e-12 * np.abs(ref).max()
    img4, _ = oracle.image(oracle.Params(**{**p.__dict__, "n_w": 4}), uvw, vis, wt, flags=0)
    assert np.abs(img4 - img1).max() <= 1e-13 * np.abs(ref).max()


# ---------------------------------------------------------------- the input generator

@pytest.mark.parametrize("name,n_keep", [("small", 5000), ("lofar", 20000), ("lofar", 16 * 1000 + 5)])
def test_generator_rows_times_channel_factors(name, n_keep):
    """The per-visibility uvw of the generator is the per-row uvw times the
    channel factor, one FP64 product per coordinate: the multi-channel input
    form (rows and factors) describes exactly the same visibilities."""
    obs = synth.scaled(name, n_keep=n_keep).obs
    d = synth.generate(obs, rows=True)
    nc = obs.n_chan
    assert d["uvw_rows"].shape == ((n_keep + nc - 1) // nc, 3)
    assert np.array_equal(d["chan_scale"], (obs.nu0 + np.arange(nc) * obs.dnu) / obs.nu0)
    full = (d["uvw_rows"][:, None, :] * d["chan_scale"][None, :, None]).reshape(-1, 3)[:n_keep]
    assert np.array_equal(full, d["uvw"])
    # the visibilities are those of the per-visibility call
    d2 = synth.generate(obs)
    assert np.array_equal(d2["vis"], d["vis"]) and np.array_equal(d2["uvw"], d["uvw"])


# ---------------------------------------------------------------- imaging weights

def test_density_weights_hand_example():
    """Three visibilities, two in one cell (weights 1 and 2) and one alone
    (weight 4): densities 3 and 4.  Uniform: 1/3, 2/3, 1.  Briggs R = 0:
    f^2 = 25 / ((3^2 + 4^2) / 7) = 7, weights 1/22, 2/22, 4/29."""
    n, fov = 64, 0.01
    p = oracle.Params(n=n, n_w=1, fov=fov, kernel=oracle.KB, support=1, tile=16)
    cell = 1.0 / fov
    uvw = np.array([[3 * cell, 2 * cell, 0.0], [3.2 * cell, 1.9 * cell, 0.0],
                    [-5 * cell, 7 * cell, 0.0]])
    wt = np.array([1.0, 2.0, 4.0])
    u = oracle.density_weights(p, uvw, wt, oracle.WEIGHT_UNIFORM)
    assert u == pytest.approx([1 / 3, 2 / 3, 1.0], rel=1e-15)
    b = oracle.density_weights(p, uvw, wt, oracle.WEIGHT_BRIGGS, 0.0)
    assert b == pytest.approx([1 / 22, 2 / 22, 4 / 29], rel=1e-15)


def test_density_weights_limits_and_cell_sums():
    """Uniform: the new weights of every occupied cell sum to 1.  Briggs tends
    to natural weighting as R grows and to uniform (up to one factor f^2) as R
    falls.  Dropped visibilities get 0."""
    d = synth.generate(synth.scaled("small", n_keep=20000).obs)
    wl = synth.WORKLOADS["small"]
    n = 64  # the outer uv tracks leave this grid: some visibilities are dropped
    p = oracle.Params(n=n, n_w=wl.n_w, fov=1.0 * np.pi / 180, kernel=oracle.KB, support=7,
                      tile=16)
    wt = 0.5 + rng(3).random(len(d["vis"]))
    g = oracle.coords(p, d["uvw"])
    kept = g["status"] == 0
    assert (~kept).any() and kept.any()
    uni = oracle.density_weights(p, d["uvw"], wt, oracle.WEIGHT_UNIFORM)
    assert np.all(uni[~kept] == 0.0)
    cells = (g["ay"][kept] + 3) * n + g["ax"][kept] + 3
    sums = np.bincount(cells, weights=uni[kept])
    assert np.allclose(sums[np.unique(cells)], 1.0, rtol=1e-12)
    nat = oracle.density_weights(p, d["uvw"], wt, oracle.WEIGHT_BRIGGS, 8.0)
    assert np.allclose(nat[kept], wt[kept], rtol=1e-6)
    rob = oracle.density_weights(p, d["uvw"], wt, oracle.WEIGHT_BRIGGS, -8.0)
    ratio = rob[kept] / uni[kept]
    assert np.allclose(ratio, ratio[0], rtol=1e-6)


# ---------------------------------------------------------------- sampled pixels

@pytest.mark.parametrize("W,n_w,kern", [(7, 8, oracle.KB), (4, 3, oracle.GAUSS), (1, 1, oracle.KB)])
def test_image_pixels_equal_fft_image(W, n_w, kern):
    """The per-visibility evaluation of chosen pixels equals the FFT image there
    (the two routes compute the same sums in a different order)."""
    d = synth.generate(synth.scaled("small", n_keep=3000).obs)
    wl = synth.WORKLOADS["small"]
    n = 64
    p = oracle.Params(n=n, n_w=n_w, fov=wl.fov / 4, kernel=kern, support=W, tile=16)
    wt = 0.5 + rng(9).random(len(d["vis"]))
    img, _ = oracle.image(p, d["uvw"], d["vis"], wt)
    pix = [(n // 2, n // 2), (0, 0), (n - 1, 3), (17, 40), (n // 2 + 5, n // 2 - 9), (63, 63)]
    got = oracle.image_pixels(p, d["uvw"], d["vis"], wt, pix)
    want = np.array([img[q, pp] for pp, q in pix])
    assert got == pytest.approx(want, rel=1e-10, abs=1e-12 * np.abs(img).max())


# ---------------------------------------------------------------- grid padding and crop

def _padding_case(m_img=64, fov_img=2.0 ** -4, M=3000, seed=31):
    """Three point sources, two near the edges of an m_img-pixel field, w = 0
    (so that the only error left is the gridding's aliasing)."""
    r = rng(seed)
    lim = (m_img / 2 - 5) / fov_img
    uvw = np.stack([r.uniform(-lim, lim, M), r.uniform(-lim, lim, M), np.zeros(M)], 1)
    dl = fov_img / m_img
    vis = sum(_point_source_vis(uvw, a * dl, b * dl, S)
              for a, b, S in ((28.0, -27.0, 1.0), (3.0, -2.0, 0.5), (-31.3, 29.6, 0.7)))
    return uvw, vis, fov_img


@pytest.mark.parametrize("kern,W,alpha,tol", [(oracle.KB, 7, 2, 1e-6), (oracle.KB, 9, 2, 1e-8),
                                              (oracle.KB, 7, 4, 1e-6), (oracle.GAUSS, 7, 2, 2e-3)])
def test_padding_cuts_aliasing_against_dft(kern, W, alpha, tol):
    """The central crop of a grid padded by alpha is the brute-force DFT of the
    kept field to the kernel's aliasing level, where the unpadded grid of the
    same pixel size is off by percents near the edges.  An offset crop, a wrong
    pixel size or a wrong phase centre would miss the DFT by far more."""
    uvw, vis, fov_img = _padding_case()
    m = 64
    f = oracle.N_CORRECT | oracle.NORMALIZE
    ref = oracle.dft(m, fov_img, uvw, vis, None, flags=f, sum_weight=float(len(vis)))
    peak = np.abs(ref).max()
    n = m * alpha
    p = oracle.Params(n=n, n_w=1, fov=fov_img * alpha, kernel=kern, support=W, tile=16, image_n=m)
    img, st = oracle.image(p, uvw, vis, None, flags=f)
    assert img.shape == (m, m) and st["n_binned"] == len(vis)
    err = np.abs(img - ref).max() / peak
    p1 = oracle.Params(n=m, n_w=1, fov=fov_img, kernel=kern, support=W, tile=16)
    img1, _ = oracle.image(p1, uvw, vis, None, flags=f)
    err1 = np.abs(img1 - ref).max() / peak
    print(f"padding {alpha}: {err:.2e} (unpadded {err1:.2e})")
    assert err <= tol and err1 >= 1e-2
    # image_n == n is the uncropped image
    p2 = oracle.Params(n=m, n_w=1, fov=fov_img, kernel=kern, support=W, tile=16, image_n=m)
    assert np.array_equal(oracle.image(p2, uvw, vis, None, flags=f)[0], img1)


@pytest.mark.parametrize("n,m", [(64, 32), (64, 46)])  # offsets 16 and 9 (odd)
def test_crop_adjoint_dot_product(n, m):
    """<A x, y> = Re <x, A^H y> with A the cropped image operator: the adjoint
    zero-pads the m x m image into the n x n grid frame (P9)."""
    fov, W = 0.06, 7
    r = rng(32)
    M = 600
    lim = (n / 2 - 1) / fov
    uvw = np.stack([r.uniform(-lim, lim, M), r.uniform(-lim, lim, M), r.uniform(-300, 300, M)], 1)
    x = r.normal(size=M) + 1j * r.normal(size=M)
    y = r.normal(size=(m, m))
    wt = r.uniform(0.5, 1.5, M)
    p = oracle.Params(n=n, n_w=5, fov=fov, kernel=oracle.KB, support=W, tile=16, image_n=m)
    f = oracle.N_CORRECT | oracle.NORMALIZE
    ax, st = oracle.image(p, uvw, x, wt, flags=f)
    aty = oracle.adjoint(p, uvw, y, wt, flags=f, w_min=st["w_min"], w_max=st["w_max"],
                         sum_weight=st["sum_weight"])
    lhs = np.sum(ax * y)
    rhs = np.real(np.sum(x * np.conj(aty)))
    assert abs(lhs - rhs) <= 1e-12 * np.sum(np.abs(ax * y))
    # and the crop is the central block of the uncropped image at the same pixels
    full, _ = oracle.image(oracle.Params(n=n, n_w=5, fov=fov, kernel=oracle.KB, support=W,
                                         tile=16), uvw, x, wt, flags=f)
    o = (n - m) // 2
    assert np.array_equal(ax, full[o:o + m, o:o + m])


@pytest.mark.parametrize("W,alpha", [(4, 1.5), (7, 1.5), (9, 1.5), (4, 2.0), (7, 2.0), (9, 2.0),
                                     (4, 3.0), (7, 3.0)])
def test_kb_beta_puts_first_taper_zero_past_the_alias_edge(W, alpha):
    """Beatty et al.'s KB shape for oversampling alpha: the kernel's transform C
    (here by quadrature of G, not its closed form) stays positive out to the
    first alias of the image edge, nu = 1 - 1/(2 alpha) grid units, and turns
    negative just beyond it."""
    beta = oracle.kb_beta(W, alpha)
    p = oracle.Params(n=64, n_w=1, fov=0.05, kernel=oracle.KB, support=W, kb_beta=beta, tile=16)
    edge = 1.0 - 1.0 / (2.0 * alpha)
    assert all(oracle.taper(p, nu) > 0 for nu in np.linspace(0.0, edge, 25))
    assert oracle.taper(p, edge + 0.2 / W ** 2 + 0.01 / W) < 0
    if alpha == 2.0:
        assert beta == oracle.kb_beta_default(W)
