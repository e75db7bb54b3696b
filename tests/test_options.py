"""The plan options and the imaginary-part flag, through the C ABI.

- RICK_OPT_HERMITIAN_MIRROR grids every visibility twice, V at (u, v, w) and
  conj(V) at (-u, -v, -w).  Against the oracle's image of the explicitly
  mirrored set (the input concatenated with its conjugates at -uvw); the image
  equals the unmirrored one made with the same, symmetric, w-planes (the real
  part is already the Hermitian part; with other planes the two differ by the
  w-quantisation of the method, 3e-3 of peak here);
  the imaginary part of the plane sum (RICK_IMAG_PART) vanishes to the FP32
  floor, where for the unmirrored set it is that of the oracle's plane sum;
  the adjoint (degridding) of the mirrored binning is the sum of the two
  records' adjoints.
- RICK_OPT_DETERMINISTIC: two bin + grid + transform runs give bitwise equal
  records, planes and images; the records of each bin are in input order, so
  the permutation equals the oracle's stable counting sort bit for bit; the
  image meets the same bars against the oracle.
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


def small(n_keep=40000, seed_shift=0):
    obs = synth.scaled("small", n_keep=n_keep).obs
    obs.seed += seed_shift
    return synth.generate(obs)


def params(wl, **over):
    kw = dict(n=wl.n, n_w=wl.n_w, fov=wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile)
    kw.update(over)
    return kw


def oracle_params(kw):
    return oracle.Params(n=kw["n"], n_w=kw["n_w"], fov=kw["fov"],
                         kernel=oracle.KB if kw["kernel"] == "kb" else oracle.GAUSS,
                         support=kw["support"], tile=kw["tile"])


def cc_of(op):
    c = oracle.taper_row(op)
    c = c / c[op.n // 2]
    return c[:, None] * c[None, :]


def errs(img, ref, op):
    cc = cc_of(op)
    d = img.astype(np.float64) - ref
    q = op.n // 4
    inner = (slice(op.n // 2 - q, op.n // 2 + q),) * 2
    return dict(tapered=np.abs(d * cc).max() / np.abs(ref * cc).max(),
                inner=np.abs(d[inner]).max() / np.abs(ref[inner]).max())


def mirrored(d):
    """The set with every visibility's Hermitian partner appended."""
    return dict(uvw=np.concatenate([d["uvw"], -d["uvw"]]),
                vis=np.concatenate([d["vis"], np.conj(d["vis"])]),
                weight=np.concatenate([d["weight"], d["weight"]]))


def to_dev(d, dev):
    return {k: torch.from_numpy(np.ascontiguousarray(d[k])).to(dev)
            for k in ("uvw", "vis", "weight")}


@pytest.mark.parametrize("kernel,support,fused", [("kb", 7, True), ("gauss", 5, False)])
def test_hermitian_mirror_image(P, kernel, support, fused):
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = small()
    kw = params(wl, kernel=kernel, support=support)
    t = to_dev(d, dev)
    im = P.Imager(**kw, max_vis=len(d["vis"]), device=dev, hermitian_mirror=True, fused=fused)
    img = im.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    st = im.stats()
    imag = im.image_from_binned(P.imager.IMAGE_FLAGS | P.rick.RICK_IMAG_PART).cpu().numpy()
    # the unmirrored image with the same (symmetric) w-planes: the mirrored
    # records of plane k land in plane n_w - 1 - k, whose centre is -w_k
    wm = float(np.abs(d["uvw"][:, 2]).max())
    plain = P.Imager(**kw, max_vis=len(d["vis"]), device=dev, fused=fused, w_range=(-wm, wm))
    pimg = plain.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    op = oracle_params(kw)
    m = mirrored(d)
    ref, ost = oracle.image(op, m["uvw"], m["vis"], m["weight"].astype(np.float64))
    # the records and the range are those of the mirrored set
    assert st["n_binned"] == ost["n_binned"]
    assert (st["w_min"], st["w_max"]) == (ost["w_min"], ost["w_max"])
    assert st["w_min"] == -st["w_max"] == -np.abs(d["uvw"][:, 2]).max()
    assert st["sum_weight"] == pytest.approx(ost["sum_weight"], rel=1e-12)
    e = errs(img, ref, op)
    print(f"mirror {kernel}: image vs oracle of the mirrored set: tapered {e['tapered']:.2e}, "
          f"inner {e['inner']:.2e}")
    assert e["tapered"] <= TOL and e["inner"] <= TOL
    # pin P5 on the GPU: the image of Hermitian data is real, and equal to the
    # real part of the unmirrored image
    cc = cc_of(op)
    peak = np.abs(ref * cc).max()
    assert np.abs(imag * cc).max() <= 2e-6 * peak
    assert np.abs((img - pimg) * cc).max() <= TOL * peak
    im.close()
    plain.close()


def test_imaginary_part_matches_the_oracle(P):
    """RICK_IMAG_PART writes Im of the plane sum times the pixel scale: the
    oracle's plane sum acc gives it as Im(acc) s(p, q)."""
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = small(30000, 3)
    kw = params(wl, kernel="kb", support=7)
    t = to_dev(d, dev)
    im = P.Imager(**kw, max_vis=len(d["vis"]), device=dev)
    im.bin(t["uvw"], t["vis"], t["weight"])
    flags = P.imager.IMAGE_FLAGS | P.rick.RICK_IMAG_PART
    got = im.image_from_binned(flags).cpu().numpy()
    op = oracle_params(kw)
    ref, acc, st = oracle.image(op, d["uvw"], d["vis"], d["weight"].astype(np.float64),
                                want_acc=True)
    n = op.n
    l = (np.arange(n) - n // 2) * op.fov / n
    nn = np.sqrt(1.0 - l[None, :] ** 2 - l[:, None] ** 2)
    tap = oracle.taper_row(op)
    scale = nn / (tap[None, :] * tap[:, None]) / st["sum_weight"]
    want = acc.imag * scale
    e = errs(got, want, op)
    print(f"imaginary part vs oracle: tapered {e['tapered']:.2e}, inner {e['inner']:.2e}")
    assert e["tapered"] <= TOL and e["inner"] <= TOL
    im.close()


def test_hermitian_mirror_adjoint(P):
    """Degridding a mirrored binning: each input's model value is its record's
    plus the conjugate of its mirrored record's (the transpose of gridding
    both)."""
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = small(20000, 5)
    kw = params(wl, kernel="kb", support=7)
    t = to_dev(d, dev)
    im = P.Imager(**kw, max_vis=len(d["vis"]), device=dev, hermitian_mirror=True)
    im.bin(t["uvw"], t["vis"], t["weight"])
    torch.cuda.synchronize()
    st = im.stats()
    op = oracle_params(kw)
    y = (np.random.default_rng(4).normal(size=(op.n, op.n)) * cc_of(op)).astype(np.float32)
    vg = im.adjoint(torch.from_numpy(y).to(dev), t["weight"]).cpu().numpy()
    m = mirrored(d)
    vr = oracle.adjoint(op, m["uvw"], y.astype(np.float64), m["weight"].astype(np.float64),
                        w_min=st["w_min"], w_max=st["w_max"], sum_weight=st["sum_weight"])
    n = len(d["vis"])
    want = vr[:n] + np.conj(vr[n:])
    assert np.abs(vg - want).max() <= TOL * np.abs(want).max()
    im.close()


def test_mirror_refused_where_unsupported(P):
    R = P.rick
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = small(5000)
    t = to_dev(d, dev)
    im = P.Imager(**params(wl), max_vis=5000, device=dev, hermitian_mirror=True)
    im.bin(t["uvw"], t["vis"], t["weight"])
    with pytest.raises(R.RickError) as e:
        im.density_weights("uniform", 0.0, t["weight"])
    assert e.value.status == R.RICK_EINVAL
    h = {k: v.cpu().pin_memory() for k, v in t.items()}
    with pytest.raises(R.RickError) as e:
        im.image_streamed(h["uvw"], h["vis"], h["weight"])
    assert e.value.status == R.RICK_EINVAL
    im.close()


def _det_run(P, kw, t, n, dev, fused):
    im = P.Imager(**kw, max_vis=n, device=dev, deterministic=True, fused=fused)
    img = im.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    b = im.binned()
    planes = im.planes.cpu().numpy() if not fused else None
    im.close()
    return img, b, planes


@pytest.mark.parametrize("case", ["kb7_t16", "kb9_t32", "gauss7_t32_unfused"])
def test_deterministic_is_bitwise_repeatable(P, case):
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    over = {"kb7_t16": dict(kernel="kb", support=7, tile=16),
            "kb9_t32": dict(kernel="kb", support=9, tile=32),
            "gauss7_t32_unfused": dict(kernel="gauss", support=7, tile=32)}[case]
    fused = not case.endswith("unfused")
    d = small(65536)
    kw = params(wl, **over)
    t = to_dev(d, dev)
    n = len(d["vis"])
    img1, b1, pl1 = _det_run(P, kw, t, n, dev, fused)
    img2, b2, pl2 = _det_run(P, kw, t, n, dev, fused)
    assert np.array_equal(img1.view(np.uint32), img2.view(np.uint32))
    for k in ("offsets", "perm", "rec_cell"):
        assert np.array_equal(b1[k], b2[k]), k
    assert np.array_equal(b1["rec_val"].view(np.uint64), b2["rec_val"].view(np.uint64))
    if pl1 is not None:
        assert np.array_equal(pl1.view(np.uint64), pl2.view(np.uint64))
    # P10: the records of each bin in input order: the oracle's stable sort
    op = oracle_params(kw)
    ob = oracle.bin(op, d["uvw"])
    assert np.array_equal(b1["offsets"].astype(np.int64), ob["offsets"])
    assert np.array_equal(b1["perm"].astype(np.int64), ob["perm"])
    ref, _ = oracle.image(op, d["uvw"], d["vis"], d["weight"].astype(np.float64))
    e = errs(img1, ref, op)
    print(f"deterministic {case}: image vs oracle: tapered {e['tapered']:.2e}, "
          f"inner {e['inner']:.2e}")
    assert e["tapered"] <= TOL and e["inner"] <= TOL


def test_deterministic_multi_item_tiles_and_accumulate(P):
    """Tiles dense enough to take several work items (their fixed-point sums go
    through the workspace slots), and gridding that adds into planes
    (rick_grid_accumulate): repeatable and equal to the oracle's planes."""
    R = P.rick
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = small(65536, 9)
    # a narrow field: the tracks pile up on a few tiles of a 64^2 grid
    kw = params(wl, n=64, n_w=2, fov=0.2 * math.pi / 180, kernel="kb", support=7, tile=16)
    t = to_dev(d, dev)
    n = len(d["vis"])
    outs = []
    for _ in range(2):
        im = P.Imager(**kw, max_vis=n, device=dev, deterministic=True, fused=False)
        im.bin(t["uvw"], t["vis"], t["weight"])
        im.grid()
        R.rick_grid_accumulate(im.plan, im.ws.data_ptr(), im.planes.data_ptr(),
                               torch.cuda.current_stream().cuda_stream)
        outs.append(im.planes.cpu().numpy())
        im.close()
    assert np.array_equal(outs[0].view(np.uint64), outs[1].view(np.uint64))
    op = oracle_params(kw)
    og, _ = oracle.grid(op, d["uvw"], d["vis"], d["weight"].astype(np.float64))
    i = np.arange(op.n)
    cb = np.where((i[:, None] + i[None, :]) % 2, -1.0, 1.0)
    want = 2 * og * cb[None]
    assert np.abs(outs[0] - want).max() <= TOL * np.abs(want).max()


def test_probe_throughput(P):
    """The per-SM rates the bench's rooflines divide by: positive, and within
    what one SM can issue (4 sub-partitions x 32 lanes per clock)."""
    R = P.rick
    rates = {k: R.rick_probe_throughput(getattr(R, k)) for k in
             ("RICK_PROBE_SMEM_RMW", "RICK_PROBE_SMEM_ATOMIC_F32", "RICK_PROBE_SMEM_ATOMIC_U32",
              "RICK_PROBE_SMEM_ATOMIC_U64", "RICK_PROBE_FFMA", "RICK_PROBE_FFMA2",
              "RICK_PROBE_SHFL", "RICK_PROBE_F2I")}
    print("probe (operations per SM clock):", {k: round(v, 2) for k, v in rates.items()})
    for k, v in rates.items():
        assert 0.5 < v <= 4 * 32 * (2 if k.endswith("FFMA2") else 1) * 1.05, (k, v)
    with pytest.raises(R.RickError):
        R.rick_probe_throughput(99)


def test_set_planes_retargets_a_plan(P):
    """A plan made for 16 planes and re-targeted to 8 (rick_plan_set_planes)
    images like a plan made for 8; its cuFFT stage, batched for 16, refuses."""
    R = P.rick
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = small(30000, 11)
    t = to_dev(d, dev)
    kw = params(wl, n_w=8, kernel="kb", support=7)
    fresh = P.Imager(**kw, max_vis=30000, device=dev)
    ref = fresh.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    big = P.Imager(**dict(kw, n_w=16), max_vis=65536, device=dev)
    big.image(t["uvw"], t["vis"], t["weight"])
    torch.cuda.synchronize()
    big.set_planes(8)
    got = big.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    op = oracle_params(kw)
    cc = cc_of(op)
    assert np.abs((got - ref) * cc).max() <= 1e-6 * np.abs(ref * cc).max()
    with pytest.raises(R.RickError):
        big.fft(+1)
    with pytest.raises(R.RickError):
        big.set_planes(17)
    fresh.close()
    big.close()
