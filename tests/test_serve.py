"""The continuous-batching server on the GPU.

Every request's image is the same served alone and served in a mix of
concurrent requests of different sizes (within the parity tolerance: 1e-5 of
peak on the tapered image, as in test_gpu_parity); the HBM budget is never
exceeded even when it forces requests to wait and slots to be evicted; an
invalid request or one larger than the budget fails alone while the others
complete.
"""
import numpy as np
import pytest

import oracle
import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2411_07321_gb300 import serve
    return serve


@pytest.fixture(scope="module")
def data():
    d = synth.generate(synth.scaled("lofar", n_keep=600_000).obs)
    return {k: torch.from_numpy(d[k]).pin_memory() for k in ("uvw", "vis", "weight")}


def make_jobs(S, data, specs):
    jobs = []
    for jid, (n_vis, n, n_w, kernel) in enumerate(specs):
        fov = S.fov_for(n, 7, 12000.0)
        jobs.append(S.ImagingJob(data["uvw"][:n_vis], data["vis"][:n_vis], data["weight"][:n_vis],
                                 n=n, n_w=n_w, fov=fov, kernel=kernel, support=7,
                                 tile=32 if n <= 512 else 64, job_id=jid))
    return jobs


def tapered_error(img, ref, n, kernel):
    op = oracle.Params(n=n, n_w=1, fov=0.01, kernel=oracle.KB if kernel == "kb" else oracle.GAUSS,
                       support=7)
    c = np.array([oracle.taper(op, (i - n // 2) / n) for i in range(n)])
    cc = np.outer(c, c)
    return np.abs((img - ref) * cc).max() / np.abs(ref * cc).max()


SPECS = [(20_000, 256, 4, "kb"), (600_000, 1024, 8, "kb"), (150_000, 512, 16, "gauss"),
         (333_333, 1024, 8, "kb"), (50_000, 512, 6, "kb"), (600_000, 512, 4, "gauss")]


def test_alone_equals_in_mix(S, data):
    jobs = make_jobs(S, data, SPECS)
    alone = []
    for j in jobs:
        with S.Server("cuda:0") as srv:
            alone.append(srv.submit(j).result(timeout=120).image)
    with S.Server("cuda:0", max_running=4) as srv:
        futs = [srv.submit(j) for j in jobs]
        mix = [f.result(timeout=120) for f in futs]
    for j, a, m in zip(jobs, alone, mix):
        assert m.job_id == j.job_id
        assert tapered_error(m.image, a, j.n, j.kernel) <= 1e-5, j.job_id
    # the plain per-request path gives the same images
    for j, a in zip(jobs[:3], alone):
        assert tapered_error(S.run_plain(j), a, j.n, j.kernel) <= 1e-5


def test_budget_is_respected_and_forces_waiting(S, data):
    jobs = make_jobs(S, data, SPECS * 2)
    biggest = max(S.slot_footprint(j) for j in jobs)
    budget = int(2.2 * biggest)  # room for about two slots: the rest must wait or evict
    with S.Server("cuda:0", budget_bytes=budget, max_running=8) as srv:
        futs = [srv.submit(j) for j in jobs]
        res = [f.result(timeout=300) for f in futs]
        assert srv.peak_used <= budget
        assert srv.admission.used() <= budget
    assert sorted(r.job_id for r in res) == [j.job_id for j in jobs]


def test_failures_stay_with_their_request(S, data):
    import paper_2411_07321_gb300 as P
    good = make_jobs(S, data, SPECS[:3])
    bad = S.ImagingJob(data["uvw"][:1000], data["vis"][:1000], None, n=100, n_w=4, fov=0.01,
                       job_id=99)  # n must be a power of two
    with S.Server("cuda:0", budget_bytes=int(1.5 * max(S.slot_footprint(j) for j in good))) as srv:
        huge = make_jobs(S, data, [(600_000, 8192, 32, "kb")])[0]
        futs = [srv.submit(good[0]), srv.submit(bad), srv.submit(huge), srv.submit(good[1]),
                srv.submit(good[2])]
        with pytest.raises(P.rick.RickError):
            futs[1].result(timeout=60)
        with pytest.raises(S.AdmissionError):
            futs[2].result(timeout=60)
        for f in (futs[0], futs[3], futs[4]):
            assert f.result(timeout=120).image.shape[0] in (256, 512, 1024)
        # a request that fails at launch (fewer visibilities than uvw rows): it
        # fails alone, and its slot serves the next request
        short = S.ImagingJob(data["uvw"][:1000], data["vis"][:999], data["weight"][:1000],
                             n=256, n_w=4, fov=good[0].fov, job_id=98, tile=32)
        f_short = srv.submit(short)
        with pytest.raises(RuntimeError):
            f_short.result(timeout=60)
        assert srv.submit(good[0]).result(timeout=120).image.shape[0] == 256


def test_crops_share_a_slot(S, data):
    """Requests for different crops of one grid (image_n) run on one re-targeted
    slot, each giving its plain per-request image."""
    n = 512
    fov = S.fov_for(n, 7, 12000.0)
    jobs = [S.ImagingJob(data["uvw"][:200_000], data["vis"][:200_000], data["weight"][:200_000],
                         n=n, n_w=8, fov=fov, kernel="kb", support=7, tile=32, job_id=i,
                         image_n=m) for i, m in enumerate((None, 256, 384, 256, None))]
    with S.Server("cuda:0", max_running=1) as srv:
        res = [srv.submit(j).result(timeout=120) for j in jobs]
        assert srv.counters["new_slots"] == 1 and srv.counters["reused"] == len(jobs) - 1
    op = oracle.Params(n=n, n_w=1, fov=0.01, kernel=oracle.KB, support=7)
    c = np.array([oracle.taper(op, (i - n // 2) / n) for i in range(n)])
    for j, r in zip(jobs, res):
        assert r.image.shape == (j.side, j.side)
        ref = S.run_plain(j)
        o = (n - j.side) // 2
        cc = np.outer(c[o:o + j.side], c[o:o + j.side])
        assert np.abs((r.image - ref) * cc).max() <= 1e-5 * np.abs(ref * cc).max()


def test_small_requests_share_a_gridding_launch(S, data):
    """With merge_small, small requests admitted together are gridded by one
    merged launch (rick_grid_sparse_batch on the server's batch stream) and
    still give their plain per-request images."""
    specs = [(20_000, 256, 4, "kb"), (150_000, 512, 16, "gauss"), (50_000, 512, 6, "kb"),
             (333_333, 1024, 8, "kb"), (600_000, 1024, 5, "gauss"), (80_000, 256, 9, "gauss")]
    jobs = make_jobs(S, data, specs)
    for j in jobs:
        j.tile = 32  # one group: same support and tile
    with S.Server("cuda:0", max_running=8, merge_small=True) as srv:
        futs = [srv.submit(j) for j in jobs]
        res = [f.result(timeout=120) for f in futs]
        assert srv.counters["batches"] >= 1 and srv.counters["batched"] >= 2
    for j, r in zip(jobs, res):
        assert r.job_id == j.job_id
        assert tapered_error(r.image, S.run_plain(j), j.n, j.kernel) <= 1e-5, j.job_id
