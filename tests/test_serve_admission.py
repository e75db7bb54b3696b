"""Host-side admission logic of the imaging server (no GPU needed).

Admission keeps the sum of resident slot footprints within the HBM budget,
reuses an idle slot of the same key, evicts idle slots least recently used
first, never evicts a busy slot, and rejects a request larger than the whole
budget -- a failure that touches no other request.
"""
import importlib
import os

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def load_serve():
    return importlib.import_module("paper_2411_07321_gb300.serve")


@pytest.fixture(scope="module")
def S():
    pytest.importorskip("torch")
    from paper_2411_07321_gb300 import build
    build.build()  # serve.py loads the binding (no GPU work is done here)
    return load_serve()


def test_capacity_classes(S):
    m = S.MIN_CAPACITY
    assert S.capacity_class(1) == m
    assert S.capacity_class(m) == m
    assert S.capacity_class(m + 1) == 2 * m
    assert S.capacity_class(10_000_000) == 1 << 24
    assert S.plane_class(4) == S.plane_class(S.MIN_PLANES) == S.MIN_PLANES
    assert S.plane_class(40) == 40


def test_tuple_capacities_compare_element_by_element(S):
    a = S.Admission(1000)
    k = ("A",)
    i = a.add(k, 300, now=0.0, cap=(1 << 20, 16))
    a.release(i, now=1.0)
    assert a.plan(k, 300, (1 << 20, 8)) == ("reuse", i)
    assert a.plan(k, 300, (1 << 19, 16)) == ("reuse", i)
    assert a.plan(k, 300, (1 << 21, 8)) == ("new", [])  # too few visibilities
    assert a.plan(k, 300, (1 << 20, 17)) == ("new", [])  # too few planes


def test_reuse_idle_slot_of_same_key(S):
    a = S.Admission(1000)
    k = ("A",)
    assert a.plan(k, 300) == ("new", [])
    i = a.add(k, 300, now=0.0)
    a.release(i, now=1.0)
    assert a.plan(k, 300) == ("reuse", i)
    a.acquire(i, now=2.0)
    # the only slot of that key is busy: a new one is planned
    assert a.plan(k, 300) == ("new", [])


def test_lru_eviction_and_busy_slots_never_evicted(S):
    a = S.Admission(1000)
    s1 = a.add(("A",), 400, now=0.0)
    s2 = a.add(("B",), 400, now=1.0)
    a.release(s1, now=5.0)   # s1 idle, used later than s2
    a.release(s2, now=3.0)   # s2 idle, least recently used
    # needs 500: 200 free, evict s2 (LRU) first -> 600 free
    assert a.plan(("C",), 500) == ("new", [s2])
    # with s1 busy, only s2 can go
    a.acquire(s1, now=6.0)
    assert a.plan(("C",), 500) == ("new", [s2])
    # needs 700: even evicting s2 leaves 600 free -> wait
    assert a.plan(("C",), 700) is None


def test_budget_never_exceeded(S):
    a = S.Admission(1000)
    import random
    rnd = random.Random(0)
    live = []
    for step in range(500):
        key = (rnd.randrange(4),)
        need = rnd.randrange(50, 400)
        d = a.plan(key, need)
        if d is None:
            if live:
                a.release(live.pop(rnd.randrange(len(live))), now=step)
            continue
        if d[0] == "reuse":
            a.acquire(d[1], now=step)
            live.append(d[1])
        else:
            for i in d[1]:
                assert not a.slots[i]["busy"]
                a.remove(i)
            live.append(a.add(key, need, now=step))
        assert a.used() <= a.budget
        if len(live) > 3:
            a.release(live.pop(0), now=step)


def test_request_larger_than_budget_is_rejected(S):
    a = S.Admission(1000)
    with pytest.raises(S.AdmissionError):
        a.plan(("A",), 1001)
    assert a.plan(("A",), 1000) == ("new", [])


def test_poisson_arrivals(S):
    t = S.poisson_arrivals(20000, rate=50.0, seed=3)
    import numpy as np
    assert np.all(np.diff(t) > 0)
    assert abs(np.mean(np.diff(t)) - 1 / 50.0) < 0.05 / 50.0


def test_slot_cap_evicts_idle_lru_first(S):
    a = S.Admission(10_000, max_slots=2)
    s1 = a.add(("A",), 100, now=0.0)
    s2 = a.add(("B",), 100, now=1.0)
    # both busy: a third key must wait even though the budget has room
    assert a.plan(("C",), 100) is None
    a.release(s2, now=2.0)
    a.release(s1, now=3.0)
    assert a.plan(("C",), 100) == ("new", [s2])  # s2 is least recently used
    assert a.plan(("A",), 100) == ("reuse", s1)


def test_reuse_prefers_the_smallest_idle_slot_with_enough_capacity(S):
    a = S.Admission(10_000)
    k = ("A",)
    small = a.add(k, 100, now=0.0, cap=1 << 14)
    big = a.add(k, 400, now=1.0, cap=1 << 20)
    mid = a.add(k, 200, now=2.0, cap=1 << 16)
    for i in (small, big, mid):
        a.release(i, now=3.0)
    assert a.plan(k, 100, cap=1 << 15) == ("reuse", mid)   # 2^16 is the smallest that holds it
    assert a.plan(k, 100, cap=1 << 14) == ("reuse", small)
    assert a.plan(k, 100, cap=1 << 21) == ("new", [])       # none is large enough
    a.acquire(mid, now=4.0)
    assert a.plan(k, 100, cap=1 << 15) == ("reuse", big)   # the next larger one


def test_job_key_leaves_out_kernel_planes_and_capacity(S):
    import numpy as np
    uvw = np.zeros((10, 3))
    a = S.ImagingJob(uvw, None, None, n=512, n_w=8, fov=0.01, kernel="kb", support=7)
    b = S.ImagingJob(np.zeros((100_000, 3)), None, None, n=512, n_w=12, fov=0.02,
                     kernel="gauss", support=5)
    assert a.key() == b.key()
    assert S.capacities(a) == (S.MIN_CAPACITY, S.MIN_PLANES)
    c = S.ImagingJob(uvw, None, None, n=1024, n_w=8, fov=0.01)
    assert a.key() != c.key()
    d = S.ImagingJob(uvw, None, None, n=512, n_w=8, fov=0.01, image_n=300)
    assert d.key() == a.key() and (d.side, a.side) == (300, 512)


class _FakeImager:
    def __init__(self, fused=True, options=0):
        self.fused = fused
        self.params = type("P", (), {"options": options})()


class _FakeSlot:
    def __init__(self, job, fused=True, options=0):
        self.job = job
        self.imager = _FakeImager(fused, options)
        self.future = None
        self.event = None


def _job(S, n_vis, support=7, tile=64, precision="fp32", job_id=0):
    import numpy as np
    uvw = np.zeros((n_vis, 3))
    return S.ImagingJob(uvw, None, None, n=512, n_w=4, fov=0.01, support=support, tile=tile,
                        precision=precision, job_id=job_id)


def _server(S, merge_small):
    """A Server whose launch steps are recorded instead of run (no device)."""
    srv = S.Server.__new__(S.Server)
    srv.merge_small = merge_small
    srv.launched = []
    srv.failed = []
    srv._launch = lambda slot, job: srv.launched.append(("alone", job.job_id))
    srv._launch_batch = lambda slots: srv.launched.append(
        ("merged", tuple(sl.job.job_id for sl in slots)))
    srv._fail = lambda sid, slot, err: srv.failed.append(slot.job.job_id)
    return srv


def test_merged_groups_by_support_and_tile(S):
    """Small FP32 requests on fused grids are grouped by (support, tile) and
    split at RICK_GRID_BATCH_MAX; a group of one, a large request, a
    compensated one, one on a grid outside the fused sizes and a
    deterministic plan are launched alone."""
    B = S.R.RICK_GRID_BATCH_MAX
    jobs = [_job(S, 1000, job_id=i) for i in range(B + 2)]           # one group, split
    jobs += [_job(S, 1000, support=9, job_id=100),                     # a group of one
             _job(S, 1000, tile=32, job_id=101), _job(S, 2000, tile=32, job_id=102),
             _job(S, S.BATCH_MAX_VIS + 1, job_id=103),                 # too large
             _job(S, 1000, precision="compensated", job_id=104)]
    slots = [_FakeSlot(j) for j in jobs]
    slots.append(_FakeSlot(_job(S, 1000, job_id=105), fused=False))   # no fused transform
    slots.append(_FakeSlot(_job(S, 1000, job_id=106), options=S.R.RICK_OPT_DETERMINISTIC))
    started = [(i, sl, sl.job, None) for i, sl in enumerate(slots)]
    srv = _server(S, merge_small=True)
    srv._launch_group(started)
    merged = [ids for kind, ids in srv.launched if kind == "merged"]
    alone = sorted(ids for kind, ids in srv.launched if kind == "alone")
    assert merged == [tuple(range(B)), (B, B + 1), (101, 102)]
    assert alone == [100, 103, 104, 105, 106]
    # off: every request on its own launches
    srv = _server(S, merge_small=False)
    srv._launch_group(started)
    assert sorted(ids for _, ids in srv.launched) == sorted(sl.job.job_id for sl in slots)
    assert all(kind == "alone" for kind, _ in srv.launched)


def test_a_failed_launch_fails_only_its_part(S):
    """An exception from one launch (or one merged group) fails exactly the
    requests of that launch; the others are still launched."""
    jobs = [_job(S, 1000, job_id=i) for i in range(3)] + [_job(S, 1000, tile=32, job_id=10),
                                                          _job(S, 1000, support=9, job_id=20)]
    started = [(i, _FakeSlot(j), j, None) for i, j in enumerate(jobs)]
    srv = _server(S, merge_small=True)

    def bad_batch(slots):
        raise RuntimeError("merged launch failed")
    srv._launch_batch = bad_batch
    srv._launch_group(started)
    assert sorted(srv.failed) == [0, 1, 2]          # the merged group of tile 64
    assert sorted(ids for _, ids in srv.launched) == [10, 20]
