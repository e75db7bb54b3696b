"""The binning's bounded device-side wait, made to run out.

The key pass waits on an mbarrier for the bulk (TMA) copies of its inputs into
shared memory, at most a set number of polls.  With the limit set to zero polls
(rick_plan_set_wait_limit) the wait gives up at once: each block lets its
copies finish, leaves its inputs out and returns, and the binning reports
n_binned = -1.  Nothing faults, the plan keeps no
error, and the next binning with the default limit is complete and correct.
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


def test_bounded_wait_gives_up_and_the_plan_recovers(P):
    R = P.rick
    dev = torch.device("cuda:0")
    wl = synth.WORKLOADS["small"]
    d = synth.generate(wl.obs)
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                  max_vis=len(d["vis"]), device=dev)
    R.rick_plan_set_wait_limit(im.plan, 0)
    im.bin(t["uvw"], t["vis"], t["weight"])
    torch.cuda.synchronize()
    assert im.stats()["n_binned"] == -1
    assert R.rick_plan_last_error(im.plan) == R.RICK_OK
    R.rick_plan_set_wait_limit(im.plan, R.RICK_WAIT_POLLS_DEFAULT)
    img = im.image(t["uvw"], t["vis"], t["weight"]).cpu().numpy()
    op = oracle.Params(n=wl.n, n_w=wl.n_w, fov=wl.fov, kernel=oracle.GAUSS, support=wl.support,
                       tile=wl.tile)
    ref, ost = oracle.image(op, d["uvw"], d["vis"], d["weight"].astype(np.float64))
    assert im.stats()["n_binned"] == ost["n_binned"]
    c = oracle.taper_row(op)
    c = c / c[op.n // 2]
    cc = c[:, None] * c[None, :]
    assert np.abs((img - ref) * cc).max() <= 1e-5 * np.abs(ref * cc).max()
    im.close()
