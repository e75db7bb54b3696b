"""CPU checks of the C ABI library: it loads, exports every declared entry
point, and validates arguments on the host (no GPU work is enqueued here)."""
import math
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def R():
    from paper_2411_07321_gb300 import build

    build.build()
    from paper_2411_07321_gb300 import rick

    return rick


def declared_functions():
    src = open(os.path.join(ROOT, "include", "rick.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(rick_[a-z0-9_]+)\s*\(", src)))


def test_every_declared_symbol_is_exported(R):
    names = declared_functions()
    assert "rick_bin" in names and "rick_degrid" in names and len(names) >= 13
    for name in names:
        assert hasattr(R._L, name), name
    assert sorted(R.EXPORTS) == names


def test_status_strings(R):
    for s in (R.RICK_OK, R.RICK_EINVAL, R.RICK_ENOMEM, R.RICK_ECUDA, R.RICK_ECUFFT, R.RICK_ERANGE):
        assert R.status_string(s) and R.status_string(s) != "unknown status"


def test_struct_layout_matches_header(R, tmp_path):
    """The binding's structs have the C compiler's size and field offsets."""
    import ctypes
    import subprocess
    assert ctypes.sizeof(R.rick_params) == 72
    assert ctypes.sizeof(R.rick_bin_stats) == 48
    structs = {"rick_params": R.rick_params, "rick_bin_stats": R.rick_bin_stats,
               "rick_bin_view": R.rick_bin_view}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "rick.h"', "int main(void) {"]
    for name, cls in structs.items():
        lines.append(f'printf("{name} size %zu\\n", sizeof({name}));')
        for field, _ in cls._fields_:
            lines.append(f'printf("{name} {field} %zu\\n", offsetof({name}, {field}));')
    lines += ["return 0; }"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), "-o", str(exe),
                    str(src)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True,
                               text=True).stdout.splitlines():
        name, field, v = line.split()
        got[(name, field)] = int(v)
    for name, cls in structs.items():
        assert got[(name, "size")] == ctypes.sizeof(cls), name
        for field, _ in cls._fields_:
            assert got[(name, field)] == getattr(cls, field).offset, (name, field)


@pytest.mark.parametrize("bad", [
    dict(n=100), dict(n=8), dict(n_w=0), dict(fov=0.0), dict(fov=2.0), dict(support=0),
    dict(support=17), dict(tile=4), dict(tile=48), dict(tile=256), dict(kernel=7),
    dict(w_min=1.0), dict(w_min=2.0, w_max=1.0), dict(precision=3), dict(kb_beta=-1.0),
    dict(gauss_sigma=0.0, kernel=0), dict(image_n=14), dict(image_n=101), dict(image_n=512),
    dict(image_n=-2), dict(fov=2.0, image_n=192),
])
def test_invalid_params_rejected_on_host(R, bad):
    kw = dict(n=256, n_w=8, fov=0.035, kernel=1, support=7, w_min=math.nan, w_max=math.nan,
              kb_beta=math.nan, gauss_sigma=math.nan, tile=32, precision=0)
    kw.update(bad)
    p = R.make_params(**kw)
    with pytest.raises(R.RickError) as e:
        R.rick_workspace_bytes(p, 1000)
    assert e.value.status == R.RICK_EINVAL


def test_crop_params(R):
    """A crop relaxes the unit-circle bound to the kept field; unknown option bits
    are refused."""
    kw = dict(n=256, n_w=8, fov=2.0, kernel=1, support=7, tile=32)
    R.rick_workspace_bytes(R.make_params(**kw, image_n=128), 1000)  # 2 * 0.5 / sqrt 2 < 1
    p = R.make_params(**dict(kw, fov=0.03))
    p.options = 4
    with pytest.raises(R.RickError):
        R.rick_workspace_bytes(p, 1000)


def test_kb_beta_for_oversampling(R):
    import oracle
    for W in (2, 4, 7, 9, 16):
        for alpha in (1.25, 1.5, 2.0, 3.0):
            want = oracle.kb_beta(W, alpha)
            if math.isnan(want):
                assert math.isnan(R.rick_kb_beta(W, alpha))
            else:
                assert R.rick_kb_beta(W, alpha) == pytest.approx(want, rel=1e-15)
    assert math.isnan(R.rick_kb_beta(1, 2.0))
    assert math.isnan(R.rick_kb_beta(7, 0.9))

    p = R.make_params(4096, 16, 0.1396, 1, 7, tile=64)
    b1, planes = R.rick_workspace_bytes(p, 1_000_000)
    b2, _ = R.rick_workspace_bytes(p, 2_000_000)
    assert planes == 16 * 4096 * 4096 * 8
    assert 30_000_000 < b2 - b1 < 50_000_000  # tens of bytes per visibility
    with pytest.raises(R.RickError):
        R.rick_workspace_bytes(p, -1)


def test_null_plan_rejected(R):
    import ctypes
    assert R._L.rick_grid(None, None, None, None) == R.RICK_EINVAL
    assert R._L.rick_plan_destroy(None) == R.RICK_OK
    assert R._L.rick_plan_last_error(None) == R.RICK_EINVAL
    v = R.rick_bin_view()
    assert R._L.rick_bin_layout(None, ctypes.byref(v)) == R.RICK_EINVAL


def test_grid_batch_rejected_on_host(R):
    """rick_grid_sparse_batch validates its job list before any launch."""
    import ctypes
    arr = ctypes.c_void_p * 2
    none = arr(None, None)
    assert R._L.rick_grid_sparse_batch(None, None, None, 1, None) == R.RICK_EINVAL
    assert R._L.rick_grid_sparse_batch(none, none, none, 0, None) == R.RICK_ERANGE
    assert R._L.rick_grid_sparse_batch(none, none, none, R.RICK_GRID_BATCH_MAX + 1,
                                       None) == R.RICK_ERANGE
    assert R._L.rick_grid_sparse_batch(none, none, none, 2, None) == R.RICK_EINVAL
    with pytest.raises(ValueError):
        R.rick_grid_sparse_batch([None], [None, None], [None], None)
    src = open(os.path.join(ROOT, "include", "rick.h")).read()
    assert re.search(r"#define RICK_GRID_BATCH_MAX (\d+)", src).group(1) == str(
        R.RICK_GRID_BATCH_MAX)


def test_stream_bytes(R):
    """Staging area of the streamed path: a ring of RICK_STREAM_BUFS chunk
    buffers of vis and weight, the fused transform's work buffer (tile, tile-row
    and plane flags, 128-bit tile-row and tile masks, and the transposed row
    transforms, 8 n_w n^2 bytes), plus a ring of chunk buffers of uvw (given w
    range) or two areas holding the whole set's uvw, resident while its w range
    is found and used by alternate calls (range from the data)."""
    al = lambda x: (x + 255) // 256 * 256
    B = R.RICK_STREAM_BUFS
    src = open(os.path.join(ROOT, "include", "rick.h")).read()
    assert re.search(r"#define RICK_STREAM_BUFS (\d+)", src).group(1) == str(B)
    chunk, n = 100_000, 1_234_567
    given = R.make_params(256, 8, 0.035, 1, 7, w_min=-10.0, w_max=10.0, tile=32)
    data = R.make_params(256, 8, 0.035, 1, 7, tile=32)
    nt = 256 // 32
    fwork = al(8 * nt * nt) + al(8 * nt) + al(8) + al(16 * 8) + al(16 * 8 * nt) + 8 * 8 * 256 * 256
    head = R.rick_stream_bytes(given, chunk, n) - B * (al(24 * chunk) + al(8 * chunk) +
                                                       al(4 * chunk)) - fwork
    assert 0 < head <= 4096 + 2 * 8 * 4096  # headers and two areas of channel factors
    assert R.rick_stream_bytes(data, chunk, n) == head + fwork + 2 * al(24 * n) + B * (
        al(8 * chunk) + al(4 * chunk))
    # grids the fused transform does not cover (n > 8192) stage no work buffer
    big = R.make_params(16384, 8, 0.035, 1, 7, w_min=-10.0, w_max=10.0, tile=64)
    assert R.rick_stream_bytes(big, chunk, n) - B * (al(24 * chunk) + al(8 * chunk) +
                                                     al(4 * chunk)) == head
    # a given range keeps nothing of the set resident: independent of n
    assert R.rick_stream_bytes(given, chunk, 10 * n) == R.rick_stream_bytes(given, chunk, n)
    with pytest.raises(R.RickError):
        R.rick_stream_bytes(given, -1, n)


def test_fused_work_bytes(R):
    """The fused transform's work buffer without a plan: flags and 128-bit masks, then
    the transposed row transforms (8 n_w image_n n bytes); the same bytes the
    streamed call stages; none where the fused transform does not cover n."""
    al = lambda x: (x + 255) // 256 * 256
    for n, n_w, tile, image_n in ((256, 8, 32, 0), (4096, 16, 64, 0), (8192, 3, 8, 4096),
                                  (8192, 2, 64, 4094)):
        p = R.make_params(n, n_w, 0.03, 1, 7, tile=tile, image_n=image_n)
        nt, m = n // tile, image_n or n
        want = al(n_w * nt * nt) + al(n_w * nt) + al(n_w) + al(16 * n_w) + al(16 * n_w * nt) + \
            8 * n_w * m * n
        assert R.rick_fused_work_bytes(p) == want
    assert R.rick_fused_work_bytes(R.make_params(128, 4, 0.03, 1, 7, tile=32)) == 0
    assert R.rick_fused_work_bytes(R.make_params(16384, 4, 0.03, 1, 7, tile=64)) == 0
    with pytest.raises(R.RickError) as e:
        R.rick_fused_work_bytes(R.make_params(100, 4, 0.03, 1, 7, tile=32))
    assert e.value.status == R.RICK_EINVAL
