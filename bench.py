#!/usr/bin/env python
"""Throughput of the end-to-end w-stacked image on one GB300 (or N replicas).

One step = one pass of the whole hot path over one batch of visibilities:
bin -> grid -> per-plane inverse FFT -> w-correct + stack + taper (the stages of
§2 of De Rubeis et al.), by default on the large workload: 2e8 synthetic
LOFAR-like visibilities (60 stations, 64 channels), 8192^2 grid, 32 w-planes,
Kaiser-Bessel support 9.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Prints one JSON line.  ``value`` is visibilities/s with the inputs already
resident in HBM; ``e2e`` is the same metric through the streamed host-buffer
API call (pinned host inputs streamed to the GPU in chunks, copies overlapping
binning and gridding, and the image copied back to pinned host memory, all
inside the timed region).  The inputs (7.2 GB) are larger than L2, so no L2
flush is needed between steps.  Extra keys: the LOFAR-like workload's step
(5e7 visibilities, 4096^2 x 16 planes, KB W=7), a reduced serving trace
(served vs plain), the chi^2 gradient step, and the FP64 oracle on the host
cores.  ``--impl reference`` times the FP64 oracle alone, on per-plane slabs
of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "visibilities/s end-to-end w-stacked image vs roofline; served p50/p99 vs plain"
UNIT = "vis/s"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons around the timed region."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def start(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20", "-i", str(self.index)], stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None

    def stop(self, t0: float, t1: float) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        self.proc.wait()
        self.f.seek(0)
        rows = [r.split(", ") for r in self.f.read().strip().splitlines() if r.count(",") >= 9]
        os.unlink(self.f.name)
        from datetime import datetime

        def ts(s):
            try:
                return datetime.strptime(s.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except ValueError:
                return None

        inside = [r for r in rows if (ts(r[0]) or 0) >= t0 - 0.02 and (ts(r[0]) or 0) <= t1 + 0.02]
        use = inside or rows
        sm = [float(r[2]) for r in use if r[2].strip().replace(".", "").isdigit()]
        mx = [float(r[3]) for r in use if r[3].strip().replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[j] for r in use for j in range(4)
                          if r[6 + j].strip().lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(use), "samples_in_window": len(inside)}


def algorithmic_bytes(n_vis: int, n_binned: int, n: int, n_w: int, tile: int,
                      tiles: int, tile_rows: int) -> dict:
    """Bytes each stage must move at least.  tiles / tile_rows: the (plane,
    uv-tile) and (plane, tile-row) pairs that records reach -- the only parts
    of the planes the sparse grid and the fused transform touch."""
    planes = n_w * n * n * 8
    cells = tiles * tile * tile * 8
    return {
        # read uvw f64x3, vis c64, weight f32; write records (value c64, offsets 2xf32,
        # cell u32) and the permutation u32
        "bin": n_vis * (24 + 8 + 4) + n_binned * (8 + 8 + 4 + 4),
        # read each record once, write the cells of the tiles records reach
        "grid": n_binned * (8 + 8 + 4) + cells,
        # read those cells, write and read back the transposed row transforms of
        # the tile-rows they lie in, write the image
        "fft_wcorrect": cells + 2 * tile_rows * tile * n * 8 + n * n * 4,
        # the unfused stages, for comparison: the cuFFT transform (one read and
        # one write of the planes at least) and the plane sum (read every plane,
        # write the image); their grid step writes every plane cell
        "cufft": 2 * planes,
        "wcorrect": planes + n * n * 4,
        "grid_clear": n_binned * (8 + 8 + 4) + planes,
    }


def probe_rates(P) -> dict:
    """Per-SM throughput of the units that bound the tile kernels, measured on
    this GPU by the library's probe (operations per SM clock)."""
    R = P.rick
    kinds = {"smem_rmw_f32": R.RICK_PROBE_SMEM_RMW, "smem_atomic_f32": R.RICK_PROBE_SMEM_ATOMIC_F32,
             "smem_atomic_u32": R.RICK_PROBE_SMEM_ATOMIC_U32,
             "smem_atomic_u64": R.RICK_PROBE_SMEM_ATOMIC_U64, "ffma": R.RICK_PROBE_FFMA,
             "ffma2": R.RICK_PROBE_FFMA2, "shfl": R.RICK_PROBE_SHFL, "f2i": R.RICK_PROBE_F2I}
    return {k: R.rick_probe_throughput(v) for k, v in kinds.items()}


def stage_rooflines(wl, m: dict, rates: dict, sms: int, sm_mhz: float, hbm_peak: float) -> dict:
    """Each stage against the unit that bounds it:
    - bin: HBM (algorithmic bytes / measured copy bandwidth);
    - grid: shared memory -- Eq. 3 accumulates 2 W^2 FP32 values per visibility;
      the peak is the measured plain read-modify-write rate of shared memory
      (the faster of the two ways to add into it); HBM bytes alongside;
    - fft_wcorrect: FP32 arithmetic -- 5 N log2 N flops per N-point complex
      transform (the usual count), one per row of the tile-rows with records
      plus one per image column and plane with records, against the measured
      FP32 FMA rate (2 flops per FMA)."""
    clk = sm_mhz * 1e6
    out = {}
    ms = m["stage_ms"]
    alg = m["alg"]
    hb = {k: alg[k] / (ms[k] * 1e-3) / 1e9 for k in ms}
    out["bin"] = {"bound": "hbm", "achieved": hb["bin"], "peak": hbm_peak, "unit": "GB/s",
                  "frac": hb["bin"] / hbm_peak, "work": alg["bin"]}
    smem_ops = 2 * wl.support ** 2 * m["n_binned"]
    smem_peak = rates["smem_rmw_f32"] * sms * clk
    g = smem_ops / (ms["grid"] * 1e-3)
    out["grid"] = {"bound": "smem", "achieved": g / 1e9, "peak": smem_peak / 1e9,
                   "unit": "G FP32 shared read-modify-writes/s", "frac": g / smem_peak,
                   "work": smem_ops, "hbm_frac": hb["grid"] / hbm_peak,
                   "peak_note": f"{rates['smem_rmw_f32']:.2f} RMW/clk/SM measured x {sms} SMs x "
                                f"{sm_mhz:.0f} MHz"}
    n = wl.n
    m_img = n
    transforms = m["tile_rows"] * wl.tile + m_img * m["planes_read"]
    flops = 5.0 * n * math.log2(n) * transforms
    fma = max(rates["ffma"], rates["ffma2"])  # the faster of single and paired FMAs
    fpeak = 2.0 * fma * sms * clk
    f = flops / (ms["fft_wcorrect"] * 1e-3)
    out["fft_wcorrect"] = {"bound": "alu", "achieved": f / 1e12, "peak": fpeak / 1e12,
                           "unit": "TFLOP/s (FP32)", "frac": f / fpeak, "work": flops,
                           "hbm_frac": hb["fft_wcorrect"] / hbm_peak,
                           "peak_note": f"{fma:.1f} FP32 FMA/clk/SM measured x 2 flops x "
                                        f"{sms} SMs x {sm_mhz:.0f} MHz"}
    return out


def traffic_of(stage: str, n_vis: int):
    """DRAM bytes per launch of a stage's kernels from the committed ncu summary
    (a "traffic <stage> <bytes> bytes n_vis <n> sources <file>=<sha256[:16]> ..."
    line under profiles/), if it was taken on this workload size and none of the
    named sources changed since (else None)."""
    import glob
    for path in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for line in open(path):
            f = line.split()
            if len(f) < 7 or f[0] != "traffic" or f[1] != stage or f[3] != "bytes":
                continue
            if f[4] != "n_vis" or int(f[5]) != int(n_vis) or f[6] != "sources":
                continue
            for item in f[7:]:
                src, _, digest = item.partition("=")
                try:
                    h = hashlib.sha256(open(os.path.join(ROOT, src), "rb").read()).hexdigest()
                except OSError:
                    return None
                if h[:16] != digest:
                    return None
            return int(f[2])
    return None


def max_over_ranks(ms: float, dist=None, device=None) -> float:
    """The largest of the ranks' times in ms (the whole job ends with its slowest
    replica); ``ms`` itself without a process group."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: int, steps: int, world: int, ms: float) -> float:
    """Units per second of the whole job: every replica processes units_per_rank
    units per step, and the job takes the slowest replica's ms for all steps."""
    return units_per_rank * steps * world / (ms / 1e3)


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_params(wl, n_w=None):
    import oracle
    return oracle.Params(n=wl.n, n_w=wl.n_w if n_w is None else n_w, fov=wl.fov,
                         kernel=oracle.KB if wl.kernel == "kb" else oracle.GAUSS,
                         support=wl.support, tile=wl.tile)


def oracle_slabs(wl, data):
    """The workload cut along w for timing the oracle in bounded pieces: the
    oracle's own plane of every kept visibility (wl.n_w planes over the whole w
    range), and per plane the indices of its visibilities, in input order.
    Returns the planes in an interleaved order (outer and inner planes mixed)
    and the slabs."""
    import numpy as np

    import oracle
    g = oracle.coords(oracle_params(wl), data["uvw"])
    kept = np.flatnonzero(g["status"] == 0)
    pl = g["plane"][kept]
    order = np.argsort(pl, kind="stable")
    counts = np.bincount(pl, minlength=wl.n_w)
    starts = np.concatenate([[0], np.cumsum(counts)])
    slabs = [kept[order[starts[k]:starts[k + 1]]] for k in range(wl.n_w)]
    step = 7 if wl.n_w % 7 else 5
    return [(k * step) % wl.n_w for k in range(wl.n_w)], slabs


def slab_arrays(data, idx):
    """One slab's inputs in the dtypes the oracle computes in (FP64, complex128),
    so that its call converts nothing."""
    import numpy as np
    return (np.ascontiguousarray(data["uvw"][idx]), data["vis"][idx].astype(np.complex128),
            data["weight"][idx].astype(np.float64))


def oracle_slab(wl, arrays):
    """The oracle's image of one slab: its visibilities gridded on the full
    n x n grid as one w-plane, the FFT of that plane, its w-correction and the
    taper division -- 1/n_w of the whole job's planes with their visibilities."""
    import oracle
    uvw, vis, wt = arrays
    oracle.image(oracle_params(wl, n_w=1), uvw, vis, wt)


def cpu_baseline(wl, data, budget_s: float = 20.0) -> dict:
    """The FP64 oracle as it stands on the host cores, on a bounded sample of the
    workload: whole w-plane slabs (each slab's visibilities gridded on the full
    grid, one FFT, the w-correction), until about budget_s seconds have been
    spent; plus the split of one slab into gridding, FFT and the rest."""
    import numpy as np

    import oracle
    order, slabs = oracle_slabs(wl, data)
    oracle_slab(wl, slab_arrays(data, slabs[order[0]][:1000]))  # the taper table (kept)
    done_vis, spent, planes = 0, 0.0, 0
    timed = []
    for k in order:
        arr = slab_arrays(data, slabs[k])
        t0 = time.perf_counter()
        oracle_slab(wl, arr)
        dt = time.perf_counter() - t0
        timed.append((len(slabs[k]), k, dt))
        done_vis += len(slabs[k])
        spent += dt
        planes += 1
        if spent >= budget_s:
            break
    # the split of the fullest timed slab: its gridding and one FFT again
    nv, k, dt = max(timed)
    arr = slab_arrays(data, slabs[k])
    t1 = time.perf_counter()
    oracle.grid(oracle_params(wl, n_w=1), *arr)
    t_grid = time.perf_counter() - t1
    t1 = time.perf_counter()
    oracle.fft2d(np.zeros((wl.n, wl.n), np.complex128), +1)
    t_fft = time.perf_counter() - t1
    split = {"plane": int(k), "n_vis": int(nv), "total_s": dt, "grid_s": t_grid, "fft_s": t_fft,
             "wcorrect_taper_s": max(dt - t_grid - t_fft, 0.0),
             "grid_includes": "coordinates, plane and kernel weights of every visibility"}
    n_kept = sum(len(x) for x in slabs)
    return {"value": done_vis / spent, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{planes} of the {wl.n_w} w-plane slabs of the workload ({done_vis} of its "
                      f"{n_kept} kept visibilities), each imaged by the oracle as one plane on "
                      f"the full {wl.n}^2 grid (gridding, FFT, w-correction, taper); {spent:.1f} s",
            "whole_job_estimate_s": n_kept / (done_vis / spent),
            "split_one_slab": split}


def run_reference(args, wl):
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import oracle
    import synth

    data = synth.generate(wl.obs)
    order, slabs = oracle_slabs(wl, data)
    oracle_slab(wl, slab_arrays(data, slabs[order[0]][:1000]))  # the taper table (kept)
    plan = [order[s % len(order)] for s in range(args.warmup + args.steps)]
    for k in plan[:args.warmup]:
        oracle_slab(wl, slab_arrays(data, slabs[k]))
    spent, vis = 0.0, 0
    for k in plan[args.warmup:]:
        arr = slab_arrays(data, slabs[k])
        t0 = time.perf_counter()
        oracle_slab(wl, arr)
        spent += time.perf_counter() - t0
        vis += len(slabs[k])
    value = vis / spent
    cores = oracle.max_threads()
    sample = (f"each step: one of the {wl.n_w} w-plane slabs of the workload (its visibilities "
              f"gridded by the oracle as one plane on the full {wl.n}^2 grid, one FFT, the "
              f"w-correction and taper), the planes in turn; {vis} visibilities in the timed steps")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": spent / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_of(wl),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def config_of(wl) -> dict:
    return {"workload": f"{wl.name}: {wl.obs.n_keep} visibilities ({wl.obs.n_ant} stations, "
                        f"{wl.obs.n_chan} channels), {wl.n}^2 grid, {wl.n_w} w-planes, "
                        f"{'Kaiser-Bessel' if wl.kernel == 'kb' else 'Gaussian'} support "
                        f"{wl.support}, uv-tile {wl.tile}",
            "n_vis": wl.obs.n_keep, "grid": wl.n, "w_planes": wl.n_w, "kernel": wl.kernel,
            "support": wl.support, "tile": wl.tile, "precision": "fp32",
            "l2": "inputs (uvw+vis+weight) larger than L2; no flush"}


def device_step(P, wl, data, dev, steps, warmup, dist=None, local=0, sample_clocks=False):
    """Time `steps` steps (bin, sparse grid, fused FFT + w-correct) of a workload
    with its inputs resident in HBM: CUDA events on the current stream, the
    whole region and each stage.  Returns the measurements and the imager
    (still open) with the device inputs."""
    import torch
    n_vis = len(data["vis"])
    uvw = torch.from_numpy(data["uvw"]).to(dev)
    vis = torch.from_numpy(data["vis"]).to(dev)
    wt = torch.from_numpy(data["weight"]).to(dev)
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                  max_vis=n_vis, device=dev)
    img = torch.empty((wl.n, wl.n), dtype=torch.float32, device=dev)

    def step(ev=None):
        if ev is not None:
            ev[0].record()
        im.bin(uvw, vis, wt)
        if ev is not None:
            ev[1].record()
        im.grid_sparse()
        if ev is not None:
            ev[2].record()
        im.fft_wcorrect(out=img)
        if ev is not None:
            ev[3].record()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    n_binned = im.stats()["n_binned"]
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    t_start, t_end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clocks = Clocks(local) if sample_clocks else None
    if clocks:
        clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    l0 = im.launches()
    h0 = time.time()
    t_start.record()
    for k in range(steps):
        step(evs[k])
    t_end.record()
    torch.cuda.synchronize()
    h1 = time.time()
    if dist:
        dist.barrier()
    out = {"clocks": clocks.stop(h0, h1) if clocks else None,
           "launches": im.launches() - l0,
           "ms": max_over_ranks(t_start.elapsed_time(t_end), dist, dev),
           "stage_ms": {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in evs)
                        for i, name in enumerate(["bin", "grid", "fft_wcorrect"])},
           "n_vis": n_vis, "n_binned": n_binned}
    out["tiles"], out["tile_rows"], out["planes_read"] = im.fused_tiles(planes=True)
    alg = algorithmic_bytes(n_vis, n_binned, wl.n, wl.n_w, wl.tile, out["tiles"], out["tile_rows"])
    out["alg"] = alg
    out["gbps"] = {k: alg[k] / (out["stage_ms"][k] * 1e-3) / 1e9 for k in out["stage_ms"]}
    return out, im, (uvw, vis, wt, img)


def timed_calls(call, steps, warmup, dist=None, dev=None, finish=None):
    """ms of `steps` calls of `call` on the current stream (CUDA events), after
    `warmup` untimed calls; `finish` (enqueue-only) runs before the end event,
    e.g. to join copies that the calls left on another stream."""
    import torch
    for _ in range(max(1, warmup)):
        call()
    if finish:
        finish()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        call()
    if finish:
        finish()
    e1.record()
    torch.cuda.synchronize()
    t = max_over_ranks(e0.elapsed_time(e1), dist, dev)
    if dist:
        dist.barrier()
    return t


def run_ours(args, wl):
    import torch

    import synth
    import paper_2411_07321_gb300 as P

    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    data = synth.generate(wl.obs, rows=True)
    n_vis = len(data["vis"])
    m, im, (uvw, vis, wt, img) = device_step(P, wl, data, dev, args.steps, args.warmup, dist,
                                              local, sample_clocks=True)
    ms = m["ms"]
    value = whole_job_rate(n_vis, args.steps, world, ms)

    # the unfused stages (grid clearing every tile, cuFFT in place, plane sum),
    # timed after the headline steps, for comparison
    uevs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)]
            for _ in range(max(3, args.steps // 2))]
    for e in uevs:
        e[0].record()
        im.bin(uvw, vis, wt)
        e[1].record()
        im.grid()
        e[2].record()
        im.fft(+1)
        e[3].record()
        im.wcorrect(out=img)
        e[4].record()
    torch.cuda.synchronize()
    unfused_ms = {name: statistics.mean(e[i].elapsed_time(e[i + 1]) for e in uevs[1:])
                  for i, name in enumerate(["bin", "grid_clear", "cufft", "wcorrect"])}

    # the w-phase ablation: the fused transform with the phase argument in
    # plain FP32 instead of double-single arithmetic, on the same binning
    im.bin(uvw, vis, wt)
    im.grid_sparse()
    fp32_phase_ms = timed_calls(
        lambda: im.fft_wcorrect(flags=P.imager.IMAGE_FLAGS | P.rick.RICK_PHASE_FP32, out=img),
        args.steps, args.warmup, dist, dev) / args.steps
    ds_phase_ms = timed_calls(lambda: im.fft_wcorrect(out=img), args.steps, args.warmup,
                              dist, dev) / args.steps

    # Briggs-robust weighting: the extra passes per image, after a binning of
    # the same visibilities -- density weights, then re-weighting the records
    im.bin(uvw, vis, wt)

    def reweight():
        w2 = im.density_weights("briggs", 0.0, wt)
        im.bin_values(vis, w2)

    weighting_ms = timed_calls(reweight, args.steps, args.warmup, dist, dev)

    # end to end through the host-buffer calls (pinned host in, image back to
    # pinned host memory, every copy inside the timed region): the streamed
    # path (chunks of args.chunk visibilities, copies overlapping binning and
    # gridding) is the headline; the resident path (all inputs copied, then
    # imaged) is kept for comparison
    uvw_h = torch.from_numpy(data["uvw"]).pin_memory()
    vis_h = torch.from_numpy(data["vis"]).pin_memory()
    wt_h = torch.from_numpy(data["weight"]).pin_memory()
    out_h = torch.empty((wl.n, wl.n), dtype=torch.float32).pin_memory()
    ims = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                   max_vis=min(args.chunk, n_vis), device=dev)
    e2e_vis_ms = timed_calls(lambda: ims.image_streamed(uvw_h, vis_h, wt_h, out_h), args.steps,
                             args.warmup, dist, dev, finish=ims.join_out)
    e2e_resident_ms = timed_calls(lambda: im.image_from_host(uvw_h, vis_h, wt_h, out_h),
                                  args.steps, args.warmup, dist, dev)
    # the same visibilities as rows of n_chan channels (a measurement set's
    # layout): uvw once per row and a factor per channel
    n_chan = wl.obs.n_chan
    if n_vis % n_chan == 0:
        rows_h = torch.from_numpy(data["uvw_rows"]).pin_memory()
        scale_h = torch.from_numpy(data["chan_scale"]).pin_memory()
        e2e_ms = timed_calls(
            lambda: ims.image_streamed(rows_h, vis_h, wt_h, out_h, chan_scale=scale_h),
            args.steps, args.warmup, dist, dev, finish=ims.join_out)
        h2d = rows_h.numel() * 8 + scale_h.numel() * 8 + n_vis * (8 + 4)
        call = (f"Imager.image_streamed with chan_scale (rick_image_host_rows, one "
                f"correlation): rows of {n_chan} channels with uvw once per row, chunks of "
                f"{min(args.chunk, n_vis)} visibilities, w range from the data; the image "
                f"copied back to pinned host memory inside the timed region")
    else:
        e2e_ms, h2d = e2e_vis_ms, n_vis * (24 + 8 + 4)
        call = (f"Imager.image_streamed (rick_image_host), chunks of {min(args.chunk, n_vis)} "
                f"visibilities, w range from the data")
    ims.close()
    im.close()
    del uvw, vis, wt, img, ims, im
    torch.cuda.empty_cache()
    e2e_value = whole_job_rate(n_vis, args.steps, world, e2e_ms)

    stage_ms, alg, gbps = m["stage_ms"], m["alg"], m["gbps"]
    peak, peak_kind = peaks()
    rates = probe_rates(P)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    sm_mhz = (m["clocks"] or {}).get("sm_mhz") or (m["clocks"] or {}).get("sm_max_mhz") or 2070.0
    roofs = stage_rooflines(wl, m, rates, sms, sm_mhz, peak)
    dom = max(stage_ms, key=lambda k: stage_ms[k])
    kernel_name = {"bin": "rick_bin (all binning kernels)", "grid": "grid_kernel",
                   "fft_wcorrect": "fft_rows_kernel + fft_cols_kernel"}[dom]
    roofline = {**roofs[dom], "kernel": kernel_name, "stage": dom,
                "traffic": traffic_of(dom, n_vis), "algorithmic_bytes": alg[dom],
                "peak_source": ("measured HBM copy bandwidth" if roofs[dom]["bound"] == "hbm"
                                else "measured by rick_probe_throughput on this GPU") +
                               f" ({peak_kind} MEASURED_PEAKS.json for HBM)"}
    unfused = {"ms": unfused_ms, "ms_per_step": sum(unfused_ms.values()),
               "gbps": {k: alg[k] / (unfused_ms[k] * 1e-3) / 1e9 for k in unfused_ms},
               "calls": "rick_bin, rick_grid (clears record-free tiles), rick_fft_wplanes "
                        "(cuFFT in place), rick_wcorrect_stack"}

    extras = {}
    if world == 1 and args.n_vis is None and not args.no_extras and args.workload != "lofar":
        # the LOFAR-like workload's step (device-resident inputs)
        lw = synth.WORKLOADS["lofar"]
        ld = synth.generate(lw.obs)
        lm, lim, (luvw, lvis, lwt, _) = device_step(P, lw, ld, dev, args.steps, args.warmup)
        lim.close()
        # the precision ablation of this workload: compensated FP32 gridding
        # (sums of rounds of 4096 records folded by Neumaier's summation)
        cim = P.Imager(lw.n, lw.n_w, lw.fov, kernel=lw.kernel, support=lw.support, tile=lw.tile,
                       max_vis=len(ld["vis"]), device=dev, precision="compensated")
        cim.bin(luvw, lvis, lwt)
        comp_grid_ms = timed_calls(cim.grid_sparse, args.steps, args.warmup) / args.steps
        cim.close()
        del lim, cim, luvw, lvis, lwt
        torch.cuda.empty_cache()
        extras["lofar"] = {
            "workload": config_of(lw)["workload"], "value": len(ld["vis"]) / (lm["ms"] / args.steps * 1e-3),
            "unit": UNIT, "ms_per_step": lm["ms"] / args.steps, "stage_ms": lm["stage_ms"],
            "gbps": lm["gbps"], "launches": lm["launches"],
            "compensated_grid_ms": comp_grid_ms}
        del ld
        extras["serving"] = serve_measure(args.extra_serve_jobs, args.serve_slots)
        extras["grad"] = grad_measure(args.steps, args.warmup)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    cpu = None
    if world == 1 and not args.no_cpu_baseline and args.n_vis is None:
        cpu = cpu_baseline(wl, data, args.cpu_budget)
    line = {
        **({"profiling_subset": True} if args.n_vis is not None else {}),
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {**config_of(wl), "parallelism": f"replicas{world}"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": wl.n * wl.n * 4, "ms_per_step": e2e_ms / args.steps,
                "call": call,
                "per_visibility_uvw": {
                    "value": whole_job_rate(n_vis, args.steps, world, e2e_vis_ms),
                    "ms_per_step": e2e_vis_ms / args.steps,
                    "h2d_bytes_per_step": n_vis * (24 + 8 + 4),
                    "call": "Imager.image_streamed (rick_image_host), uvw per visibility"},
                "resident_call_ms_per_step": e2e_resident_ms / args.steps},
        "roofline": roofline,
        "stages": {"ms": stage_ms, "gbps": gbps, "algorithmic_bytes": alg, "roofline": roofs,
                   "probe_ops_per_clock_per_sm": rates, "planes_read": m["planes_read"],
                   "n_binned": m["n_binned"], "tiles_with_records": m["tiles"],
                   "tile_rows_with_records": m["tile_rows"],
                   "calls": "rick_bin, rick_grid_sparse, rick_fft_wcorrect (sparse)"},
        "unfused": unfused,
        "phase_ablation": {"fft_wcorrect_ms": {"double_single": ds_phase_ms,
                                               "fp32": fp32_phase_ms},
                           "what": "rick_fft_wcorrect with the w-phase argument in "
                                   "double-single arithmetic (default) and with "
                                   "RICK_PHASE_FP32, same binning and planes"},
        "weighting": {"scheme": "briggs, robust 0", "ms_per_image": weighting_ms / args.steps,
                      "passes": "rick_density_weights + rick_bin_values, after a binning"},
        **extras,
        "cpu_baseline": cpu,
        "clocks": m["clocks"],
        "gpu_launches": m["launches"],
    }
    print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def serve_measure(n_jobs: int, slots: int) -> dict:
    """The serving workload: n_jobs imaging requests with Poisson arrivals,
    log-uniform 1e4..1e7 visibilities (prefixes of the LOFAR-like tracks), grids
    512^2..4096^2, 4..16 w-planes, Gaussian or Kaiser-Bessel W=7.  The plain
    per-request path (fresh plan and buffers per request) is run first,
    back to back, to measure its mean service time; both paths then serve the
    same arrival trace at 0.8 / (that mean)."""
    import threading

    import numpy as np
    import torch

    import synth
    from paper_2411_07321_gb300 import serve as S

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    d = synth.generate(synth.scaled("lofar", n_keep=10_000_000).obs)
    host = {k: torch.from_numpy(d[k]).pin_memory() for k in ("uvw", "vis", "weight")}
    rng = np.random.default_rng(5)
    specs = []
    for jid in range(n_jobs):
        n_vis = int(np.exp(rng.uniform(np.log(1e4), np.log(1e7))))
        n = int(rng.choice([512, 1024, 2048, 4096]))
        specs.append(dict(n_vis=n_vis, n=n, n_w=int(rng.integers(4, 17)),
                          kernel=str(rng.choice(["gauss", "kb"])), job_id=jid))

    def job(sp, arrival=None):
        nv = sp["n_vis"]
        j = S.ImagingJob(host["uvw"][:nv], host["vis"][:nv], host["weight"][:nv], n=sp["n"],
                         n_w=sp["n_w"], fov=S.fov_for(sp["n"], 7, 12000.0), kernel=sp["kernel"],
                         support=7, tile=64, job_id=sp["job_id"])
        if arrival is not None:
            j.arrival = arrival
        return j

    # plain service times, back to back
    S.run_plain(job(specs[0]))  # CUDA context, cuFFT and allocator warm-up
    service, plain_imgs = [], {}
    for sp in specs:
        t0 = time.perf_counter()
        img = S.run_plain(job(sp))
        service.append(time.perf_counter() - t0)
        if sp["job_id"] < 8:
            plain_imgs[sp["job_id"]] = img
    mean_service = float(np.mean(service))
    plain_saturated = n_jobs / float(np.sum(service))
    total_vis = sum(sp["n_vis"] for sp in specs)

    def summary(lat, wall):
        return {"jobs_per_s": n_jobs / wall, "vis_per_s": total_vis / wall,
                "p50_ms": 1e3 * S.percentile(lat, 50), "p99_ms": 1e3 * S.percentile(lat, 99),
                "mean_ms": 1e3 * float(np.mean(lat)), "wall_s": wall}

    def plain_trace(offsets):
        """The plain path on an arrival trace: one request at a time, in order."""
        t_base = time.perf_counter() + 0.2
        lat, done = [], t_base
        for sp, off in zip(specs, offsets):
            arrival = t_base + off
            while time.perf_counter() < arrival:
                time.sleep(2e-4)
            S.run_plain(job(sp))
            done = time.perf_counter()
            lat.append(done - arrival)
        return summary(lat, done - t_base)

    def served_trace(srv, offsets):
        t_base = time.perf_counter() + 0.2
        futs = [None] * n_jobs

        def feed():
            for i, (sp, off) in enumerate(zip(specs, offsets)):
                arrival = t_base + off
                while time.perf_counter() < arrival:
                    time.sleep(2e-4)
                futs[i] = srv.submit(job(sp, arrival))

        th = threading.Thread(target=feed)
        th.start()
        th.join()
        res = [f.result() for f in futs]
        wall = max(t_base + off + r.latency_s for off, r in zip(offsets, res)) - t_base
        return summary([r.latency_s for r in res], wall), res

    # arrival traces at 0.8 and 1.5 times the plain path's capacity (1 / its
    # mean service time): at 0.8 both paths keep up and latency tells them
    # apart; at 1.5 the plain path falls behind and throughput does
    loads = {"0.8": 0.8, "1.5": 1.5}
    offsets = {k: S.poisson_arrivals(n_jobs, v / mean_service, seed=6) for k, v in loads.items()}
    plain = {k: plain_trace(o) for k, o in offsets.items()}
    served = {}
    with S.Server(dev, max_running=slots) as srv:
        # saturated throughput: every request queued at once (also warms the slots)
        t0 = time.perf_counter()
        sat = [srv.submit(job(sp)) for sp in specs]
        for f in sat:
            f.result()
        served_saturated = n_jobs / (time.perf_counter() - t0)
        for k, o in offsets.items():
            served[k], res = served_trace(srv, o)
            if k == "0.8":
                res08 = res
        peak_used = srv.peak_used
        counters = dict(srv.counters)
    # the same saturated run (a fresh server, as above) with the small requests
    # admitted together gridded by one merged launch
    with S.Server(dev, max_running=slots, merge_small=True) as srv:
        t0 = time.perf_counter()
        for f in [srv.submit(job(sp)) for sp in specs]:
            f.result()
        served_merged = n_jobs / (time.perf_counter() - t0)
        merged_counters = {k: srv.counters[k] for k in ("batches", "batched")}
    err = 0.0  # inner region |l|, |m| < fov/4: clear of the taper's corner amplification
    for jid, img in plain_imgs.items():
        n = img.shape[0]
        inner = (slice(n // 4, 3 * n // 4),) * 2
        ref = img[inner].astype(np.float64)
        err = max(err, float(np.abs(res08[jid].image[inner] - ref).max() / np.abs(ref).max()))

    return {
        "n_jobs": n_jobs, "unit": "jobs/s", "value": served["1.5"]["jobs_per_s"],
        "value_is": "served throughput on the 1.5-load trace",
        "config": {"workload": f"{n_jobs} requests, Poisson arrivals at 0.8 and 1.5 / mean "
                               "plain service time; n_vis log-uniform 1e4..1e7 (LOFAR-like "
                               "tracks); grids 512..4096; 4..16 w-planes; Gaussian or KB W=7",
                   "arrival_rate_hz": {k: v / mean_service for k, v in loads.items()},
                   "slots": slots},
        "served": served["0.8"], "plain": plain["0.8"],
        "overload_1_5": {"served": served["1.5"], "plain": plain["1.5"]},
        "saturated_jobs_per_s": {"served": served_saturated, "plain": plain_saturated,
                                 "served_with_merged_gridding": served_merged,
                                 "merged_gridding_counters": merged_counters},
        "plain_mean_service_ms": 1e3 * mean_service, "served_peak_hbm_bytes": peak_used,
        "max_rel_diff_served_vs_plain_inner": err, "server_counters": counters,
    }


def run_serve(args):
    r = serve_measure(args.serve_jobs, args.serve_slots)
    print(json.dumps({"metric": METRIC, "mode": "serve", "n_gpus": 1, "higher_is_better": True,
                      "data": "synthetic", **r}), flush=True)


def grad_measure(steps: int, warmup: int) -> dict:
    """The differentiable workload: the gradient of chi^2 = sum w |V_obs - D x|^2
    with respect to a float32 image x of 50 point sources, on 1e7 visibilities
    (4 channels of the LOFAR-like tracks), a 2048^2 grid, 16 w-planes, KB W=7.
    One step = forward (DegridFn: w-spread, forward cuFFT per plane, degrid) +
    backward (GridFn of the residual: re-weight the records, sparse grid, fused
    inverse FFT + w-correction)."""
    import numpy as np
    import torch

    import synth
    import paper_2411_07321_gb300 as P
    from paper_2411_07321_gb300.autograd import chi2

    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    wl = synth.WORKLOADS["diff"]
    d = synth.generate(wl.obs)
    n_vis = len(d["vis"])
    t = {k: torch.from_numpy(d[k]).to(dev) for k in ("uvw", "vis", "weight")}
    im = P.Imager(wl.n, wl.n_w, wl.fov, kernel=wl.kernel, support=wl.support, tile=wl.tile,
                  max_vis=n_vis, device=dev)
    im.bin(t["uvw"], t["vis"], t["weight"])
    rng = np.random.default_rng(4)
    x = np.zeros((wl.n, wl.n), np.float32)
    x.flat[rng.choice(wl.n * wl.n, 50, replace=False)] = \
        np.exp(rng.uniform(np.log(0.1), np.log(10.0), 50))
    xt = torch.from_numpy(x).to(dev).requires_grad_(True)

    def step(ev=None):
        xt.grad = None
        if ev is not None:
            ev[0].record()
        loss = chi2(xt, im, t["vis"], t["weight"])
        if ev is not None:
            ev[1].record()
        loss.backward()
        if ev is not None:
            ev[2].record()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        step()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    for ev in evs:
        step(ev)
    torch.cuda.synchronize()
    fwd = statistics.mean(ev[0].elapsed_time(ev[1]) for ev in evs)
    bwd = statistics.mean(ev[1].elapsed_time(ev[2]) for ev in evs)
    out = {
        "unit": "vis/s", "value": n_vis / (ms * 1e-3),
        "ms_per_step": ms, "steps": steps, "warmup": warmup,
        "ms_forward": fwd, "ms_backward": bwd,
        "config": {"workload": f"diff: {n_vis} visibilities (60 stations, 4 channels), "
                               f"{wl.n}^2 grid, {wl.n_w} w-planes, Kaiser-Bessel support "
                               f"{wl.support}; gradient of chi^2 wrt a 50-source float32 image",
                   "step": "chi2 forward (predict) + backward (grid of the residual)",
                   "fused_transform": im.fused},
    }
    im.close()
    return out


def run_grad(args):
    r = grad_measure(args.steps, args.warmup)
    print(json.dumps({"metric": METRIC, "mode": "grad", "n_gpus": 1, "higher_is_better": True,
                      "dtype": "f32", "data": "synthetic", **r}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default="large")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle work in cpu_baseline (whole w-plane slabs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the extra keys (LOFAR-like step, serving trace, gradient)")
    ap.add_argument("--extra-serve-jobs", type=int, default=64,
                    help="requests of the serving trace in the default line")
    ap.add_argument("--chunk", type=int, default=1 << 26,
                    help="visibilities per chunk of the streamed end-to-end call")
    ap.add_argument("--serve", action="store_true",
                    help="run the serving workload instead (its own JSON line)")
    ap.add_argument("--grad", action="store_true",
                    help="time the chi^2 gradient on the differentiable workload (own JSON line)")
    ap.add_argument("--serve-jobs", type=int, default=256)
    ap.add_argument("--serve-slots", type=int, default=8)
    ap.add_argument("--n-vis", type=int, default=None,
                    help="profiling aid: image only the first N visibilities (not a bench line)")
    ap.add_argument("--n-w", type=int, default=None,
                    help="profiling aid: this many w-planes (not a bench line)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("bench.py: --warmup must be at least 3")
    import synth

    wl = synth.WORKLOADS[args.workload]
    if args.n_vis is not None or args.n_w is not None:
        wl = synth.scaled(args.workload, n_keep=args.n_vis,
                          **({"n_w": args.n_w} if args.n_w is not None else {}))
        args.n_vis = wl.obs.n_keep
    if args.serve:
        run_serve(args)
    elif args.grad:
        run_grad(args)
    elif args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
