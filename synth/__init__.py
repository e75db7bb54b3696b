"""Seeded synthetic observations and the named imaging workloads.

The only module both the CUDA path's tests/benchmark and the FP64 oracle take
inputs from.  It contains no imaging arithmetic: it draws LOFAR-like earth-
rotation uvw tracks and a point-source sky (the measurement equation, Eq. 1 of
De Rubeis et al., evaluated directly) in ``synth.c``.

The paper measured on LOFAR HBA measurement sets (its Table 1: 62 / 72 stations,
8 h at 4 s, 150.5 / 144.6 MHz, Dec +27.5 / +64 deg), which are not available;
these workloads stand in for them with the same structure: a dense station core
(half the stations within 2 km) plus log-radially spread remote stations, so the
uv coverage piles up at the centre as in real LOFAR data.
"""
from __future__ import annotations

import ctypes
import math
import os
import platform
import subprocess
from dataclasses import dataclass, field, replace

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "synth.c")
_LIB = os.path.join(_HERE, "libsynth.so")


def build(force: bool = False) -> str:
    stamp = _LIB + ".arch"
    try:
        same_arch = open(stamp).read().strip() == platform.machine()
    except OSError:
        same_arch = False
    if force or not same_arch or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off",
                        "-fopenmp", "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(platform.machine())
    return _LIB


class _Cfg(ctypes.Structure):
    _fields_ = [("seed", ctypes.c_int64), ("n_ant", ctypes.c_int32), ("n_steps", ctypes.c_int32),
                ("n_chan", ctypes.c_int32), ("n_src", ctypes.c_int32),
                ("core_frac", ctypes.c_double), ("core_radius", ctypes.c_double),
                ("max_radius", ctypes.c_double), ("latitude", ctypes.c_double),
                ("dec", ctypes.c_double), ("hours", ctypes.c_double), ("nu0", ctypes.c_double),
                ("dnu", ctypes.c_double), ("uv_max", ctypes.c_double), ("w_max", ctypes.c_double),
                ("field", ctypes.c_double), ("flux_min", ctypes.c_double),
                ("flux_max", ctypes.c_double), ("flux_index", ctypes.c_double),
                ("noise_sigma", ctypes.c_double), ("weight_mode", ctypes.c_int32),
                ("pad", ctypes.c_int32)]


DEG = math.pi / 180.0


@dataclass
class Observation:
    """Generator settings (metres, radians, Hz, wavelengths)."""
    seed: int
    n_ant: int
    n_steps: int
    n_chan: int
    n_src: int
    n_keep: int
    uv_max: float
    w_max: float
    field: float
    flux_min: float
    flux_max: float
    flux_index: float = 0.0
    noise_sigma: float = 0.01
    weight_mode: int = 0
    dec: float = 64.0 * DEG
    latitude: float = 52.9 * DEG
    hours: float = 8.0
    nu0: float = 144.6e6
    dnu: float = 12.207e3
    core_frac: float = 0.5
    core_radius: float = 2000.0
    max_radius: float = 80000.0

    def c(self) -> _Cfg:
        return _Cfg(self.seed, self.n_ant, self.n_steps, self.n_chan, self.n_src, self.core_frac,
                    self.core_radius, self.max_radius, self.latitude, self.dec, self.hours,
                    self.nu0, self.dnu, self.uv_max, self.w_max, self.field, self.flux_min,
                    self.flux_max, self.flux_index, self.noise_sigma, self.weight_mode, 0)


@dataclass
class Workload:
    """A named imaging job: the observation and the imaging parameters."""
    name: str
    obs: Observation
    n: int
    n_w: int
    fov: float
    kernel: str            # "gauss" | "kb"
    support: int
    tile: int = 64
    extra: dict = field(default_factory=dict)


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        L.sx_observation.restype = ctypes.c_int64
        D = ctypes.POINTER(ctypes.c_double)
        F = ctypes.POINTER(ctypes.c_float)
        L.sx_observation.argtypes = [ctypes.POINTER(_Cfg), ctypes.c_int64, D, F, F, D, D, D, D, D]
        _lib = L
    return _lib


def generate(obs: Observation, rows: bool = False):
    """Returns dict(uvw f64 [n,3], vis c64 [n], weight f32 [n], src_l, src_m, src_flux);
    with rows=True also uvw_rows f64 [ceil(n / n_chan), 3] and chan_scale f64
    [n_chan], with uvw[r * n_chan + c] = uvw_rows[r] * chan_scale[c] exactly."""
    n = obs.n_keep
    uvw = np.empty((n, 3), np.float64)
    n_rows = (n + obs.n_chan - 1) // obs.n_chan
    ur = np.empty((n_rows, 3), np.float64) if rows else None
    cf = np.empty(obs.n_chan, np.float64) if rows else None
    vis = np.empty(n, np.complex64)
    wt = np.empty(n, np.float32)
    k = max(obs.n_src, 1)
    sl, sm, ss = np.empty(k), np.empty(k), np.empty(k)
    D = ctypes.POINTER(ctypes.c_double)
    F = ctypes.POINTER(ctypes.c_float)
    got = lib().sx_observation(ctypes.byref(obs.c()), n, uvw.ctypes.data_as(D),
                               vis.ctypes.data_as(F), wt.ctypes.data_as(F), sl.ctypes.data_as(D),
                               sm.ctypes.data_as(D), ss.ctypes.data_as(D),
                               ur.ctypes.data_as(D) if rows else None,
                               cf.ctypes.data_as(D) if rows else None)
    out = dict(uvw=uvw[:got], vis=vis[:got], weight=wt[:got], src_l=sl[:obs.n_src],
               src_m=sm[:obs.n_src], src_flux=ss[:obs.n_src])
    if rows:
        out.update(uvw_rows=ur[:(got + obs.n_chan - 1) // obs.n_chan], chan_scale=cf)
    return out


# The five workloads.  Sizes follow the paper's Table 2 shapes scaled to one GPU.
WORKLOADS = {
    # 32 stations (496 baselines) x 133 steps, first 65,536; 1 channel; Dec +27.5 (LOFAR Dutch).
    "small": Workload(
        "small", Observation(seed=1, n_ant=32, n_steps=133, n_chan=1, n_src=20, n_keep=65536,
                             uv_max=2000.0, w_max=300.0, field=2.0 * DEG, flux_min=0.1,
                             flux_max=10.0, flux_index=0.0, noise_sigma=0.01, weight_mode=0,
                             dec=27.5 * DEG, nu0=150.5e6, dnu=97.656e3),
        n=256, n_w=8, fov=2.0 * DEG, kernel="gauss", support=7, tile=32),
    # 60 stations (1770 baselines) x 1766 steps x 16 channels, first 5e7; Dec +64 (LOFAR ILT).
    "lofar": Workload(
        "lofar", Observation(seed=2, n_ant=60, n_steps=1766, n_chan=16, n_src=200,
                             n_keep=50_000_000, uv_max=12000.0, w_max=5000.0, field=8.0 * DEG,
                             flux_min=0.05, flux_max=10.0, flux_index=-1.8, noise_sigma=0.01,
                             weight_mode=1),
        n=4096, n_w=16, fov=8.0 * DEG, kernel="kb", support=7, tile=64),
    # same generator, 64 channels, first 2e8.
    "large": Workload(
        "large", Observation(seed=3, n_ant=60, n_steps=1766, n_chan=64, n_src=200,
                             n_keep=200_000_000, uv_max=12000.0, w_max=5000.0, field=8.0 * DEG,
                             flux_min=0.05, flux_max=10.0, flux_index=-1.8, noise_sigma=0.01,
                             weight_mode=1),
        n=8192, n_w=32, fov=8.0 * DEG, kernel="kb", support=9, tile=64),
    # 4 channels, first 1e7, 2048^2 grid.
    "diff": Workload(
        "diff", Observation(seed=4, n_ant=60, n_steps=1766, n_chan=4, n_src=50,
                            n_keep=10_000_000, uv_max=6000.0, w_max=2500.0, field=4.0 * DEG,
                            flux_min=0.1, flux_max=10.0, flux_index=0.0, noise_sigma=0.01,
                            weight_mode=1),
        n=2048, n_w=16, fov=4.0 * DEG, kernel="kb", support=7, tile=64),
}


def scaled(name: str, n_keep: int | None = None, **image_overrides) -> Workload:
    """A copy of a named workload with fewer visibilities and/or other imaging sizes."""
    w = WORKLOADS[name]
    obs = w.obs if n_keep is None else replace(w.obs, n_keep=n_keep)
    return replace(w, obs=obs, **image_overrides)
