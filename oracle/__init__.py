"""FP64 reference of the w-stacking imaging path (RICK, De Rubeis et al., §2).

TEST INFRASTRUCTURE ONLY.  The tests, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` are the only callers.  The product path (the CUDA
library and its Python binding) never imports this package, and this package
imports nothing from the product.

The arithmetic lives in ``oracle.c`` (plain C, FP64, compiled with
``-ffp-contract=off`` so that every ``a*b+c`` rounds twice unless the source
calls ``fma`` explicitly).  This module only marshals numpy arrays.

Functions and the passage each follows:
  kernel / i0 / taper   -- §2 ("G kernel is a Kaiser-Bessel function"), plus the
                           Gaussian and the taper correction (readings listed in
                           oracle.c's header)
  fft1d / fft2d         -- radix-2 Cooley-Tukey, the transform of §2 step 3
  coords / bin          -- §2 closest w-plane + gridding sub-step 1 (binning)
  grid                  -- Eq. 3
  image                 -- §2 steps 2-4, Eq. 2 (optionally the central image_n x
                           image_n pixels of a padded grid)
  adjoint               -- exact transpose of ``image`` (degridding)
  kb_beta               -- KB shape for a grid oversampling (Beatty et al. 2005)
  dft                   -- brute-force inverse of Eq. 1 at pixel centres
"""
from __future__ import annotations

import ctypes
import os
import platform
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

GAUSS, KB = 0, 1
N_CORRECT, NORMALIZE, N_DIVIDE = 1, 2, 4


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, FP64, no contraction)."""
    stamp = _LIB + ".arch"
    try:
        same_arch = open(stamp).read().strip() == platform.machine()
    except OSError:
        same_arch = False
    if force or not same_arch or not os.path.exists(_LIB) or \
            os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
        with open(stamp, "w") as f:
            f.write(platform.machine())
    return _LIB


class _Params(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("n_w", ctypes.c_int32), ("fov", ctypes.c_double),
                ("w_min", ctypes.c_double), ("w_max", ctypes.c_double),
                ("kernel", ctypes.c_int32), ("support", ctypes.c_int32),
                ("kb_beta", ctypes.c_double), ("gauss_sigma", ctypes.c_double),
                ("tile", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("image_n", ctypes.c_int32), ("reserved_", ctypes.c_int32)]


@dataclass
class Params:
    """Imaging parameters in the paper's terms (uvw in wavelengths, §2)."""
    n: int
    n_w: int
    fov: float
    kernel: int = KB
    support: int = 7
    w_min: float = float("nan")
    w_max: float = float("nan")
    kb_beta: float = float("nan")
    gauss_sigma: float = float("nan")
    tile: int = 64
    image_n: int = 0  # side of the central crop kept (grid padding n / image_n); 0: n

    def side(self) -> int:
        return self.image_n if self.image_n > 0 else self.n

    def c(self) -> _Params:
        return _Params(self.n, self.n_w, self.fov, self.w_min, self.w_max, self.kernel,
                       self.support, self.kb_beta, self.gauss_sigma, self.tile, 0,
                       self.image_n, 0)


_lib = None
_D = ctypes.POINTER(ctypes.c_double)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        P = ctypes.POINTER(_Params)
        L.or_i0.restype = ctypes.c_double
        L.or_i0.argtypes = [ctypes.c_double]
        L.or_kb_beta_default.restype = ctypes.c_double
        L.or_kb_beta_default.argtypes = [ctypes.c_int32]
        L.or_kb_beta.restype = ctypes.c_double
        L.or_kb_beta.argtypes = [ctypes.c_int32, ctypes.c_double]
        L.or_kernel.restype = ctypes.c_double
        L.or_kernel.argtypes = [P, ctypes.c_double]
        L.or_taper.restype = ctypes.c_double
        L.or_taper.argtypes = [P, ctypes.c_double]
        L.or_taper_row.argtypes = [P, _D]
        L.or_fft1d.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.or_fft2d.argtypes = [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]
        L.or_wrange.argtypes = [ctypes.c_int64, _D, _D, _D]
        L.or_coords.restype = ctypes.c_int64
        L.or_coords.argtypes = [P, ctypes.c_int64, _D, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int32, _I32, _I32, _I32, _D, _D, _I32]
        L.or_plane_centre.restype = ctypes.c_double
        L.or_plane_centre.argtypes = [P, ctypes.c_int32, ctypes.c_double, ctypes.c_double]
        L.or_nbins.restype = ctypes.c_int64
        L.or_nbins.argtypes = [P]
        L.or_bin.argtypes = [P, ctypes.c_int64, _I32, _I32, _I32, _I32, _I32, _I64, _I64]
        L.or_image.argtypes = [P, ctypes.c_int64, _D, ctypes.c_void_p, ctypes.c_void_p,
                               ctypes.c_uint32, _D, ctypes.c_void_p, _D]
        L.or_grid.argtypes = [P, ctypes.c_int64, _D, ctypes.c_void_p, ctypes.c_void_p,
                              ctypes.c_void_p, _D]
        L.or_adjoint.argtypes = [P, ctypes.c_int64, _D, ctypes.c_void_p, ctypes.c_uint32, _D,
                                 ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_void_p]
        L.or_dft.argtypes = [ctypes.c_int32, ctypes.c_double, ctypes.c_int64, _D,
                             ctypes.c_void_p, ctypes.c_void_p, ctypes.c_uint32, ctypes.c_double,
                             _D]
        L.or_image_pixels.argtypes = [P, ctypes.c_int64, _D, ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_uint32, ctypes.c_int32, _I32, _I32, _D]
        L.or_density_weights.argtypes = [P, ctypes.c_int64, _D, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.c_double, _D]
        L.or_max_threads.restype = ctypes.c_int32
        _lib = L
    return _lib


def _p(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _vp(a):
    return None if a is None else ctypes.c_void_p(a.ctypes.data)


def _uvw(uvw):
    return np.ascontiguousarray(uvw, dtype=np.float64).reshape(-1, 3)


def _vis(vis):
    return np.ascontiguousarray(vis, dtype=np.complex128)


def _wt(weight):
    return None if weight is None else np.ascontiguousarray(weight, dtype=np.float64)


def i0(x: float) -> float:
    return lib().or_i0(float(x))


def kb_beta_default(W: int) -> float:
    return lib().or_kb_beta_default(int(W))


def kb_beta(W: int, alpha: float) -> float:
    return lib().or_kb_beta(int(W), float(alpha))


def kernel(p: Params, d: float) -> float:
    return lib().or_kernel(ctypes.byref(p.c()), float(d))


def taper(p: Params, nu: float) -> float:
    return lib().or_taper(ctypes.byref(p.c()), float(nu))


def taper_row(p: Params) -> np.ndarray:
    """C((i - n/2) / n) for i = 0 .. n-1 (the taper along one grid axis)."""
    out = np.empty(p.n, np.float64)
    lib().or_taper_row(ctypes.byref(p.c()), out.ctypes.data_as(_D))
    return out


def fft1d(a, sign: int) -> np.ndarray:
    out = np.array(a, dtype=np.complex128, copy=True)
    lib().or_fft1d(ctypes.c_void_p(out.ctypes.data), out.shape[0], int(sign))
    return out


def fft2d(a, sign: int) -> np.ndarray:
    out = np.array(a, dtype=np.complex128, copy=True, order="C")
    lib().or_fft2d(ctypes.c_void_p(out.ctypes.data), out.shape[0], int(sign))
    return out


def wrange(uvw):
    uvw = _uvw(uvw)
    lo, hi = ctypes.c_double(), ctypes.c_double()
    lib().or_wrange(uvw.shape[0], _p(uvw, ctypes.c_double), ctypes.byref(lo), ctypes.byref(hi))
    return lo.value, hi.value


def coords(p: Params, uvw):
    """Per-visibility geometry: dict(plane, ax, ay, fx, fy, status, w_min, w_max)."""
    uvw = _uvw(uvw)
    n = uvw.shape[0]
    given = not (np.isnan(p.w_min) or np.isnan(p.w_max))
    wmin, wmax = (p.w_min, p.w_max) if given else wrange(uvw)
    out = dict(plane=np.empty(n, np.int32), ax=np.empty(n, np.int32), ay=np.empty(n, np.int32),
               fx=np.empty(n, np.float64), fy=np.empty(n, np.float64),
               status=np.empty(n, np.int32))
    lib().or_coords(ctypes.byref(p.c()), n, _p(uvw, ctypes.c_double), wmin, wmax, int(given),
                    _p(out["plane"], ctypes.c_int32), _p(out["ax"], ctypes.c_int32),
                    _p(out["ay"], ctypes.c_int32), _p(out["fx"], ctypes.c_double),
                    _p(out["fy"], ctypes.c_double), _p(out["status"], ctypes.c_int32))
    out["w_min"], out["w_max"] = wmin, wmax
    return out


def plane_centre(p: Params, k: int, wmin: float, wmax: float) -> float:
    return lib().or_plane_centre(ctypes.byref(p.c()), int(k), float(wmin), float(wmax))


def nbins(p: Params) -> int:
    return lib().or_nbins(ctypes.byref(p.c()))


def bin(p: Params, uvw):
    """Binning: dict(key (-1 = dropped), perm (sorted position -> input index),
    offsets (nbins + 1), and the per-visibility geometry of ``coords``)."""
    g = coords(p, uvw)
    n = g["plane"].shape[0]
    key = np.empty(n, np.int32)
    kept = int((g["status"] == 0).sum())
    perm = np.empty(max(kept, 1), np.int64)
    offsets = np.empty(nbins(p) + 1, np.int64)
    lib().or_bin(ctypes.byref(p.c()), n, _p(g["plane"], ctypes.c_int32),
                 _p(g["ax"], ctypes.c_int32), _p(g["ay"], ctypes.c_int32),
                 _p(g["status"], ctypes.c_int32), _p(key, ctypes.c_int32),
                 _p(perm, ctypes.c_int64), _p(offsets, ctypes.c_int64))
    g.update(key=key, perm=perm[:kept], offsets=offsets)
    return g


def _stats(st):
    return dict(n_binned=int(st[0]), n_dropped_uv=int(st[1]), n_dropped_w=int(st[2]),
                sum_weight=float(st[3]), w_min=float(st[4]), w_max=float(st[5]))


def image(p: Params, uvw, vis, weight=None, flags: int = N_CORRECT | NORMALIZE,
          want_acc: bool = False):
    """The w-stacked image (FP64), image_n x image_n (the central crop of the n x n
    grid's image).  Returns (image, stats) or (image, acc, stats); acc is the
    n x n plane sum before scaling."""
    uvw, vis, wt = _uvw(uvw), _vis(vis), _wt(weight)
    img = np.empty((p.side(), p.side()), np.float64)
    acc = np.empty((p.n, p.n), np.complex128) if want_acc else None
    st = np.zeros(6, np.float64)
    lib().or_image(ctypes.byref(p.c()), uvw.shape[0], _p(uvw, ctypes.c_double), _vp(vis), _vp(wt),
                   int(flags), _p(img, ctypes.c_double), _vp(acc), _p(st, ctypes.c_double))
    return (img, acc, _stats(st)) if want_acc else (img, _stats(st))


def grid(p: Params, uvw, vis, weight=None):
    """Gridded planes g_k (no checkerboard, no FFT), complex128 [n_w, n, n]."""
    uvw, vis, wt = _uvw(uvw), _vis(vis), _wt(weight)
    planes = np.empty((p.n_w, p.n, p.n), np.complex128)
    st = np.zeros(6, np.float64)
    lib().or_grid(ctypes.byref(p.c()), uvw.shape[0], _p(uvw, ctypes.c_double), _vp(vis),
                  _vp(wt), _vp(planes), _p(st, ctypes.c_double))
    return planes, _stats(st)


def adjoint(p: Params, uvw, image_in, weight=None, flags: int = N_CORRECT | NORMALIZE,
            w_min=None, w_max=None, sum_weight=None):
    """Transpose of ``image`` (weights applied) or, with weight=None and other
    flags, the degridding predictor.  image_in is image_n x image_n.  Geometry
    (w range, weight sum) defaults to the forward operator's."""
    uvw, wt = _uvw(uvw), _wt(weight)
    y = np.ascontiguousarray(image_in, dtype=np.float64)
    assert y.shape == (p.side(), p.side())
    if w_min is None or w_max is None:
        given = not (np.isnan(p.w_min) or np.isnan(p.w_max))
        w_min, w_max = (p.w_min, p.w_max) if given else wrange(uvw)
    if sum_weight is None:
        st = coords(p, uvw)["status"] == 0
        sum_weight = float(np.sum(wt[st])) if wt is not None else float(st.sum())
    out = np.empty(uvw.shape[0], np.complex128)
    lib().or_adjoint(ctypes.byref(p.c()), uvw.shape[0], _p(uvw, ctypes.c_double), _vp(wt),
                     int(flags), _p(y, ctypes.c_double), float(w_min), float(w_max),
                     float(sum_weight), _vp(out))
    return out


def dft(n: int, fov: float, uvw, vis, weight=None, flags: int = 0, sum_weight: float = 1.0):
    """Brute-force direct transform at pixel centres (inverse of Eq. 1)."""
    uvw, vis, wt = _uvw(uvw), _vis(vis), _wt(weight)
    img = np.empty((n, n), np.float64)
    lib().or_dft(int(n), float(fov), uvw.shape[0], _p(uvw, ctypes.c_double), _vp(vis), _vp(wt),
                 int(flags), float(sum_weight), _p(img, ctypes.c_double))
    return img


def image_pixels(p: Params, uvw, vis, weight, pixels, flags: int = N_CORRECT | NORMALIZE):
    """The w-stacked image at the given (p, q) pixels of the n x n grid frame
    (a crop's pixel p' is p' + (n - image_n)/2 there), evaluated per visibility
    (no FFT): for checking a few pixels of a large image."""
    uvw, vis, wt = _uvw(uvw), _vis(vis), _wt(weight)
    pix = np.asarray(pixels, np.int32).reshape(-1, 2)
    px, py = np.ascontiguousarray(pix[:, 0]), np.ascontiguousarray(pix[:, 1])
    out = np.empty(len(pix), np.float64)
    lib().or_image_pixels(ctypes.byref(p.c()), uvw.shape[0], _p(uvw, ctypes.c_double), _vp(vis),
                          _vp(wt), int(flags), len(pix), _p(px, ctypes.c_int32),
                          _p(py, ctypes.c_int32), _p(out, ctypes.c_double))
    return out


WEIGHT_UNIFORM, WEIGHT_BRIGGS = 1, 2


def density_weights(p: Params, uvw, weight=None, scheme: int = WEIGHT_BRIGGS,
                    robust: float = 0.0) -> np.ndarray:
    """Uniform or Briggs-robust imaging weights (FP64), 0 for dropped visibilities."""
    uvw, wt = _uvw(uvw), _wt(weight)
    out = np.empty(uvw.shape[0], np.float64)
    lib().or_density_weights(ctypes.byref(p.c()), uvw.shape[0], _p(uvw, ctypes.c_double),
                             _vp(wt), int(scheme), float(robust), _p(out, ctypes.c_double))
    return out


def max_threads() -> int:
    return int(lib().or_max_threads())
