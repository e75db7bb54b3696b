"""Torch-facing wrapper of the C ABI: device buffers, streams and stage order.

``Imager`` keeps one configuration's state resident on the GPU -- the plan
(cuFFT plan, taper table), the binning workspace, the w-planes and the image
-- and calls the library's stages on the current torch stream.  It does no
arithmetic of its own: every stage is a librick.so kernel (or cuFFT).
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import rick as R

KERNELS = {"gauss": R.RICK_KERNEL_GAUSS, "kb": R.RICK_KERNEL_KB}
PRECISIONS = {"fp32": R.RICK_PREC_FP32, "compensated": R.RICK_PREC_FP32_COMPENSATED}
IMAGE_FLAGS = R.RICK_N_CORRECT | R.RICK_NORMALIZE     # the image of Eq. 2, flux-normalised
PREDICT_FLAGS = R.RICK_N_DIVIDE                       # the 1/n of Eq. 1, for model visibilities


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stats_from_bytes(raw: np.ndarray) -> dict:
    i = raw[:24].view(np.int64)
    d = raw[24:48].view(np.float64)
    return dict(n_binned=int(i[0]), n_dropped_uv=int(i[1]), n_dropped_w=int(i[2]),
                sum_weight=float(d[0]), w_min=float(d[1]), w_max=float(d[2]))


class Imager:
    def __init__(self, n: int, n_w: int, fov: float, kernel: str = "kb", support: int = 7,
                 tile: int = 64, w_range: tuple[float, float] | None = None,
                 kb_beta: float = math.nan, gauss_sigma: float = math.nan,
                 precision: str = "fp32", max_vis: int = 1 << 20, device=None,
                 image_n: int | None = None, fused: bool = True,
                 hermitian_mirror: bool = False, deterministic: bool = False):
        """n is the grid side; the image is the central image_n x image_n crop
        (default n: no padding), with pixel size fov / n.  With ``fused`` (and n
        in 256 ... 8192) images are made by the fused sparse transform +
        w-correction (rick_grid_sparse, rick_fft_wcorrect); otherwise, and in
        the explicit grid / fft / wcorrect stages, by cuFFT in place and the
        plane-sum kernel.  ``hermitian_mirror`` grids every visibility also as
        conj(V) at -uvw (RICK_OPT_HERMITIAN_MIRROR); ``deterministic`` makes
        binning and gridding bitwise repeatable (RICK_OPT_DETERMINISTIC)."""
        self.device = torch.device(device if device is not None else "cuda")
        if self.device.type != "cuda":
            raise ValueError("Imager runs on a CUDA device only")
        wmin, wmax = (math.nan, math.nan) if w_range is None else map(float, w_range)
        self.params = R.make_params(n, n_w, fov, KERNELS[kernel], support, wmin, wmax, kb_beta,
                                    gauss_sigma, tile, PRECISIONS[precision],
                                    0 if image_n is None else image_n,
                                    (R.RICK_OPT_HERMITIAN_MIRROR if hermitian_mirror else 0) |
                                    (R.RICK_OPT_DETERMINISTIC if deterministic else 0))
        self.n, self.n_w, self.max_vis = int(n), int(n_w), int(max_vis)
        self.m = int(image_n) if image_n else self.n
        with torch.cuda.device(self.device):
            self.plan = R.rick_plan_create(self.params, self.max_vis)
            self.ws_bytes, self.plane_bytes = R.rick_workspace_bytes(self.params, self.max_vis)
            self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
            self._planes_all = torch.empty((self.n_w, self.n, self.n), dtype=torch.complex64,
                                           device=self.device)
            self.planes = self._planes_all
            self.stats_buf = torch.zeros(48, dtype=torch.uint8, device=self.device)
        self.fft_bytes = R.rick_plan_fft_bytes(self.plan)
        self.n_vis = 0
        self.fused = bool(fused) and R.rick_fft_wcorrect_bytes(self.plan) is not None
        self._fwork = None

    # ---------------------------------------------------------------- helpers
    def _stream(self) -> int:
        return torch.cuda.current_stream(self.device).cuda_stream

    def _check(self, t: torch.Tensor, dtype, shape=None, name="tensor"):
        if t.device != self.device or t.dtype != dtype or not t.is_contiguous():
            raise ValueError(f"{name} must be a contiguous {dtype} tensor on {self.device}")
        if shape is not None and tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")

    def footprint_bytes(self) -> int:
        """Device bytes this imager holds (workspace, planes, cuFFT area, and the
        fused transform's work buffer)."""
        fb = R.rick_fft_wcorrect_bytes(self.plan) if self.fused else 0
        return self.ws_bytes + self.plane_bytes + self.fft_bytes + (fb or 0) + 48

    # ---------------------------------------------------------------- stages
    def bin(self, uvw: torch.Tensor, vis: torch.Tensor, weight: torch.Tensor | None = None):
        n = uvw.shape[0]
        self._check(uvw, torch.float64, (n, 3), "uvw")
        self._check(vis, torch.complex64, (n,), "vis")
        if weight is not None:
            self._check(weight, torch.float32, (n,), "weight")
        R.rick_bin(self.plan, n, uvw.data_ptr(), vis.data_ptr(), _ptr(weight), self.ws.data_ptr(),
                   self.ws_bytes, self.stats_buf.data_ptr(), self._stream())
        self.n_vis = n

    def bin_channels(self, uvw_rows: torch.Tensor, chan_scale: torch.Tensor, vis: torch.Tensor,
                     weight: torch.Tensor | None = None, n_corr: int = 1):
        """Binning of rows of n_chan channels: uvw once per row, times a factor per
        channel (vis and weight hold n_rows * n_chan * n_corr values, correlation
        fastest, then channel).  With n_corr > 1 each (row, channel) is gridded
        as the weighted sum of its correlations (rick_bin_rows)."""
        n_rows, n_chan = uvw_rows.shape[0], chan_scale.shape[0]
        nv = n_rows * n_chan * n_corr
        self._check(uvw_rows, torch.float64, (n_rows, 3), "uvw_rows")
        self._check(chan_scale, torch.float64, (n_chan,), "chan_scale")
        self._check(vis.reshape(-1), torch.complex64, (nv,), "vis")
        if weight is not None:
            self._check(weight.reshape(-1), torch.float32, (nv,), "weight")
        R.rick_bin_rows(self.plan, n_rows, n_chan, n_corr, uvw_rows.data_ptr(),
                        chan_scale.data_ptr(), vis.data_ptr(), _ptr(weight), self.ws.data_ptr(),
                        self.ws_bytes, self.stats_buf.data_ptr(), self._stream())
        self.n_vis = n_rows * n_chan

    def bin_values(self, vis: torch.Tensor, weight: torch.Tensor | None = None):
        self._check(vis, torch.complex64, (self.n_vis,), "vis")
        if weight is not None:
            self._check(weight, torch.float32, (self.n_vis,), "weight")
        R.rick_bin_values(self.plan, vis.data_ptr(), _ptr(weight), self.ws.data_ptr(),
                          self.stats_buf.data_ptr(), self._stream())

    def density_weights(self, scheme: str = "briggs", robust: float = 0.0,
                        weight: torch.Tensor | None = None) -> torch.Tensor:
        """Uniform or Briggs-robust imaging weights (float32, input order) from the
        uv-cell density of the last binning; ``weight`` are the weights that
        binning was given (None: unit)."""
        schemes = {"uniform": R.RICK_WEIGHT_UNIFORM, "briggs": R.RICK_WEIGHT_BRIGGS}
        if weight is not None:
            self._check(weight, torch.float32, (self.n_vis,), "weight")
        need = R.rick_density_scratch_bytes(self.params)
        if getattr(self, "_dens", None) is None or self._dens.numel() < need:
            self._dens = torch.empty(need, dtype=torch.uint8, device=self.device)
        out = torch.empty(self.n_vis, dtype=torch.float32, device=self.device)
        R.rick_density_weights(self.plan, self.n_vis, _ptr(weight), self.ws.data_ptr(),
                               schemes[scheme], robust, self._dens.data_ptr(), self._dens.numel(),
                               out.data_ptr(), self._stream())
        return out

    def image_weighted(self, uvw, vis, weight=None, scheme: str = "briggs", robust: float = 0.0,
                       flags: int = IMAGE_FLAGS, out=None) -> torch.Tensor:
        """The image with uniform or Briggs-robust weighting: bin, density
        weights, re-weight the records, grid, FFT, w-correct."""
        self.bin(uvw, vis, weight)
        w2 = self.density_weights(scheme, robust, weight)
        self.bin_values(vis, w2)
        return self.image_from_binned(flags, out)

    def grid(self):
        R.rick_grid(self.plan, self.ws.data_ptr(), self.planes.data_ptr(), self._stream())

    def fft(self, direction: int):
        R.rick_fft_wplanes(self.plan, self.planes.data_ptr(), direction, self._stream())

    def wcorrect(self, flags: int = IMAGE_FLAGS, out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty((self.m, self.m), dtype=torch.float32, device=self.device)
        self._check(out, torch.float32, (self.m, self.m), "image")
        R.rick_wcorrect_stack(self.plan, self.planes.data_ptr(), self.ws.data_ptr(),
                              out.data_ptr(), flags, self._stream())
        return out

    def grid_sparse(self):
        """Gridding that writes only the tiles records reach (for fft_wcorrect)."""
        R.rick_grid_sparse(self.plan, self.ws.data_ptr(), self.planes.data_ptr(), self._stream())

    def fft_wcorrect(self, flags: int = IMAGE_FLAGS, out: torch.Tensor | None = None,
                     sparse: bool = True) -> torch.Tensor:
        """The inverse FFT of the planes fused with the w-correction and plane
        sum (rick_fft_wcorrect): the image of planes from grid() or
        grid_sparse() (sparse: read only the tiles with records); the planes
        are not modified."""
        self._fused_work()
        if out is None:
            out = torch.empty((self.m, self.m), dtype=torch.float32, device=self.device)
        self._check(out, torch.float32, (self.m, self.m), "image")
        R.rick_fft_wcorrect(self.plan, self.planes.data_ptr(), self.ws.data_ptr(), int(sparse),
                            self._fwork.data_ptr(), self._fwork.numel(), out.data_ptr(), flags,
                            self._stream())
        return out

    def _fused_work(self) -> torch.Tensor:
        need = R.rick_fft_wcorrect_bytes(self.plan)
        if need is None:
            raise ValueError(f"the fused transform does not cover n = {self.n}")
        if self._fwork is None or self._fwork.numel() < need:
            self._fwork = None
            self._fwork = torch.empty(need, dtype=torch.uint8, device=self.device)
        return self._fwork

    def wspread_fft(self, image: torch.Tensor, flags: int = IMAGE_FLAGS):
        """w-spreading fused with the forward FFT of the planes (rick_wspread_fft):
        the adjoint's planes, written for the tiles the last binning's records
        reach (what degrid reads)."""
        self._check(image, torch.float32, (self.m, self.m), "image")
        w = self._fused_work()
        R.rick_wspread_fft(self.plan, image.data_ptr(), self.ws.data_ptr(), w.data_ptr(),
                           w.numel(), self.planes.data_ptr(), flags, self._stream())

    def fused_tiles(self, planes: bool = False):
        """(plane, uv-tile) and (plane, tile-row) pairs the last fft_wcorrect read
        (from the flags at the head of its work buffer); with ``planes`` also the
        number of planes it transformed."""
        if self._fwork is None:
            return (0, 0, 0) if planes else (0, 0)
        nt = self.n // self.params.tile
        al = lambda x: (x + 255) // 256 * 256
        nf = self.n_w * nt * nt
        tiles = int(self._fwork[:nf].sum())
        o = al(nf)
        rows = int(self._fwork[o:o + self.n_w * nt].sum())
        if not planes:
            return tiles, rows
        o += al(self.n_w * nt)
        return tiles, rows, int(self._fwork[o:o + self.n_w].sum())

    def wspread(self, image: torch.Tensor, flags: int = IMAGE_FLAGS):
        self._check(image, torch.float32, (self.m, self.m), "image")
        R.rick_wspread(self.plan, image.data_ptr(), self.ws.data_ptr(), self.planes.data_ptr(),
                       flags, self._stream())

    def degrid(self, weight: torch.Tensor | None = None,
               out: torch.Tensor | None = None) -> torch.Tensor:
        if out is None:
            out = torch.empty(self.n_vis, dtype=torch.complex64, device=self.device)
        self._check(out, torch.complex64, (self.n_vis,), "vis_out")
        if weight is not None:
            self._check(weight, torch.float32, (self.n_vis,), "weight")
        R.rick_degrid(self.plan, self.ws.data_ptr(), self.planes.data_ptr(), _ptr(weight),
                      out.data_ptr(), self._stream())
        return out

    # ---------------------------------------------------------------- compositions
    def image(self, uvw, vis, weight=None, flags: int = IMAGE_FLAGS, out=None) -> torch.Tensor:
        """bin -> grid -> inverse FFT per plane -> w-correct + stack (§2 steps 2-4)."""
        self.bin(uvw, vis, weight)
        return self.image_from_binned(flags, out)

    def image_from_binned(self, flags: int = IMAGE_FLAGS, out=None) -> torch.Tensor:
        if self.fused:
            self.grid_sparse()
            return self.fft_wcorrect(flags, out, sparse=True)
        self.grid()
        self.fft(+1)
        return self.wcorrect(flags, out)

    def adjoint(self, image: torch.Tensor, weight=None, flags: int = IMAGE_FLAGS,
                out=None, fused: bool | None = None) -> torch.Tensor:
        """Transpose of image_from_binned: w-spread -> forward FFT -> degrid (the
        first two fused where the imager uses the fused transform, unless
        ``fused`` is False)."""
        if self.fused if fused is None else fused:
            self.wspread_fft(image, flags)
        else:
            self.wspread(image, flags)
            self.fft(-1)
        return self.degrid(weight, out)

    def predict(self, image: torch.Tensor, out=None) -> torch.Tensor:
        """Model visibilities of a sky image through the binned geometry (Eq. 1)."""
        return self.adjoint(image, None, PREDICT_FLAGS, out)

    def image_from_host(self, uvw_host: torch.Tensor, vis_host: torch.Tensor,
                        weight_host: torch.Tensor | None, out_host: torch.Tensor,
                        flags: int = IMAGE_FLAGS) -> torch.Tensor:
        """The image from host buffers (pinned for asynchronous copies): the
        inputs are copied into resident device buffers, imaged, and the image is
        copied back into ``out_host``, all on the current stream."""
        self.bin_from_host(uvw_host, vis_host, weight_host)
        self.image_from_binned(flags, out=self._image_buffer())
        out_host.copy_(self._out_img, non_blocking=True)
        return out_host

    def bin_from_host(self, uvw_host: torch.Tensor, vis_host: torch.Tensor,
                      weight_host: torch.Tensor | None):
        """The first half of image_from_host: the host inputs copied into the
        resident device buffers and binned, on the current stream."""
        n = uvw_host.shape[0]
        if n > self.max_vis:
            raise ValueError(f"{n} visibilities exceed this imager's capacity {self.max_vis}")
        if getattr(self, "_in_uvw", None) is None:
            self._in_uvw = torch.empty((self.max_vis, 3), dtype=torch.float64, device=self.device)
            self._in_vis = torch.empty(self.max_vis, dtype=torch.complex64, device=self.device)
            self._in_wt = torch.empty(self.max_vis, dtype=torch.float32, device=self.device)
        uvw, vis = self._in_uvw[:n], self._in_vis[:n]
        uvw.copy_(uvw_host, non_blocking=True)
        vis.copy_(vis_host, non_blocking=True)
        wt = None
        if weight_host is not None:
            wt = self._in_wt[:n]
            wt.copy_(weight_host, non_blocking=True)
        self.bin(uvw, vis, wt)

    def transform_to_host(self, out_host: torch.Tensor, flags: int = IMAGE_FLAGS) -> torch.Tensor:
        """The second half of image_from_host after gridding: the fused
        transform of the gridded planes (rick_fft_wcorrect, sparse) and the
        image copied into ``out_host``, on the current stream."""
        self.fft_wcorrect(flags, self._image_buffer(), sparse=True)
        out_host.copy_(self._out_img, non_blocking=True)
        return out_host

    def _image_buffer(self) -> torch.Tensor:
        if getattr(self, "_out_img", None) is None or self._out_img.shape[0] != self.m:
            self._out_img = torch.empty((self.m, self.m), dtype=torch.float32, device=self.device)
        return self._out_img

    def image_streamed(self, uvw_host: torch.Tensor, vis_host: torch.Tensor,
                       weight_host: torch.Tensor | None, out_host: torch.Tensor | None = None,
                       flags: int = IMAGE_FLAGS,
                       chan_scale: torch.Tensor | None = None, n_corr: int = 1) -> torch.Tensor:
        """The image of a visibility set in host memory, of any size, streamed
        through the GPU in chunks of this imager's ``max_vis`` (copies of the
        next chunk overlap binning and gridding of the current one; pinned
        host tensors give the overlap).  With ``chan_scale`` (float64
        [n_chan]) the input is multi-channel: ``uvw_host`` holds one row per
        n_chan visibilities, scaled per channel, and each visibility may carry
        ``n_corr`` correlations (vis and weight [rows][chan][corr], folded into
        one record as in ``bin_channels``).  Returns the device image,
        ordered on the current stream.  If ``out_host`` is given the image is
        also copied there on this imager's copy-out stream, so that the copy
        overlaps the next call's work: synchronise the device (or call
        ``wait_out()``) before reading it.  Consecutive calls alternate between
        two device image buffers."""
        n_units = uvw_host.shape[0]
        n_chan = 0 if chan_scale is None else chan_scale.shape[0]
        if n_corr != 1 and not n_chan:
            raise ValueError("correlations need the row form (chan_scale)")
        n = n_units * max(n_chan, 1)
        nv = n * n_corr
        vis_host = vis_host.reshape(-1)
        weight_host = None if weight_host is None else weight_host.reshape(-1)
        for t, dt, shape, name in ((uvw_host, torch.float64, (n_units, 3), "uvw"),
                                   (vis_host, torch.complex64, (nv,), "vis"),
                                   (weight_host, torch.float32, (nv,), "weight"),
                                   (chan_scale, torch.float64, (n_chan,), "chan_scale")):
            if t is None:
                continue
            if t.device.type != "cpu" or t.dtype != dt or not t.is_contiguous() or \
                    tuple(t.shape) != shape:
                raise ValueError(f"{name} must be a contiguous {dt} host tensor of shape {shape}")
        need = R.rick_stream_bytes(self.params, self.max_vis, n)
        if getattr(self, "_stage", None) is None or self._stage.numel() < need:
            self._stage = None
            self._stage = torch.empty(need, dtype=torch.uint8, device=self.device)
        if getattr(self, "_out_imgs", None) is None:
            self._out_imgs = [None, None]
            self._out_done = [None, None]
            self._out_i = 0
            self._copy_out = torch.cuda.Stream(device=self.device)
        i = self._out_i
        self._out_i ^= 1
        cur = torch.cuda.current_stream(self.device)
        if self._out_done[i] is not None:  # the copy-out of this buffer two calls ago
            cur.wait_event(self._out_done[i])
        if self._out_imgs[i] is None or self._out_imgs[i].shape[0] != self.m:
            self._out_imgs[i] = torch.empty((self.m, self.m), dtype=torch.float32,
                                            device=self.device)
        img = self._out_imgs[i]
        if n_chan:
            R.rick_image_host_rows(self.plan, n_units, n_chan, n_corr, uvw_host.data_ptr(),
                                   chan_scale.data_ptr(), vis_host.data_ptr(),
                                   _ptr(weight_host), self.ws.data_ptr(), self.ws_bytes,
                                   self._stage.data_ptr(), self._stage.numel(),
                                   self.planes.data_ptr(), img.data_ptr(), flags,
                                   self.stats_buf.data_ptr(), self._stream())
            rows = max(self.max_vis // (n_chan * n_corr), 1)
            last = n_units - (n_units - 1) // rows * rows if n_units else 0
            self.n_vis = last * n_chan  # the last chunk
        else:
            R.rick_image_host(self.plan, n, uvw_host.data_ptr(), vis_host.data_ptr(),
                              _ptr(weight_host), self.ws.data_ptr(), self.ws_bytes,
                              self._stage.data_ptr(), self._stage.numel(), self.planes.data_ptr(),
                              img.data_ptr(), flags, self.stats_buf.data_ptr(), self._stream())
            self.n_vis = n - (n - 1) // self.max_vis * self.max_vis if n else 0  # the last chunk
        if out_host is not None:
            ready = torch.cuda.Event()
            ready.record(cur)
            self._copy_out.wait_event(ready)
            with torch.cuda.stream(self._copy_out):
                out_host.copy_(img, non_blocking=True)
            done = torch.cuda.Event()
            done.record(self._copy_out)
            self._out_done[i] = done
        else:
            self._out_done[i] = None
        return img

    def join_out(self):
        """Make the current stream wait for this imager's pending copies into
        ``out_host`` (enqueue only): work or events recorded on the stream
        afterwards follow those copies."""
        cur = torch.cuda.current_stream(self.device)
        for ev in getattr(self, "_out_done", None) or ():
            if ev is not None:
                cur.wait_event(ev)

    def wait_out(self):
        """Wait until the copies into ``out_host`` of ``image_streamed`` are done."""
        if getattr(self, "_copy_out", None) is not None:
            self._copy_out.synchronize()

    def set_geometry(self, fov: float, w_range: tuple[float, float] | None = None):
        """Re-target the resident plan to another field of view / w range."""
        wmin, wmax = (math.nan, math.nan) if w_range is None else map(float, w_range)
        R.rick_plan_set_geometry(self.plan, fov, wmin, wmax)
        self.params.fov, self.params.w_min, self.params.w_max = float(fov), wmin, wmax

    def set_planes(self, n_w: int):
        """Re-target the resident plan to n_w w-planes, at most the count it was
        created with (rick_plan_set_planes): the buffers stay, the planes are
        their first n_w."""
        R.rick_plan_set_planes(self.plan, n_w)
        self.params.n_w = self.n_w = int(n_w)
        self.planes = self._planes_all[:self.n_w]

    def set_image_n(self, image_n: int | None):
        """Re-target the resident plan to another crop of its grid (None: no crop)."""
        R.rick_plan_set_image_n(self.plan, 0 if image_n is None else image_n)
        self.params.image_n = 0 if image_n is None else int(image_n)
        self.m = int(image_n) if image_n else self.n

    def set_kernel(self, kernel: str, support: int, kb_beta: float = math.nan,
                   gauss_sigma: float = math.nan):
        """Re-target the resident plan to another gridding kernel (the taper
        table and kernel fits are rebuilt, the cuFFT plan stays).  Work this
        imager enqueued must be complete."""
        R.rick_plan_set_kernel(self.plan, KERNELS[kernel], support, kb_beta, gauss_sigma)
        self.params.kernel, self.params.support = KERNELS[kernel], int(support)
        self.params.kb_beta, self.params.gauss_sigma = float(kb_beta), float(gauss_sigma)

    def launches(self) -> int:
        """Library kernels this imager's plan has enqueued so far."""
        return R.rick_plan_launch_count(self.plan)

    def stats(self) -> dict:
        return _stats_from_bytes(self.stats_buf.cpu().numpy())

    def binned(self) -> dict:
        """Copies of the binned records (host numpy), via the C ABI's layout view."""
        v = R.rick_bin_layout(self.plan)
        st = self.stats()
        nb = st["n_binned"]
        raw = self.ws

        def take(off, nbytes):
            return raw[off:off + nbytes].cpu().numpy()

        rec = take(v.rec, 16 * nb).view(np.float32).reshape(-1, 4)
        return dict(offsets=take(v.offsets, 4 * (v.n_bins + 1)).view(np.uint32),
                    perm=take(v.perm, 4 * nb).view(np.uint32),
                    rec_val=np.ascontiguousarray(rec[:, :2]).view(np.complex64).reshape(-1),
                    rec_frac=np.ascontiguousarray(rec[:, 2:]),
                    rec_cell=take(v.rec_cell, 4 * nb).view(np.uint32), stats=st)

    def close(self):
        """Release the plan.  Work this imager enqueued must be complete (its
        stream synchronised) -- the server only closes idle slots."""
        if getattr(self, "plan", None):
            torch.cuda.current_stream(self.device).synchronize()
            self.wait_out()
            R.rick_plan_destroy(self.plan)
            self.plan = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_sparse_batch(imagers) -> None:
    """rick_grid_sparse of several imagers' last binnings in one launch
    (rick_grid_sparse_batch), on the current stream of the first imager's
    device.  The imagers share support and tile, use FP32 sums and are not
    deterministic; at most RICK_GRID_BATCH_MAX of them."""
    imagers = list(imagers)
    if not imagers:
        return
    st = torch.cuda.current_stream(imagers[0].device).cuda_stream
    R.rick_grid_sparse_batch([im.plan for im in imagers], [im.ws.data_ptr() for im in imagers],
                             [im.planes.data_ptr() for im in imagers], st)
