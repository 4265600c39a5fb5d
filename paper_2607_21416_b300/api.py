"""Tensor-level binding of libgs: device buffers (PyTorch tensors) in, C-ABI
calls out.  PyTorch supplies device memory and streams only; every step of the
rendering path runs in libgs kernels.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, field

import numpy as np
import torch

from . import _lib as L


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


# ---------------------------------------------------------------------------
class Views:
    """A batch of keyframes: resolutions (host) and cameras (device)."""

    def __init__(self, cams, wh, device="cuda"):
        cams = torch.as_tensor(np.asarray(cams, np.float32)).reshape(-1, 16)
        wh = np.asarray(wh, np.int32).reshape(-1, 2)
        self.V = int(wh.shape[0])
        if self.V < 1 or self.V > L.GS_MAX_VIEWS:
            raise ValueError("1..64 views per batch")
        self.wh = wh
        self.cams = cams.to(device).contiguous()
        self._views = (L.gs_view * self.V)(*[L.gs_view(int(w), int(h)) for w, h in wh])
        lib = L.load()
        self.total_tiles = int(lib.gs_total_tiles(self._views, self.V))
        self.total_pixels = int(lib.gs_total_pixels(self._views, self.V))
        self.pix_base = np.concatenate([[0], np.cumsum(wh[:, 0].astype(np.int64) * wh[:, 1])])

    @property
    def ptr(self):
        return self._views

    def set_cams(self, cams):
        self.cams.copy_(torch.as_tensor(np.asarray(cams, np.float32)).reshape(-1, 16))

    def image_of(self, flat, v):
        w, h = (int(x) for x in self.wh[v])
        b = int(self.pix_base[v]) * 3
        return flat[b:b + 3 * w * h].view(3, h, w)


@dataclass
class Anchors:
    xyz: torch.Tensor
    feat: torch.Tensor
    log_scaling: torch.Tensor
    offsets: torch.Tensor
    part: torch.Tensor
    mlp: torch.Tensor
    F: int
    k: int
    hidden: int
    M: int

    @property
    def N(self):
        return int(self.xyz.shape[0])

    @staticmethod
    def from_scene(scene, device="cuda"):
        t = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a)).to(device, dt).contiguous()
        return Anchors(t(scene.xyz), t(scene.feat), t(scene.log_scaling), t(scene.offsets),
                       t(scene.part, torch.int32), t(scene.mlp), scene.F, scene.k, scene.hidden,
                       scene.M)

    def struct(self):
        return L.gs_anchors(self.N, self.F, self.k, self.hidden, self.M, self.xyz.data_ptr(),
                            self.feat.data_ptr(), self.log_scaling.data_ptr(),
                            self.offsets.data_ptr(), self.part.data_ptr(), self.mlp.data_ptr())


@dataclass
class Gauss3D:
    k: int
    cap_rows: int
    row_anchor: torch.Tensor | None
    view_start: torch.Tensor
    mu: torch.Tensor
    scale: torch.Tensor
    quat: torch.Tensor
    opacity: torch.Tensor
    colour: torch.Tensor

    @staticmethod
    def alloc(cap_rows, k, V, device="cuda"):
        C_ = max(cap_rows * k, 1)
        z = lambda *s: torch.zeros(*s, device=device, dtype=torch.float32)
        return Gauss3D(k, cap_rows, torch.zeros(max(cap_rows, 1), device=device, dtype=torch.int32),
                       torch.zeros(V + 1, device=device, dtype=torch.int32), z(C_, 3), z(C_, 3),
                       z(C_, 4), z(C_), z(C_, 3))

    @staticmethod
    def explicit(mu, scale, quat, opacity, colour, device="cuda"):
        t = lambda a: torch.as_tensor(np.ascontiguousarray(a, np.float32)).to(device).contiguous()
        G = int(np.asarray(mu).shape[0])
        vs = torch.tensor([0, G], device=device, dtype=torch.int32)
        return Gauss3D(1, G, None, vs, t(mu), t(scale), t(quat), t(opacity), t(colour))

    def struct(self):
        return L.gs_gauss3d(self.k, self.cap_rows,
                            self.row_anchor.data_ptr() if self.row_anchor is not None else None,
                            self.view_start.data_ptr(), self.mu.data_ptr(), self.scale.data_ptr(),
                            self.quat.data_ptr(), self.opacity.data_ptr(), self.colour.data_ptr())


@dataclass
class Gauss3DGrad:
    dmu: torch.Tensor
    dscale: torch.Tensor
    dquat: torch.Tensor
    dopacity: torch.Tensor
    dcolour: torch.Tensor

    @staticmethod
    def like(g: Gauss3D):
        return Gauss3DGrad(torch.empty_like(g.mu), torch.empty_like(g.scale), torch.empty_like(g.quat),
                           torch.empty_like(g.opacity), torch.empty_like(g.colour))

    def struct(self):
        return L.gs_gauss3d_grad(self.dmu.data_ptr(), self.dscale.data_ptr(), self.dquat.data_ptr(),
                                 self.dopacity.data_ptr(), self.dcolour.data_ptr())


@dataclass
class Splats:
    rec: torch.Tensor     # [C, 12] float32 (48-byte records)
    tiles: torch.Tensor   # [C] int32

    @staticmethod
    def alloc(cap_cand, device="cuda"):
        return Splats(torch.zeros(max(cap_cand, 1), 12, device=device, dtype=torch.float32),
                      torch.zeros(max(cap_cand, 1), device=device, dtype=torch.int32))

    def struct(self):
        return L.gs_splats(int(self.rec.shape[0]), self.rec.data_ptr(), self.tiles.data_ptr())


@dataclass
class Bins:
    cap_pairs: int
    vals: torch.Tensor     # int32 storage of uint32 ids
    keys: torch.Tensor | None
    ranges: torch.Tensor   # [T, 2] int32 storage of uint32
    n_pairs: torch.Tensor  # [1] int32

    @staticmethod
    def alloc(cap_pairs, total_tiles, device="cuda", keys=False):
        return Bins(cap_pairs, torch.zeros(max(cap_pairs, 1), device=device, dtype=torch.int32),
                    torch.zeros(max(cap_pairs, 1), device=device, dtype=torch.int64) if keys else None,
                    torch.zeros(max(total_tiles, 1), 2, device=device, dtype=torch.int32),
                    torch.zeros(1, device=device, dtype=torch.int32))

    def struct(self):
        return L.gs_bins(self.cap_pairs, self.vals.data_ptr(),
                         self.keys.data_ptr() if self.keys is not None else None,
                         self.ranges.data_ptr(), self.n_pairs.data_ptr())


@dataclass
class AnchorGrad:
    dxyz: torch.Tensor
    dfeat: torch.Tensor
    dlog_scaling: torch.Tensor
    doffsets: torch.Tensor
    dmlp: torch.Tensor

    @staticmethod
    def like(a: Anchors):
        return AnchorGrad(torch.empty_like(a.xyz), torch.empty_like(a.feat),
                          torch.empty_like(a.log_scaling), torch.empty_like(a.offsets),
                          torch.empty_like(a.mlp))

    def struct(self):
        return L.gs_anchor_grad(self.dxyz.data_ptr(), self.dfeat.data_ptr(),
                                self.dlog_scaling.data_ptr(), self.doffsets.data_ptr(),
                                self.dmlp.data_ptr())


def new_status(device="cuda"):
    return torch.zeros(2, dtype=torch.int64, device=device)


TUNING_FIELDS = ("fwd_ctas_per_sm", "bwd_ctas_per_sm", "sort_ctas_per_sm", "emit_ctas_per_sm")


def set_tuning(tuning: dict | None):
    """Launch shapes for later calls (gs_set_tuning); None or {} restores the
    library's defaults, missing keys are 0 (the library's choice)."""
    lib = L.load()
    if not tuning:
        L.check("gs_set_tuning", lib.gs_set_tuning(None))
        return
    unknown = set(tuning) - set(TUNING_FIELDS)
    if unknown:
        raise ValueError(f"unknown tuning keys {sorted(unknown)}")
    t = L.gs_tuning(*(int(tuning.get(k, 0)) for k in TUNING_FIELDS))
    L.check("gs_set_tuning", lib.gs_set_tuning(C.byref(t)))


def get_tuning() -> dict:
    t = L.gs_tuning()
    L.check("gs_get_tuning", L.load().gs_get_tuning(C.byref(t)))
    return {k: int(getattr(t, k)) for k in TUNING_FIELDS}


def set_wait_limit(ns: int | None):
    """Limit (ns) of the tensor-core kernels' MMA completion waits for later
    calls; None restores the default (1 s), 0 gives up at the first wait."""
    L.check("gs_set_wait_limit", L.load().gs_set_wait_limit(-1 if ns is None else int(ns)))


def read_status(status):
    s = status.cpu().numpy()
    code = int(np.int32(s[0] & 0xFFFFFFFF))
    where = int(np.int32((s[0] >> 32) & 0xFFFFFFFF))
    return code, where, int(s[1])


def workspace(nbytes, device="cuda"):
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


# ---------------------------------------------------------------- the calls
def decode(anchors: Anchors, views: Views, out: Gauss3D, ws, status, precision=L.GS_PREC_FP32,
           stream=None):
    lib = L.load()
    a, g = anchors.struct(), out.struct()
    L.check("gs_decode", lib.gs_decode(C.byref(a), _ptr(views.cams), views.ptr, views.V, precision,
                                       C.byref(g), _ptr(ws), ws.numel(), _ptr(status),
                                       _stream(stream)))


def decode_noalloc(anchors: Anchors, views: Views, out: Gauss3D, status, precision=L.GS_PREC_FP32,
                   stream=None):
    """gs_decode without a workspace (scratch in a static device array)."""
    lib = L.load()
    a, g = anchors.struct(), out.struct()
    L.check("gs_decode_noalloc", lib.gs_decode_noalloc(C.byref(a), _ptr(views.cams), views.ptr, views.V,
                                                       precision, C.byref(g), _ptr(status),
                                                       _stream(stream)))


def decode_workspace(anchors: Anchors, views: Views, cap_rows):
    return int(L.load().gs_decode_workspace(anchors.N, views.V, anchors.M, cap_rows))


def decode_project(anchors: Anchors, views: Views, g: Gauss3D, sp: Splats, ws, status, precision=L.GS_PREC_FP32,
                   stream=None):
    """Visible rows, decoding and projection in one call (the tensor-core
    path writes the splat records straight from the decoder)."""
    lib = L.load()
    a, gs_, s = anchors.struct(), g.struct(), sp.struct()
    L.check("gs_decode_project", lib.gs_decode_project(C.byref(a), _ptr(views.cams), views.ptr, views.V, precision,
                                                       C.byref(gs_), C.byref(s), _ptr(ws), ws.numel(), _ptr(status),
                                                       _stream(stream)))


def project(g: Gauss3D, views: Views, out: Splats, status, stream=None):
    lib = L.load()
    gs, sp = g.struct(), out.struct()
    L.check("gs_project", lib.gs_project(C.byref(gs), _ptr(views.cams), views.ptr, views.V,
                                         C.byref(sp), _ptr(status), _stream(stream)))


def bin_sort_workspace(views: Views, cap_cand, cap_pairs):
    return int(L.load().gs_bin_sort_workspace(views.ptr, views.V, cap_cand, cap_pairs))


def bin_sort(sp: Splats, g: Gauss3D, views: Views, bins: Bins, ws, status, stream=None):
    lib = L.load()
    s, b = sp.struct(), bins.struct()
    L.check("gs_bin_sort", lib.gs_bin_sort(C.byref(s), g.k, _ptr(g.view_start), g.cap_rows,
                                           views.ptr, views.V, C.byref(b), _ptr(ws), ws.numel(),
                                           _ptr(status), _stream(stream)))


def _bg(bg):
    return (C.c_float * 3)(*[float(x) for x in bg])


def render_workspace(views: Views, cap_pairs, chunk=0):
    return int(L.load().gs_render_workspace(views.ptr, views.V, cap_pairs, chunk))


def render_fwd(sp: Splats, bins: Bins, views: Views, bg, image, status, ws, chunk=0, T_final=None,
               last=None, n_eval=None, stream=None):
    lib = L.load()
    s, b = sp.struct(), bins.struct()
    L.check("gs_render_fwd", lib.gs_render_fwd(C.byref(s), C.byref(b), views.ptr, views.V, _bg(bg), chunk,
                                               _ptr(ws), ws.numel(), _ptr(image), _ptr(T_final),
                                               _ptr(last), _ptr(n_eval), _ptr(status), _stream(stream)))


def l1_loss(image, target, views: Views, loss, d_image, stream=None):
    lib = L.load()
    L.check("gs_l1_loss", lib.gs_l1_loss(_ptr(image), _ptr(target), views.ptr, views.V, _ptr(loss),
                                         _ptr(d_image), _stream(stream)))


def photometric_workspace(views: Views):
    return int(L.load().gs_photometric_workspace(views.ptr, views.V))


def photometric_loss(image, target, views: Views, lam, ws, loss, d_image, stream=None):
    """Eq. 3: loss[0:3] = (lam L1 + (1 - lam) L_SSIM, L1, L_SSIM); d_image = dL/dimage."""
    lib = L.load()
    L.check("gs_photometric_loss", lib.gs_photometric_loss(_ptr(image), _ptr(target), views.ptr, views.V,
                                                           float(lam), _ptr(ws), ws.numel(), _ptr(loss),
                                                           _ptr(d_image), _stream(stream)))


def adam_step(groups, step, beta1=0.9, beta2=0.999, eps=1e-15, stream=None):
    """One Adam step over `groups` = [(param, grad, m, v, lr), ...] (contiguous
    float32 device tensors, updated in place), one launch."""
    lib = L.load()
    arr = (L.gs_adam_group * len(groups))(*[
        L.gs_adam_group(_ptr(p), _ptr(g), _ptr(m), _ptr(v), int(p.numel()), float(lr))
        for p, g, m, v, lr in groups])
    L.check("gs_adam_step", lib.gs_adam_step(arr, len(groups), int(step), float(beta1), float(beta2),
                                             float(eps), _stream(stream)))


def densify_stats(g: Gauss3D, views: Views, sp: Splats, sgrad, N, grad_accum, offset_denom, opacity_accum,
                  anchor_denom, status, stream=None):
    lib = L.load()
    gs_ = g.struct()
    L.check("gs_densify_stats", lib.gs_densify_stats(C.byref(gs_), views.V, _ptr(sp.tiles), _ptr(sgrad), int(N),
                                                     _ptr(grad_accum), _ptr(offset_denom), _ptr(opacity_accum),
                                                     _ptr(anchor_denom), _ptr(status), _stream(stream)))


def densify_masks(k, grad_accum, offset_denom, opacity_accum, anchor_denom, grad_thr, opacity_thr, min_count,
                  grow, prune, stream=None):
    lib = L.load()
    N = int(opacity_accum.numel())
    L.check("gs_densify_masks", lib.gs_densify_masks(N, int(k), _ptr(grad_accum), _ptr(offset_denom),
                                                     _ptr(opacity_accum), _ptr(anchor_denom), float(grad_thr),
                                                     float(opacity_thr), int(min_count), _ptr(grow), _ptr(prune),
                                                     _stream(stream)))


def voxelize_workspace(P):
    return int(L.load().gs_voxelize_workspace(int(P)))


def voxelize(points, eps, keys_out, centers_out, n_out, ws, status, existing=None, stream=None):
    """Eq. 4 on device points [P, 3] float32: new voxel keys (ascending, int64
    tensor holding the uint64 keys) and centres; n_out: uint32[1] count."""
    lib = L.load()
    P = int(points.shape[0]) if points.dim() > 1 else int(points.numel()) // 3
    ne = 0 if existing is None else int(existing.numel())
    L.check("gs_voxelize", lib.gs_voxelize(_ptr(points), P, float(eps), _ptr(existing) if ne else None, ne,
                                           _ptr(keys_out), _ptr(centers_out), int(keys_out.numel()), _ptr(n_out),
                                           _ptr(ws), ws.numel(), _ptr(status), _stream(stream)))


def loop_closure(xyz, old_cams, new_cams, wh, z_far, assigned=None, stream=None):
    """Eq. 7: moves the anchors xyz [N, 3] (device, in place) by the pose
    updates of the keyframes (old_cams / new_cams: device [K, 16] float32;
    wh: device int32 [K, 2]); assigned: optional int32 [N] (-1: none)."""
    lib = L.load()
    L.check("gs_loop_closure", lib.gs_loop_closure(_ptr(xyz), int(xyz.shape[0]), _ptr(old_cams), _ptr(new_cams),
                                                   _ptr(wh), int(old_cams.shape[0]), float(z_far),
                                                   _ptr(assigned), _stream(stream)))


def flow_workspace(N):
    return int(L.load().gs_flow_workspace(int(N)))


def flow_triangulate(cams, wh, flow, samples, tau, kept, points, n_kept, ws, status, residual=None, stream=None):
    """Eq. 5 filtering and triangulation: cams device [2, 16] float32
    (keyframes 1, 2), flow device [H, W, 2], samples device int32 [N]."""
    lib = L.load()
    c1 = C.c_void_p(cams.data_ptr())
    c2 = C.c_void_p(cams.data_ptr() + 64)
    L.check("gs_flow_triangulate", lib.gs_flow_triangulate(c1, c2, int(wh[0]), int(wh[1]), _ptr(flow), _ptr(samples),
                                                           int(samples.numel()), float(tau), _ptr(residual),
                                                           _ptr(kept), _ptr(points), int(kept.numel()),
                                                           _ptr(n_kept), _ptr(ws), ws.numel(), _ptr(status),
                                                           _stream(stream)))


def splat_grad_alloc(g: Gauss3D, layout=L.GS_SGRAD_CANDIDATE, device="cuda"):
    """Splat-gradient buffer for g's capacity: [C][9] candidate-major, or in
    row tiles of 128 (GS_SGRAD_ROW_TILES: the whole last tile)."""
    rows = g.cap_rows if layout == L.GS_SGRAD_CANDIDATE else (g.cap_rows + 127) // 128 * 128
    return torch.zeros(max(rows * g.k, 1), 9, device=device)


def render_bwd(g: Gauss3D, sp: Splats, bins: Bins, views: Views, image, d_image, sgrad, out: Gauss3DGrad,
               status, ws, chunk=0, last=None, stream=None, sgrad_layout=L.GS_SGRAD_CANDIDATE):
    """Reverse of the compositing and (unless out is None) of the projection.
    image: the forward's output; last: its optional per-pixel last
    composited position; sgrad_layout: GS_SGRAD_* of sgrad."""
    lib = L.load()
    gs_, s, b = g.struct(), sp.struct(), bins.struct()
    sg = L.gs_splat_grad(sgrad.data_ptr(), sgrad_layout)
    o = C.byref(out.struct()) if out is not None else None
    L.check("gs_render_bwd", lib.gs_render_bwd(C.byref(gs_), _ptr(views.cams), C.byref(s), C.byref(b),
                                               views.ptr, views.V, chunk, _ptr(ws), ws.numel(), _ptr(image),
                                               _ptr(d_image), _ptr(last), C.byref(sg), o,
                                               _ptr(status), _stream(stream)))


def project_bwd(g: Gauss3D, sp: Splats, views: Views, sgrad, out: Gauss3DGrad, status, stream=None):
    """Chain rule of the projection from the splat gradients of render_bwd."""
    lib = L.load()
    gs_, s = g.struct(), sp.struct()
    sg = L.gs_splat_grad(sgrad.data_ptr())
    o = out.struct()
    L.check("gs_project_bwd", lib.gs_project_bwd(C.byref(gs_), _ptr(views.cams), C.byref(s), views.ptr, views.V,
                                                 C.byref(sg), C.byref(o), _ptr(status), _stream(stream)))


def decode_project_bwd_workspace(g: Gauss3D, precision=L.GS_PREC_FP32):
    return int(L.load().gs_decode_project_bwd_workspace(g.k, g.cap_rows, precision))


def decode_project_bwd(anchors: Anchors, views: Views, g: Gauss3D, sp: Splats, sgrad, out: AnchorGrad, ws,
                       status, precision=L.GS_PREC_FP32, stream=None, sgrad_layout=L.GS_SGRAD_CANDIDATE):
    """Reverse of the projection and the decoders from render_bwd's splat
    gradients (tensor-core path fused; FP32 path through ws).  Row-tiled
    splat gradients (tensor-core path only) need no workspace."""
    lib = L.load()
    a, gs_, s = anchors.struct(), g.struct(), sp.struct()
    sg = L.gs_splat_grad(sgrad.data_ptr(), sgrad_layout)
    o = out.struct()
    L.check("gs_decode_project_bwd", lib.gs_decode_project_bwd(C.byref(a), _ptr(views.cams), views.ptr, views.V,
                                                               precision, C.byref(gs_), C.byref(s), C.byref(sg),
                                                               C.byref(o), _ptr(ws), 0 if ws is None else ws.numel(),
                                                               _ptr(status), _stream(stream)))


def decode_bwd_workspace(anchors: Anchors, views: Views, cap_rows):
    return int(L.load().gs_decode_bwd_workspace(anchors.N, views.V, anchors.M, cap_rows))


def decode_bwd(anchors: Anchors, views: Views, g: Gauss3D, dg: Gauss3DGrad, out: AnchorGrad, ws,
               status, precision=L.GS_PREC_FP32, stream=None):
    lib = L.load()
    a, gs_, d, o = anchors.struct(), g.struct(), dg.struct(), out.struct()
    L.check("gs_decode_bwd", lib.gs_decode_bwd(C.byref(a), _ptr(views.cams), views.ptr, views.V,
                                               precision, C.byref(gs_), C.byref(d), C.byref(o),
                                               _ptr(ws), ws.numel(), _ptr(status), _stream(stream)))


def probe_peak(kind: int, blocks: int | None = None, iters: int = 4096, device="cuda"):
    """Issue rate of FP32 fused multiply-adds (kind 0) or SFU ex2 (kind 1) on
    the current device, in operations per second (measurement helper)."""
    if blocks is None:
        blocks = torch.cuda.get_device_properties(device).multi_processor_count * 8
    sink = torch.zeros(blocks, device=device)
    ops = C.c_int64(0)
    lib = L.load()
    for _ in range(2):   # warm-up launch, then the timed one
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        L.check("gs_probe_peak", lib.gs_probe_peak(kind, blocks, iters, _ptr(sink), C.byref(ops), _stream()))
        e1.record()
        torch.cuda.synchronize()
    return ops.value / (e0.elapsed_time(e1) * 1e-3)
