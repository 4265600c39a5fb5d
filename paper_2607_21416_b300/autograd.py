"""PyTorch autograd front end of libgs.

`decode`, `render` and `l1_loss` are differentiable functions whose forward
and backward passes run in libgs kernels:

    g = decode(anchors..., views)            # GsDecode: a0 visibility + a1 decoding (Eq. 2, Eq. 6)
    image = render(g, views)                 # GsRender: a2 projection, a3 binning, a4 compositing (Eq. 1)
    loss = l1_loss(image, target, views)     # GsL1: Eq. 3, L1 term
    (or photometric_loss(image, target, views, lam=0.8): all of Eq. 3)
    loss.backward()                          # a6 render backward (with the projection), a7 decode backward

They run eagerly and synchronise with the host once per call to check the
status word (and to grow the pair buffers on a capacity overflow), so they
suit training loops written in PyTorch; the graph-captured batched iteration
is `pipeline.MappingStep`.  Rows of a decoded batch are in view-major anchor
order; rows past the batch's row count (g.view_start[-1]) are zero and get no
gradient.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import torch

from . import _lib as L
from . import api


def _check(status, call):
    code, where, needed = api.read_status(status)
    if code != L.GS_OK:
        raise L.GsError(f"{call} (stage {where}, needed {needed})", code)


@dataclass
class Decoded:
    """Differentiable decoded Gaussians of a keyframe batch (capacity N x V rows)."""
    mu: torch.Tensor
    scale: torch.Tensor
    quat: torch.Tensor
    opacity: torch.Tensor
    colour: torch.Tensor
    row_anchor: torch.Tensor | None
    view_start: torch.Tensor
    k: int


class GsDecode(torch.autograd.Function):
    @staticmethod
    def forward(ctx, xyz, feat, log_scaling, offsets, mlp, part, views, k, hidden, M, precision):
        A = api.Anchors(xyz.detach().contiguous(), feat.detach().contiguous(), log_scaling.detach().contiguous(),
                        offsets.detach().contiguous(), part.contiguous(), mlp.detach().contiguous(),
                        int(feat.shape[1]), k, hidden, M)
        cap = max(A.N * views.V, 1)   # every (anchor, view) row fits: no capacity overflow
        g = api.Gauss3D.alloc(cap, k, views.V, xyz.device)
        st = api.new_status(xyz.device)
        ws = api.workspace(api.decode_workspace(A, views, cap), xyz.device)
        api.decode(A, views, g, ws, st, precision)
        _check(st, "gs_decode")
        ctx.A, ctx.g, ctx.views, ctx.precision = A, g, views, precision
        ctx.mark_non_differentiable(g.row_anchor, g.view_start)
        return g.mu, g.scale, g.quat, g.opacity, g.colour, g.row_anchor, g.view_start

    @staticmethod
    def backward(ctx, dmu, dscale, dquat, dopacity, dcolour, _ra, _vs):
        A, g, views = ctx.A, ctx.g, ctx.views
        z = lambda d, like: (d if d is not None else torch.zeros_like(like)).contiguous()
        dg = api.Gauss3DGrad(z(dmu, g.mu), z(dscale, g.scale), z(dquat, g.quat), z(dopacity, g.opacity),
                             z(dcolour, g.colour))
        out = api.AnchorGrad.like(A)
        st = api.new_status(g.mu.device)
        ws = api.workspace(api.decode_bwd_workspace(A, views, g.cap_rows), g.mu.device)
        api.decode_bwd(A, views, g, dg, out, ws, st, ctx.precision)
        _check(st, "gs_decode_bwd")
        return out.dxyz, out.dfeat, out.dlog_scaling, out.doffsets, out.dmlp, None, None, None, None, None, None


def decode(xyz, feat, log_scaling, offsets, mlp, part, views: api.Views, k: int, hidden: int, M: int,
           precision: int = L.GS_PREC_FP32) -> Decoded:
    """Anchor visibility and decoding of every visible (anchor, view) row."""
    mu, scale, quat, opacity, colour, ra, vs = GsDecode.apply(xyz, feat, log_scaling, offsets, mlp, part, views, k,
                                                             hidden, M, precision)
    return Decoded(mu, scale, quat, opacity, colour, ra, vs, k)


class Renderer:
    """Pair-buffer capacity shared by successive `render` calls (grown on
    overflow); every call allocates its own buffers, so several forward
    passes may be alive before their backward passes."""

    def __init__(self, chunk: int = 0, pairs_per_candidate: float = 4.0):
        self.chunk = int(chunk)
        self.ppc = float(pairs_per_candidate)
        self.cap_pairs = 0


class GsRender(torch.autograd.Function):
    @staticmethod
    def forward(ctx, mu, scale, quat, opacity, colour, k, row_anchor, view_start, views, bg, renderer):
        dev = mu.device
        C_ = int(mu.shape[0])
        g = api.Gauss3D(k, C_ // k, row_anchor, view_start, mu.detach().contiguous(), scale.detach().contiguous(),
                        quat.detach().contiguous(), opacity.detach().contiguous(), colour.detach().contiguous())
        sp = api.Splats.alloc(C_, dev)
        st = api.new_status(dev)
        api.project(g, views, sp, st)
        _check(st, "gs_project")   # before the retries below reset the status word
        cap = max(renderer.cap_pairs, int(renderer.ppc * C_), 1024)
        for _ in range(4):
            bins = api.Bins.alloc(cap, views.total_tiles, dev)
            st.zero_()
            api.bin_sort(sp, g, views, bins, api.workspace(api.bin_sort_workspace(views, C_, cap), dev), st)
            code, where, needed = api.read_status(st)
            if code != L.GS_ERR_CAPACITY:
                break
            cap = int(math.ceil(needed * 1.15)) + 1024
        _check(st, "gs_bin_sort")
        renderer.cap_pairs = max(renderer.cap_pairs, cap)
        npix = views.total_pixels
        image = torch.zeros(3 * npix, device=dev)
        T_final = torch.zeros(npix, device=dev)
        last = torch.zeros(npix, device=dev, dtype=torch.int32)
        ws = api.workspace(api.render_workspace(views, cap, renderer.chunk), dev)
        api.render_fwd(sp, bins, views, bg, image, st, ws, renderer.chunk, T_final, last)
        _check(st, "gs_render_fwd")
        ctx.state = (g, sp, bins, ws, image, last, views, renderer.chunk)
        return image

    @staticmethod
    def backward(ctx, d_image):
        g, sp, bins, ws, image, last, views, chunk = ctx.state
        dev = g.mu.device
        sgrad = torch.zeros(max(g.mu.shape[0], 1), 9, device=dev)
        out = api.Gauss3DGrad.like(g)
        st = api.new_status(dev)
        api.render_bwd(g, sp, bins, views, image, d_image.contiguous(), sgrad, out, st, ws, chunk, last)
        _check(st, "gs_render_bwd")
        return out.dmu, out.dscale, out.dquat, out.dopacity, out.dcolour, None, None, None, None, None, None


def render(g: Decoded, views: api.Views, bg=(0.0, 0.0, 0.0), renderer: Renderer | None = None) -> torch.Tensor:
    """Composited images of all views, planar [3, H, W] per view, concatenated."""
    r = renderer if renderer is not None else Renderer()
    return GsRender.apply(g.mu, g.scale, g.quat, g.opacity, g.colour, g.k, g.row_anchor, g.view_start, views,
                          tuple(float(x) for x in bg), r)


def explicit(mu, scale, quat, opacity, colour) -> Decoded:
    """Explicit Gaussians (one view batch, k = 1) as renderable input."""
    G = int(mu.shape[0])
    vs = torch.tensor([0, G], device=mu.device, dtype=torch.int32)
    return Decoded(mu, scale, quat, opacity, colour, None, vs, 1)


class GsL1(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image, target, views):
        loss = torch.zeros(1, device=image.device)
        d_image = torch.zeros_like(image)
        api.l1_loss(image.detach().contiguous(), target.contiguous(), views, loss, d_image)
        ctx.save_for_backward(d_image)
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        (d_image,) = ctx.saved_tensors
        return d_image * grad, None, None


def l1_loss(image, target, views: api.Views) -> torch.Tensor:
    """Sum over views of the per-view mean absolute error (Eq. 3, L1 term)."""
    return GsL1.apply(image, target, views)


class GsPhotometric(torch.autograd.Function):
    @staticmethod
    def forward(ctx, image, target, views, lam):
        loss = torch.zeros(3, device=image.device)
        d_image = torch.zeros_like(image)
        ws = api.workspace(api.photometric_workspace(views), image.device)
        api.photometric_loss(image.detach().contiguous(), target.contiguous(), views, lam, ws, loss, d_image)
        ctx.save_for_backward(d_image)
        return loss[0]

    @staticmethod
    def backward(ctx, grad):
        (d_image,) = ctx.saved_tensors
        return d_image * grad, None, None, None


def photometric_loss(image, target, views: api.Views, lam: float = 0.8) -> torch.Tensor:
    """Eq. 3: lam L1 + (1 - lam)(1 - SSIM), each a per-view mean summed over views."""
    return GsPhotometric.apply(image, target, views, float(lam))
