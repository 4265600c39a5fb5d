"""One mapping iteration of the rendering path, built from the libgs calls.

`RenderPass` owns capacity-sized device buffers for a keyframe batch and runs
decode -> project -> bin/sort -> render -> loss (L1 term of Eq. 3, or all of
Eq. 3 with its SSIM term) -> render backward -> decode
backward on one CUDA stream with no host synchronisation in between, so the
whole sequence can be captured into one CUDA graph.  Capacity overflow is
detected on the device (status word) and handled by `ensure_capacity`, which
grows the buffers outside any capture.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

from . import _lib as L
from . import api


@dataclass
class PassOutputs:
    image: torch.Tensor
    loss: torch.Tensor
    d_image: torch.Tensor


class RenderPass:
    """Buffers + call sequence for one keyframe batch.

    anchors: api.Anchors or None (explicit Gaussians passed to `set_explicit`).
    store_state: keep the forward's per-pixel T_final / last contributor for
    the backward (plain path), or let the backward decide the stop rule again
    on its front-to-back walk (batched path: nothing per pixel is stored).
    fuse_projection: decode and project in one call (gs_decode_project); with
    BF16 decoding the 3D Gaussians then never reach device memory (g's
    candidate arrays stay unwritten) -- turn it off when the decoded
    Gaussians themselves are needed (densification statistics).
    """

    def __init__(self, views: api.Views, anchors: api.Anchors | None = None, k: int = 1,
                 cap_rows: int | None = None, cap_pairs: int | None = None,
                 precision: int = L.GS_PREC_FP32, store_state: bool = True,
                 bg=(0.0, 0.0, 0.0), device="cuda", keys=False, chunk=0, loss="l1", lam=0.8,
                 fuse_projection=True):
        self.views = views
        self.anchors = anchors
        self.k = anchors.k if anchors is not None else k
        self.precision = precision
        self.store_state = store_state
        self.bg = tuple(float(x) for x in bg)
        self.device = device
        self.want_keys = keys
        self.chunk = int(chunk)
        self.fuse_projection = bool(fuse_projection)
        if loss not in ("l1", "photometric"):
            raise ValueError(f"loss must be 'l1' or 'photometric', not {loss!r}")
        self.loss_kind = loss
        self.lam = float(lam)
        V = views.V
        if cap_rows is None:
            cap_rows = (anchors.N * V) if anchors is not None else 1
        self.cap_rows = int(cap_rows)
        self.cap_pairs = int(cap_pairs) if cap_pairs is not None else max(4 * self.cap_rows * self.k, 1024)
        self.status = api.new_status(device)
        npix = views.total_pixels
        self.image = torch.zeros(3 * npix, device=device)
        self.d_image = torch.zeros(3 * npix, device=device)
        # l1: [L1]; photometric: [lam L1 + (1 - lam) L_SSIM, L1, L_SSIM]
        self.loss = torch.zeros(1 if loss == "l1" else 3, device=device)
        self.photo_ws = (api.workspace(api.photometric_workspace(views), device) if loss == "photometric"
                         else None)
        self.T_final = torch.zeros(npix, device=device) if store_state else None
        self.last = torch.zeros(npix, device=device, dtype=torch.int32) if store_state else None
        self.n_eval = torch.zeros(4, device=device, dtype=torch.int64)
        self._alloc()

    def _alloc(self):
        dev, V = self.device, self.views.V
        C_ = self.cap_rows * self.k
        if self.anchors is not None:
            self.g = api.Gauss3D.alloc(self.cap_rows, self.k, V, dev)
            self.dec_ws = api.workspace(api.decode_workspace(self.anchors, self.views, self.cap_rows), dev)
            self.agrad = api.AnchorGrad.like(self.anchors)
            self.dbwd_ws = api.workspace(api.decode_bwd_workspace(self.anchors, self.views, self.cap_rows), dev)
            self.dpbwd_ws = api.workspace(api.decode_project_bwd_workspace(self.g, self.precision), dev)
        self.splats = api.Splats.alloc(C_, dev)
        self.bins = api.Bins.alloc(self.cap_pairs, self.views.total_tiles, dev, keys=self.want_keys)
        self.sort_ws = api.workspace(api.bin_sort_workspace(self.views, C_, self.cap_pairs), dev)
        self.render_ws = api.workspace(api.render_workspace(self.views, self.cap_pairs, self.chunk), dev)
        # the fused tensor-core reverse reads the splat gradients in row tiles, written so by render_bwd
        self.sgrad_layout = (L.GS_SGRAD_ROW_TILES if self.anchors is not None and not self.gaussians_written
                             else L.GS_SGRAD_CANDIDATE)
        rows = self.cap_rows if self.sgrad_layout == L.GS_SGRAD_CANDIDATE else (self.cap_rows + 127) // 128 * 128
        self.sgrad = torch.zeros(max(rows * self.k, 1), 9, device=dev)
        self.ggrad = None

    def set_explicit(self, g: api.Gauss3D):
        """Use explicit Gaussians (k = 1) instead of decoding anchors."""
        if g.cap_rows * g.k > self.cap_rows * self.k:
            self.cap_rows = g.cap_rows
            self.k = g.k
            self._alloc()
        self.g = g

    @property
    def gaussians_written(self) -> bool:
        """Whether the forward leaves the decoded 3D Gaussians in g."""
        return self.anchors is None or not self.fuse_projection or self.precision != L.GS_PREC_BF16

    # ---------------------------------------------------------------- passes
    def forward(self, count_evals=False, stream=None):
        """decode + project (one call: with BF16 decoding the decoder writes the
        splat records itself and g's candidate arrays are not written), then
        bin/sort and composite."""
        self.status.zero_()
        if self.anchors is not None and self.fuse_projection:
            api.decode_project(self.anchors, self.views, self.g, self.splats, self.dec_ws, self.status,
                               self.precision, stream)
        else:
            if self.anchors is not None:
                api.decode(self.anchors, self.views, self.g, self.dec_ws, self.status, self.precision, stream)
            api.project(self.g, self.views, self.splats, self.status, stream)
        api.bin_sort(self.splats, self.g, self.views, self.bins, self.sort_ws, self.status, stream)
        api.render_fwd(self.splats, self.bins, self.views, self.bg, self.image, self.status,
                       self.render_ws, self.chunk,
                       self.T_final if self.store_state else None,
                       self.last if self.store_state else None,
                       self.n_eval if count_evals else None, stream)
        return self.image

    def loss_l1(self, target, stream=None):
        """The configured loss of Eq. 3 (its L1 term, or all of it) and dL/dimage."""
        if self.loss_kind == "l1":
            api.l1_loss(self.image, target, self.views, self.loss, self.d_image, stream)
        else:
            api.photometric_loss(self.image, target, self.views, self.lam, self.photo_ws, self.loss,
                                 self.d_image, stream)
        return self.loss

    def backward(self, d_image=None, stream=None):
        """Reverse of the iteration: the compositing's (splat gradients), then
        for anchors the projection's and the decoders' in one call (fused on
        the tensor-core path), for explicit Gaussians the projection's."""
        dimg = self.d_image if d_image is None else d_image
        last = self.last if self.store_state else None
        if self.anchors is not None:
            api.render_bwd(self.g, self.splats, self.bins, self.views, self.image, dimg, self.sgrad, None,
                           self.status, self.render_ws, self.chunk, last, stream, self.sgrad_layout)
            api.decode_project_bwd(self.anchors, self.views, self.g, self.splats, self.sgrad, self.agrad,
                                   self.dpbwd_ws, self.status, self.precision, stream, self.sgrad_layout)
            return self.agrad
        if self.ggrad is None or self.ggrad.dmu.shape[0] != self.g.mu.shape[0]:
            self.ggrad = api.Gauss3DGrad.like(self.g)
        api.render_bwd(self.g, self.splats, self.bins, self.views, self.image, dimg, self.sgrad, self.ggrad,
                       self.status, self.render_ws, self.chunk, last, stream)
        return self.ggrad

    def step(self, target, stream=None):
        """forward + loss + backward (one mapping iteration without the optimizer)."""
        self.forward(stream=stream)
        self.loss_l1(target, stream)
        self.backward(stream=stream)
        return self.loss

    # ------------------------------------------------------------ capacity
    def check(self):
        code, where, needed = api.read_status(self.status)
        return code, where, needed

    def ensure_capacity(self, target=None, max_tries=4):
        """Runs one pass and grows the buffers until no capacity error is left
        (outside of any graph capture).  Returns the final status code."""
        for _ in range(max_tries):
            self.forward()
            if target is not None:
                self.loss_l1(target)
                self.backward()
            torch.cuda.synchronize()
            code, where, needed = self.check()
            if code == 0:
                return 0
            if code != L.GS_ERR_CAPACITY:
                raise L.GsError(f"stage {where}", code)
            if where == 1:
                self.cap_rows = int(math.ceil(needed * 1.1)) + 16
                # one pair per candidate at least; a pair overflow on the next try sizes them exactly
                self.cap_pairs = max(self.cap_pairs, self.cap_rows * self.k)
            else:
                self.cap_pairs = int(math.ceil(needed * 1.15)) + 1024
            self._alloc()
        return self.check()[0]

    def n_rows(self):
        return int(self.g.view_start[-1].item())

    def n_pairs(self):
        return int(self.bins.n_pairs.item())


class MappingStep:
    """One mapping iteration of a keyframe batch (decode -> ... -> decode
    backward, no optimizer step) captured once into a CUDA graph and replayed.

    `prepare(target)` sizes the buffers with one host-synchronised eager pass
    and captures the graph (with tune=True it first picks the chunk length
    and launch shapes with `autotune.tune`, cached in `tune_cache`, and
    captures with them); `run()` replays it on device-resident inputs;
    `step(target_host, cams_host)` is the end-to-end call: it copies the
    iteration's target images (and optionally cameras) from pinned host memory,
    replays the graph and reads back the loss and the status word (one stream
    synchronisation).  With `next_target_host`, the next iteration's images are
    copied into a second device buffer on a copy stream while this iteration
    runs (the step returns once both are done; the next step then replays the
    graph captured on that buffer), so the host-to-device copy overlaps the
    compute; the next call must pass the same tensor, unchanged.  A capacity
    overflow found there re-prepares the buffers and repeats the iteration.
    """

    def __init__(self, views: api.Views, anchors: api.Anchors, precision: int = L.GS_PREC_BF16,
                 cap_rows: int | None = None, store_state: bool = False, chunk: int = 0, device="cuda",
                 loss: str = "l1", lam: float = 0.8, tune: bool = False, tune_cache: str | None = None,
                 fuse_projection: bool = True):
        self.views = views
        self.anchors = anchors
        self._args = dict(cap_rows=cap_rows, precision=precision, store_state=store_state, device=device,
                          loss=loss, lam=lam, fuse_projection=fuse_projection)
        self.rp = RenderPass(views, anchors, chunk=chunk, **self._args)
        self.target = torch.zeros(3 * views.total_pixels, device=device)
        self._target_b = torch.zeros(3 * views.total_pixels, device=device)   # the prefetch buffer
        self.stream = torch.cuda.Stream(device=device)
        self._copy_stream = torch.cuda.Stream(device=device)
        self.graph = None
        self._graph_b = None   # the same iteration captured on the prefetch buffer
        self._pending = None   # (host tensor, buffer index, event) of a prefetched target
        self.tune = bool(tune)
        self.tune_cache = tune_cache
        self.tuned = None      # the autotuner's pick and its measurements (tune=True)
        self.tuning = None     # launch shapes the graph is captured with (None: the process-wide ones)
        self._loss_host = torch.zeros(1, dtype=torch.float32).pin_memory()
        self._status_host = torch.zeros(2, dtype=torch.int64).pin_memory()

    @property
    def h2d_bytes(self):
        return self.target.numel() * 4

    def _autotune(self):
        """Picks the chunk length and launch shapes for this batch (measured
        with CUDA events on it, or from the cache) and rebuilds the buffers
        when the chunk length changes."""
        from . import autotune
        code = self.rp.ensure_capacity(self.target)   # the batch's sizes, for the candidates' buffers
        if code != 0:
            raise L.GsError("capacity handling", code)
        cfg, info = autotune.tune(self.views, self.anchors, self.target, self._args["precision"],
                                  self._args["loss"], cache_path=self.tune_cache, cap_rows=self.rp.cap_rows,
                                  cap_pairs=self.rp.cap_pairs)
        self.tuned = dict(config=cfg, **info)
        if int(cfg["chunk"]) != self.rp.chunk:
            cap_pairs = self.rp.cap_pairs
            self._args["cap_rows"] = self.rp.cap_rows
            self.rp = RenderPass(self.views, self.anchors, chunk=int(cfg["chunk"]), **self._args)
            self.rp.cap_pairs = cap_pairs
            self.rp._alloc()
        self.tuning = {k: int(cfg[k]) for k in api.TUNING_FIELDS}

    def prepare(self, target=None):
        if target is not None:
            self.target.copy_(target)
        if self.tune and self.tuned is None:
            self._autotune()
        code = self.rp.ensure_capacity(self.target)
        if code != 0:
            raise L.GsError("capacity handling", code)
        self.recapture()

    def recapture(self):
        """Captures the iteration into a new CUDA graph with the current
        buffers (and this step's launch shapes, when tuned)."""
        prev = api.get_tuning()
        if self.tuning is not None:
            api.set_tuning(self.tuning)
        try:
            with torch.cuda.stream(self.stream):
                self.rp.step(self.target)   # kernel attributes and workspaces settle outside the capture
            torch.cuda.synchronize()
            self.graph = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self.graph, stream=self.stream):
                self.rp.step(self.target)
            self._graph_b = torch.cuda.CUDAGraph()
            with torch.cuda.graph(self._graph_b, stream=self.stream):
                self.rp.step(self._target_b)
            torch.cuda.synchronize()
            self._pending = None
        finally:
            if self.tuning is not None:
                api.set_tuning(prev)

    def run(self):
        """Replays the captured iteration on the current inputs; returns the device loss."""
        with torch.cuda.stream(self.stream):
            self.graph.replay()
        return self.rp.loss

    def step(self, target_host, cams_host=None, next_target_host=None, retries=2):
        """End-to-end iteration from host inputs; returns the loss as a Python float."""
        if self.graph is None:
            self.prepare(target_host.to(self.target.device))
        pend, self._pending = self._pending, None
        for _ in range(retries + 1):
            buf = 0
            with torch.cuda.stream(self.stream):
                if pend is not None and pend[0] is target_host:   # copied during the previous step
                    buf = pend[1]
                    self.stream.wait_event(pend[2])
                else:
                    self.target.copy_(target_host, non_blocking=True)
                if cams_host is not None:
                    self.views.cams.copy_(cams_host, non_blocking=True)
                (self._graph_b if buf else self.graph).replay()
                self._loss_host.copy_(self.rp.loss[:1], non_blocking=True)
                self._status_host.copy_(self.rp.status, non_blocking=True)
            ev = None
            if next_target_host is not None:
                # the other buffer's last reader finished with the previous step (synchronised)
                nxt = 1 - buf
                with torch.cuda.stream(self._copy_stream):
                    (self._target_b if nxt else self.target).copy_(next_target_host, non_blocking=True)
                    ev = torch.cuda.Event()
                    ev.record(self._copy_stream)
            self.stream.synchronize()
            if ev is not None:
                ev.synchronize()
            code = int(np.int32(int(self._status_host[0]) & 0xFFFFFFFF))
            if code == 0:
                if ev is not None:
                    self._pending = (next_target_host, nxt, ev)
                return float(self._loss_host[0])
            if code != L.GS_ERR_CAPACITY:
                raise L.GsError("mapping step", code)
            self.prepare()
            pend = None
        raise L.GsError("mapping step: capacity", L.GS_ERR_CAPACITY)

    @property
    def d2h_bytes(self):
        return 4 + 16


class Optimizer:
    """Adam over the anchor parameters the paper optimises -- features,
    offsets, log-scalings and the packed decoder weights -- in one launch per
    step (`gs_adam_step`).  Anchor positions are left out: the paper moves
    them only at loop closures.  The learning rates default to the
    Scaffold-GS values (the paper gives none); `lr` overrides them by name.
    Run it after the iteration's reverse pass (outside a captured graph: the
    bias correction changes every step)."""

    DEFAULT_LR = {"feat": 0.0075, "offsets": 0.01, "log_scaling": 0.007, "mlp": 0.004}

    def __init__(self, anchors: api.Anchors, grads: api.AnchorGrad, lr=None, betas=(0.9, 0.999), eps=1e-15):
        rates = dict(self.DEFAULT_LR)
        rates.update(lr or {})
        self.betas, self.eps, self.t = betas, float(eps), 0
        self.names = list(rates)
        self.groups = []
        for n in self.names:
            p, g = getattr(anchors, n), getattr(grads, "d" + n)
            self.groups.append([p, g, torch.zeros_like(p), torch.zeros_like(p), float(rates[n])])

    def set_lr(self, name, lr):
        self.groups[self.names.index(name)][4] = float(lr)

    def step(self, stream=None):
        self.t += 1
        api.adam_step([tuple(g) for g in self.groups], self.t, self.betas[0], self.betas[1], self.eps, stream)


class DensifyStats:
    """Accumulators of the growth / pruning statistics (`gs_densify_stats`)
    over a densification interval, and the candidate masks from them."""

    def __init__(self, anchors: api.Anchors, device="cuda"):
        self.N, self.k = anchors.N, anchors.k
        self.grad_accum = torch.zeros(self.N * self.k, device=device)
        self.offset_denom = torch.zeros(self.N * self.k, device=device, dtype=torch.int32)
        self.opacity_accum = torch.zeros(self.N, device=device)
        self.anchor_denom = torch.zeros(self.N, device=device, dtype=torch.int32)

    def reset(self):
        for t in (self.grad_accum, self.offset_denom, self.opacity_accum, self.anchor_denom):
            t.zero_()

    def accumulate(self, rp: RenderPass, stream=None):
        """Adds the statistics of the iteration `rp` has just run (after its backward).
        They read the decoded opacities: `rp` must leave them in g
        (RenderPass / MappingStep with fuse_projection=False for BF16)."""
        if not rp.gaussians_written:
            raise ValueError("densification statistics need the decoded Gaussians: build the pass with "
                             "fuse_projection=False")
        api.densify_stats(rp.g, rp.views, rp.splats, rp.sgrad, self.N, self.grad_accum, self.offset_denom,
                          self.opacity_accum, self.anchor_denom, rp.status, stream)

    def masks(self, grad_thr, opacity_thr, min_count=1, stream=None):
        grow = torch.zeros(self.N * self.k, device=self.grad_accum.device, dtype=torch.uint8)
        prune = torch.zeros(self.N, device=self.grad_accum.device, dtype=torch.uint8)
        api.densify_masks(self.k, self.grad_accum, self.offset_denom, self.opacity_accum, self.anchor_denom,
                          grad_thr, opacity_thr, min_count, grow, prune, stream)
        return grow, prune
