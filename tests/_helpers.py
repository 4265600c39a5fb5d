"""Test glue: feeds oracle outputs (rounded to FP32) to the CUDA path, and
compares results element by element with masks for decisions that FP32 and
FP64 may legitimately take differently near a threshold."""
from __future__ import annotations

import numpy as np
import torch

from oracle import oracle as O

PIX_TOL = 1e-4        # FP32 pixels vs FP64 oracle (absolute)
GRAD_REL = 1e-3       # gradients, per tensor ||g - g*|| / ||g*||
GRAD_ELEM = 1e-3      # gradients, per element, relative to max |g*| of the tensor


def f32(a):
    return np.ascontiguousarray(np.asarray(a, np.float64).astype(np.float32))


def pack_records(prj: O.Projected, opacity, colour):
    """[C,12] float32 records in the library's layout from oracle projection
    outputs (culled candidates get an empty record)."""
    C_ = prj.tiles.shape[0]
    rec = np.zeros((C_, 12), np.float32)
    ok = prj.tiles > 0
    rec[:, 0:2] = f32(prj.mean2d)
    # exponent coefficients in base 2 and log2 opacity (the library's record layout)
    l2e = 1.0 / np.log(2.0)
    conic = np.asarray(prj.conic, np.float64)
    rec[:, 2] = f32(-0.5 * l2e * conic[:, 0])
    rec[:, 3] = f32(-l2e * conic[:, 1])
    rec[:, 4] = f32(-0.5 * l2e * conic[:, 2])
    with np.errstate(divide="ignore"):
        rec[:, 5] = f32(np.log2(np.maximum(np.asarray(opacity, np.float64), 1e-30)))
    rec[:, 6:9] = f32(colour)
    rec[:, 9] = f32(prj.depth)
    rx = (prj.rect[:, 0].astype(np.uint32) | (prj.rect[:, 2].astype(np.uint32) << 16))
    ry = (prj.rect[:, 1].astype(np.uint32) | (prj.rect[:, 3].astype(np.uint32) << 16))
    rec[:, 10] = rx.view(np.float32)
    rec[:, 11] = ry.view(np.float32)
    rec[~ok] = 0
    return rec, np.where(ok, prj.tiles, 0).astype(np.int32)


def rounded_projection(prj: O.Projected, opacity, colour):
    """The oracle projection as the library's FP32 records carry it (as doubles):
    conic and opacity recovered from the rounded base-2 coefficients."""
    r = lambda a: np.asarray(a, np.float64).astype(np.float32).astype(np.float64)
    rec, _ = pack_records(prj, opacity, colour)
    rec = rec.astype(np.float64)
    l2e = 1.0 / np.log(2.0)
    conic = np.stack([-2.0 * rec[:, 2] / l2e, -rec[:, 3] / l2e, -2.0 * rec[:, 4] / l2e], 1)
    op = np.where(np.asarray(opacity) > 0, np.exp2(rec[:, 5]), 0.0)
    return dict(mean2d=r(prj.mean2d), conic=conic, opacity=op, colour=r(colour),
                depth_bits=prj.depth_bits, rect=prj.rect, status=prj.status)


def tile_mask_from_splats(wh, view_start, k, rect, presence, edge=None):
    """Pixels whose result may legitimately differ because a splat decision is
    near its threshold: every tile of the rectangle (grown by one tile) of a
    splat whose presence may flip, and the ring of tiles along the rectangle
    border of a splat whose rectangle may flip."""
    wh = np.asarray(wh).reshape(-1, 2)
    masks = [np.zeros((int(h), int(w)), bool) for w, h in wh]
    edge = np.zeros_like(presence) if edge is None else edge
    for c in np.nonzero(presence | edge)[0]:
        v = int(np.searchsorted(view_start, c // k, side="right") - 1)
        x0, y0, x1, y1 = (int(x) for x in rect[c])
        m = masks[v]
        if presence[c]:
            m[max(0, y0 - 1) * 16:(y1 + 1) * 16, max(0, x0 - 1) * 16:(x1 + 1) * 16] = True
        else:
            for xx in (x0 - 1, x0, x1 - 1, x1):
                if xx >= 0:
                    m[max(0, y0 - 1) * 16:(y1 + 1) * 16, xx * 16:(xx + 1) * 16] = True
            for yy in (y0 - 1, y0, y1 - 1, y1):
                if yy >= 0:
                    m[yy * 16:(yy + 1) * 16, max(0, x0 - 1) * 16:(x1 + 1) * 16] = True
    return np.concatenate([m.reshape(-1) for m in masks])


def image_mask(wh, pix_mask):
    """Per-pixel mask -> per-(channel, pixel) mask in the planar image layout."""
    wh = np.asarray(wh).reshape(-1, 2)
    out, b = [], 0
    for w, h in wh:
        n = int(w) * int(h)
        out.append(np.tile(pix_mask[b:b + n], 3))
        b += n
    return np.concatenate(out)


def assert_grad_close(got, want, name, rel=GRAD_REL, elem=GRAD_ELEM):
    got = np.asarray(got, np.float64).reshape(-1)
    want = np.asarray(want, np.float64).reshape(-1)
    nw = np.linalg.norm(want)
    scale = np.max(np.abs(want)) if want.size else 0.0
    if nw == 0:
        assert np.max(np.abs(got)) <= 1e-6, f"{name}: expected zero gradient"
        return
    err = np.linalg.norm(got - want) / nw
    worst = float(np.max(np.abs(got - want))) / scale if scale > 0 else 0.0
    print(f"[grad] {name}: per-tensor {err:.3e} (bar {rel}), worst element {worst:.3e} of max|g*| (bar {elem})")
    assert err <= rel, f"{name}: relative error {err:.3e} > {rel}"
    bad = np.abs(got - want) > elem * scale + 1e-7
    assert not bad.any(), f"{name}: {bad.sum()} elements off (max {np.max(np.abs(got - want)):.3e})"


def to_np(t):
    return t.detach().cpu().numpy()


def u32(t):
    return to_np(t).view(np.uint32)
