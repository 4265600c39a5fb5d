"""A third opinion on the oracle's hand-derived reverse passes: PyTorch float64
autograd (CPU) of independent formulations of the same forward steps.

* Compositing (Eq. 1) per tile as one vectorised exclusive cumulative product
  of (1 - alpha) over the tile's sorted list, the skip and stop decisions
  taken on the forward values; autograd through alpha = min(0.99, o
  exp(power)), the transmittances and the colours, against the oracle's
  reverse pass (d mean2d, d conic, d opacity, d colour).
* The EWA projection (mean2d and conic of each Gaussian from its position,
  scale and quaternion, tangent clamp included) against the oracle's
  projection chain rule.
"""
import numpy as np
import torch

from oracle import oracle as O
from paper_2607_21416_b300 import scenes

T = torch.float64


def _composite_tile(x0, y0, W, H, ids, mean2d, conic, opacity, colour, bg):
    """Image values of the tile's pixels from its sorted list `ids` (torch)."""
    ys, xs = torch.meshgrid(torch.arange(y0, min(y0 + 16, H), dtype=T), torch.arange(x0, min(x0 + 16, W), dtype=T),
                            indexing="ij")
    px, py = xs.reshape(-1, 1), ys.reshape(-1, 1)
    if len(ids) == 0:
        return torch.tensor(bg, dtype=T).view(3, 1).expand(3, px.shape[0]), xs, ys
    m, k = mean2d[ids], conic[ids]
    dx, dy = m[:, 0].view(1, -1) - px, m[:, 1].view(1, -1) - py
    power = -0.5 * (k[:, 0] * dx * dx + k[:, 2] * dy * dy) - k[:, 1] * dx * dy
    ag = opacity[ids].view(1, -1) * torch.exp(power)
    alpha = torch.minimum(ag, torch.full_like(ag, 0.99))
    with torch.no_grad():
        valid = (power <= 0) & (alpha >= 1.0 / 255.0)
    a = torch.where(valid, alpha, torch.zeros_like(alpha))
    one_m = 1.0 - a
    t_after = torch.cumprod(one_m, dim=1)
    t_before = torch.cat([torch.ones_like(t_after[:, :1]), t_after[:, :-1]], dim=1)
    with torch.no_grad():   # the stop: the first composited splat whose T' falls below 1e-4 (not composited)
        stop_hit = valid & (t_after < 1e-4)
        n = a.shape[1]
        first = torch.where(stop_hit.any(1), stop_hit.float().argmax(1), torch.full((a.shape[0],), n))
        keep = torch.arange(n).view(1, -1) < first.view(-1, 1)
    w = torch.where(keep, a * t_before, torch.zeros_like(a))
    C = w @ colour[ids]                                                   # [pixels, 3]
    last_T = torch.where(first < n, t_before.gather(1, first.clamp(max=n - 1).view(-1, 1)).squeeze(1),
                         t_after[:, -1])
    img = C.T + last_T.view(1, -1) * torch.tensor(bg, dtype=T).view(3, 1)
    return img, xs, ys


def test_torch_autograd_of_compositing_matches_the_oracle_reverse_pass():
    s = scenes.explicit_frustum(seed=4, n=150, width=40, height=32, fx=40, fy=40, cx=20, cy=16)
    W, H = 40, 32
    vs = np.array([0, 150], np.int64)
    prj = O.project(s.mu, s.scale, s.quat, s.opacity, s.cams, s.wh, vs)
    keys, vals, ranges = O.bin_sort(prj.depth_bits, prj.rect, s.wh, vs)
    bg = (0.1, 0.2, 0.3)
    ren = O.render(s.wh, vs, 1, prj.mean2d, prj.conic, s.opacity.astype(np.float64), s.colour.astype(np.float64),
                   prj.depth_bits, prj.rect, prj.status, 0, ranges, vals, bg)
    mean2d = torch.tensor(prj.mean2d, dtype=T, requires_grad=True)
    conic = torch.tensor(prj.conic, dtype=T, requires_grad=True)
    opacity = torch.tensor(s.opacity.astype(np.float64), dtype=T, requires_grad=True)
    colour = torch.tensor(s.colour.astype(np.float64), dtype=T, requires_grad=True)
    img = torch.zeros(3, H, W, dtype=T)
    TX = (W + 15) // 16
    for t in range(len(ranges)):
        ids = torch.as_tensor(vals[ranges[t, 0]:ranges[t, 1]].astype(np.int64))
        x0, y0 = 16 * (t % TX), 16 * (t // TX)
        v, xs, ys = _composite_tile(x0, y0, W, H, ids, mean2d, conic, opacity, colour, bg)
        img[:, y0:y0 + xs.shape[0], x0:x0 + xs.shape[1]] = v.reshape(3, xs.shape[0], xs.shape[1])
    # the independent forward agrees with the oracle's image
    assert np.allclose(img.detach().numpy().reshape(-1), ren.image, rtol=1e-12, atol=1e-12)
    w = np.random.default_rng(5).normal(size=3 * H * W)
    (img.reshape(-1) * torch.tensor(w, dtype=T)).sum().backward()
    dm, dk, do, dc = O.render_bwd(s.wh, prj.mean2d, prj.conic, s.opacity.astype(np.float64),
                                  s.colour.astype(np.float64), ranges, vals, w, bg)
    for got, want in ((mean2d.grad, dm), (conic.grad, dk), (opacity.grad, do), (colour.grad, dc)):
        want = np.asarray(want).reshape(got.shape)
        scale = np.abs(want).max()
        assert scale > 0
        assert np.allclose(got.numpy(), want, rtol=1e-9, atol=1e-10 * scale)


def _rot(q):
    w, x, y, z = q[:, 0], q[:, 1], q[:, 2], q[:, 3]
    return torch.stack([
        torch.stack([1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)], -1),
        torch.stack([2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)], -1),
        torch.stack([2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)], -1)], -2)


def test_torch_autograd_of_projection_matches_the_oracle_chain_rule():
    s = scenes.explicit_frustum(seed=7, n=60)
    s.mu[:8, 0] *= 3.0                                   # some off-axis enough for the tangent clamp
    W, H = s.wh[0]
    cam = s.cams[0].astype(np.float64)
    fx, fy, cx, cy = cam[:4]
    Rw, tw = torch.tensor(cam[4:13].reshape(3, 3)), torch.tensor(cam[13:16])
    vs = np.array([0, 60], np.int64)
    prj = O.project(s.mu, s.scale, s.quat, s.opacity, s.cams, s.wh, vs)
    live = prj.status == 1
    assert live.sum() > 40
    mu = torch.tensor(s.mu.astype(np.float64), requires_grad=True)
    sc = torch.tensor(s.scale.astype(np.float64), requires_grad=True)
    qt = torch.tensor(s.quat.astype(np.float64), requires_grad=True)
    p = mu @ Rw.T + tw
    Rq = _rot(qt)
    M = Rq * sc.view(-1, 1, 3)
    S3 = M @ M.transpose(1, 2)
    limx, limy = 1.3 * W / (2 * fx), 1.3 * H / (2 * fy)
    txz = torch.clamp(p[:, 0] / p[:, 2], -limx, limx)
    tyz = torch.clamp(p[:, 1] / p[:, 2], -limy, limy)
    z = p[:, 2]
    zero = torch.zeros_like(z)
    J = torch.stack([torch.stack([fx / z, zero, -fx * txz / z], -1),
                     torch.stack([zero, fy / z, -fy * tyz / z], -1)], -2)
    Tm = J @ Rw
    S2 = Tm @ S3 @ Tm.transpose(1, 2)
    a, b, c = S2[:, 0, 0] + 0.3, S2[:, 0, 1], S2[:, 1, 1] + 0.3
    det = a * c - b * b
    conic = torch.stack([c / det, -b / det, a / det], -1)
    mean2d = torch.stack([fx * p[:, 0] / z + cx, fy * p[:, 1] / z + cy], -1)
    assert np.allclose(conic.detach().numpy()[live], prj.conic[live], rtol=1e-11)
    assert np.allclose(mean2d.detach().numpy()[live], prj.mean2d[live], rtol=1e-12)
    rng = np.random.default_rng(8)
    wm, wk = rng.normal(size=(60, 2)) * live[:, None], rng.normal(size=(60, 3)) * live[:, None]
    ((mean2d * torch.tensor(wm)).sum() + (conic * torch.tensor(wk)).sum()).backward()
    dmu, ds, dq = O.project_bwd(s.mu, s.scale, s.quat, prj.status, s.cams, s.wh, vs, wm, wk)
    for got, want in ((mu.grad, dmu), (sc.grad, ds), (qt.grad, dq)):
        scale = np.abs(want).max()
        assert np.allclose(got.numpy()[live], want[live], rtol=1e-9, atol=1e-10 * scale)
