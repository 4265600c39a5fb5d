"""Central finite differences of the autograd front end on the GPU (FP32):
GsDecode -> GsRender (gs_decode_bwd, gs_render_bwd with the projection chain
rule) for the anchor map, and GsRender alone for explicit Gaussians.

The scenes are built so that no discrete decision of the method lies near
its threshold: every splat covers the whole image with alpha well above
1/255 at every pixel (no skip, no tile-rectangle edge inside the view), the
transmittance stays far above the 1e-4 stop, opacities are far from the 0.99
clamp and from the decoder's opacity > 0 cull, and depths are 0.5 m apart (no
order swap), and every decoder hidden unit is at least 0.1 from its ReLU
kink.  The image is then a smooth function of every parameter and
central differences of a weighted sum of the FP32 image must match the
analytic directional derivative.  The FP64 oracle confirms the design (every
pair composited, nothing flagged near a threshold) before the GPU runs."""
import math

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2607_21416_b300 import api, autograd, scenes

pytestmark = pytest.mark.gpu

W, H, FX = 48, 32, 40.0
FD_REL = 1e-2      # relative size of the step (per tensor, against its RMS; the path is smooth here)
FD_TOL = 1e-3      # |FD - analytic| <= FD_TOL |analytic| + the FP32 noise floor


def smooth_anchor_scene(seed=0, F=8, k=4, hidden=16):
    """Two anchors in two partitions (one decoder each, Eq. 6) 6 m and 9.5 m in
    front of a 48x32 camera; offsets put their k Gaussians 0.5 m apart in
    depth; log-scalings [3:6] of ln 16 make every Gaussian cover the view;
    the opacity heads are damped around tanh(0.35) and the covariance heads
    around sigmoid(0) (draw order: features, offsets x/y, decoder weights)."""
    rng = np.random.default_rng(seed)
    xyz = np.array([[0.3, -0.2, 6.0], [-0.4, 0.25, 9.5]])
    feat = rng.normal(0.0, 0.1, (2, F))
    off = np.zeros((2, k, 3))
    off[:, :, :2] = rng.normal(0.0, 0.1, (2, k, 2))
    off[:, :, 2] = (np.arange(k) - (k - 1) / 2.0) * 0.5
    ls = np.zeros((2, 6))
    ls[:, 3:6] = math.log(16.0)
    mlp = scenes.init_mlp(rng, 2, F, k, hidden).astype(np.float64)
    din = F + 4
    for m in range(2):
        o = 0
        for h, dout in enumerate((k, 3 * k, 7 * k)):
            w2 = o + hidden * din + hidden
            b2 = w2 + dout * hidden
            if h == 0:      # opacity head: tanh(0.35 + small)
                mlp[m, w2:b2] *= 0.1
                mlp[m, b2:b2 + dout] = 0.35
            elif h == 2:    # covariance head: sigmoid(~0) scales
                mlp[m, w2:b2] *= 0.3
                mlp[m, b2:b2 + 3 * k] = 0.0
            o = b2 + dout
    cams = scenes.camera(FX, FX, W / 2.0, H / 2.0, (0.0, 0.0, 0.0))[None]
    # every hidden unit's pre-activation at least 0.1 away from the ReLU kink
    # (each partition decodes one anchor here, so its biases can be shifted)
    for a in range(2):
        o = 0
        for dout in (k, 3 * k, 7 * k):
            pre = _preactivations(mlp[a], o, feat[a], xyz[a], F, hidden)
            b1 = o + hidden * din
            shift = np.where(np.abs(pre) < 0.1, np.where(pre >= 0, 0.1, -0.1), 0.0)
            mlp[a, b1:b1 + hidden] += shift
            o = b1 + hidden + dout * hidden + dout
    wh = np.array([[W, H]], np.int32)
    return scenes.Scene(name="smooth_anchors", xyz=xyz.astype(np.float32), feat=feat.astype(np.float32),
                        log_scaling=ls.astype(np.float32), offsets=off.astype(np.float32),
                        part=np.array([0, 1], np.int32), mlp=mlp.astype(np.float32), F=F, k=k,
                        hidden=hidden, M=2, cams=cams, wh=wh,
                        targets=[rng.uniform(0, 1, (3, H, W)).astype(np.float32)])


def _preactivations(P, o, feat, xyz, F, hidden):
    """First-layer pre-activations W1 u + b1 of the head at offset o of a
    packed decoder P, for an anchor seen from a camera at the origin (Eq. 2:
    u = [f_a, direction, distance])."""
    din = F + 4
    d = np.asarray(xyz, np.float64)
    dist = np.linalg.norm(d)
    u = np.concatenate([np.asarray(feat, np.float64), d / dist, [dist]])
    W1 = np.asarray(P[o:o + hidden * din], np.float64).reshape(hidden, din)
    return W1 @ u + np.asarray(P[o + hidden * din:o + hidden * din + hidden], np.float64)


def _relu_margin(s):
    out = []
    for a in range(s.N):
        o = 0
        for dout in (s.k, 3 * s.k, 7 * s.k):
            out.append(np.abs(_preactivations(s.mlp[s.part[a]], o, s.feat[a], s.xyz[a], s.F, s.hidden)).min())
            o += s.hidden * (s.F + 4) + s.hidden + dout * s.hidden + dout
    return min(out)


def smooth_explicit_scene(seed=0, n=6):
    """n Gaussians 4..9 m deep (1 m apart) near the optical axis, scales
    U[5, 8] m, random rotations, opacities U[0.25, 0.35], colours U[0, 1]."""
    rng = np.random.default_rng(seed)
    z = 4.0 + np.arange(n)
    mu = np.stack([rng.uniform(-0.1, 0.1, n) * z, rng.uniform(-0.1, 0.1, n) * z, z], 1)
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return scenes.Scene(name="smooth_explicit", mu=mu.astype(np.float32),
                        scale=rng.uniform(5.0, 8.0, (n, 3)).astype(np.float32), quat=q.astype(np.float32),
                        opacity=rng.uniform(0.25, 0.35, n).astype(np.float32),
                        colour=rng.uniform(0.0, 1.0, (n, 3)).astype(np.float32),
                        cams=scenes.camera(FX, FX, W / 2.0, H / 2.0, (0.0, 0.0, 0.0))[None],
                        wh=np.array([[W, H]], np.int32), targets=[])


def _assert_smooth(fw, n_splats):
    """The oracle's forward: every pixel composites every splat, nothing is
    flagged near a threshold, transmittance far above the stop."""
    assert (fw.ren.pix_flag == 0).all()
    assert (fw.ren.last == n_splats).all()
    assert fw.ren.T_final.min() > 1e-2


def _weights(seed, n):
    return torch.as_tensor(np.random.default_rng(seed).uniform(-0.5, 1.5, n).astype(np.float32)).cuda()


def _fd_check(f, leaves, names, w, seed):
    """Analytic directional derivative of sum(w * f(leaves)) along a random
    direction per tensor against central differences."""
    out = f(*leaves)
    (out * w).sum().backward()
    rng = np.random.default_rng(seed)
    for i, name in enumerate(names):
        p = leaves[i]
        d = torch.as_tensor(rng.normal(size=tuple(p.shape)).astype(np.float32)).cuda()
        h = FD_REL * (float(p.detach().pow(2).mean().sqrt()) + 1e-3) / float(d.pow(2).mean().sqrt())
        with torch.no_grad():
            plus = [t.detach().clone() for t in leaves]
            minus = [t.detach().clone() for t in leaves]
            plus[i] += h * d
            minus[i] -= h * d
            lp = float((f(*plus).double() * w.double()).sum())
            lm = float((f(*minus).double() * w.double()).sum())
        fd = (lp - lm) / 2.0
        an = h * float((p.grad.double() * d.double()).sum())
        noise = 1e-6 * float((out.detach().double().abs() * w.double().abs()).sum()) / math.sqrt(out.numel())
        print(f"[fd] {name}: finite difference {fd:.6e}, analytic {an:.6e}")
        assert abs(fd - an) <= FD_TOL * abs(an) + noise, f"{name}: FD {fd:.6e} vs analytic {an:.6e}"


def test_finite_differences_through_decode_and_render():
    s = smooth_anchor_scene()
    _assert_smooth(O.forward_anchor(s), s.N * s.k)
    assert _relu_margin(s) >= 0.099
    views = api.Views(s.cams, s.wh)
    leaf = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda().requires_grad_(True)
    leaves = [leaf(s.xyz), leaf(s.feat), leaf(s.log_scaling), leaf(s.offsets), leaf(s.mlp)]
    part = torch.as_tensor(s.part).cuda()

    def f(xyz, feat, ls, off, mlp):
        return autograd.render(autograd.decode(xyz, feat, ls, off, mlp, part, views, s.k, s.hidden, s.M), views)

    _fd_check(f, leaves, ["xyz", "feat", "log_scaling", "offsets", "mlp"], _weights(7, 3 * W * H), 8)


def test_finite_differences_through_render_of_explicit_gaussians():
    s = smooth_explicit_scene()
    _assert_smooth(O.forward_explicit(s), s.mu.shape[0])
    views = api.Views(s.cams, s.wh)
    leaf = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda().requires_grad_(True)
    leaves = [leaf(s.mu), leaf(s.scale), leaf(s.quat), leaf(s.opacity), leaf(s.colour)]

    def f(mu, scale, quat, opacity, colour):
        return autograd.render(autograd.explicit(mu, scale, quat, opacity, colour), views)

    _fd_check(f, leaves, ["mu", "scale", "quat", "opacity", "colour"], _weights(9, 3 * W * H), 10)


def test_finite_differences_of_the_l1_loss_through_the_whole_path():
    """The composed GsDecode -> GsRender -> GsL1 loss along one direction over
    all anchor parameters at once.  The target sits 0.05 above the image at
    the expansion point, so the L1 kink is never crossed and the loss stays
    small (its FP32 sum then carries little rounding); the step is 1e-2 of
    each tensor's RMS (the path is smooth here: truncation error ~1e-4)."""
    s = smooth_anchor_scene(seed=3)
    _assert_smooth(O.forward_anchor(s), s.N * s.k)
    assert _relu_margin(s) >= 0.099
    views = api.Views(s.cams, s.wh)
    leaf = lambda a: torch.as_tensor(np.ascontiguousarray(a)).cuda().requires_grad_(True)
    leaves = [leaf(s.xyz), leaf(s.feat), leaf(s.log_scaling), leaf(s.offsets), leaf(s.mlp)]
    part = torch.as_tensor(s.part).cuda()

    def image(*ps):
        return autograd.render(autograd.decode(*ps, part, views, s.k, s.hidden, s.M), views)

    with torch.no_grad():
        tgt = image(*[p.detach() for p in leaves]) + 0.05

    def loss(*ps):
        return autograd.l1_loss(image(*ps), tgt, views)

    L0 = loss(*leaves)
    L0.backward()
    rng = np.random.default_rng(11)
    ds = [torch.as_tensor(rng.normal(size=tuple(p.shape)).astype(np.float32)).cuda() for p in leaves]
    hs = [1e-2 * (float(p.detach().pow(2).mean().sqrt()) + 1e-3) / float(d.pow(2).mean().sqrt())
          for p, d in zip(leaves, ds)]
    with torch.no_grad():
        lp = float(loss(*[p.detach() + h * d for p, h, d in zip(leaves, hs, ds)]).double())
        lm = float(loss(*[p.detach() - h * d for p, h, d in zip(leaves, hs, ds)]).double())
    fd = (lp - lm) / 2.0
    an = sum(h * float((p.grad.double() * d.double()).sum()) for p, h, d in zip(leaves, hs, ds))
    print(f"[fd] L1 loss: finite difference {fd:.6e}, analytic {an:.6e} (loss {float(L0.detach()):.4e})")
    assert abs(fd - an) <= FD_TOL * abs(an) + 4 * 2.0 ** -24 * float(L0.detach())
