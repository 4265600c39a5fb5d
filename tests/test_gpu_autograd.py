"""The autograd front end (GsDecode, GsRender, GsL1) and the graph-captured
MappingStep: values and gradients against the FP64 oracle, a finite-difference
check of the composed backward, and the end-to-end step from host inputs."""
import numpy as np
import pytest
import torch

from _helpers import PIX_TOL, assert_grad_close, f32, image_mask, to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, autograd, pipeline, scenes
from test_gpu_parity import _e2e_masks, tiny

pytestmark = pytest.mark.gpu


def _leaf(a, dt=torch.float32):
    return torch.as_tensor(np.ascontiguousarray(a)).to("cuda", dt).requires_grad_(dt == torch.float32)


def _anchor_leaves(s):
    return (_leaf(s.xyz), _leaf(s.feat), _leaf(s.log_scaling), _leaf(s.offsets), _leaf(s.mlp),
            torch.as_tensor(np.ascontiguousarray(s.part)).to("cuda", torch.int32))


def test_autograd_anchor_path_matches_oracle():
    """decode -> render -> backward of a given image gradient, against the
    oracle's forward image and its hand-derived reverse pass (Eq. 1, Eq. 2, Eq. 6)."""
    s = tiny()
    fw = O.forward_anchor(s)
    ok = _e2e_masks(s, fw)
    assert ok.mean() > 0.97
    m = image_mask(s.wh, ok)
    views = api.Views(s.cams, s.wh)
    xyz, feat, ls, off, mlp, part = _anchor_leaves(s)
    dec = autograd.decode(xyz, feat, ls, off, mlp, part, views, s.k, s.hidden, s.M)
    img = autograd.render(dec, views)
    err = np.abs(to_np(img) - fw.ren.image)[m]
    assert err.max() <= PIX_TOL, f"max pixel error {err.max():.3e}"
    _, dimg = O.l1(s.wh, fw.ren.image, O.targets_flat(s))
    dimg = dimg * m
    img.backward(torch.as_tensor(f32(dimg)).cuda())
    _, want, _ = O.loss_and_grads_anchor(s, dimage=dimg)
    for name, t in (("xyz", xyz), ("feat", feat), ("log_scaling", ls), ("offsets", off), ("mlp", mlp)):
        assert t.grad is not None, name
        assert_grad_close(to_np(t.grad), want[name], "d" + name)


def test_autograd_l1_loss_and_its_gradient():
    s = tiny()
    views = api.Views(s.cams, s.wh)
    fw = O.forward_anchor(s)
    img = torch.as_tensor(f32(fw.ren.image)).cuda().requires_grad_(True)
    tgt = O.targets_flat(s)
    loss = autograd.l1_loss(img, torch.as_tensor(f32(tgt)).cuda(), views)
    L_o, dimg = O.l1(s.wh, fw.ren.image, tgt)
    assert float(loss.detach()) == pytest.approx(L_o, abs=1e-4)
    (2.0 * loss).backward()
    assert np.allclose(to_np(img.grad), 2.0 * dimg, rtol=1e-5, atol=1e-9)


def test_autograd_explicit_gaussians_gradients():
    """Explicit Gaussians through GsRender: the colour gradient against central
    differences of FP32 renders (the image is linear in colour), and every
    input's gradient against the oracle's reverse pass (Eq. 1 and the EWA
    projection chain rule).  Means and opacities are not differenced: the
    alpha >= 1/255 skip makes the image jump under their perturbations."""
    s = scenes.explicit_frustum(seed=1, n=600)
    views = api.Views(s.cams, s.wh)
    leaves = [_leaf(a) for a in (s.mu, s.scale, s.quat, s.opacity, s.colour)]
    fw = O.forward_explicit(s)
    ok = _e2e_masks(s, fw)
    assert ok.mean() > 0.97
    m = image_mask(s.wh, ok)
    wts_np = np.random.default_rng(2).uniform(-1, 1, 3 * views.total_pixels) * m
    wts = torch.as_tensor(f32(wts_np)).cuda()
    r = autograd.Renderer()

    def f(mu, scale, quat, opacity, colour):
        return autograd.render(autograd.explicit(mu, scale, quat, opacity, colour), views, renderer=r)

    img = f(*leaves)
    (img * wts).sum().backward()
    d = torch.as_tensor(np.random.default_rng(3).normal(size=s.colour.shape).astype(np.float32)).cuda()
    eps = 1e-2
    with torch.no_grad():
        args_p = [t.detach().clone() for t in leaves]
        args_m = [t.detach().clone() for t in leaves]
        args_p[4] += eps * d
        args_m[4] -= eps * d
        numeric = float(((f(*args_p).double() - f(*args_m).double()) * wts.double()).sum()) / (2 * eps)
    analytic = float((leaves[4].grad * d).sum())
    assert analytic == pytest.approx(numeric, rel=1e-3, abs=1e-4)
    wts64 = f32(wts_np).astype(np.float64)
    dm, dk, do, dc = O.render_bwd(s.wh, fw.prj.mean2d, fw.prj.conic, fw.opacity, fw.colour, fw.ranges,
                                  fw.vals, wts64)
    dmu, ds, dq = O.project_bwd(s.mu, s.scale, s.quat, fw.prj.status, s.cams, s.wh, fw.view_start_c, dm, dk)
    for name, t, want in (("dmu", leaves[0], dmu), ("dscale", leaves[1], ds), ("dquat", leaves[2], dq),
                          ("dopacity", leaves[3], do), ("dcolour", leaves[4], dc)):
        assert_grad_close(to_np(t.grad), want, name)


def test_autograd_bf16_decode_gradients_close_to_fp32():
    s = scenes.tiny_corridor(seed=0, n_anchors=4000, F=32, k=10, hidden=32)
    views = api.Views(s.cams, s.wh)
    grads = {}
    for prec in (L.GS_PREC_FP32, L.GS_PREC_BF16):
        xyz, feat, ls, off, mlp, part = _anchor_leaves(s)
        dec = autograd.decode(xyz, feat, ls, off, mlp, part, views, s.k, s.hidden, s.M, precision=prec)
        loss = autograd.l1_loss(autograd.render(dec, views), torch.as_tensor(f32(O.targets_flat(s))).cuda(), views)
        loss.backward()
        grads[prec] = [to_np(t.grad).ravel().astype(np.float64) for t in (xyz, feat, ls, off, mlp)]
    for a, b in zip(grads[L.GS_PREC_BF16], grads[L.GS_PREC_FP32]):
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        assert cos >= 0.999


def test_mapping_step_from_host_inputs_matches_render_pass():
    s = scenes.tiny_corridor(seed=0, n_anchors=4000, F=32, k=10, hidden=32)
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    tgt_host = torch.as_tensor(f32(O.targets_flat(s))).pin_memory()
    ref = pipeline.RenderPass(views, A, precision=L.GS_PREC_BF16, store_state=False)
    assert ref.ensure_capacity(tgt_host.cuda()) == 0
    ref.step(tgt_host.cuda())
    torch.cuda.synchronize()
    want = float(ref.loss.item())
    dfeat = to_np(ref.agrad.dfeat).copy()
    # deliberately small capacities: the step grows them and re-captures
    ms = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16, cap_rows=64)
    ms.rp.cap_pairs = 1024
    ms.rp._alloc()
    got = ms.step(tgt_host)
    assert got == pytest.approx(want, rel=1e-5, abs=1e-6)
    assert np.allclose(to_np(ms.rp.agrad.dfeat), dfeat, rtol=1e-4, atol=1e-6)
    got2 = ms.step(tgt_host)   # replay only
    assert got2 == pytest.approx(want, rel=1e-5, abs=1e-6)


def test_mapping_step_prefetched_targets():
    """Each step copying the next step's images into the second buffer during
    its run: the losses are those of the images each step was given, through
    both captured graphs, and a step given other images than the prefetched
    ones copies its own."""
    s = scenes.tiny_corridor(seed=0, n_anchors=4000, F=32, k=10, hidden=32)
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    t0 = f32(O.targets_flat(s))
    tgts = [torch.as_tensor(t0).pin_memory(), torch.as_tensor(f32(t0[::-1].copy())).pin_memory(),
            torch.as_tensor(f32(0.5 * t0)).pin_memory()]
    ref = pipeline.RenderPass(views, A, precision=L.GS_PREC_BF16, store_state=False)
    assert ref.ensure_capacity(tgts[0].cuda()) == 0
    want = []
    for t in tgts:
        ref.step(t.cuda())
        torch.cuda.synchronize()
        want.append(float(ref.loss.item()))
    assert len(set(want)) == 3
    ms = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16)
    order = [0, 1, 2, 0, 1]
    for i, j in enumerate(order):
        nxt = tgts[order[i + 1]] if i + 1 < len(order) else None
        assert ms.step(tgts[j], next_target_host=nxt) == pytest.approx(want[j], rel=1e-5, abs=1e-6)
    # a prefetched buffer the next call does not use
    assert ms.step(tgts[2], next_target_host=tgts[0]) == pytest.approx(want[2], rel=1e-5, abs=1e-6)
    assert ms.step(tgts[1]) == pytest.approx(want[1], rel=1e-5, abs=1e-6)
