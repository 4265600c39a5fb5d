"""gs_photometric_loss (Eq. 3: lam L1 + (1 - lam)(1 - SSIM)) against the FP64
oracle, element by element: ragged view sets (sizes that leave partial 16x16
tiles, images smaller than the 11x11 window, a 1x1 view), uncorrelated,
nearly identical and identical image pairs, the lam = 1 and lam = 0 ends, the
full keyframe resolution, repeated calls on one workspace, the autograd front
end and the graph-captured mapping step."""
import numpy as np
import pytest
import torch

from _helpers import assert_grad_close, f32, to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, autograd, pipeline, scenes

pytestmark = pytest.mark.gpu

LOSS_TOL = 2e-5   # absolute, on loss values of order 1 (FP32 window sums, per-tile partials)


def _views(wh):
    return api.Views(np.zeros((len(wh), 16), np.float32), np.asarray(wh))


def _pair(wh, seed, noise=None):
    rng = np.random.default_rng(seed)
    n = 3 * int(sum(w * h for w, h in wh))
    x = rng.uniform(size=n)
    y = rng.uniform(size=n) if noise is None else np.clip(x + noise * rng.normal(size=n), 0, 1)
    return f32(x), f32(y)


def _gpu(views, x, y, lam, ws=None):
    img, tgt = torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda()
    loss = torch.full((3,), float("nan"), device="cuda")
    d = torch.full_like(img, float("nan"))
    if ws is None:
        ws = api.workspace(api.photometric_workspace(views))
    api.photometric_loss(img, tgt, views, lam, ws, loss, d)
    torch.cuda.synchronize()
    return to_np(loss), to_np(d)


def _check(wh, x, y, lam, got_loss, got_d):
    L_, d, L1, Ls = O.photometric(wh, x.astype(np.float64), y.astype(np.float64), lam)
    assert got_loss[0] == pytest.approx(L_, abs=LOSS_TOL * len(wh))
    assert got_loss[1] == pytest.approx(L1, abs=LOSS_TOL * len(wh))
    assert got_loss[2] == pytest.approx(Ls, abs=LOSS_TOL * len(wh))
    assert_grad_close(got_d, d, "dL/dimage")


RAGGED = [(37, 23), (64, 48), (5, 3), (1, 1), (17, 16), (100, 7)]


@pytest.mark.parametrize("noise", [None, 0.05])
def test_ragged_views_match_oracle(noise):
    wh = RAGGED
    views = _views(wh)
    x, y = _pair(wh, 1, noise)
    got_loss, got_d = _gpu(views, x, y, 0.8)
    _check(np.asarray(wh), x, y, 0.8, got_loss, got_d)


def test_identical_images_are_the_optimum():
    """x = y: both terms vanish and so does the gradient (S = 1 is the maximum
    of every SSIM map entry; the L1 sign is 0).  What is left is FP32 rounding
    of terms that cancel: per view, far below the 1 / (3 H W) scale of its
    gradients in the other cases."""
    wh = RAGGED
    views = _views(wh)
    x, _ = _pair(wh, 1)
    got_loss, got_d = _gpu(views, x, x.copy(), 0.8)
    assert got_loss[1] == 0.0
    assert abs(got_loss[2]) < 1e-5 and abs(got_loss[0]) < 1e-5
    at = 0
    for w, h in wh:
        n = 3 * w * h
        assert np.abs(got_d[at:at + n]).max() < 1e-5 / n, (w, h)
        at += n


@pytest.mark.parametrize("lam", [1.0, 0.0, 0.35])
def test_lambda_ends_and_l1_agreement(lam):
    wh = [(29, 31), (16, 16)]
    views = _views(wh)
    x, y = _pair(wh, 2, 0.1)
    got_loss, got_d = _gpu(views, x, y, lam)
    _check(np.asarray(wh), x, y, lam, got_loss, got_d)
    if lam == 1.0:   # pure L1: the same result as gs_l1_loss
        l1 = torch.zeros(1, device="cuda")
        d1 = torch.zeros(len(x), device="cuda")
        api.l1_loss(torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda(), views, l1, d1)
        torch.cuda.synchronize()
        assert got_loss[0] == pytest.approx(float(l1[0]), rel=1e-5)
        assert np.allclose(got_d, to_np(d1), rtol=1e-6, atol=1e-12)


def test_full_keyframe_resolution_two_views():
    wh = [(1241, 376), (1241, 376)]
    views = _views(wh)
    x, y = _pair(wh, 3, 0.2)
    got_loss, got_d = _gpu(views, x, y, 0.8)
    _check(np.asarray(wh), x, y, 0.8, got_loss, got_d)


def test_repeated_calls_share_the_workspace():
    wh = [(40, 33), (9, 70)]
    views = _views(wh)
    ws = api.workspace(api.photometric_workspace(views))
    for seed in (4, 5):
        x, y = _pair(wh, seed, 0.1 if seed == 4 else None)
        got_loss, got_d = _gpu(views, x, y, 0.8, ws)
        _check(np.asarray(wh), x, y, 0.8, got_loss, got_d)


def test_invalid_arguments_are_rejected():
    views = _views([(8, 8)])
    img = torch.zeros(192, device="cuda")
    loss = torch.zeros(3, device="cuda")
    ws = api.workspace(api.photometric_workspace(views))
    lib = L.load()
    for lam in (-0.1, 1.5, float("nan")):
        code = lib.gs_photometric_loss(img.data_ptr(), img.data_ptr(), views.ptr, 1, lam, ws.data_ptr(),
                                       ws.numel(), loss.data_ptr(), img.data_ptr(), None)
        assert code == L.GS_ERR_INVALID_ARG
    code = lib.gs_photometric_loss(img.data_ptr(), img.data_ptr(), views.ptr, 1, 0.8, ws.data_ptr(), 16,
                                   loss.data_ptr(), img.data_ptr(), None)
    assert code == L.GS_ERR_INVALID_ARG


def test_autograd_photometric_loss():
    wh = [(33, 20), (12, 41)]
    views = _views(wh)
    x, y = _pair(wh, 6, 0.1)
    img = torch.as_tensor(x).cuda().requires_grad_(True)
    loss = autograd.photometric_loss(img, torch.as_tensor(y).cuda(), views, lam=0.8)
    (3.0 * loss).backward()
    L_, d, _, _ = O.photometric(np.asarray(wh), x.astype(np.float64), y.astype(np.float64), 0.8)
    assert float(loss.detach()) == pytest.approx(L_, abs=LOSS_TOL * 2)
    assert_grad_close(to_np(img.grad), 3.0 * d, "autograd dL/dimage")


def test_mapping_step_with_the_full_objective():
    s = scenes.tiny_corridor(seed=0, n_anchors=4000, F=32, k=10, hidden=32)
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    tgt_host = torch.as_tensor(f32(O.targets_flat(s))).pin_memory()
    ref = pipeline.RenderPass(views, A, precision=L.GS_PREC_BF16, store_state=False, loss="photometric", lam=0.8)
    assert ref.ensure_capacity(tgt_host.cuda()) == 0
    ref.step(tgt_host.cuda())
    torch.cuda.synchronize()
    image = to_np(ref.image).astype(np.float64)
    L_, d, _, _ = O.photometric(np.asarray(s.wh), image, O.targets_flat(s), 0.8)
    assert float(ref.loss[0]) == pytest.approx(L_, abs=LOSS_TOL * views.V)
    assert_grad_close(to_np(ref.d_image), d, "dL/dimage")
    ms = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16, loss="photometric", lam=0.8)
    got = ms.step(tgt_host)
    assert got == pytest.approx(float(ref.loss[0]), rel=1e-5, abs=1e-6)
    assert np.allclose(to_np(ms.rp.agrad.dfeat), to_np(ref.agrad.dfeat), rtol=1e-4, atol=1e-6)
