"""BF16 tensor-core decoding: against the FP64 oracle within BF16 tolerances,
multi-partition decoding (Eq. 6) in both precisions, and the batched BF16 path
against the plain FP32 path (PSNR and gradient cosine)."""
import numpy as np
import pytest
import torch

from _helpers import to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, pipeline, scenes

pytestmark = pytest.mark.gpu


def small_partitions():
    # 16 lognormal partitions scaled down to a few thousand anchors each, mixed resolutions
    s = scenes.uneven_partitions(seed=0, scale_count=0.04, F=32, k=10, hidden=32, n_views=3)
    s.wh = np.array([[160, 64], [128, 64], [128, 96]], np.int32)
    s.cams[:, 0:2] = s.cams[:, 0:2] * 0.125
    s.cams[:, 2] = s.wh[:, 0] / 2.0
    s.cams[:, 3] = s.wh[:, 1] / 2.0
    s.targets = [np.random.default_rng(1).uniform(0, 1, (3, h, w)).astype(np.float32) for w, h in s.wh]
    return s


def gpu_decode(s, precision):
    A = api.Anchors.from_scene(s)
    vw = api.Views(s.cams, s.wh)
    cap = s.N * s.V
    g = api.Gauss3D.alloc(cap, s.k, s.V)
    st = api.new_status()
    api.decode(A, vw, g, api.workspace(api.decode_workspace(A, vw, cap)), st, precision)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    return g


@pytest.mark.parametrize("make", [lambda: scenes.tiny_corridor(seed=0, n_anchors=900, hidden=16),
                                  scenes.anchor_single_view, small_partitions])
def test_bf16_decode_close_to_oracle(make):
    s = make()
    g = gpu_decode(s, L.GS_PREC_BF16)
    dec = O.decode(s)
    R = dec.av_anchor.shape[0]
    assert np.array_equal(to_np(g.row_anchor)[:R], dec.av_anchor)
    C = R * s.k
    # BF16 inputs and weights (2^-9 relative rounding) through two layers
    assert np.abs(to_np(g.opacity)[:C] - dec.opacity).max() < 3e-2
    assert np.abs(to_np(g.colour)[:C] - dec.colour).max() < 3e-2
    assert np.abs(to_np(g.quat)[:C] - dec.quat).max() < 5e-2
    assert np.allclose(to_np(g.scale)[:C], dec.scale, rtol=3e-2, atol=1e-6)
    assert np.allclose(to_np(g.mu)[:C], dec.mu, rtol=1e-6, atol=1e-5)
    # typical error much smaller than the worst case
    assert np.abs(to_np(g.opacity)[:C] - dec.opacity).mean() < 3e-3


def test_multi_partition_decode_fp32_matches_oracle():
    s = small_partitions()
    assert s.M == 16
    g = gpu_decode(s, L.GS_PREC_FP32)
    dec = O.decode(s)
    R = dec.av_anchor.shape[0]
    parts = s.part[dec.av_anchor]
    assert len(np.unique(parts)) > 3
    assert np.array_equal(to_np(g.row_anchor)[:R], dec.av_anchor)
    C = R * s.k
    assert np.allclose(to_np(g.opacity)[:C], dec.opacity, atol=2e-5)
    assert np.allclose(to_np(g.colour)[:C], dec.colour, atol=2e-5)


def _run(s, precision, store, chunk=0):
    vw = api.Views(s.cams, s.wh)
    rp = pipeline.RenderPass(vw, api.Anchors.from_scene(s), precision=precision, store_state=store, chunk=chunk)
    tgt = torch.as_tensor(O.targets_flat(s).astype(np.float32)).cuda()
    assert rp.ensure_capacity(tgt) == 0
    rp.step(tgt)
    torch.cuda.synchronize()
    assert rp.check()[0] == 0
    return rp


def _psnr(a, b):
    mse = float(((a - b) ** 2).mean())
    return 10 * np.log10(1.0 / max(mse, 1e-30))


@pytest.mark.parametrize("make", [lambda: scenes.tiny_corridor(seed=0, n_anchors=4000, F=32, k=10, hidden=32),
                                  small_partitions])
def test_batched_bf16_path_matches_plain_fp32_path(make):
    """Batched BF16-decode pass (recomputed state) vs the plain FP32 pass:
    PSNR >= 45 dB and gradient cosine >= 0.999 for every anchor tensor and
    the MLP weights."""
    s = make()
    plain = _run(s, L.GS_PREC_FP32, True)
    batched = _run(s, L.GS_PREC_BF16, False, chunk=256)
    psnr = _psnr(to_np(batched.image), to_np(plain.image))
    assert psnr >= 45.0, f"PSNR {psnr:.2f} dB"
    for name in ("dxyz", "dfeat", "dlog_scaling", "doffsets", "dmlp"):
        a = to_np(getattr(batched.agrad, name)).ravel().astype(np.float64)
        b = to_np(getattr(plain.agrad, name)).ravel().astype(np.float64)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        assert cos >= 0.999, f"{name}: cosine {cos:.5f}"


@pytest.mark.parametrize("make", [lambda: scenes.tiny_corridor(seed=0, n_anchors=900, hidden=16),
                                  scenes.anchor_single_view, small_partitions])
def test_bf16_decode_bwd_close_to_oracle(make):
    """BF16 tensor-core reverse of the decoders against the FP64 oracle on the
    same upstream gradients: cosine >= 0.999 and relative error <= 3e-2 for
    every anchor tensor and the MLP weights."""
    s = make()
    A = api.Anchors.from_scene(s)
    vw = api.Views(s.cams, s.wh)
    cap = s.N * s.V
    g = api.Gauss3D.alloc(cap, s.k, s.V)
    st = api.new_status()
    api.decode(A, vw, g, api.workspace(api.decode_workspace(A, vw, cap)), st, L.GS_PREC_BF16)
    dec = O.decode(s)
    Cn = dec.opacity.shape[0]
    rng = np.random.default_rng(4)
    # upstream only where both precisions keep the candidate (opacity sign agrees)
    live = ((dec.opacity > 0) & (to_np(g.opacity)[:Cn] > 0) & (np.abs(dec.opacity) > 3e-2)).astype(np.float64)
    up = dict(mu=rng.normal(size=(Cn, 3)) * live[:, None], scale=rng.normal(size=(Cn, 3)) * live[:, None],
              quat=rng.normal(size=(Cn, 4)) * live[:, None], opacity=rng.normal(size=Cn) * live,
              colour=rng.normal(size=(Cn, 3)) * live[:, None])
    up = {k_: v.astype(np.float32) for k_, v in up.items()}
    dg = api.Gauss3DGrad.like(g)
    for name, t in (("mu", dg.dmu), ("scale", dg.dscale), ("quat", dg.dquat), ("opacity", dg.dopacity),
                    ("colour", dg.dcolour)):
        t.zero_()
        t[:Cn] = torch.as_tensor(up[name]).cuda()
    out = api.AnchorGrad.like(A)
    api.decode_bwd(A, vw, g, dg, out, api.workspace(api.decode_bwd_workspace(A, vw, cap)), st, L.GS_PREC_BF16)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    want = O.decode_bwd(s, dec, up["mu"], up["scale"], up["quat"], up["opacity"], up["colour"])
    for name, key in (("dxyz", "xyz"), ("dfeat", "feat"), ("dlog_scaling", "log_scaling"),
                      ("doffsets", "offsets"), ("dmlp", "mlp")):
        a = to_np(getattr(out, name)).ravel().astype(np.float64)
        b = want[key].ravel()
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300)
        assert cos >= 0.999 and rel <= 3e-2, f"{name}: cosine {cos:.5f}, relative error {rel:.3e}"


@pytest.mark.parametrize("make", [lambda: scenes.tiny_corridor(seed=0, n_anchors=900, hidden=16),
                                  scenes.anchor_single_view, small_partitions])
def test_bf16_fused_projection_and_decode_bwd(make):
    """gs_decode_project_bwd with the tensor-core decoder (the projection's
    chain rule applied inside the reverse decoder to the recomputed
    Gaussians) against the FP64 oracle's projection and decoder reverse on
    the same splat gradients (cosine >= 0.999, relative error <= 3e-2), and
    against the unfused GPU path (gs_project_bwd then gs_decode_bwd) on the
    same inputs (cosine >= 0.9999)."""
    s = make()
    A = api.Anchors.from_scene(s)
    vw = api.Views(s.cams, s.wh)
    cap = s.N * s.V
    g = api.Gauss3D.alloc(cap, s.k, s.V)
    st = api.new_status()
    api.decode(A, vw, g, api.workspace(api.decode_workspace(A, vw, cap)), st, L.GS_PREC_BF16)
    sp = api.Splats.alloc(cap * s.k)
    api.project(g, vw, sp, st)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    dec = O.decode(s)
    prj = O.project(dec.mu, dec.scale, dec.quat, dec.opacity, s.cams, s.wh, dec.view_start, s.k)
    Cn = dec.opacity.shape[0]
    tiles = to_np(sp.tiles)[:Cn]
    # splat gradients where both sides draw the candidate, away from every threshold
    keep = ((prj.tiles > 0) & (tiles > 0) & (prj.flag == 0) & (dec.cand_flag == 0) &
            (np.abs(dec.opacity) > 3e-2)).astype(np.float64)
    assert keep.sum() > 100
    rng = np.random.default_rng(6)
    sg = (rng.normal(size=(Cn, 9)) * keep[:, None]).astype(np.float32)
    sg[:, 2:5] *= 1e-2   # conic gradients at the scale of the mean gradients
    sgrad = torch.zeros(cap * s.k, 9, device="cuda")
    sgrad[:Cn] = torch.as_tensor(sg).cuda()
    fused = api.AnchorGrad.like(A)
    api.decode_project_bwd(A, vw, g, sp, sgrad, fused, api.workspace(api.decode_project_bwd_workspace(g, L.GS_PREC_BF16)),
                           st, L.GS_PREC_BF16)
    # the same gradients in row tiles of 128 ([tile][i][9][128]): read in place, no workspace
    nt = (cap + 127) // 128
    sgt = np.zeros((nt * 128, s.k, 9), np.float32)
    sgt[:cap] = to_np(sgrad).reshape(cap, s.k, 9)
    sgt = np.ascontiguousarray(sgt.reshape(nt, 128, s.k, 9).transpose(0, 2, 3, 1))
    tiled = api.AnchorGrad.like(A)
    api.decode_project_bwd(A, vw, g, sp, torch.as_tensor(sgt).cuda(), tiled, None, st, L.GS_PREC_BF16, None,
                           L.GS_SGRAD_ROW_TILES)
    dg = api.Gauss3DGrad.like(g)
    api.project_bwd(g, sp, vw, sgrad, dg, st)
    unfused = api.AnchorGrad.like(A)
    api.decode_bwd(A, vw, g, dg, unfused, api.workspace(api.decode_bwd_workspace(A, vw, cap)), st, L.GS_PREC_BF16)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    sg64 = sg.astype(np.float64)
    dmu, ds, dq = O.project_bwd(dec.mu, dec.scale, dec.quat, prj.status * (prj.tiles > 0), s.cams, s.wh,
                                dec.view_start, sg64[:, 0:2], sg64[:, 2:5], s.k)
    want = O.decode_bwd(s, dec, dmu, ds, dq, sg64[:, 5], sg64[:, 6:9])
    for name, key in (("dxyz", "xyz"), ("dfeat", "feat"), ("dlog_scaling", "log_scaling"),
                      ("doffsets", "offsets"), ("dmlp", "mlp")):
        a = to_np(getattr(fused, name)).ravel().astype(np.float64)
        b = want[key].ravel()
        u = to_np(getattr(unfused, name)).ravel().astype(np.float64)
        cos = a @ b / (np.linalg.norm(a) * np.linalg.norm(b) + 1e-300)
        rel = np.linalg.norm(a - b) / (np.linalg.norm(b) + 1e-300)
        cos_u = a @ u / (np.linalg.norm(a) * np.linalg.norm(u) + 1e-300)
        print(f"[fused] {name}: cosine {cos:.6f} / {cos_u:.7f} (oracle / unfused), relative error {rel:.3e}")
        assert cos >= 0.999 and rel <= 3e-2, f"{name}: cosine {cos:.5f}, relative error {rel:.3e}"
        assert cos_u >= 0.9999, f"{name}: cosine to the unfused path {cos_u:.6f}"
        t = to_np(getattr(tiled, name)).ravel().astype(np.float64)   # same sums, other atomic order
        assert np.linalg.norm(t - a) <= 1e-5 * (np.linalg.norm(a) + 1e-30), f"{name}: row-tiled input differs"
