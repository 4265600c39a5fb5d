"""gs_render_bwd writing the splat gradients in row tiles of 128
(GS_SGRAD_ROW_TILES, the layout the fused tensor-core reverse decoder reads)
gives the candidate-major gradients rearranged, and the API takes each layout
only where it is supported."""
import numpy as np
import pytest
import torch

from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, pipeline, scenes

pytestmark = pytest.mark.gpu


def _pass(s):
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    rp = pipeline.RenderPass(views, A, precision=L.GS_PREC_BF16, cap_rows=s.N * views.V + 77)
    rp.forward()
    target = torch.rand(3 * views.total_pixels, device="cuda")
    rp.loss_l1(target)
    torch.cuda.synchronize()
    return views, A, rp


@pytest.mark.parametrize("make", [lambda: scenes.tiny_corridor(seed=3, n_anchors=2500),
                                  lambda: scenes.keyframe_batch(seed=1, n_anchors=20000, n_views=2)])
def test_row_tiled_splat_gradients_match_candidate_major(make):
    s = make()
    views, A, rp = _pass(s)
    g, k = rp.g, rp.k
    rows = int(g.view_start[-1].item())
    cand = api.splat_grad_alloc(g)
    tiled = api.splat_grad_alloc(g, L.GS_SGRAD_ROW_TILES)
    tiled.fill_(7.0)   # every entry up to the last tile of rows must be overwritten
    for sg, lay in ((cand, L.GS_SGRAD_CANDIDATE), (tiled, L.GS_SGRAD_ROW_TILES)):
        api.render_bwd(g, rp.splats, rp.bins, views, rp.image, rp.d_image, sg, None, rp.status, rp.render_ws,
                       rp.chunk, None, None, lay)
    torch.cuda.synchronize()
    assert api.read_status(rp.status)[0] == 0
    c = cand.cpu().numpy()[:rows * k].reshape(rows, k, 9)
    nt = (rows + 127) // 128
    t = tiled.cpu().numpy().ravel()[:nt * 128 * k * 9].reshape(nt, k, 9, 128).transpose(0, 3, 1, 2)
    t = t.reshape(nt * 128, k, 9)
    assert np.all(t[rows:] == 0.0), "rows past the row count in the last tile are zeroed"
    t = t[:rows]
    scale = np.abs(c).max()
    assert scale > 0
    assert np.abs(t - c).max() <= 1e-5 * scale, "same per-splat sums (atomic order aside)"


def test_layouts_are_checked_by_the_api():
    s = scenes.tiny_corridor(seed=4, n_anchors=600)
    views, A, rp = _pass(s)
    g = rp.g
    tiled = api.splat_grad_alloc(g, L.GS_SGRAD_ROW_TILES)
    out = api.Gauss3DGrad.like(g)
    # the projection chain rule inside render_bwd, gs_project_bwd and the FP32 fused reverse need [C][9]
    with pytest.raises(L.GsError):
        api.render_bwd(g, rp.splats, rp.bins, views, rp.image, rp.d_image, tiled, out, rp.status, rp.render_ws,
                       rp.chunk, None, None, L.GS_SGRAD_ROW_TILES)
    with pytest.raises(L.GsError):
        api.decode_project_bwd(A, views, g, rp.splats, tiled, rp.agrad, rp.dpbwd_ws, rp.status, L.GS_PREC_FP32,
                               None, L.GS_SGRAD_ROW_TILES)
    with pytest.raises(L.GsError):
        api.render_bwd(g, rp.splats, rp.bins, views, rp.image, rp.d_image, tiled, None, rp.status, rp.render_ws,
                       rp.chunk, None, None, 5)
