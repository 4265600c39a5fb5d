"""Parity at the full sizes of the larger mapping workloads, run through the
graph-captured MappingStep with BF16 decoding, on sampled outputs the FP64
oracle computes one by one:

  uneven partitions: 16 lognormal partitions (648k anchors), 16 keyframes at
      1241x376 / 1024x384 / 1024x768, 4.6M rows -- decode tiles that span
      several partitions (Eq. 6), mixed view sizes;
  loop road: 2M anchors on a 5 km loop with ground relief, 16 equal-arc
      partitions, 32 keyframes drawn by the recent-window rule, 17.1M rows.

Checked: visibility rows exact (near-threshold rows excepted); 1000 sampled
decoded rows; 20k sampled candidates projected by the oracle from the GPU's
decoded Gaussians; all pairs (each (splat, covered tile) once, inside the
splat's rectangle, (depth bits, id) order in every tile, ranges partitioning
the pairs); per view the heaviest tile and random busy tiles composited by
the oracle from the GPU's lists (every tile's list ordered by (depth bits, id));
the render backward of an image gradient confined to those tiles; the decode
backward of candidate gradients confined to the sampled rows."""
import numpy as np
import pytest
import torch

from _helpers import PIX_TOL, assert_grad_close, f32, image_mask, to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, pipeline, scenes
from test_gpu_fullsize import (_at, _records, _row_subset, _sample_rows, _tile_pixel_mask, check_pairs,
                               check_projection, decoded)

pytestmark = pytest.mark.gpu

CONFIGS = {"uneven_partitions": lambda: scenes.uneven_partitions(seed=0),
           "loop_road": lambda: scenes.loop_road(seed=0)}


@pytest.fixture(scope="module", params=sorted(CONFIGS))
def run(request):
    s = CONFIGS[request.param]()
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    # initial capacities near the expected sizes (about 0.3 rows per anchor and view, 20 pairs per
    # row); the step grows them if a capacity is exceeded
    cap_rows = int(0.3 * s.N * views.V)
    ms = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16, cap_rows=cap_rows)
    ms.rp.cap_pairs = 20 * cap_rows
    ms.rp._alloc()
    tgt_host = torch.from_numpy(np.concatenate([t.reshape(-1) for t in s.targets]).astype(np.float32)).pin_memory()
    ms.step(tgt_host)
    torch.cuda.synchronize()
    gdec = decoded(ms, A, views)
    yield s, views, A, ms, gdec
    del ms, gdec
    torch.cuda.empty_cache()


def _tiles_and_lists(ms, views, n_per_view, seed, n_views=6):
    """In n_views evenly spaced views, the heaviest tile and random busy tiles;
    their lists with the splats they use renumbered 0..n-1 (oracle inputs),
    read tile by tile."""
    ranges = to_np(ms.rp.bins.ranges).view(np.uint32).astype(np.int64)
    lens = ranges[:, 1] - ranges[:, 0]
    tb = np.concatenate([[0], np.cumsum([((w + 15) // 16) * ((h + 15) // 16) for w, h in views.wh])])
    rng = np.random.default_rng(seed)
    sel = []
    for v in np.unique(np.linspace(0, views.V - 1, min(n_views, views.V)).astype(int)):
        t0, t1 = tb[v], tb[v + 1]
        busy = np.nonzero(lens[t0:t1] > 0)[0] + t0
        sel += [t0 + int(np.argmax(lens[t0:t1]))] + list(rng.choice(busy, size=n_per_view - 1, replace=False))
    sel = np.array(sorted(set(sel)))
    lists = {int(t): to_np(ms.rp.bins.vals[int(ranges[t, 0]):int(ranges[t, 1])]).view(np.uint32) for t in sel}
    used = np.unique(np.concatenate(list(lists.values())))
    r_sub = np.zeros_like(ranges)
    v_sub, pos = [], 0
    for t in range(len(ranges)):
        if t in lists:
            lst = np.searchsorted(used, lists[t])
            r_sub[t] = (pos, pos + len(lst))
            v_sub.append(lst)
            pos += len(lst)
        else:
            r_sub[t] = (pos, pos)
    return sel, used, r_sub.astype(np.uint32), np.concatenate(v_sub).astype(np.uint32)


def test_visibility_rows_exact(run):
    s, views, A, ms, gdec = run
    vs_g = to_np(ms.rp.g.view_start).astype(np.int64)
    R = int(vs_g[-1])
    ra = to_np(ms.rp.g.row_anchor)[:R].astype(np.int64)
    av, vs, rf = O.visibility(s.xyz, s.cams, s.wh)
    gpu = (np.searchsorted(vs_g, np.arange(R), side="right") - 1) * s.N + ra
    ora = (np.searchsorted(vs, np.arange(len(av)), side="right") - 1) * s.N + av.astype(np.int64)
    flagged = ora[rf.astype(bool)]
    diff = np.setxor1d(gpu, ora)
    assert np.isin(diff, flagged).all()
    assert R > 4_000_000


def test_decode_sampled_rows(run):
    s, views, A, ms, gdec = run
    g = gdec
    vs_g = to_np(g.view_start).astype(np.int64)
    rows = _sample_rows(int(vs_g[-1]), 1000, 11)
    dec = O.decode(s, rows=_row_subset(rows, vs_g, to_np(g.row_anchor)))
    assert len(np.unique(s.part[dec.av_anchor])) > 4
    c = (rows[:, None] * s.k + np.arange(s.k)[None, :]).ravel()
    assert np.abs(_at(g.opacity, c) - dec.opacity).max() < 3e-2
    assert np.abs(_at(g.colour, c) - dec.colour).max() < 3e-2
    assert np.abs(_at(g.quat, c) - dec.quat).max() < 5e-2
    assert np.allclose(_at(g.scale, c), dec.scale, rtol=3e-2, atol=1e-6)
    assert np.allclose(_at(g.mu, c), dec.mu, rtol=1e-6, atol=5e-5)
    assert np.abs(_at(g.opacity, c) - dec.opacity).mean() < 3e-3


def test_project_sampled_candidates(run):
    s, views, A, ms, gdec = run
    check_projection(s, views, gdec, ms.rp, 20000, 16)


def test_bin_sort_invariants_all_pairs(run):
    s, views, A, ms, gdec = run
    check_pairs(s, views, ms.rp, 10_000_000)


def test_render_sampled_tiles(run):
    s, views, A, ms, gdec = run
    rp = ms.rp
    tiles_sel, used, r_sub, v_sub = _tiles_and_lists(ms, views, 2, 12)
    r = _records(_at(rp.splats.rec, used))
    # every sampled list is ordered by (depth bits, id)
    for t in tiles_sel:
        lst = v_sub[r_sub[t, 0]:r_sub[t, 1]].astype(np.int64)
        key = r["depth_bits"][lst].astype(np.int64) * (1 << 32) + used[lst]
        assert (np.diff(key) > 0).all()
    one_view = np.array([0] + [len(used)] * views.V, np.int64)
    ren = O.render(s.wh, one_view, 1, r["mean2d"], r["conic"], r["opacity"], r["colour"], r["depth_bits"],
                   r["rect"], np.ones(len(used), np.int32), 0, r_sub, v_sub)
    pm = _tile_pixel_mask(views, tiles_sel)
    ok = pm & (ren.pix_flag == 0)
    assert ok.sum() > 0.9 * pm.sum()   # heavy tiles carry more near-threshold (flagged) pixels
    m = image_mask(s.wh, ok)
    err = np.abs(to_np(rp.image) - ren.image)[m]
    assert err.max() <= PIX_TOL, f"max pixel error {err.max():.3e}"
    dimg = np.random.default_rng(13).normal(size=3 * views.total_pixels) * m
    sgrad = torch.zeros_like(rp.sgrad)
    out = api.Gauss3DGrad.like(gdec)
    st = api.new_status()
    api.render_bwd(gdec, rp.splats, rp.bins, views, rp.image, torch.as_tensor(f32(dimg)).cuda(), sgrad, out, st,
                   rp.render_ws, rp.chunk)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    dm, dk, do, dc = O.render_bwd(s.wh, r["mean2d"], r["conic"], r["opacity"], r["colour"], r_sub, v_sub,
                                  f32(dimg).astype(np.float64))
    sg = _at(sgrad, used)
    assert_grad_close(sg[:, 0:2], dm, "dmean2d")
    assert_grad_close(sg[:, 2:5], dk, "dconic")
    assert_grad_close(sg[:, 5], do, "dopacity")
    assert_grad_close(sg[:, 6:9], dc, "dcolour")
    # no other splat received a gradient
    assert float(sgrad.abs().sum()) == pytest.approx(float(np.abs(sg).astype(np.float64).sum()), rel=1e-5)


def test_decode_bwd_sampled_rows(run):
    s, views, A, ms, gdec = run
    g = gdec
    vs_g = to_np(g.view_start).astype(np.int64)
    rows = _sample_rows(int(vs_g[-1]), 1000, 14)
    dec = O.decode(s, rows=_row_subset(rows, vs_g, to_np(g.row_anchor)))
    c = (rows[:, None] * s.k + np.arange(s.k)[None, :]).ravel()
    live = ((dec.opacity > 3e-2) & (_at(g.opacity, c) > 3e-2)).astype(np.float64)
    rng = np.random.default_rng(15)
    n = len(c)
    up = dict(mu=rng.normal(size=(n, 3)) * live[:, None], scale=rng.normal(size=(n, 3)) * live[:, None],
              quat=rng.normal(size=(n, 4)) * live[:, None], opacity=rng.normal(size=n) * live,
              colour=rng.normal(size=(n, 3)) * live[:, None])
    up = {k_: v.astype(np.float32) for k_, v in up.items()}
    dg = api.Gauss3DGrad.like(g)
    idx = torch.as_tensor(c).cuda()
    for name, t in (("mu", dg.dmu), ("scale", dg.dscale), ("quat", dg.dquat), ("opacity", dg.dopacity),
                    ("colour", dg.dcolour)):
        t.zero_()
        t[idx] = torch.as_tensor(up[name]).cuda()
    out = api.AnchorGrad.like(A)
    st = api.new_status()
    api.decode_bwd(A, views, g, dg, out, ms.rp.dbwd_ws, st, L.GS_PREC_BF16)
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
