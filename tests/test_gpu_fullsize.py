"""Parity at the full size of the 8-keyframe mapping batch (200k anchors,
8 x 1241x376, BF16 decoding, state recomputed), run through the same
graph-captured iteration the benchmark times, checked stage by stage on
sampled outputs the FP64 oracle computes one by one, and on properties that
hold at any size:

  a0  visibility rows: exact against the oracle (near-threshold rows excepted)
  a1  decoded candidates of 3000 sampled rows (BF16 tolerances)
  a2  splat records of sampled candidates, projected by the oracle from the
      GPU's decoded Gaussians
  a3  all 12M pairs: each (splat, tile) pair exactly once, every pair inside
      its splat's rectangle, per-splat counts, ranges partitioning the pairs,
      (depth bits, id) order inside every tile
  a4  24 sampled tiles composited by the oracle from the GPU's lists
  a6  the render backward of an image gradient confined to those tiles
  a7  the decode backward of candidate gradients confined to the sampled rows
"""
import numpy as np
import pytest
import torch

from _helpers import PIX_TOL, assert_grad_close, f32, image_mask, to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, pipeline, scenes

pytestmark = pytest.mark.gpu


def u32(t):
    return to_np(t).view(np.uint32)


@pytest.fixture(scope="module")
def run():
    s = scenes.keyframe_batch(seed=0)
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    ms = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16, cap_rows=int(1.2 * s.N * 0.6 * views.V))
    tgt_host = torch.from_numpy(np.concatenate([t.reshape(-1) for t in s.targets]).astype(np.float32)).pin_memory()
    ms.step(tgt_host)
    torch.cuda.synchronize()
    return s, views, A, ms, decoded(ms, A, views)


def decoded(ms, A, views):
    """The batch's decoded Gaussians: the benchmarked step decodes and projects
    in one kernel and keeps no 3D Gaussians, so the tests decode again (same
    BF16 decoder, same rows) to check them and the projection."""
    g = api.Gauss3D.alloc(ms.rp.cap_rows, A.k, views.V)
    st = api.new_status()
    api.decode(A, views, g, ms.rp.dec_ws, st, L.GS_PREC_BF16)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    assert torch.equal(g.view_start, ms.rp.g.view_start)
    return g


def _records(rec):
    """Oracle-side splat inputs from the library's FP32 records (as doubles)."""
    r = rec.astype(np.float64)
    l2e = 1.0 / np.log(2.0)
    conic = np.stack([-2.0 * r[:, 2] / l2e, -r[:, 3] / l2e, -2.0 * r[:, 4] / l2e], 1)
    rx, ry = rec[:, 10].view(np.uint32), rec[:, 11].view(np.uint32)
    rect = np.stack([rx & 0xFFFF, ry & 0xFFFF, rx >> 16, ry >> 16], 1).astype(np.int32)
    return dict(mean2d=r[:, 0:2], conic=conic, opacity=np.exp2(r[:, 5]), colour=r[:, 6:9],
                depth_bits=rec[:, 9].view(np.uint32), rect=rect)


def _sample_rows(R, n, seed):
    return np.sort(np.random.default_rng(seed).choice(R, size=min(n, R), replace=False))


def _row_subset(rows, view_start, row_anchor):
    """Oracle row list (anchors grouped by view) of the given GPU rows."""
    v = np.searchsorted(view_start, rows, side="right") - 1
    vs = np.zeros(len(view_start), np.int64)
    np.add.at(vs, v + 1, 1)
    return row_anchor[rows].astype(np.int32), np.cumsum(vs), np.zeros(len(rows), np.uint8)


def test_visibility_rows_exact(run):
    s, views, A, ms, gdec = run
    vs_g = to_np(ms.rp.g.view_start).astype(np.int64)
    R = int(vs_g[-1])
    ra = to_np(ms.rp.g.row_anchor)[:R]
    av, vs, rf = O.visibility(s.xyz, s.cams, s.wh)
    assert R > 700_000
    gpu = set(zip(np.searchsorted(vs_g, np.arange(R), side="right") - 1, ra))
    ora = set(zip(np.searchsorted(vs, np.arange(len(av)), side="right") - 1, av))
    flagged = set(zip(np.searchsorted(vs, np.nonzero(rf)[0], side="right") - 1, av[rf.astype(bool)]))
    assert (gpu ^ ora) <= flagged


def test_decode_sampled_rows(run):
    s, views, A, ms, gdec = run
    g = gdec
    vs_g = to_np(g.view_start).astype(np.int64)
    rows = _sample_rows(int(vs_g[-1]), 3000, 1)
    dec = O.decode(s, rows=_row_subset(rows, vs_g, to_np(g.row_anchor)))
    c = (rows[:, None] * s.k + np.arange(s.k)[None, :]).ravel()
    assert np.abs(to_np(g.opacity)[c] - dec.opacity).max() < 3e-2
    assert np.abs(to_np(g.colour)[c] - dec.colour).max() < 3e-2
    assert np.abs(to_np(g.quat)[c] - dec.quat).max() < 5e-2
    assert np.allclose(to_np(g.scale)[c], dec.scale, rtol=3e-2, atol=1e-6)
    assert np.allclose(to_np(g.mu)[c], dec.mu, rtol=1e-6, atol=2e-5)
    assert np.abs(to_np(g.opacity)[c] - dec.opacity).mean() < 3e-3


def _at(t, idx):
    """Host copy of t[idx], gathered on the device (the buffers can hold 10^8 rows)."""
    return to_np(t[torch.as_tensor(np.asarray(idx, np.int64)).to(t.device)])


def check_projection(s, views, g, rp, n, seed):
    """Splat records of n sampled candidates against the oracle's projection
    of the GPU's own decoded Gaussians g (3DGS preliminaries of Sec. III-A)."""
    vs_g = to_np(g.view_start).astype(np.int64)
    C_ = int(vs_g[-1]) * s.k
    cand = _sample_rows(C_, n, seed)
    cand = cand[_at(g.opacity, cand) > 0]
    v = np.searchsorted(vs_g * s.k, cand, side="right") - 1
    vs_sub = np.concatenate([[0], np.cumsum(np.bincount(v, minlength=views.V))]).astype(np.int64)
    mu, sc, q, op = (_at(t, cand).astype(np.float64) for t in (g.mu, g.scale, g.quat, g.opacity))
    prj = O.project(mu, sc, q, op, s.cams, s.wh, vs_sub, 1)
    rec = _at(rp.splats.rec, cand)
    tiles = _at(rp.splats.tiles, cand)
    ok = prj.flag == 0
    assert ok.mean() > 0.95
    assert np.array_equal(tiles[ok], prj.tiles[ok])
    live = ok & (prj.tiles > 0)
    assert live.sum() > 1000
    r = _records(rec)
    # FP32 bound: the camera-space point R mu + t of world coordinates ~1e3 m
    # carries ~|R||mu| + |t| times 2^-24 absolute error, relative to its depth z
    cams = np.asarray(s.cams, np.float64)[v]
    t = cams[:, 13:16]
    z = prj.depth
    rel_z = 8 * 2.0 ** -24 * (np.abs(mu).sum(1) + np.abs(t).sum(1)) / z
    f = cams[:, 0:2]
    uv = np.abs((prj.mean2d - cams[:, 2:4]) / f)
    tol_px = f * rel_z[:, None] * (1 + uv) + 1e-4
    assert np.all(np.abs(r["mean2d"] - prj.mean2d)[live] <= tol_px[live])
    scale = np.max(np.abs(prj.conic[live]), axis=1, keepdims=True)
    assert np.all(np.abs(r["conic"][live] - prj.conic[live]) <= (2e-5 + 8 * rel_z[live, None]) * scale)
    # opacity (log2 in the record) and colour pass through unchanged
    # (the record keeps log2 of the opacity: two ulps of log2 relative to its magnitude)
    lg = np.maximum(1.0, np.abs(np.log2(op[live])))
    assert np.all(np.abs(r["opacity"][live] / op[live] - 1.0) <= 4 * 2.0 ** -24 * lg + 1e-7)
    assert np.array_equal(rec[live, 6:9], _at(g.colour, cand)[live])
    # the depth key is the camera-space z
    assert np.all(np.abs(rec[live, 9] - z[live]) <= (4 * 2.0 ** -24 + rel_z[live]) * z[live])
    # rectangles: equal except where that position error moves a bound across a tile edge
    same = np.all(r["rect"] == prj.rect, axis=1)
    assert same[live].mean() > 0.999


def check_pairs(s, views, rp, min_pairs):
    """Invariants of all (tile, splat) pairs, checked on the device: ranges
    partition the pairs in tile order; every pair lies inside its splat's tile
    rectangle in the splat's own view; per-splat pair counts equal the tiles
    the rectangle covers; (depth bits, id) strictly increase inside every tile
    (so no pair repeats).  Together: each (splat, covered tile) exactly once,
    in the order of the (tile, depth, id) key."""
    dev = rp.bins.vals.device
    P = int(rp.bins.n_pairs.item())
    assert P > min_pairs
    i64 = lambda t: t.to(torch.int64) & 0xFFFFFFFF
    vals = i64(rp.bins.vals[:P])
    ranges = i64(rp.bins.ranges.view(-1, 2))
    T = ranges.shape[0]
    lens = ranges[:, 1] - ranges[:, 0]
    assert bool((lens >= 0).all()) and int(lens.sum()) == P
    starts = torch.cumsum(lens, 0) - lens
    busy = lens > 0
    assert torch.equal(ranges[busy, 0], starts[busy])
    tile = torch.repeat_interleave(torch.arange(T, device=dev), lens)
    vs = rp.g.view_start.to(torch.int64)
    C_ = int(vs[-1]) * s.k
    tiles_touched = rp.splats.tiles[:C_].to(torch.int64)
    assert int(tiles_touched.sum()) == P
    assert bool((vals < C_).all())
    assert torch.equal(torch.bincount(vals, minlength=C_), tiles_touched)
    rec = rp.splats.rec.view(-1, 12)
    words = rec[:, 9:12].contiguous().view(torch.int32)
    rx, ry = i64(words[vals, 1]), i64(words[vals, 2])
    tb = torch.as_tensor(np.concatenate([[0], np.cumsum([((w + 15) // 16) * ((h + 15) // 16)
                                                         for w, h in views.wh])]), device=dev)
    tv = torch.searchsorted(tb, tile, right=True) - 1
    TX = torch.as_tensor(np.array([(w + 15) // 16 for w, h in views.wh]), device=dev)[tv]
    loc = tile - tb[tv]
    tx, ty = loc % TX, loc // TX
    inside = (tx >= (rx & 0xFFFF)) & (tx < (rx >> 16)) & (ty >= (ry & 0xFFFF)) & (ty < (ry >> 16))
    assert bool(inside.all())
    v_of_c = torch.searchsorted(vs * s.k, vals, right=True) - 1
    assert torch.equal(v_of_c, tv)
    key = i64(words[vals, 0]) * (1 << 32) + vals
    same = tile[1:] == tile[:-1]
    assert bool((key[1:][same] > key[:-1][same]).all())


def test_project_sampled_candidates(run):
    s, views, A, ms, gdec = run
    check_projection(s, views, gdec, ms.rp, 20000, 2)


def test_bin_sort_invariants_all_pairs(run):
    s, views, A, ms, gdec = run
    check_pairs(s, views, ms.rp, 10_000_000)


def _sampled_tiles(ms, views, n_per_view=3, seed=3):
    ranges = u32(ms.rp.bins.ranges).astype(np.int64)
    lens = ranges[:, 1] - ranges[:, 0]
    tb = np.concatenate([[0], np.cumsum([((w + 15) // 16) * ((h + 15) // 16) for w, h in views.wh])])
    rng = np.random.default_rng(seed)
    out = []
    for v in range(views.V):
        t0, t1 = tb[v], tb[v + 1]
        heavy = t0 + int(np.argmax(lens[t0:t1]))
        busy = np.nonzero(lens[t0:t1] > 0)[0] + t0
        out += [heavy] + list(rng.choice(busy, size=n_per_view - 1, replace=False))
    return np.array(sorted(set(out)))


def _compact(ms, tiles_sel):
    """Oracle inputs restricted to the sampled tiles: their lists, with the
    splats they use renumbered 0..n-1."""
    ranges = u32(ms.rp.bins.ranges).astype(np.int64)
    vals = u32(ms.rp.bins.vals)
    used = np.unique(np.concatenate([vals[ranges[t, 0]:ranges[t, 1]] for t in tiles_sel]))
    remap = {int(c): i for i, c in enumerate(used)}
    r_sub = np.zeros_like(ranges)
    v_sub = []
    pos = 0
    sel = set(tiles_sel.tolist())
    for t in range(len(ranges)):
        if t in sel:
            lst = [remap[int(c)] for c in vals[ranges[t, 0]:ranges[t, 1]]]
            r_sub[t] = (pos, pos + len(lst))
            v_sub += lst
            pos += len(lst)
        else:
            r_sub[t] = (pos, pos)
    return used, r_sub.astype(np.uint32), np.array(v_sub, np.uint32)


def _tile_pixel_mask(views, tiles_sel):
    m = np.zeros(views.total_pixels, bool)
    tb = np.concatenate([[0], np.cumsum([((w + 15) // 16) * ((h + 15) // 16) for w, h in views.wh])])
    for t in tiles_sel:
        v = int(np.searchsorted(tb, t, side="right") - 1)
        w, h = (int(x) for x in views.wh[v])
        TX = (w + 15) // 16
        loc = t - tb[v]
        x0, y0 = (loc % TX) * 16, (loc // TX) * 16
        img = np.zeros((h, w), bool)
        img[y0:y0 + 16, x0:x0 + 16] = True
        m[int(views.pix_base[v]):int(views.pix_base[v + 1])] |= img.reshape(-1)
    return m


def test_render_sampled_tiles_forward_and_backward(run):
    s, views, A, ms, gdec = run
    rp = ms.rp
    tiles_sel = _sampled_tiles(ms, views)
    used, r_sub, v_sub = _compact(ms, tiles_sel)
    assert len(v_sub) > 20_000
    rec = to_np(rp.splats.rec)[used]
    r = _records(rec)
    one_view = np.array([0] + [len(used)] * views.V, np.int64)
    ren = O.render(s.wh, one_view, 1, r["mean2d"], r["conic"], r["opacity"], r["colour"], r["depth_bits"],
                   r["rect"], np.ones(len(used), np.int32), 0, r_sub, v_sub)
    pm = _tile_pixel_mask(views, tiles_sel)
    ok = pm & (ren.pix_flag == 0)
    assert ok.sum() > 0.97 * pm.sum()
    m = image_mask(s.wh, ok)
    err = np.abs(to_np(rp.image) - ren.image)[m]
    assert err.max() <= PIX_TOL, f"max pixel error {err.max():.3e}"
    # backward of an image gradient on those tiles, same launch as the batched iteration
    dimg = np.random.default_rng(4).normal(size=3 * views.total_pixels) * m
    sgrad = torch.zeros_like(rp.sgrad)
    out = api.Gauss3DGrad.like(gdec)
    st = api.new_status()
    api.render_bwd(gdec, rp.splats, rp.bins, views, rp.image, torch.as_tensor(f32(dimg)).cuda(), sgrad, out, st,
                   rp.render_ws, rp.chunk)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    dm, dk, do, dc = O.render_bwd(s.wh, r["mean2d"], r["conic"], r["opacity"], r["colour"], r_sub, v_sub,
                                  f32(dimg).astype(np.float64))
    sg = to_np(sgrad)
    assert_grad_close(sg[used, 0:2], dm, "dmean2d")
    assert_grad_close(sg[used, 2:5], dk, "dconic")
    assert_grad_close(sg[used, 5], do, "dopacity")
    assert_grad_close(sg[used, 6:9], dc, "dcolour")
    rest = np.ones(sg.shape[0], bool)
    rest[used] = False
    assert np.abs(sg[rest]).max() == 0.0
    # projection chain rule of those splats, from the GPU's decoded Gaussians
    g = gdec
    vs_c = to_np(g.view_start).astype(np.int64) * s.k
    v = np.searchsorted(vs_c, used, side="right") - 1
    vs_sub = np.concatenate([[0], np.cumsum(np.bincount(v, minlength=views.V))]).astype(np.int64)
    mu, sc, q = (to_np(t)[used].astype(np.float64) for t in (g.mu, g.scale, g.quat))
    dmu, ds, dq = O.project_bwd(mu, sc, q, np.ones(len(used), np.int32), s.cams, s.wh, vs_sub,
                                sg[used, 0:2].astype(np.float64), sg[used, 2:5].astype(np.float64), 1)
    assert_grad_close(to_np(out.dmu)[used], dmu, "dmu")
    assert_grad_close(to_np(out.dscale)[used], ds, "dscale")
    assert_grad_close(to_np(out.dquat)[used], dq, "dquat")


def test_decode_bwd_sampled_rows(run):
    s, views, A, ms, gdec = run
    g = gdec
    vs_g = to_np(g.view_start).astype(np.int64)
    rows = _sample_rows(int(vs_g[-1]), 3000, 5)
    dec = O.decode(s, rows=_row_subset(rows, vs_g, to_np(g.row_anchor)))
    c = (rows[:, None] * s.k + np.arange(s.k)[None, :]).ravel()
    live = ((dec.opacity > 3e-2) & (to_np(g.opacity)[c] > 3e-2)).astype(np.float64)
    rng = np.random.default_rng(6)
    n = len(c)
    up = dict(mu=rng.normal(size=(n, 3)) * live[:, None], scale=rng.normal(size=(n, 3)) * live[:, None],
              quat=rng.normal(size=(n, 4)) * live[:, None], opacity=rng.normal(size=n) * live,
              colour=rng.normal(size=(n, 3)) * live[:, None])
    up = {k_: v.astype(np.float32) for k_, v in up.items()}
    dg = api.Gauss3DGrad.like(g)
    for name, t in (("mu", dg.dmu), ("scale", dg.dscale), ("quat", dg.dquat), ("opacity", dg.dopacity),
                    ("colour", dg.dcolour)):
        t.zero_()
        t[torch.as_tensor(c).cuda()] = torch.as_tensor(up[name]).cuda()
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
