"""CUDA path vs the FP64 oracle, stage by stage and end to end, through the
C ABI.  Each stage is fed the oracle's own previous-stage output rounded to
FP32, so a mismatch points at one kernel."""
import numpy as np
import pytest
import torch

from _helpers import (PIX_TOL, assert_grad_close, f32, image_mask, pack_records, rounded_projection,
                      tile_mask_from_splats, to_np, u32)
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, pipeline, scenes

pytestmark = pytest.mark.gpu


def explicit_1():
    return scenes.explicit_frustum(seed=0)


def explicit_ragged():
    return scenes.explicit_frustum(seed=7, n=3000, width=83, height=61, fx=70.0, fy=75.0, cx=41.0, cy=30.5)


def tiny():
    return scenes.tiny_corridor(seed=0, n_anchors=900)


def explicit_dense_tiles(n=80000, seed=21):
    """80k small, faint splats clustered on a 64x48 view: eight of its twelve
    tiles hold 39-144 chunks of 256 (the segmented combine), and pixels stop in
    chunks of every segment of them while others never stop."""
    s = scenes.explicit_frustum(seed=seed, n=n, width=64, height=48, fx=64.0, fy=64.0, cx=32.0, cy=24.0)
    rng = np.random.default_rng(seed + 1)
    u = np.clip(32.0 + rng.normal(0.0, 12.0, n), 0.0, 63.9)
    v = np.clip(24.0 + rng.normal(0.0, 9.0, n), 0.0, 47.9)
    z = s.mu[:, 2].astype(np.float64)
    s.mu = np.stack([(u - 32.0) / 64.0 * z, (v - 24.0) / 64.0 * z, z], 1).astype(np.float32)
    s.scale = np.exp(rng.normal(-3.0, 0.3, (n, 3))).astype(np.float32)
    s.opacity = rng.uniform(0.02, 0.1, n).astype(np.float32)
    return s


EXPLICIT = [explicit_1, explicit_ragged]


def oracle_explicit(s):
    vs = np.array([0, s.mu.shape[0]], np.int64)
    prj = O.project(s.mu, s.scale, s.quat, s.opacity, s.cams, s.wh, vs)
    keys, vals, ranges = O.bin_sort(prj.depth_bits, prj.rect, s.wh, vs)
    return vs, prj, keys, vals, ranges


def gpu_bins_from(keys, vals, ranges, total_tiles):
    b = api.Bins.alloc(len(vals), total_tiles, keys=False)
    b.vals[: len(vals)] = torch.as_tensor(vals.view(np.int32)).cuda()
    b.ranges.copy_(torch.as_tensor(ranges.astype(np.uint32).view(np.int32)).cuda())
    b.n_pairs.fill_(len(vals))
    return b


def gpu_splats_from(rec, tiles):
    return api.Splats(torch.as_tensor(rec).cuda().contiguous(), torch.as_tensor(tiles).cuda().contiguous())


# ------------------------------------------------------------------ project
@pytest.mark.parametrize("make", EXPLICIT)
def test_project_matches_oracle(make):
    s = make()
    vw = api.Views(s.cams, s.wh)
    g = api.Gauss3D.explicit(s.mu, s.scale, s.quat, s.opacity, s.colour)
    sp = api.Splats.alloc(s.mu.shape[0])
    st = api.new_status()
    api.project(g, vw, sp, st)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    rec, tiles = to_np(sp.rec), to_np(sp.tiles)
    _, prj, _, _, _ = oracle_explicit(s)
    ok = prj.flag == 0
    assert ok.mean() > 0.95
    assert np.array_equal(tiles[ok], prj.tiles[ok])
    v = ok & (prj.tiles > 0)
    assert v.sum() > 100
    assert np.allclose(rec[v, 0:2], prj.mean2d[v], rtol=2e-6, atol=2e-5)
    l2e = 1.0 / np.log(2.0)
    r64 = rec.astype(np.float64)
    conic = np.stack([-2.0 * r64[:, 2] / l2e, -r64[:, 3] / l2e, -2.0 * r64[:, 4] / l2e], 1)
    scale = np.max(np.abs(prj.conic[v]), axis=1, keepdims=True)
    assert np.all(np.abs(conic[v] - prj.conic[v]) <= 2e-5 * scale)
    assert np.allclose(np.exp2(r64[v, 5]), s.opacity[v], rtol=2e-6) and np.allclose(rec[v, 6:9], s.colour[v])
    assert np.allclose(rec[v, 9], prj.depth[v], rtol=1e-6)
    rx = rec[v, 10].view(np.uint32)
    ry = rec[v, 11].view(np.uint32)
    assert np.array_equal(rx & 0xFFFF, prj.rect[v, 0]) and np.array_equal(rx >> 16, prj.rect[v, 2])
    assert np.array_equal(ry & 0xFFFF, prj.rect[v, 1]) and np.array_equal(ry >> 16, prj.rect[v, 3])


# ----------------------------------------------------------------- bin sort
def _bin_sort_case(s, rows_view_start, k, prj, opacity, colour):
    rec, tiles = pack_records(prj, opacity, colour)
    vw = api.Views(s.cams, s.wh)
    sp = gpu_splats_from(rec, tiles)
    P = int(prj.tiles.sum())
    bins = api.Bins.alloc(max(P, 1), vw.total_tiles, keys=True)
    vs_t = torch.as_tensor(np.asarray(rows_view_start, np.int32)).cuda()
    g = api.Gauss3D(k, int(rows_view_start[-1]), None, vs_t, *([torch.zeros(1, device="cuda")] * 5))
    ws = api.workspace(api.bin_sort_workspace(vw, len(tiles), max(P, 1)))
    st = api.new_status()
    api.bin_sort(sp, g, vw, bins, ws, st)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0, f"device status (code, site, index) = {api.read_status(st)}"
    keys, vals, ranges = O.bin_sort(prj.depth_bits, prj.rect, s.wh, rows_view_start, k)
    assert int(bins.n_pairs.item()) == P
    assert np.array_equal(to_np(bins.keys)[:P].view(np.uint64), keys)
    assert np.array_equal(u32(bins.vals)[:P], vals)
    assert np.array_equal(u32(bins.ranges), ranges)


@pytest.mark.parametrize("make", EXPLICIT)
def test_bin_sort_bit_exact_explicit(make):
    s = make()
    vs, prj, _, _, _ = oracle_explicit(s)
    _bin_sort_case(s, vs, 1, prj, s.opacity, s.colour)


def test_bin_sort_bit_exact_anchor_views():
    s = tiny()
    fw = O.forward_anchor(s)
    _bin_sort_case(s, fw.dec.view_start, s.k, fw.prj, fw.dec.opacity, fw.dec.colour)


def test_bin_sort_bit_exact_many_tiles_per_sort_block():
    """Enough splats (~700k) that every block of the radix passes walks several
    2048-element tiles, with dirty shared memory left by a previous kernel."""
    s = scenes.explicit_frustum(seed=11, n=700_000, width=1024, height=768, fx=600.0, fy=600.0,
                                cx=512.0, cy=384.0)
    s.scale *= 0.3
    vs, prj, _, _, _ = oracle_explicit(s)
    assert (prj.tiles > 0).sum() > 296 * 2048
    _bin_sort_case(s, vs, 1, prj, s.opacity, s.colour)


def test_bin_sort_bit_exact_depth_ties():
    """Equal depths: the tie is broken by splat id."""
    s = explicit_1()
    s.mu[:, 2] = np.round(s.mu[:, 2] * 2) / 2       # only 17 distinct depths
    s.mu[:, 0] = s.mu[:, 0] * 0 + np.repeat(np.linspace(-3, 3, 40), 50)[: s.mu.shape[0]]
    vs, prj, _, _, _ = oracle_explicit(s)
    assert len(np.unique(prj.depth_bits[prj.tiles > 0])) < 30
    _bin_sort_case(s, vs, 1, prj, s.opacity, s.colour)


# ------------------------------------------------------------ render forward
def _render_fwd_case(s, view_start, k, prj, opacity, colour, keys, vals, ranges, bg=(0.0, 0.0, 0.0), chunk=0,
                     min_ok=0.99):
    rec, tiles = pack_records(prj, opacity, colour)
    vw = api.Views(s.cams, s.wh)
    sp = gpu_splats_from(rec, tiles)
    bins = gpu_bins_from(keys, vals, ranges, vw.total_tiles)
    img = torch.zeros(3 * vw.total_pixels, device="cuda")
    Tf = torch.zeros(vw.total_pixels, device="cuda")
    last = torch.zeros(vw.total_pixels, device="cuda", dtype=torch.int32)
    nev = torch.zeros(4, device="cuda", dtype=torch.int64)
    st = api.new_status()
    ws = api.workspace(api.render_workspace(vw, bins.cap_pairs, chunk))
    api.render_fwd(sp, bins, vw, bg, img, st, ws, chunk, Tf, last, nev)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    r = rounded_projection(prj, opacity, colour)
    ren = O.render(s.wh, view_start, k, r["mean2d"], r["conic"], r["opacity"], r["colour"],
                   r["depth_bits"], r["rect"], r["status"], 0, ranges, vals, bg)
    ok = ren.pix_flag == 0
    assert ok.mean() > min_ok, f"near-threshold pixels {1 - ok.mean():.4%}"
    m = image_mask(s.wh, ok)
    err = np.abs(to_np(img) - ren.image)[m]
    assert err.max() <= PIX_TOL, f"max pixel error {err.max():.3e}"
    assert np.array_equal(to_np(last)[ok], ren.last[ok])
    assert np.allclose(to_np(Tf)[ok], ren.T_final[ok], rtol=1e-3, atol=1e-6)
    assert int(nev[0].item()) == pytest.approx(ren.nev, rel=1e-3)
    assert 0 < int(nev[1].item()) <= int(nev[0].item())
    # the same counts over the tiles whose list is a single work item
    lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
    L_ = chunk if chunk else L.DEFAULT_CHUNK
    assert 0 <= int(nev[2].item()) <= int(nev[0].item()) and 0 <= int(nev[3].item()) <= int(nev[1].item())
    if (lens <= L_).all():
        assert int(nev[2].item()) == int(nev[0].item()) and int(nev[3].item()) == int(nev[1].item())
    if chunk:
        lens = ranges[:, 1].astype(np.int64) - ranges[:, 0]
        assert (lens > chunk).any(), "case should contain tiles cut into several chunks"
    return sp, bins, img, to_np(last), ren, ws


@pytest.mark.parametrize("chunk", [0, 256])
@pytest.mark.parametrize("make", EXPLICIT)
def test_render_fwd_matches_oracle(make, chunk):
    s = make()
    vs, prj, keys, vals, ranges = oracle_explicit(s)
    _render_fwd_case(s, vs, 1, prj, s.opacity, s.colour, keys, vals, ranges, bg=(0.1, 0.3, 0.7), chunk=chunk)


@pytest.mark.parametrize("chunk", [0, 256])
def test_render_fwd_anchor_views_matches_oracle(chunk):
    s = tiny() if chunk == 0 else scenes.tiny_corridor(seed=0, n_anchors=4000)
    fw = O.forward_anchor(s)
    _render_fwd_case(s, fw.dec.view_start, s.k, fw.prj, fw.dec.opacity, fw.dec.colour, fw.keys,
                     fw.vals, fw.ranges, chunk=chunk)


# ----------------------------------------------------------- render backward
@pytest.mark.parametrize("make,store,chunk", [(explicit_1, True, 0), (explicit_1, False, 0),
                                              (explicit_ragged, False, 0), (explicit_1, True, 256),
                                              (explicit_1, False, 256), (explicit_ragged, False, 256),
                                              (explicit_dense_tiles, False, 256), (explicit_dense_tiles, True, 256)])
def test_render_bwd_matches_oracle(make, store, chunk):
    s = make()
    bg = (0.2, 0.1, 0.4)
    vs, prj, keys, vals, ranges = oracle_explicit(s)
    dense = make is explicit_dense_tiles
    if dense:   # tiles past the combine's long-tile threshold (32 chunks)
        assert ((ranges[:, 1].astype(np.int64) - ranges[:, 0]) > 32 * chunk).sum() >= 4
    sp, bins, img, last, ren, ws = _render_fwd_case(s, vs, 1, prj, s.opacity, s.colour, keys, vals, ranges, bg,
                                                    chunk, min_ok=0.95 if dense else 0.99)
    rng = np.random.default_rng(5)
    ok = ren.pix_flag == 0
    dimg = rng.normal(size=ren.image.shape) * image_mask(s.wh, ok)
    vw = api.Views(s.cams, s.wh)
    g = api.Gauss3D.explicit(s.mu, s.scale, s.quat, s.opacity, s.colour)
    sgrad = torch.zeros(s.mu.shape[0], 9, device="cuda")
    out = api.Gauss3DGrad.like(g)
    st = api.new_status()
    dimg_t = torch.as_tensor(f32(dimg)).cuda()
    if store:
        api.render_bwd(g, sp, bins, vw, img, dimg_t, sgrad, out, st, ws, chunk, torch.as_tensor(last).cuda())
    else:
        api.render_bwd(g, sp, bins, vw, img, dimg_t, sgrad, out, st, ws, chunk)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    r = rounded_projection(prj, s.opacity, s.colour)
    dm, dk, do, dc = O.render_bwd(s.wh, r["mean2d"], r["conic"], r["opacity"], r["colour"], ranges, vals,
                                  f32(dimg).astype(np.float64), bg)
    sg = to_np(sgrad)
    assert_grad_close(sg[:, 0:2], dm, "dmean2d")
    assert_grad_close(sg[:, 2:5], dk, "dconic")
    assert_grad_close(sg[:, 5], do, "dopacity")
    assert_grad_close(sg[:, 6:9], dc, "dcolour")
    dmu, ds, dq = O.project_bwd(s.mu, s.scale, s.quat, prj.status * (prj.tiles > 0), s.cams, s.wh, vs,
                                sg[:, 0:2].astype(np.float64), sg[:, 2:5].astype(np.float64))
    assert_grad_close(to_np(out.dmu), dmu, "dmu")
    assert_grad_close(to_np(out.dscale), ds, "dscale")
    assert_grad_close(to_np(out.dquat), dq, "dquat")
    assert np.array_equal(to_np(out.dopacity), sg[:, 5]) and np.array_equal(to_np(out.dcolour), sg[:, 6:9])


# ------------------------------------------------------------------- decode
@pytest.mark.parametrize("make", [tiny, scenes.anchor_single_view])
def test_decode_matches_oracle(make):
    s = make()
    A = api.Anchors.from_scene(s)
    vw = api.Views(s.cams, s.wh)
    cap = s.N * s.V
    g = api.Gauss3D.alloc(cap, s.k, s.V)
    ws = api.workspace(api.decode_workspace(A, vw, cap))
    st = api.new_status()
    api.decode(A, vw, g, ws, st)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    dec = O.decode(s)
    R = dec.av_anchor.shape[0]
    assert dec.row_flag.sum() == 0
    assert np.array_equal(to_np(g.view_start), dec.view_start.astype(np.int32))
    assert np.array_equal(to_np(g.row_anchor)[:R], dec.av_anchor)
    Cn = R * s.k
    assert np.allclose(to_np(g.mu)[:Cn], dec.mu, rtol=1e-6, atol=1e-5)
    assert np.allclose(to_np(g.scale)[:Cn], dec.scale, rtol=2e-5, atol=1e-7)
    assert np.allclose(to_np(g.quat)[:Cn], dec.quat, rtol=0, atol=2e-5)
    assert np.allclose(to_np(g.opacity)[:Cn], dec.opacity, rtol=0, atol=2e-5)
    assert np.allclose(to_np(g.colour)[:Cn], dec.colour, rtol=0, atol=2e-5)
    assert np.array_equal(to_np(g.opacity)[:Cn] > 0, dec.opacity > 0) or dec.cand_flag.any()


@pytest.mark.parametrize("make", [tiny, scenes.anchor_single_view])
def test_decode_bwd_matches_oracle(make):
    s = make()
    A = api.Anchors.from_scene(s)
    vw = api.Views(s.cams, s.wh)
    cap = s.N * s.V
    g = api.Gauss3D.alloc(cap, s.k, s.V)
    st = api.new_status()
    api.decode(A, vw, g, api.workspace(api.decode_workspace(A, vw, cap)), st)
    dec = O.decode(s)
    Cn = dec.opacity.shape[0]
    rng = np.random.default_rng(8)
    live = ((dec.opacity > 0) & (dec.cand_flag == 0)).astype(np.float64)
    up = dict(mu=rng.normal(size=(Cn, 3)) * live[:, None], scale=rng.normal(size=(Cn, 3)) * live[:, None],
              quat=rng.normal(size=(Cn, 4)) * live[:, None], opacity=rng.normal(size=Cn) * live,
              colour=rng.normal(size=(Cn, 3)) * live[:, None])
    up = {k_: f32(v) for k_, v in up.items()}
    dg = api.Gauss3DGrad.like(g)
    for name, t in (("mu", dg.dmu), ("scale", dg.dscale), ("quat", dg.dquat), ("opacity", dg.dopacity),
                    ("colour", dg.dcolour)):
        t.zero_()
        t[:Cn] = torch.as_tensor(up[name]).cuda()
    out = api.AnchorGrad.like(A)
    api.decode_bwd(A, vw, g, dg, out, api.workspace(api.decode_bwd_workspace(A, vw, cap)), st)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    want = O.decode_bwd(s, dec, up["mu"], up["scale"], up["quat"], up["opacity"], up["colour"])
    assert_grad_close(to_np(out.dxyz), want["xyz"], "dxyz")
    assert_grad_close(to_np(out.dfeat), want["feat"], "dfeat")
    assert_grad_close(to_np(out.dlog_scaling), want["log_scaling"], "dlog_scaling")
    assert_grad_close(to_np(out.doffsets), want["offsets"], "doffsets")
    assert_grad_close(to_np(out.dmlp), want["mlp"], "dmlp")


# --------------------------------------------------------------- end to end
def _e2e_masks(s, fw):
    ok = fw.ren.pix_flag == 0
    presence = (fw.prj.flag & 1).astype(bool)
    edge = (fw.prj.flag & 2).astype(bool)
    if fw.dec is not None:
        presence |= fw.dec.cand_flag.astype(bool) | np.repeat(fw.dec.row_flag.astype(bool), s.k)
    ok &= ~tile_mask_from_splats(s.wh, fw.view_start_c, fw.k, fw.prj.rect, presence, edge)
    return ok


@pytest.mark.parametrize("make,chunk,store", [(explicit_1, 0, True), (tiny, 0, True), (explicit_1, 256, False),
                                              (tiny, 256, False)])
def test_end_to_end(make, chunk, store):
    s = make()
    vw = api.Views(s.cams, s.wh)
    if s.xyz is None:
        fw = O.forward_explicit(s)
        rp = pipeline.RenderPass(vw, None, cap_rows=s.mu.shape[0], chunk=chunk, store_state=store)
        g = api.Gauss3D.explicit(s.mu, s.scale, s.quat, s.opacity, s.colour)
        rp.set_explicit(g)
    else:
        fw = O.forward_anchor(s)
        rp = pipeline.RenderPass(vw, api.Anchors.from_scene(s), chunk=chunk, store_state=store)
    tgt = O.targets_flat(s)
    assert rp.ensure_capacity() == 0
    img = rp.forward()
    rp.loss_l1(torch.as_tensor(f32(tgt)).cuda())
    torch.cuda.synchronize()
    ok = _e2e_masks(s, fw)
    assert ok.mean() > 0.97
    m = image_mask(s.wh, ok)
    err = np.abs(to_np(img) - fw.ren.image)[m]
    assert err.max() <= PIX_TOL, f"max pixel error {err.max():.3e}"
    L_o, dimg = O.l1(s.wh, fw.ren.image, tgt)
    assert float(rp.loss.item()) == pytest.approx(L_o, abs=1e-4)
    # same upstream gradient for both reverse passes (masked pixels zeroed)
    dimg = dimg * m
    rp.backward(torch.as_tensor(f32(dimg)).cuda())
    torch.cuda.synchronize()
    assert rp.check()[0] == 0
    dm, dk, do, dc = O.render_bwd(s.wh, fw.prj.mean2d, fw.prj.conic, fw.opacity, fw.colour, fw.ranges,
                                  fw.vals, dimg)
    if s.xyz is None:
        dmu, ds, dq = O.project_bwd(s.mu, s.scale, s.quat, fw.prj.status, s.cams, s.wh, fw.view_start_c,
                                    dm, dk)
        assert_grad_close(to_np(rp.ggrad.dmu), dmu, "dmu")
        assert_grad_close(to_np(rp.ggrad.dscale), ds, "dscale")
        assert_grad_close(to_np(rp.ggrad.dquat), dq, "dquat")
        assert_grad_close(to_np(rp.ggrad.dopacity), do, "dopacity")
        assert_grad_close(to_np(rp.ggrad.dcolour), dc, "dcolour")
    else:
        dmu, ds, dq = O.project_bwd(fw.dec.mu, fw.dec.scale, fw.dec.quat, fw.prj.status, s.cams, s.wh,
                                    fw.dec.view_start, dm, dk, s.k)
        want = O.decode_bwd(s, fw.dec, dmu, ds, dq, do, dc)
        for name, got in (("xyz", rp.agrad.dxyz), ("feat", rp.agrad.dfeat),
                          ("log_scaling", rp.agrad.dlog_scaling), ("offsets", rp.agrad.doffsets),
                          ("mlp", rp.agrad.dmlp)):
            assert_grad_close(to_np(got), want[name], "d" + name)


# ------------------------------------------------------------- capacities
def test_capacity_overflow_is_reported_and_recovered():
    s = tiny()
    vw = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    rp = pipeline.RenderPass(vw, A, cap_rows=10, cap_pairs=64)
    rp.forward()
    torch.cuda.synchronize()
    code, where, needed = rp.check()
    assert code == L.GS_ERR_CAPACITY and where == 1
    assert needed == O.visibility(s.xyz, s.cams, s.wh)[0].shape[0]
    assert rp.ensure_capacity() == 0
    ref = pipeline.RenderPass(vw, A)
    assert ref.ensure_capacity() == 0
    torch.cuda.synchronize()
    assert torch.equal(rp.forward(), ref.forward())
    # pair overflow
    rp2 = pipeline.RenderPass(vw, A, cap_pairs=8)
    rp2.forward()
    torch.cuda.synchronize()
    code, where, needed = rp2.check()
    assert code == L.GS_ERR_CAPACITY and where == 3
    assert needed == ref.n_pairs()


# ------------------------------------------------------------- edge cases
def test_everything_behind_camera_renders_background():
    s = explicit_1()
    s.mu[:, 2] = -s.mu[:, 2]
    vw = api.Views(s.cams, s.wh)
    rp = pipeline.RenderPass(vw, None, cap_rows=s.mu.shape[0], bg=(0.25, 0.5, 0.75))
    rp.set_explicit(api.Gauss3D.explicit(s.mu, s.scale, s.quat, s.opacity, s.colour))
    img = to_np(rp.forward()).reshape(3, -1)
    rp.backward(torch.ones(3 * vw.total_pixels, device="cuda"))
    torch.cuda.synchronize()
    assert rp.n_pairs() == 0
    assert np.allclose(img[0], 0.25) and np.allclose(img[1], 0.5) and np.allclose(img[2], 0.75)
    assert float(rp.ggrad.dmu.abs().max()) == 0.0


def test_no_visible_anchor():
    s = tiny()
    s.cams = np.stack([scenes.camera(60.0, 60.0, 36.0, 20.0, (0.0, 0.0, -5.0), 180.0),
                       scenes.camera(45.0, 45.0, 25.0, 17.0, (0.0, 0.0, -6.0), 180.0)])
    vw = api.Views(s.cams, s.wh)
    rp = pipeline.RenderPass(vw, api.Anchors.from_scene(s))
    img = rp.forward()
    rp.loss_l1(torch.zeros_like(img))
    rp.backward()
    torch.cuda.synchronize()
    assert rp.check()[0] == 0 and rp.n_rows() == 0
    assert float(img.abs().max()) == 0.0
    assert float(rp.agrad.dmlp.abs().max()) == 0.0


def test_invalid_arguments_are_rejected_on_the_host():
    s = explicit_1()
    vw = api.Views(s.cams, s.wh)
    g = api.Gauss3D.explicit(s.mu, s.scale, s.quat, s.opacity, s.colour)
    sp = api.Splats.alloc(s.mu.shape[0])
    bad = api.Splats(sp.rec.view(-1)[1:13].view(1, 12), sp.tiles)   # misaligned records
    with pytest.raises(L.GsError) as e:
        api.project(g, vw, bad, api.new_status())
    assert e.value.code == L.GS_ERR_INVALID_ARG
    with pytest.raises(ValueError):
        api.Views(np.zeros((0, 16)), np.zeros((0, 2)))


def test_l1_ragged_views_match_oracle():
    """Eq. 3's L1 term over views whose element counts are not multiples of
    four (view boundaries inside the kernel's 16-byte groups) and an odd
    total, against the oracle; the gradient is sign(d) / (3 H W) exactly."""
    wh = np.array([[29, 31], [16, 16], [7, 5]], np.int32)
    rng = np.random.default_rng(12)
    n = int(3 * (wh[:, 0] * wh[:, 1]).sum())
    x = rng.uniform(0, 1, n).astype(np.float32)
    y = rng.uniform(0, 1, n).astype(np.float32)
    y[::17] = x[::17]   # some exact zeros of the difference
    cams = np.stack([scenes.camera(30.0, 30.0, 14.5, 15.5, (0.0, 0.0, 0.0))] * 3)
    vw = api.Views(cams, wh)
    loss = torch.zeros(1, device="cuda")
    d = torch.zeros(n, device="cuda")
    api.l1_loss(torch.as_tensor(x).cuda(), torch.as_tensor(y).cuda(), vw, loss, d)
    torch.cuda.synchronize()
    want_loss, want_d = O.l1(wh, x.astype(np.float64), y.astype(np.float64))
    assert float(loss[0]) == pytest.approx(float(want_loss), rel=1e-5)
    assert np.array_equal(to_np(d), f32(want_d))


def test_bin_sort_bit_exact_three_tile_passes():
    """More than 2^16 tiles (40 views of 1241x376: 74,880 tiles), so the tile
    sort takes three 8-bit passes and the ranges come from the third."""
    V, n = 40, 1500
    s = scenes.explicit_frustum(seed=23, n=n, width=1241, height=376, fx=718.0, fy=718.0, cx=620.5, cy=188.0)
    s.scale *= 0.1
    s.cams = np.repeat(s.cams, V, axis=0)
    s.wh = np.repeat(s.wh, V, axis=0)
    for name in ("mu", "scale", "quat", "opacity", "colour"):
        setattr(s, name, np.tile(getattr(s, name), (V, 1)) if getattr(s, name).ndim == 2
                else np.tile(getattr(s, name), V))
    vs = np.arange(V + 1, dtype=np.int64) * n
    prj = O.project(s.mu, s.scale, s.quat, s.opacity, s.cams, s.wh, vs)
    assert api.Views(s.cams, s.wh).total_tiles > (1 << 16)
    _bin_sort_case(s, vs, 1, prj, s.opacity, s.colour)
