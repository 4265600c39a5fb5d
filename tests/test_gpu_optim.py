"""gs_adam_step, gs_densify_stats and gs_densify_masks against the FP64 oracle
on seeded synthetic inputs (none taken from the CUDA path): several tensors of
ragged sizes in one launch (one spanning many CTAs, one misaligned, one
empty), several steps; statistics accumulated over two calls with rows of
several views hitting the same anchors; masks bit-exact (the means are taken
in single precision on both sides); invalid arguments; and a few optimizer
steps of the mapping iteration lowering its loss."""
import numpy as np
import pytest
import torch

from _helpers import f32, to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, pipeline, scenes

pytestmark = pytest.mark.gpu


def test_adam_groups_match_oracle_over_steps():
    rng = np.random.default_rng(0)
    sizes = [100_003, 37, 0, 4096 * 3 + 5, 1]
    lrs = [0.01, 0.1, 0.5, 0.003, 1.0]
    base = torch.zeros(sum(sizes) + 1, device="cuda")   # group 1 starts at an odd float: scalar path
    params, grads, ms, vs, ref = [], [], [], [], []
    at = 0
    for i, n in enumerate(sizes):
        p0 = rng.normal(size=n)
        if i == 1:
            at += 1
        p = base[at:at + n] if i == 1 else torch.zeros(n, device="cuda")
        p.copy_(torch.as_tensor(f32(p0)))
        at += n if i == 1 else 0
        params.append(p)
        grads.append(torch.zeros(n, device="cuda"))
        ms.append(torch.zeros(n, device="cuda"))
        vs.append(torch.zeros(n, device="cuda"))
        ref.append([f32(p0).astype(np.float64), np.zeros(n), np.zeros(n)])
    for step in range(1, 5):
        for i, n in enumerate(sizes):
            g = f32(rng.normal(size=n) * (10.0 ** rng.uniform(-3, 1)))
            grads[i].copy_(torch.as_tensor(g))
            ref[i] = list(O.adam(ref[i][0], g.astype(np.float64), ref[i][1], ref[i][2], step, lrs[i],
                                 0.9, 0.999, 1e-8))
        api.adam_step([(params[i], grads[i], ms[i], vs[i], lrs[i]) for i in range(len(sizes))], step,
                      0.9, 0.999, 1e-8)
        torch.cuda.synchronize()
        for i, n in enumerate(sizes):
            if n == 0:
                continue
            assert np.allclose(to_np(params[i]), ref[i][0], rtol=2e-6, atol=2e-6 * lrs[i]), (step, i)
            # m = b1 m + (1 - b1) g cancels where g changes sign: absolute slack of FP32 rounding
            assert np.allclose(to_np(ms[i]), ref[i][1], rtol=1e-5, atol=1e-6 * np.abs(ref[i][1]).max()), (step, i)
            assert np.allclose(to_np(vs[i]), ref[i][2], rtol=1e-5, atol=1e-12), (step, i)


def test_adam_rejects_invalid_arguments():
    lib = L.load()
    p = torch.zeros(8, device="cuda")
    grp = (L.gs_adam_group * 1)(L.gs_adam_group(p.data_ptr(), p.data_ptr(), p.data_ptr(), p.data_ptr(), 8, 0.1))
    assert lib.gs_adam_step(grp, 1, 0, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG      # step 0
    assert lib.gs_adam_step(grp, 1, 1, 1.0, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG      # beta1 = 1
    assert lib.gs_adam_step(grp, 0, 1, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG      # no group
    many = (L.gs_adam_group * 17)(*[grp[0]] * 17)
    assert lib.gs_adam_step(many, 17, 1, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG
    bad = (L.gs_adam_group * 1)(L.gs_adam_group(p.data_ptr(), None, p.data_ptr(), p.data_ptr(), 8, 0.1))
    assert lib.gs_adam_step(bad, 1, 1, 0.9, 0.999, 1e-8, None) == L.GS_ERR_INVALID_ARG


def _synthetic_rows(rng, N, k, V, rows_per_view):
    """Decoded rows of V views over N anchors (each view sees a random subset, in anchor order)."""
    ra = np.concatenate([np.sort(rng.choice(N, size=rows_per_view, replace=False)) for _ in range(V)])
    vs = np.arange(V + 1) * rows_per_view
    R = len(ra)
    tiles = rng.integers(0, 3, R * k) * (rng.uniform(size=R * k) < 0.7)
    opacity = f32(rng.uniform(-0.3, 1.0, R * k))
    sgrad = f32(rng.normal(size=(R * k, 9)) * 1e-3)
    return ra, vs, tiles, opacity, sgrad


def test_densify_stats_match_oracle_over_two_calls():
    rng = np.random.default_rng(1)
    N, k, V = 5000, 10, 6
    views = api.Views(np.zeros((V, 16), np.float32), np.full((V, 2), 64))
    acc_g = (torch.zeros(N * k, device="cuda"), torch.zeros(N * k, device="cuda", dtype=torch.int32),
             torch.zeros(N, device="cuda"), torch.zeros(N, device="cuda", dtype=torch.int32))
    want = None
    status = api.new_status()
    for call in range(2):
        ra, vs, tiles, opacity, sgrad = _synthetic_rows(rng, N, k, V, 3000)
        R = len(ra)
        g = api.Gauss3D.alloc(R + 7, k, V)   # capacity above the row count
        g.row_anchor[:R] = torch.as_tensor(ra.astype(np.int32)).cuda()
        g.view_start.copy_(torch.as_tensor(vs.astype(np.int32)))
        g.opacity[:R * k] = torch.as_tensor(opacity).cuda()
        sp = api.Splats.alloc((R + 7) * k)
        sp.tiles[:R * k] = torch.as_tensor(tiles.astype(np.int32)).cuda()
        sg = torch.zeros((R + 7) * k, 9, device="cuda")
        sg[:R * k] = torch.as_tensor(sgrad).cuda()
        api.densify_stats(g, views, sp, sg, N, *acc_g, status)
        want = O.densify_stats(ra, tiles, opacity.astype(np.float64), sgrad.astype(np.float64), N, k, accum=want)
    torch.cuda.synchronize()
    assert api.read_status(status)[0] == 0
    assert np.array_equal(to_np(acc_g[1]), want[1]) and np.array_equal(to_np(acc_g[3]), want[3])
    assert np.allclose(to_np(acc_g[0]), want[0], rtol=1e-5, atol=1e-9)
    assert np.allclose(to_np(acc_g[2]), want[2], rtol=1e-5, atol=1e-6)
    assert want[3].max() > 1 and want[1].max() > 1   # anchors seen by several views


def test_densify_stats_reports_an_anchor_outside_the_map():
    N, k, V = 10, 2, 1
    views = api.Views(np.zeros((V, 16), np.float32), [(16, 16)])
    g = api.Gauss3D.alloc(3, k, V)
    g.row_anchor.copy_(torch.tensor([0, 12, 1], dtype=torch.int32))
    g.view_start.copy_(torch.tensor([0, 3], dtype=torch.int32))
    sp = api.Splats.alloc(3 * k)
    sg = torch.zeros(3 * k, 9, device="cuda")
    acc = (torch.zeros(N * k, device="cuda"), torch.zeros(N * k, device="cuda", dtype=torch.int32),
           torch.zeros(N, device="cuda"), torch.zeros(N, device="cuda", dtype=torch.int32))
    status = api.new_status()
    api.densify_stats(g, views, sp, sg, N, *acc, status)
    torch.cuda.synchronize()
    assert api.read_status(status)[0] == L.GS_ERR_INVALID_ARG
    assert int(acc[3].sum()) == 2   # the two rows with valid anchors were counted


def test_densify_masks_bit_exact():
    rng = np.random.default_rng(2)
    N, k = 20000, 10
    ga = f32(rng.uniform(0, 1e-2, N * k))
    od = rng.integers(0, 6, N * k).astype(np.int32)
    oa = f32(rng.uniform(0, 3, N))
    ad = rng.integers(0, 6, N).astype(np.int32)
    # put some means exactly on the thresholds
    ga[:50] = f32(0.002 * od[:50])
    grow, prune = torch.zeros(N * k, device="cuda", dtype=torch.uint8), torch.zeros(N, device="cuda", dtype=torch.uint8)
    t = lambda a: torch.as_tensor(a).cuda()
    api.densify_masks(k, t(ga), t(od), t(oa), t(ad), 0.002, 0.5, 2, grow, prune)
    torch.cuda.synchronize()
    wg, wp = O.densify_masks(ga, od, oa, ad, k, 0.002, 0.5, 2)
    assert np.array_equal(to_np(grow), wg) and np.array_equal(to_np(prune), wp)
    assert 0 < wg.sum() < N * k and 0 < wp.sum() < N


def test_optimizer_steps_lower_the_mapping_loss():
    s = scenes.tiny_corridor(seed=0, n_anchors=4000, F=32, k=10, hidden=32)
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    tgt_host = torch.as_tensor(f32(O.targets_flat(s))).pin_memory()
    ms = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16, fuse_projection=False)
    opt = pipeline.Optimizer(A, ms.rp.agrad)
    stats = pipeline.DensifyStats(A)
    xyz0 = A.xyz.clone()
    losses = []
    for _ in range(6):
        losses.append(ms.step(tgt_host))
        stats.accumulate(ms.rp, ms.stream)
        with torch.cuda.stream(ms.stream):
            opt.step()
    torch.cuda.synchronize()
    assert losses[-1] < losses[0]
    assert torch.equal(A.xyz, xyz0)   # anchor positions are not optimised
    assert int(stats.anchor_denom.sum()) == 6 * ms.rp.n_rows()
    grow, prune = stats.masks(1e-4, 0.05, min_count=1)
    assert grow.numel() == A.N * A.k and prune.numel() == A.N
