"""Pins of the oracle's optimizer step (Adam with bias correction) and of the
densification statistics and masks: PyTorch's own Adam in float64, the
closed forms of the first step and of a constant gradient, a hand-worked
statistics example and its invariants, and the mask edges."""
import numpy as np
import pytest
import torch

from oracle import oracle as O


def test_adam_matches_torch_adam_in_float64():
    rng = np.random.default_rng(0)
    p0 = rng.normal(size=37)
    grads = [rng.normal(size=37) * s for s in (1.0, 0.1, 3.0, 1e-3, 0.5)]
    t = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([t], lr=0.01, betas=(0.9, 0.999), eps=1e-8)
    p, m, v = p0.copy(), np.zeros(37), np.zeros(37)
    for step, g in enumerate(grads, start=1):
        t.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        p, m, v = O.adam(p, g, m, v, step, 0.01, 0.9, 0.999, 1e-8)
        assert np.allclose(p, t.detach().numpy(), rtol=1e-13, atol=1e-15)
    st = opt.state[t]
    assert np.allclose(m, st["exp_avg"].numpy(), rtol=1e-13)
    assert np.allclose(v, st["exp_avg_sq"].numpy(), rtol=1e-13)


def test_adam_first_step_and_constant_gradient_closed_forms():
    g = np.array([2.0, -0.5, 0.0, 1e-3])
    p, m, v = O.adam(np.ones(4), g, np.zeros(4), np.zeros(4), 1, 0.1)
    assert np.allclose(p, 1.0 - 0.1 * np.sign(g), rtol=1e-12)   # m/(1-b1) = g, v/(1-b2) = g^2
    # a constant gradient keeps the bias-corrected moments at g and g^2: each step moves lr sign(g)
    p, m, v = np.zeros(4), np.zeros(4), np.zeros(4)
    for t in range(1, 8):
        p, m, v = O.adam(p, g, m, v, t, 0.05)
    assert np.allclose(p, -7 * 0.05 * np.sign(g), rtol=1e-10, atol=1e-12)
    assert np.allclose(m, g * (1 - 0.9 ** 7), rtol=1e-12)
    assert np.allclose(v, g * g * (1 - 0.999 ** 7), rtol=1e-12)


def test_densify_stats_hand_example():
    # 3 anchors, k = 2; rows: view 0 sees anchors 0 and 2, view 1 sees anchors 2 and 1
    row_anchor = np.array([0, 2, 2, 1])
    tiles = np.array([1, 0,   3, 2,   1, 1,   0, 0])
    opacity = np.array([0.5, -0.2,   0.1, 0.3,   0.7, 0.0,   0.4, 0.4])
    sg = np.zeros((8, 9))
    sg[:, 0:2] = [[3, 4], [9, 9], [1, 0], [0, 2], [6, 8], [1, 1], [5, 5], [7, 7]]
    ga, od, oa, ad = O.densify_stats(row_anchor, tiles, opacity, sg, N=3, k=2)
    assert np.allclose(ga, [5.0, 0.0, 0.0, 0.0, 1.0 + 10.0, 2.0 + np.sqrt(2.0)])
    assert od.tolist() == [1, 0, 0, 0, 2, 2]
    assert np.allclose(oa, [0.5, 0.8, 0.4 + 0.7])
    assert ad.tolist() == [1, 1, 2]


def test_densify_stats_invariants_and_accumulation():
    rng = np.random.default_rng(1)
    N, k, rows = 50, 4, 160
    row_anchor = rng.integers(0, N, rows)
    tiles = rng.integers(0, 3, rows * k)
    opacity = rng.uniform(-0.5, 1, rows * k)
    sg = rng.normal(size=(rows * k, 9))
    ga, od, oa, ad = O.densify_stats(row_anchor, tiles, opacity, sg, N, k)
    assert od.sum() == (tiles > 0).sum() and ad.sum() == rows
    assert ga.sum() == pytest.approx(np.hypot(sg[:, 0], sg[:, 1])[tiles > 0].sum(), rel=1e-13)
    assert oa.sum() == pytest.approx(np.maximum(opacity, 0).sum(), rel=1e-13)
    # accumulating two halves equals one pass over all rows
    h = rows // 2
    acc = O.densify_stats(row_anchor[:h], tiles[:h * k], opacity[:h * k], sg[:h * k], N, k)
    acc = O.densify_stats(row_anchor[h:], tiles[h * k:], opacity[h * k:], sg[h * k:], N, k, accum=acc)
    for a, b in zip(acc, (ga, od, oa, ad)):
        assert np.allclose(a, b, rtol=1e-13)


def test_densify_masks_edges():
    ga = np.array([0.3, 0.3, 0.1, 0.0], np.float32)
    od = np.array([3, 2, 1, 0], np.int32)
    oa = np.array([0.01, 0.05], np.float32)
    ad = np.array([2, 1], np.int32)
    grow, prune = O.densify_masks(ga, od, oa, ad, k=2, grad_thr=0.1, opacity_thr=0.05, min_count=1)
    # means 0.1 (>= 0.1: grows), 0.15, 0.1, and an offset never rendered
    assert grow.tolist() == [1, 1, 1, 0]
    assert prune.tolist() == [1, 0]      # 0.005 < 0.05; 0.05 is not < 0.05
    grow, prune = O.densify_masks(ga, od, oa, ad, k=2, grad_thr=0.1, opacity_thr=0.05, min_count=2)
    assert grow.tolist() == [1, 1, 0, 0] and prune.tolist() == [1, 0]
