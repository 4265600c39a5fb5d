"""Host-side logic that needs no GPU: the optimizer's parameter groups (the
anchor positions are not optimised), the densification accumulators, the
loss selection of the render pass, and the synthetic flow pairs' recipe."""
import numpy as np
import pytest
import torch

from paper_2607_21416_b300 import api, pipeline, scenes


def _cpu_anchors(N=50, F=8, k=4, hidden=16, M=2):
    z = lambda *s: torch.zeros(*s)
    return api.Anchors(z(N, 3), z(N, F), z(N, 6), z(N, k, 3), torch.zeros(N, dtype=torch.int32),
                       z(M, 1000), F, k, hidden, M)


def test_optimizer_groups_leave_the_anchor_positions_out():
    A = _cpu_anchors()
    g = api.AnchorGrad.like(A)
    opt = pipeline.Optimizer(A, g, lr={"mlp": 0.001})
    assert opt.names == ["feat", "offsets", "log_scaling", "mlp"]
    params = [grp[0] for grp in opt.groups]
    assert all(p is not A.xyz for p in params)
    assert [grp[4] for grp in opt.groups] == [0.0075, 0.01, 0.007, 0.001]
    for p, gr, m, v, _ in opt.groups:
        assert m.shape == p.shape and v.shape == p.shape and float(m.abs().sum()) == 0.0
        assert gr.shape == p.shape
    opt.set_lr("offsets", 0.5)
    assert opt.groups[1][4] == 0.5


def test_densify_accumulators_have_the_documented_shapes():
    A = _cpu_anchors(N=30, k=5)
    st = pipeline.DensifyStats(A, device="cpu")
    assert st.grad_accum.shape == (150,) and st.offset_denom.dtype == torch.int32
    assert st.opacity_accum.shape == (30,) and st.anchor_denom.dtype == torch.int32
    st.grad_accum += 1
    st.reset()
    assert float(st.grad_accum.sum()) == 0.0


def test_render_pass_rejects_an_unknown_loss():
    views = api.Views(np.zeros((1, 16), np.float32), [(32, 32)], device="cpu")
    with pytest.raises(ValueError):
        pipeline.RenderPass(views, _cpu_anchors(), loss="l2", device="cpu")


def test_flow_pair_recipe():
    a = scenes.flow_pair(seed=3, width=200, height=80, fx=150.0, outlier_frac=0.25, n_samples=5000)
    b = scenes.flow_pair(seed=3, width=200, height=80, fx=150.0, outlier_frac=0.25, n_samples=5000)
    assert np.array_equal(a.flow, b.flow) and np.array_equal(a.samples, b.samples)   # seeded
    assert a.flow.shape == (80, 200, 2) and a.flow.dtype == np.float32
    assert abs(a.outlier.mean() - 0.25) < 0.02
    assert len(np.unique(a.samples)) == 5000 and a.samples.max() < 200 * 80
    assert 4.0 <= a.depth.min() and a.depth.max() <= 44.0
