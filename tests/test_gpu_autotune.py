"""The autotuner on the GPU: MappingStep(tune=True) picks the chunk length
and launch shapes for a batch by measuring them, caches the pick, renders
the same image and loss as the default shapes (chunking and launch shapes
change no result beyond floating-point rounding of the chunk combine), and a
second step on the same workload takes the cached pick without measuring."""
import numpy as np
import pytest
import torch

from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, pipeline, scenes

pytestmark = pytest.mark.gpu


def test_tuned_mapping_step_matches_default_and_caches(tmp_path):
    s = scenes.keyframe_batch(seed=0, n_anchors=40000, n_views=2)
    views = api.Views(s.cams, s.wh)
    A = api.Anchors.from_scene(s)
    tgt = torch.from_numpy(np.concatenate([t.reshape(-1) for t in s.targets]).astype(np.float32)).pin_memory()
    ref = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16)
    loss_ref = ref.step(tgt)
    img_ref = ref.rp.image.clone()
    dfeat_ref = ref.rp.agrad.dfeat.clone()
    cache = str(tmp_path / "tune.json")
    ms = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16, tune=True, tune_cache=cache)
    loss = ms.step(tgt)
    info = ms.tuned
    print("tuned", info)
    assert info["cached"] is False and info["evaluated"] >= 10
    assert info["ms"] <= info["default_ms"] * 1.02
    assert api.get_tuning() == {k: 0 for k in api.TUNING_FIELDS}   # the process-wide shapes are left as found
    assert loss == pytest.approx(loss_ref, rel=1e-5, abs=1e-7)
    assert float((ms.rp.image - img_ref).abs().max()) <= 1e-5
    a, b = ms.rp.agrad.dfeat.double().ravel(), dfeat_ref.double().ravel()
    assert float((a - b).norm() / b.norm()) <= 1e-4
    again = pipeline.MappingStep(views, A, precision=L.GS_PREC_BF16, tune=True, tune_cache=cache)
    again.step(tgt)
    assert again.tuned["cached"] is True and again.tuned["config"] == info["config"]
