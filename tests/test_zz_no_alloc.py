"""gs_decode_noalloc: the decode entry point for callers that cannot allocate
device memory (its scratch is a static device array instead of a caller
workspace).  Its output must equal that of gs_decode on the same inputs, on
two calls in a row with different problem sizes (the second call finds the
first call's counts in the shared scratch), with the FP32 decoder and with
the BF16 tensor-core decoder.  This file is collected last so that a stop at
the first failure has already run every other test."""
import numpy as np
import pytest
import torch

from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, scenes

pytestmark = pytest.mark.gpu

PREC_TOL = 0.0   # same kernels and inputs: outputs match bit for bit


def _decode_both(s, precision):
    A = api.Anchors.from_scene(s)
    vw = api.Views(s.cams, s.wh)
    cap = s.N * s.V
    ref = api.Gauss3D.alloc(cap, s.k, s.V)
    st = api.new_status()
    api.decode(A, vw, ref, api.workspace(api.decode_workspace(A, vw, cap)), st, precision)
    got = api.Gauss3D.alloc(cap, s.k, s.V)
    got.row_anchor.fill_(-7)
    got.opacity.fill_(123.0)
    st2 = api.new_status()
    api.decode_noalloc(A, vw, got, st2, precision)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0 and api.read_status(st2)[0] == 0
    rows = int(ref.view_start[-1].item())
    assert rows > 0
    assert torch.equal(got.view_start, ref.view_start)
    assert torch.equal(got.row_anchor[:rows], ref.row_anchor[:rows])
    C = rows * s.k
    for name in ("mu", "scale", "quat", "opacity", "colour"):
        a, b = getattr(got, name)[:C], getattr(ref, name)[:C]
        assert torch.allclose(a, b, rtol=PREC_TOL, atol=PREC_TOL), name


@pytest.mark.parametrize("precision", [L.GS_PREC_FP32, L.GS_PREC_BF16])
def test_noalloc_decode_matches_decode_on_two_calls_in_a_row(precision):
    # two different problems back to back: several anchor chunks and views,
    # then a larger single view
    _decode_both(scenes.tiny_corridor(seed=2, n_anchors=5000), precision)
    _decode_both(scenes.anchor_single_view(seed=1), precision)


def test_noalloc_decode_rejects_sizes_beyond_its_scratch():
    s = scenes.tiny_corridor(seed=0, n_anchors=600)
    A = api.Anchors.from_scene(s)
    views = np.tile(s.wh[:1], (64, 1))
    cams = np.tile(s.cams[:1], (64, 1))
    vw = api.Views(cams, views)
    # 64 views x ceil(N / 2048) chunks above 131072 counts: N just over 4M anchors
    big = api.Anchors(A.xyz.repeat(7000, 1)[: 4_194_305], A.feat.repeat(7000, 1)[: 4_194_305],
                      A.log_scaling.repeat(7000, 1)[: 4_194_305], A.offsets.repeat(7000, 1, 1)[: 4_194_305],
                      A.part.repeat(7000)[: 4_194_305], A.mlp, A.F, A.k, A.hidden, A.M)
    g = api.Gauss3D.alloc(16, s.k, 64)
    with pytest.raises(L.GsError) as e:
        api.decode_noalloc(big, vw, g, api.new_status())
    assert e.value.code == L.GS_ERR_CAPACITY
