"""Failure detection of the tensor-core decoders without a GPU fault: the
bounded wait of a tcgen05 kernel for its MMAs is made to run out (a limit of
0 gives up at the first wait), and the call must record GS_ERR_TIMEOUT in the
status word, drain its MMAs, free its tensor memory and leave the context
usable -- the next call, with the default limit, gives the normal result."""
import pytest
import torch

from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, scenes

pytestmark = pytest.mark.gpu

SITE_DECODE_TC = 15       # status `where` of the forward decoder's timeout
SITE_DECODE_BWD_TC = 65   # and of the reverse decoder's


def _decode(A, vw, cap, s):
    g = api.Gauss3D.alloc(cap, s.k, s.V)
    st = api.new_status()
    api.decode(A, vw, g, api.workspace(api.decode_workspace(A, vw, cap)), st, L.GS_PREC_BF16)
    torch.cuda.synchronize()
    return g, api.read_status(st)


def _decode_bwd(A, vw, g, cap):
    dg = api.Gauss3DGrad.like(g)
    for t in (dg.dmu, dg.dscale, dg.dquat, dg.dopacity, dg.dcolour):
        t.copy_(torch.linspace(-1.0, 1.0, t.numel(), device=t.device).view_as(t))
    out = api.AnchorGrad.like(A)
    st = api.new_status()
    api.decode_bwd(A, vw, g, dg, out, api.workspace(api.decode_bwd_workspace(A, vw, cap)), st, L.GS_PREC_BF16)
    torch.cuda.synchronize()
    return out, api.read_status(st)


def test_tensor_core_wait_timeout_is_reported_and_the_next_call_succeeds():
    s = scenes.tiny_corridor(seed=0, n_anchors=4000, F=32, k=10, hidden=32)
    A = api.Anchors.from_scene(s)
    vw = api.Views(s.cams, s.wh)
    cap = s.N * s.V
    ref, code = _decode(A, vw, cap, s)
    assert code[0] == L.GS_OK
    ref_grad, code = _decode_bwd(A, vw, ref, cap)
    assert code[0] == L.GS_OK
    rows = int(ref.view_start[-1].item())
    assert rows > 128
    try:
        api.set_wait_limit(0)
        _, (code, where, _) = _decode(A, vw, cap, s)
        assert (code, where) == (L.GS_ERR_TIMEOUT, SITE_DECODE_TC)
        _, (code, where, _) = _decode_bwd(A, vw, ref, cap)
        assert (code, where) == (L.GS_ERR_TIMEOUT, SITE_DECODE_BWD_TC)
    finally:
        api.set_wait_limit(None)
    # the context is usable and the tensor memory was given back: same results as before
    for _ in range(2):
        g, code = _decode(A, vw, cap, s)
        assert code[0] == L.GS_OK
        C = rows * s.k
        for name in ("mu", "scale", "quat", "opacity", "colour"):
            assert torch.equal(getattr(g, name)[:C], getattr(ref, name)[:C]), name
        out, code = _decode_bwd(A, vw, g, cap)
        assert code[0] == L.GS_OK
        for name in ("dxyz", "dfeat", "dlog_scaling", "doffsets", "dmlp"):
            a, b = getattr(out, name), getattr(ref_grad, name)
            assert torch.allclose(a, b, rtol=1e-4, atol=1e-6 * float(b.abs().max())), name
