"""gs_flow_triangulate (Eq. 5 filtering and linear triangulation) against the
FP64 oracle on synthetic flow pairs: the keep decisions exact away from
pairs flagged within the FP64 rounding band of tau, kept positions in sample
order, residuals and points within single-precision rounding of the output;
samples spanning several CTAs with a ragged tail; no sample; a capacity
overflow; a sample outside the image."""
import numpy as np
import pytest
import torch

from _helpers import to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api, scenes

pytestmark = pytest.mark.gpu


def _gpu(fp, tau, samples=None, cap=None):
    samples = fp.samples if samples is None else samples
    N = len(samples)
    cap = max(N, 1) if cap is None else cap
    cams = torch.as_tensor(np.ascontiguousarray(fp.cams, np.float32)).cuda()
    flow = torch.as_tensor(fp.flow).cuda()
    smp = torch.as_tensor(np.asarray(samples, np.int32)).cuda()
    kept = torch.full((cap,), -1, dtype=torch.int32, device="cuda")
    pts = torch.zeros(cap, 3, device="cuda")
    res = torch.zeros(max(N, 1), device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = api.workspace(api.flow_workspace(N))
    st = api.new_status()
    api.flow_triangulate(cams, fp.wh, flow, smp, tau, kept, pts, n, ws, st, residual=res)
    torch.cuda.synchronize()
    k = int(n[0])
    return api.read_status(st), to_np(kept[:k]), to_np(pts[:k]), to_np(res[:N])


@pytest.mark.parametrize("seed,n_samples", [(0, 2048 * 5 + 77), (1, 200_000)])
def test_flow_triangulate_matches_oracle(seed, n_samples):
    fp = scenes.flow_pair(seed=seed, outlier_frac=0.3, noise_px=0.05, n_samples=n_samples)
    tau = 200.0
    (code, _, _), kept, pts, res = _gpu(fp, tau)
    assert code == 0
    r, keep, flag, wpts = O.flow_triangulate(fp.cams[0], fp.cams[1], fp.wh, fp.flow, fp.samples, tau)
    assert not flag.any()
    assert np.array_equal(kept, np.nonzero(keep)[0])
    assert np.allclose(res, r, rtol=1e-6, atol=1e-6)
    # points: FP64 on both sides, rounded to FP32 at the output; badly conditioned pairs (near the
    # epipole: little parallax) amplify the FP64 rounding differences of the two solvers
    par = np.hypot(*fp.flow.reshape(-1, 2)[fp.samples[keep]].T) > 2.0
    assert par.mean() > 0.5
    assert np.allclose(pts[par], wpts[par], rtol=1e-5, atol=1e-5)
    assert np.isfinite(pts).all()


def test_flow_triangulate_edges():
    fp = scenes.flow_pair(seed=3, width=64, height=48, fx=60.0, outlier_frac=0.2, n_samples=1000)
    (code, _, _), kept, _, _ = _gpu(fp, 200.0, samples=np.zeros(0, np.int32))
    assert code == 0 and len(kept) == 0
    r, keep, _, _ = O.flow_triangulate(fp.cams[0], fp.cams[1], fp.wh, fp.flow, fp.samples, 200.0)
    (code, _, needed), kept, _, _ = _gpu(fp, 200.0, cap=5)
    assert code == L.GS_ERR_CAPACITY and needed == keep.sum() and len(kept) == 0
    bad = fp.samples.copy()
    bad[17] = 64 * 48
    (code, where, _), _, _, _ = _gpu(fp, 200.0, samples=bad)
    assert code == L.GS_ERR_INVALID_ARG and where == 90
