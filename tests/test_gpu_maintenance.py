"""gs_voxelize (Eq. 4) and gs_loop_closure (Eq. 7) against the oracle on
seeded synthetic inputs: voxel keys and centres bit-exact (the rounding is
decided in single precision on both sides), with ties, near-duplicates,
several sort tiles, existing keys excluded, an empty input, a capacity
overflow and an out-of-range index; the loop-closure assignment exact away
from flagged frustum edges and distance ties, positions within FP32
rounding, on a corridor of anchors and keyframes with perturbed poses."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from _helpers import to_np
from oracle import oracle as O
from paper_2607_21416_b300 import _lib as L
from paper_2607_21416_b300 import api

pytestmark = pytest.mark.gpu


def _gpu_voxelize(pts, eps, existing=None, cap=None):
    P = len(pts)
    cap = max(P, 1) if cap is None else cap
    d_pts = torch.as_tensor(np.ascontiguousarray(pts, np.float32)).cuda().reshape(-1, 3)
    keys = torch.zeros(cap, dtype=torch.int64, device="cuda")
    cen = torch.zeros(cap, 3, device="cuda")
    n = torch.zeros(1, dtype=torch.int32, device="cuda")
    ws = api.workspace(api.voxelize_workspace(P))
    st = api.new_status()
    ex = None if existing is None else torch.as_tensor(existing.view(np.int64)).cuda()
    api.voxelize(d_pts, eps, keys, cen, n, ws, st, existing=ex)
    torch.cuda.synchronize()
    code, where, needed = api.read_status(st)
    k = int(n[0])
    return code, where, needed, to_np(keys[:k]).view(np.uint64), to_np(cen[:k])


@pytest.mark.parametrize("P", [0, 1, 37, 5000, 300_000])
def test_voxelize_matches_oracle(P):
    rng = np.random.default_rng(P)
    pts = (rng.normal(size=(P, 3)) * [40, 3, 40]).astype(np.float32)
    if P > 10:
        pts[: P // 10] = pts[P // 10: 2 * (P // 10)] + np.float32(1e-5)   # near-duplicates
        pts[0] = [0.25, -0.15, 0.05]                                     # ties to even at eps = 0.1
    eps = 0.1 if P < 1000 else 0.2
    code, _, _, keys, cen = _gpu_voxelize(pts, eps)
    wk, wc, n = O.voxelize(pts, eps)
    assert code == 0
    assert len(keys) == n and np.array_equal(keys, wk) and np.array_equal(cen, wc)


def test_voxelize_excludes_existing_and_reports_capacity():
    rng = np.random.default_rng(7)
    pts = rng.uniform(-30, 30, (100_000, 3)).astype(np.float32)
    all_keys, _, n_all = O.voxelize(pts, 0.5)
    existing = np.ascontiguousarray(np.sort(np.concatenate([all_keys[1::4], all_keys[:1]])), np.uint64)
    code, _, _, keys, cen = _gpu_voxelize(pts, 0.5, existing=existing)
    wk, wc, n = O.voxelize(pts, 0.5, existing=existing)
    assert code == 0 and np.array_equal(keys, wk) and np.array_equal(cen, wc)
    code, _, needed, keys, _ = _gpu_voxelize(pts, 0.5, existing=existing, cap=100)
    assert code == L.GS_ERR_CAPACITY and needed == n and len(keys) == 0


def test_voxelize_reports_an_index_out_of_range():
    pts = np.array([[0, 0, 0], [2.0e5, 0, 0]], np.float32)
    code, where, _, _, _ = _gpu_voxelize(pts, 0.1)
    assert code == L.GS_ERR_INVALID_ARG and where == 80


def _corridor_keyframes(rng, K):
    """Keyframes along +z every 4 m looking forward with small yaw, and perturbed new poses."""
    old, new = [], []
    for i in range(K):
        c = np.array([rng.uniform(-0.5, 0.5), 0.0, 4.0 * i])
        R = Rotation.from_euler("y", rng.uniform(-3, 3), degrees=True).as_matrix()
        t = -R @ c
        old.append(np.concatenate([[600.0, 600.0, 400.0, 150.0], R.reshape(9), t]))
        dR = Rotation.from_euler("xyz", rng.normal(size=3) * 0.3, degrees=True).as_matrix()
        Rn = dR @ R
        tn = -Rn @ (c + rng.normal(size=3) * 0.2)
        new.append(np.concatenate([[600.0, 600.0, 400.0, 150.0], Rn.reshape(9), tn]))
    return np.array(old), np.array(new)


@pytest.mark.parametrize("K", [1, 7, 300])
def test_loop_closure_matches_oracle(K):
    rng = np.random.default_rng(K)
    N = 200_000
    xyz = np.stack([rng.uniform(-8, 8, N), rng.uniform(-3, 2, N), rng.uniform(-5, 4.0 * K + 40, N)], 1)
    xyz32 = xyz.astype(np.float32)
    old, new = _corridor_keyframes(rng, K)
    wh = np.tile([[800, 300]], (K, 1)).astype(np.int32)
    old32, new32 = old.astype(np.float32), new.astype(np.float32)
    d_xyz = torch.as_tensor(xyz32).cuda()
    assigned = torch.full((N,), -7, dtype=torch.int32, device="cuda")
    api.loop_closure(d_xyz, torch.as_tensor(old32).cuda(), torch.as_tensor(new32).cuda(),
                     torch.as_tensor(wh).cuda(), 30.0, assigned)
    torch.cuda.synchronize()
    want, wa, flag = O.loop_closure(xyz32.astype(np.float64), old32.astype(np.float64), new32.astype(np.float64),
                                    wh, 30.0, band=1e-4)
    ok = flag == 0
    assert ok.mean() > 0.99
    got_a = to_np(assigned)
    assert np.array_equal(got_a[ok], wa[ok])
    assert (wa >= 0).mean() > 0.3 and (wa < 0).any()
    got = to_np(d_xyz).astype(np.float64)
    scale = np.abs(xyz).max() + 100.0
    assert np.abs(got[ok] - want[ok]).max() <= 2e-6 * scale
    assert np.array_equal(got[wa < 0], xyz32[wa < 0].astype(np.float64))
