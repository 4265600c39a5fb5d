"""Pins of the oracle's map maintenance: voxelisation (Eq. 4) against NumPy's
unique of the single-precision rounded indices, a hand example with a tie,
the exclusion of existing voxels, the centre property and the range check;
the loop-closure deformation (Eq. 7) against its closed forms (no update, a
pure shift of the world, a rotation about a camera centre), the
nearest-keyframe rule on a hand example and rigidity."""
import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O

B = O.KEY_BIAS


def _key(i, j, l):
    return np.uint64(((i + B) << 42) | ((j + B) << 21) | (l + B))


def test_voxelize_hand_example_with_ties_to_even():
    pts = np.array([[0.04, 0, 0], [0.06, 0, 0], [0.1, 0, 0], [0.25, 0.0, -0.15], [-0.31, 0, 0]])
    keys, centres, n = O.voxelize(pts, 0.1)
    # 0.4 -> 0, 0.6 -> 1, 1.0 -> 1, (2.5, 0, -1.5) -> (2, 0, -2) (ties to even), -3.1 -> -3
    want = sorted([_key(0, 0, 0), _key(1, 0, 0), _key(2, 0, -2), _key(-3, 0, 0)])
    assert n == 4 and keys.tolist() == [int(k) for k in want]
    idx = {int(_key(2, 0, -2)): (2, 0, -2)}
    at = keys.tolist().index(int(_key(2, 0, -2)))
    assert np.array_equal(centres[at], np.float32(idx[int(_key(2, 0, -2))]) * np.float32(0.1))


def test_voxelize_equals_numpy_unique_of_rounded_indices():
    rng = np.random.default_rng(0)
    pts = (rng.normal(size=(20000, 3)) * [30, 2, 30]).astype(np.float32)
    pts = np.concatenate([pts, pts[:3000] + 1e-4])          # near-duplicates
    eps = np.float32(0.2)
    keys, centres, n = O.voxelize(pts, eps)
    idx = np.rint(pts / eps).astype(np.int64)                # float32 division, ties to even
    u = np.unique(idx, axis=0)
    want = ((u[:, 0] + B) << 42) | ((u[:, 1] + B) << 21) | (u[:, 2] + B)
    assert np.array_equal(keys.astype(np.int64), np.sort(want))
    assert np.array_equal(centres, (u[np.argsort(want)].astype(np.float32) * eps))
    # every point lies within half a voxel (plus rounding) of its voxel's centre
    c = np.rint(pts / eps).astype(np.float32) * eps
    assert np.abs(pts - c).max() <= 0.5 * eps * (1 + 1e-5)


def test_voxelize_excludes_existing_voxels():
    rng = np.random.default_rng(1)
    pts = rng.uniform(-5, 5, (5000, 3)).astype(np.float32)
    all_keys, _, n_all = O.voxelize(pts, 0.5)
    existing = np.sort(np.concatenate([all_keys[::3], np.array([_key(900, 0, 0)], np.uint64)]))
    keys, _, n = O.voxelize(pts, 0.5, existing=existing)
    assert n == n_all - len(all_keys[::3])
    assert not np.isin(keys, existing).any()
    assert np.array_equal(np.union1d(keys, all_keys[::3]), all_keys)
    _, _, needed = O.voxelize(pts, 0.5, existing=existing, cap=10)
    assert needed == n


def test_voxelize_rejects_indices_out_of_range():
    with pytest.raises(ValueError):
        O.voxelize(np.array([[1.1e5, 0, 0]]), 0.1)


def _cam(R, t, fx=500.0, W=640, H=480):
    return np.concatenate([[fx, fx, W / 2, H / 2], np.asarray(R, float).reshape(9), t])


def test_loop_closure_no_update_and_world_shift():
    rng = np.random.default_rng(2)
    xyz = rng.uniform([-20, -5, 1], [20, 5, 60], (3000, 3))
    old = np.stack([_cam(np.eye(3), [0, 0, 0]), _cam(Rotation.from_euler("y", 30, degrees=True).as_matrix(),
                                                     [1, 0, -5])])
    wh = [(640, 480), (640, 480)]
    out, assigned, _ = O.loop_closure(xyz, old, old, wh, z_far=50.0)
    assert np.allclose(out, xyz, atol=1e-12) and (assigned >= 0).any() and (assigned < 0).any()
    # new poses that see the world shifted by s: T_new x = T_old (x - s) moves frustum anchors by +s
    s = np.array([0.3, -0.1, 2.0])
    new = old.copy()
    for i in range(2):
        R = old[i, 4:13].reshape(3, 3)
        new[i, 13:16] = old[i, 13:16] - R @ s
    out, assigned2, _ = O.loop_closure(xyz, old, new, wh, z_far=50.0)
    assert np.array_equal(assigned, assigned2)
    moved = assigned >= 0
    assert np.allclose(out[moved], xyz[moved] + s, atol=1e-12)
    assert np.array_equal(out[~moved], xyz[~moved])


def test_loop_closure_rotation_about_the_camera_centre_and_rigidity():
    rng = np.random.default_rng(3)
    xyz = rng.uniform([-10, -5, 2], [10, 5, 40], (2000, 3))
    old = _cam(np.eye(3), [0, 0, 0])
    Rn = Rotation.from_euler("xyz", [3, -8, 5], degrees=True).as_matrix()
    new = _cam(Rn, [0, 0, 0])          # same centre, rotated: x -> Rn^T x
    out, assigned, _ = O.loop_closure(xyz, old[None], new[None], [(640, 480)], z_far=45.0)
    m = assigned == 0
    assert m.sum() > 100
    assert np.allclose(out[m], xyz[m] @ Rn, atol=1e-12)
    d0 = np.linalg.norm(xyz[m][:, None] - xyz[m][None], axis=2)
    d1 = np.linalg.norm(out[m][:, None] - out[m][None], axis=2)
    assert np.allclose(d0, d1, atol=1e-10)


def test_loop_closure_takes_the_nearest_keyframe():
    # keyframe 0 at the origin looking along +z, keyframe 1 at z = 30 looking back along -z:
    # both see the anchors on the axis between them; each anchor takes the nearer one
    R1 = np.diag([-1.0, 1.0, -1.0])
    old = np.stack([_cam(np.eye(3), [0, 0, 0]), _cam(R1, -R1 @ np.array([0, 0, 30.0]))])
    new = old.copy()
    new[0, 13:16] -= [1, 0, 0]     # keyframe 0 sees the world shifted by +x: its anchors move by +1 in x
    new[1, 13:16] -= [0, 1, 0]     # keyframe 1: its anchors move by +1 in y (R1 keeps y)
    z = np.array([5, 12, 14.999, 15.001, 20, 25.0])
    xyz = np.stack([np.zeros_like(z), np.zeros_like(z), z], 1)
    out, assigned, flag = O.loop_closure(xyz, old, new, [(640, 480)] * 2, z_far=100.0)
    assert assigned.tolist() == [0, 0, 0, 1, 1, 1] and not flag.any()
    assert np.allclose(out[:3], xyz[:3] + [1, 0, 0], atol=1e-12)
    assert np.allclose(out[3:], xyz[3:] + [0, 1, 0], atol=1e-12)
    # an exact tie goes to the lower index and is flagged
    out, assigned, flag = O.loop_closure(np.array([[0, 0, 15.0]]), old, new, [(640, 480)] * 2, z_far=100.0)
    assert assigned.tolist() == [0] and flag.tolist() == [1]
