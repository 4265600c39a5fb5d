"""Pins of the oracle's flow-densification geometry (Eq. 5): the fundamental
matrix of Eq. 5 against the textbook relative-pose form, its epipoles,
zero residuals and exact depths for noise-free flow, and the separation of
outlier correspondences."""
import numpy as np

from oracle import oracle as O
from paper_2607_21416_b300 import scenes


def _K(cam):
    return np.array([[cam[0], 0, cam[2]], [0, cam[1], cam[3]], [0, 0, 1.0]])


def test_fundamental_matches_the_relative_pose_form_and_its_epipoles():
    fp = scenes.flow_pair(seed=0, n_samples=10)
    c1, c2 = fp.cams.astype(np.float64)
    F = O.fundamental(c1, c2)
    R1, t1 = c1[4:13].reshape(3, 3), c1[13:16]
    R2, t2 = c2[4:13].reshape(3, 3), c2[13:16]
    R, t = R2 @ R1.T, t2 - R2 @ R1.T @ t1            # keyframe-1 camera frame -> keyframe-2 frame
    tx = np.array([[0, -t[2], t[1]], [t[2], 0, -t[0]], [-t[1], t[0], 0]])
    Fr = np.linalg.inv(_K(c2)).T @ tx @ R @ np.linalg.inv(_K(c1))
    a, b = F / np.linalg.norm(F), Fr / np.linalg.norm(Fr)
    assert min(np.abs(a - b).max(), np.abs(a + b).max()) < 1e-12
    C1 = -R1.T @ t1
    C2 = -R2.T @ t2
    e1 = _K(c1) @ (R1 @ C2 + t1)
    e2 = _K(c2) @ (R2 @ C1 + t2)
    assert np.abs(F @ e1).max() <= 1e-12 * np.linalg.norm(F) * np.linalg.norm(e1)
    assert np.abs(F.T @ e2).max() <= 1e-12 * np.linalg.norm(F) * np.linalg.norm(e2)
    assert abs(np.linalg.det(F)) <= 1e-12 * np.linalg.norm(F) ** 3


def test_noise_free_flow_gives_zero_residuals_and_the_true_depths():
    fp = scenes.flow_pair(seed=1, width=320, height=120, fx=200.0, outlier_frac=0.0, n_samples=3000)
    W, H = fp.wh
    # the float32 flow carries ~1e-5 px of rounding: residuals stay at that level
    r, keep, flag, pts = O.flow_triangulate(fp.cams[0], fp.cams[1], fp.wh, fp.flow, fp.samples, tau=1e-2)
    assert keep.all() and not flag.any()
    q = fp.samples
    c1 = fp.cams[0].astype(np.float64)
    Xc = pts @ c1[4:13].reshape(3, 3).T + c1[13:16]          # keyframe-1 camera frame
    depth = fp.depth.reshape(-1)[q].astype(np.float64)
    parallax = np.hypot(*fp.flow.reshape(-1, 2)[q].T) > 2.0   # away from the epipole
    assert parallax.mean() > 0.5
    assert np.allclose(Xc[parallax, 2], depth[parallax], rtol=1e-3)
    u = c1[0] * Xc[:, 0] / Xc[:, 2] + c1[2]
    assert np.allclose(u[parallax], (q % W)[parallax], atol=1e-3)   # the point reprojects onto its pixel


def test_outliers_separate_from_inliers():
    fp = scenes.flow_pair(seed=2, outlier_frac=0.3, noise_px=0.05, n_samples=20000)
    # F of Eq. 5 is not normalised (|F| ~ 3.7e3 here): 0.05 px of flow noise gives residuals up to ~170
    r, keep, flag, pts = O.flow_triangulate(fp.cams[0], fp.cams[1], fp.wh, fp.flow, fp.samples, tau=200.0)
    out = fp.outlier.reshape(-1)[fp.samples]
    assert keep[~out].mean() > 0.99
    assert keep[out].mean() < 0.05
    assert len(pts) == keep.sum()
