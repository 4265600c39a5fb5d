"""The projection's conic against the FP64 oracle over a sweep of condition
numbers of the 2D covariance, 1e0 ... 1e7: needle-like Gaussians whose major
axis projects to sqrt(0.3 (c - 1)) pixels while the minor axis is held at the
0.3 px^2 low-pass.  The device forms the 2D covariance in FP32 and, when
det < 1e-3 a c, the determinant and conic in FP64, so the error left is the
FP32 rounding of the covariance entries amplified by the conditioning of the
inverse: |d conic| / |conic| <= K c 2^-24 (K = 16 covers the rounding of the
entries' several products and sums).  The measured errors per decade are
printed (run with -s)."""
import numpy as np
import pytest
import torch
from scipy.spatial.transform import Rotation

from _helpers import to_np
from oracle import oracle as O
from paper_2607_21416_b300 import api, scenes
from test_gpu_fullsize import _records

pytestmark = pytest.mark.gpu


def test_conic_error_over_condition_numbers():
    rng = np.random.default_rng(0)
    f, W, H, z = 500.0, 640, 480, 10.0
    cams = scenes.camera(f, f, W / 2, H / 2, (0.0, 0.0, 0.0))[None]
    per = 40
    conds = 10.0 ** np.arange(0, 8)
    mu, scale, quat = [], [], []
    for c in conds:
        major = z / f * np.sqrt(0.3 * max(c - 1.0, 1e-6))        # metres: (f s / z)^2 = 0.3 (c - 1)
        for _ in range(per):
            mu.append([rng.uniform(-2, 2), rng.uniform(-1.5, 1.5), z + rng.uniform(-0.01, 0.01)])
            scale.append([major, 1e-5, 1e-5])
            quat.append(Rotation.from_euler("zyx", [rng.uniform(0, 180), rng.uniform(-2, 2), rng.uniform(-2, 2)],
                                            degrees=True).as_quat()[[3, 0, 1, 2]])
    mu, scale, quat = (np.array(a, np.float32) for a in (mu, scale, quat))
    G = len(mu)
    opacity = np.full(G, 0.5, np.float32)
    colour = np.full((G, 3), 0.5, np.float32)
    views = api.Views(cams, [(W, H)])
    g = api.Gauss3D.explicit(mu, scale, quat, opacity, colour)
    sp = api.Splats.alloc(G)
    st = api.new_status()
    api.project(g, views, sp, st)
    torch.cuda.synchronize()
    assert api.read_status(st)[0] == 0
    got = _records(to_np(sp.rec))["conic"]
    prj = O.project(mu, scale, quat, opacity, cams.astype(np.float64), [(W, H)], np.array([0, G], np.int64))
    assert (prj.status == 1).all() and (to_np(sp.tiles) > 0).all()
    a, b, cc = prj.cov2d[:, 0], prj.cov2d[:, 1], prj.cov2d[:, 2]
    lam = 0.5 * (a + cc) + np.sqrt(0.25 * (a - cc) ** 2 + b * b)
    cond = lam / (a * cc - b * b) * lam                         # lambda_max / lambda_min
    err = np.abs(got - prj.conic).max(1) / np.abs(prj.conic).max(1)
    assert (err <= 16.0 * np.maximum(cond, 1.0) * 2.0 ** -24 + 1e-7).all(), err.max()
    print("\n  condition  conic relative error (max over %d needles)  FP64 branch" % per)
    for i, c in enumerate(conds):
        sl = slice(i * per, (i + 1) * per)
        print("  %9.0e  %10.2e  %4d / %d" % (np.median(cond[sl]), err[sl].max(), prj.fp64_branch[sl].sum(), per))
    # needles at an angle to the image axes take the FP64 branch (b^2 close to a c); well-conditioned
    # covariances never do
    assert prj.fp64_branch[-2 * per:].mean() > 0.75 and not prj.fp64_branch[:3 * per].any()
