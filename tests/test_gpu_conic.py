"""The projection's conic against the FP64 oracle over a sweep of condition
numbers of the 2D covariance, 1e0 ... 1e7: needle-like Gaussians whose major
axis projects to sqrt(0.3 (c - 1)) pixels while the minor axis is held at the
0.3 px^2 low-pass.  The device forms the 2D covariance in FP32; where det <
1e-3 a c (near-degenerate) it forms it again in compensated single precision
and takes determinant and conic in FP64.  Well-conditioned splats keep the
FP32 error of the inverse, |d conic| / |conic| <= K c 2^-24 (K = 16 covers the
rounding of the entries' several products and sums); near-degenerate ones
must come out at FP32 output precision whatever their condition number, far
below what an inverse of FP32 entries gives there (emulated on the host from
the oracle's covariance rounded to FP32, with the determinant in FP32 or in
FP64 -- about the same, since the rounding of the entries dominates).  The
measured errors per decade are printed (run with -s)."""
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
    # inverses of the FP32-rounded covariance: determinant in FP32, or in FP64
    a32, b32, c32 = (x.astype(np.float32) for x in (a, b, cc))
    det32 = a32 * c32 - b32 * b32
    det64 = a32.astype(np.float64) * c32 - b32.astype(np.float64) ** 2
    with np.errstate(divide="ignore", invalid="ignore"):
        rel = lambda k: np.abs(k - prj.conic).max(1) / np.abs(prj.conic).max(1)
        e32 = np.where(det32 > 0, rel(np.stack([c32 / det32, -b32 / det32, a32 / det32], 1).astype(np.float64)),
                       np.inf)
        e64 = np.where(det64 > 0, rel(np.stack([c32 / det64, -b32 / det64, a32 / det64], 1)), np.inf)
    print("\n  condition  conic relative error (max over %d needles): GPU | FP32 entries, FP32 / FP64 "
          "inverse  FP64 branch" % per)
    for i, c in enumerate(conds):
        sl = slice(i * per, (i + 1) * per)
        print("  %9.0e  %10.2e | %10.2e %10.2e  %4d / %d" % (np.median(cond[sl]), err[sl].max(), e32[sl].max(),
                                                            e64[sl].max(), prj.fp64_branch[sl].sum(), per))
    br = prj.fp64_branch.astype(bool)
    # well-conditioned covariances never take the branch and keep the FP32 bound
    assert not br[:3 * per].any()
    assert (err[~br] <= 16.0 * np.maximum(cond[~br], 1.0) * 2.0 ** -24 + 1e-7).all(), err[~br].max()
    # near-degenerate ones come out at FP32 output precision whatever their condition number ...
    assert br[-2 * per:].mean() > 0.75
    deep = br & (cond > 1e4)
    assert deep.sum() > 60
    assert err[deep].max() <= 8 * 2.0 ** -24, err[deep].max()
    # ... where an inverse of FP32 entries is off by orders of magnitude, FP64 determinant or not
    assert np.median(e32[deep]) > 100 * err[deep].max() and np.median(e64[deep]) > 100 * err[deep].max()
