"""Pins of the FP64 oracle against facts the paper and the mathematics fix.

None of these re-types the oracle's own formulas: each checks a closed form
(single-splat alpha, EWA covariance on the optical axis, conic inverse,
two-splat composite), an invariant (transmittance telescoping, permutation
invariance), a reduction to a library routine (SciPy rotations, Python's
sort), brute force (every pixel against every splat), or central finite
differences of the hand-derived reverse pass.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from oracle import oracle as O
from paper_2607_21416_b300 import scenes


def cam1(fx=100.0, fy=100.0, cx=32.0, cy=24.0, centre=(0.0, 0.0, 0.0), yaw=0.0, pitch=0.0):
    return scenes.camera(fx, fy, cx, cy, centre, yaw, pitch)[None].astype(np.float64)


def explicit_forward(mu, scale, quat, opa, col, cams, wh, mode=0, bg=(0.0, 0.0, 0.0)):
    mu = np.asarray(mu, np.float64)
    vs = np.array([0, mu.shape[0]], np.int64)
    prj = O.project(mu, scale, quat, opa, cams, wh, vs, 1)
    keys, vals, ranges = O.bin_sort(prj.depth_bits, prj.rect, wh, vs, 1)
    ren = O.render(wh, vs, 1, prj.mean2d, prj.conic, opa, col, prj.depth_bits, prj.rect,
                   prj.status, mode, ranges, vals, bg)
    return prj, keys, vals, ranges, ren


# ---------------------------------------------------------------- closed forms
def test_single_isotropic_gaussian_alpha_equals_opacity_at_centre():
    """Eq. 1 with one splat: at the projected centre power = 0, so alpha = o and
    C = o c, T = 1 - o.  One pixel away, the EWA covariance of an isotropic
    Gaussian on the optical axis is ((f/z)^2 s^2 + 0.3) I."""
    wh = np.array([[64, 48]], np.int32)
    o, s, z, f = 0.7, 0.05, 5.0, 100.0
    col = np.array([[0.2, 0.5, 0.9]])
    prj, _, _, _, ren = explicit_forward([[0, 0, z]], [[s] * 3], [[1, 0, 0, 0]], [o], col,
                                         cam1(), wh)
    img = ren.view_image(wh, 0)
    assert np.allclose(prj.mean2d[0], [32.0, 24.0], atol=0, rtol=0)
    assert img[:, 24, 32] == pytest.approx(o * col[0], abs=1e-15)
    assert ren.T_final[24 * 64 + 32] == pytest.approx(1 - o, abs=1e-15)
    var = (f / z * s) ** 2 + 0.3
    for (u, v) in [(33, 24), (32, 26), (35, 21)]:
        d2 = (u - 32) ** 2 + (v - 24) ** 2
        a = o * math.exp(-0.5 * d2 / var)
        expect = a * col[0] if a >= 1 / 255 else 0 * col[0]
        assert img[:, v, u] == pytest.approx(expect, rel=1e-12, abs=1e-15)


def test_ewa_covariance_closed_forms():
    """Sigma2 = J W Sigma3 W^T J^T + 0.3 I evaluated by hand:
    on the optical axis with axis-aligned scales, diag((f s_x/z)^2 + .3,
    (f s_y/z)^2 + .3); off-axis at (x, 0, z) the x-variance gains the depth
    term (f x s_z / z^2)^2."""
    wh = np.array([[200, 150]], np.int32)
    f, z = 150.0, 4.0
    sx, sy, sz = 0.03, 0.07, 0.11
    cams = cam1(fx=f, fy=f, cx=100, cy=75)
    prj = O.project(np.array([[0.0, 0.0, z]]), np.array([[sx, sy, sz]]), np.array([[1.0, 0, 0, 0]]),
                    np.array([0.5]), cams, wh, np.array([0, 1], np.int64))
    a, b, c = prj.cov2d[0]
    assert a == pytest.approx((f * sx / z) ** 2 + 0.3, rel=1e-13)
    assert c == pytest.approx((f * sy / z) ** 2 + 0.3, rel=1e-13)
    assert b == pytest.approx(0.0, abs=1e-15)
    x = 0.4
    prj = O.project(np.array([[x, 0.0, z]]), np.array([[sx, sy, sz]]), np.array([[1.0, 0, 0, 0]]),
                    np.array([0.5]), cams, wh, np.array([0, 1], np.int64))
    a, b, c = prj.cov2d[0]
    assert a == pytest.approx((f * sx / z) ** 2 + (f * x * sz / z ** 2) ** 2 + 0.3, rel=1e-13)
    assert c == pytest.approx((f * sy / z) ** 2 + 0.3, rel=1e-13)
    assert prj.mean2d[0, 0] == pytest.approx(100 + f * x / z, rel=1e-15)


def test_conic_is_inverse_of_cov2d():
    s = scenes.explicit_frustum(seed=3, n=300)
    vs = np.array([0, 300], np.int64)
    prj = O.project(s.mu, s.scale, s.quat, s.opacity, s.cams, s.wh, vs)
    ok = prj.status == 1
    for i in np.nonzero(ok)[0]:
        a, b, c = prj.cov2d[i]
        ca, cb, cc = prj.conic[i]
        prod = np.array([[a, b], [b, c]]) @ np.array([[ca, cb], [cb, cc]])
        assert np.allclose(prod, np.eye(2), atol=1e-10)


def test_quaternion_convention_matches_scipy():
    """Sigma3 = R(q) S^2 R(q)^T with q = (w, x, y, z): on the optical axis of an
    identity camera, Sigma2 = (f/z)^2 Sigma3[:2,:2] + 0.3 I."""
    rng = np.random.default_rng(11)
    wh = np.array([[64, 64]], np.int32)
    f, z = 80.0, 3.0
    cams = cam1(fx=f, fy=f, cx=32, cy=32)
    for _ in range(20):
        q = rng.normal(size=4)
        q /= np.linalg.norm(q)
        s = rng.uniform(0.01, 0.1, 3)
        prj = O.project(np.array([[0.0, 0.0, z]]), s[None], q[None], np.array([0.5]), cams, wh,
                        np.array([0, 1], np.int64))
        Rm = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        S3 = Rm @ np.diag(s ** 2) @ Rm.T
        S2 = (f / z) ** 2 * S3[:2, :2] + 0.3 * np.eye(2)
        assert np.allclose(prj.cov2d[0], [S2[0, 0], S2[0, 1], S2[1, 1]], rtol=1e-12, atol=1e-14)


def test_camera_pose_projects_axis_point_to_principal_point():
    """A point on a posed camera's optical axis lands on (cx, cy); one metre to
    the camera's right at depth d lands f/d pixels right of cx."""
    wh = np.array([[120, 90]], np.int32)
    for yaw, pitch in [(0, 0), (30, 0), (-75, 10), (140, -20)]:
        c = np.array([3.0, -1.0, 7.0])
        cams = cam1(fx=90, fy=90, cx=60, cy=45, centre=c, yaw=yaw, pitch=pitch)
        Rcw = (Rotation.from_euler("y", yaw, degrees=True) *
               Rotation.from_euler("x", pitch, degrees=True)).as_matrix()
        fwd, right = Rcw[:, 2], Rcw[:, 0]
        d = 4.0
        pts = np.stack([c + d * fwd, c + d * fwd + right])
        prj = O.project(pts, np.full((2, 3), 0.05), np.tile([1.0, 0, 0, 0], (2, 1)),
                        np.array([0.5, 0.5]), cams, wh, np.array([0, 2], np.int64))
        assert np.allclose(prj.mean2d[0], [60, 45], atol=1e-10)
        assert np.allclose(prj.mean2d[1], [60 + 90 / d, 45], atol=1e-10)
        assert np.allclose(prj.depth, [d, d], atol=1e-12)


def test_two_splat_composite_by_hand():
    """Two splats centred on the same pixel: C = c1 o1 + c2 o2 (1 - o1),
    T = (1 - o1)(1 - o2); swapping their depths swaps the roles."""
    wh = np.array([[32, 32]], np.int32)
    c1, c2 = np.array([1.0, 0.2, 0.1]), np.array([0.0, 0.4, 0.8])
    o1, o2 = 0.6, 0.5
    for z1, z2 in [(2.0, 3.0), (3.0, 2.0)]:
        mu = [[0, 0, z1], [0, 0, z2]]
        _, _, _, _, ren = explicit_forward(mu, [[0.03] * 3] * 2, [[1, 0, 0, 0]] * 2, [o1, o2],
                                           np.stack([c1, c2]), cam1(cx=16, cy=16), wh)
        img = ren.view_image(wh, 0)[:, 16, 16]
        if z1 < z2:
            exp_c = c1 * o1 + c2 * o2 * (1 - o1)
        else:
            exp_c = c2 * o2 + c1 * o1 * (1 - o2)
        assert np.allclose(img, exp_c, rtol=1e-14, atol=1e-15)
        assert ren.T_final[16 * 32 + 16] == pytest.approx((1 - o1) * (1 - o2), rel=1e-14)


def test_alpha_clamp_and_early_stop():
    """Opacity 1 clamps to 0.99.  Five such splats: T goes 1, .01, 1e-4; the
    third would take T' to 1e-6 < 1e-4 and is not composited, and the second
    (T' = 1e-4 exactly) is."""
    wh = np.array([[16, 16]], np.int32)
    n = 5
    mu = [[0, 0, 2.0 + i] for i in range(n)]
    col = np.eye(3)[np.arange(n) % 3]
    _, _, _, _, ren = explicit_forward(mu, [[0.05] * 3] * n, [[1, 0, 0, 0]] * n, [1.0] * n, col,
                                       cam1(cx=8, cy=8), wh)
    img = ren.view_image(wh, 0)[:, 8, 8]
    T1 = 0.01
    T2 = T1 * 0.01
    expect = col[0] * 0.99 + col[1] * 0.99 * T1
    assert np.allclose(img, expect, rtol=1e-13)
    assert ren.T_final[8 * 16 + 8] == pytest.approx(T2, rel=1e-10)
    assert ren.last[8 * 16 + 8] == 2


@pytest.mark.parametrize("o3,stops", [(0.6, True), (0.4, False)])
def test_stop_threshold_is_1e4(o3, stops):
    """After opacities 0.99 and 0.98 the transmittance is 2e-4.  A third splat
    of opacity 0.6 would leave T' = 0.8e-4 < 1e-4: compositing stops before it.
    With opacity 0.4, T' = 1.2e-4 and it is composited."""
    wh = np.array([[16, 16]], np.int32)
    ops = [0.99, 0.98, o3]
    col = np.array([[1.0, 0, 0], [0, 1.0, 0], [0, 0, 1.0]])
    _, _, _, _, ren = explicit_forward([[0, 0, 2.0 + i] for i in range(3)], [[0.05] * 3] * 3,
                                       [[1, 0, 0, 0]] * 3, ops, col, cam1(cx=8, cy=8), wh)
    img = ren.view_image(wh, 0)[:, 8, 8]
    T2 = (1 - 0.99) * (1 - 0.98)
    expect = col[0] * 0.99 + col[1] * 0.98 * (1 - 0.99)
    if stops:
        assert ren.last[8 * 16 + 8] == 2
        assert ren.T_final[8 * 16 + 8] == pytest.approx(T2, rel=1e-12)
    else:
        expect = expect + col[2] * o3 * T2
        assert ren.last[8 * 16 + 8] == 3
        assert ren.T_final[8 * 16 + 8] == pytest.approx(T2 * (1 - o3), rel=1e-12)
    assert np.allclose(img, expect, rtol=1e-12, atol=1e-16)


def test_transmittance_telescopes_to_one():
    """sum_i alpha_i T_i + T_final = 1 at every pixel (white splats, bg 0),
    early-stopped pixels included."""
    s = scenes.explicit_frustum(seed=0)
    white = np.ones_like(s.colour, dtype=np.float64)
    _, _, _, _, ren = explicit_forward(s.mu, s.scale, s.quat, s.opacity, white, s.cams, s.wh)
    img = ren.view_image(s.wh, 0)
    for ch in range(3):
        assert np.max(np.abs(img[ch].reshape(-1) + ren.T_final - 1.0)) < 1e-12
    assert (ren.T_final < 1e-3).any(), "scene should contain early-stopped pixels"


def test_background_enters_with_final_transmittance():
    s = scenes.explicit_frustum(seed=1, n=200)
    bg = (0.25, 0.5, 1.0)
    _, _, _, _, r0 = explicit_forward(s.mu, s.scale, s.quat, s.opacity, s.colour, s.cams, s.wh)
    _, _, _, _, r1 = explicit_forward(s.mu, s.scale, s.quat, s.opacity, s.colour, s.cams, s.wh,
                                      bg=bg)
    i0, i1 = r0.view_image(s.wh, 0), r1.view_image(s.wh, 0)
    T = r0.T_final.reshape(i0.shape[1:])
    for ch in range(3):
        assert np.allclose(i1[ch], i0[ch] + T * bg[ch], rtol=0, atol=1e-14)


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_binned_equals_brute_force(seed):
    """Tile binning + sort (mode 0) against every pixel scanning every splat
    whose rectangle covers it (mode 1): bit-identical images."""
    rng = np.random.default_rng(seed)
    n = int(rng.integers(1, 65))
    s = scenes.explicit_frustum(seed=seed, n=n, width=32 + seed * 5, height=32 - seed * 3,
                                fx=30.0, fy=30.0, cx=16.0, cy=15.0)
    # a few splats exactly on tile edges
    s.mu[: min(4, n), 0] = (16.0 - 16.0) / 30.0 * s.mu[: min(4, n), 2]
    a = explicit_forward(s.mu, s.scale, s.quat, s.opacity, s.colour, s.cams, s.wh, mode=0)[4]
    b = explicit_forward(s.mu, s.scale, s.quat, s.opacity, s.colour, s.cams, s.wh, mode=1)[4]
    assert np.array_equal(a.image, b.image)
    assert np.array_equal(a.T_final, b.T_final)


@pytest.mark.parametrize("seed", [0, 5])
def test_tile_cutoff_is_lossless_for_faint_splats(seed):
    """With opacities below 0.35, every pixel outside a splat's 3-sigma tile
    rectangle has alpha < 1/255 and is skipped anyway, so scanning every splat
    at every pixel with no tile cutoff (mode 2) gives the binned image."""
    s = scenes.explicit_frustum(seed=seed, n=48, width=40, height=36, fx=35.0, fy=35.0,
                                cx=20.0, cy=18.0)
    opa = s.opacity * 0.34
    a = explicit_forward(s.mu, s.scale, s.quat, opa, s.colour, s.cams, s.wh, mode=0)[4]
    b = explicit_forward(s.mu, s.scale, s.quat, opa, s.colour, s.cams, s.wh, mode=2)[4]
    assert np.array_equal(a.image, b.image)


def test_sort_matches_python_sorted_and_ranges_partition_pairs():
    s = scenes.tiny_corridor()
    fw = O.forward_anchor(s)
    prj, vs, k = fw.prj, fw.dec.view_start, s.k
    tx, ty, base, T = O.tiles_of(s.wh)
    pairs = []
    for c in range(prj.tiles.shape[0]):
        v = int(np.searchsorted(vs, c // k, side="right") - 1)
        x0, y0, x1, y1 = prj.rect[c]
        for yy in range(y0, y1):
            for xx in range(x0, x1):
                t = int(base[v] + yy * tx[v] + xx)
                pairs.append(((t << 32) | int(prj.depth_bits[c]), c))
    pairs.sort()
    assert np.array_equal(fw.keys, np.array([p[0] for p in pairs], np.uint64))
    assert np.array_equal(fw.vals, np.array([p[1] for p in pairs], np.uint32))
    covered = np.zeros(len(pairs), int)
    for t in range(T):
        s0, e0 = fw.ranges[t]
        covered[s0:e0] += 1
        assert np.all((fw.keys[s0:e0] >> np.uint64(32)) == t)
    assert np.all(covered == 1)


def test_permutation_invariance():
    """Reordering the input Gaussians (ids remapped) leaves the image unchanged
    after the depth sort."""
    s = scenes.explicit_frustum(seed=4, n=500)
    rng = np.random.default_rng(9)
    perm = rng.permutation(500)
    a = explicit_forward(s.mu, s.scale, s.quat, s.opacity, s.colour, s.cams, s.wh)[4]
    b = explicit_forward(s.mu[perm], s.scale[perm], s.quat[perm], s.opacity[perm], s.colour[perm],
                         s.cams, s.wh)[4]
    assert np.array_equal(a.image, b.image)


# ------------------------------------------------------------ decode
def _decode_scene(F=4, k=3, hidden=8, M=2, n=12, seed=0):
    s = scenes.tiny_corridor(seed=seed, n_anchors=n, F=F, k=k, hidden=hidden, length=4.0,
                             views=((40, 30, 40.0, 40.0, 20.0, 15.0, (0.0, 0.0, -3.0), 0.0),))
    s.M = M
    s.part = (np.arange(n) * M // n).astype(np.int32)
    rng = np.random.default_rng(seed + 100)
    s.mlp = scenes.init_mlp(rng, M, F, k, hidden)
    return s


def _head_slices(F, k, hidden):
    din = F + 4
    out, p = [], 0
    for dout in (k, 3 * k, 7 * k):
        sl = {}
        for name, size in (("W1", hidden * din), ("b1", hidden), ("W2", dout * hidden),
                           ("b2", dout)):
            sl[name] = slice(p, p + size)
            p += size
        out.append(sl)
    return out


def test_decode_bias_only_closed_form():
    """All weights zero: every head outputs its b2, so opacity = tanh(b2),
    colour = sigmoid(b2), scale = exp(l) sigmoid(b2), rotation = b2/|b2|, and
    mu = x_a + offset exp(l) -- per partition (the indicator of Eq. 6)."""
    s = _decode_scene()
    hs = _head_slices(s.F, s.k, s.hidden)
    for m in range(s.M):
        for h in hs:
            s.mlp[m, h["W1"]] = 0
            s.mlp[m, h["b1"]] = 0
            s.mlp[m, h["W2"]] = 0
    dec = O.decode(s)
    assert dec.av_anchor.size > 0
    for r, a in enumerate(dec.av_anchor):
        m = s.part[a]
        b_o = s.mlp[m, hs[0]["b2"]].astype(np.float64)
        b_c = s.mlp[m, hs[1]["b2"]].astype(np.float64).reshape(s.k, 3)
        b_v = s.mlp[m, hs[2]["b2"]].astype(np.float64).reshape(s.k, 7)
        ls = s.log_scaling[a].astype(np.float64)
        for i in range(s.k):
            c = r * s.k + i
            assert dec.opacity[c] == pytest.approx(math.tanh(b_o[i]), rel=1e-14)
            assert np.allclose(dec.colour[c], 1 / (1 + np.exp(-b_c[i])), rtol=1e-14)
            assert np.allclose(dec.scale[c], np.exp(ls[3:]) / (1 + np.exp(-b_v[i, :3])), rtol=1e-14)
            assert np.allclose(dec.quat[c], b_v[i, 3:] / np.linalg.norm(b_v[i, 3:]), rtol=1e-14)
            mu = s.xyz[a].astype(np.float64) + s.offsets[a, i].astype(np.float64) * np.exp(ls[:3])
            assert np.allclose(dec.mu[c], mu, rtol=1e-14)


def test_decode_view_inputs_distance_and_direction():
    """Eq. 2: a hidden unit that reads only the distance input, or only one
    component of the direction, passes it through ReLU and an identity W2 row
    into z; with tanh undone this recovers |x_a - x_c| and (x_a - x_c)/|.|."""
    s = _decode_scene(M=1, k=4)
    hs = _head_slices(s.F, s.k, s.hidden)
    din = s.F + 4
    W = np.zeros_like(s.mlp, dtype=np.float64)
    # head 0 (opacity): hidden j reads input F+j (dir_x, dir_y, dir_z, delta) with weight 0.1,
    # bias 1 keeps it positive; W2 row j picks hidden j.
    W1 = np.zeros((s.hidden, din)); b1 = np.zeros(s.hidden); W2 = np.zeros((s.k, s.hidden))
    for j in range(min(4, s.k)):
        W1[j, s.F + j] = 0.1
        b1[j] = 1.0
        W2[j, j] = 1.0
    W[0, hs[0]["W1"]] = W1.ravel(); W[0, hs[0]["b1"]] = b1; W[0, hs[0]["W2"]] = W2.ravel()
    s.mlp = W
    dec = O.decode(s)
    xc = np.array([0.0, 0.0, -3.0])
    for r, a in enumerate(dec.av_anchor):
        d = s.xyz[a].astype(np.float64) - xc
        delta = np.linalg.norm(d)
        want = np.concatenate([d / delta, [delta]])[: min(4, s.k)]
        got = (np.arctanh(dec.opacity[r * s.k: r * s.k + min(4, s.k)]) - 1.0) / 0.1
        assert np.allclose(got, want, rtol=1e-9, atol=1e-9)


def test_visibility_rule():
    """An anchor is decoded iff it is in front of the near plane (z > 0.2) and
    projects inside the image grown by 15 % per side."""
    wh = np.array([[100, 80]], np.int32)
    cams = cam1(fx=100, fy=100, cx=50, cy=40)
    z = 2.0
    # u = 100 x / z + 50: the grown image spans u in [-15, 115)
    pts = np.array([[0, 0, z], [0, 0, -z], [0, 0, 0.19], [0, 0, 0.21],
                    [(114.9 - 50) * z / 100, 0, z], [(115.1 - 50) * z / 100, 0, z],
                    [(-14.9 - 50) * z / 100, 0, z], [(-15.1 - 50) * z / 100, 0, z],
                    [0, (91.9 - 40) * z / 100, z], [0, (92.1 - 40) * z / 100, z]])
    av, vs, _ = O.visibility(pts, cams, wh)
    assert list(av) == [0, 3, 4, 6, 8]
    assert list(vs) == [0, 5]


# ------------------------------------------------------------ finite differences
def _fd(f, x, idxs, g, fingerprint, rel_h=1e-6):
    """Central differences of scalar f at x[idxs] against g[idxs]; entries
    whose +-h evaluations change a discrete decision are skipped."""
    base_fp = fingerprint()
    checked = 0
    scale = max(np.max(np.abs(g)), 1e-30)
    for idx in idxs:
        x0 = x[idx]
        h = rel_h * max(1.0, abs(x0))
        x[idx] = x0 + h
        fp, fpp = f(), fingerprint()
        x[idx] = x0 - h
        fm, fpm = f(), fingerprint()
        x[idx] = x0
        if fpp != base_fp or fpm != base_fp:
            continue
        num = (fp - fm) / (2 * h)
        assert abs(num - g[idx]) <= 2e-6 * scale + 1e-9, (idx, num, g[idx])
        checked += 1
    return checked


def _sample(shape, n, rng):
    flat = rng.choice(int(np.prod(shape)), size=min(n, int(np.prod(shape))), replace=False)
    return [np.unravel_index(i, shape) for i in flat]


def test_fd_render_backward_fixed_lists():
    """Reverse pass of Eq. 1 (per-splat mean2d, conic, opacity, colour) against
    central differences of a linear functional of the image, bins held fixed."""
    s = scenes.explicit_frustum(seed=2, n=120, width=48, height=40, fx=45, fy=45, cx=24, cy=20)
    vs = np.array([0, 120], np.int64)
    prj = O.project(s.mu, s.scale, s.quat, s.opacity, s.cams, s.wh, vs)
    keys, vals, ranges = O.bin_sort(prj.depth_bits, prj.rect, s.wh, vs)
    rng = np.random.default_rng(0)
    w = rng.normal(size=3 * 48 * 40)
    st = dict(mean2d=prj.mean2d.copy(), conic=prj.conic.copy(),
              opacity=s.opacity.astype(np.float64).copy(), colour=s.colour.astype(np.float64).copy())
    bg = (0.1, 0.2, 0.3)

    def run():
        return O.render(s.wh, vs, 1, st["mean2d"], st["conic"], st["opacity"], st["colour"],
                        prj.depth_bits, prj.rect, prj.status, 0, ranges, vals, bg)

    f = lambda: float(w @ run().image)
    fpr = lambda: run().hash
    dm, dk, do, dc = O.render_bwd(s.wh, st["mean2d"], st["conic"], st["opacity"], st["colour"],
                                  ranges, vals, w, bg)
    grads = dict(mean2d=dm, conic=dk, opacity=do, colour=dc)
    total = 0
    for name, g in grads.items():
        live = [i for i in _sample(g.shape, 400, rng) if prj.status[i[0]]]
        total += _fd(f, st[name], live[:60], g, fpr)
    assert total > 150


def test_fd_projection_backward():
    """Chain rule of the projection (mean2d and conic w.r.t. mu, scale and the
    quaternion) against central differences of a linear functional."""
    s = scenes.explicit_frustum(seed=6, n=80)
    # push some splats off-axis enough to hit the tangent clamp
    s.mu[:10, 0] *= 3.0
    vs = np.array([0, 80], np.int64)
    rng = np.random.default_rng(1)
    wm, wk = rng.normal(size=(80, 2)), rng.normal(size=(80, 3))
    st = dict(mu=s.mu.astype(np.float64).copy(), scale=s.scale.astype(np.float64).copy(),
              quat=s.quat.astype(np.float64).copy())

    def run():
        return O.project(st["mu"], st["scale"], st["quat"], s.opacity, s.cams, s.wh, vs)

    base = run()
    mask = base.status == 1
    f = lambda: float(np.sum(wm[mask] * run().mean2d[mask]) + np.sum(wk[mask] * run().conic[mask]))
    fpr = lambda: run().status.tobytes()
    dmu, ds, dq = O.project_bwd(st["mu"], st["scale"], st["quat"], base.status, s.cams, s.wh, vs,
                                wm * mask[:, None], wk * mask[:, None])
    total = 0
    for name, g in dict(mu=dmu, scale=ds, quat=dq).items():
        live = [i for i in _sample(g.shape, 300, rng) if mask[i[0]]]
        total += _fd(f, st[name], live[:60], g, fpr)
    assert total > 150


def test_fd_decode_backward():
    """Reverse pass of the partitioned decoder (Eq. 6, Eq. 2) against central
    differences of a linear functional of its outputs."""
    s = _decode_scene(F=4, k=3, hidden=8, M=2, n=16, seed=3)
    rng = np.random.default_rng(2)
    dec = O.decode(s)
    C_ = dec.opacity.shape[0]
    live = (dec.opacity > 0).astype(np.float64)
    W = dict(mu=rng.normal(size=(C_, 3)), scale=rng.normal(size=(C_, 3)),
             quat=rng.normal(size=(C_, 4)), opacity=rng.normal(size=C_),
             colour=rng.normal(size=(C_, 3)))
    for k_ in W:
        W[k_] = W[k_] * (live[:, None] if W[k_].ndim == 2 else live)
    params = dict(xyz=s.xyz.astype(np.float64), feat=s.feat.astype(np.float64),
                  log_scaling=s.log_scaling.astype(np.float64),
                  offsets=s.offsets.astype(np.float64), mlp=s.mlp.astype(np.float64))
    for k_, v in params.items():
        setattr(s, k_, v)
    rows = (dec.av_anchor, dec.view_start, dec.row_flag)

    def f():
        d = O.decode(s, rows=rows)
        return float(sum(np.sum(W[n] * getattr(d, n)) for n in W))

    fpr = lambda: (O.decode(s, rows=rows).opacity > 0).tobytes()
    g = O.decode_bwd(s, dec, W["mu"], W["scale"], W["quat"], W["opacity"], W["colour"])
    total = 0
    for name in params:
        total += _fd(f, params[name], _sample(params[name].shape, 60, rng), g[name], fpr)
    assert total > 150


def test_fd_end_to_end_l1_anchor_path():
    """L1 loss (Eq. 3, L1 term) of the whole anchor path against central
    differences w.r.t. anchor positions, features, scalings, offsets and MLP
    weights; entries whose perturbation flips any discrete decision
    (visibility, culling, tile rectangles, sort order, skip/stop, sign of the
    residual) are skipped."""
    s = scenes.tiny_corridor(seed=3, n_anchors=150, F=4, k=3, hidden=8, length=12.0,
                             views=((40, 28, 36.0, 36.0, 20.0, 14.0, (0.0, 0.0, 2.0), 0.0),
                                    (34, 20, 30.0, 30.0, 17.0, 10.0, (0.2, 0.0, 2.5), 4.0)))
    for k_ in ("xyz", "feat", "log_scaling", "offsets", "mlp"):
        setattr(s, k_, getattr(s, k_).astype(np.float64))
    L, g, fw0 = O.loss_and_grads_anchor(s)
    tgt = O.targets_flat(s)
    rng = np.random.default_rng(3)

    def f():
        return O.l1(s.wh, O.forward_anchor(s).ren.image, tgt)[0]

    def fpr():
        fw = O.forward_anchor(s)
        return (fw.dec.av_anchor.tobytes(), (fw.dec.opacity > 0).tobytes(), fw.prj.status.tobytes(),
                fw.prj.rect.tobytes(), fw.vals.tobytes(), fw.ranges.tobytes(), fw.ren.hash,
                np.sign(fw.ren.image - tgt).tobytes())

    total = 0
    for name in ("xyz", "feat", "log_scaling", "offsets", "mlp"):
        x = getattr(s, name)
        total += _fd(f, x, _sample(x.shape, 40, rng), g[name], fpr)
    assert total > 100
    assert np.abs(g["mlp"]).max() > 0 and np.abs(g["xyz"]).max() > 0


def test_l1_closed_form():
    wh = np.array([[2, 1], [1, 1]], np.int32)
    img = np.array([0.5, 0.1, 0.2, 0.9, 0.3, 0.3, 1.0, 0.0, 0.5])
    tgt = np.array([0.0, 0.3, 0.2, 0.4, 0.3, 0.7, 0.0, 0.5, 0.25])
    L, d = O.l1(wh, img, tgt)
    v0 = np.abs(img[:6] - tgt[:6]).mean()
    v1 = np.abs(img[6:] - tgt[6:]).mean()
    assert L == pytest.approx(v0 + v1, rel=1e-15)
    assert np.allclose(d[:6], np.sign(img[:6] - tgt[:6]) / 6)
    assert np.allclose(d[6:], np.sign(img[6:] - tgt[6:]) / 3)
