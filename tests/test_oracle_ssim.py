"""Pins of the oracle's structural term of Eq. 3 (L_SSIM = 1 - SSIM, 11x11
Gaussian window, sigma 1.5, zero padding, C1 = 0.01^2, C2 = 0.03^2), each
against something other than the oracle itself: the fixed point x = y, closed
forms on constant and checkerboard images, SciPy's Gaussian filter for the
windowed moments, symmetry, additivity over views and central differences of
its own loss for the hand-derived gradient."""
import numpy as np
import pytest
from scipy import ndimage

from oracle import oracle as O

C1, C2 = 0.01 ** 2, 0.03 ** 2


def _planes(wh, a):
    out, at = [], 0
    for w, h in wh:
        out.append(a[at:at + 3 * w * h].reshape(3, h, w))
        at += 3 * w * h
    return out


def test_identical_images_give_zero_loss_and_zero_gradient():
    rng = np.random.default_rng(0)
    wh = np.array([[23, 17], [8, 5]])
    x = rng.uniform(size=3 * (23 * 17 + 8 * 5))
    L, d, m = O.ssim(wh, x, x, want_map=True)
    assert abs(L) < 1e-13
    assert np.abs(m - 1).max() < 1e-13
    assert np.abs(d).max() < 1e-15   # S = 1 is the maximum of every map entry


def test_constant_images_interior_closed_form():
    a, b = 0.3, 0.7
    wh = np.array([[30, 24]])
    x = np.full(3 * 30 * 24, a)
    y = np.full(3 * 30 * 24, b)
    _, _, m = O.ssim(wh, x, y, want_map=True, want_grad=False)
    m = m.reshape(3, 24, 30)
    want = (2 * a * b + C1) / (a * a + b * b + C1)   # zero variances: the second factor is C2 / C2
    interior = m[:, 5:19, 5:25]
    assert np.allclose(interior, want, rtol=1e-12, atol=0)
    # the zero padding lowers the means at the border: the border differs
    assert abs(m[0, 0, 0] - want) > 1e-3


def test_checkerboard_anticorrelated_closed_form():
    """x = a + d (-1)^(i+j), y = 2a - x.  With the separable window g, the
    windowed mean of the checkerboard is s e^2 (e = sum_i g_i (-1)^i, s the
    parity sign), so mu_x = a + d s e^2, mu_y = a - d s e^2, var_x = var_y =
    d^2 (1 - e^4) and cov = -var_x."""
    a, d = 0.5, 0.2
    W, H = 28, 26
    jj, ii = np.meshgrid(np.arange(W), np.arange(H))
    chk = np.where((ii + jj) % 2 == 0, 1.0, -1.0)
    x = np.tile((a + d * chk).ravel(), 3)
    y = 2 * a - x
    _, _, m = O.ssim(np.array([[W, H]]), x, y, want_map=True, want_grad=False)
    m = m.reshape(3, H, W)
    k = np.arange(-5, 6)
    g = np.exp(-k * k / (2 * 1.5 ** 2))
    g /= g.sum()
    e = float(np.sum(g * (-1.0) ** np.abs(k)))
    var = d * d * (1 - e ** 4)
    for s in (1.0, -1.0):
        mx, my = a + d * s * e * e, a - d * s * e * e
        want = (2 * mx * my + C1) * (-2 * var + C2) / ((mx * mx + my * my + C1) * (2 * var + C2))
        sel = chk[5:H - 5, 5:W - 5] == s
        assert np.allclose(m[:, 5:H - 5, 5:W - 5][:, sel], want, rtol=1e-10, atol=1e-14)
    assert want < 0   # anti-correlated structure: negative SSIM


def test_windowed_moments_match_scipy_gaussian_filter():
    rng = np.random.default_rng(1)
    wh = np.array([[19, 14]])
    x = rng.uniform(size=3 * 19 * 14)
    y = rng.uniform(size=3 * 19 * 14)
    _, _, m = O.ssim(wh, x, y, want_map=True, want_grad=False)
    X, Y = x.reshape(3, 14, 19), y.reshape(3, 14, 19)

    def blur(z):   # radius int(truncate * sigma + 0.5) = 5, normalised, zero padding
        return ndimage.gaussian_filter(z, 1.5, mode="constant", cval=0.0, truncate=5 / 1.5)

    for c in range(3):
        mx, my = blur(X[c]), blur(Y[c])
        vx, vy, cv = blur(X[c] ** 2) - mx ** 2, blur(Y[c] ** 2) - my ** 2, blur(X[c] * Y[c]) - mx * my
        S = (2 * mx * my + C1) * (2 * cv + C2) / ((mx ** 2 + my ** 2 + C1) * (vx + vy + C2))
        assert np.allclose(m.reshape(3, 14, 19)[c], S, rtol=1e-11, atol=1e-13)


def test_symmetric_and_additive_over_views():
    rng = np.random.default_rng(2)
    wh = np.array([[11, 9], [6, 13]])
    n = 3 * (11 * 9 + 6 * 13)
    x, y = rng.uniform(size=n), rng.uniform(size=n)
    L, _, m = O.ssim(wh, x, y, want_map=True, want_grad=False)
    L2, _, m2 = O.ssim(wh, y, x, want_map=True, want_grad=False)
    assert L == pytest.approx(L2, rel=1e-14)
    assert np.allclose(m, m2, rtol=1e-13)
    n0 = 3 * 11 * 9
    La = O.ssim(wh[:1], x[:n0], y[:n0], want_grad=False)[0]
    Lb = O.ssim(wh[1:], x[n0:], y[n0:], want_grad=False)[0]
    assert L == pytest.approx(La + Lb, rel=1e-14)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(3)
    wh = np.array([[12, 9], [7, 6]])
    n = 3 * (12 * 9 + 7 * 6)
    x, y = rng.uniform(size=n), rng.uniform(size=n)
    _, d, _ = O.ssim(wh, x, y)
    for i in rng.choice(n, size=40, replace=False):
        h = 1e-6
        xp, xm = x.copy(), x.copy()
        xp[i] += h
        xm[i] -= h
        num = (O.ssim(wh, xp, y, want_grad=False)[0] - O.ssim(wh, xm, y, want_grad=False)[0]) / (2 * h)
        assert num == pytest.approx(d[i], rel=1e-6, abs=1e-10)


def test_photometric_combines_both_terms():
    rng = np.random.default_rng(4)
    wh = np.array([[10, 8]])
    x, y = rng.uniform(size=240), rng.uniform(size=240)
    L, d, L1, Ls = O.photometric(wh, x, y, lam=0.8)
    assert L == pytest.approx(0.8 * L1 + 0.2 * Ls, rel=1e-15)
    assert L1 == pytest.approx(np.abs(x - y).mean(), rel=1e-14)
    _, d1 = O.l1(wh, x, y)
    _, ds, _ = O.ssim(wh, x, y)
    assert np.allclose(d, 0.8 * d1 + 0.2 * ds, rtol=1e-14, atol=1e-18)
