"""ctypes front-end of the FP64 CPU oracle (`gs_oracle.c`).

TEST INFRASTRUCTURE ONLY: imported by the test-suite, by the smoke check and
by the CPU-baseline leg of the benchmark, never by the product path.  It does
not import the CUDA package and the CUDA package does not import it.

Each wrapper takes NumPy arrays (any float dtype; converted to float64) and
returns NumPy arrays.  The paper passages each step follows are cited in the
C source next to each function.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gs_oracle.c")
_LIB = os.path.join(_HERE, "libgs_oracle.so")

BAND = 1e-4      # relative band around a threshold inside which FP32 may decide differently
BAND_T = 2e-4    # same for the transmittance stop test (a product of many FP32 factors, ~1e-5 off)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               "-o", _LIB, _SRC, "-lm"]
        subprocess.check_call(cmd)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        _declare(_lib)
    return _lib


_dp = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
_ip = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_lp = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
_u8 = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_u32 = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_u64 = np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")


class _u64n:
    """uint64 array pointer that also accepts None (NULL)."""
    @classmethod
    def from_param(cls, a):
        return None if a is None else _u64.from_param(a)


class _dpn:
    """float64 array pointer that also accepts None (NULL)."""
    @classmethod
    def from_param(cls, a):
        return None if a is None else _dp.from_param(a)


def _declare(L):
    i, l, d = C.c_int, C.c_long, C.c_double
    L.gso_visibility.restype = l
    L.gso_visibility.argtypes = [i, _dp, i, _dp, _ip, d, _ip, _lp, l, _u8]
    L.gso_decode.restype = i
    L.gso_decode.argtypes = [i, i, i, i, i, _dp, _dp, _dp, _dp, _ip, _dp, i, _dp, _ip, l, _ip,
                             _lp, d, _dp, _dp, _dp, _dp, _dp, _u8]
    L.gso_project.restype = i
    L.gso_project.argtypes = [l, i, i, _lp, _dp, _ip, _dp, _dp, _dp, _dp, d, _dp, _dp, _dp, _dp,
                              _ip, _ip, _ip, _u8, _ip]
    L.gso_bin_sort.restype = l
    L.gso_bin_sort.argtypes = [l, i, i, _lp, _ip, _u32, _ip, l, _u64, _u32, _u32]
    L.gso_render.restype = i
    L.gso_render.argtypes = [i, _ip, l, i, _lp, _dp, _dp, _dp, _dp, _u32, _ip, _ip, i, _u32,
                             _u32, _dp, d, d, _dp, _dp, _ip, C.POINTER(C.c_long), _u8,
                             C.POINTER(C.c_uint64)]
    L.gso_l1.restype = d
    L.gso_l1.argtypes = [i, _ip, _dp, _dp, _dp]
    L.gso_ssim.restype = d
    L.gso_ssim.argtypes = [i, _ip, _dp, _dp, _dpn, _dpn]
    L.gso_adam.restype = None
    L.gso_adam.argtypes = [l, _dp, _dp, _dp, _dp, l, d, d, d, d]
    L.gso_densify_stats.restype = None
    L.gso_densify_stats.argtypes = [l, i, _ip, _ip, _dp, _dp, _dp, _ip, _dp, _ip]
    L.gso_voxelize.restype = l
    L.gso_voxelize.argtypes = [l, _f32p, C.c_float, _u64n, l, _u64, _f32p, l]
    L.gso_loop_closure.restype = None
    L.gso_loop_closure.argtypes = [i, _dp, i, _dp, _dp, _ip, d, d, _dp, _ip, _u8]
    L.gso_densify_masks.restype = None
    L.gso_densify_masks.argtypes = [l, i, _f32p, _ip, _f32p, _ip, C.c_float, C.c_float, i, _u8, _u8]
    L.gso_render_bwd.restype = i
    L.gso_render_bwd.argtypes = [i, _ip, l, _dp, _dp, _dp, _dp, _u32, _u32, _dp, _dp, _dp,
                                 _dp, _dp, _dp]
    L.gso_project_bwd.restype = i
    L.gso_project_bwd.argtypes = [l, i, i, _lp, _dp, _ip, _dp, _dp, _dp, _ip, _dp, _dp, _dp,
                                  _dp, _dp]
    L.gso_decode_bwd.restype = i
    L.gso_decode_bwd.argtypes = [i, i, i, i, i, _dp, _dp, _dp, _dp, _ip, _dp, i, _dp, _ip, l,
                                 _ip, _lp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp, _dp]
    L.gso_mlp_size.restype = l
    L.gso_mlp_size.argtypes = [i, i, i]


def _f64(a):
    return np.ascontiguousarray(np.asarray(a, np.float64))


def _i32(a):
    return np.ascontiguousarray(np.asarray(a, np.int32))


def tiles_of(wh):
    """(TX, TY, tile_base, total tiles) for each view of a 16x16 tiling."""
    wh = np.asarray(wh, np.int64).reshape(-1, 2)
    tx = (wh[:, 0] + 15) // 16
    ty = (wh[:, 1] + 15) // 16
    n = tx * ty
    base = np.concatenate([[0], np.cumsum(n)[:-1]])
    return tx, ty, base, int(n.sum())


# --------------------------------------------------------------------------
@dataclass
class Decoded:
    av_anchor: np.ndarray   # [R] int32
    view_start: np.ndarray  # [V+1] int64 (rows)
    row_flag: np.ndarray    # [R] uint8
    k: int
    mu: np.ndarray = None
    scale: np.ndarray = None
    quat: np.ndarray = None
    opacity: np.ndarray = None
    colour: np.ndarray = None
    cand_flag: np.ndarray = None


def visibility(xyz, cams, wh, band=BAND):
    xyz = _f64(xyz); cams = _f64(cams); wh = _i32(wh)
    N, V = xyz.shape[0], cams.shape[0]
    cap = N * V
    av = np.zeros(max(cap, 1), np.int32)
    vs = np.zeros(V + 1, np.int64)
    fl = np.zeros(max(cap, 1), np.uint8)
    r = lib().gso_visibility(N, xyz, V, cams, wh, band, av, vs, cap, fl)
    assert r >= 0
    return av[:r].copy(), vs, fl[:r].copy()


def decode(scene, band=BAND, rows=None):
    """Visibility (a0) + decode (a1) of every (view, anchor) row."""
    s = scene
    if rows is None:
        av, vs, rf = visibility(s.xyz, s.cams, s.wh, band)
    else:
        av, vs, rf = rows
    R = av.shape[0]
    C_ = R * s.k
    mu = np.zeros((C_, 3)); sc = np.zeros((C_, 3)); q = np.zeros((C_, 4))
    op = np.zeros(C_); col = np.zeros((C_, 3)); cf = np.zeros(max(C_, 1), np.uint8)
    lib().gso_decode(s.N, s.F, s.k, s.hidden, s.M, _f64(s.xyz), _f64(s.feat),
                     _f64(s.log_scaling), _f64(s.offsets), _i32(s.part), _f64(s.mlp),
                     s.V, _f64(s.cams), _i32(s.wh), R, _i32(av), vs, band, mu, sc, q, op, col, cf)
    return Decoded(av, vs, rf, s.k, mu, sc, q, op, col, cf[:C_])


@dataclass
class Projected:
    mean2d: np.ndarray
    conic: np.ndarray
    cov2d: np.ndarray
    depth: np.ndarray
    rect: np.ndarray      # [C,4] int32 x0,y0,x1,y1
    tiles: np.ndarray
    status: np.ndarray
    flag: np.ndarray          # bit 0: presence decision near a threshold; bit 1: tile rectangle
    fp64_branch: np.ndarray

    @property
    def depth_bits(self):
        return self.depth.astype(np.float32).view(np.uint32)


def project(mu, scale, quat, opacity, cams, wh, view_start, k=1, band=BAND):
    C_ = mu.shape[0]
    V = np.asarray(cams).shape[0]
    out = Projected(np.zeros((C_, 2)), np.zeros((C_, 3)), np.zeros((C_, 3)), np.zeros(C_),
                    np.zeros((C_, 4), np.int32), np.zeros(C_, np.int32), np.zeros(C_, np.int32),
                    np.zeros(C_, np.uint8), np.zeros(C_, np.int32))
    lib().gso_project(C_, k, V, np.ascontiguousarray(view_start, np.int64), _f64(cams), _i32(wh),
                      _f64(mu), _f64(scale), _f64(quat), _f64(opacity), band, out.mean2d,
                      out.conic, out.cov2d, out.depth, out.rect, out.tiles, out.status, out.flag,
                      out.fp64_branch)
    return out


def bin_sort(depth_bits, rect, wh, view_start, k=1):
    depth_bits = np.ascontiguousarray(depth_bits, np.uint32)
    rect = _i32(rect)
    C_ = depth_bits.shape[0]
    V = np.asarray(wh).reshape(-1, 2).shape[0]
    P = int(((rect[:, 2] - rect[:, 0]) * (rect[:, 3] - rect[:, 1])).sum()) if C_ else 0
    _, _, _, T = tiles_of(wh)
    keys = np.zeros(max(P, 1), np.uint64)
    vals = np.zeros(max(P, 1), np.uint32)
    ranges = np.zeros(2 * T, np.uint32)
    n = lib().gso_bin_sort(C_, k, V, np.ascontiguousarray(view_start, np.int64), _i32(wh),
                           depth_bits, rect, P, keys, vals, ranges)
    assert n == P
    return keys[:P].copy(), vals[:P].copy(), ranges.reshape(T, 2)


@dataclass
class Rendered:
    image: np.ndarray      # flat [sum_v 3*H*W], per view planar [3,H,W]
    T_final: np.ndarray    # flat [sum_v H*W]
    last: np.ndarray
    pix_flag: np.ndarray
    nev: int
    hash: int

    def view_image(self, wh, v):
        wh = np.asarray(wh).reshape(-1, 2)
        base = int(sum(3 * int(w) * int(h) for w, h in wh[:v]))
        w, h = (int(x) for x in wh[v])
        return self.image[base:base + 3 * w * h].reshape(3, h, w)


def render(wh, view_start, k, mean2d, conic, opacity, colour, depth_bits, rect, status,
           mode=0, ranges=None, vals=None, bg=(0.0, 0.0, 0.0), band=BAND, band_t=BAND_T):
    wh = _i32(wh).reshape(-1, 2)
    V = wh.shape[0]
    npix = int((wh[:, 0].astype(np.int64) * wh[:, 1]).sum())
    C_ = np.asarray(opacity).shape[0]
    if ranges is None:
        ranges = np.zeros((1, 2), np.uint32)
        vals = np.zeros(1, np.uint32)
    image = np.zeros(3 * npix); Tf = np.zeros(npix); last = np.zeros(npix, np.int32)
    pf = np.zeros(npix, np.uint8)
    nev = C.c_long(0); h = C.c_uint64(0)
    lib().gso_render(V, wh, C_, k, np.ascontiguousarray(view_start, np.int64), _f64(mean2d),
                     _f64(conic), _f64(opacity), _f64(colour),
                     np.ascontiguousarray(depth_bits, np.uint32), _i32(rect), _i32(status), mode,
                     np.ascontiguousarray(ranges, np.uint32).reshape(-1),
                     np.ascontiguousarray(vals, np.uint32), _f64(bg), band, band_t, image, Tf,
                     last, C.byref(nev), pf, C.byref(h))
    return Rendered(image, Tf, last, pf, int(nev.value), int(h.value))


def l1(wh, image, target):
    image = _f64(image).reshape(-1); target = _f64(target).reshape(-1)
    d = np.zeros_like(image)
    L = lib().gso_l1(np.asarray(wh).reshape(-1, 2).shape[0], _i32(wh), image, target, d)
    return L, d


def ssim(wh, image, target, want_map=False, want_grad=True):
    """Structural term of Eq. 3: L_SSIM = sum over views of (1 - mean SSIM),
    its gradient with respect to image and (optionally) the SSIM map."""
    image = _f64(image).reshape(-1); target = _f64(target).reshape(-1)
    wh = _i32(wh).reshape(-1, 2)
    d = np.zeros_like(image) if want_grad else None
    m = np.zeros_like(image) if want_map else None
    L = lib().gso_ssim(wh.shape[0], wh, image, target, m, d)
    return L, d, m


def photometric(wh, image, target, lam=0.8):
    """Eq. 3: L = lam L1 + (1 - lam) L_SSIM and dL/dimage; also the two terms."""
    L1, d1 = l1(wh, image, target)
    Ls, ds, _ = ssim(wh, image, target)
    return lam * L1 + (1 - lam) * Ls, lam * d1 + (1 - lam) * ds, L1, Ls


def adam(param, grad, m, v, step, lr, b1=0.9, b2=0.999, eps=1e-15):
    """One Adam step with bias correction (t = step >= 1); returns new (param, m, v)."""
    p, m, v = _f64(param).copy(), _f64(m).copy(), _f64(v).copy()
    lib().gso_adam(p.size, p.reshape(-1), _f64(grad).reshape(-1), m.reshape(-1), v.reshape(-1), int(step),
                   float(lr), float(b1), float(b2), float(eps))
    return p, m, v


def densify_stats(row_anchor, tiles, opacity, sgrad, N, k, accum=None):
    """Accumulates one iteration's densification statistics into `accum` =
    (grad_accum [N k], offset_denom [N k], opacity_accum [N], anchor_denom [N])."""
    if accum is None:
        accum = (np.zeros(N * k), np.zeros(N * k, np.int32), np.zeros(N), np.zeros(N, np.int32))
    ga, od, oa, ad = (np.ascontiguousarray(a) for a in accum)
    ra = _i32(row_anchor)
    lib().gso_densify_stats(ra.size, int(k), ra, _i32(tiles), _f64(opacity).reshape(-1),
                            _f64(sgrad).reshape(-1), ga, od, oa, ad)
    return ga, od, oa, ad


def densify_masks(grad_accum, offset_denom, opacity_accum, anchor_denom, k, grad_thr, opacity_thr, min_count):
    """Growth mask [N k] and pruning mask [N] (uint8) from float32 statistics."""
    ga = np.ascontiguousarray(grad_accum, np.float32)
    oa = np.ascontiguousarray(opacity_accum, np.float32)
    N = oa.size
    grow = np.zeros(N * k, np.uint8)
    prune = np.zeros(N, np.uint8)
    lib().gso_densify_masks(N, int(k), ga, _i32(offset_denom), oa, _i32(anchor_denom), float(grad_thr),
                            float(opacity_thr), int(min_count), grow, prune)
    return grow, prune


KEY_BIAS = 1 << 20


def voxelize(points, eps, existing=None, cap=None):
    """Eq. 4: the new voxel keys (ascending uint64) of float32 points at voxel
    size eps, minus `existing` (sorted uint64), and their float32 centres.
    Raises ValueError for a voxel index outside (-2^20, 2^20)."""
    pts = np.ascontiguousarray(points, np.float32).reshape(-1, 3)
    P = pts.shape[0]
    cap = P if cap is None else int(cap)
    keys = np.zeros(max(cap, 1), np.uint64)
    centres = np.zeros((max(cap, 1), 3), np.float32)
    ex = None if existing is None or len(existing) == 0 else np.ascontiguousarray(existing, np.uint64)
    n = lib().gso_voxelize(P, pts.reshape(-1), np.float32(eps), ex, 0 if ex is None else ex.size, keys,
                           centres.reshape(-1), cap)
    if n == np.iinfo(np.int64).min:
        raise ValueError("voxel index out of range")
    if n < 0:
        return None, None, -n
    return keys[:n], centres[:n], n


def loop_closure(xyz, cams_old, cams_new, wh, z_far, band=BAND):
    """Eq. 7 applied with the nearest-keyframe rule: new anchor positions,
    the keyframe used per anchor (-1: none) and near-threshold flags."""
    x = _f64(xyz).reshape(-1, 3)
    N = x.shape[0]
    wh = _i32(wh).reshape(-1, 2)
    K = wh.shape[0]
    out = np.zeros_like(x)
    assigned = np.zeros(N, np.int32)
    flag = np.zeros(N, np.uint8)
    lib().gso_loop_closure(N, x.reshape(-1), K, _f64(cams_old).reshape(-1), _f64(cams_new).reshape(-1), wh,
                           float(z_far), float(band), out.reshape(-1), assigned, flag)
    return out, assigned, flag


def _proj_matrix(cam):
    """P = K [R | t] of a camera record (fx, fy, cx, cy, R, t), zero skew."""
    c = _f64(cam).reshape(-1)
    K = np.array([[c[0], 0, c[2]], [0, c[1], c[3]], [0, 0, 1.0]])
    return K @ np.hstack([c[4:13].reshape(3, 3), c[13:16, None]])


def _skew(v):
    return np.array([[0, -v[2], v[1]], [v[2], 0, -v[0]], [-v[1], v[0], 0]])


def fundamental(cam1, cam2):
    """Eq. 5: F = [e2]x P2 P1^+ with e2 = P2 C1, C1 the centre of camera 1
    (the right null space of P1, here -R1^T t1 in homogeneous form)."""
    P1, P2 = _proj_matrix(cam1), _proj_matrix(cam2)
    c = _f64(cam1).reshape(-1)
    C1 = np.append(-c[4:13].reshape(3, 3).T @ c[13:16], 1.0)
    e2 = P2 @ C1
    return _skew(e2) @ P2 @ np.linalg.pinv(P1)


def flow_triangulate(cam1, cam2, wh, flow, samples, tau, band=1e-9):
    """Correspondence filtering (Eq. 5) and linear triangulation (Sec. III,
    Flow Densification), FP64.  For each sampled pixel x = (px, py, 1) of
    keyframe 1 and x' = x + flow: residual = |x'^T F x|, kept iff < tau.
    Kept pairs are triangulated by linear least squares on the four DLT rows
    (x P1[2] - P1[0], y P1[2] - P1[1], x' P2[2] - P2[0], y' P2[2] - P2[1]) with
    the homogeneous coordinate fixed to 1.  Returns (residual [N], keep [N],
    flag [N]: |residual - tau| within band of the terms' scale, points [M, 3]
    of the kept samples in sample order)."""
    W, H = int(wh[0]), int(wh[1])
    F = fundamental(cam1, cam2)
    q = np.asarray(samples, np.int64)
    fl = _f64(flow).reshape(H * W, 2)[q]
    x = np.stack([q % W, q // W, np.ones(len(q))], 1).astype(np.float64)
    xp = x.copy()
    xp[:, :2] += fl
    r = np.abs(np.einsum("ni,ij,nj->n", xp, F, x))
    scale = np.einsum("ni,ij,nj->n", np.abs(xp), np.abs(F), np.abs(x))
    keep = r < tau
    flag = np.abs(r - tau) <= band * (tau + scale)
    P1, P2 = _proj_matrix(cam1), _proj_matrix(cam2)
    pts = []
    for i in np.nonzero(keep)[0]:
        A = np.stack([x[i, 0] * P1[2] - P1[0], x[i, 1] * P1[2] - P1[1],
                      xp[i, 0] * P2[2] - P2[0], xp[i, 1] * P2[2] - P2[1]])
        pts.append(np.linalg.lstsq(A[:, :3], -A[:, 3], rcond=None)[0])
    return r, keep, flag, np.array(pts).reshape(-1, 3)


def render_bwd(wh, mean2d, conic, opacity, colour, ranges, vals, dimage, bg=(0.0, 0.0, 0.0)):
    wh = _i32(wh).reshape(-1, 2)
    C_ = np.asarray(opacity).shape[0]
    dm = np.zeros((C_, 2)); dk = np.zeros((C_, 3)); do = np.zeros(C_); dc = np.zeros((C_, 3))
    lib().gso_render_bwd(wh.shape[0], wh, C_, _f64(mean2d), _f64(conic), _f64(opacity),
                         _f64(colour), np.ascontiguousarray(ranges, np.uint32).reshape(-1),
                         np.ascontiguousarray(vals, np.uint32), _f64(bg), _f64(dimage), dm, dk,
                         do, dc)
    return dm, dk, do, dc


def project_bwd(mu, scale, quat, status, cams, wh, view_start, dmean2d, dconic, k=1):
    C_ = mu.shape[0]
    V = np.asarray(cams).shape[0]
    dmu = np.zeros((C_, 3)); ds = np.zeros((C_, 3)); dq = np.zeros((C_, 4))
    lib().gso_project_bwd(C_, k, V, np.ascontiguousarray(view_start, np.int64), _f64(cams),
                          _i32(wh), _f64(mu), _f64(scale), _f64(quat), _i32(status),
                          _f64(dmean2d), _f64(dconic), dmu, ds, dq)
    return dmu, ds, dq


def decode_bwd(scene, dec: Decoded, dmu, dscale, dquat, dopacity, dcolour):
    s = scene
    N = s.N
    dxyz = np.zeros((N, 3)); dfeat = np.zeros((N, s.F)); dls = np.zeros((N, 6))
    doff = np.zeros((N, s.k, 3)); dmlp = np.zeros_like(_f64(s.mlp))
    lib().gso_decode_bwd(N, s.F, s.k, s.hidden, s.M, _f64(s.xyz), _f64(s.feat),
                         _f64(s.log_scaling), _f64(s.offsets), _i32(s.part), _f64(s.mlp), s.V,
                         _f64(s.cams), _i32(s.wh), dec.av_anchor.shape[0], _i32(dec.av_anchor),
                         dec.view_start, _f64(dmu), _f64(dscale), _f64(dquat), _f64(dopacity),
                         _f64(dcolour), dxyz, dfeat, dls, doff, dmlp)
    return dict(xyz=dxyz, feat=dfeat, log_scaling=dls, offsets=doff, mlp=dmlp)


def mlp_size(F, k, hidden):
    return int(lib().gso_mlp_size(F, k, hidden))


# --------------------------------------------------------------------------
# Whole-path helpers (forward and reverse) used by the self-checks and the
# CPU baseline.

@dataclass
class Forward:
    dec: Decoded | None
    prj: Projected
    keys: np.ndarray
    vals: np.ndarray
    ranges: np.ndarray
    ren: Rendered
    colour: np.ndarray
    opacity: np.ndarray
    view_start_c: np.ndarray   # candidate offsets per view, in rows
    k: int


def forward_explicit(scene, bg=(0.0, 0.0, 0.0), mode=0):
    s = scene
    vs = np.array([0, s.mu.shape[0]], np.int64)
    prj = project(s.mu, s.scale, s.quat, s.opacity, s.cams, s.wh, vs, 1)
    keys, vals, ranges = bin_sort(prj.depth_bits, prj.rect, s.wh, vs, 1)
    ren = render(s.wh, vs, 1, prj.mean2d, prj.conic, s.opacity, s.colour, prj.depth_bits,
                 prj.rect, prj.status, mode, ranges, vals, bg)
    return Forward(None, prj, keys, vals, ranges, ren, _f64(s.colour), _f64(s.opacity), vs, 1)


def forward_anchor(scene, bg=(0.0, 0.0, 0.0), mode=0):
    s = scene
    dec = decode(s)
    prj = project(dec.mu, dec.scale, dec.quat, dec.opacity, s.cams, s.wh, dec.view_start, s.k)
    keys, vals, ranges = bin_sort(prj.depth_bits, prj.rect, s.wh, dec.view_start, s.k)
    ren = render(s.wh, dec.view_start, s.k, prj.mean2d, prj.conic, dec.opacity, dec.colour,
                 prj.depth_bits, prj.rect, prj.status, mode, ranges, vals, bg)
    return Forward(dec, prj, keys, vals, ranges, ren, dec.colour, dec.opacity, dec.view_start,
                   s.k)


def targets_flat(scene):
    return np.concatenate([t.reshape(-1) for t in scene.targets]).astype(np.float64)


def loss_and_grads_anchor(scene, bg=(0.0, 0.0, 0.0), dimage=None):
    """L1 loss of the anchor path and its gradient w.r.t. every anchor
    parameter and MLP weight (oracle end to end)."""
    s = scene
    fw = forward_anchor(s, bg)
    L, dimg = l1(s.wh, fw.ren.image, targets_flat(s))
    if dimage is not None:
        dimg = dimage
    dm, dk, do, dc = render_bwd(s.wh, fw.prj.mean2d, fw.prj.conic, fw.opacity, fw.colour,
                                fw.ranges, fw.vals, dimg, bg)
    dmu, ds, dq = project_bwd(fw.dec.mu, fw.dec.scale, fw.dec.quat, fw.prj.status, s.cams, s.wh,
                              fw.dec.view_start, dm, dk, s.k)
    g = decode_bwd(s, fw.dec, dmu, ds, dq, do, dc)
    return L, g, fw
