"""Seeded synthetic inputs for the anchor-Gaussian rendering path.

This module only *draws* inputs; it holds none of the method's arithmetic
(no decoding, projection of Gaussians, sorting, compositing, fundamental
matrix or triangulation).  Both the CUDA path and the FP64 CPU oracle are fed
from here, so the two always see byte-identical inputs.  The one pinhole
reprojection here (`flow_pair`) synthesises what the optical-flow network of
Sec. III would deliver: the input of the flow densification, not its method.

Every generator uses NumPy's PCG64 (`np.random.default_rng`), draws in the
fixed order written in its docstring, draws in FP64 and casts to FP32.

World frame (OpenCV): x right, y down, z forward.  Cameras sit 1.6 m above
the ground plane (ground at y = +1.6), facades stand at x = +-7 m and are 10 m
tall (y in [-8.4, 1.6]).  These corridors stand in for the long outdoor
driving sequences the paper maps (KITTI / Oxford RobotCar / Malaga, Sec. IV-A),
which are not available here.

Data formats shared with the library (interfaces, not arithmetic):

* camera  : float32[16] = fx, fy, cx, cy, R (3x3 row-major, world->camera), t (3)
* view    : int32[2]    = width, height in pixels
* MLP set : one float32 vector per partition, heads in the order
            (opacity, colour, covariance), each head stored as
            W1[H][Din], b1[H], W2[Dout][H], b2[Dout] with Din = F + 4 and
            Dout = k, 3k, 7k (Scaffold-GS decoder heads, Sec. III-A / Eq. 6).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Corridor geometry (metres).
CELL = 0.2            # anchor voxel pitch of the synthetic corridors
HALF_WIDTH = 7.0      # facades at x = +-7
GROUND_Y = 1.6        # ground plane (camera height 1.6 m)
FACADE_TOP = -8.4     # facades are 10 m tall
N_GROUND = int(round(2 * HALF_WIDTH / CELL))            # 70 cells across
N_FACADE = int(round((GROUND_Y - FACADE_TOP) / CELL))   # 50 cells up each facade
CELLS_PER_SLICE = N_GROUND + 2 * N_FACADE               # 170 cells per 0.2 m slice


def mlp_param_count(F: int, k: int, hidden: int) -> int:
    """Floats in one packed partition MLP set (three two-layer heads)."""
    din = F + 4
    total = 0
    for dout in (k, 3 * k, 7 * k):
        total += hidden * din + hidden + dout * hidden + dout
    return total


@dataclass
class Scene:
    """A seeded synthetic mapping problem (anchors + MLP sets + keyframes)."""
    name: str
    # anchors
    xyz: np.ndarray | None = None          # [N,3] f32
    feat: np.ndarray | None = None         # [N,F] f32
    log_scaling: np.ndarray | None = None  # [N,6] f32
    offsets: np.ndarray | None = None      # [N,k,3] f32
    part: np.ndarray | None = None         # [N] i32, non-decreasing
    mlp: np.ndarray | None = None          # [M, P] f32 packed per partition
    F: int = 0
    k: int = 0
    hidden: int = 0
    M: int = 0
    # explicit Gaussians (scene that enters at projection)
    mu: np.ndarray | None = None           # [G,3]
    scale: np.ndarray | None = None        # [G,3]
    quat: np.ndarray | None = None         # [G,4] (w,x,y,z), unit
    opacity: np.ndarray | None = None      # [G]
    colour: np.ndarray | None = None       # [G,3]
    # keyframes
    cams: np.ndarray = field(default_factory=lambda: np.zeros((0, 16), np.float32))
    wh: np.ndarray = field(default_factory=lambda: np.zeros((0, 2), np.int32))
    targets: list = field(default_factory=list)   # per view [3,H,W] f32

    @property
    def N(self) -> int:
        return 0 if self.xyz is None else int(self.xyz.shape[0])

    @property
    def V(self) -> int:
        return int(self.cams.shape[0])

    @property
    def pixels(self) -> int:
        return int(sum(int(w) * int(h) for w, h in self.wh))


def camera(fx, fy, cx, cy, centre, yaw_deg=0.0, pitch_deg=0.0):
    """World->camera pose of a camera at `centre` looking along +z turned by
    `yaw_deg` about the (down-pointing) y axis, then `pitch_deg` about x."""
    ps = math.radians(yaw_deg)
    th = math.radians(pitch_deg)
    ry = np.array([[math.cos(ps), 0.0, math.sin(ps)],
                   [0.0, 1.0, 0.0],
                   [-math.sin(ps), 0.0, math.cos(ps)]])
    rx = np.array([[1.0, 0.0, 0.0],
                   [0.0, math.cos(th), -math.sin(th)],
                   [0.0, math.sin(th), math.cos(th)]])
    r_cw = ry @ rx                      # camera->world rotation
    r = r_cw.T                          # world->camera
    t = -r @ np.asarray(centre, np.float64)
    out = np.zeros(16, np.float64)
    out[:4] = (fx, fy, cx, cy)
    out[4:13] = r.reshape(-1)
    out[13:16] = t
    return out.astype(np.float32)


def init_mlp(rng, M: int, F: int, k: int, hidden: int, dist_ref: float = 100.0):
    """Per-partition decoder weights, U(+-1/sqrt(fan_in)) like a default linear
    layer.  The distance input column of W1 is further divided by `dist_ref`
    so that a raw distance of O(dist_ref) metres contributes O(1) to the
    pre-activations, like the other inputs.  Draw order: partition-major, then
    head (opacity, colour, covariance), then W1, b1, W2, b2."""
    din = F + 4
    P = mlp_param_count(F, k, hidden)
    out = np.zeros((M, P), np.float64)
    for m in range(M):
        parts = []
        for dout in (k, 3 * k, 7 * k):
            b1lim = 1.0 / math.sqrt(din)
            w1 = rng.uniform(-b1lim, b1lim, (hidden, din))
            w1[:, din - 1] /= dist_ref
            b1 = rng.uniform(-b1lim, b1lim, hidden)
            b2lim = 1.0 / math.sqrt(hidden)
            w2 = rng.uniform(-b2lim, b2lim, (dout, hidden))
            b2 = rng.uniform(-b2lim, b2lim, dout)
            parts += [w1.ravel(), b1, w2.ravel(), b2]
        out[m] = np.concatenate(parts)
    return out.astype(np.float32)


def _targets(rng, wh):
    return [rng.uniform(0.0, 1.0, (3, int(h), int(w))).astype(np.float32) for w, h in wh]


def corridor_cell_xyz(idx: np.ndarray, z0: float) -> np.ndarray:
    """Centre of corridor cell `idx` (slice-major: slice = idx // 170)."""
    idx = np.asarray(idx, np.int64)
    sl = idx // CELLS_PER_SLICE
    s = idx % CELLS_PER_SLICE
    z = z0 + (sl + 0.5) * CELL
    x = np.empty(idx.shape, np.float64)
    y = np.empty(idx.shape, np.float64)
    g = s < N_GROUND
    x[g] = -HALF_WIDTH + (s[g] + 0.5) * CELL
    y[g] = GROUND_Y
    f = ~g
    sf = s[f] - N_GROUND
    side = np.where(sf < N_FACADE, -1.0, 1.0)
    h = sf % N_FACADE
    x[f] = side * HALF_WIDTH
    y[f] = GROUND_Y - (h + 0.5) * CELL
    return np.stack([x, y, z], 1)


def _anchor_attributes(rng, N, F, k):
    feat = rng.normal(0.0, 0.1, (N, F))
    offsets = rng.normal(0.0, 1.0, (N, k, 3))
    log_scaling = np.full((N, 6), math.log(0.2))
    return (feat.astype(np.float32), offsets.astype(np.float32),
            log_scaling.astype(np.float32))


def explicit_frustum(seed=0, n=2000, width=128, height=96, fx=100.0, fy=100.0,
                     cx=64.0, cy=48.0):
    """Plain explicit 3DGS view: `n` Gaussians uniform in the pinhole frustum.

    Draw order: u ~ U[0,W), v ~ U[0,H), z ~ U[2,10] (each [n]); log-scale ~
    N(-2, 0.5) [n,3]; quaternion ~ N(0,1) [n,4] then unit-normalised; opacity
    logit ~ N(0,1) [n] then logistic; RGB ~ U[0,1] [n,3]; target ~ U[0,1]
    [3,H,W].  The camera is at the origin looking along +z."""
    rng = np.random.default_rng(seed)
    u = rng.uniform(0.0, width, n)
    v = rng.uniform(0.0, height, n)
    z = rng.uniform(2.0, 10.0, n)
    log_s = rng.normal(-2.0, 0.5, (n, 3))
    q = rng.normal(0.0, 1.0, (n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    opa = 1.0 / (1.0 + np.exp(-rng.normal(0.0, 1.0, n)))
    rgb = rng.uniform(0.0, 1.0, (n, 3))
    wh = np.array([[width, height]], np.int32)
    target = _targets(rng, wh)
    mu = np.stack([(u - cx) / fx * z, (v - cy) / fy * z, z], 1)
    cams = camera(fx, fy, cx, cy, (0.0, 0.0, 0.0))[None]
    return Scene(name=f"explicit_{n}_{width}x{height}", mu=mu.astype(np.float32),
                 scale=np.exp(log_s).astype(np.float32), quat=q.astype(np.float32),
                 opacity=opa.astype(np.float32), colour=rgb.astype(np.float32),
                 cams=cams, wh=wh, targets=target)


def corridor(seed=0, length=200.0, n_anchors=20000, F=32, k=10, hidden=32,
             views=((1241, 376, 718.0, 718.0, 620.5, 188.0, (0.0, 0.0, 100.0), 0.0),),
             yaw_jitter_deg=0.0, name=None):
    """Straight corridor along +z over [0, length): ground + two facades.

    Anchors are distinct cells of the 0.2 m corridor grid sampled without
    replacement (then kept in cell order), one partition.  Views are tuples
    (W, H, fx, fy, cx, cy, centre, yaw_deg).

    Draw order: cell choice [N]; features N(0,0.1) [N,F]; offsets N(0,1)
    [N,k,3]; MLP weights (see `init_mlp`); yaw jitter U[-j,j] per view;
    targets U[0,1] per view."""
    rng = np.random.default_rng(seed)
    n_slices = int(round(length / CELL))
    ncell = n_slices * CELLS_PER_SLICE
    if n_anchors > ncell:
        raise ValueError("more anchors than corridor cells")
    idx = np.sort(rng.choice(ncell, n_anchors, replace=False))
    xyz = corridor_cell_xyz(idx, 0.0)
    feat, offsets, log_scaling = _anchor_attributes(rng, n_anchors, F, k)
    mlp = init_mlp(rng, 1, F, k, hidden)
    cams, wh = [], []
    for (w, h, fx, fy, cx, cy, c, yaw) in views:
        j = rng.uniform(-yaw_jitter_deg, yaw_jitter_deg) if yaw_jitter_deg > 0 else 0.0
        cams.append(camera(fx, fy, cx, cy, c, yaw + j))
        wh.append((w, h))
    wh = np.asarray(wh, np.int32)
    targets = _targets(rng, wh)
    return Scene(name=name or f"corridor_{n_anchors}", xyz=xyz.astype(np.float32), feat=feat,
                 log_scaling=log_scaling, offsets=offsets,
                 part=np.zeros(n_anchors, np.int32), mlp=mlp, F=F, k=k, hidden=hidden,
                 M=1, cams=np.stack(cams), wh=wh, targets=targets)


def anchor_single_view(seed=0):
    """20k anchors on a 200 m corridor, one 1241x376 view (fx=fy=718) at the
    corridor centre (0, 0, 100), FP32 features."""
    return corridor(seed=seed, length=200.0, n_anchors=20000, name="anchor_grid_20k_1view")


def keyframe_batch(seed=0, n_anchors=200000, n_views=8):
    """200k anchors over a 1 km corridor; 8 keyframes of 1241x376 at 1 m pose
    spacing (z = 500..507) with +-2 deg yaw jitter."""
    views = tuple((1241, 376, 718.0, 718.0, 620.5, 188.0, (0.0, 0.0, 500.0 + i), 0.0)
                  for i in range(n_views))
    return corridor(seed=seed, length=1000.0, n_anchors=n_anchors, views=views,
                    yaw_jitter_deg=2.0, name=f"keyframe_batch_{n_anchors // 1000}k_{n_views}v")


def tiny_corridor(seed=0, n_anchors=600, F=8, k=4, hidden=16, length=30.0,
                  views=((72, 40, 60.0, 60.0, 36.0, 20.0, (0.0, 0.0, 5.0), 0.0),
                         (50, 34, 45.0, 45.0, 25.0, 17.0, (0.3, 0.0, 6.0), 3.0))):
    """Small anchor scene for oracle self-checks and parity tests: several
    tiles per view, ragged tile tails, two views of different resolution."""
    return corridor(seed=seed, length=length, n_anchors=n_anchors, F=F, k=k,
                    hidden=hidden, views=views, name=f"tiny_corridor_{n_anchors}")


def uneven_partitions(seed=0, n_parts=16, mu_log=math.log(40000.0), sigma=0.8,
                      cap=150000, F=32, k=10, hidden=32, n_views=16, scale_count=1.0):
    """Spatial decomposition with uneven partitions: partition m holds
    n_m = min(round(lognormal(mu, sigma)), cap) anchors on its own straight
    corridor segment of length n_m / 425 m (50 % cell occupancy); segments
    follow each other along +z.  One keyframe per segment start; resolutions
    cycle 1241x376, 1024x384, 1024x768 with fx = fy ~ U[400, 720].

    Draw order: counts [M]; per partition: cell choice, features, offsets;
    MLP weights for all partitions; per view fx; targets."""
    rng = np.random.default_rng(seed)
    counts = np.minimum(np.round(rng.lognormal(mu_log, sigma, n_parts)), cap).astype(np.int64)
    counts = np.maximum((counts * scale_count).astype(np.int64), 1)
    xyz_l, feat_l, off_l, ls_l, part_l, starts = [], [], [], [], [], []
    z0 = 0.0
    for m in range(n_parts):
        n = int(counts[m])
        seg = n / 425.0
        n_slices = max(1, int(math.ceil(seg / CELL)))
        ncell = n_slices * CELLS_PER_SLICE
        idx = np.sort(rng.choice(ncell, min(n, ncell), replace=False))
        xyz_l.append(corridor_cell_xyz(idx, z0))
        f, o, ls = _anchor_attributes(rng, len(idx), F, k)
        feat_l.append(f); off_l.append(o); ls_l.append(ls)
        part_l.append(np.full(len(idx), m, np.int32))
        starts.append(z0)
        z0 += n_slices * CELL
    mlp = init_mlp(rng, n_parts, F, k, hidden)
    res = [(1241, 376), (1024, 384), (1024, 768)]
    cams, wh = [], []
    for v in range(n_views):
        w, h = res[v % 3]
        f = rng.uniform(400.0, 720.0)
        cams.append(camera(f, f, w / 2.0, h / 2.0, (0.0, 0.0, starts[v % n_parts])))
        wh.append((w, h))
    wh = np.asarray(wh, np.int32)
    targets = _targets(rng, wh)
    return Scene(name=f"uneven_{n_parts}parts_{n_views}v",
                 xyz=np.concatenate(xyz_l).astype(np.float32), feat=np.concatenate(feat_l),
                 log_scaling=np.concatenate(ls_l), offsets=np.concatenate(off_l),
                 part=np.concatenate(part_l), mlp=mlp, F=F, k=k, hidden=hidden, M=n_parts,
                 cams=np.stack(cams), wh=wh, targets=targets)


def loop_road(seed=0, n_anchors=2_000_000, circumference=5000.0, relief=1.0,
              n_parts=16, n_views=32, current_s=4000.0, window=25, p_recent=0.7,
              F=32, k=10, hidden=32, scale_count=1.0):
    """Long-horizon map: a closed circular road of the given circumference
    with ground height relief*sin(2*pi*s/1000 m), ground + facades, 16
    equal-arc partitions.  Keyframes every 1 m up to `current_s`; the batch of
    `n_views` keyframes is drawn without replacement by the rule of the
    paper's implementation details (recent window of 25 with p = 0.7, else
    older), each with +-2 deg yaw jitter.

    Draw order: cell choice; features; offsets; MLP weights; keyframe draws
    (one U[0,1] and one index per pick); yaw jitter per view; targets."""
    rng = np.random.default_rng(seed)
    n_anchors = int(n_anchors * scale_count)
    R = circumference / (2.0 * math.pi)
    n_slices = int(round(circumference / CELL))
    ncell = n_slices * CELLS_PER_SLICE
    idx = np.sort(rng.choice(ncell, n_anchors, replace=False))
    sl = idx // CELLS_PER_SLICE
    s_arc = (sl + 0.5) * CELL
    local = corridor_cell_xyz(idx % CELLS_PER_SLICE, 0.0)   # x (lateral), y (height), z unused
    lift = relief * np.sin(2.0 * math.pi * s_arc / 1000.0)
    ang = s_arc / R
    # centre line (R sin a, y, R(1 - cos a)) heading (cos a, 0, sin a) rotated: tangent
    # (cos a, 0, sin a) is the +z of the road frame, lateral +x is (sin a, 0, -cos a)... use
    # tangent = (sin a, 0, cos a) so that a = 0 heads along +z like the straight corridor.
    cx = R * (1.0 - np.cos(ang))
    cz = R * np.sin(ang)
    tx, tz = np.sin(ang), np.cos(ang)          # tangent
    lx, lz = np.cos(ang), -np.sin(ang)         # lateral (+x at a = 0)
    xyz = np.stack([cx + local[:, 0] * lx, local[:, 1] - lift, cz + local[:, 0] * lz], 1)
    feat, offsets, log_scaling = _anchor_attributes(rng, n_anchors, F, k)
    part = np.minimum((s_arc / (circumference / n_parts)).astype(np.int32), n_parts - 1)
    mlp = init_mlp(rng, n_parts, F, k, hidden)
    n_kf = int(current_s) + 1
    recent = list(range(max(0, n_kf - window), n_kf))
    older = list(range(0, max(0, n_kf - window)))
    picks = []
    while len(picks) < n_views:
        pool = recent if (rng.uniform() < p_recent and recent) or not older else older
        j = int(rng.integers(len(pool)))
        picks.append(pool.pop(j))
    cams, wh = [], []
    for s in picks:
        a = s / R
        c = (R * (1.0 - math.cos(a)), -relief * math.sin(2.0 * math.pi * s / 1000.0),
             R * math.sin(a))
        yaw = math.degrees(a) + rng.uniform(-2.0, 2.0)
        cams.append(camera(718.0, 718.0, 620.5, 188.0, c, yaw))
        wh.append((1241, 376))
    wh = np.asarray(wh, np.int32)
    targets = _targets(rng, wh)
    return Scene(name=f"loop_{n_anchors // 1000}k_{n_views}v", xyz=xyz.astype(np.float32),
                 feat=feat, log_scaling=log_scaling, offsets=offsets, part=part, mlp=mlp,
                 F=F, k=k, hidden=hidden, M=n_parts, cams=np.stack(cams), wh=wh,
                 targets=targets)


@dataclass
class FlowPair:
    cams: np.ndarray       # [2, 16] float32, keyframes 1 and 2
    wh: tuple              # (width, height)
    flow: np.ndarray       # [H, W, 2] float32, keyframe 1 -> keyframe 2 (pixels)
    depth: np.ndarray      # [H, W] float32, depth of each keyframe-1 pixel (its true 3D point)
    outlier: np.ndarray    # [H, W] bool, pixels whose flow was replaced by a random vector
    samples: np.ndarray    # [n_samples] int32 pixel indices y W + x, drawn without replacement


def flow_pair(seed=0, width=1241, height=376, fx=718.0, step=(0.3, 0.0, 1.2), yaw_deg=1.5,
              outlier_frac=0.2, noise_px=0.0, n_samples=200_000):
    """Two consecutive keyframes of a forward-moving camera and the dense flow
    between them, standing in for the flow network's output (Sec. III, Flow
    Densification).  Draw order: depth-field phases (8 uniform), outlier mask
    (H W uniform), outlier vectors (2 H W uniform in [-40, 40] px), flow
    noise (2 H W normal, times noise_px), samples (a permutation prefix).
    Depth: 4 + 40 (1 + sum of 4 random plane waves / 4) / 2 m, smooth in the
    image.  Flow of an inlier pixel: its depth-scaled ray, moved into
    keyframe 2 and reprojected (pixels at integer coordinates)."""
    rng = np.random.default_rng(seed)
    cx, cy = width / 2.0, height / 2.0
    c1 = camera(fx, fx, cx, cy, (0.0, 0.0, 0.0))
    c2 = camera(fx, fx, cx, cy, step, yaw_deg=yaw_deg)
    ph = rng.uniform(0, 2 * np.pi, 8)
    yy, xx = np.mgrid[0:height, 0:width].astype(np.float64)
    wave = sum(np.sin(xx * (0.004 + 0.002 * i) + yy * (0.01 - 0.002 * i) + ph[i]) for i in range(4)) / 4.0
    depth = 4.0 + 40.0 * (1.0 + wave) / 2.0
    X1 = np.stack([(xx - cx) / fx * depth, (yy - cy) / fx * depth, depth], -1)     # keyframe-1 camera frame
    R1, t1 = c1[4:13].astype(np.float64).reshape(3, 3), c1[13:16].astype(np.float64)
    R2, t2 = c2[4:13].astype(np.float64).reshape(3, 3), c2[13:16].astype(np.float64)
    Xw = (X1 - t1) @ R1                                                              # R1^T (X1 - t1)
    X2 = Xw @ R2.T + t2
    u2 = fx * X2[..., 0] / X2[..., 2] + cx
    v2 = fx * X2[..., 1] / X2[..., 2] + cy
    flow = np.stack([u2 - xx, v2 - yy], -1)
    out = rng.uniform(size=(height, width)) < outlier_frac
    rnd = rng.uniform(-40, 40, (height, width, 2))
    flow[out] = rnd[out]
    flow += noise_px * rng.normal(size=(height, width, 2))
    samples = rng.permutation(width * height)[:n_samples].astype(np.int32)
    return FlowPair(np.stack([c1, c2]), (width, height), flow.astype(np.float32), depth.astype(np.float32),
                    out, samples)
