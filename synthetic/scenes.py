"""Seeded synthetic structure-from-motion scenes.

This module is the one input generator shared by the oracle tests, the CUDA
parity tests, ``bench.py`` and ``smoke()``.  It places pinhole cameras and 3D
points, projects the points (plus per-observation Gaussian pixel noise), forms
every pairwise combination of the cameras that see a point (the completed
tracks of the paper's track completion, Appendix "Tracks"), replaces a fraction
of keypoint pairs by uniform-random outlier pixels, and groups the keypoint
pairs by image pair.  It holds none of the method's arithmetic: no objective,
gradient, optimizer or estimator lives here.

Conventions (shared with the C ABI):
  * world-to-camera pose: ``x_cam = R @ X + t``; camera centre ``o = -R^T t``;
  * pixel ``u = f * x/z + cx``, ``v = f * y/z + cy``; principal point at the
    image centre (Sec. 3.1, camera assumptions);
  * an image pair is ``(i, j)`` with ``i < j``; in a keypoint pair the first
    keypoint lies in image ``i`` and the second in image ``j``;
  * keypoint pairs are sorted by (image pair, track) and ``kp_img_pair`` is
    non-decreasing.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from itertools import combinations

import numpy as np

__all__ = ["Scene", "make_scene", "scene_c1", "scene_c2", "perturb_params",
           "gt_relative_poses", "CONFIGS", "concat_scenes", "batch_c4"]


@dataclass
class Scene:
    name: str
    seed: int
    width: int
    height: int
    focal: np.ndarray        # [N] float64
    cx: np.ndarray           # [N]
    cy: np.ndarray           # [N]
    R_gt: np.ndarray         # [N,3,3] world-to-camera
    t_gt: np.ndarray         # [N,3]
    points: np.ndarray       # [T,3] one point per track
    pair_i: np.ndarray       # [P] int32, pair_i < pair_j
    pair_j: np.ndarray       # [P] int32
    kp_img_pair: np.ndarray  # [Z] int32, non-decreasing
    kp1_px: np.ndarray       # [Z,2] float32, keypoint in image pair_i
    kp2_px: np.ndarray       # [Z,2] float32, keypoint in image pair_j
    kp_track: np.ndarray     # [Z] int32
    kp_inlier: np.ndarray    # [Z] bool, False where the pair was replaced by an outlier
    meta: dict = field(default_factory=dict)
    scene_cam_off: np.ndarray | None = None   # [S+1] camera offsets of a batch of scenes

    @property
    def n_cams(self) -> int:
        return int(self.focal.shape[0])

    @property
    def n_pairs(self) -> int:
        return int(self.pair_i.shape[0])

    @property
    def n_kp(self) -> int:
        return int(self.kp_img_pair.shape[0])

    @property
    def centers_gt(self) -> np.ndarray:
        return -np.einsum("nji,nj->ni", self.R_gt, self.t_gt)

    def seg_off(self) -> np.ndarray:
        """CSR offsets of the keypoint pairs of each image pair, [P+1] int64."""
        counts = np.bincount(self.kp_img_pair, minlength=self.n_pairs)
        off = np.zeros(self.n_pairs + 1, dtype=np.int64)
        np.cumsum(counts, out=off[1:])
        return off


# --------------------------------------------------------------------------
# camera placement helpers (scene construction only)
# --------------------------------------------------------------------------

def _frame_looking(forward: np.ndarray, up: np.ndarray) -> np.ndarray:
    """Rows are the camera x, y, z axes in world coordinates (right-handed)."""
    z = forward / np.linalg.norm(forward)
    x = np.cross(z, up)
    nx = np.linalg.norm(x)
    if nx < 1e-9:  # forward parallel to up: pick any perpendicular axis
        x = np.cross(z, np.array([1.0, 0.0, 0.0]))
        nx = np.linalg.norm(x)
    x = x / nx
    y = np.cross(z, x)
    return np.stack([x, y, z])


def _rot_axis(axis: int, ang: float) -> np.ndarray:
    c, s = np.cos(ang), np.sin(ang)
    if axis == 0:
        return np.array([[1, 0, 0], [0, c, -s], [0, s, c]])
    if axis == 1:
        return np.array([[c, 0, s], [0, 1, 0], [-s, 0, c]])
    return np.array([[c, -s, 0], [s, c, 0], [0, 0, 1]])


def _project(R, t, f, cx, cy, X):
    """Project points X [M,3] into cameras [N]: returns (u, v, depth) of shape [M,N]."""
    Xc = np.einsum("nij,mj->mni", R, X) + t[None, :, :]
    z = Xc[..., 2]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = f[None, :] * Xc[..., 0] / z + cx[None, :]
        v = f[None, :] * Xc[..., 1] / z + cy[None, :]
    return u, v, z


# --------------------------------------------------------------------------
# track -> keypoint pairs
# --------------------------------------------------------------------------

def _tracks_to_pairs(rng, track_cams, track_uv, width, height, outlier_frac,
                     min_pairs_per_image_pair):
    """All C(k,2) camera combinations of every track, grouped by image pair.

    track_cams: list of int arrays (sorted camera ids per track)
    track_uv:   list of [k,2] arrays (noisy pixels, one per observation)
    """
    by_k = {}
    for tid, cams in enumerate(track_cams):
        by_k.setdefault(len(cams), []).append(tid)
    ci, cj, p1, p2, tr = [], [], [], [], []
    for k, tids in by_k.items():
        tids = np.asarray(tids)
        cams = np.stack([track_cams[t] for t in tids])      # [n,k]
        uv = np.stack([track_uv[t] for t in tids])          # [n,k,2]
        comb = np.array(list(combinations(range(k), 2)))    # [c,2]
        a, b = comb[:, 0], comb[:, 1]
        ci.append(cams[:, a].reshape(-1))
        cj.append(cams[:, b].reshape(-1))
        p1.append(uv[:, a].reshape(-1, 2))
        p2.append(uv[:, b].reshape(-1, 2))
        tr.append(np.repeat(tids, len(comb)))
    ci = np.concatenate(ci).astype(np.int64)
    cj = np.concatenate(cj).astype(np.int64)
    p1 = np.concatenate(p1)
    p2 = np.concatenate(p2)
    tr = np.concatenate(tr).astype(np.int64)
    return _group_pairs(rng, ci, cj, p1, p2, tr, width, height, outlier_frac,
                        min_pairs_per_image_pair)


def _grouped_tracks_to_pairs(rng, cams_by_k, uv_by_k, width, height, outlier_frac,
                             min_pairs_per_image_pair):
    """Same as _tracks_to_pairs with tracks already grouped by length: lists of
    [n,k] camera arrays and [n,k,2] pixel arrays; track ids run over the groups
    in order."""
    ci, cj, p1, p2, tr = [], [], [], [], []
    base = 0
    for cams, uv in zip(cams_by_k, uv_by_k):
        n, k = cams.shape
        comb = np.array(list(combinations(range(k), 2)))
        a, b = comb[:, 0], comb[:, 1]
        ci.append(cams[:, a].reshape(-1))
        cj.append(cams[:, b].reshape(-1))
        p1.append(uv[:, a].reshape(-1, 2))
        p2.append(uv[:, b].reshape(-1, 2))
        tr.append(np.repeat(np.arange(base, base + n), len(comb)))
        base += n
    ci = np.concatenate(ci).astype(np.int64)
    cj = np.concatenate(cj).astype(np.int64)
    p1 = np.concatenate(p1)
    p2 = np.concatenate(p2)
    tr = np.concatenate(tr).astype(np.int64)
    return _group_pairs(rng, ci, cj, p1, p2, tr, width, height, outlier_frac,
                        min_pairs_per_image_pair)


def _group_pairs(rng, ci, cj, p1, p2, tr, width, height, outlier_frac,
                 min_pairs_per_image_pair):
    n_cam_key = int(max(ci.max(), cj.max())) + 1
    key = ci * n_cam_key + cj
    order = np.lexsort((tr, key))
    ci, cj, p1, p2, tr, key = ci[order], cj[order], p1[order], p2[order], tr[order], key[order]
    uniq, inv, counts = np.unique(key, return_inverse=True, return_counts=True)
    keep_pair = counts >= min_pairs_per_image_pair
    keep_kp = keep_pair[inv]
    ci, cj, p1, p2, tr, inv = ci[keep_kp], cj[keep_kp], p1[keep_kp], p2[keep_kp], tr[keep_kp], inv[keep_kp]
    new_index = np.cumsum(keep_pair) - 1
    kp_img_pair = new_index[inv]
    uniq = uniq[keep_pair]
    pair_i = (uniq // n_cam_key).astype(np.int32)
    pair_j = (uniq % n_cam_key).astype(np.int32)
    # outliers: the second keypoint of the pair becomes a uniform random pixel
    z = len(kp_img_pair)
    is_out = rng.random(z) < outlier_frac
    n_out = int(is_out.sum())
    p2 = p2.copy()
    p2[is_out, 0] = rng.uniform(0.0, width, n_out)
    p2[is_out, 1] = rng.uniform(0.0, height, n_out)
    return dict(pair_i=pair_i, pair_j=pair_j,
                kp_img_pair=kp_img_pair.astype(np.int32),
                kp1_px=p1.astype(np.float32), kp2_px=p2.astype(np.float32),
                kp_track=tr.astype(np.int32), kp_inlier=~is_out)


# --------------------------------------------------------------------------
# configurations
# --------------------------------------------------------------------------

def scene_c1(seed: int = 0, n_points: int = 2000, sigma_px: float = 0.5,
             outlier_frac: float = 0.05, n_cams: int = 20) -> Scene:
    """Tiny scene: 20 cameras on a circle of radius 5 looking at the origin
    with yaw jitter U(-10deg, 10deg), f = 500 px, 640x480, points uniform in a
    unit cube, each seen by k ~ U{2..6} random cameras."""
    rng = np.random.default_rng(seed)
    W, H = 640, 480
    N = n_cams
    f = np.full(N, 500.0)
    cx = np.full(N, W / 2.0)
    cy = np.full(N, H / 2.0)
    R = np.zeros((N, 3, 3))
    t = np.zeros((N, 3))
    up = np.array([0.0, 1.0, 0.0])
    for k in range(N):
        th = 2.0 * np.pi * k / N
        C = 5.0 * np.array([np.cos(th), 0.0, np.sin(th)])
        Rk = _frame_looking(-C, up)
        yaw = np.deg2rad(rng.uniform(-10.0, 10.0))
        Rk = _rot_axis(1, yaw) @ Rk
        R[k] = Rk
        t[k] = -Rk @ C
    X = rng.uniform(-0.5, 0.5, size=(n_points, 3))
    u, v, z = _project(R, t, f, cx, cy, X)
    track_cams, track_uv = [], []
    for p in range(n_points):
        k = min(int(rng.integers(2, 7)), N)
        cams = np.sort(rng.choice(N, size=k, replace=False))
        uv = np.stack([u[p, cams], v[p, cams]], axis=1) + rng.normal(0.0, sigma_px, size=(k, 2))
        track_cams.append(cams)
        track_uv.append(uv)
    g = _tracks_to_pairs(rng, track_cams, track_uv, W, H, outlier_frac, 8)
    return Scene(name="c1", seed=seed, width=W, height=H, focal=f, cx=cx, cy=cy,
                 R_gt=R, t_gt=t, points=X, meta=dict(sigma_px=sigma_px,
                 outlier_frac=outlier_frac), **g)


def _bspline(ctrl: np.ndarray, s: np.ndarray):
    """Uniform cubic B-spline through (approximating) the control points, with
    end points clamped by tripling; returns positions and tangents at s in [0,1]."""
    P = np.concatenate([ctrl[:1], ctrl[:1], ctrl, ctrl[-1:], ctrl[-1:]])
    nseg = len(P) - 3
    x = np.clip(s, 0.0, 1.0 - 1e-12) * nseg
    i = np.floor(x).astype(int)
    u = (x - i)[:, None]
    b0 = (1 - u) ** 3 / 6
    b1 = (3 * u ** 3 - 6 * u ** 2 + 4) / 6
    b2 = (-3 * u ** 3 + 3 * u ** 2 + 3 * u + 1) / 6
    b3 = u ** 3 / 6
    d0 = -(1 - u) ** 2 / 2
    d1 = (9 * u ** 2 - 12 * u) / 6
    d2 = (-9 * u ** 2 + 6 * u + 3) / 6
    d3 = u ** 2 / 2
    pos = b0 * P[i] + b1 * P[i + 1] + b2 * P[i + 2] + b3 * P[i + 3]
    tan = d0 * P[i] + d1 * P[i + 1] + d2 * P[i + 2] + d3 * P[i + 3]
    return pos, tan


def _distort(uv, alpha, cx, cy):
    """Observed pixels of ideal pixels uv [...,2] under the division model
    x_u = x_d / (1 + alpha r_d^2) (x about the centre, in half-diagonal
    units): the radius solving that equation closest to r_u,
    r_d = 2 r_u / (1 + sqrt(1 - 4 alpha r_u^2))."""
    c = np.stack([cx, cy], axis=-1)
    h = np.linalg.norm(c, axis=-1, keepdims=True)
    x = (uv - c) / h
    r2 = np.sum(x * x, axis=-1, keepdims=True)
    disc = 1.0 - 4.0 * alpha[..., None] * r2
    if np.any(disc < 0.0):
        raise ValueError("alpha too large for the image: no distorted radius")
    return c + h * x * (2.0 / (1.0 + np.sqrt(disc)))


def _observe_c2(seed: int = 0, n_cams: int = 300, n_points: int = 100_000,
             sigma_px: float = 1.0, outlier_frac: float = 0.10,
             box=(50.0, 50.0, 10.0), max_depth: float = 30.0,
             track_mean: float = 4.0, jitter_deg: float = 15.0,
             focal_range=(400.0, 900.0), chunk: int = 8192, focal_groups: int = 0,
             alpha=0.0):
    """Cameras, points and noisy track observations of ``scene_c2`` (same
    arguments; ``outlier_frac`` is not used here).  Returns the generator and
    a dict of the scene's parts."""
    rng = np.random.default_rng(seed)
    W, H = 640, 480
    N = n_cams
    bx = np.asarray(box, dtype=np.float64)
    ctrl = rng.uniform(0.0, 1.0, size=(8, 3)) * bx
    pos, tan = _bspline(ctrl, np.linspace(0.0, 1.0, N))
    up = np.array([0.0, 0.0, 1.0])
    R = np.zeros((N, 3, 3))
    t = np.zeros((N, 3))
    for k in range(N):
        fwd = tan[k].copy()
        fwd[2] *= 0.2  # keep the view roughly level
        if np.linalg.norm(fwd) < 1e-9:
            fwd = np.array([1.0, 0.0, 0.0])
        Rk = _frame_looking(fwd, up)
        yaw = np.deg2rad(rng.uniform(-jitter_deg, jitter_deg))
        pitch = np.deg2rad(rng.uniform(-jitter_deg, jitter_deg))
        Rk = _rot_axis(1, yaw) @ _rot_axis(0, pitch) @ Rk
        R[k] = Rk
        t[k] = -Rk @ pos[k]
    f = rng.uniform(focal_range[0], focal_range[1], size=N)
    group = np.arange(N, dtype=np.int32)
    if focal_groups > 0:
        group = (np.arange(N) * focal_groups // N).astype(np.int32)
        f = f[np.searchsorted(group, np.arange(focal_groups))][group]
    cx = np.full(N, W / 2.0)
    cy = np.full(N, H / 2.0)
    a = np.asarray(alpha, np.float64)
    alpha_cam = np.full(N, float(a)) if a.ndim == 0 else a[group]
    X = rng.uniform(0.0, 1.0, size=(n_points, 3)) * bx
    p_geom = 1.0 / (track_mean - 1.0)   # k = 2 + (Geometric(p) - 1), mean track_mean
    groups = {}                          # k -> list of (cams [n,k], uv [n,k,2], point ids [n])
    for s0 in range(0, n_points, chunk):
        Xs = X[s0:s0 + chunk]
        u, v, z = _project(R, t, f, cx, cy, Xs)
        vis = (z > 0.1) & (z <= max_depth) & (u >= 0) & (u < W) & (v >= 0) & (v < H)
        nvis = vis.sum(axis=1)
        want = 2 + rng.geometric(p_geom, size=len(Xs)) - 1
        k = np.minimum(want, nvis)
        keys = rng.random(vis.shape)
        keys[~vis] = np.inf
        order = np.argsort(keys, axis=1)
        for kk in np.unique(k[k >= 2]):
            rows = np.nonzero(k == kk)[0]
            cams = np.sort(order[rows, :kk], axis=1)
            uv = np.stack([u[rows[:, None], cams], v[rows[:, None], cams]], axis=2)
            groups.setdefault(int(kk), []).append((cams, uv, s0 + rows))
    track_cams, track_uv, track_pts = [], [], []
    for kk in sorted(groups):
        cams = np.concatenate([g[0] for g in groups[kk]])
        uv = np.concatenate([g[1] for g in groups[kk]])
        pts = np.concatenate([g[2] for g in groups[kk]])
        if np.any(alpha_cam != 0.0):
            uv = _distort(uv, alpha_cam[cams], cx[cams], cy[cams])
        # per-observation noise (shared by every pair that uses the observation)
        uv = uv + rng.normal(0.0, sigma_px, size=uv.shape)
        track_cams.append(cams)
        track_uv.append(uv)
        track_pts.append(pts)
    return rng, dict(W=W, H=H, R=R, t=t, f=f, cx=cx, cy=cy, X=X, group=group, alpha_cam=alpha_cam,
                     track_cams=track_cams, track_uv=track_uv, track_pts=track_pts)


def scene_c2(seed: int = 0, n_cams: int = 300, n_points: int = 100_000,
             sigma_px: float = 1.0, outlier_frac: float = 0.10,
             box=(50.0, 50.0, 10.0), max_depth: float = 30.0,
             track_mean: float = 4.0, jitter_deg: float = 15.0,
             focal_range=(400.0, 900.0), chunk: int = 8192, focal_groups: int = 0,
             alpha=0.0) -> Scene:
    """Scene at scale: cameras on a smooth random trajectory (cubic B-spline
    through 8 random control points inside a 50x50x10 box) looking along the
    tangent with +-15deg jitter, f ~ U(400, 900) px, points uniform in the box,
    track length 2 + Geometric (mean ``track_mean``) capped by visibility (in
    front, inside the image, depth <= 30).  focal_groups = g > 0: the images
    form g contiguous blocks along the trajectory, each sharing one focal
    length (``meta["focal_group"]``); 0: one focal length per image.
    alpha: radial distortion of the observed pixels (one-parameter division
    model about the image centre, radii in units of the half diagonal), a
    scalar for every image or one value per focal group; the visibility test
    uses the undistorted projection, the pixel noise is added after the
    distortion (``meta["alpha"]`` per image)."""
    rng, o = _observe_c2(seed, n_cams, n_points, sigma_px, outlier_frac, box, max_depth, track_mean,
                         jitter_deg, focal_range, chunk, focal_groups, alpha)
    W, H = o["W"], o["H"]
    track_cams, track_uv, track_pts = o["track_cams"], o["track_uv"], o["track_pts"]
    R, t, f, cx, cy, X = o["R"], o["t"], o["f"], o["cx"], o["cy"], o["X"]
    group, alpha_cam = o["group"], o["alpha_cam"]
    g = _grouped_tracks_to_pairs(rng, track_cams, track_uv, W, H, outlier_frac, 8)
    track_pts = np.concatenate(track_pts)
    return Scene(name="c2", seed=seed, width=W, height=H, focal=f, cx=cx, cy=cy,
                 R_gt=R, t_gt=t, points=X[track_pts],
                 meta=dict(sigma_px=sigma_px, outlier_frac=outlier_frac,
                           n_points_sampled=n_points, focal_group=group, alpha=alpha_cam), **g)


@dataclass
class RawMatches:
    """Keypoints per image and raw pairwise matches (before track completion).

    Keypoints are grouped by image: those of image c are kp_off[c] ..
    kp_off[c+1]-1, in a random order (a detector's order carries no meaning).
    matches [M,2] holds keypoint ids (the first in the lower image), grouped by
    image pair.  true_track [K] is the generator's track of each keypoint (-1
    for distractors that observe no point)."""
    kp_off: np.ndarray       # [N+1] int32
    kp_px: np.ndarray        # [K,2] float32
    matches: np.ndarray      # [M,2] int32
    true_track: np.ndarray   # [K] int32
    n_spurious: int
    focal: np.ndarray
    cx: np.ndarray
    cy: np.ndarray
    R_gt: np.ndarray
    t_gt: np.ndarray
    width: int
    height: int

    @property
    def n_cams(self) -> int:
        return int(self.kp_off.shape[0] - 1)

    @property
    def n_kp(self) -> int:
        return int(self.kp_off[-1])


def raw_matches_c2(seed: int = 0, n_cams: int = 300, n_points: int = 100_000, recall: float = 0.5,
                   spurious_frac: float = 0.0, distractors: int = 0, sigma_px: float = 1.0,
                   **scene_kw) -> RawMatches:
    """Raw matches of the ``scene_c2`` geometry with low matching recall:
    every observation of a track is one keypoint of its image; each pair of
    observations of a track is matched independently with probability
    ``recall`` (a track may fall apart into several components); a fraction
    ``spurious_frac`` of extra matches join a random keypoint of the lower
    image of a matched image pair to a random keypoint of the other (these
    merge unrelated tracks); ``distractors`` unmatched keypoints per image."""
    _, o = _observe_c2(seed, n_cams, n_points, sigma_px, 0.0, **scene_kw)
    rng = np.random.default_rng(1_000_003 + seed)   # the matching draws, apart from the scene's
    N = n_cams
    cams = [c.reshape(-1) for c in o["track_cams"]]
    uvs = [u.reshape(-1, 2) for u in o["track_uv"]]
    tids, base = [], 0
    for c in o["track_cams"]:
        n, k = c.shape
        tids.append(np.repeat(np.arange(base, base + n), k))
        base += n
    obs_cam = np.concatenate(cams).astype(np.int64)
    obs_uv = np.concatenate(uvs)
    obs_track = np.concatenate(tids).astype(np.int64)
    n_obs = len(obs_cam)
    # distractors
    d_cam = np.repeat(np.arange(N), distractors)
    d_uv = rng.uniform([0.0, 0.0], [o["W"], o["H"]], size=(len(d_cam), 2))
    all_cam = np.concatenate([obs_cam, d_cam])
    all_uv = np.concatenate([obs_uv, d_uv])
    all_track = np.concatenate([obs_track, np.full(len(d_cam), -1)])
    # keypoint ids: grouped by image, random order inside an image
    order = np.lexsort((rng.random(len(all_cam)), all_cam))
    node_of = np.empty(len(all_cam), np.int64)
    node_of[order] = np.arange(len(all_cam))
    kp_off = np.concatenate([[0], np.cumsum(np.bincount(all_cam, minlength=N))]).astype(np.int32)
    kp_px = all_uv[order].astype(np.float32)
    true_track = all_track[order].astype(np.int32)
    # matches inside tracks: observations of a track are contiguous (cameras
    # increasing); each pair of them is matched with probability `recall`
    o1, o2, off = [], [], 0
    for c in o["track_cams"]:
        n, k = c.shape
        first = off + np.arange(n) * k
        for a in range(k):
            for b in range(a + 1, k):
                keep = rng.random(n) < recall
                o1.append(first[keep] + a)
                o2.append(first[keep] + b)
        off += n * k
    o1 = np.concatenate(o1) if o1 else np.zeros(0, np.int64)
    o2 = np.concatenate(o2) if o2 else np.zeros(0, np.int64)
    u, v = node_of[o1], node_of[o2]
    # spurious matches between images already matched
    n_sp = int(round(spurious_frac * len(u)))
    if n_sp > 0 and len(u) > 0:
        pick = rng.integers(0, len(u), n_sp)
        ci, cj = all_cam[o1[pick]], all_cam[o2[pick]]
        su = kp_off[ci] + (rng.random(n_sp) * (kp_off[ci + 1] - kp_off[ci])).astype(np.int64)
        sv = kp_off[cj] + (rng.random(n_sp) * (kp_off[cj + 1] - kp_off[cj])).astype(np.int64)
        u = np.concatenate([u, su])
        v = np.concatenate([v, sv])
    # group by image pair (lower image first), then by keypoint ids
    ci, cj = np.searchsorted(kp_off, u, side="right") - 1, np.searchsorted(kp_off, v, side="right") - 1
    swap = ci > cj
    u, v = np.where(swap, v, u), np.where(swap, u, v)
    ci, cj = np.where(swap, cj, ci), np.where(swap, ci, cj)
    order = np.lexsort((v, u, cj, ci))
    matches = np.stack([u[order], v[order]], axis=1).astype(np.int32)
    return RawMatches(kp_off=kp_off, kp_px=kp_px, matches=matches, true_track=true_track, n_spurious=n_sp,
                      focal=o["f"], cx=o["cx"], cy=o["cy"], R_gt=o["R"], t_gt=o["t"], width=o["W"], height=o["H"])


CONFIGS = {
    # the small case the oracle finishes in seconds
    "c1": dict(fn=scene_c1, kwargs={}),
    # the scene at scale as specified (about 0.9-1.2M keypoint pairs)
    "c2": dict(fn=scene_c2, kwargs={}),
    # the scene at scale with the point count raised so that the number of
    # keypoint pairs is about 5M, the pair count the workload is quoted at
    "c2_5m": dict(fn=scene_c2, kwargs=dict(n_points=605_000)),
}


def concat_scenes(scenes, name="batch") -> Scene:
    """One Scene holding several independent scenes: cameras, image pairs,
    keypoint pairs and tracks concatenated scene by scene, with the camera
    offsets in ``scene_cam_off``.  Image-pair and track indices are shifted."""
    cam_off = np.zeros(len(scenes) + 1, dtype=np.int64)
    pair_off = np.zeros(len(scenes) + 1, dtype=np.int64)
    trk_off = np.zeros(len(scenes) + 1, dtype=np.int64)
    for k, sc in enumerate(scenes):
        cam_off[k + 1] = cam_off[k] + sc.n_cams
        pair_off[k + 1] = pair_off[k] + sc.n_pairs
        trk_off[k + 1] = trk_off[k] + (int(sc.kp_track.max()) + 1 if sc.n_kp else 0)
    cat = np.concatenate
    return Scene(
        name=name, seed=scenes[0].seed, width=scenes[0].width, height=scenes[0].height,
        focal=cat([sc.focal for sc in scenes]), cx=cat([sc.cx for sc in scenes]),
        cy=cat([sc.cy for sc in scenes]), R_gt=cat([sc.R_gt for sc in scenes]),
        t_gt=cat([sc.t_gt for sc in scenes]), points=cat([sc.points for sc in scenes]),
        pair_i=cat([sc.pair_i + cam_off[k] for k, sc in enumerate(scenes)]).astype(np.int32),
        pair_j=cat([sc.pair_j + cam_off[k] for k, sc in enumerate(scenes)]).astype(np.int32),
        kp_img_pair=cat([sc.kp_img_pair + pair_off[k] for k, sc in enumerate(scenes)]).astype(np.int32),
        kp1_px=cat([sc.kp1_px for sc in scenes]), kp2_px=cat([sc.kp2_px for sc in scenes]),
        kp_track=cat([sc.kp_track + trk_off[k] for k, sc in enumerate(scenes)]).astype(np.int32),
        kp_inlier=cat([sc.kp_inlier for sc in scenes]),
        meta=dict(pair_off=pair_off, track_off=trk_off,
                  kp_off=np.concatenate([[0], np.cumsum([sc.n_kp for sc in scenes])])),
        scene_cam_off=cam_off.astype(np.int32))


def batch_c4(seed: int = 0, n_scenes: int = 64, cams=(20, 500), points=(2_000, 150_000),
             outliers=(0.05, 0.20), point_scale: float = 1.0):
    """Scenes of uneven size for batched solving: per scene (seed-indexed)
    N ~ logU(cams), point count ~ logU(points) times point_scale, outlier
    fraction ~ U(outliers), sigma = 1 px, the geometry of ``scene_c2``
    (trajectory through a 50x50x10 box).  Returns the list of scenes."""
    rng = np.random.default_rng(10_000 + seed)
    out = []
    for k in range(n_scenes):
        n = int(round(np.exp(rng.uniform(np.log(cams[0]), np.log(cams[1])))))
        m = int(round(point_scale * np.exp(rng.uniform(np.log(points[0]), np.log(points[1])))))
        of = float(rng.uniform(*outliers))
        sc = scene_c2(seed=1000 * (seed + 1) + k, n_cams=n, n_points=m, outlier_frac=of)
        sc.name = f"c4[{k}]"
        out.append(sc)
    return out


def make_scene(config: str = "c1", seed: int = 0, **overrides) -> Scene:
    spec = CONFIGS[config]
    kw = dict(spec["kwargs"])
    kw.update(overrides)
    sc = spec["fn"](seed=seed, **kw)
    sc.name = config
    return sc


# --------------------------------------------------------------------------
# inputs for the per-stage evaluations (seeded; no method arithmetic)
# --------------------------------------------------------------------------

def gt_relative_poses(scene: Scene, rot_noise_deg: float = 0.0,
                      dir_noise_deg: float = 0.0, seed: int = 0):
    """Relative rotations R^{i->j} = R_j R_i^T and unit relative translations
    t^{i->j} (direction of t_j - R^{i->j} t_i) of every image pair, optionally
    perturbed by small random rotations.  Returns float64 arrays [P,3,3], [P,3]."""
    rng = np.random.default_rng(seed)
    Ri = scene.R_gt[scene.pair_i]
    Rj = scene.R_gt[scene.pair_j]
    Rij = Rj @ np.transpose(Ri, (0, 2, 1))
    tij = scene.t_gt[scene.pair_j] - np.einsum("pab,pb->pa", Rij, scene.t_gt[scene.pair_i])
    tij /= np.linalg.norm(tij, axis=1, keepdims=True)
    P = scene.n_pairs
    if rot_noise_deg > 0:
        for p in range(P):
            Rij[p] = _small_rotation(rng, rot_noise_deg) @ Rij[p]
    if dir_noise_deg > 0:
        for p in range(P):
            tij[p] = _small_rotation(rng, dir_noise_deg) @ tij[p]
    return Rij, tij


def _small_rotation(rng, deg):
    axis = rng.normal(size=3)
    axis /= np.linalg.norm(axis)
    ang = np.deg2rad(deg) * rng.normal()
    K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
    return np.eye(3) + np.sin(ang) * K + (1 - np.cos(ang)) * K @ K


def perturb_params(base: np.ndarray, sigma: float, seed: int) -> np.ndarray:
    """Gaussian perturbation of a parameter array (seeded)."""
    rng = np.random.default_rng(seed)
    return base + rng.normal(0.0, sigma, size=base.shape)
