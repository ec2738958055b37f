"""Sparse reconstruction for the oracle (float64).  Test infrastructure only.

Appendix "Sparse Reconstruction": every keypoint pair of a (completed) track
is triangulated, the points of a track are averaged, each keypoint's
reprojection error is measured against the averaged point, keypoints with a
large error are outliers, a point with fewer than 3 inlier keypoints is
dropped, and so is a point whose largest triangulation angle is below a
threshold.  The paper names no triangulation method, error threshold or
angle threshold; the readings here:
  * two-ray midpoint triangulation of each keypoint pair; a pair whose rays
    are within ~0.057 deg of parallel gives no point (PARALLEL_SIN2);
  * a track's keypoints are its distinct (camera, pixel) observations; an
    observation is an inlier if its reprojection error is <= max_err_px;
    the point needs inliers in >= 3 distinct cameras;
  * the triangulation angle of a keypoint pair is the angle at the averaged
    point between the rays to the two camera centres; the largest over the
    pairs whose two keypoints are inliers must be >= min_angle_deg.
"""
import numpy as np


# Rays closer than this to parallel (sin^2 of the angle between them) give
# no point: their intersection is not determined at the float32 precision
# of the inputs (an angle below ~0.057 deg).
PARALLEL_SIN2 = 1e-6


def midpoint(o1, d1, o2, d2):
    """Midpoint of the shortest segment between rays o1 + s d1 and o2 + u d2.
    The normal equations of min |o1 + s d1 - o2 - u d2|^2 have determinant
    |d1|^2 |d2|^2 - (d1.d2)^2 = |d1 x d2|^2 (Lagrange's identity); the cross
    product form keeps it exact for parallel directions.  ok is False when
    |d1 x d2|^2 <= PARALLEL_SIN2 |d1|^2 |d2|^2."""
    w0 = o1 - o2
    a = np.sum(d1 * d1, -1)
    b = np.sum(d1 * d2, -1)
    c = np.sum(d2 * d2, -1)
    d = np.sum(d1 * w0, -1)
    e = np.sum(d2 * w0, -1)
    den = np.sum(np.cross(d1, d2) ** 2, -1)
    ok = den > PARALLEL_SIN2 * a * c
    dd = np.where(ok, den, 1.0)
    s = np.where(ok, (b * e - c * d) / dd, 0.0)
    u = np.where(ok, (a * e - b * d) / dd, 0.0)
    return 0.5 * (o1 + s[..., None] * d1 + o2 + u[..., None] * d2), ok


def triangulate(R, t, pair_i, pair_j, kp_img_pair, x1, x2, kp_track, n_tracks, focal,
                max_err_px=4.0, min_angle_deg=2.0, diag=False):
    """R [N,3,3], t [N,3] world-to-camera; x1, x2 calibrated [Z,3]; returns
    (points [T,3], valid [T] bool, n_inlier_cams [T]), and with diag=True a
    fourth value: a dict of the intermediate quantities the decisions are
    taken on (per keypoint pair: err1, err2 in pixels, angle_deg, pair_ok,
    pair_sin2 = sin^2 of the angle between its rays;
    per track: max_angle_deg), for tests that locate decisions lying within
    rounding of a threshold."""
    R = np.asarray(R, np.float64)
    t = np.asarray(t, np.float64)
    o = -np.einsum("nba,nb->na", R, t)
    ci = np.asarray(pair_i)[kp_img_pair]
    cj = np.asarray(pair_j)[kp_img_pair]
    d1 = np.einsum("mba,mb->ma", R[ci], x1)     # R_i^T x~1
    d2 = np.einsum("mba,mb->ma", R[cj], x2)
    Xm, ok = midpoint(o[ci], d1, o[cj], d2)
    T = n_tracks
    pts = np.zeros((T, 3))
    cnt = np.zeros(T)
    np.add.at(pts, kp_track[ok], Xm[ok])
    np.add.at(cnt, kp_track[ok], 1.0)
    pts = pts / np.maximum(cnt, 1.0)[:, None]

    def reproj_err(X, cam, x):
        Xc = np.einsum("mab,mb->ma", R[cam], X) + t[cam]
        z = Xc[:, 2]
        zz = np.where(np.abs(z) > 1e-12, z, 1e-12)
        u = Xc[:, 0] / zz - x[:, 0]
        v = Xc[:, 1] / zz - x[:, 1]
        e = np.asarray(focal, np.float64)[cam] * np.sqrt(u * u + v * v)
        return np.where(z > 0, e, np.inf)

    P = pts[kp_track]
    in1 = reproj_err(P, ci, x1) <= max_err_px
    in2 = reproj_err(P, cj, x2) <= max_err_px
    inlier_cams = [set() for _ in range(T)]
    for m in np.nonzero(in1)[0]:
        inlier_cams[kp_track[m]].add(int(ci[m]))
    for m in np.nonzero(in2)[0]:
        inlier_cams[kp_track[m]].add(int(cj[m]))
    ncam = np.array([len(s) for s in inlier_cams])
    r1 = o[ci] - P
    r2 = o[cj] - P
    cosang = np.sum(r1 * r2, 1) / np.maximum(np.linalg.norm(r1, axis=1) * np.linalg.norm(r2, axis=1), 1e-300)
    ang = np.degrees(np.arccos(np.clip(cosang, -1.0, 1.0)))
    ang = np.where(in1 & in2, ang, 0.0)
    max_ang = np.zeros(T)
    np.maximum.at(max_ang, kp_track, ang)
    valid = (cnt > 0) & (ncam >= 3) & (max_ang >= min_angle_deg)
    if diag:
        return pts, valid, ncam, {"err1": reproj_err(P, ci, x1), "err2": reproj_err(P, cj, x2),
                                  "angle_deg": np.degrees(np.arccos(np.clip(cosang, -1.0, 1.0))),
                                  "pair_ok": ok, "max_angle_deg": max_ang,
                                  "pair_sin2": np.sum(np.cross(d1, d2) ** 2, 1) /
                                               np.maximum(np.sum(d1 * d1, 1) * np.sum(d2 * d2, 1), 1e-300)}
    return pts, valid, ncam
