"""Hand-built one-track scenes whose triangulation decisions are known from
the geometry alone (Appendix "Sparse Reconstruction"; the readings of the
inlier test, the 3-camera rule and the angle rule are those of
oracle/triangulation.py).

Every camera has R = I and sits on the plane z = -5 looking along +z at the
track's point X = 0, with its principal point at (320, 240).  A camera at
o = (ox, oy, -5) sees X at the calibrated point (-ox/5, -oy/5), i.e. at the
pixel (320 - f ox/5, 240 - f oy/5).  The focal lengths differ from camera to
camera, so that measuring an error with the wrong camera's focal length, or in
calibrated units, changes a decision.

Two devices make the expected decisions exact:
  * an observation that is displaced on purpose is paired only with a camera
    whose ray is parallel to the displaced ray (same calibrated point, R = I,
    so bit-identical ray directions): that keypoint pair is degenerate and
    contributes no midpoint, so the averaged point stays at X;
  * displacements are dyadic (4 +- 2^-10 px) and the two focal lengths of a
    degenerate pair differ by a factor of 2, so the pixels are exact in
    float32 and the two calibrated points are equal bit for bit.
"""
import numpy as np

from synthetic.scenes import Scene

CX, CY = 320.0, 240.0


def _scene(name, focal, centres, pairs, track_len):
    """pairs: list of (i, j, (u1, v1), (u2, v2)) with i < j, in image-pair
    order; one keypoint pair per image pair, all of track 0."""
    N = len(focal)
    R = np.repeat(np.eye(3)[None], N, axis=0)
    o = np.asarray(centres, np.float64)
    t = -o                                  # t = -R o with R = I
    pi = np.array([p[0] for p in pairs], np.int32)
    pj = np.array([p[1] for p in pairs], np.int32)
    kp1 = np.array([p[2] for p in pairs], np.float32)
    kp2 = np.array([p[3] for p in pairs], np.float32)
    # every pixel of the construction is exact in float32
    assert np.array_equal(kp1.astype(np.float64), np.array([p[2] for p in pairs], np.float64))
    assert np.array_equal(kp2.astype(np.float64), np.array([p[3] for p in pairs], np.float64))
    Z = len(pairs)
    return Scene(name=name, seed=0, width=640, height=480, focal=np.asarray(focal, np.float64),
                 cx=np.full(N, CX), cy=np.full(N, CY), R_gt=R, t_gt=t, points=np.zeros((1, 3)),
                 pair_i=pi, pair_j=pj, kp_img_pair=np.arange(Z, dtype=np.int32), kp1_px=kp1, kp2_px=kp2,
                 kp_track=np.zeros(Z, np.int32), kp_inlier=np.ones(Z, bool), meta={"track_len": track_len})


def _px(f, o):
    """exact pixel of X = 0 seen from a camera at o with R = I"""
    return (CX - f * o[0] / 5.0, CY - f * o[1] / 5.0)


def reprojection_case(delta_px, displaced_first):
    """Cameras A (f 500), B (f 700), D (f 1000).  A and B see X exactly
    (image pair A-B).  D, on the axis through X, sees X at the principal point;
    its keypoint is displaced by delta_px along u, and it is paired with A only.
    A sits where its ray to X has the direction of D's displaced ray, so the
    pair A-D is degenerate and the averaged point is X.  D's reprojection
    error is then delta_px exactly (D's focal length; in A's it would be
    delta_px / 2).  Expected: D is an inlier iff delta_px <= 4; the track has
    3 inlier cameras (kept: angle A-X-B ~ 16 deg) or 2 (dropped).
    displaced_first: D is the first camera of its image pair (x~1) instead of
    the second (x~2)."""
    fA, fB, fD = 500.0, 700.0, 1000.0
    oA = (-5.0 * delta_px / fD, 0.0, -5.0)
    oB = (1.0, 1.0, -5.0)
    oD = (0.0, 0.0, -5.0)
    pA = (CX + delta_px / 2.0, CY)             # = _px(fA, oA): A's ray points at X
    pB = _px(fB, oB)
    pD = (CX + delta_px, CY)                    # true projection (320, 240), displaced
    if displaced_first:                          # cameras D=0, A=1, B=2
        return _scene("tri_reproj_first", [fD, fA, fB], [oD, oA, oB],
                      [(0, 1, pD, pA), (1, 2, pA, pB)], 3)
    return _scene("tri_reproj_second", [fA, fB, fD], [oA, oB, oD],   # cameras A=0, B=1, D=2
                  [(0, 1, pA, pB), (0, 2, pA, pD)], 3)


def angle_case(theta_deg):
    """Cameras A, C, B with exact observations; seen from X, C is theta/2 and
    B theta away from A in the x-z plane (angles A-X-C = C-X-B = theta/2,
    A-X-B = theta).  Expected: 3 inlier cameras, largest angle theta; kept iff
    theta >= 2 deg."""
    th = np.radians(theta_deg)
    fA, fC, fB = 500.0, 650.0, 800.0
    oA = (0.0, 0.0, -5.0)
    oC = (5.0 * np.tan(th / 2.0), 0.0, -5.0)
    oB = (5.0 * np.tan(th), 0.0, -5.0)
    f = [fA, fC, fB]
    o = [oA, oC, oB]
    # pixels rounded to float32 (the construction stays exact to ~1e-7 deg)
    px = [tuple(float(np.float32(v)) for v in _px(f[k], o[k])) for k in range(3)]
    return _scene("tri_angle", f, o, [(0, 1, px[0], px[1]), (0, 2, px[0], px[2]), (1, 2, px[1], px[2])], 3)


def exclusion_case(displace):
    """Cameras A (f 500), B (f 800, 3 deg from A seen from X), C (f 650,
    1.5 deg).  Image pairs A-B, A-C, B-C.  With displace=True, B's keypoint in
    A-B sits at B's principal point: its ray is parallel to A's (pair A-B
    degenerate, no midpoint) and ~42 px from X's projection (outlier), while
    B's keypoint in B-C is exact, so B is still an inlier camera.  The largest
    angle over pairs whose two keypoints are inliers is then 1.5 deg (A-C,
    B-C): dropped, with 3 inlier cameras.  With displace=False every
    observation is exact and A-B's 3 deg counts: kept."""
    fA, fB, fC = 500.0, 800.0, 650.0
    oA = (0.0, 0.0, -5.0)
    oB = (5.0 * np.tan(np.radians(3.0)), 0.0, -5.0)
    oC = (5.0 * np.tan(np.radians(1.5)), 0.0, -5.0)
    pA = _px(fA, oA)
    pB = tuple(float(np.float32(v)) for v in _px(fB, oB))
    pC = tuple(float(np.float32(v)) for v in _px(fC, oC))
    pB_ab = (CX, CY) if displace else pB
    return _scene("tri_exclusion", [fA, fB, fC], [oA, oB, oC],
                  [(0, 1, pA, pB_ab), (0, 2, pA, pC), (1, 2, pB, pC)], 3)


# (scene, expected valid, expected inlier cameras)
def all_cases():
    d = 2.0 ** -10
    out = []
    for first in (False, True):
        out.append((reprojection_case(4.0 - d, first), True, 3))
        out.append((reprojection_case(4.0 + d, first), False, 2))
    out.append((angle_case(2.01), True, 3))
    out.append((angle_case(1.99), False, 3))
    out.append((exclusion_case(True), False, 3))
    out.append((exclusion_case(False), True, 3))
    return out
