"""Two-view setup steps for the oracle (float64).  Test infrastructure only.

* Relative pose of an image pair from its keypoint pairs.  The paper takes
  R^{i->j}, t^{i->j} from decomposing the fundamental / homography matrix of
  geometric verification (Sec. 3.3, "Global Rotation"; Appendix
  "Limitations": of the four decompositions the cheirality check keeps one,
  lowest index on ties).  Here the essential matrix comes from the same
  keypoint pairs: the unit vector e minimising sum_m (v_m . e)^2 (v_m =
  vec(x~2 x~1^T)), i.e. the eigenvector of W_n (Eq. 17) with the smallest
  eigenvalue, optionally re-solved a few times with IRLS weights
  1/max(|r|, delta) -- the linear eight-point estimate in calibrated
  coordinates.  It is projected onto the essential matrices (singular values
  (1, 1, 0), Sec. 3.1: the characterisation of essential matrices) and
  decomposed.
* Relative translation re-estimation (Appendix "Relative Translation"): with
  R_ij from the global rotations, candidate unit translations on the sphere
  are scored by the mean absolute epipolar error and the best one is kept.
  The candidate set (a reading: the paper does not give it) is a Fibonacci
  lattice on the hemisphere, refined twice by Fibonacci lattices on spherical
  caps around the best candidate; the error is even in t, so the sign is
  chosen by cheirality.
"""
import numpy as np

from .so3 import skew

GOLDEN_ANGLE = np.pi * (3.0 - np.sqrt(5.0))


# ------------------------------------------------------------ cheirality

def depths(R, t, x1, x2):
    """Depths (l1, l2) with l2 x2 = l1 R x1 + t, least squares per pair."""
    a = np.einsum("ab,mb->ma", R, x1)       # R x1
    # [a, -x2] [l1, l2]^T = -t
    A11 = np.sum(a * a, 1)
    A12 = -np.sum(a * x2, 1)
    A22 = np.sum(x2 * x2, 1)
    b1 = -np.sum(a * t, 1)
    b2 = np.sum(x2 * t, 1)
    det = A11 * A22 - A12 * A12
    ok = np.abs(det) > 1e-12
    dd = np.where(ok, det, 1.0)
    l1 = (A22 * b1 - A12 * b2) / dd
    l2 = (A11 * b2 - A12 * b1) / dd
    return np.where(ok, l1, 0.0), np.where(ok, l2, 0.0)


def cheirality_count(R, t, x1, x2):
    l1, l2 = depths(R, t, x1, x2)
    return int(np.sum((l1 > 0) & (l2 > 0)))


# ------------------------------------------------------------ eight point

def essential_from_pairs(x1, x2, weights=None):
    """Smallest-eigenvalue eigenvector of sum_m w_m v_m v_m^T, as a 3x3 matrix."""
    v = np.einsum("ma,mb->mab", x2, x1).reshape(-1, 9)
    w = np.ones(len(v)) if weights is None else weights
    W = np.einsum("m,ma,mb->ab", w, v, v)
    _, V = np.linalg.eigh(W)
    return V[:, 0].reshape(3, 3)


def project_essential(E):
    U, s, Vt = np.linalg.svd(E)
    return U @ np.diag([1.0, 1.0, 0.0]) @ Vt, s


def decompositions(E):
    """The four (R, t) with E ~ [t]_x R, in the order (R1, t), (R1, -t),
    (R2, t), (R2, -t)."""
    U, _, Vt = np.linalg.svd(E)
    if np.linalg.det(U) < 0:
        U = -U
    if np.linalg.det(Vt) < 0:
        Vt = -Vt
    Wm = np.array([[0.0, -1.0, 0.0], [1.0, 0.0, 0.0], [0.0, 0.0, 1.0]])
    R1 = U @ Wm @ Vt
    R2 = U @ Wm.T @ Vt
    t = U[:, 2]
    return [(R1, t), (R1, -t), (R2, t), (R2, -t)]


def relative_pose(x1, x2, irls_iters=0, delta=1e-5):
    """(R_ij, unit t_ij) of one image pair from its calibrated keypoint pairs."""
    E = essential_from_pairs(x1, x2)
    for _ in range(irls_iters):
        r = np.abs(np.einsum("ma,ab,mb->m", x2, E, x1))
        E = essential_from_pairs(x1, x2, 1.0 / np.maximum(r, delta))
    E, _ = project_essential(E)
    cands = decompositions(E)
    counts = [cheirality_count(R, t, x1, x2) for R, t in cands]
    best = int(np.argmax(counts))          # first maximum: lowest index on ties
    R, t = cands[best]
    return R, t / np.linalg.norm(t)


# ------------------------------------------------------------ grid search

def hemisphere_lattice(K):
    """K Fibonacci points on the unit hemisphere z > 0."""
    k = np.arange(K, dtype=np.float64)
    z = 1.0 - (k + 0.5) / K
    r = np.sqrt(1.0 - z * z)
    phi = k * GOLDEN_ANGLE
    return np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)


def cap_lattice(K, radius, centre):
    """K Fibonacci points on the spherical cap of angular radius `radius`
    around the unit vector `centre`."""
    k = np.arange(K, dtype=np.float64)
    z = 1.0 - (1.0 - np.cos(radius)) * (k + 0.5) / K
    r = np.sqrt(np.maximum(1.0 - z * z, 0.0))
    phi = k * GOLDEN_ANGLE
    pts = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    return pts @ _rotation_to(centre).T


def _rotation_to(c):
    """Rotation taking (0, 0, 1) to the unit vector c (Rodrigues)."""
    c = np.asarray(c, np.float64)
    z = np.array([0.0, 0.0, 1.0])
    v = np.cross(z, c)
    s = np.linalg.norm(v)
    cth = float(np.dot(z, c))
    if s < 1e-12:
        return np.eye(3) if cth > 0 else np.diag([1.0, -1.0, -1.0])
    K = skew(v / s)
    ang = np.arctan2(s, cth)
    return np.eye(3) + np.sin(ang) * K + (1.0 - np.cos(ang)) * (K @ K)


def mean_epipolar_error(t, R, x1, x2):
    """mean_m |x2^T [t]_x R x1| for each candidate t [K,3] (= |t . (R x1 x x2)|)."""
    a = np.cross(np.einsum("ab,mb->ma", R, x1), x2)
    return np.mean(np.abs(t @ a.T), axis=1)


GRID_LEVELS = ((4096, None), (1024, 2.0), (1024, 2.0))   # (points, cap radius in spacings)


def lattice_spacing(K, area):
    return np.sqrt(area / K)


def relative_translation(R, x1, x2, levels=GRID_LEVELS):
    """Best unit t for the pair (grid search of the appendix), sign by
    cheirality (+t on ties).  Returns (t, mean error)."""
    K0 = levels[0][0]
    cand = hemisphere_lattice(K0)
    err = mean_epipolar_error(cand, R, x1, x2)
    best = int(np.argmin(err))
    t, e = cand[best], err[best]
    spacing = lattice_spacing(K0, 2.0 * np.pi)
    for K, mult in levels[1:]:
        radius = mult * spacing
        cand = cap_lattice(K, radius, t)
        err = mean_epipolar_error(cand, R, x1, x2)
        b = int(np.argmin(err))
        if err[b] < e:
            t, e = cand[b], err[b]
        spacing = lattice_spacing(K, 2.0 * np.pi * (1.0 - np.cos(radius)))
    if cheirality_count(R, -t, x1, x2) > cheirality_count(R, t, x1, x2):
        t = -t
    return t / np.linalg.norm(t), e
