"""Rotations for the oracle (float64).  Test infrastructure only.

* 6D representation (Sec. 3.3, global rotation; Zhou et al.): two 3-vectors
  a1, a2 are the first two columns before orthonormalisation; b1 = a1/|a1|, b2 = normalise(a2 -
  (b1.a2) b1), b3 = b1 x b2, R = [b1 b2 b3] (columns).
* geodesic distance d(R, R') = arccos((tr(R^T R') - 1) / 2)   (Eq. 4).
"""
import numpy as np


def skew(v):
    """[v]_x for v of shape [..., 3]."""
    v = np.asarray(v, dtype=np.float64)
    z = np.zeros(v.shape[:-1])
    return np.stack([
        np.stack([z, -v[..., 2], v[..., 1]], -1),
        np.stack([v[..., 2], z, -v[..., 0]], -1),
        np.stack([-v[..., 1], v[..., 0], z], -1),
    ], -2)


def rot_from_6d(a):
    """a [..., 6] = (a1, a2) -> R [..., 3, 3] with columns b1, b2, b3."""
    a = np.asarray(a, dtype=np.float64)
    a1, a2 = a[..., 0:3], a[..., 3:6]
    b1 = a1 / np.linalg.norm(a1, axis=-1, keepdims=True)
    u2 = a2 - np.sum(b1 * a2, -1, keepdims=True) * b1
    b2 = u2 / np.linalg.norm(u2, axis=-1, keepdims=True)
    b3 = np.cross(b1, b2)
    return np.stack([b1, b2, b3], axis=-1)


def rot_to_6d(R):
    """The first two columns of R, concatenated: the 6D vector that maps back to R."""
    R = np.asarray(R, dtype=np.float64)
    return np.concatenate([R[..., :, 0], R[..., :, 1]], axis=-1)


def rot_from_6d_vjp(a, gR):
    """Gradient with respect to a of <gR, rot_from_6d(a)>; written out by hand
    along the Gram-Schmidt steps above (each step's transpose, in reverse)."""
    a = np.asarray(a, dtype=np.float64)
    gR = np.asarray(gR, dtype=np.float64)
    a1, a2 = a[..., 0:3], a[..., 3:6]
    n1 = np.linalg.norm(a1, axis=-1, keepdims=True)
    b1 = a1 / n1
    d12 = np.sum(b1 * a2, -1, keepdims=True)
    u2 = a2 - d12 * b1
    n2 = np.linalg.norm(u2, axis=-1, keepdims=True)
    b2 = u2 / n2
    gb1 = gR[..., :, 0].copy()
    gb2 = gR[..., :, 1].copy()
    gb3 = gR[..., :, 2]
    # b3 = b1 x b2
    gb1 += np.cross(b2, gb3)
    gb2 += np.cross(gb3, b1)
    # b2 = u2 / |u2|
    gu2 = (gb2 - b2 * np.sum(b2 * gb2, -1, keepdims=True)) / n2
    # u2 = a2 - (b1.a2) b1
    ga2 = gu2 - b1 * np.sum(b1 * gu2, -1, keepdims=True)
    gb1 += -d12 * gu2 - a2 * np.sum(b1 * gu2, -1, keepdims=True)
    # b1 = a1 / |a1|
    ga1 = (gb1 - b1 * np.sum(b1 * gb1, -1, keepdims=True)) / n1
    return np.concatenate([ga1, ga2], axis=-1)


def geodesic(R, Rp):
    """d(R, R') = arccos((tr(R^T R') - 1)/2), argument clipped to [-1, 1] (Eq. 4)."""
    c = (np.einsum("...ij,...ij->...", R, Rp) - 1.0) / 2.0
    return np.arccos(np.clip(c, -1.0, 1.0))


def project_to_rotation(M):
    """Nearest rotation (Frobenius) of each 3x3 matrix: U diag(1, 1, det(U V^T)) V^T
    from the SVD M = U S V^T.  A float32 copy of a rotation is a rotation only
    to ~1e-7; the geodesic distance of Eq. 4 is defined for rotations, so the
    oracle evaluates it on the rotation the given matrix stands for."""
    M = np.asarray(M, dtype=np.float64)
    U, _, Vt = np.linalg.svd(M)
    d = np.sign(np.linalg.det(U @ Vt))
    D = np.zeros(M.shape)
    D[..., 0, 0] = 1.0
    D[..., 1, 1] = 1.0
    D[..., 2, 2] = d
    return U @ D @ Vt


def angle_axis(axis, ang):
    """Rodrigues' formula (used by tests to build exact rotations)."""
    axis = np.asarray(axis, dtype=np.float64)
    axis = axis / np.linalg.norm(axis)
    K = skew(axis)
    return np.eye(3) + np.sin(ang) * K + (1.0 - np.cos(ang)) * (K @ K)
