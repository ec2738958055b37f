"""Global rotation for the oracle (float64).  Test infrastructure only.

* loss  L_R = 1/|P| sum_{(i,j)} d(R_j, R^{i->j} R_i)             (Eq. 3)
  with d the geodesic distance arccos((tr(R^T R') - 1)/2)         (Eq. 4)
  and R_i from the 6D representation (Sec. 3.3).
* initialisation: the modified Martinec-Pajdla scheme of Appendix
  "Global Rotation / Initialization" (Eqs. 10-14): first columns from the
  least-squares problem L^(1) (Eq. 12), second columns from L^(2) with the
  orthogonality penalty (Eq. 13), each solved as the eigenvector of the
  smallest eigenvalue of its quadratic form (the "SVD" step), normalised per
  camera, Gram-Schmidt, third column = c1 x c2 (Eq. 14).
"""
import numpy as np

from .so3 import project_to_rotation, rot_from_6d, rot_from_6d_vjp


def loss_grad(params6, pair_i, pair_j, rel_R, project=True):
    """L_R and its gradient with respect to the 6D parameters [N,6].

    With M = R_j^T R_ij R_i, c = (tr M - 1)/2 and d = arccos(c):
    dd/dc = -1/sqrt(1 - c^2); tr M = <R_j, R_ij R_i> so
    d tr/dR_j = R_ij R_i and d tr/dR_i = R_ij^T R_j.
    Where 1 - c^2 <= 0 (d = 0 or pi) the subgradient 0 is used.
    project: take each given R_ij as its nearest rotation first (arccos near 1
    is ill-conditioned, so a 1e-7 departure from orthogonality of a float32
    input would otherwise move d by ~1e-7/d).
    """
    params6 = np.asarray(params6, dtype=np.float64)
    n = params6.shape[0]
    P = len(pair_i)
    R = rot_from_6d(params6)
    Ri, Rj = R[pair_i], R[pair_j]
    Rij = np.asarray(rel_R, dtype=np.float64)
    if project:
        Rij = project_to_rotation(Rij)
    K = Rij @ Ri
    c = (np.einsum("pab,pab->p", Rj, K) - 1.0) / 2.0
    cc = np.clip(c, -1.0, 1.0)
    d = np.arccos(cc)
    L = np.sum(d) / P
    s2 = 1.0 - cc * cc
    dd_dc = np.where(s2 > 0.0, -1.0 / np.sqrt(np.where(s2 > 0.0, s2, 1.0)), 0.0)
    coef = dd_dc * 0.5 / P                    # dL/d tr M
    dRj = coef[:, None, None] * K
    dRi = coef[:, None, None] * (np.transpose(Rij, (0, 2, 1)) @ Rj)
    gR = np.zeros((n, 3, 3))
    np.add.at(gR, pair_i, dRi)
    np.add.at(gR, pair_j, dRj)
    return L, rot_from_6d_vjp(params6, gR)


def pairwise_errors(params6, pair_i, pair_j, rel_R):
    R = rot_from_6d(np.asarray(params6, np.float64))
    K = np.asarray(rel_R, np.float64) @ R[pair_i]
    c = (np.einsum("pab,pab->p", R[pair_j], K) - 1.0) / 2.0
    return np.arccos(np.clip(c, -1.0, 1.0))


def _column_form(n, pair_i, pair_j, rel_R):
    """Matrix A [3N,3N] with x^T A x = sum ||x_j - R_ij x_i||^2 (x stacks one
    3-vector per camera); uses R_ij^T R_ij = I."""
    A = np.zeros((3 * n, 3 * n))
    for p, (i, j) in enumerate(zip(pair_i, pair_j)):
        Rp = np.asarray(rel_R[p], np.float64)
        A[3 * i:3 * i + 3, 3 * i:3 * i + 3] += np.eye(3)
        A[3 * j:3 * j + 3, 3 * j:3 * j + 3] += np.eye(3)
        A[3 * j:3 * j + 3, 3 * i:3 * i + 3] -= Rp
        A[3 * i:3 * i + 3, 3 * j:3 * j + 3] -= Rp.T
    return A


def _smallest_eigvec(A):
    w, V = np.linalg.eigh(A)
    return V[:, 0]


def martinec_init(n, pair_i, pair_j, rel_R):
    """World-to-camera rotations [N,3,3] from relative rotations (Eqs. 10-14)."""
    A = _column_form(n, pair_i, pair_j, rel_R)
    # first columns: minimise L^(1) over a non-zero vector (Eq. 12)
    c1 = _smallest_eigvec(A).reshape(n, 3)
    c1 = c1 / np.linalg.norm(c1, axis=1, keepdims=True)
    # second columns: L^(2) = 1/|P| sum ||.||^2 + 1/|I| sum (c1_i^T c2_i)^2 (Eq. 13)
    B = A / len(pair_i)
    for i in range(n):
        B[3 * i:3 * i + 3, 3 * i:3 * i + 3] += np.outer(c1[i], c1[i]) / n
    c2 = _smallest_eigvec(B).reshape(n, 3)
    c2 = c2 / np.linalg.norm(c2, axis=1, keepdims=True)
    # Gram-Schmidt against the first column, then the cross product (Eq. 14)
    c2 = c2 - np.sum(c1 * c2, axis=1, keepdims=True) * c1
    c2 = c2 / np.linalg.norm(c2, axis=1, keepdims=True)
    c3 = np.cross(c1, c2)
    return np.stack([c1, c2, c3], axis=-1)
