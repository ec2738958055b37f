"""Epipolar adjustment for the oracle (float64).  Test infrastructure only.

Sec. 3.3 "Epipolar Adjustment" and Appendix "Epipolar Adjustment":
  * point pairs in normalised homogeneous coordinates x~ = K^-1 [u, v, 1]^T
    with the principal point at the image centre and z = 1;
  * E_n is the essential matrix of image pair n = (i_n, j_n) computed from the
    world-to-camera rotations and translations of both images:
        R_ij = R_j R_i^T,  t_ij = t_j - R_ij t_i,  E_n = [t_ij/|t_ij|]_x R_ij
    (the direction of t_ij is used, so the loss does not shrink to zero by
    shrinking the baseline);
  * direct L1 objective  L = 1/Z sum_n sum_m |x2^T E_n x1|          (Eq. 7);
  * L2 objective         L = 1/Z sum_n sum_m (x2^T E_n x1)^2        (Eq. 8);
  * IRLS objective       L = 1/Z sum_n sum_m (x2^T E_n x1)^2/|eps^| (Eq. 9);
  * compact form         L = 1/Z sum_n e_n^T W_n e_n,
                         W_n = sum_m w_m w_m^T, w_m = vec(x2 x1^T), e_n = vec(E_n)
    (Eq. 8 right-hand side and Eqs. 16-17; row-major vec; the factor is 1/Z so
    that the two sides of Eq. 8 are equal).

Parameters of the epipolar stage, per camera: [a1 (3), a2 (3), t (3)] with
(a1, a2) the 6D rotation and t the world-to-camera translation.
"""
import numpy as np

from .so3 import rot_from_6d, rot_from_6d_vjp, skew

_BASIS_SKEW = np.stack([skew(np.eye(3)[k]) for k in range(3)])   # [3,3,3]


def calibrate(px, focal, cx, cy):
    """Pixels [...,2] -> homogeneous calibrated coordinates [...,3] with z = 1."""
    px = np.asarray(px, dtype=np.float64)
    x = (px[..., 0] - cx) / focal
    y = (px[..., 1] - cy) / focal
    return np.stack([x, y, np.ones_like(x)], axis=-1)


def calibrated_pairs(kp1_px, kp2_px, kp_img_pair, pair_i, pair_j, focal, cx, cy):
    """x~1 (in image i_n) and x~2 (in image j_n) of every keypoint pair, [Z,3] each."""
    ci = np.asarray(pair_i)[kp_img_pair]
    cj = np.asarray(pair_j)[kp_img_pair]
    f = np.asarray(focal, dtype=np.float64)
    x1 = calibrate(kp1_px, f[ci], np.asarray(cx, np.float64)[ci], np.asarray(cy, np.float64)[ci])
    x2 = calibrate(kp2_px, f[cj], np.asarray(cx, np.float64)[cj], np.asarray(cy, np.float64)[cj])
    return x1, x2


def pair_geometry(params, pair_i, pair_j):
    """Per image pair: R_i, R_j, t_i, R_ij, t_ij, |t_ij|, t^ = t_ij/|t_ij|, E."""
    params = np.asarray(params, dtype=np.float64)
    R = rot_from_6d(params[:, 0:6])
    t = params[:, 6:9]
    Ri, Rj = R[pair_i], R[pair_j]
    ti, tj = t[pair_i], t[pair_j]
    Rij = Rj @ np.transpose(Ri, (0, 2, 1))
    tij = tj - np.einsum("pab,pb->pa", Rij, ti)
    nrm = np.linalg.norm(tij, axis=1)
    that = tij / nrm[:, None]
    E = skew(that) @ Rij
    return dict(R=R, Ri=Ri, Rj=Rj, ti=ti, Rij=Rij, tij=tij, nrm=nrm, that=that, E=E)


def essential_matrices(params, pair_i, pair_j):
    return pair_geometry(params, pair_i, pair_j)["E"]


def residuals(E, x1, x2, kp_img_pair):
    """Algebraic epipolar error r_m = x2^T E_n x1 of every keypoint pair."""
    return np.einsum("ma,mab,mb->m", x2, E[kp_img_pair], x1)


def _rho(r, weights, loss):
    w = np.ones_like(r) if weights is None else np.asarray(weights, dtype=np.float64)
    if loss == "l1":
        return w * np.abs(r), w * np.sign(r)
    if loss == "l2":
        return w * r * r, 2.0 * w * r
    raise ValueError(loss)


def backward_E(G, geo, n_cams, pair_i, pair_j, params):
    """Chain rule from dL/dE_n (G [P,3,3]) to the per-camera parameters.

    E = [t^]_x R_ij with t^ = t_ij/|t_ij|, t_ij = t_j - R_ij t_i, R_ij = R_j R_i^T.
    Each step is differentiated on its own and the pieces are summed per
    camera; the 6D step is ``so3.rot_from_6d_vjp``.
    """
    Rij, that, nrm = geo["Rij"], geo["that"], geo["nrm"]
    Ri, Rj, ti = geo["Ri"], geo["Rj"], geo["ti"]
    # through E = [t^]_x R_ij with t^ held fixed
    dRij = np.transpose(skew(that), (0, 2, 1)) @ G
    # dL/dt^_k = <G, [e_k]_x R_ij>
    dthat = np.einsum("pab,kac,pcb->pk", G, _BASIS_SKEW, Rij)
    # t^ = t_ij / |t_ij|
    dtij = (dthat - that * np.sum(that * dthat, axis=1, keepdims=True)) / nrm[:, None]
    # t_ij = t_j - R_ij t_i
    dRij = dRij - np.einsum("pa,pb->pab", dtij, ti)
    dtj = dtij
    dti = -np.einsum("pba,pb->pa", Rij, dtij)
    # R_ij = R_j R_i^T
    dRj = dRij @ Ri
    dRi = np.transpose(dRij, (0, 2, 1)) @ Rj
    gR = np.zeros((n_cams, 3, 3))
    gt = np.zeros((n_cams, 3))
    np.add.at(gR, pair_i, dRi)
    np.add.at(gR, pair_j, dRj)
    np.add.at(gt, pair_i, dti)
    np.add.at(gt, pair_j, dtj)
    g6 = rot_from_6d_vjp(np.asarray(params, np.float64)[:, 0:6], gR)
    return np.concatenate([g6, gt], axis=1)


def direct_loss_grad(params, pair_i, pair_j, x1, x2, kp_img_pair, weights=None,
                     loss="l1", inv_z=None):
    """Loss and gradient of the direct per-keypoint-pair objective.

    loss="l1": L = inv_z * sum w |r|   (Eq. 7 with w = 1, inv_z = 1/Z)
    loss="l2": L = inv_z * sum w r^2   (Eq. 8 with w = 1; Eq. 9 with w = 1/|eps^|)
    Subgradient of |r| at r = 0 is 0.  Returns (loss, grad [N,9], G [P,3,3]).
    """
    params = np.asarray(params, dtype=np.float64)
    n_cams = params.shape[0]
    P = len(pair_i)
    Z = len(kp_img_pair)
    if inv_z is None:
        inv_z = 1.0 / max(Z, 1)
    geo = pair_geometry(params, pair_i, pair_j)
    r = residuals(geo["E"], x1, x2, kp_img_pair)
    rho, drho = _rho(r, weights, loss)
    L = inv_z * np.sum(rho)
    # dL/dE_n = inv_z * sum_m drho_m x2 x1^T
    G = np.zeros((P, 3, 3))
    np.add.at(G, kp_img_pair, inv_z * drho[:, None, None] * np.einsum("ma,mb->mab", x2, x1))
    grad = backward_E(G, geo, n_cams, pair_i, pair_j, params)
    return L, grad, G


def build_W(x1, x2, kp_img_pair, n_pairs, weights=None):
    """W_n = sum_m w_m vec(x2 x1^T) vec(x2 x1^T)^T, [P,9,9] (Eq. 17)."""
    v = np.einsum("ma,mb->mab", x2, x1).reshape(-1, 9)
    wt = np.ones(len(v)) if weights is None else np.asarray(weights, np.float64)
    W = np.zeros((n_pairs, 9, 9))
    np.add.at(W, kp_img_pair, wt[:, None, None] * np.einsum("ma,mb->mab", v, v))
    return W


def compact_loss_grad(params, pair_i, pair_j, W, inv_z):
    """L = inv_z * sum_n e_n^T W_n e_n and its gradient (Eq. 8, right-hand side).
    dL/de_n = 2 inv_z W_n e_n.  Returns (loss, grad [N,9], G [P,3,3])."""
    params = np.asarray(params, dtype=np.float64)
    geo = pair_geometry(params, pair_i, pair_j)
    e = geo["E"].reshape(-1, 9)
    We = np.einsum("pab,pb->pa", W, e)
    L = inv_z * np.sum(e * We)
    G = (2.0 * inv_z * We).reshape(-1, 3, 3)
    grad = backward_E(G, geo, params.shape[0], pair_i, pair_j, params)
    return L, grad, G


def irls_weights(r_hat, tau, delta):
    """IRLS weight of every keypoint pair (Eq. 9 and the filtering that follows
    it): 1/max(|eps^|, delta) for |eps^| < tau, and 0 (filtered out) otherwise."""
    a = np.abs(np.asarray(r_hat, np.float64))
    keep = a < tau
    return np.where(keep, 1.0 / np.maximum(a, delta), 0.0), keep
