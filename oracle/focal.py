"""Focal lengths inside epipolar adjustment, for the oracle (float64).  Test
infrastructure only.

Sec. 3.3, end of "Epipolar Adjustment": besides the poses, the focal lengths
can be optimised by folding them into the matrices of the epipolar
objective, which then become fundamental rather than essential matrices.
The paper gives no formula; the reading used here (and on the GPU):

  * camera c carries a log focal ratio phi_c: f_c = f0_c exp(phi_c), with the
    keypoints calibrated once at the initial focal f0 (principal point fixed);
  * recalibrating at f_c scales the first two coordinates of x~ by
    s_c = exp(-phi_c):  x~(phi) = S_c x~0,  S_c = diag(s_c, s_c, 1);
  * so r = x2~(phi)^T E_n x1~(phi) = x2~0^T E'_n x1~0 with
        E'_n = S_j E_n S_i,
    and every objective of epipolar.py (L1, L2, IRLS, compact) applies to
    E' unchanged;
  * chain rule, with G' = dL/dE'_n and D = diag(1, 1, 0):
        dL/dE_n = S_j G' S_i,
        dL/ds_i = <G', S_j E_n D>,   dL/ds_j = <G', D E_n S_i>,
        dL/dphi_c = -s_c dL/ds_c (summed over the image pairs of camera c).
"""
import numpy as np

from . import epipolar as ep

_D = np.diag([1.0, 1.0, 0.0])


def scale_matrices(phi):
    """S_c = diag(exp(-phi_c), exp(-phi_c), 1), [N,3,3]."""
    s = np.exp(-np.asarray(phi, np.float64))
    S = np.zeros((len(s), 3, 3))
    S[:, 0, 0] = s
    S[:, 1, 1] = s
    S[:, 2, 2] = 1.0
    return S


def focal_matrices(E, phi, pair_i, pair_j):
    """E'_n = S_j E_n S_i for every image pair, [P,3,3]."""
    S = scale_matrices(phi)
    return S[pair_j] @ E @ S[pair_i]


def _backward(Gp, geo, phi, pair_i, pair_j, params):
    """(grad [N,9], gphi [N]) from G' = dL/dE'."""
    S = scale_matrices(phi)
    Si, Sj = S[pair_i], S[pair_j]
    E = geo["E"]
    G = Sj @ Gp @ Si
    grad = ep.backward_E(G, geo, len(phi), pair_i, pair_j, params)
    ds_i = np.einsum("pab,pab->p", Gp, Sj @ E @ _D)
    ds_j = np.einsum("pab,pab->p", Gp, _D @ E @ Si)
    s = np.exp(-np.asarray(phi, np.float64))
    gphi = np.zeros(len(phi))
    np.add.at(gphi, pair_i, -s[pair_i] * ds_i)
    np.add.at(gphi, pair_j, -s[pair_j] * ds_j)
    return grad, gphi


def direct_loss_grad(params, phi, pair_i, pair_j, x1, x2, kp_img_pair, weights=None, loss="l1", inv_z=None):
    """The direct objective of epipolar.direct_loss_grad at E' = S_j E S_i,
    with x1, x2 calibrated at f0.  Returns (loss, grad [N,9], gphi [N])."""
    params = np.asarray(params, np.float64)
    phi = np.asarray(phi, np.float64)
    Z = len(kp_img_pair)
    if inv_z is None:
        inv_z = 1.0 / max(Z, 1)
    geo = ep.pair_geometry(params, pair_i, pair_j)
    Ep = focal_matrices(geo["E"], phi, pair_i, pair_j)
    r = ep.residuals(Ep, x1, x2, kp_img_pair)
    rho, drho = ep._rho(r, weights, loss)
    L = inv_z * np.sum(rho)
    Gp = np.zeros((len(pair_i), 3, 3))
    np.add.at(Gp, kp_img_pair, inv_z * drho[:, None, None] * np.einsum("ma,mb->mab", x2, x1))
    grad, gphi = _backward(Gp, geo, phi, pair_i, pair_j, params)
    return L, grad, gphi


def compact_loss_grad(params, phi, pair_i, pair_j, W, inv_z):
    """The compact objective inv_z sum_n e'_n^T W_n e'_n with e' = vec(E'),
    W_n built from the keypoints calibrated at f0.  Returns (loss, grad, gphi)."""
    params = np.asarray(params, np.float64)
    phi = np.asarray(phi, np.float64)
    geo = ep.pair_geometry(params, pair_i, pair_j)
    e = focal_matrices(geo["E"], phi, pair_i, pair_j).reshape(-1, 9)
    We = np.einsum("pab,pb->pa", W, e)
    L = inv_z * np.sum(e * We)
    Gp = (2.0 * inv_z * We).reshape(-1, 3, 3)
    grad, gphi = _backward(Gp, geo, phi, pair_i, pair_j, params)
    return L, grad, gphi
