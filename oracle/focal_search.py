"""Focal length interval search for the oracle (float64).  Test infrastructure
only.

Sec. 3.1 "Focal Length Estimation" (Eq. focal-vote) and Appendix "Focal
Length Estimation" (which follows Appendix "Distortion Estimation",
"Multiple cameras"):

  * a 3x3 matrix is essential iff its singular values are (s, s, 0); with the
    right intrinsics K, E = K^T F K has lambda1 / lambda2 = 1;
  * a candidate focal length is scored over a set of image pairs by
        v = sum_pairs exp((1 - lambda1 / lambda2) / tau),
    lambda1 >= lambda2 the two largest singular values, and the candidate with
    the highest score is kept (the first on ties);
  * several cameras (groups of images sharing intrinsics): the groups are
    estimated one by one; an image pair is "ready" for a group when both of its
    images belong to the group, or one does and the other's group is already
    estimated; the group with the most ready pairs goes next (the lowest index
    on ties), scored on its ready pairs with the known focal lengths fixed.

Readings (the paper gives no numbers): the two-view matrix of an image pair is
the linear eight-point estimate in coordinates calibrated at initial focal
lengths f0 (relpose.essential_from_pairs, optional IRLS re-solves); with a
fixed principal point, K0^-1 K = diag(rho, rho, 1) for rho = f / f0, so the
candidate essential matrix is D_j E0 D_i with D = diag(rho, rho, 1); the
candidates are rho_k = exp of n points spaced evenly in [log rho_min,
log rho_max]; image pairs with fewer than 8 keypoint pairs take no part.
"""
import numpy as np

from . import relpose as rp


def initial_essentials(x1, x2, kp_img_pair, n_pairs, irls_iters=0, delta=1e-5):
    """E0 [P,3,3] (unit Frobenius norm) and valid [P] (>= 8 keypoint pairs)."""
    off = np.concatenate([[0], np.cumsum(np.bincount(kp_img_pair, minlength=n_pairs))])
    E0 = np.zeros((n_pairs, 3, 3))
    valid = np.zeros(n_pairs, bool)
    for p in range(n_pairs):
        a, b = off[p], off[p + 1]
        if b - a < 8:
            continue
        E = rp.essential_from_pairs(x1[a:b], x2[a:b])
        for _ in range(irls_iters):
            r = np.abs(np.einsum("ma,ab,mb->m", x2[a:b], E, x1[a:b]))
            E = rp.essential_from_pairs(x1[a:b], x2[a:b], 1.0 / np.maximum(r, delta))
        E0[p] = E
        valid[p] = True
    return E0, valid


def candidates(rho_min, rho_max, n):
    return np.exp(np.linspace(np.log(rho_min), np.log(rho_max), n))


def vote_terms(E0, rho_i, rho_j, tau):
    """exp((1 - lambda1/lambda2)/tau) of D_j E0 D_i for every image pair
    (rho_i, rho_j scalars or [P])."""
    ri = np.broadcast_to(np.asarray(rho_i, np.float64), (len(E0),))
    rj = np.broadcast_to(np.asarray(rho_j, np.float64), (len(E0),))
    Di = np.zeros((len(E0), 3, 3))
    Dj = np.zeros((len(E0), 3, 3))
    Di[:, 0, 0] = Di[:, 1, 1] = ri
    Dj[:, 0, 0] = Dj[:, 1, 1] = rj
    Di[:, 2, 2] = Dj[:, 2, 2] = 1.0
    s = np.linalg.svd(Dj @ E0 @ Di, compute_uv=False)
    return np.exp((1.0 - s[:, 0] / s[:, 1]) / tau)


def search_shared(E0, valid, rhos, tau):
    """One focal length for every image: (best index, votes [n])."""
    v = np.array([np.sum(vote_terms(E0[valid], r, r, tau)) for r in rhos])
    return int(np.argmax(v)), v


def search_groups(E0, valid, pair_i, pair_j, group, n_groups, rhos, tau):
    """Greedy group order of the appendix.  Returns (rho [n_groups], with NaN
    for groups never ready, order of estimation)."""
    gi, gj = np.asarray(group)[pair_i], np.asarray(group)[pair_j]
    rho = np.full(n_groups, np.nan)
    done = np.zeros(n_groups, bool)
    order = []
    while not done.all():
        best_g, best_n = -1, 0
        for g in range(n_groups):
            if done[g]:
                continue
            ready = valid & (((gi == g) & (gj == g)) | ((gi == g) & done[gj]) | ((gj == g) & done[gi]))
            if ready.sum() > best_n:
                best_g, best_n = g, int(ready.sum())
        if best_g < 0:
            break
        g = best_g
        ready = valid & (((gi == g) & (gj == g)) | ((gi == g) & done[gj]) | ((gj == g) & done[gi]))
        idx = np.nonzero(ready)[0]
        v = np.zeros(len(rhos))
        for k, r in enumerate(rhos):
            ri = np.where(gi[idx] == g, r, rho[gi[idx]])
            rj = np.where(gj[idx] == g, r, rho[gj[idx]])
            v[k] = np.sum(vote_terms(E0[idx], ri, rj, tau))
        rho[g] = rhos[int(np.argmax(v))]
        done[g] = True
        order.append(g)
    return rho, order
