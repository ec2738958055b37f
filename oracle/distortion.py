"""Distortion interval search for the oracle (float64).  Test infrastructure
only.

Sec. 3.1 "Camera Assumptions" / "Distortion Estimation" (Eq. 1) and Appendix
"Distortion Estimation" ("Hierarchical search", "Multiple cameras"):

  * one-parameter division model: an observed (distorted) point x_d with
    radius r_d maps to x_u = x_d / (1 + alpha r_d^2); the principal point is
    the image centre;
  * a candidate alpha is scored on a set of image pairs by undistorting their
    keypoints, re-estimating each pair's fundamental matrix and averaging the
    epipolar error over all keypoint pairs of all those image pairs; the
    candidate with the lowest average wins (the first on ties);
  * hierarchical search: candidates spaced evenly over [alpha_min,
    alpha_max]; after each level the winner's two neighbours become the next
    level's interval; the last level's winner is the estimate;
  * several cameras: the same greedy "ready pair" order as the focal search;
    a pair with one image of an estimated camera undistorts that image with
    its known alpha.

Readings (the paper gives no numbers or normalisation): x_d = (pixel -
centre) / h with h = |centre| (the half diagonal, so r_d <= 1 inside the
image); points are homogeneous (x_u, y_u, 1); the fundamental matrix is the
normalised linear eight-point estimate (Hartley, "In defense of the
eight-point algorithm", 1997): each image's points of the pair are moved to
their centroid and scaled to an RMS distance of sqrt(2) (y = T x), F^ is the
eigenvector of the smallest eigenvalue of W = sum a a^T with a = y_2 (x) y_1,
projected to rank 2 (smallest singular value zeroed) and scaled to unit
Frobenius norm (F = T_2^T F^ T_1 in the undistorted coordinates); the
epipolar error of a keypoint pair is |y_2^T F^ y_1|, measured in the pair's
normalised frame of the candidate, so that a candidate cannot lower the error
by shrinking the coordinates (in the undistorted coordinates alpha > 0 shrinks
every point and with it the algebraic error: a few percent of outliers then
pull the search to alpha_max); candidates per level n = 32, levels 3,
interval [-0.5, 0.5]; at an end of the interval the missing neighbour is the
end candidate itself; image pairs with fewer than 8 keypoint pairs take no
part.
"""
import numpy as np


def normalised(kp_px, cx, cy):
    """x_d of pixel keypoints [Z,2] of images with centres (cx, cy) [Z]."""
    c = np.stack([np.asarray(cx, np.float64), np.asarray(cy, np.float64)], axis=-1)
    h = np.linalg.norm(c, axis=-1, keepdims=True)
    return (np.asarray(kp_px, np.float64) - c) / h


def undistort(xd, alpha):
    """Eq. 1: x_u = x_d / (1 + alpha r_d^2); alpha scalar or [Z]."""
    r2 = np.sum(xd * xd, axis=-1, keepdims=True)
    return xd / (1.0 + np.asarray(alpha, np.float64).reshape(-1, 1) * r2)


def homogeneous(x):
    return np.concatenate([x, np.ones(x.shape[:-1] + (1,))], axis=-1)


def hartley(x):
    """T moving homogeneous points [m,3] (w = 1) to their centroid and
    scaling them to an RMS distance of sqrt(2)."""
    c = x[:, :2].mean(axis=0)
    k = np.sqrt(2.0) / np.sqrt(np.mean(np.sum((x[:, :2] - c) ** 2, axis=1)))
    return np.array([[k, 0.0, -k * c[0]], [0.0, k, -k * c[1]], [0.0, 0.0, 1.0]])


def normalised_8pt(x1u, x2u):
    """(F^, y1, y2): the rank-2, unit-Frobenius eight-point estimate in the
    Hartley-normalised coordinates y = T x of homogeneous points [m,3]
    (r = y2^T F^ y1)."""
    y1, y2 = x1u @ hartley(x1u).T, x2u @ hartley(x2u).T
    a = np.einsum("mp,mq->mpq", y2, y1).reshape(-1, 9)
    w, V = np.linalg.eigh(a.T @ a)
    Fh = V[:, 0].reshape(3, 3)
    U, s, Vt = np.linalg.svd(Fh)
    Fh = U @ np.diag([s[0], s[1], 0.0]) @ Vt
    return Fh / np.linalg.norm(Fh), y1, y2


def fundamental_8pt(x1u, x2u):
    """The same estimate in the undistorted coordinates, F = T_2^T F^ T_1 at
    unit Frobenius norm (r = x2^T F x1)."""
    Fh, _, _ = normalised_8pt(x1u, x2u)
    F = hartley(x2u).T @ Fh @ hartley(x1u)
    return F / np.linalg.norm(F)


def error_sum(x1u, x2u):
    """Sum over the image pair's keypoint pairs of the epipolar error
    |y2^T F^ y1| in the pair's normalised frame."""
    Fh, y1, y2 = normalised_8pt(x1u, x2u)
    return float(np.sum(np.abs(np.einsum("mp,pq,mq->m", y2, Fh, y1))))


def pair_offsets(kp_img_pair, n_pairs):
    return np.concatenate([[0], np.cumsum(np.bincount(kp_img_pair, minlength=n_pairs))])


def average_error(xd1, xd2, off, pairs, alpha_i, alpha_j):
    """Mean epipolar error over all keypoint pairs of the listed image pairs,
    image i_n undistorted with alpha_i[q], image j_n with alpha_j[q]."""
    tot, cnt = 0.0, 0
    for q, n in enumerate(pairs):
        a, b = off[n], off[n + 1]
        x1u = homogeneous(undistort(xd1[a:b], alpha_i[q]))
        x2u = homogeneous(undistort(xd2[a:b], alpha_j[q]))
        tot += error_sum(x1u, x2u)
        cnt += b - a
    return tot / cnt


def level_candidates(lo, hi, n):
    return np.linspace(lo, hi, n)


def search(score, alpha_min, alpha_max, n_cand, n_levels):
    """Hierarchical interval search of the scalar function score(alpha).
    Returns (estimate, [candidates of each level], [scores of each level])."""
    lo, hi = alpha_min, alpha_max
    cands, scores = [], []
    best = lo
    for _ in range(n_levels):
        c = level_candidates(lo, hi, n_cand)
        s = np.array([score(a) for a in c])
        k = int(np.argmin(s))
        best = c[k]
        lo, hi = c[max(k - 1, 0)], c[min(k + 1, n_cand - 1)]
        cands.append(c)
        scores.append(s)
    return best, cands, scores


def search_groups(xd1, xd2, kp_img_pair, pair_i, pair_j, group, n_groups, alpha_min=-0.5, alpha_max=0.5,
                  n_cand=32, n_levels=3):
    """Greedy camera order of the appendix.  Returns (alpha [n_groups], NaN
    for cameras never ready, order of estimation)."""
    P = len(pair_i)
    off = pair_offsets(kp_img_pair, P)
    valid = np.diff(off) >= 8
    gi, gj = np.asarray(group)[pair_i], np.asarray(group)[pair_j]
    alpha = np.full(n_groups, np.nan)
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
        pairs = np.nonzero(ready)[0]

        def score(a):
            ai = np.where(gi[pairs] == g, a, alpha[gi[pairs]])
            aj = np.where(gj[pairs] == g, a, alpha[gj[pairs]])
            return average_error(xd1, xd2, off, pairs, ai, aj)

        alpha[g], _, _ = search(score, alpha_min, alpha_max, n_cand, n_levels)
        done[g] = True
        order.append(g)
    return alpha, order
