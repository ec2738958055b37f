"""Global translation for the oracle (float64).  Test infrastructure only.

* target direction  o^{i->j} = -R_j^T t^{i->j}                          (Eq. 5)
* loss  L_t = 1/|P| sum || (o_j - o_i)/||o_j - o_i||_2 - o^{i->j} ||_1    (Eq. 6)
* multiple random initialisations merged per camera (Appendix "Multiple
  Initializations"): each run is moved to zero centroid and scaled to unit
  mean norm, and every camera takes the run with the lowest mean loss over
  the image pairs it belongs to.
"""
import numpy as np


def targets(R, pair_j, rel_t):
    """o^{i->j} = -R_j^T t^{i->j} for every image pair, [P,3] (Eq. 5)."""
    R = np.asarray(R, np.float64)
    return -np.einsum("pba,pb->pa", R[pair_j], np.asarray(rel_t, np.float64))


def pair_terms(o, pair_i, pair_j, tgt):
    """|| u_ij - o^{i->j} ||_1 per image pair with u_ij = (o_j - o_i)/|o_j - o_i|."""
    d = o[pair_j] - o[pair_i]
    n = np.linalg.norm(d, axis=1, keepdims=True)
    u = d / np.where(n > 1e-12, n, 1.0)
    return np.sum(np.abs(u - tgt), axis=1)


def loss_grad(o, pair_i, pair_j, tgt):
    """L_t and dL_t/do [N,3].  sign(0) = 0; a pair with |o_j - o_i| <= 1e-12
    contributes a zero gradient."""
    o = np.asarray(o, np.float64)
    P = len(pair_i)
    d = o[pair_j] - o[pair_i]
    n = np.linalg.norm(d, axis=1, keepdims=True)
    ok = n[:, 0] > 1e-12
    u = d / np.where(n > 1e-12, n, 1.0)
    e = u - tgt
    L = np.sum(np.abs(e)) / P
    gu = np.sign(e) / P
    gd = (gu - u * np.sum(u * gu, axis=1, keepdims=True)) / np.where(n > 1e-12, n, 1.0)
    gd[~ok] = 0.0
    g = np.zeros_like(o)
    np.add.at(g, pair_j, gd)
    np.add.at(g, pair_i, -gd)
    return L, g


def normalise_run(o):
    """Zero centroid, unit mean norm (the alignment of Appendix "Multiple
    Initializations"; the rotations are shared so no rotation is needed)."""
    o = np.asarray(o, np.float64)
    c = o - o.mean(axis=0, keepdims=True)
    return c / np.mean(np.linalg.norm(c, axis=1))


def camera_mean_loss(o, pair_i, pair_j, tgt, n_cams):
    terms = pair_terms(o, pair_i, pair_j, tgt)
    s = np.zeros(n_cams)
    c = np.zeros(n_cams)
    np.add.at(s, pair_i, terms)
    np.add.at(s, pair_j, terms)
    np.add.at(c, pair_i, 1.0)
    np.add.at(c, pair_j, 1.0)
    return s / np.maximum(c, 1.0)


def merge_runs(runs, pair_i, pair_j, tgt):
    """runs [m,N,3] -> merged [N,3]: normalise each run, then per camera take
    the run with the lowest mean incident loss (lowest index on ties)."""
    runs = np.asarray(runs, np.float64)
    m, n, _ = runs.shape
    normed = np.stack([normalise_run(runs[k]) for k in range(m)])
    scores = np.stack([camera_mean_loss(normed[k], pair_i, pair_j, tgt, n) for k in range(m)])
    best = np.argmin(scores, axis=0)
    return normed[best, np.arange(n)], best
