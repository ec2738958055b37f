"""Helpers shared by the GPU parity tests: build the library, create problems
from seeded scenes, evaluate the oracle on exactly the same float32 inputs."""
import itertools

import numpy as np

from oracle import epipolar as ep

GAMMA = 2e-6   # |r| below which float32 and float64 may disagree on sign(r)


def f32(x):
    return np.asarray(x, dtype=np.float32).astype(np.float64)


def lib_ready():
    from paper_2505_04612_b300 import build as B
    B.build()


def make_problem(sc, device=True, rel_R=None, rel_t=None):
    lib_ready()
    from paper_2505_04612_b300.fastmap import problem_from_scene
    return problem_from_scene(sc, rel_R=rel_R, rel_t=rel_t, device=device)


def oracle_xs(sc):
    return ep.calibrated_pairs(sc.kp1_px, sc.kp2_px, sc.kp_img_pair, sc.pair_i, sc.pair_j,
                               f32(sc.focal), f32(sc.cx), f32(sc.cy))


def rel_err(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def ea_oracle(sc, params, loss, weights=None, inv_z=None, xs=None, sign_override=None):
    """Oracle loss/grad of the epipolar stage on the float32-rounded inputs the
    GPU sees.  sign_override: {pair index: sign} replacing sign(r) (L1)."""
    x1, x2 = xs if xs is not None else oracle_xs(sc)
    p = f32(params).reshape(-1, 9)
    w = None if weights is None else f32(weights)
    if sign_override:
        geo = ep.pair_geometry(p, sc.pair_i, sc.pair_j)
        r = ep.residuals(geo["E"], x1, x2, sc.kp_img_pair)
        s = np.sign(r)
        for m, v in sign_override.items():
            s[m] = v
        wt = np.ones_like(r) if w is None else w
        iz = 1.0 / max(len(r), 1) if inv_z is None else inv_z
        L = iz * np.sum(wt * np.abs(r))
        G = np.zeros((sc.n_pairs, 3, 3))
        np.add.at(G, sc.kp_img_pair, iz * (wt * s)[:, None, None] * np.einsum("ma,mb->mab", x2, x1))
        return L, ep.backward_E(G, geo, p.shape[0], sc.pair_i, sc.pair_j, p)
    L, g, _ = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, weights=w,
                                  loss=loss, inv_z=inv_z)
    return L, g


def ambiguous_pairs(sc, params, xs=None):
    x1, x2 = xs if xs is not None else oracle_xs(sc)
    p = f32(params).reshape(-1, 9)
    r = ep.residuals(ep.essential_matrices(p, sc.pair_i, sc.pair_j), x1, x2, sc.kp_img_pair)
    return np.nonzero(np.abs(r) < GAMMA)[0]


def l1_grad_matches(sc, params, g_gpu, tol, weights=None, inv_z=None, xs=None, max_amb=3):
    """sign(r) is decided in float32 on the GPU; pairs with |r| < GAMMA may
    take either sign (or 0).  The unique part (all other pairs) must match; the
    ambiguous ones must take one of the valid values.  Returns (ok, err, n_amb)
    or None when too many pairs are ambiguous to enumerate."""
    amb = ambiguous_pairs(sc, params, xs)
    if len(amb) > max_amb:
        return None
    best = np.inf
    for signs in itertools.product([-1.0, 0.0, 1.0], repeat=len(amb)):
        _, g = ea_oracle(sc, params, "l1", weights, inv_z, xs,
                         sign_override=dict(zip(amb.tolist(), signs)) if len(amb) else None)
        best = min(best, rel_err(g_gpu.reshape(g.shape), g))
    return best < tol, best, len(amb)


def l1_grad_within_bound(sc, params, g_gpu, tol, weights=None, inv_z=None, xs=None):
    """For scenes with too many sign-ambiguous pairs to enumerate: the GPU
    gradient is within tol (relative) of the oracle's plus, for each pair with
    |r| < GAMMA, the largest change its sign can make, 2 w_m inv_z
    |d r_m / d params|.  Returns (ok, err, bound, n_ambiguous)."""
    x1, x2 = xs if xs is not None else oracle_xs(sc)
    p = f32(params).reshape(-1, 9)
    _, go = ea_oracle(sc, params, "l1", weights, inv_z, xs)
    amb = ambiguous_pairs(sc, params, xs)
    iz = 1.0 / max(sc.n_kp, 1) if inv_z is None else inv_z
    geo = ep.pair_geometry(p, sc.pair_i, sc.pair_j)
    bound = 0.0
    for m in amb:
        wm = 1.0 if weights is None else float(weights[m])
        Gm = np.zeros((sc.n_pairs, 3, 3))
        Gm[sc.kp_img_pair[m]] = wm * iz * np.outer(x2[m], x1[m])
        bound += 2.0 * np.linalg.norm(ep.backward_E(Gm, geo, p.shape[0], sc.pair_i, sc.pair_j, p))
    err = np.linalg.norm(np.asarray(g_gpu, np.float64).reshape(go.shape) - go)
    return err <= tol * np.linalg.norm(go) + bound, err, bound, len(amb)
