"""End-to-end first-order solve for the oracle (float64).  Test infrastructure.

The order of the paper's pipeline after matching and intrinsics (Sec. 3,
Fig. "pipeline"; Appendix "Global Rotation", "Global Translation",
"Epipolar Adjustment", "Sparse Reconstruction"):
  1. rotation initialisation (Eqs. 10-14) from the relative rotations;
  2. Adam on the global rotation loss (Eqs. 3-4);
  3. relative translations re-estimated by grid search with the relative
     rotations recomputed from the global ones (Appendix "Relative
     Translation");
  4. m translation runs from random initialisations (Eqs. 5-6), merged per
     camera (Appendix "Multiple Initializations"), then a final run;
  5. epipolar adjustment: rounds of IRLS reweighting with a decreasing
     filtering threshold, each followed by Adam steps on the compact form
     (Eqs. 8-9);
  6. sparse reconstruction.
The paper gives no learning rates, iteration counts or thresholds; the ones
here are readings (the defaults of SolveOpts), shared with the C ABI's
fm_solve_opts.  Random initial centres come from a counter-based generator
(below) that the CUDA side implements from the same definition.
"""
from dataclasses import dataclass

import numpy as np

from . import epipolar as ep
from . import relpose as rp
from . import rotation as rot
from . import translation as trn
from . import triangulation as tri
from .adam import Adam
from .so3 import rot_from_6d


@dataclass
class SolveOpts:
    rot_iters: int = 2000
    rot_lr: float = 1e-3
    reestimate_rel_t: bool = True
    trn_runs: int = 4
    trn_iters: int = 2000
    trn_lr: float = 1e-2
    trn_final_iters: int = 1000
    seed: int = 0
    ea_rounds: int = 5
    ea_iters: int = 500
    ea_lr: float = 1e-4
    ea_tau0: float = 0.05
    ea_tau_min: float = 0.005
    ea_delta: float = 1e-5
    tri_max_err_px: float = 4.0
    tri_min_angle_deg: float = 2.0
    # each Adam loop runs in four equal phases with the learning rate scaled by
    # these factors (Adam's moments carry over between phases)
    lr_phases: tuple = (1.0, 0.3, 0.1, 0.03)


def hash_uniform(n, salt):
    """n values in [-1, 1): value k is fmix32(k * 0x9E3779B9 + salt) >> 8,
    scaled by 2^-23, minus 1 (a Weyl step then the MurmurHash3 32-bit
    finaliser; uint32 arithmetic)."""
    k = np.arange(n, dtype=np.uint64)
    z = (k * np.uint64(0x9E3779B9) + np.uint64(salt)) & np.uint64(0xFFFFFFFF)
    z = ((z ^ (z >> np.uint64(16))) * np.uint64(0x85EBCA6B)) & np.uint64(0xFFFFFFFF)
    z = ((z ^ (z >> np.uint64(13))) * np.uint64(0xC2B2AE35)) & np.uint64(0xFFFFFFFF)
    z = z ^ (z >> np.uint64(16))
    return (z >> np.uint64(8)).astype(np.float64) * (1.0 / 8388608.0) - 1.0


def _adam_loop(x, grad_fn, iters, lr, phases):
    opt = Adam(x.shape, lr=lr)
    per = max(iters // len(phases), 0)
    L = None
    for ph, f in enumerate(phases):
        opt.lr = lr * f
        n = per if ph < len(phases) - 1 else iters - per * (len(phases) - 1)
        for _ in range(n):
            L, g = grad_fn(x)
            x = opt.step(x, g)
    return x, L


def solve(n_cams, pair_i, pair_j, x1, x2, kp_img_pair, rel_R, rel_t, focal, kp_track=None,
          opts=SolveOpts()):
    """Returns dict(R [N,3,3], t [N,3], centres, points, point_valid, losses)."""
    P = len(pair_i)
    # 1-2. rotations
    R0 = rot.martinec_init(n_cams, pair_i, pair_j, rel_R)
    p6 = np.concatenate([R0[:, :, 0], R0[:, :, 1]], axis=1)
    p6, L_rot = _adam_loop(p6, lambda q: rot.loss_grad(q, pair_i, pair_j, rel_R), opts.rot_iters,
                           opts.rot_lr, opts.lr_phases)
    R = rot_from_6d(p6)
    # 3. relative translations
    if opts.reestimate_rel_t:
        off = np.zeros(P + 1, dtype=np.int64)
        np.cumsum(np.bincount(kp_img_pair, minlength=P), out=off[1:])
        rel_t = np.zeros((P, 3))
        for n in range(P):
            s = slice(off[n], off[n + 1])
            Rij = R[pair_j[n]] @ R[pair_i[n]].T
            if off[n + 1] > off[n]:
                rel_t[n], _ = rp.relative_translation(Rij, x1[s], x2[s])
            else:
                rel_t[n] = np.array([0.0, 0.0, 1.0])
    tgt = trn.targets(R, pair_j, rel_t)
    # 4. translation runs, merge, final run
    m = opts.trn_runs
    o_all = hash_uniform(m * n_cams * 3, opts.seed).reshape(m, n_cams, 3)
    runs = []
    for k in range(m):
        o, _ = _adam_loop(o_all[k], lambda q: trn.loss_grad(q, pair_i, pair_j, tgt), opts.trn_iters,
                          opts.trn_lr, opts.lr_phases)
        runs.append(o)
    merged, best = trn.merge_runs(np.stack(runs), pair_i, pair_j, tgt) if m > 1 else (trn.normalise_run(runs[0]), np.zeros(n_cams, int))
    o, L_trn = _adam_loop(merged, lambda q: trn.loss_grad(q, pair_i, pair_j, tgt), opts.trn_final_iters,
                          opts.trn_lr, opts.lr_phases)
    # 5. epipolar adjustment
    t = -np.einsum("nab,nb->na", R, o)
    params = np.concatenate([p6, t], axis=1)
    L_ea = None
    n_kept = len(kp_img_pair)
    for k in range(opts.ea_rounds):
        tau = max(opts.ea_tau0 * 0.5 ** k, opts.ea_tau_min)
        r = ep.residuals(ep.essential_matrices(params, pair_i, pair_j), x1, x2, kp_img_pair)
        w, keep = ep.irls_weights(r, tau, opts.ea_delta)
        n_kept = int(keep.sum())
        W = ep.build_W(x1, x2, kp_img_pair, P, weights=w)
        inv_z = 1.0 / max(n_kept, 1)
        params, L_ea = _adam_loop(params, lambda q: ep.compact_loss_grad(q, pair_i, pair_j, W, inv_z)[:2],
                                  opts.ea_iters, opts.ea_lr, opts.lr_phases)
    R = rot_from_6d(params[:, :6])
    t = params[:, 6:]
    out = dict(R=R, t=t, centres=-np.einsum("nba,nb->na", R, t), loss_rot=L_rot, loss_trn=L_trn,
               loss_ea=L_ea, n_kept=n_kept, rel_t=rel_t, best_run=best)
    # 6. points
    if kp_track is not None:
        T = int(np.max(kp_track)) + 1
        pts, valid, _ = tri.triangulate(R, t, pair_i, pair_j, kp_img_pair, x1, x2, kp_track, T, focal,
                                        opts.tri_max_err_px, opts.tri_min_angle_deg)
        out.update(points=pts, point_valid=valid)
    return out


def rotation_errors_deg(R_est, R_gt):
    """Per-camera angle of R_gt G - R_est after the best global alignment
    R_est ~ R_gt G (Kabsch on the stacked matrices)."""
    M = np.einsum("nki,nkj->ij", R_gt, R_est)
    U, _, Vt = np.linalg.svd(M)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
    G = U @ D @ Vt
    c = (np.einsum("nij,nij->n", R_gt @ G, R_est) - 1.0) / 2.0
    return np.degrees(np.arccos(np.clip(c, -1.0, 1.0)))


def centre_errors(c_est, c_gt):
    """Camera-centre errors after the best similarity alignment (Umeyama)."""
    mu_e, mu_g = c_est.mean(0), c_gt.mean(0)
    A, B = c_est - mu_e, c_gt - mu_g
    U, S, Vt = np.linalg.svd(B.T @ A)
    D = np.diag([1.0, 1.0, np.sign(np.linalg.det(U @ Vt))])
    Q = U @ D @ Vt
    s = np.trace(np.diag(S) @ D) / np.sum(A * A)
    aligned = s * A @ Q.T + mu_g
    return np.linalg.norm(aligned - c_gt, axis=1)
