"""Pins of the oracle's global rotation (Eqs. 3-4, Appendix "Global Rotation",
Eqs. 10-14), global translation (Eqs. 5-6, Appendix "Multiple
Initializations") and Adam against closed forms, ground truth, invariances,
exact recovery and finite differences (no CUDA)."""
import json
import os

import numpy as np

from oracle import rotation as rot
from oracle import translation as trn
from oracle.adam import Adam
from oracle.so3 import angle_axis, rot_from_6d
from synthetic.scenes import gt_relative_poses
from tests._util import gt_params6, scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _fd(fun, p, h):
    g = np.zeros_like(p)
    for idx in np.ndindex(p.shape):
        a, b = p.copy(), p.copy()
        a[idx] += h
        b[idx] -= h
        g[idx] = (fun(a) - fun(b)) / (2 * h)
    return g


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


# ----------------------------------------------------------------- rotation

def test_rotation_loss_zero_at_ground_truth():
    sc = scene("c1", 0)
    Rij, _ = gt_relative_poses(sc)
    L, g = rot.loss_grad(gt_params6(sc), sc.pair_i, sc.pair_j, Rij)
    assert L < 1e-7   # arccos(1 - 1e-16) ~ 1.5e-8 per pair
    # the subgradient at d = 0 may pick either side of the kink; it stays bounded
    assert np.all(np.isfinite(g))


def test_rotation_loss_closed_form_single_pair():
    # R_i = I, R_ij = I, R_j a rotation by theta: L_R = theta
    for theta in [0.05, 0.4, 1.3, 3.0]:
        Rj = angle_axis([1.0, 2.0, -0.5], theta)
        p = np.stack([np.r_[1.0, 0, 0, 0, 1.0, 0], np.r_[Rj[:, 0], Rj[:, 1]]])
        L, _ = rot.loss_grad(p, np.array([0]), np.array([1]), np.eye(3)[None])
        assert abs(L - theta) < 1e-9


def test_rotation_gauge_invariance():
    sc = scene("c1", 1)
    Rij, _ = gt_relative_poses(sc, rot_noise_deg=2.0, seed=1)
    rng = np.random.default_rng(1)
    p = gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6))
    R = rot_from_6d(p)
    G = angle_axis([0.2, 0.9, -0.4], 1.1)
    RG = R @ G
    q = np.concatenate([RG[:, :, 0], RG[:, :, 1]], axis=1)
    La, _ = rot.loss_grad(p, sc.pair_i, sc.pair_j, Rij)
    Lb, _ = rot.loss_grad(q, sc.pair_i, sc.pair_j, Rij)
    assert abs(La - Lb) < 1e-12 * La


def test_rotation_gradient_central_differences():
    sc = scene("c1", 2)
    Rij, _ = gt_relative_poses(sc, rot_noise_deg=2.0, seed=2)
    rng = np.random.default_rng(2)
    p = gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6))
    L, g = rot.loss_grad(p, sc.pair_i, sc.pair_j, Rij)
    fd = _fd(lambda q: rot.loss_grad(q, sc.pair_i, sc.pair_j, Rij)[0], p, 1e-6)
    assert _rel(g, fd) < 1e-6


def test_martinec_init_exact_recovery_on_noise_free_rotations():
    sc = scene("c1", 3)
    Rij, _ = gt_relative_poses(sc)
    R0 = rot.martinec_init(sc.n_cams, sc.pair_i, sc.pair_j, Rij)
    assert np.allclose(np.linalg.det(R0), 1.0, atol=1e-10)
    # recovered up to the gauge R_i -> R_i G
    G = sc.R_gt[0].T @ R0[0]
    err = np.max(np.abs(R0 - sc.R_gt @ G))
    assert err < 1e-9
    p = np.concatenate([R0[:, :, 0], R0[:, :, 1]], axis=1)
    assert rot.loss_grad(p, sc.pair_i, sc.pair_j, Rij)[0] < 1e-6


def test_martinec_init_close_under_noise():
    sc = scene("c1", 4)
    Rij, _ = gt_relative_poses(sc, rot_noise_deg=1.0, seed=4)
    R0 = rot.martinec_init(sc.n_cams, sc.pair_i, sc.pair_j, Rij)
    # align with the best global rotation (Kabsch on the stacked matrices)
    M = np.einsum("nki,nkj->ij", sc.R_gt, R0)
    U, _, Vt = np.linalg.svd(M)
    G = U @ Vt
    ang = np.degrees(np.arccos(np.clip((np.einsum("nij,nij->n", sc.R_gt @ G, R0) - 1) / 2, -1, 1)))
    assert np.mean(ang) < 1.5


# -------------------------------------------------------------- translation

def _translation_inputs(sc, dir_noise_deg=0.0, seed=0):
    _, tij = gt_relative_poses(sc, dir_noise_deg=dir_noise_deg, seed=seed)
    return trn.targets(sc.R_gt, sc.pair_j, tij)


def test_translation_target_is_unit_centre_direction_at_ground_truth():
    sc = scene("c1", 0)
    tgt = _translation_inputs(sc)
    c = sc.centers_gt
    d = c[sc.pair_j] - c[sc.pair_i]
    np.testing.assert_allclose(tgt, d / np.linalg.norm(d, axis=1, keepdims=True), atol=1e-12)


def test_translation_loss_zero_at_ground_truth_and_invariances():
    sc = scene("c1", 1)
    tgt = _translation_inputs(sc)
    c = sc.centers_gt
    assert trn.loss_grad(c, sc.pair_i, sc.pair_j, tgt)[0] < 1e-12
    rng = np.random.default_rng(1)
    o = c + rng.normal(0, 0.3, size=c.shape)
    La = trn.loss_grad(o, sc.pair_i, sc.pair_j, tgt)[0]
    Lb = trn.loss_grad(4.2 * o + np.array([3.0, -1.0, 7.0]), sc.pair_i, sc.pair_j, tgt)[0]
    assert La > 1e-2 and abs(La - Lb) < 1e-12 * La
    # a negative scale is not a symmetry (the directions flip)
    assert trn.loss_grad(-o, sc.pair_i, sc.pair_j, tgt)[0] > 2 * La


def test_translation_gradient_central_differences():
    sc = scene("c1", 2)
    tgt = _translation_inputs(sc, dir_noise_deg=2.0, seed=2)
    rng = np.random.default_rng(2)
    o = sc.centers_gt + rng.normal(0, 0.3, size=(sc.n_cams, 3))
    _, g = trn.loss_grad(o, sc.pair_i, sc.pair_j, tgt)
    fd = _fd(lambda q: trn.loss_grad(q, sc.pair_i, sc.pair_j, tgt)[0], o, 1e-8)
    assert _rel(g, fd) < 1e-5


def test_translation_merge_picks_the_better_run_per_camera():
    sc = scene("c1", 3)
    tgt = _translation_inputs(sc)
    good = sc.centers_gt
    rng = np.random.default_rng(3)
    bad_a, bad_b = good.copy(), good.copy()
    bad_a[:5] = rng.normal(0, 3.0, size=(5, 3))     # run 0 wrong on cameras 0-4
    bad_b[10:14] = rng.normal(0, 3.0, size=(4, 3))  # run 1 wrong on cameras 10-13
    merged, best = trn.merge_runs(np.stack([bad_a, 2.0 * bad_b + 1.0]), sc.pair_i, sc.pair_j, tgt)
    assert np.all(best[:5] == 1) and np.all(best[10:14] == 0)
    ref = trn.normalise_run(good)
    np.testing.assert_allclose(trn.normalise_run(merged), ref, atol=0.5)
    # the merged centres have zero centroid... only up to the mixing of runs;
    # each run on its own is normalised exactly
    n0 = trn.normalise_run(bad_a)
    assert abs(np.mean(np.linalg.norm(n0, axis=1)) - 1.0) < 1e-12
    assert np.max(np.abs(n0.mean(axis=0))) < 1e-12


# --------------------------------------------------------------------- Adam

def test_adam_hand_computed_two_steps():
    with open(os.path.join(GOLDEN, "adam_two_steps.json")) as f:
        gold = json.load(f)
    opt = Adam((1,), lr=gold["lr"], beta1=gold["beta1"], beta2=gold["beta2"], eps=gold["eps"])
    x = np.array([gold["x0"]])
    for g, want in zip(gold["grads"], gold["x"]):
        x = opt.step(x, np.array([g]))
        assert abs(x[0] - want) < 1e-14
