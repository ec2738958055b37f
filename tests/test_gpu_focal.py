"""Focal length interval search on the GPU (fm_focal_search; Sec. 3.1 Eq.
focal-vote, Appendix "Focal Length Estimation") against the FP64 oracle
(oracle/focal_search: float64 eigh eight-point E0, SVD singular-value ratio,
the same greedy group order) on the same float32 keypoints, and the
recalibration of a problem at new focal lengths (fm_set_focal)."""
import dataclasses

import numpy as np
import pytest

from oracle import epipolar as ep
from oracle import focal_search as fs
from synthetic.scenes import gt_relative_poses, scene_c2
from tests import _gpu as G

pytestmark = pytest.mark.gpu

RHO_MIN, RHO_MAX, N_CAND, TAU = 1.0 / 3.0, 3.0, 1024, 0.01
STEP = np.log(RHO_MAX / RHO_MIN) / (N_CAND - 1)


def _scene(groups, sigma=0.0, seed=5, n_cams=40):
    return scene_c2(seed=seed, n_cams=n_cams, n_points=5000, sigma_px=sigma, outlier_frac=0.0,
                    focal_groups=groups)


def _at(sc, f0):
    """The same scene, calibrated at the focal lengths f0 (scalar or [N])."""
    return dataclasses.replace(sc, focal=np.broadcast_to(np.asarray(f0, np.float64), (sc.n_cams,)).copy())


def _oracle_e0(sc, f0):
    x1, x2 = ep.calibrated_pairs(sc.kp1_px, sc.kp2_px, sc.kp_img_pair, sc.pair_i, sc.pair_j,
                                 G.f32(np.full(sc.n_cams, f0)), G.f32(sc.cx), G.f32(sc.cy))
    return fs.initial_essentials(x1, x2, sc.kp_img_pair, sc.n_pairs)


def _index(rho):
    return int(np.round(np.log(rho / RHO_MIN) / STEP))


@pytest.mark.parametrize("f0", [450.0, 900.0])
def test_shared_focal_matches_the_oracle_on_noise_free_scenes(f0):
    sc = _scene(1)
    E0, valid = _oracle_e0(sc, f0)
    rhos = fs.candidates(RHO_MIN, RHO_MAX, N_CAND)
    k_o, _ = fs.search_shared(E0, valid, rhos, TAU)
    with G.make_problem(_at(sc, f0)) as pr:
        focal, n_est = pr.focal_search(rho_min=RHO_MIN, rho_max=RHO_MAX, n_cand=N_CAND, tau=TAU)
    assert n_est == 1
    assert np.all(focal == focal[0])
    assert abs(_index(focal[0] / np.float32(f0)) - k_o) <= 1
    assert abs(np.log(focal[0] / sc.focal[0])) <= 1.5 * STEP


def test_noisy_shared_focal_is_an_oracle_optimum():
    """1 px noise: the vote landscape is flat near its top, so the float32 GPU
    and the float64 oracle may pick neighbouring candidates; the GPU's choice
    must score within 2 % of the oracle's best under the oracle's own vote,
    and lie within a few grid steps of it."""
    sc = _scene(1, sigma=1.0)
    f0 = 700.0
    E0, valid = _oracle_e0(sc, f0)
    rhos = fs.candidates(RHO_MIN, RHO_MAX, N_CAND)
    k_o, v = fs.search_shared(E0, valid, rhos, TAU)
    with G.make_problem(_at(sc, f0)) as pr:
        focal, n_est = pr.focal_search(rho_min=RHO_MIN, rho_max=RHO_MAX, n_cand=N_CAND, tau=TAU)
    k_g = _index(focal[0] / np.float32(f0))
    assert n_est == 1
    assert v[k_g] >= 0.98 * v[k_o], (k_g, k_o, v[k_g], v[k_o])
    assert abs(k_g - k_o) <= 4


@pytest.mark.parametrize("sigma", [0.0, 1.0])
def test_groups_match_the_oracle(sigma):
    """Three blocks of images along the trajectory, each with its own focal
    length, estimated in the greedy ready-pair order."""
    sc = _scene(3, sigma=sigma)
    g = sc.meta["focal_group"]
    f0 = 700.0
    E0, valid = _oracle_e0(sc, f0)
    rhos = fs.candidates(RHO_MIN, RHO_MAX, N_CAND)
    rho_o, order = fs.search_groups(E0, valid, sc.pair_i, sc.pair_j, g, 3, rhos, TAU)
    assert sorted(order) == [0, 1, 2]
    with G.make_problem(_at(sc, f0)) as pr:
        focal, n_est = pr.focal_search(group=g, n_groups=3, rho_min=RHO_MIN, rho_max=RHO_MAX, n_cand=N_CAND,
                                       tau=TAU)
    assert n_est == 3
    tol = 1 if sigma == 0.0 else 4
    for q in range(3):
        fq = focal[g == q]
        assert np.all(fq == fq[0])
        assert abs(_index(fq[0] / np.float32(f0)) - _index(rho_o[q])) <= tol, (q, fq[0], rho_o[q] * f0)
        f_true = sc.focal[g == q][0]
        assert abs(np.log(fq[0] / f_true)) <= (2 if sigma == 0.0 else 6) * STEP


def test_group_without_images_and_groups_never_ready():
    """An id with no image is never estimated; with a group per image no image
    pair starts ready, so nothing is estimated and focal_out keeps f0."""
    sc = _scene(1, n_cams=24)
    f0 = 700.0
    with G.make_problem(_at(sc, f0)) as pr:
        focal, n_est = pr.focal_search(group=np.zeros(sc.n_cams, np.int32), n_groups=2, n_cand=N_CAND)
        assert n_est == 1
        assert abs(np.log(focal[0] / sc.focal[0])) <= 1.5 * STEP
        focal, n_est = pr.focal_search(group=np.arange(sc.n_cams, dtype=np.int32), n_groups=sc.n_cams,
                                       n_cand=N_CAND)
        assert n_est == 0
        np.testing.assert_array_equal(focal, np.float32(f0))


def test_chain_of_single_image_groups_matches_the_oracle():
    """The first half of the images share one focal length, every later image
    is its own group: the order grows outward from the shared block, each
    image scored on its pairs to images already estimated."""
    sc = _scene(1, n_cams=24)
    N = sc.n_cams
    g = np.where(np.arange(N) < N // 2, 0, np.arange(N) - N // 2 + 1).astype(np.int32)
    n_groups = N - N // 2 + 1
    f0 = 700.0
    E0, valid = _oracle_e0(sc, f0)
    rhos = fs.candidates(RHO_MIN, RHO_MAX, N_CAND)
    rho_o, order = fs.search_groups(E0, valid, sc.pair_i, sc.pair_j, g, n_groups, rhos, TAU)
    with G.make_problem(_at(sc, f0)) as pr:
        focal, n_est = pr.focal_search(group=g, n_groups=n_groups, n_cand=N_CAND)
    assert n_est == len(order) == np.sum(np.isfinite(rho_o))
    for q in range(n_groups):
        if np.isfinite(rho_o[q]):
            assert abs(_index(focal[g == q][0] / np.float32(f0)) - _index(rho_o[q])) <= 1, q


def test_invalid_arguments_are_rejected():
    from paper_2505_04612_b300.fastmap import FastMapError
    sc = _scene(1, n_cams=12)
    with G.make_problem(sc) as pr:
        for kw in [dict(n_cand=1), dict(rho_min=0.0), dict(rho_min=2.0, rho_max=1.0), dict(tau=0.0),
                   dict(group=np.full(sc.n_cams, 3, np.int32), n_groups=2), dict(n_groups=2)]:
            with pytest.raises(FastMapError):
                pr.focal_search(**kw)
        with pytest.raises(FastMapError):
            pr.set_focal(np.zeros(sc.n_cams, np.float32))


def test_set_focal_matches_a_problem_built_at_those_focal_lengths():
    """Keypoints calibrated at f0 and rescaled by f0 / f against keypoints
    calibrated at f directly: the epipolar loss and gradient at the true
    poses agree to float32 rounding."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    from tests._util import perturbed_params_ea
    sc = _scene(1, sigma=1.0)
    params = torch.from_numpy(np.asarray(perturbed_params_ea(sc, 3), np.float32).reshape(-1)).cuda()
    with G.make_problem(sc) as ref:
        L_ref, g_ref = ref.loss_grad(F.FM_STAGE_EPIPOLAR, params)
        g_ref = g_ref.cpu().numpy().astype(np.float64)
    with G.make_problem(_at(sc, 700.0)) as pr:
        L0, _ = pr.loss_grad(F.FM_STAGE_EPIPOLAR, params)
        pr.set_focal(sc.focal.astype(np.float32))
        L1, g1 = pr.loss_grad(F.FM_STAGE_EPIPOLAR, params)
    assert abs(L0 - L_ref) > 1e-2 * abs(L_ref)   # the calibration really changed
    assert abs(L1 - L_ref) <= 1e-5 * abs(L_ref), (L1, L_ref)
    assert G.rel_err(g1.cpu().numpy(), g_ref) < 1e-4


def test_search_then_recalibrate_gives_the_relative_poses():
    """End to end on a noise-free scene with a wrong initial focal length:
    interval search, recalibration, relative poses from the keypoints."""
    sc = _scene(1)
    with G.make_problem(_at(sc, 800.0)) as pr:
        focal, _ = pr.focal_search(n_cand=N_CAND)
        pr.set_focal(focal)
        n = pr.relative_poses()
        R, _ = pr.get_rel_poses()
    Rg, _ = gt_relative_poses(sc)
    M = np.transpose(R.astype(np.float64), (0, 2, 1)) @ Rg
    ang = np.degrees(np.arccos(np.clip(0.5 * (np.trace(M, axis1=1, axis2=2) - 1.0), -1.0, 1.0)))
    assert n == sc.n_pairs
    assert np.median(ang) < 0.1, np.median(ang)
