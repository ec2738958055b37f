"""Distortion interval search on the GPU (fm_distortion_search,
fm_distortion_pair_errors, fm_set_distortion; Sec. 3.1 Eq. 1, Appendix
"Distortion Estimation") against the FP64 oracle (oracle/distortion: float64
eigh eight-point, SVD rank-2 projection, the same hierarchical levels and
camera order) on the same float32 pixels."""
import dataclasses

import numpy as np
import pytest

from oracle import distortion as D
from synthetic.scenes import gt_relative_poses, scene_c2
from tests import _gpu as G

pytestmark = pytest.mark.gpu

N_CAND, N_LEVELS = 32, 3


def _resolution():
    step = 1.0 / (N_CAND - 1)
    for _ in range(N_LEVELS - 1):
        step = 2 * step / (N_CAND - 1)
    return step


def _scene(alpha, groups=1, sigma=0.0, seed=5, n_cams=40):
    return scene_c2(seed=seed, n_cams=n_cams, n_points=5000, sigma_px=sigma, outlier_frac=0.0,
                    focal_groups=groups, alpha=alpha)


def _xd(sc):
    ci = sc.pair_i[sc.kp_img_pair]
    cj = sc.pair_j[sc.kp_img_pair]
    return (D.normalised(G.f32(sc.kp1_px), sc.cx[ci], sc.cy[ci]),
            D.normalised(G.f32(sc.kp2_px), sc.cx[cj], sc.cy[cj]))


def _oracle_pair_errors(sc, cands):
    """Oracle error sums [P, K] and the relative eigen-gap (lambda2 - lambda1)
    / lambda9 of each normalised moment matrix W (its conditioning)."""
    xd1, xd2 = _xd(sc)
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    out = np.zeros((sc.n_pairs, len(cands)))
    gap = np.ones((sc.n_pairs, len(cands)))
    for n in range(sc.n_pairs):
        a, b = off[n], off[n + 1]
        if b - a < 8:
            continue
        for k, al in enumerate(cands):
            x1 = D.homogeneous(D.undistort(xd1[a:b], al))
            x2 = D.homogeneous(D.undistort(xd2[a:b], al))
            out[n, k] = D.error_sum(x1, x2)
            T1, T2 = D.hartley(x1), D.hartley(x2)
            A = np.einsum("mp,mq->mpq", x2 @ T2.T, x1 @ T1.T).reshape(-1, 9)
            w = np.linalg.eigvalsh(A.T @ A)
            gap[n, k] = (w[1] - w[0]) / w[-1]
    return out, gap


def _oracle_score(sc, a):
    xd1, xd2 = _xd(sc)
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    pairs = np.nonzero(np.diff(off) >= 8)[0]
    return D.average_error(xd1, xd2, off, pairs, np.full(len(pairs), a), np.full(len(pairs), a))


@pytest.mark.parametrize("sigma,dense", [(0.0, False), (1.0, False), (1.0, True)])
def test_pair_errors_match_the_oracle(sigma, dense):
    """Every (image pair, candidate) score of one level, element by element.
    The tolerance follows the conditioning of the eigenvector: float32
    moments perturb W by about eps32 sqrt(m) of its largest eigenvalue, which
    turns F^ by theta ~ eps32 sqrt(m) / gap (first-order perturbation; gap =
    (lambda2 - lambda1) / lambda9), and moves each of the m residuals by about
    theta, so a sum may differ by 5e-4 of itself plus 10 m theta (the factor
    10 is a margin over the ~0.75 seen in a float32 emulation of the kernel).
    On well-separated pairs that is ~1e-3 relative; on near-degenerate ones
    (exactly 8-9 keypoint pairs, or two nearly equal smallest eigenvalues) no
    float32 result is unique and the bound opens up.  Sums near the float32
    rounding of the residuals (the noise-free truth) are compared in absolute
    terms."""
    if dense:   # image pairs of more than 1,024 keypoint pairs: one CTA of warps each
        sc = scene_c2(seed=2, n_cams=10, n_points=40000, sigma_px=sigma, outlier_frac=0.0, alpha=-0.2)
    else:
        sc = _scene(-0.2, sigma=sigma)
    cands = np.linspace(-0.5, 0.5, N_CAND).astype(np.float32)
    with G.make_problem(sc) as pr:
        err = pr.distortion_pair_errors(cands).astype(np.float64)
    ref, gap = _oracle_pair_errors(sc, cands.astype(np.float64))
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    if dense:
        assert np.sum(np.diff(off) > 1024) >= 3 and np.sum((np.diff(off) >= 8) & (np.diff(off) <= 1024)) >= 3
    m = np.broadcast_to(np.diff(off)[:, None], err.shape)
    far = ref > 1e-4 * m          # mean |r| above 1e-4: well above float32 rounding
    rel = np.abs(err - ref) / np.maximum(ref, 1e-30)
    theta = 2.0 ** -24 * np.sqrt(m) / gap
    tol = 5e-4 * ref + 10 * m * theta
    assert far.sum() > 0.8 * far.size
    bad = far & (np.abs(err - ref) > tol)
    assert not bad.any(), (np.argwhere(bad)[:5], rel[bad][:5], (tol / ref)[bad][:5])
    assert np.median(rel[far]) < 1e-4, np.median(rel[far])
    assert np.all(np.abs(err - ref)[~far] <= 2e-4 * m[~far])


def test_pair_errors_of_thin_image_pairs_are_zero():
    sc = _scene(-0.2)
    keep = np.ones(sc.n_kp, bool)
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    thin = [0, 7, sc.n_pairs - 1]
    for p in thin:
        keep[off[p] + 5:off[p + 1]] = False
    from tests.test_gpu_epipolar import _subscene
    sub = _subscene(sc, sc.pair_i, sc.pair_j, sc.kp_img_pair[keep], np.nonzero(keep)[0])
    with G.make_problem(sub) as pr:
        err = pr.distortion_pair_errors(np.array([-0.2, 0.0], np.float32))
    assert np.all(err[thin] == 0.0)
    assert np.all(np.delete(err, thin, axis=0)[:, 1] > 0.0)


@pytest.mark.parametrize("alpha,sigma", [(-0.2, 0.0), (-0.3, 1.0), (0.1, 1.0)])
def test_one_camera_matches_the_oracle(alpha, sigma):
    """The GPU's estimate scores as well as the oracle's under the oracle's own
    average error (the flat bottom of the noisy landscape may let float32 and
    float64 pick neighbouring candidates) and lies near it and the truth."""
    sc = _scene(alpha, sigma=sigma)
    xd1, xd2 = _xd(sc)
    est_o, _ = D.search_groups(xd1, xd2, sc.kp_img_pair, sc.pair_i, sc.pair_j, np.zeros(sc.n_cams, int), 1)
    with G.make_problem(sc) as pr:
        est, n_est = pr.distortion_search(n_cand=N_CAND, n_levels=N_LEVELS)
    assert n_est == 1 and np.all(est == est[0])
    tol = 2 * _resolution() if sigma == 0.0 else 0.01
    assert abs(est[0] - est_o[0]) <= tol, (est[0], est_o[0])
    assert abs(est[0] - alpha) <= tol
    if sigma > 0.0:
        s_g, s_o = _oracle_score(sc, float(est[0])), _oracle_score(sc, est_o[0])
        assert s_g <= s_o * (1 + 2e-3), (s_g, s_o)


def test_cameras_match_the_oracle():
    alphas = np.array([-0.3, 0.05, -0.1])
    sc = _scene(alphas, groups=3)
    g = sc.meta["focal_group"]
    xd1, xd2 = _xd(sc)
    est_o, order = D.search_groups(xd1, xd2, sc.kp_img_pair, sc.pair_i, sc.pair_j, g, 3)
    with G.make_problem(sc) as pr:
        est, n_est = pr.distortion_search(group=g, n_groups=3)
    assert n_est == 3
    for q in range(3):
        aq = est[g == q]
        assert np.all(aq == aq[0])
        assert abs(aq[0] - est_o[q]) <= 2 * _resolution(), (q, aq[0], est_o[q])
    np.testing.assert_allclose([est[g == q][0] for q in range(3)], alphas, atol=2e-3)


def test_set_distortion_matches_a_problem_built_from_undistorted_pixels():
    """Keypoints undistorted in place against pixels undistorted by the oracle
    before the problem is built: the epipolar loss and gradient agree."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    from tests._util import perturbed_params_ea
    alpha = -0.25
    sc = _scene(alpha, sigma=1.0)
    ci = sc.pair_i[sc.kp_img_pair]
    cj = sc.pair_j[sc.kp_img_pair]
    h = np.hypot(sc.cx[0], sc.cy[0])
    c1 = np.stack([sc.cx[ci], sc.cy[ci]], 1)
    c2 = np.stack([sc.cx[cj], sc.cy[cj]], 1)
    xd1, xd2 = _xd(sc)
    und = dataclasses.replace(sc, kp1_px=(c1 + h * D.undistort(xd1, alpha)).astype(np.float32),
                              kp2_px=(c2 + h * D.undistort(xd2, alpha)).astype(np.float32))
    params = torch.from_numpy(np.asarray(perturbed_params_ea(sc, 3), np.float32).reshape(-1)).cuda()
    with G.make_problem(und) as ref:
        L_ref, g_ref = ref.loss_grad(F.FM_STAGE_EPIPOLAR, params)
        g_ref = g_ref.cpu().numpy().astype(np.float64)
    with G.make_problem(sc) as pr:
        L0, _ = pr.loss_grad(F.FM_STAGE_EPIPOLAR, params)
        pr.set_distortion(np.full(sc.n_cams, alpha, np.float32))
        L1, g1 = pr.loss_grad(F.FM_STAGE_EPIPOLAR, params)
    assert abs(L0 - L_ref) > 1e-2 * abs(L_ref)
    assert abs(L1 - L_ref) <= 1e-5 * abs(L_ref), (L1, L_ref)
    assert G.rel_err(g1.cpu().numpy(), g_ref) < 1e-4


def test_invalid_arguments_and_points_without_an_undistortion():
    from paper_2505_04612_b300.fastmap import FastMapError
    sc = _scene(0.0, n_cams=12)
    with G.make_problem(sc) as pr:
        for kw in [dict(n_cand=1), dict(n_cand=33), dict(n_levels=0), dict(alpha_min=0.5, alpha_max=0.5),
                   dict(group=np.full(sc.n_cams, 2, np.int32), n_groups=2)]:
            with pytest.raises(FastMapError):
                pr.distortion_search(**kw)
        with pytest.raises(FastMapError):
            pr.distortion_pair_errors(np.zeros(33, np.float32))
        # corners of the image have r_d = 1: 1 + alpha r^2 <= 0 for alpha <= -1
        with pytest.raises(FastMapError):
            pr.set_distortion(np.full(sc.n_cams, -3.0, np.float32))


def test_distortion_then_focal_then_relative_poses():
    """End to end from distorted pixels with a wrong focal length: distortion
    search, undistortion, focal search, recalibration, relative poses."""
    sc = _scene(-0.25)
    f_true = sc.focal[0]
    wrong = dataclasses.replace(sc, focal=np.full(sc.n_cams, 700.0))
    with G.make_problem(wrong) as pr:
        alpha, _ = pr.distortion_search()
        pr.set_distortion(alpha)
        focal, _ = pr.focal_search()
        pr.set_focal(focal)
        n = pr.relative_poses()
        R, _ = pr.get_rel_poses()
    assert abs(alpha[0] + 0.25) <= 2 * _resolution()
    assert abs(np.log(focal[0] / f_true)) < 0.005
    Rg, _ = gt_relative_poses(sc)
    M = np.transpose(R.astype(np.float64), (0, 2, 1)) @ Rg
    ang = np.degrees(np.arccos(np.clip(0.5 * (np.trace(M, axis1=1, axis2=2) - 1.0), -1.0, 1.0)))
    assert n == sc.n_pairs
    assert np.median(ang) < 0.1, np.median(ang)
