"""Relative poses from the keypoints on the GPU (fm_relative_poses) against
the ground truth on noise-free scenes and against the FP64 oracle
(oracle/relpose.relative_pose: eigh of W_n, SVD projection, four
decompositions, cheirality) on noisy ones, plus the degenerate image pairs
and fm_solve without given relative rotations."""
import numpy as np
import pytest

from oracle import relpose as rp
from oracle.solve import rotation_errors_deg
from synthetic.scenes import gt_relative_poses, make_scene
from tests import _gpu as G
from tests._util import clean_scene

pytestmark = pytest.mark.gpu


def _angle_deg(Ra, Rb):
    """Angle of Ra^T Rb by atan2 (arccos of the trace cannot resolve the
    small angles of float32 matrices)."""
    M = np.transpose(Ra, (0, 2, 1)) @ Rb
    v = np.stack([M[:, 2, 1] - M[:, 1, 2], M[:, 0, 2] - M[:, 2, 0], M[:, 1, 0] - M[:, 0, 1]], 1)
    return np.degrees(np.arctan2(0.5 * np.linalg.norm(v, axis=1), 0.5 * (np.trace(M, axis1=1, axis2=2) - 1.0)))


def _dir_deg(ta, tb):
    return np.degrees(np.arctan2(np.linalg.norm(np.cross(ta, tb), axis=1), np.sum(ta * tb, 1)))


def _gpu_relposes(sc, irls=0):
    with G.make_problem(sc) as pr:
        n = pr.relative_poses(irls_iters=irls, delta=1e-5)
        R, t = pr.get_rel_poses()
    return n, R.astype(np.float64), t.astype(np.float64)


@pytest.mark.parametrize("seed", [0, 3])
def test_noise_free_scenes_give_the_true_relative_poses(seed):
    sc = clean_scene(seed)
    n, R, t = _gpu_relposes(sc)
    Rg, tg = gt_relative_poses(sc)
    assert n == sc.n_pairs
    # float32 W_n and Jacobi: ~1e-4 rad at worst on these narrow-view pairs
    assert np.max(_angle_deg(R, Rg)) < 0.01
    assert np.max(_dir_deg(t, tg)) < 0.05


@pytest.mark.parametrize("irls", [0, 2])
def test_noisy_scenes_match_the_oracle(irls):
    """c1 geometry with 0.5 px noise and no outliers: the GPU's float32 Jacobi
    eight-point estimate against the oracle's float64 eigh on the same pairs."""
    sc = make_scene("c1", 4, outlier_frac=0.0)
    n, R, t = _gpu_relposes(sc, irls)
    x1, x2 = G.oracle_xs(sc)
    off = sc.seg_off()
    Ro = np.zeros_like(R)
    to = np.zeros_like(t)
    for p in range(sc.n_pairs):
        s = slice(off[p], off[p + 1])
        Ro[p], to[p] = rp.relative_pose(x1[s], x2[s], irls_iters=irls, delta=1e-5)
    assert n == sc.n_pairs
    dR, dt = _angle_deg(R, Ro), _dir_deg(t, to)
    assert np.median(dR) < 0.005 and np.max(dR) < 0.1, (np.median(dR), np.max(dR))
    assert np.median(dt) < 0.05 and np.max(dt) < 1.0, (np.median(dt), np.max(dt))
    # (the linear estimate itself is degrees off the truth on c1's narrow
    # views: the oracle shares that, it is the method's, not the kernel's)


def test_image_pairs_with_fewer_than_eight_pairs():
    sc = clean_scene(1)
    keep = np.ones(sc.n_kp, bool)
    off = sc.seg_off()
    thin = [0, 5, sc.n_pairs - 1]
    for p in thin:   # leave 5 keypoint pairs in these image pairs
        keep[off[p] + 5:off[p + 1]] = False
    from tests.test_gpu_epipolar import _subscene
    sub = _subscene(sc, sc.pair_i, sc.pair_j, sc.kp_img_pair[keep], np.nonzero(keep)[0])
    n, R, t = _gpu_relposes(sub)
    assert n == sc.n_pairs - len(thin)
    for p in thin:
        np.testing.assert_array_equal(R[p], np.eye(3))
        np.testing.assert_array_equal(t[p], np.zeros(3))
    Rg, _ = gt_relative_poses(sc)
    others = np.setdiff1d(np.arange(sc.n_pairs), thin)
    assert np.max(_angle_deg(R[others], Rg[others])) < 0.01


def test_solve_estimates_relative_poses_when_none_are_given():
    """fm_solve on a noise-free scene without rel_R: the relative poses come
    from the keypoints and the solve recovers the cameras."""
    sc = clean_scene(2)
    with G.make_problem(sc) as pr:
        out = pr.solve(rot_iters=400, trn_iters=400, trn_final_iters=200, ea_rounds=2, ea_iters=200)
    ok = out["cam_valid"]
    err = rotation_errors_deg(out["R"].astype(np.float64)[ok], sc.R_gt[ok])
    assert np.mean(err) < 0.05, np.mean(err)
