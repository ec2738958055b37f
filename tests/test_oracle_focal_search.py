"""Pins of the oracle's focal length interval search (Sec. 3.1, Eq.
focal-vote; Appendix "Focal Length Estimation" with the multi-camera order of
"Distortion Estimation"): the essential-matrix characterisation at the true
focal length, invariance to the two-view matrix's scale and sign, recovery on
noise-free scenes for one shared focal length and for groups (no CUDA)."""
import numpy as np
import pytest

from oracle import epipolar as ep
from oracle import focal_search as fs
from synthetic.scenes import scene_c2


def _scene(groups, seed=5, sigma=0.0, outliers=0.0):
    return scene_c2(seed=seed, n_cams=40, n_points=5000, sigma_px=sigma, outlier_frac=outliers,
                    focal_groups=groups)


def _e0(sc, f0):
    x1, x2 = ep.calibrated_pairs(sc.kp1_px, sc.kp2_px, sc.kp_img_pair, sc.pair_i, sc.pair_j,
                                 np.full(sc.n_cams, f0), sc.cx, sc.cy)
    return fs.initial_essentials(x1, x2, sc.kp_img_pair, sc.n_pairs)


def test_true_focal_makes_every_matrix_essential():
    """Noise-free keypoints: at rho = f/f0 every valid pair's D E0 D has equal
    leading singular values, so each vote term is exp(0) = 1 and the score is
    the number of valid pairs; a wrong candidate scores less."""
    sc = _scene(1)
    f0 = 700.0
    E0, valid = _e0(sc, f0)
    rho = sc.focal[0] / f0
    terms = fs.vote_terms(E0[valid], rho, rho, 0.01)
    # the pixels are stored in float32: lambda1/lambda2 - 1 stays below ~2e-5
    np.testing.assert_allclose(terms, 1.0, atol=2e-3)
    assert np.sum(fs.vote_terms(E0[valid], 1.1 * rho, 1.1 * rho, 0.01)) < 0.5 * valid.sum()


def test_vote_ignores_scale_and_sign_of_the_two_view_matrix():
    sc = _scene(1, sigma=1.0)
    E0, valid = _e0(sc, 650.0)
    s = np.where(np.arange(len(E0)) % 2 == 0, -3.0, 0.25)[:, None, None]
    a = fs.vote_terms(E0[valid], 0.9, 0.9, 0.02)
    b = fs.vote_terms((s * E0)[valid], 0.9, 0.9, 0.02)
    np.testing.assert_allclose(a, b, rtol=1e-12)


@pytest.mark.parametrize("f0", [450.0, 900.0])
def test_shared_focal_recovered_within_the_grid_spacing(f0):
    sc = _scene(1)
    E0, valid = _e0(sc, f0)
    rhos = fs.candidates(1 / 3, 3, 1024)
    k, v = fs.search_shared(E0, valid, rhos, 0.01)
    step = np.log(rhos[1] / rhos[0])
    assert abs(np.log(rhos[k] * f0 / sc.focal[0])) <= step


def test_groups_recovered_in_ready_pair_order():
    """Three groups of images along the trajectory, each with its own focal
    length: the greedy order estimates all three, each within the grid
    spacing; the first group estimated is the one with the most pairs inside
    it."""
    sc = _scene(3)
    g = sc.meta["focal_group"]
    f0 = 700.0
    E0, valid = _e0(sc, f0)
    rhos = fs.candidates(1 / 3, 3, 1024)
    rho, order = fs.search_groups(E0, valid, sc.pair_i, sc.pair_j, g, 3, rhos, 0.01)
    step = np.log(rhos[1] / rhos[0])
    f_true = np.array([sc.focal[np.nonzero(g == q)[0][0]] for q in range(3)])
    assert sorted(order) == [0, 1, 2]
    assert np.all(np.abs(np.log(rho * f0 / f_true)) <= 2 * step)
    inside = [np.sum(valid & (g[sc.pair_i] == q) & (g[sc.pair_j] == q)) for q in range(3)]
    assert order[0] == int(np.argmax(inside))
