"""Pins of the oracle's focal lengths inside epipolar adjustment (Sec. 3.3,
end of "Epipolar Adjustment"; reading in oracle/focal.py) against the
pose-only objective, recalibration of the pixels at another focal length,
noise-free geometry, the compact-form identity and finite differences (no
CUDA)."""
import numpy as np
import pytest

from oracle import epipolar as ep
from oracle import focal as fo
from tests._util import clean_scene, gt_params_ea, perturbed_params_ea, scene


def _xs(sc, focal=None):
    f = sc.focal if focal is None else focal
    return ep.calibrated_pairs(sc.kp1_px, sc.kp2_px, sc.kp_img_pair, sc.pair_i, sc.pair_j, f, sc.cx, sc.cy)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_zero_log_ratio_is_the_pose_only_objective(loss):
    sc = scene("c1", 1)
    x1, x2 = _xs(sc)
    p = perturbed_params_ea(sc, 3)
    L0, g0, _ = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss=loss)
    L, g, gphi = fo.direct_loss_grad(p, np.zeros(sc.n_cams), sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair,
                                     loss=loss)
    assert L == pytest.approx(L0, rel=1e-14)
    np.testing.assert_allclose(g, g0, rtol=1e-12, atol=1e-15)
    assert np.all(np.isfinite(gphi))


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_recalibrating_the_pixels_equals_shifting_the_log_ratio(loss):
    """Keypoints calibrated at f0 exp(d) and evaluated at phi - d give the
    loss (and gradients) of keypoints calibrated at f0 evaluated at phi: the
    scale matrices are built with the right sign and on the right axes."""
    sc = scene("c1", 2)
    rng = np.random.default_rng(5)
    p = perturbed_params_ea(sc, 1)
    phi = rng.normal(0.0, 0.05, sc.n_cams)
    d = rng.normal(0.0, 0.1, sc.n_cams)
    x1, x2 = _xs(sc)
    y1, y2 = _xs(sc, sc.focal * np.exp(d))
    La, ga, gpa = fo.direct_loss_grad(p, phi, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss=loss)
    Lb, gb, gpb = fo.direct_loss_grad(p, phi - d, sc.pair_i, sc.pair_j, y1, y2, sc.kp_img_pair, loss=loss)
    assert Lb == pytest.approx(La, rel=1e-12)
    np.testing.assert_allclose(gb, ga, rtol=1e-9, atol=1e-13)
    np.testing.assert_allclose(gpb, gpa, rtol=1e-9, atol=1e-13)


def test_true_focal_recovered_from_miscalibrated_noise_free_keypoints():
    """Keypoints calibrated at a wrong focal f0 = f exp(-d): the L2 loss at the
    true poses vanishes at phi = d (the true focal) and not at 0 (the pixels
    are stored in float32, so "vanishes" is ~1e-8 residuals, 1e-16 loss)."""
    sc = clean_scene(3)
    d = np.random.default_rng(2).uniform(-0.1, 0.1, sc.n_cams)
    x1, x2 = _xs(sc, sc.focal * np.exp(-d))
    p = gt_params_ea(sc)
    L_true, g_true, gphi_true = fo.direct_loss_grad(p, d, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss="l2")
    L_zero, _, gphi_zero = fo.direct_loss_grad(p, np.zeros(sc.n_cams), sc.pair_i, sc.pair_j, x1, x2,
                                               sc.kp_img_pair, loss="l2")
    assert L_true < 1e-14 and L_true < 1e-9 * L_zero
    assert np.max(np.abs(gphi_true)) < 1e-5 * np.max(np.abs(gphi_zero))


def test_finite_differences_of_the_log_ratio_and_the_poses():
    """Central differences of the L2 objective (smooth) in float64, h = 1e-5."""
    sc = scene("c1", 4)
    x1, x2 = _xs(sc)
    rng = np.random.default_rng(9)
    p = perturbed_params_ea(sc, 2)
    phi = rng.normal(0.0, 0.05, sc.n_cams)
    f = lambda q, ph: fo.direct_loss_grad(q, ph, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss="l2")[0]
    _, g, gphi = fo.direct_loss_grad(p, phi, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss="l2")
    h = 1e-5
    fd_phi = np.array([(f(p, phi + h * e) - f(p, phi - h * e)) / (2 * h) for e in np.eye(sc.n_cams)])
    assert _rel(gphi, fd_phi) < 1e-6
    fd = np.zeros_like(p)
    for n in range(sc.n_cams):
        for k in range(9):
            a, b = p.copy(), p.copy()
            a[n, k] += h
            b[n, k] -= h
            fd[n, k] = (f(a, phi) - f(b, phi)) / (2 * h)
    assert _rel(g, fd) < 1e-6


def test_compact_form_equals_direct_form_with_focal():
    """Eq. 8's identity holds at E' = S_j E S_i with W built at f0."""
    sc = scene("c1", 5)
    x1, x2 = _xs(sc)
    rng = np.random.default_rng(4)
    p = perturbed_params_ea(sc, 4)
    phi = rng.normal(0.0, 0.05, sc.n_cams)
    w = rng.uniform(0.2, 2.0, sc.n_kp)
    W = ep.build_W(x1, x2, sc.kp_img_pair, sc.n_pairs, weights=w)
    inv_z = 1.0 / sc.n_kp
    Ld, gd, gpd = fo.direct_loss_grad(p, phi, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, weights=w, loss="l2",
                                      inv_z=inv_z)
    Lc, gc, gpc = fo.compact_loss_grad(p, phi, sc.pair_i, sc.pair_j, W, inv_z)
    assert Lc == pytest.approx(Ld, rel=1e-10)
    np.testing.assert_allclose(gc, gd, rtol=1e-8, atol=1e-14)
    np.testing.assert_allclose(gpc, gpd, rtol=1e-8, atol=1e-14)
