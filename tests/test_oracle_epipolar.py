"""Pins of the oracle's epipolar adjustment (Sec. 3.3, Eqs. 7-9, Appendix
"Epipolar Adjustment") against geometry, invariances, the compact-form
identity and finite differences (no CUDA)."""
import numpy as np
import pytest

from oracle import epipolar as ep
from oracle.so3 import rot_from_6d
from tests._util import (clean_scene, gt_params_ea, perturbed_params_ea, scene,
                         similarity_transform_ea)


def _xs(sc):
    return ep.calibrated_pairs(sc.kp1_px, sc.kp2_px, sc.kp_img_pair, sc.pair_i, sc.pair_j,
                               sc.focal, sc.cx, sc.cy)


def _fd_grad(fun, p, h):
    g = np.zeros_like(p)
    for n in range(p.shape[0]):
        for k in range(p.shape[1]):
            a, b = p.copy(), p.copy()
            a[n, k] += h
            b[n, k] -= h
            g[n, k] = (fun(a) - fun(b)) / (2 * h)
    return g


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def test_calibration_is_inverse_intrinsics():
    sc = scene("c1", 0)
    x1, x2 = _xs(sc)
    i = sc.pair_i[sc.kp_img_pair]
    K = np.zeros((len(i), 3, 3))
    K[:, 0, 0] = sc.focal[i]
    K[:, 1, 1] = sc.focal[i]
    K[:, 0, 2] = sc.cx[i]
    K[:, 1, 2] = sc.cy[i]
    K[:, 2, 2] = 1.0
    uv1 = np.concatenate([sc.kp1_px.astype(np.float64), np.ones((len(i), 1))], axis=1)
    np.testing.assert_allclose(np.einsum("mab,mb->ma", K, x1), uv1, atol=1e-9)
    assert np.all(x2[:, 2] == 1.0)


def test_residual_is_the_coplanarity_determinant():
    """x2^T [t^]_x R x1 = det[x2, t^, R x1]: the three rays are coplanar for a
    true match.  Checked pair by pair with rotation matrices built directly
    from ground truth (not through the 6D map)."""
    sc = scene("c1", 0)
    x1, x2 = _xs(sc)
    rng = np.random.default_rng(0)
    p = perturbed_params_ea(sc, 0)
    geo = ep.pair_geometry(p, sc.pair_i, sc.pair_j)
    r = ep.residuals(geo["E"], x1, x2, sc.kp_img_pair)
    R = rot_from_6d(p[:, :6])
    for m in rng.choice(sc.n_kp, 40, replace=False):
        n = sc.kp_img_pair[m]
        i, j = sc.pair_i[n], sc.pair_j[n]
        Rij = R[j] @ R[i].T
        tij = p[j, 6:] - Rij @ p[i, 6:]
        that = tij / np.linalg.norm(tij)
        ref = np.linalg.det(np.stack([x2[m], that, Rij @ x1[m]], axis=1))
        assert abs(r[m] - ref) < 1e-12


def test_zero_loss_at_noise_free_ground_truth():
    sc = clean_scene(0)
    x1, x2 = _xs(sc)
    p = gt_params_ea(sc)
    L1, _, _ = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss="l1")
    L2, g2, _ = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss="l2")
    # keypoints are stored as float32 pixels (as the C ABI takes them): a pixel
    # of magnitude < 1024 rounds by <= 2^-24*1024 = 6.1e-5 px, i.e. <= 1.3e-7 in
    # calibrated units at f >= 500; |r| <= |x2| |E| |dx1| + ... stays below ~1e-6.
    assert L1 < 1e-7 and L2 < 1e-13
    assert np.max(np.abs(g2)) < 1e-10
    # and clearly non-zero away from it / with noise
    Lp, _, _ = ep.direct_loss_grad(perturbed_params_ea(sc, 1), sc.pair_i, sc.pair_j, x1, x2,
                                   sc.kp_img_pair, loss="l1")
    assert Lp > 1e-3


def test_noise_free_W_annihilates_true_essential_matrix():
    sc = clean_scene(1)
    x1, x2 = _xs(sc)
    W = ep.build_W(x1, x2, sc.kp_img_pair, sc.n_pairs)
    e = ep.essential_matrices(gt_params_ea(sc), sc.pair_i, sc.pair_j).reshape(-1, 9)
    We = np.einsum("pab,pb->pa", W, e)
    # zero up to the float32 pixel rounding of the keypoints (|w^T e| ~ 1e-7)
    assert np.max(np.abs(We).max(axis=1) / np.linalg.norm(W, axis=(1, 2))) < 1e-7
    e_bad = ep.essential_matrices(perturbed_params_ea(sc, 1), sc.pair_i, sc.pair_j).reshape(-1, 9)
    assert np.median(np.abs(np.einsum("pab,pb->pa", W, e_bad)).max(axis=1) / np.linalg.norm(W, axis=(1, 2))) > 1e-4
    # W is symmetric positive semi-definite
    np.testing.assert_allclose(W, np.transpose(W, (0, 2, 1)), atol=0)
    assert np.min(np.linalg.eigvalsh(W)) > -1e-9


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_world_similarity_invariance(loss):
    sc = scene("c1", 0)
    x1, x2 = _xs(sc)
    p = perturbed_params_ea(sc, 2)
    from oracle.so3 import angle_axis
    Q = angle_axis([0.3, -1.0, 0.5], 0.7)
    q = similarity_transform_ea(p, Q, np.array([1.0, -2.0, 0.5]), 3.7)
    La, _, _ = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss=loss)
    Lb, _, _ = ep.direct_loss_grad(q, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss=loss)
    assert abs(La - Lb) <= 1e-12 * La


def test_direct_l2_equals_compact_quadratic_form():
    """Eq. 8: the per-pair L2 sum equals the sum of 9x9 quadratic forms, for
    loss and gradient, with and without IRLS weights (Eq. 9)."""
    sc = scene("c1", 3)
    x1, x2 = _xs(sc)
    p = perturbed_params_ea(sc, 3)
    rng = np.random.default_rng(3)
    for w in [None, rng.uniform(0.0, 5.0, size=sc.n_kp)]:
        inv_z = 1.0 / sc.n_kp
        Ld, gd, Gd = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair,
                                         weights=w, loss="l2", inv_z=inv_z)
        W = ep.build_W(x1, x2, sc.kp_img_pair, sc.n_pairs, weights=w)
        Lc, gc, Gc = ep.compact_loss_grad(p, sc.pair_i, sc.pair_j, W, inv_z)
        assert abs(Ld - Lc) <= 1e-12 * Ld
        assert _rel(gc, gd) < 1e-10
        assert _rel(Gc, Gd) < 1e-10


def test_l2_gradient_central_differences():
    sc = scene("c1", 4)
    x1, x2 = _xs(sc)
    p = perturbed_params_ea(sc, 4)
    w = 1.0 / np.maximum(np.abs(ep.residuals(ep.essential_matrices(p, sc.pair_i, sc.pair_j), x1, x2, sc.kp_img_pair)), 1e-6)

    def f(q):
        return ep.direct_loss_grad(q, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, weights=w, loss="l2")[0]

    _, g, _ = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, weights=w, loss="l2")
    assert _rel(g, _fd_grad(f, p, 1e-6)) < 1e-6
    # the step the workload description fixes (1e-3): only O(h^2) truncation remains
    assert _rel(g, _fd_grad(f, p, 1e-3)) < 1e-3


def test_l1_gradient_central_differences():
    """|r| has a kink at 0; a step of 1e-7 crosses it for essentially no pair at
    these perturbed parameters (checked: the smallest |r| is reported)."""
    sc = scene("c1", 5)
    x1, x2 = _xs(sc)
    p = perturbed_params_ea(sc, 5)

    def f(q):
        return ep.direct_loss_grad(q, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss="l1")[0]

    _, g, _ = ep.direct_loss_grad(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, loss="l1")
    assert _rel(g, _fd_grad(f, p, 1e-8)) < 1e-4


def test_irls_weights_closed_form():
    r = np.array([0.5, -1e-9, 2e-3, -0.2, 0.0])
    w, keep = ep.irls_weights(r, tau=0.3, delta=1e-6)
    np.testing.assert_allclose(w, [0.0, 1e6, 500.0, 5.0, 1e6])
    assert keep.tolist() == [False, True, True, True, True]
