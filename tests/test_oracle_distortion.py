"""Pins of the oracle's distortion interval search (Sec. 3.1 "Distortion
Estimation", Eq. 1; Appendix "Distortion Estimation"): undistortion inverts
the generator's distortion (an independent closed-form root), the eight-point
fundamental matrix equals K^-T [t]x R K^-1 of the true poses, the average
epipolar error vanishes only at the true alpha, the hierarchical search on
functions with known minima, and recovery on noise-free and noisy scenes
with one and with several cameras (no CUDA)."""
import numpy as np
import pytest

from oracle import distortion as D
from synthetic.scenes import _distort, scene_c2


def _scene(alpha, groups=1, sigma=0.0, seed=5, n_cams=40):
    return scene_c2(seed=seed, n_cams=n_cams, n_points=5000, sigma_px=sigma, outlier_frac=0.0,
                    focal_groups=groups, alpha=alpha)


def _xd(sc):
    ci = sc.pair_i[sc.kp_img_pair]
    cj = sc.pair_j[sc.kp_img_pair]
    return (D.normalised(sc.kp1_px, sc.cx[ci], sc.cy[ci]), D.normalised(sc.kp2_px, sc.cx[cj], sc.cy[cj]))


def _resolution(n_cand=32, n_levels=3, width=1.0):
    step = width / (n_cand - 1)
    for _ in range(n_levels - 1):
        step = 2 * step / (n_cand - 1)
    return step


@pytest.mark.parametrize("alpha", [-0.4, -0.1, 0.0, 0.15])
def test_undistortion_inverts_the_generator(alpha):
    rng = np.random.default_rng(1)
    W, H = 640.0, 480.0
    uv = rng.uniform([0, 0], [W, H], size=(1000, 2))
    cx, cy = np.full(1000, W / 2), np.full(1000, H / 2)
    obs = _distort(uv, np.full(1000, alpha), cx, cy)
    xu = D.undistort(D.normalised(obs, cx, cy), alpha)
    np.testing.assert_allclose(xu, D.normalised(uv, cx, cy), rtol=0, atol=1e-12)
    if alpha == 0.0:
        np.testing.assert_allclose(obs, uv, rtol=0, atol=1e-9)


def test_fundamental_matrix_of_noise_free_pairs_is_the_true_one():
    sc = _scene(0.0)
    xd1, xd2 = _xd(sc)
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    h = np.hypot(sc.cx[0], sc.cy[0])
    for n in [0, sc.n_pairs // 2, sc.n_pairs - 1]:
        i, j = sc.pair_i[n], sc.pair_j[n]
        s = slice(off[n], off[n + 1])
        F = D.fundamental_8pt(D.homogeneous(xd1[s]), D.homogeneous(xd2[s]))
        R = sc.R_gt[j] @ sc.R_gt[i].T
        t = sc.t_gt[j] - R @ sc.t_gt[i]
        tx = np.array([[0, -t[2], t[1]], [t[2], 0, -t[0]], [-t[1], t[0], 0]])
        Ki = np.diag([h / sc.focal[i], h / sc.focal[i], 1.0])
        Kj = np.diag([h / sc.focal[j], h / sc.focal[j], 1.0])
        Ft = Kj.T @ tx @ R @ Ki
        Ft /= np.linalg.norm(Ft)
        assert abs(np.linalg.norm(F) - 1.0) < 1e-12
        assert abs(np.linalg.det(F)) < 1e-12
        # pixels are stored in float32: agreement to ~1e-5
        assert abs(abs(np.sum(F * Ft)) - 1.0) < 1e-6, np.sum(F * Ft)


def test_normalisation_moves_points_to_the_centroid_at_rms_sqrt2():
    rng = np.random.default_rng(3)
    x = D.homogeneous(rng.normal([0.3, -0.2], [0.05, 0.2], size=(50, 2)))
    y = x @ D.hartley(x).T
    np.testing.assert_allclose(y[:, :2].mean(axis=0), 0.0, atol=1e-12)
    assert abs(np.sqrt(np.mean(np.sum(y[:, :2] ** 2, axis=1))) - np.sqrt(2.0)) < 1e-12
    np.testing.assert_array_equal(y[:, 2], 1.0)


def test_error_is_scale_free():
    """The epipolar error is measured in the normalised frame: scaling the
    undistorted points about the origin (what a positive alpha does to the
    outer points) leaves it unchanged, while the algebraic error of the
    undistorted coordinates shrinks with the points."""
    sc = _scene(0.0, sigma=1.0)
    xd1, xd2 = _xd(sc)
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    s = slice(off[3], off[4])
    x1, x2 = D.homogeneous(xd1[s]), D.homogeneous(xd2[s])
    y1, y2 = D.homogeneous(0.5 * xd1[s]), D.homogeneous(0.5 * xd2[s])
    assert abs(D.error_sum(y1, y2) / D.error_sum(x1, x2) - 1.0) < 1e-9

    def raw(a, b):
        F = D.fundamental_8pt(a, b)
        return np.sum(np.abs(np.einsum("mp,pq,mq->m", b, F, a)))
    assert raw(y1, y2) < 0.6 * raw(x1, x2)


def test_error_vanishes_only_at_the_true_alpha():
    sc = _scene(-0.2)
    xd1, xd2 = _xd(sc)
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    pairs = np.arange(sc.n_pairs)

    def err(a):
        return D.average_error(xd1, xd2, off, pairs, np.full(len(pairs), a), np.full(len(pairs), a))

    e0 = err(-0.2)
    assert e0 < 1e-6
    assert err(-0.15) > 20 * e0 and err(-0.25) > 20 * e0 and err(0.0) > 100 * e0


def test_hierarchical_search_on_known_functions():
    res = _resolution()
    best, cands, _ = D.search(lambda a: (a - 0.1234) ** 2, -0.5, 0.5, 32, 3)
    assert abs(best - 0.1234) <= res
    assert len(cands) == 3 and np.isclose(cands[1][-1] - cands[1][0], 2.0 / 31)
    assert D.search(lambda a: a, -0.5, 0.5, 32, 3)[0] == -0.5      # minimum at the left end
    assert D.search(lambda a: -a, -0.5, 0.5, 32, 3)[0] == 0.5      # right end
    assert D.search(lambda a: 1.0, -0.5, 0.5, 32, 3)[0] == -0.5    # ties: the first candidate
    # a single level is the plain grid
    best, cands, _ = D.search(lambda a: abs(a - 0.2), -0.5, 0.5, 11, 1)
    assert np.isclose(best, 0.2) and len(cands) == 1


@pytest.mark.parametrize("alpha,sigma,tol", [(-0.2, 0.0, None), (-0.3, 1.0, 0.01), (0.1, 1.0, 0.01)])
def test_one_camera_recovered(alpha, sigma, tol):
    sc = _scene(alpha, sigma=sigma)
    xd1, xd2 = _xd(sc)
    est, order = D.search_groups(xd1, xd2, sc.kp_img_pair, sc.pair_i, sc.pair_j, np.zeros(sc.n_cams, int), 1)
    assert order == [0]
    assert abs(est[0] - alpha) <= (2 * _resolution() if tol is None else tol), est


def test_cameras_recovered_in_ready_pair_order():
    alphas = np.array([-0.3, 0.05, -0.1])
    sc = _scene(alphas, groups=3)
    g = sc.meta["focal_group"]
    xd1, xd2 = _xd(sc)
    est, order = D.search_groups(xd1, xd2, sc.kp_img_pair, sc.pair_i, sc.pair_j, g, 3)
    assert sorted(order) == [0, 1, 2]
    np.testing.assert_allclose(est, alphas, atol=2e-3)
    off = D.pair_offsets(sc.kp_img_pair, sc.n_pairs)
    valid = np.diff(off) >= 8
    inside = [np.sum(valid & (g[sc.pair_i] == q) & (g[sc.pair_j] == q)) for q in range(3)]
    assert order[0] == int(np.argmax(inside))
