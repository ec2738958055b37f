"""Pins of the oracle's sparse reconstruction (Appendix "Sparse
Reconstruction") on hand-built tracks whose decisions follow from the
geometry alone (tests/_tri_cases.py): the reprojection threshold in the
observing camera's own pixels, the 3-distinct-camera rule, the angle
threshold, and the angle taken only over pairs whose two keypoints are
inliers."""
import numpy as np
import pytest

from oracle import epipolar as ep
from oracle import triangulation as tri
from tests import _tri_cases as C


def _run(sc):
    x1, x2 = ep.calibrated_pairs(sc.kp1_px, sc.kp2_px, sc.kp_img_pair, sc.pair_i, sc.pair_j,
                                 sc.focal, sc.cx, sc.cy)
    return tri.triangulate(sc.R_gt, sc.t_gt, sc.pair_i, sc.pair_j, sc.kp_img_pair, x1, x2, sc.kp_track, 1,
                           sc.focal, 4.0, 2.0, diag=True)


@pytest.mark.parametrize("first", [False, True])
@pytest.mark.parametrize("delta", [4.0 - 2.0 ** -10, 4.0 + 2.0 ** -10])
def test_reprojection_threshold_in_the_observing_camera_pixels(delta, first):
    sc = C.reprojection_case(delta, first)
    pts, valid, ncam, d = _run(sc)
    # the displaced pair is degenerate, the other one meets at X
    deg = 0 if first else 1
    assert not d["pair_ok"][deg] and d["pair_ok"][1 - deg]
    np.testing.assert_allclose(pts[0], 0.0, atol=1e-12)
    # D's error is delta in D's pixels (A's focal length would give delta / 2)
    err_d = d["err1"][0] if first else d["err2"][1]
    assert abs(err_d - delta) < 1e-9
    inlier = delta <= 4.0
    assert ncam[0] == (3 if inlier else 2)
    # with D out, three inlier keypoints remain (A twice, B) but only two cameras
    assert bool(valid[0]) == inlier


@pytest.mark.parametrize("theta", [1.99, 2.01])
def test_angle_threshold(theta):
    sc = C.angle_case(theta)
    pts, valid, ncam, d = _run(sc)
    assert ncam[0] == 3 and d["pair_ok"].all()
    assert abs(d["max_angle_deg"][0] - theta) < 1e-5
    assert bool(valid[0]) == (theta >= 2.0)


def test_angle_only_over_inlier_pairs():
    kept = _run(C.exclusion_case(False))
    dropped = _run(C.exclusion_case(True))
    assert kept[1][0] and kept[2][0] == 3 and abs(kept[3]["max_angle_deg"][0] - 3.0) < 1e-5
    _, valid, ncam, d = dropped
    assert not d["pair_ok"][0]                       # A-B degenerate
    assert d["err2"][0] > 40.0                       # B's displaced keypoint is an outlier
    assert ncam[0] == 3                              # B still counts through B-C
    assert abs(d["max_angle_deg"][0] - 1.5) < 1e-5   # A-B's 3 deg left out
    assert not valid[0]


def test_expected_outcomes_table():
    for sc, want_valid, want_ncam in C.all_cases():
        _, valid, ncam, _ = _run(sc)
        assert bool(valid[0]) == want_valid and ncam[0] == want_ncam, sc.name


def test_parallel_rays_give_no_point():
    o1, o2 = np.array([[0.0, 0.0, 0.0]]), np.array([[1.0, 0.0, 0.0]])
    d = np.array([[0.3, -0.2, 1.0]])
    _, ok = tri.midpoint(o1, d, o2, d)
    assert not ok[0]
    # just above / below the parallel threshold (sin^2 = 1e-6)
    for s2, want in ((1.2e-6, True), (0.8e-6, False)):
        ang = np.arcsin(np.sqrt(s2))
        d2 = np.array([[np.sin(ang), 0.0, np.cos(ang)]])
        _, ok = tri.midpoint(o1, np.array([[0.0, 0.0, 1.0]]), o2, d2)
        assert ok[0] == want
