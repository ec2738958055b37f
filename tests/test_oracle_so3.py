"""Pins of the oracle's rotation helpers against closed forms and finite
differences (no CUDA)."""
import numpy as np

from oracle.so3 import (angle_axis, geodesic, project_to_rotation, rot_from_6d, rot_from_6d_vjp,
                        rot_to_6d, skew)


def _random_rotations(rng, n):
    return np.stack([angle_axis(rng.normal(size=3), rng.uniform(0, np.pi)) for _ in range(n)])


def test_skew_is_cross_product():
    rng = np.random.default_rng(0)
    a, b = rng.normal(size=(2, 5, 3))
    np.testing.assert_allclose(np.einsum("nij,nj->ni", skew(a), b), np.cross(a, b), atol=1e-14)


def test_6d_round_trip_and_orthonormality():
    rng = np.random.default_rng(1)
    R = _random_rotations(rng, 50)
    np.testing.assert_allclose(rot_from_6d(rot_to_6d(R)), R, atol=1e-13)
    a = rng.normal(size=(200, 6))
    Q = rot_from_6d(a)
    np.testing.assert_allclose(np.einsum("nki,nkj->nij", Q, Q), np.broadcast_to(np.eye(3), Q.shape), atol=1e-13)
    np.testing.assert_allclose(np.linalg.det(Q), 1.0, atol=1e-13)
    # first column is the direction of a1; second lies in span(a1, a2) on a2's side
    np.testing.assert_allclose(Q[:, :, 0], a[:, :3] / np.linalg.norm(a[:, :3], axis=1, keepdims=True), atol=1e-13)
    assert np.all(np.einsum("ni,ni->n", Q[:, :, 1], a[:, 3:]) > 0)


def test_6d_invariances():
    # positive scaling of a1, and adding a multiple of a1 to a2, leave R unchanged
    rng = np.random.default_rng(2)
    a = rng.normal(size=(20, 6))
    b = a.copy()
    b[:, :3] *= rng.uniform(0.1, 5.0, size=(20, 1))
    b[:, 3:] += rng.normal(size=(20, 1)) * a[:, :3]
    b[:, 3:] *= rng.uniform(0.1, 5.0, size=(20, 1))
    np.testing.assert_allclose(rot_from_6d(a), rot_from_6d(b), atol=1e-12)


def test_6d_vjp_finite_differences():
    rng = np.random.default_rng(3)
    a = rng.normal(size=(4, 6))
    gR = rng.normal(size=(4, 3, 3))
    g = rot_from_6d_vjp(a, gR)
    h = 1e-6
    fd = np.zeros_like(a)
    for n in range(4):
        for k in range(6):
            ap, am = a.copy(), a.copy()
            ap[n, k] += h
            am[n, k] -= h
            fd[n, k] = (np.sum(gR[n] * rot_from_6d(ap)[n]) - np.sum(gR[n] * rot_from_6d(am)[n])) / (2 * h)
    np.testing.assert_allclose(g, fd, rtol=1e-7, atol=1e-8)


def test_geodesic_closed_form():
    rng = np.random.default_rng(4)
    for ang in [0.0, 1e-3, 0.3, 1.0, 2.5, np.pi - 1e-3]:
        axis = rng.normal(size=3)
        R0 = _random_rotations(rng, 1)[0]
        R1 = angle_axis(axis, ang) @ R0
        assert abs(geodesic(R0, R1) - ang) < 2e-8
        assert abs(geodesic(R1, R0) - ang) < 2e-8


def test_projection_to_rotation():
    rng = np.random.default_rng(5)
    R = _random_rotations(rng, 20)
    np.testing.assert_allclose(project_to_rotation(R), R, atol=1e-14)
    # a float32 copy is brought back to an exact rotation within float32 rounding
    Rf = R.astype(np.float32).astype(np.float64)
    Q = project_to_rotation(Rf)
    np.testing.assert_allclose(np.einsum("nki,nkj->nij", Q, Q), np.broadcast_to(np.eye(3), Q.shape), atol=1e-14)
    assert np.max(np.abs(Q - R)) < 2e-7
    # a reflection is mapped to a proper rotation
    F = R[0] @ np.diag([1.0, 1.0, -1.0])
    assert abs(np.linalg.det(project_to_rotation(F)) - 1.0) < 1e-12
