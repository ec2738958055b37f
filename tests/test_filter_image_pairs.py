"""Adaptive image-pair filtering through the C ABI (host code, no GPU)
against the oracle (Appendix "Filtering"): bit-exact keep flags, image
validity and threshold on hand-made and random view graphs."""
import numpy as np
import pytest

from oracle import tracks as T
from paper_2505_04612_b300 import build as B
from paper_2505_04612_b300 import fastmap as F


@pytest.fixture(scope="module", autouse=True)
def _lib():
    B.build()


def _same(n, pi, pj, c, t0, tmin):
    k, v, t = F.filter_image_pairs(n, pi, pj, c, t0, tmin)
    ko, vo, to = T.filter_image_pairs(n, pi, pj, c, t0, tmin)
    np.testing.assert_array_equal(k, ko)
    np.testing.assert_array_equal(v, vo)
    assert t == to
    return k, v, t


def test_hand_made_graphs():
    pi, pj, c = np.array([0, 1, 2, 0]), np.array([1, 2, 3, 3]), np.array([10, 3, 10, 1])
    assert _same(4, pi, pj, c, 8, 1)[2] == 2.0
    k, v, t = _same(4, pi, pj, c, 8, 4)
    assert v.tolist() == [True, True, False, False]
    _same(5, np.array([0, 1, 0]), np.array([1, 2, 2]), np.array([50, 40, 30]), 100, 2)   # image 4 isolated


@pytest.mark.parametrize("seed", range(6))
def test_random_view_graphs(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(5, 60))
    P = int(rng.integers(0, 3 * n))
    pi = rng.integers(0, n, P)
    pj = rng.integers(0, n, P)
    ok = pi != pj
    pi, pj = np.minimum(pi, pj)[ok], np.maximum(pi, pj)[ok]
    c = rng.integers(1, 400, len(pi))
    _same(n, pi, pj, c, float(rng.choice([512, 100, 37.5])), float(rng.choice([1, 4, 15])))


def test_invalid_arguments():
    with pytest.raises(F.FastMapError):
        F.filter_image_pairs(3, [0], [3], [5], 10, 1)        # image out of range
    with pytest.raises(F.FastMapError):
        F.filter_image_pairs(3, [1], [1], [5], 10, 1)        # one image twice
    with pytest.raises(F.FastMapError):
        F.filter_image_pairs(3, [0], [1], [5], 1, 10)        # t_start < t_min
