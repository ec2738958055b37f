"""Pins of the oracle's track completion and adaptive image-pair filtering
(Appendix "Tracks" and "Filtering"): hand-checked graphs, connected
components against networkx, completion against the generator's true tracks,
the count identity, and the halving schedule (no CUDA)."""
from itertools import combinations

import networkx as nx
import numpy as np
import pytest

from oracle import tracks as T
from synthetic.scenes import raw_matches_c2


def test_chain_is_completed():
    # images 0, 1, 2 with one keypoint each; matches 0-1 and 1-2
    out = T.complete_tracks([0, 1, 2, 3], [[0, 1], [1, 2]])
    assert out["n_tracks"] == 1 and out["consistent"].tolist() == [True]
    assert list(zip(out["pair_i"], out["pair_j"])) == [(0, 1), (0, 2), (1, 2)]
    assert out["kp_img_pair"].tolist() == [0, 1, 2]
    assert list(zip(out["node1"], out["node2"])) == [(0, 1), (0, 2), (1, 2)]
    assert out["kp_track"].tolist() == [0, 0, 0]


def test_inconsistent_track_passes_its_raw_matches():
    # image 0: keypoints 0, 1; image 1: keypoint 2; image 2: keypoint 3
    # 0-2 and 1-2 join two keypoints of image 0: not completed
    out = T.complete_tracks([0, 2, 3, 4], [[2, 1], [0, 2], [2, 3]])
    assert out["consistent"].tolist() == [False]
    assert list(zip(out["pair_i"], out["pair_j"])) == [(0, 1), (1, 2)]
    # raw matches in input order, oriented from the lower image
    assert list(zip(out["node1"], out["node2"])) == [(1, 2), (0, 2), (2, 3)]
    assert out["kp_img_pair"].tolist() == [0, 0, 1]


def test_components_match_networkx():
    rng = np.random.default_rng(4)
    for K, M in [(50, 30), (200, 180), (300, 600)]:
        e = rng.integers(0, K, size=(M, 2))
        e = e[e[:, 0] != e[:, 1]]
        lab = T.components(K, e)
        g = nx.Graph()
        g.add_nodes_from(range(K))
        g.add_edges_from(e.tolist())
        ref = np.empty(K, np.int64)
        for comp in nx.connected_components(g):
            ref[list(comp)] = min(comp)
        np.testing.assert_array_equal(lab, ref)


def _track_pairs(out):
    pairs = {}
    for a, b, t in zip(out["node1"], out["node2"], out["kp_track"]):
        pairs.setdefault(int(t), set()).add((int(a), int(b)))
    return pairs


def test_full_recall_reproduces_the_true_tracks():
    rm = raw_matches_c2(seed=2, n_cams=15, n_points=1500, recall=1.0, distractors=3)
    out = T.complete_tracks(rm.kp_off, rm.matches)
    img = T.image_of(rm.kp_off)
    truth = {}
    for x in range(rm.n_kp):
        if rm.true_track[x] >= 0:
            truth.setdefault(int(rm.true_track[x]), []).append(x)
    truth = {t: m for t, m in truth.items() if len(m) >= 2}
    assert out["n_tracks"] == len(truth) and out["consistent"].all()
    want = sorted(tuple(sorted((a, b), key=lambda z: img[z])) for m in truth.values() for a, b in combinations(m, 2))
    got = sorted(zip(out["node1"].tolist(), out["node2"].tolist()))
    assert got == want
    # grouped by image pair, lower image first
    assert np.all(np.diff(out["kp_img_pair"]) >= 0)
    assert np.all(img[out["node1"]] == out["pair_i"][out["kp_img_pair"]])
    assert np.all(img[out["node2"]] == out["pair_j"][out["kp_img_pair"]])


def test_low_recall_tracks_are_parts_of_true_tracks():
    rm = raw_matches_c2(seed=3, n_cams=15, n_points=1500, recall=0.3)
    out = T.complete_tracks(rm.kp_off, rm.matches)
    assert out["consistent"].all()
    for t, ps in _track_pairs(out).items():
        nodes = {a for p in ps for a in p}
        assert len({int(rm.true_track[x]) for x in nodes}) == 1
        assert len(ps) == len(nodes) * (len(nodes) - 1) // 2   # complete
    # completion adds pairs: more than the raw matches
    assert len(out["node1"]) > len(rm.matches)


def test_count_identity_with_spurious_matches():
    rm = raw_matches_c2(seed=5, n_cams=12, n_points=1200, recall=0.6, spurious_frac=0.05)
    out = T.complete_tracks(rm.kp_off, rm.matches)
    lab = T.components(rm.n_kp, rm.matches)
    roots = np.nonzero((np.arange(rm.n_kp) == lab) & (np.bincount(lab, minlength=rm.n_kp) >= 2))[0]
    sizes = np.bincount(lab, minlength=rm.n_kp)[roots]
    raw_per_root = {int(r): 0 for r in roots}
    for u, v in rm.matches:
        raw_per_root[int(lab[u])] += 1
    expect = sum(int(k * (k - 1) // 2) if c else raw_per_root[int(r)]
                 for r, k, c in zip(roots, sizes, out["consistent"]))
    assert (~out["consistent"]).sum() > 0
    assert len(out["node1"]) == expect
    # min_pairs drops whole image pairs
    out8 = T.complete_tracks(rm.kp_off, rm.matches, min_pairs=8)
    cnt = np.bincount(out["kp_img_pair"])
    assert len(out8["pair_i"]) == int(np.sum(cnt >= 8))
    assert len(out8["node1"]) == int(cnt[cnt >= 8].sum())


def test_filter_halves_until_connected():
    pi, pj = np.array([0, 1, 2, 0]), np.array([1, 2, 3, 3])
    counts = np.array([10, 3, 10, 1])
    keep, valid, t = T.filter_image_pairs(4, pi, pj, counts, 8, 1)
    assert t == 2.0 and valid.all() and keep.tolist() == [True, True, True, False]
    # stopped at t_min = 4 while still disconnected: the tie between {0, 1}
    # and {2, 3} goes to the component with the smallest image
    keep, valid, t = T.filter_image_pairs(4, pi, pj, counts, 8, 4)
    assert t == 4.0 and valid.tolist() == [True, True, False, False]
    assert keep.tolist() == [True, False, False, False]


@pytest.mark.parametrize("t_start", [100, 7])
def test_filter_drops_an_isolated_image(t_start):
    pi, pj = np.array([0, 1, 0]), np.array([1, 2, 2])
    counts = np.array([50, 40, 30])
    keep, valid, t = T.filter_image_pairs(4, pi, pj, counts, t_start, 2)   # image 3 has no pair
    assert t == 2.0 and valid.tolist() == [True, True, True, False] and keep.all()
