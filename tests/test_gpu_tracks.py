"""Track completion on the GPU (fm_tracks_complete; Appendix "Tracks")
against the oracle (oracle/tracks: plain union-find, explicit emission and
sort): every output array bit-exact, on hand-made graphs, generated raw
matches of low recall with spurious matches and distractors, host and device
inputs, min_pairs, empty inputs and invalid matches; at a larger size the
components are checked against scipy's and the counts against the identity
of the reading."""
import numpy as np
import pytest

from oracle import tracks as T
from synthetic.scenes import raw_matches_c2
from tests import _gpu as G

pytestmark = pytest.mark.gpu

KEYS = ["pair_i", "pair_j", "kp_img_pair", "node1", "node2", "kp_track"]


def _gpu(kp_off, matches, kp_px=None, min_pairs=1, device=False):
    G.lib_ready()
    from paper_2505_04612_b300 import fastmap as F
    if device:
        import torch
        t = lambda a, dt: torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).cuda()  # noqa: E731
        out = F.complete_tracks(t(kp_off, np.int32), t(np.asarray(matches).reshape(-1, 2), np.int32),
                                None if kp_px is None else t(kp_px, np.float32), min_pairs)
        return {k: (v.cpu().numpy() if hasattr(v, "cpu") else v) for k, v in out.items()}
    return F.complete_tracks(kp_off, matches, kp_px, min_pairs)


def _check(kp_off, matches, min_pairs=1, device=False, kp_px=None):
    out = _gpu(kp_off, matches, kp_px, min_pairs, device)
    ref = T.complete_tracks(kp_off, matches, min_pairs)
    for k in KEYS:
        np.testing.assert_array_equal(out[k], ref[k], err_msg=k)
    assert out["n_tracks"] == ref["n_tracks"]
    assert out["n_inconsistent"] == int((~ref["consistent"]).sum())
    if kp_px is not None:
        np.testing.assert_array_equal(out["kp1_px"], np.asarray(kp_px)[ref["node1"]])
        np.testing.assert_array_equal(out["kp2_px"], np.asarray(kp_px)[ref["node2"]])
    return out


def test_hand_made_graphs():
    _check([0, 1, 2, 3], [[0, 1], [1, 2]])                     # chain -> completed
    _check([0, 2, 3, 4], [[2, 1], [0, 2], [2, 3]])             # inconsistent: raw matches
    _check([0, 1, 2, 3, 4], [[3, 0], [2, 1]])                  # two tracks, reversed orientation


@pytest.mark.parametrize("recall,spurious,distractors", [(1.0, 0.0, 0), (0.5, 0.0, 4), (0.3, 0.05, 2),
                                                         (0.6, 0.2, 0)])
def test_generated_raw_matches(recall, spurious, distractors):
    rm = raw_matches_c2(seed=7, n_cams=25, n_points=2500, recall=recall, spurious_frac=spurious,
                        distractors=distractors)
    out = _check(rm.kp_off, rm.matches, kp_px=rm.kp_px)
    assert len(out["node1"]) >= len(rm.matches) * (1 if spurious else 1)


@pytest.mark.parametrize("min_pairs", [2, 8])
def test_min_pairs_and_device_inputs(min_pairs):
    rm = raw_matches_c2(seed=8, n_cams=20, n_points=2000, recall=0.5, spurious_frac=0.02)
    _check(rm.kp_off, rm.matches, min_pairs=min_pairs, device=True, kp_px=rm.kp_px)


def test_shuffled_matches_give_the_same_consistent_tracks():
    """The labels and the consistent tracks' pairs do not depend on the order
    or orientation of the raw matches."""
    rm = raw_matches_c2(seed=9, n_cams=20, n_points=2000, recall=0.5)
    a = _gpu(rm.kp_off, rm.matches)
    rng = np.random.default_rng(0)
    m = rm.matches[rng.permutation(len(rm.matches))]
    flip = rng.random(len(m)) < 0.5
    m[flip] = m[flip][:, ::-1]
    b = _gpu(rm.kp_off, m)
    for k in KEYS:
        np.testing.assert_array_equal(a[k], b[k])


def test_empty_inputs_and_invalid_matches():
    from paper_2505_04612_b300.fastmap import FastMapError
    out = _check([0, 3, 5, 9], np.zeros((0, 2), np.int32))
    assert len(out["pair_i"]) == 0 and len(out["node1"]) == 0
    with pytest.raises(FastMapError):
        _gpu([0, 2, 4], [[0, 1]])          # both keypoints in image 0
    with pytest.raises(FastMapError):
        _gpu([0, 2, 4], [[0, 4]])          # keypoint 4 does not exist
    with pytest.raises(FastMapError):
        _gpu([0, 2, 4], [[7, 1], [0, 3]])  # first keypoint out of range (never dereferenced)
    with pytest.raises(FastMapError):
        _gpu([0, 2, 4], [[-1, 3], [0, 3]])


def test_larger_scene_against_independent_components():
    """~100k keypoints: labels against scipy's connected components, counts
    against the reading's identity, grouping and orientation."""
    from scipy.sparse import coo_matrix
    from scipy.sparse.csgraph import connected_components
    rm = raw_matches_c2(seed=11, n_cams=150, n_points=40000, recall=0.4, spurious_frac=0.01, distractors=10)
    out = _gpu(rm.kp_off, rm.matches)
    K = rm.n_kp
    g = coo_matrix((np.ones(len(rm.matches)), (rm.matches[:, 0], rm.matches[:, 1])), shape=(K, K))
    nc, lab = connected_components(g, directed=False)
    first = np.full(nc, K)
    np.minimum.at(first, lab, np.arange(K))
    label = first[lab]
    size = np.bincount(label, minlength=K)
    img = T.image_of(rm.kp_off)
    roots = np.nonzero((np.arange(K) == label) & (size >= 2))[0]
    assert out["n_tracks"] == len(roots)
    # consistency: a component with two keypoints in one image
    key = label.astype(np.int64) * len(rm.kp_off) + img
    dup = np.zeros(K, bool)
    u, c = np.unique(key, return_counts=True)
    dup[(u[c > 1] // len(rm.kp_off))] = True
    raw = np.bincount(label[rm.matches[:, 0]], minlength=K)
    expect = int(sum(int(size[r]) * (int(size[r]) - 1) // 2 if not dup[r] else int(raw[r]) for r in roots))
    assert len(out["node1"]) == expect and out["n_inconsistent"] == int(dup[roots].sum())
    # grouping, orientation, track of every pair = its keypoints' component
    assert np.all(np.diff(out["kp_img_pair"]) >= 0)
    pk = out["pair_i"].astype(np.int64) * len(rm.kp_off) + out["pair_j"]
    assert np.all(np.diff(pk) > 0)
    assert np.all(img[out["node1"]] == out["pair_i"][out["kp_img_pair"]])
    assert np.all(img[out["node2"]] == out["pair_j"][out["kp_img_pair"]])
    assert np.all(label[out["node1"]] == label[out["node2"]])
    np.testing.assert_array_equal(roots[out["kp_track"]], label[out["node1"]])
