"""Keypoint pairs in any order at creation (Sec. 3.3 groups the keypoint
pairs Q_n by image pair; Sec. 4 does the marshalling on the GPU): the
library sorts them on the device by (image pair, track, caller index) and
keeps the permutation.  With tracks that order is canonical, so a shuffled
scene gives the sorted scene's results bit for bit; per-pair weights go in
and out in the caller's order."""
import dataclasses

import numpy as np
import pytest

from tests import _gpu as G
from tests._util import perturbed_params_ea, scene

pytestmark = pytest.mark.gpu


def _shuffled(sc, seed, tracks=True):
    rng = np.random.default_rng(seed)
    q = rng.permutation(sc.n_kp)
    return dataclasses.replace(sc, name=sc.name + "_shuffled", kp_img_pair=sc.kp_img_pair[q],
                               kp1_px=sc.kp1_px[q], kp2_px=sc.kp2_px[q],
                               kp_track=sc.kp_track[q] if tracks else None, kp_inlier=sc.kp_inlier[q]), q


def _loss_grad(pr, p):
    import torch
    from paper_2505_04612_b300 import fastmap as F
    L, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(p.reshape(-1)).cuda())
    return L, g.cpu().numpy()


def test_permutation_is_the_stable_lexicographic_order():
    sc = scene("c1", 2)
    sh, _ = _shuffled(sc, 1)
    with G.make_problem(sh) as pr:
        perm = pr.kp_order()
    want = np.lexsort((np.arange(sh.n_kp), sh.kp_track, sh.kp_img_pair))
    assert np.array_equal(perm, want)
    # without tracks: the image pair alone, ties in the caller's order
    sh2, _ = _shuffled(sc, 2, tracks=False)
    with G.make_problem(sh2) as pr:
        perm = pr.kp_order()
    assert np.array_equal(perm, np.argsort(sh2.kp_img_pair, kind="stable"))
    # an input already in order is kept as it is
    with G.make_problem(sc) as pr:
        assert np.array_equal(pr.kp_order(), np.arange(sc.n_kp))


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_shuffled_scene_equals_sorted_scene_bitwise(loss):
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 3)
    sh, _ = _shuffled(sc, 3)
    code = F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2
    with G.make_problem(sc) as a, G.make_problem(sh) as b:
        a.set_ea_loss(code)
        b.set_ea_loss(code)
        for k in range(3):
            p = perturbed_params_ea(sc, 30 + k).astype(np.float32)
            La, ga = _loss_grad(a, p)
            Lb, gb = _loss_grad(b, p)
            assert La == Lb and np.array_equal(ga, gb), (loss, k)
        # and the oracle on the shuffled inputs
        Lo, go = G.ea_oracle(sh, p, loss)
        assert abs(Lb - Lo) <= 1e-5 * Lo
        if loss == "l2":
            assert G.rel_err(gb.reshape(go.shape), go) < 1e-4


def test_shuffled_scene_without_tracks_matches_the_oracle():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 4)
    sh, _ = _shuffled(sc, 4, tracks=False)
    with G.make_problem(sh) as pr:
        pr.set_ea_loss(F.FM_EA_L2)
        p = perturbed_params_ea(sc, 40).astype(np.float32)
        L, g = _loss_grad(pr, p)
    Lo, go = G.ea_oracle(sh, p, "l2")
    assert abs(L - Lo) <= 1e-5 * Lo
    assert G.rel_err(g.reshape(go.shape), go) < 1e-4


def test_weights_in_the_callers_order():
    """Weights given in the shuffled order land on the same keypoint pairs:
    the loss equals the sorted problem's with the same weights moved along,
    bit for bit, and fm_ea_get_weights gives back the caller's array."""
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 5)
    sh, q = _shuffled(sc, 5)
    rng = np.random.default_rng(5)
    w_sorted = rng.uniform(0.2, 3.0, size=sc.n_kp).astype(np.float32)
    w_sh = w_sorted[q]                      # caller order of the shuffled scene
    inv_z = np.float32(1.0 / sc.n_kp)
    with G.make_problem(sc) as a, G.make_problem(sh) as b:
        for pr, w in ((a, w_sorted), (b, w_sh)):
            pr.set_ea_loss(F.FM_EA_L1)
            pr.set_ea_weights(w, inv_z)
        p = perturbed_params_ea(sc, 50).astype(np.float32)
        La, ga = _loss_grad(a, p)
        Lb, gb = _loss_grad(b, p)
        assert La == Lb and np.array_equal(ga, gb)
        back, _ = b.get_weights()
        assert np.array_equal(back.cpu().numpy(), w_sh)
        # host and device buffers alike
        import torch
        b.set_ea_weights(torch.from_numpy(w_sh).cuda(), inv_z)
        assert np.array_equal(b.get_weights()[0].cpu().numpy(), w_sh)
        # the IRLS reweighting writes weights in the internal order; read back,
        # they are the caller's view of the same pairs
        for pr in (a, b):
            pr.set_params(F.FM_STAGE_EPIPOLAR, p.reshape(-1))
            pr.reweight(0.05, 1e-5)
        wa = a.get_weights()[0].cpu().numpy()
        wb = b.get_weights()[0].cpu().numpy()
        assert np.array_equal(wb, wa[q])


def test_shuffled_scene_triangulates_the_same_points():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 6)
    sh, _ = _shuffled(sc, 6)
    p = perturbed_params_ea(sc, 60, sigma_rot=1e-4, sigma_t=1e-4).astype(np.float32)
    out = []
    for s in (sc, sh):
        with G.make_problem(s) as pr:
            pr.set_params(F.FM_STAGE_EPIPOLAR, p.reshape(-1))
            out.append(pr.triangulate(4.0, 2.0))
    for x, y in zip(out[0], out[1]):
        assert np.array_equal(x, y)
    assert out[1][1].sum() > 0.3 * len(out[1][1])   # (parity with the oracle: test_gpu_setup.py)
