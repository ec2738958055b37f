"""GPU parity of the rotation stage (Eqs. 3-4), the translation stage (Eqs. 5-6,
batched initialisation runs) and the Adam steps of all three stages against the
FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import epipolar as ep
from oracle import rotation as rot
from oracle import translation as trn
from oracle.adam import Adam
from oracle.so3 import rot_from_6d
from synthetic.scenes import gt_relative_poses
from tests import _gpu as G
from tests._util import gt_params6, perturbed_params_ea, scene

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _torch():
    import torch
    return torch


def _rot_inputs(seed):
    sc = scene("c1", seed)
    Rij, tij = gt_relative_poses(sc, rot_noise_deg=2.0, dir_noise_deg=2.0, seed=seed)
    return sc, Rij.astype(np.float32), tij.astype(np.float32)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rotation_loss_grad(seed):
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    sc, Rij, tij = _rot_inputs(seed)
    rng = np.random.default_rng(seed)
    with G.make_problem(sc, rel_R=Rij, rel_t=tij) as pr:
        for k in range(4):
            p = (gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6))).astype(np.float32)
            L, g = pr.loss_grad(F.FM_STAGE_ROTATION, torch.from_numpy(p.reshape(-1)).cuda())
            Lo, go = rot.loss_grad(G.f32(p), sc.pair_i, sc.pair_j, G.f32(Rij))
            assert abs(L - Lo) <= LOSS_TOL * Lo, (L, Lo)
            assert G.rel_err(g.cpu().numpy().reshape(go.shape), go) < GRAD_TOL


def test_rotation_near_zero_distance():
    """Noise-free relative rotations at ground truth: every pair distance is
    ~0; the float32 kernel must still return a loss at the float32 rounding
    level (the arccos form would return ~1e-3 there)."""
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 3)
    Rij, tij = gt_relative_poses(sc)
    with G.make_problem(sc, rel_R=Rij.astype(np.float32), rel_t=tij.astype(np.float32)) as pr:
        p = gt_params6(sc).astype(np.float32)
        L, g = pr.loss_grad(F.FM_STAGE_ROTATION, torch.from_numpy(p.reshape(-1)).cuda())
    assert L < 1e-6
    assert torch.isfinite(g).all()


@pytest.mark.parametrize("runs", [1, 4])
def test_translation_loss_grad(runs):
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    sc, Rij, tij = _rot_inputs(4)
    rot6 = gt_params6(sc).astype(np.float32)
    rng = np.random.default_rng(4)
    o = np.stack([sc.centers_gt + rng.normal(0, 0.3, size=(sc.n_cams, 3)) for _ in range(runs)]).astype(np.float32)
    with G.make_problem(sc, rel_R=Rij, rel_t=tij) as pr:
        pr.set_params(F.FM_STAGE_ROTATION, rot6.reshape(-1))
        pr.set_translation_runs(runs)
        L, g = pr.loss_grad(F.FM_STAGE_TRANSLATION, torch.from_numpy(o.reshape(-1)).cuda())
    L = np.atleast_1d(L)
    g = g.cpu().numpy().reshape(runs, sc.n_cams, 3)
    tgt = trn.targets(rot_from_6d(G.f32(rot6)), sc.pair_j, G.f32(tij))
    for r in range(runs):
        Lo, go = trn.loss_grad(G.f32(o[r]), sc.pair_i, sc.pair_j, tgt)
        assert abs(L[r] - Lo) <= LOSS_TOL * Lo
        assert G.rel_err(g[r], go) < GRAD_TOL


def test_translation_needs_rotation_state():
    from paper_2505_04612_b300 import fastmap as F
    sc, Rij, tij = _rot_inputs(5)
    with G.make_problem(sc, rel_R=Rij, rel_t=tij) as pr:
        with pytest.raises(F.FastMapError) as e:
            pr.loss_grad(F.FM_STAGE_TRANSLATION, np.zeros(3 * sc.n_cams, np.float32))
        assert e.value.status == F.FM_ERR_STATE


# --------------------------------------------------------------- Adam steps

def _adam_compare(pr, stage, p0, oracle_grad, lr, n_steps, atol):
    from paper_2505_04612_b300 import fastmap as F
    pr.set_params(stage, p0.reshape(-1))
    pr.step(stage, n_steps, lr)
    got = pr.get_params(stage).cpu().numpy().astype(np.float64).reshape(p0.shape)
    opt = Adam(p0.shape, lr=lr)
    x = G.f32(p0)
    for _ in range(n_steps):
        x = opt.step(x, oracle_grad(x))
    err = np.max(np.abs(got - x))
    assert err < atol, err
    assert np.max(np.abs(got - G.f32(p0))) > 0.5 * lr   # it moved


def test_adam_epipolar():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 6)
    xs = G.oracle_xs(sc)
    p0 = perturbed_params_ea(sc, 6).astype(np.float32)
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_L2)

        def og(x):
            return ep.direct_loss_grad(x, sc.pair_i, sc.pair_j, xs[0], xs[1], sc.kp_img_pair, loss="l2")[1]
        _adam_compare(pr, F.FM_STAGE_EPIPOLAR, p0, og, lr=1e-3, n_steps=5, atol=5e-6)


def test_adam_rotation():
    from paper_2505_04612_b300 import fastmap as F
    sc, Rij, tij = _rot_inputs(7)
    rng = np.random.default_rng(7)
    p0 = (gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6))).astype(np.float32)
    with G.make_problem(sc, rel_R=Rij, rel_t=tij) as pr:
        _adam_compare(pr, F.FM_STAGE_ROTATION, p0,
                      lambda x: rot.loss_grad(x, sc.pair_i, sc.pair_j, G.f32(Rij))[1], lr=1e-3, n_steps=5,
                      atol=5e-6)


def test_adam_translation():
    from paper_2505_04612_b300 import fastmap as F
    sc, Rij, tij = _rot_inputs(8)
    rot6 = gt_params6(sc).astype(np.float32)
    rng = np.random.default_rng(8)
    o0 = (sc.centers_gt + rng.normal(0, 0.3, size=(sc.n_cams, 3))).astype(np.float32)
    tgt = trn.targets(rot_from_6d(G.f32(rot6)), sc.pair_j, G.f32(tij))
    with G.make_problem(sc, rel_R=Rij, rel_t=tij) as pr:
        pr.set_params(F.FM_STAGE_ROTATION, rot6.reshape(-1))
        _adam_compare(pr, F.FM_STAGE_TRANSLATION, o0,
                      lambda x: trn.loss_grad(x, sc.pair_i, sc.pair_j, tgt)[1], lr=1e-2, n_steps=5, atol=5e-5)


def test_loss_trace_and_timing():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 9)
    p0 = perturbed_params_ea(sc, 9).astype(np.float32)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, p0.reshape(-1))
        pr.track_loss(1, 16)
        pr.timing(True)
        last = pr.step(F.FM_STAGE_EPIPOLAR, 20, 1e-4, want_loss=True)
        hist = pr.loss_history(16)
        kt = pr.timing_read()
    assert len(hist) == 16 and hist[-1] == last
    assert hist[-1] < hist[0]
    assert kt["k_ea_direct"][0] == 20 and kt["k_ea_direct"][1] > 0
    # after the streaming kernel, one launch: the image pairs' chain rule, the
    # cameras' Adam update and the loss (trace and returned value alike)
    assert kt["k_cam_ea"][0] == 20 and kt["k_ea_tables"][0] == 20
    assert not {"k_ea_segments", "k_cam", "k_sum_fixed"} & set(kt)


def test_rotation_and_translation_at_scale():
    """Both stages on a 600-camera scene (thousands of image pairs, up to a
    few hundred per camera) against the oracle; the translation stage with 4
    runs batched."""
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    from synthetic.scenes import make_scene
    sc = make_scene("c2", 8, n_cams=600, n_points=120000)
    Rij, tij = gt_relative_poses(sc, rot_noise_deg=2.0, dir_noise_deg=2.0, seed=8)
    Rij, tij = Rij.astype(np.float32), tij.astype(np.float32)
    rng = np.random.default_rng(8)
    p6 = (gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6))).astype(np.float32)
    runs = 4
    o = np.stack([sc.centers_gt + rng.normal(0, 0.3, size=(sc.n_cams, 3)) for _ in range(runs)]).astype(np.float32)
    with G.make_problem(sc, rel_R=Rij, rel_t=tij) as pr:
        L, g = pr.loss_grad(F.FM_STAGE_ROTATION, torch.from_numpy(p6.reshape(-1)).cuda())
        Lo, go = rot.loss_grad(G.f32(p6), sc.pair_i, sc.pair_j, G.f32(Rij))
        assert abs(L - Lo) <= LOSS_TOL * Lo, (L, Lo)
        assert G.rel_err(g.cpu().numpy().reshape(go.shape), go) < GRAD_TOL
        pr.set_params(F.FM_STAGE_ROTATION, p6.reshape(-1))
        pr.set_translation_runs(runs)
        Lt, gt = pr.loss_grad(F.FM_STAGE_TRANSLATION, torch.from_numpy(o.reshape(-1)).cuda())
    Lt = np.atleast_1d(Lt)
    gt = gt.cpu().numpy().reshape(runs, sc.n_cams, 3)
    tgt = trn.targets(rot_from_6d(G.f32(p6)), sc.pair_j, G.f32(tij))
    for r in range(runs):
        Lo, go = trn.loss_grad(G.f32(o[r]), sc.pair_i, sc.pair_j, tgt)
        assert abs(Lt[r] - Lo) <= LOSS_TOL * Lo
        assert G.rel_err(gt[r], go) < GRAD_TOL
