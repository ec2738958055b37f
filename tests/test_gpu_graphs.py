"""fm_step replays captured CUDA graphs of its iterations; the results must be
those of launching every kernel from the host, bit for bit, for every stage
(and across the events that change captured state: a new loss, new weights,
a new number of translation runs)."""
import numpy as np
import pytest

from synthetic.scenes import concat_scenes, gt_relative_poses, make_scene
from tests import _gpu as G
from tests._util import gt_params6, perturbed_params_ea

pytestmark = pytest.mark.gpu


def _run(sc, rel_R, rel_t, graphs):
    import torch
    from paper_2505_04612_b300 import fastmap as F
    out = {}
    rng = np.random.default_rng(1)
    with G.make_problem(sc, rel_R=rel_R, rel_t=rel_t) as pr:
        pr.graphs(graphs)
        p6 = (gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6))).astype(np.float32).reshape(-1)
        pr.set_params(F.FM_STAGE_ROTATION, torch.from_numpy(p6).cuda())
        out["rot_loss"] = pr.step(F.FM_STAGE_ROTATION, 50, lr=1e-3, want_loss=True)
        out["rot"] = pr.get_params(F.FM_STAGE_ROTATION).cpu().numpy()
        pr.set_translation_runs(3)
        pr.translation_random_init(7)
        out["trn_loss"] = pr.step(F.FM_STAGE_TRANSLATION, 40, lr=1e-2, want_loss=True)
        out["trn"] = pr.get_params(F.FM_STAGE_TRANSLATION).cpu().numpy()
        pe = perturbed_params_ea(sc, 2, sigma_rot=0.005, sigma_t=0.005).astype(np.float32).reshape(-1)
        pr.set_params(F.FM_STAGE_EPIPOLAR, torch.from_numpy(pe).cuda())
        pr.set_ea_loss(F.FM_EA_L1)
        pr.step(F.FM_STAGE_EPIPOLAR, 33, lr=1e-4)
        pr.reweight(0.05, 1e-5)
        pr.set_ea_loss(F.FM_EA_COMPACT)
        out["ea_loss"] = pr.step(F.FM_STAGE_EPIPOLAR, 37, lr=1e-4, want_loss=True)
        pr.set_ea_loss(F.FM_EA_L2)
        pr.step(F.FM_STAGE_EPIPOLAR, 20, lr=1e-4)
        out["ea"] = pr.get_params(F.FM_STAGE_EPIPOLAR).cpu().numpy()
        out["launches"] = {k: v[0] for k, v in pr.timing_read().items()}
    return out


@pytest.mark.parametrize("batch", [False, True])
def test_graph_replay_is_bitwise_identical(batch):
    scs = [make_scene("c1", 1), make_scene("c1", 2, n_points=800)] if batch else [make_scene("c1", 1)]
    sc = concat_scenes(scs) if batch else scs[0]
    rel = [gt_relative_poses(s, rot_noise_deg=0.5, dir_noise_deg=0.5, seed=3) for s in scs]
    rel_R = np.concatenate([r[0] for r in rel]).astype(np.float32)
    rel_t = np.concatenate([r[1] for r in rel]).astype(np.float32)
    a = _run(sc, rel_R, rel_t, graphs=True)
    b = _run(sc, rel_R, rel_t, graphs=False)
    for k in ["rot", "trn", "ea"]:
        np.testing.assert_array_equal(a[k], b[k], err_msg=k)
    for k in ["rot_loss", "trn_loss", "ea_loss"]:
        assert a[k] == b[k], k
    # the launch counters count the kernels of every replayed iteration
    assert a["launches"] == b["launches"]


def test_rotation_init_graph_is_bitwise_identical():
    from paper_2505_04612_b300 import fastmap as F
    sc = make_scene("c1", 6)
    Rij, _ = gt_relative_poses(sc, rot_noise_deg=2.0, seed=6)
    res = []
    for graphs in (True, False):
        with G.make_problem(sc, rel_R=Rij.astype(np.float32)) as pr:
            pr.graphs(graphs)
            pr.rotation_init(200)          # 6 replays of 32 iterations + 8 direct ones
            res.append(pr.get_params(F.FM_STAGE_ROTATION).cpu().numpy())
    np.testing.assert_array_equal(res[0], res[1])


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_weighted_direct_steps_repeatable(loss):
    """Weighted direct epipolar steps, launched kernel by kernel with
    programmatic dependent launch and replayed from graphs, give one result:
    a kernel that starts before its predecessor finishes reads the
    predecessor's output through L2, never through the read-only cache."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    sc = make_scene("c1", 1)
    pe = perturbed_params_ea(sc, 2, sigma_rot=0.005, sigma_t=0.005).astype(np.float32).reshape(-1)
    w = np.random.default_rng(0).uniform(0.5, 2.0, sc.n_kp).astype(np.float32)
    outs = []
    for graphs in (False, False, False, True):
        with G.make_problem(sc) as pr:
            pr.graphs(graphs)
            pr.set_params(F.FM_STAGE_EPIPOLAR, torch.from_numpy(pe).cuda())
            pr.set_ea_weights(w)
            pr.set_ea_loss(F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2)
            pr.step(F.FM_STAGE_EPIPOLAR, 20, lr=1e-4)
            outs.append(pr.get_params(F.FM_STAGE_EPIPOLAR).cpu().numpy())
    for o in outs[1:]:
        np.testing.assert_array_equal(o, outs[0])


def test_host_loss_grad_graph_is_bitwise_identical():
    """fm_loss_grad with host buffers runs directly on the first call at an
    epoch and through a captured graph afterwards: every call, for every
    stage and after every change of captured state (loss form, weights,
    translation runs), returns the bits of the device-buffer path."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    sc = make_scene("c1", 3)
    rel_R, rel_t = gt_relative_poses(sc, rot_noise_deg=0.5, dir_noise_deg=0.5, seed=5)
    rng = np.random.default_rng(2)
    p6 = (gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6))).astype(np.float32).reshape(-1)
    pe = perturbed_params_ea(sc, 4).astype(np.float32).reshape(-1)

    def same(pr, stage, host):
        dev = torch.from_numpy(host).cuda()
        Ld, gd = pr.loss_grad(stage, dev)
        for _ in range(4):   # direct, capture + replay, replays
            Lh, gh = pr.loss_grad(stage, host)
            np.testing.assert_array_equal(np.asarray(Lh), np.asarray(Ld))
            np.testing.assert_array_equal(gh, gd.cpu().numpy())
        Lg, _ = pr.loss_grad(stage, host, want_grad=False)   # loss only: another graph
        np.testing.assert_array_equal(np.asarray(Lg), np.asarray(Ld))

    with G.make_problem(sc, rel_R=rel_R.astype(np.float32), rel_t=rel_t.astype(np.float32)) as pr:
        same(pr, F.FM_STAGE_ROTATION, p6)
        same(pr, F.FM_STAGE_ROTATION, (p6 * 1.01).astype(np.float32))   # other parameters, same graph
        pr.set_params(F.FM_STAGE_ROTATION, torch.from_numpy(p6).cuda())
        pr.set_translation_runs(2)
        pr.translation_random_init(3)
        t = pr.get_params(F.FM_STAGE_TRANSLATION).cpu().numpy().reshape(-1)
        same(pr, F.FM_STAGE_TRANSLATION, t)
        pr.set_translation_runs(3)
        pr.translation_random_init(4)
        same(pr, F.FM_STAGE_TRANSLATION, pr.get_params(F.FM_STAGE_TRANSLATION).cpu().numpy().reshape(-1))
        for loss in (F.FM_EA_L1, F.FM_EA_L2):
            pr.set_ea_loss(loss)
            same(pr, F.FM_STAGE_EPIPOLAR, pe)
        pr.set_ea_weights(rng.uniform(0.0, 2.0, sc.n_kp).astype(np.float32))
        same(pr, F.FM_STAGE_EPIPOLAR, pe)
        pr.set_params(F.FM_STAGE_EPIPOLAR, torch.from_numpy(pe).cuda())
        pr.reweight(0.05, 1e-5)
        pr.set_ea_loss(F.FM_EA_COMPACT)
        same(pr, F.FM_STAGE_EPIPOLAR, pe)
