"""Several independent scenes in one problem (scene_cam_off): every loss is
the scene's own and every kernel touches a scene's cameras and image pairs
only, so a batch must give each scene what solving it alone gives.  The
rotation and translation stages, the IRLS/compact epipolar path and the whole
fm_solve do the same float32 operations per element in the same order
whether batched or not (checked bit for bit); the direct epipolar kernel
splits a batch into warp runs at other places than a scene alone, so its
sums are compared within the parity tolerance, and against the oracle."""
import numpy as np
import pytest

from synthetic.scenes import concat_scenes, gt_relative_poses, make_scene
from tests import _gpu as G
from tests._util import gt_params6, perturbed_params_ea

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _F():
    from paper_2505_04612_b300 import fastmap as F
    return F


def _scenes():
    # uneven sizes: two c1 scenes, a small and a larger c2-geometry scene
    return [make_scene("c1", 0), make_scene("c1", 3, n_points=900),
            make_scene("c2", 1, n_cams=24, n_points=4000), make_scene("c2", 2, n_cams=60, n_points=12000)]


def _rel(scenes, noise=1.0):
    R, t = [], []
    for k, sc in enumerate(scenes):
        a, b = gt_relative_poses(sc, rot_noise_deg=noise, dir_noise_deg=noise, seed=k)
        R.append(a.astype(np.float32))
        t.append(b.astype(np.float32))
    return R, t


def _cat_params(per_scene):
    return np.concatenate([np.asarray(p, np.float32).reshape(-1) for p in per_scene])


def _split(x, scenes, dim):
    out, o = [], 0
    for sc in scenes:
        out.append(x[o:o + dim * sc.n_cams])
        o += dim * sc.n_cams
    return out


def test_invalid_batches_are_rejected():
    F = _F()
    scenes = _scenes()[:2]
    b = concat_scenes(scenes)
    bad = b.scene_cam_off.copy()
    bad[1] += 1                                   # the first scene's last pair now crosses scenes
    b.scene_cam_off = bad
    with pytest.raises(F.FastMapError) as e:
        G.make_problem(b)
    assert e.value.status == F.FM_ERR_INVALID_ARG
    b = concat_scenes(scenes)
    b.scene_cam_off = np.array([0, 2, b.n_cams], np.int32)   # image pairs of cameras 0-1 with others cross
    with pytest.raises(F.FastMapError):
        G.make_problem(b)
    b = concat_scenes(scenes)
    b.scene_cam_off = np.array([0, 5, b.n_cams - 1], np.int32)   # does not end at n_cams
    with pytest.raises(F.FastMapError):
        G.make_problem(b)


def test_rotation_and_translation_stages_bitwise():
    """Loss per scene and gradient of the rotation and translation stages,
    and ten Adam steps of each, equal the per-scene results bit for bit."""
    import torch
    F = _F()
    scenes = _scenes()
    b = concat_scenes(scenes)
    R, t = _rel(scenes)
    rng = np.random.default_rng(0)
    p6 = [gt_params6(sc) + rng.normal(0, 0.05, size=(sc.n_cams, 6)) for sc in scenes]
    o = [sc.centers_gt + rng.normal(0, 0.3, size=(sc.n_cams, 3)) for sc in scenes]
    with G.make_problem(b, rel_R=np.concatenate(R), rel_t=np.concatenate(t)) as pb:
        assert pb.info().n_scenes == len(scenes)
        Lb, gb = pb.loss_grad(F.FM_STAGE_ROTATION, torch.from_numpy(_cat_params(p6)).cuda())
        pb.set_params(F.FM_STAGE_ROTATION, torch.from_numpy(_cat_params(p6)).cuda())
        pb.step(F.FM_STAGE_ROTATION, 10, lr=1e-3)
        rb = pb.get_params(F.FM_STAGE_ROTATION).cpu().numpy()
        Ltb, gtb = pb.loss_grad(F.FM_STAGE_TRANSLATION, torch.from_numpy(_cat_params(o)).cuda())
        gb, gtb = gb.cpu().numpy(), gtb.cpu().numpy()
    for k, sc in enumerate(scenes):
        with G.make_problem(sc, rel_R=R[k], rel_t=t[k]) as ps:
            L, g = ps.loss_grad(F.FM_STAGE_ROTATION, torch.from_numpy(_cat_params([p6[k]])).cuda())
            assert L == Lb[k]
            np.testing.assert_array_equal(g.cpu().numpy(), _split(gb, scenes, 6)[k])
            ps.set_params(F.FM_STAGE_ROTATION, torch.from_numpy(_cat_params([p6[k]])).cuda())
            ps.step(F.FM_STAGE_ROTATION, 10, lr=1e-3)
            np.testing.assert_array_equal(ps.get_params(F.FM_STAGE_ROTATION).cpu().numpy(),
                                          _split(rb, scenes, 6)[k])
            Lt, gt = ps.loss_grad(F.FM_STAGE_TRANSLATION, torch.from_numpy(_cat_params([o[k]])).cuda())
            assert Lt == Ltb[k]
            np.testing.assert_array_equal(gt.cpu().numpy(), _split(gtb, scenes, 3)[k])


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_direct_epipolar_per_scene(loss):
    """Direct epipolar loss and gradient of a batch: each scene's loss and
    gradient match the scene alone and the oracle (L1 up to sign-ambiguous
    pairs, as in the single-scene parity tests)."""
    import torch
    F = _F()
    scenes = _scenes()
    b = concat_scenes(scenes)
    ps = [perturbed_params_ea(sc, 3 + k) for k, sc in enumerate(scenes)]
    with G.make_problem(b) as pb:
        pb.set_ea_loss(F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2)
        Lb, gb = pb.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(_cat_params(ps)).cuda())
        gb = gb.cpu().numpy().astype(np.float64)
    for k, sc in enumerate(scenes):
        g = _split(gb, scenes, 9)[k]
        Lo, go = G.ea_oracle(sc, ps[k], loss)
        assert abs(Lb[k] - Lo) <= LOSS_TOL * abs(Lo)
        if loss == "l2":
            assert G.rel_err(g.reshape(go.shape), go) < GRAD_TOL
        else:
            res = G.l1_grad_matches(sc, ps[k], g, GRAD_TOL)
            if res is not None:
                assert res[0], res
        with G.make_problem(sc) as p1:
            p1.set_ea_loss(F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2)
            L1, g1 = p1.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(_cat_params([ps[k]])).cuda())
        assert abs(Lb[k] - L1) <= 1e-6 * abs(L1)
        assert G.rel_err(g, g1.cpu().numpy()) < 1e-5


def test_reweight_and_compact_bitwise():
    """IRLS reweighting counts kept pairs per scene; the compact steps that
    follow equal the per-scene ones bit for bit."""
    import torch
    F = _F()
    scenes = _scenes()
    b = concat_scenes(scenes)
    ps = [perturbed_params_ea(sc, k, sigma_rot=0.002, sigma_t=0.002) for k, sc in enumerate(scenes)]
    with G.make_problem(b) as pb:
        pb.set_params(F.FM_STAGE_EPIPOLAR, torch.from_numpy(_cat_params(ps)).cuda())
        kept_b = pb.reweight(0.02, 1e-5)
        pb.set_ea_loss(F.FM_EA_COMPACT)
        Lb = pb.step(F.FM_STAGE_EPIPOLAR, 20, lr=1e-4, want_loss=True)
        eb = pb.get_params(F.FM_STAGE_EPIPOLAR).cpu().numpy()
    kept = 0
    for k, sc in enumerate(scenes):
        with G.make_problem(sc) as p1:
            p1.set_params(F.FM_STAGE_EPIPOLAR, torch.from_numpy(_cat_params([ps[k]])).cuda())
            kept += p1.reweight(0.02, 1e-5)
            p1.set_ea_loss(F.FM_EA_COMPACT)
            L1 = p1.step(F.FM_STAGE_EPIPOLAR, 20, lr=1e-4, want_loss=True)
            assert L1 == Lb[k]
            np.testing.assert_array_equal(p1.get_params(F.FM_STAGE_EPIPOLAR).cpu().numpy(),
                                          _split(eb, scenes, 9)[k])
    assert kept == kept_b


def test_solve_batch_equals_solves_one_at_a_time():
    """fm_solve on a batch returns, per scene, the poses and points of
    fm_solve on the scene alone, bit for bit (fewer iterations than the
    defaults, to keep the test short)."""
    scenes = _scenes()
    b = concat_scenes(scenes)
    R, _ = _rel(scenes)
    opts = dict(rot_iters=200, trn_iters=200, trn_final_iters=100, ea_rounds=2, ea_iters=100)
    T = int(b.kp_track.max()) + 1
    with G.make_problem(b, rel_R=np.concatenate(R)) as pb:
        ob = pb.solve(n_tracks=T, **opts)
    toff = b.meta["track_off"]
    for k, sc in enumerate(scenes):
        c0, c1 = b.scene_cam_off[k], b.scene_cam_off[k + 1]
        with G.make_problem(sc, rel_R=R[k]) as p1:
            o1 = p1.solve(n_tracks=int(sc.kp_track.max()) + 1, **opts)
        np.testing.assert_array_equal(o1["cam_valid"], ob["cam_valid"][c0:c1])
        np.testing.assert_array_equal(o1["R"], ob["R"][c0:c1])
        np.testing.assert_array_equal(o1["t"], ob["t"][c0:c1])
        np.testing.assert_array_equal(o1["points"], ob["points"][toff[k]:toff[k + 1]])
        np.testing.assert_array_equal(o1["point_valid"], ob["point_valid"][toff[k]:toff[k + 1]])


def test_connectivity_filter_marks_the_largest_component():
    """A camera without image pairs and a two-camera island beside the main
    view graph: only the main component's cameras are valid (per scene in a
    batch)."""
    from synthetic.scenes import Scene
    sc = make_scene("c1", 0)
    N = sc.n_cams
    m = np.nonzero(sc.kp_img_pair == 0)[0]                 # reuse the first image pair's keypoints
    extra = Scene(name="x", seed=0, width=sc.width, height=sc.height,
                  focal=np.concatenate([sc.focal, sc.focal[:3]]), cx=np.concatenate([sc.cx, sc.cx[:3]]),
                  cy=np.concatenate([sc.cy, sc.cy[:3]]), R_gt=np.concatenate([sc.R_gt, sc.R_gt[:3]]),
                  t_gt=np.concatenate([sc.t_gt, sc.t_gt[:3]]), points=sc.points,
                  pair_i=np.concatenate([sc.pair_i, [N]]).astype(np.int32),
                  pair_j=np.concatenate([sc.pair_j, [N + 1]]).astype(np.int32),
                  kp_img_pair=np.concatenate([sc.kp_img_pair, np.full(len(m), sc.n_pairs)]).astype(np.int32),
                  kp1_px=np.concatenate([sc.kp1_px, sc.kp1_px[m]]), kp2_px=np.concatenate([sc.kp2_px, sc.kp2_px[m]]),
                  kp_track=np.concatenate([sc.kp_track, sc.kp_track[m]]).astype(np.int32),
                  kp_inlier=np.concatenate([sc.kp_inlier, sc.kp_inlier[m]]))
    Rij, _ = gt_relative_poses(sc, rot_noise_deg=0.5, seed=1)
    rel_R = np.concatenate([Rij, np.eye(3)[None]]).astype(np.float32)
    want = np.r_[np.ones(N, bool), np.zeros(3, bool)]
    opts = dict(rot_iters=100, trn_iters=100, trn_final_iters=50, ea_rounds=1, ea_iters=50)
    with G.make_problem(extra, rel_R=rel_R) as pr:
        assert pr.info().n_cams_connected == N
        out = pr.solve(**opts)
    np.testing.assert_array_equal(out["cam_valid"], want)
    b = concat_scenes([extra, make_scene("c1", 2)])
    with G.make_problem(b, rel_R=np.concatenate([rel_R, gt_relative_poses(make_scene("c1", 2))[0].astype(np.float32)])) as pr:
        assert pr.info().n_cams_connected == N + 20
        out = pr.solve(**opts)
    np.testing.assert_array_equal(out["cam_valid"], np.r_[want, np.ones(20, bool)])


def test_solve_reports_the_output_gauge_per_scene():
    """fm_solve's gauge, per scene: the first valid camera has R = I, the
    valid cameras' centres have centroid 0 and mean norm 1, and the points
    share the frame (in front of the cameras that see them)."""
    scenes = _scenes()
    b = concat_scenes(scenes)
    R, _ = _rel(scenes)
    T = int(b.kp_track.max()) + 1
    with G.make_problem(b, rel_R=np.concatenate(R)) as pb:
        out = pb.solve(n_tracks=T, rot_iters=200, trn_iters=200, trn_final_iters=100, ea_rounds=2, ea_iters=100)
    Rs = out["R"].astype(np.float64)
    c = -np.einsum("nba,nb->na", Rs, out["t"].astype(np.float64))
    for k in range(len(scenes)):
        c0, c1 = b.scene_cam_off[k], b.scene_cam_off[k + 1]
        valid = np.nonzero(out["cam_valid"][c0:c1])[0] + c0
        np.testing.assert_allclose(Rs[valid[0]], np.eye(3), atol=2e-6)
        cv = c[valid]
        np.testing.assert_allclose(cv.mean(0), 0.0, atol=2e-5)
        assert abs(np.mean(np.linalg.norm(cv, axis=1)) - 1.0) < 2e-5
    # points in the same frame: in front of the cameras that see them
    pts, ok = out["points"], out["point_valid"]
    assert ok.sum() > 0
    m = np.nonzero(ok[b.kp_track])[0][:2000]
    X = pts[b.kp_track[m]].astype(np.float64)
    ci = b.pair_i[b.kp_img_pair[m]]
    depth = np.einsum("nab,nb->na", Rs[ci], X)[:, 2] + out["t"].astype(np.float64)[ci, 2]
    assert np.mean(depth > 0) > 0.99


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_direct_adam_step_uses_the_start_parameters(loss):
    """One direct epipolar Adam step over 2,400 cameras: the camera pass runs
    in several waves of CTAs and updates the parameters in place while other
    CTAs still form their image pairs' chain rule, which must use the
    parameters the step started from.  With lr = 1 and eps = 1 the first Adam
    update is -g / (|g| + 1) (bias-corrected moments m = g, v = g^2), so a
    chain rule evaluated at partly updated parameters would move the result
    by ~1e-2 relative; the step must reproduce fm_loss_grad's gradient at the
    start within float32 rounding."""
    import torch
    F = _F()
    scenes = [make_scene("c2", 10 + k, n_cams=300, n_points=6000) for k in range(8)]
    b = concat_scenes(scenes)
    p0 = _cat_params([perturbed_params_ea(sc, 20 + k) for k, sc in enumerate(scenes)])
    with G.make_problem(b) as pr:
        assert b.n_cams == 2400
        pr.set_ea_loss(F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2)
        _, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(p0).cuda())
        g = g.cpu().numpy().astype(np.float64)
        pr.set_params(F.FM_STAGE_EPIPOLAR, torch.from_numpy(p0).cuda())
        pr.step(F.FM_STAGE_EPIPOLAR, 1, lr=1.0, beta1=0.9, beta2=0.999, eps=1.0)
        p1 = pr.get_params(F.FM_STAGE_EPIPOLAR).cpu().numpy().astype(np.float64)
    # Adam's first step in float64 from the float32 gradient
    m, v = 0.1 * g, 0.001 * g * g
    want = p0.astype(np.float64) - (m / 0.1) / (np.sqrt(v / 0.001) + 1.0)
    err = np.abs(p1 - want)
    scale = np.abs(p0.astype(np.float64) - want)
    assert np.all(err <= 1e-5 * scale + 2e-7 * (1.0 + np.abs(want))), float(np.max(err))
