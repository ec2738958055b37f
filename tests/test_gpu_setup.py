"""GPU parity of the setup steps -- rotation initialisation (Eqs. 10-14),
relative-translation grid search (Appendix "Relative Translation"),
multi-run merge (Appendix "Multiple Initializations"), triangulation
(Appendix "Sparse Reconstruction") -- and of the end-to-end solve, against
the FP64 oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import relpose as rp
from oracle import rotation as rot
from oracle import solve as S
from oracle import translation as trn
from oracle import triangulation as tri
from oracle.so3 import rot_from_6d
from synthetic.scenes import gt_relative_poses, make_scene
from tests import _gpu as G
from tests import _tri_cases as TC
from tests._util import clean_scene, gt_params6, perturbed_params_ea, scene

pytestmark = pytest.mark.gpu


def _rot6_to_R(p):
    return rot_from_6d(G.f32(p).reshape(-1, 6))


def _aligned_err_deg(A, B):
    """Per-camera angle between A and B after the best global right-alignment."""
    return S.rotation_errors_deg(A, B)


@pytest.mark.parametrize("noise", [0.0, 1.0])
def test_rotation_init_matches_oracle(noise):
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 0)
    Rij, tij = gt_relative_poses(sc, rot_noise_deg=noise, seed=1)
    Rij32 = Rij.astype(np.float32)
    with G.make_problem(sc, rel_R=Rij32) as pr:
        pr.rotation_init(2000)
        Rg = _rot6_to_R(pr.get_params(F.FM_STAGE_ROTATION).cpu().numpy())
    Ro = rot.martinec_init(sc.n_cams, sc.pair_i, sc.pair_j, G.f32(Rij32))
    assert np.allclose(np.linalg.det(Rg), 1.0, atol=1e-5)
    err = _aligned_err_deg(Rg, Ro)
    assert err.max() < 0.05, err.max()
    if noise == 0.0:
        assert _aligned_err_deg(Rg, sc.R_gt).max() < 2e-3


def test_relative_translations_are_valid_grid_minima():
    """The float32 argmin may pick a different lattice point than the oracle
    where two candidates tie to rounding; every choice must then have the
    oracle's minimum error (to float32 rounding) and the same sign."""
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 1)
    x1, x2 = G.oracle_xs(sc)
    p6 = gt_params6(sc).astype(np.float32)
    R = _rot6_to_R(p6)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_ROTATION, p6.reshape(-1))
        err_g = pr.relative_translations()
        _, t_g = pr.get_rel_poses(want_R=False)
    off = sc.seg_off()
    for n in range(sc.n_pairs):
        s = slice(off[n], off[n + 1])
        Rij = R[sc.pair_j[n]] @ R[sc.pair_i[n]].T
        t_o, e_o = rp.relative_translation(Rij, x1[s], x2[s])
        tg = G.f32(t_g[n])
        e_g = rp.mean_epipolar_error(tg[None], Rij, x1[s], x2[s])[0]
        assert e_g <= e_o * (1 + 1e-3) + 1e-7, (n, e_g, e_o)
        assert abs(err_g[n] - e_g) <= 1e-4 * e_g + 1e-7
        c_p = rp.cheirality_count(Rij, tg, x1[s], x2[s])
        c_m = rp.cheirality_count(Rij, -tg, x1[s], x2[s])
        assert c_p >= c_m


def test_translation_merge_matches_oracle():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 2)
    _, tij = gt_relative_poses(sc, dir_noise_deg=2.0, seed=2)
    p6 = gt_params6(sc).astype(np.float32)
    rng = np.random.default_rng(2)
    runs = np.stack([sc.centers_gt + rng.normal(0, s, size=(sc.n_cams, 3)) for s in (0.05, 1.0, 0.2, 2.0)])
    runs = runs.astype(np.float32)
    runs[0, :4] += 3.0                       # run 0 is wrong on cameras 0-3
    with G.make_problem(sc, rel_t=tij.astype(np.float32)) as pr:
        pr.set_params(F.FM_STAGE_ROTATION, p6.reshape(-1))
        pr.set_translation_runs(4)
        pr.set_params(F.FM_STAGE_TRANSLATION, runs.reshape(-1))
        best_g = pr.translation_merge()
        merged_g = pr.get_params(F.FM_STAGE_TRANSLATION).cpu().numpy().reshape(-1, 3)
    tgt = trn.targets(_rot6_to_R(p6), sc.pair_j, G.f32(tij.astype(np.float32)))
    merged_o, best_o = trn.merge_runs(G.f32(runs), sc.pair_i, sc.pair_j, tgt)
    # the per-camera choice is an argmin over run losses: compare where it is clear
    scores = np.stack([trn.camera_mean_loss(trn.normalise_run(G.f32(runs[k])), sc.pair_i, sc.pair_j, tgt, sc.n_cams)
                       for k in range(4)])
    srt = np.sort(scores, axis=0)
    clear = (srt[1] - srt[0]) > 1e-5
    assert np.array_equal(best_g[clear], best_o[clear])
    assert np.max(np.abs(merged_g[clear] - merged_o[clear])) < 1e-5


def _tri_params(sc):
    return np.concatenate([sc.R_gt[:, :, 0], sc.R_gt[:, :, 1], sc.t_gt], axis=1).astype(np.float32)


def test_triangulation_matches_oracle():
    """Points within float32 rounding; every keep flag and inlier-camera count
    equal to the oracle's except on tracks where a decision lies within
    rounding of its threshold (an observation's reprojection error within the
    float32 point error of max_err_px, a pair's rays at the parallel threshold,
    the largest angle within rounding of min_angle), which are enumerated."""
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 3)
    x1, x2 = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 3, sigma_rot=1e-4, sigma_t=1e-4).astype(np.float32)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, p.reshape(-1))
        pts_g, valid_g, ncam_g = pr.triangulate(4.0, 2.0)
    pp = G.f32(p)
    R = rot_from_6d(pp[:, :6])
    t = pp[:, 6:]
    T = int(sc.kp_track.max()) + 1
    pts_o, valid_o, ncam_o, d = tri.triangulate(R, t, sc.pair_i, sc.pair_j, sc.kp_img_pair, x1, x2,
                                                sc.kp_track, T, G.f32(sc.focal), 4.0, 2.0, diag=True)
    assert len(valid_g) == T
    seen = np.bincount(sc.kp_track, minlength=T) > 0
    scale = np.max(np.abs(pts_o[seen]))
    dP = np.linalg.norm(pts_g.astype(np.float64) - pts_o, axis=1)
    assert np.max(dP[seen]) < 1e-4 * scale
    # decision margins: an error moves by at most ~ f |dP| / depth, an angle by
    # (1/|r1| + 1/|r2|) |dP| (factor 4 of slack), plus float32 rounding of the
    # quantity itself
    tr = sc.kp_track
    ci, cj = sc.pair_i[sc.kp_img_pair], sc.pair_j[sc.kp_img_pair]
    o = -np.einsum("nba,nb->na", R, t)
    zi = np.einsum("mab,mb->ma", R[ci], pts_o[tr])[:, 2] + t[ci, 2]
    zj = np.einsum("mab,mb->ma", R[cj], pts_o[tr])[:, 2] + t[cj, 2]
    f = G.f32(sc.focal)
    be1 = 4.0 * f[ci] * dP[tr] / np.maximum(np.abs(zi), 1e-6) + 1e-3
    be2 = 4.0 * f[cj] * dP[tr] / np.maximum(np.abs(zj), 1e-6) + 1e-3
    amb_obs = (np.abs(d["err1"] - 4.0) < be1) | (np.abs(d["err2"] - 4.0) < be2)
    amb_par = np.abs(d["pair_sin2"] - tri.PARALLEL_SIN2) < 1e-8
    inv_r = 1.0 / np.linalg.norm(o[ci] - pts_o[tr], axis=1) + 1.0 / np.linalg.norm(o[cj] - pts_o[tr], axis=1)
    band_a = np.degrees(4.0 * inv_r * dP[tr]) + 1e-3
    amb_track = np.zeros(T, bool)
    np.logical_or.at(amb_track, tr, amb_obs | amb_par)
    worst_band = np.zeros(T)
    np.maximum.at(worst_band, tr, band_a)
    amb_track |= np.abs(d["max_angle_deg"] - 2.0) < worst_band
    check = seen & ~amb_track
    assert check.sum() > 0.99 * seen.sum(), (int(seen.sum()), int(check.sum()))
    bad = np.nonzero(check & ((valid_g != valid_o) | (ncam_g != ncam_o)))[0]
    assert len(bad) == 0, [(int(k), bool(valid_g[k]), bool(valid_o[k]), int(ncam_g[k]), int(ncam_o[k]))
                           for k in bad[:10]]


@pytest.mark.parametrize("case", range(len(TC.all_cases())))
def test_triangulation_hand_built_tracks(case):
    """The hand-built tracks of the oracle's pins through the C ABI: the
    displaced observation is measured in its own camera's pixels, the
    3-camera rule counts distinct cameras, the angle rule uses only pairs of
    two inlier keypoints, and exactly parallel rays give no point."""
    from paper_2505_04612_b300 import fastmap as F
    sc, want_valid, want_ncam = TC.all_cases()[case]
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, _tri_params(sc).reshape(-1))
        pts_g, valid_g, ncam_g = pr.triangulate(4.0, 2.0)
    assert len(valid_g) == 1
    assert np.max(np.abs(pts_g[0])) < 1e-5, pts_g
    assert bool(valid_g[0]) == want_valid and int(ncam_g[0]) == want_ncam, (sc.name, valid_g, ncam_g)


def test_random_translation_starts_match_the_oracle_hash():
    """fm_translation_random_init draws the same counter-based values as the
    oracle's hash_uniform (itself pinned by published vectors), bit for bit."""
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 0)
    with G.make_problem(sc) as pr:
        for runs, seed in ((1, 0), (4, 7), (3, 0xFFFFFFFF)):
            pr.set_translation_runs(runs)
            pr.translation_random_init(seed)
            got = pr.get_params(F.FM_STAGE_TRANSLATION).cpu().numpy().reshape(-1)
            want = S.hash_uniform(runs * sc.n_cams * 3, seed).astype(np.float32)
            assert np.array_equal(got, want), (runs, seed)


def test_solve_noise_free_recovers_ground_truth():
    sc = clean_scene(4)
    Rij, tij = gt_relative_poses(sc)
    T = int(sc.kp_track.max()) + 1
    with G.make_problem(sc, rel_R=Rij.astype(np.float32)) as pr:
        out = pr.solve(n_tracks=T)
    R = out["R"].astype(np.float64)
    c = -np.einsum("nba,nb->na", R, out["t"].astype(np.float64))
    assert S.rotation_errors_deg(R, sc.R_gt).max() < 0.05
    scale = np.mean(np.linalg.norm(sc.centers_gt - sc.centers_gt.mean(0), axis=1))
    assert S.centre_errors(c, sc.centers_gt).max() < 1e-2 * scale
    assert out["n_points_valid"] > 0.3 * T


def test_solve_matches_oracle_accuracy():
    """c1 with pixel noise and outliers: the float32 solve and the float64
    oracle solve follow the same algorithm; their final mean rotation errors
    against ground truth agree within 0.05 deg."""
    sc = scene("c1", 5)
    x1, x2 = G.oracle_xs(sc)
    Rij, tij = gt_relative_poses(sc, rot_noise_deg=1.0, seed=5)
    Rij32 = Rij.astype(np.float32)
    with G.make_problem(sc, rel_R=Rij32) as pr:
        out = pr.solve(n_tracks=int(sc.kp_track.max()) + 1)
    o = S.solve(sc.n_cams, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, G.f32(Rij32), None, G.f32(sc.focal),
                sc.kp_track, S.SolveOpts())
    e_g = S.rotation_errors_deg(out["R"].astype(np.float64), sc.R_gt).mean()
    e_o = S.rotation_errors_deg(o["R"], sc.R_gt).mean()
    assert abs(e_g - e_o) < 0.05, (e_g, e_o)


def test_relative_translations_leave_out_zero_weight_pairs():
    """With per-pair weights set, the grid search scores and signs each image
    pair on its pairs of positive weight only (all of them when none has one):
    every choice attains the oracle's minimum over the kept pairs."""
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 2)
    x1, x2 = G.oracle_xs(sc)
    p6 = gt_params6(sc).astype(np.float32)
    R = _rot6_to_R(p6)
    rng = np.random.default_rng(3)
    w = (rng.random(sc.n_kp) < 0.6).astype(np.float32)
    off = sc.seg_off()
    w[off[5]:off[6]] = 0.0                     # an image pair with nothing kept: all its pairs count
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_ROTATION, p6.reshape(-1))
        pr.set_ea_weights(w)
        err_g = pr.relative_translations()
        _, t_g = pr.get_rel_poses(want_R=False)
    for n in range(sc.n_pairs):
        idx = np.arange(off[n], off[n + 1])
        kept = idx[w[idx] > 0] if np.any(w[idx] > 0) else idx
        Rij = R[sc.pair_j[n]] @ R[sc.pair_i[n]].T
        t_o, e_o = rp.relative_translation(Rij, x1[kept], x2[kept])
        tg = G.f32(t_g[n])
        e_g = rp.mean_epipolar_error(tg[None], Rij, x1[kept], x2[kept])[0]
        assert e_g <= e_o * (1 + 1e-3) + 1e-7, (n, e_g, e_o)
        assert abs(err_g[n] - e_g) <= 1e-4 * e_g + 1e-7
        assert rp.cheirality_count(Rij, tg, x1[kept], x2[kept]) >= rp.cheirality_count(Rij, -tg, x1[kept], x2[kept])


@pytest.mark.parametrize("stage,override", [("rotation", {"rot_lr": 1e38}),
                                            ("translation", {"trn_lr": 1e38}),
                                            ("epipolar", {"ea_lr": 1e38})])
def test_solve_reports_divergence(stage, override):
    """A learning rate that drives a stage's parameters to overflow (Adam's
    first steps move each parameter by about lr) makes its final loss
    non-finite; fm_solve stops there with FM_ERR_NAN and names the
    stage (plain float arithmetic on the GPU: nothing faults)."""
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 1)
    Rij, tij = gt_relative_poses(sc, rot_noise_deg=1.0, seed=1)
    with G.make_problem(sc, rel_R=Rij.astype(np.float32), rel_t=tij.astype(np.float32)) as pr:
        with pytest.raises(F.FastMapError) as ei:
            pr.solve(rot_iters=40, trn_iters=40, trn_final_iters=20, ea_rounds=1, ea_iters=40, **override)
        assert ei.value.status == F.FM_ERR_NAN, str(ei.value)
        # the stage whose loss first goes non-finite: the overridden one, or a
        # later one (the translation loss compares directions, which stay
        # finite while the centres overflow together)
        later = {"rotation": ["rotation"], "translation": ["translation", "epipolar"],
                 "epipolar": ["epipolar"]}[stage]
        assert any(s + " stage" in str(ei.value) for s in later), str(ei.value)
        # the problem stays usable: a normal solve afterwards succeeds
        out = pr.solve(rot_iters=40, trn_iters=40, trn_final_iters=20, ea_rounds=1, ea_iters=40)
        assert np.all(np.isfinite(out["R"]))
