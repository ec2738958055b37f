"""What the trained network gains over the method without it: trained on the
method's own converged solves of small synthetic scenes (the library's
trainer), the learned filter reaches a better rotation accuracy in one
epipolar round than the plain filter in five on a held-out scene; its kept
pairs are cleaner against the generator's inlier flags.  (Wall time is
measured by bench.py --config learned_c5, not asserted here: a timing
comparison on a shared machine is not a parity check.)"""
import time

import numpy as np
import pytest

from oracle.solve import centre_errors, rotation_errors_deg
from synthetic.scenes import concat_scenes, gt_relative_poses, scene_c2
from tests import _gpu as G

pytestmark = pytest.mark.gpu


def _train():
    import torch
    from paper_2505_04612_b300 import fastmap as F
    from paper_2505_04612_b300 import learned as Lm
    G.lib_ready()
    rng = np.random.default_rng(5)
    scs = [scene_c2(seed=3000 + k, n_cams=int(rng.integers(40, 70)), n_points=int(rng.integers(4000, 9000)),
                    outlier_frac=float(rng.uniform(0.05, 0.4))) for k in range(16)]
    Xs, ys = [], []
    for b in range(2):
        grp = scs[8 * b:8 * b + 8]
        R = np.concatenate([gt_relative_poses(s, rot_noise_deg=1.0, seed=k)[0] for k, s in enumerate(grp)])
        with F.problem_from_scene(concat_scenes(grp), rel_R=R.astype(np.float32)) as pr:
            X, y = Lm.training_rows(pr, keep_frac=0.5, seed=b)
        Xs.append(X)
        ys.append(y)
    X, y = torch.cat(Xs), torch.cat(ys)
    theta, losses = Lm.train(X, y, steps=600, batch=32768)
    return theta, losses, X, y


def _solve(sc, R, theta, learned, rounds):
    import torch
    from paper_2505_04612_b300 import fastmap as F
    with F.problem_from_scene(sc, rel_R=R) as pr:
        if learned:
            pr.mlp_set_params(theta)
        pr.solve(learned=int(learned), ea_rounds=rounds)            # warm-up
        torch.cuda.synchronize()
        t = time.perf_counter()
        out = pr.solve(learned=int(learned), ea_rounds=rounds)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t
        w, _ = pr.get_weights()
        keep = (w > 0).cpu().numpy()
    ok = out["cam_valid"]
    Rr = out["R"].astype(np.float64)
    c = -np.einsum("nba,nb->na", Rr, out["t"].astype(np.float64))
    scale = np.mean(np.linalg.norm(sc.centers_gt[ok] - sc.centers_gt[ok].mean(0), axis=1))
    return dict(time=dt, rot=float(rotation_errors_deg(Rr[ok], sc.R_gt[ok]).mean()),
                ctr=float(centre_errors(c[ok], sc.centers_gt[ok]).mean() / scale),
                precision=float(sc.kp_inlier[keep].mean()))


def test_learned_filter_gains_over_the_plain_one():
    from paper_2505_04612_b300 import learned as Lm
    theta, losses, X, y = _train()
    assert losses[-1] < 0.6 * losses[0]
    acc = float(((Lm.logits(theta, X) >= 0).float() == y).float().mean())
    assert acc > 0.9, acc
    sc = scene_c2(seed=4242, n_cams=150, n_points=40000, outlier_frac=0.15)
    R = gt_relative_poses(sc, rot_noise_deg=1.0, seed=9)[0].astype(np.float32)
    plain = _solve(sc, R, theta, learned=False, rounds=5)
    learned = _solve(sc, R, theta, learned=True, rounds=1)
    assert learned["rot"] < plain["rot"], (learned, plain)
    assert learned["ctr"] < 1.25 * plain["ctr"] + 0.01, (learned, plain)
    assert learned["precision"] > plain["precision"] - 0.005, (learned, plain)
