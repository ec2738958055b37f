"""Learned inlier weights on the GPU (tensor-core network, features, trainer)
against the FP64 oracle (oracle/mlp.py).  The network's products take
bfloat16 operands: the oracle reproduces the same roundings (quantise=True),
so what is left is float32 accumulation order, float32 erf/exp, and rare
bfloat16 rounding flips of values that sit next to a rounding boundary."""
import numpy as np
import pytest

from oracle import mlp as M
from oracle.adam import Adam
from synthetic.scenes import make_scene
from tests import _gpu as G
from tests._util import perturbed_params_ea

pytestmark = pytest.mark.gpu


def _mods():
    import torch
    from paper_2505_04612_b300 import fastmap as F
    return torch, F


def _batch(B, seed):
    rng = np.random.default_rng(seed)
    # feature ranges like the real ones: residual ratios, log distances, angles
    x = np.stack([rng.exponential(1.0, B), rng.exponential(0.8, B), rng.uniform(0.7, 1.8, B),
                  rng.uniform(0.0, 0.5, B), rng.uniform(0.0, 0.8, B), rng.uniform(0, 1, B),
                  rng.uniform(2, 8, B), rng.uniform(0, 1, B)], axis=1)
    y = (rng.random(B) < 0.7).astype(np.float64)
    return x, y


def _theta(seed):
    th = M.init_params(seed)
    th[M.N_PARAMS - 1] = 0.3
    rng = np.random.default_rng(seed + 1)
    P = M.unpack(th)
    P = {k: v.copy() for k, v in P.items()}
    P["b1"] += rng.normal(0, 0.1, 64)
    P["b2"] += rng.normal(0, 0.1, 64)
    return M.pack(P)


def _dev(a):
    torch, _ = _mods()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


@pytest.mark.parametrize("B", [1, 127, 128, 129, 1000, 20000, 100003])
def test_loss_and_gradient_match_the_oracle(B):
    """The tcgen05 training kernel: one row, a ragged tile, one full tile,
    one row past it, and more 128-row tiles than resident CTAs (the weight
    accumulators carried across a CTA's tiles in tensor memory)."""
    torch, F = _mods()
    G.lib_ready()
    x, y = _batch(B, B)
    th = _theta(B)
    x32 = x.astype(np.float32).astype(np.float64)
    th32 = th.astype(np.float32).astype(np.float64)
    Lo, go = M.loss_grad(th32, x32, y, quantise=True)
    tr = F.MlpTrainer(max(B, 64))
    tr.set_params(th)
    L, g = tr.loss_grad(_dev(x), _dev(y))
    L, g = float(L.item()), g.cpu().numpy().astype(np.float64)
    assert abs(L - Lo) <= 1e-5 * abs(Lo), (L, Lo)
    assert G.rel_err(g, go) < 1e-4, G.rel_err(g, go)
    # and the same numbers again (fixed-order reductions)
    L2, g2 = tr.loss_grad(_dev(x), _dev(y))
    assert float(L2.item()) == L
    np.testing.assert_array_equal(g2.cpu().numpy(), g.astype(np.float32))
    # the unquantised float64 gradient is within the bfloat16 error
    _, gf = M.loss_grad(th32, x32, y)
    assert G.rel_err(g, gf) < 3e-2
    tr.close()


def test_empty_batch_gives_zero_loss_and_gradient():
    torch, F = _mods()
    G.lib_ready()
    tr = F.MlpTrainer(64)
    tr.set_params(_theta(3))
    L, g = tr.loss_grad(_dev(np.zeros((0, 8))), _dev(np.zeros(0)))
    assert float(L.item()) == 0.0
    assert not g.cpu().numpy().any()
    tr.close()


@pytest.mark.parametrize("B", [1, 127, 128, 5000, 200003])
def test_forward_logits_match_the_oracle(B):
    """The tcgen05 forward pass: single rows, one ragged tile, one full tile,
    many tiles, and more tiles than resident CTAs (persistent loop)."""
    torch, F = _mods()
    G.lib_ready()
    x, _ = _batch(B, 7)
    th = _theta(11)
    tr = F.MlpTrainer(B)
    tr.set_params(th)
    o = tr.forward(_dev(x)).cpu().numpy().astype(np.float64)
    oq, _ = M.forward(th.astype(np.float32).astype(np.float64), x.astype(np.float32).astype(np.float64),
                      quantise=True)
    err = np.abs(o - oq)
    tol = 1e-4 * (1 + np.abs(oq))
    assert np.mean(err <= tol) > 0.995, np.mean(err <= tol)   # rare bfloat16 rounding flips
    assert err.max() < 2e-2
    tr.close()


def test_adam_step_matches_the_oracle_adam():
    torch, F = _mods()
    G.lib_ready()
    x, y = _batch(3000, 3)
    th = _theta(5).astype(np.float32)
    tr = F.MlpTrainer(3000)
    tr.set_params(th)
    _, g = tr.loss_grad(_dev(x), _dev(y))
    tr.step(_dev(x), _dev(y), lr=1e-3)
    th1 = tr.get_params().astype(np.float64)
    opt = Adam(th.shape, lr=1e-3)
    want = opt.step(th.astype(np.float64), g.cpu().numpy().astype(np.float64))
    np.testing.assert_allclose(th1, want, rtol=1e-6, atol=1e-7)
    tr.close()


def test_training_reduces_the_loss():
    torch, F = _mods()
    G.lib_ready()
    rng = np.random.default_rng(0)
    x, _ = _batch(20000, 8)
    y = (x[:, 0] + 0.3 * rng.normal(size=len(x)) < 1.0).astype(np.float64)   # learnable rule
    tr = F.MlpTrainer(20000)
    tr.set_params(M.init_params(1))
    xd, yd = _dev(x), _dev(y)
    L0 = float(tr.loss_grad(xd, yd)[0].item())
    for _ in range(200):
        tr.step(xd, yd, lr=3e-3)
    L1 = float(tr.loss_grad(xd, yd)[0].item())
    assert L1 < 0.6 * L0, (L0, L1)
    tr.close()


def test_features_residuals_and_probabilities_on_a_scene():
    torch, F = _mods()
    sc = make_scene("c1", 4)
    x1, x2 = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 6)
    w = np.random.default_rng(2).uniform(0.0, 100.0, sc.n_kp).astype(np.float32)
    th = _theta(21)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, _dev(p.reshape(-1)))
        pr.set_ea_weights(w)
        pr.mlp_set_params(th)
        feat, resid, prob = pr.mlp_eval(iter_frac=0.4, delta=1e-5, want_prob=True)
        feat, resid, prob = feat.cpu().numpy(), resid.cpu().numpy(), prob.cpu().numpy()
    fo, ro = M.features(G.f32(p), sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, G.f32(sc.focal), 0.4,
                        kp_track=sc.kp_track, weights=G.f32(w), delta=1e-5)
    np.testing.assert_allclose(resid, ro, rtol=1e-4, atol=2e-7)
    # float32 residuals carry an absolute error of ~1e-7: f0 and f1 inherit it
    np.testing.assert_allclose(feat[:, 0], fo[:, 0], rtol=1e-3, atol=2e-4)
    np.testing.assert_allclose(feat[:, 1], fo[:, 1], rtol=1e-3, atol=1e-4)
    np.testing.assert_allclose(feat[:, 2:], fo[:, 2:], rtol=1e-5, atol=2e-6)
    # the network on the GPU's own features
    o, _ = M.forward(th.astype(np.float32).astype(np.float64), feat.astype(np.float64), quantise=True)
    po = M.sigmoid(o)
    assert np.mean(np.abs(prob - po) < 1e-5) > 0.995
    assert np.abs(prob - po).max() < 5e-3


def test_learned_reweight_keeps_the_predicted_inliers():
    torch, F = _mods()
    sc = make_scene("c1", 5)
    x1, x2 = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 1, sigma_rot=0.002, sigma_t=0.002)
    th = _theta(31)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, _dev(p.reshape(-1)))
        pr.mlp_set_params(th)
        _, resid, prob = pr.mlp_eval(iter_frac=0.0, delta=1e-5, want_prob=True)
        kept = pr.mlp_reweight(0.0, delta=1e-5, p_min=0.5, irls=True)
        w, inv_z = pr.get_weights()
        prob, resid, w = prob.cpu().numpy(), resid.cpu().numpy(), w.cpu().numpy()
    keep = prob >= 0.5
    assert kept == int(keep.sum())
    np.testing.assert_array_equal(w[~keep], 0.0)
    np.testing.assert_allclose(w[keep], 1.0 / np.maximum(np.abs(resid[keep]), 1e-5), rtol=1e-6)
    assert abs(inv_z - 1.0 / max(kept, 1)) < 1e-9


def test_errors():
    torch, F = _mods()
    sc = make_scene("c1", 0)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, _dev(perturbed_params_ea(sc, 0).reshape(-1)))
        with pytest.raises(F.FastMapError) as e:
            pr.mlp_eval(want_prob=True)
        assert e.value.status == F.FM_ERR_STATE
        bad = _theta(1)
        bad[100] = np.nan
        with pytest.raises(F.FastMapError) as e:
            pr.mlp_set_params(bad)
        assert e.value.status == F.FM_ERR_NAN
        with pytest.raises(F.FastMapError) as e:
            pr.mlp_eval(iter_frac=1.5)
        assert e.value.status == F.FM_ERR_INVALID_ARG
    tr = F.MlpTrainer(10)
    x, y = _batch(11, 0)
    with pytest.raises(F.FastMapError) as e:
        tr.loss_grad(_dev(x), _dev(y))
    assert e.value.status == F.FM_ERR_INVALID_ARG
    tr.close()


def test_relative_features_and_early_pruning():
    """Features from the global rotations and relative translations (before
    any centre is known) against the oracle; pruning keeps exactly the pairs
    whose probability reaches p_min, with weight 1."""
    torch, F = _mods()
    from tests._util import gt_params6
    from synthetic.scenes import gt_relative_poses
    sc = make_scene("c1", 6)
    x1, x2 = G.oracle_xs(sc)
    Rij, tij = gt_relative_poses(sc, rot_noise_deg=0.5, dir_noise_deg=2.0, seed=4)
    p6 = (gt_params6(sc) + np.random.default_rng(1).normal(0, 0.01, (sc.n_cams, 6))).astype(np.float32)
    th = _theta(41)
    with G.make_problem(sc, rel_R=Rij.astype(np.float32), rel_t=tij.astype(np.float32)) as pr:
        pr.set_params(F.FM_STAGE_ROTATION, p6.reshape(-1))
        pr.mlp_set_params(th)
        feat, resid, prob = pr.mlp_eval_relative(iter_frac=0.0, delta=1e-5, want_prob=True)
        p_min = float(prob.median().item())    # about half the pairs on each side
        kept = pr.mlp_prune(0.0, delta=1e-5, p_min=p_min)
        w, inv_z = pr.get_weights()
        feat, resid, prob, w = feat.cpu().numpy(), resid.cpu().numpy(), prob.cpu().numpy(), w.cpu().numpy()
    fo, ro = M.features_relative(G.f32(p6), G.f32(tij), sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair,
                                 G.f32(sc.focal), 0.0, kp_track=sc.kp_track, delta=1e-5)
    np.testing.assert_allclose(resid, ro, rtol=1e-4, atol=2e-7)
    np.testing.assert_allclose(feat[:, 0], fo[:, 0], rtol=1e-3, atol=2e-4)
    np.testing.assert_allclose(feat[:, 1], fo[:, 1], rtol=1e-3, atol=1e-4)
    np.testing.assert_allclose(feat[:, 2:], fo[:, 2:], rtol=1e-5, atol=2e-6)
    keep = prob >= p_min
    assert 0 < kept == int(keep.sum()) < len(keep)
    np.testing.assert_array_equal(w, keep.astype(np.float32))
    assert abs(inv_z - 1.0 / kept) < 1e-9
