"""GPU parity of IRLS reweighting / filtering (Sec. 3.3, Eq. 9) and of the
compact per-image-pair form (Eq. 8, Appendix Eqs. 15-17) against the FP64
oracle, through the C ABI."""
import numpy as np
import pytest

from oracle import epipolar as ep
from oracle.adam import Adam
from tests import _gpu as G
from tests._util import perturbed_params_ea, scene

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _near(sc, seed, s=0.003):
    return perturbed_params_ea(sc, seed, sigma_rot=s, sigma_t=s).astype(np.float32)


@pytest.mark.parametrize("irls", [True, False])
def test_reweight_matches_oracle(irls):
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 0)
    x1, x2 = G.oracle_xs(sc)
    p = _near(sc, 0)
    tau, delta = 0.01, 1e-5
    r = ep.residuals(ep.essential_matrices(G.f32(p), sc.pair_i, sc.pair_j), x1, x2, sc.kp_img_pair)
    w_o, keep_o = ep.irls_weights(r, tau, delta)
    if not irls:
        w_o = keep_o.astype(np.float64)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, p.reshape(-1))
        kept = pr.reweight(tau, delta, irls)
        w_g, inv_z = pr.get_weights()
    w_g = w_g.cpu().numpy().astype(np.float64)
    a = np.abs(r)
    sure = np.abs(a - tau) > G.GAMMA                      # the keep decision is unique here
    assert np.array_equal(w_g[sure] > 0, keep_o[sure])
    assert abs(kept - int(keep_o.sum())) <= int((~sure).sum())
    assert kept < sc.n_kp and kept > 0.8 * sc.n_kp       # the outliers (5%) went
    assert abs(inv_z - 1.0 / kept) <= 1e-7 / kept
    k = sure & keep_o
    # 1/max(|r|, delta) inherits the float32 error of r: relative GAMMA/max(|r|, delta)
    tol = w_o[k] * (G.GAMMA / np.maximum(a[k], delta) + 1e-6)
    assert np.all(np.abs(w_g[k] - w_o[k]) <= tol)


def _oracle_weights(sc, p0, tau=0.01, delta=1e-5):
    x1, x2 = G.oracle_xs(sc)
    r = ep.residuals(ep.essential_matrices(G.f32(p0), sc.pair_i, sc.pair_j), x1, x2, sc.kp_img_pair)
    w, keep = ep.irls_weights(r, tau, delta)
    return w.astype(np.float32), np.float32(1.0 / keep.sum())


@pytest.mark.parametrize("seed", [1, 2])
def test_compact_matches_oracle(seed):
    torch = pytest.importorskip("torch")
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", seed)
    x1, x2 = G.oracle_xs(sc)
    p0 = _near(sc, seed)
    w, inv_z = _oracle_weights(sc, p0)
    W = ep.build_W(x1, x2, sc.kp_img_pair, sc.n_pairs, weights=G.f32(w))
    rng = np.random.default_rng(seed)
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, p0.reshape(-1))
        pr.set_ea_weights(w, inv_z)
        for s in [0.0, 1e-3, 5e-3]:
            p = (p0 + rng.normal(0, s, size=p0.shape)).astype(np.float32)
            pr.set_ea_loss(F.FM_EA_COMPACT)
            Lc, gc = pr.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(p.reshape(-1)).cuda())
            Lo, go, _ = ep.compact_loss_grad(G.f32(p), sc.pair_i, sc.pair_j, W, float(inv_z))
            assert abs(Lc - Lo) <= LOSS_TOL * Lo, (s, Lc, Lo)
            assert G.rel_err(gc.cpu().numpy().reshape(go.shape), go) < GRAD_TOL
            # the direct weighted L2 kernel evaluates the same objective
            pr.set_ea_loss(F.FM_EA_L2)
            Ld, gd = pr.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(p.reshape(-1)).cuda())
            assert abs(Ld - Lo) <= LOSS_TOL * Lo
            assert G.rel_err(gd.cpu().numpy().reshape(go.shape), go) < GRAD_TOL


def test_compact_without_weights_is_unweighted_l2():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 3)
    x1, x2 = G.oracle_xs(sc)
    p = _near(sc, 3)
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_COMPACT)
        L, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, p.reshape(-1))
    W = ep.build_W(x1, x2, sc.kp_img_pair, sc.n_pairs)
    Lo, go, _ = ep.compact_loss_grad(G.f32(p), sc.pair_i, sc.pair_j, W, 1.0 / sc.n_kp)
    assert abs(L - Lo) <= LOSS_TOL * Lo
    assert G.rel_err(g.reshape(go.shape), go) < GRAD_TOL


def test_compact_adam_steps():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 4)
    x1, x2 = G.oracle_xs(sc)
    p0 = _near(sc, 4)
    w, inv_z = _oracle_weights(sc, p0)
    W = ep.build_W(x1, x2, sc.kp_img_pair, sc.n_pairs, weights=G.f32(w))
    lr, n = 2e-4, 10
    with G.make_problem(sc) as pr:
        pr.set_params(F.FM_STAGE_EPIPOLAR, p0.reshape(-1))
        pr.set_ea_weights(w, inv_z)
        pr.set_ea_loss(F.FM_EA_COMPACT)
        pr.step(F.FM_STAGE_EPIPOLAR, n, lr)
        got = pr.get_params(F.FM_STAGE_EPIPOLAR).cpu().numpy().astype(np.float64).reshape(p0.shape)
    opt = Adam(p0.shape, lr=lr)
    x = G.f32(p0)
    for _ in range(n):
        x = opt.step(x, ep.compact_loss_grad(x, sc.pair_i, sc.pair_j, W, float(inv_z))[1])
    assert np.max(np.abs(got - x)) < 1e-5
    assert np.max(np.abs(got - G.f32(p0))) > 0.5 * lr


def test_compact_at_scale_matches_oracle():
    """The compact step on a 600-camera scene (thousands of image pairs: many
    32-pair tiles of W, a ragged last one, camera passes over up to a few
    hundred incident image pairs read in camera-CSR order) against the
    oracle, unweighted and IRLS-weighted."""
    from paper_2505_04612_b300 import fastmap as F
    from synthetic.scenes import make_scene
    sc = make_scene("c2", 7, n_cams=600, n_points=120000)
    assert sc.n_pairs > 5000 and sc.n_pairs % 32 != 0
    x1, x2 = G.oracle_xs(sc)
    p0 = _near(sc, 7)
    w, inv_z = _oracle_weights(sc, p0)
    for weighted in (False, True):
        W = ep.build_W(x1, x2, sc.kp_img_pair, sc.n_pairs, weights=G.f32(w) if weighted else None)
        iz = float(inv_z) if weighted else 1.0 / sc.n_kp
        with G.make_problem(sc) as pr:
            pr.set_params(F.FM_STAGE_EPIPOLAR, p0.reshape(-1))
            if weighted:
                pr.set_ea_weights(w, inv_z)
            pr.set_ea_loss(F.FM_EA_COMPACT)
            p = (p0 + np.random.default_rng(8).normal(0, 1e-3, size=p0.shape)).astype(np.float32)
            L, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, p.reshape(-1))
        Lo, go, _ = ep.compact_loss_grad(G.f32(p), sc.pair_i, sc.pair_j, W, iz)
        assert abs(L - Lo) <= LOSS_TOL * Lo, (weighted, L, Lo)
        assert G.rel_err(np.asarray(g).reshape(go.shape), go) < GRAD_TOL
