"""Focal lengths inside epipolar adjustment on the GPU (fm_ea_focal_forward /
fm_ea_focal_backward; Sec. 3.3, last paragraph of "Epipolar Adjustment")
against the FP64 oracle (oracle/focal.direct_loss_grad) on the same float32
inputs; phi = 0 against the pose-only split (bitwise); recalibration
equivalence; and a short Adam run recovering the focal lengths on
noise-free keypoints."""
import dataclasses

import numpy as np
import pytest

from oracle import epipolar as ep
from oracle import focal as fo
from tests import _gpu as G
from tests._util import gt_params_ea, perturbed_params_ea, scene

pytestmark = pytest.mark.gpu

LOSS_TOL, GRAD_TOL = 1e-5, 1e-4


def _torch():
    import torch
    return torch


def _gpu(pr, params, phi, grad_loss=None):
    torch = _torch()
    from paper_2505_04612_b300.autograd import epipolar_focal_loss
    p = torch.tensor(np.asarray(params, np.float32).reshape(-1), device="cuda", requires_grad=True)
    f = torch.tensor(np.asarray(phi, np.float32), device="cuda", requires_grad=True)
    L = epipolar_focal_loss(p, f, pr)
    (L * (1.0 if grad_loss is None else grad_loss)).backward()
    return float(L.detach()), p.grad.cpu().numpy().astype(np.float64), f.grad.cpu().numpy().astype(np.float64)


def _l1_grads_with_signs(sc, params, phi, xs, max_amb=3):
    """The oracle's L1 gradients for every valid sign (-1, 0, 1) of the
    residuals within float32 reach of 0 (GAMMA), or None if there are more
    than max_amb of them."""
    import itertools
    p = G.f32(params).reshape(-1, 9)
    f = G.f32(phi)
    geo = ep.pair_geometry(p, sc.pair_i, sc.pair_j)
    Ep = fo.focal_matrices(geo["E"], f, sc.pair_i, sc.pair_j)
    r = ep.residuals(Ep, xs[0], xs[1], sc.kp_img_pair)
    amb = np.nonzero(np.abs(r) < G.GAMMA)[0]
    if len(amb) > max_amb:
        return None
    outer = np.einsum("ma,mb->mab", xs[1], xs[0]) / len(r)
    out = []
    for signs in itertools.product([-1.0, 0.0, 1.0], repeat=len(amb)):
        sg = np.sign(r)
        sg[amb] = signs
        Gp = np.zeros((sc.n_pairs, 3, 3))
        np.add.at(Gp, sc.kp_img_pair, sg[:, None, None] * outer)
        out.append(fo._backward(Gp, geo, f, sc.pair_i, sc.pair_j, p))
    return out


@pytest.mark.parametrize("loss", ["l2", "l1"])
@pytest.mark.parametrize("seed", [0, 1])
def test_matches_the_oracle(loss, seed):
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", seed)
    xs = G.oracle_xs(sc)
    rng = np.random.default_rng(40 + seed)
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2)
        checked = 0
        for k in range(6):
            params = perturbed_params_ea(sc, 10 * seed + k)
            phi = rng.normal(0.0, 0.05, sc.n_cams)
            L, g, gphi = _gpu(pr, params, phi)
            Lo, go, gpo = fo.direct_loss_grad(G.f32(params).reshape(-1, 9), G.f32(phi), sc.pair_i, sc.pair_j,
                                              xs[0], xs[1], sc.kp_img_pair, loss=loss)
            assert abs(L - Lo) <= LOSS_TOL * abs(Lo), (L, Lo)   # continuous through r = 0
            cands = [(go, gpo)] if loss == "l2" else _l1_grads_with_signs(sc, params, phi, xs)
            if cands is None:
                continue   # too many residuals within float32 reach of 0 to enumerate their signs
            err = min(max(G.rel_err(g.reshape(a.shape), a), G.rel_err(gphi, b)) for a, b in cands)
            assert err < GRAD_TOL, err
            checked += 1
        assert checked >= 2


def test_zero_phi_is_the_pose_only_split_bitwise():
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    from paper_2505_04612_b300.autograd import epipolar_loss
    sc = scene("c1", 2)
    params = perturbed_params_ea(sc, 7)
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_L2)
        L, g, gphi = _gpu(pr, params, np.zeros(sc.n_cams))
        p = torch.tensor(np.asarray(params, np.float32).reshape(-1), device="cuda", requires_grad=True)
        L0 = epipolar_loss(p, pr, "fused")
        L0.backward()
        assert L == float(L0.detach())
        np.testing.assert_array_equal(g, p.grad.cpu().numpy().astype(np.float64))
    _, _, gpo = fo.direct_loss_grad(G.f32(params).reshape(-1, 9), np.zeros(sc.n_cams), sc.pair_i, sc.pair_j,
                                    *G.oracle_xs(sc), sc.kp_img_pair, loss="l2")
    assert G.rel_err(gphi, gpo) < GRAD_TOL


def test_recalibration_equivalence_and_upstream_scale():
    """phi = delta on keypoints calibrated at f0 is the plain objective on the
    same pixels calibrated at f0 e^delta; an upstream factor scales both
    gradients."""
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    from paper_2505_04612_b300.autograd import epipolar_loss
    sc = scene("c1", 3)
    rng = np.random.default_rng(5)
    delta = rng.normal(0.0, 0.03, sc.n_cams)
    params = perturbed_params_ea(sc, 3)
    moved = dataclasses.replace(sc, focal=sc.focal * np.exp(delta))
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_L2)
        L, g, gphi = _gpu(pr, params, delta)
        L3, g3, gphi3 = _gpu(pr, params, delta, grad_loss=3.0)
    with G.make_problem(moved) as pr2:
        pr2.set_ea_loss(F.FM_EA_L2)
        p = torch.tensor(np.asarray(params, np.float32).reshape(-1), device="cuda", requires_grad=True)
        L2 = epipolar_loss(p, pr2, "fused")
        L2.backward()
        g2 = p.grad.cpu().numpy().astype(np.float64)
    assert abs(L - float(L2.detach())) <= 1e-4 * abs(float(L2.detach()))
    assert G.rel_err(g, g2) < 1e-3
    # the factor enters before the chain rule: equal up to float32 rounding
    assert G.rel_err(g3, 3.0 * g) < 1e-6 and G.rel_err(gphi3, 3.0 * gphi) < 1e-6


def test_adam_recovers_focal_lengths_without_noise():
    """Noise-free c1 keypoints calibrated at focal lengths 2 % off (per
    camera), poses at the truth: Adam on phi alone drives the L2 loss down
    and phi toward the true log ratios (the noisy case drifts: the objective
    is biased there, as the oracle shows)."""
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    from paper_2505_04612_b300.autograd import epipolar_focal_loss
    from tests._util import clean_scene
    sc = clean_scene(4)
    rng = np.random.default_rng(9)
    phi_true = rng.normal(0.0, 0.02, sc.n_cams)
    wrong = dataclasses.replace(sc, focal=sc.focal * np.exp(-phi_true))   # f0 = f e^-phi*
    params = torch.tensor(np.asarray(gt_params_ea(sc), np.float32).reshape(-1), device="cuda")
    phi = torch.zeros(sc.n_cams, device="cuda", requires_grad=True)
    opt = torch.optim.Adam([phi], lr=1e-3)
    with G.make_problem(wrong) as pr:
        pr.set_ea_loss(F.FM_EA_L2)
        L_start = float(epipolar_focal_loss(params, phi.detach().contiguous(), pr))
        for _ in range(600):
            opt.zero_grad()
            L = epipolar_focal_loss(params, phi, pr)
            L.backward()
            opt.step()
        L_end = float(epipolar_focal_loss(params, phi.detach().contiguous(), pr))
    err0 = np.mean(np.abs(phi_true))
    err = np.mean(np.abs(phi.detach().cpu().numpy() - phi_true))
    assert L_end < 0.05 * L_start, (L_start, L_end)
    assert err < 0.3 * err0, (err0, err)
