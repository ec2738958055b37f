"""The hand-written adjoint of the epipolar objective behind
torch.autograd.Function (Sec. 3.3, Eqs. 7-9), in its three modes, against the
FP64 oracle's gradient and against central finite differences (h = 1e-3, FP64)
of the oracle's loss.  Tolerances as for the fused evaluation: loss relative
1e-5, gradient relative L2 1e-4."""
import numpy as np
import pytest

from oracle import epipolar as ep
from synthetic.scenes import Scene
from tests import _gpu as G
from tests._util import perturbed_params_ea, scene

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4
MODES = ["recompute", "stored", "fused"]


def _mods():
    import torch
    from paper_2505_04612_b300 import autograd as A
    from paper_2505_04612_b300 import fastmap as F
    return torch, A, F


def _set_loss(pr, loss):
    _, _, F = _mods()
    pr.set_ea_loss(F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2)


def _autograd(pr, params, mode, scale=None):
    """(loss, grad) through EpipolarLoss; `scale` multiplies the loss first."""
    torch, A, _ = _mods()
    p = torch.from_numpy(np.asarray(params, np.float32).reshape(-1)).cuda().requires_grad_(True)
    L = A.epipolar_loss(p, pr, mode)
    (L if scale is None else L * scale).backward()
    return float(L.item()), p.grad.detach().cpu().numpy().astype(np.float64), p.grad.detach().clone()


def _fused_reference(pr, params):
    torch, _, F = _mods()
    p = torch.from_numpy(np.asarray(params, np.float32).reshape(-1)).cuda()
    L, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, p)
    return L, g


def _check_vs_oracle(sc, L, g, params, loss, xs, weights=None, inv_z=None):
    Lo, go = G.ea_oracle(sc, params, loss, weights, inv_z, xs)
    assert abs(L - Lo) <= LOSS_TOL * abs(Lo), (L, Lo)
    if loss == "l2":
        err = G.rel_err(g.reshape(go.shape), go)
        assert err < GRAD_TOL, err
        return True
    res = G.l1_grad_matches(sc, params, g, GRAD_TOL, weights, inv_z, xs)
    if res is None:
        return False
    ok, err, n_amb = res
    assert ok, (err, n_amb)
    return True


def test_c3_64_perturbations_all_modes():
    """The c1 seed-0 scene, 64 perturbations: each mode's loss and gradient
    match the oracle (L2 strictly, L1 up to sign-ambiguous pairs), and the
    three modes give the gradient of the one-pass evaluation bit for bit."""
    torch, _, _ = _mods()
    sc = scene("c1", 0)
    xs = G.oracle_xs(sc)
    n_l1 = 0
    with G.make_problem(sc) as pr:
        for loss in ["l2", "l1"]:
            _set_loss(pr, loss)
            for k in range(64):
                p = perturbed_params_ea(sc, k)
                L_ref, g_ref = _fused_reference(pr, p)
                checked = True
                for mode in MODES:
                    L, g, g_dev = _autograd(pr, p, mode)
                    assert torch.equal(g_dev, g_ref), (mode, k)
                    assert abs(L - L_ref) <= 1e-6 * abs(L_ref)
                    checked = _check_vs_oracle(sc, L, g, p, loss, xs) and checked
                n_l1 += (loss == "l1") and checked
    assert n_l1 >= 40


def test_central_differences_of_the_oracle():
    """GPU adjoint (each mode) against central differences of the FP64 oracle
    loss, h = 1e-3: the full 180-entry gradient at one perturbation (L2) and
    16 random directional derivatives at three more (the FD truncation error
    here is ~1e-8 of |grad|)."""
    sc = scene("c1", 0)
    x1, x2 = G.oracle_xs(sc)

    def L_oracle(q):
        return ep.direct_loss_grad(q.reshape(-1, 9), sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair,
                                   loss="l2")[0]

    h = 1e-3
    with G.make_problem(sc) as pr:
        _set_loss(pr, "l2")
        p = G.f32(perturbed_params_ea(sc, 7)).reshape(-1)
        fd = np.empty_like(p)
        for i in range(p.size):
            e = np.zeros_like(p)
            e[i] = h
            fd[i] = (L_oracle(p + e) - L_oracle(p - e)) / (2 * h)
        for mode in MODES:
            _, g, _ = _autograd(pr, p, mode)
            assert G.rel_err(g, fd) < GRAD_TOL, mode
        rng = np.random.default_rng(11)
        for k in (8, 9, 10):
            p = G.f32(perturbed_params_ea(sc, k)).reshape(-1)
            grads = {m: _autograd(pr, p, m)[1] for m in MODES}
            gn = np.linalg.norm(grads["recompute"])
            for _ in range(16):
                v = rng.normal(size=p.shape)
                v /= np.linalg.norm(v)
                d = (L_oracle(p + h * v) - L_oracle(p - h * v)) / (2 * h)
                for m in MODES:
                    assert abs(grads[m] @ v - d) <= GRAD_TOL * gn, (m, grads[m] @ v, d)


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_weighted_and_scaled_upstream_gradient(loss):
    """Per-pair weights (with filtered pairs) and an upstream gradient g:
    backward returns g * dL/dparams (g enters on the device)."""
    torch, A, _ = _mods()
    sc = scene("c1", 3)
    xs = G.oracle_xs(sc)
    rng = np.random.default_rng(5)
    w = rng.uniform(0.0, 3.0, size=sc.n_kp).astype(np.float32)
    w[rng.random(sc.n_kp) < 0.2] = 0.0
    inv_z = float(np.float32(1.0 / np.count_nonzero(w)))
    p = perturbed_params_ea(sc, 4)
    with G.make_problem(sc) as pr:
        pr.set_ea_weights(w, np.float32(inv_z))
        _set_loss(pr, loss)
        for mode in MODES:
            L, g, _ = _autograd(pr, p, mode)
            _check_vs_oracle(sc, L, g, p, loss, xs, weights=w, inv_z=inv_z)
            _, g3, _ = _autograd(pr, p, mode, scale=-2.5)
            # g scales dL/dE_n before the chain rule: equal up to rounding
            np.testing.assert_allclose(g3, -2.5 * g, rtol=1e-5, atol=1e-6 * np.abs(g).max())


def test_stored_coefficients_are_w_rho_prime():
    """The stored intermediate is c_m = w_m rho'(r_m): sign(r) (L1) or 2r
    (L2), per keypoint pair in the input order (the input is already sorted by
    image pair)."""
    torch, _, F = _mods()
    sc = scene("c1", 2)
    x1, x2 = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 1)
    r = ep.residuals(ep.essential_matrices(G.f32(p), sc.pair_i, sc.pair_j), x1, x2, sc.kp_img_pair)
    pt = torch.from_numpy(np.asarray(p, np.float32).reshape(-1)).cuda()
    with G.make_problem(sc) as pr:
        for loss in ["l1", "l2"]:
            _set_loss(pr, loss)
            coef = torch.empty(sc.n_kp, dtype=torch.float32, device="cuda")
            L = torch.empty((), dtype=torch.float32, device="cuda")
            F.fm_ea_forward(pr.handle, pt.data_ptr(), L.data_ptr(), F.FM_EA_SAVE_COEF, coef.data_ptr())
            c = coef.cpu().numpy().astype(np.float64)
            if loss == "l1":
                sure = np.abs(r) >= G.GAMMA
                np.testing.assert_array_equal(c[sure], np.sign(r[sure]))
                assert np.all(np.isin(c[~sure], [-1.0, 0.0, 1.0]))
            else:
                # r is a sum of nine O(1) products: float32 evaluation error < 1e-6
                np.testing.assert_allclose(c, 2.0 * r, rtol=1e-4, atol=2e-6)


def _subscene(sc, pair_i, pair_j, kp_img_pair, keep):
    return Scene(name="edge", seed=0, width=sc.width, height=sc.height, focal=sc.focal, cx=sc.cx,
                 cy=sc.cy, R_gt=sc.R_gt, t_gt=sc.t_gt, points=sc.points,
                 pair_i=np.asarray(pair_i, np.int32), pair_j=np.asarray(pair_j, np.int32),
                 kp_img_pair=np.asarray(kp_img_pair, np.int32), kp1_px=sc.kp1_px[keep],
                 kp2_px=sc.kp2_px[keep], kp_track=sc.kp_track[keep], kp_inlier=sc.kp_inlier[keep])


@pytest.mark.parametrize("n_kp", [0, 1, 31, 481, 959])
def test_ragged_and_empty(n_kp):
    """Partial last warp run (zero-filled tail, coefficient copy-out) and the
    empty problem (loss 0, gradient 0)."""
    torch, _, _ = _mods()
    sc = scene("c1", 9)
    keep = np.arange(n_kp)
    sub = _subscene(sc, sc.pair_i, sc.pair_j, sc.kp_img_pair[keep], keep)
    p = perturbed_params_ea(sub, 4)
    with G.make_problem(sub) as pr:
        for loss in ["l2", "l1"]:
            _set_loss(pr, loss)
            L_ref, g_ref = _fused_reference(pr, p)
            for mode in MODES:
                L, g, g_dev = _autograd(pr, p, mode)
                assert torch.equal(g_dev, g_ref), mode
                if n_kp == 0:
                    assert L == 0.0 and np.all(g == 0.0)
                else:
                    assert abs(L - L_ref) <= 1e-6 * abs(L_ref)


def test_tiny_image_pairs_slow_path():
    """Image pairs of 1-3 keypoint pairs (lanes crossing several image-pair
    ends, table entries past the 32 in registers) in every mode."""
    torch, _, _ = _mods()
    sc = scene("c1", 7)
    xs_sc = sc
    rng = np.random.default_rng(7)
    pi, pj, kp_pair = [], [], np.zeros(sc.n_kp, np.int64)
    off = sc.seg_off()
    for n in range(sc.n_pairs):
        m = off[n]
        while m < off[n + 1]:
            k = int(rng.integers(1, 4))
            kp_pair[m:m + k] = len(pi)
            pi.append(sc.pair_i[n]); pj.append(sc.pair_j[n])
            m += k
    sub = _subscene(xs_sc, pi, pj, kp_pair, np.arange(sc.n_kp))
    xs = G.oracle_xs(sub)
    p = perturbed_params_ea(sub, 2)
    with G.make_problem(sub) as pr:
        _set_loss(pr, "l2")
        L_ref, g_ref = _fused_reference(pr, p)
        for mode in MODES:
            L, g, g_dev = _autograd(pr, p, mode)
            assert torch.equal(g_dev, g_ref), mode
            _check_vs_oracle(sub, L, g, p, "l2", xs)


def test_errors():
    torch, A, F = _mods()
    sc = scene("c1", 1)
    p = torch.from_numpy(np.asarray(perturbed_params_ea(sc, 0), np.float32).reshape(-1)).cuda()
    L = torch.empty((), dtype=torch.float32, device="cuda")
    buf = torch.empty(sc.n_kp + 8, dtype=torch.float32, device="cuda")
    with G.make_problem(sc) as pr:
        with pytest.raises(F.FastMapError) as e:
            F.fm_ea_forward(pr.handle, p.data_ptr(), L.data_ptr(), 7, None)
        assert e.value.status == F.FM_ERR_INVALID_ARG
        with pytest.raises(F.FastMapError) as e:
            F.fm_ea_forward(pr.handle, p.data_ptr(), L.data_ptr(), F.FM_EA_SAVE_COEF, buf.data_ptr() + 4)
        assert e.value.status == F.FM_ERR_INVALID_ARG and "aligned" in str(e.value)
        with pytest.raises(F.FastMapError) as e:
            F.fm_ea_backward(pr.handle, p.data_ptr(), F.FM_EA_SAVE_COEF, None, None, buf.data_ptr())
        assert e.value.status == F.FM_ERR_INVALID_ARG
        pr.set_ea_loss(F.FM_EA_COMPACT)
        with pytest.raises(F.FastMapError) as e:
            A.epipolar_loss(p.clone().requires_grad_(True), pr, "recompute")
        assert e.value.status == F.FM_ERR_STATE
        with pytest.raises(ValueError):
            A.epipolar_loss(p, pr, "bogus")


def test_batch_of_scenes_per_scene_losses():
    """A problem holding several scenes returns one loss per scene; backward
    with upstream gradients g_s gives sum_s g_s dL_s/dparams (each scene's
    cameras get g_s times their own gradient)."""
    torch, A, F = _mods()
    from synthetic.scenes import concat_scenes
    scenes = [scene("c1", 0), scene("c1", 2), scene("c1", 4)]
    b = concat_scenes(scenes)
    ps = [np.asarray(perturbed_params_ea(sc, 5 + k), np.float32) for k, sc in enumerate(scenes)]
    gs = torch.tensor([1.0, -0.5, 2.0], device="cuda")
    with G.make_problem(b) as pb:
        _set_loss(pb, "l2")
        for mode in MODES:
            p = torch.from_numpy(np.concatenate([q.reshape(-1) for q in ps])).cuda().requires_grad_(True)
            L = A.epipolar_loss(p, pb, mode)
            assert L.shape == (3,)
            (L * gs).sum().backward()
            g = p.grad.cpu().numpy()
            o = 0
            for k, sc in enumerate(scenes):
                Lo, go = G.ea_oracle(sc, ps[k], "l2")
                assert abs(float(L.detach()[k]) - Lo) <= LOSS_TOL * abs(Lo)
                gk = g[o:o + 9 * sc.n_cams].astype(np.float64)
                assert G.rel_err(gk, float(gs[k]) * go.reshape(-1)) < GRAD_TOL, (mode, k)
                o += 9 * sc.n_cams
