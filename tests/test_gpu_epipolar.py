"""GPU parity of the epipolar stage (Sec. 3.3, Eqs. 7-9) against the FP64
oracle, through the C ABI.  Tolerances (fixed by the workload description):
loss relative 1e-5, gradient relative L2 1e-4."""
import numpy as np
import pytest

from synthetic.scenes import Scene, make_scene
from tests import _gpu as G
from tests._util import gt_params_ea, perturbed_params_ea, scene

pytestmark = pytest.mark.gpu

LOSS_TOL = 1e-5
GRAD_TOL = 1e-4


def _torch():
    import torch
    return torch


def _eval(pr, params, device=True):
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    p = np.asarray(params, np.float32).reshape(-1)
    if device:
        L, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, torch.from_numpy(p).cuda())
        return L, g.cpu().numpy().astype(np.float64)
    L, g = pr.loss_grad(F.FM_STAGE_EPIPOLAR, p)
    return L, g.astype(np.float64)


def _check(sc, pr, params, loss, weights=None, inv_z=None, xs=None, device=True):
    from paper_2505_04612_b300 import fastmap as F
    pr.set_ea_loss(F.FM_EA_L1 if loss == "l1" else F.FM_EA_L2)
    L, g = _eval(pr, params, device)
    Lo, go = G.ea_oracle(sc, params, loss, weights, inv_z, xs)
    assert abs(L - Lo) <= LOSS_TOL * abs(Lo), (L, Lo)
    if loss == "l2":
        assert G.rel_err(g.reshape(go.shape), go) < GRAD_TOL
        return True
    res = G.l1_grad_matches(sc, params, g, GRAD_TOL, weights, inv_z, xs)
    if res is None:
        return False
    ok, err, n_amb = res
    assert ok, (err, n_amb)
    return True


@pytest.mark.parametrize("seed", [0, 1, 2])
@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_c1_perturbed(seed, loss):
    sc = scene("c1", seed)
    xs = G.oracle_xs(sc)
    with G.make_problem(sc) as pr:
        checked = 0
        for k in range(4):
            checked += _check(sc, pr, perturbed_params_ea(sc, 10 * seed + k), loss, xs=xs)
        assert checked >= 2


def test_c3_64_perturbations():
    """64 random perturbations of the c1 seed-0 scene (6D + N(0, 0.02),
    t + N(0, 0.02 * mean baseline)); L2 strictly, L1 with sign ambiguity."""
    sc = scene("c1", 0)
    xs = G.oracle_xs(sc)
    n_l1 = 0
    with G.make_problem(sc) as pr:
        for k in range(64):
            p = perturbed_params_ea(sc, k)
            _check(sc, pr, p, "l2", xs=xs)
            n_l1 += _check(sc, pr, p, "l1", xs=xs)
    assert n_l1 >= 40


@pytest.mark.parametrize("loss", ["l1", "l2"])
def test_weighted_and_host_path(loss):
    sc = scene("c1", 3)
    xs = G.oracle_xs(sc)
    rng = np.random.default_rng(7)
    w = rng.uniform(0.0, 3.0, size=sc.n_kp).astype(np.float32)
    w[rng.random(sc.n_kp) < 0.2] = 0.0          # filtered pairs
    inv_z = 1.0 / float(np.count_nonzero(w))
    p = perturbed_params_ea(sc, 3)
    with G.make_problem(sc, device=False) as pr:    # host inputs, host params
        pr.set_ea_weights(w, np.float32(inv_z))
        _check(sc, pr, p, loss, weights=w, inv_z=float(np.float32(inv_z)), xs=xs, device=False)
        _check(sc, pr, p, loss, weights=w, inv_z=float(np.float32(inv_z)), xs=xs, device=True)
        pr.set_ea_weights(None)
        _check(sc, pr, p, loss, xs=xs)


def test_near_ground_truth():
    sc = scene("c1", 4)
    p = gt_params_ea(sc)
    with G.make_problem(sc) as pr:
        _check(sc, pr, p, "l2")
        _check(sc, pr, p, "l1")


def test_deterministic_bitwise():
    torch = _torch()
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 5)
    p = torch.from_numpy(perturbed_params_ea(sc, 5).astype(np.float32).reshape(-1)).cuda()
    with G.make_problem(sc) as pr:
        outs = [pr.loss_grad(F.FM_STAGE_EPIPOLAR, p) for _ in range(5)]
    for L, g in outs[1:]:
        assert L == outs[0][0]
        assert torch.equal(g, outs[0][1])


# ------------------------------------------------------------- edge cases

def _subscene(sc, pair_i, pair_j, kp_img_pair, keep):
    return Scene(name="edge", seed=0, width=sc.width, height=sc.height, focal=sc.focal, cx=sc.cx,
                 cy=sc.cy, R_gt=sc.R_gt, t_gt=sc.t_gt, points=sc.points,
                 pair_i=np.asarray(pair_i, np.int32), pair_j=np.asarray(pair_j, np.int32),
                 kp_img_pair=np.asarray(kp_img_pair, np.int32), kp1_px=sc.kp1_px[keep],
                 kp2_px=sc.kp2_px[keep], kp_track=sc.kp_track[keep], kp_inlier=sc.kp_inlier[keep])


def test_empty_image_pairs_first_middle_last():
    sc = scene("c1", 6)
    P = sc.n_pairs
    # new image-pair list: an empty pair before every 7th pair, plus first and last
    pi, pj, remap = [], [], np.zeros(P, np.int64)
    pi.append(0); pj.append(1)
    for n in range(P):
        if n % 7 == 3:
            pi.append(2); pj.append(5)
        remap[n] = len(pi)
        pi.append(sc.pair_i[n]); pj.append(sc.pair_j[n])
    pi.append(3); pj.append(4)
    sub = _subscene(sc, pi, pj, remap[sc.kp_img_pair], np.arange(sc.n_kp))
    with G.make_problem(sub) as pr:
        assert pr.info().n_empty_img_pairs == len(pi) - P
        for loss in ["l2", "l1"]:
            _check(sub, pr, perturbed_params_ea(sub, 1), loss)


def test_many_tiny_image_pairs_per_warp_run():
    """Image pairs of 1-3 keypoint pairs: each takes a lane of its own, so a
    warp run holds 32 image pairs and most lanes are partly empty."""
    sc = scene("c1", 7)
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
    sub = _subscene(sc, pi, pj, kp_pair, np.arange(sc.n_kp))
    with G.make_problem(sub) as pr:
        for loss in ["l2", "l1"]:
            _check(sub, pr, perturbed_params_ea(sub, 2), loss)


def test_one_image_pair_spanning_many_warp_runs():
    # three cameras: every image pair holds thousands of keypoint pairs
    sub = make_scene("c1", 8, n_points=6000, n_cams=3)
    assert sub.n_pairs == 3 and sub.n_kp > 5000
    with G.make_problem(sub) as pr:
        for loss in ["l2", "l1"]:
            _check(sub, pr, perturbed_params_ea(sub, 3), loss)


@pytest.mark.parametrize("n_kp", [1, 31, 479, 480, 481, 959])
def test_ragged_sizes(n_kp):
    sc = scene("c1", 9)
    keep = np.arange(n_kp)
    sub = _subscene(sc, sc.pair_i, sc.pair_j, sc.kp_img_pair[keep], keep)
    with G.make_problem(sub) as pr:
        for loss in ["l2", "l1"]:
            _check(sub, pr, perturbed_params_ea(sub, 4), loss)


def test_no_keypoint_pairs():
    sc = scene("c1", 10)
    keep = np.arange(0)
    sub = _subscene(sc, sc.pair_i, sc.pair_j, sc.kp_img_pair[keep], keep)
    with G.make_problem(sub) as pr:
        L, g = _eval(pr, perturbed_params_ea(sub, 5))
        assert L == 0.0 and np.all(g == 0.0)


def test_invalid_inputs_are_rejected():
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 11)
    # (keypoint pairs in any order are accepted: tests/test_gpu_order.py)
    bad = sc.kp_img_pair.copy()
    bad[-1] = sc.n_pairs                                 # out of range
    sub = _subscene(sc, sc.pair_i, sc.pair_j, bad, np.arange(sc.n_kp))
    with pytest.raises(F.FastMapError) as e:
        G.make_problem(sub)
    assert e.value.status == F.FM_ERR_INVALID_ARG
    bad[-1] = -1                                         # negative
    sub = _subscene(sc, sc.pair_i, sc.pair_j, bad, np.arange(sc.n_kp))
    with pytest.raises(F.FastMapError) as e:
        G.make_problem(sub)
    assert e.value.status == F.FM_ERR_INVALID_ARG
    kp = sc.kp1_px.copy()
    kp[5, 0] = np.nan
    sub = _subscene(sc, sc.pair_i, sc.pair_j, sc.kp_img_pair, np.arange(sc.n_kp))
    sub.kp1_px = kp
    with pytest.raises(F.FastMapError) as e:
        G.make_problem(sub)
    assert e.value.status == F.FM_ERR_NAN
    with G.make_problem(sc) as pr:
        p = perturbed_params_ea(sc, 0).astype(np.float32)
        p[3, 2] = np.inf
        with pytest.raises(F.FastMapError) as e:
            pr.set_params(F.FM_STAGE_EPIPOLAR, p.reshape(-1))
        assert e.value.status == F.FM_ERR_NAN


# ----------------------------------------------------------- full size

def test_full_size_5m_pairs():
    """The 5M-keypoint-pair scene in the launch configuration the benchmark
    times: loss and L2 gradient everywhere; the L1 gradient on the unique part
    plus a bound for the sign-ambiguous pairs."""
    from oracle import epipolar as ep
    sc = make_scene("c2_5m", 0)
    xs = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 0, sigma_rot=0.01, sigma_t=0.01)
    with G.make_problem(sc) as pr:
        _check(sc, pr, p, "l2", xs=xs)
        from paper_2505_04612_b300 import fastmap as F
        pr.set_ea_loss(F.FM_EA_L1)
        L, g = _eval(pr, p)
    Lo, go = G.ea_oracle(sc, p, "l1", xs=xs)
    assert abs(L - Lo) <= LOSS_TOL * Lo
    amb = G.ambiguous_pairs(sc, p, xs)
    # each ambiguous pair moves the gradient by at most 2 |d r_m / d params| / Z
    x1, x2 = xs
    pp = G.f32(p).reshape(-1, 9)
    geo = ep.pair_geometry(pp, sc.pair_i, sc.pair_j)
    bound = 0.0
    for m in amb:
        Gm = np.zeros((sc.n_pairs, 3, 3))
        Gm[sc.kp_img_pair[m]] = np.outer(x2[m], x1[m]) / sc.n_kp
        bound += 2.0 * np.linalg.norm(ep.backward_E(Gm, geo, sc.n_cams, sc.pair_i, sc.pair_j, pp))
    err = np.linalg.norm(g.reshape(go.shape) - go)
    assert err <= GRAD_TOL * np.linalg.norm(go) + bound, (err, bound, len(amb))
