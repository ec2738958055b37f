"""Pins of the learned-weight oracle (oracle/mlp.py) against things other
than itself: torch's bfloat16 conversion and float64 autograd (library
routines), central finite differences, closed forms with zero weights, a
per-pair loop for the features, invariances and the generator's own track
lengths."""
import numpy as np
import pytest

from oracle import mlp as M
from synthetic.scenes import make_scene
from tests import _gpu as G
from tests._util import clean_scene, gt_params_ea, perturbed_params_ea, similarity_transform_ea


def _data(B=96, seed=0):
    rng = np.random.default_rng(seed)
    x = rng.normal(0, 1.0, size=(B, 8))
    y = (rng.random(B) < 0.6).astype(np.float64)
    return x, y


def test_bf16_matches_torch_conversion():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.normal(0, 10, 5000), rng.normal(0, 1e-3, 5000),
                        # exact ties between two bfloat16 values (both parities)
                        (np.arange(1, 200) * 2 + 1) * 2.0 ** -8 + 1.0, [0.0, -0.0, 1.0, -3.5]])
    v32 = v.astype(np.float32)
    want = torch.from_numpy(v32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(M.bf16(v32), want)


def test_gelu_and_its_derivative():
    z = np.linspace(-6, 6, 101)
    from scipy.stats import norm
    np.testing.assert_allclose(M.gelu(z), z * norm.cdf(z), rtol=1e-13, atol=1e-15)
    h = 1e-6
    np.testing.assert_allclose(M.gelu_grad(z), (M.gelu(z + h) - M.gelu(z - h)) / (2 * h), rtol=1e-7, atol=1e-9)


def test_gradient_central_differences():
    x, y = _data()
    th = M.init_params(3) + np.random.default_rng(4).normal(0, 0.05, M.N_PARAMS)
    L, g = M.loss_grad(th, x, y)
    rng = np.random.default_rng(5)
    idx = rng.choice(M.N_PARAMS, 60, replace=False)
    h = 1e-6
    for k in idx:
        e = np.zeros(M.N_PARAMS)
        e[k] = h
        fd = (M.bce(M.forward(th + e, x)[0], y) - M.bce(M.forward(th - e, x)[0], y)) / (2 * h)
        assert abs(fd - g[k]) <= 1e-6 * max(1.0, abs(g[k])) + 1e-9, (k, fd, g[k])


def test_matches_torch_autograd_float64():
    torch = pytest.importorskip("torch")
    x, y = _data(64, 2)
    th = M.init_params(7)
    L, g = M.loss_grad(th, x, y)
    P = {k: torch.tensor(v, dtype=torch.float64, requires_grad=True) for k, v in M.unpack(th).items()}
    X = torch.tensor(x)
    h1 = torch.nn.functional.gelu(X @ P["W1"] + P["b1"], approximate="none")
    h2 = torch.nn.functional.gelu(h1 @ P["W2"] + P["b2"], approximate="none")
    o = h2 @ P["w3"] + P["b3"][0]
    Lt = torch.nn.functional.binary_cross_entropy_with_logits(o, torch.tensor(y))
    Lt.backward()
    gt = np.concatenate([P[k].grad.numpy().reshape(-1) for k in M.SIZES])
    assert abs(L - Lt.item()) < 1e-12
    np.testing.assert_allclose(g, gt, rtol=1e-9, atol=1e-13)


def test_closed_form_with_zero_weights():
    """W1 = W2 = w3 = 0: the output is b3 for every pair, the loss is
    softplus(b3) - mean(y) b3, dL/db3 = sigmoid(b3) - mean(y), and
    dL/dw3 = GELU(b2) (sigmoid(b3) - mean(y))."""
    x, y = _data(50, 3)
    P = M.unpack(np.zeros(M.N_PARAMS))
    P = {k: v.copy() for k, v in P.items()}
    P["b3"][0] = 0.7
    P["b2"][:] = np.linspace(-1, 1, 64)
    th = M.pack(P)
    L, g = M.loss_grad(th, x, y)
    s = 1 / (1 + np.exp(-0.7))
    assert abs(L - (np.log1p(np.exp(0.7)) - y.mean() * 0.7)) < 1e-14
    G_ = M.unpack(g)
    assert abs(G_["b3"][0] - (s - y.mean())) < 1e-14
    np.testing.assert_allclose(G_["w3"], M.gelu(P["b2"]) * (s - y.mean()), rtol=1e-12, atol=1e-15)
    assert np.all(G_["W1"] == 0) and np.all(G_["W2"] == 0)


def test_quantised_pass_stays_within_bfloat16_error():
    x, y = _data(256, 4)
    th = M.init_params(9)
    L, g = M.loss_grad(th, x, y)
    Lq, gq = M.loss_grad(th, x, y, quantise=True)
    assert abs(Lq - L) < 5e-3 * L
    assert np.linalg.norm(gq - g) < 3e-2 * np.linalg.norm(g)
    # operands that are bfloat16 already are left alone
    xb = M.bf16(x)
    assert np.array_equal(M.bf16(xb), xb)


def _small_scene():
    sc = make_scene("c1", 0)
    keep = np.nonzero(sc.kp_img_pair < 12)[0]
    return sc, keep


def test_features_match_a_per_pair_loop():
    sc, keep = _small_scene()
    x1, x2 = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 1)
    w = np.random.default_rng(0).uniform(0.0, 50.0, sc.n_kp)
    args = (sc.pair_i, sc.pair_j)
    f, r = M.features(p, *args, x1[keep], x2[keep], sc.kp_img_pair[keep], sc.focal, 0.25,
                      kp_track=sc.kp_track[keep], weights=w[keep])
    fl, rl = M.features_loop(p, *args, x1[keep], x2[keep], sc.kp_img_pair[keep], sc.focal, 0.25,
                             kp_track=sc.kp_track[keep], weights=w[keep])
    np.testing.assert_allclose(r, rl, rtol=1e-10, atol=1e-14)
    np.testing.assert_allclose(f, fl, rtol=1e-9, atol=1e-12)


def test_feature_invariances_and_known_values():
    """Zero residual features at noise-free ground truth; the residual,
    epipolar-distance and parallax features do not change under a similarity
    of the world; the track-length feature is the log of the number of
    cameras that see the point."""
    sc = clean_scene(2)
    x1, x2 = G.oracle_xs(sc)
    p = gt_params_ea(sc)
    f, r = M.features(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, sc.focal, 0.0, kp_track=sc.kp_track)
    # pixels are stored in float32: a coordinate of up to 640 px is off by up
    # to 640 * 2^-24 = 4e-5 px, and so is the epipolar distance
    assert np.abs(f[:, 1]).max() < 1e-4
    cams = {}
    for m in range(sc.n_kp):
        cams.setdefault(int(sc.kp_track[m]), set()).update([int(sc.pair_i[sc.kp_img_pair[m]]),
                                                            int(sc.pair_j[sc.kp_img_pair[m]])])
    want = np.array([np.log(len(cams[int(t)])) for t in sc.kp_track])
    np.testing.assert_allclose(f[:, 2], want, rtol=1e-12)
    sc2 = make_scene("c1", 3)
    x1, x2 = G.oracle_xs(sc2)
    p = perturbed_params_ea(sc2, 2)
    f0, _ = M.features(p, sc2.pair_i, sc2.pair_j, x1, x2, sc2.kp_img_pair, sc2.focal, 0.5)
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    Q *= np.sign(np.linalg.det(Q))
    p2 = similarity_transform_ea(p, Q, rng.normal(size=3), 2.5)
    f1, _ = M.features(p2, sc2.pair_i, sc2.pair_j, x1, x2, sc2.kp_img_pair, sc2.focal, 0.5)
    np.testing.assert_allclose(f1[:, [0, 1, 3]], f0[:, [0, 1, 3]], rtol=1e-7, atol=1e-9)


def test_relative_features_equal_the_camera_features_when_consistent():
    """With the relative translations of the epipolar-stage parameters
    themselves, E_n is the same either way, and so are the features."""
    from oracle.epipolar import pair_geometry
    sc = make_scene("c1", 5)
    x1, x2 = G.oracle_xs(sc)
    p = perturbed_params_ea(sc, 3)
    geo = pair_geometry(p, sc.pair_i, sc.pair_j)
    f_a, r_a = M.features(p, sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair, sc.focal, 0.0, kp_track=sc.kp_track)
    f_b, r_b = M.features_relative(p[:, :6], 3.0 * geo["that"], sc.pair_i, sc.pair_j, x1, x2, sc.kp_img_pair,
                                   sc.focal, 0.0, kp_track=sc.kp_track)
    np.testing.assert_allclose(r_b, r_a, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(f_b, f_a, rtol=1e-10, atol=1e-12)
