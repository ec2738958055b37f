"""Learned per-pair inlier weights for the oracle (float64).  Test infrastructure.

The paper handles outlier keypoint pairs with IRLS weights and a periodic
filter whose threshold decreases (Sec. 3.3, Eq. 9; Appendix "Epipolar
Adjustment").  The learned extension replaces the filter by a small network
that predicts, per keypoint pair, the probability that the pair is an inlier.
The paper has no learned component: everything below is a reading, stated
once here and implemented the same way by the CUDA library.

Features of keypoint pair m of image pair n = (i, j) at epipolar-stage
parameters, with r_m = x~2^T E_n x~1 (the residual of Eq. 7):
  f0  |r_m| / (mean over the pairs of n of |r| + 1e-12)      normalised residual
  f1  log1p(d_m), d_m = fbar |r_m| / sqrt(a0^2 + a1^2 + b0^2 + b1^2),
      a = E_n x~1, b = E_n^T x~2, fbar = (f_i + f_j)/2  epipolar (Sampson)
      distance in pixels
  f2  log(k_m), k_m = (1 + sqrt(1 + 8 c_m))/2 the track length recovered from
      the number c_m of keypoint pairs of the pair's track (0 without tracks)
  f3  the angle (radians) between the viewing rays R_i^T x~1 and R_j^T x~2
      (the pair's parallax; the triangulation angle of its two rays)
  f4  (|x~1[:2]| + |x~2[:2]|)/2, the keypoint radius in calibrated units
  f5  the iteration fraction (given)
  f6  log(Z_n), Z_n the keypoint pairs of image pair n
  f7  log1p(w_m)/log1p(1/delta) with w_m the current IRLS weight (1 without
      weights; delta the IRLS floor)

Network (8 -> 64 -> 64 -> 1): h1 = GELU(x W1 + b1), h2 = GELU(h1 W2 + b2),
o = h2 . w3 + b3, p = sigmoid(o); GELU(z) = z Phi(z) = z (1 + erf(z/sqrt 2))/2
(exact, with erf).  Parameters, flat: W1 [8][64], b1 [64], W2 [64][64],
b2 [64], w3 [64], b3 [1] (4801 values).  Loss: binary cross-entropy averaged
over the pairs, mean(softplus(o) - y o) = mean(-y log p - (1-y) log(1-p)).

Tensor-core emulation (quantise=True): the kernels multiply bfloat16 operands
and accumulate in float32; the operands rounded to bfloat16 (round to nearest
even) are x, W1, h1 and W2 in the forward pass and, in the backward pass, the
pre-activation gradients dz2 and dz1 (with W2 and the inputs x, h1 as above);
everything else is float32 arithmetic.  Here the rounding is applied at the
same points to float64 values.

Pins (tests/test_oracle_mlp.py): central finite differences of the loss;
torch float64 autograd on the same network; closed forms with zero weights;
the bfloat16 rounding against torch's conversion; features against a brute
force per-pair loop and their invariances.
"""
from math import erf, sqrt

import numpy as np

from .so3 import rot_from_6d
from .epipolar import pair_geometry

N_IN, N_HID = 8, 64
SIZES = dict(W1=(N_IN, N_HID), b1=(N_HID,), W2=(N_HID, N_HID), b2=(N_HID,), w3=(N_HID,), b3=(1,))
N_PARAMS = sum(int(np.prod(s)) for s in SIZES.values())   # 4801

_erf = np.vectorize(erf)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64)
    out, o = {}, 0
    for k, s in SIZES.items():
        n = int(np.prod(s))
        out[k] = theta[o:o + n].reshape(s)
        o += n
    return out


def pack(parts):
    return np.concatenate([np.asarray(parts[k], np.float64).reshape(-1) for k in SIZES])


def init_params(seed):
    """He-style initial parameters (seeded): W ~ N(0, 2/fan_in), biases 0."""
    rng = np.random.default_rng(seed)
    return pack(dict(W1=rng.normal(0, sqrt(2 / N_IN), SIZES["W1"]), b1=np.zeros(N_HID),
                     W2=rng.normal(0, sqrt(2 / N_HID), SIZES["W2"]), b2=np.zeros(N_HID),
                     w3=rng.normal(0, sqrt(1 / N_HID), SIZES["w3"]), b3=np.zeros(1)))


def bf16(x):
    """Round to bfloat16 (8-bit significand, round to nearest, ties to even),
    returned as float64: round to float32 first, then keep the top 16 bits of
    the float32 pattern after adding 0x7FFF plus the lowest kept bit."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / sqrt(2.0)))


def gelu_grad(z):
    """d/dz z Phi(z) = Phi(z) + z phi(z)."""
    return 0.5 * (1.0 + _erf(z / sqrt(2.0))) + z * np.exp(-0.5 * z * z) / sqrt(2.0 * np.pi)


def softplus(o):
    return np.logaddexp(0.0, o)


def sigmoid(o):
    return 0.5 * (1.0 + np.tanh(0.5 * o))


def forward(theta, x, quantise=False):
    """Returns (o [B], cache).  x: [B, 8]."""
    P = unpack(theta)
    q = bf16 if quantise else (lambda v: np.asarray(v, np.float64))
    xq = q(x)
    z1 = xq @ q(P["W1"]) + P["b1"]
    h1 = gelu(z1)
    h1q = q(h1)
    z2 = h1q @ q(P["W2"]) + P["b2"]
    h2 = gelu(z2)
    o = h2 @ P["w3"] + P["b3"][0]
    return o, dict(xq=xq, z1=z1, h1q=h1q, z2=z2, h2=h2, P=P)


def bce(o, y):
    return float(np.mean(softplus(o) - y * o))


def loss_grad(theta, x, y, quantise=False):
    """BCE loss and its gradient with respect to the flat parameters,
    derived by hand (reverse order of `forward`)."""
    o, c = forward(theta, x, quantise)
    q = bf16 if quantise else (lambda v: np.asarray(v, np.float64))
    P = c["P"]
    B = len(o)
    do = (sigmoid(o) - y) / B                       # dL/do
    g = {}
    g["w3"] = c["h2"].T @ do
    g["b3"] = np.array([do.sum()])
    dz2 = np.outer(do, P["w3"]) * gelu_grad(c["z2"])
    dz2q = q(dz2)
    g["W2"] = c["h1q"].T @ dz2q
    g["b2"] = dz2.sum(axis=0)
    dh1 = dz2q @ q(P["W2"]).T
    dz1 = dh1 * gelu_grad(c["z1"])
    dz1q = q(dz1)
    g["W1"] = c["xq"].T @ dz1q
    g["b1"] = dz1.sum(axis=0)
    return bce(o, y), pack(g)


# ----------------------------------------------------------------- features

def features(params, pair_i, pair_j, x1, x2, kp_img_pair, focal, iter_frac, kp_track=None,
             weights=None, delta=1e-5):
    """[Z, 8] features of every keypoint pair (definitions in the module
    docstring) at epipolar-stage parameters [N, 9].  x1, x2: [Z, 3]
    calibrated.  Returns (features, residuals)."""
    params = np.asarray(params, np.float64)
    geo = pair_geometry(params, pair_i, pair_j)
    return _features(geo["E"], geo["R"], pair_i, pair_j, x1, x2, kp_img_pair, focal, iter_frac, kp_track,
                     weights, delta)


def features_relative(params6, rel_t, pair_i, pair_j, x1, x2, kp_img_pair, focal, iter_frac, kp_track=None,
                      weights=None, delta=1e-5):
    """The same before any camera centre is known: E_n = [t^{i->j}]_x R_j R_i^T
    from rotation-stage parameters [N, 6] and unit relative translations
    [P, 3]."""
    from .so3 import skew
    R = rot_from_6d(np.asarray(params6, np.float64))
    t = np.asarray(rel_t, np.float64)
    t = t / np.linalg.norm(t, axis=1, keepdims=True)
    Rij = R[pair_j] @ np.transpose(R[pair_i], (0, 2, 1))
    E = skew(t) @ Rij
    return _features(E, R, pair_i, pair_j, x1, x2, kp_img_pair, focal, iter_frac, kp_track, weights, delta)


def _features(E_pairs, R, pair_i, pair_j, x1, x2, kp_img_pair, focal, iter_frac, kp_track, weights, delta):
    E = E_pairs[kp_img_pair]
    a = np.einsum("mab,mb->ma", E, x1)
    b = np.einsum("mba,mb->ma", E, x2)
    r = np.einsum("ma,ma->m", x2, a)
    P = len(pair_i)
    Zn = np.bincount(kp_img_pair, minlength=P).astype(np.float64)
    mean_abs = np.bincount(kp_img_pair, weights=np.abs(r), minlength=P) / np.maximum(Zn, 1)
    f = np.zeros((len(r), 8))
    f[:, 0] = np.abs(r) / (mean_abs[kp_img_pair] + 1e-12)
    fbar = 0.5 * (np.asarray(focal, np.float64)[np.asarray(pair_i)[kp_img_pair]] +
                  np.asarray(focal, np.float64)[np.asarray(pair_j)[kp_img_pair]])
    den = np.sqrt(a[:, 0] ** 2 + a[:, 1] ** 2 + b[:, 0] ** 2 + b[:, 1] ** 2)
    f[:, 1] = np.log1p(fbar * np.abs(r) / den)
    if kp_track is not None:
        c = np.bincount(kp_track).astype(np.float64)[kp_track]
        f[:, 2] = np.log(0.5 * (1.0 + np.sqrt(1.0 + 8.0 * c)))
    d1 = np.einsum("mba,mb->ma", R[np.asarray(pair_i)[kp_img_pair]], x1)   # R_i^T x1
    d2 = np.einsum("mba,mb->ma", R[np.asarray(pair_j)[kp_img_pair]], x2)
    cosang = np.einsum("ma,ma->m", d1, d2) / (np.linalg.norm(d1, axis=1) * np.linalg.norm(d2, axis=1))
    f[:, 3] = np.arccos(np.clip(cosang, -1.0, 1.0))
    f[:, 4] = 0.5 * (np.linalg.norm(x1[:, :2], axis=1) + np.linalg.norm(x2[:, :2], axis=1))
    f[:, 5] = iter_frac
    f[:, 6] = np.log(Zn[kp_img_pair])
    w = np.ones(len(r)) if weights is None else np.asarray(weights, np.float64)
    f[:, 7] = np.log1p(w) / np.log1p(1.0 / delta)
    return f, r


def features_loop(params, pair_i, pair_j, x1, x2, kp_img_pair, focal, iter_frac, kp_track=None,
                  weights=None, delta=1e-5):
    """The same features pair by pair with plain loops (small inputs only)."""
    params = np.asarray(params, np.float64)
    Z = len(kp_img_pair)
    out = np.zeros((Z, 8))
    rs = np.zeros(Z)
    R = rot_from_6d(params[:, :6])
    t = params[:, 6:]
    tcount = {}
    if kp_track is not None:
        for tr in kp_track:
            tcount[int(tr)] = tcount.get(int(tr), 0) + 1
    for m in range(Z):
        n = int(kp_img_pair[m])
        i, j = int(pair_i[n]), int(pair_j[n])
        Rij = R[j] @ R[i].T
        tij = t[j] - Rij @ t[i]
        th = tij / np.linalg.norm(tij)
        E = np.array([[0, -th[2], th[1]], [th[2], 0, -th[0]], [-th[1], th[0], 0]]) @ Rij
        rs[m] = x2[m] @ E @ x1[m]
    for m in range(Z):
        n = int(kp_img_pair[m])
        i, j = int(pair_i[n]), int(pair_j[n])
        same = [k for k in range(Z) if kp_img_pair[k] == n]
        mean_abs = sum(abs(rs[k]) for k in same) / len(same)
        Rij = R[j] @ R[i].T
        tij = t[j] - Rij @ t[i]
        th = tij / np.linalg.norm(tij)
        E = np.array([[0, -th[2], th[1]], [th[2], 0, -th[0]], [-th[1], th[0], 0]]) @ Rij
        a = E @ x1[m]
        b = E.T @ x2[m]
        fb = 0.5 * (focal[i] + focal[j])
        out[m, 0] = abs(rs[m]) / (mean_abs + 1e-12)
        out[m, 1] = np.log1p(fb * abs(rs[m]) / sqrt(a[0] ** 2 + a[1] ** 2 + b[0] ** 2 + b[1] ** 2))
        if kp_track is not None:
            c = tcount[int(kp_track[m])]
            k = (1 + sqrt(1 + 8 * c)) / 2
            out[m, 2] = np.log(k)
        d1 = R[i].T @ x1[m]
        d2 = R[j].T @ x2[m]
        out[m, 3] = np.arccos(np.clip(d1 @ d2 / (np.linalg.norm(d1) * np.linalg.norm(d2)), -1, 1))
        out[m, 4] = 0.5 * (np.hypot(x1[m, 0], x1[m, 1]) + np.hypot(x2[m, 0], x2[m, 1]))
        out[m, 5] = iter_frac
        out[m, 6] = np.log(len(same))
        w = 1.0 if weights is None else float(weights[m])
        out[m, 7] = np.log1p(w) / np.log1p(1.0 / delta)
    return out, rs


def labels(r, tau):
    """Training labels: a pair is an inlier when its residual at the converged
    plain solve is below the final filter threshold."""
    return (np.abs(r) < tau).astype(np.float64)
