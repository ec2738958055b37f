"""Training data, training and evaluation of the learned inlier filter.

The network and its features are defined in ``include/fastmap.h`` (learned
inlier weights).  This module sequences C-ABI calls; every feature, forward
and backward pass, optimiser step, solve stage and reweighting runs in the
library's kernels.

Training data: each training problem (one scene, or a batch of scenes in one
problem) goes through the stages of ``fm_solve`` call by call; at the start
of every epipolar round the features of every keypoint pair are captured
(iteration fraction k/rounds, the weights of the previous round), and after
the last round the converged residuals give the labels: a pair is an inlier
when |r| < tau_min, the final filter threshold (the labels of the method's
own converged solves).
"""
from __future__ import annotations

import numpy as np

from . import fastmap as F

PHASES = (1.0, 0.3, 0.1, 0.03)   # the learning-rate phases of fm_solve's Adam loops


def init_params(seed: int) -> np.ndarray:
    """He-style initial network parameters (seeded), flat float32 [4801]."""
    rng = np.random.default_rng(seed)
    parts = [rng.normal(0.0, np.sqrt(2.0 / 8), (8, 64)), np.zeros(64),
             rng.normal(0.0, np.sqrt(2.0 / 64), (64, 64)), np.zeros(64),
             rng.normal(0.0, np.sqrt(1.0 / 64), 64), np.zeros(1)]
    return np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)


def _stepped(pr, stage, lr, iters, opts, want_loss=False):
    per = iters // len(PHASES)
    loss = None
    for k, f in enumerate(PHASES):
        n = per if k < len(PHASES) - 1 else iters - per * (len(PHASES) - 1)
        last = k == len(PHASES) - 1
        loss = pr.step(stage, n, lr * f, opts.beta1, opts.beta2, opts.eps, want_loss=want_loss and last)
    return loss


def solve_with_snapshots(pr, snapshot=None, **overrides):
    """The stages of the plain fm_solve, call by call with the same options;
    calls ``snapshot(None, rounds)`` after the relative translations are
    estimated and ``snapshot(k, rounds)`` at the start of epipolar round k
    (before its reweighting) -- the two places the learned solve evaluates the
    network.  Returns the options used."""
    o = F.solve_opts(**overrides)
    pr.set_ea_weights(None)
    pr.rotation_init(o.rot_init_iters)
    _stepped(pr, F.FM_STAGE_ROTATION, o.rot_lr, o.rot_iters, o)
    if o.reestimate_rel_t:
        pr.relative_translations()
    if snapshot is not None:
        snapshot(None, o.ea_rounds)
    pr.set_translation_runs(o.trn_runs)
    pr.translation_random_init(o.seed)
    _stepped(pr, F.FM_STAGE_TRANSLATION, o.trn_lr, o.trn_iters, o)
    pr.translation_merge()
    _stepped(pr, F.FM_STAGE_TRANSLATION, o.trn_lr, o.trn_final_iters, o)
    pr.epipolar_init_from_stages()
    pr.set_ea_loss(F.FM_EA_COMPACT)
    for k in range(o.ea_rounds):
        if snapshot is not None:
            snapshot(k, o.ea_rounds)
        tau = max(o.ea_tau0 * 0.5 ** k, o.ea_tau_min)
        pr.reweight(tau, o.ea_delta)
        _stepped(pr, F.FM_STAGE_EPIPOLAR, o.ea_lr, o.ea_iters, o)
    return o


def training_rows(pr, keep_frac=0.25, seed=0, **overrides):
    """Features captured where the learned solve evaluates the network -- after
    the first relative translations (iteration fraction 0, E from the global
    rotations and the relative translations) and at the start of every
    epipolar round k of R (fraction (k+1)/(R+1)) -- during a plain solve of
    `pr`, and the labels from its converged residuals.  Returns CUDA tensors
    X [n, 8], y [n] (a seeded random `keep_frac` of the rows of every
    snapshot)."""
    import torch
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    snaps = []
    o_holder = {}

    def snap(k, rounds):
        delta = o_holder["delta"]
        if k is None:
            feat, _, _ = pr.mlp_eval_relative(iter_frac=0.0, delta=delta, want_feat=True, want_resid=False)
        else:
            feat, _, _ = pr.mlp_eval(iter_frac=(k + 1) / (rounds + 1), delta=delta, want_feat=True,
                                     want_resid=False)
        idx = torch.nonzero(torch.rand(feat.shape[0], generator=g, device="cuda") < keep_frac).squeeze(1)
        snaps.append((idx, feat[idx]))

    o_holder["delta"] = F.solve_opts(**overrides).ea_delta
    o = solve_with_snapshots(pr, snap, **overrides)
    _, resid, _ = pr.mlp_eval(iter_frac=1.0, delta=o.ea_delta, want_feat=False, want_resid=True)
    label = (resid.abs() < o.ea_tau_min).float()
    X = torch.cat([f for _, f in snaps])
    y = torch.cat([label[i] for i, _ in snaps])
    return X, y


def train(X, y, steps=2000, batch=65536, lr=3e-3, seed=0, theta0=None, stream=None):
    """Adam on minibatches of (X, y) with the library's trainer; the learning
    rate decays by 10x over the run.  Returns (theta [4801] float32, losses)."""
    import torch
    n = int(y.numel())
    b = min(batch, n)
    tr = F.MlpTrainer(b, stream=stream)
    tr.set_params(init_params(seed) if theta0 is None else theta0)
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    losses = []
    loss = torch.empty(1, dtype=torch.float32, device=X.device)
    for k in range(steps):
        idx = torch.randint(0, n, (b,), generator=g, device="cuda")
        xb, yb = X[idx].contiguous(), y[idx].contiguous()
        tr.step(xb, yb, lr * 0.1 ** (k / max(steps - 1, 1)), loss_out=loss)
        if k % 100 == 0 or k == steps - 1:
            losses.append(float(loss.item()))
    theta = tr.get_params()
    tr.close()
    return theta, losses


def logits(theta, X):
    """Network outputs o of feature rows X (CUDA tensor [n, 8]); a pair is
    predicted an inlier when o >= 0 (p >= 0.5)."""
    tr = F.MlpTrainer(max(int(X.shape[0]), 1))
    tr.set_params(theta)
    o = tr.forward(X.contiguous())
    tr.close()
    return o
