"""Shared helpers for the tests: seeded scenes and parameter sets.

Parameters are laid out as the C ABI lays them out:
  rotation stage     [N,6]  = (a1, a2)           6D rotation (first two columns)
  translation stage  [N,3]  = o                  camera centre
  epipolar stage     [N,9]  = (a1, a2, t)        6D rotation + world-to-camera t
"""
import functools

import numpy as np

from synthetic.scenes import make_scene


@functools.lru_cache(maxsize=16)
def scene(config="c1", seed=0, **kw):
    return make_scene(config, seed, **kw)


def clean_scene(seed=0, **kw):
    """c1 geometry without pixel noise and without outliers."""
    return make_scene("c1", seed, sigma_px=0.0, outlier_frac=0.0, **kw)


def gt_params6(sc):
    return np.concatenate([sc.R_gt[:, :, 0], sc.R_gt[:, :, 1]], axis=1)


def gt_params_ea(sc):
    return np.concatenate([gt_params6(sc), sc.t_gt], axis=1)


def perturbed_params_ea(sc, seed, sigma_rot=0.02, sigma_t=0.02):
    """c3-style perturbation: 6D + N(0, sigma_rot), t + N(0, sigma_t * mean baseline)."""
    rng = np.random.default_rng(100 + seed)
    p = gt_params_ea(sc).copy()
    c = sc.centers_gt
    base = np.mean(np.linalg.norm(c[sc.pair_j] - c[sc.pair_i], axis=1))
    p[:, :6] += rng.normal(0.0, sigma_rot, size=(sc.n_cams, 6))
    p[:, 6:] += rng.normal(0.0, sigma_t * base, size=(sc.n_cams, 3))
    return p


def similarity_transform_ea(params, Q, d, s):
    """World similarity X -> s Q X + d applied to epipolar-stage parameters:
    R -> R Q^T and t -> s t - R Q^T d (camera centres o -> s Q o + d)."""
    from oracle.so3 import rot_from_6d
    R = rot_from_6d(params[:, :6])
    t = params[:, 6:]
    Rn = R @ Q.T
    tn = s * t - np.einsum("nab,b->na", Rn, d)
    return np.concatenate([Rn[:, :, 0], Rn[:, :, 1], tn], axis=1)
