"""From raw matches to poses, in the order of the paper (Sec. 3 with
Appendix "Filtering" and "Tracks"): image pairs whose raw-match count does
not exceed an adaptive threshold are dropped (``fm_filter_image_pairs``);
the global rotations are aligned on the raw matches; the tracks are completed
(``fm_tracks_complete``) and the completed keypoint pairs, only introduced
after the rotation alignment, drive the translation and epipolar stages and
the triangulation (``fm_solve`` with ``rot_given``).  Every step is a call of
the C ABI; this module only moves arrays between them.
"""
from __future__ import annotations

import numpy as np

from . import fastmap as F


def group_raw_matches(kp_off, matches):
    """Image pairs of raw matches (keypoint ids): matches oriented from the
    lower image, grouped by image pair (a stable order inside one).  Returns
    (pair_i, pair_j, kp_img_pair, oriented matches [M,2])."""
    kp_off = np.asarray(kp_off, np.int64)
    m = np.asarray(matches, np.int64).reshape(-1, 2)
    n_img = len(kp_off) - 1
    img = np.searchsorted(kp_off, m, side="right") - 1
    swap = img[:, 0] > img[:, 1]
    m = np.where(swap[:, None], m[:, ::-1], m)
    img = np.where(swap[:, None], img[:, ::-1], img)
    key = img[:, 0] * n_img + img[:, 1]
    order = np.argsort(key, kind="stable")
    key, m = key[order], m[order]
    uniq, kp_img_pair = np.unique(key, return_inverse=True)
    return ((uniq // n_img).astype(np.int32), (uniq % n_img).astype(np.int32),
            kp_img_pair.astype(np.int32), m.astype(np.int32))


def solve_from_raw_matches(kp_off, matches, kp_px, focal, cx, cy, t_start=256.0, t_min=16.0, complete=True,
                           min_pairs=8, rot_opts=None, **solve_opts):
    """Poses (and points) of the images from raw matches.

    kp_off [N+1], kp_px [K,2]: keypoints grouped by image with their pixels;
    matches [M,2]: keypoint ids of raw matches between two images; focal, cx,
    cy [N]: intrinsics.  The image pairs are filtered on their raw-match
    counts (threshold from t_start halved down to t_min until the images are
    connected); the rotation stage runs on the kept raw matches; with
    ``complete`` the translation and epipolar stages run on the completed
    tracks of those matches (image pairs with fewer than ``min_pairs``
    completed pairs dropped), otherwise on the raw matches themselves.
    ``rot_opts`` / ``solve_opts`` override fm_solve's options for the two
    solves.  Returns fm_solve's dict plus "threshold", "image_valid" and the
    sizes of both problems."""
    kp_off = np.asarray(kp_off, np.int32)
    kp_px = np.asarray(kp_px, np.float32)
    n_img = len(kp_off) - 1
    pi, pj, kp_pair, m = group_raw_matches(kp_off, matches)
    counts = np.bincount(kp_pair, minlength=len(pi))
    keep, image_valid, t = F.filter_image_pairs(n_img, pi, pj, counts, t_start, t_min)
    km = keep[kp_pair]
    new_index = np.cumsum(keep) - 1
    raw = dict(pair_i=pi[keep], pair_j=pj[keep], kp_img_pair=new_index[kp_pair[km]].astype(np.int32),
               kp1_px=kp_px[m[km, 0]], kp2_px=kp_px[m[km, 1]])
    intr = dict(focal=np.asarray(focal, np.float32), cx=np.asarray(cx, np.float32), cy=np.asarray(cy, np.float32))
    # rotations on the raw matches (the translation / epipolar work of this
    # solve is cut to the minimum: only its rotation stage is kept)
    ro = dict(trn_runs=1, trn_iters=1, trn_final_iters=1, ea_rounds=0)
    ro.update(rot_opts or {})
    with F.Problem(raw["pair_i"], raw["pair_j"], raw["kp_img_pair"], raw["kp1_px"], raw["kp2_px"],
                   intr["focal"], intr["cx"], intr["cy"]) as pr_raw:
        pr_raw.solve(**ro)
        rot = pr_raw.get_params(F.FM_STAGE_ROTATION).cpu().numpy()
        sizes = dict(raw_img_pairs=pr_raw.n_pairs, raw_kp_pairs=pr_raw.n_kp)
    if complete:
        tr = F.complete_tracks(kp_off, m[km], kp_px, min_pairs=min_pairs)
        args = (tr["pair_i"], tr["pair_j"], tr["kp_img_pair"], tr["kp1_px"], tr["kp2_px"])
        track = tr["kp_track"]
        n_tracks = int(tr["n_tracks"])
    else:
        args = (raw["pair_i"], raw["pair_j"], raw["kp_img_pair"], raw["kp1_px"], raw["kp2_px"])
        track, n_tracks = None, None
    with F.Problem(*args, intr["focal"], intr["cx"], intr["cy"], kp_track=track) as pr:
        pr.set_params(F.FM_STAGE_ROTATION, np.asarray(rot, np.float32).reshape(-1))
        out = pr.solve(n_tracks=n_tracks, rot_given=1, **solve_opts)
        sizes.update(img_pairs=pr.n_pairs, kp_pairs=pr.n_kp)
    out.update(threshold=t, image_valid=image_valid, **sizes)
    return out
