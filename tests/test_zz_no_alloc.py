"""The allocation-free entry point, fm_ea_loss_grad_static, against the
problem-based fm_loss_grad.

fm_ea_loss_grad_static is for callers that cannot allocate device memory
when they evaluate (code under another framework's allocator, latency-
critical loops, fixed-footprint deployments): its temporary tables live in a
16 MiB array the library holds on each GPU.  This file is collected last so
that a run stopping at the first failure has run everything else first; the
test also passes alone in a fresh process (the first call on the device looks
the array's address up)."""
import ctypes

import numpy as np
import pytest

from oracle.so3 import rot_from_6d_vjp
from tests import _gpu as G
from tests._util import perturbed_params_ea, scene

pytestmark = pytest.mark.gpu


def _calibrated(sc):
    """float4 (x1, y1, x2, y2) computed as the library computes it (float32)."""
    f = sc.focal.astype(np.float32)
    cx = sc.cx.astype(np.float32)
    cy = sc.cy.astype(np.float32)
    i = sc.pair_i[sc.kp_img_pair]
    j = sc.pair_j[sc.kp_img_pair]
    k1 = sc.kp1_px.astype(np.float32)
    k2 = sc.kp2_px.astype(np.float32)
    return np.stack([(k1[:, 0] - cx[i]) / f[i], (k1[:, 1] - cy[i]) / f[i],
                     (k2[:, 0] - cx[j]) / f[j], (k2[:, 1] - cy[j]) / f[j]], axis=1).astype(np.float32)


def _per_camera(sc, params, blocks):
    """Sum the per-image-pair blocks (dR_i, dt_i, dR_j, dt_j) per camera and
    apply the 6D adjoint, giving the layout fm_loss_grad returns."""
    b = blocks.reshape(-1, 24).astype(np.float64)
    N = sc.n_cams
    gR = np.zeros((N, 3, 3))
    gt = np.zeros((N, 3))
    np.add.at(gR, sc.pair_i, b[:, 0:9].reshape(-1, 3, 3))
    np.add.at(gt, sc.pair_i, b[:, 9:12])
    np.add.at(gR, sc.pair_j, b[:, 12:21].reshape(-1, 3, 3))
    np.add.at(gt, sc.pair_j, b[:, 21:24])
    p = np.asarray(params, np.float64).reshape(N, 9)
    return np.concatenate([rot_from_6d_vjp(p[:, :6], gR), gt], axis=1)


@pytest.mark.parametrize("config,seed", [("c1", 0), ("c2", 1)])
def test_static_entry_matches_problem_entry(config, seed):
    import torch
    from paper_2505_04612_b300 import fastmap as F
    sc = scene(config, seed)
    dev = torch.device("cuda")
    kp = torch.from_numpy(_calibrated(sc)).to(dev)
    seg_off = torch.from_numpy(sc.seg_off().astype(np.int32)).to(dev)
    pi = torch.from_numpy(sc.pair_i.astype(np.int32)).to(dev)
    pj = torch.from_numpy(sc.pair_j.astype(np.int32)).to(dev)
    rng = np.random.default_rng(seed)
    w = rng.uniform(0.5, 2.0, size=sc.n_kp).astype(np.float32)
    inv_z = np.float32(1.0 / sc.n_kp)
    with G.make_problem(sc) as pr:
        for loss in (F.FM_EA_L1, F.FM_EA_L2):
            pr.set_ea_loss(loss)
            for weighted in (False, True):
                if weighted:
                    pr.set_ea_weights(w, inv_z)
                else:
                    pr.set_ea_weights(None)
                # two calls in a row: the shared array keeps the first call's
                # contents, which must not leak into the second
                for k in range(2):
                    p = perturbed_params_ea(sc, 10 * seed + k).astype(np.float32).reshape(-1)
                    p_dev = torch.from_numpy(p).to(dev)
                    L_ref, g_ref = pr.loss_grad(F.FM_STAGE_EPIPOLAR, p_dev)
                    loss_out = torch.empty(1, dtype=torch.float32, device=dev)
                    blocks = torch.empty(24 * sc.n_pairs, dtype=torch.float32, device=dev)
                    F.fm_ea_loss_grad_static(kp, seg_off, pi, pj, p_dev,
                                             torch.from_numpy(w).to(dev) if weighted else None,
                                             sc.n_cams, loss, float(inv_z), loss_out, blocks)
                    torch.cuda.synchronize()
                    L = float(loss_out.item())
                    g = _per_camera(sc, p, blocks.cpu().numpy())
                    gr = g_ref.cpu().numpy().astype(np.float64).reshape(g.shape)
                    assert abs(L - L_ref) <= 1e-5 * abs(L_ref), (loss, weighted, k, L, L_ref)
                    assert G.rel_err(g, gr) < 1e-4, (loss, weighted, k)


def test_static_entry_rejects_problems_beyond_its_array():
    """A problem whose tables would not fit is refused on the host, before any
    GPU work (the buffers passed are never touched)."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    F.lib()
    buf = torch.zeros(64, dtype=torch.float32, device="cuda")
    ib = torch.zeros(64, dtype=torch.int32, device="cuda")
    st = F.lib().fm_ea_loss_grad_static(buf.data_ptr(), ib.data_ptr(), ib.data_ptr(), ib.data_ptr(),
                                        buf.data_ptr(), None, 2, 1, 200_000_000, F.FM_EA_L1,
                                        ctypes.c_float(1.0), buf.data_ptr(), buf.data_ptr(), None)
    assert st == F.FM_ERR_INVALID_ARG
    assert "static array holds" in F.fm_last_error(None)
