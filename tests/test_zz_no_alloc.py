"""The allocation-free entry point, fm_ea_loss_grad_static, against the
problem-based fm_loss_grad and against the float64 oracle.

fm_ea_loss_grad_static is for callers that cannot allocate device memory
when they evaluate (code under another framework's allocator, latency-
critical loops, fixed-footprint deployments): its temporary tables live in a
16 MiB array the library holds on each GPU.  The array keeps whatever the
previous call left in it, so the tests call it in sequences that would
expose stale contents: two calls in a row, a large problem then a smaller one
then the large one again, image pairs without keypoint pairs, no keypoint
pairs at all.  This file is collected last so that a run stopping at the
first failure has run everything else first; the tests also pass alone in a
fresh process (the first call on the device looks the array's address up)."""
import ctypes
import dataclasses

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


def _xs(kp):
    """the oracle's calibrated points for the exact float32 inputs passed"""
    k = kp.astype(np.float64)
    one = np.ones((len(k), 1))
    return np.concatenate([k[:, 0:2], one], 1), np.concatenate([k[:, 2:4], one], 1)


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


class _Inputs:
    """device copies of one scene's inputs of fm_ea_loss_grad_static"""

    def __init__(self, sc, seed):
        import torch
        dev = torch.device("cuda")
        self.sc = sc
        self.kp_host = _calibrated(sc)
        self.kp = torch.from_numpy(self.kp_host).to(dev)
        self.seg_off = torch.from_numpy(sc.seg_off().astype(np.int32)).to(dev)
        self.pi = torch.from_numpy(sc.pair_i.astype(np.int32)).to(dev)
        self.pj = torch.from_numpy(sc.pair_j.astype(np.int32)).to(dev)
        rng = np.random.default_rng(seed)
        self.w_host = rng.uniform(0.5, 2.0, size=sc.n_kp).astype(np.float32)
        self.w = torch.from_numpy(self.w_host).to(dev)
        self.inv_z = np.float32(1.0 / max(sc.n_kp, 1))
        self.loss_out = torch.empty(1, dtype=torch.float32, device=dev)
        self.blocks = torch.empty(24 * sc.n_pairs, dtype=torch.float32, device=dev)

    def call(self, p_dev, loss, weighted, seg_off=None):
        from paper_2505_04612_b300 import fastmap as F
        F.fm_ea_loss_grad_static(self.kp, self.seg_off if seg_off is None else seg_off, self.pi, self.pj, p_dev,
                                 self.w if weighted else None, self.sc.n_cams, loss, float(self.inv_z),
                                 self.loss_out, self.blocks)


def _check_against_problem_and_oracle(pr, inp, p, loss, weighted):
    """loss and per-camera gradient equal fm_loss_grad's (1e-5 / 1e-4) and the
    oracle's on the same float32 inputs (L1: signs of |r| < GAMMA enumerated)."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    sc = inp.sc
    p_dev = torch.from_numpy(p).cuda()
    L_ref, g_ref = pr.loss_grad(F.FM_STAGE_EPIPOLAR, p_dev)
    inp.call(p_dev, loss, weighted)
    torch.cuda.synchronize()
    L = float(inp.loss_out.item())
    g = _per_camera(sc, p, inp.blocks.cpu().numpy())
    gr = g_ref.cpu().numpy().astype(np.float64).reshape(g.shape)
    assert abs(L - L_ref) <= 1e-5 * abs(L_ref), (loss, weighted, L, L_ref)
    assert G.rel_err(g, gr) < 1e-4, (loss, weighted)
    xs = _xs(inp.kp_host)
    w = inp.w_host if weighted else None
    name = "l1" if loss == F.FM_EA_L1 else "l2"
    Lo, go = G.ea_oracle(sc, p, name, w, float(inp.inv_z), xs)
    assert abs(L - Lo) <= 1e-5 * abs(Lo), (loss, weighted, L, Lo)
    if name == "l2":
        assert G.rel_err(g, go) < 1e-4
    else:
        res = G.l1_grad_matches(sc, p, g, 1e-4, w, float(inp.inv_z), xs)
        if res is None:   # too many sign-ambiguous pairs to enumerate: bound them
            res = G.l1_grad_within_bound(sc, p, g, 1e-4, w, float(inp.inv_z), xs)
        assert res[0], res


def _with_empty_image_pairs(sc, every=7):
    """sc with an image pair without keypoint pairs inserted after every
    `every`-th image pair (and one at the start and one at the end)."""
    P = sc.n_pairs
    new_index = np.zeros(P, np.int64)
    pi, pj = [0], [1]                     # an empty image pair first
    for n in range(P):
        new_index[n] = len(pi)
        pi.append(int(sc.pair_i[n]))
        pj.append(int(sc.pair_j[n]))
        if n % every == every - 1:
            pi.append(int(sc.pair_i[n]))
            pj.append(int(sc.pair_j[n]))
    pi.append(0)
    pj.append(2)                          # and one last
    return dataclasses.replace(sc, name=sc.name + "_empty", pair_i=np.array(pi, np.int32),
                               pair_j=np.array(pj, np.int32),
                               kp_img_pair=new_index[sc.kp_img_pair].astype(np.int32))


@pytest.mark.parametrize("config,seed", [("c1", 0), ("c2", 1)])
def test_static_entry_matches_problem_entry_and_oracle(config, seed):
    from paper_2505_04612_b300 import fastmap as F
    sc = scene(config, seed)
    inp = _Inputs(sc, seed)
    with G.make_problem(sc) as pr:
        for loss in (F.FM_EA_L1, F.FM_EA_L2):
            pr.set_ea_loss(loss)
            for weighted in (False, True):
                pr.set_ea_weights(inp.w_host if weighted else None, inp.inv_z)
                # two calls in a row: the shared array keeps the first call's
                # contents, which must not leak into the second
                for k in range(2):
                    p = perturbed_params_ea(sc, 10 * seed + k).astype(np.float32).reshape(-1)
                    _check_against_problem_and_oracle(pr, inp, p, loss, weighted)


def test_large_then_small_then_large():
    """c2 (0.8M pairs, 16k image pairs) then c1 (14k pairs) then c2 again: the
    smaller call runs over tables the larger one left behind, and the larger
    one over the smaller one's."""
    from paper_2505_04612_b300 import fastmap as F
    big, small = scene("c2", 2), scene("c1", 2)
    ib, i_s = _Inputs(big, 2), _Inputs(small, 3)
    with G.make_problem(big) as pb, G.make_problem(small) as ps:
        for pr in (pb, ps):
            pr.set_ea_loss(F.FM_EA_L1)
            pr.set_ea_weights(None)
        for k, (pr, inp) in enumerate(((pb, ib), (ps, i_s), (pb, ib))):
            p = perturbed_params_ea(inp.sc, 40 + k).astype(np.float32).reshape(-1)
            _check_against_problem_and_oracle(pr, inp, p, F.FM_EA_L1, False)


def test_empty_image_pairs_give_zero_blocks():
    import torch
    from paper_2505_04612_b300 import fastmap as F
    sc = _with_empty_image_pairs(scene("c1", 4))
    off = sc.seg_off()
    empty = np.nonzero(off[1:] == off[:-1])[0]
    assert len(empty) > 20 and empty[0] == 0 and empty[-1] == sc.n_pairs - 1
    inp = _Inputs(sc, 4)
    with G.make_problem(sc) as pr:
        for loss in (F.FM_EA_L1, F.FM_EA_L2):
            pr.set_ea_loss(loss)
            pr.set_ea_weights(None)
            p = perturbed_params_ea(sc, 50).astype(np.float32).reshape(-1)
            inp.blocks.fill_(7.0)          # every block, empty ones included, is written
            _check_against_problem_and_oracle(pr, inp, p, loss, False)
            blocks = inp.blocks.cpu().numpy().reshape(-1, 24)
            assert np.all(blocks[empty] == 0.0)
    torch.cuda.synchronize()


def test_no_keypoint_pairs_and_rejected_offsets():
    """Z = 0 gives a zero loss and zero blocks.  An offset table that is not a
    CSR table of Z pairs (decreasing, or not ending at Z) is caught on the
    device before any keypoint is read: the loss is NaN, the blocks zero, and
    the next valid call is unaffected."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 5)
    inp = _Inputs(sc, 5)
    p = perturbed_params_ea(sc, 60).astype(np.float32).reshape(-1)
    p_dev = torch.from_numpy(p).cuda()
    # no keypoint pairs
    zero = torch.zeros(sc.n_pairs + 1, dtype=torch.int32, device="cuda")
    F.fm_ea_loss_grad_static(inp.kp, zero, inp.pi, inp.pj, p_dev, None, sc.n_cams, F.FM_EA_L1, 1.0,
                             inp.loss_out, inp.blocks, n_kp_pairs=0)
    torch.cuda.synchronize()
    assert float(inp.loss_out.item()) == 0.0
    assert torch.count_nonzero(inp.blocks).item() == 0
    good = inp.seg_off.clone()
    bad_tables = []
    dec = good.clone()
    dec[5], dec[6] = good[6], good[5]               # decreasing at 5
    bad_tables.append(dec)
    short = good.clone()
    short[-1] = good[-1] - 1                        # does not end at Z
    bad_tables.append(short)
    start = good.clone()
    start[0] = 1                                    # does not start at 0
    bad_tables.append(start)
    with G.make_problem(sc) as pr:
        pr.set_ea_loss(F.FM_EA_L1)
        pr.set_ea_weights(None)
        for bad in bad_tables:
            inp.call(p_dev, F.FM_EA_L1, False, seg_off=bad)
            torch.cuda.synchronize()
            assert np.isnan(float(inp.loss_out.item()))
            assert torch.count_nonzero(inp.blocks).item() == 0
            _check_against_problem_and_oracle(pr, inp, p, F.FM_EA_L1, False)


def test_calls_allocate_no_device_memory():
    """After a first round of calls (which may load the kernels' code), further
    calls leave the device's free memory unchanged."""
    import torch
    from paper_2505_04612_b300 import fastmap as F
    sc = scene("c1", 6)
    inp = _Inputs(sc, 6)
    p_dev = torch.from_numpy(perturbed_params_ea(sc, 70).astype(np.float32).reshape(-1)).cuda()

    def round_of_calls():
        for loss in (F.FM_EA_L1, F.FM_EA_L2):
            for weighted in (False, True):
                inp.call(p_dev, loss, weighted)
        torch.cuda.synchronize()

    round_of_calls()
    free0, _ = torch.cuda.mem_get_info()
    for _ in range(5):
        round_of_calls()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0, (free0, free1)


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
