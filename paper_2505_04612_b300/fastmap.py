"""ctypes binding of the C ABI in ``include/fastmap.h``.

The functions below carry the C names and only marshal arguments: every
computation runs in ``lib/libfastmap.so``.  Arrays may be torch tensors
(CUDA tensors are passed as device pointers, CPU tensors and numpy arrays as
host pointers).  If the library is missing, loading raises: there is no
fallback implementation.

``Problem`` is a small owner of one ``fm_problem`` handle built on these calls.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

FM_OK = 0
FM_ERR_INVALID_ARG = 1
FM_ERR_CUDA = 2
FM_ERR_OOM = 3
FM_ERR_NAN = 4
FM_ERR_TIMEOUT = 5
FM_ERR_NOT_CONVERGED = 6
FM_ERR_STATE = 7

FM_STAGE_ROTATION = 0
FM_STAGE_TRANSLATION = 1
FM_STAGE_EPIPOLAR = 2
STAGE_DIM = {FM_STAGE_ROTATION: 6, FM_STAGE_TRANSLATION: 3, FM_STAGE_EPIPOLAR: 9}

FM_EA_L1 = 0
FM_EA_L2 = 1
FM_EA_COMPACT = 2

FM_EA_SAVE_NONE = 0
FM_EA_SAVE_COEF = 1
FM_EA_SAVE_DLDE = 2

_c_i32p = ctypes.POINTER(ctypes.c_int32)
_c_f32p = ctypes.POINTER(ctypes.c_float)


class fm_problem_desc(ctypes.Structure):
    _fields_ = [
        ("n_cams", ctypes.c_int32),
        ("n_img_pairs", ctypes.c_int32),
        ("n_kp_pairs", ctypes.c_int64),
        ("pair_cam_i", ctypes.c_void_p),
        ("pair_cam_j", ctypes.c_void_p),
        ("kp_img_pair", ctypes.c_void_p),
        ("kp1_px", ctypes.c_void_p),
        ("kp2_px", ctypes.c_void_p),
        ("kp_track", ctypes.c_void_p),
        ("focal", ctypes.c_void_p),
        ("cx", ctypes.c_void_p),
        ("cy", ctypes.c_void_p),
        ("rel_R", ctypes.c_void_p),
        ("rel_t", ctypes.c_void_p),
        ("inputs_on_device", ctypes.c_int32),
        ("cuda_stream", ctypes.c_void_p),
        ("n_scenes", ctypes.c_int32),
        ("scene_cam_off", ctypes.c_void_p),
    ]


class fm_problem_info(ctypes.Structure):
    _fields_ = [
        ("n_cams", ctypes.c_int32),
        ("n_img_pairs", ctypes.c_int32),
        ("n_kp_pairs", ctypes.c_int64),
        ("n_empty_img_pairs", ctypes.c_int32),
        ("pairs_per_lane", ctypes.c_int32),
        ("n_records", ctypes.c_int64),
        ("device_bytes", ctypes.c_int64),
        ("n_scenes", ctypes.c_int32),
        ("n_cams_connected", ctypes.c_int32),
    ]


class fm_kernel_time(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64), ("total_ms", ctypes.c_double)]


class fm_tri_opts(ctypes.Structure):
    _fields_ = [("max_err_px", ctypes.c_float), ("min_angle_deg", ctypes.c_float)]


class fm_solve_opts(ctypes.Structure):
    _fields_ = [
        ("rot_init_iters", ctypes.c_int32), ("rot_iters", ctypes.c_int32), ("rot_lr", ctypes.c_float),
        ("reestimate_rel_t", ctypes.c_int32), ("trn_runs", ctypes.c_int32), ("trn_iters", ctypes.c_int32),
        ("trn_lr", ctypes.c_float), ("trn_final_iters", ctypes.c_int32), ("seed", ctypes.c_uint32),
        ("ea_rounds", ctypes.c_int32), ("ea_iters", ctypes.c_int32), ("ea_lr", ctypes.c_float),
        ("ea_tau0", ctypes.c_float), ("ea_tau_min", ctypes.c_float), ("ea_delta", ctypes.c_float),
        ("tri_max_err_px", ctypes.c_float), ("tri_min_angle_deg", ctypes.c_float),
        ("beta1", ctypes.c_float), ("beta2", ctypes.c_float), ("eps", ctypes.c_float),
        ("learned", ctypes.c_int32), ("learned_p_min", ctypes.c_float), ("learned_prune_passes", ctypes.c_int32),
        ("rot_given", ctypes.c_int32),
    ]


class fm_result(ctypes.Structure):
    _fields_ = [
        ("R", ctypes.c_void_p), ("t", ctypes.c_void_p), ("points", ctypes.c_void_p),
        ("point_valid", ctypes.c_void_p), ("n_tracks", ctypes.c_int32), ("n_points_valid", ctypes.c_int32),
        ("loss_rotation", ctypes.c_float), ("loss_translation", ctypes.c_float),
        ("loss_epipolar", ctypes.c_float), ("n_kept", ctypes.c_int64),
        ("cam_valid", ctypes.c_void_p),
    ]


class fm_tuning(ctypes.Structure):
    _fields_ = [("pairs_per_lane", ctypes.c_int32), ("ctas_per_sm", ctypes.c_int32),
                ("us_per_eval", ctypes.c_float)]


class fm_adam_opts(ctypes.Structure):
    _fields_ = [("lr", ctypes.c_float), ("beta1", ctypes.c_float),
                ("beta2", ctypes.c_float), ("eps", ctypes.c_float)]


# name -> (restype, argtypes); kept in the order of include/fastmap.h
_SIGNATURES = {
    "fm_problem_create": (ctypes.c_int, [ctypes.POINTER(fm_problem_desc), ctypes.POINTER(ctypes.c_void_p)]),
    "fm_problem_destroy": (None, [ctypes.c_void_p]),
    "fm_last_error": (ctypes.c_char_p, [ctypes.c_void_p]),
    "fm_problem_info_get": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fm_problem_info)]),
    "fm_kp_order": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int32]),
    "fm_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_int32]),
    "fm_set_rel_poses": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_translation_set_runs": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fm_ea_set_loss": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int]),
    "fm_ea_set_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_float]),
    "fm_ea_reweight": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int64)]),
    "fm_ea_get_weights": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_float)]),
    "fm_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_int32]),
    "fm_ea_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32,
                                     ctypes.c_void_p]),
    "fm_ea_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_void_p]),
    "fm_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int, ctypes.POINTER(fm_adam_opts), ctypes.c_int32,
                               ctypes.c_void_p]),
    "fm_mlp_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_mlp_eval": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_float, ctypes.c_float,
                                   ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fm_mlp_eval_relative": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p]),
    "fm_mlp_prune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                    ctypes.POINTER(ctypes.c_int64)]),
    "fm_mlp_reweight": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                       ctypes.c_int32, ctypes.POINTER(ctypes.c_int64)]),
    "fm_mlp_trainer_create": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "fm_mlp_trainer_destroy": (None, [ctypes.c_void_p]),
    "fm_mlp_trainer_set_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_mlp_trainer_get_params": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_mlp_trainer_loss_grad": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                                ctypes.c_void_p, ctypes.c_void_p]),
    "fm_mlp_trainer_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64,
                                           ctypes.POINTER(fm_adam_opts), ctypes.c_void_p]),
    "fm_mlp_trainer_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p]),
    "fm_set_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fm_tuning)]),
    "fm_get_tuning": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fm_tuning)]),
    "fm_autotune": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(fm_tuning)]),
    "fm_graphs_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fm_timing_enable": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fm_timing_read": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fm_kernel_time), ctypes.c_int32,
                                      ctypes.POINTER(ctypes.c_int32)]),
    "fm_track_loss": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32]),
    "fm_loss_history": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_float), ctypes.c_int32,
                                       ctypes.POINTER(ctypes.c_int32)]),
    "fm_rotation_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "fm_relative_translations": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_relative_poses": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                         ctypes.POINTER(ctypes.c_int32)]),
    "fm_focal_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                       ctypes.c_float, ctypes.c_int32, ctypes.c_float, ctypes.c_int32,
                                       ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32)]),
    "fm_set_focal": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_distortion_search": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_float,
                                            ctypes.c_float, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                            ctypes.POINTER(ctypes.c_int32)]),
    "fm_distortion_pair_errors": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p,
                                                 ctypes.c_int32]),
    "fm_set_distortion": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_ea_focal_forward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                           ctypes.c_void_p]),
    "fm_ea_focal_backward": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                            ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p]),
    "fm_tracks_complete": (ctypes.c_int, [ctypes.c_int32, ctypes.c_void_p, ctypes.c_int64, ctypes.c_void_p,
                                          ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                          ctypes.POINTER(ctypes.c_void_p)]),
    "fm_tracks_info": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64),
                                      ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]),
    "fm_tracks_copy": (ctypes.c_int, [ctypes.c_void_p] + [ctypes.c_void_p] * 8 + [ctypes.c_int32]),
    "fm_tracks_destroy": (None, [ctypes.c_void_p]),
    "fm_filter_image_pairs": (ctypes.c_int, [ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.c_double, ctypes.c_double, ctypes.c_void_p,
                                             ctypes.c_void_p, ctypes.POINTER(ctypes.c_double)]),
    "fm_get_rel_poses": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32]),
    "fm_translation_random_init": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_uint32]),
    "fm_translation_merge": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "fm_epipolar_init_from_stages": (ctypes.c_int, [ctypes.c_void_p]),
    "fm_triangulate": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fm_tri_opts), ctypes.c_void_p, ctypes.c_void_p,
                                      ctypes.c_void_p, ctypes.c_int32, ctypes.POINTER(ctypes.c_int32)]),
    "fm_solve_opts_default": (None, [ctypes.POINTER(fm_solve_opts)]),
    "fm_solve": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(fm_solve_opts), ctypes.POINTER(fm_result)]),
    "fm_ea_loss_grad_static": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                              ctypes.c_int64, ctypes.c_int32, ctypes.c_float, ctypes.c_void_p,
                                              ctypes.c_void_p, ctypes.c_void_p]),
}

_LIB = None


def library_path() -> str:
    return _build.LIB


def lib():
    """Loads lib/libfastmap.so (raises if it has not been built)."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with `python -m paper_2505_04612_b300.build`")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _LIB = L
    return _LIB


class FastMapError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"fastmap status {status}: {message}")
        self.status = status


def _check(status, handle=None):
    if status != FM_OK:
        msg = lib().fm_last_error(handle)
        raise FastMapError(status, msg.decode() if msg else "")


# ------------------------------------------------------------- marshalling

def _ptr(x):
    """(address, on_device, keepalive) of a torch tensor / numpy array / None."""
    if x is None:
        return None, False, None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if not x.is_contiguous():
                x = x.contiguous()
            return x.data_ptr(), x.is_cuda, x
    except ImportError:  # pragma: no cover
        pass
    a = np.ascontiguousarray(x)
    return a.ctypes.data, False, a


def _as(x, dtype):
    """Convert to the given numpy dtype unless it is a tensor of the right dtype."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            want = {np.float32: torch.float32, np.int32: torch.int32}[dtype]
            if x.dtype == want and x.is_contiguous():   # nothing to convert: no dispatch
                return x
            return x.to(want).contiguous()
    except ImportError:  # pragma: no cover
        pass
    return np.ascontiguousarray(x, dtype=dtype)


def _stream_handle(stream):
    if stream is not None:
        return stream
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except ImportError:  # pragma: no cover
        pass
    return None


# ------------------------------------------------------------ C-named calls

def fm_problem_create(desc: fm_problem_desc) -> int:
    h = ctypes.c_void_p()
    _check(lib().fm_problem_create(ctypes.byref(desc), ctypes.byref(h)), None)
    return h.value


def fm_problem_destroy(handle):
    lib().fm_problem_destroy(handle)


def fm_last_error(handle=None) -> str:
    return lib().fm_last_error(handle).decode()


def fm_problem_info_get(handle) -> fm_problem_info:
    info = fm_problem_info()
    _check(lib().fm_problem_info_get(handle, ctypes.byref(info)), handle)
    return info


def fm_set_params(handle, stage, params):
    p, dev, keep = _ptr(_as(params, np.float32))
    _check(lib().fm_set_params(handle, stage, p, int(dev)), handle)


def fm_get_params(handle, stage, out):
    p, dev, keep = _ptr(out)
    _check(lib().fm_get_params(handle, stage, p, int(dev)), handle)
    return out


def fm_set_rel_poses(handle, rel_R=None, rel_t=None):
    rR = _as(rel_R, np.float32) if rel_R is not None else None
    rt = _as(rel_t, np.float32) if rel_t is not None else None
    pR, dR, kR = _ptr(rR)
    pt, dt, kt = _ptr(rt)
    if rR is not None and rt is not None and dR != dt:
        raise ValueError("rel_R and rel_t must both be on the device or both on the host")
    _check(lib().fm_set_rel_poses(handle, pR, pt, int(dR or dt)), handle)


def fm_translation_set_runs(handle, n_runs):
    _check(lib().fm_translation_set_runs(handle, int(n_runs)), handle)


def fm_ea_set_loss(handle, loss):
    _check(lib().fm_ea_set_loss(handle, int(loss)), handle)


def fm_ea_set_weights(handle, weights, inv_z):
    if weights is None:
        _check(lib().fm_ea_set_weights(handle, None, 0, ctypes.c_float(0.0)), handle)
        return
    p, dev, keep = _ptr(_as(weights, np.float32))
    _check(lib().fm_ea_set_weights(handle, p, int(dev), ctypes.c_float(inv_z)), handle)


def fm_ea_reweight(handle, tau, delta, irls=True):
    kept = ctypes.c_int64()
    _check(lib().fm_ea_reweight(handle, ctypes.c_float(tau), ctypes.c_float(delta), int(bool(irls)),
                                ctypes.byref(kept)), handle)
    return kept.value


def fm_kp_order(handle, out):
    """The library's keypoint-pair order: out[k] = caller index of internal
    position k (a numpy int32 array or a CUDA int32 tensor of Z entries)."""
    p, dev, keep = _ptr(out)
    _check(lib().fm_kp_order(handle, p, int(dev)), handle)
    return out


def fm_ea_get_weights(handle, out):
    p, dev, keep = _ptr(out)
    inv_z = ctypes.c_float()
    _check(lib().fm_ea_get_weights(handle, p, int(dev), ctypes.byref(inv_z)), handle)
    return out, inv_z.value


def fm_loss_grad(handle, stage, params, loss_out, grad_out, mem_on_device):
    """Raw call: params / grad_out are addresses (int) or None, loss_out a
    ctypes float array or None."""
    _check(lib().fm_loss_grad(handle, stage, params, loss_out, grad_out, int(mem_on_device)), handle)


def fm_ea_forward(handle, params_dev, loss_dev, save, saved_dev):
    """Raw call: device addresses (int) or None."""
    _check(lib().fm_ea_forward(handle, params_dev, loss_dev, int(save), saved_dev), handle)


def fm_ea_backward(handle, params_dev, save, saved_dev, grad_loss_dev, grad_dev):
    """Raw call: device addresses (int) or None."""
    _check(lib().fm_ea_backward(handle, params_dev, int(save), saved_dev, grad_loss_dev, grad_dev), handle)


def fm_step(handle, stage, opts: fm_adam_opts, n_iters, loss_out=None):
    _check(lib().fm_step(handle, stage, ctypes.byref(opts), int(n_iters), loss_out), handle)


def fm_timing_enable(handle, enable):
    _check(lib().fm_timing_enable(handle, int(bool(enable))), handle)


def fm_timing_read(handle):
    """{kernel name: (launches, total device ms)} since timing was enabled."""
    cap = 32
    arr = (fm_kernel_time * cap)()
    n = ctypes.c_int32()
    _check(lib().fm_timing_read(handle, arr, cap, ctypes.byref(n)), handle)
    return {arr[k].name.decode(): (int(arr[k].launches), float(arr[k].total_ms)) for k in range(min(n.value, cap))}


def fm_track_loss(handle, every, capacity=4096):
    _check(lib().fm_track_loss(handle, int(every), int(capacity)), handle)


def fm_loss_history(handle, capacity=4096):
    out = (ctypes.c_float * capacity)()
    n = ctypes.c_int32()
    _check(lib().fm_loss_history(handle, out, capacity, ctypes.byref(n)), handle)
    return [out[k] for k in range(n.value)]


def fm_ea_loss_grad_static(kp, seg_off, pair_i, pair_j, params, weights, n_cams, loss, inv_z,
                           loss_out, pair_grad_out, stream=None, n_kp_pairs=None):
    """Allocation-free direct epipolar loss + per-image-pair gradient blocks.
    Every array is a CUDA tensor (kp float32 [Z,4], seg_off int32 [P+1],
    pair_i/pair_j int32 [P], params float32 [N*9], weights float32 [Z] or
    None, loss_out float32 [1], pair_grad_out float32 [P*24]).  Z is taken
    from kp unless n_kp_pairs is given (at most the pairs kp holds)."""
    args = [_ptr(a) for a in (kp, seg_off, pair_i, pair_j, params, weights, loss_out, pair_grad_out)]
    for a, (addr, dev, _) in zip(("kp", "seg_off", "pair_i", "pair_j", "params", "weights", "loss_out",
                                  "pair_grad_out"), args):
        if addr is not None and not dev:
            raise ValueError(f"{a} must be a CUDA tensor")
    P = int(pair_i.numel())
    Z = int(kp.numel() // 4)
    if n_kp_pairs is not None:
        if not 0 <= int(n_kp_pairs) <= Z:
            raise ValueError("n_kp_pairs must lie in [0, the pairs kp holds]")
        Z = int(n_kp_pairs)
    st = lib().fm_ea_loss_grad_static(args[0][0], args[1][0], args[2][0], args[3][0], args[4][0], args[5][0],
                                      int(n_cams), P, Z, int(loss), ctypes.c_float(inv_z), args[6][0],
                                      args[7][0], _stream_handle(stream))
    _check(st, None)


def complete_tracks(kp_off, matches, kp_px=None, min_pairs=1):
    """fm_tracks_complete + fm_tracks_copy.  Inputs as numpy arrays (host) or
    CUDA tensors (device; outputs then stay on the device as tensors).
    Returns a dict: pair_i, pair_j [P]; kp_img_pair, node1, node2, kp_track
    [Z]; kp1_px, kp2_px [Z,2] when kp_px is given; n_tracks, n_inconsistent."""
    dev = hasattr(matches, "is_cuda") and matches.is_cuda
    if dev:
        import torch
        off = kp_off.to(torch.int32).contiguous()
        m = matches.to(torch.int32).contiguous().reshape(-1, 2)
        px = None if kp_px is None else kp_px.to(torch.float32).contiguous()
        torch.cuda.current_stream().synchronize()   # the library reads them on its own stream
        a_off, a_m, a_px = off.data_ptr(), m.data_ptr(), (None if px is None else px.data_ptr())
        n_img, n_m = off.numel() - 1, m.shape[0]
    else:
        off = np.ascontiguousarray(kp_off, dtype=np.int32)
        m = np.ascontiguousarray(matches, dtype=np.int32).reshape(-1, 2)
        px = None if kp_px is None else np.ascontiguousarray(kp_px, dtype=np.float32)
        a_off, a_m, a_px = off.ctypes.data, m.ctypes.data, (None if px is None else px.ctypes.data)
        n_img, n_m = len(off) - 1, len(m)
    h = ctypes.c_void_p()
    _check(lib().fm_tracks_complete(int(n_img), a_off, int(n_m), a_m if n_m else None, a_px, int(min_pairs),
                                    int(dev), ctypes.byref(h)))
    try:
        nt, P, Z, ni = (ctypes.c_int64() for _ in range(4))
        _check(lib().fm_tracks_info(h, ctypes.byref(nt), ctypes.byref(P), ctypes.byref(Z), ctypes.byref(ni)))
        P, Z = P.value, Z.value
        if dev:
            import torch
            mk = lambda *shape, dt=torch.int32: torch.empty(shape, dtype=dt, device=m.device)  # noqa: E731
            ptr = lambda a: a.data_ptr()  # noqa: E731
        else:
            mk = lambda *shape, dt=np.int32: np.empty(shape, dtype=dt)  # noqa: E731
            ptr = lambda a: a.ctypes.data  # noqa: E731
        f32 = (torch.float32 if dev else np.float32)
        out = dict(pair_i=mk(P), pair_j=mk(P), kp_img_pair=mk(Z), node1=mk(Z), node2=mk(Z), kp_track=mk(Z))
        if px is not None:
            out["kp1_px"] = mk(Z, 2, dt=f32)
            out["kp2_px"] = mk(Z, 2, dt=f32)
        _check(lib().fm_tracks_copy(h, *(ptr(out[k]) for k in ["pair_i", "pair_j", "kp_img_pair", "node1", "node2",
                                                              "kp_track"]),
                                    ptr(out["kp1_px"]) if px is not None else None,
                                    ptr(out["kp2_px"]) if px is not None else None, int(dev)))
        out["n_tracks"] = nt.value
        out["n_inconsistent"] = ni.value
        return out
    finally:
        lib().fm_tracks_destroy(h)


def filter_image_pairs(n_images, pair_i, pair_j, counts, t_start, t_min):
    """fm_filter_image_pairs (host): returns (keep [P] bool, image_valid [N]
    bool, threshold used)."""
    pi = np.ascontiguousarray(pair_i, dtype=np.int32)
    pj = np.ascontiguousarray(pair_j, dtype=np.int32)
    c = np.ascontiguousarray(counts, dtype=np.int32)
    keep = np.empty(len(pi), np.int32)
    valid = np.empty(int(n_images), np.int32)
    t = ctypes.c_double()
    _check(lib().fm_filter_image_pairs(int(n_images), len(pi), pi.ctypes.data, pj.ctypes.data, c.ctypes.data,
                                       ctypes.c_double(t_start), ctypes.c_double(t_min), keep.ctypes.data,
                                       valid.ctypes.data, ctypes.byref(t)))
    return keep.astype(bool), valid.astype(bool), t.value


def fm_mlp_set_params(handle, theta):
    p, dev, keep = _ptr(None if theta is None else _as(theta, np.float32))
    _check(lib().fm_mlp_set_params(handle, p, int(dev)), handle)


class MlpTrainer:
    """Owner of an fm_mlp_trainer (device parameters + Adam state)."""

    def __init__(self, max_batch, stream=None):
        h = ctypes.c_void_p()
        _check(lib().fm_mlp_trainer_create(int(max_batch), _stream_handle(stream), ctypes.byref(h)), None)
        self.handle = h.value
        self.max_batch = int(max_batch)

    def close(self):
        if getattr(self, "handle", None):
            lib().fm_mlp_trainer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_params(self, theta):
        p, dev, keep = _ptr(_as(theta, np.float32))
        _check(lib().fm_mlp_trainer_set_params(self.handle, p, int(dev)), None)

    def get_params(self):
        out = np.empty(4801, np.float32)
        _check(lib().fm_mlp_trainer_get_params(self.handle, out.ctypes.data, 0), None)
        return out

    def loss_grad(self, x, y):
        """x [B,8], y [B] CUDA float32 tensors -> (loss, grad [4801]) tensors."""
        import torch
        loss = torch.empty(1, dtype=torch.float32, device=x.device)
        grad = torch.empty(4801, dtype=torch.float32, device=x.device)
        _check(lib().fm_mlp_trainer_loss_grad(self.handle, x.data_ptr(), y.data_ptr(), int(y.numel()),
                                              loss.data_ptr(), grad.data_ptr()), None)
        return loss, grad

    def step(self, x, y, lr, beta1=0.9, beta2=0.999, eps=1e-8, loss_out=None):
        opts = fm_adam_opts(lr, beta1, beta2, eps)
        _check(lib().fm_mlp_trainer_step(self.handle, x.data_ptr(), y.data_ptr(), int(y.numel()),
                                         ctypes.byref(opts), None if loss_out is None else loss_out.data_ptr()),
               None)

    def forward(self, x):
        import torch
        out = torch.empty(x.shape[0], dtype=torch.float32, device=x.device)
        _check(lib().fm_mlp_trainer_forward(self.handle, x.data_ptr(), int(x.shape[0]), out.data_ptr()), None)
        return out


def solve_opts(**overrides) -> fm_solve_opts:
    o = fm_solve_opts()
    lib().fm_solve_opts_default(ctypes.byref(o))
    for k, v in overrides.items():
        setattr(o, k, v)
    return o


# ------------------------------------------------------------ owner class

class Problem:
    """One fm_problem.  Inputs may be numpy arrays / CPU tensors (copied from
    the host) or CUDA tensors (read on the device); all of them must be on the
    same side.  scene_cam_off ([S+1] camera offsets, host) makes a problem of
    S independent scenes whose losses come back per scene."""

    def __init__(self, pair_i, pair_j, kp_img_pair, kp1_px, kp2_px, focal, cx, cy,
                 rel_R=None, rel_t=None, kp_track=None, stream=None, scene_cam_off=None):
        arrs = dict(
            pair_cam_i=_as(pair_i, np.int32), pair_cam_j=_as(pair_j, np.int32),
            kp_img_pair=_as(kp_img_pair, np.int32),
            kp1_px=_as(kp1_px, np.float32), kp2_px=_as(kp2_px, np.float32),
            focal=_as(focal, np.float32), cx=_as(cx, np.float32), cy=_as(cy, np.float32),
            rel_R=_as(rel_R, np.float32) if rel_R is not None else None,
            rel_t=_as(rel_t, np.float32) if rel_t is not None else None,
            kp_track=_as(kp_track, np.int32) if kp_track is not None else None,
        )
        d = fm_problem_desc()
        d.n_cams = int(len(arrs["focal"]))
        d.n_img_pairs = int(len(arrs["pair_cam_i"]))
        d.n_kp_pairs = int(len(arrs["kp_img_pair"]))
        self._keep = []
        sides = set()
        for k, v in arrs.items():
            p, dev, keep = _ptr(v)
            setattr(d, k, p)
            if v is not None:
                sides.add(dev)
                self._keep.append(keep)
        if len(sides) > 1:
            raise ValueError("all inputs must be on the device or all on the host")
        d.inputs_on_device = int(sides == {True})
        d.cuda_stream = _stream_handle(stream)
        self.S = 1
        if scene_cam_off is not None:
            off = np.ascontiguousarray(np.asarray(scene_cam_off), dtype=np.int32)
            self._keep.append(off)
            d.n_scenes = int(len(off) - 1)
            d.scene_cam_off = off.ctypes.data
            self.S = max(int(len(off) - 1), 1)
        self.n_cams, self.n_pairs, self.n_kp = d.n_cams, d.n_img_pairs, d.n_kp_pairs
        self.handle = fm_problem_create(d)
        self._keep = []
        self.runs = 1

    def close(self):
        if getattr(self, "handle", None):
            fm_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def info(self):
        return fm_problem_info_get(self.handle)

    def n_params(self, stage):
        return STAGE_DIM[stage] * self.n_cams * (self.runs if stage == FM_STAGE_TRANSLATION else 1)

    def set_params(self, stage, params):
        fm_set_params(self.handle, stage, params)

    def get_params(self, stage):
        import torch
        out = torch.empty(self.n_params(stage), dtype=torch.float32, device="cuda")
        fm_get_params(self.handle, stage, out)
        return out

    def set_rel_poses(self, rel_R=None, rel_t=None):
        fm_set_rel_poses(self.handle, rel_R, rel_t)

    def set_translation_runs(self, n_runs):
        fm_translation_set_runs(self.handle, n_runs)
        self.runs = int(n_runs)

    def set_ea_loss(self, loss):
        fm_ea_set_loss(self.handle, loss)

    def set_ea_weights(self, weights, inv_z=None):
        """inv_z None: each scene's 1/(number of its positive weights),
        computed by the library."""
        fm_ea_set_weights(self.handle, weights, inv_z if inv_z is not None else 0.0)

    def reweight(self, tau, delta, irls=True):
        """IRLS weights + filtering at the current epipolar parameters; returns #kept."""
        return fm_ea_reweight(self.handle, tau, delta, irls)

    def kp_order(self):
        """numpy int32 [Z]: the caller index of each internal keypoint-pair
        position (fm_kp_order)."""
        return fm_kp_order(self.handle, np.empty(self.n_kp, np.int32))

    def get_weights(self):
        import torch
        out = torch.empty(self.n_kp, dtype=torch.float32, device="cuda")
        return fm_ea_get_weights(self.handle, out)

    def loss_grad(self, stage, params, want_loss=True, want_grad=True, grad_out=None):
        """params: CUDA tensor (device path), or numpy array / CPU tensor (host
        path).  Returns (loss, grad) with grad of the same kind as params, or
        grad_out when given (same side as params)."""
        nruns = self.runs if stage == FM_STAGE_TRANSLATION else 1
        loss = (ctypes.c_float * (nruns * self.S))() if want_loss else None
        p = _as(params, np.float32)
        addr, dev, keep = _ptr(p)
        grad = None
        gaddr = None
        if want_grad:
            if grad_out is not None:
                grad = grad_out
                gaddr, gdev, _ = _ptr(grad_out)
                if gdev != dev:
                    raise ValueError("grad_out must be on the same side as params")
            elif dev:
                import torch
                grad = torch.empty_like(p)
                gaddr = grad.data_ptr()
            else:
                grad = np.empty(np.asarray(p).shape, dtype=np.float32)
                gaddr = grad.ctypes.data
        fm_loss_grad(self.handle, stage, addr, loss, gaddr, int(dev))
        lv = self._losses(loss, nruns) if want_loss else None
        return lv, grad

    def _losses(self, loss, nruns):
        """One scene: a float ([m] for m translation runs); S scenes: [S]
        (or [m][S])."""
        vals = [loss[k] for k in range(nruns * self.S)]
        if self.S == 1:
            return vals[0] if nruns == 1 else vals
        if nruns == 1:
            return vals
        return [vals[r * self.S:(r + 1) * self.S] for r in range(nruns)]

    def mlp_set_params(self, theta):
        fm_mlp_set_params(self.handle, theta)

    def mlp_eval(self, params=None, iter_frac=0.0, delta=1e-5, want_feat=True, want_resid=True, want_prob=False):
        """fm_mlp_eval on the device; returns (feat [Z,8], resid [Z], prob [Z])
        (None for outputs not asked for)."""
        import torch
        feat = torch.empty((self.n_kp, 8), dtype=torch.float32, device="cuda") if want_feat else None
        resid = torch.empty(self.n_kp, dtype=torch.float32, device="cuda") if want_resid else None
        prob = torch.empty(self.n_kp, dtype=torch.float32, device="cuda") if want_prob else None
        pp = None if params is None else _ptr(_as(params, np.float32))[0]
        _check(lib().fm_mlp_eval(self.handle, pp, ctypes.c_float(iter_frac), ctypes.c_float(delta),
                                 None if feat is None else feat.data_ptr(),
                                 None if resid is None else resid.data_ptr(),
                                 None if prob is None else prob.data_ptr()), self.handle)
        return feat, resid, prob

    def mlp_eval_relative(self, iter_frac=0.0, delta=1e-5, want_feat=True, want_resid=True, want_prob=False):
        """fm_mlp_eval_relative (rotation stage + relative translations)."""
        import torch
        feat = torch.empty((self.n_kp, 8), dtype=torch.float32, device="cuda") if want_feat else None
        resid = torch.empty(self.n_kp, dtype=torch.float32, device="cuda") if want_resid else None
        prob = torch.empty(self.n_kp, dtype=torch.float32, device="cuda") if want_prob else None
        _check(lib().fm_mlp_eval_relative(self.handle, ctypes.c_float(iter_frac), ctypes.c_float(delta),
                                          None if feat is None else feat.data_ptr(),
                                          None if resid is None else resid.data_ptr(),
                                          None if prob is None else prob.data_ptr()), self.handle)
        return feat, resid, prob

    def mlp_prune(self, iter_frac=0.0, delta=1e-5, p_min=0.5):
        kept = ctypes.c_int64()
        _check(lib().fm_mlp_prune(self.handle, ctypes.c_float(iter_frac), ctypes.c_float(delta),
                                  ctypes.c_float(p_min), ctypes.byref(kept)), self.handle)
        return kept.value

    def mlp_reweight(self, iter_frac, delta=1e-5, p_min=0.5, irls=True):
        kept = ctypes.c_int64()
        _check(lib().fm_mlp_reweight(self.handle, ctypes.c_float(iter_frac), ctypes.c_float(delta),
                                     ctypes.c_float(p_min), int(bool(irls)), ctypes.byref(kept)), self.handle)
        return kept.value

    def autotune(self, repeats=5):
        """fm_autotune; returns the chosen fm_tuning as a dict."""
        t = fm_tuning()
        _check(lib().fm_autotune(self.handle, int(repeats), ctypes.byref(t)), self.handle)
        return dict(pairs_per_lane=t.pairs_per_lane, ctas_per_sm=t.ctas_per_sm, us_per_eval=t.us_per_eval)

    def set_tuning(self, pairs_per_lane=15, ctas_per_sm=0):
        t = fm_tuning(pairs_per_lane, ctas_per_sm, 0.0)
        _check(lib().fm_set_tuning(self.handle, ctypes.byref(t)), self.handle)

    def get_tuning(self):
        t = fm_tuning()
        _check(lib().fm_get_tuning(self.handle, ctypes.byref(t)), self.handle)
        return dict(pairs_per_lane=t.pairs_per_lane, ctas_per_sm=t.ctas_per_sm)

    def graphs(self, enable=True):
        _check(lib().fm_graphs_enable(self.handle, int(bool(enable))), self.handle)

    def timing(self, enable=True):
        fm_timing_enable(self.handle, enable)

    def timing_read(self):
        return fm_timing_read(self.handle)

    def track_loss(self, every, capacity=4096):
        fm_track_loss(self.handle, every, capacity)

    def loss_history(self, capacity=4096):
        return fm_loss_history(self.handle, capacity)

    def rotation_init(self, n_iters=2000):
        _check(lib().fm_rotation_init(self.handle, int(n_iters)), self.handle)

    def relative_translations(self):
        err = np.empty(self.n_pairs, np.float32)
        _check(lib().fm_relative_translations(self.handle, err.ctypes.data, 0), self.handle)
        return err

    def relative_poses(self, irls_iters=0, delta=1e-5):
        """fm_relative_poses: estimates rel_R / rel_t from the keypoints; returns
        the number of image pairs estimated."""
        n = ctypes.c_int32()
        _check(lib().fm_relative_poses(self.handle, int(irls_iters), ctypes.c_float(delta), ctypes.byref(n)),
               self.handle)
        return n.value

    def focal_search(self, group=None, n_groups=1, rho_min=1.0 / 3.0, rho_max=3.0, n_cand=1024, tau=0.01,
                     irls_iters=0):
        """fm_focal_search; returns (focal [N] float32, number of groups estimated)."""
        out = np.empty(self.n_cams, np.float32)
        g = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
        n = ctypes.c_int32()
        _check(lib().fm_focal_search(self.handle, None if g is None else g.ctypes.data, int(n_groups),
                                     ctypes.c_float(rho_min), ctypes.c_float(rho_max), int(n_cand),
                                     ctypes.c_float(tau), int(irls_iters), out.ctypes.data, ctypes.byref(n)),
               self.handle)
        return out, n.value

    def set_focal(self, focal):
        f = np.ascontiguousarray(focal, dtype=np.float32)
        _check(lib().fm_set_focal(self.handle, f.ctypes.data, 0), self.handle)

    def distortion_search(self, group=None, n_groups=1, alpha_min=-0.5, alpha_max=0.5, n_cand=32, n_levels=3):
        """fm_distortion_search; returns (alpha [N] float32, number of groups estimated)."""
        out = np.empty(self.n_cams, np.float32)
        g = None if group is None else np.ascontiguousarray(group, dtype=np.int32)
        n = ctypes.c_int32()
        _check(lib().fm_distortion_search(self.handle, None if g is None else g.ctypes.data, int(n_groups),
                                          ctypes.c_float(alpha_min), ctypes.c_float(alpha_max), int(n_cand),
                                          int(n_levels), out.ctypes.data, ctypes.byref(n)), self.handle)
        return out, n.value

    def distortion_pair_errors(self, alpha_cand):
        """fm_distortion_pair_errors; returns [P, n_cand] float32 on the side
        of alpha_cand (numpy array or CUDA tensor)."""
        if hasattr(alpha_cand, "is_cuda") and alpha_cand.is_cuda:
            import torch
            c = alpha_cand.to(torch.float32).contiguous().reshape(-1)
            out = torch.empty((self.n_pairs, c.numel()), dtype=torch.float32, device=c.device)
            _check(lib().fm_distortion_pair_errors(self.handle, c.data_ptr(), c.numel(), out.data_ptr(), 1),
                   self.handle)
            return out
        c = np.ascontiguousarray(alpha_cand, dtype=np.float32).reshape(-1)
        out = np.empty((self.n_pairs, len(c)), np.float32)
        _check(lib().fm_distortion_pair_errors(self.handle, c.ctypes.data, len(c), out.ctypes.data, 0),
               self.handle)
        return out

    def set_distortion(self, alpha):
        a = np.ascontiguousarray(alpha, dtype=np.float32)
        _check(lib().fm_set_distortion(self.handle, a.ctypes.data, 0), self.handle)

    def get_rel_poses(self, want_R=True, want_t=True):
        R = np.empty((self.n_pairs, 3, 3), np.float32) if want_R else None
        t = np.empty((self.n_pairs, 3), np.float32) if want_t else None
        _check(lib().fm_get_rel_poses(self.handle, R.ctypes.data if want_R else None,
                                      t.ctypes.data if want_t else None, 0), self.handle)
        return R, t

    def translation_random_init(self, seed=0):
        _check(lib().fm_translation_random_init(self.handle, ctypes.c_uint32(seed)), self.handle)

    def translation_merge(self):
        best = np.empty(self.n_cams, np.int32)
        _check(lib().fm_translation_merge(self.handle, best.ctypes.data), self.handle)
        self.runs = 1
        return best

    def epipolar_init_from_stages(self):
        _check(lib().fm_epipolar_init_from_stages(self.handle), self.handle)

    def triangulate(self, max_err_px=4.0, min_angle_deg=2.0):
        T = ctypes.c_int32()
        opts = fm_tri_opts(max_err_px, min_angle_deg)
        _check(lib().fm_triangulate(self.handle, ctypes.byref(opts), None, None, None, 0, ctypes.byref(T)),
               self.handle)
        n = T.value
        pts = np.empty((n, 3), np.float32)
        valid = np.empty(n, np.int32)
        ncam = np.empty(n, np.int32)
        _check(lib().fm_triangulate(self.handle, ctypes.byref(opts), pts.ctypes.data, valid.ctypes.data,
                                    ncam.ctypes.data, 0, ctypes.byref(T)), self.handle)
        return pts, valid.astype(bool), ncam

    def solve(self, n_tracks=None, **overrides):
        """fm_solve; returns a dict with R [N,3,3], t [N,3], points/valid (if
        the problem has tracks) and the final losses."""
        opts = solve_opts(**overrides)
        R = np.empty((self.n_cams, 3, 3), np.float32)
        t = np.empty((self.n_cams, 3), np.float32)
        res = fm_result()
        res.R = R.ctypes.data
        res.t = t.ctypes.data
        cam_valid = np.empty(self.n_cams, np.int32)
        res.cam_valid = cam_valid.ctypes.data
        pts = valid = None
        if n_tracks:
            pts = np.empty((n_tracks, 3), np.float32)
            valid = np.empty(n_tracks, np.int32)
            res.points = pts.ctypes.data
            res.point_valid = valid.ctypes.data
        _check(lib().fm_solve(self.handle, ctypes.byref(opts), ctypes.byref(res)), self.handle)
        self.runs = 1
        out = dict(R=R, t=t, loss_rotation=res.loss_rotation, loss_translation=res.loss_translation,
                   loss_epipolar=res.loss_epipolar, n_kept=res.n_kept, n_points_valid=res.n_points_valid,
                   cam_valid=cam_valid.astype(bool))
        if n_tracks:
            out.update(points=pts[:res.n_tracks], point_valid=valid[:res.n_tracks].astype(bool))
        return out

    def step(self, stage, n_iters, lr, beta1=0.9, beta2=0.999, eps=1e-8, want_loss=False):
        opts = fm_adam_opts(lr, beta1, beta2, eps)
        nruns = self.runs if stage == FM_STAGE_TRANSLATION else 1
        loss = (ctypes.c_float * (nruns * self.S))() if want_loss else None
        fm_step(self.handle, stage, opts, n_iters, loss)
        if want_loss:
            return self._losses(loss, nruns)
        return None


def problem_from_scene(scene, rel_R=None, rel_t=None, device=True, stream=None):
    """Builds a Problem from a ``synthetic.scenes.Scene``-like object (fields
    pair_i, pair_j, kp_img_pair, kp1_px, kp2_px, focal, cx, cy, kp_track, and
    scene_cam_off for a batch of scenes)."""
    arrays = [scene.pair_i, scene.pair_j, scene.kp_img_pair, scene.kp1_px, scene.kp2_px,
              scene.focal, scene.cx, scene.cy]
    extra = dict(rel_R=rel_R, rel_t=rel_t, kp_track=scene.kp_track)
    if device:
        import torch

        def dv(a, dt):
            return None if a is None else torch.as_tensor(np.ascontiguousarray(a, dtype=dt)).cuda()
        dts = [np.int32, np.int32, np.int32, np.float32, np.float32, np.float32, np.float32, np.float32]
        arrays = [dv(a, dt) for a, dt in zip(arrays, dts)]
        extra = dict(rel_R=dv(rel_R, np.float32), rel_t=dv(rel_t, np.float32),
                     kp_track=dv(scene.kp_track, np.int32))
    return Problem(*arrays, stream=stream, scene_cam_off=getattr(scene, "scene_cam_off", None), **extra)
