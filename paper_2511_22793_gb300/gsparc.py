"""Thin Python binding of libgsparc.so (the C ABI declared in include/gsparc.h).

Argument marshalling only: every function takes torch tensors that already
live on the GPU (outputs included), passes their device pointers, sizes and
the current CUDA stream to the C entry point of the same name, and raises
GsparcError on a non-zero status.  No step of the computation runs here.
The library is loaded on first use; if it has not been built the call fails
loudly instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes
import os

import torch

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libgsparc.so")

GSPARC_OK = 0
GSPARC_ERR_INVALID = -1
GSPARC_ERR_WORKSPACE = -2
GSPARC_ERR_CUDA = -3
GSPARC_ERR_TIMEOUT = -4
GSPARC_ERR_CAPACITY = -5
GSPARC_ERR_TOO_LARGE = -6
GSPARC_ERR_INPUT = -7
GSPARC_NOALLOC_MAX_N = 65536
GSPARC_NOALLOC_MAX_PAIRS = 524288
GSPARC_OVERLAP_BIN_SORT, GSPARC_OVERLAP_FORWARD, GSPARC_OVERLAP_SCHEDULE = 1, 2, 4
GSPARC_OVERLAP_BACKWARD, GSPARC_OVERLAP_NETWORK, GSPARC_OVERLAP_ALL = 8, 16, 31
GSPARC_FP32, GSPARC_BF16, GSPARC_BF16X2 = 0, 1, 2
TILE = 16
PROJ_STRIDE = 8

EXPORTS = [
    "gsparc_num_tiles", "gsparc_project", "gsparc_project_bwd", "gsparc_bin_sort_workspace",
    "gsparc_bin_sort", "gsparc_bin_sort_noalloc", "gsparc_attr_mlp", "gsparc_attr_mlp_bwd",
    "gsparc_attr_mlp_bwd_tc", "gsparc_emission_stride", "gsparc_emission_fwd", "gsparc_emission_bwd", "gsparc_render_fwd", "gsparc_render_fwd_l2", "gsparc_render_fwd_tc",
    "gsparc_render_bwd", "gsparc_render_bwd_workspace", "gsparc_render_bwd_balanced",
    "gsparc_render_bwd_tc", "gsparc_render_bwd_tc_workspace", "gsparc_render_bwd_tc_balanced",
    "gsparc_l2_loss", "gsparc_csi_head", "gsparc_csi_loss", "gsparc_csi_head_bwd",
    "gsparc_spectrum_loss_workspace", "gsparc_spectrum_loss",
    "gsparc_render_csi_tc", "gsparc_render_fwd_l2_tc", "gsparc_confidence", "gsparc_densify_accumulate",
    "gsparc_densify_workspace", "gsparc_densify", "gsparc_opacity_reset", "gsparc_adam", "gsparc_adam_segments", "gsparc_scale_rows",
    "gsparc_set_wait_limit", "gsparc_set_launch_overlap",
    "gsparc_check", "gsparc_strerror",
]


class GsparcError(RuntimeError):
    def __init__(self, fn, code):
        self.code = code
        super().__init__("%s failed: %d (%s)" % (fn, code, strerror(code)))


class View(ctypes.Structure):
    _fields_ = [("H", ctypes.c_int32), ("W", ctypes.c_int32), ("rx", ctypes.c_float * 3),
                ("V", ctypes.c_float * 9), ("near_dist", ctypes.c_float)]


class Band(ctypes.Structure):
    _fields_ = [("K", ctypes.c_int32), ("reserved", ctypes.c_int32), ("f_c", ctypes.c_double),
                ("df", ctypes.c_double)]


class MLP(ctypes.Structure):
    _fields_ = [("hidden", ctypes.c_int32), ("reserved", ctypes.c_int32)] + \
               [(n, ctypes.c_void_p) for n in ("W1", "b1", "W2", "b2", "W3", "b3")]


class DensifyParams(ctypes.Structure):
    _fields_ = [("tau_grad", ctypes.c_float), ("clone_scale", ctypes.c_float), ("sigma_min", ctypes.c_float),
                ("r_max", ctypes.c_float), ("n_split", ctypes.c_int32)]


class MLPGrad(ctypes.Structure):
    _fields_ = [(n, ctypes.c_void_p) for n in ("W1", "b1", "W2", "b2", "W3", "b3")]


_lib = None


def lib():
    """The loaded library; raises if libgsparc.so is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libgsparc.so is not built (%s); run __graft_entry__.build() or "
                               "python -m paper_2511_22793_gb300.build" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, i64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        f32 = ctypes.c_float
        P = ctypes.POINTER
        sig = {
            "gsparc_num_tiles": (i32, [P(View)]),
            "gsparc_project": (ctypes.c_int, [P(View), i32, vp, vp, vp, vp, vp, vp]),
            "gsparc_project_bwd": (ctypes.c_int, [P(View), i32, vp, vp, vp, vp, vp, vp, vp, vp]),
            "gsparc_bin_sort_workspace": (ctypes.c_int, [P(View), i32, i64, P(ctypes.c_size_t)]),
            "gsparc_bin_sort": (ctypes.c_int, [P(View), i32, vp, i64, vp, ctypes.c_size_t, vp, vp, vp,
                                               vp, vp, vp]),
            "gsparc_bin_sort_noalloc": (ctypes.c_int, [P(View), i32, vp, i64, vp, vp, vp, vp, vp, vp]),
            "gsparc_attr_mlp": (ctypes.c_int, [i32, i32, vp, P(f32), vp, vp, vp, P(MLP), i32, vp, vp, vp]),
            "gsparc_attr_mlp_bwd": (ctypes.c_int, [i32, i32, vp, P(f32), vp, vp, vp, P(MLP), vp, vp,
                                                   vp, vp, P(MLPGrad), vp, vp]),
            "gsparc_attr_mlp_bwd_tc": (ctypes.c_int, [i32, i32, vp, P(f32), vp, vp, vp, P(MLP), i32, vp,
                                                      vp, vp, vp, P(MLPGrad), vp]),
            "gsparc_emission_stride": (i32, [i32]),
            "gsparc_emission_fwd": (ctypes.c_int, [i32, i32, i32, vp, P(f32), vp, vp, vp, i32, vp, vp]),
            "gsparc_emission_bwd": (ctypes.c_int, [i32, i32, i32, vp, P(f32), vp, vp, vp, i32, vp, vp, vp, vp,
                                                   vp]),
            "gsparc_render_fwd": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp, vp,
                                                 vp, vp, vp, vp]),
            "gsparc_render_fwd_tc": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp, vp,
                                                    vp, vp, vp, vp]),
            "gsparc_render_fwd_l2": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp, vp,
                                                    vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "gsparc_render_bwd_workspace": (ctypes.c_int, [P(View), P(Band), i32, P(ctypes.c_size_t)]),
            "gsparc_render_bwd_balanced": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp,
                                                          vp, vp, vp, vp, vp, i32, vp, ctypes.c_size_t, vp,
                                                          vp, vp, vp]),
            "gsparc_render_bwd": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp, vp,
                                                 vp, vp, vp, vp, vp]),
            "gsparc_render_bwd_tc": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp, vp,
                                                    vp, vp, vp, vp, vp]),
            "gsparc_l2_loss": (ctypes.c_int, [i64, vp, vp, vp, vp, vp]),
            "gsparc_csi_head": (ctypes.c_int, [i32, i32, i64, vp, f32, vp, vp]),
            "gsparc_csi_loss": (ctypes.c_int, [i32, i32, vp, vp, vp, vp, vp]),
            "gsparc_csi_head_bwd": (ctypes.c_int, [i32, i32, i64, vp, f32, vp, vp]),
            "gsparc_spectrum_loss_workspace": (ctypes.c_int, [i32, i32, i32, i32, P(ctypes.c_size_t)]),
            "gsparc_spectrum_loss": (ctypes.c_int, [i32, i32, i32, i32, vp, vp, f32, vp, ctypes.c_size_t, vp, vp,
                                                    vp]),
            "gsparc_render_csi_tc": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp, vp,
                                                    vp, vp, vp, vp, vp]),
            "gsparc_render_fwd_l2_tc": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp, vp,
                                                       vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "gsparc_render_bwd_tc_workspace": (ctypes.c_int, [P(View), P(Band), i32, P(ctypes.c_size_t)]),
            "gsparc_render_bwd_tc_balanced": (ctypes.c_int, [P(View), P(Band), i32, i32, vp, vp, vp, vp, vp,
                                                             vp, vp, vp, vp, vp, i32, vp, ctypes.c_size_t, vp,
                                                             vp, vp, vp]),
            "gsparc_confidence": (ctypes.c_int, [i32, i32, vp, vp, vp, f32, vp, vp, vp, vp, vp]),
            "gsparc_densify_accumulate": (ctypes.c_int, [i32, vp, vp, vp, vp, vp]),
            "gsparc_densify_workspace": (ctypes.c_int, [i32, P(ctypes.c_size_t)]),
            "gsparc_densify": (ctypes.c_int, [i32, i32, vp, vp, vp, vp, vp, vp, vp, vp, vp, P(DensifyParams), i32,
                                              vp, ctypes.c_size_t, vp, vp, vp, vp, vp, vp, vp, vp, vp]),
            "gsparc_opacity_reset": (ctypes.c_int, [i32, f32, vp, vp]),
            "gsparc_adam": (ctypes.c_int, [i64, vp, vp, vp, vp, f32, f32, f32, f32, i32, vp]),
            "gsparc_adam_segments": (ctypes.c_int, [i64, vp, vp, vp, vp, i32, P(i64), P(f32), f32, f32, f32, i32,
                                                    vp]),
            "gsparc_scale_rows": (ctypes.c_int, [i32, i64, vp, vp, vp]),
            "gsparc_set_wait_limit": (ctypes.c_uint32, [ctypes.c_uint32]),
            "gsparc_set_launch_overlap": (ctypes.c_int32, [ctypes.c_int32]),
            "gsparc_check": (ctypes.c_int, [vp, vp]),
            "gsparc_strerror": (ctypes.c_char_p, [ctypes.c_int]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def strerror(code: int) -> str:
    try:
        return lib().gsparc_strerror(int(code)).decode()
    except Exception:
        return "status %d" % code


def _call(name, *args):
    rc = getattr(lib(), name)(*args)
    if rc != GSPARC_OK:
        raise GsparcError(name, rc)


def _p(t):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


def make_view(H, W, rx=(0.0, 0.0, 0.0), V=(1, 0, 0, 0, 1, 0, 0, 0, 1), near_dist=0.1) -> View:
    v = View()
    v.H, v.W = int(H), int(W)
    for i in range(3):
        v.rx[i] = float(rx[i])
    for i in range(9):
        v.V[i] = float(V[i])
    v.near_dist = float(near_dist)
    return v


def make_band(K, f_c=2.4e9, df=312.5e3) -> Band:
    b = Band()
    b.K, b.reserved, b.f_c, b.df = int(K), 0, float(f_c), float(df)
    return b


def make_mlp(hidden, W1, b1, W2, b2, W3, b3) -> MLP:
    m = MLP()
    m.hidden, m.reserved = int(hidden), 0
    for n, t in zip(("W1", "b1", "W2", "b2", "W3", "b3"), (W1, b1, W2, b2, W3, b3)):
        setattr(m, n, _p(t).value)
    return m


def make_mlp_grad(W1, b1, W2, b2, W3, b3) -> MLPGrad:
    g = MLPGrad()
    for n, t in zip(("W1", "b1", "W2", "b2", "W3", "b3"), (W1, b1, W2, b2, W3, b3)):
        setattr(g, n, _p(t).value)
    return g


def gsparc_num_tiles(view: View) -> int:
    return int(lib().gsparc_num_tiles(ctypes.byref(view)))


def gsparc_project(view, means, log_scales, quats, proj, stream=None, d_status=None):
    _call("gsparc_project", ctypes.byref(view), means.shape[0], _p(means), _p(log_scales), _p(quats),
          _p(proj), _p(d_status), _stream(stream))


def gsparc_project_bwd(view, means, log_scales, quats, d_proj, d_means, d_log_scales, d_quats,
                       stream=None):
    _call("gsparc_project_bwd", ctypes.byref(view), means.shape[0], _p(means), _p(log_scales),
          _p(quats), _p(d_proj), _p(d_means), _p(d_log_scales), _p(d_quats), _stream(stream))


def gsparc_bin_sort_workspace(view, n, pair_capacity) -> int:
    out = ctypes.c_size_t(0)
    _call("gsparc_bin_sort_workspace", ctypes.byref(view), int(n), int(pair_capacity),
          ctypes.byref(out))
    return int(out.value)


def gsparc_bin_sort(view, n, proj, pair_capacity, ws, sorted_ids, sorted_keys, tile_ranges, n_pairs,
                    d_status, stream=None):
    _call("gsparc_bin_sort", ctypes.byref(view), int(n), _p(proj), int(pair_capacity), _p(ws),
          ws.numel() * ws.element_size(), _p(sorted_ids), _p(sorted_keys), _p(tile_ranges),
          _p(n_pairs), _p(d_status), _stream(stream))


def gsparc_bin_sort_noalloc(view, n, proj, pair_capacity, sorted_ids, sorted_keys, tile_ranges,
                            n_pairs, d_status, stream=None):
    """gsparc_bin_sort with its scratch in the library's fixed device array (no workspace)."""
    _call("gsparc_bin_sort_noalloc", ctypes.byref(view), int(n), _p(proj), int(pair_capacity),
          _p(sorted_ids), _p(sorted_keys), _p(tile_ranges), _p(n_pairs), _p(d_status),
          _stream(stream))


def hidden_ld(rows: int) -> int:
    """Leading dimension of the network's stored activations (gsparc_attr_mlp's `hidden`)."""
    return (int(rows) + 3) // 4 * 4


def gsparc_attr_mlp(tx, rx, means, opacity_logit, latent, mlp: MLP, precision, attr, stream=None, hidden=None):
    """hidden (FP32 only): [2 * mlp.hidden * hidden_ld(B * N)] floats that receive the activations
    gsparc_attr_mlp_bwd can take instead of recomputing them."""
    rxa = (ctypes.c_float * 3)(*[float(v) for v in rx])
    _call("gsparc_attr_mlp", means.shape[0], tx.shape[0], _p(tx), rxa, _p(means), _p(opacity_logit),
          _p(latent), ctypes.byref(mlp), int(precision), _p(attr), _p(hidden), _stream(stream))


def gsparc_attr_mlp_bwd(tx, rx, means, opacity_logit, latent, mlp: MLP, d_attr, d_means,
                        d_opacity_logit, d_latent, grads: MLPGrad, stream=None, hidden=None):
    rxa = (ctypes.c_float * 3)(*[float(v) for v in rx])
    _call("gsparc_attr_mlp_bwd", means.shape[0], tx.shape[0], _p(tx), rxa, _p(means),
          _p(opacity_logit), _p(latent), ctypes.byref(mlp), _p(d_attr), _p(d_means),
          _p(d_opacity_logit), _p(d_latent), ctypes.byref(grads), _p(hidden), _stream(stream))


def gsparc_attr_mlp_bwd_tc(tx, rx, means, opacity_logit, latent, mlp: MLP, precision, d_attr, d_means,
                           d_opacity_logit, d_latent, grads: MLPGrad, stream=None):
    rxa = (ctypes.c_float * 3)(*[float(v) for v in rx])
    _call("gsparc_attr_mlp_bwd_tc", means.shape[0], tx.shape[0], _p(tx), rxa, _p(means),
          _p(opacity_logit), _p(latent), ctypes.byref(mlp), int(precision), _p(d_attr), _p(d_means),
          _p(d_opacity_logit), _p(d_latent), ctypes.byref(grads), _stream(stream))


def gsparc_render_fwd(view, band, B, n, proj, tile_ranges, sorted_ids, attr, spectrum,
                      final_logT=None, n_contrib=None, n_used=None, stream=None, d_status=None):
    _call("gsparc_render_fwd", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(spectrum), _p(final_logT), _p(n_contrib),
          _p(n_used), _p(d_status), _stream(stream))


def gsparc_render_fwd_tc(view, band, B, n, proj, tile_ranges, sorted_ids, attr, spectrum,
                         final_logT=None, n_contrib=None, n_used=None, stream=None, d_status=None):
    _call("gsparc_render_fwd_tc", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(spectrum), _p(final_logT), _p(n_contrib),
          _p(n_used), _p(d_status), _stream(stream))


def gsparc_render_bwd(view, band, B, n, proj, tile_ranges, sorted_ids, attr, final_logT, n_contrib,
                      d_spectrum, d_attr, d_proj, stream=None, d_status=None):
    _call("gsparc_render_bwd", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(final_logT), _p(n_contrib), _p(d_spectrum),
          _p(d_attr), _p(d_proj), _p(d_status), _stream(stream))


def gsparc_render_bwd_tc(view, band, B, n, proj, tile_ranges, sorted_ids, attr, final_logT, n_contrib,
                         d_spectrum, d_attr, d_proj, stream=None, d_status=None):
    _call("gsparc_render_bwd_tc", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(final_logT), _p(n_contrib), _p(d_spectrum),
          _p(d_attr), _p(d_proj), _p(d_status), _stream(stream))


def gsparc_emission_stride(hidden) -> int:
    """Floats per Gaussian in the emission buffer (6 hidden + 2, rounded up to a multiple of 4)."""
    v = int(lib().gsparc_emission_stride(int(hidden)))
    if v <= 0:
        raise GsparcError("gsparc_emission_stride", -1)
    return v


def gsparc_emission_fwd(tx, rx, means, opacity_logit, weights, hidden, attr, inv_d=True, stream=None):
    """tx [B,3] device, rx 3 host floats, weights [N, stride] -> attr [B,N,4]."""
    n, B = int(means.shape[0]), int(tx.shape[0])
    rxa = (ctypes.c_float * 3)(*[float(v) for v in rx])
    _call("gsparc_emission_fwd", n, B, int(hidden), _p(tx), rxa, _p(means), _p(opacity_logit), _p(weights),
          1 if inv_d else 0, _p(attr), _stream(stream))


def gsparc_emission_bwd(tx, rx, means, opacity_logit, weights, hidden, d_attr, d_means, d_opacity_logit,
                        d_weights, inv_d=True, stream=None):
    """Adds the gradients of gsparc_emission_fwd for d_attr [B,N,4] into d_means, d_opacity_logit and
    d_weights."""
    n, B = int(means.shape[0]), int(tx.shape[0])
    rxa = (ctypes.c_float * 3)(*[float(v) for v in rx])
    _call("gsparc_emission_bwd", n, B, int(hidden), _p(tx), rxa, _p(means), _p(opacity_logit), _p(weights),
          1 if inv_d else 0, _p(d_attr), _p(d_means), _p(d_opacity_logit), _p(d_weights), _stream(stream))


def gsparc_render_fwd_l2(view, band, B, n, proj, tile_ranges, sorted_ids, attr, target, loss, d_spectrum,
                         spectrum=None, final_logT=None, n_contrib=None, n_used=None, s_tot=None, tile_walk=None,
                         stream=None, d_status=None):
    """FP32 forward with the complex L2 loss fused (dL/dz, loss, optional s_tot and tile walks)."""
    _call("gsparc_render_fwd_l2", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(target), _p(loss), _p(d_spectrum), _p(spectrum),
          _p(final_logT), _p(n_contrib), _p(n_used), _p(s_tot), _p(tile_walk), _p(d_status), _stream(stream))


def gsparc_render_bwd_workspace(view, band, B) -> int:
    out = ctypes.c_size_t(0)
    _call("gsparc_render_bwd_workspace", ctypes.byref(view), ctypes.byref(band), int(B), ctypes.byref(out))
    return int(out.value)


def fp32_strips(K) -> int:
    """Strips of the FP32 kernels' s_tot buffer [B, strips, H, W] for K subcarriers."""
    return 1 if K <= 32 else (K + 31) // 32


def gsparc_render_bwd_balanced(view, band, B, n, proj, tile_ranges, sorted_ids, attr, spectrum, s_tot,
                               final_logT, n_contrib, d_spectrum, ws, d_attr, d_proj, split_min=0,
                               tile_walk=None, stream=None, d_status=None):
    """FP32 backward scheduled over the SMs.  ws: a uint8 device tensor of
    gsparc_render_bwd_workspace() bytes, zeroed once (torch.zeros) before its first use."""
    _call("gsparc_render_bwd_balanced", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(spectrum), _p(s_tot), _p(tile_walk), _p(final_logT),
          _p(n_contrib), _p(d_spectrum), int(split_min), _p(ws), ws.numel() * ws.element_size(), _p(d_attr),
          _p(d_proj), _p(d_status), _stream(stream))


def gsparc_render_bwd_tc_workspace(view, band, B) -> int:
    out = ctypes.c_size_t(0)
    _call("gsparc_render_bwd_tc_workspace", ctypes.byref(view), ctypes.byref(band), int(B), ctypes.byref(out))
    return int(out.value)


def s_tot_strips(K) -> int:
    """Strips of the s_tot buffer [B, strips, H, W] for K subcarriers."""
    return 1 if K <= 64 else (K + 63) // 64


def gsparc_render_bwd_tc_balanced(view, band, B, n, proj, tile_ranges, sorted_ids, attr, spectrum, s_tot,
                                  final_logT, n_contrib, d_spectrum, ws, d_attr, d_proj, split_min=0,
                                  tile_walk=None, stream=None, d_status=None):
    """ws: a uint8 device tensor of gsparc_render_bwd_tc_workspace() bytes, zeroed once
    (torch.zeros) before its first use."""
    _call("gsparc_render_bwd_tc_balanced", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(spectrum), _p(s_tot), _p(tile_walk), _p(final_logT),
          _p(n_contrib), _p(d_spectrum), int(split_min), _p(ws), ws.numel() * ws.element_size(), _p(d_attr),
          _p(d_proj), _p(d_status), _stream(stream))


def gsparc_l2_loss(z, target, loss, d_z=None, stream=None):
    count = z.numel() // 2
    _call("gsparc_l2_loss", count, _p(z), _p(target), _p(loss), _p(d_z), _stream(stream))


def gsparc_spectrum_loss_workspace(B, K, H, W) -> int:
    out = ctypes.c_size_t(0)
    _call("gsparc_spectrum_loss_workspace", int(B), int(K), int(H), int(W), ctypes.byref(out))
    return int(out.value)


def gsparc_spectrum_loss(spectrum, target, ws, loss, d_spectrum=None, lam=0.2, stream=None):
    """spectrum [B,K,H,W,2], target [B,K,H,W] magnitudes -> loss [1] (Eq. 4, L1 + SSIM) and dL/dz."""
    B, K, H, W = (int(v) for v in target.shape)
    _call("gsparc_spectrum_loss", B, K, H, W, _p(spectrum), _p(target), float(lam), _p(ws),
          ws.numel() * ws.element_size(), _p(loss), _p(d_spectrum), _stream(stream))


def gsparc_confidence(pos, task_loss, weights, hidden, objective, confidence=None, d_task_loss=None,
                      d_weights=None, alpha=0.3, stream=None):
    """Eq. 5: pos [B,3], task_loss [B], weights [5 hidden + 1] -> objective [1] = mean (C L - alpha
    ln C), C = 1 + exp(g(pos)) [B], dObj/dL [B] (written) and the weight gradients (accumulated)."""
    B = int(task_loss.shape[0])
    _call("gsparc_confidence", B, int(hidden), _p(pos), _p(task_loss), _p(weights), float(alpha),
          _p(confidence), _p(objective), _p(d_task_loss), _p(d_weights), _stream(stream))


def densify_params(tau_grad=2e-4, clone_scale=0.01 * 5.0 * 3.0 ** 0.5, sigma_min=0.005, r_max=20.0,
                   n_split=2) -> DensifyParams:
    p = DensifyParams()
    p.tau_grad, p.clone_scale, p.sigma_min, p.r_max = float(tau_grad), float(clone_scale), float(sigma_min), \
        float(r_max)
    p.n_split = int(n_split)
    return p


def gsparc_densify_accumulate(proj, d_means, norm_sum, count, stream=None):
    """Adds ||dL/dmu|| and 1 for every Gaussian whose projection record [N,8] was not culled."""
    _call("gsparc_densify_accumulate", int(norm_sum.shape[0]), _p(proj), _p(d_means), _p(norm_sum), _p(count),
          _stream(stream))


def gsparc_densify_workspace(N) -> int:
    out = ctypes.c_size_t(0)
    _call("gsparc_densify_workspace", int(N), ctypes.byref(out))
    return int(out.value)


def gsparc_densify(means, log_scales, quats, opacity_logit, payload, proj, norm_sum, count, xi, params, ws,
                   out, n_out, d_status=None, stream=None):
    """Algorithm 1's clone / split / prune over N Gaussians.  payload [N,P] or None; out: dict of
    preallocated outputs (means, log_scales, quats, opacity_logit, payload, parent), capacity rows
    each; n_out [1] int32/uint32 device count of the rows produced."""
    N = int(means.shape[0])
    P = 0 if payload is None else int(payload.shape[1])
    cap = int(out["parent"].shape[0])
    _call("gsparc_densify", N, P, _p(means), _p(log_scales), _p(quats), _p(opacity_logit), _p(payload), _p(proj),
          _p(norm_sum), _p(count), _p(xi), ctypes.byref(params), cap, _p(ws), ws.numel() * ws.element_size(),
          _p(out["means"]), _p(out["log_scales"]), _p(out["quats"]), _p(out["opacity_logit"]),
          _p(out.get("payload")), _p(out["parent"]), _p(n_out), _p(d_status), _stream(stream))


def gsparc_opacity_reset(opacity_logit, max_opacity=0.01, stream=None):
    _call("gsparc_opacity_reset", int(opacity_logit.numel()), float(max_opacity), _p(opacity_logit),
          _stream(stream))


def gsparc_csi_head(spectrum, csi, scale, stream=None):
    """spectrum [B, K, H, W, 2] -> csi [B, K, 2] = scale * sum over pixels (Eq. 2 with 1/HW)."""
    B, K = spectrum.shape[0], spectrum.shape[1]
    P = spectrum.numel() // (2 * B * K)
    _call("gsparc_csi_head", int(B), int(K), int(P), _p(spectrum), float(scale), _p(csi), _stream(stream))


def gsparc_csi_loss(csi, target, loss, d_csi=None, stream=None):
    B, K = csi.shape[0], csi.shape[1]
    _call("gsparc_csi_loss", int(B), int(K), _p(csi), _p(target), _p(loss), _p(d_csi), _stream(stream))


def gsparc_csi_head_bwd(d_csi, d_spectrum, scale, stream=None):
    B, K = d_csi.shape[0], d_csi.shape[1]
    P = d_spectrum.numel() // (2 * B * K)
    _call("gsparc_csi_head_bwd", int(B), int(K), int(P), _p(d_csi), float(scale), _p(d_spectrum),
          _stream(stream))


def gsparc_render_csi_tc(view, band, B, n, proj, tile_ranges, sorted_ids, attr, csi, spectrum=None,
                         final_logT=None, n_contrib=None, n_used=None, stream=None, d_status=None):
    _call("gsparc_render_csi_tc", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(csi), _p(spectrum), _p(final_logT), _p(n_contrib),
          _p(n_used), _p(d_status), _stream(stream))


def gsparc_render_fwd_l2_tc(view, band, B, n, proj, tile_ranges, sorted_ids, attr, target, loss, d_spectrum,
                            spectrum=None, final_logT=None, n_contrib=None, n_used=None, s_tot=None,
                            tile_walk=None, stream=None, d_status=None):
    _call("gsparc_render_fwd_l2_tc", ctypes.byref(view), ctypes.byref(band), int(B), int(n), _p(proj),
          _p(tile_ranges), _p(sorted_ids), _p(attr), _p(target), _p(loss), _p(d_spectrum), _p(spectrum),
          _p(final_logT), _p(n_contrib), _p(n_used), _p(s_tot), _p(tile_walk), _p(d_status), _stream(stream))


def gsparc_adam(param, grad, m, v, lr, step, b1=0.9, b2=0.999, eps=1e-15, stream=None):
    _call("gsparc_adam", param.numel(), _p(param), _p(grad), _p(m), _p(v), float(lr), float(b1),
          float(b2), float(eps), int(step), _stream(stream))


def gsparc_adam_segments(param, grad, m, v, seg_end, seg_lr, step, b1=0.9, b2=0.999, eps=1e-15, stream=None):
    """One Adam launch over a flat buffer whose groups end at seg_end (host ints, the last = numel)
    with learning rates seg_lr (host floats)."""
    k = len(seg_end)
    ends = (ctypes.c_int64 * k)(*[int(e) for e in seg_end])
    lrs = (ctypes.c_float * k)(*[float(x) for x in seg_lr])
    _call("gsparc_adam_segments", param.numel(), _p(param), _p(grad), _p(m), _p(v), k, ends, lrs, float(b1),
          float(b2), float(eps), int(step), _stream(stream))


def gsparc_scale_rows(x, w, stream=None):
    """x [rows, ...] scaled in place row by row by w [rows] (device)."""
    rows = int(x.shape[0])
    _call("gsparc_scale_rows", rows, x.numel() // max(rows, 1), _p(w), _p(x), _stream(stream))


def gsparc_set_wait_limit(polls: int) -> int:
    """Polls before a pipeline wait of the tensor-core compositing kernels gives up (0: the
    default); returns the previous setting.  For tests of the timeout path."""
    return int(lib().gsparc_set_wait_limit(int(polls)))


def gsparc_set_launch_overlap(groups) -> int:
    """Programmatic dependent launch of the library's follow-on kernels: True / False for every
    group or none, or a mask of GSPARC_OVERLAP_* groups (every group by default); returns the
    previous mask."""
    if isinstance(groups, bool):
        groups = GSPARC_OVERLAP_ALL if groups else 0
    return int(lib().gsparc_set_launch_overlap(int(groups)))


def gsparc_check(d_status=None, stream=None) -> int:
    return int(lib().gsparc_check(_p(d_status), _stream(stream)))
