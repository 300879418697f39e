"""ctypes wrapper of the FP64 per-pixel renderer in render_oracle.c.

TEST INFRASTRUCTURE (see the package docstring).  build() compiles the C file
with the host compiler; tests and the benchmark's CPU baseline load it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "render_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

C_LIGHT = 299792458.0


def build(force: bool = False) -> str:
    """Compile liboracle.so next to its source (OpenMP over pixels)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            bp = ctypes.POINTER(ctypes.c_ubyte)
            common = [ctypes.c_int] + [dp] * 6 + [bp] + [dp] * 4 + [ctypes.c_int] * 3 + \
                     [ctypes.c_double] * 2 + [ctypes.c_int] * 2 + [ip]
            lib.oracle_render_fwd.argtypes = common + [dp, dp, ip, ctypes.POINTER(ctypes.c_ulonglong),
                                                       ctypes.c_int]
            lib.oracle_render_fwd.restype = ctypes.c_int
            lib.oracle_render_bwd.argtypes = common + [dp, dp, ctypes.c_int]
            lib.oracle_render_bwd.restype = ctypes.c_int
            _lib = lib
    return _lib


def _d(a):
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _ptr(a, t):
    return a.ctypes.data_as(ctypes.POINTER(t))


def _geom_args(geo, attr):
    arrs = [_d(geo[k]) for k in ("px", "py", "cxx", "cxy", "cyy", "r")]
    valid = np.ascontiguousarray(np.asarray(geo["valid"], dtype=np.uint8))
    att = [_d(attr[k]) for k in ("sigma", "a", "phi0", "L")]
    return arrs, valid, att


def first_frequency(K: int, f_c: float, df: float) -> float:
    """f_k = f_c + (k - floor(K/2)) df, so K = 1 renders the carrier itself."""
    return f_c - (K // 2) * df


def render_fwd(geo, attr, H, W, K, f_c, df, pixels=None, exact=False, threads=0, signature=False):
    """Render the given pixels (linear ids y*W + x; all when None).

    geo: dict with px, py, cxx, cxy, cyy, r, valid (numpy or torch, any float).
    attr: dict with sigma, a, phi0, L.
    Returns (z [npix, K] complex128, T_final [npix], n_used [npix]); with
    signature=True also the per-pixel composited-set signature.
    """
    lib = _load()
    arrs, valid, att = _geom_args(geo, attr)
    N = arrs[0].shape[0]
    pix = np.arange(H * W, dtype=np.int32) if pixels is None else \
        np.ascontiguousarray(np.asarray(pixels, dtype=np.int32))
    npix = pix.shape[0]
    z = np.zeros((npix, K, 2), dtype=np.float64)
    tf = np.zeros(npix, dtype=np.float64)
    nu = np.zeros(npix, dtype=np.int32)
    sg = np.zeros(npix, dtype=np.uint64)
    dp = ctypes.c_double
    rc = lib.oracle_render_fwd(
        N, *[_ptr(a, dp) for a in arrs], _ptr(valid, ctypes.c_ubyte), *[_ptr(a, dp) for a in att],
        H, W, K, first_frequency(K, f_c, df), df, int(bool(exact)), npix, _ptr(pix, ctypes.c_int),
        _ptr(z, dp), _ptr(tf, dp), _ptr(nu, ctypes.c_int), _ptr(sg, ctypes.c_ulonglong),
        int(threads))
    if rc != 0:
        raise RuntimeError("oracle_render_fwd failed: %d" % rc)
    zc = z[..., 0] + 1j * z[..., 1]
    if signature:
        return zc, tf, nu, sg
    return zc, tf, nu


def render_bwd(geo, attr, H, W, K, f_c, df, gz, pixels=None, exact=False, threads=0):
    """Gradient of a real loss given gz = dL/dRe z + j dL/dIm z, [npix, K] complex.

    Returns grad [N, 9] float64 with columns
    (p_x, p_y, c_xx, c_xy, c_yy, sigma, a, phi0, L).
    """
    lib = _load()
    arrs, valid, att = _geom_args(geo, attr)
    N = arrs[0].shape[0]
    pix = np.arange(H * W, dtype=np.int32) if pixels is None else \
        np.ascontiguousarray(np.asarray(pixels, dtype=np.int32))
    npix = pix.shape[0]
    gz = np.asarray(gz)
    g = np.ascontiguousarray(np.stack([gz.real, gz.imag], -1).astype(np.float64).reshape(npix, K, 2))
    grad = np.zeros((N, 9), dtype=np.float64)
    dp = ctypes.c_double
    rc = lib.oracle_render_bwd(
        N, *[_ptr(a, dp) for a in arrs], _ptr(valid, ctypes.c_ubyte), *[_ptr(a, dp) for a in att],
        H, W, K, first_frequency(K, f_c, df), df, int(bool(exact)), npix, _ptr(pix, ctypes.c_int),
        _ptr(g, dp), _ptr(grad, dp), int(threads))
    if rc != 0:
        raise RuntimeError("oracle_render_bwd failed: %d" % rc)
    return grad
