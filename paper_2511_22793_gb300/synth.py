"""Seeded synthetic inputs for the equirectangular splatting path.

This module only draws random numbers and packs them into arrays.  It holds
none of the method's arithmetic (no projection, no attribute network, no
compositing), so both the CUDA path and the FP64 oracle can consume what it
produces without sharing any code with each other.

Distributions follow the scene recipe used for every workload: Gaussian means
uniform in a 10 m cube centred on the receiver, restricted to the upper
hemisphere (y >= 0); log-scales N(-1.5, 0.5) in metres; unit quaternions from
normalised N(0, 1)^4 in (w, x, y, z) order; opacity logits N(0, 1); 16-dim
per-Gaussian latents N(0, 1); transmitter positions uniform in the full cube.
The paper's datasets (Sec. 5) are not available, so these scenes stand in for
them.

Seeds: scene 0, target scene 1, transmitters 2, network 3, request stream 4.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

CUBE_HALF = 5.0          # metres; the cube is [-5, 5]^3 around the receiver
LATENT_DIM = 16
MLP_IN = 3 + LATENT_DIM + 1   # transmitter position, latent, log-distance feature


def _bf16_round(x: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even), kept as float32."""
    x = np.ascontiguousarray(x, dtype=np.float32)
    u = x.view(np.uint32).astype(np.uint64)
    rounding = ((u >> 16) & 1) + 0x7FFF
    u = ((u + rounding) >> 16) << 16
    return u.astype(np.uint32).view(np.float32).copy()


@dataclass
class Scene:
    means: np.ndarray          # [N, 3] float32
    log_scales: np.ndarray     # [N, 3] float32
    quats: np.ndarray          # [N, 4] float32, (w, x, y, z), unit norm
    opacity_logit: np.ndarray  # [N] float32
    latent: np.ndarray         # [N, 16] float32

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logit, self.latent)


@dataclass
class MLPWeights:
    hidden: int
    W1: np.ndarray   # [20, Hd]  (input-major: row j multiplies input feature j)
    b1: np.ndarray   # [Hd]
    W2: np.ndarray   # [Hd, Hd]
    b2: np.ndarray   # [Hd]
    W3: np.ndarray   # [Hd, 3]
    b3: np.ndarray   # [3]

    def arrays(self):
        return (self.W1, self.b1, self.W2, self.b2, self.W3, self.b3)


@dataclass
class View:
    H: int
    W: int
    rx: tuple = (0.0, 0.0, 0.0)
    V: tuple = (1.0, 0.0, 0.0, 0.0, 1.0, 0.0, 0.0, 0.0, 1.0)   # row-major 3x3
    near: float = 0.1


@dataclass
class Band:
    K: int
    f_c: float = 2.4e9
    df: float = 312.5e3


def make_scene(n: int, seed: int = 0, upper_only: bool = True, bf16_latent: bool = False) -> Scene:
    rng = np.random.default_rng(seed)
    means = rng.uniform(-CUBE_HALF, CUBE_HALF, size=(n, 3))
    if upper_only:
        means[:, 1] = rng.uniform(0.0, CUBE_HALF, size=n)
    log_scales = rng.normal(-1.5, 0.5, size=(n, 3))
    q = rng.normal(0.0, 1.0, size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    ologit = rng.normal(0.0, 1.0, size=n)
    latent = rng.normal(0.0, 1.0, size=(n, LATENT_DIM))
    latent = latent.astype(np.float32)
    if bf16_latent:
        latent = _bf16_round(latent)
    return Scene(
        means=means.astype(np.float32),
        log_scales=log_scales.astype(np.float32),
        quats=q.astype(np.float32),
        opacity_logit=ologit.astype(np.float32),
        latent=latent,
    )


def make_mlp(hidden: int = 32, seed: int = 3, bf16_weights: bool = False) -> MLPWeights:
    """Weights N(0,1)/sqrt(fan_in), biases N(0, 0.1^2).

    The paper initialises the network from a standard normal (Sec. 4.1,
    initialisation paragraph); with 20 inputs that saturates every unit, so
    the synthetic scenes scale by 1/sqrt(fan_in).  Both sides read the same
    weights, so this choice does not affect parity.
    """
    rng = np.random.default_rng(seed)

    def w(fi, fo):
        x = (rng.normal(0.0, 1.0, size=(fi, fo)) / np.sqrt(fi)).astype(np.float32)
        return _bf16_round(x) if bf16_weights else x

    def b(fo):
        return (0.1 * rng.normal(0.0, 1.0, size=fo)).astype(np.float32)

    W1, b1 = w(MLP_IN, hidden), b(hidden)
    W2, b2 = w(hidden, hidden), b(hidden)
    W3, b3 = w(hidden, 3), b(3)
    return MLPWeights(hidden, W1, b1, W2, b2, W3, b3)


def make_tx(b: int, seed: int = 2) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.uniform(-CUBE_HALF, CUBE_HALF, size=(b, 3)).astype(np.float32)


def make_proj_records(n: int, H: int, W: int, seed: int = 5, frac_culled: float = 0.05,
                      frac_wide: float = 0.02) -> np.ndarray:
    """Random FP32 projection records [n, 8] for exercising binning on its own.

    Layout per record: (p_x, p_y, ext_x, ext_y, c_xx, c_xy, c_yy, r).  Positions
    cover the whole image plus a margin, extents span sub-pixel to wider than
    half the azimuth range, a fraction is marked culled (extents -1), and a
    fraction repeats the depth of an earlier record so that ties occur.
    """
    rng = np.random.default_rng(seed)
    rec = np.zeros((n, 8), dtype=np.float32)
    rec[:, 0] = rng.uniform(0.0, W, size=n)
    rec[:, 1] = rng.uniform(-4.0, H + 4.0, size=n)
    ext = np.exp(rng.uniform(np.log(0.2), np.log(60.0), size=(n, 2)))
    wide = rng.uniform(size=n) < frac_wide
    ext[wide, 0] = rng.uniform(0.45 * W, 2.0 * W, size=int(wide.sum()))
    rec[:, 2:4] = ext
    rec[:, 4] = 1.0
    rec[:, 6] = 1.0
    rec[:, 7] = rng.uniform(0.1, 9.0, size=n)
    ties = rng.uniform(size=n) < 0.05
    idx = np.nonzero(ties)[0]
    if idx.size:
        src = rng.integers(0, n, size=idx.size)
        rec[idx, 7] = rec[src, 7]
    culled = rng.uniform(size=n) < frac_culled
    rec[culled, 2:4] = -1.0
    return rec


def make_target_grad(shape, seed: int = 6) -> np.ndarray:
    """A random upstream gradient dL/dz (complex, stored as float32 pairs)."""
    rng = np.random.default_rng(seed)
    return rng.normal(0.0, 1.0, size=tuple(shape) + (2,)).astype(np.float32)
