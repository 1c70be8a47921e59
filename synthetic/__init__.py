"""Seeded synthetic inputs shared by the FP64 oracle and the CUDA path.

This module holds no arithmetic of the tokenizer itself: it only draws the
random pixels, weights, drop rates and arrival times that both sides consume.
Neither side's arithmetic lives here, and nothing here imports either side.

Workload shapes follow the paper's evaluation setup (1080p test videos at
30/60 fps, Sec. 8.1, and their 2x/3x downscales, Sec. 5 and Appendix A.2).
The datasets themselves (UVG, UHD, UGC, Inter4K) are not available, so these
generators stand in for them with seeded noise of the same shape.
"""
from __future__ import annotations

import zlib

import numpy as np
from scipy.ndimage import gaussian_filter1d

__all__ = [
    "blurred_noise_clip",
    "moving_rects_clip",
    "he_normal",
    "weights_for",
    "drop_rates",
    "poisson_arrivals",
    "to_bf16_f32",
]


def _gauss_blur_hw(a: np.ndarray, sigma: float, radius: int) -> np.ndarray:
    """Separable Gaussian blur over the two spatial axes (-3, -2) of a
    (..., H, W, C) array, zero-extended at the borders ('constant')."""
    truncate = radius / sigma
    a = gaussian_filter1d(a, sigma, axis=-3, mode="constant", truncate=truncate)
    a = gaussian_filter1d(a, sigma, axis=-2, mode="constant", truncate=truncate)
    return a


def blurred_noise_clip(seed: int, N: int, T: int, H: int, W: int, C: int = 3) -> np.ndarray:
    """Gaussian-blurred uniform noise in [-1, 1], shape (N, T, H, W, C) float32.

    Recipe: U[-1, 1] i.i.d. per sample, a separable spatial Gaussian with
    sigma = 1.5 px (radius 4) applied to every frame, then each clip is
    rescaled by 1 / max|.| so that its values span [-1, 1].
    """
    rng = np.random.default_rng(seed)
    u = rng.uniform(-1.0, 1.0, size=(N, T, H, W, C))
    b = _gauss_blur_hw(u, 1.5, 4)
    m = np.abs(b).reshape(N, -1).max(axis=1)
    b = b / m[:, None, None, None, None]
    return b.astype(np.float32)


def moving_rects_clip(seed: int, T: int, H: int, W: int, C: int = 3,
                      n_rects: int = 4, noise_sigma: float = 0.05) -> np.ndarray:
    """Structured content for the variable-resolution and streaming workloads.

    Smooth noise (U[-1, 1] blurred with sigma = 8 px per frame, rescaled to
    [-1, 1]), plus ``n_rects`` moving rectangles (sides 10-30% of H/W, colour
    U[-1, 1], velocity 2-8 px/frame, bouncing off the borders), plus
    per-pixel N(0, noise_sigma^2), clamped to [-1, 1]. Shape (T, H, W, C)
    float32. The background is static over time; the rectangles move.
    """
    rng = np.random.default_rng(seed)
    bg = rng.uniform(-1.0, 1.0, size=(H, W, C))
    bg = _gauss_blur_hw(bg, 8.0, 24)
    bg = bg / max(np.abs(bg).max(), 1e-12)
    rects = []
    for _ in range(n_rects):
        rh = int(rng.uniform(0.1, 0.3) * H) + 1
        rw = int(rng.uniform(0.1, 0.3) * W) + 1
        y = rng.uniform(0, H - rh)
        x = rng.uniform(0, W - rw)
        speed = rng.uniform(2.0, 8.0)
        ang = rng.uniform(0, 2 * np.pi)
        vy, vx = speed * np.sin(ang), speed * np.cos(ang)
        col = rng.uniform(-1.0, 1.0, size=C)
        rects.append([y, x, vy, vx, rh, rw, col])
    out = np.empty((T, H, W, C), dtype=np.float64)
    for t in range(T):
        f = bg.copy()
        for r in rects:
            y, x, vy, vx, rh, rw, col = r
            iy, ix = int(round(y)), int(round(x))
            f[iy:iy + rh, ix:ix + rw, :] = col
            y, x = y + vy, x + vx
            if y < 0 or y > H - rh:
                vy = -vy
                y = min(max(y, 0.0), H - rh)
            if x < 0 or x > W - rw:
                vx = -vx
                x = min(max(x, 0.0), W - rw)
            r[0], r[1], r[2], r[3] = y, x, vy, vx
        out[t] = f
    out += rng.normal(0.0, noise_sigma, size=out.shape)
    return np.clip(out, -1.0, 1.0).astype(np.float32)


def he_normal(name: str, shape, fan_in: int, seed: int = 0, gain: float = 1.0) -> np.ndarray:
    """He-normal N(0, gain^2 * 2 / fan_in) weights, float32, drawn from a
    stream keyed by (seed, crc32(name)) so that every named tensor is the same
    whatever order the two sides ask for them in."""
    rng = np.random.default_rng([seed, zlib.crc32(name.encode())])
    std = gain * np.sqrt(2.0 / fan_in)
    return (rng.standard_normal(size=tuple(shape)) * std).astype(np.float32)


def weights_for(spec, seed: int = 0, out_gain: float = 1.0) -> dict:
    """Draw every parameter of a parameter list.

    ``spec`` is an iterable of (name, shape, kind) with kind one of
    'conv' (He-normal, fan_in = prod(shape[1:])), 'bias' (zeros),
    'gn_gamma' (ones), 'gn_beta' (zeros). Tensors whose name is listed with
    kind 'conv_out' use He-normal scaled by ``out_gain``.
    """
    out = {}
    for name, shape, kind in spec:
        shape = tuple(int(s) for s in shape)
        if kind in ("conv", "conv_out"):
            fan_in = int(np.prod(shape[1:]))
            g = out_gain if kind == "conv_out" else 1.0
            out[name] = he_normal(name, shape, fan_in, seed, g)
        elif kind in ("bias", "gn_beta"):
            out[name] = np.zeros(shape, dtype=np.float32)
        elif kind == "gn_gamma":
            out[name] = np.ones(shape, dtype=np.float32)
        else:
            raise ValueError(f"unknown parameter kind {kind!r} for {name}")
    return out


def drop_rates(seed: int, n: int, lo: float = 0.0, hi: float = 0.30) -> np.ndarray:
    """Per-chunk token drop rates ~ U[lo, hi] (float32)."""
    rng = np.random.default_rng(seed)
    return rng.uniform(lo, hi, size=n).astype(np.float32)


def poisson_arrivals(seed: int, n_streams: int, horizon_s: float, start_rate_hz: float = 4.0):
    """Stream start times: a Poisson process of rate ``start_rate_hz`` over
    [0, horizon_s); returns a sorted float64 array of length n_streams
    (clipped to the horizon)."""
    rng = np.random.default_rng(seed)
    gaps = rng.exponential(1.0 / start_rate_hz, size=n_streams)
    t = np.cumsum(gaps) - gaps[0]
    return np.minimum(t, horizon_s)


def to_bf16_f32(a: np.ndarray) -> np.ndarray:
    """Round float32 values to the nearest bfloat16 (ties to even) and return
    them as float32. Used to hand the oracle exactly the values a bf16 tensor
    holds; plain bit manipulation, no tokenizer arithmetic."""
    a = np.ascontiguousarray(a, dtype=np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    nan = np.isnan(a)
    rounding = ((u >> 16) & 1) + 0x7FFF
    r = ((u + rounding) >> 16) << 16
    r = (r & 0xFFFFFFFF).astype(np.uint32).view(np.float32)
    r = np.where(nan, a, r)
    return r
