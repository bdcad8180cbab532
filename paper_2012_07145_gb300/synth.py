"""Seeded synthetic input images (host side, numpy).

This module only draws random inputs; it holds none of the pipelines'
arithmetic, so both the CUDA path's tests and the oracle's tests take their
inputs from here.  Images stand in for the Halide-repository test images used by
the paper's evaluation (Sec. 6), which are not available; they have the shapes
and value distributions of the workloads.

Generator: a counter-based splitmix64.  Element n of a stream (row-major over
the whole [C][H][W] array) is mixed from its counter as

    z = (seed << 40) ^ (stream << 56) ^ n        (seed < 2^16, stream < 2^8)
    z = z + 0x9E3779B97F4A7C15
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
    z = (z ^ (z >> 27)) * 0x94D049BB133111EB
    z =  z ^ (z >> 31)

A uniform float in [0, 1) is (z >> 40) * 2^-24, exactly representable in
float32.  Gaussian samples use Box-Muller in float64 on two streams.
"""

import numpy as np

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(counter: np.ndarray) -> np.ndarray:
    """splitmix64 finaliser of a uint64 counter array (wrapping arithmetic)."""
    z = counter.astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15)
    z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
    return z ^ (z >> np.uint64(31))


def raw_u64(n: int, seed: int = 0, stream: int = 0) -> np.ndarray:
    base = (np.uint64(seed & 0xFFFF) << np.uint64(40)) ^ (np.uint64(stream & 0xFF) << np.uint64(56))
    with np.errstate(over="ignore"):
        return splitmix64(np.arange(n, dtype=np.uint64) ^ base)


def uniform_f32(shape, seed: int = 0, stream: int = 0) -> np.ndarray:
    """float32 values (z >> 40) * 2^-24 in [0, 1)."""
    n = int(np.prod(shape))
    z = raw_u64(n, seed, stream)
    return ((z >> np.uint64(40)).astype(np.float64) * (2.0 ** -24)).astype(np.float32).reshape(shape)


def gaussian_f64(shape, seed: int = 0, stream: int = 0) -> np.ndarray:
    """Standard normal samples by Box-Muller from streams (stream, stream+1)."""
    n = int(np.prod(shape))
    u1 = ((raw_u64(n, seed, stream) >> np.uint64(11)).astype(np.float64) + 1.0) * (2.0 ** -53)
    u2 = (raw_u64(n, seed, stream + 1) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return (np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)).reshape(shape)


def stencil_input(h: int, w: int, seed: int = 0) -> np.ndarray:
    """Single-channel float32 [1][H][W], uniform [0,1) (stencil-chain workloads)."""
    return uniform_f32((1, h, w), seed, stream=1)


def rgb_f32(h: int, w: int, seed: int = 0) -> np.ndarray:
    """Planar float32 RGB [3][H][W], uniform [0,1) per channel (Harris, unsharp)."""
    return uniform_f32((3, h, w), seed, stream=2)


def rgb_u16_gradient_noise(h: int, w: int, seed: int = 0, sigma: float = 0.02) -> np.ndarray:
    """Planar uint16 RGB [3][H][W] for the local Laplacian workload.

    R = x/(W-1), G = y/(H-1), B = (R+G)/2, plus N(0, sigma) per channel and pixel,
    clamped to [0,1], scaled by 65535 and rounded to nearest (half to even).
    """
    xs = np.arange(w, dtype=np.float64) / max(w - 1, 1)
    ys = np.arange(h, dtype=np.float64) / max(h - 1, 1)
    r = np.broadcast_to(xs[None, :], (h, w))
    g = np.broadcast_to(ys[:, None], (h, w))
    b = (r + g) / 2.0
    base = np.stack([r, g, b])
    noisy = base + sigma * gaussian_f64((3, h, w), seed, stream=3)
    return np.rint(np.clip(noisy, 0.0, 1.0) * 65535.0).astype(np.uint16)


def gray_u8_lowcontrast(h: int, w: int, seed: int = 0) -> np.ndarray:
    """uint8 [1][H][W]: clamp(rint(N(100, 20)), 0, 255) (histogram-equalize workload)."""
    v = 100.0 + 20.0 * gaussian_f64((1, h, w), seed, stream=5)
    return np.clip(np.rint(v), 0, 255).astype(np.uint8)


def rgba_sparse_f32(h: int, w: int, seed: int = 0, coverage: float = 0.25) -> np.ndarray:
    """Planar float32 RGBA [4][H][W] for the interpolate workload: RGB uniform
    [0,1); alpha 1 on a seeded random fraction `coverage` of the pixels (the
    samples to interpolate between), 0 elsewhere."""
    rgb = uniform_f32((3, h, w), seed, stream=6)
    a = (uniform_f32((1, h, w), seed, stream=7) < coverage).astype(np.float32)
    return np.concatenate([rgb, a])


def gray_f32_gradient_noise(h: int, w: int, seed: int = 0, sigma: float = 0.05) -> np.ndarray:
    """float32 [1][H][W] for the bilateral-grid workload: (x/(W-1) + y/(H-1))/2
    plus N(0, sigma) per pixel, clamped to [0, 1]."""
    xs = np.arange(w, dtype=np.float64) / max(w - 1, 1)
    ys = np.arange(h, dtype=np.float64) / max(h - 1, 1)
    base = (xs[None, :] + ys[:, None]) / 2.0
    noisy = base + sigma * gaussian_f64((1, h, w), seed, stream=9)[0]
    return np.clip(noisy, 0.0, 1.0).astype(np.float32)[None]
