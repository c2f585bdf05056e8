"""Seeded synthetic hyperspectral cubes shaped like the paper's workloads.

The real scenes of the paper (AVIRIS Cuprite, Jasper Ridge, World Trade
Center) and the USGS spectral library are not available here; these
generators stand in for them.  Every cube is built from a numpy
``default_rng(seed)`` with a fixed draw order (endmember spectra, then
abundances, then noise) so that the GPU path and the CPU oracle consume the
same bytes.

This module holds no arithmetic of the PCA method itself (no band means, no
covariance, no eigen-solver, no projection): only linear mixing of
spectra, orthonormal bases for planted spectra, and noise.

Workloads (pixels x bands, component count k):
  linear_mixing     100x100 x 128, 5 endmembers U[0,1], Dirichlet(1), sigma 0.01, k=5
  paper_scene       610x340 x 103 and 512x217 x 224: 12 smooth spectra in [0, 8000],
                    Dirichlet(0.5) abundances correlated over 8x8 blocks,
                    Poisson-like noise, k=10
  planted_spectrum  2048x2048 x 224, s_i = 0.7^(i-1) over 20 components,
                    1e-3 floor, values in [0, 1] rounded to bf16 (or fp16), k=20
                    (planted_spectrum_device: the same recipe drawn on a GPU)
  tile_batch        256 tiles, N log-uniform in [4096, 262144],
                    B in {64,96,128,160,200,224,256}, 3-15 endmembers, k=8
                    (tile: numpy on the host; tile_device: torch on a GPU)
  gradient_cube     512x512 x 200 planted spectrum (s_i = 0.9^(i-1), i <= 11,
                    0.05 floor), upstream gradient N(0,1), k=10
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


@dataclass
class Cube:
    name: str
    Y: np.ndarray            # [N, B] pixel-major (band-interleaved-by-pixel)
    k: int
    tol: float
    sweeps_max: int
    shape2d: tuple = ()       # (rows, cols) of the image, when it has one
    meta: dict = field(default_factory=dict)

    @property
    def N(self) -> int:
        return int(self.Y.shape[0])

    @property
    def B(self) -> int:
        return int(self.Y.shape[1])


def _dirichlet(rng, alpha, n):
    return rng.dirichlet(alpha, size=n)


def linear_mixing(seed: int = 0, rows: int = 100, cols: int = 100, bands: int = 128,
                  endmembers: int = 5, sigma: float = 0.01, k: int = 5,
                  tol: float = 1e-10, sweeps_max: int = 30, name: str = "linear_mixing") -> Cube:
    """Y = A M + sigma * noise; M ~ U[0,1]^(e x B), rows of A ~ Dirichlet(1_e); float32."""
    rng = np.random.default_rng(seed)
    M = rng.uniform(0.0, 1.0, size=(endmembers, bands))
    N = rows * cols
    A = _dirichlet(rng, np.ones(endmembers), N)
    noise = rng.standard_normal((N, bands))
    Y = (A @ M + sigma * noise).astype(np.float32)
    return Cube(name, Y, k, tol, sweeps_max, (rows, cols),
                dict(seed=seed, endmembers=endmembers, sigma=sigma))


def _smooth_spectra(rng, count: int, bands: int, lo: float, hi: float) -> np.ndarray:
    """Cumulative Gaussian random walks, Gaussian-smoothed (sigma = bands/20), min-max to [lo, hi]."""
    walk = np.cumsum(rng.standard_normal((count, bands)), axis=1)
    sig = max(bands / 20.0, 1e-6)
    half = int(math.ceil(3 * sig))
    t = np.arange(-half, half + 1)
    g = np.exp(-0.5 * (t / sig) ** 2)
    g /= g.sum()
    out = np.empty_like(walk)
    for i in range(count):
        padded = np.pad(walk[i], half, mode="reflect")
        out[i] = np.convolve(padded, g, mode="valid")
    mn = out.min(axis=1, keepdims=True)
    mx = out.max(axis=1, keepdims=True)
    return lo + (hi - lo) * (out - mn) / np.maximum(mx - mn, 1e-12)


def paper_scene(seed: int, rows: int, cols: int, bands: int, endmembers: int = 12,
                k: int = 10, tol: float = 1e-10, sweeps_max: int = 30,
                name: str = "paper_scene") -> Cube:
    """Scene-like cube: smooth spectra in [0, 8000], block-correlated Dirichlet(0.5)
    abundances (0.9 * per-8x8-block draw + 0.1 * per-pixel draw), Poisson-like noise
    y + sqrt(max(y, 0)) * N(0, 1); float32."""
    rng = np.random.default_rng(seed)
    M = _smooth_spectra(rng, endmembers, bands, 0.0, 8000.0)
    br, bc = -(-rows // 8), -(-cols // 8)
    alpha = np.full(endmembers, 0.5)
    Ablk = _dirichlet(rng, alpha, br * bc).reshape(br, bc, endmembers)
    Apix = _dirichlet(rng, alpha, rows * cols).reshape(rows, cols, endmembers)
    r = np.arange(rows)[:, None] // 8
    c = np.arange(cols)[None, :] // 8
    A = (0.9 * Ablk[r, c] + 0.1 * Apix).reshape(rows * cols, endmembers)
    clean = A @ M
    noise = rng.standard_normal(clean.shape)
    Y = (clean + np.sqrt(np.maximum(clean, 0.0)) * noise).astype(np.float32)
    return Cube(name, Y, k, tol, sweeps_max, (rows, cols), dict(seed=seed, endmembers=endmembers))


def paper_scenes(scale: float = 1.0):
    """The two scene-shaped cubes (610x340 x 103, seed 1; 512x217 x 224, seed 2).
    `scale` < 1 shrinks the image side lengths (tests), bands unchanged."""
    def s(v):
        return max(8, int(round(v * scale)))
    return [paper_scene(1, s(610), s(340), 103, name="scene_610x340x103"),
            paper_scene(2, s(512), s(217), 224, name="scene_512x217x224")]


def orthonormal_basis(rng, B: int) -> np.ndarray:
    """B x B orthonormal matrix from the QR factorisation of a Gaussian matrix."""
    Wq, R = np.linalg.qr(rng.standard_normal((B, B)))
    return Wq * np.sign(np.diag(R))[None, :]


def planted_spectrum(seed: int = 20, side: int = 2048, bands: int = 224, comps: int = 20,
                     ratio: float = 0.7, floor: float = 1e-3, dtype: str = "bf16",
                     k: int = 20, tol: float = 1e-10, sweeps_max: int = 30,
                     chunk: int = 1 << 18, name: str = "planted_spectrum",
                     pixels: int | None = None):
    """Y = clip(0.5 + 0.08 U diag(s) W^T, 0, 1) rounded to bf16 or fp16, U ~ N(0,1),
    W orthonormal, s_i = ratio^(i-1) for i <= comps, floor otherwise.
    Returns a Cube whose Y is a torch tensor of the requested 16-bit dtype (CPU).
    pixels: only the first `pixels` rows of the side x side cube (the same values
    the whole cube has there; a bounded sample for a slow consumer)."""
    import torch
    rng = np.random.default_rng(seed)
    W = orthonormal_basis(rng, bands)
    s = np.full(bands, floor)
    s[:comps] = ratio ** np.arange(comps)
    Ms = (s[:, None] * W.T).astype(np.float32)          # diag(s) W^T
    N = side * side if pixels is None else min(side * side, int(pixels))
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float16
    out = torch.empty((N, bands), dtype=tdt)
    for n0 in range(0, N, chunk):
        n1 = min(N, n0 + chunk)
        U = rng.standard_normal((n1 - n0, bands), dtype=np.float32)
        blk = np.clip(0.5 + 0.08 * (U @ Ms), 0.0, 1.0)
        out[n0:n1] = torch.from_numpy(blk).to(tdt)
    return Cube(name, out, k, tol, sweeps_max, (side, side),
                dict(seed=seed, s=s, W=W, dtype=dtype))


def planted_spectrum_device(device, seed: int = 20, side: int = 2048, bands: int = 224,
                            comps: int = 20, ratio: float = 0.7, floor: float = 1e-3,
                            dtype: str = "bf16", k: int = 20, tol: float = 1e-10,
                            sweeps_max: int = 30, chunk: int = 1 << 20,
                            name: str = "planted_spectrum"):
    """The recipe of ``planted_spectrum`` (same W and s from the same numpy seed)
    with U ~ N(0, 1) drawn on a CUDA device by a torch generator seeded with
    `seed`, for the full-size cube that would take long to draw on the host.
    The values differ from ``planted_spectrum``'s (another generator of U); the
    distribution is the same.  Y is a device tensor of the 16-bit dtype."""
    import torch
    rng = np.random.default_rng(seed)
    W = orthonormal_basis(rng, bands)
    s = np.full(bands, floor)
    s[:comps] = ratio ** np.arange(comps)
    Ms = torch.from_numpy((s[:, None] * W.T).astype(np.float32)).to(device)
    N = side * side
    tdt = torch.bfloat16 if dtype == "bf16" else torch.float16
    out = torch.empty((N, bands), dtype=tdt, device=device)
    gen = torch.Generator(device=device)
    gen.manual_seed(int(seed))
    for n0 in range(0, N, chunk):
        n1 = min(N, n0 + chunk)
        U = torch.randn(n1 - n0, bands, generator=gen, device=device, dtype=torch.float32)
        out[n0:n1] = (U @ Ms).mul_(0.08).add_(0.5).clamp_(0.0, 1.0).to(tdt)
    return Cube(name, out, k, tol, sweeps_max, (side, side),
                dict(seed=seed, s=s, W=W, dtype=dtype, generator="torch-device"))


TILE_BANDS = (64, 96, 128, 160, 200, 224, 256)


def tile_batch_specs(seed: int = 3, tiles: int = 256, n_lo: int = 4096, n_hi: int = 262144):
    """(N_t, B_t, e_t, seed_t) for every tile; N log-uniform, B and e uniform."""
    rng = np.random.default_rng(seed)
    N = np.rint(np.exp(rng.uniform(math.log(n_lo), math.log(n_hi), size=tiles))).astype(np.int64)
    Bt = rng.choice(np.array(TILE_BANDS), size=tiles)
    e = rng.integers(3, 16, size=tiles)
    seeds = rng.integers(0, 2**31 - 1, size=tiles)
    return [(int(N[i]), int(Bt[i]), int(e[i]), int(seeds[i])) for i in range(tiles)]


def tile(spec, k: int = 8, tol: float = 1e-8, sweeps_max: int = 30) -> Cube:
    N, B, e, sd = spec
    rng = np.random.default_rng(sd)
    M = rng.uniform(0.0, 1.0, size=(e, B))
    A = _dirichlet(rng, np.ones(e), N)
    Y = (A @ M + 0.01 * rng.standard_normal((N, B))).astype(np.float32)
    return Cube(f"tile_{N}x{B}_e{e}", Y, k, tol, sweeps_max, (), dict(seed=sd, endmembers=e))


def tile_device(spec, device, k: int = 8, tol: float = 1e-8, sweeps_max: int = 30) -> Cube:
    """The same recipe as ``tile`` (U[0,1] endmembers, Dirichlet(1) abundances as
    normalised exponential draws, 0.01 Gaussian noise, FP32) drawn on a CUDA
    device with a torch generator seeded by the tile seed -- for full-size
    batches whose 10 GB would take minutes to draw on the host.  The values
    differ from ``tile``'s (another generator); the distribution is the same."""
    import torch
    N, B, e, sd = spec
    gen = torch.Generator(device=device)
    gen.manual_seed(int(sd))
    M = torch.rand(e, B, generator=gen, device=device, dtype=torch.float32)
    A = torch.empty(N, e, device=device, dtype=torch.float32).exponential_(generator=gen)
    A /= A.sum(dim=1, keepdim=True)
    Y = torch.randn(N, B, generator=gen, device=device, dtype=torch.float32).mul_(0.01)
    Y.addmm_(A, M)
    return Cube(f"tile_{N}x{B}_e{e}", Y, k, tol, sweeps_max, (), dict(seed=sd, endmembers=e))


def gradient_cube(seed: int = 4, side: int = 512, bands: int = 200, comps: int = 11,
                  ratio: float = 0.9, floor: float = 0.05, scale: float = 0.1,
                  k: int = 10, grad_seed: int = 40, name: str = "gradient_cube"):
    """Planted cube Y = 0.5 + scale * U diag(s) W^T (float32) and an upstream
    gradient dQ ~ N(0, 1) of shape [N, k] (float32, its own seed)."""
    rng = np.random.default_rng(seed)
    W = orthonormal_basis(rng, bands)
    s = np.full(bands, floor)
    s[:comps] = ratio ** np.arange(comps)
    N = side * side
    U = rng.standard_normal((N, bands))
    Y = (0.5 + scale * (U * s[None, :]) @ W.T).astype(np.float32)
    dQ = np.random.default_rng(grad_seed).standard_normal((N, k)).astype(np.float32)
    return Cube(name, Y, k, 1e-10, 30, (side, side), dict(seed=seed, s=s, W=W, dQ=dQ))
