"""Seeded synthetic 3DGS scenes and search grids.

This module only draws random inputs. It holds none of the method's
arithmetic (no quantisation, no ordering, no entropy), so both the CUDA path
and the CPU oracle can be fed from it.

Attribute layout (Sec. 2, "Preliminary": mu in R^3, q in R^4, s in R^3,
SH in R^{3(f+1)^2} with f = 3, opacity): 59 FP32 channels per Gaussian, in
this channel order:

    0-2    position (mu)
    3-5    SH DC (degree-0 colour)
    6-50   SH rest (45 higher-degree coefficients)
    51     opacity logit
    52-54  log-scale (s)
    55-58  rotation quaternion (q)

The paper's datasets (Mip-NeRF 360 etc.) are not available; these
distributions stand in for a trained scene of the same size (Sec. 1 quotes
5.27 M Gaussians for *bicycle*):

    position   mixture of 32 isotropic Gaussians (sigma 0.05) with centres
               uniform in [0.1, 0.9]^3, clipped to [0, 1]
    SH DC      N(0, 0.5^2)
    SH rest    Laplace(0, 0.05)
    opacity    N(0, 2^2)
    log-scale  N(-4, 1)
    rotation   4 x N(0, 1), normalised to a unit quaternion
    importance LogNormal(0, 1)   (stands in for I_g = I_d * I_i, Sec. 3.1)
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

N_CHANNELS = 59
CH_POS = slice(0, 3)
CH_SH_DC = slice(3, 6)
CH_SH_REST = slice(6, 51)
CH_OPACITY = 51
CH_LOG_SCALE = slice(52, 55)
CH_ROTATION = slice(55, 59)

_CHUNK = 1 << 20


def make_scene(n: int, seed: int) -> tuple[np.ndarray, np.ndarray]:
    """Return (attrs float32 [n, 59] C-contiguous, importance float32 [n])."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x3D65]))
    attrs = np.empty((n, N_CHANNELS), dtype=np.float32)
    centres = rng.uniform(0.1, 0.9, size=(32, 3)).astype(np.float32)
    for lo in range(0, n, _CHUNK):
        hi = min(n, lo + _CHUNK)
        m = hi - lo
        comp = rng.integers(0, 32, size=m)
        pos = centres[comp] + np.float32(0.05) * rng.standard_normal((m, 3), dtype=np.float32)
        attrs[lo:hi, CH_POS] = np.clip(pos, 0.0, 1.0)
        attrs[lo:hi, CH_SH_DC] = np.float32(0.5) * rng.standard_normal((m, 3), dtype=np.float32)
        mag = rng.standard_exponential((m, 45), dtype=np.float32) * np.float32(0.05)
        sign = rng.random((m, 45), dtype=np.float32) < 0.5
        attrs[lo:hi, CH_SH_REST] = np.where(sign, -mag, mag)
        attrs[lo:hi, CH_OPACITY] = np.float32(2.0) * rng.standard_normal(m, dtype=np.float32)
        attrs[lo:hi, CH_LOG_SCALE] = np.float32(-4.0) + rng.standard_normal((m, 3), dtype=np.float32)
        quat = rng.standard_normal((m, 4), dtype=np.float32)
        quat /= np.linalg.norm(quat, axis=1, keepdims=True).astype(np.float32)
        attrs[lo:hi, CH_ROTATION] = quat
    importance = np.exp(rng.standard_normal(n, dtype=np.float32)).astype(np.float32)
    return attrs, importance


def keep_counts(n: int, ratios: list[tuple[int, int]]) -> np.ndarray:
    """Kept-set sizes K_r = floor(p * n / q) for reserve ratios p/q, in int64."""
    return np.array([(p * int(n)) // q for p, q in ratios], dtype=np.int64)


@dataclass(frozen=True)
class Workload:
    """A named search workload: scene size, reserve ratios, bit-widths, group size."""
    name: str
    n: int
    ratios: tuple[tuple[int, int], ...]
    bits: tuple[int, ...]
    group_size: int
    budget_bytes: float | None = None
    seed: int = 0

    def keep(self) -> np.ndarray:
        return keep_counts(self.n, list(self.ratios))


def tenths() -> tuple[tuple[int, int], ...]:
    return tuple((k, 10) for k in range(1, 11))


def twentieths() -> tuple[tuple[int, int], ...]:
    return tuple((k, 20) for k in range(1, 21))


# The paper's workloads, as synthetic stand-ins (sizes: Sec. 1; grids: Sec. 3.6).
SMALL = Workload("single scene N=100k, r=1/2, b={4,6,8,10,12,16}, G=4096",
                 100_000, ((1, 2),), (4, 6, 8, 10, 12, 16), 4096)
SCENE = Workload("scene-scale search N=5.27M, r=0.1..1.0, b={2,3,4,5,6,8,10,12,14,16}, G=4096, 40 MB",
                 5_270_000, tenths(), (2, 3, 4, 5, 6, 8, 10, 12, 14, 16), 4096, 40e6)
LARGE = Workload("large grid N=6M, r=0.05..1.00, b=1..16, G=2048, 8 budgets",
                 6_000_000, twentieths(), tuple(range(1, 17)), 2048)


def batch_sizes(n_scenes: int, lo: int, hi: int, seed: int) -> np.ndarray:
    """Scene sizes drawn log-uniformly from [lo, hi]."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0xBA7C]))
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=n_scenes)).astype(np.int64)


def poisson_arrivals(n_jobs: int, rate_per_s: float, seed: int,
                     n_lo: int = 100_000, n_hi: int = 6_000_000,
                     budget_lo: float = 5e6, budget_hi: float = 60e6):
    """Job stream for the serving workload: (arrival time s, scene size, byte budget)."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x5E7F]))
    gaps = rng.exponential(1.0 / rate_per_s, size=n_jobs)
    t = np.cumsum(gaps) - gaps[0]
    sizes = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), size=n_jobs)).astype(np.int64)
    budgets = rng.uniform(budget_lo, budget_hi, size=n_jobs)
    return t, sizes, budgets


def vq_batches(n: int, iters: int, batch: int, seed: int) -> np.ndarray:
    """Row indices of the mini-batches of the SH clustering: [iters, batch]
    int32, drawn uniformly (with replacement) from range(n)."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0x51A]))
    return rng.integers(0, n, size=(iters, batch), dtype=np.int64).astype(np.int32)


def vq_init_rows(n: int, K: int, seed: int) -> np.ndarray:
    """K distinct rows whose vectors seed the codebook (int32 [K])."""
    rng = np.random.default_rng(np.random.SeedSequence([int(seed), 0xC0DE]))
    return np.sort(rng.choice(n, size=K, replace=False)).astype(np.int32)


# SH clustering stand-in: the 45 SH-rest coefficients of the scene-scale
# scene, a 4096-entry codebook, 50 mini-batches of 65536 vectors.
VQ_K, VQ_ITERS, VQ_BATCH = 4096, 50, 65536
