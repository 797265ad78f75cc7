"""Seeded synthetic inputs shaped like the paper's workloads.

The paper measures on SDRBench quantization codes (hurricane, HACC, Nyx;
uint16 from cuSZ), the RTM float32 field and TPC-H int32/string columns
(section 4.1).  Those datasets are not available here; these generators
stand in for them with the same element types and similar structure.  This
module holds no compression arithmetic: it only draws numbers, so both the
CUDA path and the CPU oracle can consume the same bytes.

Every generator is a pure function of its arguments (numpy ``default_rng``
seeded explicitly; large arrays are drawn in fixed-size blocks, each from
its own child seed, so the result does not depend on memory limits).
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

_BLOCK = 1 << 22  # elements per independently seeded block


def sha256(a: np.ndarray) -> str:
    return hashlib.sha256(np.ascontiguousarray(a).view(np.uint8)).hexdigest()


def _block_rngs(seed: int, n: int):
    nblk = math.ceil(n / _BLOCK)
    seqs = np.random.SeedSequence(seed).spawn(nblk)
    for i, s in enumerate(seqs):
        lo = i * _BLOCK
        yield lo, min(n, lo + _BLOCK), np.random.default_rng(s)


def quant_codes_laplace(n: int, seed: int = 0, b: float = 2.0,
                        copy_prob: float = 0.3) -> np.ndarray:
    """uint16 codes: 512 + round(Laplace(0, b)) clipped to [0, 1023], where a
    fraction ``copy_prob`` of positions repeat the previous value (runs).
    Stand-in for cuSZ quantization codes (paper section 4.1)."""
    out = np.empty(n, np.uint16)
    last = None
    for lo, hi, rng in _block_rngs(seed, n):
        m = hi - lo
        v = np.clip(512 + np.rint(rng.laplace(0.0, b, m)), 0, 1023)
        copy = rng.random(m) < copy_prob
        if lo == 0:
            copy[0] = False
        idx = np.where(copy, -1, np.arange(m))
        src = np.maximum.accumulate(np.maximum(idx, -1))
        vals = np.where(src >= 0, v[np.maximum(src, 0)],
                        last if last is not None else 512)
        out[lo:hi] = vals.astype(np.uint16)
        last = out[hi - 1]
    return out


def markov_codes(n: int, seed: int = 0, stay: float = 0.6,
                 b: float = 4.0) -> np.ndarray:
    """First-order Markov chain of codes in [0, 1023] (as uint32): start at
    512; each step keeps the previous value with probability ``stay``, else
    jumps to 512 + round(Laplace(0, b)) clipped.  Store as uint8 (mod 256),
    uint16 or uint32 to get 1-, 2- or 4-byte symbols."""
    out = np.empty(n, np.uint32)
    last = 512
    for lo, hi, rng in _block_rngs(seed, n):
        m = hi - lo
        jump = rng.random(m) >= stay
        v = np.clip(512 + np.rint(rng.laplace(0.0, b, m)), 0, 1023)
        idx = np.where(jump, np.arange(m), -1)
        src = np.maximum.accumulate(idx)
        out[lo:hi] = np.where(src >= 0, v[np.maximum(src, 0)], last)
        last = int(out[hi - 1])
    return out


def gaussian_field(shape=(512, 512, 256), n_gauss: int = 16, seed: int = 0,
                   noise: float = 1e-4) -> np.ndarray:
    """float32 smooth field: sum of ``n_gauss`` isotropic 3-D Gaussians
    (centres uniform in the grid, sigma ~ U[8, 64] voxels, amplitude ~
    N(0, 1)) plus N(0, noise) noise; computed in float64, C order.
    Stand-in for the RTM float32 field."""
    rng = np.random.default_rng(seed)
    nx, ny, nz = shape
    centres = rng.uniform(0.0, 1.0, (n_gauss, 3)) * np.array(shape, float)
    sigma = rng.uniform(8.0, 64.0, n_gauss)
    amp = rng.normal(0.0, 1.0, n_gauss)
    gx = [np.exp(-((np.arange(nx) - c[0]) ** 2) / (2 * s * s))
          for c, s in zip(centres, sigma)]
    gy = [np.exp(-((np.arange(ny) - c[1]) ** 2) / (2 * s * s))
          for c, s in zip(centres, sigma)]
    gz = [np.exp(-((np.arange(nz) - c[2]) ** 2) / (2 * s * s))
          for c, s in zip(centres, sigma)]
    out = np.empty(shape, np.float32)
    slab = max(1, (1 << 22) // (ny * nz))
    for x0 in range(0, nx, slab):
        x1 = min(nx, x0 + slab)
        acc = np.zeros((x1 - x0, ny, nz))
        for g in range(n_gauss):
            acc += amp[g] * gx[g][x0:x1, None, None] * np.outer(gy[g], gz[g])[None]
        acc += rng.normal(0.0, noise, acc.shape)
        out[x0:x1] = acc
    return out


def sorted_indices(n: int, p: float = 0.3, seed: int = 0) -> np.ndarray:
    """int32 strictly increasing indices: cumulative sum of geometric(p)
    gaps (support >= 1).  Stand-in for TPC-H int32 columns."""
    out = np.empty(n, np.int32)
    carry = 0
    for lo, hi, rng in _block_rngs(seed, n):
        c = np.cumsum(rng.geometric(p, hi - lo), dtype=np.int64) + carry
        out[lo:hi] = c
        carry = int(c[-1])
    return out


def uniform_bytes(n: int, seed: int = 0) -> np.ndarray:
    """Incompressible control: uniform random bytes."""
    out = np.empty(n, np.uint8)
    for lo, hi, rng in _block_rngs(seed, n):
        out[lo:hi] = rng.integers(0, 256, hi - lo, dtype=np.uint8)
    return out


def constant_run(n_sym: int, value: int, dtype) -> np.ndarray:
    return np.full(n_sym, value, dtype)


def periodic(n_sym: int, q: int, dtype) -> np.ndarray:
    """x[i] = i mod q."""
    return (np.arange(n_sym) % q).astype(dtype)


# --- configuration recipes ---------------------------------------------------

def workload_small(seed: int = 0) -> np.ndarray:
    """1 MiB of uint16 quantization-code-like symbols (524,288)."""
    return quant_codes_laplace(524_288, seed=seed)


def batch_buffers(n_buffers: int = 10_000, seed: int = 0,
                  lo_bytes: int = 4096, hi_bytes: int = 16 << 20):
    """Sizes and dtypes of a batch of independent buffers: sizes log-uniform
    in [lo_bytes, hi_bytes] rounded down to a multiple of 16, dtype uniform
    over {uint8 codes, uint16 codes, float32 field slices, int32 indices}.
    Returns (sizes, kinds) where kind 0..3 is that order."""
    rng = np.random.default_rng(seed)
    sizes = np.exp(rng.uniform(math.log(lo_bytes), math.log(hi_bytes),
                               n_buffers))
    sizes = (sizes.astype(np.int64) // 16) * 16
    sizes = np.maximum(sizes, 16)
    kinds = rng.integers(0, 4, n_buffers)
    return sizes, kinds


def serving_trace(rate: float = 2000.0, duration: float = 60.0,
                  seed: int = 0, median_bytes: int = 256 << 10,
                  sigma: float = 1.5, cap_bytes: int = 64 << 20,
                  compress_frac: float = 0.7):
    """Poisson arrivals: (arrival_s, is_compress, size_bytes, symbol_bytes)
    arrays.  Sizes lognormal(ln median, sigma) capped, rounded down to the
    symbol size (and to at least one symbol)."""
    rng = np.random.default_rng(seed)
    n = int(rng.poisson(rate * duration))
    arrivals = np.sort(rng.uniform(0.0, duration, n))
    is_comp = rng.random(n) < compress_frac
    sizes = np.minimum(rng.lognormal(math.log(median_bytes), sigma, n),
                       cap_bytes).astype(np.int64)
    sym = np.array([1, 2, 4])[rng.integers(0, 3, n)]
    sizes = np.maximum((sizes // sym) * sym, sym)
    return arrivals, is_comp, sizes, sym
