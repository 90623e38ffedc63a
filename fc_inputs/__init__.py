"""Seeded synthetic inputs for the fibre-bundle CG solve.

This module only draws random numbers and lays them out; it holds none of the
method's arithmetic (no Green's function, no convolution, no solver).  It is the
one piece shared by the CPU oracle's tests, the CUDA path's tests and the
benchmark, so both sides always see identical arrays.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used in its counter form: draw k of stream
``seed`` is ``mix64(seed + (k + 1) * 0x9E3779B97F4A7C15)``.

Conventions (the paper gives no RNG, only distributions):
  * uniform in (0, 1): ``((z >> 11) + 0.5) * 2**-53``, never exactly 0 or 1;
  * N(0, 1): Box-Muller on consecutive pairs of uniforms (cos branch first);
  * fields are row-major, flat index ``i = iy * L + ix``;
  * per problem the stream is consumed in the order s, then b, then t.
"""
from __future__ import annotations

import math

import numpy as np

__all__ = [
    "splitmix64",
    "uniform",
    "normal",
    "problem",
    "request_stream",
    "padded_side",
]

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Draws ``start .. start+count-1`` of SplitMix64 stream ``seed`` (uint64)."""
    k = np.arange(start + 1, start + 1 + count, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, start: int, count: int) -> np.ndarray:
    """Uniform float64 draws in the open interval (0, 1)."""
    z = splitmix64(seed, start, count)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (2.0 ** -53)


def normal(seed: int, start: int, count: int) -> tuple[np.ndarray, int]:
    """N(0,1) draws by Box-Muller; returns (values, uniforms consumed)."""
    pairs = (count + 1) // 2
    u = uniform(seed, start, 2 * pairs)
    u1, u2 = u[0::2], u[1::2]
    rad = np.sqrt(-2.0 * np.log(u1))
    out = np.empty(2 * pairs, dtype=np.float64)
    out[0::2] = rad * np.cos(2.0 * math.pi * u2)
    out[1::2] = rad * np.sin(2.0 * math.pi * u2)
    return out[:count], 2 * pairs


def padded_side(L: int) -> int:
    """Side M of the zero-padded FFT grid: the smallest power of two >= 2L."""
    if L < 1:
        raise ValueError("L must be >= 1")
    m = 2
    while m < 2 * L:
        m *= 2
    return m


def problem(L: int, seed: int, b_kind: str = "ones", with_t: bool = False,
            s_lo: float = 0.5, s_hi: float = 1.5, t_gradient: float = 0.0) -> dict:
    """One synthetic system (C + diag(s)) x = b on an L x L grid.

    s ~ U[s_lo, s_hi] (the fibres' compliances), b = 1 (uniform plate
    displacement) or b ~ N(0, 1), and optionally breaking thresholds
    t = xi + t_gradient (iy + 1/2) / L with xi ~ U(0, 1): a threshold
    gradient along y directs the fracture front (Section 2 of the paper
    names a gradient in the threshold distribution as the simplest way to
    load the system with one).  All arrays are float64 of length L*L,
    row-major.
    """
    n = L * L
    pos = 0
    s = s_lo + (s_hi - s_lo) * uniform(seed, pos, n)
    pos += n
    if b_kind == "ones":
        b = np.ones(n, dtype=np.float64)
    elif b_kind == "normal":
        b, used = normal(seed, pos, n)
        pos += used
    else:
        raise ValueError(f"unknown b_kind {b_kind!r}")
    out = {"L": L, "seed": seed, "s": s, "b": b}
    if with_t:
        t = uniform(seed, pos, n)
        pos += n
        if t_gradient:
            t = t + t_gradient * (np.arange(n) // L + 0.5) / L
        out["t"] = t
    return out


def request_stream(count: int, seed: int, rate_per_s: float,
                   log2_lo: int = 5, log2_hi: int = 11,
                   tols: tuple = (1e-6, 1e-8)) -> list[dict]:
    """Serving workload: Poisson arrivals, L = 2**round(U[log2_lo, log2_hi]).

    Each request gets its own problem seed (``seed * 1_000_003 + k``), a
    tolerance drawn uniformly from ``tols`` and an arrival time from
    exponential gaps of mean 1/rate.  Rounding the log-uniform exponent gives
    the two end sizes half weight.
    """
    u = uniform(seed, 0, 3 * count).reshape(count, 3)
    reqs = []
    t = 0.0
    for k in range(count):
        t += -math.log(u[k, 0]) / rate_per_s
        e = log2_lo + (log2_hi - log2_lo) * u[k, 1]
        L = 1 << int(math.floor(e + 0.5))
        tol = tols[min(int(u[k, 2] * len(tols)), len(tols) - 1)]
        reqs.append({"k": k, "arrival_s": t, "L": L, "tol": tol,
                     "seed": seed * 1_000_003 + k})
    return reqs
