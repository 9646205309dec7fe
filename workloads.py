"""Seeded synthetic inputs shared by the tests, the smoke check and the bench.

This module holds only random-number recipes (numpy ``default_rng``, PCG64);
it contains none of the transform's arithmetic, so both the CUDA path's
tests and the CPU oracle can draw the same inputs from it.

The paper times power-of-two vector lengths 2^3..2^24 and never states the
data content; these recipes stand in for that workload (uniform [-1, 1] real
and imaginary parts unless stated).
"""
from __future__ import annotations

import numpy as np


def uniform_complex(n: int, batch: int = 1, seed: int = 0) -> np.ndarray:
    """batch x n complex128, re then im drawn as two arrays of n*batch
    i.i.d. uniform[-1, 1] values from ``default_rng(seed)``."""
    rng = np.random.default_rng(seed)
    re = rng.uniform(-1.0, 1.0, n * batch)
    im = rng.uniform(-1.0, 1.0, n * batch)
    return (re + 1j * im).reshape(batch, n)


def gaussian_complex(n: int, batch: int = 1, seed: int = 0, sigma: float = 1.0) -> np.ndarray:
    """batch x n complex128 with i.i.d. N(0, sigma^2) real and imaginary parts."""
    rng = np.random.default_rng(seed)
    re = rng.normal(0.0, sigma, n * batch)
    im = rng.normal(0.0, sigma, n * batch)
    return (re + 1j * im).reshape(batch, n)


def dynamic_range_complex(n: int, batch: int = 1, seed: int = 0, lo: float = -4.0,
                          hi: float = 4.0) -> np.ndarray:
    """batch x n complex128 with amplitude 10^U(lo, hi) and phase U(0, 2 pi)."""
    rng = np.random.default_rng(seed)
    amp = 10.0 ** rng.uniform(lo, hi, n * batch)
    ph = rng.uniform(0.0, 2.0 * np.pi, n * batch)
    return (amp * np.cos(ph) + 1j * amp * np.sin(ph)).reshape(batch, n)


def closed_form_inputs(n: int):
    """Named length-n inputs whose DFT has a closed form:
    delta_0, delta_5, constant one, cos(2 pi f k / n) and sin(2 pi f k / n)
    with f = 37 (f reduced mod n for small n)."""
    k = np.arange(n)
    f = 37 % max(n, 1)
    d0 = np.zeros(n, np.complex128)
    d0[0] = 1.0
    d5 = np.zeros(n, np.complex128)
    d5[5 % n] = 1.0
    return {
        "delta0": d0,
        "delta5": d5,
        "const": np.ones(n, np.complex128),
        "cos37": np.cos(2.0 * np.pi * f * k / n).astype(np.complex128),
        "sin37": np.sin(2.0 * np.pi * f * k / n).astype(np.complex128),
    }


def uneven_sizes(count: int = 20000, seed: int = 1, lo_exp: int = 6, hi_exp: int = 16):
    """Log-uniform power-of-two sizes: exponents i.i.d. uniform integers in
    [lo_exp, hi_exp] from ``default_rng(seed)``.  Returns (sizes, rng) so the
    caller draws the data next from the same generator."""
    rng = np.random.default_rng(seed)
    k = rng.integers(lo_exp, hi_exp + 1, size=count)
    return (np.int64(1) << k.astype(np.int64)), rng


def uneven_batch(count: int = 20000, seed: int = 1, lo_exp: int = 6, hi_exp: int = 16):
    """The uneven batch: sizes as in :func:`uneven_sizes`, then the packed
    data (re then im, uniform[-1, 1]) drawn next from the same generator."""
    sizes, rng = uneven_sizes(count, seed, lo_exp, hi_exp)
    total = int(sizes.sum())
    re = rng.uniform(-1.0, 1.0, total)
    im = rng.uniform(-1.0, 1.0, total)
    return sizes, re + 1j * im


def loss_problem(n: int, batch: int, seed_x: int = 0, seed_h: int = 2, seed_y: int = 3):
    """The differentiation workload: x uniform from ``default_rng(seed_x)``,
    H and y complex Gaussian from ``default_rng(seed_h)`` and
    ``default_rng(seed_y)``; all batch x n complex128."""
    x = uniform_complex(n, batch, seed_x)
    H = gaussian_complex(n, batch, seed_h)
    y = gaussian_complex(n, batch, seed_y)
    return x, H, y
