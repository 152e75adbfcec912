"""Seeded densities and incident directions."""
from __future__ import annotations

import numpy as np


def random_density(n: int, seed: int = 0, nrhs: int = 1, dtype=np.complex128):
    """Complex standard-normal density, shape [n] (nrhs == 1) or [nrhs, n].

    Real and imaginary parts are independent N(0, 1/2) so E|x|^2 = 1.
    """
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs == 1 else (nrhs, n)
    x = (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / np.sqrt(2.0)
    return x.astype(dtype)


def fibonacci_directions(n: int, seed: int = 0):
    """n unit vectors on a golden-angle Fibonacci sphere, randomly rotated.

    The rotation is a seeded uniform random orthogonal matrix (QR of a
    Gaussian matrix with the sign fix), so the set is deterministic per seed.
    """
    i = np.arange(n, dtype=np.float64)
    z = 1.0 - 2.0 * (i + 0.5) / n
    r = np.sqrt(np.maximum(0.0, 1.0 - z * z))
    ga = np.pi * (3.0 - np.sqrt(5.0))
    phi = ga * i
    d = np.stack([r * np.cos(phi), r * np.sin(phi), z], axis=1)
    rng = np.random.default_rng(seed)
    q, rr = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(rr))[None, :]
    return d @ q.T
