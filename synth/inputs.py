"""Seeded random inputs (numpy PCG64 generators).

noise_field   xi ~ U[-1, 1] per cell, for the "h <- h (1 + a xi)" perturbations of the
              ensemble workload (seed, member index)
bump_centres  n points uniform on the sphere as (lon, lat) pairs (Gaussian-bump centres)
fd_direction  a N(0, 1) field (finite-difference direction of gradient checks)
perturb_h     applies h <- h (1 + a xi) to a state: each cell's three conserved
              variables scale together (velocity unchanged)
"""
import numpy as np


def noise_field(shape, seed, member=0):
    rng = np.random.default_rng([int(seed), int(member)])
    return rng.uniform(-1.0, 1.0, size=shape)


def bump_centres(n, seed):
    rng = np.random.default_rng(int(seed))
    lon = rng.uniform(-np.pi, np.pi, size=n)
    lat = np.arcsin(rng.uniform(-1.0, 1.0, size=n))
    return np.stack([lon, lat], axis=1)


def fd_direction(shape, seed):
    rng = np.random.default_rng(int(seed))
    return rng.standard_normal(size=shape)


def perturb_h(q, xi, amp=0.01):
    """q: array (3, 6, N, N) (numpy or torch); xi: (6, N, N)."""
    return q * (1.0 + amp * xi)[None]
