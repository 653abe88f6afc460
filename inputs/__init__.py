"""Seeded synthetic inputs shared by the oracle side and the CUDA side of the tests.

This module holds no arithmetic of the method: it only draws reproducible random
arrays (numpy PCG64 from an integer seed) in the layouts the two sides take.
Positions are in units of the box side, as uint32 ticks (2^32 per side) or FP64
fractions; momenta are in Mpc/h; fields are C-ordered (x slowest, z fastest).

Shapes follow the paper's workloads: particles in Lagrangian (lattice) order with
displacements of a few mesh cells, as in a particle-mesh run whose lattice
matches or is coarser than its mesh (Sec. 3), clustered tails for the late-time
deposit, and Gaussian fields for the FFT estimators.
"""
import numpy as np


def rng(seed):
    return np.random.default_rng(np.random.PCG64(int(seed)))


def lattice_order_ticks(seed, n_side, sigma_cells, n_mesh=None, tail_fraction=0.0, tail_cells=8.0):
    """uint32 positions (3, n_side^3): lattice nodes plus Gaussian offsets in mesh cells.

    A fraction ``tail_fraction`` of particles gets offsets of width ``tail_cells``
    (the clustered, far-travelled population of a late-time run).
    """
    r = rng(seed)
    n_mesh = n_side if n_mesh is None else n_mesh
    i = np.arange(n_side, dtype=np.float64) / n_side
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    q = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    off = r.normal(0.0, sigma_cells / n_mesh, size=q.shape)
    if tail_fraction > 0:
        tail = r.random(q.shape[1]) < tail_fraction
        off[:, tail] = r.normal(0.0, tail_cells / n_mesh, size=(3, int(tail.sum())))
    u = q + off
    u = u - np.floor(u)
    t = np.floor(u * 2.0**32).astype(np.uint64) % np.uint64(2**32)
    return t.astype(np.uint32)


def uniform_ticks(seed, count):
    """uint32 positions (3, count) uniform in the box (any count: ragged tails)."""
    return rng(seed).integers(0, 2**32, size=(3, count), dtype=np.uint64).astype(np.uint32)


def clustered_ticks(seed, count, n_clusters=16, width=0.01):
    """uint32 positions (3, count) in Gaussian blobs (heavy atomic contention)."""
    r = rng(seed)
    centres = r.random((3, n_clusters))
    which = r.integers(0, n_clusters, size=count)
    u = centres[:, which] + r.normal(0.0, width, size=(3, count))
    u = u - np.floor(u)
    return (np.floor(u * 2.0**32).astype(np.uint64) % np.uint64(2**32)).astype(np.uint32)


def ticks_to_fractions(t):
    """Exact FP64 box fractions of uint32 ticks (a change of unit, not a computation)."""
    return np.asarray(t, dtype=np.float64) * 2.0**-32


def momenta(seed, count, scale):
    """FP64 momenta (3, count), Gaussian with standard deviation ``scale`` Mpc/h."""
    return rng(seed).normal(0.0, scale, size=(3, count))


def gaussian_field(seed, n, dtype=np.float64):
    """Real white-noise field (n, n, n), unit variance."""
    return rng(seed).standard_normal((n, n, n)).astype(dtype)


def lognormal_field(seed, n, sigma=1.0, dtype=np.float64):
    """Positive, skewed field exp(sigma g) - mean (late-time density-like values)."""
    g = rng(seed).standard_normal((n, n, n))
    f = np.exp(sigma * g)
    return (f / f.mean() - 1.0).astype(dtype)
