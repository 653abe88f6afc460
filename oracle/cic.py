"""Cloud-in-cell (CIC) mass assignment, force interpolation, cell keys and order.

Oracle (test infrastructure only).

The paper measures the counting density delta = rho / rho_bar - 1 with the CIC
scheme of Pylians3 (Sec. 4) and runs particle-mesh codes (Sec. 2).  Reading used
here: mesh nodes sit at the cell centres x_j = (j + 1/2) L / N, while the
particle lattice of the initial conditions sits at q_i = i L / N_p (cell
corners).  A particle at mesh coordinate s = x N / L - 1/2 has base node
i = floor(s) mod N and fraction d = s - floor(s), with weights (1 - d, d) per
axis.  With particles starting half a cell away from the nodes the CIC density
responds linearly to sub-cell displacements; with particles on the nodes it would
respond to |displacement| and shift the density by half a cell.  Positions
arrive in units of the box side, either as uint32 ticks (2^32 per side) or as FP64
fractions; for power-of-two N the conversion to s is exact in both cases
(ticks: subtract half a cell, 2^(31 - log2 N) ticks, modulo 2^32), so the base
node is exact.
"""
import numpy as np


def mesh_coords(x, n):
    """Base node (3, Np) int64 and fraction (3, Np) FP64 of each particle."""
    x = np.asarray(x)
    if x.dtype == np.uint32:
        half = 2**31 // n
        t = (x.astype(np.int64) - half) % 2**32
        s = t.astype(np.float64) * (n / 2.0**32)
    else:
        s = x.astype(np.float64) * n - 0.5
    base = np.floor(s)
    frac = s - base
    return base.astype(np.int64) % n, frac


def _corners(base, frac, n):
    """Yield (linear node index, weight) for the 8 CIC corners."""
    for dx in (0, 1):
        wx = frac[0] if dx else 1.0 - frac[0]
        ix = (base[0] + dx) % n
        for dy in (0, 1):
            wy = frac[1] if dy else 1.0 - frac[1]
            iy = (base[1] + dy) % n
            for dz in (0, 1):
                wz = frac[2] if dz else 1.0 - frac[2]
                iz = (base[2] + dz) % n
                yield (ix * n + iy) * n + iz, wx * wy * wz


def deposit(x, n, mass=None):
    """Density rho on the n^3 mesh; mass per particle defaults to n^3 / N_particles.

    With that mass the mean of rho is exactly 1, and delta = rho - 1.
    """
    base, frac = mesh_coords(x, n)
    npart = base.shape[1]
    m = (n**3 / npart) if mass is None else mass
    rho = np.zeros(n**3)
    for idx, w in _corners(base, frac, n):
        rho += np.bincount(idx, weights=w * m, minlength=n**3)
    return rho.reshape(n, n, n)


def density_contrast(x, n):
    """Counting density contrast delta = rho / rho_bar - 1 (Sec. 4)."""
    return deposit(x, n) - 1.0


def interpolate(field, x):
    """CIC gather of a scalar mesh field at the particles (same weights as deposit)."""
    n = field.shape[0]
    base, frac = mesh_coords(x, n)
    flat = field.ravel()
    out = np.zeros(base.shape[1])
    for idx, w in _corners(base, frac, n):
        out += w * flat[idx]
    return out


def interpolate_gradient(field, x, box):
    """Gradient of the CIC (trilinear) interpolant of a mesh field at the particles.

    Returns (3, Np) in field units per Mpc/h.  Reading of the first-order gradient of the
    paper's PM code (Sec. 4.1 attributes its large-scale power deficit to it): inside the
    particle's cell the interpolant is linear along each axis, so its x derivative is the
    difference of the field between the cell's two x planes over the spacing L/N, weighted
    bilinearly in y and z with the CIC weights (likewise for y and z).  It uses the same
    eight corners as ``interpolate``.
    """
    n = field.shape[0]
    base, frac = mesh_coords(x, n)
    flat = field.ravel()
    inv_d = n / box
    out = np.zeros((3, base.shape[1]))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                d = (dx, dy, dz)
                idx = (((base[0] + dx) % n) * n + (base[1] + dy) % n) * n + (base[2] + dz) % n
                v = flat[idx]
                w = [frac[j] if d[j] else 1.0 - frac[j] for j in range(3)]
                s = [inv_d if d[j] else -inv_d for j in range(3)]
                out[0] += s[0] * w[1] * w[2] * v
                out[1] += w[0] * s[1] * w[2] * v
                out[2] += w[0] * w[1] * s[2] * v
    return out


def cell_keys(x, n):
    """Linear base-cell index (ix n + iy) n + iz of each particle."""
    base, _ = mesh_coords(x, n)
    return (base[0] * n + base[1]) * n + base[2]


def cell_order(x, n):
    """Particle order sorted by cell key, stable in particle id."""
    return np.argsort(cell_keys(x, n), kind="stable")
