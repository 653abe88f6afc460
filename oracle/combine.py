"""GR displacement field and the combined positions (Eqs. xiGR and combined, Sec. 2).

Oracle (test infrastructure only).

Eq. xiGR: xi = x_GR - x_Newton per particle id (the runs share their initial
phases and ids).  Eq. combined: x = x_Newton,target + xi.  Both equations are in
configuration space.  Readings used here:

* The difference is the minimum periodic image; on uint32 ticks the wrapping
  int32 difference is exactly that.
* When the GR/Newton pair runs on a coarser particle lattice (n_c per side) than
  the target run (n_t = r n_c, r a power of two), xi is interpolated trilinearly
  in Lagrangian coordinates q (periodic).  Target id (i, j, k) sits at coarse
  coordinate (i, j, k) / r, so the weights are integers over r^3: on ticks the
  interpolated value is round-half-even(sum_c W_c xi_c / r^3) (exact integer
  arithmetic); on FP64 fractions it is the plain weighted sum.
"""
import numpy as np


def displacement(x_gr, x_newton):
    """xi = minimum-image(x_GR - x_Newton) in box units (int32 ticks or FP64)."""
    if x_gr.dtype == np.uint32:
        d = (x_gr.astype(np.int64) - x_newton.astype(np.int64)) % 2**32
        d = np.where(d >= 2**31, d - 2**32, d)
        return d.astype(np.int32)
    d = x_gr.astype(np.float64) - x_newton.astype(np.float64)
    return d - np.rint(d)


def interpolate_lagrangian(xi, n_c, n_t):
    """Trilinear interpolation in q from the n_c^3 lattice to the n_t^3 lattice."""
    if n_t % n_c:
        raise ValueError("target lattice must be a multiple of the source lattice")
    r = n_t // n_c
    src = xi.reshape(3, n_c, n_c, n_c)
    if r == 1:
        return xi.copy()
    it = np.arange(n_t)
    base = it // r
    off = it % r
    out = np.zeros((3, n_t, n_t, n_t), dtype=np.int64 if xi.dtype == np.int32 else np.float64)
    for dx in (0, 1):
        wx = off if dx else r - off
        ix = (base + dx) % n_c
        for dy in (0, 1):
            wy = off if dy else r - off
            iy = (base + dy) % n_c
            for dz in (0, 1):
                wz = off if dz else r - off
                iz = (base + dz) % n_c
                W = wx[:, None, None] * wy[None, :, None] * wz[None, None, :]
                for j in range(3):
                    vals = src[j][np.ix_(ix, iy, iz)]
                    if xi.dtype == np.int32:
                        out[j] += W.astype(np.int64) * vals.astype(np.int64)
                    else:
                        out[j] += W * vals
    if xi.dtype == np.int32:
        res = np.rint(out.astype(np.float64) / r**3).astype(np.int64)
        return res.reshape(3, -1).astype(np.int32)
    return (out / r**3).reshape(3, -1)


def combine(x_target, xi_target):
    """x = x_target + xi (Eq. combined), wrapped into the box."""
    if x_target.dtype == np.uint32:
        return ((x_target.astype(np.int64) + xi_target.astype(np.int64)) % 2**32).astype(np.uint32)
    x = x_target + xi_target
    return x - np.floor(x)
