"""Zel'dovich (first-order LPT) and second-order LPT initial conditions on a particle lattice.

Oracle (test infrastructure only).

Sec. 2 combines Newtonian and relativistic runs that start from the same random
phases; Sec. 2 also names first-order LPT ("1LPT") as a way to produce particle
positions.  Sec. 3 starts the runs at z = 50.  Reading used here:

* delta_n = N^3 g_n sqrt(P(k_n)/V) on the N_p^3 lattice, with g_n the unit complex
  Gaussian of ``philox.hermitian_noise_half`` or g = FFT(w)/N^{3/2} for a caller's
  real white-noise field w; P is the z = 0 linear spectrum (D(1) = 1).
* Pairing (Sec. 4.2 uses the pairing method of Angulo & Pontzen 2016): "paired" flips
  the sign of every g_n; "fixed amplitude" replaces g_n by g_n/|g_n| (unit modulus,
  the same phase), so that |delta_n|^2 = N^6 P(k_n)/V holds mode by mode.
* Psi_n = i k delta_n / k^2 (the zero mode and Nyquist components are zero).
* x = q + D(a) Psi(q),  p = a^2 E(a) f(a) D(a) Psi(q), with q the lattice node
  i L / N_p and p = a^2 dx/dt / H0 (Mpc/h in H0 = 1 units).
* Positions are returned in units of the box side: as uint32 ticks
  (2^32 per side, exact periodic wrap) or as FP64 fractions in [0, 1).
"""
import numpy as np

from . import philox


def fix_amplitude(g):
    """g / |g| where g != 0, else 0 (the fixed-amplitude phases)."""
    r = np.abs(g)
    return np.where(r > 0, g / np.where(r > 0, r, 1.0), 0.0)


def linear_delta_k(cosmo, n, box, seed=None, white_noise=None, paired=False, fixed_amplitude=False):
    """delta_n at a = 1 on the rfftn half grid (n, n, n/2+1)."""
    if white_noise is not None:
        w = np.asarray(white_noise, dtype=np.float64).reshape(n, n, n)
        g = np.fft.rfftn(w) / n**1.5
        f = philox.signed_freqs(n)
        fz = np.arange(n // 2 + 1)
        NX, NY, NZ = np.meshgrid(f, f, fz, indexing="ij")
        nyq = (np.abs(NX) == n // 2) | (np.abs(NY) == n // 2) | (NZ == n // 2)
        g = np.where(nyq, 0.0, g)
        g[0, 0, 0] = 0.0
    else:
        g = philox.hermitian_noise_half(seed, n)
    if fixed_amplitude:
        g = fix_amplitude(g)
    if paired:
        g = -g
    kf = 2.0 * np.pi / box
    n2 = mode_n2(n)
    k = kf * np.sqrt(n2.astype(np.float64))
    pk = np.zeros_like(k)
    nz = n2 > 0
    pk[nz] = cosmo.power_linear(k[nz])
    return n**3 * g * np.sqrt(pk / box**3)


def mode_n2(n):
    """|n|^2 on the rfftn half grid, with signed integer wavenumbers."""
    f = philox.signed_freqs(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64)
    NX, NY, NZ = np.meshgrid(f, f, fz, indexing="ij")
    return NX * NX + NY * NY + NZ * NZ


def za_displacement(delta_k, n, box):
    """Psi_j(q) = IFFT[i k_j delta_k / k^2] on the lattice, shape (3, n, n, n) in Mpc/h."""
    kf = 2.0 * np.pi / box
    f = philox.signed_freqs(n).astype(np.float64)
    fz = np.arange(n // 2 + 1, dtype=np.float64)
    f_nyq0 = np.where(np.abs(f) == n // 2, 0.0, f)
    fz_nyq0 = np.where(fz == n // 2, 0.0, fz)
    NX, NY, NZ = np.meshgrid(f_nyq0, f_nyq0, fz_nyq0, indexing="ij")
    n2 = mode_n2(n).astype(np.float64)
    inv_k2 = np.zeros_like(n2)
    inv_k2[n2 > 0] = 1.0 / (kf * kf * n2[n2 > 0])
    psi = np.empty((3, n, n, n))
    for j, Nj in enumerate((NX, NY, NZ)):
        psi[j] = np.fft.irfftn(1j * kf * Nj * delta_k * inv_k2, s=(n, n, n), axes=(0, 1, 2))
    return psi


def za_displacement_at(cosmo, n, box, seed, ids, paired=False, fixed_amplitude=False):
    """Psi_j(q) at the lattice nodes of the given particle ids, shape (3, len(ids)) in Mpc/h.

    The same field as za_displacement(linear_delta_k(cosmo, n, box, seed)), evaluated by the
    direct sum over modes one x frequency at a time, so that memory stays at one plane of
    modes times the number of nodes (for full-size meshes).  The inverse transform of a
    Hermitian half spectrum is N^-3 sum over the half grid of w Re(Psi_n exp(2 pi i n.q / N))
    with w = 1 on the nz = 0 plane and 2 elsewhere (the nz = n/2 plane is zero here).
    """
    ids = np.asarray(ids, dtype=np.int64).ravel()
    q = np.stack([ids // (n * n), (ids // n) % n, ids % n])
    kf = 2.0 * np.pi / box
    f = philox.signed_freqs(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64)
    NY, NZ = np.meshgrid(f, fz, indexing="ij")
    w = np.where(NZ == 0, 1.0, 2.0)
    ey = np.exp(2j * np.pi * np.outer(f, q[1]) / n)    # (n, S)
    ez = np.exp(2j * np.pi * np.outer(fz, q[2]) / n)   # (n/2+1, S)
    dNY = np.where(np.abs(NY) == n // 2, 0, NY).astype(np.float64)
    dNZ = np.where(NZ == n // 2, 0, NZ).astype(np.float64)
    out = np.zeros((3, ids.size))
    for ix in range(n):
        nx = int(f[ix])
        g = philox.hermitian_noise_plane(seed, n, ix)
        if fixed_amplitude:
            g = fix_amplitude(g)
        if paired:
            g = -g
        n2 = nx * nx + NY * NY + NZ * NZ
        pos = n2 > 0
        pk = np.zeros(n2.shape)
        pk[pos] = cosmo.power_linear(kf * np.sqrt(n2[pos].astype(np.float64)))
        inv_k2 = np.zeros(n2.shape)
        inv_k2[pos] = 1.0 / (kf * kf * n2[pos])
        dk = n**3 * g * np.sqrt(pk / box**3)
        ex = np.exp(2j * np.pi * nx * q[0] / n)
        dnx = 0.0 if abs(nx) == n // 2 else float(nx)
        for j, Nj in enumerate((dnx, dNY, dNZ)):
            coef = 1j * kf * Nj * dk * inv_k2 * w
            out[j] += np.real(ex * np.sum((coef @ ez) * ey, axis=0))
    return out / n**3


def lpt2_displacement(delta_k, n, box):
    """Second-order Lagrangian displacement Psi2 (shape (3, n, n, n), Mpc/h) at D = 1.

    Bouchet et al. (1995), Scoccimarro (1998): with the first-order potential
    laplacian(phi1) = delta (so Psi1 = -grad phi1), the second-order potential solves
    laplacian(phi2) = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2), and Psi2 = grad phi2; the
    position is x = q + D Psi1 + D2 Psi2 with D2 < 0.  Derivatives are spectral on the
    n^3 lattice; the source is the product of the mesh fields (no de-aliasing); the zero
    mode and every mode with a Nyquist component of phi2 are dropped (as for Psi1).
    """
    kf = 2.0 * np.pi / box
    f = philox.signed_freqs(n).astype(np.float64)
    fz = np.arange(n // 2 + 1, dtype=np.float64)
    KX, KY, KZ = np.meshgrid(kf * f, kf * f, kf * fz, indexing="ij")
    K = (KX, KY, KZ)
    k2 = KX * KX + KY * KY + KZ * KZ
    inv_k2 = np.zeros_like(k2)
    inv_k2[k2 > 0] = 1.0 / k2[k2 > 0]
    phi1_k = -delta_k * inv_k2
    # phi1_ij = IFFT[(i k_i)(i k_j) phi1_k] = IFFT[-k_i k_j phi1_k]
    d2 = {}
    for i in range(3):
        for j in range(i, 3):
            d2[i, j] = np.fft.irfftn(-K[i] * K[j] * phi1_k, s=(n, n, n), axes=(0, 1, 2))
    src = (d2[0, 0] * d2[1, 1] - d2[0, 1]**2) + (d2[0, 0] * d2[2, 2] - d2[0, 2]**2) \
        + (d2[1, 1] * d2[2, 2] - d2[1, 2]**2)
    src_k = np.fft.rfftn(src)
    NX, NY, NZ = np.meshgrid(philox.signed_freqs(n), philox.signed_freqs(n), np.arange(n // 2 + 1), indexing="ij")
    nyq = (np.abs(NX) == n // 2) | (np.abs(NY) == n // 2) | (NZ == n // 2)
    phi2_k = np.where(nyq, 0.0, -src_k * inv_k2)
    return np.stack([np.fft.irfftn(1j * K[j] * phi2_k, s=(n, n, n), axes=(0, 1, 2)) for j in range(3)])


def lattice_ticks(n):
    """Lattice node coordinates in ticks, particle id = (ix n + iy) n + iz."""
    step = 2**32 // n
    i = np.arange(n, dtype=np.uint64) * np.uint64(step)
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()]).astype(np.uint32)


def zeldovich(cosmo, n, box, a_init, seed=None, white_noise=None, paired=False, fixed=True,
              fixed_amplitude=False, lpt_order=1):
    """Lagrangian ICs at a_init: returns (x, p) with x (3, n^3) ticks (fixed=True) or
    fractions, p (3, n^3); fixed_amplitude selects unit-modulus phases; lpt_order = 2
    adds D2 Psi2 to the positions and a^2 E f2 D2 Psi2 to the momenta."""
    dk = linear_delta_k(cosmo, n, box, seed=seed, white_noise=white_noise, paired=paired,
                        fixed_amplitude=fixed_amplitude)
    psi = za_displacement(dk, n, box).reshape(3, -1)
    D = cosmo.growth_D(a_init)
    f = cosmo.growth_f(a_init)
    E = float(cosmo.E(a_init))
    disp = D * psi
    p = a_init**2 * E * f * D * psi
    if lpt_order == 2:
        psi2 = lpt2_displacement(dk, n, box).reshape(3, -1)
        D2 = cosmo.growth_D2(a_init)
        disp = disp + D2 * psi2
        p = p + a_init**2 * E * cosmo.growth_f2(a_init) * D2 * psi2
    if fixed:
        q = lattice_ticks(n).astype(np.int64)
        x = ((q + np.rint(disp * (2.0**32 / box)).astype(np.int64)) % 2**32).astype(np.uint32)
    else:
        i = np.arange(n, dtype=np.float64) / n
        X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
        q = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
        x = q + disp / box
        x = x - np.floor(x)
    return x, p
