"""Philox4x32-10 and the per-wavevector Gaussian phases of the initial conditions.

Oracle (test infrastructure only).

The paper runs its three simulations from "the same initial random perturbation
phases" (Sec. 2, Sec. 3) but does not say how they are drawn (MonofonIC does it
in the paper).  Reading used here: each Fourier mode n = (nx, ny, nz) of the
half grid draws one unit complex Gaussian g_n from Philox4x32-10 (Salmon, Moraes,
Dror & Shaw, SC'11, "Parallel random numbers: as easy as 1, 2, 3") with
key = (seed mod 2^32, seed div 2^32) and counter = (nx, ny, nz, 0) as 32-bit
two's-complement words, followed by a Box-Muller transform in FP64.  The draw
depends on n and the seed only, so two resolutions share their common modes.
"""
import numpy as np

_MASK = np.uint64(0xFFFFFFFF)
_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = np.uint64(0x9E3779B9)
_W1 = np.uint64(0xBB67AE85)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Ten Philox-4x32 rounds (Salmon et al. 2011, Sec. 4.2).

    Each round multiplies words 0 and 2 by the two Philox multipliers, takes the
    high and low halves of the 64-bit products, xors the high halves with the
    other counter words and the key, and permutes; the key is bumped by the two
    Weyl constants between rounds.  All arguments are uint32-valued arrays.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for r in range(10):
        if r > 0:
            k0 = (k0 + _W0) & _MASK
            k1 = (k1 + _W1) & _MASK
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> np.uint64(32), p0 & _MASK
        hi1, lo1 = p1 >> np.uint64(32), p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
    return (c0.astype(np.uint32), c1.astype(np.uint32),
            c2.astype(np.uint32), c3.astype(np.uint32))


def unit_gaussian_modes(seed, nx, ny, nz):
    """Unit complex Gaussian g_n (E|g|^2 = 1) for integer wavevectors (nx, ny, nz).

    Box-Muller in FP64 on the first two Philox words:
    u = (r + 1/2) 2^-32, |g| = sqrt(-ln u1), arg g = 2 pi u2.
    """
    seed = int(seed)
    to_u32 = lambda v: (np.asarray(v, dtype=np.int64) & 0xFFFFFFFF).astype(np.uint64)
    r0, r1, _, _ = philox4x32_10(to_u32(nx), to_u32(ny), to_u32(nz), np.zeros_like(to_u32(nx)),
                                 np.uint64(seed & 0xFFFFFFFF), np.uint64((seed >> 32) & 0xFFFFFFFF))
    u1 = (r0.astype(np.float64) + 0.5) * 2.0**-32
    u2 = (r1.astype(np.float64) + 0.5) * 2.0**-32
    amp = np.sqrt(-np.log(u1))
    return amp * np.cos(2.0 * np.pi * u2) + 1j * amp * np.sin(2.0 * np.pi * u2)


def signed_freqs(n):
    """Integer wavenumbers in FFT order: 0..n/2-1, -n/2..-1."""
    return np.fft.fftfreq(n, d=1.0 / n).round().astype(np.int64)


def _hermitian_noise(seed, n, NX, NY, NZ):
    """g_n on the given integer wavevectors (nz >= 0) with the rule of hermitian_noise_half."""
    canonical = (NZ > 0) | ((NZ == 0) & ((NY > 0) | ((NY == 0) & (NX > 0))))
    cx = np.where(canonical, NX, -NX)
    cy = np.where(canonical, NY, -NY)
    g = unit_gaussian_modes(seed, cx, cy, NZ)
    g = np.where(canonical, g, np.conj(g))
    zero = (np.abs(NX) == n // 2) | (np.abs(NY) == n // 2) | (NZ == n // 2) | ((NX == 0) & (NY == 0) & (NZ == 0))
    return np.where(zero, 0.0, g)


def hermitian_noise_half(seed, n):
    """g_n on the rfftn half grid (n, n, n/2+1), Hermitian on the nz = 0 plane.

    Canonical modes (nz > 0, or nz = 0 with ny > 0, or nz = 0, ny = 0, nx > 0) draw
    their own g_n; the remaining nz = 0 modes are the complex conjugates of their
    partners at -n.  The zero mode and every mode with a Nyquist component
    (|n_i| = n/2) are set to zero (reading: keeps the field and the Zel'dovich
    displacement real without special cases).
    """
    f = signed_freqs(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64)
    NX, NY, NZ = np.meshgrid(f, f, fz, indexing="ij")
    return _hermitian_noise(seed, n, NX, NY, NZ)


def hermitian_noise_plane(seed, n, ix):
    """hermitian_noise_half(seed, n)[ix]: the (ny, nz) plane of one x frequency."""
    f = signed_freqs(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64)
    NY, NZ = np.meshgrid(f, fz, indexing="ij")
    return _hermitian_noise(seed, n, np.full_like(NY, f[ix]), NY, NZ)
