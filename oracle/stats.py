"""Power spectrum, bispectrum and halo-proxy linear bias.

Oracle (test infrastructure only).

Conventions: delta_n = sum_x delta(x) exp(-2 pi i n.x/N) (unnormalised DFT) and the
continuous transform is (V/N^3) delta_n, so

* Eq. powerspectrum, <delta(k1) delta(k2)> = (2pi)^3 delta_D P(k1):
  P_b = (V/N^6) sum_{n in b} w_n |delta_n / W(n)|^2 / sum_{n in b} w_n,
  averaged over the full sphere of modes (w_n = 1 on the nz = 0 and nz = N/2
  planes of the half grid, 2 elsewhere);
* Eq. bispectre, <delta(k1) delta(k2) delta(k3)> = (2pi)^3 delta_D B:
  B_ijl = (V^2/N^9) sum_{n1+n2+n3=0, n_a in bins i,j,l} delta_n1 delta_n2 delta_n3 / N_ijl.

W(n) = prod_j sinc^2(pi n_j / N) is the CIC window (deconvolution on by default,
as in Pylians3, Sec. 4).  Bins are given by edges e_0 < ... < e_B in units of the
fundamental mode k_f = 2 pi / L; a mode belongs to bin b when
e_b^2 <= |n|^2 < e_{b+1}^2 (the last bin is closed), which both sides decide on
the exact integer |n|^2.  The zero mode and modes with |n| > N/2 are excluded;
the bispectrum also leaves out modes with a Nyquist component (reading).
"""
import math

import numpy as np

from . import philox


def cic_window_half(n):
    f = philox.signed_freqs(n).astype(np.float64)
    fz = np.arange(n // 2 + 1, dtype=np.float64)
    wx = np.sinc(f / n)**2
    wz = np.sinc(fz / n)**2
    return wx[:, None, None] * wx[None, :, None] * wz[None, None, :]


def _half_grid(n):
    f = philox.signed_freqs(n)
    fz = np.arange(n // 2 + 1, dtype=np.int64)
    NX, NY, NZ = np.meshgrid(f, f, fz, indexing="ij")
    n2 = NX * NX + NY * NY + NZ * NZ
    w = np.full(n2.shape, 2.0)
    w[:, :, 0] = 1.0
    w[:, :, n // 2] = 1.0
    return n2, w


def assign_bins(n2, edges):
    """Bin index of each |n|^2 (or -1): e_b^2 <= n2 < e_{b+1}^2, last bin closed."""
    e2 = np.asarray(edges, dtype=np.float64)**2
    b = np.searchsorted(e2, n2.astype(np.float64), side="right") - 1
    b = np.where(n2.astype(np.float64) == e2[-1], len(e2) - 2, b)
    return np.where((b >= 0) & (b < len(e2) - 1), b, -1)


def power_spectrum(delta, box, edges, deconvolve=True, delta2=None):
    """Binned auto (or cross, with delta2) power spectrum of mesh fields.

    Returns (k_mean [h/Mpc], P [(Mpc/h)^3], n_modes).  Eq. powerspectrum.
    """
    n = delta.shape[0]
    d1 = np.fft.rfftn(delta)
    d2 = d1 if delta2 is None else np.fft.rfftn(delta2)
    if deconvolve:
        W = cic_window_half(n)
        d1 = d1 / W
        d2 = d2 / W
    n2, w = _half_grid(n)
    b = assign_bins(n2, edges)
    b = np.where((n2 > 0) & (n2 <= (n // 2)**2), b, -1)
    sel = b >= 0
    nb = len(edges) - 1
    kf = 2.0 * np.pi / box
    power = np.real(d1 * np.conj(d2))
    wsum = np.bincount(b[sel], weights=w[sel], minlength=nb)
    psum = np.bincount(b[sel], weights=(w * power)[sel], minlength=nb)
    ksum = np.bincount(b[sel], weights=(w * kf * np.sqrt(n2))[sel], minlength=nb)
    with np.errstate(invalid="ignore", divide="ignore"):
        pk = box**3 / n**6 * psum / wsum
        kk = ksum / wsum
    return kk, pk, wsum


def log_edges(nbins, k_min_over_kf, k_max_over_kf):
    """Logarithmic edges in units of k_f."""
    return k_min_over_kf * (k_max_over_kf / k_min_over_kf)**(np.arange(nbins + 1) / nbins)


def triangles(nbins):
    """All bin triplets i <= j <= l in lexicographic order."""
    return [(i, j, l) for i in range(nbins) for j in range(i, nbins) for l in range(j, nbins)]


def bispectrum(delta, box, edges, M=None, deconvolve=True):
    """FFT bispectrum estimator for all triangles i <= j <= l (Eq. bispectre).

    sum_{n1+n2+n3=0} prod_a delta_{n_a} = M^-3 sum_x I_i I_j I_l with
    I_b(x) = sum_{n in b} delta_n exp(2 pi i n.x/M), exact (no aliasing) on any grid
    M > 3 max |n_a|_inf; the triangle count N_ijl is the same sum with delta -> 1.
    Returns (tri (T, 3) int, B [(Mpc/h)^6], N_tri).
    """
    n = delta.shape[0]
    dk = np.fft.fftn(delta)
    f = philox.signed_freqs(n)
    NX, NY, NZ = np.meshgrid(f, f, f, indexing="ij")
    if deconvolve:
        W = (np.sinc(NX / n) * np.sinc(NY / n) * np.sinc(NZ / n))**2
        dk = dk / W
    n2 = NX * NX + NY * NY + NZ * NZ
    b = assign_bins(n2, edges)
    # modes with a Nyquist component have no distinct partner at -n; they are left
    # out of every triangle so that each I_b stays a real field
    nyq = (np.abs(NX) == n // 2) | (np.abs(NY) == n // 2) | (np.abs(NZ) == n // 2)
    b = np.where((n2 > 0) & (n2 <= (n // 2)**2) & ~nyq, b, -1)
    nb = len(edges) - 1
    inbin = b >= 0
    nmax = int(max(np.abs(NX[inbin]).max(), np.abs(NY[inbin]).max(), np.abs(NZ[inbin]).max()))
    if M is None:
        M = 1
        while M < 3 * nmax + 1:
            M *= 2
    if M < 3 * nmax + 1:
        raise ValueError("grid too small for an alias-free triangle sum")
    I = np.zeros((nb, M**3))
    C = np.zeros((nb, M**3))
    for bb in range(nb):
        m = b == bb
        grid = np.zeros((M, M, M), dtype=np.complex128)
        grid[NX[m] % M, NY[m] % M, NZ[m] % M] = dk[m]
        I[bb] = np.real(np.fft.ifftn(grid)).ravel() * M**3
        grid[:] = 0.0
        grid[NX[m] % M, NY[m] % M, NZ[m] % M] = 1.0
        C[bb] = np.real(np.fft.ifftn(grid)).ravel() * M**3
    tri = np.array(triangles(nb), dtype=np.int64).reshape(-1, 3)
    S = np.zeros(len(tri))
    T = np.zeros(len(tri))
    pos = {tuple(t): q for q, t in enumerate(tri)}
    for i in range(nb):
        for j in range(i, nb):
            s_ij = I[j:] @ (I[i] * I[j])
            c_ij = C[j:] @ (C[i] * C[j])
            for off, l in enumerate(range(j, nb)):
                q = pos[(i, j, l)]
                S[q] = s_ij[off]
                T[q] = c_ij[off]
    ntri = np.rint(T / M**3)
    with np.errstate(invalid="ignore", divide="ignore"):
        B = (box**3)**2 / float(n)**9 * S / T
    B = np.where(ntri > 0, B, np.nan)
    return tri, B, ntri


def top_fraction_mask(delta, fraction=0.05):
    """Halo proxy: the ceil(fraction N^3) densest cells, ties by lower linear index."""
    v = np.asarray(delta).ravel()
    count = int(math.ceil(fraction * v.size))
    order = np.lexsort((np.arange(v.size), -v))
    mask = np.zeros(v.size, dtype=bool)
    mask[order[:count]] = True
    return mask.reshape(delta.shape)


def halo_proxy_contrast(delta, fraction=0.05):
    """delta_h = n_h / mean(n_h) - 1 with n_h the indicator of the selected cells."""
    m = top_fraction_mask(delta, fraction).astype(np.float64)
    return m / m.mean() - 1.0


def fit_linear_bias(k, ratio, weights, k_max, calH=None, with_k2=False):
    """Weighted least squares of P_hm/P_mm = b1 [+ b1GR calH^2/k^2] [+ c k^2] on k < k_max.

    Eq. b1 (Sec. 5.2); weights are mode counts.  Returns the coefficient vector.
    """
    k = np.asarray(k, dtype=np.float64)
    sel = (k < k_max) & (weights > 0) & np.isfinite(ratio)
    cols = [np.ones(sel.sum())]
    if calH is not None:
        cols.append(calH**2 / k[sel]**2)
    if with_k2:
        cols.append(k[sel]**2)
    A = np.stack(cols, axis=1)
    sw = np.sqrt(weights[sel])
    coef, *_ = np.linalg.lstsq(A * sw[:, None], ratio[sel] * sw, rcond=None)
    return coef


def b1_gr_theory(b1, f, omega_m_a):
    """Eq. bgr: b1^GR = 3 (f + (3/2) Omega_m(z)) (1 - b1)."""
    return 3.0 * (f + 1.5 * omega_m_a) * (1.0 - b1)
