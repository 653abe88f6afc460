"""Pins of the P(k) / B(k) estimators, the bias fit and the displacement combination."""
import itertools

import numpy as np
import pytest

import inputs
from oracle import combine, stats


def _full_dft(delta):
    """Direct O(N^6) DFT: delta_n = sum_x delta(x) exp(-2 pi i n.x / N), full grid, signed n."""
    n = delta.shape[0]
    f = np.fft.fftfreq(n, 1.0 / n).round().astype(int)
    g = np.arange(n)
    E = np.exp(-2j * np.pi * np.outer(f, g) / n)  # (n_freq, n_pos)
    return np.einsum("ax,by,cz,xyz->abc", E, E, E, delta), f


def test_power_spectrum_against_direct_dft():
    n, box = 8, 250.0
    delta = inputs.lognormal_field(21, n)
    dk, f = _full_dft(delta)
    NX, NY, NZ = np.meshgrid(f, f, f, indexing="ij")
    n2 = NX**2 + NY**2 + NZ**2
    edges = np.array([0.5, 1.7, 2.5, 3.3, 4.0])
    for deconv in (False, True):
        W = (np.sinc(NX / n) * np.sinc(NY / n) * np.sinc(NZ / n))**2 if deconv else 1.0
        kk, pk, nm = stats.power_spectrum(delta, box, edges, deconvolve=deconv)
        for b in range(4):
            m = (n2 >= edges[b]**2) & ((n2 < edges[b + 1]**2) | ((b == 3) & (n2 == edges[-1]**2))) \
                & (n2 > 0) & (n2 <= (n // 2)**2)
            assert nm[b] == m.sum()
            want = box**3 / n**6 * np.mean(np.abs(dk[m] / (W[m] if deconv else 1.0))**2)
            assert pk[b] == pytest.approx(want, rel=1e-12)
            assert kk[b] == pytest.approx(2 * np.pi / box * np.mean(np.sqrt(n2[m])), rel=1e-12)


def test_single_cosine_power():
    # delta = A cos(2 pi n.x/N): the two modes +-n carry |delta_n|^2 = A^2 N^6/4 each,
    # so sum_b P_b n_b = 2 * V A^2 / 4 (deconvolution off).
    n, box, A = 16, 100.0, 0.3
    g = np.arange(n)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    delta = A * np.cos(2 * np.pi * (3 * X - 2 * Y + 1 * Z) / n)
    edges = stats.log_edges(6, 1.0, 8.0)
    _, pk, nm = stats.power_spectrum(delta, box, edges, deconvolve=False)
    tot = np.nansum(pk * nm)
    assert tot == pytest.approx(2 * box**3 * A * A / 4, rel=1e-12)
    assert np.count_nonzero(np.nan_to_num(pk) > 1e-20) == 1


def _cic_window(n, nvec):
    """Prod_j [sin(pi n_j / N) / (pi n_j / N)]^2: the Fourier transform of the CIC kernel."""
    w = 1.0
    for nj in nvec:
        x = np.pi * nj / n
        w *= 1.0 if nj == 0 else (np.sin(x) / x)**2
    return w


def _brute_bispectrum(delta, box, edges, deconvolve=False):
    n = delta.shape[0]
    dk, f = _full_dft(delta)
    NX, NY, NZ = np.meshgrid(f, f, f, indexing="ij")
    if deconvolve:
        for i in np.ndindex(dk.shape):
            dk[i] /= _cic_window(n, (NX[i], NY[i], NZ[i]))
    n2 = NX**2 + NY**2 + NZ**2
    b = stats.assign_bins(n2, edges)
    nyq = (np.abs(NX) == n // 2) | (np.abs(NY) == n // 2) | (np.abs(NZ) == n // 2)
    b = np.where((n2 > 0) & (n2 <= (n // 2)**2) & ~nyq, b, -1)
    modes = [(int(NX[i]), int(NY[i]), int(NZ[i]), int(b[i]), dk[i]) for i in zip(*np.nonzero(b >= 0))]
    lookup = {(m[0], m[1], m[2]): (m[3], m[4]) for m in modes}
    nb = len(edges) - 1
    S = np.zeros((nb, nb, nb), dtype=complex)
    C = np.zeros((nb, nb, nb))
    for m1, m2 in itertools.product(modes, modes):
        k3 = (-m1[0] - m2[0], -m1[1] - m2[1], -m1[2] - m2[2])
        if k3 not in lookup:
            continue
        b3, d3 = lookup[k3]
        S[m1[3], m2[3], b3] += m1[4] * m2[4] * d3
        C[m1[3], m2[3], b3] += 1
    return S, C


@pytest.mark.parametrize("deconvolve,top", [(False, 3.5), (True, 3.5), (False, 4.0)])
def test_bispectrum_against_brute_force_triplets(deconvolve, top):
    # each mode divided by its own CIC window W(n) before the triplet product when deconvolving;
    # top = 4.0 closes the last bin at the 8^3 Nyquist frequency, so modes with a Nyquist
    # component (|n_j| = 4, no distinct partner at -n) fall in it and must be left out
    n, box = 8, 300.0
    delta = inputs.lognormal_field(22, n, sigma=0.8)
    edges = np.array([0.5, 1.5, 2.5, top])
    tri, B, ntri = stats.bispectrum(delta, box, edges, deconvolve=deconvolve)
    S, C = _brute_bispectrum(delta, box, edges, deconvolve)
    for (i, j, l), bval, nt in zip(tri, B, ntri):
        assert nt == C[i, j, l]
        if nt > 0:
            assert abs(S[i, j, l].imag) < 1e-9 * abs(S[i, j, l])
            assert bval == pytest.approx(box**6 / n**9 * S[i, j, l].real / nt, rel=1e-10)
        else:
            assert np.isnan(bval)


def test_bispectrum_triple_cosine():
    # delta = A sum_a cos(2 pi n_a.x/N) with n1+n2+n3 = 0 in three distinct bins:
    # B_123 = V^2 A^3 / (4 N_123) (deconvolution off).
    n, box, A = 16, 200.0, 0.1
    g = np.arange(n)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    n1, n2v = np.array([1, 0, 0]), np.array([0, 2, 0])
    n3 = -(n1 + n2v)
    delta = sum(A * np.cos(2 * np.pi * (v[0] * X + v[1] * Y + v[2] * Z) / n) for v in (n1, n2v, n3))
    edges = np.array([0.5, 1.5, 2.1, 2.5])  # |n1| = 1, |n2| = 2, |n3| = sqrt 5
    tri, B, ntri = stats.bispectrum(delta, box, edges, deconvolve=False)
    q = [t for t in range(len(tri)) if tuple(tri[t]) == (0, 1, 2)][0]
    assert B[q] == pytest.approx(box**6 * A**3 / (4 * ntri[q]), rel=1e-10)


def test_bias_fit_recovers_exact_coefficients():
    k = np.linspace(0.002, 0.05, 30)
    w = np.arange(30) + 5.0
    H = 3.3e-4
    ratio = 2.5 + (-7.0) * H**2 / k**2
    b1, bgr = stats.fit_linear_bias(k, ratio, w, 0.02, calH=H)
    assert b1 == pytest.approx(2.5, rel=1e-10) and bgr == pytest.approx(-7.0, rel=1e-8)
    # delta_h = b delta_m exactly -> P_hm / P_mm = b
    d = inputs.gaussian_field(23, 16)
    edges = stats.log_edges(8, 1.0, 8.0)
    kk, phm, nm = stats.power_spectrum(2.7 * d, 1000.0, edges, delta2=d)
    _, pmm, _ = stats.power_spectrum(d, 1000.0, edges)
    (b,) = stats.fit_linear_bias(kk, phm / pmm, nm, 1.0)
    assert b == pytest.approx(2.7, rel=1e-12)


def test_cross_spectrum_is_the_real_part():
    # Eq. powerspectrum for two fields: Re <delta_1 delta_2*>, so delta against -delta gives -P
    d = inputs.gaussian_field(25, 16)
    edges = stats.log_edges(6, 1.0, 8.0)
    _, p, _ = stats.power_spectrum(d, 500.0, edges)
    _, px, _ = stats.power_spectrum(d, 500.0, edges, delta2=-d)
    np.testing.assert_allclose(px, -p, rtol=1e-14)


def test_bias_fit_weights_modes_and_cuts_at_k_max():
    # Eq. b1 fitted by least squares weighted with the mode counts on k < k_max: a constant
    # fit is the mode-weighted mean of the ratios of the bins below k_max
    k = np.array([0.01, 0.02, 0.04])
    ratio = np.array([1.0, 3.0, 50.0])
    w = np.array([3.0, 1.0, 100.0])
    (b,) = stats.fit_linear_bias(k, ratio, w, 0.03)
    assert b == pytest.approx((3.0 * 1.0 + 1.0 * 3.0) / 4.0, rel=1e-14)


def test_halo_proxy_contrast_values():
    # delta_h = n_h / mean(n_h) - 1 of the indicator of the selected cells: 1/f' - 1 on the
    # selected cells (f' the selected fraction) and -1 elsewhere, zero mean
    d = inputs.gaussian_field(24, 4)
    dh = stats.halo_proxy_contrast(d, 0.05)  # ceil(3.2) = 4 of 64 cells
    sel = stats.top_fraction_mask(d, 0.05)
    assert np.all(dh[sel] == 15.0) and np.all(dh[~sel] == -1.0)
    assert abs(dh.mean()) < 1e-15


def test_top_fraction_mask_count_and_ties():
    d = np.zeros((4, 4, 4))
    d.ravel()[[5, 9, 40]] = 3.0
    d.ravel()[[1, 2, 3, 60]] = 1.0
    m = stats.top_fraction_mask(d, 0.05)  # ceil(3.2) = 4 cells
    assert m.sum() == 4
    assert set(np.flatnonzero(m.ravel())) == {5, 9, 40, 1}


def test_displacement_identity_and_min_image():
    x = inputs.uniform_ticks(24, 1000)
    assert np.all(combine.displacement(x, x) == 0)
    np.testing.assert_array_equal(combine.combine(x, np.zeros((3, 1000), np.int32)), x)
    d = inputs.rng(25).integers(-2**30, 2**30, size=(3, 1000)).astype(np.int64)
    y = ((x.astype(np.int64) + d) % 2**32).astype(np.uint32)
    np.testing.assert_array_equal(combine.displacement(y, x), d)
    xf = inputs.ticks_to_fractions(x)
    yf = inputs.ticks_to_fractions(y)
    np.testing.assert_allclose(combine.displacement(yf, xf), d / 2.0**32, atol=1e-15)


def test_lagrangian_interpolation_reproduces_constant_and_linear():
    nc, nt = 4, 8
    const = np.full((3, nc**3), 123456, dtype=np.int32)
    np.testing.assert_array_equal(combine.interpolate_lagrangian(const, nc, nt), np.full((3, nt**3), 123456))
    # a field linear in the coarse x index (away from the periodic seam) is interpolated exactly
    i = np.arange(nc)
    lin = np.broadcast_to((1000 * i)[:, None, None], (nc, nc, nc)).ravel()
    xi = np.stack([lin, lin, lin]).astype(np.int32)
    out = combine.interpolate_lagrangian(xi, nc, nt).reshape(3, nt, nt, nt)
    it = np.arange(nt - 2)
    np.testing.assert_array_equal(out[0, :nt - 2, 0, 0], 500 * it)
    # same lattice: identity
    np.testing.assert_array_equal(combine.interpolate_lagrangian(xi, nc, nc), xi)
    # FP64 form agrees with the tick form up to rounding
    outf = combine.interpolate_lagrangian(xi.astype(np.float64) * 2.0**-32, nc, nt)
    assert np.max(np.abs(outf * 2**32 - out.reshape(3, -1))) <= 0.5
    # a target halfway between two coarse nodes gets their mean; on ticks a tie rounds half to
    # even (the reading both sides share): 0 and 1 -> 0, 1 and 2 -> 2, -1 and 0 -> 0, 3 and 4 -> 4
    for lo, hi, want in ((0, 1, 0), (1, 2, 2), (-1, 0, 0), (3, 4, 4), (5, 6, 6)):
        v = np.where(np.arange(nc) % 2 == 0, lo, hi)
        f = np.broadcast_to(v[:, None, None], (nc, nc, nc)).ravel()
        t = combine.interpolate_lagrangian(np.stack([f, f, f]).astype(np.int32), nc, nt).reshape(3, nt, nt, nt)
        assert t[0, 1, 0, 0] == want, (lo, hi, t[0, 1, 0, 0])
