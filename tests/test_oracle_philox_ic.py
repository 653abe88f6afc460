"""Pins of the Philox phases and the Zel'dovich initial conditions."""
import os

import numpy as np
import pytest

from oracle import ic, philox
from oracle.cosmology import Cosmology

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")) if l.strip() and not l.startswith("#")]
    assert len(rows) == 3
    for r in rows:
        v = [int(t, 16) for t in r]
        out = philox.philox4x32_10(*[np.uint64(t) for t in v[:6]])
        assert [int(o) for o in out] == v[6:]


def test_gaussian_moments():
    n = np.arange(200_000)
    g = philox.unit_gaussian_modes(7, n % 97, n // 97, np.ones_like(n))
    se = 1.0 / np.sqrt(n.size)
    assert abs(g.real.mean()) < 5 * se and abs(g.imag.mean()) < 5 * se
    assert np.mean(np.abs(g)**2) == pytest.approx(1.0, abs=5 * se)
    assert np.var(g.real) == pytest.approx(0.5, abs=5 * se)
    # Box-Muller: |g|^2 is exponential with unit mean -> P(|g|^2 > 1) = e^-1
    assert np.mean(np.abs(g)**2 > 1.0) == pytest.approx(np.exp(-1.0), abs=5 * se)


@pytest.mark.parametrize("n", [8, 16])
def test_noise_is_hermitian(n):
    # A half-grid spectrum is the rfft of a real field iff it is Hermitian on the nz=0 plane:
    # the round trip irfftn -> rfftn must reproduce it exactly.
    g = philox.hermitian_noise_half(3, n)
    back = np.fft.rfftn(np.fft.irfftn(g, s=(n, n, n), axes=(0, 1, 2)))
    assert np.max(np.abs(back - g)) < 1e-12


def test_noise_shared_across_resolutions():
    g16 = philox.hermitian_noise_half(11, 16)
    g32 = philox.hermitian_noise_half(11, 32)
    f16 = philox.signed_freqs(16)
    for ix in range(16):
        for iy in range(16):
            nx, ny = f16[ix], f16[iy]
            if abs(nx) == 8 or abs(ny) == 8:
                continue
            np.testing.assert_array_equal(g16[ix, iy, :8], g32[nx % 32, ny % 32, :8])


def test_za_single_mode_displacement():
    # A single cosine in the white noise gives an analytic Zel'dovich displacement:
    # delta = eps cos(k x) -> Psi_x = -(eps/k) sin(k x), Psi_y = Psi_z = 0.
    n, box = 16, 100.0
    x = np.arange(n) / n
    eps = 0.01
    delta = eps * np.cos(2 * np.pi * 2 * x)[:, None, None] * np.ones((n, n, n))
    psi = ic.za_displacement(np.fft.rfftn(delta), n, box)
    k = 2 * np.pi * 2 / box
    expect = -(eps / k) * np.sin(2 * np.pi * 2 * x)[:, None, None] * np.ones((n, n, n))
    assert np.max(np.abs(psi[0] - expect)) < 1e-14 * box
    assert np.max(np.abs(psi[1])) < 1e-15 * box and np.max(np.abs(psi[2])) < 1e-15 * box


def test_za_divergence_is_minus_delta():
    # Linear continuity: div Psi = -delta (every non-Nyquist mode).
    n, box = 16, 500.0
    dk = ic.linear_delta_k(Cosmology(), n, box, seed=5)
    psi = ic.za_displacement(dk, n, box)
    kf = 2 * np.pi / box
    f = philox.signed_freqs(n)
    div = np.zeros_like(dk)
    for j, axis_f in enumerate((f[:, None, None], f[None, :, None], np.arange(n // 2 + 1)[None, None, :])):
        div = div + 1j * kf * axis_f * np.fft.rfftn(psi[j])
    assert np.max(np.abs(div + dk)) < 1e-10 * np.max(np.abs(dk))


def test_ic_spectrum_amplitude_exact():
    # |delta_n|^2 = N^6 |g_n|^2 P(k_n) / V mode by mode (Eq. powerspectrum normalisation).
    n, box, c = 16, 1000.0, Cosmology()
    dk = ic.linear_delta_k(c, n, box, seed=9)
    g = philox.hermitian_noise_half(9, n)
    n2 = ic.mode_n2(n)
    m = (n2 > 0) & (np.abs(g) > 0)
    P = c.power_linear(2 * np.pi / box * np.sqrt(n2[m]))
    np.testing.assert_allclose(np.abs(dk[m])**2, n**6 * np.abs(g[m])**2 * P / box**3, rtol=1e-12)


def test_zeldovich_particles_fixed_and_float_agree():
    c = Cosmology()
    xt, pt = ic.zeldovich(c, 8, 1000.0, 1 / 51, seed=2, fixed=True)
    xf, pf = ic.zeldovich(c, 8, 1000.0, 1 / 51, seed=2, fixed=False)
    np.testing.assert_array_equal(pt, pf)
    d = xt.astype(np.float64) / 2**32 - xf
    d -= np.rint(d)
    assert np.max(np.abs(d)) <= 2**-32
    assert abs(pt.mean()) < 1e-12 * np.abs(pt).max()


def test_plane_noise_and_direct_mode_sum_match_the_full_grid():
    # the one-plane-at-a-time forms used for full-size meshes against the full-grid FFT forms
    c = Cosmology()
    for n, box, seed in ((16, 300.0, 7), (32, 700.0, 11)):
        g = philox.hermitian_noise_half(seed, n)
        for i in range(n):
            assert np.array_equal(philox.hermitian_noise_plane(seed, n, i), g[i])
        psi = ic.za_displacement(ic.linear_delta_k(c, n, box, seed=seed), n, box).reshape(3, -1)
        ids = np.array([0, 1, n * n * 3 + n * 5 + 7, n**3 - 1, 977 % n**3])
        got = ic.za_displacement_at(c, n, box, seed, ids)
        assert np.max(np.abs(got - psi[:, ids])) < 1e-12 * np.max(np.abs(psi))
    # paired phases flip the sign
    assert np.allclose(ic.za_displacement_at(c, 16, 300.0, 7, [5], paired=True),
                       -ic.za_displacement_at(c, 16, 300.0, 7, [5]), rtol=0, atol=0)


def _bin_mean_linear_power(c, n, box, edges):
    """Per bin, the mean of P_lin(k_n) over every full-grid wavevector n (components in
    [-n/2, n/2), |n| <= n/2, n != 0) of the bin, counting the modes with a Nyquist
    component (which carry no phase) as zero power: brute force over the whole grid."""
    f = np.arange(-(n // 2), n // 2)
    NX, NY, NZ = np.meshgrid(f, f, f, indexing="ij")
    n2 = (NX * NX + NY * NY + NZ * NZ).ravel()
    nyq = ((NX == -(n // 2)) | (NY == -(n // 2)) | (NZ == -(n // 2))).ravel()
    kf = 2 * np.pi / box
    nb = len(edges) - 1
    num, den = np.zeros(nb), np.zeros(nb)
    for m2, q in zip(n2, nyq):
        if m2 == 0 or m2 > (n // 2)**2:
            continue
        kn = np.sqrt(float(m2))
        b = int(np.searchsorted(edges, kn, side="right")) - 1
        if kn == edges[-1]:
            b = nb - 1
        if not 0 <= b < nb:
            continue
        den[b] += 1.0
        if not q:
            num[b] += c.power_linear(kf * kn)
    return num / den


def test_paired_phases_invert_the_linear_field():
    # the pairing method (Sec. 4.2): the partner run starts from the same field with every phase
    # shifted by pi, i.e. delta -> -delta (and the Zel'dovich displacements change sign)
    c = Cosmology()
    d = ic.linear_delta_k(c, 16, 500.0, seed=4)
    dp = ic.linear_delta_k(c, 16, 500.0, seed=4, paired=True)
    np.testing.assert_array_equal(dp, -d)
    df = ic.linear_delta_k(c, 16, 500.0, seed=4, fixed_amplitude=True)
    dfp = ic.linear_delta_k(c, 16, 500.0, seed=4, fixed_amplitude=True, paired=True)
    np.testing.assert_array_equal(dfp, -df)


def test_fixed_amplitude_ic_has_the_input_spectrum_exactly():
    # Fixed amplitudes (|g_n| = 1): the measured P(k) of the linear field equals the bin
    # mean of the input spectrum with no cosmic variance; Gaussian amplitudes scatter.
    from oracle import stats
    n, box, c = 16, 800.0, Cosmology()
    # edges between integer |n|^2 (no mode on an inner edge), the last one at n/2, closed
    edges = np.sqrt([0.5, 2.5, 6.5, 12.5, 24.5, 40.5, 64.0])
    want = _bin_mean_linear_power(c, n, box, edges)
    for seed in (3, 4):
        for paired in (False, True):
            dk = ic.linear_delta_k(c, n, box, seed=seed, paired=paired, fixed_amplitude=True)
            delta = np.fft.irfftn(dk, s=(n, n, n), axes=(0, 1, 2))
            _, pk, _ = stats.power_spectrum(delta, box, edges, deconvolve=False)
            np.testing.assert_allclose(pk, want, rtol=1e-12)
    dk = ic.linear_delta_k(c, n, box, seed=3)
    _, pk, _ = stats.power_spectrum(np.fft.irfftn(dk, s=(n, n, n), axes=(0, 1, 2)), box, edges, deconvolve=False)
    assert np.max(np.abs(pk / want - 1.0)) > 1e-2


def test_fixed_amplitude_keeps_phases_and_hermitian_symmetry():
    n = 16
    g = philox.hermitian_noise_half(5, n)
    gf = ic.fix_amplitude(g)
    live = np.abs(g) > 0
    assert np.max(np.abs(np.abs(gf[live]) - 1.0)) < 1e-15
    assert np.array_equal(gf[~live], g[~live])
    # same phase: g_fixed * |g| reproduces g
    assert np.max(np.abs(gf * np.abs(g) - g)) < 1e-15 * np.max(np.abs(g))
    back = np.fft.rfftn(np.fft.irfftn(gf, s=(n, n, n), axes=(0, 1, 2)))
    assert np.max(np.abs(back - gf)) < 1e-12
    # the one-plane form for full-size meshes agrees with the full grid
    c = Cosmology()
    psi = ic.za_displacement(ic.linear_delta_k(c, n, 300.0, seed=5, fixed_amplitude=True), n, 300.0).reshape(3, -1)
    ids = np.array([0, 7, n**3 - 1, 1234])
    got = ic.za_displacement_at(c, n, 300.0, 5, ids, fixed_amplitude=True)
    assert np.max(np.abs(got - psi[:, ids])) < 1e-12 * np.max(np.abs(psi))
