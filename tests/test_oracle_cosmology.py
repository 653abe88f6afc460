"""Pins of the FP64 background / growth / leapfrog factors / linear spectrum oracle."""
import math
import os

import numpy as np
import pytest
from scipy import integrate

from oracle.cosmology import Cosmology
from oracle.stats import b1_gr_theory

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_einstein_de_sitter_growth_is_a():
    # Omega_m = 1: D(a) = a exactly and f = 1 (textbook EdS limit).
    c = Cosmology(omega_m=1.0)
    for a in (0.02, 0.1, 0.5, 0.9):
        assert c.growth_D(a) == pytest.approx(a, rel=1e-10)
        assert c.growth_f(a) == pytest.approx(1.0, rel=1e-10)


def test_einstein_de_sitter_kick_and_drift_closed_forms():
    # E = a^-3/2: int da/(a^2 E) = 2(sqrt a1 - sqrt a0); int da/(a^3 E) = 2(a0^-1/2 - a1^-1/2).
    c = Cosmology(omega_m=1.0)
    a0, a1 = 0.13, 0.57
    assert c.kick_factor(a0, a1) == pytest.approx(2 * (math.sqrt(a1) - math.sqrt(a0)), rel=1e-12)
    assert c.drift_factor(a0, a1) == pytest.approx(2 * (a0**-0.5 - a1**-0.5), rel=1e-12)


def test_lcdm_growth_matches_growth_ode():
    # Independent route: integrate D'' + (3/a + dlnE/da) D' - 3/2 Om a^-5 E^-2 D = 0
    # from deep matter domination (D = a) and normalise at a = 1.
    c = Cosmology(omega_m=0.31)

    def rhs(a, y):
        D, dD = y
        E = float(c.E(a))
        dlnE = -1.5 * c.omega_m / a**4 / E**2
        return [dD, -(3.0 / a + dlnE) * dD + 1.5 * c.omega_m / (a**5 * E**2) * D]

    a_eval = [0.02, 0.1, 0.3, 0.6, 1.0]
    sol = integrate.solve_ivp(rhs, (1e-4, 1.0), [1e-4, 1.0], t_eval=a_eval, rtol=1e-12, atol=1e-16,
                              method="DOP853")
    D_ode = sol.y[0] / sol.y[0][-1]
    f_ode = sol.y[1] * np.array(a_eval) / sol.y[0]
    for a, d, f in zip(a_eval, D_ode, f_ode):
        assert c.growth_D(a) == pytest.approx(d, rel=2e-7)
        assert c.growth_f(a) == pytest.approx(f, rel=2e-7)


def test_tophat_window_is_fourier_transform_of_ball():
    # W(kR) = (3/R^3) int_0^R r^2 sin(kr)/(kr) dr, evaluated by direct quadrature.
    R = 8.0
    for k in (0.01, 0.3, 1.7):
        direct, _ = integrate.quad(lambda r: r * r * math.sin(k * r) / (k * r), 0.0, R, epsrel=1e-12)
        assert Cosmology.tophat_window(k * R) == pytest.approx(3.0 * direct / R**3, rel=1e-9, abs=1e-12)


def test_tophat_window_near_zero_against_extended_precision():
    # the small-x branch (a series) against 3 (sin x - x cos x) / x^3 evaluated in 50-digit
    # arithmetic, on both sides of the switch to the closed form; in FP64 the closed form
    # loses digits to cancellation just above the switch (sin x - x cos x ~ x^3 / 3: about
    # 3e-10 at x = 1e-3), the series is exact to rounding below it
    mpmath = pytest.importorskip("mpmath")
    mpmath.mp.dps = 50
    for x, tol in ((1e-5, 1e-14), (5e-4, 1e-14), (9.99e-4, 1e-14), (1.001e-3, 1e-9), (3e-3, 1e-9)):
        xm = mpmath.mpf(x)
        exact = float(3 * (mpmath.sin(xm) - xm * mpmath.cos(xm)) / xm**3)
        assert float(Cosmology.tophat_window(x)) == pytest.approx(exact, rel=0, abs=tol)


def test_transfer_function_limits_and_bbks_shape():
    c = Cosmology()
    assert c.transfer_eh_nowiggle(1e-6) == pytest.approx(1.0, abs=1e-4)
    k = np.logspace(-3, 0, 40)
    T = c.transfer_eh_nowiggle(k)
    assert np.all(np.diff(T) < 0)
    # BBKS (Bardeen et al. 1986) with the Sugiyama (1995) shape parameter: an independent
    # fit of the same physics; the two agree to within ~5% over these scales.
    gam = c.omega_m * c.h * math.exp(-c.omega_b * (1 + math.sqrt(2 * c.h) / c.omega_m))
    q = k / gam
    bbks = np.log(1 + 2.34 * q) / (2.34 * q) * (1 + 3.89 * q + (16.1 * q)**2 + (5.46 * q)**3 + (6.71 * q)**4)**-0.25
    assert np.max(np.abs(T / bbks - 1)) < 0.08


def test_eh_sound_horizon_against_the_measured_drag_scale():
    # Eisenstein & Hu (1998) Eq. 26 is a fit, stated to about 2%, to the sound horizon at the drag
    # epoch.  Planck 2018 (results VI, Table 2, TT,TE,EE+lowE+lensing) measures r_drag =
    # 147.09 +- 0.26 Mpc for Omega_m = 0.3153, Omega_b h^2 = 0.02237, h = 0.6736: a dropped square
    # root, a log10 for ln or a wrong exponent on omega_b moves the fit far outside 3%.
    h = 0.6736
    c = Cosmology(omega_m=0.3153, omega_b=0.02237 / h**2, h=h)
    assert abs(c.sound_horizon_mpc() / 147.09 - 1.0) < 0.03


@pytest.mark.parametrize("om,ob,h", [(0.31, 0.049, 0.67), (0.25, 0.04, 0.72), (0.4, 0.05, 0.65),
                                     (0.3, 0.02, 0.7), (0.3, 0.07, 0.7), (0.35, 0.03, 0.6)])
def test_eh_baryon_suppression_against_sugiyama(om, ob, h):
    # Eq. 31's alpha_Gamma (the small-scale shape Gamma_eff = alpha_Gamma Omega_m h) against the
    # independent fit of Sugiyama (1995), Gamma = Omega_m h exp(-Omega_b - sqrt(2h) Omega_b / Omega_m):
    # they agree to better than 1% for baryon fractions 0.07-0.23; a coefficient off by a digit
    # or a sign moves alpha_Gamma by several percent.
    c = Cosmology(omega_m=om, omega_b=ob, h=h)
    sugiyama = math.exp(-ob - math.sqrt(2.0 * h) * ob / om)
    assert abs(c.alpha_gamma() / sugiyama - 1.0) < 0.015
    # and the transfer function takes that shape well below the sound horizon: there it is the
    # zero-baryon transfer function (Gamma = Omega_m h) at k / alpha_Gamma
    no_baryons = Cosmology(omega_m=om, omega_b=0.0, h=h)
    for k in (20.0, 50.0, 200.0):
        assert c.transfer_eh_nowiggle(k) == pytest.approx(no_baryons.transfer_eh_nowiggle(k / c.alpha_gamma()), rel=1e-9)


def test_sigma8_normalisation_and_growth_scaling():
    c = Cosmology()
    assert c.sigma_R(8.0) == pytest.approx(0.81, rel=1e-9)
    a = 1.0 / 51.0
    assert c.power_linear(0.05, a) / c.power_linear(0.05) == pytest.approx(c.growth_D(a)**2, rel=1e-12)


def test_eq_bgr_from_the_gauge_relations_of_linear_theory():
    # Eq. bgr derived, not restated: for the growing mode of pressureless matter + Lambda the
    # comoving density delta_c grows as D on all scales, its velocity divergence in the Poisson
    # (longitudinal) gauge is theta = -calH f delta_c, and k^2 Phi = -(3/2) calH^2 Om(a) delta_c.
    # The Poisson-gauge density is delta_P = delta_c - 3 calH theta / k^2; halos with comoving bias
    # b1 move with the matter, so they take the same gauge term; the counting densities are
    # delta_P - 3 Phi (Eq. physical_density).  The coefficient of calH^2/k^2 in their ratio at
    # k >> calH is b1^GR.
    c = Cosmology()
    for z, b1 in ((0.0, 2.0), (0.5, 3.0), (1.0, 1.5), (2.0, 4.5)):
        a = 1.0 / (1.0 + z)
        H, f, om = float(c.conformal_hubble(a)), c.growth_f(a), float(c.omega_m_a(a))
        k = 1e4 * H
        x = (H / k)**2
        dc = 1.0
        theta = -H * f * dc
        phi = -1.5 * H * H * om * dc / k**2
        d_m = dc - 3.0 * H * theta / k**2 - 3.0 * phi
        d_h = b1 * dc - 3.0 * H * theta / k**2 - 3.0 * phi
        slope = (d_h / d_m - b1) / x
        assert slope == pytest.approx(b1_gr_theory(b1, f, om), rel=1e-6)
    # the gauge term's sign: a superhorizon mode in matter domination (f = Om = 1) has the
    # textbook Poisson-gauge density delta_P = -2 Phi
    x = 1e8
    d_p = 1.0 + 3.0 * x  # delta_c - 3 calH theta / k^2 with theta = -calH delta_c
    phi = -1.5 * x
    assert d_p / (-2.0 * phi) == pytest.approx(1.0, rel=1e-7)


def test_paper_table1_gr_bias_consistent_with_eq_bgr():
    # Table 1 b1GR at z <= 0.5 lies within 1.5 sigma of Eq. bgr evaluated with the oracle's
    # f(z) and Omega_m(z) in the Sec. 3 cosmology (the paper reports agreement with theory).
    rows = np.loadtxt(os.path.join(GOLDEN, "table1_bias.txt"))
    c = Cosmology(omega_m=0.263771 + 0.0482754, omega_b=0.0482754, h=0.67556, n_s=0.9619)
    for z, b1, b1gr, sig in rows:
        if z > 0.5:
            continue
        a = 1.0 / (1.0 + z)
        th = b1_gr_theory(b1, c.growth_f(a), float(c.omega_m_a(a)))
        assert abs(th - b1gr) < 1.5 * sig, (z, th, b1gr, sig)
