"""FP64 LambdaCDM background, linear growth, leapfrog factors and linear P(k).

Oracle (test infrastructure only).  Units: lengths in Mpc/h, wavenumbers in h/Mpc,
H0 = 1 so that velocities are in units of 100 km/s and c = 2997.92458.

Paper: Sec. 3 ("Simulation setup") fixes a matter + Lambda background with the
radiation term removed, Omega_Lambda = 1 - Omega_m.  The linear spectrum is the
Eisenstein & Hu (1998) no-wiggle fit normalised to sigma_8 (the paper itself
uses CLASS with A_s; sigma_8 normalisation is this oracle's reading).
"""
import math

import numpy as np
from scipy import integrate

C_LIGHT = 2997.92458  # speed of light in units of 100 km/s


class Cosmology:
    """Flat matter + Lambda background (no radiation, Sec. 3)."""

    def __init__(self, omega_m=0.31, omega_b=0.049, h=0.67, n_s=0.965,
                 sigma8=0.81, t_cmb=2.7255):
        self.omega_m = float(omega_m)
        self.omega_b = float(omega_b)
        self.h = float(h)
        self.n_s = float(n_s)
        self.sigma8 = float(sigma8)
        self.t_cmb = float(t_cmb)
        self.omega_l = 1.0 - self.omega_m
        self._amp = None

    # ---------------------------------------------------------------- background
    def E(self, a):
        """H(a)/H0 = sqrt(Omega_m a^-3 + Omega_Lambda) (Sec. 3: no radiation)."""
        a = np.asarray(a, dtype=np.float64)
        return np.sqrt(self.omega_m / a**3 + self.omega_l)

    def omega_m_a(self, a):
        """Omega_m(a) = Omega_m a^-3 / E(a)^2."""
        return self.omega_m / np.asarray(a, dtype=np.float64)**3 / self.E(a)**2

    def conformal_hubble(self, a):
        """Conformal Hubble rate calH = a H / c in h/Mpc (H0 = 1 units)."""
        return a * self.E(a) / C_LIGHT

    # ---------------------------------------------------------------- growth
    def _growth_integral(self, a):
        """I(a) = int_0^a da' / (a' E(a'))^3 (Heath 1977 integral form)."""
        val, _ = integrate.quad(lambda x: 1.0 / (x * self.E(x))**3, 0.0, float(a),
                                epsabs=0.0, epsrel=1e-13, limit=200)
        return val

    def growth_D(self, a):
        """Linear growth D(a) = (5 Omega_m / 2) E(a) I(a), normalised to D(1) = 1."""
        raw = lambda x: 2.5 * self.omega_m * float(self.E(x)) * self._growth_integral(x)
        return raw(a) / raw(1.0)

    def growth_f(self, a):
        """f = dlnD/dlna = dlnE/dlna + 1 / (a^2 E^3 I(a))."""
        a = float(a)
        E = float(self.E(a))
        dlnE = -1.5 * self.omega_m / a**3 / E**2
        return dlnE + 1.0 / (a**2 * E**3 * self._growth_integral(a))

    # ---------------------------------------------------------------- leapfrog
    def growth_D2(self, a):
        """Second-order growth D2 = -(3/7) D^2 Om(a)^(-1/143) (Bouchet et al. 1995 fit;
        exact -3/7 D^2 for Om = 1).  Sec. 3: the paper's ICs are second-order LPT."""
        return -3.0 / 7.0 * self.growth_D(a)**2 * self.omega_m_a(a)**(-1.0 / 143.0)

    def growth_f2(self, a):
        """dln D2 / dln a = 2 Om(a)^(6/11) (Bouchet et al. 1995 fit)."""
        return 2.0 * self.omega_m_a(a)**(6.0 / 11.0)

    def kick_factor(self, a0, a1):
        """K(a0, a1) = int_{a0}^{a1} da / (a^2 E(a)): dp/da = -grad(phi)/(a^2 E)."""
        val, _ = integrate.quad(lambda a: 1.0 / (a * a * self.E(a)), float(a0), float(a1),
                                epsabs=0.0, epsrel=1e-13, limit=200)
        return val

    def drift_factor(self, a0, a1):
        """D(a0, a1) = int_{a0}^{a1} da / (a^3 E(a)): dx/da = p/(a^3 E)."""
        val, _ = integrate.quad(lambda a: 1.0 / (a**3 * self.E(a)), float(a0), float(a1),
                                epsabs=0.0, epsrel=1e-13, limit=200)
        return val

    def growth_p(self, a):
        """Momentum growth of the linear growing mode: p = a^3 E dx/da = a^2 E f D Psi for
        x = q + D Psi (the Zel'dovich momenta of ``ic``)."""
        return float(a)**2 * float(self.E(a)) * self.growth_f(a) * self.growth_D(a)

    def kick_factor_growth(self, a0, a1, a_force):
        """Kick factor that is exact for the linear growing mode (the growth-matched factors of
        FastPM, Feng et al. 2016): the linear force at a_force is g = (3/2) Om D(a_force) Psi
        and p must go from growth_p(a0) Psi to growth_p(a1) Psi."""
        return (self.growth_p(a1) - self.growth_p(a0)) / (1.5 * self.omega_m * self.growth_D(a_force))

    def drift_factor_growth(self, a0, a1, a_mom):
        """Drift factor exact for the linear growing mode: x goes from D(a0) Psi to D(a1) Psi
        with the momenta growth_p(a_mom) Psi held over the drift."""
        return (self.growth_D(a1) - self.growth_D(a0)) / self.growth_p(a_mom)

    def delta_tau(self, a0, a1):
        """Conformal-time interval in Mpc/h: dtau = c da / (a^2 E)."""
        return C_LIGHT * self.kick_factor(a0, a1)

    # ---------------------------------------------------------------- linear P(k)
    def sound_horizon_mpc(self):
        """Eisenstein & Hu (1998) Eq. 26: fitted sound horizon at the drag epoch (Mpc)."""
        omh2 = self.omega_m * self.h * self.h
        obh2 = self.omega_b * self.h * self.h
        return 44.5 * np.log(9.83 / omh2) / np.sqrt(1.0 + 10.0 * obh2**0.75)

    def alpha_gamma(self):
        """Eisenstein & Hu (1998) Eq. 31: the baryons' suppression of the shape parameter on
        scales well below the sound horizon, Gamma_eff -> alpha_Gamma Omega_m h."""
        omh2 = self.omega_m * self.h * self.h
        fb = self.omega_b / self.omega_m
        return 1.0 - 0.328 * np.log(431.0 * omh2) * fb + 0.38 * np.log(22.3 * omh2) * fb * fb

    def transfer_eh_nowiggle(self, k):
        """Eisenstein & Hu (1998) zero-baryon-oscillation transfer function.

        Their Eqs. 26 (sound horizon), 28-31 (alpha_Gamma, Gamma_eff, q, L0, C0);
        k in h/Mpc.
        """
        k = np.asarray(k, dtype=np.float64)
        om, h = self.omega_m, self.h
        theta = self.t_cmb / 2.7
        s = self.sound_horizon_mpc()
        alpha = self.alpha_gamma()
        k_mpc = k * h
        gamma_eff = om * h * (alpha + (1.0 - alpha) / (1.0 + (0.43 * k_mpc * s)**4))
        q = k * theta * theta / gamma_eff
        L0 = np.log(2.0 * math.e + 1.8 * q)
        C0 = 14.2 + 731.0 / (1.0 + 62.5 * q)
        return L0 / (L0 + C0 * q * q)

    def _unnormalised_power(self, k):
        return np.asarray(k, dtype=np.float64)**self.n_s * self.transfer_eh_nowiggle(k)**2

    @staticmethod
    def tophat_window(x):
        """Fourier transform of a real-space spherical top hat, 3 (sin x - x cos x)/x^3."""
        x = np.asarray(x, dtype=np.float64)
        small = np.abs(x) < 1e-3
        xs = np.where(small, 1.0, x)
        w = 3.0 * (np.sin(xs) - xs * np.cos(xs)) / xs**3
        return np.where(small, 1.0 - x * x / 10.0, w)

    def _sigma2_unnormalised(self, R):
        f = lambda lnk: (np.exp(lnk)**3 * self._unnormalised_power(np.exp(lnk))
                         * self.tophat_window(np.exp(lnk) * R)**2 / (2.0 * np.pi**2))
        val, _ = integrate.quad(f, math.log(1e-7), math.log(1e3), epsabs=0.0,
                                epsrel=1e-12, limit=1000)
        return val

    @property
    def amplitude(self):
        """A such that sigma(R = 8 Mpc/h, a = 1) = sigma_8."""
        if self._amp is None:
            self._amp = self.sigma8**2 / self._sigma2_unnormalised(8.0)
        return self._amp

    def power_linear(self, k, a=1.0):
        """P(k, a) = A k^n_s T(k)^2 D(a)^2 in (Mpc/h)^3."""
        D = 1.0 if a == 1.0 else self.growth_D(a)
        return self.amplitude * self._unnormalised_power(k) * D * D

    def sigma_R(self, R, a=1.0):
        D = 1.0 if a == 1.0 else self.growth_D(a)
        return math.sqrt(self.amplitude * self._sigma2_unnormalised(R)) * D
