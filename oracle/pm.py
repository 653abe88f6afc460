"""Particle-mesh kick-drift-kick leapfrog in the scale factor.

Oracle (test infrastructure only).

One force evaluation per step on a uniform a-grid a_n = a_i + n (a_f - a_i)/N_steps
(reading; the paper's codes use their own integrators):

    p_{n+1/2} = p_{n-1/2} + K(a_{n-1/2}, a_{n+1/2}) g(x_n)    (first step: K(a_0, a_{1/2}))
    x_{n+1}   = x_n + D(a_n, a_{n+1}) p_{n+1/2}
    closing   : p_N = p_{N-1/2} + K(a_{N-1/2}, a_N) g(x_N)     after the last step,

with a_{n+1/2} the arithmetic midpoint, g = -grad(phi) interpolated with CIC, and
K, D the FP64 integrals of ``cosmology`` (stepping = INTEGRALS) or the growth-matched
factors that make every step exact for the linear growing mode (stepping = GROWTH:
``cosmology.kick_factor_growth`` with the force taken at a_n, a_N for the closing kick, and
``cosmology.drift_factor_growth`` with the momenta at a_{n+1/2}).  A force evaluation is: CIC deposit of
the counting density, FFT, Green's function (Newtonian or the linearised
Poisson-gauge constraint of ``gravity``), spectral gradient, inverse FFT, CIC
interpolation.  With gradient = FD1 the potential itself is transformed back and
g = -grad of its CIC interpolant at the particle (the first-order finite difference
across the particle's cell, ``cic.interpolate_gradient``).  Fixed-point drift: Delta u = round-half-even(D p 2^32 / L),
u <- (u + Delta u) mod 2^32; FP64 drift: u <- frac(u + D p / L).
"""
import numpy as np

from . import cic, gravity

NEWTON = 0
GR_POISSON = 1
SPECTRAL = 0
FD1 = 1
INTEGRALS = 0
GROWTH = 1


class PMRun:
    def __init__(self, cosmo, n_mesh, box, a_init, a_final, n_steps, x, p, mode=NEWTON, gradient=SPECTRAL,
                 stepping=INTEGRALS):
        self.cosmo = cosmo
        self.n = int(n_mesh)
        self.box = float(box)
        self.a_grid = a_init + (a_final - a_init) * np.arange(n_steps + 1) / n_steps
        self.n_steps = int(n_steps)
        self.x = np.array(x, copy=True)
        self.p = np.array(p, dtype=np.float64, copy=True)
        self.fixed = self.x.dtype == np.uint32
        self.mode = mode
        self.gradient = gradient
        self.stepping = stepping
        self.i = 0
        self.synced = True
        self.phi_old_k = None
        self.a_last_force = None

    # ------------------------------------------------------------------ force
    def potential_k(self, a):
        """Code potential phi_k of the current particles at scale factor a."""
        delta = cic.density_contrast(self.x, self.n)
        dk = np.fft.rfftn(delta)
        if self.mode == NEWTON:
            return gravity.newton_potential_k(dk, self.n, self.box, self.cosmo.omega_m)
        dtau = None
        if self.phi_old_k is not None:
            dtau = self.cosmo.delta_tau(self.a_last_force, a)
        Phi = gravity.gr_potential_k(dk, self.n, self.box, self.cosmo, a,
                                     phi_old_k=self.phi_old_k, dtau=dtau)
        self.phi_old_k = Phi
        self.a_last_force = a
        return gravity.gr_code_potential_k(Phi, a)

    def accel(self, a):
        """g(x) = -grad(phi) at the particles, shape (3, Np)."""
        phi_k = self.potential_k(a)
        if self.gradient == FD1:
            return -cic.interpolate_gradient(gravity.potential_mesh(phi_k, self.n), self.x, self.box)
        g_mesh = gravity.gradient_force(phi_k, self.n, self.box)
        return np.stack([cic.interpolate(g_mesh[j], self.x) for j in range(3)])

    # ------------------------------------------------------------------ update
    def _drift(self, dfac):
        if self.fixed:
            du = np.rint(dfac * self.p * (2.0**32 / self.box)).astype(np.int64)
            self.x = ((self.x.astype(np.int64) + du) % 2**32).astype(np.uint32)
        else:
            x = self.x + dfac * self.p / self.box
            self.x = x - np.floor(x)

    def step(self, nsteps=1):
        for _ in range(nsteps):
            if self.i >= self.n_steps:
                raise ValueError("past the end of the a-grid")
            a0, a1 = self.a_grid[self.i], self.a_grid[self.i + 1]
            ah = 0.5 * (a0 + a1)
            g = self.accel(a0)
            a_from = a0 if self.synced else 0.5 * (self.a_grid[self.i - 1] + a0)
            self.p += self._kick(a_from, ah, a0) * g
            self._drift(self._drift_fac(a0, a1, ah))
            self.i += 1
            self.synced = False
            if self.i == self.n_steps:
                g = self.accel(a1)
                self.p += self._kick(ah, a1, a1) * g
                self.synced = True

    def _kick(self, a0, a1, a_force):
        if self.stepping == GROWTH:
            return self.cosmo.kick_factor_growth(a0, a1, a_force)
        return self.cosmo.kick_factor(a0, a1)

    def _drift_fac(self, a0, a1, a_mom):
        if self.stepping == GROWTH:
            return self.cosmo.drift_factor_growth(a0, a1, a_mom)
        return self.cosmo.drift_factor(a0, a1)

    def positions_mpc(self):
        """Positions in Mpc/h in [0, L)."""
        if self.fixed:
            return self.x.astype(np.float64) * (self.box / 2.0**32)
        return self.x * self.box
