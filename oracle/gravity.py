"""Newtonian Poisson solve, linearised Poisson-gauge constraint and spectral gradient.

Oracle (test infrastructure only).

Code potential phi (Mpc/h)^2 in H0 = 1 units.  Newtonian gauge (Sec. 2: the
N-body-gauge Poisson equation is the Newtonian one): the comoving peculiar
potential Phi_N obeys lap Phi_N = (3/2) Omega_m delta / a, and with phi = a Phi_N
the kick is dp/da = -grad(phi) / (a^2 E).  Hence

    phi_k = -(3/2) Omega_m delta_k / k^2,   phi_0 = 0,

with the continuous 1/k^2 and no CIC deconvolution in the force (readings).

Poisson gauge (Sec. 2: gevolution's relativistic run; Eq. physical_density relates
the counting and physical densities, delta_count = delta_phys - 3 phi).  Reading:
scalar sector with Phi = Psi and no anisotropic stress, the linear 00 constraint

    lap Phi - 3 calH (Phi' + calH Phi) = (3/2) calH^2 Omega_m(a) delta_phys,

sourced by delta_phys = delta_count + 3 Phi, with Phi' the backward difference
(Phi - Phi_old) / dtau between consecutive force evaluations (Phi' = 0 at the
first).  Per Fourier mode

    Phi_k = [3 calH Phi_old,k / dtau - (3/2) calH^2 Om(a) delta_k]
            / [k^2 + 3 calH / dtau + 3 calH^2 + (9/2) calH^2 Om(a)],

and the particles feel phi = a c^2 Phi, which reduces to the Newtonian phi for
k >> calH.  Gradient: g_j = IFFT[-i k_j phi_k] with k_j = 0 at the Nyquist index.
"""
import numpy as np

from . import philox
from .cosmology import C_LIGHT


def _wavenumbers(n, box):
    kf = 2.0 * np.pi / box
    f = philox.signed_freqs(n).astype(np.float64)
    fz = np.arange(n // 2 + 1, dtype=np.float64)
    NX, NY, NZ = np.meshgrid(f, f, fz, indexing="ij")
    k2 = kf * kf * (NX * NX + NY * NY + NZ * NZ)
    return kf, (NX, NY, NZ), k2


def newton_potential_k(delta_k, n, box, omega_m):
    """phi_k = -(3/2) Omega_m delta_k / k^2 with phi_0 = 0."""
    _, _, k2 = _wavenumbers(n, box)
    phi = np.zeros_like(delta_k)
    nz = k2 > 0
    phi[nz] = -1.5 * omega_m * delta_k[nz] / k2[nz]
    return phi


def gr_potential_k(delta_k, n, box, cosmo, a, phi_old_k=None, dtau=None):
    """Poisson-gauge Phi_k (dimensionless) from the counting density delta_k."""
    _, _, k2 = _wavenumbers(n, box)
    H = float(cosmo.conformal_hubble(a))
    om = float(cosmo.omega_m_a(a))
    src = -1.5 * H * H * om * delta_k
    den = k2 + 3.0 * H * H + 4.5 * H * H * om
    if phi_old_k is not None:
        src = src + 3.0 * H * phi_old_k / dtau
        den = den + 3.0 * H / dtau
    Phi = src / den
    Phi[0, 0, 0] = 0.0
    return Phi


def gr_code_potential_k(Phi_k, a):
    """phi = a c^2 Phi, the potential that enters the Newtonian-form kick."""
    return a * C_LIGHT**2 * Phi_k


def gradient_force(phi_k, n, box):
    """Force meshes g_j = IFFT[-i k_j phi_k], j = x, y, z; Nyquist k_j set to 0."""
    kf, (NX, NY, NZ), _ = _wavenumbers(n, box)
    out = np.empty((3, n, n, n))
    for j, Nj in enumerate((NX, NY, NZ)):
        kj = kf * np.where(np.abs(Nj) == n // 2, 0.0, Nj)
        out[j] = np.fft.irfftn(-1j * kj * phi_k, s=(n, n, n), axes=(0, 1, 2))
    return out


def potential_mesh(phi_k, n):
    """Real-space potential on the mesh."""
    return np.fft.irfftn(phi_k, s=(n, n, n), axes=(0, 1, 2))
