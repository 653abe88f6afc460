"""Pins of the second-order LPT initial conditions (Sec. 3: the paper's ICs are 2LPT)."""
import numpy as np
import pytest
from scipy.integrate import solve_ivp

from oracle import ic
from oracle.cosmology import Cosmology


def _mesh_k(field):
    return np.fft.rfftn(field)


def _nodes(n):
    i = np.arange(n) / n
    return np.meshgrid(i, i, i, indexing="ij")


@pytest.mark.parametrize("direction", [(2, 0, 0), (0, 0, 3), (1, 1, 0), (2, 0, 2), (1, 1, 1), (1, 2, 0)])
def test_single_plane_wave_has_no_second_order_displacement(direction):
    # a one-dimensional perturbation (along any lattice direction) has phi1_ii phi1_jj =
    # phi1_ij^2 for every pair, so the source and Psi2 vanish; Zel'dovich is exact in 1-D
    n, box = 16, 400.0
    X, Y, Z = _nodes(n)
    dx, dy, dz = direction
    delta = 0.3 * np.cos(2 * np.pi * (dx * X + dy * Y + dz * Z) + 0.4)
    psi2 = ic.lpt2_displacement(_mesh_k(delta), n, box)
    psi1 = ic.za_displacement(_mesh_k(delta), n, box)
    assert np.max(np.abs(psi1)) > 0.1
    assert np.max(np.abs(psi2)) < 1e-13 * np.max(np.abs(psi1))


def test_crossed_plane_waves_match_the_closed_form():
    # delta = A cos(k1 x) + B cos(k2 y): phi1_xx = A cos(k1 x), phi1_yy = B cos(k2 y), phi1_xy = 0,
    # so laplacian(phi2) = A B cos(k1 x) cos(k2 y), phi2 = -A B cos cos / (k1^2 + k2^2), Psi2 = grad phi2
    n, box = 16, 500.0
    A, B, m1, m2 = 0.2, -0.15, 2, 3
    k1, k2 = 2 * np.pi * m1 / box, 2 * np.pi * m2 / box
    X, Y, Z = _nodes(n)
    cx, sx = np.cos(2 * np.pi * m1 * X), np.sin(2 * np.pi * m1 * X)
    cy, sy = np.cos(2 * np.pi * m2 * Y), np.sin(2 * np.pi * m2 * Y)
    psi2 = ic.lpt2_displacement(_mesh_k(A * cx + B * cy), n, box)
    amp = A * B / (k1 * k1 + k2 * k2)
    want = np.stack([amp * k1 * sx * cy, amp * k2 * cx * sy, np.zeros_like(X)])
    assert np.max(np.abs(psi2 - want)) < 1e-12 * np.max(np.abs(want))


def test_second_order_displacement_divergence_is_the_source():
    # div Psi2 = laplacian(phi2) = S for every mode kept (no Nyquist component, not zero)
    n, box, c = 16, 600.0, Cosmology()
    dk = ic.linear_delta_k(c, n, box, seed=17)
    psi2 = ic.lpt2_displacement(dk, n, box)
    kf = 2 * np.pi / box
    f = np.fft.fftfreq(n, 1.0 / n)
    fz = np.arange(n // 2 + 1)
    div = sum(1j * kf * ax * np.fft.rfftn(psi2[j])
              for j, ax in enumerate((f[:, None, None], f[None, :, None], fz[None, None, :])))
    # the source from finite products of spectral second derivatives, written out again
    phi = -dk / np.where(ic.mode_n2(n) > 0, (kf**2) * ic.mode_n2(n), np.inf)
    kk = (f[:, None, None] * kf, f[None, :, None] * kf, fz[None, None, :] * kf)
    d = {(i, j): np.fft.irfftn(-kk[i] * kk[j] * phi, s=(n, n, n), axes=(0, 1, 2)) for i in range(3) for j in range(i, 3)}
    S = sum(d[i, i] * d[j, j] - d[i, j]**2 for i in range(3) for j in range(i + 1, 3))
    NX, NY, NZ = np.meshgrid(f, f, fz, indexing="ij")
    keep = (np.abs(NX) != n // 2) & (np.abs(NY) != n // 2) & (NZ != n // 2) & (ic.mode_n2(n) > 0)
    Sk = np.fft.rfftn(S)
    assert np.max(np.abs(Sk[keep])) > 0
    assert np.max(np.abs(div[keep] - Sk[keep])) < 1e-10 * np.max(np.abs(Sk[keep]))
    assert np.max(np.abs(div[~keep])) < 1e-10 * np.max(np.abs(Sk[keep]))


def test_second_order_growth_fits():
    # Einstein-de Sitter: D2 = -(3/7) a^2 and f2 = 2 exactly
    eds = Cosmology(omega_m=1.0)
    for a in (0.02, 0.3, 1.0):
        assert eds.growth_D2(a) == pytest.approx(-3.0 / 7.0 * a * a, rel=1e-12)
        assert eds.growth_f2(a) == pytest.approx(2.0, rel=1e-12)
    # LambdaCDM: the fits against the second-order growth equation
    #   D2'' + (2 + dlnE/dlna) D2' - 3/2 Om(a) D2 = -3/2 Om(a) D^2   (' = d/dlna)
    # integrated from the matter era (D2 = -3/7 D^2) with D from the first-order equation
    c = Cosmology()

    def rhs(lna, y):
        a = np.exp(lna)
        om = c.omega_m_a(a)
        dlnE = -1.5 * c.omega_m * a**-3 / c.E(a)**2
        D, dD, D2, dD2 = y
        return [dD, -(2 + dlnE) * dD + 1.5 * om * D, dD2, -(2 + dlnE) * dD2 + 1.5 * om * D2 - 1.5 * om * D * D]

    a0 = 1e-4
    sol = solve_ivp(rhs, [np.log(a0), 0.0], [a0, a0, -3 / 7 * a0**2, -6 / 7 * a0**2], rtol=1e-12, atol=1e-22,
                    dense_output=True)
    d1_today = sol.y[0, -1]
    for a, tol_d2, tol_f2 in ((1 / 51, 1e-10, 1e-6), (0.5, 1e-4, 5e-3), (1.0, 5e-4, 5e-3)):
        D, dD, D2, dD2 = sol.sol(np.log(a))
        assert D / d1_today == pytest.approx(c.growth_D(a), rel=1e-10)
        assert D2 / d1_today**2 == pytest.approx(c.growth_D2(a), rel=tol_d2)
        assert dD2 / D2 == pytest.approx(c.growth_f2(a), rel=tol_f2)


def test_2lpt_particles_add_the_second_order_term():
    c = Cosmology()
    n, box, a = 16, 700.0, 0.3
    x1, p1 = ic.zeldovich(c, n, box, a, seed=8, fixed=False)
    x2, p2 = ic.zeldovich(c, n, box, a, seed=8, fixed=False, lpt_order=2)
    psi2 = ic.lpt2_displacement(ic.linear_delta_k(c, n, box, seed=8), n, box).reshape(3, -1)
    d = (x2 - x1) * box
    d -= box * np.rint(d / box)
    assert np.max(np.abs(d - c.growth_D2(a) * psi2)) < 1e-9 * np.max(np.abs(c.growth_D2(a) * psi2))
    pf = a * a * c.E(a) * c.growth_f2(a) * c.growth_D2(a)
    assert np.max(np.abs(p2 - p1 - pf * psi2)) < 1e-12 * np.max(np.abs(p1))
    # the second-order term is a correction: well below the first-order displacement here
    assert 1e-4 < np.max(np.abs(d)) / np.max(np.abs(p1 / (a * a * c.E(a) * c.growth_f(a)))) < 0.3
