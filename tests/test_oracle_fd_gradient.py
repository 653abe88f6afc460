"""Pins of the first-order (CIC-interpolant) gradient used by the finite-difference force
option (Sec. 4.1: the paper's PM code computes the force with a first-order gradient)."""
import numpy as np
import pytest

import inputs
from oracle import cic, gravity, ic, pm as opm
from oracle.cosmology import Cosmology


def _random_fractions(seed, count):
    return np.random.default_rng(seed).random((3, count))


def test_plane_wave_difference_across_the_cell_closed_form():
    # phi = cos(k x) on the nodes x_j = (j + 1/2) L/n: inside the cell [x_i, x_i+1] the x
    # derivative is (phi_{i+1} - phi_i)/dx = -(2/dx) sin(k dx/2) sin(k (x_i + dx/2)),
    # whatever the particle's place in the cell; the y and z derivatives vanish
    n, box, m = 16, 320.0, 3
    dx = box / n
    k = 2 * np.pi * m / box
    xn = (np.arange(n) + 0.5) * dx
    phi = np.cos(k * xn)[:, None, None] * np.ones((n, n, n))
    x = _random_fractions(1, 500)
    g = cic.interpolate_gradient(phi, x, box)
    s = x[0] * n - 0.5
    i = np.floor(s)
    want = -(2 / dx) * np.sin(k * dx / 2) * np.sin(k * (i + 1) * dx)
    assert np.max(np.abs(g[0] - want)) < 1e-12 * np.max(np.abs(want))
    assert np.max(np.abs(g[1])) < 1e-12 and np.max(np.abs(g[2])) < 1e-12


def test_is_the_derivative_of_the_cic_interpolation():
    # the CIC interpolant is linear along each axis inside a cell: a central difference of
    # cic.interpolate in the particle position reproduces the gradient (away from cell edges)
    n, box = 16, 500.0
    field = inputs.gaussian_field(3, n)
    x = _random_fractions(2, 400)
    s = x * n - 0.5
    inner = np.all(np.abs(s - np.floor(s) - 0.5) < 0.4, axis=0)
    x = x[:, inner]
    g = cic.interpolate_gradient(field, x, box)
    eps = 1e-3 / n
    for j in range(3):
        e = np.zeros((3, 1))
        e[j] = eps
        fd = (cic.interpolate(field, x + e) - cic.interpolate(field, x - e)) / (2 * eps * box)
        assert np.max(np.abs(fd - g[j])) < 1e-8 * np.max(np.abs(g[j]))


def test_first_order_convergence_to_the_analytic_gradient():
    # for a smooth potential the error against the exact gradient falls as the first power
    # of the spacing at general positions (the one-sided difference of a first-order scheme)
    box, m = 100.0, 1
    k = 2 * np.pi * m / box
    x = _random_fractions(4, 2000)
    errs = []
    for n in (16, 32, 64, 128):
        xn = (np.arange(n) + 0.5) * box / n
        phi = np.cos(k * xn)[:, None, None] * np.ones((n, n, n))
        g = cic.interpolate_gradient(phi, x, box)
        errs.append(np.max(np.abs(g[0] + k * np.sin(k * x[0] * box))))
    ratios = np.array(errs[:-1]) / np.array(errs[1:])
    assert np.all((ratios > 1.8) & (ratios < 2.2))


def test_fd1_run_differs_from_spectral_only_at_the_force():
    # one step of both force options from the same ICs: the densities agree (same ICs), the
    # FD1 force is the gradient of the CIC interpolant of the same potential
    c = Cosmology()
    n, box, a_i = 16, 400.0, 0.2
    x0, p0 = ic.zeldovich(c, n, box, a_i, seed=6, fixed=False)
    spec = opm.PMRun(c, n, box, a_i, 1.0, 4, x0, p0)
    fd = opm.PMRun(c, n, box, a_i, 1.0, 4, x0, p0, gradient=opm.FD1)
    phi = gravity.potential_mesh(fd.potential_k(a_i), n)
    g_fd = fd.accel(a_i)
    np.testing.assert_allclose(g_fd, -cic.interpolate_gradient(phi, x0, box), rtol=0, atol=1e-14 * np.abs(g_fd).max())
    g_sp = spec.accel(a_i)
    # the two gradients agree on large scales: correlated to better than 10% here
    assert np.linalg.norm(g_fd - g_sp) < 0.2 * np.linalg.norm(g_sp)


def test_fd1_force_is_minus_the_gradient_of_the_mesh_energy():
    # With rho(c) = m sum_p W(x_p - c) (CIC) and a symmetric Green's function, the mesh energy
    # E = 1/2 sum_c delta(c) phi(c) has dE/dx_p = m sum_c dW(x_p - c)/dx_p phi(c), i.e. m times
    # the gradient of the CIC interpolant of phi at x_p: the first-order force is the exact
    # negative gradient of the energy (E is piecewise quadratic in x_p, so a central difference
    # inside the cell reproduces it to rounding)
    n, box, om = 16, 400.0, 0.31
    rng = np.random.default_rng(9)
    x = rng.random((3, 6))
    m = n**3 / x.shape[1]

    def energy(xx):
        delta = cic.density_contrast(xx, n)
        phi = gravity.potential_mesh(gravity.newton_potential_k(np.fft.rfftn(delta), n, box, om), n)
        return 0.5 * np.sum(delta * phi), phi

    _, phi = energy(x)
    grad = cic.interpolate_gradient(phi, x, box)
    s = x * n - 0.5
    frac = s - np.floor(s)
    eps = 1e-4 / n
    checked = 0
    for p in range(x.shape[1]):
        for j in range(3):
            if not (0.01 < frac[j, p] < 0.99):
                continue
            e = np.zeros_like(x)
            e[j, p] = eps
            dE = (energy(x + e)[0] - energy(x - e)[0]) / (2 * eps * box)
            assert dE == pytest.approx(m * grad[j, p], rel=1e-7, abs=1e-10 * m * np.abs(grad).max())
            checked += 1
    assert checked >= 12
