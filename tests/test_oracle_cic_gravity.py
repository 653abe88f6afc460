"""Pins of the CIC deposit/interpolation, cell keys, Poisson solves and gradient."""
import numpy as np
import pytest

import inputs
from oracle import cic, gravity
from oracle.cosmology import C_LIGHT, Cosmology


def test_mass_conservation_any_positions():
    for x in (inputs.uniform_ticks(1, 10_007), inputs.clustered_ticks(2, 5_003),
              inputs.ticks_to_fractions(inputs.uniform_ticks(3, 999))):
        rho = cic.deposit(x, 16)
        assert rho.sum() == pytest.approx(16**3, rel=1e-13)


def test_uniform_lattice_gives_zero_contrast():
    n = 8
    i = (np.arange(n, dtype=np.uint64) * (2**32 // n)).astype(np.uint32)
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    assert np.all(cic.density_contrast(x, n) == 0.0)
    # a lattice of 8^3 particles on a 16^3 mesh: the lattice sits half a cell off the
    # cell-centred nodes, so every node gets (1/2)^3 of one particle of mass 8
    rho = cic.deposit(x, 16)
    assert np.all(rho == 1.0)


def test_single_particle_weights():
    n = 8
    s = np.array([2.25, 5.5, 7.75])  # mesh coordinates (nodes at cell centres); z wraps to node 0
    x = np.floor((s + 0.5) / n * 2**32).astype(np.uint64).astype(np.uint32).reshape(3, 1)
    rho = cic.deposit(x, n, mass=1.0)
    w = {(2, 0.75), (3, 0.25)}, {(5, 0.5), (6, 0.5)}, {(7, 0.25), (0, 0.75)}
    expect = np.zeros((n, n, n))
    for ix, wx in w[0]:
        for iy, wy in w[1]:
            for iz, wz in w[2]:
                expect[ix, iy, iz] = wx * wy * wz
    np.testing.assert_array_equal(rho, expect)
    # a particle of mass m deposits m times the weights
    np.testing.assert_array_equal(cic.deposit(x, n, mass=2.5), 2.5 * expect)


def test_interpolation_is_transpose_of_deposit():
    n = 16
    x = inputs.uniform_ticks(4, 3000)
    f = inputs.gaussian_field(5, n)
    lhs = np.sum(cic.deposit(x, n, mass=1.0) * f)
    rhs = np.sum(cic.interpolate(f, x))
    assert lhs == pytest.approx(rhs, rel=1e-12)


def test_interpolation_exact_for_linear_field():
    n = 16
    g = np.arange(n, dtype=np.float64)
    f = 0.5 * g[:, None, None] - 2.0 * g[None, :, None] + 3.0 * g[None, None, :] + np.zeros((n, n, n))
    u = inputs.rng(6).uniform(0.5 / n, (n - 0.5) / n, size=(3, 500))  # away from the periodic seam
    s = u * n - 0.5  # mesh coordinate of a cell-centred node grid
    want = 0.5 * s[0] - 2.0 * s[1] + 3.0 * s[2]
    np.testing.assert_allclose(cic.interpolate(f, u), want, rtol=0, atol=1e-12)


def test_cell_keys_match_integer_shifts():
    # Base node from the float path equals the top log2(N) bits of the tick minus half a cell.
    x = inputs.uniform_ticks(7, 20_000)
    for n in (8, 64, 512):
        sh = 32 - int(np.log2(n))
        b = ((x.astype(np.int64) - (1 << (sh - 1))) & 0xFFFFFFFF) >> sh
        want = (b[0] * n + b[1]) * n + b[2]
        np.testing.assert_array_equal(cic.cell_keys(x, n), want)
        f = inputs.ticks_to_fractions(x)
        np.testing.assert_array_equal(cic.cell_keys(f, n), want)


def test_cell_order_is_stable_sort():
    x = inputs.lattice_order_ticks(8, 8, 1.5, n_mesh=4)
    keys = cic.cell_keys(x, 4)
    order = cic.cell_order(x, 4)
    k = keys[order]
    assert np.all(np.diff(k) >= 0)
    same = np.diff(k) == 0
    assert np.all(np.diff(order)[same] > 0)


def _cos_mode(n, nvec, eps):
    g = np.arange(n)
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    ph = 2 * np.pi * (nvec[0] * X + nvec[1] * Y + nvec[2] * Z) / n
    return eps * np.cos(ph), ph


@pytest.mark.parametrize("nvec", [(1, 0, 0), (2, -3, 1), (0, 5, 7)])
def test_single_mode_poisson_and_gradient(nvec):
    # delta = eps cos(k.x): phi = -(3/2) Om eps cos(k.x)/k^2, g = -grad phi = -(3/2) Om eps k sin(k.x)/k^2
    n, box, om = 16, 300.0, 0.31
    delta, ph = _cos_mode(n, nvec, 1e-2)
    phik = gravity.newton_potential_k(np.fft.rfftn(delta), n, box, om)
    k = 2 * np.pi / box * np.array(nvec, dtype=np.float64)
    k2 = k @ k
    phi = gravity.potential_mesh(phik, n)
    np.testing.assert_allclose(phi, -1.5 * om * delta / k2, rtol=0, atol=1e-13 / k2)
    g = gravity.gradient_force(phik, n, box)
    for j in range(3):
        want = -1.5 * om * 1e-2 * k[j] * np.sin(ph) / k2
        np.testing.assert_allclose(g[j], want, rtol=0, atol=1e-13 / np.sqrt(k2))


def test_nyquist_gradient_is_zero():
    n, box = 8, 100.0
    delta, _ = _cos_mode(n, (4, 0, 0), 1.0)  # the x-Nyquist plane wave
    g = gravity.gradient_force(gravity.newton_potential_k(np.fft.rfftn(delta), n, box, 0.3), n, box)
    assert np.max(np.abs(g)) < 1e-15


def test_gr_constraint_reduces_to_newton_inside_horizon():
    n, box, a = 16, 20.0, 1.0  # k >= 0.3 h/Mpc >> calH ~ 3e-4 h/Mpc
    c = Cosmology()
    dk = np.fft.rfftn(inputs.gaussian_field(9, n))
    Phi = gravity.gr_potential_k(dk, n, box, c, a)
    phi_gr = gravity.gr_code_potential_k(Phi, a)
    phi_n = gravity.newton_potential_k(dk, n, box, c.omega_m)
    assert np.max(np.abs(phi_gr - phi_n)) < 1e-5 * np.max(np.abs(phi_n))


def test_gr_matter_era_identity():
    # Omega_m = 1, Phi' = 0: the 00 constraint reads -k^2 Phi - 3 calH^2 Phi = (3/2) calH^2 delta_phys,
    # i.e. delta_phys = -2 Phi - (2/3)(k^2/calH^2) Phi, with delta_phys = delta_count + 3 Phi.
    n, box, a = 8, 20000.0, 0.1
    c = Cosmology(omega_m=1.0)
    dk = np.fft.rfftn(inputs.gaussian_field(10, n))
    Phi = gravity.gr_potential_k(dk, n, box, c, a)
    _, _, k2 = gravity._wavenumbers(n, box)
    H = float(c.conformal_hubble(a))
    lhs = dk + 3 * Phi
    rhs = -2 * Phi - (2.0 / 3.0) * k2 / H**2 * Phi
    lhs[0, 0, 0] = rhs[0, 0, 0] = 0
    assert np.max(np.abs(lhs - rhs)) < 1e-12 * np.max(np.abs(dk))


def test_gr_lag_fixed_point():
    # A static potential (Phi_old equal to the Phi' = 0 solution) is a fixed point of the lagged solve.
    n, box, a = 8, 4000.0, 0.5
    c = Cosmology()
    dk = np.fft.rfftn(inputs.gaussian_field(11, n))
    Phi0 = gravity.gr_potential_k(dk, n, box, c, a)
    Phi1 = gravity.gr_potential_k(dk, n, box, c, a, phi_old_k=Phi0, dtau=37.0)
    assert np.max(np.abs(Phi1 - Phi0)) < 1e-14 * np.max(np.abs(Phi0))
    assert C_LIGHT == pytest.approx(299792.458 / 100.0)


def _linear_theory_history(c, n, box, a):
    """Linear Lambda-CDM in Poisson gauge for pressureless matter: Phi(k, a) = Phi_0(k) D(a)/a
    on every scale, so Phi' = (f - 1) calH Phi, and the 00 constraint fixes
    delta_phys = -Phi (k^2 + 3 calH^2 f) / ((3/2) calH^2 Om(a)); delta_count = delta_phys - 3 Phi
    (Eq. physical_density).  Returns (Phi, delta_count) at a."""
    _, _, k2 = gravity._wavenumbers(n, box)
    phi0 = np.fft.rfftn(inputs.gaussian_field(12, n)) * 1e-5
    phi0[0, 0, 0] = 0.0
    H, om, f = float(c.conformal_hubble(a)), float(c.omega_m_a(a)), c.growth_f(a)
    phi = phi0 * c.growth_D(a) / a
    dcount = -phi * (k2 + 3.0 * H * H * f) / (1.5 * H * H * om) - 3.0 * phi
    dcount[0, 0, 0] = 0.0
    return phi, dcount


def _lagged_history_error(c, steps, n=8, box=40000.0, a_i=1.0 / 101.0):
    """Largest error of the lagged solve along a uniform a-grid, fed the closed-form counting
    density (Phi' = 0 at the first evaluation, backward difference over dtau afterwards)."""
    grid = a_i + (1.0 - a_i) * np.arange(steps + 1) / steps
    old, a_old, err = None, None, 0.0
    for a in grid:
        truth, dcount = _linear_theory_history(c, n, box, a)
        if old is None:
            Phi = gravity.gr_potential_k(dcount, n, box, c, a)
        else:
            Phi = gravity.gr_potential_k(dcount, n, box, c, a, phi_old_k=old, dtau=c.delta_tau(a_old, a))
        err = max(err, np.max(np.abs(Phi - truth)) / np.max(np.abs(truth)))
        old, a_old = Phi, a
    return err


def test_gr_lag_term_follows_linear_theory_on_superhorizon_modes():
    # L = 40 Gpc/h on 8^3: k = 1.6e-4 .. 6e-4 h/Mpc, at or above the horizon (calH(a = 1) = 3.3e-4),
    # where Phi' weighs as much as calH Phi.  The lagged constraint must follow Phi_0 D(a)/a with an
    # error of first order in dtau (halving the step halves it), 1e-3 at 100 steps; a lag term with
    # another coefficient than 3 calH misses it by 5-12%.
    c = Cosmology()
    e50, e100, e200 = (_lagged_history_error(c, s) for s in (50, 100, 200))
    assert e100 < 1.5e-3
    assert 1.8 < e50 / e100 < 2.2 and 1.8 < e100 / e200 < 2.2


def test_pm_run_threads_phi_old_and_dtau_through_its_force_evaluations(monkeypatch):
    # the same history through PMRun's own bookkeeping of Phi_old and dtau between the force
    # evaluations of its steps (the counting density is handed in, the particles are not used)
    from oracle import pm as opm
    n, box, steps, a_i = 8, 40000.0, 100, 1.0 / 101.0
    c = Cosmology()
    now = {}
    monkeypatch.setattr(opm.cic, "density_contrast",
                        lambda x, nn: np.fft.irfftn(_linear_theory_history(c, n, box, now["a"])[1], s=(n, n, n), axes=(0, 1, 2)))
    x = np.zeros((3, 1), dtype=np.uint32)
    run = opm.PMRun(c, n, box, a_i, 1.0, steps, x, np.zeros((3, 1)), mode=opm.GR_POISSON)
    err = 0.0
    for a in run.a_grid:
        now["a"] = a
        Phi = run.potential_k(a) / (a * C_LIGHT**2)
        truth = _linear_theory_history(c, n, box, a)[0]
        err = max(err, np.max(np.abs(Phi - truth)) / np.max(np.abs(truth)))
    assert err < 1.5e-3
