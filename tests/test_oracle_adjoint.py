"""Pin of the FP64 reverse-mode gradient: central finite differences of the forward
oracle itself (no shared arithmetic with the reverse sweep)."""
import numpy as np
import pytest

import inputs
from oracle import adjoint, cic
from oracle.cosmology import Cosmology


@pytest.mark.parametrize("n_p,n_mesh", [(16, 16), (8, 16)])
def test_gradient_matches_central_differences(n_p, n_mesh):
    c = Cosmology()
    box, ai, af, steps = 300.0, 0.2, 0.6, 4
    w = inputs.gaussian_field(1, n_p)
    ut, _, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, inputs.gaussian_field(2, n_p))
    target = cic.density_contrast(ut, n_mesh)
    L, g = adjoint.loss_and_grad(c, n_p, n_mesh, box, ai, af, steps, w, target)
    assert L == pytest.approx(adjoint.loss(c, n_p, n_mesh, box, ai, af, steps, w, target), rel=1e-14)
    rng = np.random.default_rng(3)
    eps = 1e-5  # small enough that no particle crosses a CIC cell boundary
    for _ in range(3):
        v = rng.standard_normal((n_p,) * 3)
        fd = (adjoint.loss(c, n_p, n_mesh, box, ai, af, steps, w + eps * v, target)
              - adjoint.loss(c, n_p, n_mesh, box, ai, af, steps, w - eps * v, target)) / (2 * eps)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)


def test_gradient_vanishes_at_the_target():
    c = Cosmology()
    w = inputs.gaussian_field(4, 8)
    u, _, _, _ = adjoint.forward(c, 8, 16, 300.0, 0.2, 0.6, 3, w)
    L, g = adjoint.loss_and_grad(c, 8, 16, 300.0, 0.2, 0.6, 3, w, cic.density_contrast(u, 16))
    assert L < 1e-28 and np.max(np.abs(g)) < 1e-12


@pytest.mark.parametrize("n_p,n_mesh", [(8, 16), (16, 16)])
def test_vector_jacobian_product_of_density_and_displacements(n_p, n_mesh):
    # a loss that is not the MSE: L = sum_k W(k) |delta_k|^2 / N^6 (a power-spectrum weighted
    # norm of the final density) + sum_p g_p . d_p (the final displacements in Mpc/h); the
    # cotangents go into vjp and its product with random directions must equal the central
    # differences of the forward oracle itself
    c = Cosmology()
    box, ai, af, steps = 300.0, 0.2, 0.6, 4
    w = inputs.gaussian_field(5, n_p)
    r = np.random.default_rng(6)
    f = np.fft.fftfreq(n_mesh, 1.0 / n_mesh)
    K2 = f[:, None, None]**2 + f[None, :, None]**2 + f[None, None, :]**2
    Wk = 1.0 / (1.0 + K2)
    gdisp = r.standard_normal((3, n_p**3)) * 1e-3

    def L_of(ww):
        u, _, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, ww)
        dk = np.fft.fftn(cic.density_contrast(u, n_mesh))
        return float(np.sum(Wk * np.abs(dk)**2) / n_mesh**6 + np.sum(gdisp * adjoint.displacement(u, n_p, box)))

    u, _, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, w)
    dk = np.fft.fftn(cic.density_contrast(u, n_mesh))
    lam_delta = 2.0 * np.real(np.fft.ifftn(Wk * dk)) / n_mesh**3  # dL/d delta of the spectral norm
    g = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=lam_delta, lam_disp=gdisp)
    eps = 1e-5
    for _ in range(3):
        v = r.standard_normal((n_p,) * 3)
        fd = (L_of(w + eps * v) - L_of(w - eps * v)) / (2 * eps)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)
    # each cotangent alone: the products add up
    g1 = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=lam_delta)
    g2 = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_disp=gdisp)
    np.testing.assert_allclose(g1 + g2, g, rtol=0, atol=1e-12 * np.max(np.abs(g)))


def test_vector_jacobian_product_of_the_final_momenta():
    # L = sum_p h_p . p_p on the synchronised final momenta (after the closing half kick), alone
    # and with a displacement term: the reverse sweep starting from lam_p = h must equal the
    # central differences of the forward oracle; h = 0 gives the displacement term's gradient
    c = Cosmology()
    n_p, n_mesh = 8, 16
    box, ai, af, steps = 300.0, 0.2, 0.6, 4
    w = inputs.gaussian_field(7, n_p)
    r = np.random.default_rng(8)
    h = r.standard_normal((3, n_p**3)) * 1e-2
    gdisp = r.standard_normal((3, n_p**3)) * 1e-3

    def L_of(ww, with_disp):
        u, p, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, ww)
        extra = np.sum(gdisp * adjoint.displacement(u, n_p, box)) if with_disp else 0.0
        return float(np.sum(h * p) + extra)

    eps = 1e-5
    for with_disp in (False, True):
        g = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_disp=gdisp if with_disp else None, lam_mom=h)
        for _ in range(3):
            v = r.standard_normal((n_p,) * 3)
            fd = (L_of(w + eps * v, with_disp) - L_of(w - eps * v, with_disp)) / (2 * eps)
            assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)
    g0 = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_disp=gdisp, lam_mom=np.zeros_like(h))
    np.testing.assert_array_equal(g0, adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_disp=gdisp))


def _ics_of(c, n_p, box, a_i, w):
    """The Zel'dovich state the adjoint's forward map starts from (box units, Mpc/h)."""
    from oracle import ic
    psi = ic.za_displacement(ic.linear_delta_k(c, n_p, box, white_noise=w), n_p, box).reshape(3, -1)
    D, f, E = c.growth_D(a_i), c.growth_f(a_i), float(c.E(a_i))
    u = adjoint.lattice_fractions(n_p) + D * psi / box
    return u - np.floor(u), a_i**2 * E * f * D * psi


@pytest.mark.parametrize("gradient", [adjoint.SPECTRAL, adjoint.FD1])
@pytest.mark.parametrize("mode", [adjoint.NEWTON, adjoint.GR_POISSON])
def test_forward_map_is_the_oracle_run(mode, gradient):
    # the adjoint's own forward map (kept as a list of kicks and drifts) against oracle.pm's run
    # from the same ICs, Newtonian and Poisson gauge (20 Gpc/h, where the lag term matters),
    # spectral and first-order gradient
    from oracle import pm as opm
    c = Cosmology()
    n_p, n_mesh, box, ai, af, steps = 8, 16, 20000.0, 0.1, 0.5, 4
    w = inputs.gaussian_field(9, n_p)
    u, p, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, w, mode, gradient)
    u0, p0 = _ics_of(c, n_p, box, ai, w)
    run = opm.PMRun(c, n_mesh, box, ai, af, steps, u0, p0, mode=opm.GR_POISSON if mode else opm.NEWTON,
                    gradient=opm.FD1 if gradient else opm.SPECTRAL)
    run.step(steps)
    d = run.x - u
    assert np.max(np.abs(d - np.rint(d))) < 1e-13
    np.testing.assert_allclose(run.p, p, rtol=0, atol=1e-12 * np.max(np.abs(p)))


def test_growth_matched_stepping_forward_map_and_vector_jacobian_product():
    # with the growth-matched kick and drift factors: the adjoint's forward map equals oracle.pm's
    # run with the same factors, and its vector-Jacobian product for a loss of the final density,
    # displacements and momenta matches central differences of that map
    from oracle import pm as opm
    c = Cosmology()
    n_p, n_mesh, box, ai, af, steps = 8, 16, 1000.0, 0.05, 1.0, 4
    w = inputs.gaussian_field(12, n_p)
    u, p, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, w, stepping=opm.GROWTH)
    u0, p0 = _ics_of(c, n_p, box, ai, w)
    run = opm.PMRun(c, n_mesh, box, ai, af, steps, u0, p0, stepping=opm.GROWTH)
    run.step(steps)
    d = run.x - u
    assert np.max(np.abs(d - np.rint(d))) < 1e-13
    np.testing.assert_allclose(run.p, p, rtol=0, atol=1e-12 * np.max(np.abs(p)))
    r = np.random.default_rng(13)
    f = np.fft.fftfreq(n_mesh, 1.0 / n_mesh)
    Wk = 1.0 / (1.0 + f[:, None, None]**2 + f[None, :, None]**2 + f[None, None, :]**2)
    gdisp = r.standard_normal((3, n_p**3)) * 1e-3
    h = r.standard_normal((3, n_p**3)) * 1e-2

    def L_of(ww):
        uu, pp, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, ww, stepping=opm.GROWTH)
        dk = np.fft.fftn(cic.density_contrast(uu, n_mesh))
        return float(np.sum(Wk * np.abs(dk)**2) / n_mesh**6 + np.sum(gdisp * adjoint.displacement(uu, n_p, box))
                     + np.sum(h * pp))

    dk = np.fft.fftn(cic.density_contrast(u, n_mesh))
    lam_delta = 2.0 * np.real(np.fft.ifftn(Wk * dk)) / n_mesh**3
    g = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=lam_delta, lam_disp=gdisp, lam_mom=h,
                    stepping=opm.GROWTH)
    gi = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=lam_delta, lam_disp=gdisp, lam_mom=h)
    assert np.linalg.norm(g - gi) > 0.01 * np.linalg.norm(g)  # the factors matter for the gradient
    eps = 1e-5
    for _ in range(3):
        v = r.standard_normal((n_p,) * 3)
        fd = (L_of(w + eps * v) - L_of(w - eps * v)) / (2 * eps)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)


def test_poisson_gauge_vector_jacobian_product():
    # Poisson gauge at 20 Gpc/h (the lag term 3 calH / dtau is larger than k^2 on the low modes):
    # a loss of the final density, displacements and momenta; the reverse sweep with the carried
    # spectrum Z against central differences of the forward map, and far from the Newtonian
    # gradient of the same loss (so the Poisson-gauge chain is what is checked)
    c = Cosmology()
    n_p, n_mesh, box, ai, af, steps = 8, 16, 20000.0, 0.1, 0.5, 4
    w = inputs.gaussian_field(10, n_p)
    r = np.random.default_rng(11)
    f = np.fft.fftfreq(n_mesh, 1.0 / n_mesh)
    Wk = 1.0 / (1.0 + f[:, None, None]**2 + f[None, :, None]**2 + f[None, None, :]**2)
    gdisp = r.standard_normal((3, n_p**3)) * 1e-3
    h = r.standard_normal((3, n_p**3)) * 1e-2
    mode = adjoint.GR_POISSON

    def L_of(ww, m=mode):
        u, p, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, ww, m)
        dk = np.fft.fftn(cic.density_contrast(u, n_mesh))
        return float(np.sum(Wk * np.abs(dk)**2) / n_mesh**6 + np.sum(gdisp * adjoint.displacement(u, n_p, box))
                     + np.sum(h * p))

    def cotangents(m):
        u, _, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, w, m)
        dk = np.fft.fftn(cic.density_contrast(u, n_mesh))
        return 2.0 * np.real(np.fft.ifftn(Wk * dk)) / n_mesh**3

    g = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=cotangents(mode), lam_disp=gdisp, lam_mom=h,
                    mode=mode)
    eps = 1e-5
    for _ in range(3):
        v = r.standard_normal((n_p,) * 3)
        fd = (L_of(w + eps * v) - L_of(w - eps * v)) / (2 * eps)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)
    gn = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=cotangents(adjoint.NEWTON), lam_disp=gdisp,
                     lam_mom=h, mode=adjoint.NEWTON)
    assert np.linalg.norm(g - gn) > 0.05 * np.linalg.norm(g)


@pytest.mark.parametrize("mode,box", [(adjoint.NEWTON, 300.0), (adjoint.GR_POISSON, 20000.0)])
def test_first_order_gradient_vector_jacobian_product(mode, box):
    # the first-order gradient g = -grad interp(phi): the transposed chain is a scalar deposit with
    # the CIC derivative weights, the transposed potential map, and the interpolant's mixed second
    # derivatives for the direct term; a loss of the final density, displacements and momenta
    # against central differences of the forward map, and far from the spectral-gradient result
    c = Cosmology()
    n_p, n_mesh, ai, af, steps = 8, 16, 0.1 if mode else 0.2, 0.5 if mode else 0.6, 4
    w = inputs.gaussian_field(12, n_p)
    r = np.random.default_rng(13)
    f = np.fft.fftfreq(n_mesh, 1.0 / n_mesh)
    Wk = 1.0 / (1.0 + f[:, None, None]**2 + f[None, :, None]**2 + f[None, None, :]**2)
    gdisp = r.standard_normal((3, n_p**3)) * 1e-3
    h = r.standard_normal((3, n_p**3)) * 1e-2
    fd1 = adjoint.FD1

    def L_of(ww):
        u, p, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, ww, mode, fd1)
        dk = np.fft.fftn(cic.density_contrast(u, n_mesh))
        return float(np.sum(Wk * np.abs(dk)**2) / n_mesh**6 + np.sum(gdisp * adjoint.displacement(u, n_p, box))
                     + np.sum(h * p))

    def lam_delta(grad):
        u, _, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, w, mode, grad)
        dk = np.fft.fftn(cic.density_contrast(u, n_mesh))
        return 2.0 * np.real(np.fft.ifftn(Wk * dk)) / n_mesh**3

    g = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=lam_delta(fd1), lam_disp=gdisp, lam_mom=h,
                    mode=mode, gradient=fd1)
    # 20 Gpc/h: displacements far below a cell (1250 Mpc/h), so a larger eps crosses no CIC
    # boundary and keeps the differences above the rounding of the positions
    eps = 1e-4 if box > 10000.0 else 1e-5
    for _ in range(3):
        v = r.standard_normal((n_p,) * 3)
        fd = (L_of(w + eps * v) - L_of(w - eps * v)) / (2 * eps)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)
    gs = adjoint.vjp(c, n_p, n_mesh, box, ai, af, steps, w, lam_delta=lam_delta(adjoint.SPECTRAL), lam_disp=gdisp,
                     lam_mom=h, mode=mode, gradient=adjoint.SPECTRAL)
    assert np.linalg.norm(g - gs) > 0.01 * np.linalg.norm(g)
