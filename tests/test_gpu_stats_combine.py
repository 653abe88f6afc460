"""GPU parity of the estimators (P(k), B(k)) and the GR displacement combination."""
import numpy as np
import pytest

import inputs
from oracle import cic, combine, ic, pm as opm, stats
from oracle.cosmology import Cosmology
from tests.gpu_util import bk_abs_scale, lib, min_image, positions_box_units, ticks_to_host, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FP32, FP64 = 0, 1


def _ctx(pm, np_side, nmesh, box, prec, mode=0, steps=4, a_i=0.1, a_f=1.0):
    return pm.PMRun(pm.make_config(np_side, nmesh, box, a_i, a_f, steps, mode=mode, precision=prec))


def _field(f, prec):
    return to_dev(f.astype(np.float64 if prec == FP64 else np.float32))


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("deconv", [True, False])
def test_power_of_fields_auto_and_cross(prec, deconv):
    pm = lib()
    n, box = 64, 1500.0
    run = _ctx(pm, 16, n, box, prec)
    f1 = inputs.lognormal_field(51, n, sigma=0.9)
    f2 = 0.5 * f1 + inputs.gaussian_field(52, n)
    cast = (lambda a: a) if prec == FP64 else (lambda a: a.astype(np.float32).astype(np.float64))
    edges = stats.log_edges(20, 1.0, n / 2.0)
    k, p, nm = run.power(edges, field=_field(f1, prec), deconvolve=deconv)
    ko, po, no = stats.power_spectrum(cast(f1), box, edges, deconvolve=deconv)
    np.testing.assert_array_equal(nm, no)
    tol = 2e-6 if prec == FP32 else 1e-12
    np.testing.assert_allclose(p, po, rtol=tol)
    np.testing.assert_allclose(k, ko, rtol=1e-13)
    k, p, nm = run.power(edges, field=_field(f1, prec), field2=_field(f2, prec), deconvolve=deconv)
    _, po, _ = stats.power_spectrum(cast(f1), box, edges, deconvolve=deconv, delta2=cast(f2))
    np.testing.assert_allclose(p, po, rtol=10 * tol)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_power_of_particles_and_empty_bins(prec):
    pm = lib()
    np_side, n, box = 32, 64, 800.0
    run = _ctx(pm, np_side, n, box, prec)
    x = inputs.lattice_order_ticks(53, np_side, 2.0, n_mesh=n)
    xs = x if prec == FP32 else inputs.ticks_to_fractions(x)
    p = inputs.momenta(54, np_side**3, 10.0)
    pm.pm_set_particles(run.ctx, to_dev(xs), _field(p, prec))
    edges = np.array([0.1, 0.5, 1.0, 3.0, 8.0, 32.0, 40.0])  # first two bins hold no mode
    k, pg, ng = run.power(edges)
    ko, po, no = stats.power_spectrum(cic.density_contrast(xs, n), box, edges)
    np.testing.assert_array_equal(ng, no)
    assert np.isnan(pg[0]) and np.isnan(pg[1]) and ng[0] == 0
    ok = no > 0
    # FP32 atomics sum the CIC weights in arbitrary order: density-level 1e-5 tolerance
    np.testing.assert_allclose(pg[ok], po[ok], rtol=1e-5 if prec == FP32 else 1e-12)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_bispectrum_matches_oracle(prec):
    pm = lib()
    n, box, m = 32, 1000.0, 64
    run = _ctx(pm, 16, n, box, prec)
    f = inputs.lognormal_field(55, n, sigma=0.8)
    edges = np.linspace(0.5, 15.0, 9)  # 8 bins up to |n| = 15 -> alias free on m = 64 (3 * 15 < 64)
    b, nt = run.bispectrum(edges, m, field=_field(f, prec))
    cast = f if prec == FP64 else f.astype(np.float32).astype(np.float64)
    tri, bo, nto = stats.bispectrum(cast, box, edges, M=m)
    assert len(b) == len(bo) == 120
    np.testing.assert_array_equal(nt, nto)  # integer counts of configurations
    ok = nto > 0
    assert np.array_equal(np.isnan(b), ~ok)
    # every triangle against the absolute sum of its terms, and relative to B itself where the
    # sum does not cancel below 1% of that scale
    sc = bk_abs_scale(cast, box, edges, m)
    tol = 1e-4 if prec == FP32 else 1e-10
    assert np.all(np.abs(b[ok] - bo[ok]) <= tol * sc[ok])
    big = ok & (np.abs(bo) > 1e-2 * sc)
    np.testing.assert_allclose(b[big], bo[big], rtol=1e-3 if prec == FP32 else 1e-9)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_bispectrum_many_bins_matches_oracle(prec):
    # 20 bins: triangles (i, j, l) span three blocks of eight l's, with partial first and last
    # blocks, as in the 24-bin estimator of the benchmark
    pm = lib()
    n, box, m = 64, 2000.0, 64
    run = _ctx(pm, 16, n, box, prec)
    f = inputs.lognormal_field(57, n, sigma=0.6)
    edges = np.linspace(0.5, 20.5, 21)  # |n| <= 20 -> alias free on m = 64 (3 * 20 < 64)
    b, nt = run.bispectrum(edges, m, field=_field(f, prec))
    cast = f if prec == FP64 else f.astype(np.float32).astype(np.float64)
    tri, bo, nto = stats.bispectrum(cast, box, edges, M=m)
    assert len(b) == len(bo) == 20 * 21 * 22 // 6
    np.testing.assert_array_equal(nt, nto)
    ok = nto > 0
    assert np.array_equal(np.isnan(b), ~ok)
    sc = bk_abs_scale(cast, box, edges, m)
    assert np.all(np.abs(b[ok] - bo[ok]) <= (1e-4 if prec == FP32 else 1e-10) * sc[ok])
    big = ok & (np.abs(bo) > 1e-2 * sc)
    np.testing.assert_allclose(b[big], bo[big], rtol=1e-3 if prec == FP32 else 1e-9)


def test_bispectrum_refuses_aliasing_grid():
    pm = lib()
    run = _ctx(pm, 16, 32, 1000.0, FP32)
    f = _field(inputs.gaussian_field(56, 32), FP32)
    with pytest.raises(pm.PMError) as e:
        run.bispectrum(np.linspace(0.5, 15.0, 5), 32, field=f)
    assert e.value.status == 1


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("ratio", [1, 2, 4])
def test_displacement_correction_exact(prec, ratio):
    pm = lib()
    nc = 16
    nt = nc * ratio
    box = 1000.0
    gr, newton = _ctx(pm, nc, nc, box, prec), _ctx(pm, nc, nc, box, prec)
    target = _ctx(pm, nt, nt, box, prec)
    xg = inputs.lattice_order_ticks(61, nc, 1.0)
    xn = inputs.lattice_order_ticks(62, nc, 1.0)
    xt = inputs.lattice_order_ticks(63, nt, 1.0)
    if prec == FP64:
        xg, xn, xt = (inputs.ticks_to_fractions(a) for a in (xg, xn, xt))
    zero_c = _field(np.zeros((3, nc**3)), prec)
    pm.pm_set_particles(gr.ctx, to_dev(xg), zero_c)
    pm.pm_set_particles(newton.ctx, to_dev(xn), zero_c)
    pm.pm_set_particles(target.ctx, to_dev(xt), _field(np.zeros((3, nt**3)), prec))
    xi = torch.empty((3, nt**3), dtype=torch.float64 if prec == FP64 else torch.int32, device="cuda")
    pm.pm_displacement_correction(target.ctx, gr.ctx, newton.ctx, xi)
    x_out, _ = target.particles()
    torch.cuda.synchronize()
    xi_o = combine.interpolate_lagrangian(combine.displacement(xg, xn), nc, nt)
    want = combine.combine(xt, xi_o)
    if prec == FP32:
        np.testing.assert_array_equal(to_host(xi), xi_o)
        np.testing.assert_array_equal(ticks_to_host(x_out), want)
    else:
        assert np.max(np.abs(to_host(xi) - xi_o)) < 1e-16
        assert np.max(np.abs(min_image(to_host(x_out) - want))) < 1e-15


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_paired_gr_newton_combination_pipeline(prec):
    # Eqs. xiGR and combined end to end on a horizon-scale box: a 16^3 GR/Newton pair from one
    # seed corrects a 32^3 Newtonian run of the same seed.
    pm = lib()
    box, a_i, a_f, steps = 20000.0, 1.0 / 51.0, 1.0, 8
    c = Cosmology()
    runs = {}
    for name, npd, mode in (("gr", 16, 1), ("n", 16, 0), ("t", 32, 0)):
        r = pm.PMRun(pm.make_config(npd, 2 * npd, box, a_i, a_f, steps, mode=mode, precision=prec, n_lo=2))
        r.ic(seed=77)
        r.step(steps)
        runs[name] = r
    pm.pm_displacement_correction(runs["t"].ctx, runs["gr"].ctx, runs["n"].ctx)
    xg, _ = runs["t"].particles()
    torch.cuda.synchronize()
    xg = ticks_to_host(xg) if prec == FP32 else to_host(xg)
    ref = {}
    for name, npd, mode in (("gr", 16, opm.GR_POISSON), ("n", 16, opm.NEWTON), ("t", 32, opm.NEWTON)):
        x0, p0 = ic.zeldovich(c, npd, box, a_i, seed=77, fixed=(prec == FP32))
        r = opm.PMRun(c, 2 * npd, box, a_i, a_f, steps, x0, p0, mode=mode)
        r.step(steps)
        ref[name] = r.x
    xi = combine.interpolate_lagrangian(combine.displacement(ref["gr"], ref["n"]), 16, 32)
    want = combine.combine(ref["t"], xi)
    d_g = min_image(positions_box_units(xg) - positions_box_units(ref["t"]))
    d_o = min_image(positions_box_units(want) - positions_box_units(ref["t"]))
    # FP32: the GR displacement is a difference of two FP32 runs (~0.5% relative noise)
    assert np.linalg.norm(d_g - d_o) < (2e-2 if prec == FP32 else 1e-9) * np.linalg.norm(d_o)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_paired_fixed_bispectrum_slices_match_oracle(prec):
    # Sec. 4.2: B(k) averaged over a paired-and-fixed pair of Zel'dovich ICs, reported on
    # the equilateral and the squeezed (k3 = 4 k_f) triangles of the table
    pm = lib()
    np_side, n, box, m, a_i = 32, 32, 1000.0, 64, 0.5
    run = _ctx(pm, np_side, n, box, prec, a_i=a_i)
    edges = np.arange(0.5, 16.0, 1.0)       # unit-width shells centred on |n| = 1..15
    nb = len(edges) - 1
    k3_bin = int(np.searchsorted(edges, 4.0)) - 1
    assert edges[k3_bin] < 4.0 < edges[k3_bin + 1]
    c = Cosmology()
    got, want, scale = [], [], 0.0
    for paired in (False, True):
        run.ic(seed=21, paired=paired, fixed=True)
        b, nt = run.bispectrum(edges, m)
        x, _ = ic.zeldovich(c, np_side, box, a_i, seed=21, paired=paired, fixed=(prec == FP32),
                            fixed_amplitude=True)
        _, bo, nto = stats.bispectrum(cic.density_contrast(x, n), box, edges, M=m)
        np.testing.assert_allclose(nt, nto, rtol=1e-5 if prec == FP32 else 1e-12, atol=0.1 if prec == FP32 else 1e-6)
        got.append(b)
        want.append(bo)
        scale = max(scale, np.nanmax(np.abs(bo)))
    ok = nto > 0
    b_avg, bo_avg = 0.5 * (got[0] + got[1]), 0.5 * (want[0] + want[1])
    assert np.array_equal(np.isnan(b_avg), ~ok)
    # the pair average cancels the leading (Gaussian) part: tolerances against the single-run scale
    tol = (2e-4 if prec == FP32 else 1e-9) * scale
    assert np.max(np.abs(b_avg[ok] - bo_avg[ok])) < tol
    eq, sq = pm.bispectrum_configurations(nb, k3_bin)
    tri = stats.triangles(nb)
    assert [tri[t] for t in sq] == [(k3_bin, j, j) for j in range(k3_bin, nb)]
    for rows in (eq, sq):
        live = ok[rows]
        assert live.sum() >= 3
        assert np.max(np.abs(b_avg[rows][live] - bo_avg[rows][live])) < tol


@pytest.mark.parametrize("np_side,n", [(64, 64), (32, 64), (32, 32)])
def test_power_after_a_step_reuses_the_step_density(np_side, n):
    # after a step P(k) of the particles and the potential transform the density the update
    # left in rho (fused update), or a deposit made once (unfused); the same numbers as a
    # fresh deposit of the same positions, up to FP32 summation order
    pm = lib()
    run = _ctx(pm, np_side, n, 800.0, FP32, steps=6)
    run.ic(seed=44)
    run.step(2)
    edges = stats.log_edges(12, 1.0, n / 2.0)
    _, p_step, nm = run.power(edges)
    phi_step = torch.empty((n, n, n), dtype=torch.float32, device="cuda")
    pm.pm_potential(run.ctx, phi_step)
    _, p_again, _ = run.power(edges)
    x, p = run.particles()
    xs, ps = x.clone(), p.clone()
    pm.pm_set_particles(run.ctx, xs, ps)
    _, p_fresh, nm2 = run.power(edges)
    phi_fresh = torch.empty_like(phi_step)
    pm.pm_potential(run.ctx, phi_fresh)
    np.testing.assert_array_equal(nm, nm2)
    ok = nm > 0
    np.testing.assert_allclose(p_step[ok], p_fresh[ok], rtol=1e-5)
    np.testing.assert_allclose(p_step[ok], p_again[ok], rtol=1e-12)  # FP64 bin sums, any order
    d = (phi_step - phi_fresh).double().norm() / phi_fresh.double().norm()
    assert float(d) < 1e-5
