"""GPU parity of the PM run: Zel'dovich ICs, density and potential, single steps,
a full Newtonian run (32^3 particles, 20 steps to z = 0) and the Poisson-gauge mode.

The oracle builds its own ICs from the same seed (Philox phases) or the same seeded
white noise; nothing it uses comes from the GPU.
"""
import numpy as np
import pytest

import inputs
from oracle import cic, gravity, ic, pm as opm, stats
from oracle.cosmology import Cosmology
from tests.gpu_util import lib, min_image, positions_box_units, rel_l2, ticks_to_host, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FP32, FP64 = 0, 1


def _run(pm, np_side, nmesh, box, a_i, a_f, steps, prec, mode=0, n_lo=0):
    cfg = pm.make_config(np_side, nmesh, box, a_i, a_f, steps, mode=mode, precision=prec, n_lo=n_lo)
    return pm.PMRun(cfg)


def _host_particles(run):
    x, p = run.particles()
    torch.cuda.synchronize()
    xh = ticks_to_host(x) if not run.fp64 else to_host(x)
    return xh.copy(), to_host(p).astype(np.float64).copy()


def _disp(x, np_side):
    """Displacement from the lattice node in box units (minimum image)."""
    q = ic.lattice_ticks(np_side).astype(np.float64) * 2.0**-32
    return min_image(positions_box_units(x) - q)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("source", ["philox", "white_noise", "paired", "fixed", "paired_fixed", "white_noise_fixed",
                                    "lpt2", "white_noise_lpt2", "paired_fixed_lpt2"])
def test_zeldovich_ic_matches_oracle(prec, source):
    pm = lib()
    np_side, nmesh, box, a_i = 32, 64, 1000.0, 1.0 / 51.0
    run = _run(pm, np_side, nmesh, box, a_i, 1.0, 10, prec)
    c = Cosmology()
    fixed = "fixed" in source
    order = 2 if source.endswith("lpt2") else 1
    kw = {"fixed_amplitude": fixed, "lpt_order": order}
    if source.startswith("white_noise"):
        w = inputs.gaussian_field(41, np_side)
        run.ic(white_noise=to_dev(w if prec == FP64 else w.astype(np.float32)), fixed=fixed, lpt_order=order)
        kw["white_noise"] = w if prec == FP64 else w.astype(np.float32).astype(np.float64)
    else:
        paired = source.startswith("paired")
        run.ic(seed=12345, paired=paired, fixed=fixed, lpt_order=order)
        kw["seed"] = 12345
        kw["paired"] = paired
    xg, pg = _host_particles(run)
    xo, po = ic.zeldovich(c, np_side, box, a_i, fixed=(prec == FP32), **kw)
    tol = 2e-6 if prec == FP32 else 1e-11
    assert rel_l2(_disp(xg, np_side), _disp(xo, np_side)) < tol
    assert rel_l2(pg, po) < tol
    assert run.state() == (0, a_i, True)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("np_side,nmesh", [(32, 32), (32, 64), (16, 64)])
def test_second_order_lpt_term_matches_oracle(prec, np_side, nmesh):
    # late start (a = 0.5, delta_rms ~ 0.2 per cell) so that D2 Psi2 is resolved in ticks:
    # the second-order part alone, x_2LPT - x_ZA and p_2LPT - p_ZA, against the oracle's
    pm = lib()
    box, a_i = 1000.0, 0.5
    run = _run(pm, np_side, nmesh, box, a_i, 1.0, 4, prec)
    c = Cosmology()
    out = []
    for order in (1, 2):
        run.ic(seed=77, lpt_order=order)
        out.append(_host_particles(run))
    (x1, p1), (x2, p2) = out
    xo1, po1 = ic.zeldovich(c, np_side, box, a_i, seed=77, fixed=(prec == FP32))
    xo2, po2 = ic.zeldovich(c, np_side, box, a_i, seed=77, fixed=(prec == FP32), lpt_order=2)
    dg = min_image(positions_box_units(x2) - positions_box_units(x1))
    do = min_image(positions_box_units(xo2) - positions_box_units(xo1))
    assert np.max(np.abs(do)) > 1e-4
    tol = 2e-3 if prec == FP32 else 1e-9
    assert rel_l2(dg, do) < tol
    assert rel_l2(p2 - p1, po2 - po1) < tol
    assert rel_l2(_disp(x2, np_side), _disp(xo2, np_side)) < (1e-5 if prec == FP32 else 1e-11)


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_density_and_potential_after_one_step(prec):
    pm = lib()
    np_side, nmesh, box, a_i, a_f, steps = 32, 64, 500.0, 0.1, 1.0, 10
    run = _run(pm, np_side, nmesh, box, a_i, a_f, steps, prec)
    run.ic(seed=5)
    run.step(1)
    delta_g = to_host(run.density()).astype(np.float64)
    phi_g = to_host(run.potential()).astype(np.float64)
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=5, fixed=(prec == FP32))
    ref = opm.PMRun(c, nmesh, box, a_i, a_f, steps, x0, p0)
    ref.step(1)
    delta_o = cic.density_contrast(ref.x, nmesh)
    phi_o = gravity.potential_mesh(gravity.newton_potential_k(np.fft.rfftn(delta_o), nmesh, box, c.omega_m), nmesh)
    tol = 1e-5 if prec == FP32 else 1e-11
    assert rel_l2(delta_g, delta_o) < tol
    assert rel_l2(phi_g, phi_o) < tol
    xg, pg = _host_particles(run)
    assert rel_l2(min_image(positions_box_units(xg) - positions_box_units(x0)),
                  min_image(positions_box_units(ref.x) - positions_box_units(x0))) < tol
    assert rel_l2(pg, ref.p) < tol


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_full_run_power_spectrum(prec):
    # 32^3 particles on a 32^3 mesh, L = 2000 Mpc/h, ZA at z = 50, 20 KDK steps to z = 0,
    # P(k) in 16 log bins on [k_f, k_Ny].
    pm = lib()
    np_side = nmesh = 32
    box, a_i, a_f, steps = 2000.0, 1.0 / 51.0, 1.0, 20
    run = _run(pm, np_side, nmesh, box, a_i, a_f, steps, prec)
    run.ic(seed=1)
    run.step(steps)
    st = run.state()
    assert st[0] == steps and st[1] == pytest.approx(a_f, abs=1e-15) and st[2]
    edges = stats.log_edges(16, 1.0, nmesh / 2.0)
    kg, pg, ng = run.power(edges)
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=1, fixed=(prec == FP32))
    ref = opm.PMRun(c, nmesh, box, a_i, a_f, steps, x0, p0)
    ref.step(steps)
    ko, po, no = stats.power_spectrum(cic.density_contrast(ref.x, nmesh), box, edges)
    np.testing.assert_array_equal(ng, no)
    ok = no > 0
    # FP32 measured: P(k) 5.9e-6, positions within 3.1e-5 Mpc/h of the FP64 run's
    assert np.max(np.abs(pg[ok] / po[ok] - 1)) < (1e-4 if prec == FP32 else 1e-9)
    assert np.max(np.abs(kg[ok] / ko[ok] - 1)) < 1e-12
    xg, pgm = _host_particles(run)
    assert np.max(np.abs(min_image(positions_box_units(xg) - positions_box_units(ref.x)))) * box < \
        (1e-3 if prec == FP32 else 1e-8)
    # momentum is conserved by the CIC + symmetric Green's function + odd gradient
    assert np.max(np.abs(pgm.sum(axis=1) - p0.sum(axis=1))) < (1e-4 if prec == FP32 else 1e-9) * np.abs(pgm).sum()


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_growth_matched_stepping_matches_oracle(prec):
    # PM_STEP_GROWTH: kick and drift factors exact for the linear growing mode (the force of a
    # step taken at a_n, its drift's momenta at a_{n+1/2}); 32^3 particles on a 32^3 mesh,
    # L = 2000 Mpc/h, ZA at z = 50, 6 steps to z = 0, against the oracle's run with the same factors
    pm = lib()
    np_side = nmesh = 32
    box, a_i, a_f, steps = 2000.0, 1.0 / 51.0, 1.0, 6
    run = pm.PMRun(pm.make_config(np_side, nmesh, box, a_i, a_f, steps, precision=prec,
                                  stepping=pm.PM_STEP_GROWTH))
    run.ic(seed=1)
    run.step(steps)
    assert run.state()[2]
    edges = stats.log_edges(16, 1.0, nmesh / 2.0)
    kg, pg, ng = run.power(edges)
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=1, fixed=(prec == FP32))
    ref = opm.PMRun(c, nmesh, box, a_i, a_f, steps, x0, p0, stepping=opm.GROWTH)
    ref.step(steps)
    plain = opm.PMRun(c, nmesh, box, a_i, a_f, steps, x0, p0)
    plain.step(steps)
    ko, po, no = stats.power_spectrum(cic.density_contrast(ref.x, nmesh), box, edges)
    ok = no > 0
    assert np.max(np.abs(pg[ok] / po[ok] - 1)) < (1e-4 if prec == FP32 else 1e-9)
    xg, pgm = _host_particles(run)
    d = lambda u, v: min_image(positions_box_units(u) - positions_box_units(v))
    dref = d(ref.x, x0)
    assert rel_l2(d(xg, x0), dref) < (1e-4 if prec == FP32 else 1e-10)
    assert rel_l2(pgm, ref.p) < (1e-4 if prec == FP32 else 1e-10)
    assert rel_l2(d(plain.x, x0), dref) > 1e-3  # the plain integrals' six steps differ


def test_stepping_past_the_grid_is_refused():
    pm = lib()
    run = _run(pm, 16, 16, 100.0, 0.5, 1.0, 2, FP32)
    run.ic(seed=3)
    run.step(2)
    with pytest.raises(pm.PMError) as e:
        run.step(1)
    assert e.value.status == 7


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_poisson_gauge_run_matches_oracle(prec):
    # horizon-scale box (L = 20 Gpc/h, 16^3 particles on a 32^3 mesh, z = 100 -> 1): the GR run
    # departs from the Newtonian one; both sides solve the lagged linear constraint.
    pm = lib()
    np_side, nmesh, box, a_i, a_f, steps = 16, 32, 20000.0, 1.0 / 101.0, 1.0, 12
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=21, fixed=(prec == FP32))
    ref_gr = opm.PMRun(c, nmesh, box, a_i, a_f, steps, x0, p0, mode=opm.GR_POISSON)
    ref_gr.step(steps)
    ref_n = opm.PMRun(c, nmesh, box, a_i, a_f, steps, x0, p0, mode=opm.NEWTON)
    ref_n.step(steps)
    out = {}
    for mode, n_lo in ((1, 4), (1, 0), (0, 0)):
        run = _run(pm, np_side, nmesh, box, a_i, a_f, steps, prec, mode=mode, n_lo=n_lo)
        run.ic(seed=21)
        run.step(steps)
        out[(mode, n_lo)] = _host_particles(run)
    xi_o = min_image(positions_box_units(ref_gr.x) - positions_box_units(ref_n.x))
    assert np.max(np.abs(xi_o)) * box > 1e-3  # the GR displacement is not negligible here
    for key in ((1, 4), (1, 0)):
        xg, pg = out[key]
        xn, _ = out[(0, 0)]
        xi_g = min_image(positions_box_units(xg) - positions_box_units(xn))
        # xi is the difference of two runs, so FP32 rounding in either shows up relative to the
        # difference: measured 1.0e-3 in FP32 on this 20 Gpc/h box (the same with and without the
        # FP64 island; 6.2e-3 while the forward transform carried the density's mean), roundoff
        # in FP64
        assert rel_l2(xi_g, xi_o) < (3e-3 if prec == FP32 else 1e-9)
        d_g = min_image(positions_box_units(xg) - positions_box_units(x0))
        d_o = min_image(positions_box_units(ref_gr.x) - positions_box_units(x0))
        # FP32 stores rho ~ 1 + delta and resolves delta to ~6e-8; with delta ~ 1e-4 on these
        # 625 Mpc/h cells at z = 100 the FP32 forces, hence displacements, carry ~1e-3 errors
        # (measured 4.2e-4)
        assert rel_l2(d_g, d_o) < (1e-3 if prec == FP32 else 1e-11)


@pytest.mark.slow
def test_poisson_gauge_pair_at_the_horizon_scale_configuration():
    # the paired runs of the horizon-scale configuration at the same cell size on a 64^3 lattice:
    # 64^3 particles on a 128^3 mesh, L = 4000 Mpc/h, ZA at z = 100, 20 steps to z = 0; xi^GR of
    # the FP32 runs within 1e-4 of the FP64 oracle's for n_lo = 0, 4 and 16 (measured 1.3e-5
    # each, displacements 4.9e-6)
    pm = lib()
    np_side, nmesh, box, a_i, steps = 64, 128, 4000.0, 1.0 / 101.0, 20
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=1, fixed=True)
    ref = {}
    for mode in (opm.GR_POISSON, opm.NEWTON):
        r = opm.PMRun(c, nmesh, box, a_i, 1.0, steps, x0, p0, mode=mode)
        r.step(steps)
        ref[mode] = positions_box_units(r.x)
    xi_o = min_image(ref[opm.GR_POISSON] - ref[opm.NEWTON])
    d_o = min_image(ref[opm.GR_POISSON] - positions_box_units(x0))
    assert np.linalg.norm(xi_o) > 0.1 * np.linalg.norm(d_o)  # a horizon-scale effect, not roundoff
    newton = _run(pm, np_side, nmesh, box, a_i, 1.0, steps, FP32)
    newton.ic(seed=1)
    newton.step(steps)
    xn, _ = _host_particles(newton)
    for n_lo in (0, 4, 16):
        gr = _run(pm, np_side, nmesh, box, a_i, 1.0, steps, FP32, mode=1, n_lo=n_lo)
        gr.ic(seed=1)
        gr.step(steps)
        xg, _ = _host_particles(gr)
        xi_g = min_image(positions_box_units(xg) - positions_box_units(xn))
        assert rel_l2(xi_g, xi_o) < 1e-4
        d_g = min_image(positions_box_units(xg) - positions_box_units(x0))
        assert rel_l2(d_g, d_o) < 2e-5


@pytest.mark.parametrize("prec,np_side,nmesh", [(FP32, 32, 32), (FP32, 32, 64), (FP32, 64, 64), (FP32, 16, 64),
                                                (FP64, 32, 32), (FP64, 16, 32)])
@pytest.mark.parametrize("mode", [0, 1])
def test_first_order_gradient_run_matches_oracle(prec, np_side, nmesh, mode):
    # PM_GRAD_FD1: the force is the gradient of the CIC interpolant of the potential (one
    # inverse transform; the update gathers the potential's eight corners).  Covers the
    # unfused update (nmesh 32), the fused row sweep (64/64) and the fused tiles (32/64, 16/64).
    pm = lib()
    box, a_i, a_f, steps = 500.0 if mode == 0 else 20000.0, 0.1, 1.0, 10
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=31, fixed=(prec == FP32))
    ref = opm.PMRun(c, nmesh, box, a_i, a_f, steps, x0, p0, mode=mode, gradient=opm.FD1)
    ref.step(3)
    cfg = pm.make_config(np_side, nmesh, box, a_i, a_f, steps, mode=mode, precision=prec, gradient=pm.PM_GRAD_FD1)
    run = pm.PMRun(cfg)
    run.ic(seed=31)
    run.step(3)
    xg, pg = _host_particles(run)
    d_g = min_image(positions_box_units(xg) - positions_box_units(x0))
    d_o = min_image(positions_box_units(ref.x) - positions_box_units(x0))
    # FP32 on the 20 Gpc/h box: rho ~ 1 + delta with delta ~ 1e-4 per cell carries ~1e-3
    # relative density errors (as in the Poisson-gauge run test)
    tol = (1e-4 if mode == 0 else 3e-3) if prec == FP32 else 1e-10
    assert rel_l2(d_g, d_o) < tol
    assert rel_l2(pg, ref.p) < tol
    # and it is not the spectral force
    spec = _run(pm, np_side, nmesh, box, a_i, a_f, steps, prec, mode=mode)
    spec.ic(seed=31)
    spec.step(3)
    _, ps = _host_particles(spec)
    assert rel_l2(pg, ps) > 1e-3


def test_first_order_gradient_is_refused_by_batches_and_the_fp64_gradient():
    # batches keep the spectral force; the loss gradient takes the first-order force in FP32
    # (checked against the oracle in test_gpu_adjoint.py) and refuses FP64 contexts
    pm = lib()
    cfg = pm.make_config(32, 64, 500.0, 0.1, 1.0, 4, gradient=pm.PM_GRAD_FD1)
    with pytest.raises(pm.PMError) as e:
        pm.PMBatch(cfg, boxes=[500.0, 600.0])
    assert e.value.status == 1
    w = to_dev(inputs.gaussian_field(3, 32).astype(np.float32))
    target = torch.zeros((64, 64, 64), dtype=torch.float32, device="cuda")
    L, g = pm.PMRun(cfg).loss_grad(w, target)
    assert np.isfinite(L) and L > 0 and torch.isfinite(g).all()
    run64 = pm.PMRun(pm.make_config(32, 64, 500.0, 0.1, 1.0, 4, precision=pm.PM_FP64))
    with pytest.raises(pm.PMError) as e:
        run64.loss_grad(w, target)
    assert e.value.status == 6


@pytest.mark.parametrize("in_place", [False, True])
def test_set_state_resumes_a_run_where_it_was_saved(in_place):
    # a snapshot (x, p, step, synchronised) taken between steps and restored into a fresh
    # context continues as the original run: the same integrator position and the same
    # particles after the remaining steps (up to the summation order of the deposit atomics);
    # in_place: the snapshot is written into the context's own arrays (pm_particles) and
    # pm_set_state, handed those arrays, copies nothing
    pm = lib()
    np_side = nmesh = 64
    box, steps, k = 1000.0, 40, 25
    runs = [pm.PMRun(pm.make_config(np_side, nmesh, box, 1.0 / 51.0, 1.0, steps)) for _ in range(2)]
    a, b = runs
    b.ic(seed=10)  # other particles, overwritten by the snapshot
    a.ic(seed=9)
    a.step(k)
    st = a.state()
    assert st[0] == k and not st[2]
    x, p = (t.clone() for t in a.particles())
    if in_place:
        xb0, pb0 = b.particles()
        xb0.copy_(x)
        pb0.copy_(p)
        pm.pm_set_state(b.ctx, xb0, pb0, st[0], st[2])
    else:
        pm.pm_set_state(b.ctx, x, p, st[0], st[2])
    assert b.state() == st
    a.step(steps - k)
    b.step(steps - k)
    assert a.state() == b.state() and a.state()[2]
    xa, pa = _host_particles(a)
    xb, pb = _host_particles(b)
    da = min_image(positions_box_units(xa) - positions_box_units(x.cpu().numpy().view(np.uint32)))
    db = min_image(positions_box_units(xb) - positions_box_units(x.cpu().numpy().view(np.uint32)))
    assert rel_l2(db, da) < 1e-5
    assert rel_l2(pb, pa) < 1e-5


def test_set_state_checks_its_arguments():
    pm = lib()
    run = _run(pm, 16, 16, 100.0, 0.5, 1.0, 4, FP32)
    run.ic(seed=3)
    x, p = (t.clone() for t in run.particles())
    for step, sync in ((5, 1), (-1, 1), (0, 0), (4, 0)):
        with pytest.raises(pm.PMError) as e:
            pm.pm_set_state(run.ctx, x, p, step, sync)
        assert e.value.status == 1
    gr = _run(pm, 16, 16, 20000.0, 0.5, 1.0, 4, FP32, mode=1)
    with pytest.raises(pm.PMError) as e:
        pm.pm_set_state(gr.ctx, x, p, 2, 0)
    assert e.value.status == 6
    pm.pm_set_state(gr.ctx, x, p, 0, 1)


@pytest.mark.parametrize("bad", [1.0, 1.5, -1e-3, float("nan"), float("inf")])
def test_fp64_positions_outside_the_box_are_refused(bad):
    # FP64 positions are box fractions in [0, 1): anything else is outside the mesh's bounds
    pm = lib()
    run = _run(pm, 16, 16, 100.0, 0.5, 1.0, 4, FP64)
    run.ic(seed=3)
    run.step(1)
    x, p = (t.clone() for t in run.particles())
    x[1, 77] = bad
    with pytest.raises(pm.PMError) as e:
        pm.pm_set_particles(run.ctx, x, p)
    assert e.value.status == 5
    with pytest.raises(pm.PMError) as e:
        pm.pm_set_state(run.ctx, x, p, 2, 0)
    assert e.value.status == 5
    assert run.state()[0] == 1  # nothing was taken over
    x[1, 77] = 0.25
    pm.pm_set_particles(run.ctx, x, p)
    assert run.state()[0] == 0


@pytest.mark.parametrize("precision", ["fp32", "fp64"])
def test_positions_in_mpc(precision):
    # pm_positions: ticks times L / 2^32 rounded down to float (FP32), fractions times L (FP64),
    # bit for bit; all in [0, L)
    pm = lib()
    prec = pm.PM_FP32_FIXED if precision == "fp32" else pm.PM_FP64
    box = 700.0
    run = pm.PMRun(pm.make_config(16, 32, box, 0.1, 1.0, 6, precision=prec))
    run.ic(seed=5)
    run.step(4)
    pos = to_host(run.positions())
    x = to_host(run.particles()[0])
    if precision == "fp32":
        exact = x.view(np.uint32).astype(np.float64) * (box / 2.0**32)
        want = exact.astype(np.float32)
        up = want.astype(np.float64) > exact  # rounded up to nearest: one float below
        want[up] = np.nextafter(want[up], np.float32(-np.inf))
    else:
        want = x * box
    assert pos.dtype == want.dtype and np.array_equal(pos, want)
    assert pos.min() >= 0.0 and pos.max() < box


@pytest.mark.parametrize("n_lo", [0, 4])
def test_poisson_gauge_run_resumes_from_a_snapshot_with_its_history(n_lo):
    # a Poisson-gauge snapshot between steps (particles, integrator state, Phi_old and the FP64
    # island) restored into a fresh context with pm_set_state_gr continues as the original run;
    # without the history pm_set_state refuses it, and a run resumed with a wrong (zero) history
    # departs from the original
    pm = lib()
    cfg = pm.make_config(32, 64, 8000.0, 0.02, 1.0, 12, mode=1, n_lo=n_lo)
    a = pm.PMRun(cfg)
    a.ic(seed=4)
    a.step(7)
    x, p = (t.clone() for t in a.particles())
    step, _, synced = a.state()
    phi, island = a.gr_history()
    a.step(5)
    xa, pa = _host_particles(a)
    b = pm.PMRun(cfg)
    with pytest.raises(pm.PMError) as e:
        pm.pm_set_state(b.ctx, x, p, step, synced)
    assert e.value.status == 6
    pm.pm_set_state_gr(b.ctx, x, p, step, synced, phi, island)
    b.step(5)
    xb, pb = _host_particles(b)
    x0 = ticks_to_host(x).copy()
    assert rel_l2(_disp(xb, 32) - _disp(x0, 32), _disp(xa, 32) - _disp(x0, 32)) < 1e-5
    assert rel_l2(pb, pa) < 1e-5
    z = pm.PMRun(cfg)
    pm.pm_set_state_gr(z.ctx, x, p, step, synced, torch.zeros_like(phi),
                       None if island is None else torch.zeros_like(island))
    z.step(5)
    _, pz = _host_particles(z)
    assert rel_l2(pz, pa) > 1e-3
