"""The fused middle passes of the force evaluation (forward y, x with the Green's function or
the Poisson-gauge constraint, inverse y, in one persistent launch over the kz planes) against
the three separate passes and against the FP64 oracle, on the mesh sizes that use them
(FP32, 256^3 and up)."""
import numpy as np
import pytest

from oracle import cic, gravity, ic
from oracle.cosmology import Cosmology
from tests.gpu_util import lib, rel_l2, to_host, torch

pytestmark = pytest.mark.gpu


def _kicks(pm, cfg, seed, steps, threads):
    run = pm.PMRun(cfg)
    pm.pm_set_fused_fft(run.ctx, threads)
    run.ic(seed=seed)
    _, p = run.particles()
    p0 = p.to(torch.float64).clone()
    run.step(steps)
    _, p = run.particles()
    dp = (p.to(torch.float64) - p0).cpu().numpy()
    x = run.density().cpu().numpy()
    del run
    torch.cuda.empty_cache()
    return dp, x


@pytest.mark.parametrize("mode,n_lo", [(0, 0), (1, 4)])
@pytest.mark.parametrize("np_side,nmesh", [(128, 256), (256, 256), (256, 512)])
def test_fused_middle_passes_equal_the_separate_passes(mode, n_lo, np_side, nmesh):
    # the same butterflies, twiddles and per-mode operator in either form and for every CTA size:
    # the runs differ only by the summation order of the deposit's float atomics (~1e-7 of the density)
    pm = lib()
    box = 2000.0 if mode == 0 else 8000.0
    cfg = pm.make_config(np_side, nmesh, box, 1.0 / 51.0, 1.0, 20, mode=mode, n_lo=n_lo)
    dps, ds = _kicks(pm, cfg, 4, 3, 0)
    assert np.max(np.abs(dps)) > 0
    for threads in (256, 512, 1024):
        dpf, df = _kicks(pm, cfg, 4, 3, threads)
        assert rel_l2(dpf, dps) < 1e-5
        assert rel_l2(df, ds) < 1e-5


def test_fft_autotuner_keeps_a_candidate_and_the_run_goes_on():
    pm = lib()
    run = pm.PMRun(pm.make_config(128, 256, 2000.0, 1.0 / 51.0, 1.0, 20))
    run.ic(seed=2)
    run.step(2)
    threads, ms = pm.pm_autotune_fft(run.ctx)
    assert threads in (0, 256, 512, 1024) and ms > 0
    run.step(1)  # the tuning touched only the spectrum buffers
    ref = pm.PMRun(pm.make_config(128, 256, 2000.0, 1.0 / 51.0, 1.0, 20))
    ref.ic(seed=2)
    ref.step(3)
    xa, pa = run.particles()
    xb, pb = ref.particles()
    assert rel_l2(to_host(pa).astype(np.float64), to_host(pb).astype(np.float64)) < 1e-5
    small = pm.PMRun(pm.make_config(16, 32, 500.0, 0.1, 1.0, 4))
    assert pm.pm_autotune_fft(small.ctx) == (0, 0.0)  # no other form applies to a 32^3 mesh
    with pytest.raises(pm.PMError):
        pm.pm_set_fused_fft(run.ctx, 128)


@pytest.mark.slow
def test_fused_force_of_one_step_matches_the_oracle():
    # 128^3 particles on a 256^3 mesh, L = 2000 Mpc/h: the kick of the first step from the ZA ICs
    # is K(a0, a_1/2) g(x0); the oracle evaluates g from its own ICs of the same seed
    pm = lib()
    np_side, n, box, steps, a_i = 128, 256, 2000.0, 20, 1.0 / 51.0
    dp, _ = _kicks(pm, pm.make_config(np_side, n, box, a_i, 1.0, steps), 6, 1, 512)
    c = Cosmology()
    x0, _ = ic.zeldovich(c, np_side, box, a_i, seed=6, fixed=True)
    a1 = a_i + (1.0 - a_i) / steps
    K = c.kick_factor(a_i, 0.5 * (a_i + a1))
    phik = gravity.newton_potential_k(np.fft.rfftn(cic.density_contrast(x0, n)), n, box, c.omega_m)
    g = gravity.gradient_force(phik, n, box)
    want = K * np.stack([cic.interpolate(g[j], x0) for j in range(3)])
    assert rel_l2(dp, want) < 1e-5


@pytest.mark.parametrize("mode,n_lo", [(0, 0), (1, 4)])
@pytest.mark.parametrize("np_side,nmesh", [(64, 64), (32, 128), (64, 128), (128, 128)])
def test_whole_plane_middle_passes_equal_the_separate_passes(mode, n_lo, np_side, nmesh):
    # form 1: each kz plane transformed in shared memory (forward y, x, per-mode operator, and the
    # three inverse x and y transforms of -i k_j phi): the same butterflies and operator as the
    # separate passes, so the runs differ only by the deposit's atomic order
    pm = lib()
    box = 1000.0 if mode == 0 else 8000.0
    cfg = pm.make_config(np_side, nmesh, box, 1.0 / 51.0, 1.0, 20, mode=mode, n_lo=n_lo)
    dps, ds = _kicks(pm, cfg, 5, 3, 0)
    dpp, dp_ = _kicks(pm, cfg, 5, 3, 1)
    assert np.max(np.abs(dps)) > 0
    # the plane form applies -i k_y and -i k_z before the inverse transforms instead of between
    # or after them: the same values up to FP32 rounding order; on the 8 Gpc/h Poisson-gauge box
    # at z = 50 (delta ~ 1e-3 a cell) the runs then differ by up to 3e-5 (both are checked
    # against the oracle below and in the Poisson-gauge run tests)
    tol = 1e-5 if mode == 0 else 1e-4
    assert rel_l2(dpp, dps) < tol
    assert rel_l2(dp_, ds) < tol


def test_whole_plane_form_against_the_oracle():
    # 64^3 particles on a 128^3 mesh, L = 1000 Mpc/h: the first kick from the ZA ICs, K g(x0),
    # against the oracle's own force evaluation of its ICs from the same seed
    pm = lib()
    np_side, n, box, steps, a_i = 64, 128, 1000.0, 20, 1.0 / 51.0
    dp, _ = _kicks(pm, pm.make_config(np_side, n, box, a_i, 1.0, steps), 8, 1, 1)
    c = Cosmology()
    x0, _ = ic.zeldovich(c, np_side, box, a_i, seed=8, fixed=True)
    a1 = a_i + (1.0 - a_i) / steps
    K = c.kick_factor(a_i, 0.5 * (a_i + a1))
    phik = gravity.newton_potential_k(np.fft.rfftn(cic.density_contrast(x0, n)), n, box, c.omega_m)
    g = gravity.gradient_force(phik, n, box)
    want = K * np.stack([cic.interpolate(g[j], x0) for j in range(3)])
    assert rel_l2(dp, want) < 1e-5


@pytest.mark.parametrize("form", [0, 1])
def test_whole_plane_form_of_a_poisson_gauge_run_against_the_oracle(form):
    # 32^3 particles on a 64^3 mesh, L = 20 Gpc/h, z = 100 -> 1, 12 steps, n_lo = 4: both forms
    # against the FP64 oracle's Poisson-gauge run, to the FP32 tolerance of the Poisson-gauge tests
    from oracle import pm as opm
    from tests.gpu_util import min_image, positions_box_units, ticks_to_host
    pm = lib()
    np_side, n, box, a_i, steps = 32, 64, 20000.0, 1.0 / 101.0, 12
    c = Cosmology()
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=21, fixed=True)
    ref = opm.PMRun(c, n, box, a_i, 1.0, steps, x0, p0, mode=opm.GR_POISSON)
    ref.step(steps)
    run = pm.PMRun(pm.make_config(np_side, n, box, a_i, 1.0, steps, mode=1, n_lo=4))
    pm.pm_set_fused_fft(run.ctx, form)
    run.ic(seed=21)
    run.step(steps)
    x, _ = run.particles()
    torch.cuda.synchronize()
    xg = ticks_to_host(x)
    d_g = min_image(positions_box_units(xg) - positions_box_units(x0))
    d_o = min_image(positions_box_units(ref.x) - positions_box_units(x0))
    assert rel_l2(d_g, d_o) < 2e-3
