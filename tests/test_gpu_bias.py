"""GPU parity of the halo proxy and the linear-bias fit (Sec. 5.2, Eq. b1)."""
import math

import numpy as np
import pytest

import inputs
from oracle import cic, ic, pm as opm, stats
from oracle.cosmology import Cosmology
from tests.gpu_util import lib, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FP32, FP64 = 0, 1


def _cast(a, prec):
    return a if prec == FP64 else a.astype(np.float32).astype(np.float64)


def _run(pm, n, box, prec, a_i=0.5):
    return pm.PMRun(pm.make_config(16, n, box, a_i, 1.0, 4, precision=prec))


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("quantise", [False, True])
def test_halo_proxy_selection_exact(prec, quantise):
    pm = lib()
    n = 64
    f = inputs.lognormal_field(91, n, sigma=1.0)
    if quantise:  # many exact ties: the lower linear index must win
        f = np.round(f * 4.0) / 4.0
    f = _cast(f, prec)
    run = _run(pm, n, 1000.0, prec)
    out = torch.empty((n, n, n), dtype=torch.float64 if prec == FP64 else torch.float32, device="cuda")
    K = pm.pm_halo_proxy(run.ctx, out, field=to_dev(f if prec == FP64 else f.astype(np.float32)), fraction=0.05)
    assert K == math.ceil(0.05 * n**3)
    got = to_host(out).astype(np.float64)
    want_mask = stats.top_fraction_mask(f, 0.05)
    np.testing.assert_array_equal(got > 0, want_mask)
    np.testing.assert_allclose(got, stats.halo_proxy_contrast(f, 0.05), rtol=1e-6 if prec == FP32 else 1e-14)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("terms", [1, 2, 3])
def test_linear_bias_fit_matches_oracle(prec, terms):
    pm = lib()
    n, box = 64, 4000.0
    dm = _cast(inputs.lognormal_field(92, n, sigma=0.6), prec)
    run = _run(pm, n, box, prec)
    dev = to_dev(dm if prec == FP64 else dm.astype(np.float32))
    dh = torch.empty_like(dev)
    pm.pm_halo_proxy(run.ctx, dh, field=dev, fraction=0.05)
    edges = stats.log_edges(12, 1.0, n / 2.0)
    kf = 2 * np.pi / box
    kmax = 0.02
    coef, k, ratio, nm = pm.pm_linear_bias(run.ctx, dh, dev, edges, kmax, terms=terms)
    dh_o = stats.halo_proxy_contrast(dm, 0.05)
    ko, phm, no = stats.power_spectrum(dh_o, box, edges, delta2=dm)
    _, pmm, _ = stats.power_spectrum(dm, box, edges)
    np.testing.assert_array_equal(nm, no)
    ok = no > 0
    np.testing.assert_allclose(ratio[ok], (phm / pmm)[ok], rtol=2e-5 if prec == FP32 else 1e-11)
    c = Cosmology()
    calH = float(c.conformal_hubble(0.5)) if terms >= 2 else None
    want = stats.fit_linear_bias(ko, phm / pmm, no, kmax, calH=calH, with_k2=(terms == 3))
    np.testing.assert_allclose(coef, want, rtol=1e-4 if prec == FP32 else 1e-9)
    assert np.all(k[ok] * 0 == 0) and kf > 0


def test_gr_bias_study_pipeline_matches_oracle():
    # Sec. 5.2 on a horizon-scale box: the halo proxy of the Poisson-gauge and the Newtonian
    # runs from the same ICs, the fit of P_hm / P_mm = b1 + b1^GR calH^2/k^2 + c k^2 in each,
    # the relativistic bias with the Newtonian systematic subtracted, Eq. bgr beside it, and
    # B_hhh / B_mmm on the equilateral and squeezed (k3 = 4 k_f) triangles (Sec. 5.3); FP64
    pm = lib()
    np_side, n, box, a_i, a_f, steps = 16, 32, 20000.0, 1.0 / 101.0, 1.0, 12
    c = Cosmology()
    edges = np.arange(0.5, 16.0, 1.0)
    nb = len(edges) - 1
    k3_bin = 3
    eq, sq = pm.bispectrum_configurations(nb, k3_bin)
    kmax = 15.0 * 2 * np.pi / box
    got, want = {}, {}
    x0, p0 = ic.zeldovich(c, np_side, box, a_i, seed=21, fixed=False)
    for mode in (0, 1):
        run = pm.PMRun(pm.make_config(np_side, n, box, a_i, a_f, steps, mode=mode, precision=FP64, n_lo=4 * mode))
        run.ic(seed=21)
        run.step(steps)
        dm = torch.empty((n, n, n), dtype=torch.float64, device="cuda")
        pm.pm_density(run.ctx, dm)
        dh = torch.empty_like(dm)
        pm.pm_halo_proxy(run.ctx, dh, field=dm, fraction=0.05)
        coef, _, _, _ = pm.pm_linear_bias(run.ctx, dh, dm, edges, kmax, terms=3)
        bh, _ = run.bispectrum(edges, 64, field=dh)
        bm, _ = run.bispectrum(edges, 64, field=dm)
        got[mode] = (coef, bh / bm)
        ref = opm.PMRun(c, n, box, a_i, a_f, steps, x0, p0, mode=mode)
        ref.step(steps)
        dmo = cic.density_contrast(ref.x, n)
        dho = stats.halo_proxy_contrast(dmo, 0.05)
        ko, phm, no = stats.power_spectrum(dho, box, edges, delta2=dmo)
        _, pmm, _ = stats.power_spectrum(dmo, box, edges)
        coef_o = stats.fit_linear_bias(ko, phm / pmm, no, kmax, calH=float(c.conformal_hubble(a_f)), with_k2=True)
        _, bho, _ = stats.bispectrum(dho, box, edges, M=64)
        _, bmo, _ = stats.bispectrum(dmo, box, edges, M=64)
        want[mode] = (coef_o, bho / bmo)
        assert np.array_equal(to_host(dh).astype(np.float64) > 0, dho > 0)  # same cells selected
    for mode in (0, 1):
        np.testing.assert_allclose(got[mode][0], want[mode][0], rtol=1e-7)
        for rows in (eq, sq):
            g, w = got[mode][1][rows], want[mode][1][rows]
            live = np.isfinite(w)
            assert live.sum() >= 3
            np.testing.assert_allclose(g[live], w[live], rtol=1e-7)
    b1gr_corrected = got[1][0][1] - got[0][0][1]
    assert b1gr_corrected == pytest.approx(want[1][0][1] - want[0][0][1], rel=1e-6, abs=1e-9)
    cfg = pm.make_config(np_side, n, box, a_i, a_f, steps)
    theory = pm.pm_b1_gr_theory(cfg, a_f, got[1][0][0])
    assert theory == pytest.approx(stats.b1_gr_theory(want[1][0][0], c.growth_f(a_f), float(c.omega_m_a(a_f))),
                                   rel=1e-6)
