"""GPU parity of the halo proxy and the linear-bias fit (Sec. 5.2, Eq. b1)."""
import math

import numpy as np
import pytest

import inputs
from oracle import stats
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
@pytest.mark.parametrize("terms", [1, 2])
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
    want = stats.fit_linear_bias(ko, phm / pmm, no, kmax, calH=calH)
    np.testing.assert_allclose(coef, want, rtol=1e-4 if prec == FP32 else 1e-9)
    assert np.all(k[ok] * 0 == 0) and kf > 0
