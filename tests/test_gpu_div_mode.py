"""The FP64 per-mode divide of the spectral operators (Newton-Raphson reciprocal from the
FP32 one, two steps) against the correctly rounded division, over the operand range the
Green's function and the Poisson-gauge constraint give it and over the FP32 normal range."""
import numpy as np
import pytest

from tests.gpu_util import lib, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _ulps(got, want):
    a = np.asarray(got, dtype=np.float64).view(np.int64)
    b = np.asarray(want, dtype=np.float64).view(np.int64)
    return np.abs(a - b)


def _check(a, d):
    pm = lib()
    out = torch.empty(a.size, dtype=torch.float64, device="cuda")
    pm.pm_div_mode_check(to_dev(a), to_dev(d), out)
    torch.cuda.synchronize()
    got = to_host(out)
    want = a / d  # numpy: IEEE correctly rounded
    assert np.all(np.sign(got) == np.sign(want))
    return _ulps(np.abs(got), np.abs(want))


def test_green_function_operands():
    # coef / (kf^2 |n|^2): every |n|^2 of a 512^3 mesh, boxes from 100 Mpc/h to 20 Gpc/h
    n2 = np.arange(1, 3 * 256**2 + 1, dtype=np.float64)
    for box in (100.0, 2000.0, 5000.0, 20000.0):
        kf = 2 * np.pi / box
        d = kf * kf * n2
        a = np.full_like(d, -1.5 * 0.31 / 512.0**3)
        assert _check(a, d).max() <= 2


def test_constraint_denominators():
    # k^2 + 3 calH / dtau + 3 calH^2 + (9/2) calH^2 Om(a): calH ~ 3e-5 .. 3e-4 h/Mpc,
    # dtau ~ 5 .. 500 Mpc/h, k from the fundamental mode of a 20 Gpc/h box to the Nyquist of a 100 Mpc/h one
    r = np.random.default_rng(1)
    m = 200_000
    H = 10**r.uniform(np.log10(3e-5), np.log10(3e-4), m)
    dtau = 10**r.uniform(np.log10(5.0), np.log10(500.0), m)
    k = 10**r.uniform(np.log10(3e-4), np.log10(16.0), m)
    om = r.uniform(0.3, 1.0, m)
    d = k * k + 3 * H / dtau + 3 * H * H + 4.5 * H * H * om
    a = r.standard_normal(m) * 10**r.uniform(-12, 2, m)
    assert _check(a, d).max() <= 2


def test_fp32_normal_range():
    r = np.random.default_rng(2)
    m = 200_000
    d = 10**r.uniform(-37.0, 38.0, m) * r.choice([-1.0, 1.0], m)
    a = 10**r.uniform(-30.0, 30.0, m) * r.choice([-1.0, 1.0], m)
    d = np.concatenate([d, 2.0**np.arange(-120, 121), [1.0, 3.0, 7.0, 1.0 / 3.0]])
    a = np.concatenate([a, np.ones(241), [1.0, 1.0, 1.0, 1.0]])
    assert _check(a, d).max() <= 2
