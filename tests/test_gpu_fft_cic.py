"""GPU parity: 3D FFT passes, CIC deposit / interpolation, cell keys and order.

Every CUDA call goes through the C ABI (libpm.so); expected values come from the
FP64 oracle or numpy's FFT on the same seeded inputs.
"""
import numpy as np
import pytest

import inputs
from oracle import cic
from tests.gpu_util import empty_spec, lib, rel_l2, spec_to_rfftn, to_dev, to_host, torch

pytestmark = pytest.mark.gpu
FP32, FP64 = 0, 1
TOL = {FP32: 2e-6, FP64: 1e-13}


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("n", [16, 32, 64, 128, 256])
def test_r2c_matches_rfftn(n, prec):
    pm = lib()
    f = inputs.lognormal_field(100 + n, n, sigma=0.7)
    dt = np.float64 if prec == FP64 else np.float32
    spec = empty_spec(n, prec == FP64)
    pm.pm_fft_r2c(to_dev(f.astype(dt)), spec, n, prec)
    torch.cuda.synchronize()
    got = spec_to_rfftn(spec)
    ref = np.fft.rfftn(f.astype(dt).astype(np.float64))
    assert rel_l2(got, ref) < TOL[prec]


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("n", [16, 64, 128])
def test_c2r_inverts_r2c(n, prec):
    pm = lib()
    f = inputs.gaussian_field(200 + n, n)
    dt = np.float64 if prec == FP64 else np.float32
    spec = empty_spec(n, prec == FP64)
    out = torch.empty((n, n, n), dtype=torch.float64 if prec == FP64 else torch.float32, device="cuda")
    pm.pm_fft_r2c(to_dev(f.astype(dt)), spec, n, prec)
    pm.pm_fft_c2r(spec, out, n, prec)
    torch.cuda.synchronize()
    assert rel_l2(to_host(out) / n**3, f.astype(dt)) < TOL[prec]


@pytest.mark.parametrize("prec", [FP32, FP64])
def test_c2r_matches_irfftn_on_hermitian_input(prec):
    # the c2r of an arbitrary Hermitian spectrum (built from a real field's rfftn)
    pm = lib()
    n = 32
    ref_field = inputs.lognormal_field(301, n)
    F = np.fft.rfftn(ref_field)
    dt = np.float64 if prec == FP64 else np.float32
    s = np.stack([F.real, F.imag], axis=-1).transpose(2, 0, 1, 3).astype(dt)
    spec = to_dev(np.ascontiguousarray(s))
    out = torch.empty((n, n, n), dtype=torch.float64 if prec == FP64 else torch.float32, device="cuda")
    pm.pm_fft_c2r(spec, out, n, prec)
    torch.cuda.synchronize()
    assert rel_l2(to_host(out), np.fft.irfftn(F, s=(n, n, n), axes=(0, 1, 2)) * n**3) < TOL[prec]


def _positions(kind, seed, count, n_side=None):
    if kind == "uniform":
        return inputs.uniform_ticks(seed, count)
    if kind == "clustered":
        return inputs.clustered_ticks(seed, count)
    return inputs.lattice_order_ticks(seed, n_side, 1.5, tail_fraction=0.01)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("kind,count,n", [("uniform", 100_003, 16), ("clustered", 77_777, 64),
                                          ("lattice", 32**3, 32), ("uniform", 0, 16), ("uniform", 1, 16)])
def test_deposit_matches_oracle(kind, count, n, prec):
    pm = lib()
    x = _positions(kind, 7, count, 32)
    xs = x if prec == FP32 else inputs.ticks_to_fractions(x)
    rho = torch.zeros((n, n, n), dtype=torch.float64 if prec == FP64 else torch.float32, device="cuda")
    pm.pm_cic_deposit(to_dev(xs) if count else None, count, prec, n, 1.0, rho)
    torch.cuda.synchronize()
    got = to_host(rho)
    if count == 0:
        assert np.all(got == 0)
        return
    ref = cic.deposit(xs, n, mass=1.0)
    assert rel_l2(got, ref) < (1e-6 if prec == FP32 else 1e-14)
    assert got.sum() == pytest.approx(count, rel=1e-6 if prec == FP32 else 1e-12)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("count", [50_001, 1, 0])
def test_interp_matches_oracle(prec, count):
    pm = lib()
    n = 32
    x = inputs.clustered_ticks(8, count, width=0.05)
    xs = x if prec == FP32 else inputs.ticks_to_fractions(x)
    f = inputs.gaussian_field(9, n)
    dt = torch.float64 if prec == FP64 else torch.float32
    out = torch.empty(count, dtype=dt, device="cuda")
    pm.pm_cic_interp(to_dev(f.astype(np.float64 if prec == FP64 else np.float32)), n, to_dev(xs), count, prec, out)
    torch.cuda.synchronize()
    if count == 0:
        return
    ref = cic.interpolate(f.astype(np.float64 if prec == FP64 else np.float32).astype(np.float64), xs)
    assert rel_l2(to_host(out), ref) < (1e-6 if prec == FP32 else 1e-14)


@pytest.mark.parametrize("prec", [FP32, FP64])
@pytest.mark.parametrize("kind,count,n", [("uniform", 123_457, 8), ("lattice", 32**3, 16), ("clustered", 65_536, 64),
                                          ("uniform", 5, 512), ("uniform", 1, 16), ("uniform", 0, 16)])
def test_cell_keys_and_order_bit_exact(kind, count, n, prec):
    pm = lib()
    x = _positions(kind, 11, count, 32)
    xs = x if prec == FP32 else inputs.ticks_to_fractions(x)
    keys = torch.empty(count, dtype=torch.int32, device="cuda")
    order = torch.empty(count, dtype=torch.int32, device="cuda")
    scratch = torch.empty(pm.pm_cell_sort_scratch_size(count, n), dtype=torch.uint8, device="cuda")
    pm.pm_cell_sort(to_dev(xs), count, prec, n, keys, order, scratch)
    torch.cuda.synchronize()
    if count == 0:
        return
    np.testing.assert_array_equal(to_host(keys).view(np.uint32), cic.cell_keys(xs, n))
    np.testing.assert_array_equal(to_host(order).view(np.uint32), cic.cell_order(xs, n))


def test_lattice_on_nodes_and_boundaries():
    # particles exactly half a cell off the nodes and exactly on the periodic seam
    pm = lib()
    n = 16
    t = (np.arange(n, dtype=np.uint64) * (2**32 // n)).astype(np.uint32)
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    x = np.stack([X.ravel(), Y.ravel(), Z.ravel()])
    x[:, :5] = np.array([0, 2**32 - 1, 2**31], dtype=np.uint32)[:, None]
    rho = torch.zeros((n, n, n), dtype=torch.float32, device="cuda")
    pm.pm_cic_deposit(to_dev(x), x.shape[1], FP32, n, 1.0, rho)
    torch.cuda.synchronize()
    assert rel_l2(to_host(rho), cic.deposit(x, n, mass=1.0)) < 1e-7
