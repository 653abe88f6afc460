"""The C-ABI library loads, exports every symbol include/pm.h declares, and checks
its arguments on the host (no GPU needed)."""
import ctypes
import os
import re
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pm.h")


@pytest.fixture(scope="session")
def pm():
    import paper_2404_02783_gb300 as pm
    if not os.path.exists(pm.LIB_PATH):
        from paper_2404_02783_gb300 import build
        build.build()
    pm.lib()
    return pm


def declared_functions():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:pm_status|const char\*)\s+(pm_\w+)\s*\(", src, flags=re.M)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for core in ("pm_init", "pm_ic_zeldovich", "pm_step", "pm_displacement_correction", "pm_power",
                 "pm_bispectrum"):
        assert core in names


def test_library_exports_every_declared_symbol(pm):
    names = declared_functions()
    L = pm.lib()
    for name in names:
        assert hasattr(L, name), name
    assert set(names) == set(pm.EXPORTS)
    out = subprocess.run(["nm", "-D", "--defined-only", pm.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (pm_\w+)$", out, flags=re.M))
    assert set(names) <= exported


def declared_arities():
    """Number of parameters of every pm_* function declared in the header."""
    src = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for name, params in re.findall(r"^\s*(?:pm_status|const char\*)\s+(pm_\w+)\s*\(([^)]*)\)\s*;", src, flags=re.M | re.S):
        params = params.strip()
        out[name] = 0 if params in ("", "void") else params.count(",") + 1
    return out


def test_binding_argument_lists_match_the_header(pm):
    # each ctypes argument list the binding installs has as many entries as the declaration
    ar = declared_arities()
    assert set(ar) == set(declared_functions())
    L = pm.lib()
    for name, n in ar.items():
        argtypes = getattr(L, name).argtypes
        assert argtypes is not None and len(argtypes) == n, (name, n, argtypes)


def test_workspace_size_and_validation(pm):
    cfg = pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10)
    n = pm.pm_workspace_size(cfg)
    # particles (24 B) + 4 meshes (16 B) + 3 half spectra (24 B per cell-ish) at least
    assert n >= 24 * 32**3 + 16 * 64**3 + 3 * 8 * 33 * 64 * 64
    gr = pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10, mode=pm.PM_GR_POISSON, n_lo=8)
    assert pm.pm_workspace_size(gr) > n
    f64 = pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10, precision=pm.PM_FP64)
    assert pm.pm_workspace_size(f64) > 1.9 * n
    for bad in (pm.make_config(24, 64, 1000.0, 0.02, 1.0, 10),      # not a power of two
                pm.make_config(64, 32, 1000.0, 0.02, 1.0, 10),      # mesh coarser than lattice
                pm.make_config(32, 64, -1.0, 0.02, 1.0, 10),        # box
                pm.make_config(32, 64, 1000.0, 1.0, 0.5, 10),       # a-grid
                pm.make_config(32, 64, 1000.0, 0.02, 1.0, 0),       # steps
                pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10, mode=5),
                pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10, n_lo=40),
                pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10, gradient=2)):
        with pytest.raises(pm.PMError) as e:
            pm.pm_workspace_size(bad)
        assert e.value.status == 1


def test_stateless_calls_check_arguments_before_the_device(pm):
    L = pm.lib()
    assert L.pm_cic_deposit(None, 10, 0, 16, 1.0, None, None) == 1
    assert L.pm_fft_r2c(None, None, 16, 0, None) == 1
    assert L.pm_fft_r2c(ctypes.c_void_p(256), ctypes.c_void_p(256), 12, 0, None) == 1
    sz = ctypes.c_size_t()
    assert L.pm_cell_sort_scratch_size(1000, 16, ctypes.byref(sz)) == 0 and sz.value >= 3 * 16**3 * 4
    assert "pm-gb300" in pm.pm_version()


def test_no_cpu_fallback_without_a_device(pm):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    L = pm.lib()
    # valid arguments but no GPU: the library refuses instead of computing on the host
    st = L.pm_cic_deposit(ctypes.c_void_p(4096), 1, 0, 16, 1.0, ctypes.c_void_p(4096), None)
    assert st == 6
    assert "device" in L.pm_last_error().decode().lower()


def test_triangle_index_follows_the_bispectrum_table_order(pm):
    # host-only: the position of (i, j, l) in pm_bispectrum's output is the oracle's
    # lexicographic enumeration of the triangles i <= j <= l
    from oracle import stats
    for nb in (1, 2, 5, 24):
        tri = stats.triangles(nb)
        assert len(tri) == nb * (nb + 1) * (nb + 2) // 6
        for k, (i, j, l) in enumerate(tri):
            assert pm.pm_triangle_index(nb, i, j, l) == k
    for bad in ((5, 2, 1, 3), (5, 0, 0, 5), (5, -1, 0, 0), (0, 0, 0, 0)):
        with pytest.raises(pm.PMError) as e:
            pm.pm_triangle_index(*bad)
        assert e.value.status == 1
    eq, sq = pm.bispectrum_configurations(6, 2)
    tri = stats.triangles(6)
    assert [tri[k] for k in eq] == [(j, j, j) for j in range(6)]
    assert [tri[k] for k in sq] == [(2, j, j) for j in range(2, 6)]


def test_b1_gr_theory_matches_the_oracle(pm):
    # host-only Eq. bgr from the library's background against the oracle's growth rate and
    # Omega_m(a), at the four redshifts of the paper's bias table
    from oracle.cosmology import Cosmology
    from oracle.stats import b1_gr_theory
    cfg = pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10)
    c = Cosmology()
    for z, b1 in ((1.0, 9.0), (0.5, 5.7), (0.1, 3.9), (0.0, 3.6)):
        a = 1.0 / (1.0 + z)
        want = b1_gr_theory(b1, c.growth_f(a), float(c.omega_m_a(a)))
        assert pm.pm_b1_gr_theory(cfg, a, b1) == pytest.approx(want, rel=1e-9)
    assert pm.pm_b1_gr_theory(cfg, 0.7, 1.0) == 0.0
    with pytest.raises(pm.PMError):
        pm.pm_b1_gr_theory(cfg, -1.0, 2.0)


def test_linear_power_matches_the_oracle(pm):
    # host-only: the library's Eisenstein-Hu no-wiggle spectrum, sigma_8 normalisation and growth
    # (C++ quadrature) against the oracle's (scipy), which the ICs of both sides draw from
    from oracle.cosmology import Cosmology
    c = Cosmology()
    cfg = pm.make_config(32, 64, 1000.0, 0.02, 1.0, 10)
    k = np.geomspace(1e-4, 10.0, 23)
    for a in (1.0, 0.5, 1.0 / 51.0):
        p, D, f = pm.pm_linear_power(cfg, a, k)
        np.testing.assert_allclose(p, c.power_linear(k, a), rtol=1e-9)
        assert D == pytest.approx(c.growth_D(a), rel=1e-10) and f == pytest.approx(c.growth_f(a), rel=1e-10)
    assert pm.pm_linear_power(cfg, 1.0, np.zeros(1))[0][0] == 0.0
    with pytest.raises(pm.PMError):
        pm.pm_linear_power(cfg, 1.0, np.array([-1.0]))


@pytest.mark.parametrize("stepping", [0, 1])
def test_step_factors_match_the_oracle(pm, stepping):
    # host-only: the FP64 kick and drift factors pm_step uses (its own Gauss-Legendre quadrature
    # or the growth-matched factors) against the oracle's (scipy quadrature, its growth ODE), for
    # the first, a middle and the last step of a run from z = 50 and its closing half kick
    from oracle import pm as opm
    from oracle.cosmology import Cosmology
    n, a_i, a_f = 20, 1.0 / 51.0, 1.0
    cfg = pm.make_config(32, 64, 1000.0, a_i, a_f, n, stepping=stepping)
    c = Cosmology()
    ref = opm.PMRun(c, 64, 1000.0, a_i, a_f, n, np.zeros((3, 1)), np.zeros((3, 1)), stepping=stepping)
    grid = ref.a_grid
    for s in (0, 1, 9, n - 1):
        a0, a1 = grid[s], grid[s + 1]
        ah = 0.5 * (a0 + a1)
        a_from = a0 if s == 0 else 0.5 * (grid[s - 1] + a0)
        kick, drift, close = pm.pm_step_factors(cfg, s)
        assert kick == pytest.approx(ref._kick(a_from, ah, a0), rel=1e-10)
        assert drift == pytest.approx(ref._drift_fac(a0, a1, ah), rel=1e-10)
        assert close == pytest.approx(ref._kick(0.5 * (grid[n - 1] + a_f), a_f, a_f), rel=1e-10)
    for bad in (-1, n):
        with pytest.raises(pm.PMError):
            pm.pm_step_factors(cfg, bad)
