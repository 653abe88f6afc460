"""GPU parity of the FP32 step whose update fuses interpolation, kick, drift and the
next deposit over Lagrangian tiles: particles that stay near their lattice site, a
population that travels several cells (leaving the tile's staged box), and particles
anywhere in the box, for lattice-to-mesh ratios n / np of 1 and 2."""
import numpy as np
import pytest

import inputs
from oracle import cic, pm as opm
from oracle.cosmology import Cosmology
from tests.gpu_util import lib, min_image, positions_box_units, rel_l2, ticks_to_host, to_dev, to_host, torch

pytestmark = pytest.mark.gpu

BOX, A_I, A_F, STEPS = 1000.0, 0.3, 1.0, 8


def _positions(layout, np_side, nmesh):
    if layout == "uniform":
        return inputs.uniform_ticks(41, np_side**3)
    tail = 0.05 if layout == "tails" else 0.0
    return inputs.lattice_order_ticks(41, np_side, 0.7, nmesh, tail_fraction=tail, tail_cells=6.0)


@pytest.mark.parametrize("np_side,nmesh", [(64, 64), (32, 64), (128, 128)])
@pytest.mark.parametrize("layout", ["near", "tails", "uniform"])
def test_fused_update_matches_oracle(np_side, nmesh, layout):
    pm = lib()
    x0 = _positions(layout, np_side, nmesh)
    p0 = inputs.momenta(42, np_side**3, 10.0).astype(np.float32)
    run = pm.PMRun(pm.make_config(np_side, nmesh, BOX, A_I, A_F, STEPS))
    pm.pm_set_particles(run.ctx, to_dev(x0), to_dev(p0))
    ref = opm.PMRun(Cosmology(), nmesh, BOX, A_I, A_F, STEPS, x0, p0.astype(np.float64))

    def compare(tol):
        xg, pg = run.particles()
        torch.cuda.synchronize()
        xg, pg = ticks_to_host(xg), to_host(pg).astype(np.float64)
        dg = min_image(positions_box_units(xg) - positions_box_units(x0))
        do = min_image(positions_box_units(ref.x) - positions_box_units(x0))
        assert rel_l2(dg, do) < tol
        assert rel_l2(pg, ref.p) < tol

    run.step(1)
    ref.step(1)
    compare(1e-5)
    assert rel_l2(to_host(run.density()), cic.density_contrast(ref.x, nmesh)) < 1e-5
    # every later force comes from the density the fused update deposited
    run.step(STEPS - 1)
    ref.step(STEPS - 1)
    compare(1e-4)
