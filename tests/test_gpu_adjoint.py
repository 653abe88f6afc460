"""GPU gradient of the field-level loss (pm_loss_grad) against the FP64 oracle's reverse
sweep, the oracle's finite differences, and across checkpoint intervals."""
import numpy as np
import pytest

import inputs
from oracle import adjoint, cic
from oracle.cosmology import Cosmology
from tests.gpu_util import lib, rel_l2, to_dev, to_host, torch

pytestmark = pytest.mark.gpu


def _setup(pm, np_side, nmesh, box=300.0, a_i=0.2, a_f=0.6, steps=4):
    c = Cosmology()
    w = inputs.gaussian_field(31, np_side).astype(np.float32)
    ut, _, _, _ = adjoint.forward(c, np_side, nmesh, box, a_i, a_f, steps, inputs.gaussian_field(32, np_side))
    target = cic.density_contrast(ut, nmesh).astype(np.float32)
    run = pm.PMRun(pm.make_config(np_side, nmesh, box, a_i, a_f, steps))
    return c, w, target, run, (box, a_i, a_f, steps)


@pytest.mark.parametrize("np_side,nmesh", [(16, 16), (32, 64)])
def test_gradient_matches_fp64_oracle(np_side, nmesh):
    pm = lib()
    c, w, target, run, (box, a_i, a_f, steps) = _setup(pm, np_side, nmesh)
    L, g = run.loss_grad(to_dev(w), to_dev(target), checkpoint_every=2)
    Lo, go = adjoint.loss_and_grad(c, np_side, nmesh, box, a_i, a_f, steps, w.astype(np.float64),
                                   target.astype(np.float64))
    assert L == pytest.approx(Lo, rel=1e-4)
    assert rel_l2(to_host(g).astype(np.float64), go) < 1e-3


def test_checkpoint_interval_does_not_change_the_gradient():
    pm = lib()
    c, w, target, run, (box, a_i, a_f, steps) = _setup(pm, 32, 64)
    out = [run.loss_grad(to_dev(w), to_dev(target), checkpoint_every=k) for k in (1, 3, steps)]
    for L, g in out[1:]:
        assert L == pytest.approx(out[0][0], rel=1e-6)
        assert rel_l2(to_host(g), to_host(out[0][1])) < 1e-5


def test_loss_differences_match_oracle_and_autograd():
    """The FP32 loss needs a step eps far above its rounding, and at that eps the
    central difference of this piecewise-smooth loss (CIC kinks at cell boundaries)
    is not the derivative; the oracle's own small-eps test pins the derivative.  Here
    the GPU's central differences match the oracle's at the same eps and direction,
    and torch.autograd reaches the same reverse sweep."""
    pm = lib()
    c, w, target, run, (box, a_i, a_f, steps) = _setup(pm, 32, 64)
    wd, td = to_dev(w), to_dev(target)
    L, g = run.loss_grad(wd, td, checkpoint_every=2)
    rng = np.random.default_rng(7)
    eps = 3e-3
    t64 = target.astype(np.float64)
    for _ in range(2):
        v = to_dev(rng.standard_normal(w.shape).astype(np.float32))
        wp, wm = wd + eps * v, wd - eps * v
        lp, _ = run.loss_grad(wp, td)
        lm, _ = run.loss_grad(wm, td)
        fd = (lp - lm) / (2 * eps)
        lpo = adjoint.loss(c, 32, 64, box, a_i, a_f, steps, to_host(wp).astype(np.float64), t64)
        lmo = adjoint.loss(c, 32, 64, box, a_i, a_f, steps, to_host(wm).astype(np.float64), t64)
        fdo = (lpo - lmo) / (2 * eps)
        assert abs(fd - fdo) < 2e-2 * abs(fdo) + 1e-9
    # torch.autograd through the same reverse sweep
    wv = wd.clone().requires_grad_(True)
    loss = pm.field_loss(run, wv, td, checkpoint_every=2)
    loss.backward()
    assert float(loss) == pytest.approx(L, rel=1e-6)
    assert rel_l2(to_host(wv.grad), to_host(g)) < 1e-5


def test_overlapped_reruns_match_a_single_segment():
    # 9 steps with checkpoints every 2: five segments (the last one of a single step); the
    # forward run records the last two, the first three are re-run on the second stream
    # into alternating records while the reverse sweep runs.  One segment of 9 re-runs nothing.
    pm = lib()
    c, w, target, run, (box, a_i, a_f, _) = _setup(pm, 32, 64, steps=9)
    wd, td = to_dev(w), to_dev(target)
    L1, g1 = run.loss_grad(wd, td, checkpoint_every=9)
    for every in (2, 1):
        L, g = run.loss_grad(wd, td, checkpoint_every=every)
        assert L == pytest.approx(L1, rel=1e-6)
        assert rel_l2(to_host(g), to_host(g1)) < 1e-5
