"""Pin of the FP64 reverse-mode gradient: central finite differences of the forward
oracle itself (no shared arithmetic with the reverse sweep)."""
import numpy as np
import pytest

import inputs
from oracle import adjoint, cic
from oracle.cosmology import Cosmology


@pytest.mark.parametrize("n_p,n_mesh", [(16, 16), (8, 16)])
def test_gradient_matches_central_differences(n_p, n_mesh):
    c = Cosmology()
    box, ai, af, steps = 300.0, 0.2, 0.6, 4
    w = inputs.gaussian_field(1, n_p)
    ut, _, _, _ = adjoint.forward(c, n_p, n_mesh, box, ai, af, steps, inputs.gaussian_field(2, n_p))
    target = cic.density_contrast(ut, n_mesh)
    L, g = adjoint.loss_and_grad(c, n_p, n_mesh, box, ai, af, steps, w, target)
    assert L == pytest.approx(adjoint.loss(c, n_p, n_mesh, box, ai, af, steps, w, target), rel=1e-14)
    rng = np.random.default_rng(3)
    eps = 1e-5  # small enough that no particle crosses a CIC cell boundary
    for _ in range(3):
        v = rng.standard_normal((n_p,) * 3)
        fd = (adjoint.loss(c, n_p, n_mesh, box, ai, af, steps, w + eps * v, target)
              - adjoint.loss(c, n_p, n_mesh, box, ai, af, steps, w - eps * v, target)) / (2 * eps)
        assert np.sum(g * v) == pytest.approx(fd, rel=1e-6)


def test_gradient_vanishes_at_the_target():
    c = Cosmology()
    w = inputs.gaussian_field(4, 8)
    u, _, _, _ = adjoint.forward(c, 8, 16, 300.0, 0.2, 0.6, 3, w)
    L, g = adjoint.loss_and_grad(c, 8, 16, 300.0, 0.2, 0.6, 3, w, cic.density_contrast(u, 16))
    assert L < 1e-28 and np.max(np.abs(g)) < 1e-12
