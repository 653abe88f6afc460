"""The usage example of README.md runs as written (GPU)."""
import os
import re

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_readme_example_runs():
    text = open(os.path.join(ROOT, "README.md")).read()
    code = re.search(r"```python\n(.*?)```", text, flags=re.S).group(1)
    scope = {}
    exec(compile(code, "README.md", "exec"), scope)
    k, P, nm = scope["k"], scope["P"], scope["nmodes"]
    assert np.all(np.isfinite(P[nm > 0])) and np.all(P[nm > 0] > 0)
    B, ntri, eq, sq = scope["B"], scope["ntri"], scope["eq"], scope["sq"]
    assert len(B) == 29 * 30 * 31 // 6 and len(eq) == 29 and len(sq) == 26
    assert scope["batch"].state()[0] == 50
    g = scope["w"].grad
    assert g is not None and bool(torch.isfinite(g).all()) and float(g.abs().max()) > 0
