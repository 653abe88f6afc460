"""Helpers shared by the GPU parity tests: device transfer and layout conversions."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")


def lib():
    import paper_2404_02783_gb300 as pm
    pm.lib()
    return pm


def to_dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def ticks_to_host(t):
    return t.detach().cpu().numpy().view(np.uint32)


def to_host(t):
    return t.detach().cpu().numpy()


def empty_spec(n, fp64, batch=1):
    dt = torch.float64 if fp64 else torch.float32
    shape = (n // 2 + 1, n, n, 2) if batch == 1 else (batch, n // 2 + 1, n, n, 2)
    return torch.empty(shape, dtype=dt, device="cuda")


def spec_to_rfftn(spec):
    """Library layout [kz][kx][ky] -> numpy rfftn layout [kx][ky][kz]."""
    s = spec.detach().cpu().numpy()
    c = s[..., 0] + 1j * s[..., 1]
    return np.transpose(c, (1, 2, 0))


def rel_l2(a, b):
    a = np.asarray(a, dtype=np.float64) if not np.iscomplexobj(a) else np.asarray(a)
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


def min_image(d):
    return d - np.rint(d)


def positions_box_units(x):
    """Box-fraction positions from ticks (exact) or FP64 fractions."""
    return x.astype(np.float64) * 2.0**-32 if x.dtype == np.uint32 else x
