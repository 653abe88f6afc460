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


def bk_abs_scale(delta, box, edges, m):
    """Per triangle (V^2/N^9) sum |d1 d2 d3| / N_tri, the oracle's estimator applied to the mode
    moduli |delta_n|: the scale to which any floating-point evaluation of a triangle's sum of
    products is accurate (its terms' absolute sum)."""
    from oracle import stats
    n = delta.shape[0]
    mod = np.fft.irfftn(np.abs(np.fft.rfftn(delta)), s=(n, n, n), axes=(0, 1, 2))
    return stats.bispectrum(mod, box, edges, M=m)[1]
