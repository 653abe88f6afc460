"""Python binding of libpm.so, the sm_103a particle-mesh library of arXiv:2404.02783.

Argument marshalling only: every step of the path runs in the CUDA kernels behind
``include/pm.h``.  PyTorch supplies device memory (workspaces, outputs) and the
current CUDA stream.  The functions keep the C names (``pm_init``, ``pm_step``, ...)
and raise :class:`PMError` on a non-zero status.  There is no CPU fallback: if
``libpm.so`` is missing, :func:`lib` raises instead of computing anything.

:class:`PMRun` bundles a configuration, its torch-allocated workspace and the
context handle for the common case of one simulation.
"""
import ctypes
import math
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpm.so")

PM_OK = 0
PM_NEWTON, PM_GR_POISSON = 0, 1
PM_FP32_FIXED, PM_FP64 = 0, 1
PM_GRAD_SPECTRAL, PM_GRAD_FD1 = 0, 1
PM_STEP_INTEGRALS, PM_STEP_GROWTH = 0, 1
PM_IC_PAIRED, PM_IC_FIXED, PM_IC_2LPT = 1, 2, 4
# FP64 island of the Poisson-gauge constraint used by the workloads: |n| <= DEFAULT_N_LO
DEFAULT_N_LO = 4
_STATUS = {0: "PM_OK", 1: "PM_ERR_INVALID_ARG", 2: "PM_ERR_CUDA", 3: "PM_ERR_WORKSPACE", 4: "PM_ERR_TIMEOUT",
           5: "PM_ERR_BOUNDS", 6: "PM_ERR_UNSUPPORTED", 7: "PM_ERR_STATE"}

# every entry point declared in include/pm.h
EXPORTS = ("pm_workspace_size", "pm_init", "pm_destroy", "pm_ic_zeldovich", "pm_step", "pm_particles",
           "pm_set_particles", "pm_set_state", "pm_state", "pm_set_fused_fft", "pm_autotune_fft", "pm_profile", "pm_timings", "pm_density", "pm_potential", "pm_displacement_correction", "pm_power", "pm_halo_proxy", "pm_linear_bias",
           "pm_bispectrum_scratch_size", "pm_bispectrum", "pm_triangle_index", "pm_b1_gr_theory", "pm_step_factors", "pm_linear_power", "pm_cic_deposit", "pm_cic_interp",
           "pm_adjoint_scratch_size", "pm_adjoint_record", "pm_adjoint_run", "pm_loss_grad", "pm_displacement", "pm_positions", "pm_gr_history", "pm_set_state_gr", "pm_batch_workspace_size", "pm_batch_init", "pm_batch_destroy", "pm_batch_context", "pm_batch_ic",
           "pm_batch_step", "pm_batch_state", "pm_batch_power", "pm_batch_bias", "pm_batch_set_chunk", "pm_batch_autotune", "pm_batch_set_fft", "pm_batch_tuning",
           "pm_cell_sort_scratch_size", "pm_cell_sort", "pm_cell_sort_static", "pm_div_mode_check", "pm_fft_r2c", "pm_fft_c2r", "pm_version", "pm_last_error")


class PMError(RuntimeError):
    def __init__(self, status, message):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


class PMConfig(ctypes.Structure):
    """Mirror of ``pm_config`` (include/pm.h)."""
    _fields_ = [("np", ctypes.c_int), ("nmesh", ctypes.c_int), ("box", ctypes.c_double),
                ("omega_m", ctypes.c_double), ("omega_b", ctypes.c_double), ("h", ctypes.c_double),
                ("n_s", ctypes.c_double), ("sigma8", ctypes.c_double), ("a_init", ctypes.c_double),
                ("a_final", ctypes.c_double), ("n_steps", ctypes.c_int), ("mode", ctypes.c_int),
                ("precision", ctypes.c_int), ("n_lo", ctypes.c_int), ("gradient", ctypes.c_int),
                ("stepping", ctypes.c_int)]


def make_config(np_side, nmesh, box, a_init, a_final, n_steps, mode=PM_NEWTON, precision=PM_FP32_FIXED,
                omega_m=0.31, omega_b=0.049, h=0.67, n_s=0.965, sigma8=0.81, n_lo=0, gradient=0, stepping=0):
    return PMConfig(np_side, nmesh, box, omega_m, omega_b, h, n_s, sigma8, a_init, a_final, n_steps, mode,
                    precision, n_lo, gradient, stepping)


_lib = None


def lib():
    """Load libpm.so from the package directory (built by ``build.py``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with __graft_entry__.build() "
                           "(nvcc, sm_103a); there is no CPU fallback")
    L = ctypes.CDLL(LIB_PATH)
    vp, sz, i, d, i64, u64 = (ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_double, ctypes.c_int64,
                              ctypes.c_uint64)
    pd = ctypes.POINTER(ctypes.c_double)
    cfgp = ctypes.POINTER(PMConfig)
    sig = {
        "pm_workspace_size": (cfgp, ctypes.POINTER(sz)),
        "pm_init": (cfgp, vp, sz, vp, ctypes.POINTER(vp)),
        "pm_destroy": (vp,),
        "pm_ic_zeldovich": (vp, u64, vp, i),
        "pm_step": (vp, i),
        "pm_particles": (vp, ctypes.POINTER(vp), ctypes.POINTER(vp)),
        "pm_set_particles": (vp, vp, vp),
        "pm_set_state": (vp, vp, vp, i, i),
        "pm_state": (vp, ctypes.POINTER(i), pd, ctypes.POINTER(i)),
        "pm_set_fused_fft": (vp, i),
        "pm_autotune_fft": (vp, ctypes.POINTER(i), pd),
        "pm_profile": (vp, i),
        "pm_timings": (vp, pd, ctypes.POINTER(i64)),
        "pm_density": (vp, vp),
        "pm_potential": (vp, vp),
        "pm_displacement_correction": (vp, vp, vp, vp),
        "pm_power": (vp, vp, vp, i, pd, i, pd, pd, pd),
        "pm_halo_proxy": (vp, vp, d, vp, ctypes.POINTER(i64)),
        "pm_linear_bias": (vp, vp, vp, i, pd, d, i, pd, pd, pd, pd),
        "pm_bispectrum_scratch_size": (vp, i, i, ctypes.POINTER(sz)),
        "pm_bispectrum": (vp, vp, i, pd, i, i, vp, sz, pd, pd),
        "pm_triangle_index": (i, i, i, i, ctypes.POINTER(i64)),
        "pm_b1_gr_theory": (cfgp, d, d, pd),
        "pm_step_factors": (cfgp, i, pd, pd, pd),
        "pm_linear_power": (cfgp, d, pd, i64, pd, pd, pd),
        "pm_adjoint_scratch_size": (vp, i, ctypes.POINTER(sz)),
        "pm_loss_grad": (vp, vp, vp, i, vp, sz, pd, vp),
        "pm_adjoint_record": (vp, vp, i, vp, sz),
        "pm_gr_history": (vp, ctypes.POINTER(vp), ctypes.POINTER(sz), ctypes.POINTER(vp), ctypes.POINTER(sz)),
        "pm_set_state_gr": (vp, vp, vp, i, i, vp, vp),
        "pm_positions": (vp, vp),
        "pm_adjoint_run": (vp, vp, vp, vp, vp),
        "pm_displacement": (vp, vp),
        "pm_batch_workspace_size": (cfgp, i, ctypes.POINTER(sz)),
        "pm_batch_init": (cfgp, i, pd, vp, sz, vp, ctypes.POINTER(vp)),
        "pm_batch_destroy": (vp,),
        "pm_batch_context": (vp, i, ctypes.POINTER(vp)),
        "pm_batch_ic": (vp, ctypes.POINTER(u64), i),
        "pm_batch_step": (vp, i, i),
        "pm_batch_state": (vp, ctypes.POINTER(i), pd, ctypes.POINTER(i)),
        "pm_batch_power": (vp, i, pd, i, pd, pd, pd),
        "pm_batch_bias": (vp, d, i, pd, d, i, pd),
        "pm_batch_set_chunk": (vp, i),
        "pm_batch_autotune": (vp, ctypes.POINTER(i), pd),
        "pm_batch_set_fft": (vp, i),
        "pm_batch_tuning": (vp, ctypes.POINTER(i), ctypes.POINTER(i)),
        "pm_cic_deposit": (vp, i64, i, i, d, vp, vp),
        "pm_cic_interp": (vp, i, vp, i64, i, vp, vp),
        "pm_cell_sort_scratch_size": (i64, i, ctypes.POINTER(sz)),
        "pm_cell_sort": (vp, i64, i, i, vp, vp, vp, sz, vp),
        "pm_cell_sort_static": (vp, i64, i, i, vp, vp, vp),
        "pm_div_mode_check": (vp, vp, i64, vp, vp),
        "pm_fft_r2c": (vp, vp, i, i, vp),
        "pm_fft_c2r": (vp, vp, i, i, vp),
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = list(args)
        fn.restype = ctypes.c_int
    for name in ("pm_version", "pm_last_error"):
        getattr(L, name).restype = ctypes.c_char_p
        getattr(L, name).argtypes = []
    _lib = L
    return L


def _check(status):
    if status != PM_OK:
        raise PMError(status, lib().pm_last_error().decode())


def _ptr(t):
    """Device (or host) address of a tensor/array, or None."""
    if t is None:
        return None
    if hasattr(t, "data_ptr"):
        return ctypes.c_void_p(t.data_ptr())
    if isinstance(t, np.ndarray):
        return ctypes.c_void_p(t.ctypes.data)
    return ctypes.c_void_p(int(t))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _stream(stream=None):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


# --------------------------------------------------------------------------- C names
def pm_version():
    return lib().pm_version().decode()


def pm_workspace_size(cfg):
    out = ctypes.c_size_t()
    _check(lib().pm_workspace_size(ctypes.byref(cfg), ctypes.byref(out)))
    return out.value


def pm_init(cfg, workspace, stream=None):
    h = ctypes.c_void_p()
    _check(lib().pm_init(ctypes.byref(cfg), _ptr(workspace), workspace.numel() * workspace.element_size(),
                         _stream(stream), ctypes.byref(h)))
    return h


def pm_destroy(ctx):
    _check(lib().pm_destroy(ctx))


def _ic_flags(paired, fixed, lpt_order):
    if lpt_order not in (1, 2):
        raise ValueError("lpt_order must be 1 (Zel'dovich) or 2")
    return (PM_IC_PAIRED if paired else 0) | (PM_IC_FIXED if fixed else 0) | (PM_IC_2LPT if lpt_order == 2 else 0)


def pm_ic_zeldovich(ctx, seed, white_noise=None, paired=False, fixed=False, lpt_order=1):
    _check(lib().pm_ic_zeldovich(ctx, ctypes.c_uint64(seed), _ptr(white_noise), _ic_flags(paired, fixed, lpt_order)))


def pm_step(ctx, n_steps=1):
    _check(lib().pm_step(ctx, int(n_steps)))


def pm_particles(ctx):
    x, p = ctypes.c_void_p(), ctypes.c_void_p()
    _check(lib().pm_particles(ctx, ctypes.byref(x), ctypes.byref(p)))
    return x.value, p.value


def pm_set_particles(ctx, x, p):
    _check(lib().pm_set_particles(ctx, _ptr(x), _ptr(p)))


def pm_set_state(ctx, x, p, step, synchronised):
    _check(lib().pm_set_state(ctx, _ptr(x), _ptr(p), int(step), int(bool(synchronised))))


def pm_state(ctx):
    s, a, y = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    _check(lib().pm_state(ctx, ctypes.byref(s), ctypes.byref(a), ctypes.byref(y)))
    return s.value, a.value, bool(y.value)


PHASES = ("deposit", "fft_zy_fwd", "fft_x_green", "fft_yz_inv", "kick_drift")


def pm_set_fused_fft(ctx, form):
    """Form of the middle FFT passes: 0 separate launches, 1 whole kz planes in shared memory
    (64^3, 128^3), 256 / 512 / 1024 the CTA size of the persistent kernel (256^3 and up)."""
    _check(lib().pm_set_fused_fft(ctx, int(form)))


def pm_autotune_fft(ctx):
    """Time the middle FFT passes in each form and keep the fastest: (threads, ms)."""
    t, ms = ctypes.c_int(), ctypes.c_double()
    _check(lib().pm_autotune_fft(ctx, ctypes.byref(t), ctypes.byref(ms)))
    return t.value, ms.value


def pm_profile(ctx, enable=True):
    _check(lib().pm_profile(ctx, int(bool(enable))))


def pm_timings(ctx):
    """{phase: (ms, launches)} summed since the previous call (synchronises)."""
    ms = np.zeros(len(PHASES))
    n = np.zeros(len(PHASES), dtype=np.int64)
    _check(lib().pm_timings(ctx, _dptr(ms), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int64))))
    return {name: (float(ms[i]), int(n[i])) for i, name in enumerate(PHASES)}


def pm_density(ctx, out):
    _check(lib().pm_density(ctx, _ptr(out)))


def pm_displacement(ctx, out):
    _check(lib().pm_displacement(ctx, _ptr(out)))


def pm_adjoint_scratch_size(ctx, checkpoint_every):
    out = ctypes.c_size_t()
    _check(lib().pm_adjoint_scratch_size(ctx, int(checkpoint_every), ctypes.byref(out)))
    return out.value


def pm_adjoint_record(ctx, white_noise, checkpoint_every, scratch):
    _check(lib().pm_adjoint_record(ctx, _ptr(white_noise), int(checkpoint_every), _ptr(scratch),
                                   scratch.numel() * scratch.element_size()))


def pm_adjoint_run(ctx, d_delta, d_disp, grad_w, d_mom=None):
    _check(lib().pm_adjoint_run(ctx, _ptr(d_delta), _ptr(d_disp), _ptr(d_mom), _ptr(grad_w)))


def pm_gr_history(ctx):
    """(phi_old address, bytes, island address or None, bytes) of a Poisson-gauge context."""
    ph, isl = ctypes.c_void_p(), ctypes.c_void_p()
    pb, ib = ctypes.c_size_t(), ctypes.c_size_t()
    _check(lib().pm_gr_history(ctx, ctypes.byref(ph), ctypes.byref(pb), ctypes.byref(isl), ctypes.byref(ib)))
    return ph.value, pb.value, isl.value, ib.value


def pm_set_state_gr(ctx, x, p, step, synchronised, phi_old, island=None):
    _check(lib().pm_set_state_gr(ctx, _ptr(x), _ptr(p), int(step), int(bool(synchronised)), _ptr(phi_old),
                                 _ptr(island)))


def pm_positions(ctx, out):
    _check(lib().pm_positions(ctx, _ptr(out)))


def pm_potential(ctx, out):
    _check(lib().pm_potential(ctx, _ptr(out)))


def pm_displacement_correction(target, gr, newton, xi_out=None):
    _check(lib().pm_displacement_correction(target, gr, newton, _ptr(xi_out)))


def pm_power(ctx, edges, field=None, field2=None, deconvolve=True):
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nb = len(edges) - 1
    k, p, nm = np.empty(nb), np.empty(nb), np.empty(nb)
    _check(lib().pm_power(ctx, _ptr(field), _ptr(field2), nb, _dptr(edges), int(bool(deconvolve)), _dptr(k),
                          _dptr(p), _dptr(nm)))
    return k, p, nm


def pm_halo_proxy(ctx, out, field=None, fraction=0.05):
    """delta_h of the ceil(fraction n^3) densest cells (ties by lower index); returns K."""
    k = ctypes.c_int64()
    _check(lib().pm_halo_proxy(ctx, _ptr(field), float(fraction), _ptr(out), ctypes.byref(k)))
    return k.value


def pm_linear_bias(ctx, delta_h, delta_m, edges, k_max, terms=1):
    """Eq. b1 fit: returns (coef, k, ratio, nmodes)."""
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nb = len(edges) - 1
    coef = np.zeros(3)
    k, r, nm = np.empty(nb), np.empty(nb), np.empty(nb)
    _check(lib().pm_linear_bias(ctx, _ptr(delta_h), _ptr(delta_m), nb, _dptr(edges), float(k_max), int(terms),
                                _dptr(coef), _dptr(k), _dptr(r), _dptr(nm)))
    return coef[:terms], k, r, nm


def pm_bispectrum_scratch_size(ctx, m, nbins):
    out = ctypes.c_size_t()
    _check(lib().pm_bispectrum_scratch_size(ctx, int(m), int(nbins), ctypes.byref(out)))
    return out.value


def pm_bispectrum(ctx, edges, m, scratch, field=None, deconvolve=True):
    edges = np.ascontiguousarray(edges, dtype=np.float64)
    nb = len(edges) - 1
    nt = nb * (nb + 1) * (nb + 2) // 6
    b, c = np.empty(nt), np.empty(nt)
    _check(lib().pm_bispectrum(ctx, _ptr(field), nb, _dptr(edges), int(m), int(bool(deconvolve)), _ptr(scratch),
                               scratch.numel() * scratch.element_size(), _dptr(b), _dptr(c)))
    return b, c


def pm_triangle_index(nbins, i, j, l):
    out = ctypes.c_int64()
    _check(lib().pm_triangle_index(int(nbins), int(i), int(j), int(l), ctypes.byref(out)))
    return out.value


def pm_b1_gr_theory(cfg, a, b1):
    out = ctypes.c_double()
    _check(lib().pm_b1_gr_theory(ctypes.byref(cfg), float(a), float(b1), ctypes.byref(out)))
    return out.value


def pm_step_factors(cfg, s):
    """(kick, drift, closing kick) of step s of a run from cfg (host only)."""
    k, dr, kc = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().pm_step_factors(ctypes.byref(cfg), int(s), ctypes.byref(k), ctypes.byref(dr), ctypes.byref(kc)))
    return k.value, dr.value, kc.value


def pm_linear_power(cfg, a, k):
    """(P(k, a) [(Mpc/h)^3], D(a), f(a)) of the linear theory the ICs are drawn from (host only)."""
    k = np.ascontiguousarray(k, dtype=np.float64)
    p = np.empty_like(k)
    D, f = ctypes.c_double(), ctypes.c_double()
    _check(lib().pm_linear_power(ctypes.byref(cfg), float(a), _dptr(k), k.size, _dptr(p), ctypes.byref(D),
                                 ctypes.byref(f)))
    return p, D.value, f.value


def bispectrum_configurations(nbins, k3_bin):
    """Rows of pm_bispectrum's table for the equilateral triangles (j, j, j), j = 0..nbins-1,
    and the squeezed ones (k3_bin, j, j), j = k3_bin..nbins-1 (Sec. 4.2, Fig. Bk)."""
    eq = np.array([pm_triangle_index(nbins, j, j, j) for j in range(nbins)], dtype=np.int64)
    sq = np.array([pm_triangle_index(nbins, k3_bin, j, j) for j in range(k3_bin, nbins)], dtype=np.int64)
    return eq, sq


def pm_cic_deposit(x, count, precision, n, mass, rho, stream=None):
    _check(lib().pm_cic_deposit(_ptr(x), int(count), precision, int(n), float(mass), _ptr(rho), _stream(stream)))


def pm_cic_interp(field, n, x, count, precision, out, stream=None):
    _check(lib().pm_cic_interp(_ptr(field), int(n), _ptr(x), int(count), precision, _ptr(out), _stream(stream)))


def pm_cell_sort_scratch_size(count, n):
    out = ctypes.c_size_t()
    _check(lib().pm_cell_sort_scratch_size(int(count), int(n), ctypes.byref(out)))
    return out.value


def pm_cell_sort(x, count, precision, n, keys, order, scratch, stream=None):
    nbytes = 0 if scratch is None else scratch.numel() * scratch.element_size()
    _check(lib().pm_cell_sort(_ptr(x), int(count), precision, int(n), _ptr(keys), _ptr(order), _ptr(scratch), nbytes,
                              _stream(stream)))


def pm_cell_sort_static(x, count, precision, n, keys, order, stream=None):
    """pm_cell_sort with the library's fixed device scratch (meshes up to 64^3 cells).

    For callers that cannot allocate device memory per call; calls on one GPU share
    that scratch, so they must not overlap.
    """
    _check(lib().pm_cell_sort_static(_ptr(x), int(count), precision, int(n), _ptr(keys), _ptr(order),
                                     _stream(stream)))


def pm_div_mode_check(a, d, out, stream=None):
    _check(lib().pm_div_mode_check(_ptr(a), _ptr(d), int(a.numel()), _ptr(out), _stream(stream)))


def pm_fft_r2c(real, spec, n, precision, stream=None):
    _check(lib().pm_fft_r2c(_ptr(real), _ptr(spec), int(n), precision, _stream(stream)))


def pm_fft_c2r(spec, real, n, precision, stream=None):
    _check(lib().pm_fft_c2r(_ptr(spec), _ptr(real), int(n), precision, _stream(stream)))


# --------------------------------------------------------------------------- convenience
def log_edges(nbins, lo, hi):
    """Logarithmic bin edges (any unit; pass them in units of k_f to the estimators)."""
    return lo * (hi / lo)**(np.arange(nbins + 1) / nbins)


class PMRun:
    """One simulation: configuration + torch workspace on the current device + context."""

    def __init__(self, cfg, device="cuda", stream=None):
        import torch
        self.cfg = cfg
        self.device = torch.device(device)
        nbytes = pm_workspace_size(cfg)
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws = self.workspace[off:off + nbytes]
        self.stream = stream
        self.ctx = pm_init(cfg, self._ws, stream)
        self.fp64 = cfg.precision == PM_FP64
        self.rdtype = torch.float64 if self.fp64 else torch.float32
        self.count = cfg.np**3

    def __del__(self):
        ctx = getattr(self, "ctx", None)
        if ctx is not None and _lib is not None:
            _lib.pm_destroy(ctx)
            self.ctx = None

    def ic(self, seed=0, white_noise=None, paired=False, fixed=False, lpt_order=1):
        pm_ic_zeldovich(self.ctx, seed, white_noise, paired, fixed, lpt_order)

    def step(self, n=1):
        pm_step(self.ctx, n)

    def particles(self):
        """(x, p) torch views of the context's particle arrays, shape (3, np^3)."""
        import torch
        xp, pp = pm_particles(self.ctx)
        nbytes = 3 * self.count * (8 if self.fp64 else 4)
        xdt = torch.float64 if self.fp64 else torch.int32
        x = _view(self._ws, xp, nbytes).view(xdt).view(3, self.count)
        p = _view(self._ws, pp, nbytes).view(self.rdtype).view(3, self.count)
        return x, p

    def density(self):
        import torch
        n = self.cfg.nmesh
        out = torch.empty((n, n, n), dtype=self.rdtype, device=self.device)
        pm_density(self.ctx, out)
        return out

    def potential(self):
        import torch
        n = self.cfg.nmesh
        out = torch.empty((n, n, n), dtype=self.rdtype, device=self.device)
        pm_potential(self.ctx, out)
        return out

    def power(self, edges, field=None, field2=None, deconvolve=True):
        return pm_power(self.ctx, edges, field, field2, deconvolve)

    def bispectrum(self, edges, m, field=None, deconvolve=True):
        import torch
        nb = len(edges) - 1
        scratch = torch.empty(pm_bispectrum_scratch_size(self.ctx, m, nb) + 256, dtype=torch.uint8,
                              device=self.device)
        off = (-scratch.data_ptr()) % 256
        return pm_bispectrum(self.ctx, edges, m, scratch[off:], field, deconvolve)

    def state(self):
        return pm_state(self.ctx)

    def _adjoint_scratch(self, checkpoint_every):
        """Device scratch of the reverse sweep for this interval (kept for reuse)."""
        import torch
        nbytes = pm_adjoint_scratch_size(self.ctx, checkpoint_every)
        buf = getattr(self, "_adj_buf", None)
        if buf is None or buf.numel() < nbytes + 256:
            buf = torch.empty(nbytes + 256, dtype=torch.uint8, device=self.device)
            self._adj_buf = buf
        off = (-buf.data_ptr()) % 256
        return buf[off:off + nbytes]

    def loss_grad(self, white_noise, target, checkpoint_every=10):
        """(L, dL/dw) of L = mean((delta_final - target)^2) for ICs from white_noise (pm_loss_grad)."""
        import torch
        scratch = self._adjoint_scratch(checkpoint_every)
        grad = torch.empty_like(white_noise)
        loss = ctypes.c_double()
        _check(lib().pm_loss_grad(self.ctx, _ptr(white_noise), _ptr(target), int(checkpoint_every),
                                  _ptr(scratch), scratch.numel(), ctypes.byref(loss), _ptr(grad)))
        return loss.value, grad

    def record(self, white_noise, checkpoint_every=10):
        """pm_adjoint_record: the run from white_noise with its checkpoints kept for pm_adjoint_run."""
        self._adj_scratch = self._adjoint_scratch(checkpoint_every)
        pm_adjoint_record(self.ctx, white_noise, checkpoint_every, self._adj_scratch)

    def adjoint(self, d_delta=None, d_disp=None, d_mom=None):
        """pm_adjoint_run: dL/dw from the cotangents of the recorded run's final density,
        displacements and momenta."""
        import torch
        grad = torch.empty((self.cfg.np,) * 3, dtype=torch.float32, device=self.device)
        c = lambda t: None if t is None else t.contiguous()
        pm_adjoint_run(self.ctx, c(d_delta), c(d_disp), grad, d_mom=c(d_mom))
        return grad

    def gr_history(self):
        """Copies of the Poisson-gauge Phi_old spectrum and FP64 island (None when n_lo = 0), as
        uint8 device tensors for pm_set_state_gr."""
        ph, pb, isl, ib = pm_gr_history(self.ctx)
        phi = _view(self._ws, ph, pb).clone()
        island = _view(self._ws, isl, ib).clone() if isl else None
        return phi, island

    def positions(self):
        """Positions in Mpc/h in [0, L), shape (3, np^3) (float32 from the FP32 ticks)."""
        import torch
        out = torch.empty((3, self.count), dtype=self.rdtype, device=self.device)
        pm_positions(self.ctx, out)
        return out

    def displacement(self):
        """Lagrangian displacements x - q (minimum image, Mpc/h), shape (3, np^3)."""
        import torch
        out = torch.empty((3, self.count), dtype=self.rdtype, device=self.device)
        pm_displacement(self.ctx, out)
        return out

    @property
    def kf(self):
        return 2 * math.pi / self.cfg.box


def run_fields(run, white_noise, checkpoint_every=10, momenta=False):
    """(delta_final, disp_final) -- and p_final with momenta=True -- of the whole PM run as
    differentiable functions of the white-noise field w: the forward pass is
    pm_adjoint_record (the run with checkpoints, ending with the closing half kick), the
    backward pass hands the incoming gradients of the outputs to pm_adjoint_run (one reverse
    sweep on the GPU).  Any torch loss of the final density (shape (n, n, n)), displacements
    (Mpc/h, shape (3, np^3)) and momenta (Mpc/h, shape (3, np^3)) composes with it; one
    backward per forward."""
    import torch

    class _RunFields(torch.autograd.Function):
        @staticmethod
        def forward(ctx, w):
            ctx.set_materialize_grads(False)
            run.record(w.detach().contiguous(), checkpoint_every)
            out = (run.density(), run.displacement())
            if momenta:
                out = out + (run.particles()[1].clone(),)
            return out

        @staticmethod
        def backward(ctx, g_delta, g_disp, g_mom=None):
            if g_delta is None and g_disp is None and g_mom is None:
                return None
            f32 = lambda g: None if g is None else g.to(torch.float32)
            return run.adjoint(f32(g_delta), f32(g_disp), f32(g_mom))

    return _RunFields.apply(white_noise)


def field_loss(run, white_noise, target, checkpoint_every=10):
    """L(w) = mean((delta_final(w) - target)^2) through the whole PM run, differentiable in w."""
    delta, _ = run_fields(run, white_noise, checkpoint_every)
    return ((delta.to(target.dtype) - target)**2).mean()


class PMBatch:
    """Independent realisations advanced together (pm_batch_*), on a torch workspace."""

    def __init__(self, cfg, boxes=None, device="cuda", stream=None):
        import torch
        self.cfg = cfg
        self.B = len(boxes)
        self.boxes = np.ascontiguousarray(boxes, dtype=np.float64)
        out = ctypes.c_size_t()
        _check(lib().pm_batch_workspace_size(ctypes.byref(cfg), self.B, ctypes.byref(out)))
        nbytes = out.value
        self.workspace = torch.empty(nbytes + 256, dtype=torch.uint8, device=device)
        off = (-self.workspace.data_ptr()) % 256
        self._ws = self.workspace[off:off + nbytes]
        h = ctypes.c_void_p()
        _check(lib().pm_batch_init(ctypes.byref(cfg), self.B, _dptr(self.boxes), _ptr(self._ws), nbytes,
                                   _stream(stream), ctypes.byref(h)))
        self.h = h
        self.count = cfg.np**3

    def __del__(self):
        h = getattr(self, "h", None)
        if h is not None and _lib is not None:
            _lib.pm_batch_destroy(h)
            self.h = None

    def set_chunk(self, chunk):
        """Realisations per launch of every pass (0: the whole batch)."""
        _check(lib().pm_batch_set_chunk(self.h, int(chunk)))

    def autotune(self):
        """Pick the realisations per launch by timing one step of each candidate (before ic);
        returns (chunk, ms per step)."""
        c, ms = ctypes.c_int(), ctypes.c_double()
        _check(lib().pm_batch_autotune(self.h, ctypes.byref(c), ctypes.byref(ms)))
        return c.value, ms.value

    def set_fft(self, form):
        """Form of the middle FFT passes: 0 separate launches, 1 whole kz planes in shared memory."""
        _check(lib().pm_batch_set_fft(self.h, int(form)))

    def tuning(self):
        """(realisations per launch, form of the middle FFT passes) in use."""
        c, f = ctypes.c_int(), ctypes.c_int()
        _check(lib().pm_batch_tuning(self.h, ctypes.byref(c), ctypes.byref(f)))
        return c.value, f.value

    def ic(self, seeds, paired=False, fixed=False, lpt_order=1):
        s = np.ascontiguousarray(seeds, dtype=np.uint64)
        _check(lib().pm_batch_ic(self.h, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)),
                                 _ic_flags(paired, fixed, lpt_order)))

    def step(self, n=1, graph=True):
        _check(lib().pm_batch_step(self.h, int(n), int(bool(graph))))

    def state(self):
        s, a, y = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
        _check(lib().pm_batch_state(self.h, ctypes.byref(s), ctypes.byref(a), ctypes.byref(y)))
        return s.value, a.value, bool(y.value)

    def context(self, r):
        v = ctypes.c_void_p()
        _check(lib().pm_batch_context(self.h, int(r), ctypes.byref(v)))
        return v

    def particles(self, r):
        import torch
        xp, pp = pm_particles(self.context(r))
        nbytes = 3 * self.count * 4
        x = _view(self._ws, xp, nbytes).view(torch.int32).view(3, self.count)
        p = _view(self._ws, pp, nbytes).view(torch.float32).view(3, self.count)
        return x, p

    def density(self, r):
        """CIC density contrast of realisation r (pm_density on its context view), (n, n, n)."""
        import torch
        n = self.cfg.nmesh
        out = torch.empty((n, n, n), dtype=torch.float32, device=self.workspace.device)
        pm_density(self.context(r), out)
        return out

    def bispectrum(self, r, edges, m, field=None, deconvolve=True):
        """B(k) of realisation r (of its particles, or of `field` on its mesh): (B, N_tri)."""
        import torch
        view = self.context(r)
        nb = len(edges) - 1
        scratch = torch.empty(pm_bispectrum_scratch_size(view, m, nb) + 256, dtype=torch.uint8,
                              device=self.workspace.device)
        off = (-scratch.data_ptr()) % 256
        return pm_bispectrum(view, edges, m, scratch[off:], field, deconvolve)

    def power(self, edges, deconvolve=True):
        edges = np.ascontiguousarray(edges, dtype=np.float64)
        nb = len(edges) - 1
        k, p, nm = (np.empty((self.B, nb)) for _ in range(3))
        _check(lib().pm_batch_power(self.h, nb, _dptr(edges), int(bool(deconvolve)), _dptr(k), _dptr(p), _dptr(nm)))
        return k, p, nm

    def bias(self, edges, k_max, fraction=0.05, terms=1):
        edges = np.ascontiguousarray(edges, dtype=np.float64)
        coef = np.empty((self.B, terms))
        _check(lib().pm_batch_bias(self.h, float(fraction), len(edges) - 1, _dptr(edges), float(k_max), int(terms),
                                   _dptr(coef)))
        return coef


def _view(ws, ptr, nbytes):
    off = ptr - ws.data_ptr()
    return ws[off:off + nbytes]
