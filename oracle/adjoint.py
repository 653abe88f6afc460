"""Reverse-mode gradient of a field-level loss through the particle-mesh run.

Oracle (test infrastructure only), FP64, positions as box fractions.

The differentiable workload fits the initial white noise w of a run at field level
(the paper's GR displacement and bias are field-level quantities, Secs. 2 and 5):

    L(w) = (1/N^3) sum_c (delta(c) - delta_t(c))^2,

with delta the CIC counting density contrast of the final particles and delta_t a
target mesh; ``vjp`` takes the cotangents of any loss of the final density, of the
final displacements d = x - q and of the final (synchronised) momenta p instead.  The forward map is the Zel'dovich IC of ``ic`` (white-noise path)
followed by the kick-drift-kick steps of ``pm``, written out here as a list of kick
and drift operations so that the reverse sweep can walk it backwards:

    drift  u <- u + D p / L          reverse: lambda_p += (D / L) lambda_u
    kick   p <- p + K g(u)           reverse: lambda_u += K J(u)^T lambda_p

with J(u)^T v = sum_j v_j grad(interp(G_j)) + m grad(interp(rho_bar)), where G_j are
the force meshes at u, rho_bar = sum_j T_j^T V_j, V_j the CIC deposit of v_j and
T_j the (real, antisymmetric) Fourier operator rho -> G_j, so T_j^T = -T_j.  The CIC
weights are piecewise linear in u; their derivative is taken on the same side as the
forward floor() (the right derivative at a cell boundary).

Poisson gauge (Sec. 2, the lagged constraint of ``gravity.gr_potential_k``): force
evaluation n gives Phi_n = src_n delta_n + carry_n Phi_{n-1} per mode, with src = s / den,
carry = (3 calH / dtau) / den (0 at the first evaluation), and G_j = T_j (a_n c^2 Phi_n).
G at evaluation n then depends on every earlier density through the products of the carry
factors, and the transposed chain runs backwards with one carried spectrum:
Z_n = K_n a_n c^2 W_n + carry_{n+1} Z_{n+1}, rho_bar_n = IFFT[src_n Z_n] = dL/d delta_n,
where W_n = sum_j i k_j FFT(V_j) of evaluation n and K_n its kick factor.
"""
import numpy as np

from . import cic, gravity, ic, philox
from .cosmology import C_LIGHT
from .pm import GROWTH, INTEGRALS

NEWTON, GR_POISSON = 0, 1  # the force of the run, as in oracle.pm
SPECTRAL, FD1 = 0, 1       # the gradient of the potential, as in oracle.pm


def _grad_gather(field, u, n):
    """sum_c F(c) dW(u_p, c)/du_i for i = x, y, z: shape (3, Np)."""
    base, frac = cic.mesh_coords(u, n)
    flat = field.ravel()
    out = np.zeros((3, base.shape[1]))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                d = (dx, dy, dz)
                idx = (((base[0] + dx) % n) * n + (base[1] + dy) % n) * n + (base[2] + dz) % n
                f = flat[idx]
                w = [frac[a] if d[a] else 1.0 - frac[a] for a in range(3)]
                dw = [n * (1.0 if d[a] else -1.0) for a in range(3)]
                out[0] += dw[0] * w[1] * w[2] * f
                out[1] += w[0] * dw[1] * w[2] * f
                out[2] += w[0] * w[1] * dw[2] * f
    return out


def _weighted_deposit(u, weights, n):
    """V(c) = sum_p weights_p W(u_p, c)."""
    base, frac = cic.mesh_coords(u, n)
    V = np.zeros(n**3)
    for dx in (0, 1):
        wx = frac[0] if dx else 1.0 - frac[0]
        for dy in (0, 1):
            wy = frac[1] if dy else 1.0 - frac[1]
            for dz in (0, 1):
                wz = frac[2] if dz else 1.0 - frac[2]
                idx = (((base[0] + dx) % n) * n + (base[1] + dy) % n) * n + (base[2] + dz) % n
                V += np.bincount(idx, weights=weights * wx * wy * wz, minlength=n**3)
    return V.reshape(n, n, n)


def _k_components(n, box):
    kf = 2.0 * np.pi / box
    f = philox.signed_freqs(n).astype(np.float64)
    fz = np.arange(n // 2 + 1, dtype=np.float64)
    NX, NY, NZ = np.meshgrid(f, f, fz, indexing="ij")
    return [kf * np.where(np.abs(Nj) == n // 2, 0.0, Nj) for Nj in (NX, NY, NZ)]


def _rho_bar(V, n, box, omega_m):
    """sum_j T_j^T V_j with T_j rho = IFFT[-i k_j C(k) FFT(rho)], C = -(3/2) Om / k^2: T_j^T = -T_j."""
    k = _k_components(n, box)
    _, _, k2 = gravity._wavenumbers(n, box)
    C = np.zeros_like(k2)
    C[k2 > 0] = -1.5 * omega_m / k2[k2 > 0]
    acc = np.zeros((n, n, n // 2 + 1), dtype=np.complex128)
    for j in range(3):
        acc += 1j * k[j] * C * np.fft.rfftn(V[j])
    return np.fft.irfftn(acc, s=(n, n, n), axes=(0, 1, 2))


def _potential_k(u, n, box, cosmo, a, mode, hist):
    """Code potential spectrum phi_k at positions u and scale factor a.  Poisson gauge: hist =
    [Phi_old_k, a_old] of the previous force evaluation ([None, None] before the first),
    updated in place, and (a, dtau) is returned beside phi_k (dtau None at the first)."""
    dk = np.fft.rfftn(cic.density_contrast(u, n))
    if mode == NEWTON:
        return gravity.newton_potential_k(dk, n, box, cosmo.omega_m), None
    dtau = None if hist[0] is None else cosmo.delta_tau(hist[1], a)
    Phi = gravity.gr_potential_k(dk, n, box, cosmo, a, phi_old_k=hist[0], dtau=dtau)
    hist[0], hist[1] = Phi, a
    return gravity.gr_code_potential_k(Phi, a), (a, dtau)


def _grad_weight_deposit(u, v, n, box):
    """V(c) = sum_p sum_j v_j,p dW(u_p, c)/dx_j (x in Mpc/h): the transpose of the first-order
    gradient gather of ``cic.interpolate_gradient``."""
    base, frac = cic.mesh_coords(u, n)
    inv_d = n / box
    V = np.zeros(n**3)
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                d = (dx, dy, dz)
                idx = (((base[0] + dx) % n) * n + (base[1] + dy) % n) * n + (base[2] + dz) % n
                w = [frac[j] if d[j] else 1.0 - frac[j] for j in range(3)]
                sg = [inv_d if d[j] else -inv_d for j in range(3)]
                wt = v[0] * sg[0] * w[1] * w[2] + v[1] * w[0] * sg[1] * w[2] + v[2] * w[0] * w[1] * sg[2]
                V += np.bincount(idx, weights=wt, minlength=n**3)
    return V.reshape(n, n, n)


def _grad_hessian_gather(phi, u, n, box, v):
    """out_i = sum_j v_j d/du_i [sum_c dW(u, c)/dx_j phi(c)] (u in box units): the position
    derivative of the first-order gradient gather, contracted with v.  The trilinear weight is
    linear along each axis, so only the mixed (i != j) derivatives survive."""
    base, frac = cic.mesh_coords(u, n)
    inv_d = n / box
    flat = phi.ravel()
    out = np.zeros((3, base.shape[1]))
    for dx in (0, 1):
        for dy in (0, 1):
            for dz in (0, 1):
                d = (dx, dy, dz)
                idx = (((base[0] + dx) % n) * n + (base[1] + dy) % n) * n + (base[2] + dz) % n
                f = flat[idx]
                w = [frac[j] if d[j] else 1.0 - frac[j] for j in range(3)]
                sg = [inv_d if d[j] else -inv_d for j in range(3)]  # d w_j / dx_j
                du = [n * (1.0 if d[j] else -1.0) for j in range(3)]  # d w_j / du_j
                for i in range(3):
                    for j in range(3):
                        if i == j:
                            continue
                        k = 3 - i - j
                        out[i] += v[j] * sg[j] * du[i] * w[k] * f
    return out


def _gr_coefficients(cosmo, n, box, a, dtau):
    """(src, carry) per mode of the lagged constraint at (a, dtau): Phi = src delta + carry
    Phi_old, src = -(3/2) calH^2 Om(a) / den, carry = (3 calH / dtau) / den; 0 at k = 0."""
    _, _, k2 = gravity._wavenumbers(n, box)
    H = float(cosmo.conformal_hubble(a))
    om = float(cosmo.omega_m_a(a))
    cc = 0.0 if dtau is None else 3.0 * H / dtau
    den = k2 + 3.0 * H * H + 4.5 * H * H * om + cc
    src = -1.5 * H * H * om / den
    carry = cc / den
    src[0, 0, 0] = 0.0
    carry[0, 0, 0] = 0.0
    return src, carry


def _za_operator(w_or_s, n_p, box, cosmo, j):
    """Psi_j = A_j w: the white-noise Zel'dovich displacement along axis j (Mpc/h)."""
    dk = ic.linear_delta_k(cosmo, n_p, box, white_noise=w_or_s)
    kf = 2.0 * np.pi / box
    f = philox.signed_freqs(n_p).astype(np.float64)
    fz = np.arange(n_p // 2 + 1, dtype=np.float64)
    axes = np.meshgrid(f, f, fz, indexing="ij")
    Nj = np.where(np.abs(axes[j]) == n_p // 2, 0.0, axes[j])
    n2 = ic.mode_n2(n_p).astype(np.float64)
    inv_k2 = np.zeros_like(n2)
    inv_k2[n2 > 0] = 1.0 / (kf * kf * n2[n2 > 0])
    return np.fft.irfftn(1j * kf * Nj * dk * inv_k2, s=(n_p,) * 3, axes=(0, 1, 2))


def forward(cosmo, n_p, n_mesh, box, a_i, a_f, n_steps, w, mode=NEWTON, gradient=SPECTRAL, stepping=INTEGRALS):
    """ZA ICs from w and the KDK run (Newtonian or Poisson-gauge force, spectral or first-order
    gradient, the kick and drift factors of ``pm.PMRun`` with the same stepping); returns
    (u_final, p_final, ops, mass).  A kick op ("kick", K, u, info) keeps in
    info the force meshes "G" (spectral) or the potential mesh "phi" (first order), and for the
    Poisson gauge "gr" = (a, dtau)."""
    psi = ic.za_displacement(ic.linear_delta_k(cosmo, n_p, box, white_noise=w), n_p, box).reshape(3, -1)
    D, f, E = cosmo.growth_D(a_i), cosmo.growth_f(a_i), float(cosmo.E(a_i))
    i = np.arange(n_p, dtype=np.float64) / n_p
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    u = np.stack([X.ravel(), Y.ravel(), Z.ravel()]) + D * psi / box
    u = u - np.floor(u)
    p = a_i**2 * E * f * D * psi
    grid = a_i + (a_f - a_i) * np.arange(n_steps + 1) / n_steps
    ops = []
    mass = (n_mesh / n_p)**3

    hist = [None, None]

    def kick(uu, a, K):
        """The kick op at positions uu and scale factor a, and the acceleration there."""
        phi_k, meta = _potential_k(uu, n_mesh, box, cosmo, a, mode, hist)
        info = {"gr": meta}
        if gradient == SPECTRAL:
            G = gravity.gradient_force(phi_k, n_mesh, box)
            info["G"] = G
            g = np.stack([cic.interpolate(G[j], uu) for j in range(3)])
        else:
            phi = gravity.potential_mesh(phi_k, n_mesh)
            info["phi"] = phi
            g = -cic.interpolate_gradient(phi, uu, box)
        return ("kick", K, uu.copy(), info), g

    def kick_fac(a, b, a_force):
        return cosmo.kick_factor_growth(a, b, a_force) if stepping == GROWTH else cosmo.kick_factor(a, b)

    def drift_fac(a, b, a_mom):
        return cosmo.drift_factor_growth(a, b, a_mom) if stepping == GROWTH else cosmo.drift_factor(a, b)

    synced = True
    for s in range(n_steps):
        a0, a1 = grid[s], grid[s + 1]
        ah = 0.5 * (a0 + a1)
        a_from = a0 if synced else 0.5 * (grid[s - 1] + a0)
        K = kick_fac(a_from, ah, a0)
        op, g = kick(u, a0, K)
        ops.append(op)
        p = p + K * g
        Dd = drift_fac(a0, a1, ah)
        ops.append(("drift", Dd))
        u = u + Dd * p / box
        u = u - np.floor(u)
        synced = False
        if s == n_steps - 1:
            K = kick_fac(ah, a1, a1)
            op, g = kick(u, a1, K)
            ops.append(op)
            p = p + K * g
    return u, p, ops, mass


def loss(cosmo, n_p, n_mesh, box, a_i, a_f, n_steps, w, delta_t, mode=NEWTON, gradient=SPECTRAL):
    u, _, _, _ = forward(cosmo, n_p, n_mesh, box, a_i, a_f, n_steps, w, mode, gradient)
    return float(np.mean((cic.density_contrast(u, n_mesh) - delta_t)**2))


def lattice_fractions(n_p):
    """Lagrangian lattice q in box units, particle order (3, n_p^3)."""
    i = np.arange(n_p, dtype=np.float64) / n_p
    X, Y, Z = np.meshgrid(i, i, i, indexing="ij")
    return np.stack([X.ravel(), Y.ravel(), Z.ravel()])


def displacement(u, n_p, box):
    """Final displacement d = x - q in Mpc/h, minimum image (3, n_p^3)."""
    d = u - lattice_fractions(n_p)
    return (d - np.rint(d)) * box


def vjp(cosmo, n_p, n_mesh, box, a_i, a_f, n_steps, w, lam_delta=None, lam_disp=None, lam_mom=None, mode=NEWTON,
        gradient=SPECTRAL, stepping=INTEGRALS):
    """dL/dw for any loss L(delta_final, d_final, p_final) given its cotangents lam_delta =
    dL/d delta (n_mesh^3 mesh), lam_disp = dL/d d ((3, n_p^3), per Mpc/h) and lam_mom =
    dL/dp ((3, n_p^3), per Mpc/h of momentum, p after the closing half kick), by the reverse
    sweep of the recorded forward run.  Since d = (u - q) L (minimum image), dL/du = L
    lam_disp; the density adds m sum_c lam_delta(c) dW(u, c)/du; lam_mom is the adjoint
    momentum the sweep starts from (the closing kick is the first operation it reverses)."""
    u, p, ops, mass = forward(cosmo, n_p, n_mesh, box, a_i, a_f, n_steps, w, mode, gradient, stepping)
    lam_u = np.zeros_like(u)
    if lam_delta is not None:
        lam_u += mass * _grad_gather(np.asarray(lam_delta, dtype=np.float64), u, n_mesh)
    if lam_disp is not None:
        lam_u += box * np.asarray(lam_disp, dtype=np.float64).reshape(3, -1)
    lam_p = None if lam_mom is None else np.asarray(lam_mom, dtype=np.float64).reshape(3, -1)
    return _reverse(cosmo, n_p, n_mesh, box, a_i, ops, mass, lam_u, lam_p)


def _reverse(cosmo, n_p, n_mesh, box, a_i, ops, mass, lam_u, lam_p0=None):
    """Walk the recorded kicks and drifts backwards from (lam_u, lam_p = lam_p0, else 0),
    then apply the transposed Zel'dovich map: returns dL/dw (n_p, n_p, n_p)."""
    lam_p = np.zeros_like(lam_u) if lam_p0 is None else np.array(lam_p0, dtype=np.float64)
    Z, carry_next = None, None  # Poisson gauge: the carried spectrum and carry_{n+1}
    k = _k_components(n_mesh, box)
    for op in reversed(ops):
        if op[0] == "drift":
            lam_p += op[1] / box * lam_u
            continue
        K, uk, info = op[1], op[2], op[3]
        gr = info["gr"]
        if "G" in info:  # spectral gradient: g_j = interp(T_j phi)
            G = info["G"]
            V = np.stack([_weighted_deposit(uk, lam_p[j], n_mesh) for j in range(3)])
            direct = sum(lam_p[j] * _grad_gather(G[j], uk, n_mesh) for j in range(3))
            if gr is None:  # Newtonian: dL/d delta of this evaluation is K rho_bar
                rho_bar = K * _rho_bar(V, n_mesh, box, cosmo.omega_m)
            else:
                W = sum(1j * k[j] * np.fft.rfftn(V[j]) for j in range(3))
        else:  # first-order gradient: g = -grad interp(phi), phi a real mesh
            phi = info["phi"]
            Vs = -_grad_weight_deposit(uk, lam_p, n_mesh, box)  # dL/dphi over K
            direct = -_grad_hessian_gather(phi, uk, n_mesh, box, lam_p)
            if gr is None:  # phi = IFFT[C FFT(delta)] with a real, even C: its own transpose
                rho_bar = K * gravity.potential_mesh(
                    gravity.newton_potential_k(np.fft.rfftn(Vs), n_mesh, box, cosmo.omega_m), n_mesh)
            else:
                W = np.fft.rfftn(Vs)
        if gr is not None:  # Poisson gauge: Z carries dL/dPhi back through the lag (each term with its own K)
            a, dtau = gr
            src, carry = _gr_coefficients(cosmo, n_mesh, box, a, dtau)
            Z = K * a * C_LIGHT**2 * W + (0.0 if Z is None else carry_next * Z)
            rho_bar = np.fft.irfftn(src * Z, s=(n_mesh,) * 3, axes=(0, 1, 2))
            carry_next = carry
        lam_u = lam_u + K * direct + mass * _grad_gather(rho_bar, uk, n_mesh)
    D, f, E = cosmo.growth_D(a_i), cosmo.growth_f(a_i), float(cosmo.E(a_i))
    s = (D / box) * lam_u + a_i**2 * E * f * D * lam_p
    # lambda_w = sum_j A_j^T s_j and A_j^T = -A_j (odd, real Fourier multiplier)
    grad = np.zeros((n_p, n_p, n_p))
    for j in range(3):
        grad -= _za_operator(s[j].reshape(n_p, n_p, n_p), n_p, box, cosmo, j)
    return grad


def loss_and_grad(cosmo, n_p, n_mesh, box, a_i, a_f, n_steps, w, delta_t, mode=NEWTON, gradient=SPECTRAL):
    """(L, dL/dw) with dL/dw of shape (n_p, n_p, n_p)."""
    u, p, ops, mass = forward(cosmo, n_p, n_mesh, box, a_i, a_f, n_steps, w, mode, gradient)
    delta = cic.density_contrast(u, n_mesh)
    L = float(np.mean((delta - delta_t)**2))
    lam_rho = 2.0 * (delta - delta_t) / n_mesh**3
    lam_u = mass * _grad_gather(lam_rho, u, n_mesh)
    return L, _reverse(cosmo, n_p, n_mesh, box, a_i, ops, mass, lam_u)
