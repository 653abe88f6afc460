/*
 * pm.h -- C ABI of the GB300 (sm_103a) particle-mesh library for arXiv:2404.02783,
 * "Simulating the Universe from the cosmological horizon to halo scales".
 *
 * The paper (Sec. 2) obtains a relativistic displacement field by running a
 * particle-mesh (PM) code twice from the same initial phases, once in the
 * Poisson gauge (general relativity, GR) and once in the Newtonian N-body gauge,
 * subtracting the particle positions (Eq. xiGR) and adding the difference to a
 * Newtonian run (Eq. combined); it then measures the matter power spectrum
 * (Eq. powerspectrum) and bispectrum (Eq. bispectre) of the counting density
 * (Sec. 4).  This library implements that data path on one GPU:
 *
 *   pm_ic_zeldovich            Lagrangian initial conditions, first (Zel'dovich) or second order
 *                              (Sec. 2 nLPT, n = 1, 2; Sec. 3 ICs at z = 50)
 *   pm_step                    CIC deposit, r2c FFT, Green's function (Newtonian, or the
 *                              linearised Poisson-gauge constraint), spectral or first-order
 *                              gradient, c2r FFT, CIC interpolation + kick + drift (KDK in a)
 *   pm_displacement_correction Eqs. xiGR and combined
 *   pm_power / pm_bispectrum   Eqs. powerspectrum / bispectre on the CIC counting density
 *   pm_linear_bias             Eq. b1 on a halo proxy (pm_halo_proxy), Eq. bgr (pm_b1_gr_theory)
 *   pm_adjoint_record / _run   gradient of any loss of the final density, displacements and
 *                              momenta with respect to the initial white noise (pm_loss_grad:
 *                              the MSE)
 *   pm_batch_*                 many realisations stepped together from one CUDA graph
 *
 * Conventions shared by every entry point
 * --------------------------------------
 * Units: lengths in Mpc/h, wavenumbers in h/Mpc, H0 = 1 (velocities in 100 km/s).
 * Positions are stored in units of the box side: PM_FP32_FIXED keeps uint32 ticks
 * (2^32 ticks per side, periodic wrap is integer overflow), PM_FP64 keeps double
 * fractions in [0, 1).  Momenta p = a^2 dx/dt / H0 are in Mpc/h (float or double).
 * Particle arrays are structure-of-arrays: x[3][count], p[3][count], axis-major.
 * Particle id = (ix np + iy) np + iz on the Lagrangian lattice q = (ix, iy, iz) L / np.
 * Meshes are C-ordered real arrays [x][y][z] of side n (z fastest), float or double.
 * Mesh nodes sit at cell centres (j + 1/2) L / n.
 * Spectra use the library's transposed half-complex layout [kz][kx][ky] of shape
 * (n/2 + 1, n, n), complex float2 / double2, unnormalised forward DFT
 * F_n = sum_x f(x) exp(-2 pi i n.x / n); it is numpy's rfftn output permuted (2, 0, 1).
 * Bin edges are given in units of the fundamental mode k_f = 2 pi / L; a mode with
 * integer wavevector n is in bin b when e_b^2 <= |n|^2 < e_{b+1}^2 (last bin closed).
 *
 * Memory ownership: the library allocates no device memory per call.  Every device
 * buffer (the context workspace, outputs, scratch) is owned by the caller, who
 * sizes it with the *_size queries; the one exception is the fixed static array of
 * pm_cell_sort_static.  Host output arrays are caller-owned too.
 * Streams: calls are asynchronous on the stream given at pm_init (or per call for
 * the stateless operators) except pm_power, pm_bispectrum and pm_linear_bias, which
 * synchronise that stream before returning host results, and pm_adjoint_run /
 * pm_loss_grad, which also run on a second stream of the context's own and synchronise both.  Host-only calls
 * (pm_triangle_index, pm_b1_gr_theory, pm_step_factors, pm_linear_power, the *_size queries)
 * touch no device.
 * Errors: every call returns a pm_status; pm_last_error() gives a static,
 * thread-local message for the last failure.  A CUDA error inside a call is
 * returned as PM_ERR_CUDA and leaves the context unusable (pm_destroy it).
 * There is no CPU fallback: without an sm_100-family device the calls that launch
 * kernels return PM_ERR_UNSUPPORTED.
 */
#ifndef PM_H
#define PM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PM_OK = 0,
    PM_ERR_INVALID_ARG = 1,   /* bad size, null pointer, unsupported combination */
    PM_ERR_CUDA = 2,          /* a CUDA runtime call or kernel launch failed */
    PM_ERR_WORKSPACE = 3,     /* caller buffer too small or misaligned (256 B) */
    PM_ERR_TIMEOUT = 4,       /* a bounded device wait gave up (the fused FFT passes; results invalid) */
    PM_ERR_BOUNDS = 5,        /* input outside the mesh's bounds (FP64 positions outside [0, 1)) */
    PM_ERR_UNSUPPORTED = 6,   /* no suitable GPU */
    PM_ERR_STATE = 7          /* call out of order (e.g. stepping past a_final) */
} pm_status;

enum { PM_NEWTON = 0, PM_GR_POISSON = 1 };
enum { PM_FP32_FIXED = 0, PM_FP64 = 1 };
/* Force gradient: spectral (-i k phi, three inverse transforms), or the first-order
 * finite difference of the paper's PM code (Sec. 4.1): the gradient of the CIC
 * (trilinear) interpolant of the real-space potential inside the particle's cell, i.e.
 * the difference across the cell over L/nmesh, weighted bilinearly on the other axes
 * (one inverse transform; the update gathers the potential's eight corners). */
enum { PM_GRAD_SPECTRAL = 0, PM_GRAD_FD1 = 1 };
/* Leapfrog factors: the FP64 integrals K = int da / (a^2 E), D = int da / (a^3 E), or the
 * growth-matched factors that make every step exact for the linear growing mode (the force
 * of step n taken at a_n, the momenta of its drift at a_{n+1/2}; FastPM, Feng et al. 2016):
 * K = [a^2 E f D]_{a}^{b} / ((3/2) Om D(a_force)), D = [D]_{a_n}^{a_{n+1}} / (a^2 E f D)(a_{n+1/2}).
 * The Poisson-gauge lag keeps the conformal time of the integral. */
enum { PM_STEP_INTEGRALS = 0, PM_STEP_GROWTH = 1 };
/* Initial-condition flags (pm_ic_zeldovich, pm_batch_ic). */
enum { PM_IC_PAIRED = 1, PM_IC_FIXED = 2, PM_IC_2LPT = 4 };

/* Run configuration (Sec. 3 "Simulation setup"; sizes are powers of two). */
typedef struct {
    int np;            /* particle lattice side, 16..1024 */
    int nmesh;         /* PM mesh side, 16..1024, a multiple of np */
    double box;        /* comoving box side L in Mpc/h */
    double omega_m;    /* Omega_m; Omega_Lambda = 1 - Omega_m (no radiation, Sec. 3) */
    double omega_b;
    double h;
    double n_s;
    double sigma8;     /* normalisation of the Eisenstein-Hu no-wiggle linear P(k) at z = 0 */
    double a_init;     /* start of the uniform a-grid */
    double a_final;    /* end of the uniform a-grid */
    int n_steps;       /* number of KDK steps on the a-grid */
    int mode;          /* PM_NEWTON or PM_GR_POISSON */
    int precision;     /* PM_FP32_FIXED or PM_FP64 */
    int n_lo;          /* GR only: modes with |n|^2 <= n_lo^2 are solved and stored in FP64 */
    int gradient;      /* PM_GRAD_SPECTRAL (0) or PM_GRAD_FD1; pm_batch_* refuse FD1
                          (PM_ERR_INVALID_ARG) */
    int stepping;      /* PM_STEP_INTEGRALS (0) or PM_STEP_GROWTH */
} pm_config;

typedef struct pm_ctx pm_ctx;   /* opaque host object owned by the library */

/* ------------------------------------------------------------------ context */

/* Bytes of device workspace a context needs for cfg (particles, meshes, spectra,
 * GR history, tables).  Returns PM_ERR_INVALID_ARG for an unsupported cfg. */
pm_status pm_workspace_size(const pm_config* cfg, size_t* bytes);

/* Create a context on caller-owned device memory `workspace` (>= pm_workspace_size,
 * 256-byte aligned, kept alive until pm_destroy).  `stream` is a cudaStream_t
 * (NULL = legacy default).  Host-side FP64 tables (a-grid, kick/drift integrals,
 * growth, Eisenstein-Hu amplitudes, FFT twiddles) are built here and copied into
 * the workspace.  Particles are undefined until pm_ic_zeldovich or pm_set_particles. */
pm_status pm_init(const pm_config* cfg, void* workspace, size_t bytes, void* stream, pm_ctx** out);

/* Release the host object; the workspace stays the caller's.  NULL is accepted. */
pm_status pm_destroy(pm_ctx* ctx);

/* Zel'dovich initial conditions at a_init (Sec. 2: same random phases for every run;
 * first-order LPT).  Phases: white_noise == NULL draws one unit complex Gaussian per
 * wavevector from Philox4x32-10 (key = seed, counter = (nx, ny, nz, 0)) with a
 * Box-Muller transform, so every resolution shares its common modes; otherwise
 * white_noise is a device real field w[np][np][np] (ctx precision) of unit variance
 * and the phases are FFT(w) / np^{3/2}.  flags: PM_IC_PAIRED flips the sign of every
 * phase, PM_IC_FIXED scales every phase to unit modulus (|g| = 1, the phase kept), and
 * both together give the paired-and-fixed pair of the pairing method cited in Sec. 4.2
 * (B(k) is averaged over the PAIRED and plain runs of one seed).  PM_IC_2LPT adds the
 * second-order Lagrangian displacement (Sec. 3: the paper's ICs at z = 50 are 2LPT):
 * x = q + D Psi1 + D2 Psi2, p = a^2 E (f D Psi1 + f2 D2 Psi2), Psi2 = grad phi2 with
 * laplacian(phi2) = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2), Psi1 = -grad phi1,
 * D2 = -(3/7) D^2 Om(a)^(-1/143), f2 = 2 Om(a)^(6/11); derivatives are spectral on the
 * np^3 lattice, the source is formed there without de-aliasing.  Modes with a Nyquist
 * component and the zero mode are 0 (Psi1 and Psi2).  Other flag bits: PM_ERR_INVALID_ARG.
 * Resets the step counter to 0 and the GR potential history. */
pm_status pm_ic_zeldovich(pm_ctx* ctx, uint64_t seed, const void* white_noise, int flags);

/* Advance n_steps KDK steps along the a-grid (one force evaluation per step; after
 * the last step of the grid a closing half kick synchronises the momenta).
 * PM_ERR_STATE when the grid would be overrun. */
pm_status pm_step(pm_ctx* ctx, int n_steps);

/* Device pointers to the context's particle arrays x[3][np^3], p[3][np^3]. */
pm_status pm_particles(pm_ctx* ctx, void** x, void** p);

/* Copy particles in (device-to-device, caller layout = context layout) and reset
 * the step counter to 0 with synchronised momenta at a_init.  x or p may be the context's
 * own array (pm_particles), written by the caller beforehand: that array is not copied.
 * FP64 positions must be finite box fractions in [0, 1): otherwise PM_ERR_BOUNDS and
 * nothing is copied (the check runs on the device and synchronises the context stream;
 * uint32 ticks are valid by construction and are not checked). */
pm_status pm_set_particles(pm_ctx* ctx, const void* x, const void* p);

/* Resume a run at a point of its a-grid (checkpoint / restart; the paper's runs write
 * snapshots at fixed redshifts, Secs. 3-5): copy x, p in as pm_set_particles does and set
 * the integrator to `step` (0..n_steps) with momenta synchronised with the positions
 * (synchronised != 0) or half a step behind (0, the state pm_step leaves between steps:
 * p at the midpoint a_{step-1/2}).  The momenta are synchronised at step 0 and at
 * n_steps (otherwise PM_ERR_INVALID_ARG).  A Poisson-gauge context resumes here only at
 * step 0 (PM_ERR_UNSUPPORTED otherwise: its lagged constraint needs the Phi history, which
 * pm_set_state_gr carries).  A snapshot taken with pm_particles + pm_state and restored here
 * continues exactly as the original run.  FP64 positions: as pm_set_particles. */
pm_status pm_set_state(pm_ctx* ctx, const void* x, const void* p, int step, int synchronised);

/* The Poisson-gauge history the lagged constraint (Sec. 2) carries between force evaluations:
 * device pointers to the context's Phi_old spectrum (layout of the spectra, ctx precision) and
 * FP64 island (NULL when n_lo = 0), with their sizes in bytes (any output may be NULL).  A
 * snapshot of a Poisson-gauge run between steps is pm_particles + pm_state + copies of these;
 * pm_set_state_gr restores it: as pm_set_state, then the history copied in (device pointers of
 * those sizes; required for step > 0, the island too when n_lo > 0), the last force evaluation
 * taken at a_{step-1} (at a_final after the closing kick).  The run then continues as the
 * original.  Non-Poisson-gauge contexts: PM_ERR_UNSUPPORTED / PM_ERR_INVALID_ARG. */
pm_status pm_gr_history(pm_ctx* ctx, void** phi_old, size_t* phi_bytes, void** island, size_t* island_bytes);
pm_status pm_set_state_gr(pm_ctx* ctx, const void* x, const void* p, int step, int synchronised, const void* phi_old,
                          const void* island);

/* Lagrangian displacement d = x - q of every particle (minimum image, Mpc/h), q its
 * lattice node, written to disp[3][np^3] (float for PM_FP32_FIXED, double for PM_FP64).
 * The position output of a run whose gradient pm_adjoint_run takes (Sec. 2: the GR
 * displacement field is a difference of such displacements, Eq. xiGR). */
pm_status pm_displacement(pm_ctx* ctx, void* disp);

/* Positions of every particle in Mpc/h in [0, L) (a float getter of the positions): device
 * array pos[3][np^3], float for PM_FP32_FIXED (ticks times L / 2^32, rounded down to float:
 * within 3e-4 Mpc/h at L = 5000, against the ticks' 1.2e-6) and double for PM_FP64
 * (fractions times L). */
pm_status pm_positions(pm_ctx* ctx, void* pos);

/* Host view of the integrator (no device work): current step index, scale factor
 * and whether the momenta are synchronised with the positions (1) or half a step
 * behind (0). */
pm_status pm_state(pm_ctx* ctx, int* step, double* a, int* synchronised);

/* The three middle passes of a force evaluation with the spectral gradient in FP32 -- forward
 * y, x with the Green's function or Poisson-gauge constraint and the x gradient, inverse y with
 * the y gradient -- run in one of these forms (`form`):
 *   0             three separate launches (the default);
 *   1             whole kz planes in shared memory (meshes of 64^3 and 128^3): one CTA takes a
 *                 plane, runs the forward y and x transforms, the per-mode operator and, for each
 *                 force component, the inverse x and y transforms of -i k_j phi there, and writes
 *                 the three gradient spectra (HBM sees one read and three writes of the plane);
 *   256/512/1024  one persistent kernel of CTAs of that size over the kz planes (meshes of 256^3
 *                 and up), each plane's intermediate spectra re-read from L2 instead of HBM; its
 *                 items wait for the items they depend on with bounded polls, and a wait that
 *                 gives up (it cannot under correct operation) sets an error word that pm_power
 *                 and pm_timings report as PM_ERR_TIMEOUT.
 * The results are the same up to the summation order of the deposit.  A form that does not
 * apply to the context runs the separate passes.  Other values: PM_ERR_INVALID_ARG.
 * pm_autotune_fft times the middle passes in each form that applies (three runs each on the
 * context's spectrum buffers, after a warm-up, CUDA events on the context stream) and keeps the
 * fastest: *threads_out the form (0 = separate), *ms_out its time (either may be NULL).  It
 * touches only the spectrum buffers, so it may run at any point of a run.  Synchronises. */
pm_status pm_set_fused_fft(pm_ctx* ctx, int form);
pm_status pm_autotune_fft(pm_ctx* ctx, int* threads_out, double* ms_out);

/* Per-phase device timing of pm_step with CUDA events recorded on the context
 * stream around each kernel of a force evaluation and update.  pm_profile(ctx, 1)
 * starts recording (0 stops); pm_timings synchronises the stream, writes the summed
 * milliseconds and the number of timed launch groups per phase since the previous
 * call into caller arrays of PM_NPHASES entries, and resets the counters. */
enum {
    PM_PHASE_DEPOSIT = 0,      /* zeroing + CIC deposit */
    PM_PHASE_FFT_ZY_FWD = 1,   /* z (real to half spectrum) and forward y passes (z alone when the
                                  fused middle passes run, pm_set_fused_fft) */
    PM_PHASE_FFT_X_GREEN = 2,  /* x pass with Green's function / constraint and x gradient (with the
                                  forward and inverse y passes when fused) */
    PM_PHASE_FFT_YZ_INV = 3,   /* inverse y (with y gradient; not when fused) and z passes of the
                                  three force components (z gradient fused) */
    PM_PHASE_KICK_DRIFT = 4,   /* CIC interpolation + kick + drift (+ next deposit when fused) */
    PM_NPHASES = 5
};
pm_status pm_profile(pm_ctx* ctx, int enable);
pm_status pm_timings(pm_ctx* ctx, double* ms, int64_t* launches);

/* CIC counting density contrast delta = rho / rho_bar - 1 of the current particles
 * on the context mesh (Sec. 4), written to the device mesh delta[n][n][n]. */
pm_status pm_density(pm_ctx* ctx, void* delta);

/* Code potential phi (Mpc/h)^2 of the current particles on the mesh, Newtonian:
 * phi_k = -(3/2) Omega_m delta_k / k^2 (phi_0 = 0), written to phi[n][n][n].
 * (The Poisson-gauge potential depends on the step history; see pm_step.) */
pm_status pm_potential(pm_ctx* ctx, void* phi);

/* Eqs. xiGR and combined: xi = x_GR - x_Newton per particle id (minimum image),
 * interpolated trilinearly in Lagrangian coordinates when the target lattice is
 * finer (target->np = r gr->np, r a power of two; integer weights over r^3 with
 * round-half-even on ticks), then x_target += xi.  gr and newton must share np and
 * precision with each other and precision with target.  xi_out (device, target
 * layout: int32[3][np^3] ticks or double[3][np^3] fractions) may be NULL. */
pm_status pm_displacement_correction(pm_ctx* target, const pm_ctx* gr, const pm_ctx* newton,
                                     void* xi_out);

/* Eq. powerspectrum: binned P(k) = (V/n^6) <|delta_k / W(k)|^2> over the full sphere
 * of modes, W = prod_j sinc^2(pi n_j / n) when deconvolve != 0 (CIC window), the zero
 * mode and |n| > n/2 excluded.  field == NULL: the CIC counting density of the
 * context's particles; otherwise a device real mesh field[n][n][n] (ctx precision).
 * field2 != NULL gives the cross spectrum Re<delta1 delta2*>.  k_out (mean |k| of the
 * modes, h/Mpc), p_out ((Mpc/h)^3) and nmodes_out are host arrays of nbins
 * (NaN where a bin holds no mode).  Synchronises.  nbins in 1..256. */
pm_status pm_power(pm_ctx* ctx, const void* field, const void* field2, int nbins,
                   const double* edges, int deconvolve,
                   double* k_out, double* p_out, double* nmodes_out);

/* Halo proxy of the linear-bias measurement (Sec. 5.2): the K = ceil(fraction n^3)
 * densest cells of field (device mesh[n][n][n], ctx precision) -- or, field == NULL, of
 * the CIC counting density of the context's particles -- ties broken by the lower linear
 * index (x slowest), written as the tracer contrast delta_h = n_h / mean(n_h) - 1 into the
 * device mesh delta_h (n_h = 1 on selected cells, 0 elsewhere).  *selected = K.  The
 * selection is exact (radix select on the IEEE bit patterns).  Uses the context's
 * spectrum buffers as scratch, so it must not run concurrently with pm_step. */
pm_status pm_halo_proxy(pm_ctx* ctx, const void* field, double fraction, void* delta_h, int64_t* selected);

/* Linear halo bias, Eq. b1: fits P_hm / P_mm = b1 [+ b1^GR calH^2 / k^2] [+ c k^2] by least
 * squares weighted with the bins' mode counts, over the bins (edges as in pm_power) whose
 * mean k is below k_max.  terms = 1: b1; 2: b1, b1^GR; 3: b1, b1^GR, c.  calH = a E(a)/c at
 * the context's current scale factor.  P_hm is the cross spectrum of delta_h and delta_m
 * (device meshes), both CIC-deconvolved.  coef[terms] receives the fit; k_out, ratio_out
 * and nmodes_out (host arrays of nbins, may be NULL) the binned k, P_hm/P_mm and mode
 * counts.  Synchronises. */
pm_status pm_linear_bias(pm_ctx* ctx, const void* delta_h, const void* delta_m, int nbins, const double* edges,
                         double k_max, int terms, double* coef, double* k_out, double* ratio_out,
                         double* nmodes_out);

/* Eq. bgr, the linear relativistic bias of the counting density in Poisson gauge,
 * b1^GR = 3 (f(a) + (3/2) Omega_m(a)) (1 - b1), with the growth rate and Omega_m(a) of
 * cfg's background (only its cosmological fields are read).  Sec. 5.2 compares it with
 * the fitted b1^GR of the relativistic run minus that of the Newtonian run (the
 * Newtonian systematic).  Host only.  omega_m outside (0, 1] or a <= 0: PM_ERR_INVALID_ARG. */
pm_status pm_b1_gr_theory(const pm_config* cfg, double a, double b1, double* b1_gr);

/* The leapfrog factors pm_step uses for step s (0..n_steps-1) of a run started at a_init with
 * synchronised momenta: kick = the kick of step s (from a_init for s = 0, else from the
 * midpoint a_{s-1/2}, to a_{s+1/2}), drift = the drift from a_s to a_{s+1}, kick_close = the
 * closing half kick from a_{N-1/2} to a_N; all in FP64 for cfg's background and stepping
 * (PM_STEP_INTEGRALS or PM_STEP_GROWTH; the p update is p += kick * g with g = -grad phi, the
 * position update x += drift * p).  Any output may be NULL.  Host only.  An invalid cfg or s
 * outside 0..n_steps-1: PM_ERR_INVALID_ARG. */
pm_status pm_step_factors(const pm_config* cfg, int s, double* kick, double* drift, double* kick_close);

/* The linear theory the initial conditions are drawn from (Sec. 3 setup): P_out[i] = P(k[i], a)
 * in (Mpc/h)^3 for k[i] in h/Mpc (Eisenstein-Hu no-wiggle transfer function, n_s, sigma_8
 * normalised with a real-space top hat of 8 Mpc/h at a = 1) times D(a)^2, and, if not NULL,
 * D_out = D(a) (D(1) = 1) and f_out = dlnD/dlna for cfg's background (only its cosmological
 * fields are read).  Host arrays of count >= 0 entries.  Host only.  omega_m outside (0, 1],
 * a <= 0, a negative k or count < 0: PM_ERR_INVALID_ARG. */
pm_status pm_linear_power(const pm_config* cfg, double a, const double* k, int64_t count, double* p_out, double* D_out,
                          double* f_out);

/* Device scratch bytes pm_bispectrum needs for grid m and nbins bins. */
pm_status pm_bispectrum_scratch_size(const pm_ctx* ctx, int m, int nbins, size_t* bytes);

/* Eq. bispectre: B_ijl = (V^2/n^9) sum_{n1+n2+n3=0, n_a in bins i,j,l} delta_1 delta_2
 * delta_3 / N_ijl for every triangle i <= j <= l (lexicographic order,
 * nbins (nbins+1)(nbins+2)/6 entries), by the FFT identity on an m^3 grid:
 * sum_x I_i I_j I_l with I_b = IFFT_m[delta 1_b].  Exact (no aliasing) when every
 * mode of every bin has |n_i| < m/3; PM_ERR_INVALID_ARG otherwise.  field as in
 * pm_power.  b_out and ntri_out are host arrays (NaN where N_ijl = 0); N_ijl, an integer
 * count of configurations, is the rounded FFT-identity sum, and B divides by it exactly.
 * scratch is caller device memory of pm_bispectrum_scratch_size bytes.  Synchronises. */
pm_status pm_bispectrum(pm_ctx* ctx, const void* field, int nbins, const double* edges,
                        int m, int deconvolve, void* scratch, size_t scratch_bytes,
                        double* b_out, double* ntri_out);

/* Position of triangle (i, j, l), 0 <= i <= j <= l < nbins, in pm_bispectrum's output:
 * the number of triangles before it in lexicographic order.  Host only (no GPU, no
 * context).  Sec. 4.2 reports two slices of the table: the equilateral configurations
 * (j, j, j) and the squeezed ones (b3, j, j), j >= b3, with b3 the bin holding
 * k3 = 4 k_f.  Indices out of order or range: PM_ERR_INVALID_ARG. */
pm_status pm_triangle_index(int nbins, int i, int j, int l, int64_t* index);

/* ------------------------------------------------------- gradients through the run
 * Field-level fits (the paper's GR displacement and bias are field-level quantities,
 * Secs. 2 and 5) need gradients of a loss on the final state with respect to the initial
 * phases.  The forward map is w -> Zel'dovich ICs of the white-noise field w (device, np^3,
 * as pm_ic_zeldovich with white_noise) -> cfg.n_steps KDK steps and the closing half kick
 * -> (delta, d, p): delta the CIC counting density contrast of the final particles (n^3
 * mesh, pm_density), d their displacements (pm_displacement) and p their synchronised
 * momenta (pm_particles).
 *
 * pm_adjoint_record runs that forward map keeping (x, p) checkpoints every
 * checkpoint_every steps in `scratch` (pm_adjoint_scratch_size bytes, 256-byte aligned),
 * the positions and force meshes of the last two segments and the force meshes of the
 * closing kick; it leaves the context at step n_steps with synchronised momenta, the final
 * particles in place (read delta, d and p from there).  pm_adjoint_run then takes the
 * cotangents d_delta = dL/d delta (device float n^3, or NULL), d_disp = dL/d d (device
 * float [3][np^3], per Mpc/h, or NULL) and d_mom = dL/dp (device float [3][np^3], per Mpc/h
 * of momentum, or NULL; not all three NULL) of any loss L and writes dL/dw (device float
 * np^3) by the reverse sweep, which starts with the transposed closing kick when d_mom is given:
 * every earlier segment is re-run from its checkpoint on a second CUDA stream the context
 * creates on first use (overlapping the reverse sweep of the segment after it), then the
 * transposed drift, kick (direct CIC-gradient term plus the transposed deposit -> Green
 * -> gradient chain) and Zel'dovich map are applied; CIC weight derivatives are taken on
 * the side of the forward floor().  The re-runs consume the checkpoints: one
 * pm_adjoint_run per pm_adjoint_record (PM_ERR_STATE otherwise, or when the context has
 * been stepped or reset in between).  The scratch must stay untouched between the two
 * calls.  pm_adjoint_run synchronises both streams before returning, also on error.
 *
 * pm_loss_grad is both calls for L(w) = mean_c (delta(c) - delta_t(c))^2 with a device
 * target mesh delta_t: it returns L and writes dL/dw.
 *
 * Newtonian and Poisson-gauge contexts (Sec. 2): in the Poisson gauge each force evaluation's
 * Phi depends on the previous one through the lagged constraint, so the checkpoints also keep
 * Phi_old (and the FP64 island), and the transposed force chain carries one spectrum back
 * through the evaluations (the scratch holds both).  With the first-order gradient
 * (PM_GRAD_FD1) the transposed chain is a scalar deposit with the CIC derivative weights, the
 * transposed potential map and the interpolant's mixed second derivatives.  FP32 positions only
 * (PM_ERR_UNSUPPORTED for PM_FP64). */
pm_status pm_adjoint_scratch_size(const pm_ctx* ctx, int checkpoint_every, size_t* bytes);
pm_status pm_adjoint_record(pm_ctx* ctx, const void* white_noise, int checkpoint_every, void* scratch,
                            size_t scratch_bytes);
pm_status pm_adjoint_run(pm_ctx* ctx, const void* d_delta, const void* d_disp, const void* d_mom, void* grad_w);
pm_status pm_loss_grad(pm_ctx* ctx, const void* white_noise, const void* delta_target, int checkpoint_every,
                       void* scratch, size_t scratch_bytes, double* loss, void* grad_w);

/* ------------------------------------------------------- batch of realisations
 * Many independent realisations (seeds, box sizes) of the same FP32 run, Newtonian or
 * Poisson gauge, advanced together: every pass of a step is one launch over all of them,
 * and a multi-step run can be recorded once and replayed as a single CUDA graph launch.
 * This serves the paper's ensembles of runs from shared phases (Secs. 2-3) and the
 * variance of b1 across realisations (Sec. 5.2).  Requirements: precision
 * PM_FP32_FIXED, the spectral gradient, nmesh >= 64 and nmesh / np in {1, 2, 4}; cfg->box
 * is the default box, boxes[r] (may be NULL) the box of realisation r.  In the Poisson gauge
 * each realisation keeps its own Phi history (and FP64 island), and the lag of force
 * evaluation e reads evaluation e - 1 (none at the first after pm_batch_ic).  Memory: one
 * caller workspace of pm_batch_workspace_size bytes, particles [r][3][np^3], meshes
 * [r][n^3].  The batch owns one extra CUDA stream and two events for graph replay. */
typedef struct pm_batch pm_batch;
pm_status pm_batch_workspace_size(const pm_config* cfg, int nreal, size_t* bytes);
pm_status pm_batch_init(const pm_config* cfg, int nreal, const double* boxes, void* workspace, size_t bytes,
                        void* stream, pm_batch** out);
pm_status pm_batch_destroy(pm_batch* batch);
/* Context view of realisation r (particles, density, estimators); valid while the batch
 * lives.  Must not be stepped or destroyed by the caller. */
pm_status pm_batch_context(pm_batch* batch, int r, pm_ctx** view);
/* Realisations per launch of the batched step: every pass runs on chunks of `chunk`
 * realisations, the passes of one chunk back to back (a chunk whose meshes fit in L2 keeps
 * them there between its passes); 0 or nreal = one launch per pass for the whole batch
 * (the default).  The results do not depend on it.  Outside 0..nreal: PM_ERR_INVALID_ARG. */
pm_status pm_batch_set_chunk(pm_batch* batch, int chunk);
/* Form of the batch's middle FFT passes (as pm_set_fused_fft): 0 = separate launches, 1 = whole
 * kz planes in shared memory (nmesh 64 or 128; otherwise the separate passes run).  Other values:
 * PM_ERR_INVALID_ARG.  The results do not depend on it. */
pm_status pm_batch_set_fft(pm_batch* batch, int form);
/* Autotuner of the batch's launch shape: for each form of the middle FFT passes that applies,
 * times one step (replayed from a CUDA graph) for chunk = nreal, nreal/2, ..., 1 (rounded up)
 * and keeps the fastest pair (chunk_out and its ms per step in ms_out; either may be NULL;
 * pm_batch_tuning reads both settings).  It runs the step on the unperturbed lattice (the FFT
 * passes' cost does not depend on the particles; the update's is that of an early step), so
 * it overwrites the particles: call it before pm_batch_ic (PM_ERR_STATE after it).
 * Synchronises. */
pm_status pm_batch_autotune(pm_batch* batch, int* chunk_out, double* ms_out);
pm_status pm_batch_tuning(pm_batch* batch, int* chunk, int* fft_form);
/* Zel'dovich ICs of every realisation from seeds[r] (as pm_ic_zeldovich, same flags). */
pm_status pm_batch_ic(pm_batch* batch, const uint64_t* seeds, int flags);
/* n_steps KDK steps of every realisation; use_graph != 0 records the run once (cached for
 * the same start step and length) and replays it as one graph launch ordered after the
 * batch stream's prior work.  PM_ERR_STATE when the a-grid would be overrun. */
pm_status pm_batch_step(pm_batch* batch, int n_steps, int use_graph);
pm_status pm_batch_state(pm_batch* batch, int* step, double* a, int* synchronised);
/* Per-realisation P(k) of the particles: host arrays [nreal][nbins].  Synchronises. */
pm_status pm_batch_power(pm_batch* batch, int nbins, const double* edges, int deconvolve, double* k_out,
                         double* p_out, double* nmodes_out);
/* Per-realisation halo-proxy linear bias (pm_halo_proxy + pm_linear_bias on the CIC
 * density): coef_out [nreal][terms].  Synchronises. */
pm_status pm_batch_bias(pm_batch* batch, double fraction, int nbins, const double* edges, double k_max, int terms,
                        double* coef_out);

/* ------------------------------------------------ stateless device operators
 * Building blocks of pm_step exposed for testing and reuse; every pointer is a
 * device pointer, sizes are element counts, `stream` is a cudaStream_t. */

/* CIC deposit (Sec. 4 counting density): rho[n][n][n] += mass * CIC weights of
 * count particles x[3][count] (ticks or fractions, per precision).  rho is NOT
 * cleared first.  n a power of two in 8..1024. */
pm_status pm_cic_deposit(const void* x, int64_t count, int precision, int n, double mass,
                         void* rho, void* stream);

/* CIC interpolation of a scalar mesh field[n][n][n] to count particles: out[count]. */
pm_status pm_cic_interp(const void* field, int n, const void* x, int64_t count, int precision,
                        void* out, void* stream);

/* Base cell (ix n + iy) n + iz of each particle (keys_out, uint32[count]) and the
 * stable counting-sort order of the particles by that key (order_out,
 * uint32[count]; NULL to skip).  scratch: pm_cell_sort_scratch_size bytes. */
pm_status pm_cell_sort_scratch_size(int64_t count, int n, size_t* bytes);
pm_status pm_cell_sort(const void* x, int64_t count, int precision, int n,
                       uint32_t* keys_out, uint32_t* order_out,
                       void* scratch, size_t scratch_bytes, void* stream);

/* pm_cell_sort without a scratch argument: the same keys and order, computed with
 * counting scratch that lives in a fixed device array inside the library.  The paper
 * has no counterpart; the entry point exists for callers that cannot allocate device
 * memory per call -- hosts that hand the whole GPU memory to their own fixed pool, or
 * plain C / Fortran drivers with no device allocator at hand -- and for whom finding
 * and passing a scratch buffer is not an option.  It allocates nothing itself.
 * Limits: n^3 <= PM_CELL_SORT_STATIC_MAX_CELLS (a 64^3 mesh); larger meshes return
 * PM_ERR_INVALID_ARG.  The array (about 3 MB) is held on every GPU that loads the
 * library until the process exits.  The first call in each CUDA context (per device;
 * again after a context is torn down and made anew, e.g. by cudaDeviceReset) looks up
 * the array's device address (cudaGetSymbolAddress); make that first call before any
 * stream capture.  Every call on a device shares the one array and clears the part it
 * counts in before use, so calls that overlap on the GPU (different streams or host
 * threads without ordering) race and give wrong results: serialise them. */
#define PM_CELL_SORT_STATIC_MAX_CELLS 262144
pm_status pm_cell_sort_static(const void* x, int64_t count, int precision, int n,
                              uint32_t* keys_out, uint32_t* order_out, void* stream);

/* out[i] = a[i] / d[i] (device double arrays of count) by the FP64 divide of the spectral
 * operators (Green's function 1/k^2, the Poisson-gauge constraint's denominator): the
 * Newton-Raphson iteration for 1/d from the FP32 reciprocal, two steps, times a.  d must
 * be in the FP32 normal range.  Exposed so that it can be compared with the division. */
pm_status pm_div_mode_check(const double* a, const double* d, int64_t count, double* out, void* stream);

/* 3D real-to-complex FFT of real[n][n][n] into spec (layout above), unnormalised. */
pm_status pm_fft_r2c(const void* real, void* spec, int n, int precision, void* stream);

/* Inverse: complex-to-real of spec (overwritten) into real[n][n][n], unnormalised
 * (sum over modes of F_n exp(+2 pi i n.x / n)). */
pm_status pm_fft_c2r(void* spec, void* real, int n, int precision, void* stream);

/* Library version string and last error message.  0.2: pm_config gained `gradient`;
 * pm_ic_zeldovich and pm_batch_ic take PM_IC_* flags. */
const char* pm_version(void);
const char* pm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PM_H */
