"""Plain FP64 CPU oracle for the particle-mesh (PM) hot path of arXiv:2404.02783.

TEST INFRASTRUCTURE ONLY.  Nothing in the product path may import this package:
only ``tests/``, ``__graft_entry__.smoke()`` and the ``cpu_baseline`` /
``--impl reference`` legs of ``bench.py`` use it.  It shares no code, tables or
constants with the CUDA library in ``paper_2404_02783_gb300/``; the two meet only
through the seeded input generators in ``inputs/``.

Everything here is written for a reader checking it against the paper by eye:
numpy FP64 arrays, ``numpy.fft`` / ``scipy.integrate`` as library primitives, no
blocking, fusion or reordering beyond what each definition states.

Modules (each function cites the passage it follows):

* ``cosmology``  -- background E(a), growth D(a), f(a), kick/drift integrals,
  Eisenstein-Hu no-wiggle linear P(k) normalised to sigma_8 (Sec. 3 "Simulation setup").
* ``philox``     -- Philox4x32-10 counter-based generator (Salmon et al. 2011) and
  the per-wavevector Gaussian draw used for the initial phases ("same initial
  random perturbation phases", Sec. 2).
* ``ic``         -- Zel'dovich (1LPT) and second-order LPT initial conditions (Sec. 2,
  nLPT with n = 1, 2; Sec. 3), paired and fixed-amplitude phases (Sec. 4.2).
* ``cic``        -- cloud-in-cell deposit / interpolation, the gradient of the CIC
  interpolant (the first-order force option, Sec. 4.1), cell keys and sort order
  (counting density, Sec. 4).
* ``gravity``    -- Newtonian Poisson solve, spectral gradient, linearised
  Poisson-gauge scalar constraint (Sec. 2; Eq. physical_density).
* ``pm``         -- kick-drift-kick leapfrog in the scale factor (spectral or first-order
  gradient).
* ``combine``    -- GR displacement field and combination (Eqs. xiGR and combined).
* ``stats``      -- power spectrum (Eq. powerspectrum), bispectrum (Eq. bispectre),
  halo-proxy linear-bias fit (Eq. b1) and the relativistic bias of Eq. bgr.

Parity status: every function is pinned by a ``-m "not gpu"`` test against a
closed form, an invariant, a brute-force evaluation or a textbook special case.
The Poisson-gauge lag term (Phi' as a backward difference) is pinned to linear
Lambda-CDM theory, Phi = Phi_0 D(a)/a on every scale, through both the solve and
the run's bookkeeping of Phi_old and dtau.  Two parts are pinned only partly:
the amplitude of the horizon-scale GR displacement itself (the paper prints no
values; pinned through the k >> calH limit, the matter-era identity and the
linear-theory history above) and the Eisenstein-Hu constants of
``cosmology.transfer_eh_nowiggle``: the sound horizon (EH98 Eq. 26) is pinned to
Planck 2018's measured r_drag within 3% and the baryon suppression alpha_Gamma
(Eq. 31) to Sugiyama's (1995) independent fit within 1.5%, but L0 and C0
(Eqs. 29-30) only through the BBKS shape within 8% (checked by eye), so a change
of a few percent in one of their constants would pass.  Eq. bgr
(``stats.b1_gr_theory``) is pinned by its derivation from the gauge relations of
linear theory (the Poisson-gauge shift of the comoving density and the counting
volume of Eq. physical_density) and against the paper's Table 1.
"""
