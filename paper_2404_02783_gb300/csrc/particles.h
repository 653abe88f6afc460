// Launchers of the particle-side kernels (particles.cu) and the estimator
// kernels (stats.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pm_common.cuh"

namespace pm {

cudaError_t deposit(const void* x, int64_t count, int precision, int n, double mass, void* rho, cudaStream_t st);
// Deposit of the np^3 lattice-ordered particles of a context (Lagrangian tiles when possible).
cudaError_t deposit_lattice(const void* x, int np, int precision, int n, double mass, void* rho, cudaStream_t st);
cudaError_t interp(const void* field, int n, const void* x, int64_t count, int precision, void* out,
                   cudaStream_t st);
// g: three force meshes; kick = K(a, b); drift = D(a, b) in Mpc/h per unit p
// fd_inv_d > 0: first-order gradient (g[0] is the potential, g[1], g[2] unused), inv_d = n / L.
cudaError_t interp_kick_drift(void* x, void* p, int64_t count, int precision, int n, void* const* g, double kick,
                              double drift, double box, cudaStream_t st, double fd_inv_d = 0.0);
// Kick + drift of the np^3 lattice-ordered particles fused with the deposit of the
// drifted positions into rho (which must be zero on entry); FP32 ticks, n / np in {1,2,4}.
bool ikd_deposit_supported(int np, int precision, int n);
// nfields > 1: a batch of runs stored back to back, box given per field as
// scale_arr[f] = 2^32 / L_f (box is then ignored).  x_out: where the drifted positions go
// (null: back into x); p is always updated in place.
cudaError_t interp_kick_drift_deposit(void* x, void* p, int np, int precision, int n, void* const* g, double kick,
                                      double drift, double box, double mass, void* rho, cudaStream_t st,
                                      int nfields = 1, const double* scale_arr = nullptr, void* x_out = nullptr,
                                      double fd_inv_d = 0.0);
cudaError_t ic_place(void* x, void* p, void* const* psi, int np, int precision, double D, double pfac, double box,
                     cudaStream_t st);
// Second-order LPT source, accumulated over three stages, one per displacement component c:
// d[j] = d Psi1_c / d x_j on the np^3 lattice; s and a are np^3 meshes (ctx precision).
cudaError_t lpt2_source(int stage, void* const* d, void* s, void* a, int64_t count, int precision, cudaStream_t st);
// x = q + D1 Psi1 + D2 Psi2, p = pfac1 Psi1 + pfac2 Psi2; psi1 may be the p array itself.
cudaError_t ic_place2(void* x, void* p, void* const* psi1, void* const* psi2, int np, int precision, double D1,
                      double D2, double pfac1, double pfac2, double box, cudaStream_t st);
template <typename T>
cudaError_t noise(cplx<T>* spec, int n, uint64_t seed, cudaStream_t st);
cudaError_t combine(void* xt, const void* xg, const void* xn, void* xi_out, int npt, int npc, int precision,
                    cudaStream_t st);
cudaError_t fill(void* a, int64_t count, int precision, double v, cudaStream_t st);
// d = x - q (minimum image, Mpc/h; float for ticks, double for fractions) of the np^3 lattice particles.
cudaError_t lagrangian_displacement(const void* x, void* d, int np, int precision, double box, cudaStream_t st);
// Positions in Mpc/h, [3][count]: float from uint32 ticks (FP32) or double from fractions (FP64).
cudaError_t positions_mpc(const void* x, void* out, int64_t count, int precision, double box, cudaStream_t st);
// *bad = the number of FP64 positions that are not finite or outside [0, 1).
cudaError_t count_outside_box(const double* x, int64_t count, unsigned long long* bad, cudaStream_t st);
size_t cell_sort_scratch_bytes(int64_t count, int n);
cudaError_t cell_sort(const void* x, int64_t count, int precision, int n, uint32_t* keys, uint32_t* order,
                      void* scratch, cudaStream_t st);
int64_t cell_sort_static_max_cells();
cudaError_t cell_sort_static(const void* x, int64_t count, int precision, int n, uint32_t* keys, uint32_t* order,
                             cudaStream_t st);

// Exclusive prefix sum of count uint32 values (scratch: scan_scratch_bytes).
cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t count, void* scratch, cudaStream_t st);
size_t scan_scratch_bytes(int64_t count);

// Halo proxy: delta_h of the K densest cells (ties by lower index); scratch: halo_proxy_scratch_bytes.
template <typename T>
cudaError_t halo_proxy(const T* field, int64_t count, int64_t K, T* out, void* scratch, cudaStream_t st);
size_t halo_proxy_scratch_bytes(int64_t count);

// Reverse sweep of the FP32 step (adjoint.cu).
cudaError_t adj_gather(const uint32_t* x, int64_t count, int n, const float* F, float scale, int accumulate,
                       float* lam_u, cudaStream_t st);
cudaError_t adj_direct(const uint32_t* x, int64_t count, int n, const float* v, const float* const* G, float K,
                       float* lam_u, cudaStream_t st);
// lam_u += K sum_j v_j grad interp(G_j) + Km grad interp(rho_bar); then v += drift_next lam_u.
cudaError_t adj_kick_particles(const uint32_t* x, int64_t count, int n, float* v, const float* const* G,
                               const float* rho_bar, float K, float Km, float drift_next, float* lam_u,
                               cudaStream_t st);
// First-order gradient: V += -sum_j v_j dW/dx_j (inv_d = n / L; V zeroed by the caller), and the
// particle side of its transposed kick (phi the recorded potential mesh; rho_bar as in
// adj_kick_particles).
cudaError_t deposit_grad(const uint32_t* x, int64_t count, int n, const float* v, double inv_d, float* V,
                         cudaStream_t st);
cudaError_t adj_kick_particles_fd(const uint32_t* x, int64_t count, int n, float* v, const float* phi,
                                  const float* rho_bar, float K, float Km, double inv_d, float drift_next, float* lam_u,
                                  cudaStream_t st);
// V_j += CIC deposit of v_j for the np^3 lattice-ordered particles x (V_j zeroed by the caller).
cudaError_t deposit_vec(const uint32_t* x, int np, int n, const float* v, float* const* V, cudaStream_t st);
cudaError_t adj_combine(const float2* const* in, float2* out, int n, double kf, double coef, const double* amp,
                        int mode, cudaStream_t st);
cudaError_t loss_mse(float* delta, const float* target, int64_t n3, double* acc, cudaStream_t st);
cudaError_t axpby(float* y, const float* a, const float* b, int64_t m, float alpha, float beta, cudaStream_t st);

// Bispectrum: fill the m-grid masked data spectra (bins x delta 1_b) from the n-grid spectrum,
// or the indicator spectra (bins x 1_b, FP64), and accumulate the triangle sums of the
// inverse transforms of one set.
template <typename T>
cudaError_t bk_masks(const cplx<T>* spec_n, int n, cplx<T>* out, int m, int nbins, const int16_t* bin_of,
                     const double* wtab, int deconv, cudaStream_t st);
cudaError_t bk_indicators(int n, double2* out, int m, int nbins, const int16_t* bin_of, cudaStream_t st);
// unit[u] = (i, j, lb, t): the triangles (i, j, l), l in [max(j, 8 lb), min(nbins, 8 lb + 8)),
// whose first has index t in the i <= j <= l order; acc indexed by triangle (zeroed by the caller).
template <typename T>
cudaError_t bk_units(const T* fields, int m, int nbins, const int4* unit, int nunit, double* acc, cudaStream_t st);

}  // namespace pm
