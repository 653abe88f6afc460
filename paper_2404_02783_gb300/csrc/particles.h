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
cudaError_t interp_kick_drift(void* x, void* p, int64_t count, int precision, int n, void* const* g, double kick,
                              double drift, double box, cudaStream_t st);
cudaError_t ic_place(void* x, void* p, void* const* psi, int np, int precision, double D, double pfac, double box,
                     cudaStream_t st);
template <typename T>
cudaError_t noise(cplx<T>* spec, int n, uint64_t seed, cudaStream_t st);
cudaError_t combine(void* xt, const void* xg, const void* xn, void* xi_out, int npt, int npc, int precision,
                    cudaStream_t st);
cudaError_t fill(void* a, int64_t count, int precision, double v, cudaStream_t st);
size_t cell_sort_scratch_bytes(int64_t count, int n);
cudaError_t cell_sort(const void* x, int64_t count, int precision, int n, uint32_t* keys, uint32_t* order,
                      void* scratch, cudaStream_t st);
int64_t cell_sort_static_max_cells();
cudaError_t cell_sort_static(const void* x, int64_t count, int precision, int n, uint32_t* keys, uint32_t* order,
                             cudaStream_t st);

// Bispectrum: fill the m-grid masked spectra (bins x {delta 1_b, 1_b}) from the
// n-grid spectrum, and accumulate the triangle sums of the inverse transforms.
template <typename T>
cudaError_t bk_masks(const cplx<T>* spec_n, int n, cplx<T>* out, int m, int nbins, const int16_t* bin_of,
                     const double* wtab, int deconv, cudaStream_t st);
template <typename T>
cudaError_t bk_triangles(const T* fields, int m, int nbins, const int4* tri, int ntri, double* accS, double* accC,
                         cudaStream_t st);

}  // namespace pm
