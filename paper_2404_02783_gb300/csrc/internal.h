// Internal launcher interfaces shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "pm_common.cuh"

namespace pm {

// Per-mode operator applied by the strided (x-axis) FFT pass between its forward
// and inverse transforms.
enum OpKind {
    OP_FWD_STORE = 0,  // forward x-FFT, store the spectrum
    OP_INV = 1,        // inverse x-FFT
    OP_NEWTON = 2,     // Newtonian Green's function, outputs IFFT_x(phi) and IFFT_x(-i kx phi)
    OP_GR = 3,         // linearised Poisson-gauge constraint, same outputs, updates Phi_old
    OP_ZA = 4,         // Zel'dovich displacement potential from unit phases, same outputs
    OP_BIN = 5,        // power-spectrum binning (auto or cross), no output
    OP_POTENTIAL = 6   // Newtonian potential only: IFFT_x(phi)
};

// Per-mode filter of OP_ZA (the same three-output gradient chain serves the Zel'dovich
// displacement, the derivatives of a real mesh and the second-order LPT displacement).
enum ZaFilter { ZA_AMP = 0, ZA_IDENTITY = 1, ZA_INV_LAPLACE = 2 };

struct SpecOp {
    int kind = OP_FWD_STORE;
    int fwd = 1;              // forward x-FFT of the input first
    double coef = 0.0;        // NEWTON/POTENTIAL: -3/2 Om / n^3; ZA: -sign * scale (both divided by kf^2 per field)
    double kf = 0.0;          // fundamental mode, h/Mpc
    const double* kf_arr = nullptr;  // per-field kf when several fields (boxes) share a launch
    int64_t amp_stride = 0;          // elements between the amplitude tables of consecutive fields
    // linearised Poisson gauge
    double calH = 0.0, omm_a = 0.0, inv_dtau = 0.0, ac2_over_n3 = 0.0;
    int first = 1;            // Phi' = 0 at the first force evaluation
    int n_lo = 0;             // |n|^2 <= n_lo^2 handled in FP64
    void* phi_old = nullptr;  // cplx<T> [kz][kx][ky]
    double2* island = nullptr;  // double2 [(n_lo+1)(2 n_lo+1)^2]
    // Zel'dovich
    const double* amp = nullptr;  // sqrt(P(k)/V) per integer |n|^2
    int fixed_amp = 0;            // phases scaled to unit modulus first (fixed amplitudes)
    int za_filter = 0;            // ZA_AMP: coef amp[|n|^2] / k^2; ZA_IDENTITY: coef; ZA_INV_LAPLACE: coef / k^2
    // power spectrum
    const int16_t* bin_of = nullptr;  // bin per integer |n|^2 (-1 = none)
    const double* wtab = nullptr;     // CIC sinc^2(pi m / n) for m = 0..n/2
    double* acc = nullptr;            // [acc_rows][nbins]: per-CTA sums of w |delta|^2 / W^2 (zeroed)
    double* acc2 = nullptr;           // cross spectra only: the same rows for |in2|^2 (null: not wanted)
    int acc_rows = 0;                 // rows available (the x pass runs at most this many CTAs)
    int nbins = 0;
    int deconv = 0;
    const void* in2 = nullptr;        // second (y-transformed) field for the cross spectrum
};

// Uploads the twiddle tables exp(-2 pi i k / 1024) of both precisions to the current
// device (once per device).
cudaError_t ensure_device_tables();
// Raises cudaFuncAttributeMaxDynamicSharedMemorySize of fn on the current device to at least
// bytes (monotone per kernel and device; only calls the runtime when it must grow).
cudaError_t set_smem_once(const void* fn, size_t bytes);
// CTAs of fn resident per SM for the launch shape (occupancy query, cached per device),
// and the device's SM count (cached): the grid of persistent kernels.
cudaError_t resident_ctas(const void* fn, int threads, size_t smem, int* per_sm);
int num_sms();

// out[i] = a[i] / d[i] by the FP64 per-mode divide of the spectral operators (fft_impl.cuh).
cudaError_t div_mode_check(const double* a, const double* d, int64_t count, double* out, cudaStream_t st);

// FFT passes.  n is the transform length (power of two, 16..1024); batch counts
// independent 3D fields stored back to back.  The forward passes subtract `sub` from every
// input value (a density's mean: only the zero mode changes).
template <typename T>
cudaError_t z_r2c(const T* in, cplx<T>* out, int n, int batch, cudaStream_t st, double sub = 0.0);
// out_j = c2r(in_j [* -i kf kz when gradz_mask bit j is set]) for the ncomp fields; zero (if
// given, a mesh of the outputs' shape that the caller has finished with) is cleared beside them
template <typename T>
cudaError_t z_c2r(const cplx<T>* const* in, T* const* out, int ncomp, int n, int batch,
                  unsigned gradz_mask, double kf, cudaStream_t st, const double* kf_arr = nullptr,
                  T* zero = nullptr);
template <typename T, bool INV>
cudaError_t y_rows(cplx<T>* data, int64_t nrows, int n, cudaStream_t st);
// A <- IFFT_y(A), B <- IFFT_y(B), C <- IFFT_y(-i ky A); kf_arr (optional) gives the kf of
// each consecutive group of rows_per_field rows.
template <typename T>
cudaError_t y_rows_grad3(cplx<T>* A, cplx<T>* B, cplx<T>* C, int64_t nrows, int n, double kf,
                         cudaStream_t st, const double* kf_arr = nullptr, int64_t rows_per_field = 0);
template <typename T>
cudaError_t x_cols(cplx<T>* data, cplx<T>* out2, int nplanes, int n, const SpecOp& op, cudaStream_t st);
// tab[s] = bin of |n|^2 = s for s <= nmax from the squared edges e2[0..nbins] (device),
// e2[b] <= s < e2[b+1], the last edge closed, -1 outside.
cudaError_t bin_table(int16_t* tab, int64_t nmax, const double* e2, int nbins, cudaStream_t st);
// out[b] = sum_r rows[r nbins + b] in row order (deterministic), r < nrows.
cudaError_t bin_rows_sum(const double* rows, int nrows, int nbins, double* out, cudaStream_t st);
// Transposed force chain on the x pass (adjoint): V holds the three y-transformed spectra
// of the deposited adjoint momenta back to back; out = IFFT_x[sum_j i k_j c(k) FFT_x V_j]
// with c = coef / (kf^2 |n|^2).  Also sets zero[0 .. nzero) to 0 (a buffer the caller is
// done with; nzero a multiple of 4, zero 16-byte aligned; null: nothing).
// Poisson gauge (gr != null): the lagged constraint Phi_n = src_n delta_n + carry_n Phi_{n-1}
// (src = -(3/2) calH^2 Om(a) / den, carry = cc / den, den = k^2 + 3 calH^2 + (9/2) calH^2 Om(a) + cc,
// cc = 3 calH / dtau, 0 at the first evaluation) makes the transposed chain carry one spectrum
// back through the evaluations: Z_n = K_n a_n c^2 / n^3 W_n + carry_{n+1} Z_{n+1} (Z in gr->Z,
// [kz][kx][ky], read and overwritten; zero before the last evaluation is reversed),
// out = IFFT_x[src_n Z_n], W_n = sum_j i k_j FFT_x V_j.  coef is then unused.
struct AdjGrOp {
    double K_ac2_n3 = 0.0;             // K_n a_n c^2 / n^3 of evaluation n
    double H = 0.0, om = 0.0, cc = 0.0;    // calH, Om(a) and cc of evaluation n
    double H1 = 0.0, om1 = 0.0, cc1 = 0.0; // the same of evaluation n + 1 (any finite values when Z is 0)
    void* Z = nullptr;
};
// fd: the first-order gradient's transposed chain: V is one scalar field (the deposit of the
// adjoint momenta with the CIC derivative weights) and W = FFT_x V, without i k_j.
template <typename T>
cudaError_t x_adj(const cplx<T>* V, cplx<T>* out, int n, double kf, double coef, cudaStream_t st,
                  float* zero = nullptr, int64_t nzero = 0, const AdjGrOp* gr = nullptr, bool fd = false);
// Forward y, x with the per-mode operator op (OP_NEWTON or OP_GR) and inverse y with the y
// gradient of nplanes kz planes in one persistent launch of CTAs of `threads` (256, 512, 1024)
// (FP32, n = 256, 512, 1024): on entry
// A holds the z pass's half spectrum; on exit A = IFFT_y(phi), B = IFFT_y(-i kx phi),
// C = IFFT_y(-i ky phi), as after x_cols + y_rows_grad3.  sync_words: mid_sync_words_count(nplanes)
// device words; the call clears all but the last, the error word, which a bounded wait that
// gave up sets (and nothing here clears).  cudaErrorNotSupported for other sizes.
template <typename T>
cudaError_t fft_middle(cplx<T>* A, cplx<T>* B, cplx<T>* C, int nplanes, int n, const SpecOp& op, unsigned* sync_words,
                       int threads, cudaStream_t st);
inline size_t mid_sync_words_count(int nplanes) { return 5 + 2 * (size_t)nplanes; }
// The same middle passes on whole kz planes in shared memory (FP32, n = 64, 128): on entry A
// holds the z pass's half spectrum; on exit GX = IFFT_xy(-i kx phi), GY = IFFT_xy(-i ky phi),
// A = IFFT_xy(-i kz phi) (the z pass takes them without its z gradient).
// cudaErrorNotSupported for other sizes.
template <typename T>
cudaError_t fft_plane(cplx<T>* A, cplx<T>* GX, cplx<T>* GY, int nplanes, int n, const SpecOp& op, cudaStream_t st);

// Forward z (r2c) and y passes of `batch` real meshes into spec ([field][kz][kx][ky]
// before the x pass).
template <typename T>
cudaError_t forward_zy(const T* in, cplx<T>* spec, int n, int batch, cudaStream_t st, double sub = 0.0);
// The three force meshes from phi and -i kx phi after the inverse x pass (A, B, full
// layout; both overwritten): out[0] = c2r(IFFT_y(B)), out[1] = c2r(IFFT_y(-i ky A)),
// out[2] = c2r(-i kz IFFT_y(A)); scratch holds one half spectrum per field.
// zero (optional): a mesh set to 0 in the same pass (rows written beside the force rows).
template <typename T>
cudaError_t inverse_yz_grad(cplx<T>* A, cplx<T>* B, cplx<T>* scratch, T* const* out, int n, int batch, double kf,
                            cudaStream_t st, const double* kf_arr = nullptr, T* zero = nullptr);

}  // namespace pm
