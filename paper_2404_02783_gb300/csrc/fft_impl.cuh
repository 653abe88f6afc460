// 3D real FFT passes and the fused spectral operators of the PM step, templated on
// precision and transform size (included by fft_f32.cu and fft_f64.cu).
//
// Data flow of a 3D r2c transform of a real mesh R[x][y][z] (side n):
//   z_r2c : rows along z -> half spectrum T[kz][x][y]  (kz = 0..n/2; transposing store)
//   y_rows: rows along y (contiguous)                  -> T[kz][x][ky]
//   x_cols: columns along x (stride n)                 -> S[kz][kx][ky]
// and the inverse runs x_cols -> y_rows -> z_c2r.  Every pass reads and writes each
// element once: loads go straight from global memory into registers, the butterflies
// run in registers, shared memory carries only the exchanges between stages.
//
// Slab rows g = field n + x index the z passes; the half spectrum of slab row g and
// frequency kz sits at row ((g / C) (n/2 + 1) + kz) C + g % C with C = n, i.e. the
// layout [field][kz][x][y].
#pragma once

#include <math.h>

#include <algorithm>

#include "fft.cuh"
#include "internal.h"

namespace pm {

template <typename T> __device__ __forceinline__ cplx<T> tw_global(int k);
cudaError_t set_smem_once(const void* fn, size_t bytes);

// The per-stage twiddle table of a length-L transform (layout: fft.cuh, tw_stage_offset).
template <typename T, int L>
__device__ __forceinline__ void load_stage_twiddles(cplx<T>* tw) {
    constexpr int TE = tw_stage_entries(L);
    for (int k = threadIdx.x; k < TE; k += blockDim.x) {
        int Ns = radix_at(L, 1), off = 0;  // stages with span Ns > 1, in order
        while (k >= off + (radix_at(L, Ns) - 1) * Ns) {
            off += (radix_at(L, Ns) - 1) * Ns;
            Ns *= radix_at(L, Ns);
        }
        const int R = radix_at(L, Ns);
        const int r = (k - off) / Ns + 1, jm = (k - off) % Ns;
        tw[k] = tw_global<T>(jm * r * (1024 / (Ns * R)));
    }
}

// First `count` entries of the length-L table.
template <typename T>
__device__ __forceinline__ void load_twiddles_head(cplx<T>* tw, int L, int count) {
    const int stride = 1024 / L;
    for (int k = threadIdx.x; k < count; k += blockDim.x) tw[k] = tw_global<T>(k * stride);
}


// a / d in the per-mode operators.  FP32 divides as written.  FP64 divides are slow on this
// part, so FP64 computes the reciprocal of d by the Newton-Raphson iteration for 1/d,
// r <- r + r (1 - d r), started from the FP32 reciprocal of d and run twice (the relative
// error squares each time: ~2^-23, then ~2^-46, then below the FP64 rounding), and returns
// a r.  d must lie in the FP32 normal range (about 1.2e-38 .. 3.4e38; the operators' k^2
// and constraint denominators do).  pm_div_mode_check compares it with the division.
template <typename T> __device__ __forceinline__ T div_mode(T a, T d) { return a / d; }
template <> __device__ __forceinline__ double div_mode<double>(double a, double d) {
    double r = (double)__frcp_rn((float)d);
    r = fma(r, fma(-d, r, 1.0), r);
    r = fma(r, fma(-d, r, 1.0), r);
    return a * r;
}

// Opts a kernel into more than 48 KB of dynamic shared memory once per device, so that
// launches (including those recorded into a CUDA graph) make no further attribute calls.
static inline cudaError_t set_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return set_smem_once(fn, bytes);
}

// Launch shapes (compile time): sequences per CTA for each pass.
template <typename T, int LOGN> struct Shape {
    static constexpr int N = 1 << LOGN;
    static constexpr int M = N / 2;
    static constexpr int QN = N / 8;            // threads per length-N sequence
    static constexpr int QM = (M >= 8) ? M / 8 : 1;
    static constexpr int YB = (512 / QM < N) ? 512 / QM : N;     // z passes: rows per CTA
    static constexpr int RB = (256 / QN > 0) ? 256 / QN : 1;     // y pass
    static constexpr int RB3 = (sizeof(T) == 8) ? ((128 / QN > 0) ? 128 / QN : 1) : RB;  // y grad3
    static constexpr int CB0 = (512 / QN < N) ? 512 / QN : N;
    // x pass columns (FP64 halves them from n = 64 so that the exchange buffers and the
    // prefetch stage stay within 227 KB of shared memory)
    static constexpr int CB = (sizeof(T) == 8 && N >= 64) ? CB0 / 2 : CB0;
};

// Row of (slab row gl = field n + x, frequency kz) in the half spectra [field][kz][x][ky].
template <int M, int LOGN>
__device__ __forceinline__ size_t spec_row(int gl, int kz) {
    return ((size_t)((gl >> LOGN) * (M + 1) + kz) << LOGN) + (gl & ((1 << LOGN) - 1));
}

// =============================================================== z: r2c
// sub is subtracted from every input value as it is loaded: the mean of a density mesh (its
// zero mode, which no operator of the path uses), so that the transform's rounding scales
// with the fluctuations rather than with the mean.  With sub = 1, v - 1 is exact for v in
// [0.5, 2^24] and below 0.5 within half the spacing of the values near 1 (2^-25 in FP32).
template <typename T, int LOGN>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 4 : 2) k_z_r2c(const T* __restrict__ in, cplx<T>* __restrict__ out,
                                                                       T sub) {
    typedef cplx<T> C;
    typedef Shape<T, LOGN> S;
    constexpr int N = S::N, M = S::M, Q = S::QM, YB = S::YB;
    typedef RowLayout<M, true> LAY;
    constexpr int RS = LAY::RS;
    constexpr int TWN = (M + 2) & ~1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twM = reinterpret_cast<C*>(smem_raw);
    C* twN = twM + M;
    C* buf = twN + TWN;
    const int tid = threadIdx.x;
    const int y0 = blockIdx.x * YB;
    const int gl = blockIdx.y;
    const size_t g = gl;
    load_stage_twiddles<T, M>(twM);
    load_twiddles_head<T>(twN, N, M + 1);
    const int b = tid / Q, t = tid % Q;
    const C* row = reinterpret_cast<const C*>(in + (g * N + y0 + b) * N);
    C v[1][8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
        v[0][m] = row[t + m * Q];
        v[0][m].x -= sub;
        v[0][m].y -= sub;
    }
    __syncthreads();
    RowEx<C, 1, false, LAY> ex{buf, YB, RS, b, 0};
    fft_regs<M, 1, false>(v, t, twM, ex);
    C* z = buf;
    __syncthreads();  // every thread has read its last exchange before the buffer is reused
#pragma unroll
    for (int m = 0; m < 8; ++m) z[b * RS + LAY::slot(t + m * Q)] = v[0][m];
    __syncthreads();
    constexpr int NT = YB * Q, ITERS = ((M + 1) * YB + NT - 1) / NT;
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int e = tid + it * NT;
        if (e >= (M + 1) * YB) break;
        const int k = e / YB, bb = e % YB;
        const C z1 = z[bb * RS + LAY::slot(k == M ? 0 : k)];
        const C z2 = cconj(z[bb * RS + LAY::slot(k == 0 ? 0 : M - k)]);
        const C E = cscale(cadd(z1, z2), T(0.5));
        const C O = cscale(cmul_mi<false>(csub(z1, z2)), T(0.5));
        out[spec_row<M, LOGN>(gl, k) * N + y0 + bb] = cadd(E, cmul(twN[k], O));
    }
}

// =============================================================== z: c2r
template <typename T> struct Ptr3 {
    const cplx<T>* in[3];
    T* out[3];
    T* zero = nullptr;  // optional mesh of the same shape as out, set to 0 by the component-0 CTAs
};

template <typename T, int LOGN>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 4 : 2) k_z_c2r(Ptr3<T> P, unsigned gradz_mask, T kf0,
                                                                       const double* __restrict__ kf_arr) {
    typedef cplx<T> C;
    typedef Shape<T, LOGN> S;
    constexpr int N = S::N, M = S::M, Q = S::QM, YB = S::YB;
    typedef RowLayout<M, true> LAY;
    constexpr int RS = LAY::RS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* twM = reinterpret_cast<C*>(smem_raw);
    C* buf = twM + M;
    const int tid = threadIdx.x;
    const int comp = blockIdx.z;
    const bool grad = (gradz_mask >> comp) & 1u;
    const int y0 = blockIdx.x * YB;
    const int gl = blockIdx.y;
    const size_t g = gl;
    load_stage_twiddles<T, M>(twM);
    const T kf = kf_arr ? T(kf_arr[gl >> LOGN]) : kf0;
    const C* inp = comp == 0 ? P.in[0] : (comp == 1 ? P.in[1] : P.in[2]);
    T* pout = comp == 0 ? P.out[0] : (comp == 1 ? P.out[1] : P.out[2]);
    C* xb = buf;  // the pre-processed half spectrum; the FFT exchanges reuse the buffer afterwards
    // Each thread loads the pairs (X_k, X_{M-k}), k = 0..M/2, of its columns -- all of its
    // strided row segments in flight together -- and forms in registers
    //   Y_k = (X_k + X*_{M-k}) + i (X_k - X*_{M-k}) exp(+2 pi i k / N)   (and Y_{M-k} likewise),
    // the M-point sequence whose inverse transform interleaves the real output.
    constexpr int NT = YB * Q, NP = (M / 2 + 1) * YB, ITERS = (NP + NT - 1) / NT;
    C X1[ITERS], X2[ITERS];
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int e = tid + it * NT;
        if (e < NP) {
            const int k = e / YB, col = y0 + e % YB;
            X1[it] = inp[spec_row<M, LOGN>(gl, k) * N + col];
            X2[it] = inp[spec_row<M, LOGN>(gl, M - k) * N + col];
        }
    }
    constexpr int TWS = 1024 / N;  // exp(-2 pi i k / N) = global table entry k TWS
#pragma unroll
    for (int it = 0; it < ITERS; ++it) {
        const int e = tid + it * NT;
        if (e < NP) {
            const int k = e / YB, bb = e % YB;
            C a = X1[it], c = X2[it];
            if (grad) {  // (-i kz) X, Nyquist kz -> 0
                const T kza = kf * T(k), kzc = (k == 0) ? T(0) : kf * T(M - k);
                a = cmake<C>(a.y * kza, -a.x * kza);
                c = cmake<C>(c.y * kzc, -c.x * kzc);
            }
            if (k == 0) {
                a.y = T(0);
                c.y = T(0);
            }
            C* r = xb + bb * RS;
            const C bconj = cconj(c);
            const C d = cmul(csub(a, bconj), cconj(tw_global<T>(k * TWS)));
            r[LAY::slot(k)] = cadd(cadd(a, bconj), cmake<C>(-d.y, d.x));
            if (k > 0 && k < M - k) {
                const C aconj = cconj(a);
                const C d2 = cmul(csub(c, aconj), cconj(tw_global<T>((M - k) * TWS)));
                r[LAY::slot(M - k)] = cadd(cadd(c, aconj), cmake<C>(-d2.y, d2.x));
            }
        }
    }
    __syncthreads();
    const int b = tid / Q, t = tid % Q;
    C v[1][8];
#pragma unroll
    for (int m = 0; m < 8; ++m) v[0][m] = xb[b * RS + LAY::slot(t + m * Q)];
    RowEx<C, 1, false, LAY> ex{buf, YB, RS, b, 0};
    fft_regs<M, 1, true>(v, t, twM, ex);
    C* orow = reinterpret_cast<C*>(pout + (g * N + y0 + b) * N);
#pragma unroll
    for (int m = 0; m < 8; ++m) orow[t + m * Q] = v[0][m];
    if (P.zero && comp == 0) {  // the same rows of the mesh the caller clears for its next use
        C* zrow = reinterpret_cast<C*>(P.zero + (g * N + y0 + b) * N);
#pragma unroll
        for (int m = 0; m < 8; ++m) zrow[t + m * Q] = cmake<C>(T(0), T(0));
    }
}

// =============================================================== y: contiguous rows
// In place when in == out.
template <typename T, int LOGN, bool INV>
__global__ void __launch_bounds__(512) k_y_rows(const cplx<T>* in, cplx<T>* out, int64_t nrows) {
    typedef cplx<T> C;
    typedef Shape<T, LOGN> S;
    constexpr int N = S::N, Q = S::QN, RB = S::RB;
    typedef RowLayout<N, false> LAY;
    constexpr int RS = LAY::RS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const int tid = threadIdx.x;
    const int b = tid / Q, t = tid % Q;
    const int64_t r = (int64_t)blockIdx.x * RB + b;
    const bool ok = r < nrows;
    load_stage_twiddles<T, N>(tw);
    C v[1][8];
    const C* irow = in + r * N;
    if (ok) {
#pragma unroll
        for (int m = 0; m < 8; ++m) v[0][m] = irow[t + m * Q];
    }
    __syncthreads();
    RowEx<C, 1, true, LAY> ex{buf, RB, RS, b, 0};
    fft_regs<N, 1, INV>(v, t, tw, ex);
    C* orow = out + r * N;
    if (ok) {
#pragma unroll
        for (int m = 0; m < 8; ++m) orow[t + m * Q] = v[0][m];
    }
}

// A' = IFFT_y(A), B' = IFFT_y(B), C' = IFFT_y(-i ky A) (in place when Aout == A, Bout == B).
template <typename T, int LOGN>
__global__ void __launch_bounds__(512) k_y_grad3(const cplx<T>* A, const cplx<T>* B, cplx<T>* Aout, cplx<T>* Bout,
                                                 cplx<T>* __restrict__ Cout, int64_t nrows, T kf0,
                                                 const double* __restrict__ kf_arr, int64_t rows_per_field) {
    typedef cplx<T> C;
    typedef Shape<T, LOGN> S;
    constexpr int N = S::N, Q = S::QN, RB = S::RB3;
    typedef RowLayout<N, false> LAY;
    constexpr int RS = LAY::RS;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const int tid = threadIdx.x;
    const int b = tid / Q, t = tid % Q;
    const int64_t r = (int64_t)blockIdx.x * RB + b;
    const bool ok = r < nrows;
    const int64_t ri = r;
    const T kf = (kf_arr && ok) ? T(kf_arr[r / rows_per_field]) : kf0;
    load_stage_twiddles<T, N>(tw);
    // two rounds keep two sequences live at a time: (A, -i ky A), then B
    C v[2][8];
    if (ok) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int i = t + m * Q;
            const C a = A[ri * N + i];
            v[0][m] = a;
            const int ny = (i < N / 2) ? i : i - N;
            const T ky = (2 * ny == -N) ? T(0) : kf * T(ny);
            v[1][m] = cmake<C>(a.y * ky, -a.x * ky);
        }
    }
    __syncthreads();
    RowEx<C, 2, false, LAY> ex{buf, RB, RS, b, 0};
    fft_regs<N, 2, true>(v, t, tw, ex);
    if (ok) {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int i = t + m * Q;
            Aout[r * N + i] = v[0][m];
            Cout[r * N + i] = v[1][m];
        }
        // Bout may alias B, never A: the rows of A written above are not read again
#pragma unroll
        for (int m = 0; m < 8; ++m) v[0][m] = B[ri * N + t + m * Q];
    }
    RowEx<C, 1, false, LAY> ex1{buf, RB, RS, b, 0};
    fft_regs<N, 1, true>(v, t, tw, ex1);
    if (ok) {
#pragma unroll
        for (int m = 0; m < 8; ++m) Bout[r * N + t + m * Q] = v[0][m];
    }
}

// =============================================================== x: strided columns + spectral operators
// 16-byte asynchronous copy global -> shared (cp.async, completion by wait_group).
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(gmem_src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
// A hint that brings the 128-byte line holding p into L2 (no register, no wait).
__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];\n" ::"l"(p)); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Persistent: each CTA walks blocks blk = blockIdx.x, + gridDim.x, ... of CB columns of one
// plane (plane = blk / (N / CB)).  The next block's columns are copied into a shared
// stage with cp.async while the current block is transformed, so the loads of one block
// overlap the butterflies and stores of the previous one.
// Column groups of the x pass: FP32 meshes of 256 and more take 1024-thread CTAs of twice
// the columns (full 128-byte row segments; the binning pass keeps 512 threads, its
// cross-spectrum stage would not fit).
template <typename T, int LOGN, int KIND> struct XShape {
    typedef Shape<T, LOGN> S;
    static constexpr bool WIDE = sizeof(T) == 4 && S::N >= 256 && KIND != OP_BIN;
    static constexpr int CB = WIDE ? 1024 / S::QN : S::CB;
    static constexpr int THREADS = CB * S::QN;
    static constexpr int MINB = WIDE ? 1 : (sizeof(T) == 4 ? 2 : 1);
};

// The per-mode operator of the x pass on mode (nx, ny, nz), |n|^2 = n2, of field `field`:
// the Newtonian Green's function (or the potential alone), the Zel'dovich filter, or the
// linearised Poisson-gauge constraint (which reads and updates its Phi history at `old` and,
// for |n| <= n_lo, the FP64 island).  Returns phi for the mode.
template <typename T, int KIND, int N>
__device__ __forceinline__ cplx<T> mode_op(const SpecOp& op, cplx<T> vv, int nx, int ny, int nz, int n2, int field,
                                           double kf, T kfT, T coefT, T kf2T, cplx<T>* old) {
    typedef cplx<T> C;
    constexpr int M = N / 2;
    C phi;
    if constexpr (KIND == OP_NEWTON || KIND == OP_POTENTIAL) {
        phi = (n2 == 0) ? cmake<C>(T(0), T(0)) : cscale(vv, div_mode(coefT, T(n2)));
    } else if constexpr (KIND == OP_ZA) {
        const bool nyq = (2 * nx == -N) || (2 * ny == -N) || (nz == M);
        const double* amp = op.amp + (int64_t)field * op.amp_stride;
        C g = vv;
        if (op.fixed_amp) {  // keep the phase, set |g| = 1
            const T r2 = g.x * g.x + g.y * g.y;
            g = (r2 > T(0)) ? cscale(g, rsqrt(r2)) : cmake<C>(T(0), T(0));
        }
        const double filt = op.za_filter == ZA_IDENTITY  ? op.coef
                            : op.za_filter == ZA_INV_LAPLACE ? op.coef / (kf * kf * (double)n2)
                                                             : op.coef / (kf * kf) * amp[n2] / (double)n2;
        phi = (n2 == 0 || nyq) ? cmake<C>(T(0), T(0)) : cscale(g, T(filt));
    } else {  // OP_GR
        // the FP64 island of field `field` ((n_lo + 1) (2 n_lo + 1)^2 modes a field)
        if (n2 == 0) {
            phi = cmake<C>(T(0), T(0));
            if (op.n_lo > 0) {
                const int L = op.n_lo, W2 = 2 * L + 1;
                op.island[(((size_t)field * (L + 1) + nz) * W2 + L) * W2 + L] = make_double2(0.0, 0.0);
            }
        } else if (n2 <= op.n_lo * op.n_lo) {
            const int L = op.n_lo, W2 = 2 * L + 1;
            const size_t id = (((size_t)field * (L + 1) + nz) * W2 + (nx + L)) * W2 + (ny + L);
            const double k2 = kf * kf * (double)n2;
            const double H = op.calH;
            const double num_s = -1.5 * H * H * op.omm_a;
            double den = k2 + 3.0 * H * H + 4.5 * H * H * op.omm_a;
            double2 P = make_double2(num_s * (double)vv.x, num_s * (double)vv.y);
            if (!op.first) {
                const double2 old = op.island[id];
                const double cc = 3.0 * H * op.inv_dtau;
                P.x += cc * old.x;
                P.y += cc * old.y;
                den += cc;
            }
            P.x /= den;
            P.y /= den;
            op.island[id] = P;
            phi = cmake<C>(T(P.x * op.ac2_over_n3), T(P.y * op.ac2_over_n3));
        } else {
            const T k2 = kf2T * T(n2);
            const T H = T(op.calH), om = T(op.omm_a);
            const T num_s = T(-1.5) * H * H * om;
            T den = k2 + T(3) * H * H + T(4.5) * H * H * om;
            C Pc = cscale(vv, num_s);
            if (!op.first) {
                const T cc = T(3) * H * T(op.inv_dtau);
                const C o = *old;
                Pc.x += cc * o.x;
                Pc.y += cc * o.y;
                den += cc;
            }
            Pc = cscale(Pc, div_mode(T(1), den));
            *old = Pc;
            phi = cscale(Pc, T(op.ac2_over_n3));
        }
    }
    return phi;
}

template <typename T, int LOGN, int KIND>
__global__ void __launch_bounds__(XShape<T, LOGN, KIND>::THREADS, XShape<T, LOGN, KIND>::MINB)
    k_x_cols(cplx<T>* __restrict__ data, cplx<T>* __restrict__ out2, SpecOp op, int nplanes) {
    typedef cplx<T> C;
    typedef Shape<T, LOGN> S;
    constexpr int N = S::N, M = S::M, Q = S::QN, CB = XShape<T, LOGN, KIND>::CB;
    constexpr int CS = CB + 1;
    constexpr int NCG = N / CB;                              // column groups per plane
    constexpr int CHUNKS_ROW = CB * (int)sizeof(C) / 16;     // 16-byte chunks per row of a group
    static_assert(CB * sizeof(C) % 16 == 0, "column groups of whole 16-byte chunks");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const bool cross = (KIND == OP_BIN) && op.in2 != nullptr;
    C* stage = buf + (size_t)2 * N * CS;                     // [1 + cross][N][CB]: field (and in2)
    // OP_BIN: 1 / W^2 of the CIC window per |n_j| (W per axis from the FP64 table), in T
    T* iw2 = reinterpret_cast<T*>(stage + (size_t)(cross ? 2 : 1) * N * CB);
    const int tid = threadIdx.x;
    const int b = tid % CB, t = tid / CB;
    const int64_t nblk = (int64_t)nplanes * NCG;
    load_stage_twiddles<T, N>(tw);
    if (KIND == OP_BIN)
        for (int e = tid; e <= M; e += blockDim.x) iw2[e] = op.deconv ? T(1.0 / (op.wtab[e] * op.wtab[e])) : T(1);
    // OP_BIN: this CTA's row of per-bin sums in global memory (zeroed by the caller)
    double* acc_row = (KIND == OP_BIN) ? op.acc + (size_t)blockIdx.x * op.nbins : nullptr;
    // with a cross spectrum, optionally the auto spectrum of the second field in the same pass
    double* acc2_row = (KIND == OP_BIN && cross && op.acc2) ? op.acc2 + (size_t)blockIdx.x * op.nbins : nullptr;
    auto issue = [&](int64_t blk) {
        const size_t pb = (size_t)(blk / NCG) * N * N + (size_t)(blk % NCG) * CB;
        if constexpr (KIND == OP_GR) {
            // the Poisson-gauge constraint reads this block's Phi_old after the forward
            // transform: its lines are brought into L2 now, one block ahead, with the data
            constexpr int LINES = CB * (int)sizeof(C) >= 128 ? CB * (int)sizeof(C) / 128 : 1;
            constexpr int THREADS = XShape<T, LOGN, KIND>::THREADS;  // the launch's block size
            const C* ph = reinterpret_cast<const C*>(op.phi_old) + pb;
#pragma unroll
            for (int q0 = 0; q0 < N * LINES; q0 += THREADS) {
                const int q = q0 + tid;
                if (q < N * LINES)
                    prefetch_l2(reinterpret_cast<const char*>(ph + (size_t)(q / LINES) * N) + 128 * (q % LINES));
            }
        }
        for (int q = tid; q < N * CHUNKS_ROW; q += blockDim.x) {
            const int r = q / CHUNKS_ROW, h = q % CHUNKS_ROW;
            cp_async16(reinterpret_cast<char*>(stage + (size_t)r * CB) + 16 * h,
                       reinterpret_cast<const char*>(data + pb + (size_t)r * N) + 16 * h);
            if (cross)
                cp_async16(reinterpret_cast<char*>(stage + (size_t)(N + r) * CB) + 16 * h,
                           reinterpret_cast<const char*>(reinterpret_cast<const C*>(op.in2) + pb + (size_t)r * N) +
                               16 * h);
        }
        cp_async_commit();
    };
    if ((int64_t)blockIdx.x < nblk) issue(blockIdx.x);
#pragma unroll 1
    for (int64_t blk = blockIdx.x; blk < nblk; blk += gridDim.x) {
        const int plane = (int)(blk / NCG);
        const int kz = plane % (M + 1);
        const int field = plane / (M + 1);
        const double kf = op.kf_arr ? op.kf_arr[field] : op.kf;
        const int c = (int)(blk % NCG) * CB + b;
        const size_t pbase = (size_t)plane * N * N;
        C* base = data + pbase;
        cp_async_wait_all();
        __syncthreads();
        C v[2][8];
#pragma unroll
        for (int m = 0; m < 8; ++m) v[0][m] = stage[(size_t)(t + m * Q) * CB + b];
        if (cross) {
#pragma unroll
            for (int m = 0; m < 8; ++m) v[1][m] = stage[(size_t)(N + t + m * Q) * CB + b];
        }
        __syncthreads();  // the stage is free: fetch the next block while this one is transformed
        if (blk + gridDim.x < nblk) issue(blk + gridDim.x);
        ColEx<C, N> ex{buf, CS, b};
        if (op.fwd) {
            if (cross) fft_regs<N, 2, false>(v, t, tw, ex);
            else fft_regs<N, 1, false>(v, t, tw, ex);
        }
        if constexpr (KIND == OP_FWD_STORE) {
#pragma unroll
            for (int m = 0; m < 8; ++m) base[(size_t)(t + m * Q) * N + c] = v[0][m];
            continue;
        }
        if constexpr (KIND == OP_INV) {
            fft_regs<N, 1, true>(v, t, tw, ex);
#pragma unroll
            for (int m = 0; m < 8; ++m) base[(size_t)(t + m * Q) * N + c] = v[0][m];
            continue;
        }
        if constexpr (KIND == OP_BIN) {
            // regroup through the exchange buffer so that the thread holds kx = 8 t + m
            // (m = 0..7): neighbouring kx mostly share a |k| bin, so runs merge in registers
            __syncthreads();  // the transform's last exchange has been read
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                buf[(size_t)(t + m * Q) * CS + b] = v[0][m];
                if (cross) buf[(size_t)(N + t + m * Q) * CS + b] = v[1][m];
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                v[0][m] = buf[(size_t)(8 * t + m) * CS + b];
                if (cross) v[1][m] = buf[(size_t)(N + 8 * t + m) * CS + b];
            }
        }
        // ---- per-mode operator on modes (kx = t + m Q, or 8 t + m when binning; ky = c, kz)
        const int ny = (c < M) ? c : c - N;
        const int nz = kz;
        // per-CTA constants, formed once in the working precision (no FP64 work per mode in FP32)
        const T kfT = T(kf);
        const T coefT = T(op.coef) / (kfT * kfT);
        const T kf2T = T(kf * kf);
        // OP_BIN: consecutive modes of a thread that fall in the same bin are summed in
        // registers, each run added once to the CTA's row (native FP64 reduction in L2)
        int run_bin = -1;
        T run_sum = T(0), run_sum2 = T(0);
        const T wyz = (KIND == OP_BIN) ? iw2[ny < 0 ? -ny : ny] * iw2[nz] * T((nz == 0 || nz == M) ? 1 : 2) : T(1);
        // OP_BIN: the thread's modes kx = 8 t .. 8 t + 7 lie on one side of the Nyquist index, so
        // |n|^2 is monotone over them, and a bin is a contiguous range of |n|^2: when the first
        // and the last mode fall in the same bin (neither the zero mode nor beyond (n/2)^2), so
        // do all eight, and two table lookups replace eight
        int bin_all = -1;
        if constexpr (KIND == OP_BIN) {
            const int ia = 8 * t, ib = 8 * t + 7;
            const int nxa = (ia < M) ? ia : ia - N, nxb = (ib < M) ? ib : ib - N;
            const int n2a = nxa * nxa + ny * ny + nz * nz, n2b = nxb * nxb + ny * ny + nz * nz;
            if (n2a > 0 && n2b > 0 && n2a <= M * M && n2b <= M * M) {
                const int ba = op.bin_of[n2a], bb = op.bin_of[n2b];
                if (ba == bb) bin_all = ba;
            }
        }
    #pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int i = (KIND == OP_BIN) ? 8 * t + m : t + m * Q;
            const int nx = (i < M) ? i : i - N;
            const int n2 = nx * nx + ny * ny + nz * nz;
            const C vv = v[0][m];
            if constexpr (KIND == OP_BIN) {
                if (n2 == 0 || n2 > M * M) continue;
                const int bin = (bin_all >= 0) ? bin_all : op.bin_of[n2];
                if (bin < 0) continue;
                const C u = cross ? v[1][m] : vv;
                // w |delta_n|^2 / W^2 (or the cross product), w = 1 on the kz = 0, n/2 planes, 2 elsewhere
                const T wgt = iw2[nx < 0 ? -nx : nx] * wyz;
                const T val = (vv.x * u.x + vv.y * u.y) * wgt;
                const T val2 = acc2_row ? (u.x * u.x + u.y * u.y) * wgt : T(0);
                if (bin != run_bin) {
                    if (run_bin >= 0) {
                        atomicAdd(acc_row + run_bin, (double)run_sum);
                        if (acc2_row) atomicAdd(acc2_row + run_bin, (double)run_sum2);
                    }
                    run_bin = bin;
                    run_sum = val;
                    run_sum2 = val2;
                } else {
                    run_sum += val;
                    run_sum2 += val2;
                }
            } else {
                const C phi = mode_op<T, KIND, N>(op, vv, nx, ny, nz, n2, field, kf, kfT, coefT, kf2T,
                                                  reinterpret_cast<C*>(op.phi_old) + pbase + (size_t)i * N + c);
                v[0][m] = phi;
                if constexpr (KIND != OP_POTENTIAL) {
                    const T kx = (2 * nx == -N) ? T(0) : kfT * T(nx);
                    v[1][m] = cmake<C>(phi.y * kx, -phi.x * kx);  // -i kx phi
                }
            }
        }
        if constexpr (KIND == OP_BIN) {
            if (run_bin >= 0) {
                atomicAdd(acc_row + run_bin, (double)run_sum);
                if (acc2_row) atomicAdd(acc2_row + run_bin, (double)run_sum2);
            }
            continue;
        }
        if constexpr (KIND == OP_POTENTIAL) {
            fft_regs<N, 1, true>(v, t, tw, ex);
    #pragma unroll
            for (int m = 0; m < 8; ++m) base[(size_t)(t + m * Q) * N + c] = v[0][m];
        } else {
            fft_regs<N, 2, true>(v, t, tw, ex);
    #pragma unroll
            for (int m = 0; m < 8; ++m) {
                base[(size_t)(t + m * Q) * N + c] = v[0][m];
                out2[pbase + (size_t)(t + m * Q) * N + c] = v[1][m];
            }
        }
    }
}

// =============================================================== fused middle passes
// The three passes between the forward z and the inverse z transforms of a force
// evaluation -- forward y, x with the Green's function (or the Poisson-gauge constraint)
// and the x gradient, inverse y with the y gradient -- touch only one kz plane of the half
// spectrum each.  One persistent launch runs them plane by plane: a CTA takes items from a
// queue (item = one phase on a block of rows or columns of one plane) in rounds; round r
// holds the forward-y items of plane r, the x items of plane r - LAG and the inverse-y items
// of plane r - 2 LAG, so a plane's intermediate spectra are read back a few planes after they
// were written, from L2, and only the z pass's spectrum (read) and the three y-inverted
// spectra (written) go through HBM: 4 half spectra instead of 10.
// An item of the x phase waits for the plane's forward-y items to be done, an inverse-y item
// for its x items.  Every item waited on was handed out earlier, to a CTA that is running,
// so every wait ends; each wait still gives up after kMidSpinLimit polls (about a second),
// sets the error word and lets the CTA go on, so that a fault cannot hang the GPU.
struct MidSync {
    unsigned* queue;   // next item
    unsigned* done_y;  // [nplanes] finished forward-y items
    unsigned* done_x;  // [nplanes] finished x items
    unsigned* error;   // nonzero: a wait gave up
};
constexpr unsigned kMidSpinLimit = 1u << 23;

template <typename T, int LOGN, int THREADS_> struct MidShape {
    static constexpr int N = 1 << LOGN, M = N / 2, QN = N / 8;
    static constexpr int THREADS = THREADS_;
    static constexpr int RB = THREADS / QN;  // rows of a y item
    static constexpr int CB = THREADS / QN;  // columns of an x item
    static constexpr int ITEMS = N / RB;     // items of each phase per plane
    static constexpr int MINB = 1024 / THREADS;  // 64 registers a thread
    typedef RowLayout<N, false> LAY;
    // twiddles + the larger of the y exchange (two rows buffers of RB rows) and the x exchange
    // (two sequences of N x (CB + 1))
    static constexpr int XWORDS = 2 * N * (CB + 1), YWORDS = 2 * RB * LAY::RS;
    static constexpr size_t SMEM = sizeof(cplx<T>) * (N + (XWORDS > YWORDS ? XWORDS : YWORDS));
};

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];\n" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0 waits until *cnt reaches target (bounded), then the CTA proceeds.
__device__ __forceinline__ void mid_wait(const unsigned* cnt, unsigned target, unsigned* error) {
    if (threadIdx.x == 0) {
        unsigned polls = 0;
        while (ld_acquire_u32(cnt) < target) {
            if (++polls > kMidSpinLimit || *(volatile unsigned*)error) {
                atomicExch(error, 1u);
                break;
            }
            __nanosleep(128);
        }
    }
    __syncthreads();
}

// lag: rounds between the phases of one plane, chosen by the launcher so that an item's
// dependencies were handed out more items earlier than there are CTAs in flight.
template <typename T, int LOGN, int KIND, int THREADS>
__global__ void __launch_bounds__(THREADS, 1024 / THREADS)
    k_mid(cplx<T>* __restrict__ A, cplx<T>* __restrict__ B, cplx<T>* __restrict__ Cs, SpecOp op, int nplanes, int lag,
          MidSync sync) {
    typedef cplx<T> C;
    typedef MidShape<T, LOGN, THREADS> SH;
    constexpr int N = SH::N, M = SH::M, Q = SH::QN, RB = SH::RB, CB = SH::CB, ITEMS = SH::ITEMS;
    typedef typename SH::LAY LAY;
    constexpr int RS = LAY::RS, CS = CB + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    __shared__ unsigned s_item;
    const int tid = threadIdx.x;
    load_stage_twiddles<T, N>(tw);
    const unsigned rounds = (unsigned)(nplanes + 2 * lag);
    const unsigned total = rounds * 3 * ITEMS;
#pragma unroll 1
    for (;;) {
        __syncthreads();  // the previous item's last reads of s_item and of the exchange buffers
        if (tid == 0) s_item = *(volatile unsigned*)sync.error ? total : atomicAdd(sync.queue, 1u);
        __syncthreads();
        const unsigned it = s_item;
        if (it >= total) break;
        const int r = (int)(it / (3 * ITEMS)), k = (int)(it % (3 * ITEMS));
        const int phase = k / ITEMS, blk = k % ITEMS;
        const int plane = r - phase * lag;
        if (plane < 0 || plane >= nplanes) continue;
        const size_t pbase = (size_t)plane * N * N;
        const int kz = plane % (M + 1);
        const int field = plane / (M + 1);
        const double kf = op.kf_arr ? op.kf_arr[field] : op.kf;
        const T kfT = T(kf);
        if (phase == 0) {
            // ---- forward y of rows x = blk RB .. + RB (in place in A)
            const int b = tid / Q, t = tid % Q;
            C* row = A + pbase + (size_t)(blk * RB + b) * N;
            C v[1][8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[0][m] = __ldcg(row + t + m * Q);
            RowEx<C, 1, true, LAY> ex{buf, RB, RS, b, 0};
            fft_regs<N, 1, false>(v, t, tw, ex);
#pragma unroll
            for (int m = 0; m < 8; ++m) row[t + m * Q] = v[0][m];
        } else if (phase == 1) {
            // ---- x pass of columns c = blk CB .. + CB: forward x, per-mode operator, phi and
            //      -i kx phi back along x (phi in place in A, -i kx phi to B)
            mid_wait(sync.done_y + plane, ITEMS, sync.error);
            const int b = tid % CB, t = tid / CB;
            const int c = blk * CB + b;
            C* base = A + pbase;
            C v[2][8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[0][m] = __ldcg(base + (size_t)(t + m * Q) * N + c);
            ColEx<C, N> ex{buf, CS, b};
            fft_regs<N, 1, false>(v, t, tw, ex);
            const int ny = (c < M) ? c : c - N;
            const T coefT = T(op.coef) / (kfT * kfT);
            const T kf2T = T(kf * kf);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int i = t + m * Q;
                const int nx = (i < M) ? i : i - N;
                const int n2 = nx * nx + ny * ny + kz * kz;
                const C phi = mode_op<T, KIND, N>(op, v[0][m], nx, ny, kz, n2, field, kf, kfT, coefT, kf2T,
                                                  reinterpret_cast<C*>(op.phi_old) + pbase + (size_t)i * N + c);
                v[0][m] = phi;
                const T kx = (2 * nx == -N) ? T(0) : kfT * T(nx);
                v[1][m] = cmake<C>(phi.y * kx, -phi.x * kx);  // -i kx phi
            }
            fft_regs<N, 2, true>(v, t, tw, ex);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                base[(size_t)(t + m * Q) * N + c] = v[0][m];
                B[pbase + (size_t)(t + m * Q) * N + c] = v[1][m];
            }
        } else {
            // ---- inverse y of rows x = blk RB .. + RB: A <- IFFT_y(A), C <- IFFT_y(-i ky A),
            //      B <- IFFT_y(B)
            mid_wait(sync.done_x + plane, ITEMS, sync.error);
            const int b = tid / Q, t = tid % Q;
            const size_t ro = pbase + (size_t)(blk * RB + b) * N;
            C v[2][8];
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int i = t + m * Q;
                const C a = __ldcg(A + ro + i);
                v[0][m] = a;
                const int ny = (i < M) ? i : i - N;
                const T ky = (2 * ny == -N) ? T(0) : kfT * T(ny);
                v[1][m] = cmake<C>(a.y * ky, -a.x * ky);
            }
            RowEx<C, 2, false, LAY> ex{buf, RB, RS, b, 0};
            fft_regs<N, 2, true>(v, t, tw, ex);
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                A[ro + t + m * Q] = v[0][m];
                Cs[ro + t + m * Q] = v[1][m];
            }
#pragma unroll
            for (int m = 0; m < 8; ++m) v[0][m] = __ldcg(B + ro + t + m * Q);
            RowEx<C, 1, false, LAY> ex1{buf, RB, RS, b, 0};
            fft_regs<N, 1, true>(v, t, tw, ex1);
#pragma unroll
            for (int m = 0; m < 8; ++m) B[ro + t + m * Q] = v[0][m];
        }
        if (phase < 2) {
            __syncthreads();  // every store of the item is made before it is counted
            if (tid == 0) {
                __threadfence();
                atomicAdd((phase == 0 ? sync.done_y : sync.done_x) + plane, 1u);
            }
        }
    }
}

// =============================================================== whole kz planes in shared memory
// On meshes of 64^3 and 128^3 one kz plane of the half spectrum (N^2 complex: 128 KB in FP32 at
// N = 128) fits in a CTA's shared memory.  k_plane runs the middle of a force evaluation on it:
// forward y (rows), forward x (columns) with the per-mode operator, then for each force
// component j the inverse x and inverse y transforms of -i k_j phi, written straight to that
// component's spectrum (x to GX, y to GY, z over A; the z pass then needs no z gradient).  HBM
// sees one read of the plane and three writes.  A row's or a column's transform uses its own
// slots of the plane as its exchange space; phi stays in registers between the components.
template <typename T, int LOGN> struct PlaneShape {
    static constexpr int N = 1 << LOGN, M = N / 2, Q = N / 8;
    static constexpr int THREADS = 8 * N;          // 64 sequences of N at a time
    static constexpr int SEQ = THREADS / Q;
    static constexpr int ROUNDS = N / SEQ;
    static constexpr int MINB = (THREADS >= 1024) ? 1 : 1024 / THREADS;  // 64 registers a thread
    static constexpr size_t SMEM = sizeof(cplx<T>) * ((size_t)N + (size_t)N * N);
    static_assert(ROUNDS >= 1 && SEQ * ROUNDS == N, "whole rounds of rows and columns");
};

template <typename T, int LOGN, int KIND>
__global__ void __launch_bounds__(PlaneShape<T, LOGN>::THREADS, PlaneShape<T, LOGN>::MINB)
    k_plane(cplx<T>* __restrict__ A, cplx<T>* __restrict__ GX, cplx<T>* __restrict__ GY, SpecOp op, int nplanes) {
    typedef cplx<T> C;
    typedef PlaneShape<T, LOGN> SH;
    constexpr int N = SH::N, M = SH::M, Q = SH::Q, SEQ = SH::SEQ, ROUNDS = SH::ROUNDS;
    typedef RowLayout<N, false> LAY;  // a permutation within each row's N slots
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* P = tw + N;
    const int tid = threadIdx.x;
    load_stage_twiddles<T, N>(tw);
#pragma unroll 1
    for (int plane = blockIdx.x; plane < nplanes; plane += gridDim.x) {
        const size_t pbase = (size_t)plane * N * N;
        const int kz = plane % (M + 1);
        const int field = plane / (M + 1);
        const double kf = op.kf_arr ? op.kf_arr[field] : op.kf;
        const T kfT = T(kf);
        __syncthreads();  // the previous plane's last reads of P and of the twiddles' set-up
        for (int e = tid; e < N * N; e += SH::THREADS) P[e] = __ldcs(A + pbase + e);
        __syncthreads();
        // ---- forward y of the N rows
#pragma unroll 1
        for (int r = 0; r < ROUNDS; ++r) {
            const int b = tid / Q, t = tid % Q;
            C* row = P + (size_t)(r * SEQ + b) * N;
            C v[1][8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[0][m] = row[t + m * Q];
            RowEx<C, 1, false, LAY> ex{P + (size_t)r * SEQ * N, SEQ, N, b, 0};
            fft_regs<N, 1, false>(v, t, tw, ex);
            __syncthreads();  // the row's last exchange has been read
#pragma unroll
            for (int m = 0; m < 8; ++m) row[t + m * Q] = v[0][m];
        }
        __syncthreads();
        // ---- forward x of the N columns and the per-mode operator: phi in registers
        C phi[ROUNDS][8];
        const T coefT = T(op.coef) / (kfT * kfT);
        const T kf2T = T(kf * kf);
#pragma unroll
        for (int r = 0; r < ROUNDS; ++r) {
            const int b = tid % SEQ, t = tid / SEQ;
            const int c = r * SEQ + b;
            C v[1][8];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[0][m] = P[(size_t)(t + m * Q) * N + c];
            ColEx<C, N> ex{P + r * SEQ, N, b};
            fft_regs<N, 1, false>(v, t, tw, ex);
            const int ny = (c < M) ? c : c - N;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int i = t + m * Q;
                const int nx = (i < M) ? i : i - N;
                const int n2 = nx * nx + ny * ny + kz * kz;
                phi[r][m] = mode_op<T, KIND, N>(op, v[0][m], nx, ny, kz, n2, field, kf, kfT, coefT, kf2T,
                                                reinterpret_cast<C*>(op.phi_old) + pbase + (size_t)i * N + c);
            }
        }
        // ---- each component: -i k_j phi back along x (columns), then along y (rows), to its spectrum
#pragma unroll 1
        for (int j = 0; j < 3; ++j) {
            C* out = (j == 0) ? GX : (j == 1 ? GY : A);
            __syncthreads();  // every read of P by the previous pass is done
#pragma unroll
            for (int r = 0; r < ROUNDS; ++r) {
                const int b = tid % SEQ, t = tid / SEQ;
                const int c = r * SEQ + b;
                const int ny = (c < M) ? c : c - N;
                const T ky = (2 * ny == -N) ? T(0) : kfT * T(ny);
                const T kzv = (kz == M) ? T(0) : kfT * T(kz);
                C v[1][8];
#pragma unroll
                for (int m = 0; m < 8; ++m) {
                    const int i = t + m * Q;
                    const int nx = (i < M) ? i : i - N;
                    const T kx = (2 * nx == -N) ? T(0) : kfT * T(nx);
                    const T kj = (j == 0) ? kx : (j == 1 ? ky : kzv);
                    v[0][m] = cmake<C>(phi[r][m].y * kj, -phi[r][m].x * kj);  // -i k_j phi
                }
                ColEx<C, N> ex{P + r * SEQ, N, b};
                fft_regs<N, 1, true>(v, t, tw, ex);
                __syncthreads();  // the column's last exchange has been read
#pragma unroll
                for (int m = 0; m < 8; ++m) P[(size_t)(t + m * Q) * N + c] = v[0][m];
            }
            __syncthreads();
#pragma unroll 1
            for (int r = 0; r < ROUNDS; ++r) {
                const int b = tid / Q, t = tid % Q;
                const C* row = P + (size_t)(r * SEQ + b) * N;
                C v[1][8];
#pragma unroll
                for (int m = 0; m < 8; ++m) v[0][m] = row[t + m * Q];
                RowEx<C, 1, false, LAY> ex{P + (size_t)r * SEQ * N, SEQ, N, b, 0};
                fft_regs<N, 1, true>(v, t, tw, ex);
                C* orow = out + pbase + (size_t)(r * SEQ + b) * N;
#pragma unroll
                for (int m = 0; m < 8; ++m) orow[t + m * Q] = v[0][m];
            }
        }
    }
}

// =============================================================== x: adjoint combine
// Transposed force chain on the x pass: the three y-transformed spectra of the deposited
// adjoint momenta V_j (fields j = 0, 1, 2 back to back, [kz][x][ky]) are transformed
// along x one after the other and accumulated as out = sum_j i k_j c(k) V_j,
// c = coef / (kf^2 |n|^2) (zero mode 0, k_j = 0 at its Nyquist index), then transformed
// back along x into out ([kz][x][ky], ready for the inverse y and z passes).  GR: the
// Poisson-gauge operator of AdjGrOp instead of c(k), with the carried spectrum gr.Z.  FD (the
// first-order gradient): V is one scalar field and W = FFT_x V, without the i k_j factors.
template <typename T, int LOGN, bool GR, bool FD>
__global__ void __launch_bounds__(512, sizeof(T) == 4 ? 2 : 1) k_x_adj(const cplx<T>* V,
                                                                      cplx<T>* out, double kf,
                                                                      double coef, float4* __restrict__ zero,
                                                                      int64_t nzero4, AdjGrOp gr) {
    typedef cplx<T> C;
    typedef Shape<T, LOGN> S;
    constexpr int N = S::N, M = S::M, Q = S::QN, CB = S::CB;
    constexpr int CS = CB + 1;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* buf = tw + N;
    const int tid = threadIdx.x;
    const int b = tid % CB, t = tid / CB;
    const int kz = blockIdx.y;
    const int c = blockIdx.x * CB + b;
    const size_t pbase = (size_t)kz * N * N;
    const size_t field = (size_t)(M + 1) * N * N;
    load_stage_twiddles<T, N>(tw);
    {  // side job: clear `zero` (a buffer the caller has finished with), grid-stride
        const int64_t nthr = (int64_t)gridDim.x * gridDim.y * blockDim.x;
        for (int64_t e = ((int64_t)blockIdx.y * gridDim.x + blockIdx.x) * blockDim.x + tid; e < nzero4; e += nthr)
            zero[e] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    const T kfT = T(kf);
    const T coefT = T(coef) / (kfT * kfT);
    const int ny = (c < M) ? c : c - N;
    const T kyT = (2 * ny == -N) ? T(0) : kfT * T(ny);
    const T kzT = (kz == M) ? T(0) : kfT * T(kz);
    C acc[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) acc[m] = cmake<C>(T(0), T(0));
    ColEx<C, N> ex{buf, CS, b};
#pragma unroll 1
    for (int j = 0; j < (FD ? 1 : 3); ++j) {
        C v[1][8];
        const C* col = V + j * field + pbase + c;
#pragma unroll
        for (int m = 0; m < 8; ++m) v[0][m] = col[(size_t)(t + m * Q) * N];
        if (j == 0) __syncthreads();  // twiddles loaded
        fft_regs<N, 1, false>(v, t, tw, ex);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int i = t + m * Q;
            const int nx = (i < M) ? i : i - N;
            const T kj = FD ? T(1) : (j == 0) ? ((2 * nx == -N) ? T(0) : kfT * T(nx)) : (j == 1 ? kyT : kzT);
            acc[m].x += kj * v[0][m].x;
            acc[m].y += kj * v[0][m].y;
        }
    }
    C w[1][8];
    if constexpr (GR) {
        // per-evaluation constants in the working precision; den and src / carry per mode
        const T kf2 = kfT * kfT, H = T(gr.H), H1 = T(gr.H1);
        const T base = T(3) * H * H + T(4.5) * H * H * T(gr.om) + T(gr.cc);
        const T base1 = T(3) * H1 * H1 + T(4.5) * H1 * H1 * T(gr.om1) + T(gr.cc1);
        const T num = T(-1.5) * H * H * T(gr.om), cc1 = T(gr.cc1), KA = T(gr.K_ac2_n3);
        C* Zc = reinterpret_cast<C*>(gr.Z);
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int i = t + m * Q;
            const int nx = (i < M) ? i : i - N;
            const int n2 = nx * nx + ny * ny + kz * kz;
            const T k2 = kf2 * T(n2);
            const T src = (n2 == 0) ? T(0) : div_mode(num, k2 + base);
            const T carry = (n2 == 0) ? T(0) : div_mode(cc1, k2 + base1);
            const size_t zi = pbase + (size_t)i * N + c;
            const C zo = Zc[zi];
            // K a c^2 W + carry Z, W = i acc (spectral gradient) or acc (first order)
            const C Z = FD ? cmake<C>(KA * acc[m].x + carry * zo.x, KA * acc[m].y + carry * zo.y)
                           : cmake<C>(-KA * acc[m].y + carry * zo.x, KA * acc[m].x + carry * zo.y);
            Zc[zi] = Z;
            w[0][m] = cscale(Z, src);
        }
    } else {
#pragma unroll
        for (int m = 0; m < 8; ++m) {
            const int i = t + m * Q;
            const int nx = (i < M) ? i : i - N;
            const int n2 = nx * nx + ny * ny + kz * kz;
            const T cc = (n2 == 0) ? T(0) : coefT / T(n2);
            w[0][m] = FD ? cscale(acc[m], cc) : cmake<C>(-cc * acc[m].y, cc * acc[m].x);  // (i) c sum_j k_j V_j
        }
    }
    fft_regs<N, 1, true>(w, t, tw, ex);
#pragma unroll
    for (int m = 0; m < 8; ++m) out[pbase + (size_t)(t + m * Q) * N + c] = w[0][m];
}

// =============================================================== launchers
template <typename T, int LOGN>
cudaError_t z_r2c_n(const T* in, cplx<T>* out, int rows, cudaStream_t st, double sub = 0.0) {
    typedef Shape<T, LOGN> S;
    const size_t smem = sizeof(cplx<T>) * (S::M + ((S::M + 2) & ~1) + (size_t)S::YB * RowLayout<S::M, true>::RS);
    cudaError_t e = set_smem((const void*)k_z_r2c<T, LOGN>, smem);
    if (e != cudaSuccess) return e;
    k_z_r2c<T, LOGN><<<dim3(S::N / S::YB, rows), S::YB * S::QM, smem, st>>>(in, out, (T)sub);
    return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t z_c2r_n(const Ptr3<T>& P, int ncomp, int rows, unsigned mask, double kf, cudaStream_t st,
                    const double* kf_arr) {
    typedef Shape<T, LOGN> S;
    const size_t smem = sizeof(cplx<T>) * (S::M + (size_t)S::YB * RowLayout<S::M, true>::RS);
    cudaError_t e = set_smem((const void*)k_z_c2r<T, LOGN>, smem);
    if (e != cudaSuccess) return e;
    k_z_c2r<T, LOGN><<<dim3(S::N / S::YB, rows, ncomp), S::YB * S::QM, smem, st>>>(P, mask, (T)kf, kf_arr);
    return cudaGetLastError();
}

template <typename T, int LOGN, bool INV>
cudaError_t y_rows_n(const cplx<T>* in, cplx<T>* out, int64_t nrows, cudaStream_t st) {
    typedef Shape<T, LOGN> S;
    const size_t smem = sizeof(cplx<T>) * (S::N + 2 * (size_t)S::RB * RowLayout<S::N, false>::RS);
    cudaError_t e = set_smem((const void*)k_y_rows<T, LOGN, INV>, smem);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (nrows + S::RB - 1) / S::RB;
    k_y_rows<T, LOGN, INV><<<(unsigned)nblk, S::RB * S::QN, smem, st>>>(in, out, nrows);
    return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t y_grad3_n(const cplx<T>* A, const cplx<T>* B, cplx<T>* Ao, cplx<T>* Bo, cplx<T>* Co, int64_t nrows, double kf,
                      cudaStream_t st, const double* kf_arr, int64_t rows_per_field) {
    typedef Shape<T, LOGN> S;
    const size_t smem = sizeof(cplx<T>) * (S::N + 2 * (size_t)S::RB3 * RowLayout<S::N, false>::RS);
    cudaError_t e = set_smem((const void*)k_y_grad3<T, LOGN>, smem);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (nrows + S::RB3 - 1) / S::RB3;
    k_y_grad3<T, LOGN><<<(unsigned)nblk, S::RB3 * S::QN, smem, st>>>(A, B, Ao, Bo, Co, nrows, (T)kf, kf_arr,
                                                                       rows_per_field);
    return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t forward_zy_n(const T* in, cplx<T>* spec, int batch, cudaStream_t st, double sub) {
    constexpr int N = 1 << LOGN, M = N / 2;
    cudaError_t e = z_r2c_n<T, LOGN>(in, spec, N * batch, st, sub);
    if (e != cudaSuccess) return e;
    return y_rows_n<T, LOGN, false>(spec, spec, (int64_t)batch * (M + 1) * N, st);
}

// A (phi after the inverse x pass) and B (-i kx phi) in the full layout; scratch holds
// one half spectrum for IFFT_y(-i ky A).
template <typename T, int LOGN>
cudaError_t inverse_yz_grad_n(cplx<T>* A, cplx<T>* B, cplx<T>* scratch, T* const* out, int batch, double kf,
                              const double* kf_arr, cudaStream_t st, T* zero) {
    constexpr int N = 1 << LOGN, M = N / 2;
    const int64_t rows = (int64_t)batch * (M + 1) * N;
    cudaError_t e = y_grad3_n<T, LOGN>(A, B, A, B, scratch, rows, kf, st, kf_arr, (int64_t)(M + 1) * N);
    if (e != cudaSuccess) return e;
    Ptr3<T> P;
    P.in[0] = B;        // IFFT_y(-i kx phi)   -> g_x
    P.in[1] = scratch;  // IFFT_y(-i ky phi)   -> g_y
    P.in[2] = A;        // IFFT_y(phi), -i kz  -> g_z
    for (int j = 0; j < 3; ++j) P.out[j] = out[j];
    P.zero = zero;
    return z_c2r_n<T, LOGN>(P, 3, N * batch, 4u, kf, st, kf_arr);
}

template <typename T, int LOGN, int KIND>
cudaError_t x_cols_n(cplx<T>* data, cplx<T>* out2, int nplanes, const SpecOp& op, cudaStream_t st) {
    typedef Shape<T, LOGN> S;
    typedef XShape<T, LOGN, KIND> X;
    const int nstage = (KIND == OP_BIN && op.in2 != nullptr) ? 2 : 1;
    const size_t smem = sizeof(cplx<T>) * (S::N + 2 * (size_t)S::N * (X::CB + 1) + nstage * (size_t)S::N * X::CB) +
                        (KIND == OP_BIN ? sizeof(T) * (S::M + 1) : 0);
    const void* fn = (const void*)k_x_cols<T, LOGN, KIND>;
    cudaError_t e = set_smem(fn, smem);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = resident_ctas(fn, X::THREADS, smem, &per_sm);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (int64_t)nplanes * (S::N / X::CB);
    int64_t grid = std::min<int64_t>(nblk, (int64_t)per_sm * num_sms());
    if (KIND == OP_BIN) grid = std::min<int64_t>(grid, op.acc_rows);  // one row of bin sums per CTA
    k_x_cols<T, LOGN, KIND><<<(unsigned)grid, X::THREADS, smem, st>>>(data, out2, op, nplanes);
    return cudaGetLastError();
}


template <typename T, int LOGN, int THREADS>
cudaError_t middle_n(cplx<T>* A, cplx<T>* B, cplx<T>* Cs, int nplanes, const SpecOp& op, unsigned* sync_words,
                     cudaStream_t st) {
    typedef MidShape<T, LOGN, THREADS> SH;
    const void* fn = op.kind == OP_GR ? (const void*)k_mid<T, LOGN, OP_GR, THREADS>
                                      : (const void*)k_mid<T, LOGN, OP_NEWTON, THREADS>;
    cudaError_t e = set_smem(fn, SH::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = resident_ctas(fn, SH::THREADS, SH::SMEM, &per_sm);
    if (e != cudaSuccess) return e;
    // the queue and the counters start at zero; the error word after them stays set once set
    e = cudaMemsetAsync(sync_words, 0, sizeof(unsigned) * (4 + 2 * (size_t)nplanes), st);
    if (e != cudaSuccess) return e;
    MidSync sync{sync_words, sync_words + 4, sync_words + 4 + nplanes, sync_words + 4 + 2 * (size_t)nplanes};
    const int grid = per_sm * num_sms();
    const int lag = std::max(2, (grid + 3 * SH::ITEMS - 1) / (3 * SH::ITEMS) + 1);
    if (op.kind == OP_GR)
        k_mid<T, LOGN, OP_GR, THREADS><<<grid, SH::THREADS, SH::SMEM, st>>>(A, B, Cs, op, nplanes, lag, sync);
    else
        k_mid<T, LOGN, OP_NEWTON, THREADS><<<grid, SH::THREADS, SH::SMEM, st>>>(A, B, Cs, op, nplanes, lag, sync);
    return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t middle_shape(cplx<T>* A, cplx<T>* B, cplx<T>* Cs, int nplanes, const SpecOp& op, unsigned* sync_words,
                         int threads, cudaStream_t st) {
    switch (threads) {
        case 256: return middle_n<T, LOGN, 256>(A, B, Cs, nplanes, op, sync_words, st);
        case 512: return middle_n<T, LOGN, 512>(A, B, Cs, nplanes, op, sync_words, st);
        case 1024: return middle_n<T, LOGN, 1024>(A, B, Cs, nplanes, op, sync_words, st);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int LOGN>
cudaError_t plane_n(cplx<T>* A, cplx<T>* GX, cplx<T>* GY, int nplanes, const SpecOp& op, cudaStream_t st) {
    typedef PlaneShape<T, LOGN> SH;
    const void* fn = op.kind == OP_GR ? (const void*)k_plane<T, LOGN, OP_GR> : (const void*)k_plane<T, LOGN, OP_NEWTON>;
    cudaError_t e = set_smem(fn, SH::SMEM);
    if (e != cudaSuccess) return e;
    int per_sm = 1;
    e = resident_ctas(fn, SH::THREADS, SH::SMEM, &per_sm);
    if (e != cudaSuccess) return e;
    const int grid = (int)std::min<int64_t>((int64_t)per_sm * num_sms(), nplanes);
    if (op.kind == OP_GR)
        k_plane<T, LOGN, OP_GR><<<grid, SH::THREADS, SH::SMEM, st>>>(A, GX, GY, op, nplanes);
    else
        k_plane<T, LOGN, OP_NEWTON><<<grid, SH::THREADS, SH::SMEM, st>>>(A, GX, GY, op, nplanes);
    return cudaGetLastError();
}

template <typename T, int LOGN, bool GR, bool FD>
cudaError_t x_adj_k(const cplx<T>* V, cplx<T>* out, double kf, double coef, float* zero, int64_t nzero, cudaStream_t st,
                    const AdjGrOp& gr) {
    typedef Shape<T, LOGN> S;
    const size_t smem = sizeof(cplx<T>) * (S::N + 2 * (size_t)S::N * (S::CB + 1));
    cudaError_t e = set_smem((const void*)k_x_adj<T, LOGN, GR, FD>, smem);
    if (e != cudaSuccess) return e;
    k_x_adj<T, LOGN, GR, FD><<<dim3(S::N / S::CB, S::M + 1), S::CB * S::QN, smem, st>>>(
        V, out, kf, coef, (float4*)zero, zero ? nzero / 4 : 0, gr);
    return cudaGetLastError();
}

template <typename T, int LOGN>
cudaError_t x_adj_n(const cplx<T>* V, cplx<T>* out, double kf, double coef, float* zero, int64_t nzero,
                    cudaStream_t st, const AdjGrOp* gr, bool fd) {
    if (nzero % 4 != 0 || (zero && (uintptr_t)zero % 16 != 0)) return cudaErrorInvalidValue;
    if (gr && !gr->Z) return cudaErrorInvalidValue;
    const AdjGrOp g = gr ? *gr : AdjGrOp();
    if (gr) return fd ? x_adj_k<T, LOGN, true, true>(V, out, kf, coef, zero, nzero, st, g)
                      : x_adj_k<T, LOGN, true, false>(V, out, kf, coef, zero, nzero, st, g);
    return fd ? x_adj_k<T, LOGN, false, true>(V, out, kf, coef, zero, nzero, st, g)
              : x_adj_k<T, LOGN, false, false>(V, out, kf, coef, zero, nzero, st, g);
}

template <typename T, int LOGN>
cudaError_t x_cols_kind(cplx<T>* data, cplx<T>* out2, int nplanes, const SpecOp& op, cudaStream_t st) {
    switch (op.kind) {
        case OP_FWD_STORE: return x_cols_n<T, LOGN, OP_FWD_STORE>(data, out2, nplanes, op, st);
        case OP_INV: return x_cols_n<T, LOGN, OP_INV>(data, out2, nplanes, op, st);
        case OP_NEWTON: return x_cols_n<T, LOGN, OP_NEWTON>(data, out2, nplanes, op, st);
        case OP_GR: return x_cols_n<T, LOGN, OP_GR>(data, out2, nplanes, op, st);
        case OP_ZA: return x_cols_n<T, LOGN, OP_ZA>(data, out2, nplanes, op, st);
        case OP_BIN: return x_cols_n<T, LOGN, OP_BIN>(data, out2, nplanes, op, st);
        case OP_POTENTIAL: return x_cols_n<T, LOGN, OP_POTENTIAL>(data, out2, nplanes, op, st);
        default: return cudaErrorInvalidValue;
    }
}

#define PM_DISPATCH_LOGN(n, CALL)      \
    switch (ilog2(n)) {                \
        case 4: { constexpr int LG = 4; return CALL; } \
        case 5: { constexpr int LG = 5; return CALL; } \
        case 6: { constexpr int LG = 6; return CALL; } \
        case 7: { constexpr int LG = 7; return CALL; } \
        case 8: { constexpr int LG = 8; return CALL; } \
        case 9: { constexpr int LG = 9; return CALL; } \
        case 10: { constexpr int LG = 10; return CALL; } \
        default: return cudaErrorInvalidValue; \
    }

template <typename T>
cudaError_t z_r2c(const T* in, cplx<T>* out, int n, int batch, cudaStream_t st, double sub) {
    PM_DISPATCH_LOGN(n, (z_r2c_n<T, LG>(in, out, n * batch, st, sub)))
}

template <typename T>
cudaError_t z_c2r(const cplx<T>* const* in, T* const* out, int ncomp, int n, int batch, unsigned gradz_mask,
                  double kf, cudaStream_t st, const double* kf_arr, T* zero) {
    Ptr3<T> P;
    for (int j = 0; j < 3; ++j) {
        P.in[j] = in[j < ncomp ? j : 0];
        P.out[j] = out[j < ncomp ? j : 0];
    }
    P.zero = zero;
    PM_DISPATCH_LOGN(n, (z_c2r_n<T, LG>(P, ncomp, n * batch, gradz_mask, kf, st, kf_arr)))
}

template <typename T, bool INV>
cudaError_t y_rows(cplx<T>* data, int64_t nrows, int n, cudaStream_t st) {
    PM_DISPATCH_LOGN(n, (y_rows_n<T, LG, INV>(data, data, nrows, st)))
}

template <typename T>
cudaError_t y_rows_grad3(cplx<T>* A, cplx<T>* B, cplx<T>* Cc, int64_t nrows, int n, double kf, cudaStream_t st,
                         const double* kf_arr, int64_t rows_per_field) {
    PM_DISPATCH_LOGN(n, (y_grad3_n<T, LG>(A, B, A, B, Cc, nrows, kf, st, kf_arr, rows_per_field)))
}

// The fused middle passes (forward y, x with op, inverse y with the y gradient) on meshes of
// 256^3 and up; cudaErrorNotSupported for other sizes (the caller runs the separate passes).
// The fused middle passes (forward y, x with op, inverse y with the y gradient) on meshes of
// 256^3 and up with CTAs of `threads` (256, 512 or 1024); cudaErrorNotSupported for other sizes
// (the caller runs the separate passes).
template <typename T>
cudaError_t fft_middle(cplx<T>* A, cplx<T>* B, cplx<T>* Cs, int nplanes, int n, const SpecOp& op, unsigned* sync_words,
                       int threads, cudaStream_t st) {
    if (op.kind != OP_NEWTON && op.kind != OP_GR) return cudaErrorInvalidValue;
    switch (ilog2(n)) {
        case 8: return middle_shape<T, 8>(A, B, Cs, nplanes, op, sync_words, threads, st);
        case 9: return middle_shape<T, 9>(A, B, Cs, nplanes, op, sync_words, threads, st);
        case 10: return middle_shape<T, 10>(A, B, Cs, nplanes, op, sync_words, threads, st);
        default: return cudaErrorNotSupported;
    }
}

// The middle passes on whole kz planes in shared memory (meshes of 64^3 and 128^3):
// GX, GY and A receive -i k_j phi transformed back along x and y (A in place); the z pass
// then runs without its z gradient.  cudaErrorNotSupported for other sizes.
template <typename T>
cudaError_t fft_plane(cplx<T>* A, cplx<T>* GX, cplx<T>* GY, int nplanes, int n, const SpecOp& op, cudaStream_t st) {
    if (op.kind != OP_NEWTON && op.kind != OP_GR) return cudaErrorInvalidValue;
    switch (ilog2(n)) {
        case 6: return plane_n<T, 6>(A, GX, GY, nplanes, op, st);
        case 7: return plane_n<T, 7>(A, GX, GY, nplanes, op, st);
        default: return cudaErrorNotSupported;
    }
}

template <typename T>
cudaError_t x_adj(const cplx<T>* V, cplx<T>* out, int n, double kf, double coef, cudaStream_t st, float* zero,
                  int64_t nzero, const AdjGrOp* gr, bool fd) {
    PM_DISPATCH_LOGN(n, (x_adj_n<T, LG>(V, out, kf, coef, zero, nzero, st, gr, fd)))
}

template <typename T>
cudaError_t forward_zy(const T* in, cplx<T>* spec, int n, int batch, cudaStream_t st, double sub) {
    PM_DISPATCH_LOGN(n, (forward_zy_n<T, LG>(in, spec, batch, st, sub)))
}

template <typename T>
cudaError_t inverse_yz_grad(cplx<T>* A, cplx<T>* B, cplx<T>* scratch, T* const* out, int n, int batch, double kf,
                            cudaStream_t st, const double* kf_arr, T* zero) {
    PM_DISPATCH_LOGN(n, (inverse_yz_grad_n<T, LG>(A, B, scratch, out, batch, kf, kf_arr, st, zero)))
}

template <typename T>
cudaError_t x_cols(cplx<T>* data, cplx<T>* out2, int nplanes, int n, const SpecOp& op, cudaStream_t st) {
    PM_DISPATCH_LOGN(n, (x_cols_kind<T, LG>(data, out2, nplanes, op, st)))
}

#define PM_INST(T)                                                                                     \
    template cudaError_t z_r2c<T>(const T*, cplx<T>*, int, int, cudaStream_t, double);                 \
    template cudaError_t z_c2r<T>(const cplx<T>* const*, T* const*, int, int, int, unsigned, double,  \
                                  cudaStream_t, const double*, T*);                                    \
    template cudaError_t y_rows<T, false>(cplx<T>*, int64_t, int, cudaStream_t);                      \
    template cudaError_t y_rows<T, true>(cplx<T>*, int64_t, int, cudaStream_t);                       \
    template cudaError_t y_rows_grad3<T>(cplx<T>*, cplx<T>*, cplx<T>*, int64_t, int, double,           \
                                         cudaStream_t, const double*, int64_t);                        \
    template cudaError_t x_cols<T>(cplx<T>*, cplx<T>*, int, int, const SpecOp&, cudaStream_t);      \
    template cudaError_t forward_zy<T>(const T*, cplx<T>*, int, int, cudaStream_t, double);             \
    template cudaError_t x_adj<T>(const cplx<T>*, cplx<T>*, int, double, double, cudaStream_t, float*, \
                                  int64_t, const AdjGrOp*, bool);                                       \
    template cudaError_t inverse_yz_grad<T>(cplx<T>*, cplx<T>*, cplx<T>*, T* const*, int, int, double,   \
                                            cudaStream_t, const double*, T*);

}  // namespace pm
