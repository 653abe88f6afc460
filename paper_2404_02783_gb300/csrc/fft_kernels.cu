// 3D real FFT passes and the fused spectral operators of the PM step.
//
// Data flow of a 3D r2c transform of a real mesh R[x][y][z] (side n):
//   z_r2c : rows along z -> half spectrum T[kz][x][y]  (kz = 0..n/2; transposing store)
//   y_rows: rows along y (contiguous)                  -> T[kz][x][ky]
//   x_cols: columns along x (stride n)                 -> S[kz][kx][ky]
// and the inverse runs x_cols -> y_rows -> z_c2r.  Every pass reads and writes
// each element once (coalesced tiles through shared memory); the Green's
// function, the Poisson-gauge constraint, the Zel'dovich filter, the x part of
// the spectral gradient and the power-spectrum binning are fused into the
// x-column pass, the y part of the gradient into the inverse y pass and the z
// part into the c2r pass, so no pass exists only to multiply a spectrum.
#include <math.h>

#include <mutex>

#include "fft.cuh"
#include "internal.h"

namespace pm {

__device__ float2 g_tw32[1024];
__device__ double2 g_tw64[1024];

template <typename T> __device__ __forceinline__ cplx<T> tw_global(int k);
template <> __device__ __forceinline__ float2 tw_global<float>(int k) { return g_tw32[k]; }
template <> __device__ __forceinline__ double2 tw_global<double>(int k) { return g_tw64[k]; }

static std::mutex g_tab_mutex;
static bool g_tab_ready[128];

cudaError_t ensure_device_tables() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    if (dev < 128 && g_tab_ready[dev]) return cudaSuccess;
    float2 h32[1024];
    double2 h64[1024];
    for (int k = 0; k < 1024; ++k) {
        // exp(-2 pi i k / 1024) from the octant-reduced angle for exact symmetry
        const double ang = -2.0 * M_PI * (double)k / 1024.0;
        double c = cos(ang), s = sin(ang);
        if (k % 256 == 0) {
            const int q = k / 256;
            c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
            s = (q == 1) ? -1.0 : (q == 3 ? 1.0 : 0.0);
        }
        h64[k] = make_double2(c, s);
        h32[k] = make_float2((float)c, (float)s);
    }
    e = cudaMemcpyToSymbol(g_tw32, h32, sizeof(h32));
    if (e != cudaSuccess) return e;
    e = cudaMemcpyToSymbol(g_tw64, h64, sizeof(h64));
    if (e != cudaSuccess) return e;
    if (dev < 128) g_tab_ready[dev] = true;
    return cudaSuccess;
}

template <typename T>
__device__ __forceinline__ void load_twiddles(cplx<T>* tw, int n) {
    const int stride = 1024 / n;
    for (int k = threadIdx.x; k < n; k += blockDim.x) tw[k] = tw_global<T>(k * stride);
}

// Row stride (in complex elements) of a padded row tile holding `len` elements;
// odd so that lanes walking across rows hit distinct banks.
__host__ __device__ __forceinline__ int row_stride(int len) { return (spad(len) + 1) | 1; }

static cudaError_t set_smem(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// =============================================================== z: r2c
template <typename T>
__global__ void __launch_bounds__(512) k_z_r2c(const T* __restrict__ in, cplx<T>* __restrict__ out,
                                                int n, int YB) {
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s = tw + n;
    const int M = n >> 1;
    const int RS = row_stride(M + 1);
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int y0 = blockIdx.x * YB;
    const int x = blockIdx.y % n;
    const size_t f = blockIdx.y / n;
    load_twiddles<T>(tw, n);
    const C* inrow = reinterpret_cast<const C*>(in + ((f * n + x) * (size_t)n + y0) * n);
    for (int e = tid; e < YB * M; e += nthr) {
        const int b = e / M, i = e - b * M;
        s[b * RS + spad(i)] = inrow[(size_t)b * M + i];
    }
    __syncthreads();
    const int tpr = M >> 3;
    const int b = tid / tpr, t = tid - b * tpr;
    fft_tile<false>(s, M, t, b, b < YB, tw, 2, RowAddr{RS});
    C* outp = out + f * (size_t)(M + 1) * n * n;
    for (int e = tid; e < (M + 1) * YB; e += nthr) {
        const int k = e / YB, bb = e - k * YB;
        const C z1 = s[bb * RS + spad(k == M ? 0 : k)];
        const C z2 = cconj(s[bb * RS + spad(k == 0 ? 0 : M - k)]);
        const C E = cscale(cadd(z1, z2), T(0.5));
        const C O = cscale(cmul_mi<false>(csub(z1, z2)), T(0.5));
        outp[((size_t)k * n + x) * n + y0 + bb] = cadd(E, cmul(tw[k], O));
    }
}

template <typename T>
cudaError_t z_r2c(const T* in, cplx<T>* out, int n, int batch, cudaStream_t st) {
    typedef cplx<T> C;
    const int M = n / 2;
    const int tpr = M / 8;
    int YB = 512 / tpr;
    if (YB > n) YB = n;
    if (YB < 1) YB = 1;
    const size_t smem = sizeof(C) * (n + (size_t)YB * row_stride(M + 1));
    cudaError_t e = set_smem((const void*)k_z_r2c<T>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(n / YB, n * batch);
    k_z_r2c<T><<<grid, YB * tpr, smem, st>>>(in, out, n, YB);
    return cudaGetLastError();
}

// =============================================================== z: c2r
template <typename T> struct Ptr3 {
    const cplx<T>* in[3];
    T* out[3];
};

template <typename T>
__global__ void __launch_bounds__(512) k_z_c2r(Ptr3<T> P, int n, int YB, unsigned gradz_mask, T kf) {
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s = tw + n;
    const int M = n >> 1;
    const int RS = row_stride(M + 1);
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int comp = blockIdx.z;
    const bool grad = (gradz_mask >> comp) & 1u;
    const int y0 = blockIdx.x * YB;
    const int x = blockIdx.y % n;
    const size_t f = blockIdx.y / n;
    load_twiddles<T>(tw, n);
    const C* inp = P.in[comp] + f * (size_t)(M + 1) * n * n;
    for (int e = tid; e < (M + 1) * YB; e += nthr) {
        const int k = e / YB, bb = e - k * YB;
        C X = inp[((size_t)k * n + x) * n + y0 + bb];
        if (grad) {  // (-i kz) X, Nyquist kz -> 0
            const T kz = (k == M) ? T(0) : kf * T(k);
            X = cmake<C>(X.y * kz, -X.x * kz);
        }
        s[bb * RS + spad(k)] = X;
    }
    __syncthreads();
    // Y_k = (X_k + X*_{M-k}) + i (X_k - X*_{M-k}) exp(+2 pi i k / n), pairs (k, M-k) per thread.
    const int half = M >> 1;
    for (int e = tid; e < (half + 1) * YB; e += nthr) {
        const int k = e / YB, bb = e - k * YB;
        C* row = s + bb * RS;
        C a = row[spad(k)];
        C c = row[spad(M - k)];
        if (k == 0) { a.y = T(0); c.y = T(0); }
        {
            const C bconj = cconj(c);
            const C d = cmul(csub(a, bconj), cconj(tw[k]));
            const C y = cadd(cadd(a, bconj), cmake<C>(-d.y, d.x));
            if (k > 0 && k < M - k) {
                const C aconj = cconj(a);
                const C d2 = cmul(csub(c, aconj), cconj(tw[M - k]));
                row[spad(M - k)] = cadd(cadd(c, aconj), cmake<C>(-d2.y, d2.x));
            }
            row[spad(k)] = y;
        }
    }
    __syncthreads();
    const int tpr = M >> 3;
    const int b = tid / tpr, t = tid - b * tpr;
    fft_tile<true>(s, M, t, b, b < YB, tw, 2, RowAddr{RS});
    C* outrow = reinterpret_cast<C*>(P.out[comp] + ((f * n + x) * (size_t)n + y0) * n);
    for (int e = tid; e < YB * M; e += nthr) {
        const int bb = e / M, i = e - bb * M;
        outrow[(size_t)bb * M + i] = s[bb * RS + spad(i)];
    }
}

template <typename T>
cudaError_t z_c2r(const cplx<T>* const* in, T* const* out, int ncomp, int n, int batch,
                  unsigned gradz_mask, double kf, cudaStream_t st) {
    typedef cplx<T> C;
    const int M = n / 2;
    const int tpr = M / 8;
    int YB = 512 / tpr;
    if (YB > n) YB = n;
    if (YB < 1) YB = 1;
    const size_t smem = sizeof(C) * (n + (size_t)YB * row_stride(M + 1));
    cudaError_t e = set_smem((const void*)k_z_c2r<T>, smem);
    if (e != cudaSuccess) return e;
    Ptr3<T> P;
    for (int j = 0; j < 3; ++j) {
        P.in[j] = in[j < ncomp ? j : 0];
        P.out[j] = out[j < ncomp ? j : 0];
    }
    dim3 grid(n / YB, n * batch, ncomp);
    k_z_c2r<T><<<grid, YB * tpr, smem, st>>>(P, n, YB, gradz_mask, (T)kf);
    return cudaGetLastError();
}

// =============================================================== y: contiguous rows
template <typename T, bool INV>
__global__ void __launch_bounds__(512) k_y_rows(cplx<T>* __restrict__ data, int64_t nrows, int n, int RB) {
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s = tw + n;
    const int RS = row_stride(n);
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    load_twiddles<T>(tw, n);
    for (int e = tid; e < RB * n; e += nthr) {
        const int b = e / n, i = e - b * n;
        if (r0 + b < nrows) s[b * RS + spad(i)] = data[(r0 + b) * n + i];
    }
    __syncthreads();
    const int tpr = n >> 3;
    const int b = tid / tpr, t = tid - b * tpr;
    fft_tile<INV>(s, n, t, b, r0 + b < nrows, tw, 1, RowAddr{RS});
    for (int e = tid; e < RB * n; e += nthr) {
        const int bb = e / n, i = e - bb * n;
        if (r0 + bb < nrows) data[(r0 + bb) * n + i] = s[bb * RS + spad(i)];
    }
}

template <typename T, bool INV>
cudaError_t y_rows(cplx<T>* data, int64_t nrows, int n, cudaStream_t st) {
    typedef cplx<T> C;
    const int tpr = n / 8;
    int RB = 512 / tpr;
    if (RB < 1) RB = 1;
    const size_t smem = sizeof(C) * (n + (size_t)RB * row_stride(n));
    cudaError_t e = set_smem((const void*)k_y_rows<T, INV>, smem);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (nrows + RB - 1) / RB;
    k_y_rows<T, INV><<<(unsigned)nblk, RB * tpr, smem, st>>>(data, nrows, n, RB);
    return cudaGetLastError();
}

template <typename T>
__global__ void __launch_bounds__(512) k_y_rows_grad3(cplx<T>* __restrict__ A, cplx<T>* __restrict__ B,
                                                       cplx<T>* __restrict__ Cout, int64_t nrows, int n,
                                                       int RB, T kf) {
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    C* s = tw + n;
    const int RS = row_stride(n);
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int64_t r0 = (int64_t)blockIdx.x * RB;
    load_twiddles<T>(tw, n);
    for (int e = tid; e < RB * n; e += nthr) {
        const int b = e / n, i = e - b * n;
        if (r0 + b < nrows) {
            const C a = A[(r0 + b) * n + i];
            s[b * RS + spad(i)] = a;
            s[(b + RB) * RS + spad(i)] = B[(r0 + b) * n + i];
            const int ny = signed_k(i, n);
            const T ky = (2 * ny == -n) ? T(0) : kf * T(ny);
            s[(b + 2 * RB) * RS + spad(i)] = cmake<C>(a.y * ky, -a.x * ky);  // -i ky a
        }
    }
    __syncthreads();
    const int tpr = n >> 3;
    const int b = tid / tpr, t = tid - b * tpr;
    fft_tile<true>(s, n, t, b, r0 + (b % RB) < nrows, tw, 1, RowAddr{RS});
    for (int e = tid; e < RB * n; e += nthr) {
        const int bb = e / n, i = e - bb * n;
        if (r0 + bb < nrows) {
            A[(r0 + bb) * n + i] = s[bb * RS + spad(i)];
            B[(r0 + bb) * n + i] = s[(bb + RB) * RS + spad(i)];
            Cout[(r0 + bb) * n + i] = s[(bb + 2 * RB) * RS + spad(i)];
        }
    }
}

template <typename T>
cudaError_t y_rows_grad3(cplx<T>* A, cplx<T>* B, cplx<T>* Cout, int64_t nrows, int n, double kf,
                         cudaStream_t st) {
    typedef cplx<T> C;
    const int tpr = n / 8;
    int RB = 512 / (3 * tpr);
    const size_t row_bytes = sizeof(C) * 3 * (size_t)row_stride(n);
    while (RB > 1 && sizeof(C) * n + RB * row_bytes > 112 * 1024) RB /= 2;
    if (RB < 1) RB = 1;
    const size_t smem = sizeof(C) * n + RB * row_bytes;
    cudaError_t e = set_smem((const void*)k_y_rows_grad3<T>, smem);
    if (e != cudaSuccess) return e;
    const int64_t nblk = (nrows + RB - 1) / RB;
    k_y_rows_grad3<T><<<(unsigned)nblk, 3 * RB * tpr, smem, st>>>(A, B, Cout, nrows, n, RB, (T)kf);
    return cudaGetLastError();
}

// =============================================================== x: strided columns + spectral operators
template <typename T, int KIND>
__global__ void __launch_bounds__(512) k_x_cols(cplx<T>* __restrict__ data, cplx<T>* __restrict__ out2,
                                                 int n, int CB, SpecOp op) {
    typedef cplx<T> C;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    C* tw = reinterpret_cast<C*>(smem_raw);
    const int CS = CB + 1;
    C* tile0 = tw + n;
    C* tile1 = tile0 + (size_t)n * CS;
    double* acc = reinterpret_cast<double*>(tile1 + (size_t)n * CS);
    const int nthr = blockDim.x, tid = threadIdx.x;
    const int M = n >> 1;
    const int plane = blockIdx.y;
    const int kz = plane % (M + 1);
    const int c0 = blockIdx.x * CB;
    const size_t pbase = (size_t)plane * n * n;
    C* base = data + pbase;
    const bool cross = (KIND == OP_BIN) && op.in2 != nullptr;
    load_twiddles<T>(tw, n);
    for (int e = tid; e < n * CB; e += nthr) {
        const int i = e / CB, bb = e - i * CB;
        tile0[i * CS + bb] = base[(size_t)i * n + c0 + bb];
        if (cross) tile1[i * CS + bb] = reinterpret_cast<const C*>(op.in2)[pbase + (size_t)i * n + c0 + bb];
    }
    if (KIND == OP_BIN)
        for (int e = tid; e < 3 * op.nbins; e += nthr) acc[e] = 0.0;
    __syncthreads();
    const int b = tid % CB, t = tid / CB;
    if (op.fwd) {
        fft_tile<false>(tile0, n, t, b, true, tw, 1, ColAddr{CS});
        if (cross) fft_tile<false>(tile1, n, t, b, true, tw, 1, ColAddr{CS});
    }
    if (KIND == OP_FWD_STORE) {
        for (int e = tid; e < n * CB; e += nthr) {
            const int i = e / CB, bb = e - i * CB;
            base[(size_t)i * n + c0 + bb] = tile0[i * CS + bb];
        }
        return;
    }
    if (KIND == OP_INV) {
        fft_tile<true>(tile0, n, t, b, true, tw, 1, ColAddr{CS});
        for (int e = tid; e < n * CB; e += nthr) {
            const int i = e / CB, bb = e - i * CB;
            base[(size_t)i * n + c0 + bb] = tile0[i * CS + bb];
        }
        return;
    }
    // ---- per-mode operator on column b: modes (kx = i, ky = c0 + b, kz)
    const int ny = signed_k(c0 + b, n);
    const int nz = kz;
    const int q8 = n >> 3;
#pragma unroll 1
    for (int q = 0; q < 8; ++q) {
        const int i = t + q * q8;
        const int nx = signed_k(i, n);
        const int n2 = nx * nx + ny * ny + nz * nz;
        const C v = tile0[i * CS + b];
        if (KIND == OP_BIN) {
            if (n2 == 0 || n2 > M * M) continue;
            const int bin = op.bin_of[n2];
            if (bin < 0) continue;
            const double w = (nz == 0 || nz == M) ? 1.0 : 2.0;
            double val;
            if (cross) {
                const C u = tile1[i * CS + b];
                val = (double)v.x * (double)u.x + (double)v.y * (double)u.y;
            } else {
                val = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
            }
            if (op.deconv) {
                const double W = op.wtab[nx < 0 ? -nx : nx] * op.wtab[ny < 0 ? -ny : ny] * op.wtab[nz];
                val /= W * W;
            }
            atomicAdd(&acc[bin], w);
            atomicAdd(&acc[op.nbins + bin], w * val);
            atomicAdd(&acc[2 * op.nbins + bin], w * op.kf * sqrt((double)n2));
            continue;
        }
        C phi;
        if (KIND == OP_NEWTON || KIND == OP_POTENTIAL) {
            phi = (n2 == 0) ? cmake<C>(T(0), T(0)) : cscale(v, T(op.coef / (double)n2));
        } else if (KIND == OP_ZA) {
            const bool nyq = (2 * nx == -n) || (2 * ny == -n) || (nz == M);
            phi = (n2 == 0 || nyq) ? cmake<C>(T(0), T(0)) : cscale(v, T(op.coef * op.amp[n2] / (double)n2));
        } else {  // OP_GR
            if (n2 == 0) {
                phi = cmake<C>(T(0), T(0));
                if (op.n_lo > 0) {
                    const int L = op.n_lo, W2 = 2 * L + 1;
                    op.island[((size_t)nz * W2 + L) * W2 + L] = make_double2(0.0, 0.0);
                }
            } else if (n2 <= op.n_lo * op.n_lo) {
                const int L = op.n_lo, W2 = 2 * L + 1;
                const size_t id = ((size_t)nz * W2 + (nx + L)) * W2 + (ny + L);
                const double k2 = op.kf * op.kf * (double)n2;
                const double H = op.calH;
                double num_s = -1.5 * H * H * op.omm_a;
                double den = k2 + 3.0 * H * H + 4.5 * H * H * op.omm_a;
                double2 P = make_double2(num_s * (double)v.x, num_s * (double)v.y);
                if (!op.first) {
                    const double2 old = op.island[id];
                    const double c = 3.0 * H * op.inv_dtau;
                    P.x += c * old.x;
                    P.y += c * old.y;
                    den += c;
                }
                P.x /= den;
                P.y /= den;
                op.island[id] = P;
                phi = cmake<C>(T(P.x * op.ac2_over_n3), T(P.y * op.ac2_over_n3));
            } else {
                C* old = reinterpret_cast<C*>(op.phi_old) + pbase + (size_t)i * n + c0 + b;
                const T k2 = T(op.kf * op.kf) * T(n2);
                const T H = T(op.calH), om = T(op.omm_a);
                const T num_s = T(-1.5) * H * H * om;
                T den = k2 + T(3) * H * H + T(4.5) * H * H * om;
                C P = cscale(v, num_s);
                if (!op.first) {
                    const T c = T(3) * H * T(op.inv_dtau);
                    const C o = *old;
                    P.x += c * o.x;
                    P.y += c * o.y;
                    den += c;
                }
                const T inv = T(1) / den;
                P = cscale(P, inv);
                *old = P;
                phi = cscale(P, T(op.ac2_over_n3));
            }
        }
        tile0[i * CS + b] = phi;
        if (KIND != OP_POTENTIAL) {
            const T kx = (2 * nx == -n) ? T(0) : T(op.kf) * T(nx);
            tile1[i * CS + b] = cmake<C>(phi.y * kx, -phi.x * kx);  // -i kx phi
        }
    }
    __syncthreads();
    if (KIND == OP_BIN) {
        for (int e = tid; e < 3 * op.nbins; e += nthr)
            if (acc[e] != 0.0) atomicAdd(&op.acc[e], acc[e]);
        return;
    }
    fft_tile<true>(tile0, n, t, b, true, tw, 1, ColAddr{CS});
    if (KIND != OP_POTENTIAL) fft_tile<true>(tile1, n, t, b, true, tw, 1, ColAddr{CS});
    for (int e = tid; e < n * CB; e += nthr) {
        const int i = e / CB, bb = e - i * CB;
        base[(size_t)i * n + c0 + bb] = tile0[i * CS + bb];
        if (KIND != OP_POTENTIAL) out2[pbase + (size_t)i * n + c0 + bb] = tile1[i * CS + bb];
    }
}

template <typename T, int KIND>
static cudaError_t launch_x(cplx<T>* data, cplx<T>* out2, int nplanes, int n, const SpecOp& op,
                            cudaStream_t st) {
    typedef cplx<T> C;
    const int tpc = n / 8;  // threads per column
    int CB = 512 / tpc;
    if (CB > n) CB = n;
    if (CB < 1) CB = 1;
    // the kernel places its bin accumulators after the second tile, so OP_BIN keeps both
    const bool two = !(KIND == OP_FWD_STORE || KIND == OP_INV || KIND == OP_POTENTIAL);
    auto smem_of = [&](int cb) {
        return sizeof(C) * (n + (size_t)(two ? 2 : 1) * n * (cb + 1)) + sizeof(double) * 3 * op.nbins + 16;
    };
    while (CB > 1 && smem_of(CB) > 150 * 1024) CB /= 2;
    const size_t smem = smem_of(CB);
    cudaError_t e = set_smem((const void*)k_x_cols<T, KIND>, smem);
    if (e != cudaSuccess) return e;
    dim3 grid(n / CB, nplanes);
    k_x_cols<T, KIND><<<grid, CB * tpc, smem, st>>>(data, out2, n, CB, op);
    return cudaGetLastError();
}

template <typename T>
cudaError_t x_cols(cplx<T>* data, cplx<T>* out2, int nplanes, int n, const SpecOp& op, cudaStream_t st) {
    switch (op.kind) {
        case OP_FWD_STORE: return launch_x<T, OP_FWD_STORE>(data, out2, nplanes, n, op, st);
        case OP_INV: return launch_x<T, OP_INV>(data, out2, nplanes, n, op, st);
        case OP_NEWTON: return launch_x<T, OP_NEWTON>(data, out2, nplanes, n, op, st);
        case OP_GR: return launch_x<T, OP_GR>(data, out2, nplanes, n, op, st);
        case OP_ZA: return launch_x<T, OP_ZA>(data, out2, nplanes, n, op, st);
        case OP_BIN: return launch_x<T, OP_BIN>(data, out2, nplanes, n, op, st);
        case OP_POTENTIAL: return launch_x<T, OP_POTENTIAL>(data, out2, nplanes, n, op, st);
        default: return cudaErrorInvalidValue;
    }
}

// =============================================================== instantiations
#define PM_INST(T)                                                                                     \
    template cudaError_t z_r2c<T>(const T*, cplx<T>*, int, int, cudaStream_t);                         \
    template cudaError_t z_c2r<T>(const cplx<T>* const*, T* const*, int, int, int, unsigned, double,  \
                                  cudaStream_t);                                                       \
    template cudaError_t y_rows<T, false>(cplx<T>*, int64_t, int, cudaStream_t);                      \
    template cudaError_t y_rows<T, true>(cplx<T>*, int64_t, int, cudaStream_t);                       \
    template cudaError_t y_rows_grad3<T>(cplx<T>*, cplx<T>*, cplx<T>*, int64_t, int, double,           \
                                         cudaStream_t);                                                \
    template cudaError_t x_cols<T>(cplx<T>*, cplx<T>*, int, int, const SpecOp&, cudaStream_t);
PM_INST(float)
PM_INST(double)

}  // namespace pm
