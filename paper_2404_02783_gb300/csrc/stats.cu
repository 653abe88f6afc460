// Bispectrum estimator kernels (Eq. bispectre, Sec. 4.2).
//
// sum_{n1+n2+n3=0, n_a in bins} delta_1 delta_2 delta_3 = m^-3 sum_x I_i(x) I_j(x) I_l(x)
// with I_b = IFFT_m[delta 1_b] (unnormalised) and the triangle count is the same sum
// over N_b = IFFT_m[1_b].  bk_masks builds the 2 nbins masked half spectra on the m
// grid (first the nbins data fields, then the nbins indicator fields); after their
// inverse transforms bk_triangles accumulates both sums for every bin triplet.
#include "internal.h"
#include "particles.h"

namespace pm {

template <typename T>
__global__ void k_bk_masks(const cplx<T>* __restrict__ spec_n, int n, cplx<T>* __restrict__ out, int m, int nbins,
                           const int16_t* __restrict__ bin_of, const double* __restrict__ wtab, int deconv) {
    typedef cplx<T> C;
    const int64_t per = (int64_t)(m / 2 + 1) * m * m;
    const int hn = n >> 1;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(e / ((int64_t)m * m));
        const int rem = (int)(e - (int64_t)kz * m * m);
        const int nx = signed_k(rem / m, m), ny = signed_k(rem % m, m), nz = kz;
        const int ax = nx < 0 ? -nx : nx, ay = ny < 0 ? -ny : ny;
        const int n2 = nx * nx + ny * ny + nz * nz;
        int bin = -1;
        C v = cmake<C>(T(0), T(0));
        if (n2 > 0 && n2 <= hn * hn && ax < hn && ay < hn && nz < hn) {
            bin = bin_of[n2];
            if (bin >= 0) {
                v = spec_n[((size_t)nz * n + (nx & (n - 1))) * n + (ny & (n - 1))];
                if (deconv) {
                    const double W = wtab[ax] * wtab[ay] * wtab[nz];
                    v = cscale(v, T(1.0 / W));
                }
            }
        }
        const C zero = cmake<C>(T(0), T(0)), one = cmake<C>(T(1), T(0));
        for (int b = 0; b < nbins; ++b) {
            out[(size_t)b * per + e] = (b == bin) ? v : zero;
            out[(size_t)(nbins + b) * per + e] = (b == bin) ? one : zero;
        }
    }
}

template <typename T>
cudaError_t bk_masks(const cplx<T>* spec_n, int n, cplx<T>* out, int m, int nbins, const int16_t* bin_of,
                     const double* wtab, int deconv, cudaStream_t st) {
    const int64_t per = (int64_t)(m / 2 + 1) * m * m;
    int64_t blocks = (per + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_bk_masks<T><<<(unsigned)blocks, 256, 0, st>>>(spec_n, n, out, m, nbins, bin_of, wtab, deconv);
    return cudaGetLastError();
}

constexpr int kTriPoints = 64;   // points staged per chunk
constexpr int kTriPerThread = 8; // triangles per thread per block row

template <typename T>
__global__ void __launch_bounds__(512) k_bk_triangles(const T* __restrict__ f, int64_t m3, int nbins,
                                                      const int4* __restrict__ tri, int ntri,
                                                      double* __restrict__ accS, double* __restrict__ accC) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    const int nb2 = 2 * nbins;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int t0 = blockIdx.y * kTriPerThread * nthr;
    int4 my[kTriPerThread];
    double sS[kTriPerThread], sC[kTriPerThread];
#pragma unroll
    for (int k = 0; k < kTriPerThread; ++k) {
        const int t = t0 + tid + k * nthr;
        my[k] = (t < ntri) ? tri[t] : make_int4(0, 0, 0, -1);
        sS[k] = 0.0;
        sC[k] = 0.0;
    }
    for (int64_t c0 = (int64_t)blockIdx.x * kTriPoints; c0 < m3; c0 += (int64_t)gridDim.x * kTriPoints) {
        __syncthreads();
        for (int e = tid; e < kTriPoints * nb2; e += nthr) {
            const int b = e / kTriPoints, pnt = e - b * kTriPoints;
            s[pnt * nb2 + b] = (c0 + pnt < m3) ? f[(size_t)b * m3 + c0 + pnt] : T(0);
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < kTriPerThread; ++k) {
            if (my[k].w < 0) continue;
            const int i = my[k].x, j = my[k].y, l = my[k].z;
            T ps = T(0), pc = T(0);
#pragma unroll 8
            for (int pnt = 0; pnt < kTriPoints; ++pnt) {
                const T* row = s + pnt * nb2;
                ps += row[i] * row[j] * row[l];
                pc += row[nbins + i] * row[nbins + j] * row[nbins + l];
            }
            sS[k] += (double)ps;
            sC[k] += (double)pc;
        }
    }
#pragma unroll
    for (int k = 0; k < kTriPerThread; ++k) {
        if (my[k].w < 0) continue;
        const int t = t0 + tid + k * nthr;
        atomicAdd(&accS[t], sS[k]);
        atomicAdd(&accC[t], sC[k]);
    }
}

template <typename T>
cudaError_t bk_triangles(const T* fields, int m, int nbins, const int4* tri, int ntri, double* accS, double* accC,
                         cudaStream_t st) {
    const int nthr = 256;
    const int64_t m3 = (int64_t)m * m * m;
    int64_t gx = (m3 + kTriPoints - 1) / kTriPoints;
    if (gx > 152 * 4) gx = 152 * 4;
    const int gy = (ntri + kTriPerThread * nthr - 1) / (kTriPerThread * nthr);
    const size_t smem = sizeof(T) * kTriPoints * 2 * nbins;
    if (smem > 48 * 1024) {
        cudaError_t e = set_smem_once((const void*)k_bk_triangles<T>, smem);
        if (e != cudaSuccess) return e;
    }
    dim3 grid((unsigned)gx, (unsigned)gy);
    k_bk_triangles<T><<<grid, nthr, smem, st>>>(fields, m3, nbins, tri, ntri, accS, accC);
    return cudaGetLastError();
}

template cudaError_t bk_masks<float>(const float2*, int, float2*, int, int, const int16_t*, const double*, int,
                                     cudaStream_t);
template cudaError_t bk_masks<double>(const double2*, int, double2*, int, int, const int16_t*, const double*, int,
                                      cudaStream_t);
template cudaError_t bk_triangles<float>(const float*, int, int, const int4*, int, double*, double*, cudaStream_t);
template cudaError_t bk_triangles<double>(const double*, int, int, const int4*, int, double*, double*, cudaStream_t);

}  // namespace pm
