// Bispectrum estimator kernels (Eq. bispectre, Sec. 4.2).
//
// sum_{n1+n2+n3=0, n_a in bins} delta_1 delta_2 delta_3 = m^-3 sum_x I_i(x) I_j(x) I_l(x)
// with I_b = IFFT_m[delta 1_b] (unnormalised) and the triangle count is the same sum
// over N_b = IFFT_m[1_b].  bk_masks builds the nbins masked data spectra on the m grid and
// bk_indicators the nbins indicator spectra (in FP64: their sums are integer counts, which
// FP32 sums of 1e6 - 1e7 configurations do not resolve); after their inverse transforms
// bk_units accumulates the triple-product sums of one set for every bin triplet.
#include "internal.h"
#include "particles.h"

namespace pm {

// Bin of every integer |n|^2 <= nmax: the largest b with e2[b] <= |n|^2 (binary search on the
// squared edges), the last edge closed, -1 outside [e2[0], e2[nbins]].  The host applies the
// same comparisons to the same doubles, so both sides agree mode by mode.
__global__ void k_bin_table(int16_t* __restrict__ tab, int64_t nmax, const double* __restrict__ e2, int nbins) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s <= nmax; s += (int64_t)gridDim.x * blockDim.x) {
        const double v = (double)s;
        int b = -1;
        if (e2[0] <= v) {
            int lo = 0, hi = nbins;  // e2[lo] <= v; find the largest such index
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (e2[mid] <= v) lo = mid;
                else hi = mid - 1;
            }
            b = lo;
        }
        if (v == e2[nbins]) b = nbins - 1;
        tab[s] = (b >= 0 && b < nbins) ? (int16_t)b : (int16_t)-1;
    }
}

cudaError_t bin_table(int16_t* tab, int64_t nmax, const double* e2, int nbins, cudaStream_t st) {
    int64_t blocks = (nmax + 256) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_bin_table<<<(unsigned)blocks, 256, 0, st>>>(tab, nmax, e2, nbins);
    return cudaGetLastError();
}

// Bin of mode e of the m-grid half spectrum [kz][kx][ky] for an n^3 field: the bin of |n|^2,
// -1 for the zero mode, modes beyond n/2 and modes with a Nyquist component of the n-grid.
__device__ __forceinline__ int bk_mode_bin(int64_t e, int m, int n, const int16_t* __restrict__ bin_of, int* nx_out,
                                           int* ny_out, int* nz_out) {
    const int hn = n >> 1;
    const int kz = (int)(e / ((int64_t)m * m));
    const int rem = (int)(e - (int64_t)kz * m * m);
    const int nx = signed_k(rem / m, m), ny = signed_k(rem % m, m), nz = kz;
    const int ax = nx < 0 ? -nx : nx, ay = ny < 0 ? -ny : ny;
    const int n2 = nx * nx + ny * ny + nz * nz;
    *nx_out = nx;
    *ny_out = ny;
    *nz_out = nz;
    return (n2 > 0 && n2 <= hn * hn && ax < hn && ay < hn && nz < hn) ? (int)bin_of[n2] : -1;
}

// The nbins masked data spectra delta 1_b on the m grid.
template <typename T>
__global__ void k_bk_masks(const cplx<T>* __restrict__ spec_n, int n, cplx<T>* __restrict__ out, int m, int nbins,
                           const int16_t* __restrict__ bin_of, const double* __restrict__ wtab, int deconv) {
    typedef cplx<T> C;
    const int64_t per = (int64_t)(m / 2 + 1) * m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
        int nx, ny, nz;
        const int bin = bk_mode_bin(e, m, n, bin_of, &nx, &ny, &nz);
        C v = cmake<C>(T(0), T(0));
        if (bin >= 0) {
            v = spec_n[((size_t)nz * n + (nx & (n - 1))) * n + (ny & (n - 1))];
            if (deconv) {
                const double W = wtab[nx < 0 ? -nx : nx] * wtab[ny < 0 ? -ny : ny] * wtab[nz];
                v = cscale(v, T(1.0 / W));
            }
        }
        const C zero = cmake<C>(T(0), T(0));
        for (int b = 0; b < nbins; ++b) out[(size_t)b * per + e] = (b == bin) ? v : zero;
    }
}

// The nbins indicator spectra 1_b on the m grid, in FP64 (their triangle sums are counts).
__global__ void k_bk_indicators(int n, double2* __restrict__ out, int m, int nbins, const int16_t* __restrict__ bin_of) {
    const int64_t per = (int64_t)(m / 2 + 1) * m * m;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < per; e += (int64_t)gridDim.x * blockDim.x) {
        int nx, ny, nz;
        const int bin = bk_mode_bin(e, m, n, bin_of, &nx, &ny, &nz);
        for (int b = 0; b < nbins; ++b) out[(size_t)b * per + e] = make_double2(b == bin ? 1.0 : 0.0, 0.0);
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

cudaError_t bk_indicators(int n, double2* out, int m, int nbins, const int16_t* bin_of, cudaStream_t st) {
    const int64_t per = (int64_t)(m / 2 + 1) * m * m;
    int64_t blocks = (per + 255) / 256;
    if (blocks > 152 * 16) blocks = 152 * 16;
    k_bk_indicators<<<(unsigned)blocks, 256, 0, st>>>(n, out, m, nbins, bin_of);
    return cudaGetLastError();
}

// Register-tiled triangle sums: a unit is (i, j-block of 4, l-block of 8) and covers the
// triangles (i, j, l) with i <= j <= l among j in [4 jb, 4 jb + 4) and l in [8 lb, 8 lb + 8).
// Per staged point a thread reads I_i, the four I_j and the eight I_l (aligned vectors), forms
// the four products I_i I_j and multiplies them into the eight I_l: 36 arithmetic operations for
// 1 + 4 / W + 8 / W shared-memory loads, so the loads no longer bound the sums.  Partial sums
// run over a chunk of points in T and across chunks in FP64.  Rows of a staged point hold the
// nbins fields at [0, nbp), nbp = nbins rounded up to 8 (zero padded), so the blocks never read
// past a row.
// unit = (i, jb, lb, index of triangle (i, i, i) in the i <= j <= l order).
template <typename T> struct Vec4;
template <> struct Vec4<float> { typedef float4 type; static constexpr int W = 4; };
template <> struct Vec4<double> { typedef double2 type; static constexpr int W = 2; };

template <typename T>
__global__ void __launch_bounds__(256, sizeof(T) == 4 ? 2 : 1) k_bk_units(const T* __restrict__ f, int64_t m3, int nbins, int nbp, int npts,
                                                  const int4* __restrict__ unit, int nunit, double* __restrict__ acc) {
    typedef typename Vec4<T>::type V;
    constexpr int W = Vec4<T>::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T* s = reinterpret_cast<T*>(smem_raw);
    const int stride = nbp;
    const int tid = threadIdx.x, nthr = blockDim.x;
    const int u = blockIdx.y * nthr + tid;
    const int4 my = (u < nunit) ? unit[u] : make_int4(0, 0, 0, -1);
    const int i = my.x, j0 = 4 * my.y, l0 = 8 * my.z;
    double sS[4][8];
#pragma unroll
    for (int d = 0; d < 4; ++d)
#pragma unroll
        for (int q = 0; q < 8; ++q) sS[d][q] = 0.0;
    for (int64_t c0 = (int64_t)blockIdx.x * npts; c0 < m3; c0 += (int64_t)gridDim.x * npts) {
        __syncthreads();
        for (int e = tid; e < npts * stride; e += nthr) {
            const int b = e / npts, pnt = e - b * npts;
            s[pnt * stride + b] = (b < nbins && c0 + pnt < m3) ? f[(size_t)b * m3 + c0 + pnt] : T(0);
        }
        __syncthreads();
        if (my.w < 0) continue;
        T ps[4][8];
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int q = 0; q < 8; ++q) ps[d][q] = T(0);
#pragma unroll 2
        for (int pnt = 0; pnt < npts; ++pnt) {
            const T* row = s + pnt * stride;
            const T fi = row[i];
            T a[4], dl[8];
#pragma unroll
            for (int h = 0; h < 4 / W; ++h) {
                const V v = reinterpret_cast<const V*>(row + j0)[h];
                const T* vv = reinterpret_cast<const T*>(&v);
#pragma unroll
                for (int w = 0; w < W; ++w) a[h * W + w] = fi * vv[w];
            }
#pragma unroll
            for (int h = 0; h < 8 / W; ++h) {
                const V v = reinterpret_cast<const V*>(row + l0)[h];
                const T* vv = reinterpret_cast<const T*>(&v);
#pragma unroll
                for (int w = 0; w < W; ++w) dl[h * W + w] = vv[w];
            }
#pragma unroll
            for (int d = 0; d < 4; ++d)
#pragma unroll
                for (int q = 0; q < 8; ++q) ps[d][q] += a[d] * dl[q];
        }
#pragma unroll
        for (int d = 0; d < 4; ++d)
#pragma unroll
            for (int q = 0; q < 8; ++q) sS[d][q] += (double)ps[d][q];
    }
    if (my.w < 0) return;
#pragma unroll
    for (int d = 0; d < 4; ++d) {
        const int j = j0 + d;
        if (j < i || j >= nbins) continue;
        // triangles (i, j', l) for i <= j' < j come first, nbins - j' of them for each j'
        const int tij = my.w + (j - i) * nbins - ((j - i) * (i + j - 1)) / 2;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int l = l0 + q;
            if (l < j || l >= nbins) continue;
            atomicAdd(&acc[tij + (l - j)], sS[d][q]);
        }
    }
}

template <typename T>
cudaError_t bk_units(const T* fields, int m, int nbins, const int4* unit, int nunit, double* acc, cudaStream_t st) {
    // one thread per unit, at most 256 a CTA, whole warps
    const int nthr = nunit >= 256 ? 256 : ((nunit + 31) & ~31);
    const int nbp = (nbins + 7) & ~7;
    const int64_t m3 = (int64_t)m * m * m;
    // points per chunk: up to 256, the staged rows within 48 KB of shared memory
    int npts = (int)((48 * 1024) / (sizeof(T) * nbp));
    npts = npts > 256 ? 256 : (npts < 32 ? 32 : npts & ~31);
    const int gy = (nunit + nthr - 1) / nthr;
    int64_t gx = (m3 + npts - 1) / npts;
    const int64_t cap = (152 * 16 + gy - 1) / gy;  // about sixteen CTAs per SM in all
    if (gx > cap) gx = cap;
    const size_t smem = sizeof(T) * (size_t)npts * nbp;
    if (smem > 48 * 1024) {
        cudaError_t e = set_smem_once((const void*)k_bk_units<T>, smem);
        if (e != cudaSuccess) return e;
    }
    k_bk_units<T><<<dim3((unsigned)gx, (unsigned)gy), nthr, smem, st>>>(fields, m3, nbins, nbp, npts, unit, nunit, acc);
    return cudaGetLastError();
}

template cudaError_t bk_masks<float>(const float2*, int, float2*, int, int, const int16_t*, const double*, int,
                                     cudaStream_t);
template cudaError_t bk_masks<double>(const double2*, int, double2*, int, int, const int16_t*, const double*, int,
                                      cudaStream_t);
template cudaError_t bk_units<float>(const float*, int, int, const int4*, int, double*, cudaStream_t);
template cudaError_t bk_units<double>(const double*, int, int, const int4*, int, double*, cudaStream_t);

}  // namespace pm
