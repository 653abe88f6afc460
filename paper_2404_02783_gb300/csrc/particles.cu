// Particle-side kernels of the PM step: CIC deposit (counting density, Sec. 4), CIC
// interpolation and the unfused kick + drift (KDK in a; the fused update with the next
// deposit is in update.cu), Zel'dovich placement, the per-wavevector Philox phases, the GR
// displacement combination (Eqs. xiGR and combined) and the cell keys / stable cell order
// of the particles.
//
// Position encodings (units of the box side):
//   FP32 path: uint32 ticks, 2^32 per side; the periodic wrap is integer overflow.
//   FP64 path: double fraction in [0, 1).
// Mesh nodes sit at cell centres, so mesh coordinate s = x n - 1/2; on ticks that
// is (u - 2^(31 - log2 n)) >> (32 - log2 n) for the base node and the low bits
// for the fraction, both exact.
#include <math.h>

#include <mutex>
#include <type_traits>

#include "internal.h"
#include "particles.h"
#include "update_dev.cuh"

namespace pm {

// ---------------------------------------------------------------- CIC decode (FP64 fractions)
struct CicD {
    int i0, i1;
    double w1;
};
__device__ __forceinline__ CicD cic_frac(double x, int n) {
    const double s = x * (double)n - 0.5;
    const double fl = floor(s);
    CicD c;
    c.w1 = s - fl;
    c.i0 = ((int)fl) & (n - 1);
    c.i1 = (c.i0 + 1) & (n - 1);
    return c;
}

// ---------------------------------------------------------------- deposit
__global__ void __launch_bounds__(256) k_deposit_ticks(const uint32_t* __restrict__ x, int64_t count, int logn,
                                                       float inv_cell_ticks, float mass, float* __restrict__ rho) {
    const size_t n = (size_t)1 << logn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const CicF cx = cic_ticks(x[i], logn, inv_cell_ticks);
        const CicF cy = cic_ticks(x[count + i], logn, inv_cell_ticks);
        const CicF cz = cic_ticks(x[2 * count + i], logn, inv_cell_ticks);
        const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
        const int ix[2] = {cx.i0, cx.i1}, iy[2] = {cy.i0, cy.i1}, iz[2] = {cz.i0, cz.i1};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float wab = mass * wx[a] * wy[b];
                float* row = rho + ((size_t)ix[a] * n + iy[b]) * n;
                atomicAdd(row + iz[0], wab * wz[0]);
                atomicAdd(row + iz[1], wab * wz[1]);
            }
    }
}

template <int R>
__global__ void __launch_bounds__(512) k_deposit_tiled(const uint32_t* __restrict__ x, int lognp, int logn,
                                                       float inv_cell_ticks, float mass, float* __restrict__ rho) {
    typedef DepTile<R> D;
    extern __shared__ __align__(16) uint32_t tile_words[];  // D::WORDS
    uint32_t* lo = tile_words;
    uint32_t* carry = tile_words + D::CELLS;
    const int ntz = (1 << lognp) / D::TZ, nty = (1 << lognp) / D::TY;
    const int bz = blockIdx.x % ntz, by = (blockIdx.x / ntz) % nty, bx = blockIdx.x / (ntz * nty);
    const int ox = bx * D::TX * R - D::H, oy = by * D::TY * R - D::H, oz = bz * D::TZ * R - D::HZ;
    const int64_t count = (int64_t)1 << (3 * lognp);
    tile_zero<D>(tile_words);
    __syncthreads();
    auto pid = [&](int e) -> int64_t {
        const int lz = e % D::TZ, ly = (e / D::TZ) % D::TY, lx = e / (D::TZ * D::TY);
        return ((((int64_t)(bx * D::TX + lx) << lognp) + by * D::TY + ly) << lognp) + bz * D::TZ + lz;
    };
    // positions are loaded one iteration ahead (their latency overlaps the deposit)
    int64_t idn = pid(threadIdx.x);
    uint32_t nu0 = x[idn], nu1 = x[count + idn], nu2 = x[2 * count + idn];
#pragma unroll 1
    for (int e = threadIdx.x; e < D::PER; e += 512) {
        const uint32_t u0 = nu0, u1 = nu1, u2 = nu2;
        if (e + 512 < D::PER) {
            idn = pid(e + 512);
            nu0 = x[idn];
            nu1 = x[count + idn];
            nu2 = x[2 * count + idn];
        }
        tile_deposit<D>(lo, carry, rho, u0, u1, u2, logn, inv_cell_ticks, ox, oy, oz, mass);
    }
    __syncthreads();
    tile_flush<D>(lo, carry, rho, ox, oy, oz, logn);
}

// R = 1: each thread walks one lattice row of the CTA's block along x and carries the upper-x
// plane of its CIC stencil to the next particle (the deposit half of the fused update kernel).
__global__ void __launch_bounds__(512, 2) k_deposit_sweep(const uint32_t* __restrict__ x, int lognp, int logn,
                                                          float inv_cell_ticks, float mass, float* __restrict__ rho) {
    typedef DepTile<1> D;
    static_assert(D::TY * D::TZ == 512, "one thread per (ly, lz); lx runs over the loop");
    extern __shared__ __align__(16) uint32_t tile_words[];  // D::WORDS
    uint32_t* lo = tile_words;
    uint32_t* carry = tile_words + D::CELLS;
    const int np = 1 << lognp;
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int ntz = np / D::TZ, nty = np / D::TY;
    const int bz = blockIdx.x % ntz, by = (blockIdx.x / ntz) % nty, bx = blockIdx.x / (ntz * nty);
    const int ox = bx * D::TX - D::H, oy = by * D::TY - D::H, oz = bz * D::TZ - D::HZ;
    tile_zero<D>(tile_words);
    __syncthreads();
    const int lz = threadIdx.x % D::TZ, ly = threadIdx.x / D::TZ;
    const int64_t id0 = ((((int64_t)(bx * D::TX) << lognp) + by * D::TY + ly) << lognp) + bz * D::TZ + lz;
    const int64_t xstride = (int64_t)1 << (2 * lognp);
    SweepCarry sc;
    uint32_t nu0 = x[id0], nu1 = x[count + id0], nu2 = x[2 * count + id0];
#pragma unroll 1
    for (int lx = 0; lx < D::TX; ++lx) {
        const uint32_t u0 = nu0, u1 = nu1, u2 = nu2;
        if (lx + 1 < D::TX) {
            const int64_t idn = id0 + (lx + 1) * xstride;
            nu0 = x[idn];
            nu1 = x[count + idn];
            nu2 = x[2 * count + idn];
        }
        sweep_deposit<D>(lo, carry, rho, u0, u1, u2, logn, inv_cell_ticks, ox, oy, oz, mass, sc);
    }
    sweep_finish<D>(lo, carry, sc);
    __syncthreads();
    tile_flush<D>(lo, carry, rho, ox, oy, oz, logn);
}

__global__ void k_deposit_frac(const double* __restrict__ x, int64_t count, int n, double mass,
                               double* __restrict__ rho) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const CicD cx = cic_frac(x[i], n), cy = cic_frac(x[count + i], n), cz = cic_frac(x[2 * count + i], n);
        const double wx[2] = {1.0 - cx.w1, cx.w1}, wy[2] = {1.0 - cy.w1, cy.w1}, wz[2] = {1.0 - cz.w1, cz.w1};
        const int ix[2] = {cx.i0, cx.i1}, iy[2] = {cy.i0, cy.i1}, iz[2] = {cz.i0, cz.i1};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const double wab = mass * wx[a] * wy[b];
                double* row = rho + ((size_t)ix[a] * n + iy[b]) * n;
                atomicAdd(row + iz[0], wab * wz[0]);
                atomicAdd(row + iz[1], wab * wz[1]);
            }
    }
}

static unsigned grid_for(int64_t count, int threads) {
    int64_t b = (count + threads - 1) / threads;
    const int64_t cap = 152 * 32;
    if (b > cap) b = cap;
    if (b < 1) b = 1;
    return (unsigned)b;
}

template <int R>
static cudaError_t deposit_tiled_r(const void* x, int np, int n, double mass, void* rho, cudaStream_t st) {
    typedef DepTile<R> D;
    const int lognp = ilog2(np), logn = ilog2(n);
    const unsigned blocks = (unsigned)((np / D::TX) * (np / D::TY) * (np / D::TZ));
    const float inv = (float)ldexp(1.0, -(32 - logn));
    const size_t smem = sizeof(uint32_t) * D::WORDS;
    if constexpr (R == 1) {
        cudaError_t e = set_smem_once((const void*)k_deposit_sweep, smem);
        if (e != cudaSuccess) return e;
        k_deposit_sweep<<<blocks, 512, smem, st>>>((const uint32_t*)x, lognp, logn, inv, (float)mass, (float*)rho);
        return cudaGetLastError();
    } else {
        cudaError_t e = set_smem_once((const void*)k_deposit_tiled<R>, smem);
        if (e != cudaSuccess) return e;
        k_deposit_tiled<R><<<blocks, 512, smem, st>>>((const uint32_t*)x, lognp, logn, inv, (float)mass, (float*)rho);
        return cudaGetLastError();
    }
}

cudaError_t deposit_lattice(const void* x, int np, int precision, int n, double mass, void* rho, cudaStream_t st) {
    const int R = n / np;
    if ((uintptr_t)rho % 16 != 0) return deposit(x, (int64_t)np * np * np, precision, n, mass, rho, st);
    // the tile box (16 + 4) x (16 + 4) x (32 + 8) cells must fit in the mesh without overlapping itself
    const bool tiled = precision == PM_FP32_FIXED && n >= 64 && (R == 1 || R == 2 || R == 4) && np >= 32 / R;
    if (!tiled) return deposit(x, (int64_t)np * np * np, precision, n, mass, rho, st);
    if (R == 1) return deposit_tiled_r<1>(x, np, n, mass, rho, st);
    if (R == 2) return deposit_tiled_r<2>(x, np, n, mass, rho, st);
    return deposit_tiled_r<4>(x, np, n, mass, rho, st);
}

cudaError_t deposit(const void* x, int64_t count, int precision, int n, double mass, void* rho,
                    cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const int logn = ilog2(n);
    if (precision == PM_FP32_FIXED) {
        const float inv = (float)ldexp(1.0, -(32 - logn));
        k_deposit_ticks<<<grid_for(count, 256), 256, 0, st>>>((const uint32_t*)x, count, logn, inv, (float)mass,
                                                              (float*)rho);
    } else {
        k_deposit_frac<<<grid_for(count, 256), 256, 0, st>>>((const double*)x, count, n, mass, (double*)rho);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- interpolation
template <typename T, typename X>
__device__ __forceinline__ T gather8(const T* __restrict__ f, size_t n, const int* ix, const int* iy,
                                     const int* iz, const T* wx, const T* wy, const T* wz) {
    T acc = T(0);
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const T* row = f + ((size_t)ix[a] * n + iy[b]) * n;
            acc += wx[a] * wy[b] * (wz[0] * __ldg(row + iz[0]) + wz[1] * __ldg(row + iz[1]));
        }
    return acc;
}

__global__ void k_interp_ticks(const float* __restrict__ f, int logn, const uint32_t* __restrict__ x,
                               int64_t count, float inv_cell_ticks, float* __restrict__ out) {
    const size_t n = (size_t)1 << logn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const CicF cx = cic_ticks(x[i], logn, inv_cell_ticks);
        const CicF cy = cic_ticks(x[count + i], logn, inv_cell_ticks);
        const CicF cz = cic_ticks(x[2 * count + i], logn, inv_cell_ticks);
        const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
        const int ix[2] = {cx.i0, cx.i1}, iy[2] = {cy.i0, cy.i1}, iz[2] = {cz.i0, cz.i1};
        out[i] = gather8<float, uint32_t>(f, n, ix, iy, iz, wx, wy, wz);
    }
}

__global__ void k_interp_frac(const double* __restrict__ f, int n, const double* __restrict__ x, int64_t count,
                              double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const CicD cx = cic_frac(x[i], n), cy = cic_frac(x[count + i], n), cz = cic_frac(x[2 * count + i], n);
        const double wx[2] = {1.0 - cx.w1, cx.w1}, wy[2] = {1.0 - cy.w1, cy.w1}, wz[2] = {1.0 - cz.w1, cz.w1};
        const int ix[2] = {cx.i0, cx.i1}, iy[2] = {cy.i0, cy.i1}, iz[2] = {cz.i0, cz.i1};
        out[i] = gather8<double, double>(f, (size_t)n, ix, iy, iz, wx, wy, wz);
    }
}

cudaError_t interp(const void* field, int n, const void* x, int64_t count, int precision, void* out,
                   cudaStream_t st) {
    if (count == 0) return cudaSuccess;
    const int logn = ilog2(n);
    if (precision == PM_FP32_FIXED) {
        const float inv = (float)ldexp(1.0, -(32 - logn));
        k_interp_ticks<<<grid_for(count, 256), 256, 0, st>>>((const float*)field, logn, (const uint32_t*)x, count,
                                                             inv, (float*)out);
    } else {
        k_interp_frac<<<grid_for(count, 256), 256, 0, st>>>((const double*)field, n, (const double*)x, count,
                                                            (double*)out);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- interp + kick + drift
template <bool FD>
__global__ void __launch_bounds__(256) k_ikd_ticks(uint32_t* __restrict__ x, float* __restrict__ p, int64_t count,
                                                   int logn, float inv_cell_ticks, const float* __restrict__ gx,
                                                   const float* __restrict__ gy, const float* __restrict__ gz,
                                                   float kick, float drift_ticks, float inv_d) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint32_t u0 = x[i], u1 = x[count + i], u2 = x[2 * count + i];
        float p0 = p[i], p1 = p[count + i], p2 = p[2 * count + i];
        ikd_particle<FD>(u0, u1, u2, p0, p1, p2, logn, inv_cell_ticks, gx, gy, gz, kick, drift_ticks, inv_d);
        p[i] = p0;
        p[count + i] = p1;
        p[2 * count + i] = p2;
        x[i] = u0;
        x[count + i] = u1;
        x[2 * count + i] = u2;
    }
}

// Same update, two neighbouring particles per thread through 8-byte loads and stores
// (count even, arrays 8-byte aligned): neighbours share most CIC corners, so the
// second particle's gathers mostly hit L1.
template <bool FD>
__global__ void __launch_bounds__(256) k_ikd_ticks2(uint32_t* __restrict__ x, float* __restrict__ p, int64_t count,
                                                    int logn, float inv_cell_ticks, const float* __restrict__ gx,
                                                    const float* __restrict__ gy, const float* __restrict__ gz,
                                                    float kick, float drift_ticks, float inv_d) {
    const int64_t pairs = count >> 1;
    uint2* x0 = reinterpret_cast<uint2*>(x);
    uint2* x1 = reinterpret_cast<uint2*>(x + count);
    uint2* x2 = reinterpret_cast<uint2*>(x + 2 * count);
    float2* p0 = reinterpret_cast<float2*>(p);
    float2* p1 = reinterpret_cast<float2*>(p + count);
    float2* p2 = reinterpret_cast<float2*>(p + 2 * count);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < pairs;
         i += (int64_t)gridDim.x * blockDim.x) {
        uint2 a = x0[i], b = x1[i], c = x2[i];
        float2 pa = p0[i], pb = p1[i], pc = p2[i];
        ikd_particle<FD>(a.x, b.x, c.x, pa.x, pb.x, pc.x, logn, inv_cell_ticks, gx, gy, gz, kick, drift_ticks, inv_d);
        ikd_particle<FD>(a.y, b.y, c.y, pa.y, pb.y, pc.y, logn, inv_cell_ticks, gx, gy, gz, kick, drift_ticks, inv_d);
        p0[i] = pa;
        p1[i] = pb;
        p2[i] = pc;
        x0[i] = a;
        x1[i] = b;
        x2[i] = c;
    }
}

template <bool FD>
__global__ void __launch_bounds__(256) k_ikd_frac(double* __restrict__ x, double* __restrict__ p, int64_t count,
                                                  int n, const double* __restrict__ gx, const double* __restrict__ gy,
                                                  const double* __restrict__ gz, double kick, double drift_box,
                                                  double inv_d) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        double xs[3] = {x[i], x[count + i], x[2 * count + i]};
        const CicD cx = cic_frac(xs[0], n), cy = cic_frac(xs[1], n), cz = cic_frac(xs[2], n);
        const double wx[2] = {1.0 - cx.w1, cx.w1}, wy[2] = {1.0 - cy.w1, cy.w1}, wz[2] = {1.0 - cz.w1, cz.w1};
        const int ix[2] = {cx.i0, cx.i1}, iy[2] = {cy.i0, cy.i1}, iz[2] = {cz.i0, cz.i1};
        double f[3];
        if constexpr (FD) {
            double P[2][4];
#pragma unroll
            for (int a = 0; a < 2; ++a)
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 2; ++c) P[a][2 * b + c] = gx[((size_t)ix[a] * n + iy[b]) * n + iz[c]];
            fd1_force<double>(P[0], P[1], wx[0], wx[1], wy, wz, inv_d, f[0], f[1], f[2]);
        } else {
            f[0] = gather8<double, double>(gx, (size_t)n, ix, iy, iz, wx, wy, wz);
            f[1] = gather8<double, double>(gy, (size_t)n, ix, iy, iz, wx, wy, wz);
            f[2] = gather8<double, double>(gz, (size_t)n, ix, iy, iz, wx, wy, wz);
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double pj = p[j * count + i] + kick * f[j];
            p[j * count + i] = pj;
            double xj = xs[j] + drift_box * pj;
            xj -= floor(xj);
            x[j * count + i] = xj;
        }
    }
}

template <bool FD>
static cudaError_t interp_kick_drift_t(void* x, void* p, int64_t count, int precision, int n, void* const* g,
                                       double kick, double drift, double box, double inv_d, cudaStream_t st) {
    const int logn = ilog2(n);
    if (precision == PM_FP32_FIXED) {
        const float inv = (float)ldexp(1.0, -(32 - logn));
        const float dt = (float)(drift * (4294967296.0 / box));
        const bool pairs = (count % 2 == 0) && ((uintptr_t)x % 8 == 0) && ((uintptr_t)p % 8 == 0);
        if (pairs)
            k_ikd_ticks2<FD><<<grid_for(count / 2, 256), 256, 0, st>>>((uint32_t*)x, (float*)p, count, logn, inv,
                                                                       (const float*)g[0], (const float*)g[1],
                                                                       (const float*)g[2], (float)kick, dt,
                                                                       (float)inv_d);
        else
            k_ikd_ticks<FD><<<grid_for(count, 256), 256, 0, st>>>((uint32_t*)x, (float*)p, count, logn, inv,
                                                                  (const float*)g[0], (const float*)g[1],
                                                                  (const float*)g[2], (float)kick, dt, (float)inv_d);
    } else {
        k_ikd_frac<FD><<<grid_for(count, 256), 256, 0, st>>>((double*)x, (double*)p, count, n, (const double*)g[0],
                                                             (const double*)g[1], (const double*)g[2], kick,
                                                             drift / box, inv_d);
    }
    return cudaGetLastError();
}

cudaError_t interp_kick_drift(void* x, void* p, int64_t count, int precision, int n, void* const* g,
                              double kick, double drift, double box, cudaStream_t st, double fd_inv_d) {
    if (count == 0) return cudaSuccess;
    if (fd_inv_d > 0.0) return interp_kick_drift_t<true>(x, p, count, precision, n, g, kick, drift, box, fd_inv_d, st);
    return interp_kick_drift_t<false>(x, p, count, precision, n, g, kick, drift, box, 0.0, st);
}

// ---------------------------------------------------------------- Zel'dovich placement
// x = q + D Psi(q), p = a^2 E f D Psi(q); q the lattice node of particle id i.
__global__ void k_ic_ticks(uint32_t* __restrict__ x, float* __restrict__ p, const float* __restrict__ psx,
                           const float* __restrict__ psy, const float* __restrict__ psz, int lognp,
                           double disp_ticks, double pfac) {
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int sh = 32 - lognp;
    const int mask = (1 << lognp) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q[3] = {(uint32_t)((i >> (2 * lognp)) & mask) << sh, (uint32_t)((i >> lognp) & mask) << sh,
                               (uint32_t)(i & mask) << sh};
        const float ps[3] = {psx[i], psy[i], psz[i]};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            x[j * count + i] = q[j] + (uint32_t)__double2ll_rn((double)ps[j] * disp_ticks);
            p[j * count + i] = (float)(pfac * (double)ps[j]);
        }
    }
}

__global__ void k_ic_frac(double* __restrict__ x, double* __restrict__ p, const double* __restrict__ psx,
                          const double* __restrict__ psy, const double* __restrict__ psz, int lognp, double disp_box,
                          double pfac) {
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int mask = (1 << lognp) - 1;
    const double inv_np = ldexp(1.0, -lognp);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double q[3] = {(double)((i >> (2 * lognp)) & mask) * inv_np, (double)((i >> lognp) & mask) * inv_np,
                             (double)(i & mask) * inv_np};
        const double ps[3] = {psx[i], psy[i], psz[i]};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double xj = q[j] + disp_box * ps[j];
            xj -= floor(xj);
            x[j * count + i] = xj;
            p[j * count + i] = pfac * ps[j];
        }
    }
}

cudaError_t ic_place(void* x, void* p, void* const* psi, int np, int precision, double D, double pfac, double box,
                     cudaStream_t st) {
    const int lognp = ilog2(np);
    const int64_t count = (int64_t)np * np * np;
    if (precision == PM_FP32_FIXED) {
        k_ic_ticks<<<grid_for(count, 256), 256, 0, st>>>((uint32_t*)x, (float*)p, (const float*)psi[0],
                                                         (const float*)psi[1], (const float*)psi[2], lognp,
                                                         D * 4294967296.0 / box, pfac);
    } else {
        k_ic_frac<<<grid_for(count, 256), 256, 0, st>>>((double*)x, (double*)p, (const double*)psi[0],
                                                        (const double*)psi[1], (const double*)psi[2], lognp, D / box,
                                                        pfac);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- second-order LPT
// With Psi1 = -grad phi1, phi1_ij = -d_j Psi1_i, and the 2LPT source
//   S = sum_{i<j} (phi1_ii phi1_jj - phi1_ij^2)
// (Bouchet et al. 1995; Scoccimarro 1998) is gathered over the three components:
//   stage 0 (Psi1_x): S = -(d_y Psi_x)^2 - (d_z Psi_x)^2,   A = d_x Psi_x
//   stage 1 (Psi1_y): S += A d_y Psi_y - (d_z Psi_y)^2,      A += d_y Psi_y
//   stage 2 (Psi1_z): S += A d_z Psi_z
template <typename T>
__global__ void k_lpt2_source(int stage, const T* __restrict__ d0, const T* __restrict__ d1, const T* __restrict__ d2,
                              T* __restrict__ s, T* __restrict__ a, int64_t count) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (stage == 0) {
            const T y = d1[i], z = d2[i];
            s[i] = -(y * y) - z * z;
            a[i] = d0[i];
        } else if (stage == 1) {
            const T y = d1[i], z = d2[i], ai = a[i];
            s[i] += ai * y - z * z;
            a[i] = ai + y;
        } else {
            s[i] += a[i] * d2[i];
        }
    }
}

cudaError_t lpt2_source(int stage, void* const* d, void* s, void* a, int64_t count, int precision, cudaStream_t st) {
    if (precision == PM_FP32_FIXED)
        k_lpt2_source<float><<<grid_for(count, 256), 256, 0, st>>>(stage, (const float*)d[0], (const float*)d[1],
                                                                   (const float*)d[2], (float*)s, (float*)a, count);
    else
        k_lpt2_source<double><<<grid_for(count, 256), 256, 0, st>>>(stage, (const double*)d[0], (const double*)d[1],
                                                                    (const double*)d[2], (double*)s, (double*)a, count);
    return cudaGetLastError();
}

// x = q + D1 Psi1 + D2 Psi2, p = pfac1 Psi1 + pfac2 Psi2.  Psi1 may live in p: each thread
// reads the three components of its particle before writing them (no __restrict__ there).
struct Psi3 {
    const void* c[3];
};

__global__ void k_ic2_ticks(uint32_t* __restrict__ x, float* p, Psi3 ps1, Psi3 ps2, int lognp, double disp1,
                            double disp2, double pfac1, double pfac2) {
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int sh = 32 - lognp;
    const int mask = (1 << lognp) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q[3] = {(uint32_t)((i >> (2 * lognp)) & mask) << sh, (uint32_t)((i >> lognp) & mask) << sh,
                               (uint32_t)(i & mask) << sh};
        double a1[3], a2[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            a1[j] = (double)((const float*)ps1.c[j])[i];
            a2[j] = (double)((const float*)ps2.c[j])[i];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            x[j * count + i] = q[j] + (uint32_t)__double2ll_rn(a1[j] * disp1 + a2[j] * disp2);
            p[j * count + i] = (float)(pfac1 * a1[j] + pfac2 * a2[j]);
        }
    }
}

__global__ void k_ic2_frac(double* __restrict__ x, double* p, Psi3 ps1, Psi3 ps2, int lognp, double disp1,
                           double disp2, double pfac1, double pfac2) {
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int mask = (1 << lognp) - 1;
    const double inv_np = ldexp(1.0, -lognp);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double q[3] = {(double)((i >> (2 * lognp)) & mask) * inv_np, (double)((i >> lognp) & mask) * inv_np,
                             (double)(i & mask) * inv_np};
        double a1[3], a2[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            a1[j] = ((const double*)ps1.c[j])[i];
            a2[j] = ((const double*)ps2.c[j])[i];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            double xj = q[j] + (disp1 * a1[j] + disp2 * a2[j]);
            xj -= floor(xj);
            x[j * count + i] = xj;
            p[j * count + i] = pfac1 * a1[j] + pfac2 * a2[j];
        }
    }
}

cudaError_t ic_place2(void* x, void* p, void* const* psi1, void* const* psi2, int np, int precision, double D1,
                      double D2, double pfac1, double pfac2, double box, cudaStream_t st) {
    const int lognp = ilog2(np);
    const int64_t count = (int64_t)np * np * np;
    const Psi3 a = {{psi1[0], psi1[1], psi1[2]}}, b = {{psi2[0], psi2[1], psi2[2]}};
    if (precision == PM_FP32_FIXED) {
        k_ic2_ticks<<<grid_for(count, 256), 256, 0, st>>>((uint32_t*)x, (float*)p, a, b, lognp,
                                                          D1 * 4294967296.0 / box, D2 * 4294967296.0 / box, pfac1,
                                                          pfac2);
    } else {
        k_ic2_frac<<<grid_for(count, 256), 256, 0, st>>>((double*)x, (double*)p, a, b, lognp, D1 / box, D2 / box,
                                                         pfac1, pfac2);
    }
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Philox phases
// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32->64
// multiplies with the Philox multipliers, xor with the key, word permutation, and
// a Weyl-sequence key bump between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint32_t k0, uint32_t k1) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k0 += W0;
            k1 += W1;
        }
        const uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        const uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
    }
    return c;
}

// Unit complex Gaussian per wavevector on the [kz][kx][ky] half grid; Hermitian
// partners on kz = 0 are conjugates of the canonical draw; Nyquist and zero modes 0.
template <typename T>
__global__ void k_noise(cplx<T>* __restrict__ spec, int n, uint32_t seed_lo, uint32_t seed_hi) {
    const int M = n >> 1;
    const int64_t total = (int64_t)(M + 1) * n * n;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int kz = (int)(e / ((int64_t)n * n));
        const int rem = (int)(e - (int64_t)kz * n * n);
        const int nx = signed_k(rem / n, n), ny = signed_k(rem % n, n), nz = kz;
        cplx<T> g;
        g.x = T(0);
        g.y = T(0);
        const bool nyq = (2 * nx == -n) || (2 * ny == -n) || (nz == M);
        if (!nyq && (nx | ny | nz) != 0) {
            const bool canonical = nz > 0 || ny > 0 || (ny == 0 && nx > 0);
            const int cx = canonical ? nx : -nx, cy = canonical ? ny : -ny;
            const uint4 r = philox4x32_10(make_uint4((uint32_t)cx, (uint32_t)cy, (uint32_t)nz, 0u), seed_lo, seed_hi);
            const double u1 = ((double)r.x + 0.5) * 2.3283064365386963e-10;  // 2^-32
            const double u2 = ((double)r.y + 0.5) * 2.3283064365386963e-10;
            const double amp = sqrt(-log(u1));
            double s, c;
            sincospi(2.0 * u2, &s, &c);
            g.x = T(amp * c);
            g.y = T(canonical ? amp * s : -amp * s);
        }
        spec[e] = g;
    }
}

template <typename T>
cudaError_t noise(cplx<T>* spec, int n, uint64_t seed, cudaStream_t st) {
    const int64_t total = (int64_t)(n / 2 + 1) * n * n;
    k_noise<T><<<grid_for(total, 256), 256, 0, st>>>(spec, n, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
    return cudaGetLastError();
}
template cudaError_t noise<float>(float2*, int, uint64_t, cudaStream_t);
template cudaError_t noise<double>(double2*, int, uint64_t, cudaStream_t);

// ---------------------------------------------------------------- GR displacement combination
// xi = x_GR - x_N on the coarse lattice (exact minimum image on ticks), trilinear in
// the Lagrangian lattice index to the target lattice (r = npt / npc), x_t += xi.
__global__ void k_combine_ticks(uint32_t* __restrict__ xt, const uint32_t* __restrict__ xg,
                                const uint32_t* __restrict__ xn, int32_t* __restrict__ xi_out, int lognt,
                                int lognc) {
    const int64_t countt = (int64_t)1 << (3 * lognt);
    const int64_t countc = (int64_t)1 << (3 * lognc);
    const int logr = lognt - lognc;
    const int r = 1 << logr;
    const int maskt = (1 << lognt) - 1, maskc = (1 << lognc) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < countt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int it[3] = {(int)((i >> (2 * lognt)) & maskt), (int)((i >> lognt) & maskt), (int)(i & maskt)};
        int base[3], off[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            base[j] = it[j] >> logr;
            off[j] = it[j] & (r - 1);
        }
        int64_t S[3] = {0, 0, 0};
#pragma unroll
        for (int dx = 0; dx < 2; ++dx)
#pragma unroll
            for (int dy = 0; dy < 2; ++dy)
#pragma unroll
                for (int dz = 0; dz < 2; ++dz) {
                    const int64_t W = (int64_t)(dx ? off[0] : r - off[0]) * (dy ? off[1] : r - off[1]) *
                                      (dz ? off[2] : r - off[2]);
                    if (W == 0) continue;
                    const int64_t c = (((int64_t)((base[0] + dx) & maskc) << (2 * lognc)) |
                                       ((int64_t)((base[1] + dy) & maskc) << lognc) | ((base[2] + dz) & maskc));
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        const int32_t d = (int32_t)(xg[j * countc + c] - xn[j * countc + c]);
                        S[j] += W * (int64_t)d;
                    }
                }
        const int s = 3 * logr;
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            int64_t q = S[j];
            if (s > 0) {  // round-half-even of S / 2^s
                const int64_t fl = S[j] >> s;
                const int64_t rem = S[j] - (fl << s);
                const int64_t half = (int64_t)1 << (s - 1);
                q = fl + ((rem > half || (rem == half && (fl & 1))) ? 1 : 0);
            }
            xt[j * countt + i] += (uint32_t)q;
            if (xi_out) xi_out[j * countt + i] = (int32_t)q;
        }
    }
}

// The same combination by blocks: one thread per coarse node b, for the r^3 targets whose
// lower coarse node is b (trilinear from the 8 nodes b + {0,1}^3; xi formed once per node).
// The r targets of a z-run sit together: their positions are read and written as one
// r-wide vector (r = 1, 2, 4), consecutive threads covering consecutive runs.
template <int LOGR>
__global__ void __launch_bounds__(256) k_combine_blocks(uint32_t* __restrict__ xt, const uint32_t* __restrict__ xg,
                                                        const uint32_t* __restrict__ xn, int32_t* __restrict__ xi_out,
                                                        int lognc) {
    constexpr int r = 1 << LOGR, s = 3 * LOGR;
    typedef typename std::conditional<r == 4, uint4, typename std::conditional<r == 2, uint2, uint32_t>::type>::type V;
    const int maskc = (1 << lognc) - 1, lognt = lognc + LOGR;
    const int64_t countc = (int64_t)1 << (3 * lognc), countt = (int64_t)1 << (3 * lognt);
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < countc;
         b += (int64_t)gridDim.x * blockDim.x) {
        const int bx = (int)(b >> (2 * lognc)), by = (int)((b >> lognc) & maskc), bz = (int)(b & maskc);
        int32_t xi[3][8];  // corner q = 4 dx + 2 dy + dz
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const int64_t c = ((int64_t)((bx + (q >> 2)) & maskc) << (2 * lognc)) |
                              ((int64_t)((by + ((q >> 1) & 1)) & maskc) << lognc) | ((bz + (q & 1)) & maskc);
#pragma unroll
            for (int j = 0; j < 3; ++j) xi[j][q] = (int32_t)(xg[j * countc + c] - xn[j * countc + c]);
        }
        // one x plane of the r^3 target block at a time: its r x 3 target vectors are loaded
        // before any arithmetic, so their latencies overlap instead of forming r^2 x 3 chains
#pragma unroll 1
        for (int ox = 0; ox < r; ++ox) {
            V v[r][3];
#pragma unroll
            for (int oy = 0; oy < r; ++oy) {
                const int64_t t0 = ((((int64_t)(r * bx + ox) << lognt) + (r * by + oy)) << lognt) + r * bz;
#pragma unroll
                for (int j = 0; j < 3; ++j) v[oy][j] = *reinterpret_cast<const V*>(xt + j * countt + t0);
            }
#pragma unroll
            for (int oy = 0; oy < r; ++oy) {
                const int64_t t0 = ((((int64_t)(r * bx + ox) << lognt) + (r * by + oy)) << lognt) + r * bz;
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    uint32_t add[r];
#pragma unroll
                    for (int oz = 0; oz < r; ++oz) {
                        // S = sum over the corners of (weights in units of 1/r per axis) xi; exact in 64 bits
                        int64_t S = 0;
#pragma unroll
                        for (int q = 0; q < 8; ++q) {
                            const int wx = (q >> 2) ? ox : r - ox, wy = ((q >> 1) & 1) ? oy : r - oy,
                                      wz = (q & 1) ? oz : r - oz;
                            S += (int64_t)xi[j][q] * (wx * wy * wz);
                        }
                        int64_t qv = S;
                        if (s > 0) {  // round-half-even of S / r^3
                            const int64_t fl = S >> s;
                            const int64_t rem = S - (fl << s);
                            const int64_t half = (int64_t)1 << (s > 0 ? s - 1 : 0);
                            qv = fl + ((rem > half || (rem == half && (fl & 1))) ? 1 : 0);
                        }
                        add[oz] = (uint32_t)qv;
                    }
                    uint32_t* vv = reinterpret_cast<uint32_t*>(&v[oy][j]);
#pragma unroll
                    for (int oz = 0; oz < r; ++oz) vv[oz] += add[oz];
                    *reinterpret_cast<V*>(xt + j * countt + t0) = v[oy][j];
                    if (xi_out) {
                        V w;
                        uint32_t* ww = reinterpret_cast<uint32_t*>(&w);
#pragma unroll
                        for (int oz = 0; oz < r; ++oz) ww[oz] = add[oz];
                        *reinterpret_cast<V*>(xi_out + j * countt + t0) = w;
                    }
                }
            }
        }
    }
}

__global__ void k_combine_frac(double* __restrict__ xt, const double* __restrict__ xg, const double* __restrict__ xn,
                               double* __restrict__ xi_out, int lognt, int lognc) {
    const int64_t countt = (int64_t)1 << (3 * lognt);
    const int64_t countc = (int64_t)1 << (3 * lognc);
    const int logr = lognt - lognc;
    const int r = 1 << logr;
    const double inv_r3 = ldexp(1.0, -3 * logr);
    const int maskt = (1 << lognt) - 1, maskc = (1 << lognc) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < countt;
         i += (int64_t)gridDim.x * blockDim.x) {
        const int it[3] = {(int)((i >> (2 * lognt)) & maskt), (int)((i >> lognt) & maskt), (int)(i & maskt)};
        int base[3], off[3];
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            base[j] = it[j] >> logr;
            off[j] = it[j] & (r - 1);
        }
        double S[3] = {0, 0, 0};
        for (int dx = 0; dx < 2; ++dx)
            for (int dy = 0; dy < 2; ++dy)
                for (int dz = 0; dz < 2; ++dz) {
                    const int W = (dx ? off[0] : r - off[0]) * (dy ? off[1] : r - off[1]) * (dz ? off[2] : r - off[2]);
                    if (W == 0) continue;
                    const int64_t c = (((int64_t)((base[0] + dx) & maskc) << (2 * lognc)) |
                                       ((int64_t)((base[1] + dy) & maskc) << lognc) | ((base[2] + dz) & maskc));
                    for (int j = 0; j < 3; ++j) {
                        double d = xg[j * countc + c] - xn[j * countc + c];
                        d -= rint(d);
                        S[j] += (double)W * d;
                    }
                }
        for (int j = 0; j < 3; ++j) {
            const double xi = S[j] * inv_r3;
            double xj = xt[j * countt + i] + xi;
            xj -= floor(xj);
            xt[j * countt + i] = xj;
            if (xi_out) xi_out[j * countt + i] = xi;
        }
    }
}

cudaError_t combine(void* xt, const void* xg, const void* xn, void* xi_out, int npt, int npc, int precision,
                    cudaStream_t st) {
    const int lognt = ilog2(npt), lognc = ilog2(npc);
    const int64_t count = (int64_t)npt * npt * npt;
    const int64_t countc = (int64_t)npc * npc * npc;
    // vector accesses need 4 r-byte alignment (the library's particle arrays are 256-byte aligned)
    const bool aligned = (uintptr_t)xt % 16 == 0 && (uintptr_t)xi_out % 16 == 0;
    if (precision == PM_FP32_FIXED && aligned && lognt - lognc <= 2) {
        const unsigned g = grid_for(countc, 256);
        if (lognt == lognc)
            k_combine_blocks<0><<<g, 256, 0, st>>>((uint32_t*)xt, (const uint32_t*)xg, (const uint32_t*)xn,
                                                   (int32_t*)xi_out, lognc);
        else if (lognt == lognc + 1)
            k_combine_blocks<1><<<g, 256, 0, st>>>((uint32_t*)xt, (const uint32_t*)xg, (const uint32_t*)xn,
                                                   (int32_t*)xi_out, lognc);
        else
            k_combine_blocks<2><<<g, 256, 0, st>>>((uint32_t*)xt, (const uint32_t*)xg, (const uint32_t*)xn,
                                                   (int32_t*)xi_out, lognc);
    } else if (precision == PM_FP32_FIXED)
        k_combine_ticks<<<grid_for(count, 256), 256, 0, st>>>((uint32_t*)xt, (const uint32_t*)xg,
                                                              (const uint32_t*)xn, (int32_t*)xi_out, lognt, lognc);
    else
        k_combine_frac<<<grid_for(count, 256), 256, 0, st>>>((double*)xt, (const double*)xg, (const double*)xn,
                                                             (double*)xi_out, lognt, lognc);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- fill
template <typename T>
__global__ void k_fill(T* __restrict__ a, int64_t count, T v) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = v;
}
cudaError_t fill(void* a, int64_t count, int precision, double v, cudaStream_t st) {
    if (precision == PM_FP32_FIXED)
        k_fill<float><<<grid_for(count, 256), 256, 0, st>>>((float*)a, count, (float)v);
    else
        k_fill<double><<<grid_for(count, 256), 256, 0, st>>>((double*)a, count, v);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- Lagrangian displacement
// d = x - q (minimum image) in Mpc/h for the np^3 lattice-ordered particles, q the node of
// particle id = (ix np + iy) np + iz.  Ticks: the uint32 difference read as int32 is the
// minimum image exactly.
__global__ void k_disp_ticks(const uint32_t* __restrict__ x, float* __restrict__ d, int lognp, float tick_mpc) {
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int mask = (1 << lognp) - 1;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t q[3] = {(uint32_t)((i >> (2 * lognp)) & mask) << (32 - lognp),
                               (uint32_t)((i >> lognp) & mask) << (32 - lognp), (uint32_t)(i & mask) << (32 - lognp)};
#pragma unroll
        for (int j = 0; j < 3; ++j) d[j * count + i] = (float)(int32_t)(x[j * count + i] - q[j]) * tick_mpc;
    }
}
__global__ void k_disp_frac(const double* __restrict__ x, double* __restrict__ d, int lognp, double box) {
    const int64_t count = (int64_t)1 << (3 * lognp);
    const int mask = (1 << lognp) - 1;
    const double inv_np = 1.0 / (double)(1 << lognp);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int q[3] = {(int)((i >> (2 * lognp)) & mask), (int)((i >> lognp) & mask), (int)(i & mask)};
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const double v = x[j * count + i] - q[j] * inv_np;
            d[j * count + i] = (v - rint(v)) * box;
        }
    }
}
cudaError_t lagrangian_displacement(const void* x, void* d, int np, int precision, double box, cudaStream_t st) {
    const int lognp = ilog2(np);
    const int64_t count = (int64_t)np * np * np;
    if (precision == PM_FP32_FIXED)
        k_disp_ticks<<<grid_for(count, 256), 256, 0, st>>>((const uint32_t*)x, (float*)d, lognp,
                                                           (float)(box / 4294967296.0));
    else
        k_disp_frac<<<grid_for(count, 256), 256, 0, st>>>((const double*)x, (double*)d, lognp, box);
    return cudaGetLastError();
}

// Positions in Mpc/h in [0, L): uint32 ticks times L / 2^32 (exact in double, then rounded
// down to float, so that no position rounds up to L), or box fractions times L.
__global__ void k_pos_ticks(const uint32_t* __restrict__ x, float* __restrict__ out, int64_t n, double tick_mpc) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = __double2float_rd((double)x[i] * tick_mpc);
}
__global__ void k_pos_frac(const double* __restrict__ x, double* __restrict__ out, int64_t n, double box) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x[i] * box;
}
cudaError_t positions_mpc(const void* x, void* out, int64_t count, int precision, double box, cudaStream_t st) {
    const int64_t n = 3 * count;
    if (n == 0) return cudaSuccess;
    if (precision == PM_FP32_FIXED)
        k_pos_ticks<<<grid_for(n, 256), 256, 0, st>>>((const uint32_t*)x, (float*)out, n, box / 4294967296.0);
    else
        k_pos_frac<<<grid_for(n, 256), 256, 0, st>>>((const double*)x, (double*)out, n, box);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- position check
// Counts FP64 box-fraction positions that are not finite or lie outside [0, 1) (one
// warp-aggregated atomic a warp).
__global__ void k_count_outside(const double* __restrict__ x, int64_t count, unsigned long long* __restrict__ bad) {
    unsigned long long mine = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const double v = x[i];
        mine += (v >= 0.0 && v < 1.0) ? 0ull : 1ull;  // false for NaN: counted
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) mine += __shfl_down_sync(0xffffffffu, mine, o);
    if ((threadIdx.x & 31) == 0 && mine) atomicAdd(bad, mine);
}
cudaError_t count_outside_box(const double* x, int64_t count, unsigned long long* bad, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(bad, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess || count == 0) return e;
    k_count_outside<<<grid_for(count, 256), 256, 0, st>>>(x, count, bad);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- cell keys and stable order
__global__ void k_cell_keys(const void* __restrict__ xv, int64_t count, int precision, int logn, float inv_cell_ticks,
                            uint32_t* __restrict__ keys, uint32_t* __restrict__ counts) {
    const int n = 1 << logn;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x) {
        int b[3];
        if (precision == PM_FP32_FIXED) {
            const uint32_t* x = (const uint32_t*)xv;
            for (int j = 0; j < 3; ++j) b[j] = cic_ticks(x[j * count + i], logn, inv_cell_ticks).i0;
        } else {
            const double* x = (const double*)xv;
            for (int j = 0; j < 3; ++j) b[j] = cic_frac(x[j * count + i], n).i0;
        }
        const uint32_t key = ((uint32_t)b[0] << (2 * logn)) | ((uint32_t)b[1] << logn) | (uint32_t)b[2];
        keys[i] = key;
        if (counts) atomicAdd(&counts[key], 1u);
    }
}

// Exclusive scan, 4 elements per thread, 1024 threads per block.
__global__ void __launch_bounds__(1024) k_scan_block(const uint32_t* __restrict__ in, uint32_t* __restrict__ out,
                                                     int64_t count, uint32_t* __restrict__ block_sums) {
    __shared__ uint32_t warp_tot[32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t base = (int64_t)blockIdx.x * 4096 + 4 * tid;
    uint32_t v[4];
    uint32_t local = 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        v[k] = (base + k < count) ? in[base + k] : 0u;
        const uint32_t t = v[k];
        v[k] = local;
        local += t;
    }
    uint32_t incl = local;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, d);
        if (lane >= d) incl += y;
    }
    if (lane == 31) warp_tot[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t w = warp_tot[lane];
        uint32_t wi = w;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, wi, d);
            if (lane >= d) wi += y;
        }
        warp_tot[lane] = wi - w;  // exclusive warp offsets
        if (lane == 31 && block_sums) block_sums[blockIdx.x] = wi;
    }
    __syncthreads();
    const uint32_t off = warp_tot[wid] + (incl - local);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (base + k < count) out[base + k] = v[k] + off;
}

__global__ void k_scan_add(uint32_t* __restrict__ out, int64_t count, const uint32_t* __restrict__ sums) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) out[i] += sums[i / 4096];
}

// Exclusive scan of count uint32 values; scratch: scan_scratch_words(count) words.
static int64_t scan_scratch_words(int64_t count) {
    int64_t words = 0;
    while (count > 4096) {
        count = (count + 4095) / 4096;
        words += count + 1;
    }
    return words + 1;
}
static cudaError_t scan_u32(const uint32_t* in, uint32_t* out, int64_t count, uint32_t* scratch, cudaStream_t st) {
    const int64_t nblk = (count + 4095) / 4096;
    if (nblk <= 1) {
        k_scan_block<<<1, 1024, 0, st>>>(in, out, count, nullptr);
        return cudaGetLastError();
    }
    uint32_t* sums = scratch;
    k_scan_block<<<(unsigned)nblk, 1024, 0, st>>>(in, out, count, sums);
    cudaError_t e = scan_u32(sums, sums, nblk, scratch + nblk + 1, st);
    if (e != cudaSuccess) return e;
    k_scan_add<<<(unsigned)((count + 255) / 256), 256, 0, st>>>(out, count, sums);
    return cudaGetLastError();
}

cudaError_t scan_exclusive_u32(const uint32_t* in, uint32_t* out, int64_t count, void* scratch, cudaStream_t st) {
    return scan_u32(in, out, count, (uint32_t*)scratch, st);
}

size_t scan_scratch_bytes(int64_t count) { return sizeof(uint32_t) * (size_t)(scan_scratch_words(count) + 64); }

__global__ void k_scatter_unstable(const uint32_t* __restrict__ keys, int64_t count, uint32_t* __restrict__ cursor,
                                   uint32_t* __restrict__ order) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count;
         i += (int64_t)gridDim.x * blockDim.x)
        order[atomicAdd(&cursor[keys[i]], 1u)] = (uint32_t)i;
}

// Within each cell the ids were placed in arbitrary order; sort them ascending
// (Shell sort with gaps 1, 4, 13, ...), which makes the whole order stable in id.
__global__ void k_sort_buckets(const uint32_t* __restrict__ start, const uint32_t* __restrict__ cursor, int64_t ncell,
                               uint32_t* __restrict__ order) {
    for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t s = start[c], e = cursor[c];
        const uint32_t len = e - s;
        if (len < 2) continue;
        uint32_t* a = order + s;
        uint32_t gap = 1;
        while (gap < len / 3) gap = 3 * gap + 1;
        for (; gap > 0; gap /= 3)
            for (uint32_t i = gap; i < len; ++i) {
                const uint32_t v = a[i];
                uint32_t j = i;
                while (j >= gap && a[j - gap] > v) {
                    a[j] = a[j - gap];
                    j -= gap;
                }
                a[j] = v;
            }
    }
}

size_t cell_sort_scratch_bytes(int64_t count, int n) {
    const int64_t ncell = (int64_t)n * n * n;
    (void)count;
    return sizeof(uint32_t) * (size_t)(3 * ncell + scan_scratch_words(ncell) + 64);
}

cudaError_t cell_sort(const void* x, int64_t count, int precision, int n, uint32_t* keys, uint32_t* order,
                      void* scratch, cudaStream_t st) {
    const int logn = ilog2(n);
    const int64_t ncell = (int64_t)n * n * n;
    uint32_t* counts = (uint32_t*)scratch;
    uint32_t* start = counts + ncell;
    uint32_t* cursor = start + ncell;
    uint32_t* sc = cursor + ncell;
    const float inv = (float)ldexp(1.0, -(32 - logn));
    cudaError_t e;
    if (order) {
        e = cudaMemsetAsync(counts, 0, sizeof(uint32_t) * ncell, st);
        if (e != cudaSuccess) return e;
    }
    if (count > 0)
        k_cell_keys<<<grid_for(count, 256), 256, 0, st>>>(x, count, precision, logn, inv, keys,
                                                          order ? counts : nullptr);
    e = cudaGetLastError();
    if (e != cudaSuccess || !order) return e;
    e = scan_u32(counts, start, ncell, sc, st);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(cursor, start, sizeof(uint32_t) * ncell, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    if (count > 0) k_scatter_unstable<<<grid_for(count, 256), 256, 0, st>>>(keys, count, cursor, order);
    k_sort_buckets<<<grid_for(ncell, 256), 256, 0, st>>>(start, cursor, ncell, order);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- cell order without caller scratch
// Counting scratch for cell_sort_static: a fixed device array that every call on this
// GPU shares (it lives until the process exits).  Host code must not use the symbol
// as an address: the device address is looked up once per device below.
constexpr int64_t kStaticSortCells = (int64_t)64 * 64 * 64;
constexpr int64_t kStaticSortWords = 3 * kStaticSortCells + 4096;
static __device__ __align__(256) uint32_t g_sort_scratch[kStaticSortWords];

static std::mutex g_sort_mutex;
struct StaticSortAddr {
    unsigned long long ctx_id = 0;  // CUDA context the address belongs to (0: none yet)
    uint32_t* ptr = nullptr;
};
static StaticSortAddr g_sort_addr[128];

int64_t cell_sort_static_max_cells() { return kStaticSortCells; }

// Unique id of the calling thread's current CUDA context (0 when there is none), from the
// driver's cuCtxGetCurrent / cuCtxGetId reached through the runtime's entry-point query.
static unsigned long long current_context_id() {
    typedef int (*GetCurrent)(void**);
    typedef int (*GetId)(void*, unsigned long long*);
    static GetCurrent get_current = nullptr;
    static GetId get_id = nullptr;
    if (!get_current || !get_id) {
        void* f1 = nullptr;
        void* f2 = nullptr;
        cudaDriverEntryPointQueryResult q1, q2;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) != cudaSuccess ||
            cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) != cudaSuccess ||
            q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
            cudaGetLastError();
            return 0;
        }
        get_current = (GetCurrent)f1;
        get_id = (GetId)f2;
    }
    void* ctx = nullptr;
    unsigned long long id = 0;
    if (get_current(&ctx) != 0 || !ctx || get_id(ctx, &id) != 0) return 0;
    return id;
}

// Device address of g_sort_scratch in the current device's current context.  It is looked
// up (cudaGetSymbolAddress) on the first call in each context and cached under the
// context's id, so a context that is torn down and made again (cudaDeviceReset, a new
// primary context) gets a fresh lookup instead of a stale address.
static cudaError_t static_sort_scratch(uint32_t** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 128) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_sort_mutex);
    StaticSortAddr& a = g_sort_addr[dev];
    unsigned long long id = current_context_id();
    if (id == 0 || id != a.ctx_id || !a.ptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_sort_scratch);  // makes the runtime's context current if needed
        if (e != cudaSuccess) return e;
        if (id == 0) id = current_context_id();
        a.ctx_id = id;
        a.ptr = (uint32_t*)p;
    }
    *out = a.ptr;
    return cudaSuccess;
}

cudaError_t cell_sort_static(const void* x, int64_t count, int precision, int n, uint32_t* keys, uint32_t* order,
                             cudaStream_t st) {
    uint32_t* scratch = nullptr;
    cudaError_t e = static_sort_scratch(&scratch);
    if (e != cudaSuccess) return e;
    // cell_sort clears the counts it needs before use, so stale contents of the
    // shared array from an earlier call do not leak into this one
    return cell_sort(x, count, precision, n, keys, order, scratch, st);
}

}  // namespace pm
