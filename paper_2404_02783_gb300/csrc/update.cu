// The fused particle update of the FP32 PM step: CIC gather of the force at the old
// position, kick, drift, and the CIC deposit of the drifted position into the density of
// the next step, one pass over the lattice-ordered particles by Lagrangian tiles (KDK in a;
// counting density, Sec. 4).  Positions are uint32 ticks (2^32 per side).
#include "internal.h"
#include "particles.h"
#include "update_dev.cuh"

namespace pm {

// ---------------------------------------------------------------- kick + drift + next deposit
// One pass per step over the lattice-ordered particles by Lagrangian tiles: gather the
// force at x, kick, drift, and deposit the new position into the (zeroed) next
// density mesh through the tile's shared-memory accumulator, exactly as
// k_deposit_tiled would have done from the drifted positions.
// blockIdx.y selects the field of a batch of independent runs stored back to back
// (particles [field][3][np^3], meshes [field][n^3]); scale = 2^32 / L of that field.
template <int R, bool FD>
__global__ void __launch_bounds__(512, 2) k_ikd_deposit(const uint32_t* __restrict__ x, uint32_t* __restrict__ xo, float* __restrict__ p, int lognp,
                                                     int logn, float inv_cell_ticks, const float* __restrict__ gx,
                                                     const float* __restrict__ gy, const float* __restrict__ gz,
                                                     float kick, double drift, double scale0,
                                                     const double* __restrict__ scale_arr, float mass,
                                                     float* __restrict__ rho, float inv_d) {
    typedef DepTile<R> D;
    extern __shared__ __align__(16) uint32_t tile_words[];  // D::WORDS
    uint32_t* lo = tile_words;
    uint32_t* carry = tile_words + D::CELLS;
    const int np = 1 << lognp;
    const int64_t count = (int64_t)1 << (3 * lognp);
    {
        const int64_t fb = blockIdx.y;
        const int64_t n3 = (int64_t)1 << (3 * logn);
        x += fb * 3 * count;
        xo += fb * 3 * count;
        p += fb * 3 * count;
        gx += fb * n3;
        if (!FD) {
            gy += fb * n3;
            gz += fb * n3;
        }
        rho += fb * n3;
    }
    const float drift_ticks = (float)(drift * (scale_arr ? scale_arr[blockIdx.y] : scale0));
    const int ntz = np / D::TZ, nty = np / D::TY;
    const int bz = blockIdx.x % ntz, by = (blockIdx.x / ntz) % nty, bx = blockIdx.x / (ntz * nty);
    const int ox = bx * D::TX * R - D::H, oy = by * D::TY * R - D::H, oz = bz * D::TZ * R - D::HZ;
    tile_zero<D>(tile_words);
    __syncthreads();
    auto pid = [&](int e) -> int64_t {
        const int lz = e % D::TZ, ly = (e / D::TZ) % D::TY, lx = e / (D::TZ * D::TY);
        return ((((int64_t)(bx * D::TX + lx) << lognp) + by * D::TY + ly) << lognp) + bz * D::TZ + lz;
    };
    // the next particle is loaded one iteration ahead (its latency overlaps this one's work)
    int64_t idn = pid(threadIdx.x);
    uint32_t nu0 = x[idn], nu1 = x[count + idn], nu2 = x[2 * count + idn];
    float np0 = p[idn], np1 = p[count + idn], np2 = p[2 * count + idn];
#pragma unroll 1
    for (int e = threadIdx.x; e < D::PER; e += 512) {
        const int64_t id = idn;
        uint32_t u0 = nu0, u1 = nu1, u2 = nu2;
        float p0 = np0, p1 = np1, p2 = np2;
        if (e + 512 < D::PER) {
            idn = pid(e + 512);
            nu0 = x[idn];
            nu1 = x[count + idn];
            nu2 = x[2 * count + idn];
            np0 = p[idn];
            np1 = p[count + idn];
            np2 = p[2 * count + idn];
        }
        ikd_particle<FD>(u0, u1, u2, p0, p1, p2, logn, inv_cell_ticks, gx, gy, gz, kick, drift_ticks, inv_d);
        p[id] = p0;
        p[count + id] = p1;
        p[2 * count + id] = p2;
        xo[id] = u0;
        xo[count + id] = u1;
        xo[2 * count + id] = u2;
        tile_deposit<D>(lo, carry, rho, u0, u1, u2, logn, inv_cell_ticks, ox, oy, oz, mass);
    }
    __syncthreads();
    tile_flush<D>(lo, carry, rho, ox, oy, oz, logn);
}

// x and xo may be the same array (in-place update): every particle's position is read once,
// one iteration before its own thread writes it, and no thread touches another's particles.
// R = 1: each thread walks its lattice row along x (lx = 0..15 at fixed ly, lz), so the
// next particle usually sits one cell further in x with the same y and z cells.  Then
// its lower-x CIC corners are this particle's upper-x corners: the gather keeps the 12
// upper-plane force values in registers and loads only the new plane, and the deposit
// carries the upper-plane weights in registers, adds them to the next particle's
// lower-plane weights and issues 4 tile atomics a particle instead of 8.  Any other
// particle takes the full path, so the result is the same CIC gather and deposit.
template <bool FD>
__global__ void __launch_bounds__(512, 2) k_ikd_deposit_sweep(const uint32_t* __restrict__ x, uint32_t* __restrict__ xo, float* __restrict__ p,
                                                              int lognp, int logn, float inv_cell_ticks,
                                                              const float* __restrict__ gx,
                                                              const float* __restrict__ gy,
                                                              const float* __restrict__ gz, float kick, double drift,
                                                              double scale0, const double* __restrict__ scale_arr,
                                                              float mass, float* __restrict__ rho, float inv_d) {
    typedef DepTile<1> D;
    static_assert(D::TY * D::TZ == 512, "one thread per (ly, lz); lx runs over the loop");
    extern __shared__ __align__(16) uint32_t tile_words[];  // D::WORDS
    uint32_t* lo = tile_words;
    uint32_t* carry = tile_words + D::CELLS;
    const int np = 1 << lognp, nm = (1 << logn) - 1;
    const int64_t count = (int64_t)1 << (3 * lognp);
    {
        const int64_t fb = blockIdx.y;
        const int64_t n3 = (int64_t)1 << (3 * logn);
        x += fb * 3 * count;
        xo += fb * 3 * count;
        p += fb * 3 * count;
        gx += fb * n3;
        if (!FD) {
            gy += fb * n3;
            gz += fb * n3;
        }
        rho += fb * n3;
    }
    const float drift_ticks = (float)(drift * (scale_arr ? scale_arr[blockIdx.y] : scale0));
    const int ntz = np / D::TZ, nty = np / D::TY;
    const int bz = blockIdx.x % ntz, by = (blockIdx.x / ntz) % nty, bx = blockIdx.x / (ntz * nty);
    const int ox = bx * D::TX - D::H, oy = by * D::TY - D::H, oz = bz * D::TZ - D::HZ;
    tile_zero<D>(tile_words);
    __syncthreads();
    const int lz = threadIdx.x % D::TZ, ly = threadIdx.x / D::TZ;
    const int64_t id0 = ((((int64_t)(bx * D::TX) << lognp) + by * D::TY + ly) << lognp) + bz * D::TZ + lz;
    const int64_t xstride = (int64_t)1 << (2 * lognp);
    uint32_t next_cell = 0xffffffffu;  // packed (ix, iy, iz) whose lower plane the registers hold
    float U[4][FD ? 1 : 3];             // force (FD: potential) at the carried plane, corner (b, c) = 2 b + c
    SweepCarry sc;                      // deposit weights carried to the next particle's plane
    // the next particle's position and momentum are loaded one iteration ahead, so their
    // memory latency overlaps the current particle's gather, update and deposit
    uint32_t nu0 = x[id0], nu1 = x[count + id0], nu2 = x[2 * count + id0];
    float np0 = p[id0], np1 = p[count + id0], np2 = p[2 * count + id0];
#pragma unroll 1
    for (int lx = 0; lx < D::TX; ++lx) {
        const int64_t id = id0 + lx * xstride;
        uint32_t u0 = nu0, u1 = nu1, u2 = nu2;
        float p0 = np0, p1 = np1, p2 = np2;
        if (lx + 1 < D::TX) {
            const int64_t idn = id + xstride;
            nu0 = x[idn];
            nu1 = x[count + idn];
            nu2 = x[2 * count + idn];
            np0 = p[idn];
            np1 = p[count + idn];
            np2 = p[2 * count + idn];
        }
        // ---- gather at the old position
        {
            const CicF cx = cic_ticks(u0, logn, inv_cell_ticks);
            const CicF cy = cic_ticks(u1, logn, inv_cell_ticks);
            const CicF cz = cic_ticks(u2, logn, inv_cell_ticks);
            const uint32_t cell = ((((uint32_t)cx.i0 << logn) | (uint32_t)cy.i0) << logn) | (uint32_t)cz.i0;
            const uint32_t iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1}, iz[2] = {(uint32_t)cz.i0, (uint32_t)cz.i1};
            constexpr int NC = FD ? 1 : 3;
            const float* g3[3] = {gx, gy, gz};
            float L[4][NC];
            if (cell == next_cell) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
#pragma unroll
                    for (int j = 0; j < NC; ++j) L[q][j] = U[q][j];
            } else {
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const uint32_t o = ((((uint32_t)cx.i0 << logn) + iy[b]) << logn) + iz[c];
#pragma unroll
                        for (int j = 0; j < NC; ++j) L[2 * b + c][j] = __ldg(g3[j] + o);
                    }
            }
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) {
                    const uint32_t o = ((((uint32_t)cx.i1 << logn) + iy[b]) << logn) + iz[c];
#pragma unroll
                    for (int j = 0; j < NC; ++j) U[2 * b + c][j] = __ldg(g3[j] + o);
                }
            next_cell = ((((uint32_t)cx.i1 << logn) | (uint32_t)cy.i0) << logn) | (uint32_t)cz.i0;
            const float wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
            const float wx0 = 1.0f - cx.w1, wx1 = cx.w1;
            float f0 = 0.f, f1 = 0.f, f2 = 0.f;
            if constexpr (FD) {
                const float Lp[4] = {L[0][0], L[1][0], L[2][0], L[3][0]};
                const float Up[4] = {U[0][0], U[1][0], U[2][0], U[3][0]};
                fd1_force<float>(Lp, Up, wx0, wx1, wy, wz, inv_d, f0, f1, f2);
            } else {
#pragma unroll
                for (int b = 0; b < 2; ++b)
#pragma unroll
                    for (int c = 0; c < 2; ++c) {
                        const float w = wy[b] * wz[c];
                        const int q = 2 * b + c;
                        f0 = fmaf(w, fmaf(wx0, L[q][0], wx1 * U[q][0]), f0);
                        f1 = fmaf(w, fmaf(wx0, L[q][1], wx1 * U[q][1]), f1);
                        f2 = fmaf(w, fmaf(wx0, L[q][2], wx1 * U[q][2]), f2);
                    }
            }
            p0 = fmaf(kick, f0, p0);
            p1 = fmaf(kick, f1, p1);
            p2 = fmaf(kick, f2, p2);
            u0 += (uint32_t)__float2int_rn(p0 * drift_ticks);
            u1 += (uint32_t)__float2int_rn(p1 * drift_ticks);
            u2 += (uint32_t)__float2int_rn(p2 * drift_ticks);
        }
        p[id] = p0;
        p[count + id] = p1;
        p[2 * count + id] = p2;
        xo[id] = u0;
        xo[count + id] = u1;
        xo[2 * count + id] = u2;
        // ---- deposit at the new position
        sweep_deposit<D>(lo, carry, rho, u0, u1, u2, logn, inv_cell_ticks, ox, oy, oz, mass, sc);
    }
    sweep_finish<D>(lo, carry, sc);
    __syncthreads();
    tile_flush<D>(lo, carry, rho, ox, oy, oz, logn);
}

template <int R, bool FD>
static cudaError_t ikd_deposit_r(void* x, void* p, int np, int n, void* const* g, double kick, double drift,
                                 double box, double mass, void* rho, cudaStream_t st, int nfields,
                                 const double* scale_arr, void* x_out, double inv_d) {
    typedef DepTile<R> D;
    const int lognp = ilog2(np), logn = ilog2(n);
    const unsigned blocks = (unsigned)((np / D::TX) * (np / D::TY) * (np / D::TZ));
    const float inv = (float)ldexp(1.0, -(32 - logn));
    const size_t smem = sizeof(uint32_t) * D::WORDS;
    if constexpr (R == 1) {
        cudaError_t e = set_smem_once((const void*)k_ikd_deposit_sweep<FD>, smem);
        if (e != cudaSuccess) return e;
        k_ikd_deposit_sweep<FD><<<dim3(blocks, nfields), 512, smem, st>>>(
            (const uint32_t*)x, (uint32_t*)(x_out ? x_out : x), (float*)p, lognp, logn, inv, (const float*)g[0],
            (const float*)g[1], (const float*)g[2],
            (float)kick, drift, 4294967296.0 / box, scale_arr, (float)mass, (float*)rho, (float)inv_d);
    } else {
        cudaError_t e = set_smem_once((const void*)k_ikd_deposit<R, FD>, smem);
        if (e != cudaSuccess) return e;
        k_ikd_deposit<R, FD><<<dim3(blocks, nfields), 512, smem, st>>>(
            (const uint32_t*)x, (uint32_t*)(x_out ? x_out : x), (float*)p, lognp, logn, inv, (const float*)g[0],
            (const float*)g[1], (const float*)g[2],
            (float)kick, drift, 4294967296.0 / box, scale_arr, (float)mass, (float*)rho, (float)inv_d);
    }
    return cudaGetLastError();
}

bool ikd_deposit_supported(int np, int precision, int n) {
    const int R = n / np;
    return precision == PM_FP32_FIXED && n >= 64 && (R == 1 || R == 2 || R == 4) && np >= 32 / R;
}

template <bool FD>
static cudaError_t ikd_deposit_any(void* x, void* p, int np, int n, void* const* g, double kick, double drift,
                                   double box, double mass, void* rho, cudaStream_t st, int nfields,
                                   const double* scale_arr, void* x_out, double inv_d) {
    const int R = n / np;
    if (R == 1)
        return ikd_deposit_r<1, FD>(x, p, np, n, g, kick, drift, box, mass, rho, st, nfields, scale_arr, x_out, inv_d);
    if (R == 2)
        return ikd_deposit_r<2, FD>(x, p, np, n, g, kick, drift, box, mass, rho, st, nfields, scale_arr, x_out, inv_d);
    return ikd_deposit_r<4, FD>(x, p, np, n, g, kick, drift, box, mass, rho, st, nfields, scale_arr, x_out, inv_d);
}

cudaError_t interp_kick_drift_deposit(void* x, void* p, int np, int precision, int n, void* const* g, double kick,
                                      double drift, double box, double mass, void* rho, cudaStream_t st, int nfields,
                                      const double* scale_arr, void* x_out, double fd_inv_d) {
    if (!ikd_deposit_supported(np, precision, n) || nfields < 1 || (uintptr_t)rho % 16 != 0)
        return cudaErrorInvalidValue;
    if (fd_inv_d > 0.0)
        return ikd_deposit_any<true>(x, p, np, n, g, kick, drift, box, mass, rho, st, nfields, scale_arr, x_out,
                                     fd_inv_d);
    return ikd_deposit_any<false>(x, p, np, n, g, kick, drift, box, mass, rho, st, nfields, scale_arr, x_out, 0.0);
}

}  // namespace pm
