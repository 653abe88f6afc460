// Device pieces of the particle update shared by particles.cu and update.cu: the CIC
// decode of uint32 tick positions, the per-particle gather + kick + drift, and the
// fixed-point deposit tile of a Lagrangian block of particles.
#pragma once

#include <stdint.h>

#include "pm_common.cuh"

namespace pm {

// ---------------------------------------------------------------- CIC decode
struct CicF {
    int i0, i1;
    float w1;
};
__device__ __forceinline__ CicF cic_ticks(uint32_t u, int logn, float inv_cell_ticks) {
    const int sh = 32 - logn;
    const uint32_t t = u - (1u << (sh - 1));
    CicF c;
    c.i0 = (int)(t >> sh);
    c.i1 = (c.i0 + 1) & ((1 << logn) - 1);
    c.w1 = __uint2float_rn(t & ((1u << sh) - 1u)) * inv_cell_ticks;
    return c;
}
// Deposit of lattice-ordered particles (count = np^3, id = (ix np + iy) np + iz) by
// Lagrangian tiles.  A CTA owns a TX x TY x TZ block of lattice sites (16 x 16 x 32
// mesh cells' worth, R = n / np cells per lattice step); particles that have not
// travelled far land in that mesh box widened by H cells on every side, which the CTA
// accumulates in shared memory and then adds to the global mesh once per cell.  A
// particle whose CIC stencil leaves the box adds its weights to global memory directly,
// so the result is the same CIC density for any displacement.
//
// The tile accumulates in fixed point: each weight is rounded to a multiple of 2^-24
// (half a quantum at most, 3e-8, below the FP32 rounding of a sum near 1) and added
// with a native 32-bit integer atomic (shared-memory float atomics are a compare-and-
// swap loop on this part).  A wrap of the 32-bit word is seen in the atomic's return
// value and counted in an 8-bit carry per cell.  A tile holds at most 8192 mass units
// (TX TY TZ R^3 = 8192 for every R), i.e. 2^37 quanta, so a cell's carry stays below 32
// and the tile sum is exact and independent of the order of the additions.
// The box starts HZ = 4 cells below the tile in z so that its rows are made of 16-byte
// chunks aligned in the mesh: the flush adds four cells per vector reduction.
template <int R>
struct DepTile {
    static constexpr int TX = 16 / R, TY = 16 / R, TZ = 32 / R, H = 2, HZ = 4;
    static constexpr int DX = TX * R + 2 * H, DY = TY * R + 2 * H, DZ = TZ * R + 2 * HZ;
    static constexpr int CELLS = DX * DY * DZ, CHUNKS = CELLS / 4;
    static constexpr int CARRY_WORDS = CHUNKS;  // one word of four 8-bit carries per chunk
    static constexpr int WORDS = CELLS + CARRY_WORDS;  // shared memory: lo[CELLS], carry[CARRY_WORDS]
    static constexpr int PER = TX * TY * TZ;
    static_assert(PER * R * R * R == 8192, "tile mass bound");
    static_assert(DZ % 4 == 0 && (TZ * R) % 4 == 0 && HZ % 4 == 0, "z box made of aligned 16-byte chunks");
};

__device__ __forceinline__ void red_add_v4(float* dst, float4 v) {
    asm volatile("red.relaxed.gpu.global.add.v4.f32 [%0], {%1, %2, %3, %4};\n" ::"l"(dst), "f"(v.x), "f"(v.y),
                 "f"(v.z), "f"(v.w)
                 : "memory");
}

constexpr float kTileQuanta = 16777216.0f;  // 2^24 quanta per unit mass
constexpr float kTileQuantum = 5.9604644775390625e-08f;  // 2^-24

__device__ __forceinline__ void tile_add(uint32_t* lo, uint32_t* carry, int c, float w) {
    const uint32_t v = __float2uint_rn(w * kTileQuanta);
    const uint32_t old = atomicAdd(lo + c, v);
    if (old + v < old) atomicAdd(carry + (c >> 2), 1u << (8 * (c & 3)));
}

template <class D>
__device__ __forceinline__ void tile_zero(uint32_t* words) {
    for (int c = threadIdx.x; c < D::WORDS; c += blockDim.x) words[c] = 0u;
}

// One particle's CIC weights into the tile (box origin o*) or, outside it, into rho.
template <class D>
__device__ __forceinline__ void tile_deposit(uint32_t* lo, uint32_t* carry, float* __restrict__ rho, uint32_t u0,
                                             uint32_t u1, uint32_t u2, int logn, float inv_cell_ticks, int ox,
                                             int oy, int oz, float mass) {
    const int nm = (1 << logn) - 1;
    const CicF cx = cic_ticks(u0, logn, inv_cell_ticks);
    const CicF cy = cic_ticks(u1, logn, inv_cell_ticks);
    const CicF cz = cic_ticks(u2, logn, inv_cell_ticks);
    const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
    const int dx = (cx.i0 - ox) & nm, dy = (cy.i0 - oy) & nm, dz = (cz.i0 - oz) & nm;
    if (dx < D::DX - 1 && dy < D::DY - 1 && dz < D::DZ - 1) {
        const int c0 = (dx * D::DY + dy) * D::DZ + dz;
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float wab = mass * wx[a] * wy[b];
                const int c = c0 + (a * D::DY + b) * D::DZ;
                tile_add(lo, carry, c, wab * wz[0]);
                tile_add(lo, carry, c + 1, wab * wz[1]);
            }
    } else {
        const uint32_t ix[2] = {(uint32_t)cx.i0, (uint32_t)cx.i1}, iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const float wab = mass * wx[a] * wy[b];
                float* row = rho + (((ix[a] << logn) + iy[b]) << logn);
                atomicAdd(row + cz.i0, wab * wz[0]);
                atomicAdd(row + cz.i1, wab * wz[1]);
            }
    }
}

// Adds the tile's cells (box origin o*, oz a multiple of 4, rho 16-byte aligned) to rho,
// four z-cells per reduction.
template <class D>
__device__ __forceinline__ void tile_flush(const uint32_t* lo, const uint32_t* carry, float* __restrict__ rho, int ox,
                                           int oy, int oz, int logn) {
    const int nm = (1 << logn) - 1;
    for (int c = threadIdx.x; c < D::CHUNKS; c += blockDim.x) {
        const uint4 l = reinterpret_cast<const uint4*>(lo)[c];
        const uint32_t h = carry[c];
        if (l.x | l.y | l.z | l.w | h) {
            const int lz4 = c % (D::DZ / 4), ly = (c / (D::DZ / 4)) % D::DY, lx = c / ((D::DZ / 4) * D::DY);
            const float4 v = make_float4(__uint2float_rn(l.x) * kTileQuantum + (float)(h & 255u) * 256.0f,
                                         __uint2float_rn(l.y) * kTileQuantum + (float)((h >> 8) & 255u) * 256.0f,
                                         __uint2float_rn(l.z) * kTileQuantum + (float)((h >> 16) & 255u) * 256.0f,
                                         __uint2float_rn(l.w) * kTileQuantum + (float)(h >> 24) * 256.0f);
            red_add_v4(rho + ((((uint32_t)((ox + lx) & nm) << logn) + (uint32_t)((oy + ly) & nm)) << logn) +
                           ((oz + 4 * lz4) & nm),
                       v);
        }
    }
}

// Deposit of a thread walking its lattice row along x (R = 1).  The next particle usually
// sits one cell further in x with the same y and z cells; its lower-x CIC corners are then
// this particle's upper-x corners, so the upper-plane weights are carried (W, for the cell
// dnext) and added with the next particle's lower plane: 4 tile atomics a particle instead
// of 8.  A particle whose stencil leaves the box adds to rho directly.
struct SweepCarry {
    int dnext = -1;  // tile cell of the carried plane's (b, c) = (0, 0) corner, -1: none
    float W[4];      // carried weights, corner (b, c) = 2 b + c
};

template <class D>
__device__ __forceinline__ void sweep_deposit(uint32_t* lo, uint32_t* carry, float* __restrict__ rho, uint32_t u0,
                                              uint32_t u1, uint32_t u2, int logn, float inv_cell_ticks, int ox,
                                              int oy, int oz, float mass, SweepCarry& sc) {
    const int nm = (1 << logn) - 1;
    const CicF cx = cic_ticks(u0, logn, inv_cell_ticks);
    const CicF cy = cic_ticks(u1, logn, inv_cell_ticks);
    const CicF cz = cic_ticks(u2, logn, inv_cell_ticks);
    const float wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
    const float m0 = mass * (1.0f - cx.w1), m1 = mass * cx.w1;
    const int dx = (cx.i0 - ox) & nm, dy = (cy.i0 - oy) & nm, dz = (cz.i0 - oz) & nm;
    if (dx < D::DX - 1 && dy < D::DY - 1 && dz < D::DZ - 1) {
        const int c0 = (dx * D::DY + dy) * D::DZ + dz;
        float w0[4];
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) w0[2 * b + c] = m0 * wy[b] * wz[c];
        if (c0 == sc.dnext) {
#pragma unroll
            for (int q = 0; q < 4; ++q) w0[q] += sc.W[q];
        } else if (sc.dnext >= 0) {
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) tile_add(lo, carry, sc.dnext + b * D::DZ + c, sc.W[2 * b + c]);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                tile_add(lo, carry, c0 + b * D::DZ + c, w0[2 * b + c]);
                sc.W[2 * b + c] = m1 * wy[b] * wz[c];
            }
        sc.dnext = c0 + D::DY * D::DZ;
    } else {
        if (sc.dnext >= 0) {
#pragma unroll
            for (int b = 0; b < 2; ++b)
#pragma unroll
                for (int c = 0; c < 2; ++c) tile_add(lo, carry, sc.dnext + b * D::DZ + c, sc.W[2 * b + c]);
        }
        sc.dnext = -1;
        const uint32_t ix[2] = {(uint32_t)cx.i0, (uint32_t)cx.i1}, iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1};
        const float mx[2] = {m0, m1};
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                float* row = rho + (((ix[a] << logn) + iy[b]) << logn);
                atomicAdd(row + cz.i0, mx[a] * wy[b] * wz[0]);
                atomicAdd(row + cz.i1, mx[a] * wy[b] * wz[1]);
            }
    }
}

// The carried plane of the row's last particle.
template <class D>
__device__ __forceinline__ void sweep_finish(uint32_t* lo, uint32_t* carry, const SweepCarry& sc) {
    if (sc.dnext >= 0) {
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
            for (int c = 0; c < 2; ++c) tile_add(lo, carry, sc.dnext + b * D::DZ + c, sc.W[2 * b + c]);
    }
}

// ---------------------------------------------------------------- interp + kick + drift
// First-order gradient (PM_GRAD_FD1): the force -grad of the CIC interpolant of the
// potential inside the particle's cell, from its eight corners: L[q] on the lower x plane,
// U[q] on the upper one, corner (b, c) = 2 b + c for (y, z); inv_d = nmesh / L.
//   g_x = inv_d sum_bc wy_b wz_c (L - U)
//   g_y = inv_d sum_c wz_c [wx0 (L_0c - L_1c) + wx1 (U_0c - U_1c)]
//   g_z = inv_d sum_b wy_b [wx0 (L_b0 - L_b1) + wx1 (U_b0 - U_b1)]
template <typename T>
__device__ __forceinline__ void fd1_force(const T* L, const T* U, T wx0, T wx1, const T* wy, const T* wz, T inv_d,
                                          T& f0, T& f1, T& f2) {
    T gx = T(0), gy = T(0), gz = T(0);
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) gx += wy[b] * wz[c] * (L[2 * b + c] - U[2 * b + c]);
#pragma unroll
    for (int c = 0; c < 2; ++c) gy += wz[c] * (wx0 * (L[c] - L[2 + c]) + wx1 * (U[c] - U[2 + c]));
#pragma unroll
    for (int b = 0; b < 2; ++b) gz += wy[b] * (wx0 * (L[2 * b] - L[2 * b + 1]) + wx1 * (U[2 * b] - U[2 * b + 1]));
    f0 = inv_d * gx;
    f1 = inv_d * gy;
    f2 = inv_d * gz;
}

// p += kick * g(x);  x += drift * p   (g = -grad phi gathered with the deposit's weights).
// The eight corner offsets are formed once in 32 bits (n^3 <= 2^30) and serve the
// three force meshes.  FD: gx is the potential and g its first-order gradient (fd1_force).
template <bool FD>
__device__ __forceinline__ void ikd_particle(uint32_t& u0, uint32_t& u1, uint32_t& u2, float& p0, float& p1,
                                             float& p2, int logn, float inv_cell_ticks, const float* __restrict__ gx,
                                             const float* __restrict__ gy, const float* __restrict__ gz, float kick,
                                             float drift_ticks, float inv_d) {
    const CicF cx = cic_ticks(u0, logn, inv_cell_ticks);
    const CicF cy = cic_ticks(u1, logn, inv_cell_ticks);
    const CicF cz = cic_ticks(u2, logn, inv_cell_ticks);
    const float wx[2] = {1.0f - cx.w1, cx.w1}, wy[2] = {1.0f - cy.w1, cy.w1}, wz[2] = {1.0f - cz.w1, cz.w1};
    const uint32_t ix[2] = {(uint32_t)cx.i0, (uint32_t)cx.i1}, iy[2] = {(uint32_t)cy.i0, (uint32_t)cy.i1};
    float f0 = 0.f, f1 = 0.f, f2 = 0.f;
    if constexpr (FD) {
        float P[2][4];
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const uint32_t row = ((ix[a] << logn) + iy[b]) << logn;
                P[a][2 * b] = __ldg(gx + row + (uint32_t)cz.i0);
                P[a][2 * b + 1] = __ldg(gx + row + (uint32_t)cz.i1);
            }
        fd1_force<float>(P[0], P[1], wx[0], wx[1], wy, wz, inv_d, f0, f1, f2);
    } else {
#pragma unroll
        for (int a = 0; a < 2; ++a)
#pragma unroll
            for (int b = 0; b < 2; ++b) {
                const uint32_t row = ((ix[a] << logn) + iy[b]) << logn;
                const uint32_t o0 = row + (uint32_t)cz.i0, o1 = row + (uint32_t)cz.i1;
                const float w0 = wx[a] * wy[b] * wz[0], w1 = wx[a] * wy[b] * wz[1];
                f0 = fmaf(w0, __ldg(gx + o0), fmaf(w1, __ldg(gx + o1), f0));
                f1 = fmaf(w0, __ldg(gy + o0), fmaf(w1, __ldg(gy + o1), f1));
                f2 = fmaf(w0, __ldg(gz + o0), fmaf(w1, __ldg(gz + o1), f2));
            }
    }
    p0 = fmaf(kick, f0, p0);
    p1 = fmaf(kick, f1, p1);
    p2 = fmaf(kick, f2, p2);
    // 32-bit conversion (the 64-bit one is several times slower here): exact for drifts under
    // half the box per step, i.e. |p drift_ticks| < 2^31, the range of any meaningful step
    u0 += (uint32_t)__float2int_rn(p0 * drift_ticks);
    u1 += (uint32_t)__float2int_rn(p1 * drift_ticks);
    u2 += (uint32_t)__float2int_rn(p2 * drift_ticks);
}

}  // namespace pm
