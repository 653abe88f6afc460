// Register-resident FFT engine (Stockham autosort, radix 8 with one radix-4 or
// radix-2 closing stage), compile-time length.
//
// A length-L sequence is owned by Q = L/8 threads; thread t holds the eight
// elements t + m Q (m = 0..7) in registers.  A stage of radix R performs 8/R
// butterflies per thread: butterfly j = t + q Q reads elements j + r L/R,
// multiplies by exp(-+2 pi i (j mod Ns) r / (Ns R)) and runs a register DFT of
// size R; the result element (j / Ns) Ns R + (j mod Ns) + r Ns goes through
// shared memory to whichever thread reads it in the next stage.  Loads of stage
// one and stores after the last stage touch elements t + m Q, i.e. consecutive
// threads touch consecutive elements, so callers stream them to and from global
// memory directly.  Only the exchanges between stages use shared memory.
//
// Twiddles come from a shared per-stage table (tw_stage_offset; values from the host
// FP64 table exp(-2 pi i k / 1024), rounded once); INV conjugates them (unnormalised
// inverse).
#pragma once

#include "pm_common.cuh"

namespace pm {

// ---------------------------------------------------------------- butterflies
template <bool INV, typename C>
__device__ __forceinline__ void dft2(C& a, C& b) {
    C t = a;
    a = cadd(t, b);
    b = csub(t, b);
}

template <bool INV, typename C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
    C t0 = cadd(v0, v2), t1 = csub(v0, v2), t2 = cadd(v1, v3);
    C t3 = cmul_mi<INV>(csub(v1, v3));
    v0 = cadd(t0, t2);
    v2 = csub(t0, t2);
    v1 = cadd(t1, t3);
    v3 = csub(t1, t3);
}

// (x + iy) exp(-+ i pi/4) and (x + iy) exp(-+ 3 i pi/4)
template <bool INV, typename C>
__device__ __forceinline__ C mul_w8_1(C a) {
    typedef decltype(a.x) T;
    const T s = T(0.70710678118654752440);
    return INV ? cmake<C>((a.x - a.y) * s, (a.x + a.y) * s) : cmake<C>((a.x + a.y) * s, (a.y - a.x) * s);
}
template <bool INV, typename C>
__device__ __forceinline__ C mul_w8_3(C a) {
    typedef decltype(a.x) T;
    const T s = T(0.70710678118654752440);
    return INV ? cmake<C>((-a.x - a.y) * s, (a.x - a.y) * s) : cmake<C>((a.y - a.x) * s, (-a.x - a.y) * s);
}

template <bool INV, typename C>
__device__ __forceinline__ void dft8(C* v) {
    // even / odd split: E = DFT4(v0 v2 v4 v6), O = DFT4(v1 v3 v5 v7); X_k = E_k + w^k O_k
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    const C o1 = mul_w8_1<INV>(v[3]);
    const C o2 = cmul_mi<INV>(v[5]);
    const C o3 = mul_w8_3<INV>(v[7]);
    const C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

template <int R, bool INV, typename C>
__device__ __forceinline__ void dftR(C* v) {
    if constexpr (R == 8) dft8<INV>(v);
    else if constexpr (R == 4) dft4<INV>(v[0], v[1], v[2], v[3]);
    else if constexpr (R == 2) dft2<INV>(v[0], v[1]);
}

template <bool INV, typename C>
__device__ __forceinline__ C twid(const C* tw, int e) {
    C w = tw[e];
    if (INV) w.y = -w.y;
    return w;
}

__host__ __device__ constexpr int radix_at(int L, int Ns) { return (L / Ns) >= 8 ? 8 : (L / Ns); }
__host__ __device__ constexpr int last_radix(int L, int Ns = 1) { return (Ns * radix_at(L, Ns) >= L) ? radix_at(L, Ns) : last_radix(L, Ns * radix_at(L, Ns)); }

// Per-stage twiddle table: the stage with span Ns > 1 and radix R keeps
// w(r, jm) = exp(-2 pi i jm r / (Ns R)) at [offset(Ns) + (r - 1) Ns + jm], r = 1..R-1,
// jm = 0..Ns-1, so the lanes of a warp (consecutive jm) read consecutive entries.  The
// table of a length-L transform holds L - radix_at(L, 1) < L entries.
__host__ __device__ constexpr int tw_stage_offset(int L, int Ns, int s = 1, int off = 0) {
    return (s >= Ns) ? off : tw_stage_offset(L, Ns, s * radix_at(L, s), off + (s > 1 ? (radix_at(L, s) - 1) * s : 0));
}
__host__ __device__ constexpr int tw_stage_entries(int L) { return tw_stage_offset(L, L); }

// ---------------------------------------------------------------- exchangers
// Shared-memory rows of the exchanges: element i of a row sits at slot
// i ^ ((i >> SH) & MK) (a permutation within aligned blocks of MK + 1 elements), rows
// RS slots apart.  The parameters are chosen per transform length, and for the z passes
// (rows of n/2 + 1 elements that the r2c / c2r post-processing also walks across rows),
// by enumerating every access pattern of a warp so that the 8-byte accesses of each
// half-warp fall in distinct banks (no pattern replays for y rows of 16..1024 elements
// and z rows of 128..512; z rows of 8..64 replay less than the plain padded layout).
template <int L, bool ZPASS>
struct RowLayout {
    static constexpr int SH = ZPASS ? (L >= 128 ? 3 : L == 64 ? 2 : L == 32 ? 1 : L == 16 ? 4 : 1) : 3;
    static constexpr int MK = ZPASS ? (L >= 64 || L == 32 ? 15 : 7) : (L >= 128 ? 15 : 7);
    static constexpr int RS = ZPASS ? (L == 512 ? 514 : L >= 128 ? L + 1 : L == 64 ? 65 : L == 32 ? 35 : L == 16 ? 19 : 13)
                                    : (L >= 128 ? L + 1 : L == 64 ? 72 : L == 32 ? 44 : 22);
    __host__ __device__ static constexpr int slot(int i) { return i ^ ((i >> SH) & MK); }
};

// Rows: sequence s of row b at base[((p NSEQ + s) RB + b) RS + slot(i)]; two
// buffers alternate (p) when PP, so one barrier per exchange suffices.
template <typename C, int NSEQ, bool PP, class LAY>
struct RowEx {
    C* base;
    int RB, RS, b, p;
    __device__ __forceinline__ C& at(int s, int i) {
        return base[(((PP ? p : 0) * NSEQ + s) * RB + b) * RS + LAY::slot(i)];
    }
    __device__ __forceinline__ void begin() {
        if (!PP) __syncthreads();
    }
    __device__ __forceinline__ void end() {
        if (PP) p ^= 1;
    }
};

// Columns: element i of column b of sequence s at base[(s L + i) CS + b] (columns
// interleaved so that lanes of consecutive columns hit consecutive banks).
template <typename C, int L>
struct ColEx {
    C* base;
    int CS, b;
    __device__ __forceinline__ C& at(int s, int i) { return base[(s * L + i) * CS + b]; }
    __device__ __forceinline__ void begin() { __syncthreads(); }
    __device__ __forceinline__ void end() {}
};

// ---------------------------------------------------------------- stages
template <int L, int Ns, int NSEQ, bool INV, typename C, class X>
__device__ __forceinline__ void fft_stages(C (*v)[8], int t, const C* __restrict__ tw, X& ex) {
    constexpr int R = radix_at(L, Ns);
    constexpr int NB = 8 / R;
    constexpr int Q = L / 8;
#pragma unroll
    for (int s = 0; s < NSEQ; ++s)
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            if constexpr (Ns > 1) {
                const int jm = (t + q * Q) & (Ns - 1);
                const C* tws = tw + tw_stage_offset(L, Ns) + jm;
#pragma unroll
                for (int r = 1; r < R; ++r) v[s][q * R + r] = cmul(v[s][q * R + r], twid<INV>(tws, (r - 1) * Ns));
            }
            dftR<R, INV>(&v[s][q * R]);
        }
    if constexpr (Ns * R < L) {
        constexpr int Ns2 = Ns * R;
        constexpr int R2 = radix_at(L, Ns2);
        constexpr int NB2 = 8 / R2;
        ex.begin();
#pragma unroll
        for (int s = 0; s < NSEQ; ++s)
#pragma unroll
            for (int q = 0; q < NB; ++q) {
                const int j = t + q * Q;
                const int base = (j / Ns) * Ns2 + (j & (Ns - 1));
#pragma unroll
                for (int r = 0; r < R; ++r) ex.at(s, base + r * Ns) = v[s][q * R + r];
            }
        __syncthreads();
#pragma unroll
        for (int s = 0; s < NSEQ; ++s)
#pragma unroll
            for (int q = 0; q < NB2; ++q) {
                const int j = t + q * Q;
#pragma unroll
                for (int r = 0; r < R2; ++r) v[s][q * R2 + r] = ex.at(s, j + r * (L / R2));
            }
        ex.end();
        fft_stages<L, Ns2, NSEQ, INV>(v, t, tw, ex);
    }
}

// Transform NSEQ sequences of length L (8 <= L <= 1024, a power of two).  On entry
// v[s][m] is element t + m L/8 of sequence s; on exit v[s][m] is transform element
// t + m L/8.  Contains barriers: every thread of the CTA must call it.
template <int L, int NSEQ, bool INV, typename C, class X>
__device__ __forceinline__ void fft_regs(C (*v)[8], int t, const C* __restrict__ tw, X& ex) {
    fft_stages<L, 1, NSEQ, INV>(v, t, tw, ex);
    constexpr int RL = last_radix(L);
    if constexpr (RL < 8) {
        // after a closing radix-RL stage, slot q RL + r holds element t + (q + r 8/RL) L/8
        constexpr int NB = 8 / RL;
#pragma unroll
        for (int s = 0; s < NSEQ; ++s) {
            C w[8];
#pragma unroll
            for (int q = 0; q < NB; ++q)
#pragma unroll
                for (int r = 0; r < RL; ++r) w[q + r * NB] = v[s][q * RL + r];
#pragma unroll
            for (int m = 0; m < 8; ++m) v[s][m] = w[m];
        }
    }
}

}  // namespace pm
