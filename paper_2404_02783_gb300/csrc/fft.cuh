// In-shared-memory FFT building blocks (Stockham autosort, radix 8/4/2).
//
// A CTA transforms a tile of independent length-L sequences held in shared
// memory.  Each sequence ("row" b) is served by L/8 threads; thread t of row b
// performs 8/R radix-R butterflies per stage, so every stage is one
// load -> twiddle -> register DFT -> barrier -> store -> barrier round, in
// place.  Stockham ordering reads element j + r L/R and writes element
// (j / Ns) Ns R + (j mod Ns) + r Ns, leaving the result in natural order
// after the last stage without a bit-reversal pass.
//
// Twiddles come from a shared table tw[k] = exp(-2 pi i k / Ltab) built on the
// host in FP64; a length-L transform uses stride Ltab / L.  INV selects the
// conjugate (inverse, unnormalised) transform.
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
    // even / odd split: E = DFT4(v0 v2 v4 v6), O = DFT4(v1 v3 v5 v7)
    dft4<INV>(v[0], v[2], v[4], v[6]);
    dft4<INV>(v[1], v[3], v[5], v[7]);
    C o1 = mul_w8_1<INV>(v[3]);
    C o2 = cmul_mi<INV>(v[5]);
    C o3 = mul_w8_3<INV>(v[7]);
    C e0 = v[0], e1 = v[2], e2 = v[4], e3 = v[6], o0 = v[1];
    v[0] = cadd(e0, o0); v[4] = csub(e0, o0);
    v[1] = cadd(e1, o1); v[5] = csub(e1, o1);
    v[2] = cadd(e2, o2); v[6] = csub(e2, o2);
    v[3] = cadd(e3, o3); v[7] = csub(e3, o3);
}

// ---------------------------------------------------------------- addressing
// Row tile: row b occupies [b * stride, b * stride + spad(L)).
struct RowAddr {
    int stride;
    __device__ __forceinline__ int operator()(int b, int i) const { return b * stride + spad(i); }
};
// Column tile: element i of column b sits at i * stride + b (columns interleaved).
struct ColAddr {
    int stride;
    __device__ __forceinline__ int operator()(int b, int i) const { return i * stride + b; }
};

template <bool INV, typename C>
__device__ __forceinline__ C twiddle(const C* tw, int e) {
    C w = tw[e];
    if (INV) w.y = -w.y;
    return w;
}

// One Stockham stage of radix R for the thread's butterflies.
template <int R, bool INV, typename C, class Addr>
__device__ __forceinline__ void stockham_stage(C* s, int L, int Ns, int t, int b, bool active,
                                               const C* tw, int tw_stride, Addr addr) {
    constexpr int NB = 8 / R;  // butterflies per thread
    C v[8];
    const int quarter = L >> 3;  // threads per row
    const int LR = L / R;
    if (active) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int j = t + q * quarter;
            const int jm = j % Ns;
            const int tstep = jm * (L / (Ns * R)) * tw_stride;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                C a = s[addr(b, j + r * LR)];
                if (r > 0) a = cmul(a, twiddle<INV>(tw, r * tstep));
                v[q * R + r] = a;
            }
            if (R == 8) dft8<INV>(v);
            if (R == 4) dft4<INV>(v[q * 4 + 0], v[q * 4 + 1], v[q * 4 + 2], v[q * 4 + 3]);
            if (R == 2) dft2<INV>(v[q * 2 + 0], v[q * 2 + 1]);
        }
    }
    __syncthreads();
    if (active) {
#pragma unroll
        for (int q = 0; q < NB; ++q) {
            const int j = t + q * quarter;
            const int jm = j % Ns;
            const int base = (j / Ns) * Ns * R + jm;
#pragma unroll
            for (int r = 0; r < R; ++r) s[addr(b, base + r * Ns)] = v[q * R + r];
        }
    }
    __syncthreads();
}

// Full length-L transform (L a power of two, 8 <= L <= 4096) of every row in the
// tile; all threads of the CTA must call it (it contains barriers).
template <bool INV, typename C, class Addr>
__device__ void fft_tile(C* s, int L, int t, int b, bool active, const C* tw, int tw_stride, Addr addr) {
    int Ns = 1;
    while (Ns < L) {
        const int rem = L / Ns;
        if (rem >= 8) {
            stockham_stage<8, INV>(s, L, Ns, t, b, active, tw, tw_stride, addr);
            Ns *= 8;
        } else if (rem == 4) {
            stockham_stage<4, INV>(s, L, Ns, t, b, active, tw, tw_stride, addr);
            Ns *= 4;
        } else {
            stockham_stage<2, INV>(s, L, Ns, t, b, active, tw, tw_stride, addr);
            Ns *= 2;
        }
    }
}

}  // namespace pm
