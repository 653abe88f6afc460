// Common device-side types and helpers for the sm_103a particle-mesh library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/pm.h"

namespace pm {

// ------------------------------------------------------------------ type traits
template <typename T> struct CT;
template <> struct CT<float> { typedef float2 type; };
template <> struct CT<double> { typedef double2 type; };

template <typename T> using cplx = typename CT<T>::type;

template <typename C> __host__ __device__ __forceinline__ C cmake(decltype(C().x) a, decltype(C().x) b) {
    C c; c.x = a; c.y = b; return c;
}
template <typename C> __device__ __forceinline__ C cadd(C a, C b) { a.x += b.x; a.y += b.y; return a; }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { a.x -= b.x; a.y -= b.y; return a; }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
    C c; c.x = a.x * b.x - a.y * b.y; c.y = a.x * b.y + a.y * b.x; return c;
}
template <typename C> __device__ __forceinline__ C cconj(C a) { a.y = -a.y; return a; }
template <typename C, typename T> __device__ __forceinline__ C cscale(C a, T s) { a.x *= s; a.y *= s; return a; }
// multiply by -i (forward) or +i (inverse)
template <bool INV, typename C> __device__ __forceinline__ C cmul_mi(C a) {
    C c;
    if (INV) { c.x = -a.y; c.y = a.x; } else { c.x = a.y; c.y = -a.x; }
    return c;
}

// ------------------------------------------------------------------ constants
constexpr int kMaxLogN = 10;  // meshes up to 1024^3 in index arithmetic

__host__ __device__ __forceinline__ int ilog2(int n) {
    int l = 0;
    while ((1 << l) < n) ++l;
    return l;
}

// Padded shared-memory index: one spare slot every 8 complex elements keeps the
// strided Stockham stores free of shared-memory bank conflicts.
__host__ __device__ __forceinline__ int spad(int i) { return i + (i >> 3); }

// Signed wavenumber of FFT index i on an n-point axis: 0..n/2-1, -n/2..-1.
__device__ __forceinline__ int signed_k(int i, int n) { return i < (n >> 1) ? i : i - n; }

}  // namespace pm
