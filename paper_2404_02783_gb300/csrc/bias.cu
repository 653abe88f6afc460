// Halo proxy for the linear-bias measurement (Sec. 5.2, Eq. b1): the ceil(f n^3)
// densest cells of a density mesh, ties broken by the lower linear index, turned into
// a tracer contrast delta_h = n_h / mean(n_h) - 1.
//
// Selection is exact: values map to order-preserving unsigned keys (sign-flip of the
// IEEE bits), a radix select finds the threshold key byte by byte from the top
// (256-bin histograms of the cells that still match the chosen prefix), and cells
// equal to the threshold are ranked by index with an exclusive scan so that exactly
// the lowest-index ones fill the remaining places.
#include <vector>

#include "internal.h"
#include "particles.h"

namespace pm {

template <typename T> struct KeyOf;
template <> struct KeyOf<float> {
    typedef uint32_t K;
    static constexpr int BITS = 32;
    __device__ __forceinline__ static K key(float f) {
        const uint32_t u = __float_as_uint(f);
        return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
    }
};
template <> struct KeyOf<double> {
    typedef unsigned long long K;
    static constexpr int BITS = 64;
    __device__ __forceinline__ static K key(double f) {
        const unsigned long long u = (unsigned long long)__double_as_longlong(f);
        return (u & 0x8000000000000000ull) ? ~u : (u | 0x8000000000000000ull);
    }
};

template <typename T>
__global__ void k_radix_hist(const T* __restrict__ f, int64_t count, unsigned long long prefix,
                             unsigned long long pmask, int shift, unsigned long long* __restrict__ hist) {
    __shared__ unsigned int h[256];
    for (int i = threadIdx.x; i < 256; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = (unsigned long long)KeyOf<T>::key(f[i]);
        if ((k & pmask) == prefix) atomicAdd(&h[(k >> shift) & 0xFF], 1u);
    }
    __syncthreads();
    for (int i = threadIdx.x; i < 256; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

template <typename T>
__global__ void k_eq_flags(const T* __restrict__ f, int64_t count, unsigned long long thr, uint32_t* __restrict__ flags) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        flags[i] = ((unsigned long long)KeyOf<T>::key(f[i]) == thr) ? 1u : 0u;
}

// delta_h = 1[selected] n^3/K - 1
template <typename T>
__global__ void k_select(const T* __restrict__ f, int64_t count, unsigned long long thr, const uint32_t* __restrict__ eq_rank,
                         uint32_t eq_needed, T scale, T* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const unsigned long long k = (unsigned long long)KeyOf<T>::key(f[i]);
        const bool sel = k > thr || (k == thr && eq_rank[i] < eq_needed);
        out[i] = sel ? scale - T(1) : T(-1);
    }
}

static unsigned blocks_for(int64_t count) {
    int64_t b = (count + 255) / 256;
    if (b > 152 * 16) b = 152 * 16;
    return (unsigned)(b < 1 ? 1 : b);
}

template <typename T>
cudaError_t halo_proxy(const T* field, int64_t count, int64_t K, T* out, void* scratch, cudaStream_t st) {
    typedef typename KeyOf<T>::K Key;
    const int bits = KeyOf<T>::BITS;
    unsigned long long* hist = (unsigned long long*)scratch;
    uint32_t* flags = (uint32_t*)((char*)scratch + 256 * sizeof(unsigned long long));
    uint32_t* rank = flags + count;
    uint32_t* sc = rank + count;
    unsigned long long prefix = 0, pmask = 0;
    int64_t remaining = K;
    std::vector<unsigned long long> h(256);
    cudaError_t e;
    for (int shift = bits - 8; shift >= 0; shift -= 8) {
        e = cudaMemsetAsync(hist, 0, 256 * sizeof(unsigned long long), st);
        if (e != cudaSuccess) return e;
        k_radix_hist<T><<<blocks_for(count), 256, 0, st>>>(field, count, prefix, pmask, shift, hist);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(h.data(), hist, 256 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
        if (e != cudaSuccess) return e;
        e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        int64_t cum = 0;
        int digit = 0;
        for (int d = 255; d >= 0; --d) {
            if (cum + (int64_t)h[d] >= remaining) {
                digit = d;
                break;
            }
            cum += (int64_t)h[d];
        }
        remaining -= cum;
        prefix |= (unsigned long long)digit << shift;
        pmask |= 0xFFull << shift;
    }
    (void)sizeof(Key);
    k_eq_flags<T><<<blocks_for(count), 256, 0, st>>>(field, count, prefix, flags);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    e = scan_exclusive_u32(flags, rank, count, sc, st);
    if (e != cudaSuccess) return e;
    k_select<T><<<blocks_for(count), 256, 0, st>>>(field, count, prefix, rank, (uint32_t)remaining,
                                                   (T)((double)count / (double)K), out);
    return cudaGetLastError();
}

size_t halo_proxy_scratch_bytes(int64_t count) {
    return 256 * sizeof(unsigned long long) + sizeof(uint32_t) * (size_t)(2 * count) + scan_scratch_bytes(count);
}

template cudaError_t halo_proxy<float>(const float*, int64_t, int64_t, float*, void*, cudaStream_t);
template cudaError_t halo_proxy<double>(const double*, int64_t, int64_t, double*, void*, cudaStream_t);

}  // namespace pm
