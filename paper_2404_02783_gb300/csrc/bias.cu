// Halo proxy for the linear-bias measurement (Sec. 5.2, Eq. b1): the ceil(f n^3)
// densest cells of a density mesh, ties broken by the lower linear index, turned into
// a tracer contrast delta_h = n_h / mean(n_h) - 1.
//
// Selection is exact: values map to order-preserving unsigned keys (sign-flip of the
// IEEE bits), a radix select finds the threshold key byte by byte from the top
// (256-bin histograms of the cells that still match the chosen prefix), and cells
// equal to the threshold are ranked by index (per-chunk counts, their scan, and warp
// ballots within each chunk) so that exactly the lowest-index ones fill the remaining
// places.
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

// Cells equal to the threshold key are ranked by index without a full-length scan: CTA b
// owns the contiguous chunk [b chunk, (b + 1) chunk); k_eq_count counts its equal cells,
// a small scan over the CTAs gives each chunk its first rank, and k_select walks its chunk
// in index order, ranking the equal cells of each 256-cell tile with warp ballots.
template <typename T>
__global__ void __launch_bounds__(256) k_eq_count(const T* __restrict__ f, int64_t count, int64_t chunk,
                                                   unsigned long long thr, uint32_t* __restrict__ cnt) {
    __shared__ uint32_t wsum[8];
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(count, lo + chunk);
    uint32_t c = 0;
    for (int64_t i = lo + threadIdx.x; i < hi; i += blockDim.x)
        c += ((unsigned long long)KeyOf<T>::key(f[i]) == thr) ? 1u : 0u;
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t s = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += wsum[w];
        cnt[blockIdx.x] = s;
    }
}

// In place: cnt[b] <- sum of cnt[0..b) (one CTA; nb is a few thousand).
__global__ void __launch_bounds__(1024) k_scan_small(uint32_t* __restrict__ cnt, int nb) {
    __shared__ uint32_t part[1024];
    const int per = (nb + 1023) / 1024, lo = threadIdx.x * per, hi = min(nb, lo + per);
    uint32_t s = 0;
    for (int i = lo; i < hi; ++i) s += cnt[i];
    part[threadIdx.x] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int t = 0; t < 1024; ++t) {
            const uint32_t v = part[t];
            part[t] = run;
            run += v;
        }
    }
    __syncthreads();
    uint32_t run = part[threadIdx.x];
    for (int i = lo; i < hi; ++i) {
        const uint32_t v = cnt[i];
        cnt[i] = run;
        run += v;
    }
}

// delta_h = 1[selected] n^3/K - 1
template <typename T>
__global__ void __launch_bounds__(256) k_select(const T* __restrict__ f, int64_t count, int64_t chunk,
                                                 unsigned long long thr, const uint32_t* __restrict__ first,
                                                 uint32_t eq_needed, T scale, T* __restrict__ out) {
    __shared__ uint32_t wcnt[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int64_t lo = (int64_t)blockIdx.x * chunk, hi = min(count, lo + chunk);
    uint32_t base = first[blockIdx.x];  // rank of the chunk's first equal cell
    for (int64_t t0 = lo; t0 < hi; t0 += blockDim.x) {
        const int64_t i = t0 + threadIdx.x;
        unsigned long long k = 0;
        bool eq = false;
        if (i < hi) {
            k = (unsigned long long)KeyOf<T>::key(f[i]);
            eq = k == thr;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, eq);
        if (lane == 0) wcnt[w] = __popc(bal);
        __syncthreads();
        uint32_t before = base;
        for (int v = 0; v < w; ++v) before += wcnt[v];
        uint32_t tile = 0;
        for (int v = 0; v < nw; ++v) tile += wcnt[v];
        if (i < hi) {
            const uint32_t rank = before + __popc(bal & ((1u << lane) - 1u));
            const bool sel = k > thr || (eq && rank < eq_needed);
            out[i] = sel ? scale - T(1) : T(-1);
        }
        base += tile;
        __syncthreads();  // wcnt is rewritten by the next tile
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
    uint32_t* flags = (uint32_t*)((char*)scratch + 256 * sizeof(unsigned long long));  // per-CTA counts
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
    const unsigned nb = blocks_for(count);
    const int64_t chunk = (count + nb - 1) / nb;
    k_eq_count<T><<<nb, 256, 0, st>>>(field, count, chunk, prefix, flags);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_scan_small<<<1, 1024, 0, st>>>(flags, (int)nb);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_select<T><<<nb, 256, 0, st>>>(field, count, chunk, prefix, flags, (uint32_t)remaining,
                                    (T)((double)count / (double)K), out);
    return cudaGetLastError();
}

size_t halo_proxy_scratch_bytes(int64_t count) {
    return 256 * sizeof(unsigned long long) + sizeof(uint32_t) * (size_t)blocks_for(count);
}

template cudaError_t halo_proxy<float>(const float*, int64_t, int64_t, float*, void*, cudaStream_t);
template cudaError_t halo_proxy<double>(const double*, int64_t, int64_t, double*, void*, cudaStream_t);

}  // namespace pm
