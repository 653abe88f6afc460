// FP32 instantiation of the FFT passes (fft_impl.cuh) and its twiddle table.
#include "fft_impl.cuh"

namespace pm {

static __device__ float2 g_tw32[1024];
template <> __device__ __forceinline__ float2 tw_global<float>(int k) { return g_tw32[k]; }

cudaError_t upload_twiddles_f32(const float2* host) {
    return cudaMemcpyToSymbol(g_tw32, host, sizeof(float2) * 1024);
}

PM_INST(float)
template cudaError_t fft_plane<float>(float2*, float2*, float2*, int, int, const SpecOp&, cudaStream_t);
template cudaError_t fft_middle<float>(float2*, float2*, float2*, int, int, const SpecOp&, unsigned*, int,
                                       cudaStream_t);

// out[b] = sum over rows r of rows[r nbins + b]: the per-CTA bin sums of the binning x pass,
// combined in a fixed order (one warp a bin: lane l sums rows l, l + 32, ... in turn, then a
// fixed shuffle tree), so the result does not depend on the scheduling.
__global__ void k_sum_rows(const double* __restrict__ rows, int nrows, int nbins, double* __restrict__ out) {
    const int lane = threadIdx.x & 31;
    const int b = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (b >= nbins) return;  // whole warps leave together
    double s = 0.0;
    for (int r = lane; r < nrows; r += 32) s += rows[(size_t)r * nbins + b];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0) out[b] = s;
}

cudaError_t bin_rows_sum(const double* rows, int nrows, int nbins, double* out, cudaStream_t st) {
    if (nbins <= 0) return cudaSuccess;
    k_sum_rows<<<(nbins + 7) / 8, 256, 0, st>>>(rows, nrows, nbins, out);
    return cudaGetLastError();
}

}  // namespace pm
