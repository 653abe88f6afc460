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

// out[b] = sum over rows r (in order) of rows[r nbins + b]: the per-CTA bin sums of the
// binning x pass, combined in a fixed order.
__global__ void k_sum_rows(const double* __restrict__ rows, int nrows, int nbins, double* __restrict__ out) {
    for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < nbins; b += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int r = 0; r < nrows; ++r) s += rows[(size_t)r * nbins + b];
        out[b] = s;
    }
}

cudaError_t bin_rows_sum(const double* rows, int nrows, int nbins, double* out, cudaStream_t st) {
    k_sum_rows<<<1, 256, 0, st>>>(rows, nrows, nbins, out);
    return cudaGetLastError();
}

}  // namespace pm
