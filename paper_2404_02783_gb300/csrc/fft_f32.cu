// FP32 instantiation of the FFT passes (fft_impl.cuh) and its twiddle table.
#include "fft_impl.cuh"

namespace pm {

static __device__ float2 g_tw32[1024];
template <> __device__ __forceinline__ float2 tw_global<float>(int k) { return g_tw32[k]; }

cudaError_t upload_twiddles_f32(const float2* host) {
    return cudaMemcpyToSymbol(g_tw32, host, sizeof(float2) * 1024);
}

PM_INST(float)

}  // namespace pm
