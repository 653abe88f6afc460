// FP64 instantiation of the FFT passes (fft_impl.cuh) and its twiddle table.
#include "fft_impl.cuh"

namespace pm {

static __device__ double2 g_tw64[1024];
template <> __device__ __forceinline__ double2 tw_global<double>(int k) { return g_tw64[k]; }

cudaError_t upload_twiddles_f64(const double2* host) {
    return cudaMemcpyToSymbol(g_tw64, host, sizeof(double2) * 1024);
}

PM_INST(double)

}  // namespace pm
