// FP64 instantiation of the FFT passes (fft_impl.cuh) and its twiddle table.
#include "fft_impl.cuh"

namespace pm {

static __device__ double2 g_tw64[1024];
template <> __device__ __forceinline__ double2 tw_global<double>(int k) { return g_tw64[k]; }

cudaError_t upload_twiddles_f64(const double2* host) {
    return cudaMemcpyToSymbol(g_tw64, host, sizeof(double2) * 1024);
}

PM_INST(double)

// The fused and whole-plane middle passes are built for FP32 only (FP64 runs the separate passes).
template <>
cudaError_t fft_plane<double>(double2*, double2*, double2*, int, int, const SpecOp&, cudaStream_t) {
    return cudaErrorNotSupported;
}
template <>
cudaError_t fft_middle<double>(double2*, double2*, double2*, int, int, const SpecOp&, unsigned*, int, cudaStream_t) {
    return cudaErrorNotSupported;
}

// div_mode<double> applied element by element (the check of its Newton-Raphson reciprocal).
__global__ void k_div_mode(const double* __restrict__ a, const double* __restrict__ d, int64_t count,
                           double* __restrict__ out) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = div_mode<double>(a[i], d[i]);
}
cudaError_t div_mode_check(const double* a, const double* d, int64_t count, double* out, cudaStream_t st) {
    if (count <= 0) return cudaSuccess;
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 152 * 8);
    k_div_mode<<<(unsigned)blocks, 256, 0, st>>>(a, d, count, out);
    return cudaGetLastError();
}

}  // namespace pm
