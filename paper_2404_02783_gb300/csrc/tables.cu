// Once-per-device constant tables: exp(-2 pi i k / 1024), k < 1024, in FP64 and
// rounded to FP32, for the FFT passes of both precisions.
#include <math.h>

#include <mutex>
#include <map>
#include <set>
#include <tuple>
#include <utility>

#include "internal.h"

namespace pm {

cudaError_t upload_twiddles_f32(const float2* host);
cudaError_t upload_twiddles_f64(const double2* host);

static std::mutex g_tab_mutex;
static bool g_tab_ready[128];

cudaError_t ensure_device_tables() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_tab_mutex);
    if (dev >= 0 && dev < 128 && g_tab_ready[dev]) return cudaSuccess;
    static float2 h32[1024];
    static double2 h64[1024];
    for (int k = 0; k < 1024; ++k) {
        double c, s;
        if (k % 256 == 0) {  // exact quarter turns
            const int q = k / 256;
            c = (q == 0) ? 1.0 : (q == 2 ? -1.0 : 0.0);
            s = (q == 1) ? -1.0 : (q == 3 ? 1.0 : 0.0);
        } else {
            const double ang = -2.0 * M_PI * (double)k / 1024.0;
            c = cos(ang);
            s = sin(ang);
        }
        h64[k] = make_double2(c, s);
        h32[k] = make_float2((float)c, (float)s);
    }
    e = upload_twiddles_f32(h32);
    if (e != cudaSuccess) return e;
    e = upload_twiddles_f64(h64);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 128) g_tab_ready[dev] = true;
    return cudaSuccess;
}

static std::mutex g_attr_mutex;
static std::map<std::pair<const void*, int>, size_t> g_attr_max;

// The attribute only ever grows: a kernel launched with several shared-memory sizes keeps
// the largest one requested so far, so every earlier size stays valid.
cudaError_t set_smem_once(const void* fn, size_t bytes) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    const auto key = std::make_pair(fn, dev);
    auto it = g_attr_max.find(key);
    if (it != g_attr_max.end() && it->second >= bytes) return cudaSuccess;
    e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e == cudaSuccess) g_attr_max[key] = bytes;
    else (void)cudaGetLastError();  // report it here, not from the next launch's check
    return e;
}

static std::map<std::tuple<const void*, int, int, size_t>, int> g_resident;

// CTAs of fn resident per SM at the given launch shape (cached per device).
cudaError_t resident_ctas(const void* fn, int threads, size_t smem, int* per_sm) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lock(g_attr_mutex);
    const auto key = std::make_tuple(fn, dev, threads, smem);
    auto it = g_resident.find(key);
    if (it != g_resident.end()) {
        *per_sm = it->second;
        return cudaSuccess;
    }
    int n = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, threads, smem);
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return e;
    }
    if (n < 1) n = 1;
    g_resident[key] = n;
    *per_sm = n;
    return cudaSuccess;
}

int num_sms() {
    static int sms[128] = {0};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return 152;
    if (sms[dev] == 0) {
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 152;
        sms[dev] = n;
    }
    return sms[dev];
}

}  // namespace pm
