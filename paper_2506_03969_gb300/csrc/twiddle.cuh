// Per-translation-unit twiddle tables in device memory: entry N + j holds
// exp(-2 pi i j / N) for N = 2..512, computed on the host in FP64 (libm) and
// rounded to the kernel precision.  Each .cu file that includes this header
// owns a copy and uploads it with upload_twiddles_here().
#pragma once

#include <cmath>

#include "common.cuh"
#include "ztile.cuh"

namespace bridge {
namespace {
constexpr int kTwTable = 1024;
__device__ float2 tw_tab_f[kTwTable];
__device__ double2 tw_tab_d[kTwTable];

inline cudaError_t upload_twiddles_here() {
    static float2 hf[kTwTable];
    static double2 hd[kTwTable];
    for (int n = 2; n <= 512; n *= 2) {
        for (int j = 0; j < n; ++j) {
            const double a = -2.0 * kPi * double(j) / double(n);
            hd[n + j] = make_double2(std::cos(a), std::sin(a));
            hf[n + j] = make_float2(float(std::cos(a)), float(std::sin(a)));
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(tw_tab_f, hf, sizeof(hf));
    if (e != cudaSuccess) return e;
    return cudaMemcpyToSymbol(tw_tab_d, hd, sizeof(hd));
}
}  // namespace

template <> __device__ __forceinline__ float2 ztw_load<float>(int N, int j) { return __ldg(&tw_tab_f[N + j]); }
template <> __device__ __forceinline__ double2 ztw_load<double>(int N, int j) { return __ldg(&tw_tab_d[N + j]); }

}  // namespace bridge
