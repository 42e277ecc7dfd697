// Per-translation-unit four-step twiddle tables in device memory, computed on
// the host in FP64 (libm) and rounded to the kernel precision.  For each
// N = N1 * N2 in 16..512 the factor exp(-2 pi i n2 k1 / N) is stored twice:
//   tw_a: entry N + k1 * N2 + n2   (step A, where the lanes of a warp run along n2)
//   tw_b: entry N + n2 * N1 + k1   (step B', where they run along k1)
// so that a warp reads consecutive words in either step.  Each .cu file that
// includes this header owns a copy and uploads it with upload_twiddles_here().
#pragma once

#include <cmath>

#include "common.cuh"
#include "ztile.cuh"

namespace bridge {
namespace {
constexpr int kTwTable = 1024;
__device__ float2 tw_a_f[kTwTable];
__device__ float2 tw_b_f[kTwTable];
__device__ double2 tw_a_d[kTwTable];
__device__ double2 tw_b_d[kTwTable];

inline cudaError_t upload_twiddles_here() {
    static float2 af[kTwTable], bf[kTwTable];
    static double2 ad[kTwTable], bd[kTwTable];
    for (int n = 16; n <= 512; n *= 2) {
        const int n1 = split_n1(n), n2s = n / n1;
        for (int k1 = 0; k1 < n1; ++k1) {
            for (int n2 = 0; n2 < n2s; ++n2) {
                const double a = -2.0 * kPi * double(n2 * k1) / double(n);
                const double c = std::cos(a), s = std::sin(a);
                ad[n + k1 * n2s + n2] = make_double2(c, s);
                bd[n + n2 * n1 + k1] = make_double2(c, s);
                af[n + k1 * n2s + n2] = make_float2(float(c), float(s));
                bf[n + n2 * n1 + k1] = make_float2(float(c), float(s));
            }
        }
    }
    cudaError_t e = cudaMemcpyToSymbol(tw_a_f, af, sizeof(af));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tw_b_f, bf, sizeof(bf));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tw_a_d, ad, sizeof(ad));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(tw_b_d, bd, sizeof(bd));
    return e;
}
}  // namespace

template <> __device__ __forceinline__ float2 ztw_a<float>(int i) { return __ldg(&tw_a_f[i]); }
template <> __device__ __forceinline__ float2 ztw_b<float>(int i) { return __ldg(&tw_b_f[i]); }
template <> __device__ __forceinline__ double2 ztw_a<double>(int i) { return __ldg(&tw_a_d[i]); }
template <> __device__ __forceinline__ double2 ztw_b<double>(int i) { return __ldg(&tw_b_d[i]); }

}  // namespace bridge
