// Common types and helpers for the BRIDGE GB300 kernels (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bridge {

// Complex vector type per precision (8- or 16-byte aligned loads/stores).
template <typename T> struct Cplx;
template <> struct Cplx<float> { using type = float2; };
template <> struct Cplx<double> { using type = double2; };
template <typename T> using cplx_t = typename Cplx<T>::type;

template <typename V> __host__ __device__ __forceinline__ V cmake(decltype(V{}.x) a, decltype(V{}.x) b) {
    V r; r.x = a; r.y = b; return r;
}
template <typename V> __device__ __forceinline__ V cadd(V a, V b) { return cmake<V>(a.x + b.x, a.y + b.y); }
template <typename V> __device__ __forceinline__ V csub(V a, V b) { return cmake<V>(a.x - b.x, a.y - b.y); }
template <typename V> __device__ __forceinline__ V cmul(V a, V b) {
    return cmake<V>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename V> __device__ __forceinline__ V cmulc(V a, V b) {  // a * conj(b)
    return cmake<V>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename V, typename S> __device__ __forceinline__ V cscale(V a, S s) { return cmake<V>(a.x * s, a.y * s); }

// ---------------------------------------------------------------------------
// Compile-time cos/sin of 2*pi*k/R (own Taylor series after an exact quadrant
// reduction of the rational angle; |phi| < pi/2 so 16 terms reach double
// precision).  Used for the fixed twiddles inside register DFTs.
// ---------------------------------------------------------------------------
constexpr double kPi = 3.141592653589793238462643383279502884;

constexpr double taylor_sin(double x) {
    double term = x, sum = x;
    for (int i = 1; i < 16; ++i) { term *= -x * x / double((2 * i) * (2 * i + 1)); sum += term; }
    return sum;
}
constexpr double taylor_cos(double x) {
    double term = 1.0, sum = 1.0;
    for (int i = 1; i < 16; ++i) { term *= -x * x / double((2 * i - 1) * (2 * i)); sum += term; }
    return sum;
}
// cos(2 pi k / R)
constexpr double cos_turn(int k, int R) {
    int kk = ((k % R) + R) % R;
    int q = (4 * kk) / R;
    int r = 4 * kk - q * R;
    double phi = 0.5 * kPi * double(r) / double(R);
    double c = taylor_cos(phi), s = taylor_sin(phi);
    return q == 0 ? c : q == 1 ? -s : q == 2 ? -c : s;
}
// sin(2 pi k / R)
constexpr double sin_turn(int k, int R) {
    int kk = ((k % R) + R) % R;
    int q = (4 * kk) / R;
    int r = 4 * kk - q * R;
    double phi = 0.5 * kPi * double(r) / double(R);
    double c = taylor_cos(phi), s = taylor_sin(phi);
    return q == 0 ? s : q == 1 ? c : q == 2 ? -s : -c;
}

// Multiply a by exp(SIGN * 2 pi i K / R), with the trivial angles done exactly.
template <int R, int K, int SIGN, typename V> __device__ __forceinline__ V twiddle_c(V a) {
    constexpr int k = ((K % R) + R) % R;
    using T = decltype(a.x);
    if constexpr (k == 0) {
        return a;
    } else if constexpr (2 * k == R) {
        return cmake<V>(-a.x, -a.y);
    } else if constexpr (4 * k == R) {        // exp(SIGN i pi/2) = SIGN i
        return cmake<V>(T(-SIGN) * a.y, T(SIGN) * a.x);
    } else if constexpr (4 * k == 3 * R) {    // exp(SIGN i 3pi/2) = -SIGN i
        return cmake<V>(T(SIGN) * a.y, T(-SIGN) * a.x);
    } else {
        constexpr double c = cos_turn(k, R);
        constexpr double s = double(SIGN) * sin_turn(k, R);
        return cmake<V>(T(c) * a.x - T(s) * a.y, T(c) * a.y + T(s) * a.x);
    }
}

// ---------------------------------------------------------------------------
// In-register radix-2 decimation-in-frequency DFT of R points stored at
// v[0], v[S], ..., v[(R-1)S].  Output X[bitrev_R(j)] lands in v[j S].
// SIGN = -1: forward transform (e^{-2 pi i n k / R}); +1: inverse (unnormalised).
// ---------------------------------------------------------------------------
template <int R, int S, int SIGN, typename V, int J = 0>
__device__ __forceinline__ void dif_butterflies(V* v) {
    if constexpr (J < R / 2) {
        V a = v[J * S], b = v[(J + R / 2) * S];
        v[J * S] = cadd(a, b);
        v[(J + R / 2) * S] = twiddle_c<R, J, SIGN>(csub(a, b));
        dif_butterflies<R, S, SIGN, V, J + 1>(v);
    }
}
template <int R, int S, int SIGN, typename V>
__device__ __forceinline__ void dft_dif(V* v) {
    if constexpr (R > 1) {
        dif_butterflies<R, S, SIGN, V>(v);
        dft_dif<R / 2, S, SIGN, V>(v);
        dft_dif<R / 2, S, SIGN, V>(v + (R / 2) * S);
    }
}

// Asynchronous 16-byte global -> shared copies (cp.async, L2 only), grouped
// per thread; wait_all returns when this thread's copies have landed (a
// __syncthreads then makes every thread's copies visible to the block).
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((unsigned)__cvta_generic_to_shared(smem)),
                 "l"(gmem)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__host__ __device__ constexpr int ilog2c(int n) { return n <= 1 ? 0 : 1 + ilog2c(n / 2); }
__host__ __device__ constexpr int bitrev(int j, int R) {
    int r = 0;
    for (int b = 1; b < R; b <<= 1) { r = (r << 1) | (j & 1); j >>= 1; }
    return r;
}

// Four-step split N = N1 * N2 with N1 >= N2 (N1 points in step A, N2 in step B).
template <int N> struct Split;
template <> struct Split<16> { static constexpr int N1 = 4, N2 = 4; };
template <> struct Split<32> { static constexpr int N1 = 8, N2 = 4; };
template <> struct Split<64> { static constexpr int N1 = 8, N2 = 8; };
template <> struct Split<128> { static constexpr int N1 = 16, N2 = 8; };
template <> struct Split<256> { static constexpr int N1 = 16, N2 = 16; };
template <> struct Split<512> { static constexpr int N1 = 32, N2 = 16; };
// N1 of Split<n> for a run-time n (host table builders).
constexpr int split_n1(int n) { return n <= 16 ? 4 : n <= 64 ? 8 : n <= 256 ? 16 : 32; }


// Signed integer frequency of index i on an axis of n points.
__device__ __forceinline__ int signed_freq(int i, int n) { return i < n / 2 ? i : i - n; }

// Block-wide sum of a double with a fixed reduction order (deterministic).
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
    #pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < NT / 32; ++i) r += sh[i];
    }
    return r;  // valid in thread 0
}

}  // namespace bridge
