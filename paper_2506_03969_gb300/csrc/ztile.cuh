// z-direction real<->half-spectrum DFT of one tile (device functions shared by
// the stand-alone z passes and the fused nodes).
//
// A tile is 16 consecutive x by GY consecutive y lines along z.  Complex line
// c (0 <= c < 8 GY) packs the real lines x0 + 2(c % 8) + {0, 1} of row
// y0 + c / 8 as a + i b; one N-point complex four-step DFT per complex line;
// the two real lines' half spectra are separated by Hermitian symmetry.
// Spectra are stored [kz][y][x] (kz = 0..N/2), so the (A, B) pair of a
// complex line is one 16-byte (float) or 32-byte (double) store.
#pragma once

#include <type_traits>

#include "common.cuh"

namespace bridge {

// Four-step twiddle exp(-2 pi i n2 k1 / N) from the [k1][n2] table (step A)
// or the [n2][k1] table (step B'); both live in twiddle.cuh.
template <typename T> __device__ __forceinline__ cplx_t<T> ztw_a(int i);
template <typename T> __device__ __forceinline__ cplx_t<T> ztw_b(int i);
template <typename T, int N> __device__ __forceinline__ cplx_t<T> tw_a(int k1, int n2) {
    return ztw_a<T>(N + k1 * Split<N>::N2 + n2);
}
template <typename T, int N> __device__ __forceinline__ cplx_t<T> tw_b(int n2, int k1) {
    return ztw_b<T>(N + n2 * Split<N>::N1 + k1);
}

template <typename T, int N, int GY_> struct ZCfg {
    using V = cplx_t<T>;
    using V4 = typename std::conditional<sizeof(T) == 4, float4, double4_32a>::type;
    static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, J = N1 / N2;
    static constexpr int GY = GY_ < N ? GY_ : N;
    static constexpr int GC = 8 * GY;                 // complex lines per tile
    static constexpr int NT = GC * N2;                // threads that run one field
    static constexpr int SM_A = GC * N1 * (N2 + 1);   // four-step transpose buffer
    static constexpr int ZS = N + 1;                  // natural-order row stride
    static constexpr int SM_Z = GC * ZS;
    static constexpr int SM_ELEMS = SM_A > SM_Z ? SM_A : SM_Z;
    static constexpr int TILES = (N / 16) * (N / GY);
    static constexpr int TILE_VOX = 16 * GY * N;
    __device__ static int sidx(int c, int k1, int n2) { return c * (N1 * (N2 + 1)) + k1 * (N2 + 1) + n2; }
    __device__ static void tile_xy(int tile, int& x0, int& y0) {
        x0 = (tile % (N / 16)) * 16;
        y0 = (tile / (N / 16)) * GY;
    }
};

// Real-line accesses (a policy hook: the fused nodes and the passes use plain
// loads and stores; an L2 evict-last variant measured no difference).
struct PlainLineIO {
    template <typename T> __device__ __forceinline__ T ld(const T* p) const { return *p; }
    template <typename T> __device__ __forceinline__ void st(T* p, T v) const { *p = v; }
};
// 16/32-byte spectrum accesses; STREAM marks data touched once (evict-first in L2).
template <bool STREAM, typename V4> __device__ __forceinline__ V4 zld4(const V4* p) {
    if constexpr (STREAM && std::is_same<V4, float4>::value) return __ldcs(p);
    else return *p;
}
template <bool STREAM, typename V4> __device__ __forceinline__ void zst4(V4* p, const V4& v) {
    if constexpr (STREAM && std::is_same<V4, float4>::value) __stcs(p, v);
    else *p = v;
}

// Forward: real lines -> spectrum.  line(c) returns the pointer of real line
// a of complex line c; line b is at line(c) + bstride.  Must be called by all
// threads t < C::NT of the block (it synchronises with __syncthreads).
template <typename C, typename LineFn, bool STREAM = false, typename IO = PlainLineIO>
__device__ __forceinline__ void ztile_fwd(LineFn line, long long bstride, typename C::V* __restrict__ spec,
                                          int x0, int y0, typename C::V* sm, int t, const IO& io = IO()) {
    using V = typename C::V;
    using T = decltype(V{}.x);
    using V4 = typename C::V4;
    constexpr int N = C::N1 * C::N2;
    {
        const int n2 = t % C::N2, c = t / C::N2;
        const T* la = line(c);
        const T* lb = la + bstride;
        V v[C::N1];
#pragma unroll
        for (int n1 = 0; n1 < C::N1; ++n1) v[n1] = cmake<V>(io.ld(la + C::N2 * n1 + n2), io.ld(lb + C::N2 * n1 + n2));
        dft_dif<C::N1, 1, -1>(v);
#pragma unroll
        for (int i = 0; i < C::N1; ++i) {
            const int k1 = bitrev(i, C::N1);
            sm[C::sidx(c, k1, n2)] = cmul(v[i], tw_a<T, N>(k1, n2));
        }
    }
    __syncthreads();
    {
        const int c = t / C::N2;
        V X[C::J][C::N2];
#pragma unroll
        for (int j = 0; j < C::J; ++j) {
            const int k1 = t % C::N2 + j * C::N2;
#pragma unroll
            for (int n2 = 0; n2 < C::N2; ++n2) X[j][n2] = sm[C::sidx(c, k1, n2)];
            dft_dif<C::N2, 1, -1>(X[j]);
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < C::J; ++j) {
            const int k1 = t % C::N2 + j * C::N2;
#pragma unroll
            for (int i = 0; i < C::N2; ++i) sm[c * C::ZS + k1 + C::N1 * bitrev(i, C::N2)] = X[j][i];
        }
    }
    __syncthreads();
    constexpr int ROWS = C::NT / 8;
    const int pair = t % 8;
    for (int idx = t / 8; idx < (N / 2 + 1) * C::GY; idx += ROWS) {
        const int kz = idx / C::GY, yl = idx % C::GY;
        const int c = yl * 8 + pair;
        const V z1 = sm[c * C::ZS + kz];
        const V z2 = sm[c * C::ZS + ((N - kz) & (N - 1))];
        const T h = T(0.5);
        V4 ab;
        ab.x = h * (z1.x + z2.x);
        ab.y = h * (z1.y - z2.y);
        ab.z = h * (z1.y + z2.y);
        ab.w = h * (z2.x - z1.x);
        zst4<STREAM>(reinterpret_cast<V4*>(spec + (size_t(kz) * N + (y0 + yl)) * N + x0 + 2 * pair), ab);
    }
    __syncthreads();
}

// Inverse: spectrum -> real lines (unnormalised).  Same calling rules.
// LOADS: spectrum rows a thread keeps in flight (0: 9 in FP32, 5 in FP64).  The
// fused nodes pass 1: with 8-9 CTAs per SM their load phases already overlap
// other CTAs' arithmetic, and more rows in flight only raised their registers.
template <typename C, typename LineFn, bool STREAM = false, typename IO = PlainLineIO, int LOADS = 0>
__device__ __forceinline__ void ztile_inv(const typename C::V* __restrict__ spec, LineFn line, long long bstride,
                                          int x0, int y0, typename C::V* sm, int t, const IO& io = IO()) {
    using V = typename C::V;
    using T = decltype(V{}.x);
    using V4 = typename C::V4;
    constexpr int N = C::N1 * C::N2;
    constexpr int ROWS = C::NT / 8;
    constexpr int TOTAL = (N / 2 + 1) * C::GY;            // (kz, y) rows of the tile
    constexpr int ITERS = (TOTAL + ROWS - 1) / ROWS;      // rows per thread
    // all of a thread's row loads are issued before the first is used (one DRAM
    // latency per batch instead of one per row); batches bound the registers
    constexpr int MAXB = LOADS > 0 ? LOADS : (sizeof(T) == 4 ? 9 : 5);
    constexpr int NB = (ITERS + MAXB - 1) / MAXB;
    constexpr int PB = (ITERS + NB - 1) / NB;
    const int pair = t % 8;
    if constexpr (MAXB == 1) {
        for (int idx = t / 8; idx < TOTAL; idx += ROWS) {
            const int kz = idx / C::GY, yl = idx % C::GY;
            const int c = yl * 8 + pair;
            const V4 ab = zld4<STREAM>(reinterpret_cast<const V4*>(spec + (size_t(kz) * N + (y0 + yl)) * N + x0 + 2 * pair));
            if (kz == 0 || kz == N / 2) {
                sm[c * C::ZS + kz] = cmake<V>(ab.x, ab.z);   // real parts only
            } else {
                sm[c * C::ZS + kz] = cmake<V>(ab.x - ab.w, ab.y + ab.z);
                sm[c * C::ZS + (N - kz)] = cmake<V>(ab.x + ab.w, ab.z - ab.y);
            }
        }
    } else {
#pragma unroll 1
        for (int b0 = 0; b0 < ITERS; b0 += PB) {
            V4 ab[PB];
#pragma unroll
            for (int u = 0; u < PB; ++u) {
                const int idx = t / 8 + (b0 + u) * ROWS;
                if (b0 + u < ITERS && idx < TOTAL) {
                    const int kz = idx / C::GY, yl = idx % C::GY;
                    ab[u] = zld4<STREAM>(reinterpret_cast<const V4*>(spec + (size_t(kz) * N + (y0 + yl)) * N + x0 + 2 * pair));
                }
            }
#pragma unroll
            for (int u = 0; u < PB; ++u) {
                const int idx = t / 8 + (b0 + u) * ROWS;
                if (b0 + u < ITERS && idx < TOTAL) {
                    const int kz = idx / C::GY, yl = idx % C::GY;
                    const int c = yl * 8 + pair;
                    if (kz == 0 || kz == N / 2) {
                        sm[c * C::ZS + kz] = cmake<V>(ab[u].x, ab[u].z);   // real parts only
                    } else {
                        sm[c * C::ZS + kz] = cmake<V>(ab[u].x - ab[u].w, ab[u].y + ab[u].z);
                        sm[c * C::ZS + (N - kz)] = cmake<V>(ab[u].x + ab[u].w, ab[u].z - ab[u].y);
                    }
                }
            }
        }
    }
    __syncthreads();
    {
        const int c = t / C::N2;
        V Y[C::J][C::N2];
#pragma unroll
        for (int j = 0; j < C::J; ++j) {
            const int k1 = t % C::N2 + j * C::N2;
#pragma unroll
            for (int k2 = 0; k2 < C::N2; ++k2) Y[j][k2] = sm[c * C::ZS + k1 + C::N1 * k2];
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < C::J; ++j) {
            const int k1 = t % C::N2 + j * C::N2;
            dft_dif<C::N2, 1, +1>(Y[j]);
#pragma unroll
            for (int i = 0; i < C::N2; ++i) {
                const int n2 = bitrev(i, C::N2);
                sm[C::sidx(c, k1, n2)] = cmulc(Y[j][i], tw_b<T, N>(n2, k1));
            }
        }
    }
    __syncthreads();
    {
        const int n2 = t % C::N2, c = t / C::N2;
        T* la = line(c);
        T* lb = la + bstride;
        V v[C::N1];
#pragma unroll
        for (int k1 = 0; k1 < C::N1; ++k1) v[k1] = sm[C::sidx(c, k1, n2)];
        dft_dif<C::N1, 1, +1>(v);
#pragma unroll
        for (int i = 0; i < C::N1; ++i) {
            const int pos = n2 + C::N2 * bitrev(i, C::N1);
            io.st(la + pos, v[i].x);
            io.st(lb + pos, v[i].y);
        }
    }
    __syncthreads();
}

}  // namespace bridge
