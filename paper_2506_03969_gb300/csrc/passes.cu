// FFT pass kernels: the 3D real<->complex DFT of the forward model is split into
// three passes over HBM, with the k-space operators of the method fused in.
//
//   z pass : real [x][y][z] <-> half spectrum in [kz][y][x] order.  Two real
//            z lines are packed as one complex line (a + i b), transformed with
//            an N-point complex DFT and separated by Hermitian symmetry.
//   y pass : complex DFT along y on [kz][ky][x]; monomial multipliers ky^p kz^q
//            can expand one input into several outputs (inverse direction) or
//            merge several inputs into one output (forward direction).
//   x node : forward DFT along x (all of k is then known), merge the inputs into
//            one scalar spectrum Q with k-space operators, expand Q into the
//            outputs with further operators, inverse DFT along x.
//
// Each 1D DFT uses the four-step split N = N1 * N2: N1-point register DFTs
// (step A), twiddles, a shared-memory transpose, N2-point register DFTs
// (step B).  All global accesses of a warp are contiguous runs of >= 64 bytes.
#include <cmath>
#include <cstdio>
#include <type_traits>

#include "common.cuh"
#include "passes.cuh"
#include "ztile.cuh"
#include "twiddle.cuh"

namespace bridge {

cudaError_t upload_twiddles() { return upload_twiddles_here(); }

void radial_tables_host(int n, const KParams& kp, double* out) {
    const int rlen = 3 * (n / 2) * (n / 2) + 1;
    const double a = std::sqrt(kp.pk_amp / (kp.dx * kp.dx * kp.dx));
    for (int m2 = 0; m2 < rlen; ++m2) {
        const double k2 = kp.kf * kp.kf * double(m2);
        const double inv = m2 > 0 ? 1.0 / k2 : 0.0;
        // sqrt(P(k)/dx^3), P = A k^ns / (1 + (k/kc)^2)^pow, P(0) = 0   (App. A)
        const double sp = m2 > 0 ? a * std::pow(k2, 0.25 * kp.pk_ns) *
                                       std::pow(1.0 + k2 / (kp.pk_kc * kp.pk_kc), -0.5 * kp.pk_pow)
                                 : 0.0;
        const double e = -0.5 * kp.r_s * kp.r_s * k2;   // K(k) = exp(-k^2 r_s^2 / 2), Sect. 2.3
        out[0 * rlen + m2] = inv;
        out[1 * rlen + m2] = sp;
        out[2 * rlen + m2] = std::exp(e);
        out[3 * rlen + m2] = -std::expm1(e);
    }
}

// ---------------------------------------------------------------------------
// Multipliers
// ---------------------------------------------------------------------------
// k_axis^p for signed index m; odd powers vanish on the Nyquist index.
template <typename T> __device__ __forceinline__ T kpow(int m, int p, int n, T kf) {
    if (p == 0) return T(1);
    if ((p & 1) && (m == n / 2 || m == -(n / 2))) return T(0);
    const T k = kf * T(m);
    return p == 1 ? k : (p == 2 ? k * k : k * k * k);
}

// y-pass multiplier: (cre + i cim) ky^py kz^pz (no radial factor in the y pass).
template <typename T>
__device__ __forceinline__ cplx_t<T> ymult(const Term& tm, int my, int mz, int n, const KParams& kp) {
    const T kf = kf_of<T>(kp);
    const T r = kpow<T>(my, tm.py, n, kf) * kpow<T>(mz, tm.pz, n, kf);
    return cmake<cplx_t<T>>(T(tm.cre) * r, T(tm.cim) * r);
}

// ---------------------------------------------------------------------------
// Column tiles for the y pass (XM = false, lines strided by N) and the x node
// (XM = true, lines contiguous).  Spectra are [kz][ky or y][x] with N*N
// elements per kz plane and N/2+1 planes.
// ---------------------------------------------------------------------------
#ifndef BRIDGE_XNODE_T32
#define BRIDGE_XNODE_T32 128   // threads of an FP32 x-node CTA (its tile: BRIDGE_XNODE_T32 / N2 lines); four
                               // 128-thread CTAs per SM instead of two of 256: 0.646 -> 0.591 ms at 256^3
#endif
template <typename T, int N, bool XM> struct Tile {
    using V = cplx_t<T>;
    static constexpr int N1 = Split<N>::N1, N2 = Split<N>::N2, J = N1 / N2;
    // FP64 at N = 512: 8 columns, so that the forward pass's tile and its staged copy fit in shared memory
    static constexpr int GY0 = (sizeof(V) == 16 && N >= 512) ? 8
                               : ((int)(128 / sizeof(V)) > 256 / N2 ? (int)(128 / sizeof(V)) : 256 / N2);
    static constexpr int GX0 = (sizeof(V) == 8 ? BRIDGE_XNODE_T32 : 128) / N2;
    static constexpr int G0 = XM ? GX0 : GY0;
    static constexpr int G = G0 < N ? G0 : N;
    static constexpr int NT = G * N2;
    static constexpr int SM_ELEMS = XM ? G * N1 * (N2 + 1) : N * G;
    static constexpr int TILES_PER_PLANE = N / G;
    static constexpr int TILES = (N / 2 + 1) * TILES_PER_PLANE;

    __device__ static void tile_pos(int tile, int& kz, int& c0) {
        kz = tile / TILES_PER_PLANE;
        c0 = (tile % TILES_PER_PLANE) * G;
    }
    __device__ static size_t tile_base(int kz, int c0) {
        return size_t(kz) * N * N + (XM ? size_t(c0) * N : size_t(c0));
    }
    __device__ static int goff(int n, int g) { return XM ? g * N + n : n * N + g; }
    __device__ static int a_g(int t) { return XM ? t / N2 : t % G; }
    __device__ static int a_n2(int t) { return XM ? t % N2 : t / G; }
    __device__ static int b_g(int t) { return XM ? t / N2 : t % G; }
    __device__ static int b_k1(int t, int j) { return (XM ? t % N2 : t / G) + j * N2; }
    __device__ static int sidx(int g, int k1, int n2) {
        return XM ? g * (N1 * (N2 + 1)) + k1 * (N2 + 1) + n2 : (k1 * N2 + n2) * G + g;
    }
    // signed frequencies of element (n, g) of a tile at (kz, c0)
    __device__ static void freqs(int n, int g, int kz, int c0, int& mx, int& my, int& mz) {
        mz = kz;
        if (XM) { mx = signed_freq(n, N); my = signed_freq(c0 + g, N); }
        else { mx = 0; my = signed_freq(n, N); }
    }

    // Staged input tile in shared memory: the tile's ROWS rows of RLEN
    // contiguous elements (x-node: G lines of N; y pass: N rows of G columns).
    static constexpr int ROWS = XM ? G : N, RLEN = XM ? N : G;
    static constexpr int STAGE_ELEMS = ROWS * RLEN;
    __device__ static int soff(int n, int g) { return XM ? g * N + n : n * G + g; }
    // issue the asynchronous copy of the tile at src (rows N elements apart)
    __device__ static void stage(const V* __restrict__ src, V* buf, int t) {
        constexpr int CPR = int(RLEN * sizeof(V)) / 16;   // 16-byte chunks per row
        for (int c = t; c < ROWS * CPR; c += NT) {
            const int row = c / CPR, part = c % CPR;
            cp_async16(reinterpret_cast<char*>(buf + row * RLEN) + part * 16,
                       reinterpret_cast<const char*>(src + size_t(row) * N) + part * 16);
        }
        cp_async_commit();
    }
    // forward step A from the staged tile into shared memory (twiddled)
    __device__ static void fwdA_staged(const V* buf, V* sm, int t) {
        const int g = a_g(t), n2 = a_n2(t);
        V v[N1];
#pragma unroll
        for (int n1 = 0; n1 < N1; ++n1) v[n1] = buf[soff(N2 * n1 + n2, g)];
        dft_dif<N1, 1, -1>(v);
#pragma unroll
        for (int i = 0; i < N1; ++i) {
            const int k1 = bitrev(i, N1);
            sm[sidx(g, k1, n2)] = cmul(v[i], tw_a<T, N>(k1, n2));
        }
    }
    // forward step B: X[j][i] = DFT value at k = k1_j + N1 * bitrev(i)
    __device__ static void fwdB(const V* sm, int t, V (&X)[J][N2]) {
        const int g = b_g(t);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k1 = b_k1(t, j);
#pragma unroll
            for (int n2 = 0; n2 < N2; ++n2) X[j][n2] = sm[sidx(g, k1, n2)];
            dft_dif<N2, 1, -1>(X[j]);
        }
    }
    // inverse step B' from natural-order registers Y[j][k2] (k = k1_j + N1 k2)
    __device__ static void invB(V (&Y)[J][N2], V* sm, int t) {
        const int g = b_g(t);
#pragma unroll
        for (int j = 0; j < J; ++j) {
            const int k1 = b_k1(t, j);
            dft_dif<N2, 1, +1>(Y[j]);
#pragma unroll
            for (int i = 0; i < N2; ++i) {
                const int n2 = bitrev(i, N2);
                sm[sidx(g, k1, n2)] = cmulc(Y[j][i], tw_b<T, N>(n2, k1));
            }
        }
    }
    // inverse step A' to global (A layout)
    __device__ static void invA(const V* sm, V* __restrict__ dst, int t) {
        const int g = a_g(t), n2 = a_n2(t);
        V v[N1];
#pragma unroll
        for (int k1 = 0; k1 < N1; ++k1) v[k1] = sm[sidx(g, k1, n2)];
        dft_dif<N1, 1, +1>(v);
#pragma unroll
        for (int i = 0; i < N1; ++i) dst[goff(n2 + N2 * bitrev(i, N1), g)] = v[i];
    }
};

// FP32 multiplier specialised at compile time for the term shapes the programs
// use: kx^PX times 1 (RC = R_ONE) or 1/k^2 (RC = R_INVK2); HI is the
// compile-time part N1 * k2 of the element's x index k1 + HI, so the signed
// frequency and the Nyquist test reduce to one add and one compare.
// RC = R_SQRTP reads the radial table at m^2; the blend codes take the x factor
// skx[k1 + HI] times the per-thread (y, z) factor kyz (see XTerm).
template <typename T, int N, int PX, int RC, int HI>
__device__ __forceinline__ T xfac(int k1, int m2yz, const KParams& kp, const T* skx = nullptr, T kyz = T(0)) {
    const int mx = HI < N / 2 ? k1 + HI : k1 + HI - N;
    T r = T(1);
    if constexpr (PX > 0) {
        const T kx = kf_of<T>(kp) * T(mx);
        r = PX == 1 ? kx : kx * kx;
        if constexpr (PX == 1) r = (mx == -(N / 2)) ? T(0) : r;
    }
    if constexpr (RC == R_INVK2) {
        const int m2 = mx * mx + m2yz;
        r *= m2 > 0 ? T(__fdividef(kp.inv_kf2_f, float(m2))) : T(0);
    } else if constexpr (RC == R_SQRTP) {
        r *= __ldg(reinterpret_cast<const T*>(kp.rtab) + (R_SQRTP - 1) * kp.rlen + mx * mx + m2yz);
    } else if constexpr (RC == R_KBLEND) {
        r *= skx[k1 + HI] * kyz;
    } else if constexpr (RC == R_1MKBLEND) {
        r *= T(1) - skx[k1 + HI] * kyz;
    }
    return r;
}
template <int V> using IC = std::integral_constant<int, V>;
// Compile-time loop: f(IC<I>{}) for I = B .. E-1.
template <int B, int E, typename F> __device__ __forceinline__ void sfor(F&& f) {
    if constexpr (B < E) {
        f(IC<B>{});
        sfor<B + 1, E>(f);
    }
}
// Calls f(IC<PX>, IC<RC>) for the specialised shapes; false for any other term.
// FP32 up to N = 256 only (FP64 and N = 512 have no registers to spare for the
// extra code paths).
template <typename T, int N, typename F> __device__ __forceinline__ bool xdispatch(const Term& tm, F&& f) {
    if constexpr (sizeof(T) != 4 || N > 256) {
        return false;
    } else {
        switch (tm.px * 8 + tm.rcode) {
            case 0 * 8 + R_ONE: f(IC<0>{}, IC<R_ONE>{}); return true;
            case 1 * 8 + R_ONE: f(IC<1>{}, IC<R_ONE>{}); return true;
            case 2 * 8 + R_ONE: f(IC<2>{}, IC<R_ONE>{}); return true;
            case 0 * 8 + R_INVK2: f(IC<0>{}, IC<R_INVK2>{}); return true;
            case 1 * 8 + R_INVK2: f(IC<1>{}, IC<R_INVK2>{}); return true;
            case 2 * 8 + R_INVK2: f(IC<2>{}, IC<R_INVK2>{}); return true;
            case 0 * 8 + R_SQRTP: f(IC<0>{}, IC<R_SQRTP>{}); return true;
            case 0 * 8 + R_KBLEND: f(IC<0>{}, IC<R_KBLEND>{}); return true;
            case 0 * 8 + R_1MKBLEND: f(IC<0>{}, IC<R_1MKBLEND>{}); return true;
            default: return false;
        }
    }
}

// f(IC<PY>) for a y-pass term with ky power PY = 1 or 2 (FP32 up to N = 256);
// false otherwise.
template <typename T, int N, typename F> __device__ __forceinline__ bool ydispatch(const Term& tm, F&& f) {
    if constexpr (sizeof(T) != 4 || N > 256) {
        return false;
    } else {
        if (tm.py == 1) { f(IC<1>{}); return true; }
        if (tm.py == 2) { f(IC<2>{}); return true; }
        return false;
    }
}

#ifndef BRIDGE_YPASS_MINB
#define BRIDGE_YPASS_MINB 3   // FP32; the FP64 y passes (one CTA per SM by shared memory) are unbounded
#endif
// Forward (merge) column pass: out[o] = sum_{terms -> o} mult * DFT(in[src]).
// The host orders the merge terms by output; the tile of the next term is
// copied into shared memory (cp.async) while the current one is transformed.
template <typename T, int N, bool XM>
__global__ void __launch_bounds__(Tile<T, N, XM>::NT, sizeof(T) == 4 ? BRIDGE_YPASS_MINB : 1) k_col_fwd(const PassProgram P, const KParams kp) {
    using TL = Tile<T, N, XM>;
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    V* buf = sm + TL::SM_ELEMS;
    const int t = threadIdx.x, chain = blockIdx.y;
    int kz, c0;
    TL::tile_pos(blockIdx.x, kz, c0);
    const size_t base = TL::tile_base(kz, c0);
    const int g = TL::b_g(t);
    auto src_of = [&](int m) { return reinterpret_cast<const V*>(P.in[P.merge[m].src]) + chain * P.in_cs + base; };
    if (P.n_merge > 0) TL::stage(src_of(0), buf, t);
    int m = 0;
    for (int o = 0; o < P.n_out; ++o) {
        V acc[TL::J][TL::N2];
#pragma unroll
        for (int j = 0; j < TL::J; ++j)
#pragma unroll
            for (int i = 0; i < TL::N2; ++i) acc[j][i] = cmake<V>(T(0), T(0));
        for (; m < P.n_merge && P.merge[m].dst == o; ++m) {
            const Term tm = P.merge[m];
            cp_async_wait_all();
            __syncthreads();                  // tile m visible; sm free
            TL::fwdA_staged(buf, sm, t);
            __syncthreads();                  // buf free, sm complete
            if (m + 1 < P.n_merge) TL::stage(src_of(m + 1), buf, t);
            V X[TL::J][TL::N2];
            TL::fwdB(sm, t, X);
            if (!XM && tm.py == 0) {
                // no ky power: one complex factor (cre + i cim) kz^pz for the whole tile
                const V c = ymult<T>(tm, 0, kz, N, kp);
#pragma unroll
                for (int j = 0; j < TL::J; ++j)
#pragma unroll
                    for (int i = 0; i < TL::N2; ++i) acc[j][i] = cadd(acc[j][i], cmul(c, X[j][i]));
            } else if (XM || !ydispatch<T, N>(tm, [&](auto pyc) {
                           // ky^PY per element times one complex factor (cre + i cim) kz^pz
                           constexpr int PY = decltype(pyc)::value;
                           Term t0 = tm;
                           t0.py = 0;
                           const V c = ymult<T>(t0, 0, kz, N, kp);
#pragma unroll
                           for (int j = 0; j < TL::J; ++j) {
                               const int k1 = TL::b_k1(t, j);
                               sfor<0, TL::N2>([&](auto ic) {
                                   constexpr int i = decltype(ic)::value;
                                   const T r = xfac<T, N, PY, R_ONE, TL::N1 * bitrev(i, TL::N2)>(k1, 0, kp);
                                   acc[j][i] = cadd(acc[j][i], cmul(cmake<V>(c.x * r, c.y * r), X[j][i]));
                               });
                           }
                       })) {
#pragma unroll
                for (int j = 0; j < TL::J; ++j) {
                    const int k1 = TL::b_k1(t, j);
#pragma unroll
                    for (int i = 0; i < TL::N2; ++i) {
                        int mx, my, mz;
                        TL::freqs(k1 + TL::N1 * bitrev(i, TL::N2), g, kz, c0, mx, my, mz);
                        acc[j][i] = cadd(acc[j][i], cmul(ymult<T>(tm, my, mz, N, kp), X[j][i]));
                    }
                }
            }
        }
        V* dst = reinterpret_cast<V*>(P.out[o]) + chain * P.out_cs + base;
#pragma unroll
        for (int j = 0; j < TL::J; ++j) {
            const int k1 = TL::b_k1(t, j);
#pragma unroll
            for (int i = 0; i < TL::N2; ++i) dst[TL::goff(k1 + TL::N1 * bitrev(i, TL::N2), g)] = acc[j][i];
        }
    }
}

// Inverse (expand) column pass: out[dst] = IDFT(mult * in[src]) for each term.
template <typename T, int N, bool XM>
__global__ void __launch_bounds__(Tile<T, N, XM>::NT, sizeof(T) == 4 ? BRIDGE_YPASS_MINB : 1) k_col_inv(const PassProgram P, const KParams kp) {
    using TL = Tile<T, N, XM>;
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int t = threadIdx.x, chain = blockIdx.y;
    int kz, c0;
    TL::tile_pos(blockIdx.x, kz, c0);
    const size_t base = TL::tile_base(kz, c0);
    const int g = TL::b_g(t);
    for (int s = 0; s < P.n_in; ++s) {
        bool used = false;
        for (int m = 0; m < P.n_expand; ++m) used |= (P.expand[m].src == s);
        if (!used) continue;
        const V* src = reinterpret_cast<const V*>(P.in[s]) + chain * P.in_cs + base;
        V X[TL::J][TL::N2];
#pragma unroll
        for (int j = 0; j < TL::J; ++j) {
            const int k1 = TL::b_k1(t, j);
#pragma unroll
            for (int k2 = 0; k2 < TL::N2; ++k2) X[j][k2] = src[TL::goff(k1 + TL::N1 * k2, g)];
        }
        for (int m = 0; m < P.n_expand; ++m) {
            const Term tm = P.expand[m];
            if (tm.src != s) continue;
            V Y[TL::J][TL::N2];
            if (!XM && tm.py == 0) {
                // no ky power: one complex factor (cre + i cim) kz^pz for the whole tile
                const V c = ymult<T>(tm, 0, kz, N, kp);
#pragma unroll
                for (int j = 0; j < TL::J; ++j)
#pragma unroll
                    for (int k2 = 0; k2 < TL::N2; ++k2) Y[j][k2] = cmul(c, X[j][k2]);
            } else if (XM || !ydispatch<T, N>(tm, [&](auto pyc) {
                           // ky^PY per element times one complex factor (cre + i cim) kz^pz
                           constexpr int PY = decltype(pyc)::value;
                           Term t0 = tm;
                           t0.py = 0;
                           const V c = ymult<T>(t0, 0, kz, N, kp);
#pragma unroll
                           for (int j = 0; j < TL::J; ++j) {
                               const int k1 = TL::b_k1(t, j);
                               sfor<0, TL::N2>([&](auto ic) {
                                   constexpr int k2 = decltype(ic)::value;
                                   const T r = xfac<T, N, PY, R_ONE, TL::N1 * k2>(k1, 0, kp);
                                   Y[j][k2] = cmul(cmake<V>(c.x * r, c.y * r), X[j][k2]);
                               });
                           }
                       })) {
#pragma unroll
                for (int j = 0; j < TL::J; ++j) {
                    const int k1 = TL::b_k1(t, j);
#pragma unroll
                    for (int k2 = 0; k2 < TL::N2; ++k2) {
                        int mx, my, mz;
                        TL::freqs(k1 + TL::N1 * k2, g, kz, c0, mx, my, mz);
                        Y[j][k2] = cmul(ymult<T>(tm, my, mz, N, kp), X[j][k2]);
                    }
                }
            }
            __syncthreads();
            TL::invB(Y, sm, t);
            __syncthreads();
            V* dst = reinterpret_cast<V*>(P.out[tm.dst]) + chain * P.out_cs + base;
            TL::invA(sm, dst, t);
        }
    }
}

// Inverse column pass whose outputs may be fed by several terms (y pass only):
// out[d] = IDFT(sum over the terms of d of mult * in[src]), the sum formed before
// the inverse DFT (linear); each term reads its source tile.  A kernel of its
// own, so that the one-term-per-output pass above keeps its register budget.
template <typename T, int N>
__global__ void __launch_bounds__(Tile<T, N, false>::NT, 1) k_col_inv_acc(const PassProgram P, const KParams kp) {
    using TL = Tile<T, N, false>;
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int t = threadIdx.x, chain = blockIdx.y;
    int kz, c0;
    TL::tile_pos(blockIdx.x, kz, c0);
    const size_t base = TL::tile_base(kz, c0);
    const int g = TL::b_g(t);
    for (int d = 0; d < P.n_out; ++d) {
        V Y[TL::J][TL::N2];
#pragma unroll
        for (int j = 0; j < TL::J; ++j)
#pragma unroll
            for (int k2 = 0; k2 < TL::N2; ++k2) Y[j][k2] = cmake<V>(T(0), T(0));
        bool any = false;
        for (int m = 0; m < P.n_expand; ++m) {
            const Term tm = P.expand[m];
            if (tm.dst != d) continue;
            any = true;
            const V* src = reinterpret_cast<const V*>(P.in[tm.src]) + chain * P.in_cs + base;
#pragma unroll
            for (int j = 0; j < TL::J; ++j) {
                const int k1 = TL::b_k1(t, j);
#pragma unroll
                for (int k2 = 0; k2 < TL::N2; ++k2) {
                    int mx, my, mz;
                    TL::freqs(k1 + TL::N1 * k2, g, kz, c0, mx, my, mz);
                    Y[j][k2] = cadd(Y[j][k2], cmul(ymult<T>(tm, my, mz, N, kp), src[TL::goff(k1 + TL::N1 * k2, g)]));
                }
            }
        }
        if (!any) continue;
        __syncthreads();
        TL::invB(Y, sm, t);
        __syncthreads();
        TL::invA(sm, reinterpret_cast<V*>(P.out[d]) + chain * P.out_cs + base, t);
    }
}

// x node: Q = sum_merge mult * DFTx(in[src]);  out[dst] = IDFTx(mult * Q).
// Within a tile every thread has one (ky, kz), so each term's ky/kz powers and
// complex coefficient fold into one per-thread constant; per element only the
// kx power and the radial factor remain.  Radial factors other than 1/k^2 come
// from the per-context tables indexed by m^2 (exact, no transcendental work in
// the kernel).  In FP32, 1/k^2 is 1/kf^2 divided by the exact integer m^2 with
// the hardware reciprocal (within 2 ulp), which spares a gather whose addresses
// differ in every lane.
//
// The ALPT blend K(k) = exp(-r_s^2 k^2 / 2) (Sect. 2.3) is a product of an x
// factor and a (y, z) factor.  In FP32 the x factor comes from a per-CTA
// shared-memory copy of K at m^2 = mx^2 and the (y, z) factor, K at
// m^2 = my^2 + mz^2, is one per-thread constant; 1 - K is formed from that
// product.  Both factors are entries of the same FP64-computed table.
template <typename T> struct XTerm {
    T cr, ci;          // (cre + i cim) ky^py kz^pz
    T kyz;             // K at m^2 = my^2 + mz^2 (FP32 blend codes)
    int px, rcode;
};
template <typename T> __device__ __forceinline__ bool sep_blend(int rcode) {
    return sizeof(T) == 4 && (rcode == R_KBLEND || rcode == R_1MKBLEND);
}
template <typename T>
__device__ __forceinline__ XTerm<T> xterm(const Term& tm, int my, int mz, int n, const KParams& kp) {
    const T kf = kf_of<T>(kp);
    const T cyz = kpow<T>(my, tm.py, n, kf) * kpow<T>(mz, tm.pz, n, kf);
    const T kyz = sep_blend<T>(tm.rcode)
                      ? __ldg(reinterpret_cast<const T*>(kp.rtab) + (R_KBLEND - 1) * kp.rlen + my * my + mz * mz)
                      : T(0);
    return XTerm<T>{T(tm.cre) * cyz, T(tm.cim) * cyz, kyz, tm.px, tm.rcode};
}
// multiplier of element mx (x index ix); m2yz = my^2 + mz^2; skx: the CTA's
// K(mx^2) by x index (filled when the program has FP32 blend codes)
template <typename T>
__device__ __forceinline__ cplx_t<T> xmult(const XTerm<T>& x, int mx, int ix, int m2yz, int n, const KParams& kp,
                                           const T* skx) {
    T r = kpow<T>(mx, x.px, n, kf_of<T>(kp));
    if (x.rcode != R_ONE) {
        const int m2 = mx * mx + m2yz;
        if (sizeof(T) == 4 && x.rcode == R_INVK2) {
            r *= m2 > 0 ? T(__fdividef(kp.inv_kf2_f, float(m2))) : T(0);
        } else if (sep_blend<T>(x.rcode)) {
            const T k = skx[ix] * x.kyz;
            r *= x.rcode == R_KBLEND ? k : T(1) - k;
        } else {
            r *= __ldg(reinterpret_cast<const T*>(kp.rtab) + (x.rcode - 1) * kp.rlen + m2);
        }
    }
    return cmake<cplx_t<T>>(x.cr * r, x.ci * r);
}

#ifndef BRIDGE_XNODE_MINB
#define BRIDGE_XNODE_MINB 2
#endif
// FP32: as many CTAs per SM as fit 2 x 256 threads (the register budget of 128 per thread)
template <typename T, int N> constexpr int xnode_minb() {
    return sizeof(T) == 4 ? BRIDGE_XNODE_MINB * 256 / Tile<T, N, true>::NT : BRIDGE_XNODE_MINB;
}
template <typename T, int N>
__global__ void __launch_bounds__(Tile<T, N, true>::NT, (xnode_minb<T, N>())) k_x_node(const PassProgram P, const KParams kp) {
    using TL = Tile<T, N, true>;
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int t = threadIdx.x, chain = blockIdx.y;
    int kz, c0;
    TL::tile_pos(blockIdx.x, kz, c0);
    const size_t base = TL::tile_base(kz, c0);
    const int g = TL::b_g(t);
    const int my = signed_freq(c0 + g, N), mz = kz;
    const int m2yz = my * my + mz * mz;
    // x factor of the blend, when a term of the program uses it
    T* skx = reinterpret_cast<T*>(sm + TL::SM_ELEMS + TL::STAGE_ELEMS);
    bool blend = false;
    for (int m = 0; m < P.n_merge; ++m) blend |= sep_blend<T>(P.merge[m].rcode);
    for (int m = 0; m < P.n_expand; ++m) blend |= sep_blend<T>(P.expand[m].rcode);
    if (blend) {
        const T* ktab = reinterpret_cast<const T*>(kp.rtab) + (R_KBLEND - 1) * kp.rlen;
        for (int ix = t; ix < N; ix += TL::NT) {
            const int mx = signed_freq(ix, N);
            skx[ix] = __ldg(ktab + mx * mx);
        }
        __syncthreads();
    }
    V Q[TL::J][TL::N2];   // bit-reversed k2 order
#pragma unroll
    for (int j = 0; j < TL::J; ++j)
#pragma unroll
        for (int i = 0; i < TL::N2; ++i) Q[j][i] = cmake<V>(T(0), T(0));
    // the tile of input m + 1 is copied into shared memory while input m is transformed
    V* buf = sm + TL::SM_ELEMS;
    auto src_of = [&](int m) { return reinterpret_cast<const V*>(P.in[P.merge[m].src]) + chain * P.in_cs + base; };
    if (P.n_merge > 0) TL::stage(src_of(0), buf, t);
    for (int m = 0; m < P.n_merge; ++m) {
        const Term tm = P.merge[m];
        const XTerm<T> xt = xterm<T>(tm, my, mz, N, kp);
        cp_async_wait_all();
        __syncthreads();
        TL::fwdA_staged(buf, sm, t);
        __syncthreads();
        if (m + 1 < P.n_merge) TL::stage(src_of(m + 1), buf, t);
        V X[TL::J][TL::N2];
        TL::fwdB(sm, t, X);
        const bool spec = xdispatch<T, N>(tm, [&](auto pxc, auto rcc) {
            constexpr int PX = decltype(pxc)::value, RC = decltype(rcc)::value;
#pragma unroll
            for (int j = 0; j < TL::J; ++j) {
                const int k1 = TL::b_k1(t, j);
                sfor<0, TL::N2>([&](auto ic) {
                    constexpr int i = decltype(ic)::value;
                    const T r = xfac<T, N, PX, RC, TL::N1 * bitrev(i, TL::N2)>(k1, m2yz, kp, skx, xt.kyz);
                    Q[j][i] = cadd(Q[j][i], cmul(cmake<V>(xt.cr * r, xt.ci * r), X[j][i]));
                });
            }
        });
        if (!spec) {
#pragma unroll
            for (int j = 0; j < TL::J; ++j) {
                const int k1 = TL::b_k1(t, j);
#pragma unroll
                for (int i = 0; i < TL::N2; ++i) {
                    const int ix = k1 + TL::N1 * bitrev(i, TL::N2);
                    Q[j][i] = cadd(Q[j][i], cmul(xmult<T>(xt, signed_freq(ix, N), ix, m2yz, N, kp, skx), X[j][i]));
                }
            }
        }
    }
    for (int m = 0; m < P.n_expand; ++m) {
        const Term tm = P.expand[m];
        const XTerm<T> xt = xterm<T>(tm, my, mz, N, kp);
        V Y[TL::J][TL::N2];   // natural k2 order
        const bool spec = xdispatch<T, N>(tm, [&](auto pxc, auto rcc) {
            constexpr int PX = decltype(pxc)::value, RC = decltype(rcc)::value;
#pragma unroll
            for (int j = 0; j < TL::J; ++j) {
                const int k1 = TL::b_k1(t, j);
                sfor<0, TL::N2>([&](auto ic) {
                    constexpr int k2 = decltype(ic)::value;
                    const T r = xfac<T, N, PX, RC, TL::N1 * k2>(k1, m2yz, kp, skx, xt.kyz);
                    Y[j][k2] = cmul(cmake<V>(xt.cr * r, xt.ci * r), Q[j][bitrev(k2, TL::N2)]);
                });
            }
        });
        if (!spec) {
#pragma unroll
            for (int j = 0; j < TL::J; ++j) {
                const int k1 = TL::b_k1(t, j);
#pragma unroll
                for (int k2 = 0; k2 < TL::N2; ++k2) {
                    const int ix = k1 + TL::N1 * k2;
                    Y[j][k2] = cmul(xmult<T>(xt, signed_freq(ix, N), ix, m2yz, N, kp, skx), Q[j][bitrev(k2, TL::N2)]);
                }
            }
        }
        __syncthreads();
        TL::invB(Y, sm, t);
        __syncthreads();
        V* dst = reinterpret_cast<V*>(P.out[tm.dst]) + chain * P.out_cs + base;
        TL::invA(sm, dst, t);
    }
}

// ---------------------------------------------------------------------------
// stand-alone z passes (whole fields), tile functions in ztile.cuh
// ---------------------------------------------------------------------------
template <typename T, int N> using ZPass = ZCfg<T, N, 256 / (8 * Split<N>::N2)>;

#ifndef BRIDGE_ZFWD_MINB
#define BRIDGE_ZFWD_MINB 5   // FP32 up to N = 256: 48 registers, no spills, 0.351 -> 0.337 ms at 256^3 (the inverse pass loses at 5; 512 would spill)
#endif
#ifndef BRIDGE_ZINV_MINB
#define BRIDGE_ZINV_MINB 0   // 0: register count left to the compiler
#endif
template <typename T, int N>
__global__ void __launch_bounds__(ZPass<T, N>::NT, (sizeof(T) == 4 && N <= 256) ? BRIDGE_ZFWD_MINB : 0) k_z_fwd(const ZProgram P) {
    using ZT = ZPass<T, N>;
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int f = blockIdx.y, chain = blockIdx.z;
    int x0, y0;
    ZT::tile_xy(blockIdx.x, x0, y0);
    const T* rin = reinterpret_cast<const T*>(P.in[f]) + chain * P.in_cs;
    auto line = [&](int c) { return rin + (size_t(x0 + 2 * (c % 8)) * N + y0 + c / 8) * N; };
    ztile_fwd<ZT>(line, (long long)N * N, reinterpret_cast<V*>(P.out[f]) + chain * P.out_cs, x0, y0, sm,
                  threadIdx.x);
}

// Stores out[p] = v - sub[p] (the subtrahend read through the read-only path).
template <typename T> struct SubLineIO {
    const T* out;
    const T* sub;
    template <typename U> __device__ __forceinline__ void st(U* p, U v) const { *p = v - __ldg(sub + (p - out)); }
};

template <typename T, int N, bool SUB>
__global__ void __launch_bounds__(ZPass<T, N>::NT, BRIDGE_ZINV_MINB) k_z_inv(const ZProgram P) {
    using ZT = ZPass<T, N>;
    using V = cplx_t<T>;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int f = blockIdx.y, chain = blockIdx.z;
    int x0, y0;
    ZT::tile_xy(blockIdx.x, x0, y0);
    T* rout = reinterpret_cast<T*>(P.out[f]) + chain * P.out_cs;
    auto line = [&](int c) { return rout + (size_t(x0 + 2 * (c % 8)) * N + y0 + c / 8) * N; };
    const V* spec = reinterpret_cast<const V*>(P.in[f]) + chain * P.in_cs;
    if constexpr (SUB) {
        const SubLineIO<T> io{rout, reinterpret_cast<const T*>(P.sub[f]) + chain * P.out_cs};
        ztile_inv<ZT, decltype(line), false, SubLineIO<T>>(spec, line, (long long)N * N, x0, y0, sm, threadIdx.x, io);
    } else {
        ztile_inv<ZT>(spec, line, (long long)N * N, x0, y0, sm, threadIdx.x);
    }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <typename K> static cudaError_t set_smem(K kernel, size_t bytes) {
    if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, int(bytes));
    return cudaSuccess;
}

// Mesh sizes compiled in.
#ifndef BRIDGE_ONLY_N
#define BRIDGE_N_SWITCH(n, T, CALL)                                   \
    switch (n) {                                                      \
        case 16: { constexpr int NN = 16; CALL; }                     \
        case 32: { constexpr int NN = 32; CALL; }                     \
        case 64: { constexpr int NN = 64; CALL; }                     \
        case 128: { constexpr int NN = 128; CALL; }                   \
        case 256: { constexpr int NN = 256; CALL; }                   \
        case 512: { constexpr int NN = 512; CALL; }                   \
        default: return cudaErrorInvalidValue;                        \
    }
#else
#define BRIDGE_N_SWITCH(n, T, CALL)                                   \
    switch (n) {                                                      \
        case BRIDGE_ONLY_N: { constexpr int NN = BRIDGE_ONLY_N; CALL; } \
        default: return cudaErrorInvalidValue;                        \
    }
#endif

template <typename T, int N> static cudaError_t z_fwd_n(int batch, const ZProgram& p, cudaStream_t s) {
    using ZT = ZPass<T, N>;
    const size_t sm = size_t(ZT::SM_ELEMS) * sizeof(cplx_t<T>);
    cudaError_t e = set_smem(k_z_fwd<T, N>, sm);
    if (e != cudaSuccess) return e;
    k_z_fwd<T, N><<<dim3(ZT::TILES, p.n_fields, batch), ZT::NT, sm, s>>>(p);
    return cudaGetLastError();
}
template <typename T, int N, bool SUB> static cudaError_t z_inv_nk(int batch, const ZProgram& p, cudaStream_t s) {
    using ZT = ZPass<T, N>;
    const size_t sm = size_t(ZT::SM_ELEMS) * sizeof(cplx_t<T>);
    cudaError_t e = set_smem(k_z_inv<T, N, SUB>, sm);
    if (e != cudaSuccess) return e;
    k_z_inv<T, N, SUB><<<dim3(ZT::TILES, p.n_fields, batch), ZT::NT, sm, s>>>(p);
    return cudaGetLastError();
}
template <typename T, int N> static cudaError_t z_inv_n(int batch, const ZProgram& p, cudaStream_t s) {
    if (p.sub[0]) {
        for (int f = 0; f < p.n_fields; ++f)
            if (!p.sub[f]) return cudaErrorInvalidValue;
        return z_inv_nk<T, N, true>(batch, p, s);
    }
    return z_inv_nk<T, N, false>(batch, p, s);
}
template <typename T, int N, bool XM, bool FWD>
static cudaError_t col_n(int batch, const PassProgram& p, const KParams& kp, cudaStream_t s) {
    using TL = Tile<T, N, XM>;
    const size_t sm = size_t(TL::SM_ELEMS + (FWD ? TL::STAGE_ELEMS : 0)) * sizeof(cplx_t<T>);
    auto kern = FWD ? k_col_fwd<T, N, XM> : (!XM && p.accumulate ? k_col_inv_acc<T, N> : k_col_inv<T, N, XM>);
    cudaError_t e = set_smem(kern, sm);
    if (e != cudaSuccess) return e;
    if (FWD) {
        // merge terms grouped by output, in their original order within each output
        PassProgram q = p;
        int k = 0;
        for (int o = 0; o < p.n_out; ++o)
            for (int m = 0; m < p.n_merge; ++m)
                if (p.merge[m].dst == o) q.merge[k++] = p.merge[m];
        q.n_merge = k;
        kern<<<dim3(TL::TILES, batch), TL::NT, sm, s>>>(q, kp);
    } else {
        kern<<<dim3(TL::TILES, batch), TL::NT, sm, s>>>(p, kp);
    }
    return cudaGetLastError();
}
template <typename T, int N> static cudaError_t xnode_n(int batch, const PassProgram& p, const KParams& kp, cudaStream_t s) {
    using TL = Tile<T, N, true>;
    const size_t sm = size_t(TL::SM_ELEMS + TL::STAGE_ELEMS) * sizeof(cplx_t<T>) + N * sizeof(T);
    cudaError_t e = set_smem(k_x_node<T, N>, sm);
    if (e != cudaSuccess) return e;
    k_x_node<T, N><<<dim3(TL::TILES, batch), TL::NT, sm, s>>>(p, kp);
    return cudaGetLastError();
}

template <typename T> cudaError_t launch_z_fwd(int n, int batch, const ZProgram& p, cudaStream_t s) {
    BRIDGE_N_SWITCH(n, T, return (z_fwd_n<T, NN>(batch, p, s)));
}
template <typename T> cudaError_t launch_z_inv(int n, int batch, const ZProgram& p, cudaStream_t s) {
    BRIDGE_N_SWITCH(n, T, return (z_inv_n<T, NN>(batch, p, s)));
}
template <typename T> cudaError_t launch_y_fwd(int n, int batch, const PassProgram& p, const KParams& kp, cudaStream_t s) {
    BRIDGE_N_SWITCH(n, T, return (col_n<T, NN, false, true>(batch, p, kp, s)));
}
template <typename T> cudaError_t launch_y_inv(int n, int batch, const PassProgram& p, const KParams& kp, cudaStream_t s) {
    BRIDGE_N_SWITCH(n, T, return (col_n<T, NN, false, false>(batch, p, kp, s)));
}
template <typename T> cudaError_t launch_x_node(int n, int batch, const PassProgram& p, const KParams& kp, cudaStream_t s) {
    BRIDGE_N_SWITCH(n, T, return (xnode_n<T, NN>(batch, p, kp, s)));
}

#define BRIDGE_INST(T)                                                                                       \
    template cudaError_t launch_z_fwd<T>(int, int, const ZProgram&, cudaStream_t);                           \
    template cudaError_t launch_z_inv<T>(int, int, const ZProgram&, cudaStream_t);                           \
    template cudaError_t launch_y_fwd<T>(int, int, const PassProgram&, const KParams&, cudaStream_t);        \
    template cudaError_t launch_y_inv<T>(int, int, const PassProgram&, const KParams&, cudaStream_t);        \
    template cudaError_t launch_x_node<T>(int, int, const PassProgram&, const KParams&, cudaStream_t);
BRIDGE_INST(float)
BRIDGE_INST(double)

}  // namespace bridge
