// Real-space kernels: ALPT sources and adjoint (Sect. 2.3), CIC mass assignment
// and its gather adjoint, the fused eigenvalue / fuzzy-web / bias pass and its
// adjoint (Sect. 2.5-2.8, App. B), the NB likelihood (Sect. 2.6), deterministic
// FP64 reductions and the leapfrog updates (Sect. 2.2).
#include <cmath>

#include "common.cuh"
#include "pointwise.cuh"

namespace bridge {

// Thread-block partial sums: each thread accumulates its voxels, then a fixed
// warp-shuffle + shared-memory tree; thread 0 writes partial[chain][block][k].
template <int K>
__device__ __forceinline__ void write_partials(const double (&acc)[K], double* partial) {
    __shared__ double sh[kPwThreads / 32];
#pragma unroll 1
    for (int k = 0; k < K; ++k) {
        double r = block_sum<kPwThreads>(acc[k], sh);
        if (threadIdx.x == 0)
            partial[((size_t)blockIdx.y * gridDim.x + blockIdx.x) * K + k] = r;
    }
}

__device__ void reduce_body(int what, int chain, int nblk, int K, const double* partial, ChainScalars* sc,
                            const BiasD* bias, int n_regions);

// Partial sums of this block, then the last block of the chain to finish (a
// ticket counter) reduces all of them with reduce_body and resets the counter.
template <int K>
__device__ __forceinline__ void finish_partials(const double (&acc)[K], double* partial, int what, const RedArgs& ra) {
    write_partials<K>(acc, partial);
    __shared__ int last;
    __threadfence();   // this block's partials are visible before its ticket is taken
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(ra.tickets + blockIdx.y, 1) == (int)gridDim.x - 1;
    __syncthreads();
    if (last) {
        __threadfence();
        reduce_body(what, blockIdx.y, gridDim.x, K, partial, ra.sc, ra.bias, ra.n_regions);
        if (threadIdx.x == 0) ra.tickets[blockIdx.y] = 0;
    }
}

#define PW_LOOP(i, nvox) for (long long i = (long long)blockIdx.x * kPwThreads + threadIdx.x; i < (nvox); \
                              i += (long long)gridDim.x * kPwThreads)

// ---------------------------------------------------------------------------
// counts: int32 -> uint16 with range check; N_tr partial sums
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(kPwThreads) k_counts_prep(long long nvox, const int32_t* __restrict__ counts,
                                                           uint16_t* __restrict__ c16, double* partial, int* err,
                                                           RedArgs ra) {
    const size_t off = (size_t)blockIdx.y * nvox;
    double acc[1] = {0.0};
    long long s = 0;
    int bad = 0;
    // four counts per 16-byte load (nvox is a multiple of 4)
    const int4* c4 = reinterpret_cast<const int4*>(counts + off);
    ushort4* o4 = reinterpret_cast<ushort4*>(c16 + off);
    PW_LOOP(i, nvox / 4) {
        const int4 v = c4[i];
        int q[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (q[k] < 0 || q[k] > 65535) { bad = 1; q[k] = 0; }
            s += q[k];
        }
        o4[i] = make_ushort4((uint16_t)q[0], (uint16_t)q[1], (uint16_t)q[2], (uint16_t)q[3]);
    }
    if (bad) atomicOr(err, 1);
    acc[0] = (double)s;
    finish_partials<1>(acc, partial, RED_NTR, ra);
}

// Constant fill (the CIC mass is zeroed before each scatter).
template <typename T> __global__ void k_fill(long long count, T* p, T v) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        p[i] = v;
}

// ---------------------------------------------------------------------------
// CIC (mass assignment): the particle of cell q sits at q + psi (cell units);
// trilinear weights to the 8 surrounding cells, periodic.  The kernel
// accumulates the mass rho = 1 + delta (one particle per cell) into a zeroed
// field: small masses keep full relative precision, which the likelihood
// needs (d ln nbar / d rho ~ alpha / rho in nearly empty cells).  The spectra of
// rho and delta differ only at k = 0, where every tensor operator vanishes.
// ---------------------------------------------------------------------------
// The deposit runs over blocks of BX x BY x BZ particles (BZ consecutive z per
// warp, so the displacement loads are contiguous).  Each block accumulates the
// cells [x0-H, x0+BX+H) x [y0-H, y0+BY+H) x [z0-H, z0+BZ+H) in a shared-memory
// window; a particle whose 2x2x2 footprint leaves the window (|psi| beyond
// about H cells) adds straight to rho.  The window is then added to rho in
// aligned groups of four z cells (one 16-byte vector atomic for FP32, zero
// groups skipped): several times fewer global atomics than one per corner.
// FP32 windows hold fixed-point sums (weight * 2^40, exact integer adds) as
// two 32-bit counters per cell, the high and low 20 bits of each term, because
// shared-memory 32-bit integer adds run about six times faster than float or
// 64-bit adds (measured); the pair is combined and converted to FP32 once at
// the flush, so the deposit is at least as accurate as FP32 atomics (up to
// 4095 terms per cell).  No FP64 arithmetic: GB300's FP64 rate is low.  FP64 windows hold doubles.  Needs BX, BY, BZ <= N;
// windows of blocks near the periodic edges overlap, which the atomics absorb.
template <typename T> struct CicBlock;
template <> struct CicBlock<float> { static constexpr int BX = 8, BY = 8, H = 4; };    // 16x16x40 cells, 80 KB at BZ = 32
template <> struct CicBlock<double> { static constexpr int BX = 8, BY = 8, H = 4; };   // 80 KB at BZ = 32

// Shared-memory window of `cells` cells, 8 bytes per cell.  FP32: the term
// w * 2^40 is split in FP32 arithmetic into its integer part above 2^20
// (hi = floor(w 2^20)) and the next 20 bits (lo, rounded), each added to its
// own 32-bit counter; the flush forms hi 2^-20 + lo 2^-40.
template <typename T> struct CicWin;
template <> struct CicWin<float> {
    unsigned* hi;
    unsigned* lo;
    __device__ CicWin(unsigned char* raw, int cells)
        : hi(reinterpret_cast<unsigned*>(raw)), lo(reinterpret_cast<unsigned*>(raw) + cells) {}
    __device__ void zero(int i) { hi[i] = 0u; lo[i] = 0u; }
    __device__ void add(int i, float w) {   // 0 <= w <= 1
        const float s = w * 1048576.0f;      // 2^20, exact
        const float h = floorf(s);
        atomicAdd(lo + i, __float2uint_rn((s - h) * 1048576.0f));
        atomicAdd(hi + i, (unsigned)h);
    }
    __device__ float get(int i) const {
        return float(hi[i]) * 9.5367431640625e-07f + float(lo[i]) * 9.094947017729282e-13f;   // 2^-20, 2^-40
    }
};
template <> struct CicWin<double> {
    double* w;
    __device__ CicWin(unsigned char* raw, int) : w(reinterpret_cast<double*>(raw)) {}
    __device__ void zero(int i) { w[i] = 0.0; }
    __device__ void add(int i, double v) { atomicAdd(w + i, v); }
    __device__ double get(int i) const { return w[i]; }
};

__device__ __forceinline__ void cic_flush4(float* g, const CicWin<float>& W, int i) {
    const float4 v = make_float4(W.get(i), W.get(i + 1), W.get(i + 2), W.get(i + 3));
    if (v.x != 0.f || v.y != 0.f || v.z != 0.f || v.w != 0.f) atomicAdd(reinterpret_cast<float4*>(g), v);
}
__device__ __forceinline__ void cic_flush4(double* g, const CicWin<double>& W, int i) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const double v = W.get(i + q);
        if (v != 0.0) atomicAdd(g + q, v);
    }
}

// Where a particle's weights go.  CicFloat: float (or double) atomics into rho, the
// window flushed with vector atomics; the sum order varies from run to run.
// CicFixed: 64-bit fixed-point integers (FP32: the window's exact 2^-40 units; FP64:
// units of 2^-50, weights rounded once), whose sums do not depend on the order, so the
// mass assignment is bit-reproducible; k_fixed_to_mass converts afterwards.
template <typename T> struct CicFloat {
    T* r;
    __device__ void add(size_t i, T w) const { atomicAdd(r + i, w); }
    __device__ void flush4(size_t i, const CicWin<T>& W, int wi) const { cic_flush4(r + i, W, wi); }
};
template <typename T> struct CicFixedScale;
template <> struct CicFixedScale<float> { static constexpr int S = 40; };
template <> struct CicFixedScale<double> { static constexpr int S = 50; };
__device__ __forceinline__ unsigned long long fixed_units(float w) {   // the window's split: hi 2^20 + lo
    const float s = w * 1048576.0f;
    const float h = floorf(s);
    return ((unsigned long long)h << 20) + __float2uint_rn((s - h) * 1048576.0f);
}
__device__ __forceinline__ unsigned long long fixed_units(double w) { return __double2ull_rn(w * 1125899906842624.0); }   // 2^50
// FP64 windows of the fixed-point mode hold the integer units themselves
struct CicWinFx64 {
    unsigned long long* w;
    __device__ CicWinFx64(unsigned char* raw, int) : w(reinterpret_cast<unsigned long long*>(raw)) {}
    __device__ void zero(int i) { w[i] = 0ull; }
    __device__ void add(int i, double v) { atomicAdd(w + i, fixed_units(v)); }
    __device__ unsigned long long units(int i) const { return w[i]; }
};
template <typename T> struct CicFixed {
    unsigned long long* r;
    __device__ void add(size_t i, T w) const { atomicAdd(r + i, fixed_units(w)); }
    template <typename W> __device__ void flush4(size_t i, const W& win, int wi) const {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            unsigned long long v;
            if constexpr (sizeof(T) == 4) v = ((unsigned long long)win.hi[wi + q] << 20) + win.lo[wi + q];
            else v = win.units(wi + q);
            if (v != 0ull) atomicAdd(r + i + q, v);
        }
    }
};
template <typename T, bool FX> struct CicOut;
template <typename T> struct CicOut<T, false> { using type = CicFloat<T>; using win = CicWin<T>; };
template <> struct CicOut<float, true> { using type = CicFixed<float>; using win = CicWin<float>; };
template <> struct CicOut<double, true> { using type = CicFixed<double>; using win = CicWinFx64; };

// rho = units 2^-S, per chain; FP32 without FP64 arithmetic (two exact 32-bit halves).
template <typename T> __global__ void k_fixed_to_mass(long long count, const unsigned long long* acc, T* rho) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long v = acc[i];
        if constexpr (sizeof(T) == 4)
            rho[i] = __fmaf_rn(float(unsigned(v >> 32)), 0.00390625f, float(unsigned(v & 0xffffffffull)) * 9.094947017729282e-13f);   // 2^32 2^-40, 2^-40
        else
            rho[i] = double(v) * 8.881784197001252e-16;   // 2^-50
    }
}

#ifndef BRIDGE_CIC_BZ
#define BRIDGE_CIC_BZ 16   // particle block depth along z: 16 gives 16 x 16 x 24-cell windows (48 KB, four CTAs
                           // per SM), 0.33 -> 0.22 ms at 256^3 against 32 (80 KB, two CTAs per SM)
#endif
template <typename T, int BZ, bool FX, typename OutT>
__global__ void __launch_bounds__(kPwThreads) k_cic_scatter(int N, long long nvox, Fields16 psi3, OutT* out_base) {
    using CB = CicBlock<T>;
    constexpr int BX = CB::BX, BY = CB::BY, H = CB::H;
    constexpr int WX = BX + 2 * H, WY = BY + 2 * H, WZ = BZ + 2 * H, CELLS = WX * WY * WZ;
    static_assert(WZ % 4 == 0 && H % 4 == 0, "window rows are groups of four cells");
    extern __shared__ __align__(16) unsigned char smraw[];
    typename CicOut<T, FX>::win W(smraw, CELLS);
    const int t = threadIdx.x;
    const size_t off = (size_t)blockIdx.y * nvox;
    const T* p0 = (const T*)psi3.p[0] + off;
    const T* p1 = (const T*)psi3.p[1] + off;
    const T* p2 = (const T*)psi3.p[2] + off;
    const typename CicOut<T, FX>::type out{out_base + off};
    const int msk = N - 1;
    const int nbz = N / BZ, nby = N / BY;
    const int b = blockIdx.x;
    const int x0 = (b / (nbz * nby)) * BX, y0 = ((b / nbz) % nby) * BY, z0 = (b % nbz) * BZ;
    for (int i = t; i < CELLS; i += kPwThreads) W.zero(i);
    __syncthreads();
    for (int p = t; p < BX * BY * BZ; p += kPwThreads) {
        const int z = z0 + p % BZ, y = y0 + (p / BZ) % BY, x = x0 + p / (BZ * BY);
        const size_t q = ((size_t)x * N + y) * N + z;
        CicCorner<T> c;
        cic_corner<T>((long long)q, N, p0[q], p1[q], p2[q], c);
        // window coordinates of the lower corner (unwrapped)
        const int wx = c.i0[0] - (x0 - H), wy = c.i0[1] - (y0 - H), wz = c.i0[2] - (z0 - H);
        const bool inside = wx >= 0 && wx + 1 < WX && wy >= 0 && wy + 1 < WY && wz >= 0 && wz + 1 < WZ;
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            const T fx = a ? c.f[0] : T(1) - c.f[0];
#pragma unroll
            for (int bb = 0; bb < 2; ++bb) {
                const T fxy = fx * (bb ? c.f[1] : T(1) - c.f[1]);
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const T w = fxy * (e ? c.f[2] : T(1) - c.f[2]);
                    if (inside)
                        W.add(((wx + a) * WY + (wy + bb)) * WZ + wz + e, w);
                    else
                        out.add(((size_t)((c.i0[0] + a) & msk) * N + ((c.i0[1] + bb) & msk)) * N + ((c.i0[2] + e) & msk), w);
                }
            }
        }
    }
    __syncthreads();
    // flush: groups of four z cells; (z0 - H) is a multiple of 4 and so is N
    constexpr int G = WZ / 4;
    for (int i = t; i < WX * WY * G; i += kPwThreads) {
        const int g = i % G, col = i / G;
        const int wy = col % WY, wx = col / WY;
        const int gx = (x0 - H + wx) & msk, gy = (y0 - H + wy) & msk, gz = (z0 - H + 4 * g) & msk;
        out.flush4(((size_t)gx * N + gy) * N + gz, W, col * WZ + 4 * g);
    }
}

// ---------------------------------------------------------------------------
// Fused web + bias, forward (pass A): eigenvalues of T (and H), memberships,
// per-voxel parameters, ln f and beta_i; partial sums of f.
// ---------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ void load6(const Fields16& f, int base, size_t j, T out[6]) {
#pragma unroll
    for (int q = 0; q < 6; ++q) out[q] = ((const T*)f.p[base + q])[j];
}

template <typename T, int NR>
__device__ __forceinline__ void web_forward(const Fields16& th, size_t j, T rho_mass, const BiasT<T>& B,
                                            const WebParams& wp, WebState<T, NR>& S) {
    T a6[6], h6[6];
    load6<T>(th, 0, j, a6);
    if constexpr (NR == 16) load6<T>(th, 6, j, h6);
    web_eval<T, NR>(a6, h6, rho_mass, B, wp, S);
}

#ifndef BRIDGE_PASSA_MINB
#define BRIDGE_PASSA_MINB 0   // 0: register count left to the compiler
#endif
#ifndef BRIDGE_PASSB_MINB
#define BRIDGE_PASSB_MINB 0
#endif
template <typename T, int NR>
__global__ void __launch_bounds__(kPwThreads, BRIDGE_PASSA_MINB) k_pass_a(long long nvox, Fields16 th, const T* rho, T* lnf_out,
                                                      T* beta_out, const BiasT<T>* bias, WebParams wp, double* partial,
                                                      RedArgs ra) {
    __shared__ BiasT<T> B;
    const int chain = blockIdx.y;
    if (threadIdx.x == 0) B = bias[chain];
    __syncthreads();
    const size_t off = (size_t)chain * nvox;
    T accf = T(0);
    double acc[1];
    double accd = 0.0;
    int cnt = 0;
    PW_LOOP(i, nvox) {
        const size_t j = off + i;
        // re-derive the table pointer each voxel so its 112 entries are read from
        // shared memory when used instead of being kept live in registers
        const BiasT<T>* Bp = &B;
        asm volatile("" : "+l"(Bp));
        WebState<T, NR> S;
        web_forward<T, NR>(th, j, rho[j], *Bp, wp, S);
        lnf_out[j] = S.lf.lnf;
        beta_out[j] = S.q.beta;
        accf += v_exp(S.lf.lnf);
        if (++cnt == 16) { accd += (double)accf; accf = T(0); cnt = 0; }
    }
    acc[0] = accd + (double)accf;
    finish_partials<1>(acc, partial, RED_SUMF, ra);
}

// NB likelihood (pass B): ln nbar = ln f + ln C; partial sums of log P,
// d log P/d ln nbar and nu^2.  Four voxels per thread and iteration (16-byte
// loads of ln f, beta, nu; 8-byte load of the counts).
template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4_32a; };

template <typename T>
__global__ void __launch_bounds__(kPwThreads, BRIDGE_PASSB_MINB) k_pass_b(long long nvox, const T* lnf, const T* beta_i,
                                                      const uint16_t* c16, const T* nu, const ChainScalars* sc,
                                                      double* partial, RedArgs ra) {
    using V4 = typename Vec4<T>::type;
    const int chain = blockIdx.y;
    const size_t off = (size_t)chain * nvox;
    const T lnC = T(sc[chain].lnC);
    T a0 = 0, a1 = 0, a2 = 0;
    double acc[3] = {0.0, 0.0, 0.0};
    const long long n4 = nvox / 4;
    const V4* lf4 = reinterpret_cast<const V4*>(lnf + off);
    const V4* bt4 = reinterpret_cast<const V4*>(beta_i + off);
    const V4* nu4 = reinterpret_cast<const V4*>(nu + off);
    const ushort4* c4 = reinterpret_cast<const ushort4*>(c16 + off);
    int cnt = 0;
    for (long long i = (long long)blockIdx.x * kPwThreads + threadIdx.x; i < n4; i += (long long)gridDim.x * kPwThreads) {
        const V4 l = lf4[i], b = bt4[i], v = nu4[i];
        const ushort4 c = c4[i];
        const T lv[4] = {l.x, l.y, l.z, l.w}, bv[4] = {b.x, b.y, b.z, b.w}, vv[4] = {v.x, v.y, v.z, v.w};
        const int cv[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            NB<T> r;
            nb_eval<T>(cv[q], lv[q] + lnC, bv[q], true, r);
            a0 += r.logp; a1 += r.g_lnnbar; a2 += vv[q] * vv[q];
        }
        if (++cnt == 4) { acc[0] += a0; acc[1] += a1; acc[2] += a2; a0 = a1 = a2 = T(0); cnt = 0; }
    }
    acc[0] += a0; acc[1] += a1; acc[2] += a2;
    finish_partials<3>(acc, partial, RED_LIK, ra);
}

// ---------------------------------------------------------------------------
// Web + bias + NB adjoint: g_delta (direct), g_T (6), g_H (6) and, when
// requested (BIASG), the partial sums of d/d alpha_r and d/d beta_r.
// ---------------------------------------------------------------------------
#ifndef BRIDGE_WEBADJ_MINB
#define BRIDGE_WEBADJ_MINB 4   // FP32 without bias gradients: 64 registers, no spills, 0.74 -> 0.66 ms at 256^3
#endif
// FP64 and the bias-gradient variant spill more at 64 registers and keep 80 (3 blocks per SM).
template <typename T, bool BIASG> constexpr int webadj_minb() { return sizeof(T) == 4 && !BIASG ? BRIDGE_WEBADJ_MINB : 3; }
template <typename T, int NR, bool BIASG>
__global__ void __launch_bounds__(kPwThreads, (webadj_minb<T, BIASG>())) k_web_adj(long long nvox, Fields16 th, const T* rho,
                                                          const uint16_t* c16, const BiasT<T>* bias, WebParams wp,
                                                          const ChainScalars* sc, Fields16 out, double* partial) {
    __shared__ BiasT<T> B;
    const int chain = blockIdx.y;
    if (threadIdx.x == 0) B = bias[chain];
    __syncthreads();
    const size_t off = (size_t)chain * nvox;
    const T lnC = T(sc[chain].lnC);
    const T gscale = T(sc[chain].gscale);   // f_i/sum f * G = nbar_i * G / N_tr
    constexpr int NG = BIASG ? NR : 1;
    T ga[NG], gb[NG];
#pragma unroll
    for (int r = 0; r < NG; ++r) ga[r] = gb[r] = T(0);
    PW_LOOP(i, nvox) {
        const size_t j = off + i;
        const T dl = rho[j];
        const BiasT<T>* Bp = &B;            // see k_pass_a
        asm volatile("" : "+l"(Bp));
        WebState<T, NR> S;
        web_forward<T, NR>(th, j, dl, *Bp, wp, S);
        T gd, gt[6], gh[6];
        auto reload = [&](T a6[6], T h6[6]) {
            load6<T>(th, 0, j, a6);
            if constexpr (NR == 16) load6<T>(th, 6, j, h6);
        };
        // a second opaque copy, so that the region table is read again here instead of
        // the compiler keeping the 112 values of the forward phase live
        const BiasT<T>* Bq = &B;
        asm volatile("" : "+l"(Bq));
        web_adjoint_voxel<T, NR, BIASG>(S, dl, (int)c16[j], lnC, gscale, *Bq, wp, reload, gd, gt, gh, ga, gb);
        ((T*)out.p[0])[j] = gd;
#pragma unroll
        for (int q = 0; q < 6; ++q) ((T*)out.p[1 + q])[j] = gt[q];
        if constexpr (NR == 16) {
#pragma unroll
            for (int q = 0; q < 6; ++q) ((T*)out.p[7 + q])[j] = gh[q];
        }
    }
    if constexpr (BIASG) {
        double acc[2 * NR];
#pragma unroll
        for (int r = 0; r < NR; ++r) {
            acc[r] = (double)ga[r];
            acc[NR + r] = (double)gb[r];
        }
        write_partials<2 * NR>(acc, partial);
    }
}


// Radial redshift space in place: psi <- psi + f (psi1 . r) r / |r|^2 (see rsd_radial_fwd).
template <typename T>
__global__ void __launch_bounds__(kPwThreads) k_rsd_radial(int N, long long nvox, Fields16 psi, Fields16 psi1, T f) {
    const size_t off = (size_t)blockIdx.y * nvox;
    const int lg = __ffs(N) - 1, msk = N - 1;
    const T c = T(N / 2);
    T* p[3] = {(T*)psi.p[0] + off, (T*)psi.p[1] + off, (T*)psi.p[2] + off};
    const T* p1[3] = {(const T*)psi1.p[0] + off, (const T*)psi1.p[1] + off, (const T*)psi1.p[2] + off};
    PW_LOOP(i, nvox) {
        const int q[3] = {(int)(i >> (2 * lg)), (int)((i >> lg) & msk), (int)(i & msk)};
        const T v[3] = {p[0][i], p[1][i], p[2][i]};
        const T v1[3] = {p1[0][i], p1[1][i], p1[2][i]};
        RsdPoint<T> R;
        T out[3];
        rsd_radial_fwd<T>(q, c, v, v1, f, R, out);
        p[0][i] = out[0];
        p[1][i] = out[1];
        p[2][i] = out[2];
    }
}

template <typename T> __global__ void k_shift(long long count, const T* in, T* out, T c) {
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count; i += (long long)gridDim.x * blockDim.x)
        out[i] = in[i] + c;
}

// Leapfrog (Sect. 2.2): p += ck g; nu += cd p; partial sums of p^2 after the update.
template <typename T>
__global__ void __launch_bounds__(kPwThreads) k_kick_drift(long long nvox, T* p, T* nu, const T* g, T ck, T cd,
                                                          double* partial) {
    const size_t off = (size_t)blockIdx.y * nvox;
    T a = 0;
    double acc[1] = {0.0};
    int cnt = 0;
    PW_LOOP(i, nvox) {
        const size_t j = off + i;
        T pv = p[j] + ck * g[j];
        p[j] = pv;
        if (cd != T(0)) nu[j] += cd * pv;
        a += pv * pv;
        if (++cnt == 16) { acc[0] += a; a = T(0); cnt = 0; }
    }
    acc[0] += a;
    write_partials<1>(acc, partial);
}

// sum a_i b_i per chain: FP64 products, per-thread partials in FP64.
template <typename T>
__global__ void __launch_bounds__(kPwThreads) k_dot(long long nvox, const T* a, const T* b, double* partial, RedArgs ra) {
    const size_t off = (size_t)blockIdx.y * nvox;
    double acc[1] = {0.0};
    PW_LOOP(i, nvox) acc[0] += double(a[off + i]) * double(b[off + i]);
    finish_partials<1>(acc, partial, RED_DOT, ra);
}

// Joint sampling of the free bias parameters in log space (theta = ln b, Sect. 2.1
// Eq. lognormal, Sect. 2.2): with the potential U = -log post - sum theta (the
// Jacobian of b = e^theta), p_theta += ck (b d log post / d b + 1), then theta +=
// cd p_theta, and b = e^theta is written into both copies of the table.  One
// thread per entry of the (untied) free list; gbias holds d log post / d alpha_r
// then d / d beta_r, the log-normal prior included.
template <typename T>
__global__ void k_bias_kick_drift(int nr, uint32_t free_mask, double* theta, double* ptheta, const ChainScalars* sc,
                                  BiasD* bd, BiasT<T>* bt, double ck, double cd) {
    const int c = blockIdx.x, q = threadIdx.x;
    if (q >= 2 * nr || !((free_mask >> q) & 1u)) return;
    const int k = __popc(free_mask & ((1u << q) - 1u));
    double* th = theta + (size_t)c * 32 + k;
    double* pt = ptheta + (size_t)c * 32 + k;
    const double g = exp(*th) * sc[c].gbias[q] + 1.0;
    const double pv = *pt + ck * g;
    *pt = pv;
    const double t = *th + cd * pv;
    *th = t;
    const double b = exp(t);
    const int r = q % nr;
    if (q < nr) { bd[c].alpha[r] = b; bt[c].pk[r][BP_ALPHA] = T(b); }
    else { bd[c].beta[r] = b; bt[c].pk[r][BP_BETA] = T(b); }
}

// Tracer density contrast n* N^3 / N_tr - 1 of each chain (Sect. 2.2 initialisation).
template <typename T> __global__ void k_delta_tr(long long nvox, const uint16_t* c16, const ChainScalars* sc, T* out) {
    const size_t off = (size_t)blockIdx.y * nvox;
    const T scale = T(double(nvox) / sc[blockIdx.y].ntr);
    PW_LOOP(i, nvox) out[off + i] = T(c16[off + i]) * scale - T(1);
}

// g[chain] *= scale[chain] (the cotangent of a vector-Jacobian product).
template <typename T> __global__ void k_scale_chains(long long nvox, T* g, const double* scale) {
    const size_t off = (size_t)blockIdx.y * nvox;
    const T c = T(scale[blockIdx.y]);
    PW_LOOP(i, nvox) g[off + i] *= c;
}

template <typename T>
__global__ void k_lnnbar(long long nvox, const T* lnf, const ChainScalars* sc, T* out) {
    const size_t off = (size_t)blockIdx.y * nvox;
    const T lnC = T(sc[blockIdx.y].lnC);
    PW_LOOP(i, nvox) out[off + i] = lnf[off + i] + lnC;
}

template <typename T>
__global__ void k_eigs(long long nvox, Fields16 t6, Fields16 out3) {
    const size_t off = (size_t)blockIdx.y * nvox;
    PW_LOOP(i, nvox) {
        T a6[6];
        load6<T>(t6, 0, off + i, a6);
        Eig3<T> e;
        eig3<T>(a6, e);
#pragma unroll
        for (int q = 0; q < 3; ++q) ((T*)out3.p[q])[off + i] = e.m + e.mu[q];
    }
}

// ---------------------------------------------------------------------------
// Reductions (one block per chain; fixed order)
// ---------------------------------------------------------------------------
__device__ double lognormal_logpdf(double b, double mu, double sigma) {
    const double lb = log(b);
    return -lb - log(sigma * 2.5066282746310002) - (lb - mu) * (lb - mu) / (2.0 * sigma * sigma);
}
__device__ double lognormal_dlogpdf(double b, double mu, double sigma) {
    const double lb = log(b);
    return -1.0 / b - (lb - mu) / (sigma * sigma * b);
}

// Final reduction of one chain's partial sums (K components per block, nblk
// blocks) in a fixed order, and the scalars derived from them.  Called by every
// thread of one block of at least 32 K threads; partials are read past L1 (they
// may have been written by other blocks of the same launch).
__device__ void reduce_body(int what, int chain, int nblk, int K, const double* partial, ChainScalars* sc,
                            const BiasD* bias, int n_regions) {
    __shared__ double tot[32];
    ChainScalars& S = sc[chain];
    const int k = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (k < K) {
        // four independent accumulators combined in a fixed order: many loads in
        // flight, same result every run
        const double* p = partial + (size_t)chain * nblk * K + k;
        double v0 = 0.0, v1 = 0.0, v2 = 0.0, v3 = 0.0;
        int b = lane;
#pragma unroll 4
        for (; b + 96 < nblk; b += 128) {
            v0 += __ldcg(p + (size_t)b * K);
            v1 += __ldcg(p + (size_t)(b + 32) * K);
            v2 += __ldcg(p + (size_t)(b + 64) * K);
            v3 += __ldcg(p + (size_t)(b + 96) * K);
        }
        for (; b < nblk; b += 32) v0 += __ldcg(p + (size_t)b * K);
        double v = (v0 + v1) + (v2 + v3);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        if (lane == 0) tot[k] = v;
    }
    __syncthreads();
    // log-normal priors of the bias tables (Eq. lognormal), one region per lane of warp 0,
    // summed in a fixed order
    double lpr = 0.0, ga_r = 0.0, gb_r = 0.0;
    if (what == RED_LIK || what == RED_BIASGRAD) {
        const BiasD& Bd = bias[chain];
        const int r = threadIdx.x;
        if (r < n_regions && ((Bd.prior_mask >> r) & 1u)) {
            if (what == RED_LIK)
                lpr = lognormal_logpdf(Bd.alpha[r], Bd.mu_alpha, Bd.sigma_alpha) +
                      lognormal_logpdf(Bd.beta[r], Bd.mu_beta, Bd.sigma_beta);
            else {
                ga_r = lognormal_dlogpdf(Bd.alpha[r], Bd.mu_alpha, Bd.sigma_alpha);
                gb_r = lognormal_dlogpdf(Bd.beta[r], Bd.mu_beta, Bd.sigma_beta);
            }
        }
        if (threadIdx.x < 32) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) lpr += __shfl_down_sync(0xffffffffu, lpr, o);
        }
        if (what == RED_BIASGRAD && r < n_regions) {
            tot[r] += ga_r;                 // each region's own entries: no ordering question
            tot[n_regions + r] += gb_r;
        }
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if (what == RED_NTR) S.ntr = tot[0];
    else if (what == RED_SUMF) { S.sumf = tot[0]; S.lnC = log(S.ntr) - log(tot[0]); }
    else if (what == RED_P2) S.sump2 = tot[0];
    else if (what == RED_DOT) S.dot = tot[0];
    else if (what == RED_LIK) {
        S.loglik = tot[0]; S.G = tot[1]; S.sumnu2 = tot[2];
        S.gscale = tot[1] / S.ntr;
        S.logprior = lpr;
        S.logpost = -0.5 * S.sumnu2 + S.loglik + lpr;
    } else if (what == RED_BIASGRAD) {
        for (int q = 0; q < K; ++q) S.gbias[q] = tot[q];
    }
}

__global__ void __launch_bounds__(1024) k_reduce(int what, int nblk, int K, const double* partial, ChainScalars* sc,
                                                 const BiasD* bias, int n_regions) {
    reduce_body(what, blockIdx.x, nblk, K, partial, sc, bias, n_regions);
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static inline long long nvox_of(int n) { return (long long)n * n * n; }

template <typename T>
cudaError_t launch_counts_prep(int n, int batch, const int32_t* counts, uint16_t* c16, double* partial, int* err,
                               const RedArgs& ra, cudaStream_t s) {
    k_counts_prep<<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(nvox_of(n), counts, c16, partial, err, ra);
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_fill(long long count, T* p, T v, cudaStream_t s) {
    long long b = (count + 1023) / 1024;
    k_fill<T><<<(unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b)), 256, 0, s>>>(count, p, v);
    return cudaGetLastError();
}
template <typename T, bool FX, typename OutT>
static cudaError_t cic_scatter_run(int n, int batch, const Fields16& psi3, OutT* out, cudaStream_t s) {
    using CB = CicBlock<T>;
    if (n < 16) return cudaErrorInvalidValue;
    // BZ = BRIDGE_CIC_BZ (16 or 32 particles along z), 16 on the smallest mesh
    auto run = [&](auto kern, int bz) {
        const size_t sm = size_t(CB::BX + 2 * CB::H) * (CB::BY + 2 * CB::H) * (bz + 2 * CB::H) * 8;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(sm));
        if (e != cudaSuccess) return e;
        const unsigned blocks = unsigned((n / CB::BX) * (n / CB::BY) * (n / bz));
        kern<<<dim3(blocks, batch), kPwThreads, sm, s>>>(n, nvox_of(n), psi3, out);
        return cudaGetLastError();
    };
    return n >= BRIDGE_CIC_BZ ? run(k_cic_scatter<T, BRIDGE_CIC_BZ, FX, OutT>, BRIDGE_CIC_BZ)
                              : run(k_cic_scatter<T, 16, FX, OutT>, 16);
}
template <typename T>
cudaError_t launch_cic_scatter(int n, int batch, const Fields16& psi3, T* delta, cudaStream_t s) {
    return cic_scatter_run<T, false>(n, batch, psi3, delta, s);
}
template <typename T>
cudaError_t launch_cic_scatter_fixed(int n, int batch, const Fields16& psi3, unsigned long long* acc, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(acc, 0, size_t(nvox_of(n)) * batch * sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    return cic_scatter_run<T, true>(n, batch, psi3, acc, s);
}
template <typename T> cudaError_t launch_fixed_to_mass(int n, int batch, const unsigned long long* acc, T* rho, cudaStream_t s) {
    const long long count = nvox_of(n) * batch;
    long long b = (count + 1023) / 1024;
    k_fixed_to_mass<T><<<(unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b)), 256, 0, s>>>(count, acc, rho);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_pass_a(int n, int batch, const Fields16& th, const T* delta, T* lnf, T* beta_i,
                          const BiasT<T>* bias, const WebParams& wp, double* partial, const RedArgs& ra,
                          cudaStream_t s) {
    if (wp.n_regions == 16)
        k_pass_a<T, 16><<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(nvox_of(n), th, delta, lnf, beta_i, bias, wp, partial, ra);
    else
        k_pass_a<T, 4><<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(nvox_of(n), th, delta, lnf, beta_i, bias, wp, partial, ra);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_pass_b(int n, int batch, const T* lnf, const T* beta_i, const uint16_t* c16, const T* nu,
                          const ChainScalars* sc, double* partial, const RedArgs& ra, cudaStream_t s) {
    k_pass_b<T><<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(nvox_of(n), lnf, beta_i, c16, nu, sc, partial, ra);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_web_adjoint(int n, int batch, const Fields16& th, const T* delta, const uint16_t* c16,
                               const BiasT<T>* bias, const WebParams& wp, const ChainScalars* sc,
                               const Fields16& out, double* partial, bool bias_grad, cudaStream_t s, int blocks) {
    // partial sums (bias gradient) only with bias_grad: that launch keeps the reduction's grid;
    // otherwise blocks per chain as requested (grid-stride loop), else the wide grid
    const dim3 g(bias_grad ? pw_blocks(n) : (blocks > 0 ? blocks : pw_blocks_wide(n)), batch);
    if (wp.n_regions == 16) {
        if (bias_grad) k_web_adj<T, 16, true><<<g, kPwThreads, 0, s>>>(nvox_of(n), th, delta, c16, bias, wp, sc, out, partial);
        else k_web_adj<T, 16, false><<<g, kPwThreads, 0, s>>>(nvox_of(n), th, delta, c16, bias, wp, sc, out, partial);
    } else {
        if (bias_grad) k_web_adj<T, 4, true><<<g, kPwThreads, 0, s>>>(nvox_of(n), th, delta, c16, bias, wp, sc, out, partial);
        else k_web_adj<T, 4, false><<<g, kPwThreads, 0, s>>>(nvox_of(n), th, delta, c16, bias, wp, sc, out, partial);
    }
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_rsd_radial(int n, int batch, const Fields16& psi, const Fields16& psi1, double f, cudaStream_t s) {
    k_rsd_radial<T><<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(n, nvox_of(n), psi, psi1, T(f));
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_shift(long long count, const T* in, T* out, T c, cudaStream_t s) {
    long long b = (count + 1023) / 1024;
    k_shift<T><<<(unsigned)(b > 4096 ? 4096 : (b < 1 ? 1 : b)), 256, 0, s>>>(count, in, out, c);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_kick_drift(int n, int batch, T* p, T* nu, const T* g, double ck, double cd, double* partial,
                              cudaStream_t s) {
    k_kick_drift<T><<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(nvox_of(n), p, nu, g, T(ck), T(cd), partial);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_dot(int n, int batch, const T* a, const T* b, double* partial, const RedArgs& ra, cudaStream_t s) {
    k_dot<T><<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(nvox_of(n), a, b, partial, ra);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_bias_kick_drift(int batch, int nr, uint32_t free_mask, double* theta, double* ptheta,
                                   const ChainScalars* sc, BiasD* bd, BiasT<T>* bt, double ck, double cd, cudaStream_t s) {
    k_bias_kick_drift<T><<<batch, 32, 0, s>>>(nr, free_mask, theta, ptheta, sc, bd, bt, ck, cd);
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_delta_tr(int n, int batch, const uint16_t* c16, const ChainScalars* sc, T* out,
                                                  cudaStream_t s) {
    k_delta_tr<T><<<dim3(pw_blocks_wide(n), batch), kPwThreads, 0, s>>>(nvox_of(n), c16, sc, out);
    return cudaGetLastError();
}
template <typename T> cudaError_t launch_scale_chains(int n, int batch, T* g, const double* scale, cudaStream_t s) {
    k_scale_chains<T><<<dim3(pw_blocks_wide(n), batch), kPwThreads, 0, s>>>(nvox_of(n), g, scale);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_lnnbar(long long nvox, int batch, const T* lnf, const ChainScalars* sc, T* out, cudaStream_t s) {
    k_lnnbar<T><<<dim3(256, batch), kPwThreads, 0, s>>>(nvox, lnf, sc, out);
    return cudaGetLastError();
}
template <typename T>
cudaError_t launch_eigs(int n, int batch, const Fields16& t6, const Fields16& out3, cudaStream_t s) {
    k_eigs<T><<<dim3(pw_blocks(n), batch), kPwThreads, 0, s>>>(nvox_of(n), t6, out3);
    return cudaGetLastError();
}

cudaError_t launch_reduce(int what, int nblk, int batch, const double* partial, ChainScalars* sc, const BiasD* bias,
                          int n_regions, cudaStream_t s) {
    int K = what == RED_LIK ? 3 : (what == RED_BIASGRAD ? 2 * n_regions : 1);
    k_reduce<<<batch, 32 * K, 0, s>>>(what, nblk, K, partial, sc, bias, n_regions);
    return cudaGetLastError();
}

#define PW_INST(T)                                                                                                   \
    template cudaError_t launch_counts_prep<T>(int, int, const int32_t*, uint16_t*, double*, int*, const RedArgs&,   \
                                               cudaStream_t);                                                       \
    template cudaError_t launch_fill<T>(long long, T*, T, cudaStream_t);                                            \
    template cudaError_t launch_cic_scatter<T>(int, int, const Fields16&, T*, cudaStream_t);                        \
    template cudaError_t launch_cic_scatter_fixed<T>(int, int, const Fields16&, unsigned long long*, cudaStream_t);    \
    template cudaError_t launch_fixed_to_mass<T>(int, int, const unsigned long long*, T*, cudaStream_t);               \
    template cudaError_t launch_pass_a<T>(int, int, const Fields16&, const T*, T*, T*, const BiasT<T>*,             \
                                          const WebParams&, double*, const RedArgs&, cudaStream_t);                 \
    template cudaError_t launch_pass_b<T>(int, int, const T*, const T*, const uint16_t*, const T*,                  \
                                          const ChainScalars*, double*, const RedArgs&, cudaStream_t);              \
    template cudaError_t launch_web_adjoint<T>(int, int, const Fields16&, const T*, const uint16_t*,                \
                                               const BiasT<T>*, const WebParams&, const ChainScalars*,              \
                                               const Fields16&, double*, bool, cudaStream_t, int);                  \
    template cudaError_t launch_shift<T>(long long, const T*, T*, T, cudaStream_t);                                 \
    template cudaError_t launch_rsd_radial<T>(int, int, const Fields16&, const Fields16&, double, cudaStream_t);    \
    template cudaError_t launch_kick_drift<T>(int, int, T*, T*, const T*, double, double, double*, cudaStream_t);   \
    template cudaError_t launch_scale_chains<T>(int, int, T*, const double*, cudaStream_t);                         \
    template cudaError_t launch_delta_tr<T>(int, int, const uint16_t*, const ChainScalars*, T*, cudaStream_t);       \
    template cudaError_t launch_dot<T>(int, int, const T*, const T*, double*, const RedArgs&, cudaStream_t);         \
    template cudaError_t launch_bias_kick_drift<T>(int, int, uint32_t, double*, double*, const ChainScalars*,        \
                                                   BiasD*, BiasT<T>*, double, double, cudaStream_t);                \
    template cudaError_t launch_lnnbar<T>(long long, int, const T*, const ChainScalars*, T*, cudaStream_t);         \
    template cudaError_t launch_eigs<T>(int, int, const Fields16&, const Fields16&, cudaStream_t);
PW_INST(float)
PW_INST(double)

}  // namespace bridge
