// Fused node kernels (included once per precision by nodes_f32.cu / nodes_f64.cu).
//
// One CTA of 128 threads owns a tile (16 x by GY y lines along z, GY = 16/N2)
// and a scratch slab in global memory: per field, the tile's real voxels in
// [y][x][z] order.  Per tile: (1) inverse z DFT of the input spectra into the
// slab, (2) the per-voxel stage reading the slab (and a few full real fields),
// writing results back into the slab, (3) forward z DFT of the result slabs.
// CTAs are persistent (grid = resident CTAs), so each slab is rewritten tile
// after tile and stays in L2; spectra are read and written with streaming
// (evict-first) hints.  Partial sums are accumulated per CTA and chain and
// written to partial[chain][cta][k] by their single owner (deterministic).
#pragma once

#include "common.cuh"
#include "nodes.cuh"
#include "twiddle.cuh"
#include "voxel.cuh"
#include "ztile.cuh"

namespace bridge {

constexpr int kNodeThreads = 128;

template <typename T, int N> using NodeCfg = ZCfg<T, N, 16 / Split<N>::N2>;

template <int KIND, int NR> struct NodeShape;
template <int NR> struct NodeShape<NODE_WEB_FWD, NR> { static constexpr int IN = NR == 16 ? 12 : 6, SLAB = IN, OUT = 0, K = 1; };
template <int NR> struct NodeShape<NODE_WEB_ADJ, NR> { static constexpr int IN = NR == 16 ? 12 : 6, SLAB = IN + 1, OUT = IN + 1, K = 2 * NR; };
template <int NR> struct NodeShape<NODE_ALPT_FWD, NR> { static constexpr int IN = 7, SLAB = 7, OUT = 2, K = 0; };
template <int NR> struct NodeShape<NODE_ALPT_ADJ, NR> { static constexpr int IN = 9, SLAB = 9, OUT = 7, K = 0; };
template <int NR> struct NodeShape<NODE_FINAL, NR> { static constexpr int IN = 1, SLAB = 1, OUT = 0, K = 0; };
template <int NR> struct NodeShape<NODE_GATHER, NR> { static constexpr int IN = 3, SLAB = 3, OUT = 3, K = 0; };
template <int NR> struct NodeShape<NODE_SCATTER, NR> { static constexpr int IN = 3, SLAB = 3, OUT = 0, K = 0; };

// Deterministic per-(chain, CTA) accumulation of K partial sums.
template <int K>
__device__ __forceinline__ void node_flush(double (&acc)[K > 0 ? K : 1], double* partial, int chain, double* sh) {
    if constexpr (K > 0) {
        for (int k = 0; k < K; ++k) {
            double v = acc[k];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
            __syncthreads();
            if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
            __syncthreads();
            if (threadIdx.x == 0) {
                double r = 0.0;
                for (int w = 0; w < kNodeThreads / 32; ++w) r += sh[w];
                partial[((size_t)chain * gridDim.x + blockIdx.x) * K + k] += r;
            }
            acc[k] = 0.0;
        }
    }
}

template <typename T, int N, int KIND, int NR, bool BIASG>
__global__ void __launch_bounds__(kNodeThreads, 2) k_node(const NodeArgs A, int batch, long long nspec) {
    using C = NodeCfg<T, N>;
    using V = cplx_t<T>;
    using SH = NodeShape<KIND, NR>;
    static_assert(C::NT == kNodeThreads, "node tile must use 128 threads");
    constexpr long long NVOX = (long long)N * N * N;
    constexpr int TV = C::TILE_VOX;
    constexpr int KP = (KIND == NODE_WEB_FWD) ? 1 : ((KIND == NODE_WEB_ADJ && BIASG) ? 2 * NR : 0);
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    __shared__ BiasT<T> B;
    __shared__ double shred[kNodeThreads / 32];
    const int t = threadIdx.x;
    T* slab = reinterpret_cast<T*>(A.scratch) + (size_t)blockIdx.x * SH::SLAB * TV;
    auto slab_f = [&](int f) { return slab + (size_t)f * TV; };
    double acc[KP > 0 ? KP : 1];
#pragma unroll
    for (int k = 0; k < (KP > 0 ? KP : 1); ++k) acc[k] = 0.0;
    constexpr int NG = BIASG ? NR : 1;
    T ga[NG], gb[NG];
#pragma unroll
    for (int r = 0; r < NG; ++r) ga[r] = gb[r] = T(0);
    int cur_chain = -1;
    const long long items = (long long)batch * C::TILES;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int chain = (int)(item / C::TILES);
        const int tile = (int)(item % C::TILES);
        if (chain != cur_chain) {
            if (cur_chain >= 0) {
                if constexpr (KIND == NODE_WEB_ADJ && BIASG) {
#pragma unroll
                    for (int r = 0; r < NR; ++r) { acc[r] = ga[r]; acc[NR + r] = gb[r]; ga[r] = gb[r] = T(0); }
                }
                node_flush<KP>(acc, A.partial, cur_chain, shred);
            }
            cur_chain = chain;
            if constexpr (KIND == NODE_WEB_FWD || KIND == NODE_WEB_ADJ) {
                __syncthreads();
                if (t == 0) B = reinterpret_cast<const BiasT<T>*>(A.bias)[chain];
                __syncthreads();
            }
        }
        int x0, y0;
        C::tile_xy(tile, x0, y0);
        // (1) inverse z of the inputs into the slab
#pragma unroll 1
        for (int f = 0; f < SH::IN; ++f) {
            T* s = slab_f(f);
            auto line = [&](int c) { return s + ((c / 8) * 16 + 2 * (c % 8)) * N; };
            ztile_inv<C>(reinterpret_cast<const V*>(A.spec_in[f]) + chain * nspec, line, (long long)N, x0, y0, sm, t);
        }
        // (2) per-voxel stage
        const size_t coff = (size_t)chain * NVOX;
        T fsum = T(0);
        for (int v = t; v < TV; v += kNodeThreads) {
            const int z = v % N, xl = (v / N) % 16, yl = v / (16 * N);
            const size_t g = coff + ((size_t)(x0 + xl) * N + (y0 + yl)) * N + z;
            if constexpr (KIND == NODE_WEB_FWD) {
                T a6[6], h6[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) a6[q] = slab_f(q)[v];
                if constexpr (NR == 16) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) h6[q] = slab_f(6 + q)[v];
                }
                const T rho = reinterpret_cast<const T*>(A.real_in[0])[g];
                WebState<T, NR> S;
                web_eval<T, NR>(a6, h6, rho, B, A.wp, S);
                reinterpret_cast<T*>(A.real_out[0])[g] = S.lf.lnf;
                reinterpret_cast<T*>(A.real_out[1])[g] = S.q.beta;
                fsum += v_exp(S.lf.lnf);
            } else if constexpr (KIND == NODE_WEB_ADJ) {
                T a6[6], h6[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) a6[q] = slab_f(q)[v];
                if constexpr (NR == 16) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) h6[q] = slab_f(6 + q)[v];
                }
                const T rho = reinterpret_cast<const T*>(A.real_in[0])[g];
                const T lnC = T(A.sc[chain].lnC);
                const T gscale = T(A.sc[chain].G / A.sc[chain].ntr);
                WebState<T, NR> S;
                web_eval<T, NR>(a6, h6, rho, B, A.wp, S);
                T gd, gt[6], gh[6];
                web_adjoint_voxel<T, NR, BIASG>(S, rho, (int)A.c16[g], lnC, gscale, B, A.wp, gd, gt, gh, ga, gb);
#pragma unroll
                for (int q = 0; q < 6; ++q) slab_f(q)[v] = gt[q];
                if constexpr (NR == 16) {
#pragma unroll
                    for (int q = 0; q < 6; ++q) slab_f(6 + q)[v] = gh[q];
                }
                slab_f(SH::IN)[v] = gd;
            } else if constexpr (KIND == NODE_ALPT_FWD) {
                const T d0 = slab_f(0)[v];
                T phi[6];
#pragma unroll
                for (int q = 0; q < 6; ++q) phi[q] = slab_f(1 + q)[v];
                T a, b;
                alpt_sources<T>(d0, phi, T(A.growth), T(A.d2), a, b);
                slab_f(0)[v] = a;
                slab_f(1)[v] = b;
            } else if constexpr (KIND == NODE_ALPT_ADJ) {
                const T d0 = slab_f(0)[v];
                T phi[6], gphi[6], gd0;
#pragma unroll
                for (int q = 0; q < 6; ++q) phi[q] = slab_f(1 + q)[v];
                alpt_sources_adj<T>(d0, phi, T(A.growth), T(A.d2), slab_f(7)[v], slab_f(8)[v], gd0, gphi);
                slab_f(0)[v] = gd0;
#pragma unroll
                for (int q = 0; q < 6; ++q) slab_f(1 + q)[v] = gphi[q];
            } else if constexpr (KIND == NODE_FINAL) {
                reinterpret_cast<T*>(A.real_out[0])[g] = slab_f(0)[v] - reinterpret_cast<const T*>(A.real_in[0])[g];
            } else if constexpr (KIND == NODE_GATHER) {
                CicCorner<T> c;
                cic_corner<T>((long long)(g - coff), N, slab_f(0)[v], slab_f(1)[v], slab_f(2)[v], c);
                T out[3];
                cic_gather_one<T>(c, N, reinterpret_cast<const T*>(A.real_in[0]) + coff, out);
                slab_f(0)[v] = out[0];
                slab_f(1)[v] = out[1];
                slab_f(2)[v] = out[2];
            } else if constexpr (KIND == NODE_SCATTER) {
                CicCorner<T> c;
                cic_corner<T>((long long)(g - coff), N, slab_f(0)[v], slab_f(1)[v], slab_f(2)[v], c);
                cic_deposit<T>(c, N, reinterpret_cast<T*>(A.real_out[0]) + coff);
            }
        }
        if constexpr (KIND == NODE_WEB_FWD) acc[0] += (double)fsum;
        __syncthreads();
        // (3) forward z of the results
#pragma unroll 1
        for (int f = 0; f < SH::OUT; ++f) {
            // web adjoint output order: g_delta (slab IN), then the tensor slabs
            const int sf = (KIND == NODE_WEB_ADJ) ? (f == 0 ? SH::IN : f - 1) : f;
            T* s = slab_f(sf);
            auto line = [&](int c) { return s + ((c / 8) * 16 + 2 * (c % 8)) * N; };
            ztile_fwd<C>(line, (long long)N, reinterpret_cast<V*>(A.spec_out[f]) + chain * nspec, x0, y0, sm, t);
        }
    }
    if (cur_chain >= 0) {
        if constexpr (KIND == NODE_WEB_ADJ && BIASG) {
#pragma unroll
            for (int r = 0; r < NR; ++r) { acc[r] = ga[r]; acc[NR + r] = gb[r]; }
        }
        node_flush<KP>(acc, A.partial, cur_chain, shred);
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T, int N, int KIND, int NR, bool BIASG> struct NodeLaunch {
    using C = NodeCfg<T, N>;
    using SH = NodeShape<KIND, NR>;
    static size_t smem() { return size_t(C::SM_ELEMS) * sizeof(cplx_t<T>); }
    static int grid(int batch, int sms) {
        // resident CTAs, bounded so that all slabs together stay well below the 129 MB L2
        static int occ = -1;
        if (occ < 0) {
            auto kern = k_node<T, N, KIND, NR, BIASG>;
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kNodeThreads, smem()) != cudaSuccess) occ = 1;
        }
        const size_t per_cta = size_t(SH::SLAB) * C::TILE_VOX * sizeof(T);
        const size_t budget = size_t(72) << 20;
        int cps = occ < 1 ? 1 : occ;
        while (cps > 1 && size_t(cps) * sms * per_cta > budget) --cps;
        long long items = (long long)batch * C::TILES;
        long long g = (long long)cps * sms;
        return int(g < items ? g : items);
    }
    static cudaError_t run(int batch, int sms, const NodeArgs& a, cudaStream_t s, long long nspec, int* gu) {
        auto kern = k_node<T, N, KIND, NR, BIASG>;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const int g = grid(batch, sms);
        if (gu) *gu = g;
        kern<<<g, kNodeThreads, smem(), s>>>(a, batch, nspec);
        return cudaGetLastError();
    }
};

template <typename T, int N, int KIND>
static cudaError_t node_dispatch_nr(int batch, int sms, const NodeArgs& a, cudaStream_t s, long long nspec, int* gu) {
    if (a.n_regions == 16) {
        if (KIND == NODE_WEB_ADJ && a.bias_grad) return NodeLaunch<T, N, KIND, 16, true>::run(batch, sms, a, s, nspec, gu);
        return NodeLaunch<T, N, KIND, 16, false>::run(batch, sms, a, s, nspec, gu);
    }
    if (KIND == NODE_WEB_ADJ && a.bias_grad) return NodeLaunch<T, N, KIND, 4, true>::run(batch, sms, a, s, nspec, gu);
    return NodeLaunch<T, N, KIND, 4, false>::run(batch, sms, a, s, nspec, gu);
}

template <typename T, int N>
static cudaError_t node_dispatch(int batch, int sms, const NodeArgs& a, cudaStream_t s, int* gu) {
    const long long nspec = (long long)(N / 2 + 1) * N * N;
    switch (a.kind) {
        case NODE_WEB_FWD: return node_dispatch_nr<T, N, NODE_WEB_FWD>(batch, sms, a, s, nspec, gu);
        case NODE_WEB_ADJ: return node_dispatch_nr<T, N, NODE_WEB_ADJ>(batch, sms, a, s, nspec, gu);
        case NODE_ALPT_FWD: return NodeLaunch<T, N, NODE_ALPT_FWD, 4, false>::run(batch, sms, a, s, nspec, gu);
        case NODE_ALPT_ADJ: return NodeLaunch<T, N, NODE_ALPT_ADJ, 4, false>::run(batch, sms, a, s, nspec, gu);
        case NODE_FINAL: return NodeLaunch<T, N, NODE_FINAL, 4, false>::run(batch, sms, a, s, nspec, gu);
        case NODE_GATHER: return NodeLaunch<T, N, NODE_GATHER, 4, false>::run(batch, sms, a, s, nspec, gu);
        case NODE_SCATTER: return NodeLaunch<T, N, NODE_SCATTER, 4, false>::run(batch, sms, a, s, nspec, gu);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int N> static int node_grid_max(int batch, int sms) {
    int g = 0;
    auto upd = [&](int v) { g = v > g ? v : g; };
    upd(NodeLaunch<T, N, NODE_WEB_FWD, 16, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_WEB_FWD, 4, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 16, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 16, true>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 4, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 4, true>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_ALPT_FWD, 4, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_ALPT_ADJ, 4, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_FINAL, 4, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_GATHER, 4, false>::grid(batch, sms));
    upd(NodeLaunch<T, N, NODE_SCATTER, 4, false>::grid(batch, sms));
    return g;
}

template <typename T, int N> static size_t node_scratch_max(int batch, int sms) {
    size_t m = 0;
    auto upd = [&](int grid, int slab) {
        size_t v = size_t(grid) * slab * NodeCfg<T, N>::TILE_VOX * sizeof(T);
        m = v > m ? v : m;
    };
    upd(NodeLaunch<T, N, NODE_WEB_FWD, 16, false>::grid(batch, sms), NodeShape<NODE_WEB_FWD, 16>::SLAB);
    upd(NodeLaunch<T, N, NODE_WEB_FWD, 4, false>::grid(batch, sms), NodeShape<NODE_WEB_FWD, 4>::SLAB);
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 16, false>::grid(batch, sms), NodeShape<NODE_WEB_ADJ, 16>::SLAB);
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 16, true>::grid(batch, sms), NodeShape<NODE_WEB_ADJ, 16>::SLAB);
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 4, false>::grid(batch, sms), NodeShape<NODE_WEB_ADJ, 4>::SLAB);
    upd(NodeLaunch<T, N, NODE_WEB_ADJ, 4, true>::grid(batch, sms), NodeShape<NODE_WEB_ADJ, 4>::SLAB);
    upd(NodeLaunch<T, N, NODE_ALPT_FWD, 4, false>::grid(batch, sms), NodeShape<NODE_ALPT_FWD, 4>::SLAB);
    upd(NodeLaunch<T, N, NODE_ALPT_ADJ, 4, false>::grid(batch, sms), NodeShape<NODE_ALPT_ADJ, 4>::SLAB);
    upd(NodeLaunch<T, N, NODE_FINAL, 4, false>::grid(batch, sms), NodeShape<NODE_FINAL, 4>::SLAB);
    upd(NodeLaunch<T, N, NODE_GATHER, 4, false>::grid(batch, sms), NodeShape<NODE_GATHER, 4>::SLAB);
    upd(NodeLaunch<T, N, NODE_SCATTER, 4, false>::grid(batch, sms), NodeShape<NODE_SCATTER, 4>::SLAB);
    return m;
}

}  // namespace bridge
