// Fused node kernels (included once per precision by nodes_f32.cu / nodes_f64.cu).
//
// One CTA of 128 threads owns a tile (16 x by GY y lines along z, GY = 16/N2)
// and a scratch slab in global memory: per field, the tile's real voxels in
// [y][x][z] order.  Per tile: (1) inverse z DFT of the input spectra into the
// slab, (2) the per-voxel stage reading the slab (and a few full real fields),
// writing results back into the slab, (3) forward z DFT of the result slabs.
// CTAs are persistent (grid = resident CTAs), so each slab is rewritten tile
// after tile and stays in L2.
// Nodes carry the light per-voxel stages (ALPT sources and their adjoint, CIC
// gather); the arithmetic-heavy web stages and the CIC scatter (which needs 3D
// blocks of particles) run as separate kernels.
#pragma once

#include "common.cuh"
#include "nodes.cuh"
#include "twiddle.cuh"
#include "voxel.cuh"
#include "ztile.cuh"

namespace bridge {

constexpr int kNodeThreads = 128;
#ifndef BRIDGE_NODE_U
#define BRIDGE_NODE_U 8   // voxels per thread step of the per-voxel stage (4: 0.03 ms slower at 256^3)
#endif


template <typename T, int N> using NodeCfg = ZCfg<T, N, 16 / Split<N>::N2>;

template <int KIND> struct NodeShape;
template <> struct NodeShape<NODE_ALPT_FWD> { static constexpr int IN = 7, SLAB = 7, OUT = 2; };
template <> struct NodeShape<NODE_ALPT_ADJ> { static constexpr int IN = 9, SLAB = 9, OUT = 7; };
template <> struct NodeShape<NODE_GATHER> { static constexpr int IN = 3, SLAB = 3, OUT = 3; };
template <> struct NodeShape<NODE_GATHER_RSD> { static constexpr int IN = 6, SLAB = 6, OUT = 6; };

template <typename T, int N, int KIND>
__global__ void __launch_bounds__(kNodeThreads) k_node(const NodeArgs A, int batch, long long nspec) {
    using C = NodeCfg<T, N>;
    using V = cplx_t<T>;
    using SH = NodeShape<KIND>;
    static_assert(C::NT == kNodeThreads, "node tile must use 128 threads");
    constexpr long long NVOX = (long long)N * N * N;
    constexpr int TV = C::TILE_VOX;
    extern __shared__ __align__(16) unsigned char smraw[];
    V* sm = reinterpret_cast<V*>(smraw);
    const int t = threadIdx.x;
    T* slab = reinterpret_cast<T*>(A.scratch) + (size_t)blockIdx.x * SH::SLAB * TV;
    auto slab_f = [&](int f) { return slab + (size_t)f * TV; };
    const PlainLineIO io;
    const long long items = (long long)batch * C::TILES;
    for (long long item = blockIdx.x; item < items; item += gridDim.x) {
        const int chain = (int)(item / C::TILES);
        const int tile = (int)(item % C::TILES);
        int x0, y0;
        C::tile_xy(tile, x0, y0);
        // (1) inverse z of the inputs into the slab
#pragma unroll 1
        for (int f = 0; f < SH::IN; ++f) {
            T* s = slab_f(f);
            auto line = [&](int c) { return s + ((c / 8) * 16 + 2 * (c % 8)) * N; };
            ztile_inv<C, decltype(line), true, PlainLineIO, 1>(reinterpret_cast<const V*>(A.spec_in[f]) + chain * nspec, line, (long long)N, x0, y0, sm, t, io);
        }
        // (2) per-voxel stage, U voxels per thread step: the slab (and g_rho)
        // loads of all U voxels are issued before any result is stored, so a
        // step waits for one L2 round trip instead of U
        const size_t coff = (size_t)chain * NVOX;
        // FP64 and the redshift-space gather: eight voxels would spill
        constexpr int U = (sizeof(T) == 8 || KIND == NODE_GATHER_RSD) ? 4 : BRIDGE_NODE_U;
        static_assert(TV % (U * kNodeThreads) == 0, "tile voxels must split into whole steps");
        for (int v0 = t; v0 < TV; v0 += U * kNodeThreads) {
            if constexpr (KIND == NODE_ALPT_FWD) {
                T in[U][7];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int q = 0; q < 7; ++q) in[u][q] = io.ld(slab_f(q) + v0 + u * kNodeThreads);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int v = v0 + u * kNodeThreads;
                    T a, b;
                    alpt_sources<T>(in[u][0], &in[u][1], pick<T>(A.growth, A.growth_f), pick<T>(A.d2, A.d2_f), a, b);
                    io.st(slab_f(0) + v, a);
                    io.st(slab_f(1) + v, b);
                }
            } else if constexpr (KIND == NODE_ALPT_ADJ) {
                T in[U][9];
#pragma unroll
                for (int u = 0; u < U; ++u)
#pragma unroll
                    for (int q = 0; q < 9; ++q) in[u][q] = io.ld(slab_f(q) + v0 + u * kNodeThreads);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int v = v0 + u * kNodeThreads;
                    T gphi[6], gd0;
                    alpt_sources_adj<T>(in[u][0], &in[u][1], pick<T>(A.growth, A.growth_f), pick<T>(A.d2, A.d2_f), in[u][7], in[u][8], gd0, gphi);
                    io.st(slab_f(0) + v, gd0);
#pragma unroll
                    for (int q = 0; q < 6; ++q) io.st(slab_f(1 + q) + v, gphi[q]);
                }
            } else if constexpr (KIND == NODE_GATHER) {
                const T* grho = reinterpret_cast<const T*>(A.real_in[0]) + coff;
                CicCorner<T> c[U];
                T gv[U][8];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int v = v0 + u * kNodeThreads;
                    const int z = v % N, xl = (v / N) % 16, yl = v / (16 * N);
                    const long long q = ((long long)(x0 + xl) * N + (y0 + yl)) * N + z;
                    cic_corner<T>(q, N, io.ld(slab_f(0) + v), io.ld(slab_f(1) + v), io.ld(slab_f(2) + v), c[u]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) cic_gather_loads<T>(c[u], N, grho, gv[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int v = v0 + u * kNodeThreads;
                    T out[3];
                    cic_gather_combine<T>(c[u], gv[u], out);
                    io.st(slab_f(0) + v, out[0]);
                    io.st(slab_f(1) + v, out[1]);
                    io.st(slab_f(2) + v, out[2]);
                }
            } else if constexpr (KIND == NODE_GATHER_RSD) {
                // the particle at its redshift-space position (rsd_radial_fwd), the CIC gather
                // there, and the transpose of the shift (rsd_radial_adj)
                const T* grho = reinterpret_cast<const T*>(A.real_in[0]) + coff;
                const T f = pick<T>(A.rsd_f, A.rsd_f_f), cen = T(N / 2);
                CicCorner<T> c[U];
                RsdPoint<T> R[U];
                T gv[U][8];
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int v = v0 + u * kNodeThreads;
                    const int z = v % N, xl = (v / N) % 16, yl = v / (16 * N);
                    const int qv[3] = {x0 + xl, y0 + yl, z};
                    const T ps[3] = {io.ld(slab_f(0) + v), io.ld(slab_f(1) + v), io.ld(slab_f(2) + v)};
                    const T p1[3] = {io.ld(slab_f(3) + v), io.ld(slab_f(4) + v), io.ld(slab_f(5) + v)};
                    T s[3];
                    rsd_radial_fwd<T>(qv, cen, ps, p1, f, R[u], s);
                    const long long q = ((long long)qv[0] * N + qv[1]) * N + z;
                    cic_corner<T>(q, N, s[0], s[1], s[2], c[u]);
                }
#pragma unroll
                for (int u = 0; u < U; ++u) cic_gather_loads<T>(c[u], N, grho, gv[u]);
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int v = v0 + u * kNodeThreads;
                    T G[3], gp[3], gp1[3];
                    cic_gather_combine<T>(c[u], gv[u], G);
                    rsd_radial_adj<T>(R[u], f, G, gp, gp1);
#pragma unroll
                    for (int j = 0; j < 3; ++j) {
                        io.st(slab_f(j) + v, gp[j]);
                        io.st(slab_f(3 + j) + v, gp1[j]);
                    }
                }
            }
        }
        __syncthreads();
        // (3) forward z of the results
#pragma unroll 1
        for (int f = 0; f < SH::OUT; ++f) {
            T* s = slab_f(f);
            auto line = [&](int c) { return s + ((c / 8) * 16 + 2 * (c % 8)) * N; };
            ztile_fwd<C, decltype(line), true>(line, (long long)N, reinterpret_cast<V*>(A.spec_out[f]) + chain * nspec, x0, y0, sm, t, io);
        }
    }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
template <typename T, int N, int KIND> struct NodeLaunch {
    using C = NodeCfg<T, N>;
    using SH = NodeShape<KIND>;
    static size_t smem() { return size_t(C::SM_ELEMS) * sizeof(cplx_t<T>); }
    static int grid(int batch, int sms, int cps_override = 0, size_t cap = 0) {
        // resident CTAs, bounded so that all slabs together stay well below the
        // 129 MB L2 (built-in choice) or as requested, within occupancy and the
        // scratch the caller owns
        static int occ = -1;
        if (occ < 0) {
            auto kern = k_node<T, N, KIND>;
            cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kern, kNodeThreads, smem()) != cudaSuccess) occ = 1;
        }
        const size_t per_cta = size_t(SH::SLAB) * C::TILE_VOX * sizeof(T);
        const size_t budget = size_t(BRIDGE_NODE_L2_MB) << 20;
        int cps = occ < 1 ? 1 : occ;
        if (cps_override > 0) cps = min(cps_override, cps);
        else while (cps > 1 && size_t(cps) * sms * per_cta > budget) --cps;
        long long items = (long long)batch * C::TILES;
        long long g = (long long)cps * sms;
        if (cap > 0) g = min(g, (long long)(cap / per_cta));
        if (g < 1) g = 1;
        return int(g < items ? g : items);
    }
    static cudaError_t run(int batch, int sms, const NodeArgs& a, cudaStream_t s, long long nspec, int* gu) {
        auto kern = k_node<T, N, KIND>;
        static bool attr = false;
        if (!attr) {
            cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem()));
            if (e != cudaSuccess) return e;
            attr = true;
        }
        const int g = grid(batch, sms, a.cps, a.scratch_bytes);
        if (a.scratch_bytes > 0 && size_t(g) * SH::SLAB * C::TILE_VOX * sizeof(T) > a.scratch_bytes)
            return cudaErrorInvalidValue;   // not even one slab fits
        if (gu) *gu = g;
        kern<<<g, kNodeThreads, smem(), s>>>(a, batch, nspec);
        return cudaGetLastError();
    }
    static size_t scratch(int batch, int sms) { return size_t(grid(batch, sms)) * SH::SLAB * C::TILE_VOX * sizeof(T); }
};

template <typename T, int N>
static cudaError_t node_dispatch(int batch, int sms, const NodeArgs& a, cudaStream_t s, int* gu) {
    const long long nspec = (long long)(N / 2 + 1) * N * N;
    switch (a.kind) {
        case NODE_ALPT_FWD: return NodeLaunch<T, N, NODE_ALPT_FWD>::run(batch, sms, a, s, nspec, gu);
        case NODE_ALPT_ADJ: return NodeLaunch<T, N, NODE_ALPT_ADJ>::run(batch, sms, a, s, nspec, gu);
        case NODE_GATHER: return NodeLaunch<T, N, NODE_GATHER>::run(batch, sms, a, s, nspec, gu);
        case NODE_GATHER_RSD: return NodeLaunch<T, N, NODE_GATHER_RSD>::run(batch, sms, a, s, nspec, gu);
        default: return cudaErrorInvalidValue;
    }
}

template <typename T, int N> static int node_grid_max(int batch, int sms) {
    int g = NodeLaunch<T, N, NODE_ALPT_FWD>::grid(batch, sms);
    g = max(g, NodeLaunch<T, N, NODE_ALPT_ADJ>::grid(batch, sms));
    g = max(g, NodeLaunch<T, N, NODE_GATHER_RSD>::grid(batch, sms));
    return max(g, NodeLaunch<T, N, NODE_GATHER>::grid(batch, sms));
}

template <typename T, int N> static size_t node_scratch_max(int batch, int sms) {
    size_t m = NodeLaunch<T, N, NODE_ALPT_FWD>::scratch(batch, sms);
    m = max(m, NodeLaunch<T, N, NODE_ALPT_ADJ>::scratch(batch, sms));
    m = max(m, NodeLaunch<T, N, NODE_GATHER_RSD>::scratch(batch, sms));
    return max(m, NodeLaunch<T, N, NODE_GATHER>::scratch(batch, sms));
}

}  // namespace bridge
