// Fused real-space nodes: inverse z DFT of several spectra of one tile into a
// per-CTA scratch slab, a per-voxel stage, and forward z DFT of the results.
// The slab lives in global memory that stays resident in the 129 MB L2, so the
// intermediate real fields of the tensor stages never make a round trip to HBM.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "passes.cuh"
#include "pointwise.cuh"

#ifndef BRIDGE_NODE_L2_MB
#define BRIDGE_NODE_L2_MB 96   // all slabs together, MB (the L2 holds 129 MB; 72-128 MB measured within 1 %)
#endif

namespace bridge {

enum NodeKind {
    NODE_ALPT_FWD = 2,   // delta0, phi (7) -> a = -D delta0 + D2 S2, theta_SC -> r2c (2)
    NODE_ALPT_ADJ = 3,   // delta0, phi (7), g_a, g_b (2) -> g_delta0, g_phi -> r2c (7)
    NODE_GATHER = 5,     // psi (3) -> CIC gather adjoint g_psi -> r2c (3)
    NODE_GATHER_RSD = 6  // psi, psi1 (6) -> radial redshift space, CIC gather adjoint, its transpose
                         // -> g_psi, g_psi1 -> r2c (6)
};

struct NodeArgs {
    int kind;
    const void* spec_in[16];     // spectra ([kz][y][x] layout), chain stride nspec
    void* spec_out[16];          // spectra out
    const void* real_in[4];      // real fields read per voxel (g_rho for the gather), chain stride nvox
    void* real_out[4];           // real fields written per voxel (unused by the current kinds)
    void* scratch;               // slabs: [grid][F][tile voxels]
    size_t scratch_bytes;        // size of scratch; the grid is capped so that all slabs fit (0: no cap)
    int cps;                     // CTAs per SM (0: built-in choice; clamped to the occupancy limit)
    double growth, d2;
    float growth_f, d2_f;        // FP32 copies (an FP32 node reads no double parameter)
    double rsd_f;                // NODE_GATHER_RSD: f of the linear velocity
    float rsd_f_f;
};

// Launch a node; *grid_used receives the number of CTAs.
template <typename T> cudaError_t launch_node(int n, int batch, const NodeArgs& a, int* grid_used, cudaStream_t s);
// Largest grid and scratch (bytes) over all node kinds for this mesh and batch (current device).
template <typename T> int node_max_grid(int n, int batch);
template <typename T> size_t node_scratch_bytes(int n, int batch);
// Upload the twiddle tables of the node translation units (per device).
cudaError_t upload_node_twiddles();

}  // namespace bridge
