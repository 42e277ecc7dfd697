// Host-visible launch interface of the real-space kernels (pointwise.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "voxel.cuh"

namespace bridge {

constexpr int kPwThreads = 256;
// Blocks per chain of the real-space kernels (fixed per N so that the FP64
// partial sums are reduced in a fixed order: the results are deterministic).
inline int pw_blocks(int n) {
    long long v = (long long)n * n * n / (kPwThreads * 4);
    return int(v < 1 ? 1 : (v > 1024 ? 1024 : v));
}
// Kernels without partial sums run on a wider grid (at 256^3: 8192 blocks,
// eight voxels per thread), which balances the arithmetic-heavy web adjoint.
inline int pw_blocks_wide(int n) {
    long long v = (long long)n * n * n / (kPwThreads * 8);
    return int(v < 1 ? 1 : (v > 8192 ? 8192 : v));
}

// Per-chain FP64 scalars kept on the device.
struct ChainScalars {
    double ntr;       // N_tr = sum n*
    double sumf;      // sum_i f_i
    double lnC;       // ln N_tr - ln sum f
    double loglik;    // sum_i log P_i
    double G;         // sum_i d log P_i / d ln nbar_i
    double gscale;    // G / N_tr
    double sumnu2;    // sum nu^2
    double logprior;  // log-normal prior of the bias tables
    double logpost;
    double sump2;     // sum p^2 (leapfrog)
    double dot;       // sum a b (bridge_dot)
    double gbias[32]; // d/d alpha_r then d/d beta_r
};

struct BiasD {        // double copy of a chain's table and prior (device)
    double a[16], alpha[16], rho[16], eps[16], rhop[16], epsp[16], beta[16];
    uint32_t prior_mask;
    double mu_alpha, sigma_alpha, mu_beta, sigma_beta;
};

// Reduction done by the last block of the kernel that writes the partial sums
// (a per-chain ticket counter, zero between launches, picks that block).
struct RedArgs {
    int* tickets;          // [batch], zero-initialised; each fused launch leaves it at zero
    ChainScalars* sc;
    const BiasD* bias;
    int n_regions;
};

struct Fields16 { void* p[16]; };

template <typename T>
cudaError_t launch_counts_prep(int n, int batch, const int32_t* counts, uint16_t* c16, double* partial, int* err,
                               const RedArgs& ra, cudaStream_t s);
template <typename T> cudaError_t launch_fill(long long count, T* p, T v, cudaStream_t s);
template <typename T>
cudaError_t launch_cic_scatter(int n, int batch, const Fields16& psi3, T* delta, cudaStream_t s);
template <typename T>
cudaError_t launch_pass_a(int n, int batch, const Fields16& th, const T* delta, T* lnf, T* beta_i,
                          const BiasT<T>* bias, const WebParams& wp, double* partial, const RedArgs& ra, cudaStream_t s);
template <typename T>
cudaError_t launch_pass_b(int n, int batch, const T* lnf, const T* beta_i, const uint16_t* c16, const T* nu,
                          const ChainScalars* sc, double* partial, const RedArgs& ra, cudaStream_t s);
template <typename T>
cudaError_t launch_web_adjoint(int n, int batch, const Fields16& th, const T* delta, const uint16_t* c16,
                               const BiasT<T>* bias, const WebParams& wp, const ChainScalars* sc,
                               const Fields16& out, double* partial, bool bias_grad, cudaStream_t s,
                               int blocks = 0);   // blocks per chain without bias_grad (0: built-in)
template <typename T> cudaError_t launch_shift(long long count, const T* in, T* out, T c, cudaStream_t s);
// CIC mass assignment in 64-bit fixed point (order-independent sums): zeroes acc (n^3 per chain)
// and scatters into it; launch_fixed_to_mass then writes the mass rho = 1 + delta.
template <typename T>
cudaError_t launch_cic_scatter_fixed(int n, int batch, const Fields16& psi3, unsigned long long* acc, cudaStream_t s);
template <typename T>
cudaError_t launch_fixed_to_mass(int n, int batch, const unsigned long long* acc, T* rho, cudaStream_t s);
// Radial redshift-space displacement in place (Sect. 2.9): psi += f (psi1 . r) r / |r|^2,
// r = q + psi - (n/2)(1,1,1) in cell units; psi, psi1: 3 real fields each, [B][n^3].
template <typename T>
cudaError_t launch_rsd_radial(int n, int batch, const Fields16& psi, const Fields16& psi1, double f, cudaStream_t s);
template <typename T>
cudaError_t launch_kick_drift(int n, int batch, T* p, T* nu, const T* g, double ck, double cd, double* partial,
                              cudaStream_t s);
// Per-chain FP64 sum of a b (partial sums reduced by the last block into sc[chain].dot).
template <typename T>
cudaError_t launch_dot(int n, int batch, const T* a, const T* b, double* partial, const RedArgs& ra, cudaStream_t s);
template <typename T>
cudaError_t launch_bias_kick_drift(int batch, int nr, uint32_t free_mask, double* theta, double* ptheta,
                                   const ChainScalars* sc, BiasD* bd, BiasT<T>* bt, double ck, double cd, cudaStream_t s);
template <typename T>
cudaError_t launch_delta_tr(int n, int batch, const uint16_t* c16, const ChainScalars* sc, T* out, cudaStream_t s);
template <typename T> cudaError_t launch_scale_chains(int n, int batch, T* g, const double* scale, cudaStream_t s);
template <typename T>
cudaError_t launch_lnnbar(long long nvox, int batch, const T* lnf, const ChainScalars* sc, T* out, cudaStream_t s);
template <typename T>
cudaError_t launch_eigs(int n, int batch, const Fields16& t6, const Fields16& out3, cudaStream_t s);

// Reductions of the block partials (one block per chain, fixed order); nblk =
// partial slots per chain (the grid of the kernel that wrote them).
cudaError_t launch_reduce(int what, int nblk, int batch, const double* partial, ChainScalars* sc, const BiasD* bias,
                          int n_regions, cudaStream_t s);
enum { RED_NTR = 0, RED_SUMF = 1, RED_LIK = 2, RED_BIASGRAD = 3, RED_P2 = 4, RED_DOT = 5 };


}  // namespace bridge
