// Host-visible launch interface of the FFT pass kernels (passes.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace bridge {

// Multiplier radial factors R(|k|) used by pass terms.
// R_WIENER: the Wiener-filter factor of the chain initialisation, written into
// the fifth radial table per call (it depends on the chain's tracer count).
enum RCode : int8_t { R_ONE = 0, R_INVK2 = 1, R_SQRTP = 2, R_KBLEND = 3, R_1MKBLEND = 4, R_WIENER = 5 };
constexpr int kRadialTables = 5;

// One linear term of a pass program:
//   out[dst] (+)= (cre + i cim) * kx^px * ky^py * kz^pz * R(|k|) * in[src]
// Odd powers vanish on the Nyquist index of their axis.
struct Term {
    int8_t src, dst, px, py, pz, rcode;
    double cre, cim;
};

constexpr int kMaxTerms = 16;
constexpr int kMaxFields = 16;

// A pass program: fields, chain strides (elements) and terms.  For the x node
// `merge` terms map inputs into the scalar spectrum Q (dst ignored) and
// `expand` terms map Q into outputs (src ignored).
struct PassProgram {
    int n_in, n_out, n_merge, n_expand;
    int accumulate;   // y inverse pass: 1 when several expand terms share an output (summed before the inverse DFT)
    const void* in[kMaxFields];
    void* out[kMaxFields];
    long long in_cs, out_cs;
    Term merge[kMaxTerms];
    Term expand[kMaxTerms];
};

// Physical constants for multipliers.
struct KParams {
    double kf;        // 2 pi / L
    double inv_kf2;   // 1 / kf^2
    double dx;        // L / N
    double pk_amp, pk_ns, pk_kc, pk_pow;
    double r_s;
    // Radial factors tabulated by the integer m^2 = mx^2 + my^2 + mz^2 (k^2 = kf^2 m^2),
    // computed on the host in FP64: table c-1 holds R_c for c = R_INVK2 .. R_WIENER.
    const void* rtab;
    int rlen;         // entries per table: 3 (N/2)^2 + 1
    // FP32 copies of kf and 1/kf^2, so that FP32 kernels read no double
    // parameter (a double -> float conversion runs on the narrow FP64 pipe)
    float kf_f, inv_kf2_f;
    void set_fp32() { kf_f = float(kf); inv_kf2_f = float(inv_kf2); }
};
template <typename T> __device__ __forceinline__ T kf_of(const KParams& kp) {
    if constexpr (sizeof(T) == 4) return kp.kf_f;
    else return T(kp.kf);
}

// Fill the radial tables (host, FP64): out[(c-1) * rlen + m2] for c = 1..4.
void radial_tables_host(int n, const KParams& kp, double* out);

// Real-space z pass.  Fields: in[f] / out[f] for f < n_fields; chain strides in elements.
struct ZProgram {
    int n_fields;
    const void* in[kMaxFields];
    void* out[kMaxFields];
    long long in_cs, out_cs;
    // inverse pass only: when sub[0] is set, out[f] = IDFT(in[f]) - sub[f] (sub: real
    // fields with the layout and chain stride of out; may be out itself)
    const void* sub[kMaxFields];
};

template <typename T> cudaError_t launch_z_fwd(int n, int batch, const ZProgram& p, cudaStream_t s);
template <typename T> cudaError_t launch_z_inv(int n, int batch, const ZProgram& p, cudaStream_t s);
// y pass: forward (merge) or inverse (expand) with ky/kz monomial terms
template <typename T> cudaError_t launch_y_fwd(int n, int batch, const PassProgram& p, const KParams& kp, cudaStream_t s);
template <typename T> cudaError_t launch_y_inv(int n, int batch, const PassProgram& p, const KParams& kp, cudaStream_t s);
// x node: forward x DFT of the inputs, merge into Q, expand, inverse x DFT of the outputs
template <typename T> cudaError_t launch_x_node(int n, int batch, const PassProgram& p, const KParams& kp, cudaStream_t s);

// Upload the twiddle tables (host FP64 cos/sin, rounded per precision).
cudaError_t upload_twiddles();

}  // namespace bridge
