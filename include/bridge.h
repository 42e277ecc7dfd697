/*
 * bridge.h -- C ABI of the GB300 (sm_103a) library for the differentiable
 * fuzzy-cosmic-web forward model and its adjoint (arXiv 2506.03969).
 *
 * The library evaluates, for B independent chains on one GPU,
 *
 *     log P(nu | n*) = log P(nu) + log L(n* | M(nu, b)) + log P(b)       (Eq. posterior)
 *
 * with M = M_b o M_Psi o M_delta (Sect. 2.1):
 *   M_delta : white noise nu -> linear field delta0 (App. A)
 *   M_Psi   : ALPT displacement, Psi = K o Psi_2LPT + (1-K) o Psi_SC (Sect. 2.3),
 *             then cloud-in-cell mass assignment -> evolved delta
 *   M_b     : Phi-web (tidal tensor) and, for 16 regions, delta-web (density
 *             Hessian) eigenvalues -> sigmoid memberships (Eq. sigmoid,
 *             Eq. soft_cweb_p; Sect. 2.7 hierarchy) -> per-voxel bias
 *             parameters -> Eq. local_bias -> normalisation C
 *   L       : negative binomial (gamma-Poisson, Sect. 2.6, Eq. log_likelihood)
 *   priors  : -1/2 |nu|^2 (constant dropped) and log-normal (Eq. lognormal) on
 *             alpha_r, beta_r for regions r in bias.prior_mask
 * and its gradient with respect to nu (hand-written adjoint of every step)
 * and to the alpha/beta bias tables, plus HMC leapfrog trajectories (Sect. 2.2).
 *
 * Conventions.
 *   Fields are C-order [chain][x][y][z] with N^3 cells of side L/N.  FP32
 *   configurations take float buffers, FP64 configurations double buffers.
 *   Wavenumbers k_j = 2 pi m_j / L; operators with an odd power of k_j set
 *   k_j = 0 on the Nyquist plane of axis j; 1/k^2 := 0 at k = 0.
 *   Eigenvalues are ordered lambda1 >= lambda2 >= lambda3; memberships are
 *   p^V = 1 - w1, p^S = w1 - w2, p^F = w2 - w3, p^K = w3 (regions V,S,F,K =
 *   0..3); 16-region models use region 4*j + k for Phi class j, delta class k.
 *
 * Alignment.  Device buffers passed to a context (nu, counts, p, outputs) must
 * start on a 16-byte boundary (every CUDA or PyTorch allocation does, and so
 * does any chain offset of a [B][N^3] buffer); otherwise the call returns
 * BRIDGE_EINVAL.
 *
 * Ownership.  The caller owns every buffer and the CUDA stream.  A context owns
 * its device workspace (allocated once in bridge_create, sized by
 * bridge_workspace_bytes) and releases it in bridge_destroy.  Calls on one
 * context are stream-ordered on its stream and must not overlap from several
 * host threads.
 *
 * Errors.  Every int-returning call returns a BRIDGE_* status; 0 is success.
 * On error the outputs are unspecified and bridge_last_error() describes the
 * cause.  There is no CPU fallback: without a usable GPU, bridge_create
 * returns BRIDGE_ENODEVICE.
 */
#ifndef BRIDGE_H
#define BRIDGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    BRIDGE_OK = 0,
    BRIDGE_EINVAL = 1,      /* bad shape, parameter, pointer or count value    */
    BRIDGE_ENOMEM = 2,      /* device or pinned-host allocation failed         */
    BRIDGE_ECUDA = 3,       /* a CUDA runtime call or kernel launch failed     */
    BRIDGE_ENONFINITE = 4,  /* log posterior or Hamiltonian is not finite      */
    BRIDGE_ETIMEOUT = 5,    /* a bounded device-side wait gave up              */
    BRIDGE_ENODEVICE = 6    /* no CUDA device of compute capability 10.3       */
};

enum { BRIDGE_FP32 = 0, BRIDGE_FP64 = 1 };

#define BRIDGE_MAX_REGIONS 16

/* Model and mesh configuration (one per context). */
typedef struct {
    int32_t n;               /* mesh side N: power of two, 16 <= N <= 512            */
    int32_t batch;           /* independent chains B >= 1                            */
    double box;              /* box side L [Mpc/h], > 0                              */
    double pk_amp;           /* P(k) = pk_amp k^pk_ns / (1 + (k/pk_kc)^2)^pk_pow     */
    double pk_ns, pk_kc, pk_pow;
    double growth_d;         /* linear growth D (1 at z = 0)                         */
    double d2_over_d2;       /* second-order growth D2 / D^2 (-3/7)                  */
    double r_s;              /* ALPT blend radius [Mpc/h] (Sect. 2.3: 4)             */
    double lambda_th_phi;    /* Phi-web eigenvalue threshold (Sect. 2.8)             */
    double lambda_th_delta;  /* delta-web eigenvalue threshold                       */
    double sharpness;        /* sigmoid steepness s (Eq. sigmoid)                    */
    int32_t n_regions;       /* 4: Phi-web; 16: Phi x delta web (Sect. 2.7)          */
    double rho_floor;        /* 1 + delta is floored at this value (> 0)             */
    int32_t precision;       /* BRIDGE_FP32, or BRIDGE_FP64 (the comparator path)    */
    int32_t recompute_alpt;  /* 0: the ALPT spectra (delta0, phi_ij, Psi; Sect. 2.3)
                                are kept from the forward pass for the adjoint;
                                1: the adjoint recomputes them from nu (10 fewer
                                half spectra in the workspace, about 39 R more HBM
                                traffic per gradient evaluation, R = N^3 floats)   */
    double rsd_f;            /* redshift space (Sect. 2.9, Eq. of delta(s), b_v = 1) with
                                the linear velocity v/(aH) = f Psi_1 (Psi_1 the
                                Zel'dovich displacement) applied before the mass
                                assignment; 0 = real space; finite                   */
    int32_t rsd_los;         /* line of sight when rsd_f != 0: 0 = plane-parallel
                                along z, Psi_z += f Psi_1,z; 1 = radial from an
                                observer at the centre of the volume, Psi += f
                                (Psi_1 . r) r / |r|^2 with r = q + Psi - (N/2)(1,1,1)
                                the particle's real-space position in cell units
                                relative to the observer (a particle at r = 0 is not
                                moved); 6 more half spectra in the workspace.  0 or 1 */
    int32_t deterministic;   /* 1: the CIC mass assignment sums in 64-bit fixed point
                                (FP32: units of 2^-40, FP64: 2^-50), independent of the
                                order of the atomic adds, so every result is identical
                                from run to run (8 N^3 bytes more workspace per chain,
                                one more launch); 0: float atomics, whose order varies
                                (results differ by rounding).  0 or 1              */
} bridge_config;

/* Bias table of one chain; entries [0, n_regions) are used (Eq. local_bias,
 * Sect. 2.6 beta, Eq. lognormal hyper-parameters). */
typedef struct {
    double a[BRIDGE_MAX_REGIONS];      /* amplitude per region (> 0)          */
    double alpha[BRIDGE_MAX_REGIONS];  /* power-law exponent                  */
    double rho[BRIDGE_MAX_REGIONS];    /* first cut-off scale (> 0)           */
    double eps[BRIDGE_MAX_REGIONS];    /* first cut-off exponent              */
    double rhop[BRIDGE_MAX_REGIONS];   /* second cut-off scale (>= 0; 0: off) */
    double epsp[BRIDGE_MAX_REGIONS];   /* second cut-off exponent (> 0)       */
    double beta[BRIDGE_MAX_REGIONS];   /* NB dispersion (> 0)                 */
    uint32_t prior_mask;               /* bit r: log-normal prior on alpha_r and beta_r */
    double mu_alpha, sigma_alpha;      /* log-normal hyper-parameters          */
    double mu_beta, sigma_beta;
    /* Free (sampled) bias parameters, whose gradient is returned.  With P free
     * parameters per kind, bit q of free_mask selects parameter q of the list
     * alpha_0 .. alpha_{P-1}, beta_0 .. beta_{P-1}.  tie_classes = 0: P =
     * n_regions, one parameter per table entry.  tie_classes = 1 (16 regions
     * only): P = 4, and alpha_j (beta_j) shifts the four entries 4j .. 4j+3 of
     * Phi-web class j together, so its derivative is the sum of theirs --
     * Sect. 3, Table 2: alpha and beta per Phi-web class, 8 free parameters
     * with free_mask = 0xFF.  Every chain of a call must use the same
     * free_mask and tie_classes. */
    uint32_t free_mask;
    int32_t tie_classes;
} bridge_bias;

typedef struct bridge_ctx bridge_ctx;

/* Host-only check of a configuration (no device needed).  Returns BRIDGE_OK or
 * BRIDGE_EINVAL. */
int bridge_validate_config(const bridge_config* cfg);

/* Device workspace a context with this configuration allocates, in bytes;
 * 0 if the configuration is invalid.  Host-only. */
size_t bridge_workspace_bytes(const bridge_config* cfg);

/* Amplitude A such that sigma(R) = sigma for P(k) = A k^ns/(1+(k/kc)^2)^pw,
 * sigma^2(R) = 1/(2 pi^2) int k^2 P(k) W(kR)^2 dk with the spherical top-hat
 * window W (normalisation of the linear spectrum, Sect. 2.1/App. A).  Composite
 * Simpson rule in ln k; host-only.  Returns a negative value on bad input. */
double bridge_pk_amplitude(double sigma, double radius, double ns, double kc, double pw);

/* Create a context on the current CUDA device for `cfg`, ordered on `stream`
 * (a cudaStream_t; NULL = legacy default stream).  Allocates the workspace.
 * *out is set only on success.  Errors: EINVAL, ENODEVICE, ENOMEM, ECUDA. */
int bridge_create(const bridge_config* cfg, void* stream, bridge_ctx** out);

/* Release a context and its workspace (after synchronising its stream).  NULL is a no-op. */
void bridge_destroy(bridge_ctx* ctx);

/* Forward model (Sect. 2.1).
 *   nu          device, [B][N][N][N] float or double (per precision), read only
 *   counts      device, [B][N][N][N] int32 tracer counts n* in [0, 65535]
 *               (EINVAL otherwise), read only
 *   bias        host, bias[B]
 *   ln_nbar_out device, [B][N^3] float/double: ln nbar_i; may be NULL
 *   logpost_out host, [B] doubles: log posterior; may be NULL
 * Every evaluating call synchronises the context stream before it returns (it
 * reads back the FP64 scalars and the count range check). */
int bridge_forward(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                   void* ln_nbar_out, double* logpost_out);

/* Log posterior and gradient (the "single-gradient evaluation" of Sect. 3.1).
 *   nu, counts, bias   as in bridge_forward
 *   logpost_out        host [B] doubles, may be NULL
 *   grad_nu_out        device [B][N^3] float/double: d log post / d nu; required
 *   grad_bias_out      host [B][popcount(free_mask)] doubles: d log post / d
 *                      (free bias parameter), in the bit order of
 *                      bias.free_mask; may be NULL (also not written when
 *                      free_mask = 0)
 * Synchronises the context stream before returning. */
int bridge_logpost_grad(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                        double* logpost_out, void* grad_nu_out, double* grad_bias_out);

/* The same evaluation with HOST buffers: nu_host, counts_host and
 * grad_nu_host are host arrays of the shapes above (pinned memory gives
 * asynchronous copies).  The call copies nu to device staging buffers owned by
 * the context (allocated on the first call), then copies and prepares the
 * counts on a second stream while the forward fields, which do not need them,
 * run; copies the gradient back and synchronises.  The host buffers must stay
 * valid and unchanged until the call returns; on an error no copy into them is
 * left in flight. */
int bridge_logpost_grad_host(bridge_ctx* ctx, const void* nu_host, const int32_t* counts_host,
                             const bridge_bias* bias, double* logpost_out, void* grad_nu_host,
                             double* grad_bias_out);

/* Vector-Jacobian product of the log posterior, the backward pass of reverse-
 * mode differentiation (Sect. 2.2: the sampler needs the gradient).  Nothing of
 * an earlier call is reused: the forward model is evaluated again from nu --
 * the ALPT displacement included -- and then its adjoint, so a forward-only
 * bridge_forward never pays for the adjoint.
 *   nu, counts, bias   as in bridge_logpost_grad
 *   cotangent          host [B] doubles: the upstream derivative c_b of each
 *                      chain's log posterior (finite); NULL means all ones
 *   grad_nu_out        device [B][N^3]: c_b d log post_b / d nu_b; required
 *   grad_bias_out      host [B][popcount(free_mask)]: c_b times the free-
 *                      parameter gradient; may be NULL
 * Synchronises the context stream.  Errors as bridge_logpost_grad; EINVAL for
 * a non-finite cotangent. */
int bridge_logpost_vjp(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                       const double* cotangent, void* grad_nu_out, double* grad_bias_out);

/* HMC leapfrog trajectory (Sect. 2.2), identity mass matrix, U = -log post:
 *   p <- p + eps/2 grad; nu <- nu + eps p; p <- p + eps/2 grad  (n_steps times)
 *   nu, p      device [B][N^3] float/double, updated in place
 *   counts     device int32 as above; bias host [B]
 *   h0_out/h1_out host [B] doubles: H = -log post + 1/2 |p|^2 before/after
 *              (FP64 sums); may be NULL.
 * Performs n_steps + 1 gradient evaluations.  n_steps >= 1, eps finite.
 * Chains are independent: the call writes h0 and h1 for every chain.  A chain
 * whose H0 or H1 is not finite (a diverged trajectory) gets its nu and p back
 * as they were at the start of the call, and the call returns ENONFINITE after
 * the whole batch has been integrated; the other chains keep their end points,
 * so the caller can accept or reject per chain from h0/h1.  On other errors
 * (EINVAL before any work, ECUDA) the contents of nu and p are unspecified. */
int bridge_leapfrog(bridge_ctx* ctx, void* nu, void* p, const int32_t* counts, const bridge_bias* bias,
                    int32_t n_steps, double eps, double* h0_out, double* h1_out);

/* Splitting integrators of Hamilton's equations for H = -log post + 1/2 |p|^2
 * (Sect. 2.2 names second- and fourth-order integrators and the Blanes et al.
 * 2014 variant).  One step is K(k_0) D(d_0) K(k_1) ... D(d_{s-1}) K(k_s) with
 * K(c): p <- p + c eps grad log post and D(d): nu <- nu + d eps p:
 *   BRIDGE_LEAPFROG      k = 1/2, 1/2; d = 1                       (s = 1)
 *   BRIDGE_TWO_STAGE     k = b, 1 - 2b, b; d = 1/2, 1/2, b = 0.211781 (Blanes,
 *                        Casas and Sanz-Serna 2014)                 (s = 2)
 *   BRIDGE_FOURTH_ORDER  three leapfrog sub-steps of w1 eps, w0 eps, w1 eps,
 *                        w1 = 1/(2 - 2^(1/3)), w0 = 1 - 2 w1 (Yoshida 1990) (s = 3)
 * A trajectory of n_steps takes s n_steps + 1 gradient evaluations. */
enum { BRIDGE_LEAPFROG = 0, BRIDGE_TWO_STAGE = 1, BRIDGE_FOURTH_ORDER = 2 };

/* A trajectory of `scheme` with the arguments, state handling and errors of
 * bridge_leapfrog (which is this call with BRIDGE_LEAPFROG).  EINVAL for an
 * unknown scheme. */
int bridge_integrate(bridge_ctx* ctx, void* nu, void* p, const int32_t* counts, const bridge_bias* bias,
                     int32_t scheme, int32_t n_steps, double eps, double* h0_out, double* h1_out);

/* Joint trajectory of the white noise and the free bias parameters (Sect. 2.1:
 * log-normal prior Eq. lognormal on b; Sect. 2.2: the chains sample nu and b
 * together).  The bias parameters move in log space, theta = ln b, so the
 * target gains the Jacobian of b = e^theta:
 *   H = -log post(nu, b = e^theta) - sum theta + 1/2 |p|^2 + 1/2 |p_theta|^2,
 * and every kick also updates p_theta with ck (b d log post/d b + 1), every
 * drift theta with cd p_theta (identity mass for both).
 *   nu, p           device [B][N^3], in/out, as in bridge_integrate
 *   theta, p_theta  host [B][popcount(free_mask)] doubles, in/out: ln of the
 *                   free parameters (bit order of free_mask over alpha_0 ..
 *                   alpha_{n-1}, beta_0 .. beta_{n-1}) and their momenta; the
 *                   free entries of bias[] are replaced by e^theta
 *   bias            host [B]; free_mask != 0 and tie_classes = 0 (untied)
 *   scheme, n_steps, eps, h0_out, h1_out as in bridge_integrate (H as above)
 * Each evaluation also computes the bias gradient (one more reduction).  A
 * chain whose H0 or H1 is not finite gets nu, p, theta and p_theta back as
 * they were, and the call returns ENONFINITE after the whole batch.  EINVAL
 * for tied or empty free sets and non-finite theta or p_theta. */
int bridge_integrate_joint(bridge_ctx* ctx, void* nu, void* p, double* theta, double* p_theta, const int32_t* counts,
                           const bridge_bias* bias, int32_t scheme, int32_t n_steps, double eps, double* h0_out,
                           double* h1_out);

/* Leapfrog steps for a sampler that drives the trajectory from the host (the
 * No-U-Turn sampler of Sect. 2.2 grows its trajectory one step at a time in
 * either direction).  Starting from (nu, p) and the gradient `grad` of the log
 * posterior at nu (from bridge_logpost_grad or an earlier call), applies
 * n_steps leapfrog steps of size eps (negative eps integrates backward):
 *   nu, p, grad   device [B][N^3], in/out; grad returns the gradient at the new nu
 *   logpost_out   host [B]: log posterior at the new nu; may be NULL
 * One gradient evaluation per step; synchronises.  Non-finite values are
 * returned as they are (the caller decides about divergence).  Errors: EINVAL,
 * ECUDA. */
int bridge_leapfrog_steps(bridge_ctx* ctx, void* nu, void* p, void* grad, const int32_t* counts,
                          const bridge_bias* bias, int32_t n_steps, double eps, double* logpost_out);

/* Per-chain dot product sum_i a_i b_i of two device fields [B][N^3] (float or
 * double per precision), products and sums in FP64, into host out[B] (for a
 * sampler's kinetic energy and U-turn test).  Synchronises. */
int bridge_dot(bridge_ctx* ctx, const void* a, const void* b, double* out);

/* Intermediate fields of the forward model, for inspection and testing.
 * Writes the field selected by `which` for all chains to device `out`:
 *   BRIDGE_FIELD_DELTA0   [B][N^3]     linear density delta0 (App. A)
 *   BRIDGE_FIELD_PSI      [B][3][N^3]  ALPT displacement in cell units (Sect. 2.3), in redshift
 *                                      space when rsd_f != 0 (the one the mass assignment uses)
 *   BRIDGE_FIELD_DELTA    [B][N^3]     CIC density contrast
 *   BRIDGE_FIELD_TIDAL    [B][6][N^3]  tidal tensor xx,xy,xz,yy,yz,zz (Sect. 2.8)
 *   BRIDGE_FIELD_HESSIAN  [B][6][N^3]  density Hessian (App. B; 16 regions only)
 *   BRIDGE_FIELD_LAMBDA   [B][3][N^3]  Phi-web eigenvalues, descending
 *   BRIDGE_FIELD_LNNBAR   [B][N^3]     ln nbar (needs counts for N_tr)
 * Element type follows the precision.  Runs the forward model. */
enum {
    BRIDGE_FIELD_DELTA0 = 0, BRIDGE_FIELD_PSI = 1, BRIDGE_FIELD_DELTA = 2, BRIDGE_FIELD_TIDAL = 3,
    BRIDGE_FIELD_HESSIAN = 4, BRIDGE_FIELD_LAMBDA = 5, BRIDGE_FIELD_LNNBAR = 6
};
int bridge_debug_field(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                       int32_t which, void* out);

/* Starting point of a chain (Sect. 2.2): the observed tracer density contrast
 * delta*_tr = n* N^3 / N_tr - 1 Wiener-filtered (Zaroubi et al. 1995) back to an
 * approximate linear field delta0^(0) and mapped to white noise nu^(0) by the
 * inverse of App. A.  Signal: the evolved linear field D delta0 with the known
 * power D^2 P(k); noise: Poisson shot noise of power L^3 / N_tr; no peculiar
 * motions.  Per mode k != 0 (the k = 0 mode, and so the mean of nu^(0), is 0):
 *   nu^(0)_hat = D sqrt(P dx^3) / (D^2 P + L^3 / N_tr) DFT(delta*_tr).
 *   counts   device [B][N^3] int32 tracer counts in [0, 65535]; every chain needs
 *            at least one tracer (EINVAL otherwise)
 *   nu_out   device [B][N^3] float/double: nu^(0)
 * Synchronises the context stream (several times: the filter depends on each
 * chain's N_tr).  Errors: EINVAL, ECUDA. */
int bridge_wiener_init(bridge_ctx* ctx, const int32_t* counts, void* nu_out);

/* The library's 3D real DFT and its inverse, without any operator between them:
 * out = IDFT(DFT(in)) for every chain, through the same z, y and x pass kernels
 * that carry every transform of the forward model and its adjoint (App. A
 * conventions: unnormalised forward DFT, inverse with 1/N^3).  For testing the
 * transforms and for timing them against a library FFT.
 *   in, out  device [B][N^3] float/double (per precision); may be the same buffer
 * Synchronises the context stream.  Errors: EINVAL (NULL, alignment), ECUDA. */
int bridge_fft_roundtrip(bridge_ctx* ctx, const void* in, void* out);

/* Per-kernel-class timing of later calls on this context: with enable != 0
 * every launch is bracketed by CUDA events recorded on the context stream (a
 * few microseconds of overhead per launch); the table is cleared.  Host-side;
 * errors: EINVAL for a NULL context. */
int bridge_profile_enable(bridge_ctx* ctx, int enable);

/* One row per kernel class since bridge_profile_enable: launches, summed
 * event-timed duration and summed algorithmic bytes (each launch's distinct
 * inputs read once and outputs written once). */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
    double bytes;
} bridge_profile_row;

/* Synchronises the stream and writes at most max_rows rows to `rows` (host);
 * returns the number written, or a negative BRIDGE_* status. */
int bridge_profile_read(bridge_ctx* ctx, bridge_profile_row* rows, int max_rows);

/* Launch-shape autotuner (no counterpart in the paper; a GB300 launch choice).
 * Times whole gradient evaluations of (nu, counts, bias) -- same arguments and
 * layout as bridge_logpost_grad, device buffers, 16-byte aligned -- and picks
 * for this context: CTAs per SM of the three fused real-space nodes (ALPT,
 * ALPT adjoint, CIC gather) among {built-in, 1..6, 8}, clamped to the
 * occupancy limit and to the context's node scratch, and thread blocks per
 * chain of the web/bias adjoint.  The tuned kernels compute the same values
 * under every choice (each tile or voxel is handled whole by one thread block);
 * only the time differs.  About 30 evaluations of the problem; the gradient scratch
 * of the context is overwritten and the captured CUDA graphs are dropped (the
 * next call re-captures them).  choices_out (host, 4 int32, may be NULL)
 * receives the choices, 0 meaning the built-in one.  Errors: EINVAL (NULL
 * context, buffers, alignment), ECUDA; on error every choice returns to the
 * built-in one. */
int bridge_autotune(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                    int32_t* choices_out);

/* Number of kernel launches the most recent call on this context issued. */
int64_t bridge_last_launch_count(const bridge_ctx* ctx);

/* Linear density delta0 = IDFT[ sqrt(P(k)/dx^3) DFT(nu) ] (M_delta, App. A)
 * without allocating device memory and without a context.  The paper has no
 * counterpart: this is an interface for callers that cannot allocate device
 * memory at the point where they need initial conditions (a fixed memory
 * budget, a pool owned by someone else, or code where a cudaMalloc would
 * synchronise the device), while bridge_create allocates a whole workspace.
 *
 *   cfg     n, batch, box, pk_amp, pk_ns, pk_kc, pk_pow and precision are used;
 *           the whole configuration must pass bridge_validate_config.
 *   nu      device [B][N^3] white noise (float or double per precision), read.
 *   delta0  device [B][N^3] output, same type; must not overlap nu.
 *   stream  CUDA stream (cudaStream_t) or NULL for the legacy default stream.
 *
 * The result equals BRIDGE_FIELD_DELTA0 of bridge_debug_field for the same
 * configuration and nu (the same kernels; only the radial factor table is
 * computed on the device instead of the host).
 *
 * Scratch.  The intermediate half spectra and the radial table live in one
 * static device array of 4 MiB inside the library: a call needs
 *   align256(B (N/2+1) N^2 * 2 * esz) + align256(2 (3 (N/2)^2 + 1) * esz)
 * bytes (esz = 4 or 8), e.g. N <= 64 with B = 1 in either precision, or B <= 3
 * at N = 64 in FP32.  Larger problems return BRIDGE_EINVAL before anything is
 * launched.  No part of the scratch has to start at zero.  The array is one
 * per device: calls whose work can overlap on the device (different streams,
 * or host threads with their own streams) race on it and give wrong results;
 * calls on one stream are ordered and safe.
 *
 * The first call on each device, made with that device current, looks up the
 * array's address (cudaGetSymbolAddress) and uploads the FFT twiddle tables;
 * make that first call outside any stream capture.  The library remembers
 * that set-up for the life of the process: after cudaDeviceReset on a device,
 * whose context then loses the array's contents and the tables, do not call
 * this entry point on that device again in the same process.
 *
 * Asynchronous: returns once the work is enqueued on `stream`; delta0 is
 * ready, and the scratch free for another stream, when the stream reaches the
 * end of this work.  Errors: EINVAL (config, NULL pointer, size limit),
 * ENODEVICE, ECUDA (launch failure); kernel faults surface at the caller's
 * next synchronisation.  bridge_last_error(NULL) describes the last failure
 * of this call on the calling thread. */
int bridge_delta0_noalloc(const bridge_config* cfg, const void* nu, void* delta0, void* stream);

/* Text of the last error on this context (never NULL; "" if none).  With a NULL
 * context: the reason the last bridge_create or bridge_delta0_noalloc on this
 * thread failed, or "context is NULL". */
const char* bridge_last_error(const bridge_ctx* ctx);

/* Static description of a status code. */
const char* bridge_status_string(int status);

#ifdef __cplusplus
}
#endif
#endif /* BRIDGE_H */
