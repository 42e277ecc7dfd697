// C ABI of the library: context, workspace plan, the pass programs of the
// forward model and of its adjoint, and the leapfrog driver.
#include <cmath>
#include <cstdio>
#include <algorithm>
#include <cstring>
#include <initializer_list>
#include <string>
#include <vector>

#include "../../include/bridge.h"
#include "common.cuh"
#include "passes.cuh"
#include "pointwise.cuh"
#include "nodes.cuh"

using namespace bridge;

namespace {

// Spectral buffers: 19 scratch slots (peak use: adjoint y merge 13 -> 6).  The
// tidal tensor and density Hessian spectra (12) exist only inside the forward
// pass and use scratch slots 7..18.  The ALPT spectra -- linear field and
// potential Hessian (7), displacement (3) -- feed the adjoint's fused nodes:
// by default they have slots of their own (19..28) and survive from the
// forward pass to the adjoint; with recompute_alpt they are recomputed from nu
// inside the adjoint into scratch slots 7..13 and 14..16, and the workspace
// holds 19 spectra instead of 29.
// The adjoint keeps g_Psi_z (the gather node's third output) in scratch slot 17
// until the delta0 adjoint, which the redshift-space term feeds.
// The radial line of sight adds six slots after the others: the linear
// displacement Psi_1 (3, kept like Psi) and its adjoint from the gather node (3).
enum { SP_SCR = 0, SP_TH = 7, SP_ALPT_STORED = 19, SP_PSI_STORED = 26, kMaxSpec = 29,
       SP_ALPT_RECOMP = 7, SP_PSI_RECOMP = 14, SP_GPSIZ = 17, kScratchSpec = 19, kRadialSpec = 6 };
// Real buffers.
enum {
    RB_DELTA = 0,   // 1: CIC mass rho = 1 + delta
    RB_LNF = 1,     // 2: ln f, beta_i
    RB_GD = 3,      // 1: g_rho (input of the CIC gather)
    RB_TH = 4,      // 12: tidal tensor (6) and density Hessian (6) in real space
    RB_SCR = 16,    // 13: adjoint fields of the web stage; scratch for inspection fields
    kMaxReal = 29
};
// Extra real fields after the named ones: leapfrog gradient, snapshots of nu and p.
enum { kExtraReal = 3 };

Term mk(int src, int dst, int px, int py, int pz, RCode rc, double cre, double cim = 0.0) {
    Term t;
    t.src = (int8_t)src; t.dst = (int8_t)dst; t.px = (int8_t)px; t.py = (int8_t)py; t.pz = (int8_t)pz;
    t.rcode = rc; t.cre = cre; t.cim = cim;
    return t;
}

}  // namespace

struct bridge_ctx {
    bridge_config cfg{};
    cudaStream_t stream = nullptr;
    int device = 0;
    std::string err;
    int64_t launches = 0;
    int n = 0, B = 0, nr = 4;
    int sp_alpt = SP_ALPT_STORED, sp_psi = SP_PSI_STORED;   // ALPT spectrum slots (recompute_alpt moves them)
    bool recompute = false;
    bool radial = false;                 // radial line of sight (rsd_f != 0, rsd_los = 1)
    unsigned long long* fixed_acc = nullptr;   // deterministic CIC: 64-bit fixed-point mass per cell
    int sp_psi1 = 0, sp_gpsi1 = 0;       // its Psi_1 and g_Psi_1 slots
    long long nvox = 0, nspec = 0;
    size_t esz = 4;
    // workspace
    void* ws = nullptr;
    size_t ws_bytes = 0;
    void* spec[kMaxSpec + kRadialSpec] = {};
    void* real[kMaxReal] = {};
    uint16_t* c16 = nullptr;
    double* partial = nullptr;
    ChainScalars* sc = nullptr;
    BiasD* biasd = nullptr;
    void* biast = nullptr;
    int* errflag = nullptr;
    int* tickets = nullptr;     // [B] counters of the fused partial-sum reductions (zero between launches)
    void* grad_tmp = nullptr;   // gradient scratch for leapfrog
    void* snap_nu = nullptr;    // leapfrog start state, restored for chains whose Hamiltonian is not finite
    void* snap_p = nullptr;
    double* cot = nullptr;      // [B] cotangents of bridge_logpost_vjp (device)
    double* theta = nullptr;    // [B][32] log of the free bias parameters (joint integration, device)
    double* ptheta = nullptr;   // [B][32] their momenta
    uint32_t jmask = 0;         // free_mask of the joint integration in progress
    double* cot_host = nullptr; // pinned staging of cot
    void* node_scratch = nullptr;  // per-CTA slabs of the fused nodes
    size_t node_cap = 0;           // bytes of node_scratch
    // launch choices (bridge_autotune; 0 = built-in): CTAs per SM of the ALPT,
    // ALPT-adjoint and gather nodes, blocks per chain of the web adjoint
    int tune[4] = {0, 0, 0, 0};
    void* rtab = nullptr;          // radial k-space factor tables (see KParams)
    // host e2e buffers
    void* h_nu = nullptr;
    int32_t* h_counts = nullptr;
    void* h_grad = nullptr;
    // pinned host staging
    ChainScalars* sc_host = nullptr;
    BiasD* biasd_host = nullptr;
    void* biast_host = nullptr;
    int* errflag_host = nullptr;
    KParams kp{};
    WebParams wp{};
    // gradient-evaluation graph (captured once per buffer set, replayed per call)
    cudaGraphExec_t eexec = nullptr;
    const void* ekey[4] = {nullptr, nullptr, nullptr, nullptr};
    int64_t elaunches = 0;
    // leapfrog step graph (captured on a private stream, replayed per step)
    cudaStream_t gstream = nullptr;
    cudaGraphExec_t gexec = nullptr;
    const void* gkey[3] = {nullptr, nullptr, nullptr};
    std::vector<double> gck, gcd;   // unit coefficients of the captured interior step
    uint32_t gjoint = 0;            // free_mask of a captured joint step (0: fields only)
    int64_t glaunches = 0;
    cudaEvent_t gev[2] = {nullptr, nullptr};
    // host-buffer evaluation: the counts are copied and prepared on cstream while the two
    // graphs (forward fields; likelihood + adjoint) run on gstream
    cudaStream_t cstream = nullptr;
    cudaEvent_t hev[2] = {nullptr, nullptr};
    cudaGraphExec_t hexec[2] = {nullptr, nullptr};
    int64_t hlaunches[2] = {0, 0};
    int hkey = -1;                  // bias_grad of the captured second graph
    const int32_t* hcounts = nullptr;   // set by bridge_logpost_grad_host for one call
    // per-launch CUDA-event profiling (bridge_profile_enable)
    bool prof = false;
    struct ProfRec { const char* name; double bytes; cudaEvent_t a, b; };
    std::vector<ProfRec> prof_recs;
    std::vector<cudaEvent_t> prof_pool;
    size_t prof_used = 0;
};

namespace {

int fail(bridge_ctx* c, int st, const std::string& msg) {
    if (c) c->err = msg;
    return st;
}

// CK: a CUDA runtime call; CKL: a kernel launch (counted).
#define CK(call)                                                                         \
    do {                                                                                 \
        cudaError_t e_ = (call);                                                         \
        if (e_ != cudaSuccess)                                                           \
            return fail(ctx, BRIDGE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)
#define CKL(name, bytes, call)                              \
    do {                                                    \
        cudaEvent_t pa_ = nullptr, pb_ = nullptr;           \
        if (ctx->prof) {                                    \
            pa_ = prof_event(ctx); pb_ = prof_event(ctx);   \
            if (pa_) cudaEventRecord(pa_, ctx->stream);     \
        }                                                   \
        CK(call);                                           \
        ++ctx->launches;                                    \
        if (pb_) {                                          \
            cudaEventRecord(pb_, ctx->stream);              \
            ctx->prof_recs.push_back({name, double(bytes), pa_, pb_}); \
        }                                                   \
    } while (0)

cudaEvent_t prof_event(bridge_ctx* ctx) {
    if (ctx->prof_used == ctx->prof_pool.size()) {
        if (ctx->prof_pool.size() >= 1u << 16) return nullptr;
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
        ctx->prof_pool.push_back(e);
    }
    return ctx->prof_pool[ctx->prof_used++];
}
inline RedArgs red_args(bridge_ctx* c) { return RedArgs{c->tickets, c->sc, c->biasd, c->nr}; }
template <typename T> double rby(const bridge_ctx* c) { return double(c->nvox) * c->B * sizeof(T); }
template <typename T> double sby(const bridge_ctx* c) { return double(c->nspec) * c->B * 2 * sizeof(T); }
inline double c16b(const bridge_ctx* c) { return double(c->nvox) * c->B * 2; }
inline int nth_of(const bridge_ctx* c) { return c->nr == 16 ? 12 : 6; }

bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

int validate(const bridge_config* c, std::string* why) {
    auto bad = [&](const char* m) { if (why) *why = m; return BRIDGE_EINVAL; };
    if (!c) return bad("config is NULL");
    if (!is_pow2(c->n) || c->n < 16 || c->n > 512) return bad("n must be a power of two in [16, 512]");
    if (c->batch < 1 || c->batch > 4096) return bad("batch must be in [1, 4096]");
    if (!(c->box > 0) || !std::isfinite(c->box)) return bad("box must be positive and finite");
    if (!(c->pk_amp >= 0) || !std::isfinite(c->pk_amp)) return bad("pk_amp must be >= 0 and finite");
    if (!(c->pk_kc > 0) || !std::isfinite(c->pk_ns) || !std::isfinite(c->pk_pow)) return bad("bad P(k) parameters");
    if (!std::isfinite(c->growth_d) || !std::isfinite(c->d2_over_d2)) return bad("bad growth factors");
    if (!(c->r_s >= 0) || !std::isfinite(c->r_s)) return bad("r_s must be >= 0 and finite");
    if (!std::isfinite(c->lambda_th_phi) || !std::isfinite(c->lambda_th_delta)) return bad("bad thresholds");
    if (!(c->sharpness > 0) || !std::isfinite(c->sharpness)) return bad("sharpness must be positive");
    if (c->n_regions != 4 && c->n_regions != 16) return bad("n_regions must be 4 or 16");
    if (!(c->rho_floor > 0) || !(c->rho_floor < 1)) return bad("rho_floor must be in (0, 1)");
    if (c->precision != BRIDGE_FP32 && c->precision != BRIDGE_FP64) return bad("precision must be FP32 or FP64");
    if (c->recompute_alpt != 0 && c->recompute_alpt != 1) return bad("recompute_alpt must be 0 or 1");
    if (!std::isfinite(c->rsd_f)) return bad("rsd_f must be finite");
    if (c->rsd_los != 0 && c->rsd_los != 1) return bad("rsd_los must be 0 (plane-parallel) or 1 (radial)");
    if (c->deterministic != 0 && c->deterministic != 1) return bad("deterministic must be 0 or 1");
    return BRIDGE_OK;
}

int validate_bias(const bridge_ctx* ctx, const bridge_bias* b, std::string* why) {
    if (!b) { *why = "bias is NULL"; return BRIDGE_EINVAL; }
    for (int ch = 0; ch < ctx->B; ++ch) {
        const bridge_bias& x = b[ch];
        for (int r = 0; r < ctx->nr; ++r) {
            if (!(x.a[r] > 0) || !(x.rho[r] > 0) || !(x.beta[r] > 0) || !(x.rhop[r] >= 0) || !(x.epsp[r] > 0) ||
                !std::isfinite(x.alpha[r]) || !std::isfinite(x.eps[r]) || !std::isfinite(x.a[r]) ||
                !std::isfinite(x.rho[r]) || !std::isfinite(x.beta[r]) || !std::isfinite(x.rhop[r]) ||
                !std::isfinite(x.epsp[r])) {
                *why = "bias table entry out of range (a, rho, beta, eps' > 0; rho' >= 0; all finite)";
                return BRIDGE_EINVAL;
            }
        }
        if (x.prior_mask & ~((ctx->nr == 16) ? 0xFFFFu : 0xFu)) { *why = "prior_mask has bits beyond n_regions"; return BRIDGE_EINVAL; }
        if (x.tie_classes != 0 && x.tie_classes != 1) { *why = "tie_classes must be 0 or 1"; return BRIDGE_EINVAL; }
        if (x.tie_classes && ctx->nr != 16) { *why = "tie_classes needs 16 regions"; return BRIDGE_EINVAL; }
        const int np = x.tie_classes ? 4 : ctx->nr;
        if (np < 16 && (x.free_mask >> (2 * np)) != 0u) { *why = "free_mask has bits beyond 2 x (free parameters per kind)"; return BRIDGE_EINVAL; }
        if (x.free_mask != b[0].free_mask || x.tie_classes != b[0].tie_classes) {
            *why = "free_mask and tie_classes must be the same for every chain of a call";
            return BRIDGE_EINVAL;
        }
        if (x.prior_mask) {
            for (int r = 0; r < ctx->nr; ++r)
                if (((x.prior_mask >> r) & 1u) && !(x.alpha[r] > 0)) { *why = "log-normal prior needs alpha > 0"; return BRIDGE_EINVAL; }
            if (!(x.sigma_alpha > 0) || !(x.sigma_beta > 0)) { *why = "prior sigma must be > 0"; return BRIDGE_EINVAL; }
        }
    }
    return BRIDGE_OK;
}

struct Plan {
    size_t spec_bytes, real_bytes, c16_bytes, partial_bytes, sc_bytes, biasd_bytes, biast_bytes, node_bytes, rtab_bytes,
        cot_bytes, fixed_bytes, total;
    int nspec_buf, nreal_buf;
};

size_t align_up(size_t v) { return (v + 255) & ~size_t(255); }

Plan make_plan(const bridge_config* c) {
    Plan p{};
    const long long n = c->n, B = c->batch;
    const size_t esz = c->precision == BRIDGE_FP64 ? 8 : 4;
    const long long nvox = n * n * n, nspec = (n / 2 + 1) * n * n;
    p.nspec_buf = (c->recompute_alpt ? kScratchSpec : kMaxSpec) + (c->rsd_f != 0.0 && c->rsd_los == 1 ? kRadialSpec : 0);
    p.nreal_buf = kMaxReal;
    p.spec_bytes = align_up(size_t(nspec) * 2 * esz * B);
    p.real_bytes = align_up(size_t(nvox) * esz * B);
    p.c16_bytes = align_up(size_t(nvox) * 2 * B);
    // partial sums: one row per block of the real-space kernels
    const size_t max_blocks = size_t(pw_blocks(c->n));
    p.partial_bytes = align_up(size_t(B) * max_blocks * 32 * sizeof(double));
    p.sc_bytes = align_up(sizeof(ChainScalars) * B);
    p.biasd_bytes = align_up(sizeof(BiasD) * B);
    p.biast_bytes = align_up(sizeof(BiasT<double>) * B);
    p.node_bytes = align_up(size_t(BRIDGE_NODE_L2_MB + 8) << 20);   // fused-node slabs (the launcher keeps them below the budget)
    p.rtab_bytes = align_up(size_t(kRadialTables) * (3 * (n / 2) * (n / 2) + 1) * esz);
    p.cot_bytes = align_up(sizeof(double) * B) + 2 * align_up(sizeof(double) * 32 * B);
    p.fixed_bytes = c->deterministic ? align_up(size_t(nvox) * 8 * B) : 0;   // 64-bit CIC accumulator
    p.total = p.spec_bytes * p.nspec_buf + p.real_bytes * (p.nreal_buf + kExtraReal) + p.c16_bytes + p.partial_bytes +
              p.sc_bytes + p.biasd_bytes + p.biast_bytes + p.node_bytes + p.rtab_bytes + p.cot_bytes + p.fixed_bytes + 256;
    return p;
}

template <typename T> T* RB(bridge_ctx* c, int i) { return reinterpret_cast<T*>(c->real[i]); }
template <typename T> cplx_t<T>* SB(bridge_ctx* c, int i) { return reinterpret_cast<cplx_t<T>*>(c->spec[i]); }

Fields16 fields(bridge_ctx* c, int first, int count) {
    Fields16 f{};
    for (int i = 0; i < count; ++i) f.p[i] = c->real[first + i];
    return f;
}

// --- z pass helpers ---------------------------------------------------------
template <typename T> int z_fwd(bridge_ctx* ctx, std::vector<const void*> in, std::vector<void*> out) {
    ZProgram p{};
    p.n_fields = (int)in.size();
    for (int i = 0; i < p.n_fields; ++i) { p.in[i] = in[i]; p.out[i] = out[i]; }
    p.in_cs = ctx->nvox;
    p.out_cs = ctx->nspec;
    CKL("z_fwd", p.n_fields * (rby<T>(ctx) + sby<T>(ctx)), launch_z_fwd<T>(ctx->n, ctx->B, p, ctx->stream));
    return BRIDGE_OK;
}
template <typename T> int z_inv(bridge_ctx* ctx, std::vector<const void*> in, std::vector<void*> out) {
    ZProgram p{};
    p.n_fields = (int)in.size();
    for (int i = 0; i < p.n_fields; ++i) { p.in[i] = in[i]; p.out[i] = out[i]; }
    p.in_cs = ctx->nspec;
    p.out_cs = ctx->nvox;
    CKL("z_inv", p.n_fields * (rby<T>(ctx) + sby<T>(ctx)), launch_z_inv<T>(ctx->n, ctx->B, p, ctx->stream));
    return BRIDGE_OK;
}

PassProgram program(std::vector<const void*> in, std::vector<void*> out, long long cs) {
    PassProgram p{};
    p.n_in = (int)in.size();
    p.n_out = (int)out.size();
    for (int i = 0; i < p.n_in; ++i) p.in[i] = in[i];
    for (int i = 0; i < p.n_out; ++i) p.out[i] = out[i];
    p.in_cs = p.out_cs = cs;
    return p;
}
void add_merge(PassProgram& p, Term t) { p.merge[p.n_merge++] = t; }
void add_expand(PassProgram& p, Term t) { p.expand[p.n_expand++] = t; }

template <typename T> std::vector<const void*> cspec(bridge_ctx* c, int first, int count) {
    std::vector<const void*> v;
    for (int i = 0; i < count; ++i) v.push_back(c->spec[first + i]);
    return v;
}
template <typename T> std::vector<void*> mspec(bridge_ctx* c, int first, int count) {
    std::vector<void*> v;
    for (int i = 0; i < count; ++i) v.push_back(c->spec[first + i]);
    return v;
}
std::vector<const void*> creal(bridge_ctx* c, int first, int count) {
    std::vector<const void*> v;
    for (int i = 0; i < count; ++i) v.push_back(c->real[first + i]);
    return v;
}
std::vector<void*> mreal(bridge_ctx* c, int first, int count) {
    std::vector<void*> v;
    for (int i = 0; i < count; ++i) v.push_back(c->real[first + i]);
    return v;
}

// identity y pass (forward or inverse) on `count` fields, in place
template <typename T> int y_identity(bridge_ctx* ctx, int first, int count, bool fwd) {
    PassProgram p = program(cspec<T>(ctx, first, count), mspec<T>(ctx, first, count), ctx->nspec);
    for (int i = 0; i < count; ++i) {
        if (fwd) add_merge(p, mk(i, i, 0, 0, 0, R_ONE, 1.0));
        else add_expand(p, mk(i, i, 0, 0, 0, R_ONE, 1.0));
    }
    if (fwd) CKL("y_fwd", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_fwd<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    else CKL("y_inv", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_inv<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    return BRIDGE_OK;
}

#define RUN(x) do { int st_ = (x); if (st_ != BRIDGE_OK) return st_; } while (0)

// Fused node launch: fills the common arguments and reports the grid.
template <typename T> int node(bridge_ctx* ctx, NodeArgs& na, const char* name, double bytes, int* grid_used) {
    na.scratch = ctx->node_scratch;
    na.scratch_bytes = ctx->node_cap;
    na.cps = na.kind == NODE_ALPT_FWD ? ctx->tune[0] : na.kind == NODE_ALPT_ADJ ? ctx->tune[1] : ctx->tune[2];
    na.growth = ctx->cfg.growth_d;
    na.d2 = ctx->cfg.d2_over_d2 * ctx->cfg.growth_d * ctx->cfg.growth_d;
    na.growth_f = float(na.growth);
    na.d2_f = float(na.d2);
    na.rsd_f = ctx->cfg.rsd_f;
    na.rsd_f_f = float(na.rsd_f);
    int g = 0;
    CKL(name, bytes, launch_node<T>(ctx->n, ctx->B, na, &g, ctx->stream));
    if (grid_used) *grid_used = g;
    return BRIDGE_OK;
}

// ---------------------------------------------------------------------------
// M_delta and the ALPT displacement (App. A, Sect. 2.3): nu -> the spectra of
// delta0 and phi_ij (slots sp_alpt..+6) and of Psi in cell units (sp_psi..+2),
// in the [kz][y][x] layout of the z pass.  Uses scratch slots 0..4.
// ---------------------------------------------------------------------------
template <typename T> int run_alpt(bridge_ctx* ctx, const T* nu) {
    const double invn3 = 1.0 / double(ctx->nvox);
    // M_delta (App. A) and the linear potential Hessian: nu -> delta0, phi_ij spectra
    RUN(z_fwd<T>(ctx, {nu}, {ctx->spec[SP_SCR]}));
    RUN(y_identity<T>(ctx, SP_SCR, 1, true));
    {
        PassProgram p = program(cspec<T>(ctx, SP_SCR, 1), mspec<T>(ctx, SP_SCR + 1, 4), ctx->nspec);
        add_merge(p, mk(0, 0, 0, 0, 0, R_SQRTP, invn3));
        add_expand(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));    // W0 -> delta0
        add_expand(p, mk(0, 1, 2, 0, 0, R_INVK2, 1.0));  // V2 = kx^2/k^2
        add_expand(p, mk(0, 2, 1, 0, 0, R_INVK2, 1.0));  // V1 = kx/k^2
        add_expand(p, mk(0, 3, 0, 0, 0, R_INVK2, 1.0));  // V0 = 1/k^2
        CKL("x_node", (p.n_in + p.n_out) * sby<T>(ctx), launch_x_node<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    {
        PassProgram p = program(cspec<T>(ctx, SP_SCR + 1, 4), mspec<T>(ctx, ctx->sp_alpt, 7), ctx->nspec);
        add_expand(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));    // delta0
        add_expand(p, mk(1, 1, 0, 0, 0, R_ONE, 1.0));    // phi_xx
        add_expand(p, mk(2, 2, 0, 1, 0, R_ONE, 1.0));    // phi_xy
        add_expand(p, mk(2, 3, 0, 0, 1, R_ONE, 1.0));    // phi_xz
        add_expand(p, mk(3, 4, 0, 2, 0, R_ONE, 1.0));    // phi_yy
        add_expand(p, mk(3, 5, 0, 1, 1, R_ONE, 1.0));    // phi_yz
        add_expand(p, mk(3, 6, 0, 0, 2, R_ONE, 1.0));    // phi_zz
        CKL("y_inv", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_inv<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    // ALPT sources (Sect. 2.3) on the fly: inverse z of delta0, phi -> a, theta_SC -> forward z
    {
        NodeArgs na{};
        na.kind = NODE_ALPT_FWD;
        for (int f = 0; f < 7; ++f) na.spec_in[f] = ctx->spec[ctx->sp_alpt + f];
        na.spec_out[0] = ctx->spec[SP_SCR];
        na.spec_out[1] = ctx->spec[SP_SCR + 1];
        RUN(node<T>(ctx, na, "node_alpt", 9 * sby<T>(ctx), nullptr));
    }
    RUN(y_identity<T>(ctx, SP_SCR, 2, true));
    // the radial line of sight also needs V1 = kx delta0_hat / k^2 (slot 3) for Psi_1,x: the
    // blend then writes to slots 5, 6 instead of 2, 3
    const int sp_blend = ctx->radial ? SP_SCR + 5 : SP_SCR + 2;
    {
        PassProgram p = program(cspec<T>(ctx, SP_SCR, 2), mspec<T>(ctx, sp_blend, 2), ctx->nspec);
        add_merge(p, mk(0, 0, 0, 0, 0, R_KBLEND, invn3));
        add_merge(p, mk(1, 0, 0, 0, 0, R_1MKBLEND, invn3));
        const double c = -1.0 / ctx->kp.dx;               // Psi_j = -i k_j theta / (k^2 dx)
        add_expand(p, mk(0, 0, 1, 0, 0, R_INVK2, 0.0, c));
        add_expand(p, mk(0, 1, 0, 0, 0, R_INVK2, 0.0, c));
        CKL("x_node", (p.n_in + p.n_out) * sby<T>(ctx), launch_x_node<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    if (ctx->radial) {
        // radial line of sight (Sect. 2.9): Psi and the linear displacement Psi_1 = (i D / dx) k
        // delta0_hat / k^2 separately, Psi_1,x from V1 (slot 3), Psi_1,y and Psi_1,z from V0
        // (slot 4); the per-particle projection on the line of sight follows in real space
        std::vector<const void*> in = {ctx->spec[SP_SCR + 5], ctx->spec[SP_SCR + 6], ctx->spec[SP_SCR + 3],
                                       ctx->spec[SP_SCR + 4]};
        std::vector<void*> out = mspec<T>(ctx, ctx->sp_psi, 3);
        for (int j = 0; j < 3; ++j) out.push_back(ctx->spec[ctx->sp_psi1 + j]);
        PassProgram p = program(in, out, ctx->nspec);
        const double c1 = ctx->cfg.growth_d / ctx->kp.dx;
        add_expand(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));
        add_expand(p, mk(1, 1, 0, 1, 0, R_ONE, 1.0));
        add_expand(p, mk(1, 2, 0, 0, 1, R_ONE, 1.0));
        add_expand(p, mk(2, 3, 0, 0, 0, R_ONE, 0.0, c1));
        add_expand(p, mk(3, 4, 0, 1, 0, R_ONE, 0.0, c1));
        add_expand(p, mk(3, 5, 0, 0, 1, R_ONE, 0.0, c1));
        CKL("y_inv", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_inv<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
        return BRIDGE_OK;
    }
    {
        // redshift space (Sect. 2.9), plane-parallel along z with the linear velocity
        // v/(aH) = f Psi_1: Psi_z += f Psi_1,z = (i f D / dx) kz V0, V0 = delta0_hat / k^2 (the
        // first x node's output, still in slot 4), summed into Psi_z before its inverse y DFT
        const bool rsd = ctx->cfg.rsd_f != 0.0;
        PassProgram p = program(cspec<T>(ctx, SP_SCR + 2, rsd ? 3 : 2), mspec<T>(ctx, ctx->sp_psi, 3), ctx->nspec);
        add_expand(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));
        add_expand(p, mk(1, 1, 0, 1, 0, R_ONE, 1.0));
        add_expand(p, mk(1, 2, 0, 0, 1, R_ONE, 1.0));
        if (rsd) {
            add_expand(p, mk(2, 2, 0, 0, 1, R_ONE, 0.0, ctx->cfg.rsd_f * ctx->cfg.growth_d / ctx->kp.dx));
            p.accumulate = 1;
        }
        CKL("y_inv", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_inv<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    return BRIDGE_OK;
}

// The displacement the mass assignment uses, in real space at real buffers
// first..first+2: Psi, or with the radial line of sight Psi shifted by
// f (Psi_1 . r) r / |r|^2 (Psi_1 passes through first+3..first+5).
template <typename T> int psi_real(bridge_ctx* ctx, int first) {
    if (!ctx->radial) return z_inv<T>(ctx, cspec<T>(ctx, ctx->sp_psi, 3), mreal(ctx, first, 3));
    std::vector<const void*> in = cspec<T>(ctx, ctx->sp_psi, 3);
    for (int j = 0; j < 3; ++j) in.push_back(ctx->spec[ctx->sp_psi1 + j]);
    RUN(z_inv<T>(ctx, in, mreal(ctx, first, 6)));
    CKL("rsd_radial", 9 * rby<T>(ctx), launch_rsd_radial<T>(ctx->n, ctx->B, fields(ctx, first, 3), fields(ctx, first + 3, 3),
                                                            ctx->cfg.rsd_f, ctx->stream));
    return BRIDGE_OK;
}

// ---------------------------------------------------------------------------
// Forward model.  Leaves in the workspace: the ALPT and displacement spectra
// (unless recompute_alpt), rho, the tensors in real space, ln f and beta_i,
// and the scalars (ntr, sumf, lnC, loglik, G, logpost).  nu: device [B][N^3].
// ---------------------------------------------------------------------------
// run_forward_fields: every step up to the tensors in real space (needs no counts);
// run_forward_lik: the web/bias pass and the likelihood (needs the counts prepared).
template <typename T> int run_forward_fields(bridge_ctx* ctx, const T* nu) {
    const double invn3 = 1.0 / double(ctx->nvox);
    const bool hier = ctx->nr == 16;
    const int nth = nth_of(ctx);
    RUN(run_alpt<T>(ctx, nu));
    // CIC (mass rho accumulated into a zeroed field); the displacement in real
    // space borrows the tensor buffers, which are written only afterwards
    RUN(psi_real<T>(ctx, RB_TH));
    if (ctx->fixed_acc) {
        // order-independent 64-bit fixed-point sums (bit-reproducible mass assignment)
        CKL("cic_scatter", 5 * rby<T>(ctx), launch_cic_scatter_fixed<T>(ctx->n, ctx->B, fields(ctx, RB_TH, 3), ctx->fixed_acc,
                                                                       ctx->stream));   // psi in, 64-bit zero + add
        CKL("fixed_to_mass", 3 * rby<T>(ctx), launch_fixed_to_mass<T>(ctx->n, ctx->B, ctx->fixed_acc, RB<T>(ctx, RB_DELTA),
                                                                      ctx->stream));
    } else {
        CKL("fill", rby<T>(ctx), launch_fill<T>(ctx->nvox * ctx->B, RB<T>(ctx, RB_DELTA), T(0), ctx->stream));
        CKL("cic_scatter", 4 * rby<T>(ctx), launch_cic_scatter<T>(ctx->n, ctx->B, fields(ctx, RB_TH, 3), RB<T>(ctx, RB_DELTA), ctx->stream));
    }
    // tidal tensor and density Hessian spectra (Sect. 2.8, App. B)
    RUN(z_fwd<T>(ctx, creal(ctx, RB_DELTA, 1), mspec<T>(ctx, SP_SCR, 1)));
    RUN(y_identity<T>(ctx, SP_SCR, 1, true));
    {
        PassProgram p = program(cspec<T>(ctx, SP_SCR, 1), mspec<T>(ctx, SP_SCR + 1, hier ? 6 : 3), ctx->nspec);
        add_merge(p, mk(0, 0, 0, 0, 0, R_ONE, invn3));
        add_expand(p, mk(0, 0, 2, 0, 0, R_INVK2, 1.0));
        add_expand(p, mk(0, 1, 1, 0, 0, R_INVK2, 1.0));
        add_expand(p, mk(0, 2, 0, 0, 0, R_INVK2, 1.0));
        if (hier) {
            add_expand(p, mk(0, 3, 2, 0, 0, R_ONE, -1.0));
            add_expand(p, mk(0, 4, 1, 0, 0, R_ONE, -1.0));
            add_expand(p, mk(0, 5, 0, 0, 0, R_ONE, -1.0));
        }
        CKL("x_node", (p.n_in + p.n_out) * sby<T>(ctx), launch_x_node<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    {
        const int nt = hier ? 2 : 1;
        PassProgram p = program(cspec<T>(ctx, SP_SCR + 1, 3 * nt), mspec<T>(ctx, SP_TH, 6 * nt), ctx->nspec);
        for (int h = 0; h < nt; ++h) {
            const int s = 3 * h, d = 6 * h;
            add_expand(p, mk(s + 0, d + 0, 0, 0, 0, R_ONE, 1.0));
            add_expand(p, mk(s + 1, d + 1, 0, 1, 0, R_ONE, 1.0));
            add_expand(p, mk(s + 1, d + 2, 0, 0, 1, R_ONE, 1.0));
            add_expand(p, mk(s + 2, d + 3, 0, 2, 0, R_ONE, 1.0));
            add_expand(p, mk(s + 2, d + 4, 0, 1, 1, R_ONE, 1.0));
            add_expand(p, mk(s + 2, d + 5, 0, 0, 2, R_ONE, 1.0));
        }
        CKL("y_inv", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_inv<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    // tensors to real space
    RUN(z_inv<T>(ctx, cspec<T>(ctx, SP_TH, nth), mreal(ctx, RB_TH, nth)));
    return BRIDGE_OK;
}
template <typename T> int run_forward_lik(bridge_ctx* ctx, const T* nu, bool likelihood) {
    const int nth = nth_of(ctx);
    // fused eigenvalue / web / bias pass, normalisation
    CKL("web_bias", (nth + 3) * rby<T>(ctx), launch_pass_a<T>(ctx->n, ctx->B, fields(ctx, RB_TH, 12), RB<T>(ctx, RB_DELTA), RB<T>(ctx, RB_LNF),
                        RB<T>(ctx, RB_LNF + 1), reinterpret_cast<const BiasT<T>*>(ctx->biast), ctx->wp, ctx->partial,
                        red_args(ctx), ctx->stream));   // sum f and ln C reduced by the last block
    if (likelihood) {
        CKL("nb_lik", 3 * rby<T>(ctx) + c16b(ctx), launch_pass_b<T>(ctx->n, ctx->B, RB<T>(ctx, RB_LNF), RB<T>(ctx, RB_LNF + 1), ctx->c16, nu, ctx->sc,
                            ctx->partial, red_args(ctx), ctx->stream));   // log posterior reduced by the last block
    }
    return BRIDGE_OK;
}
template <typename T> int run_forward(bridge_ctx* ctx, const T* nu, bool likelihood) {
    RUN(run_forward_fields<T>(ctx, nu));
    return run_forward_lik<T>(ctx, nu, likelihood);
}

// ---------------------------------------------------------------------------
// Adjoint: every forward step transposed, ending with g_nu = d log post/d nu.
// ---------------------------------------------------------------------------
template <typename T> int run_adjoint(bridge_ctx* ctx, const T* nu, T* grad, bool bias_grad) {
    const double invn3 = 1.0 / double(ctx->nvox);
    const bool hier = ctx->nr == 16;
    const int nth = nth_of(ctx);
    // web + bias + NB adjoint: g_rho (direct), g_T, g_H in real space, then r2c
    CKL("web_bias_adj", (2 * nth + 2) * rby<T>(ctx) + c16b(ctx), launch_web_adjoint<T>(ctx->n, ctx->B, fields(ctx, RB_TH, 12), RB<T>(ctx, RB_DELTA), ctx->c16,
                             reinterpret_cast<const BiasT<T>*>(ctx->biast), ctx->wp, ctx->sc,
                             fields(ctx, RB_SCR, 1 + nth), ctx->partial, bias_grad, ctx->stream, ctx->tune[3]));
    if (bias_grad)
        CKL("reduce", 0.0, launch_reduce(RED_BIASGRAD, pw_blocks(ctx->n), ctx->B, ctx->partial, ctx->sc, ctx->biasd, ctx->nr, ctx->stream));
    RUN(z_fwd<T>(ctx, creal(ctx, RB_SCR, 1 + nth), mspec<T>(ctx, SP_SCR, 1 + nth)));
    // spectral adjoint of the tensors (transpose of the forward x node / y expansion)
    {
        const int nslot = hier ? 6 : 4;
        PassProgram p = program(cspec<T>(ctx, SP_SCR, 1 + nth), mspec<T>(ctx, SP_SCR + 13, nslot), ctx->nspec);
        for (int h = 0; h < (hier ? 2 : 1); ++h) {
            const int s = 1 + 6 * h, d = 3 * h;
            add_merge(p, mk(s + 0, d + 0, 0, 0, 0, R_ONE, 1.0));
            add_merge(p, mk(s + 1, d + 1, 0, 1, 0, R_ONE, 1.0));
            add_merge(p, mk(s + 2, d + 1, 0, 0, 1, R_ONE, 1.0));
            add_merge(p, mk(s + 3, d + 2, 0, 2, 0, R_ONE, 1.0));
            add_merge(p, mk(s + 4, d + 2, 0, 1, 1, R_ONE, 1.0));
            add_merge(p, mk(s + 5, d + 2, 0, 0, 2, R_ONE, 1.0));
        }
        if (hier) add_merge(p, mk(0, 5, 0, 0, 0, R_ONE, -1.0));   // direct g_rho joins W0' (coef -1 undone below)
        else add_merge(p, mk(0, 3, 0, 0, 0, R_ONE, 1.0));         // own slot
        CKL("y_fwd", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_fwd<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    {
        const int nslot = hier ? 6 : 4;
        PassProgram p = program(cspec<T>(ctx, SP_SCR + 13, nslot), mspec<T>(ctx, SP_SCR, 1), ctx->nspec);
        add_merge(p, mk(0, 0, 2, 0, 0, R_INVK2, invn3));
        add_merge(p, mk(1, 0, 1, 0, 0, R_INVK2, invn3));
        add_merge(p, mk(2, 0, 0, 0, 0, R_INVK2, invn3));
        if (hier) {
            add_merge(p, mk(3, 0, 2, 0, 0, R_ONE, -invn3));
            add_merge(p, mk(4, 0, 1, 0, 0, R_ONE, -invn3));
            add_merge(p, mk(5, 0, 0, 0, 0, R_ONE, -invn3));
        } else {
            add_merge(p, mk(3, 0, 0, 0, 0, R_ONE, invn3));
        }
        add_expand(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));
        CKL("x_node", (p.n_in + p.n_out) * sby<T>(ctx), launch_x_node<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    RUN(y_identity<T>(ctx, SP_SCR, 1, false));
    RUN(z_inv<T>(ctx, cspec<T>(ctx, SP_SCR, 1), mreal(ctx, RB_GD, 1)));       // g_rho (total)
    // recompute_alpt: the ALPT and displacement spectra again from nu (every
    // scratch spectrum is free here; g_rho is a real field)
    if (ctx->recompute) RUN(run_alpt<T>(ctx, nu));
    // CIC adjoint with the displacement recomputed from its spectra, then r2c
    {
        NodeArgs na{};
        na.kind = ctx->radial ? NODE_GATHER_RSD : NODE_GATHER;
        for (int f = 0; f < 3; ++f) {
            na.spec_in[f] = ctx->spec[ctx->sp_psi + f];
            na.spec_out[f] = ctx->spec[f < 2 ? SP_SCR + f : SP_GPSIZ];
            if (ctx->radial) {
                na.spec_in[3 + f] = ctx->spec[ctx->sp_psi1 + f];
                na.spec_out[3 + f] = ctx->spec[ctx->sp_gpsi1 + f];
            }
        }
        na.real_in[0] = ctx->real[RB_GD];
        RUN(node<T>(ctx, na, "node_cic_gather", (ctx->radial ? 12 : 6) * sby<T>(ctx) + rby<T>(ctx), nullptr));
    }
    {
        PassProgram p = program({ctx->spec[SP_SCR], ctx->spec[SP_SCR + 1], ctx->spec[SP_GPSIZ]},
                                mspec<T>(ctx, SP_SCR + 3, 2), ctx->nspec);
        add_merge(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));
        add_merge(p, mk(1, 1, 0, 1, 0, R_ONE, 1.0));
        add_merge(p, mk(2, 1, 0, 0, 1, R_ONE, 1.0));
        CKL("y_fwd", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_fwd<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    {
        PassProgram p = program(cspec<T>(ctx, SP_SCR + 3, 2), mspec<T>(ctx, SP_SCR + 5, 2), ctx->nspec);
        const double c = invn3 / ctx->kp.dx;              // conj(-i/dx) = +i/dx
        add_merge(p, mk(0, 0, 1, 0, 0, R_INVK2, 0.0, c));
        add_merge(p, mk(1, 0, 0, 0, 0, R_INVK2, 0.0, c));
        add_expand(p, mk(0, 0, 0, 0, 0, R_KBLEND, 1.0));
        add_expand(p, mk(0, 1, 0, 0, 0, R_1MKBLEND, 1.0));
        CKL("x_node", (p.n_in + p.n_out) * sby<T>(ctx), launch_x_node<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    RUN(y_identity<T>(ctx, SP_SCR + 5, 2, false));
    // ALPT source adjoint on the fly (delta0, phi recomputed from their spectra)
    {
        NodeArgs na{};
        na.kind = NODE_ALPT_ADJ;
        for (int f = 0; f < 7; ++f) na.spec_in[f] = ctx->spec[ctx->sp_alpt + f];
        na.spec_in[7] = ctx->spec[SP_SCR + 5];
        na.spec_in[8] = ctx->spec[SP_SCR + 6];
        for (int f = 0; f < 7; ++f) na.spec_out[f] = ctx->spec[SP_SCR + f];
        RUN(node<T>(ctx, na, "node_alpt_adj", 16 * sby<T>(ctx), nullptr));
    }
    {
        const bool rsd = ctx->cfg.rsd_f != 0.0 && !ctx->radial;
        std::vector<const void*> in = cspec<T>(ctx, SP_SCR, 7);
        if (rsd) in.push_back(ctx->spec[SP_GPSIZ]);
        if (ctx->radial)
            for (int j = 0; j < 3; ++j) in.push_back(ctx->spec[ctx->sp_gpsi1 + j]);
        PassProgram p = program(in, mspec<T>(ctx, SP_SCR + 7, 4), ctx->nspec);
        // transpose of the redshift-space term: V0' += conj(i f D / dx) kz g_Psi_z
        if (rsd) add_merge(p, mk(7, 3, 0, 0, 1, R_ONE, 0.0, -ctx->cfg.rsd_f * ctx->cfg.growth_d / ctx->kp.dx));
        if (ctx->radial) {
            // transpose of Psi_1 = (i D / dx) (V1, ky V0, kz V0): V1' += conj(i D / dx) g_Psi1,x,
            // V0' += conj(i D / dx) (ky g_Psi1,y + kz g_Psi1,z)
            const double c1 = -ctx->cfg.growth_d / ctx->kp.dx;
            add_merge(p, mk(7, 2, 0, 0, 0, R_ONE, 0.0, c1));
            add_merge(p, mk(8, 3, 0, 1, 0, R_ONE, 0.0, c1));
            add_merge(p, mk(9, 3, 0, 0, 1, R_ONE, 0.0, c1));
        }
        add_merge(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));   // W0' <- g_delta0
        add_merge(p, mk(1, 1, 0, 0, 0, R_ONE, 1.0));   // V2' <- g_phi_xx
        add_merge(p, mk(2, 2, 0, 1, 0, R_ONE, 1.0));   // V1' <- ky g_phi_xy + kz g_phi_xz
        add_merge(p, mk(3, 2, 0, 0, 1, R_ONE, 1.0));
        add_merge(p, mk(4, 3, 0, 2, 0, R_ONE, 1.0));   // V0' <- ky^2 g_yy + ky kz g_yz + kz^2 g_zz
        add_merge(p, mk(5, 3, 0, 1, 1, R_ONE, 1.0));
        add_merge(p, mk(6, 3, 0, 0, 2, R_ONE, 1.0));
        CKL("y_fwd", (p.n_in + p.n_out) * sby<T>(ctx), launch_y_fwd<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    {
        PassProgram p = program(cspec<T>(ctx, SP_SCR + 7, 4), mspec<T>(ctx, SP_SCR, 1), ctx->nspec);
        add_merge(p, mk(0, 0, 0, 0, 0, R_ONE, invn3));
        add_merge(p, mk(1, 0, 2, 0, 0, R_INVK2, invn3));
        add_merge(p, mk(2, 0, 1, 0, 0, R_INVK2, invn3));
        add_merge(p, mk(3, 0, 0, 0, 0, R_INVK2, invn3));
        add_expand(p, mk(0, 0, 0, 0, 0, R_SQRTP, 1.0));
        CKL("x_node", (p.n_in + p.n_out) * sby<T>(ctx), launch_x_node<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    RUN(y_identity<T>(ctx, SP_SCR, 1, false));
    // inverse z with the white-noise prior in its stores: g_nu = (likelihood part) - nu
    {
        ZProgram p{};
        p.n_fields = 1;
        p.in[0] = ctx->spec[SP_SCR];
        p.out[0] = grad;
        p.sub[0] = nu;
        p.in_cs = ctx->nspec;
        p.out_cs = ctx->nvox;
        CKL("z_inv", 2 * rby<T>(ctx) + sby<T>(ctx), launch_z_inv<T>(ctx->n, ctx->B, p, ctx->stream));
    }
    return BRIDGE_OK;
}

// Upload the bias tables of all chains and validate them.
template <typename T> int upload_bias(bridge_ctx* ctx, const bridge_bias* bias) {
    std::string why;
    if (validate_bias(ctx, bias, &why) != BRIDGE_OK) return fail(ctx, BRIDGE_EINVAL, why);
    BiasT<T>* bt = reinterpret_cast<BiasT<T>*>(ctx->biast_host);
    for (int c = 0; c < ctx->B; ++c) {
        BiasD& d = ctx->biasd_host[c];
        std::memset(&d, 0, sizeof(d));
        BiasT<T>& t = bt[c];
        std::memset(&t, 0, sizeof(t));
        for (int r = 0; r < 16; ++r) {
            const bool on = r < ctx->nr;
            d.a[r] = on ? bias[c].a[r] : 1.0; d.alpha[r] = on ? bias[c].alpha[r] : 0.0;
            d.rho[r] = on ? bias[c].rho[r] : 1.0; d.eps[r] = on ? bias[c].eps[r] : 1.0;
            d.rhop[r] = on ? bias[c].rhop[r] : 0.0; d.epsp[r] = on ? bias[c].epsp[r] : 1.0;
            d.beta[r] = on ? bias[c].beta[r] : 1.0;
            t.pk[r][BP_A] = T(d.a[r]); t.pk[r][BP_ALPHA] = T(d.alpha[r]); t.pk[r][BP_RHO] = T(d.rho[r]);
            t.pk[r][BP_EPS] = T(d.eps[r]); t.pk[r][BP_RHOP] = T(d.rhop[r]); t.pk[r][BP_EPSP] = T(d.epsp[r]);
            t.pk[r][BP_BETA] = T(d.beta[r]); t.pk[r][BP_FLAGS] = T(0);
        }
        // flag in slot 7 of region 0: some region of this chain has a second cut-off (rho' > 0)
        for (int r = 0; r < ctx->nr; ++r)
            if (d.rhop[r] > 0.0) t.pk[0][BP_FLAGS] = T(1);
        d.prior_mask = bias[c].prior_mask;
        d.mu_alpha = bias[c].mu_alpha; d.sigma_alpha = bias[c].sigma_alpha;
        d.mu_beta = bias[c].mu_beta; d.sigma_beta = bias[c].sigma_beta;
    }
    CK(cudaMemcpyAsync(ctx->biasd, ctx->biasd_host, sizeof(BiasD) * ctx->B, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->biast, ctx->biast_host, sizeof(BiasT<T>) * ctx->B, cudaMemcpyHostToDevice, ctx->stream));
    return BRIDGE_OK;
}

template <typename T> int prep_counts(bridge_ctx* ctx, const int32_t* counts) {
    if (!counts) return fail(ctx, BRIDGE_EINVAL, "counts is NULL");
    CK(cudaMemsetAsync(ctx->errflag, 0, sizeof(int), ctx->stream));
    // N_tr is reduced by the kernel's last block (no separate reduction launch)
    CKL("counts_prep", 3 * c16b(ctx), launch_counts_prep<T>(ctx->n, ctx->B, counts, ctx->c16, ctx->partial, ctx->errflag,
                                                             red_args(ctx), ctx->stream));
    return BRIDGE_OK;
}

// Synchronise, fetch scalars and the count-range flag.
int finish(bridge_ctx* ctx) {
    cudaError_t e = cudaMemcpyAsync(ctx->sc_host, ctx->sc, sizeof(ChainScalars) * ctx->B, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->errflag_host, ctx->errflag, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, BRIDGE_ECUDA, std::string("synchronise: ") + cudaGetErrorString(e));
    if (*ctx->errflag_host) return fail(ctx, BRIDGE_EINVAL, "counts outside [0, 65535]");
    return BRIDGE_OK;
}

template <typename T> int do_forward(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                                     void* ln_nbar_out, double* logpost_out) {
    if (!nu) return fail(ctx, BRIDGE_EINVAL, "nu is NULL");
    RUN(upload_bias<T>(ctx, bias));
    RUN(prep_counts<T>(ctx, counts));
    RUN(run_forward<T>(ctx, reinterpret_cast<const T*>(nu), true));
    if (ln_nbar_out)
        CKL("lnnbar", 2 * rby<T>(ctx), launch_lnnbar<T>(ctx->nvox, ctx->B, RB<T>(ctx, RB_LNF), ctx->sc, reinterpret_cast<T*>(ln_nbar_out), ctx->stream));
    RUN(finish(ctx));
    for (int c = 0; c < ctx->B; ++c) {
        if (!std::isfinite(ctx->sc_host[c].logpost)) return fail(ctx, BRIDGE_ENONFINITE, "log posterior is not finite");
        if (logpost_out) logpost_out[c] = ctx->sc_host[c].logpost;
    }
    return BRIDGE_OK;
}

template <typename T> int eval_body(bridge_ctx* ctx, const T* nu, const int32_t* counts, T* grad, bool bias_grad) {
    RUN(prep_counts<T>(ctx, counts));
    RUN(run_forward<T>(ctx, nu, true));
    RUN(run_adjoint<T>(ctx, nu, grad, bias_grad));
    return BRIDGE_OK;
}

int ensure_graph_stream(bridge_ctx* ctx) {
    if (!ctx->gstream) {
        CK(cudaStreamCreateWithFlags(&ctx->gstream, cudaStreamNonBlocking));
        CK(cudaEventCreateWithFlags(&ctx->gev[0], cudaEventDisableTiming));
        CK(cudaEventCreateWithFlags(&ctx->gev[1], cudaEventDisableTiming));
    }
    return BRIDGE_OK;
}

// The whole evaluation (counts preparation, forward, adjoint) replayed from a
// CUDA graph captured on a private stream; re-captured when the buffers change.
// Capture body() (which launches on ctx->stream) into *exec on the private stream.
template <typename F> int capture_exec(bridge_ctx* ctx, cudaGraphExec_t* exec, int64_t* nlaunch, F body) {
    cudaStream_t user = ctx->stream;
    const int64_t launches = ctx->launches;
    ctx->stream = ctx->gstream;
    cudaGraph_t graph = nullptr;
    CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed));
    const int st = body();
    const cudaError_t ce = cudaStreamEndCapture(ctx->gstream, &graph);
    *nlaunch = ctx->launches - launches;
    ctx->stream = user;
    ctx->launches = launches;
    if (st != BRIDGE_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (ce != cudaSuccess) return fail(ctx, BRIDGE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
    const cudaError_t ie = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) { *exec = nullptr; return fail(ctx, BRIDGE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie)); }
    return BRIDGE_OK;
}

// Evaluation on the context's device staging buffers with the inputs in host memory
// (bridge_logpost_grad_host): nu is copied in on the caller's stream; the counts are
// copied and prepared on a second stream while the forward fields, which do not need
// them, run; the web/bias pass waits for both.  The gradient is copied out last.
template <typename T> int host_eval(bridge_ctx* ctx, const void* nu_host, T* grad_host, bool bias_grad) {
    RUN(ensure_graph_stream(ctx));
    if (!ctx->cstream) {
        CK(cudaStreamCreateWithFlags(&ctx->cstream, cudaStreamNonBlocking));
        for (auto& e : ctx->hev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    }
    const T* nu = reinterpret_cast<const T*>(ctx->h_nu);
    T* g = reinterpret_cast<T*>(ctx->h_grad);
    if (!ctx->hexec[0]) RUN(capture_exec(ctx, &ctx->hexec[0], &ctx->hlaunches[0], [&] { return run_forward_fields<T>(ctx, nu); }));
    if (!ctx->hexec[1] || ctx->hkey != int(bias_grad)) {
        if (ctx->hexec[1]) { cudaGraphExecDestroy(ctx->hexec[1]); ctx->hexec[1] = nullptr; }
        RUN(capture_exec(ctx, &ctx->hexec[1], &ctx->hlaunches[1], [&] {
            RUN(run_forward_lik<T>(ctx, nu, true));
            return run_adjoint<T>(ctx, nu, g, bias_grad);
        }));
        ctx->hkey = int(bias_grad);
    }
    const size_t fb = size_t(ctx->nvox) * ctx->B * sizeof(T), cb = size_t(ctx->nvox) * ctx->B * sizeof(int32_t);
    // nu first (the forward fields need it): both copies share the host link, so the counts
    // follow it, on the second stream, and overlap the forward fields instead
    CK(cudaMemcpyAsync(ctx->h_nu, nu_host, fb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaEventRecord(ctx->hev[0], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->cstream, ctx->hev[0], 0));
    CK(cudaMemcpyAsync(ctx->h_counts, ctx->hcounts, cb, cudaMemcpyHostToDevice, ctx->cstream));
    {
        cudaStream_t user = ctx->stream;
        ctx->stream = ctx->cstream;
        const int st = prep_counts<T>(ctx, ctx->h_counts);
        ctx->stream = user;
        RUN(st);
    }
    CK(cudaEventRecord(ctx->hev[1], ctx->cstream));
    // the two halves of the evaluation, joined before the web/bias pass
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->hev[0], 0));
    CK(cudaGraphLaunch(ctx->hexec[0], ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->hev[1], 0));
    CK(cudaGraphLaunch(ctx->hexec[1], ctx->gstream));
    CK(cudaEventRecord(ctx->gev[1], ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0));
    CK(cudaMemcpyAsync(grad_host, g, fb, cudaMemcpyDeviceToHost, ctx->stream));
    ctx->launches += ctx->hlaunches[0] + ctx->hlaunches[1];
    return BRIDGE_OK;
}

template <typename T> int eval_graph(bridge_ctx* ctx, const T* nu, const int32_t* counts, T* grad, bool bias_grad) {
    RUN(ensure_graph_stream(ctx));
    const void* key[4] = {nu, counts, grad, bias_grad ? ctx : nullptr};
    bool fresh = ctx->eexec != nullptr;
    for (int i = 0; i < 4; ++i) fresh = fresh && ctx->ekey[i] == key[i];
    if (!fresh) {
        if (ctx->eexec) { cudaGraphExecDestroy(ctx->eexec); ctx->eexec = nullptr; }
        cudaStream_t user = ctx->stream;
        const int64_t launches = ctx->launches;
        ctx->stream = ctx->gstream;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed));
        const int st = eval_body<T>(ctx, nu, counts, grad, bias_grad);
        const cudaError_t ce = cudaStreamEndCapture(ctx->gstream, &graph);
        ctx->elaunches = ctx->launches - launches;
        ctx->stream = user;
        ctx->launches = launches;
        if (st != BRIDGE_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (ce != cudaSuccess) return fail(ctx, BRIDGE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&ctx->eexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) { ctx->eexec = nullptr; return fail(ctx, BRIDGE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie)); }
        for (int i = 0; i < 4; ++i) ctx->ekey[i] = key[i];
    }
    CK(cudaEventRecord(ctx->gev[0], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
    CK(cudaGraphLaunch(ctx->eexec, ctx->gstream));
    CK(cudaEventRecord(ctx->gev[1], ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0));
    ctx->launches += ctx->elaunches;
    return BRIDGE_OK;
}

// Gradient with respect to the free bias parameters of chain c (G12 reading):
// parameter p of alpha_0..alpha_{P-1}, beta_0..beta_{P-1} in bit order of
// free_mask; with tie_classes, alpha_j / beta_j move the four table entries
// 4j..4j+3 of Phi class j together, so their derivative is the sum over the four.
int pack_bias_grad(const bridge_ctx* ctx, const bridge_bias& b, const double* full, double* out) {
    const int np = b.tie_classes ? 4 : ctx->nr;
    int k = 0;
    for (int q = 0; q < 2 * np; ++q) {
        if (!((b.free_mask >> q) & 1u)) continue;
        const int kind = q / np, j = q % np;   // kind 0: alpha, 1: beta
        double v = 0.0;
        if (b.tie_classes)
            for (int i = 0; i < 4; ++i) v += full[kind * ctx->nr + 4 * j + i];
        else
            v = full[kind * ctx->nr + j];
        out[k++] = v;
    }
    return k;
}

template <typename T> int do_grad(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                                  double* logpost_out, void* grad, double* gbias_out, const double* cot = nullptr) {
    if (!nu || !grad) return fail(ctx, BRIDGE_EINVAL, "nu and grad_nu_out are required");
    if (!counts) return fail(ctx, BRIDGE_EINVAL, "counts is NULL");
    RUN(upload_bias<T>(ctx, bias));
    const T* nuT = reinterpret_cast<const T*>(nu);
    T* gT = reinterpret_cast<T*>(grad);
    const bool want_bias = gbias_out != nullptr && bias[0].free_mask != 0u;
    if (ctx->hcounts) RUN(host_eval<T>(ctx, nu, gT, want_bias));        // nu, counts and grad in host memory
    else if (ctx->prof) RUN(eval_body<T>(ctx, nuT, counts, gT, want_bias));   // per-launch events need direct launches
    else RUN(eval_graph<T>(ctx, nuT, counts, gT, want_bias));
    bool scale = false;
    if (cot) {
        for (int c = 0; c < ctx->B; ++c) {
            if (!std::isfinite(cot[c])) return fail(ctx, BRIDGE_EINVAL, "cotangent is not finite");
            ctx->cot_host[c] = cot[c];
            scale = scale || cot[c] != 1.0;
        }
    }
    if (scale) {
        CK(cudaMemcpyAsync(ctx->cot, ctx->cot_host, sizeof(double) * ctx->B, cudaMemcpyHostToDevice, ctx->stream));
        CKL("scale", 2 * rby<T>(ctx), launch_scale_chains<T>(ctx->n, ctx->B, gT, ctx->cot, ctx->stream));
    }
    RUN(finish(ctx));
    for (int c = 0; c < ctx->B; ++c) {
        if (!std::isfinite(ctx->sc_host[c].logpost)) return fail(ctx, BRIDGE_ENONFINITE, "log posterior is not finite");
        if (logpost_out) logpost_out[c] = ctx->sc_host[c].logpost;
    }
    if (want_bias) {
        const int nf = __builtin_popcount(bias[0].free_mask);
        for (int c = 0; c < ctx->B; ++c) {
            double* o = gbias_out + size_t(c) * nf;
            pack_bias_grad(ctx, bias[c], ctx->sc_host[c].gbias, o);
            if (cot)
                for (int k = 0; k < nf; ++k) o[k] *= cot[c];
        }
    }
    return BRIDGE_OK;
}

// Splitting integrators (Sect. 2.2).  One step of a scheme is K(k_0) D(d_0)
// K(k_1) ... D(d_{s-1}) K(k_s), in units of eps, with K(c): p += c eps grad log
// post and D(d): nu += d eps p.  The trajectory runs as units "gradient at nu,
// then kick and drift" (launch_kick_drift); the last kick of a step and the
// first of the next are merged into one unit.
struct Scheme {
    int s = 1;                        // drifts per step (gradient evaluations per step)
    double kick[5] = {0.5, 0.5};      // s + 1 kick coefficients
    double drift[4] = {1.0};          // s drift coefficients
};
bool make_scheme(int id, Scheme* sc) {
    Scheme r;
    if (id == BRIDGE_LEAPFROG) {
        r.s = 1; r.kick[0] = r.kick[1] = 0.5; r.drift[0] = 1.0;
    } else if (id == BRIDGE_TWO_STAGE) {
        // Blanes, Casas and Sanz-Serna (2014), b = 0.211781
        const double b = 0.211781;
        r.s = 2; r.kick[0] = b; r.kick[1] = 1.0 - 2.0 * b; r.kick[2] = b; r.drift[0] = r.drift[1] = 0.5;
    } else if (id == BRIDGE_FOURTH_ORDER) {
        // Yoshida (1990) triple jump of leapfrog sub-steps w1, w0, w1: 2 w1 + w0 = 1, 2 w1^3 + w0^3 = 0
        const double w1 = 1.0 / (2.0 - std::cbrt(2.0)), w0 = 1.0 - 2.0 * w1;
        r.s = 3; r.kick[0] = 0.5 * w1; r.kick[1] = 0.5 * (w1 + w0); r.kick[2] = 0.5 * (w0 + w1); r.kick[3] = 0.5 * w1;
        r.drift[0] = w1; r.drift[1] = w0; r.drift[2] = w1;
    } else {
        return false;
    }
    *sc = r;
    return true;
}

// Kick and drift of one unit: the fields, and with joint integration the log
// bias parameters (from the bias gradient of the same evaluation).
template <typename T> int kick_drift_unit(bridge_ctx* ctx, T* nu, T* p, const T* g, double ck, double cd, bool joint) {
    CKL("leapfrog", 5 * rby<T>(ctx), launch_kick_drift<T>(ctx->n, ctx->B, p, nu, g, ck, cd, ctx->partial, ctx->stream));
    if (joint)
        CKL("bias_leapfrog", 0.0, launch_bias_kick_drift<T>(ctx->B, ctx->nr, ctx->jmask, ctx->theta, ctx->ptheta, ctx->sc,
                                                            ctx->biasd, reinterpret_cast<BiasT<T>*>(ctx->biast), ck, cd,
                                                            ctx->stream));
    return BRIDGE_OK;
}

// Units of one interior step: gradient at nu, then p += ck g; nu += cd p.
template <typename T> int interior_step(bridge_ctx* ctx, T* nu, T* p, T* g, const std::vector<double>& ck,
                                        const std::vector<double>& cd, bool joint) {
    for (size_t j = 0; j < ck.size(); ++j) {
        RUN(run_forward<T>(ctx, nu, true));
        RUN(run_adjoint<T>(ctx, nu, g, joint));
        RUN(kick_drift_unit<T>(ctx, nu, p, g, ck[j], cd[j], joint));
    }
    return BRIDGE_OK;
}

// Replays n interior steps from a CUDA graph captured (once per nu, p and
// coefficients) on a private stream; the context stream waits for the replays.
template <typename T> int interior_graph(bridge_ctx* ctx, T* nu, T* p, T* g, const std::vector<double>& ck,
                                         const std::vector<double>& cd, int n, bool joint) {
    RUN(ensure_graph_stream(ctx));
    bool fresh = ctx->gexec && ctx->gkey[0] == nu && ctx->gkey[1] == p && ctx->gkey[2] == g &&
                 ctx->gck == ck && ctx->gcd == cd && ctx->gjoint == (joint ? ctx->jmask : 0u);
    if (!fresh) {
        if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
        cudaStream_t user = ctx->stream;
        const bool prof = ctx->prof;
        const int64_t launches = ctx->launches;
        ctx->stream = ctx->gstream;
        ctx->prof = false;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(ctx->gstream, cudaStreamCaptureModeRelaxed));
        const int st = interior_step<T>(ctx, nu, p, g, ck, cd, joint);
        const cudaError_t ce = cudaStreamEndCapture(ctx->gstream, &graph);
        ctx->glaunches = ctx->launches - launches;
        ctx->stream = user;
        ctx->prof = prof;
        ctx->launches = launches;
        if (st != BRIDGE_OK) { if (graph) cudaGraphDestroy(graph); return st; }
        if (ce != cudaSuccess) return fail(ctx, BRIDGE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
        const cudaError_t ie = cudaGraphInstantiate(&ctx->gexec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) { ctx->gexec = nullptr; return fail(ctx, BRIDGE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie)); }
        ctx->gkey[0] = nu; ctx->gkey[1] = p; ctx->gkey[2] = g;
        ctx->gck = ck; ctx->gcd = cd; ctx->gjoint = joint ? ctx->jmask : 0u;
    }
    CK(cudaEventRecord(ctx->gev[0], ctx->stream));
    CK(cudaStreamWaitEvent(ctx->gstream, ctx->gev[0], 0));
    for (int s = 0; s < n; ++s) CK(cudaGraphLaunch(ctx->gexec, ctx->gstream));
    CK(cudaEventRecord(ctx->gev[1], ctx->gstream));
    CK(cudaStreamWaitEvent(ctx->stream, ctx->gev[1], 0));
    return BRIDGE_OK;
}

// theta, ptheta: host [B][popcount(free_mask)] (joint integration) or NULL.
template <typename T> int do_integrate(bridge_ctx* ctx, void* nu_v, void* p_v, const int32_t* counts,
                                       const bridge_bias* bias, int scheme, int n_steps, double eps, double* h0,
                                       double* h1, double* theta = nullptr, double* ptheta = nullptr) {
    if (!nu_v || !p_v) return fail(ctx, BRIDGE_EINVAL, "nu and p are required");
    if (n_steps < 1 || !std::isfinite(eps)) return fail(ctx, BRIDGE_EINVAL, "n_steps >= 1 and finite eps required");
    Scheme sc;
    if (!make_scheme(scheme, &sc)) return fail(ctx, BRIDGE_EINVAL, "unknown integrator scheme");
    const bool joint = theta != nullptr;
    T* nu = reinterpret_cast<T*>(nu_v);
    T* p = reinterpret_cast<T*>(p_v);
    T* g = reinterpret_cast<T*>(ctx->grad_tmp);
    int nf = 0;
    std::vector<double> th0, pt0;   // start values of the bias state (host), for restores
    if (joint) {
        if (!bias || !ptheta) return fail(ctx, BRIDGE_EINVAL, "bias, theta and p_theta are required");
        const uint32_t m = bias[0].free_mask;
        nf = __builtin_popcount(m);
        if (m == 0u || bias[0].tie_classes != 0)
            return fail(ctx, BRIDGE_EINVAL, "joint integration needs untied free parameters (tie_classes = 0, free_mask != 0)");
        th0.assign(theta, theta + size_t(ctx->B) * nf);
        pt0.assign(ptheta, ptheta + size_t(ctx->B) * nf);
        for (double v : th0) if (!std::isfinite(v)) return fail(ctx, BRIDGE_EINVAL, "theta is not finite");
        for (double v : pt0) if (!std::isfinite(v)) return fail(ctx, BRIDGE_EINVAL, "p_theta is not finite");
        // the free entries of the tables are e^theta
        std::vector<bridge_bias> bb(bias, bias + ctx->B);
        for (int c = 0; c < ctx->B; ++c) {
            int k = 0;
            for (int q = 0; q < 2 * ctx->nr; ++q) {
                if (!((m >> q) & 1u)) continue;
                const double b = std::exp(th0[size_t(c) * nf + k++]);
                if (q < ctx->nr) bb[c].alpha[q] = b; else bb[c].beta[q - ctx->nr] = b;
            }
        }
        RUN(upload_bias<T>(ctx, bb.data()));
        ctx->jmask = m;
        std::vector<double> pad(size_t(ctx->B) * 32 * 2, 0.0);
        for (int c = 0; c < ctx->B; ++c)
            for (int k = 0; k < nf; ++k) {
                pad[size_t(c) * 32 + k] = th0[size_t(c) * nf + k];
                pad[size_t(ctx->B + c) * 32 + k] = pt0[size_t(c) * nf + k];
            }
        CK(cudaMemcpy(ctx->theta, pad.data(), pad.size() * sizeof(double), cudaMemcpyHostToDevice));
    } else {
        RUN(upload_bias<T>(ctx, bias));
    }
    RUN(prep_counts<T>(ctx, counts));
    // start state, put back for every chain whose Hamiltonian is not finite
    const size_t fb = size_t(ctx->nvox) * ctx->B * sizeof(T);
    CK(cudaMemcpyAsync(ctx->snap_nu, nu, fb, cudaMemcpyDeviceToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->snap_p, p, fb, cudaMemcpyDeviceToDevice, ctx->stream));
    // H = -log post - sum theta + 1/2 |p|^2 + 1/2 |p_theta|^2 (the theta terms for joint integration)
    auto bias_energy = [&](const double* th, const double* pt, int c) {
        double e = 0.0;
        for (int k = 0; k < nf; ++k) e += -th[size_t(c) * nf + k] + 0.5 * pt[size_t(c) * nf + k] * pt[size_t(c) * nf + k];
        return e;
    };
    std::vector<double> u0(ctx->B), k0(ctx->B);
    // initial potential and kinetic energy
    RUN(run_forward<T>(ctx, nu, true));
    RUN(run_adjoint<T>(ctx, nu, g, joint));
    CKL("leapfrog", 5 * rby<T>(ctx), launch_kick_drift<T>(ctx->n, ctx->B, p, nu, g, 0.0, 0.0, ctx->partial, ctx->stream));
    CKL("reduce", 0.0, launch_reduce(RED_P2, pw_blocks(ctx->n), ctx->B, ctx->partial, ctx->sc, ctx->biasd, ctx->nr, ctx->stream));
    RUN(finish(ctx));
    for (int c = 0; c < ctx->B; ++c) {
        u0[c] = -ctx->sc_host[c].logpost;
        k0[c] = 0.5 * ctx->sc_host[c].sump2 + (joint ? bias_energy(th0.data(), pt0.data(), c) : 0.0);
    }
    // first step: its first unit uses the gradient just computed
    RUN(kick_drift_unit<T>(ctx, nu, p, g, sc.kick[0] * eps, sc.drift[0] * eps, joint));
    {
        std::vector<double> ck, cd;
        for (int j = 1; j < sc.s; ++j) { ck.push_back(sc.kick[j] * eps); cd.push_back(sc.drift[j] * eps); }
        RUN(interior_step<T>(ctx, nu, p, g, ck, cd, joint));
    }
    // interior steps: the merged kick k_s + k_0 opens each
    if (n_steps > 1) {
        std::vector<double> ck, cd;
        ck.push_back((sc.kick[sc.s] + sc.kick[0]) * eps);
        cd.push_back(sc.drift[0] * eps);
        for (int j = 1; j < sc.s; ++j) { ck.push_back(sc.kick[j] * eps); cd.push_back(sc.drift[j] * eps); }
        if (n_steps > 2 && !ctx->prof) {
            RUN(interior_graph<T>(ctx, nu, p, g, ck, cd, n_steps - 1, joint));
            ctx->launches += ctx->glaunches * (n_steps - 1);   // kernels replayed from the graph
        } else {
            for (int s = 0; s < n_steps - 1; ++s) RUN(interior_step<T>(ctx, nu, p, g, ck, cd, joint));
        }
    }
    // last gradient and closing kick
    RUN(run_forward<T>(ctx, nu, true));
    RUN(run_adjoint<T>(ctx, nu, g, joint));
    RUN(kick_drift_unit<T>(ctx, nu, p, g, sc.kick[sc.s] * eps, 0.0, joint));
    CKL("reduce", 0.0, launch_reduce(RED_P2, pw_blocks(ctx->n), ctx->B, ctx->partial, ctx->sc, ctx->biasd, ctx->nr, ctx->stream));
    RUN(finish(ctx));
    std::vector<double> th1, pt1;
    if (joint) {
        std::vector<double> pad(size_t(ctx->B) * 32 * 2);
        CK(cudaMemcpy(pad.data(), ctx->theta, pad.size() * sizeof(double), cudaMemcpyDeviceToHost));
        th1.resize(size_t(ctx->B) * nf);
        pt1.resize(size_t(ctx->B) * nf);
        for (int c = 0; c < ctx->B; ++c)
            for (int k = 0; k < nf; ++k) {
                th1[size_t(c) * nf + k] = pad[size_t(c) * 32 + k];
                pt1[size_t(c) * nf + k] = pad[size_t(ctx->B + c) * 32 + k];
            }
    }
    int bad = 0;
    const size_t one = size_t(ctx->nvox) * sizeof(T);
    for (int c = 0; c < ctx->B; ++c) {
        const double H0 = u0[c] + k0[c];
        const double H1 = -ctx->sc_host[c].logpost + 0.5 * ctx->sc_host[c].sump2 +
                          (joint ? bias_energy(th1.data(), pt1.data(), c) : 0.0);
        if (h0) h0[c] = H0;
        if (h1) h1[c] = H1;
        const bool ok = std::isfinite(H0) && std::isfinite(H1);
        if (joint)
            for (int k = 0; k < nf; ++k) {
                theta[size_t(c) * nf + k] = ok ? th1[size_t(c) * nf + k] : th0[size_t(c) * nf + k];
                ptheta[size_t(c) * nf + k] = ok ? pt1[size_t(c) * nf + k] : pt0[size_t(c) * nf + k];
            }
        if (!ok) {
            ++bad;
            CK(cudaMemcpyAsync(reinterpret_cast<char*>(nu_v) + c * one, reinterpret_cast<const char*>(ctx->snap_nu) + c * one,
                               one, cudaMemcpyDeviceToDevice, ctx->stream));
            CK(cudaMemcpyAsync(reinterpret_cast<char*>(p_v) + c * one, reinterpret_cast<const char*>(ctx->snap_p) + c * one,
                               one, cudaMemcpyDeviceToDevice, ctx->stream));
        }
    }
    if (bad) {
        CK(cudaStreamSynchronize(ctx->stream));
        return fail(ctx, BRIDGE_ENONFINITE, "Hamiltonian is not finite for " + std::to_string(bad) + " of " +
                                                std::to_string(ctx->B) + " chains (their start state is restored)");
    }
    return BRIDGE_OK;
}

// n leapfrog steps from (nu, p) with the gradient g at nu given; g returns the
// gradient at the new nu.  One gradient evaluation per step; eps may be negative.
template <typename T> int do_steps(bridge_ctx* ctx, void* nu_v, void* p_v, void* g_v, const int32_t* counts,
                                   const bridge_bias* bias, int n, double eps, double* logpost_out) {
    if (!nu_v || !p_v || !g_v) return fail(ctx, BRIDGE_EINVAL, "nu, p and grad are required");
    if (n < 1 || !std::isfinite(eps)) return fail(ctx, BRIDGE_EINVAL, "n_steps >= 1 and finite eps required");
    T* nu = reinterpret_cast<T*>(nu_v);
    T* p = reinterpret_cast<T*>(p_v);
    T* g = reinterpret_cast<T*>(g_v);
    RUN(upload_bias<T>(ctx, bias));
    RUN(prep_counts<T>(ctx, counts));
    CKL("leapfrog", 5 * rby<T>(ctx), launch_kick_drift<T>(ctx->n, ctx->B, p, nu, g, 0.5 * eps, eps, ctx->partial, ctx->stream));
    for (int s = 1; s < n; ++s) {
        RUN(run_forward<T>(ctx, nu, true));
        RUN(run_adjoint<T>(ctx, nu, g, false));
        CKL("leapfrog", 5 * rby<T>(ctx), launch_kick_drift<T>(ctx->n, ctx->B, p, nu, g, eps, eps, ctx->partial, ctx->stream));
    }
    RUN(run_forward<T>(ctx, nu, true));
    RUN(run_adjoint<T>(ctx, nu, g, false));
    CKL("leapfrog", 5 * rby<T>(ctx), launch_kick_drift<T>(ctx->n, ctx->B, p, nu, g, 0.5 * eps, 0.0, ctx->partial, ctx->stream));
    RUN(finish(ctx));
    for (int c = 0; c < ctx->B; ++c)
        if (logpost_out) logpost_out[c] = ctx->sc_host[c].logpost;
    return BRIDGE_OK;
}

template <typename T> int do_dot(bridge_ctx* ctx, const void* a, const void* b, double* out) {
    if (!a || !b || !out) return fail(ctx, BRIDGE_EINVAL, "a, b and out are required");
    CKL("dot", 2 * rby<T>(ctx), launch_dot<T>(ctx->n, ctx->B, reinterpret_cast<const T*>(a), reinterpret_cast<const T*>(b),
                                               ctx->partial, red_args(ctx), ctx->stream));
    cudaError_t e = cudaMemcpyAsync(ctx->sc_host, ctx->sc, sizeof(ChainScalars) * ctx->B, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return fail(ctx, BRIDGE_ECUDA, std::string("dot: ") + cudaGetErrorString(e));
    for (int c = 0; c < ctx->B; ++c) out[c] = ctx->sc_host[c].dot;
    return BRIDGE_OK;
}

template <typename T> int do_debug(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                                   int which, void* out) {
    if (!nu || !out) return fail(ctx, BRIDGE_EINVAL, "nu and out are required");
    RUN(upload_bias<T>(ctx, bias));
    RUN(prep_counts<T>(ctx, counts));
    RUN(run_forward<T>(ctx, reinterpret_cast<const T*>(nu), true));
    const size_t fb = size_t(ctx->nvox) * ctx->B * sizeof(T), one = size_t(ctx->nvox) * sizeof(T);
    auto copy_fields = [&](int first, int count) -> int {
        // out layout [B][count][N^3]; workspace layout [field][B][N^3]
        for (int c = 0; c < ctx->B; ++c)
            for (int f = 0; f < count; ++f)
                CK(cudaMemcpyAsync(reinterpret_cast<char*>(out) + (size_t(c) * count + f) * one,
                                   reinterpret_cast<const char*>(ctx->real[first + f]) + size_t(c) * one, one,
                                   cudaMemcpyDeviceToDevice, ctx->stream));
        return BRIDGE_OK;
    };
    (void)fb;
    switch (which) {
        case BRIDGE_FIELD_DELTA0:
            if (ctx->recompute) RUN(run_alpt<T>(ctx, reinterpret_cast<const T*>(nu)));   // slots reused after the ALPT stage
            RUN(z_inv<T>(ctx, cspec<T>(ctx, ctx->sp_alpt, 1), mreal(ctx, RB_SCR, 1)));
            RUN(copy_fields(RB_SCR, 1));
            break;
        case BRIDGE_FIELD_PSI:
            if (ctx->recompute) RUN(run_alpt<T>(ctx, reinterpret_cast<const T*>(nu)));
            RUN(psi_real<T>(ctx, RB_SCR));
            RUN(copy_fields(RB_SCR, 3));
            break;
        case BRIDGE_FIELD_DELTA:
            CKL("shift", 2 * rby<T>(ctx), launch_shift<T>(ctx->nvox * ctx->B, RB<T>(ctx, RB_DELTA), RB<T>(ctx, RB_SCR), T(-1), ctx->stream));
            RUN(copy_fields(RB_SCR, 1));
            break;
        case BRIDGE_FIELD_TIDAL: RUN(copy_fields(RB_TH, 6)); break;
        case BRIDGE_FIELD_HESSIAN:
            if (ctx->nr != 16) return fail(ctx, BRIDGE_EINVAL, "the density Hessian exists only for 16 regions");
            RUN(copy_fields(RB_TH + 6, 6));
            break;
        case BRIDGE_FIELD_LAMBDA:
            CKL("eigs", 9 * rby<T>(ctx), launch_eigs<T>(ctx->n, ctx->B, fields(ctx, RB_TH, 6), fields(ctx, RB_SCR, 3), ctx->stream));
            RUN(copy_fields(RB_SCR, 3));
            break;
        case BRIDGE_FIELD_LNNBAR:
            CKL("lnnbar", 2 * rby<T>(ctx), launch_lnnbar<T>(ctx->nvox, ctx->B, RB<T>(ctx, RB_LNF), ctx->sc, RB<T>(ctx, RB_SCR), ctx->stream));
            RUN(copy_fields(RB_SCR, 1));
            break;
        default: return fail(ctx, BRIDGE_EINVAL, "unknown field selector");
    }
    return finish(ctx);
}

// Chain initialisation (Sect. 2.2): the tracer contrast delta*_tr = n* N^3 / N_tr - 1
// Wiener-filtered to the linear field and mapped to white noise, per mode k != 0
//   nu0_hat = D s dx^3 / (D^2 s^2 dx^3 + P_N) DFT(delta*_tr),  s = sqrt(P / dx^3),
// P_N = L^3 / N_tr (Poisson shot noise); the factor is written per chain into the
// fifth radial table and applied by the x node.
template <typename T> int do_wiener_init(bridge_ctx* ctx, const int32_t* counts, void* nu_out) {
    if (!counts || !nu_out) return fail(ctx, BRIDGE_EINVAL, "counts and nu_out are required");
    RUN(prep_counts<T>(ctx, counts));
    CKL("delta_tr", rby<T>(ctx) + c16b(ctx), launch_delta_tr<T>(ctx->n, ctx->B, ctx->c16, ctx->sc, RB<T>(ctx, RB_SCR), ctx->stream));
    RUN(z_fwd<T>(ctx, creal(ctx, RB_SCR, 1), mspec<T>(ctx, SP_SCR, 1)));
    RUN(y_identity<T>(ctx, SP_SCR, 1, true));
    RUN(finish(ctx));   // N_tr of every chain on the host
    const int rlen = ctx->kp.rlen;
    std::vector<double> tab(size_t(4) * rlen);
    radial_tables_host(ctx->n, ctx->kp, tab.data());
    const double* sq = tab.data() + (R_SQRTP - 1) * rlen;
    const double D = ctx->cfg.growth_d, dx3 = ctx->kp.dx * ctx->kp.dx * ctx->kp.dx;
    std::vector<T> w(rlen);
    T* wdev = reinterpret_cast<T*>(ctx->rtab) + size_t(R_WIENER - 1) * rlen;
    for (int c = 0; c < ctx->B; ++c) {
        const double ntr = ctx->sc_host[c].ntr;
        if (!(ntr > 0)) return fail(ctx, BRIDGE_EINVAL, "chain " + std::to_string(c) + " has no tracers");
        const double pn = ctx->cfg.box * ctx->cfg.box * ctx->cfg.box / ntr;
        for (int m2 = 0; m2 < rlen; ++m2) {
            const double sv = sq[m2];
            w[m2] = T(D * sv * dx3 / (D * D * sv * sv * dx3 + pn));
        }
        CK(cudaMemcpyAsync(wdev, w.data(), sizeof(T) * rlen, cudaMemcpyHostToDevice, ctx->stream));
        PassProgram p = program({reinterpret_cast<char*>(ctx->spec[SP_SCR]) + size_t(c) * ctx->nspec * 2 * sizeof(T)},
                                {reinterpret_cast<char*>(ctx->spec[SP_SCR + 1]) + size_t(c) * ctx->nspec * 2 * sizeof(T)},
                                ctx->nspec);
        add_merge(p, mk(0, 0, 0, 0, 0, R_WIENER, 1.0 / double(ctx->nvox)));
        add_expand(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));
        CKL("x_node", 2 * sby<T>(ctx) / ctx->B, launch_x_node<T>(ctx->n, 1, p, ctx->kp, ctx->stream));
        CK(cudaStreamSynchronize(ctx->stream));   // the host table is refilled for the next chain
    }
    RUN(y_identity<T>(ctx, SP_SCR + 1, 1, false));
    RUN(z_inv<T>(ctx, {ctx->spec[SP_SCR + 1]}, {nu_out}));
    CK(cudaStreamSynchronize(ctx->stream));
    return BRIDGE_OK;
}

// out = IDFT(DFT(in)) through the five pass kernels with the identity operator:
// z forward, y forward, x node (forward x DFT, 1/N^3, inverse x DFT), y
// inverse, z inverse -- the transforms of every other program without an
// operator, for testing them and timing them against a library FFT.
template <typename T> int do_fft_roundtrip(bridge_ctx* ctx, const void* in, void* out) {
    if (!in || !out) return fail(ctx, BRIDGE_EINVAL, "in and out are required");
    RUN(z_fwd<T>(ctx, {in}, {ctx->spec[SP_SCR]}));
    RUN(y_identity<T>(ctx, SP_SCR, 1, true));
    {
        PassProgram p = program(cspec<T>(ctx, SP_SCR, 1), mspec<T>(ctx, SP_SCR + 1, 1), ctx->nspec);
        add_merge(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0 / double(ctx->nvox)));
        add_expand(p, mk(0, 0, 0, 0, 0, R_ONE, 1.0));
        CKL("x_node", (p.n_in + p.n_out) * sby<T>(ctx), launch_x_node<T>(ctx->n, ctx->B, p, ctx->kp, ctx->stream));
    }
    RUN(y_identity<T>(ctx, SP_SCR + 1, 1, false));
    RUN(z_inv<T>(ctx, {ctx->spec[SP_SCR + 1]}, {out}));
    CK(cudaStreamSynchronize(ctx->stream));
    return BRIDGE_OK;
}

// Simpson in ln k of k^3 P(k) W(kR)^2 / (2 pi^2).
double tophat(double x) {
    if (std::fabs(x) < 1e-3) return 1.0 - x * x / 10.0 + x * x * x * x / 280.0;
    return 3.0 * (std::sin(x) - x * std::cos(x)) / (x * x * x);
}
double sigma2_unit(double R, double ns, double kc, double pw) {
    const int M = 1 << 16;
    const double a = std::log(1e-8), b = std::log(1e3 / R), h = (b - a) / M;
    double s = 0.0;
    for (int i = 0; i <= M; ++i) {
        const double k = std::exp(a + i * h);
        const double pk = std::pow(k, ns) / std::pow(1.0 + (k / kc) * (k / kc), pw);
        const double w = tophat(k * R);
        const double f = k * k * k * pk * w * w;
        s += f * ((i == 0 || i == M) ? 1.0 : (i % 2 ? 4.0 : 2.0));
    }
    return s * h / 3.0 / (2.0 * kPi * kPi);
}

// Sum of the CUDA-event times of one kernel class in the current profile.
int prof_class_ms(bridge_ctx* ctx, const char* name, double* ms_out) {
    CK(cudaStreamSynchronize(ctx->stream));
    double tot = 0.0;
    for (const auto& r : ctx->prof_recs) {
        if (std::strcmp(r.name, name) != 0) continue;
        float ms = 0.f;
        CK(cudaEventElapsedTime(&ms, r.a, r.b));
        tot += ms;
    }
    *ms_out = tot;
    return BRIDGE_OK;
}

// Captured graphs hold the launch shapes of their capture: drop them when those change.
void drop_graphs(bridge_ctx* ctx) {
    if (ctx->eexec) { cudaGraphExecDestroy(ctx->eexec); ctx->eexec = nullptr; }
    if (ctx->gexec) { cudaGraphExecDestroy(ctx->gexec); ctx->gexec = nullptr; }
    for (auto& h : ctx->hexec)
        if (h) { cudaGraphExecDestroy(h); h = nullptr; }
    ctx->hkey = -1;
    for (auto& k : ctx->ekey) k = nullptr;
    for (auto& k : ctx->gkey) k = nullptr;
}

// Launch-shape search on the caller's own problem: for each tuned kernel class
// in turn, every candidate runs three whole gradient evaluations with per-launch
// events and scores the best of the last two; the others keep their current
// choice.  The tuned kernels compute the same values under every candidate
// (each tile or voxel is handled whole by one thread block, no cross-block
// sums), so only the time differs.
template <typename T> int do_autotune(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                                      int32_t* choices) {
    if (!nu || !counts) return fail(ctx, BRIDGE_EINVAL, "nu and counts are required");
    RUN(upload_bias<T>(ctx, bias));
    const T* nuT = reinterpret_cast<const T*>(nu);
    T* g = reinterpret_cast<T*>(ctx->grad_tmp);
    const bool prof0 = ctx->prof;
    drop_graphs(ctx);
    const char* cls[4] = {"node_alpt", "node_alpt_adj", "node_cic_gather", "web_bias_adj"};
    const int wide = pw_blocks_wide(ctx->n);
    std::vector<int> cand[4];
    for (int k = 0; k < 3; ++k) cand[k] = {0, 1, 2, 3, 4, 5, 6, 8};
    cand[3] = {0, pw_blocks(ctx->n), std::max(1, wide / 4), std::max(1, wide / 2), 2 * wide};
    int st = BRIDGE_OK;
    for (int k = 0; k < 4 && st == BRIDGE_OK; ++k) {
        double best = 1e300;
        int best_c = ctx->tune[k];
        std::vector<int> seen;
        for (int c : cand[k]) {
            if (std::find(seen.begin(), seen.end(), c) != seen.end()) continue;
            seen.push_back(c);
            ctx->tune[k] = c;
            double t = 1e300;
            for (int rep = 0; rep < 3 && st == BRIDGE_OK; ++rep) {
                ctx->prof = true;
                ctx->prof_recs.clear();
                ctx->prof_used = 0;
                st = eval_body<T>(ctx, nuT, counts, g, false);
                double ms = 0.0;
                if (st == BRIDGE_OK) st = prof_class_ms(ctx, cls[k], &ms);
                if (rep > 0) t = std::min(t, ms);
            }
            if (st != BRIDGE_OK) break;
            if (t < best) { best = t; best_c = c; }
        }
        ctx->tune[k] = best_c;
    }
    ctx->prof = prof0;
    ctx->prof_recs.clear();
    ctx->prof_used = 0;
    if (st == BRIDGE_OK) st = finish(ctx);
    if (st != BRIDGE_OK) {
        for (auto& v : ctx->tune) v = 0;
        return st;
    }
    if (choices)
        for (int k = 0; k < 4; ++k) choices[k] = ctx->tune[k];
    return BRIDGE_OK;
}

}  // namespace

#define DISPATCH(ctx, fn, ...) \
    ((ctx)->cfg.precision == BRIDGE_FP64 ? fn<double>(ctx, __VA_ARGS__) : fn<float>(ctx, __VA_ARGS__))

extern "C" {

int bridge_validate_config(const bridge_config* cfg) { return validate(cfg, nullptr); }

size_t bridge_workspace_bytes(const bridge_config* cfg) {
    if (validate(cfg, nullptr) != BRIDGE_OK) return 0;
    return make_plan(cfg).total;
}

double bridge_pk_amplitude(double sigma, double radius, double ns, double kc, double pw) {
    if (!(sigma > 0) || !(radius > 0) || !(kc > 0) || !std::isfinite(ns) || !std::isfinite(pw)) return -1.0;
    const double s2 = sigma2_unit(radius, ns, kc, pw);
    if (!(s2 > 0) || !std::isfinite(s2)) return -1.0;
    return sigma * sigma / s2;
}

// Device buffers are read with 16-byte vector loads.
static bool aligned16(std::initializer_list<const void*> ptrs) {
    for (const void* p : ptrs)
        if (reinterpret_cast<uintptr_t>(p) & 15u) return false;
    return true;
}
static const char* const kAlignMsg = "device buffers must start on a 16-byte boundary";

static thread_local std::string g_create_error;

static int create_fail(bridge_ctx* ctx, int status, const std::string& why) {
    g_create_error = why;
    if (ctx) bridge_destroy(ctx);
    return status;
}

}  // extern "C"

namespace bridge {
// For the context-free entry point (noalloc.cu).
int validate_config_reason(const bridge_config* c, std::string* why) { return validate(c, why); }
void set_noctx_error(const std::string& why) { g_create_error = why; }
}  // namespace bridge

extern "C" {

int bridge_create(const bridge_config* cfg, void* stream, bridge_ctx** out) {
    g_create_error.clear();
    if (!out) return create_fail(nullptr, BRIDGE_EINVAL, "out is NULL");
    std::string why;
    if (validate(cfg, &why) != BRIDGE_OK) return create_fail(nullptr, BRIDGE_EINVAL, why);
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
        cudaGetLastError();
        return create_fail(nullptr, BRIDGE_ENODEVICE, "no CUDA device");
    }
    bridge_ctx* ctx = new bridge_ctx();
    ctx->cfg = *cfg;
    ctx->stream = reinterpret_cast<cudaStream_t>(stream);
    cudaGetDevice(&ctx->device);
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, ctx->device) != cudaSuccess || prop.major != 10 || prop.minor != 3)
        return create_fail(ctx, BRIDGE_ENODEVICE, "the current device is not of compute capability 10.3");
    ctx->n = cfg->n;
    ctx->B = cfg->batch;
    ctx->nr = cfg->n_regions;
    ctx->nvox = (long long)cfg->n * cfg->n * cfg->n;
    ctx->nspec = (long long)(cfg->n / 2 + 1) * cfg->n * cfg->n;
    ctx->esz = cfg->precision == BRIDGE_FP64 ? 8 : 4;
    ctx->recompute = cfg->recompute_alpt != 0;
    ctx->sp_alpt = ctx->recompute ? SP_ALPT_RECOMP : SP_ALPT_STORED;
    ctx->sp_psi = ctx->recompute ? SP_PSI_RECOMP : SP_PSI_STORED;
    ctx->radial = cfg->rsd_f != 0.0 && cfg->rsd_los == 1;
    ctx->sp_psi1 = ctx->recompute ? kScratchSpec : kMaxSpec;
    ctx->sp_gpsi1 = ctx->sp_psi1 + 3;
    ctx->kp.kf = 2.0 * kPi / cfg->box;
    ctx->kp.inv_kf2 = 1.0 / (ctx->kp.kf * ctx->kp.kf);
    ctx->kp.dx = cfg->box / cfg->n;
    ctx->kp.pk_amp = cfg->pk_amp; ctx->kp.pk_ns = cfg->pk_ns; ctx->kp.pk_kc = cfg->pk_kc; ctx->kp.pk_pow = cfg->pk_pow;
    ctx->kp.r_s = cfg->r_s;
    ctx->kp.set_fp32();
    ctx->wp.sharpness = cfg->sharpness;
    ctx->wp.th_phi = cfg->lambda_th_phi;
    ctx->wp.th_delta = cfg->lambda_th_delta;
    ctx->wp.rho_floor = cfg->rho_floor;
    ctx->wp.tau = cfg->precision == BRIDGE_FP64 ? 1e-10 : 1e-4;
    ctx->wp.n_regions = cfg->n_regions;
    ctx->wp.set_fp32();
    cudaError_t e = upload_twiddles();
    if (e == cudaSuccess) e = upload_node_twiddles();
    if (e != cudaSuccess) return create_fail(ctx, BRIDGE_ECUDA, std::string("twiddle upload: ") + cudaGetErrorString(e));
    const Plan pl = make_plan(cfg);
    e = cudaMalloc(&ctx->ws, pl.total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ctx->ws = nullptr;
        return create_fail(ctx, BRIDGE_ENOMEM, "workspace of " + std::to_string(pl.total) + " bytes: " + cudaGetErrorString(e));
    }
    ctx->ws_bytes = pl.total;
    e = cudaMemset(ctx->ws, 0, pl.total);
    if (e != cudaSuccess) return create_fail(ctx, BRIDGE_ECUDA, std::string("workspace clear: ") + cudaGetErrorString(e));
    char* w = reinterpret_cast<char*>(align_up(reinterpret_cast<size_t>(ctx->ws)));
    for (int i = 0; i < pl.nspec_buf; ++i) { ctx->spec[i] = w; w += pl.spec_bytes; }
    for (int i = 0; i < pl.nreal_buf; ++i) { ctx->real[i] = w; w += pl.real_bytes; }
    ctx->grad_tmp = w; w += pl.real_bytes;
    ctx->snap_nu = w; w += pl.real_bytes;
    ctx->snap_p = w; w += pl.real_bytes;
    ctx->c16 = reinterpret_cast<uint16_t*>(w); w += pl.c16_bytes;
    ctx->partial = reinterpret_cast<double*>(w); w += pl.partial_bytes;
    ctx->sc = reinterpret_cast<ChainScalars*>(w); w += pl.sc_bytes;
    ctx->biasd = reinterpret_cast<BiasD*>(w); w += pl.biasd_bytes;
    ctx->biast = w; w += pl.biast_bytes;
    ctx->node_scratch = w; w += pl.node_bytes;
    ctx->node_cap = pl.node_bytes;
    ctx->rtab = w; w += pl.rtab_bytes;
    ctx->cot = reinterpret_cast<double*>(w);
    ctx->theta = reinterpret_cast<double*>(w + align_up(sizeof(double) * ctx->B));
    ctx->ptheta = ctx->theta + 32 * size_t(ctx->B);
    w += pl.cot_bytes;
    ctx->fixed_acc = pl.fixed_bytes ? reinterpret_cast<unsigned long long*>(w) : nullptr;
    w += pl.fixed_bytes;
    {
        const int rlen = 3 * (cfg->n / 2) * (cfg->n / 2) + 1;
        std::vector<double> tab(size_t(4) * rlen);
        radial_tables_host(cfg->n, ctx->kp, tab.data());
        if (cfg->precision == BRIDGE_FP64) {
            e = cudaMemcpy(ctx->rtab, tab.data(), tab.size() * sizeof(double), cudaMemcpyHostToDevice);
        } else {
            std::vector<float> tf(tab.begin(), tab.end());
            e = cudaMemcpy(ctx->rtab, tf.data(), tf.size() * sizeof(float), cudaMemcpyHostToDevice);
        }
        if (e != cudaSuccess) return create_fail(ctx, BRIDGE_ECUDA, std::string("radial tables: ") + cudaGetErrorString(e));
        ctx->kp.rtab = ctx->rtab;
        ctx->kp.rlen = rlen;
    }
    {
        const size_t need = cfg->precision == BRIDGE_FP64 ? node_scratch_bytes<double>(cfg->n, cfg->batch)
                                                         : node_scratch_bytes<float>(cfg->n, cfg->batch);
        const int grid = cfg->precision == BRIDGE_FP64 ? node_max_grid<double>(cfg->n, cfg->batch)
                                                      : node_max_grid<float>(cfg->n, cfg->batch);
        cudaGetLastError();   // occupancy queries leave no error behind
        if (need > pl.node_bytes || grid < 1)
            return create_fail(ctx, BRIDGE_ECUDA, "node plan: scratch " + std::to_string(need) + " > " +
                                                      std::to_string(pl.node_bytes) + " or grid " + std::to_string(grid));
    }
    if (cudaMalloc(&ctx->errflag, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&ctx->tickets, sizeof(int) * ctx->B) != cudaSuccess ||
        cudaMemset(ctx->tickets, 0, sizeof(int) * ctx->B) != cudaSuccess ||
        cudaMallocHost(&ctx->sc_host, sizeof(ChainScalars) * ctx->B) != cudaSuccess ||
        cudaMallocHost(&ctx->biasd_host, sizeof(BiasD) * ctx->B) != cudaSuccess ||
        cudaMallocHost(&ctx->biast_host, sizeof(BiasT<double>) * ctx->B) != cudaSuccess ||
        cudaMallocHost(&ctx->errflag_host, sizeof(int)) != cudaSuccess ||
        cudaMallocHost(&ctx->cot_host, sizeof(double) * ctx->B) != cudaSuccess) {
        cudaGetLastError();
        return create_fail(ctx, BRIDGE_ENOMEM, "small device or pinned host buffers");
    }
    *out = ctx;
    return BRIDGE_OK;
}

void bridge_destroy(bridge_ctx* ctx) {
    if (!ctx) return;
    if (ctx->stream || ctx->ws) cudaStreamSynchronize(ctx->stream);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->errflag) cudaFree(ctx->errflag);
    if (ctx->tickets) cudaFree(ctx->tickets);
    if (ctx->h_nu) cudaFree(ctx->h_nu);
    if (ctx->h_counts) cudaFree(ctx->h_counts);
    if (ctx->h_grad) cudaFree(ctx->h_grad);
    if (ctx->sc_host) cudaFreeHost(ctx->sc_host);
    if (ctx->biasd_host) cudaFreeHost(ctx->biasd_host);
    if (ctx->biast_host) cudaFreeHost(ctx->biast_host);
    if (ctx->errflag_host) cudaFreeHost(ctx->errflag_host);
    if (ctx->cot_host) cudaFreeHost(ctx->cot_host);
    for (cudaEvent_t e : ctx->prof_pool) cudaEventDestroy(e);
    if (ctx->gexec) cudaGraphExecDestroy(ctx->gexec);
    if (ctx->eexec) cudaGraphExecDestroy(ctx->eexec);
    for (cudaGraphExec_t h : ctx->hexec) if (h) cudaGraphExecDestroy(h);
    if (ctx->gstream) cudaStreamDestroy(ctx->gstream);
    if (ctx->cstream) cudaStreamDestroy(ctx->cstream);
    for (cudaEvent_t e : ctx->gev) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : ctx->hev) if (e) cudaEventDestroy(e);
    delete ctx;
}

int bridge_forward(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                   void* ln_nbar_out, double* logpost_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({nu, counts, ln_nbar_out})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_forward, nu, counts, bias, ln_nbar_out, logpost_out);
}

int bridge_logpost_grad(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                        double* logpost_out, void* grad_nu_out, double* grad_bias_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({nu, counts, grad_nu_out})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_grad, nu, counts, bias, logpost_out, grad_nu_out, grad_bias_out);
}

int bridge_logpost_grad_host(bridge_ctx* ctx, const void* nu_host, const int32_t* counts_host, const bridge_bias* bias,
                             double* logpost_out, void* grad_nu_host, double* grad_bias_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!nu_host || !counts_host || !grad_nu_host) return fail(ctx, BRIDGE_EINVAL, "host buffers are required");
    const size_t fb = size_t(ctx->nvox) * ctx->B * ctx->esz, cb = size_t(ctx->nvox) * ctx->B * sizeof(int32_t);
    if (!ctx->h_nu) {
        if (cudaMalloc(&ctx->h_nu, fb) != cudaSuccess || cudaMalloc(&ctx->h_counts, cb) != cudaSuccess ||
            cudaMalloc(&ctx->h_grad, fb) != cudaSuccess) {
            cudaGetLastError();
            return fail(ctx, BRIDGE_ENOMEM, "device staging for host buffers");
        }
    }
    if (!ctx->prof) {
        // overlapped: the counts are copied and prepared while the forward fields run (host_eval)
        ctx->hcounts = counts_host;
        const int st = DISPATCH(ctx, do_grad, nu_host, counts_host, bias, logpost_out, grad_nu_host, grad_bias_out);
        ctx->hcounts = nullptr;
        if (st != BRIDGE_OK) {
            cudaStreamSynchronize(ctx->stream);   // no copy into the caller's buffers is left in flight
            return st;
        }
        return BRIDGE_OK;
    }
    CK(cudaMemcpyAsync(ctx->h_nu, nu_host, fb, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(ctx->h_counts, counts_host, cb, cudaMemcpyHostToDevice, ctx->stream));
    int st = DISPATCH(ctx, do_grad, ctx->h_nu, ctx->h_counts, bias, logpost_out, ctx->h_grad, grad_bias_out);
    if (st != BRIDGE_OK) return st;
    CK(cudaMemcpyAsync(grad_nu_host, ctx->h_grad, fb, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));
    return BRIDGE_OK;
}

int bridge_logpost_vjp(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                       const double* cotangent, void* grad_nu_out, double* grad_bias_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({nu, counts, grad_nu_out})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_grad, nu, counts, bias, nullptr, grad_nu_out, grad_bias_out, cotangent);
}

int bridge_integrate(bridge_ctx* ctx, void* nu, void* p, const int32_t* counts, const bridge_bias* bias, int32_t scheme,
                     int32_t n_steps, double eps, double* h0_out, double* h1_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({nu, p, counts})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_integrate, nu, p, counts, bias, scheme, n_steps, eps, h0_out, h1_out);
}

int bridge_integrate_joint(bridge_ctx* ctx, void* nu, void* p, double* theta, double* p_theta, const int32_t* counts,
                           const bridge_bias* bias, int32_t scheme, int32_t n_steps, double eps, double* h0_out,
                           double* h1_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!theta || !p_theta) return fail(ctx, BRIDGE_EINVAL, "theta and p_theta are required");
    if (!aligned16({nu, p, counts})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_integrate, nu, p, counts, bias, scheme, n_steps, eps, h0_out, h1_out, theta, p_theta);
}

int bridge_leapfrog_steps(bridge_ctx* ctx, void* nu, void* p, void* grad, const int32_t* counts, const bridge_bias* bias,
                          int32_t n_steps, double eps, double* logpost_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({nu, p, grad, counts})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_steps, nu, p, grad, counts, bias, n_steps, eps, logpost_out);
}

int bridge_dot(bridge_ctx* ctx, const void* a, const void* b, double* out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({a, b})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_dot, a, b, out);
}

int bridge_leapfrog(bridge_ctx* ctx, void* nu, void* p, const int32_t* counts, const bridge_bias* bias, int32_t n_steps,
                    double eps, double* h0_out, double* h1_out) {
    return bridge_integrate(ctx, nu, p, counts, bias, BRIDGE_LEAPFROG, n_steps, eps, h0_out, h1_out);
}

int bridge_debug_field(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias, int32_t which,
                       void* out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({nu, counts, out})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_debug, nu, counts, bias, which, out);
}

int bridge_wiener_init(bridge_ctx* ctx, const int32_t* counts, void* nu_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({counts, nu_out})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_wiener_init, counts, nu_out);
}

int bridge_fft_roundtrip(bridge_ctx* ctx, const void* in, void* out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->launches = 0;
    ctx->err.clear();
    if (!aligned16({in, out})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_fft_roundtrip, in, out);
}

int bridge_autotune(bridge_ctx* ctx, const void* nu, const int32_t* counts, const bridge_bias* bias,
                    int32_t* choices_out) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->err.clear();
    if (!aligned16({nu, counts})) return fail(ctx, BRIDGE_EINVAL, kAlignMsg);
    return DISPATCH(ctx, do_autotune, nu, counts, bias, choices_out);
}

int64_t bridge_last_launch_count(const bridge_ctx* ctx) { return ctx ? ctx->launches : 0; }

int bridge_profile_enable(bridge_ctx* ctx, int enable) {
    if (!ctx) return BRIDGE_EINVAL;
    ctx->prof = enable != 0;
    ctx->prof_recs.clear();
    ctx->prof_used = 0;
    return BRIDGE_OK;
}

int bridge_profile_read(bridge_ctx* ctx, bridge_profile_row* rows, int max_rows) {
    if (!ctx || (!rows && max_rows > 0)) return -BRIDGE_EINVAL;
    if (cudaStreamSynchronize(ctx->stream) != cudaSuccess) return -BRIDGE_ECUDA;
    std::vector<bridge_profile_row> agg;
    for (const auto& r : ctx->prof_recs) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess) return -BRIDGE_ECUDA;
        size_t i = 0;
        while (i < agg.size() && std::strcmp(agg[i].name, r.name) != 0) ++i;
        if (i == agg.size()) {
            bridge_profile_row z{};
            std::snprintf(z.name, sizeof(z.name), "%s", r.name);
            agg.push_back(z);
        }
        agg[i].launches += 1;
        agg[i].total_ms += ms;
        agg[i].bytes += r.bytes;
    }
    const int n = (int)agg.size() < max_rows ? (int)agg.size() : max_rows;
    for (int i = 0; i < n; ++i) rows[i] = agg[i];
    return n;
}

const char* bridge_last_error(const bridge_ctx* ctx) {
    if (ctx) return ctx->err.c_str();
    return g_create_error.empty() ? "context is NULL" : g_create_error.c_str();
}

const char* bridge_status_string(int s) {
    switch (s) {
        case BRIDGE_OK: return "ok";
        case BRIDGE_EINVAL: return "invalid argument";
        case BRIDGE_ENOMEM: return "out of memory";
        case BRIDGE_ECUDA: return "CUDA error";
        case BRIDGE_ENONFINITE: return "non-finite result";
        case BRIDGE_ETIMEOUT: return "device wait timed out";
        case BRIDGE_ENODEVICE: return "no suitable CUDA device";
        default: return "unknown status";
    }
}

}  // extern "C"
