// bridge_delta0_noalloc: the linear density delta0 = IDFT[ sqrt(P(k)/dx^3) DFT(nu) ]
// (M_delta, App. A) computed without allocating device memory.
//
// Who this is for: a caller that may not allocate device memory when it needs
// initial conditions -- code running under a fixed device-memory budget, inside
// a memory pool owned by someone else, or at a point where a cudaMalloc would
// synchronise the device or is not allowed -- and that has no bridge context
// (a context allocates its whole workspace in bridge_create).
//
// How: the five kernels of the delta0 step (z, y, x, y, z passes of passes.cu,
// unchanged) run with their intermediate half spectrum and the radial factor
// table placed in one file-scope device array, g_delta0_scratch, instead of a
// context workspace.  Its fixed size, kDelta0ScratchBytes, is the limit on the
// problem size; larger problems are rejected before anything is launched.
#include <cmath>
#include <mutex>
#include <string>

#include "../../include/bridge.h"
#include "common.cuh"
#include "passes.cuh"

namespace bridge {

// Defined in api.cu: configuration check with a reason, and the thread-local
// message that bridge_last_error(NULL) returns.
int validate_config_reason(const bridge_config* c, std::string* why);
void set_noctx_error(const std::string& why);

namespace {

constexpr size_t kDelta0ScratchBytes = size_t(4) << 20;   // 4 MiB
constexpr int kMaxDevices = 64;

// The only device memory this entry point uses besides the caller's nu and
// delta0.  Nothing in it has to start at zero: every call writes the spectrum
// and the table before it reads them.
static __device__ __align__(256) unsigned char g_delta0_scratch[kDelta0ScratchBytes];

std::mutex g_init_mutex;
void* g_scratch_addr[kMaxDevices];   // device address of g_delta0_scratch, per device
bool g_ready[kMaxDevices];           // twiddle tables of passes.cu uploaded, per device

inline size_t align256(size_t v) { return (v + 255) & ~size_t(255); }

// Bytes of scratch a configuration needs: B half spectra, then the radial
// table slots of codes R_INVK2 (unused here) and R_SQRTP.
size_t delta0_need(int n, int batch, int esz) {
    const size_t nspec = size_t(n / 2 + 1) * n * n;
    const size_t rlen = size_t(3) * (n / 2) * (n / 2) + 1;
    return align256(size_t(batch) * nspec * 2 * esz) + align256(2 * rlen * esz);
}

// R_SQRTP slot of the radial table: sqrt(P(k)/dx^3) with
// P(k) = A k^ns (1 + (k/kc)^2)^-pow and P(0) = 0 (App. A), at k^2 = kf^2 m2.
template <typename T>
__global__ void k_sqrtp_table(int rlen, double kf, double amp_dx3, double ns, double kc, double pw, T* tab) {
    const int m2 = blockIdx.x * blockDim.x + threadIdx.x;
    if (m2 >= rlen) return;
    const double k2 = kf * kf * double(m2);
    const double v = m2 > 0 ? sqrt(amp_dx3) * pow(k2, 0.25 * ns) * pow(1.0 + k2 / (kc * kc), -0.5 * pw) : 0.0;
    tab[rlen + m2] = T(v);
}

Term term(int src, int dst, int rcode, double cre) {
    Term t{};
    t.src = int8_t(src);
    t.dst = int8_t(dst);
    t.rcode = int8_t(rcode);
    t.cre = cre;
    return t;
}

template <typename T>
int run_delta0(const bridge_config* cfg, const void* nu, void* delta0, void* scratch, cudaStream_t s) {
    const int n = cfg->n, B = cfg->batch;
    const long long nvox = (long long)n * n * n, nspec = (long long)(n / 2 + 1) * n * n;
    const int rlen = 3 * (n / 2) * (n / 2) + 1;
    char* w = reinterpret_cast<char*>(scratch);
    void* spec = w;
    T* tab = reinterpret_cast<T*>(w + align256(size_t(B) * nspec * 2 * sizeof(T)));

    KParams kp{};
    kp.kf = 2.0 * kPi / cfg->box;
    kp.inv_kf2 = 1.0 / (kp.kf * kp.kf);
    kp.dx = cfg->box / n;
    kp.pk_amp = cfg->pk_amp;
    kp.pk_ns = cfg->pk_ns;
    kp.pk_kc = cfg->pk_kc;
    kp.pk_pow = cfg->pk_pow;
    kp.r_s = cfg->r_s;
    kp.rtab = tab;
    kp.rlen = rlen;
    kp.set_fp32();

    auto ck = [](cudaError_t e, const char* what) -> int {
        if (e == cudaSuccess) return BRIDGE_OK;
        cudaGetLastError();
        set_noctx_error(std::string(what) + ": " + cudaGetErrorString(e));
        return BRIDGE_ECUDA;
    };
    int st;
    k_sqrtp_table<T><<<(rlen + 255) / 256, 256, 0, s>>>(rlen, kp.kf, cfg->pk_amp / (kp.dx * kp.dx * kp.dx),
                                                        cfg->pk_ns, cfg->pk_kc, cfg->pk_pow, tab);
    if ((st = ck(cudaGetLastError(), "radial table")) != BRIDGE_OK) return st;

    ZProgram zf{};
    zf.n_fields = 1;
    zf.in[0] = nu;
    zf.out[0] = spec;
    zf.in_cs = nvox;
    zf.out_cs = nspec;
    if ((st = ck(launch_z_fwd<T>(n, B, zf, s), "z pass")) != BRIDGE_OK) return st;

    PassProgram p{};
    p.n_in = p.n_out = 1;
    p.in[0] = spec;
    p.out[0] = spec;
    p.in_cs = p.out_cs = nspec;
    p.n_merge = 1;
    p.merge[0] = term(0, 0, R_ONE, 1.0);
    if ((st = ck(launch_y_fwd<T>(n, B, p, kp, s), "y pass")) != BRIDGE_OK) return st;

    // x node: the whole k is known here; multiply by sqrt(P/dx^3) and 1/N^3 (the
    // single normalisation of the forward/inverse pair)
    p.merge[0] = term(0, 0, R_SQRTP, 1.0 / double(nvox));
    p.n_expand = 1;
    p.expand[0] = term(0, 0, R_ONE, 1.0);
    if ((st = ck(launch_x_node<T>(n, B, p, kp, s), "x node")) != BRIDGE_OK) return st;

    p.n_merge = 0;
    if ((st = ck(launch_y_inv<T>(n, B, p, kp, s), "y pass")) != BRIDGE_OK) return st;

    ZProgram zi{};
    zi.n_fields = 1;
    zi.in[0] = spec;
    zi.out[0] = delta0;
    zi.in_cs = nspec;
    zi.out_cs = nvox;
    return ck(launch_z_inv<T>(n, B, zi, s), "z pass");
}

}  // namespace
}  // namespace bridge

using namespace bridge;

extern "C" int bridge_delta0_noalloc(const bridge_config* cfg, const void* nu, void* delta0, void* stream) {
    set_noctx_error("");
    std::string why;
    if (validate_config_reason(cfg, &why) != BRIDGE_OK) {
        set_noctx_error(why);
        return BRIDGE_EINVAL;
    }
    if (!nu || !delta0) {
        set_noctx_error("nu and delta0 are required");
        return BRIDGE_EINVAL;
    }
    const int esz = cfg->precision == BRIDGE_FP64 ? 8 : 4;
    const size_t need = delta0_need(cfg->n, cfg->batch, esz);
    if (need > kDelta0ScratchBytes) {
        set_noctx_error("bridge_delta0_noalloc: n = " + std::to_string(cfg->n) + ", batch = " +
                        std::to_string(cfg->batch) + " needs " + std::to_string(need) +
                        " bytes of scratch; the static scratch holds " + std::to_string(kDelta0ScratchBytes) +
                        " bytes (use a context for larger problems)");
        return BRIDGE_EINVAL;
    }
    int ndev = 0, dev = -1;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1 || cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        set_noctx_error("no CUDA device");
        return BRIDGE_ENODEVICE;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        set_noctx_error("device index beyond " + std::to_string(kMaxDevices));
        return BRIDGE_EINVAL;
    }
    void* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_init_mutex);
        if (!g_ready[dev]) {
            int major = 0, minor = 0;
            cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev);
            cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev);
            if (major != 10 || minor != 3) {
                cudaGetLastError();
                set_noctx_error("the current device is not of compute capability 10.3");
                return BRIDGE_ENODEVICE;
            }
            // Once per device, with that device current: the scratch address
            // and the twiddle tables (both plain copies/lookups, no allocation).
            cudaError_t e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_delta0_scratch);
            if (e == cudaSuccess) e = upload_twiddles();
            if (e != cudaSuccess) {
                cudaGetLastError();
                g_scratch_addr[dev] = nullptr;
                set_noctx_error(std::string("first-call setup: ") + cudaGetErrorString(e));
                return BRIDGE_ECUDA;
            }
            g_ready[dev] = true;
        }
        scratch = g_scratch_addr[dev];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    return cfg->precision == BRIDGE_FP64 ? run_delta0<double>(cfg, nu, delta0, scratch, s)
                                         : run_delta0<float>(cfg, nu, delta0, scratch, s);
}
