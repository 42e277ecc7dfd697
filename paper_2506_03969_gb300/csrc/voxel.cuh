// Per-voxel arithmetic of the method (device functions shared by the kernels).
#pragma once

#include "common.cuh"

namespace bridge {

__device__ __forceinline__ float v_sqrt(float x) { return sqrtf(x); }
__device__ __forceinline__ double v_sqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float v_exp(float x) { return expf(x); }
__device__ __forceinline__ double v_exp(double x) { return exp(x); }
__device__ __forceinline__ float v_log(float x) { return logf(x); }
__device__ __forceinline__ double v_log(double x) { return log(x); }
__device__ __forceinline__ float v_log1p(float x) { return log1pf(x); }
__device__ __forceinline__ double v_log1p(double x) { return log1p(x); }
__device__ __forceinline__ float v_acos(float x) { return acosf(x); }
__device__ __forceinline__ double v_acos(double x) { return acos(x); }
// Fast single-precision exp/log/reciprocal for the web and bias arithmetic
// (hardware approximations with relative errors of a few 1e-7 on the argument
// ranges that occur; FP64 keeps the correctly rounded library functions).
// Building with -DBRIDGE_ACCURATE_WEB_MATH selects the accurate FP32 library
// functions and IEEE division instead, for measuring what the approximations cost.
#ifdef BRIDGE_ACCURATE_WEB_MATH
__device__ __forceinline__ float v_fexp(float x) { return expf(x); }
__device__ __forceinline__ float v_flog(float x) { return logf(x); }
__device__ __forceinline__ float v_fdiv(float a, float b) { return a / b; }
#else
__device__ __forceinline__ float v_fexp(float x) { return __expf(x); }
__device__ __forceinline__ float v_flog(float x) { return __logf(x); }
__device__ __forceinline__ float v_fdiv(float a, float b) { return __fdividef(a, b); }
#endif
__device__ __forceinline__ double v_fexp(double x) { return exp(x); }
__device__ __forceinline__ double v_flog(double x) { return log(x); }
__device__ __forceinline__ double v_fdiv(double a, double b) { return a / b; }

// sin/cos of pi * x (no large-argument reduction path)
__device__ __forceinline__ void v_sincospi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void v_sincospi(double x, double* s, double* c) { sincospi(x, s, c); }
__device__ __forceinline__ float v_fmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double v_fmax(double a, double b) { return fmax(a, b); }

// Stored symmetric-tensor component order: xx, xy, xz, yy, yz, zz.

// Eigen-decomposition data of a symmetric 3x3 tensor A: m = tr(A)/3, B = A - m I,
// eigenvalues mu1 >= mu2 >= mu3 of B (lambda_n = m + mu_n), by the trigonometric
// solution of the characteristic cubic (Smith 1961), App. B ordering.  Where two
// eigenvalues nearly coincide (|r| within kEigPairBand of 1, r = det B / (2 p^3)),
// the cubic fixes the pair only to about sqrt(epsilon) of the scale; there the
// isolated eigenvalue is kept and the pair is taken from the 2x2 block of B in
// the plane orthogonal to its eigenvector (eig_pair).
constexpr double kEigPairBand = 1e-3;
template <typename T> struct Eig3 {
    T m;
    T mu[3];
};

template <typename T> __device__ __forceinline__ T dot3(const T u[3], const T v[3]) {
    return u[0] * v[0] + u[1] * v[1] + u[2] * v[2];
}
template <typename T> __device__ __forceinline__ void cross3(const T u[3], const T v[3], T w[3]) {
    w[0] = u[1] * v[2] - u[2] * v[1];
    w[1] = u[2] * v[0] - u[0] * v[2];
    w[2] = u[0] * v[1] - u[1] * v[0];
}
// B v for the symmetric B stored as xx, xy, xz, yy, yz, zz
template <typename T> __device__ __forceinline__ void symv(const T b[6], const T v[3], T w[3]) {
    w[0] = b[0] * v[0] + b[1] * v[1] + b[2] * v[2];
    w[1] = b[1] * v[0] + b[3] * v[1] + b[4] * v[2];
    w[2] = b[2] * v[0] + b[4] * v[1] + b[5] * v[2];
}

// The two eigenvalues of traceless B other than an isolated one, iso, by
// deflation: v = the eigenvector of iso (the largest cross product of two rows
// of B - iso I), an orthonormal pair u, w spanning its complement, and the 2x2
// block [u.Bu, u.Bw; w.Bu, w.Bw] with trace -iso, whose eigenvalues are
// -iso/2 +- sqrt(h^2 + q^2) with h = (u.Bu - w.Bw)/2, q = u.Bw.  The gap of
// the pair comes out as a square root of a sum of squares, accurate however
// small it is, whereas from the invariants of the characteristic cubic it is
// lost to cancellation (an error of order sqrt(epsilon) times the scale).
template <typename T> __device__ __forceinline__ void eig_pair(const T b[6], T iso, T& hi, T& lo) {
    const T r0[3] = {b[0] - iso, b[1], b[2]}, r1[3] = {b[1], b[3] - iso, b[4]}, r2[3] = {b[2], b[4], b[5] - iso};
    T c01[3], c02[3], c12[3];
    cross3(r0, r1, c01);
    cross3(r0, r2, c02);
    cross3(r1, r2, c12);
    const T n01 = dot3(c01, c01), n02 = dot3(c02, c02), n12 = dot3(c12, c12);
    T v[3];
    T nv = n01;
    v[0] = c01[0]; v[1] = c01[1]; v[2] = c01[2];
    if (n02 > nv) { nv = n02; v[0] = c02[0]; v[1] = c02[1]; v[2] = c02[2]; }
    if (n12 > nv) { nv = n12; v[0] = c12[0]; v[1] = c12[1]; v[2] = c12[2]; }
    if (!(nv > T(0))) { hi = lo = T(-0.5) * iso; return; }
    const T iv = T(1) / v_sqrt(nv);
    v[0] *= iv; v[1] *= iv; v[2] *= iv;
    // u: v crossed with the coordinate axis least aligned with v
    const T ax = v[0] < T(0) ? -v[0] : v[0], ay = v[1] < T(0) ? -v[1] : v[1], az = v[2] < T(0) ? -v[2] : v[2];
    T u[3];
    if (ax <= ay && ax <= az) { u[0] = T(0); u[1] = v[2]; u[2] = -v[1]; }
    else if (ay <= az) { u[0] = -v[2]; u[1] = T(0); u[2] = v[0]; }
    else { u[0] = v[1]; u[1] = -v[0]; u[2] = T(0); }
    const T iu = T(1) / v_sqrt(dot3(u, u));
    u[0] *= iu; u[1] *= iu; u[2] *= iu;
    T w[3], bu[3], bw[3];
    cross3(v, u, w);
    symv(b, u, bu);
    symv(b, w, bw);
    const T h = T(0.5) * (dot3(u, bu) - dot3(w, bw)), q = dot3(u, bw);
    const T g = v_sqrt(h * h + q * q);
    hi = T(-0.5) * iso + g;
    lo = T(-0.5) * iso - g;
}

template <typename T> __device__ __forceinline__ void eig3(const T a[6], Eig3<T>& e) {
    e.m = (a[0] + a[3] + a[5]) * T(1.0 / 3.0);
    const T b[6] = {a[0] - e.m, a[1], a[2], a[3] - e.m, a[4], a[5] - e.m};
    const T off = b[1] * b[1] + b[2] * b[2] + b[4] * b[4];
    const T p2 = (b[0] * b[0] + b[3] * b[3] + b[5] * b[5] + T(2) * off) * T(1.0 / 6.0);
    if (!(p2 > T(0))) { e.mu[0] = e.mu[1] = e.mu[2] = T(0); return; }
    const T p = v_sqrt(p2);
    const T det = b[0] * (b[3] * b[5] - b[4] * b[4]) - b[1] * (b[1] * b[5] - b[4] * b[2]) +
                  b[2] * (b[1] * b[4] - b[3] * b[2]);
    T r = v_fdiv(det, T(2) * p2 * p);
    r = r < T(-1) ? T(-1) : (r > T(1) ? T(1) : r);
    // phi = acos(r)/3 in [0, pi/3], evaluated as sin/cos of pi * (phi / pi)
    const T phi_pi = v_acos(r) * T(0.10610329539459689051);   // 1 / (3 pi)
    T s, c;
    v_sincospi(phi_pi, &s, &c);
    // cos(phi + 2pi/3) = -c/2 - (sqrt3/2) s
    const T mu1 = T(2) * p * c;
    const T mu3 = T(2) * p * (T(-0.5) * c - T(0.86602540378443864676) * s);
    if (r > T(1) - T(kEigPairBand)) {
        // mu2 close to mu3: mu1 is isolated and accurate; the pair by deflation
        T hi, lo;
        eig_pair<T>(b, mu1, hi, lo);
        e.mu[0] = mu1; e.mu[1] = hi; e.mu[2] = lo;
        return;
    }
    if (r < T(-1) + T(kEigPairBand)) {
        // mu2 close to mu1: mu3 is isolated
        T hi, lo;
        eig_pair<T>(b, mu3, hi, lo);
        e.mu[0] = hi; e.mu[1] = lo; e.mu[2] = mu3;
        return;
    }
    T mu2 = -mu1 - mu3;
    mu2 = mu2 > mu1 ? mu1 : (mu2 < mu3 ? mu3 : mu2);
    e.mu[0] = mu1; e.mu[1] = mu2; e.mu[2] = mu3;
}

template <typename T> __device__ __forceinline__ T sigmoid(T x) { return v_fdiv(T(1), T(1) + v_fexp(-x)); }

// Fuzzy memberships (Eq. sigmoid, Eq. soft_cweb_p): w_n = sigma(s (lambda_n - th)),
// p = (V, S, F, K) = (1 - w1, w1 - w2, w2 - w3, w3).  1 - w1 is formed as
// sigma(-x1) to avoid cancellation.
template <typename T> __device__ __forceinline__ void memberships(const T lam[3], T s, T th, T w[3], T p[4]) {
    const T x1 = s * (lam[0] - th), x2 = s * (lam[1] - th), x3 = s * (lam[2] - th);
    w[0] = sigmoid(x1); w[1] = sigmoid(x2); w[2] = sigmoid(x3);
    p[0] = sigmoid(-x1);
    p[1] = w[0] - w[1];
    p[2] = w[1] - w[2];
    p[3] = w[2];
}

// Bias table of one chain (precision T), Eq. local_bias + NB beta, stored per
// region as (a, alpha, rho, eps, rhop, epsp, beta, flags) so that one region is
// two 16-byte (FP32) shared-memory loads.  flags of region 0: 1 if any region
// has a second cut-off (rho' > 0), else 0 (then rho', eps' and their
// derivatives are skipped: they would only add zeros).
template <typename T> struct __align__(16) BiasT {
    T pk[16][8];
};
enum { BP_A = 0, BP_ALPHA = 1, BP_RHO = 2, BP_EPS = 3, BP_RHOP = 4, BP_EPSP = 5, BP_BETA = 6, BP_FLAGS = 7 };

// The 7 parameters of region r (vector loads from shared memory).
__device__ __forceinline__ void region_params(const BiasT<float>& B, int r, float e[8]) {
    const float4 lo = *reinterpret_cast<const float4*>(&B.pk[r][0]);
    const float4 hi = *reinterpret_cast<const float4*>(&B.pk[r][4]);
    e[0] = lo.x; e[1] = lo.y; e[2] = lo.z; e[3] = lo.w; e[4] = hi.x; e[5] = hi.y; e[6] = hi.z; e[7] = hi.w;
}
__device__ __forceinline__ void region_params(const BiasT<double>& B, int r, double e[8]) {
#pragma unroll
    for (int q = 0; q < 8; q += 2) {
        const double2 d = *reinterpret_cast<const double2*>(&B.pk[r][q]);
        e[q] = d.x; e[q + 1] = d.y;
    }
}

// Per-voxel interpolated parameters b_i = sum_r b^(r) p_i^(r) (Sect. 2.8).
template <typename T> struct VoxParams {
    T a, alpha, rho, eps, rhop, epsp, beta;
};

// ln f = ln a + alpha ln u - (u/rho)^eps - (rho'/u)^eps'  (Eq. local_bias in logs),
// u = max(1 + delta, floor), passed in as the CIC mass rho = 1 + delta itself so
// that nearly empty cells keep full relative precision.  Returns ln f; t1, t2
// are the two cut-off terms.
template <typename T> struct LnF {
    T lnf, lnu, t1, t2, lnrho, lnrhop;
    bool floored;
};
template <typename T> __device__ __forceinline__ void log_f(T rho_mass, T floor_, const VoxParams<T>& q, LnF<T>& r) {
    T u = rho_mass;
    r.floored = !(u > floor_);
    if (r.floored) u = floor_;
    r.lnu = v_flog(u);
    r.lnrho = v_flog(q.rho);
    r.t1 = v_fexp(q.eps * (r.lnu - r.lnrho));
    if (q.rhop > T(0)) {
        r.lnrhop = v_flog(q.rhop);
        r.t2 = v_fexp(q.epsp * (r.lnrhop - r.lnu));
    } else {
        r.lnrhop = T(0);
        r.t2 = T(0);
    }
    r.lnf = v_flog(q.a) + q.alpha * r.lnu - r.t1 - r.t2;
}

// Negative-binomial log pmf with shape beta and mean nbar (Sect. 2.6):
//   log P = sum_{m<n} ln((beta+m)/(m+1)) - beta ln(1 + nbar/beta) + n (ln nbar - ln(beta + nbar))
// and its derivatives d/d ln nbar and d/d beta.
template <typename T> struct NB {
    T logp, g_lnnbar, g_beta;
};
template <typename T> __device__ __forceinline__ void nb_eval(int n, T lnnbar, T beta, bool want_grad, NB<T>& r) {
    const T nbar = v_fexp(lnnbar);
    const T l1 = v_log1p(v_fdiv(nbar, beta));        // ln((beta + nbar)/beta)
    T s = T(0), ds = T(0);
    for (int m = 0; m < n; ++m) {
        s += v_flog(v_fdiv(beta + T(m), T(m + 1)));
        if (want_grad) ds += v_fdiv(T(1), beta + T(m));
    }
    const T tn = T(n);
    r.logp = s - beta * l1 + (n > 0 ? tn * (lnnbar - v_flog(beta) - l1) : T(0));
    if (want_grad) {
        const T rden = v_fdiv(T(1), nbar + beta);
        r.g_lnnbar = beta * (tn - nbar) * rden;
        r.g_beta = ds - l1 + (nbar - tn) * rden;
    }
}

// d lambda-sum / d A for symmetric A: G = sum_n g_n v_n v_n^T written with the
// invariant (projector) form of App. B: P_n = prod_{m != n} (B - mu_m)/(mu_n - mu_m),
//   G = g2 I + (g1 - g2) P_1 + (g3 - g2) P_3.
// Near-equal eigenvalues (gap < tau * scale) share the mean of their g's (a
// subgradient; the exact gradient is not defined at a crossing).  Output is the
// derivative with respect to the stored components (off-diagonals count twice).
template <typename T>
__device__ __forceinline__ void eig_adjoint(const T a[6], const Eig3<T>& e, T g1, T g2, T g3, T tau, T out[6]) {
    const T mu1 = e.mu[0], mu2 = e.mu[1], mu3 = e.mu[2];
    const T scale = v_fmax(mu1 > T(0) ? mu1 : -mu1, mu3 > T(0) ? mu3 : -mu3) + v_fmax(e.m > T(0) ? e.m : -e.m, T(0));
    const T tol = tau * scale + T(1e-30);
    const bool t12 = (mu1 - mu2) < tol, t23 = (mu2 - mu3) < tol;
    if (t12 && t23) {
        const T gm = (g1 + g2 + g3) * T(1.0 / 3.0);
        g1 = g2 = g3 = gm;
    } else if (t12) {
        const T gm = T(0.5) * (g1 + g2);
        g1 = g2 = gm;
    } else if (t23) {
        const T gm = T(0.5) * (g2 + g3);
        g2 = g3 = gm;
    }
    const T b[6] = {a[0] - e.m, a[1], a[2], a[3] - e.m, a[4], a[5] - e.m};
    T G[6] = {g2, T(0), T(0), g2, T(0), g2};
    const T c1 = g1 - g2, c3 = g3 - g2;
    if (c1 != T(0) || c3 != T(0)) {
        T b2[6];
        b2[0] = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
        b2[1] = b[0] * b[1] + b[1] * b[3] + b[2] * b[4];
        b2[2] = b[0] * b[2] + b[1] * b[4] + b[2] * b[5];
        b2[3] = b[1] * b[1] + b[3] * b[3] + b[4] * b[4];
        b2[4] = b[1] * b[2] + b[3] * b[4] + b[4] * b[5];
        b2[5] = b[2] * b[2] + b[4] * b[4] + b[5] * b[5];
        if (c1 != T(0)) {
            const T s = v_fdiv(c1, (mu1 - mu2) * (mu1 - mu3));
            const T lin = -(mu2 + mu3), cst = mu2 * mu3;
#pragma unroll
            for (int q = 0; q < 6; ++q) G[q] += s * (b2[q] + lin * b[q]);
            G[0] += s * cst; G[3] += s * cst; G[5] += s * cst;
        }
        if (c3 != T(0)) {
            const T s = v_fdiv(c3, (mu3 - mu1) * (mu3 - mu2));
            const T lin = -(mu1 + mu2), cst = mu1 * mu2;
#pragma unroll
            for (int q = 0; q < 6; ++q) G[q] += s * (b2[q] + lin * b[q]);
            G[0] += s * cst; G[3] += s * cst; G[5] += s * cst;
        }
    }
    out[0] = G[0]; out[1] = T(2) * G[1]; out[2] = T(2) * G[2];
    out[3] = G[3]; out[4] = T(2) * G[4]; out[5] = G[5];
}

// ---------------------------------------------------------------------------
// Fused web + bias per voxel (Sect. 2.5-2.8): eigenvalues of the tidal tensor
// (and of the density Hessian for 16 regions), memberships, region weights
// p_{4j+k} = pPhi_j pdelta_k, interpolated parameters and ln f.
// ---------------------------------------------------------------------------
struct WebParams {
    double sharpness, th_phi, th_delta, rho_floor, tau;
    int n_regions;
    float f_sharpness, f_th_phi, f_th_delta, f_tau;   // FP32 copies (see KParams)
    void set_fp32() {
        f_sharpness = float(sharpness); f_th_phi = float(th_phi); f_th_delta = float(th_delta); f_tau = float(tau);
    }
};
// The FP32 copy of a parameter in FP32 code, the double itself in FP64 code.
template <typename T> __device__ __forceinline__ T pick(double d, float f) {
    if constexpr (sizeof(T) == 4) return f;
    else return T(d);
}

template <typename T, int NR> struct WebState {
    Eig3<T> ephi, edel;
    T wphi[3], pphi[4], wdel[3], pdel[4];
    VoxParams<T> q;
    LnF<T> lf;
};

// Region weight of region r = 4j + k: pPhi_j * pdelta_k (hierarchical), pPhi_r otherwise.
template <typename T, int NR, typename S>
__device__ __forceinline__ T region_w(const S& st, int j, int k) {
    if constexpr (NR == 16) return st.pphi[j] * st.pdel[k];
    else return st.pphi[j];
}

template <typename T, int NR>
__device__ __forceinline__ void web_eval(const T a6[6], const T h6[6], T rho_mass, const BiasT<T>& B,
                                         const WebParams& wp, WebState<T, NR>& S) {
    eig3<T>(a6, S.ephi);
    T lam[3] = {S.ephi.m + S.ephi.mu[0], S.ephi.m + S.ephi.mu[1], S.ephi.m + S.ephi.mu[2]};
    memberships<T>(lam, pick<T>(wp.sharpness, wp.f_sharpness), pick<T>(wp.th_phi, wp.f_th_phi), S.wphi, S.pphi);
    if constexpr (NR == 16) {
        eig3<T>(h6, S.edel);
        T ld[3] = {S.edel.m + S.edel.mu[0], S.edel.m + S.edel.mu[1], S.edel.m + S.edel.mu[2]};
        memberships<T>(ld, pick<T>(wp.sharpness, wp.f_sharpness), pick<T>(wp.th_delta, wp.f_th_delta), S.wdel, S.pdel);
    }
    VoxParams<T>& q = S.q;
    q.a = q.alpha = q.rho = q.eps = q.rhop = q.epsp = q.beta = T(0);
    constexpr int NK = NR == 16 ? 4 : 1;
    const bool cut2 = B.pk[0][BP_FLAGS] != T(0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NK; ++b) {
            const int r = NK * a + b;
            const T w = region_w<T, NR>(S, a, b);
            T e[8];
            region_params(B, r, e);
            q.a += e[BP_A] * w; q.alpha += e[BP_ALPHA] * w; q.rho += e[BP_RHO] * w; q.eps += e[BP_EPS] * w;
            q.beta += e[BP_BETA] * w;
            if (cut2) { q.rhop += e[BP_RHOP] * w; q.epsp += e[BP_EPSP] * w; }
        }
    // the floor is converted from the double parameter here: with the FP32 copy the
    // web adjoint's allocation spills at its 64-register bound
    log_f<T>(rho_mass, T(wp.rho_floor), S.q, S.lf);
}

// Adjoint of web_eval + normalisation + NB for one voxel.  Inputs: the forward
// state, the CIC mass rho, the count n, ln C and G/N_tr.  Outputs: g_rho
// (direct), g_T and g_H (stored components); accumulates d/d alpha_r and
// d/d beta_r into ga/gb when BIASG.
template <typename T, int NR, bool BIASG, typename LoadT>
__device__ __forceinline__ void web_adjoint_voxel(const WebState<T, NR>& S, T rho_mass, int n, T lnC, T gscale,
                                                  const BiasT<T>& B, const WebParams& wp, LoadT load_tensors,
                                                  T& gd, T gt[6], T gh[6], T* ga, T* gb) {
    const T s = pick<T>(wp.sharpness, wp.f_sharpness), tau = pick<T>(wp.tau, wp.f_tau);
    const T lnnbar = S.lf.lnf + lnC;
    NB<T> nb;
    nb_eval<T>(n, lnnbar, S.q.beta, true, nb);
    const T nbar = v_fexp(lnnbar);
    const T glnf = nb.g_lnnbar - nbar * gscale;      // normalisation adjoint: f_i/sum f * G = nbar_i G / N_tr
    const T gbeta = nb.g_beta;
    const T g_a = v_fdiv(glnf, S.q.a);
    const T g_al = glnf * S.lf.lnu;
    const T g_rho = v_fdiv(glnf * S.q.eps * S.lf.t1, S.q.rho);
    const T g_eps = -glnf * S.lf.t1 * (S.lf.lnu - S.lf.lnrho);
    T g_rhop = T(0), g_epsp = T(0);
    if (S.q.rhop > T(0)) {
        g_rhop = -v_fdiv(glnf * S.q.epsp * S.lf.t2, S.q.rhop);
        g_epsp = -glnf * S.lf.t2 * (S.lf.lnrhop - S.lf.lnu);
    }
    // direct density derivative (zero below the floor); u = rho
    gd = S.lf.floored ? T(0) : v_fdiv(glnf * (S.q.alpha - S.q.eps * S.lf.t1 + S.q.epsp * S.lf.t2), rho_mass);
    T gpphi[4] = {T(0), T(0), T(0), T(0)}, gpdel[4] = {T(0), T(0), T(0), T(0)};
    constexpr int NK = NR == 16 ? 4 : 1;
    const bool cut2 = B.pk[0][BP_FLAGS] != T(0);
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < NK; ++b) {
            const int r = NK * a + b;
            T e[8];
            region_params(B, r, e);
            T gw = g_a * e[BP_A] + g_al * e[BP_ALPHA] + g_rho * e[BP_RHO] + g_eps * e[BP_EPS] + gbeta * e[BP_BETA];
            if (cut2) gw += g_rhop * e[BP_RHOP] + g_epsp * e[BP_EPSP];
            if constexpr (NR == 16) {
                gpphi[a] += gw * S.pdel[b];
                gpdel[b] += gw * S.pphi[a];
            } else {
                gpphi[a] = gw;
            }
            if constexpr (BIASG) {
                const T w = region_w<T, NR>(S, a, b);
                ga[r] += g_al * w;
                gb[r] += gbeta * w;
            }
        }
    // eigenvalue adjoint with the tensors reloaded (they are no longer live)
    T a6[6], h6[6];
    load_tensors(a6, h6);
    {
        const T g1 = (gpphi[1] - gpphi[0]) * s * S.wphi[0] * (T(1) - S.wphi[0]);
        const T g2 = (gpphi[2] - gpphi[1]) * s * S.wphi[1] * (T(1) - S.wphi[1]);
        const T g3 = (gpphi[3] - gpphi[2]) * s * S.wphi[2] * (T(1) - S.wphi[2]);
        eig_adjoint<T>(a6, S.ephi, g1, g2, g3, tau, gt);
    }
    if constexpr (NR == 16) {
        const T g1 = (gpdel[1] - gpdel[0]) * s * S.wdel[0] * (T(1) - S.wdel[0]);
        const T g2 = (gpdel[2] - gpdel[1]) * s * S.wdel[1] * (T(1) - S.wdel[1]);
        const T g3 = (gpdel[3] - gpdel[2]) * s * S.wdel[2] * (T(1) - S.wdel[2]);
        eig_adjoint<T>(h6, S.edel, g1, g2, g3, tau, gh);
    }
}

// ALPT sources (Sect. 2.3): a = -D delta0 + D2 S2 (2LPT divergence) and the
// spherical-collapse divergence 3[(1 - 2/3 D delta0)^(1/2) - 1] (D delta0 < 3/2), -3 otherwise.
// phi = xx, xy, xz, yy, yz, zz of the linear potential Hessian.
template <typename T>
__device__ __forceinline__ void alpt_sources(T d0, const T phi[6], T D, T D2, T& a, T& b) {
    const T s2 = phi[0] * phi[3] + phi[0] * phi[5] + phi[3] * phi[5] - phi[1] * phi[1] - phi[2] * phi[2] - phi[4] * phi[4];
    const T x = D * d0;
    a = -x + D2 * s2;
    T arg = T(1) - T(2.0 / 3.0) * x;
    arg = arg > T(1e-12) ? arg : T(1e-12);
    b = x < T(1.5) ? T(3) * (v_sqrt(arg) - T(1)) : T(-3);
}

// Transpose of alpt_sources: g_delta0 (direct) and g_phi from g_a, g_b.
template <typename T>
__device__ __forceinline__ void alpt_sources_adj(T d0, const T phi[6], T D, T D2, T ga, T gb, T& gd0, T gphi[6]) {
    const T x = D * d0;
    const T arg = T(1) - T(2.0 / 3.0) * x;
    // d theta_SC / d delta0 = -D / sqrt(1 - 2/3 D delta0) on the uncollapsed, unclamped branch
    const T dsc = (x < T(1.5) && arg > T(1e-12)) ? -D / v_sqrt(arg) : T(0);
    const T gs2 = D2 * ga;
    gd0 = -D * ga + dsc * gb;
    gphi[0] = gs2 * (phi[3] + phi[5]);
    gphi[1] = gs2 * (T(-2) * phi[1]);
    gphi[2] = gs2 * (T(-2) * phi[2]);
    gphi[3] = gs2 * (phi[0] + phi[5]);
    gphi[4] = gs2 * (T(-2) * phi[4]);
    gphi[5] = gs2 * (phi[0] + phi[3]);
}

// Radial redshift-space displacement (Sect. 2.9, Eq. of delta(s), b_v = 1, linear
// velocity v/(aH) = f Psi_1): the particle of cell q at r = q + Psi - c relative
// to the observer c at the centre of the volume moves by f (Psi_1 . r) r / |r|^2
// (cell units; not at all when r = 0).  rsd_radial_fwd returns the shifted
// displacement; rsd_radial_adj maps the cotangent G of the shifted displacement to
// those of Psi and Psi_1:
//   g_Psi = G + (f/s) [Psi_1 (r.G) + P G - (2P/s) r (r.G)],  g_Psi1 = (f/s) r (r.G),
// with s = |r|^2, P = Psi_1 . r.
template <typename T> struct RsdPoint {
    T r[3], p1[3], pr, s;   // r, Psi_1, Psi_1 . r, |r|^2
};
template <typename T>
__device__ __forceinline__ void rsd_radial_fwd(const int q[3], T c, const T psi[3], const T psi1[3], T f, RsdPoint<T>& R,
                                               T out[3]) {
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        R.r[j] = (T(q[j]) - c) + psi[j];
        R.p1[j] = psi1[j];
    }
    R.s = R.r[0] * R.r[0] + R.r[1] * R.r[1] + R.r[2] * R.r[2];
    R.pr = psi1[0] * R.r[0] + psi1[1] * R.r[1] + psi1[2] * R.r[2];
    const T a = R.s > T(0) ? f * R.pr / R.s : T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) out[j] = psi[j] + a * R.r[j];
}
template <typename T>
__device__ __forceinline__ void rsd_radial_adj(const RsdPoint<T>& R, T f, const T G[3], T g_psi[3], T g_psi1[3]) {
    if (!(R.s > T(0))) {
#pragma unroll
        for (int j = 0; j < 3; ++j) { g_psi[j] = G[j]; g_psi1[j] = T(0); }
        return;
    }
    const T is = T(1) / R.s;
    const T rg = R.r[0] * G[0] + R.r[1] * G[1] + R.r[2] * G[2];
    const T fs = f * is, c2 = T(2) * R.pr * is * rg;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        g_psi[j] = G[j] + fs * (R.p1[j] * rg + R.pr * G[j] - c2 * R.r[j]);
        g_psi1[j] = fs * rg * R.r[j];
    }
}

// CIC geometry of the particle of cell q (cell units): lower corner and fractions.
template <typename T> struct CicCorner {
    int i0[3];
    T f[3];
};
template <typename T> __device__ __forceinline__ void cic_corner(long long q, int N, T px, T py, T pz, CicCorner<T>& c) {
    const int lg = __ffs(N) - 1;
    const int qz = (int)(q & (N - 1)), qy = (int)((q >> lg) & (N - 1)), qx = (int)(q >> (2 * lg));
    const T fx = floor(px), fy = floor(py), fz = floor(pz);
    c.f[0] = px - fx; c.f[1] = py - fy; c.f[2] = pz - fz;
    c.i0[0] = qx + (int)fx; c.i0[1] = qy + (int)fy; c.i0[2] = qz + (int)fz;
}

// CIC gather adjoint of one particle: g_psi_j = sum_corners g_rho[c] dw_c/dpsi_j.
// Split into the eight corner loads (corner index 4a + 2b + e for offsets a, b, e
// along x, y, z) and their combination, so that callers can issue the loads of
// several particles before combining any of them.
template <typename T> __device__ __forceinline__ void cic_gather_loads(const CicCorner<T>& c, int N, const T* g, T gv[8]) {
    const int msk = N - 1;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const size_t ix = (size_t)((c.i0[0] + a) & msk) * N;
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const size_t iy = (ix + (size_t)((c.i0[1] + b) & msk)) * N;
#pragma unroll
            for (int e = 0; e < 2; ++e) gv[4 * a + 2 * b + e] = g[iy + ((c.i0[2] + e) & msk)];
        }
    }
}
template <typename T> __device__ __forceinline__ void cic_gather_combine(const CicCorner<T>& c, const T gv[8], T out[3]) {
    T gx = 0, gy = 0, gz = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const T wx = a ? c.f[0] : T(1) - c.f[0], dwx = a ? T(1) : T(-1);
#pragma unroll
        for (int b = 0; b < 2; ++b) {
            const T wy = b ? c.f[1] : T(1) - c.f[1], dwy = b ? T(1) : T(-1);
#pragma unroll
            for (int e = 0; e < 2; ++e) {
                const T wz = e ? c.f[2] : T(1) - c.f[2], dwz = e ? T(1) : T(-1);
                const T v = gv[4 * a + 2 * b + e];
                gx += v * dwx * wy * wz;
                gy += v * wx * dwy * wz;
                gz += v * wx * wy * dwz;
            }
        }
    }
    out[0] = gx; out[1] = gy; out[2] = gz;
}
template <typename T> __device__ __forceinline__ void cic_gather_one(const CicCorner<T>& c, int N, const T* g, T out[3]) {
    T gv[8];
    cic_gather_loads<T>(c, N, g, gv);
    cic_gather_combine<T>(c, gv, out);
}

}  // namespace bridge
