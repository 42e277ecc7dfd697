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
__device__ __forceinline__ void v_sincos(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void v_sincos(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float v_fmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double v_fmax(double a, double b) { return fmax(a, b); }

// Stored symmetric-tensor component order: xx, xy, xz, yy, yz, zz.

// Eigen-decomposition data of a symmetric 3x3 tensor A: m = tr(A)/3, B = A - m I,
// eigenvalues mu1 >= mu2 >= mu3 of B (lambda_n = m + mu_n), by the trigonometric
// solution of the characteristic cubic (Smith 1961), App. B ordering.
template <typename T> struct Eig3 {
    T m;
    T b[6];
    T mu[3];
};

template <typename T> __device__ __forceinline__ void eig3(const T a[6], Eig3<T>& e) {
    e.m = (a[0] + a[3] + a[5]) * T(1.0 / 3.0);
    e.b[0] = a[0] - e.m; e.b[1] = a[1]; e.b[2] = a[2];
    e.b[3] = a[3] - e.m; e.b[4] = a[4]; e.b[5] = a[5] - e.m;
    const T* b = e.b;
    const T off = b[1] * b[1] + b[2] * b[2] + b[4] * b[4];
    const T p2 = (b[0] * b[0] + b[3] * b[3] + b[5] * b[5] + T(2) * off) * T(1.0 / 6.0);
    if (!(p2 > T(0))) { e.mu[0] = e.mu[1] = e.mu[2] = T(0); return; }
    const T p = v_sqrt(p2);
    const T det = b[0] * (b[3] * b[5] - b[4] * b[4]) - b[1] * (b[1] * b[5] - b[4] * b[2]) +
                  b[2] * (b[1] * b[4] - b[3] * b[2]);
    T r = det / (T(2) * p2 * p);
    r = r < T(-1) ? T(-1) : (r > T(1) ? T(1) : r);
    const T phi = v_acos(r) * T(1.0 / 3.0);
    T s, c;
    v_sincos(phi, &s, &c);
    // cos(phi + 2pi/3) = -c/2 - (sqrt3/2) s
    const T mu1 = T(2) * p * c;
    const T mu3 = T(2) * p * (T(-0.5) * c - T(0.86602540378443864676) * s);
    T mu2 = -mu1 - mu3;
    mu2 = mu2 > mu1 ? mu1 : (mu2 < mu3 ? mu3 : mu2);
    e.mu[0] = mu1; e.mu[1] = mu2; e.mu[2] = mu3;
}

template <typename T> __device__ __forceinline__ T sigmoid(T x) { return T(1) / (T(1) + v_exp(-x)); }

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

// Bias table of one chain (precision T), Eq. local_bias + NB beta.
template <typename T> struct BiasT {
    T a[16], alpha[16], rho[16], eps[16], rhop[16], epsp[16], beta[16];
};

// Per-voxel interpolated parameters b_i = sum_r b^(r) p_i^(r) (Sect. 2.8).
template <typename T> struct VoxParams {
    T a, alpha, rho, eps, rhop, epsp, beta;
};

template <typename T, int NR>
__device__ __forceinline__ void interp_params(const BiasT<T>& B, const T w[NR], VoxParams<T>& q) {
    q.a = q.alpha = q.rho = q.eps = q.rhop = q.epsp = q.beta = T(0);
#pragma unroll
    for (int r = 0; r < NR; ++r) {
        q.a += B.a[r] * w[r];
        q.alpha += B.alpha[r] * w[r];
        q.rho += B.rho[r] * w[r];
        q.eps += B.eps[r] * w[r];
        q.rhop += B.rhop[r] * w[r];
        q.epsp += B.epsp[r] * w[r];
        q.beta += B.beta[r] * w[r];
    }
}

// ln f = ln a + alpha ln u - (u/rho)^eps - (rho'/u)^eps'  (Eq. local_bias in logs),
// u = max(1 + delta, floor).  Returns ln f; t1, t2 are the two cut-off terms.
template <typename T> struct LnF {
    T lnf, lnu, t1, t2, lnrho, lnrhop;
    bool floored;
};
template <typename T> __device__ __forceinline__ void log_f(T delta, T floor_, const VoxParams<T>& q, LnF<T>& r) {
    T u = T(1) + delta;
    r.floored = !(u > floor_);
    if (r.floored) u = floor_;
    r.lnu = v_log(u);
    r.lnrho = v_log(q.rho);
    r.t1 = v_exp(q.eps * (r.lnu - r.lnrho));
    if (q.rhop > T(0)) {
        r.lnrhop = v_log(q.rhop);
        r.t2 = v_exp(q.epsp * (r.lnrhop - r.lnu));
    } else {
        r.lnrhop = T(0);
        r.t2 = T(0);
    }
    r.lnf = v_log(q.a) + q.alpha * r.lnu - r.t1 - r.t2;
}

// Negative-binomial log pmf with shape beta and mean nbar (Sect. 2.6):
//   log P = sum_{m<n} ln((beta+m)/(m+1)) - beta ln(1 + nbar/beta) + n (ln nbar - ln(beta + nbar))
// and its derivatives d/d ln nbar and d/d beta.
template <typename T> struct NB {
    T logp, g_lnnbar, g_beta;
};
template <typename T> __device__ __forceinline__ void nb_eval(int n, T lnnbar, T beta, bool want_grad, NB<T>& r) {
    const T nbar = v_exp(lnnbar);
    const T l1 = v_log1p(nbar / beta);               // ln((beta + nbar)/beta)
    T s = T(0), ds = T(0);
    for (int m = 0; m < n; ++m) {
        s += v_log((beta + T(m)) / T(m + 1));
        if (want_grad) ds += T(1) / (beta + T(m));
    }
    const T tn = T(n);
    r.logp = s - beta * l1 + tn * (lnnbar - v_log(beta) - l1);
    if (want_grad) {
        const T den = nbar + beta;
        r.g_lnnbar = beta * (tn - nbar) / den;
        r.g_beta = ds - l1 + (nbar - tn) / den;
    }
}

// d lambda-sum / d A for symmetric A: G = sum_n g_n v_n v_n^T written with the
// invariant (projector) form of App. B: P_n = prod_{m != n} (B - mu_m)/(mu_n - mu_m),
//   G = g2 I + (g1 - g2) P_1 + (g3 - g2) P_3.
// Near-equal eigenvalues (gap < tau * scale) share the mean of their g's (a
// subgradient; the exact gradient is not defined at a crossing).  Output is the
// derivative with respect to the stored components (off-diagonals count twice).
template <typename T>
__device__ __forceinline__ void eig_adjoint(const Eig3<T>& e, T g1, T g2, T g3, T tau, T out[6]) {
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
    const T* b = e.b;
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
            const T s = c1 / ((mu1 - mu2) * (mu1 - mu3));
            const T lin = -(mu2 + mu3), cst = mu2 * mu3;
#pragma unroll
            for (int q = 0; q < 6; ++q) G[q] += s * (b2[q] + lin * b[q]);
            G[0] += s * cst; G[3] += s * cst; G[5] += s * cst;
        }
        if (c3 != T(0)) {
            const T s = c3 / ((mu3 - mu1) * (mu3 - mu2));
            const T lin = -(mu1 + mu2), cst = mu1 * mu2;
#pragma unroll
            for (int q = 0; q < 6; ++q) G[q] += s * (b2[q] + lin * b[q]);
            G[0] += s * cst; G[3] += s * cst; G[5] += s * cst;
        }
    }
    out[0] = G[0]; out[1] = T(2) * G[1]; out[2] = T(2) * G[2];
    out[3] = G[3]; out[4] = T(2) * G[4]; out[5] = G[5];
}

}  // namespace bridge
