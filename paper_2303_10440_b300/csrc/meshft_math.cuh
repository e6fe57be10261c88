// Per-(frequency, triangle) math of the mesh Fourier transform and its adjoint.
//
// f_T(xi) of Eq. 8 is the second divided difference of F(x) = -exp(-i x) at the
// vertex phases phi_p = v_p . xi, and the bracket of Eq. 10 is the third divided
// difference with node p repeated: df/dphi_p = DD3[F](phi_p, phi_p, phi_q, phi_r).
// Both are translation-covariant: shifting every node by t multiplies them by
// exp(-i t). So each term is evaluated in a local frame:
//
//   f = exp(-i phi_1) * rho * f_loc,   df/dphi_p = exp(-i phi_1) * rho * D_loc[p]
//
// where phi_1 (vertex 1's phase) comes from exact integer argument reduction in
// the caller, and f_loc, D_loc depend only on the two phase differences
// a = (v2 - v1).xi and b = (v3 - v1).xi.
//
// Generic case (node spread s = max - min >= TS): with the sorted nodes
// 0 = z0 <= z1 = d1 <= z2 = d1 + d2 = s (in the frame of the smallest node,
// rho = exp(-i x0)), u = exp(-i d), E(d) = (1 - u)/(i d), q(d) = (E(d) - 1)/d:
//   f_loc = i (u1 E2 - E1) / s
//   D0 = (f_loc - i q1) / s,  D1 = (i u1 q2 - E1 + i q1) / s,  D2 = (u1 E2 - i u1 q2 - f_loc) / s
// (D0 + D1 + D2 = -i f_loc, the translation identity). E and q switch to their
// Taylor series for |d| < TG, so the paper's divergent denominators (Section
// 4.1.3, Eq. 11-12) never appear and no epsilon is needed.
//
// Near-degenerate case (s < TS, all three phases close): the convergent series
// about the node mean c, DD_m[F] = sum_k F^(m+k)(c) h_k(z - c)/(m+k)! with h_k the
// complete homogeneous symmetric polynomials; rho = exp(-i c).
#pragma once

#include "dm_common.cuh"

namespace dm {

template <class R>
struct MathCfg;
template <>
struct MathCfg<float> {
    static constexpr float TS = 0.5f;   // spread threshold for the series branch (>= 2 TG: at most one small gap)
    static constexpr float TG = 0.25f;  // gap threshold for the Taylor forms of E, q
    static constexpr int K = 8;         // series terms (truncation < 1e-8 relative at s = TS)
    static constexpr int NPR = 3;       // Taylor coefficients of pr(t) (t = d^2; truncation < 1e-9 at d = TG)
    static constexpr int NPI = 4;       // Taylor coefficients of pi(t)
};
template <>
struct MathCfg<double> {
    static constexpr double TS = 0.5;
    static constexpr double TG = 0.5;
    static constexpr int K = 18;
    static constexpr int NPR = 9;
    static constexpr int NPI = 9;
};

// 1/n! for n = 0..24
__host__ __device__ constexpr double inv_fact(int n) {
    double r = 1.0;
    for (int k = 2; k <= n; ++k) r /= (double)k;
    return r;
}

__device__ __forceinline__ void sincos_r(float x, float* s, float* c) { __sincosf(x, s, c); }
__device__ __forceinline__ void sincos_r(double x, double* s, double* c) { sincos(x, s, c); }
__device__ __forceinline__ float rcp_r(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double rcp_r(double x) { return 1.0 / x; }
template <class R>
__device__ __forceinline__ R mn(R a, R b) {
    return a < b ? a : b;
}
template <class R>
__device__ __forceinline__ R mx(R a, R b) {
    return a < b ? b : a;
}

// Taylor series of E(d) = sum_k (-i d)^k/(k+1)! and q(d) = (E(d) - 1)/d, written as
//   Re E = 1 + d^2 pr(d^2),  Im E = d pi(d^2),  Re q = d pr(d^2),  Im q = pi(d^2)
// pr(t) = sum_{j>=1} (-1)^j t^(j-1)/(2j+1)!,  pi(t) = -sum_{j>=0} (-1)^j t^j/(2j+2)!.
template <class R>
__device__ __forceinline__ void taylor_pr_pi(R d, R& pr, R& pi) {
    using C = MathCfg<R>;
    const R t = d * d;
    pr = (R)0;
#pragma unroll
    for (int j = C::NPR; j >= 1; --j) pr = pr * t + (R)((j & 1 ? -1.0 : 1.0) * inv_fact(2 * j + 1));
    pi = (R)0;
#pragma unroll
    for (int j = C::NPI - 1; j >= 0; --j) pi = pi * t + (R)((j & 1 ? 1.0 : -1.0) * inv_fact(2 * j + 2));
}

template <class R, bool ADJ>
struct TriLocal {
    Cx<R> rho;   // local-frame rotation
    Cx<R> f;     // f_loc
    Cx<R> D[3];  // ADJ: D_loc, in sorted-node order (generic) or vertex order (series)
    int p1, plo, phi;  // ADJ: position in D of vertex 1, of min(a,b), of max(a,b)
    bool ab;           // ADJ: a <= b (vertex 2 holds min(a,b))
};

// Series branch: nodes (0, a, b) in vertex order, s < TS.
template <class R, bool ADJ>
__device__ __forceinline__ void tri_series(R a, R b, TriLocal<R, ADJ>& o) {
    using C = MathCfg<R>;
    const R c = (a + b) * (R)(1.0 / 3.0);
    const R y0 = -c, y1 = a - c, y2 = b - c;
    R h[C::K];
    h[0] = (R)1;
#pragma unroll
    for (int k = 1; k < C::K; ++k) h[k] = h[k - 1] * y0;
#pragma unroll
    for (int k = 1; k < C::K; ++k) h[k] += y1 * h[k - 1];
#pragma unroll
    for (int k = 1; k < C::K; ++k) h[k] += y2 * h[k - 1];
    // f_loc = sum_k (-i)^k h_k/(k+2)!
    R fr = 0, fi = 0;
#pragma unroll
    for (int k = 0; k < C::K; ++k) {
        const R t = h[k] * (R)inv_fact(k + 2);
        if ((k & 3) == 0) fr += t;
        if ((k & 3) == 1) fi -= t;
        if ((k & 3) == 2) fr -= t;
        if ((k & 3) == 3) fi += t;
    }
    R sn, cs;
    sincos_r(c, &sn, &cs);
    o.rho = {cs, -sn};
    o.f = {fr, fi};
    if (ADJ) {
        const R yp[3] = {y0, y1, y2};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            // D_p = -i sum_k (-i)^k H_k/(k+3)!, H_k = h_k(y0, y1, y2, y_p)
            R Hk = (R)1, sr = 0, si = 0;
#pragma unroll
            for (int k = 0; k < C::K; ++k) {
                if (k > 0) Hk = h[k] + yp[p] * Hk;
                const R t = Hk * (R)inv_fact(k + 3);
                if ((k & 3) == 0) sr += t;
                if ((k & 3) == 1) si -= t;
                if ((k & 3) == 2) sr -= t;
                if ((k & 3) == 3) si += t;
            }
            o.D[p] = {si, -sr};
        }
        o.p1 = 0;
        o.plo = 1;
        o.phi = 2;
        o.ab = true;
    }
}

template <class R, bool ADJ>
__device__ __forceinline__ void tri_local(R a, R b, TriLocal<R, ADJ>& o) {
    using C = MathCfg<R>;
    const R lo = mn(a, b), hi = mx(a, b);
    const bool vmin = (R)0 <= lo;  // vertex 1 holds the smallest phase
    const bool vmax = hi <= (R)0;  // vertex 1 holds the largest phase
    const R x0 = mn(lo, (R)0), x2 = mx(hi, (R)0);
    const R x1 = vmin ? lo : (vmax ? hi : (R)0);
    const R s = x2 - x0;
    if (s < (R)C::TS) {
        tri_series<R, ADJ>(a, b, o);
        return;
    }
    const R d1 = x1 - x0, d2 = x2 - x1;
    R sn1, cs1, sn2, cs2;
    sincos_r(d1, &sn1, &cs1);
    sincos_r(d2, &sn2, &cs2);
    const Cx<R> u1 = {cs1, -sn1};
    const bool sm1 = d1 < (R)C::TG, sm2 = d2 < (R)C::TG;
    const R d1c = sm1 ? (R)1 : d1, d2c = sm2 ? (R)1 : d2;
    const R r = rcp_r(d1c * d2c * s);
    const R inv1 = r * d2c * s, inv2 = r * d1c * s, invs = r * d1c * d2c;
    R pr1, pi1, pr2, pi2;
    taylor_pr_pi(d1, pr1, pi1);
    taylor_pr_pi(d2, pr2, pi2);
    Cx<R> E1, E2;
    E1.x = sm1 ? (R)1 + d1 * d1 * pr1 : sn1 * inv1;
    E1.y = sm1 ? d1 * pi1 : ((R)-1 + cs1) * inv1;
    E2.x = sm2 ? (R)1 + d2 * d2 * pr2 : sn2 * inv2;
    E2.y = sm2 ? d2 * pi2 : ((R)-1 + cs2) * inv2;
    const Cx<R> P = cmul(u1, E2);
    // f_loc = i (P - E1) / s
    o.f = {-(P.y - E1.y) * invs, (P.x - E1.x) * invs};
    // rho = exp(-i x0): 1 (vertex 1 smallest), conj(u1) (middle), conj(u1 u2) (largest)
    const Cx<R> u12 = cmul(u1, Cx<R>{cs2, -sn2});
    o.rho.x = vmin ? (R)1 : (vmax ? u12.x : u1.x);
    o.rho.y = vmin ? (R)0 : (vmax ? -u12.y : -u1.y);
    if (ADJ) {
        Cx<R> q1, q2;
        q1.x = sm1 ? d1 * pr1 : (E1.x - (R)1) * inv1;
        q1.y = sm1 ? pi1 : E1.y * inv1;
        q2.x = sm2 ? d2 * pr2 : (E2.x - (R)1) * inv2;
        q2.y = sm2 ? pi2 : E2.y * inv2;
        const Cx<R> iq1 = {-q1.y, q1.x};
        const Cx<R> uq = cmul(u1, q2);
        const Cx<R> Pq = {-uq.y, uq.x};  // i u1 q2
        o.D[0] = {(o.f.x - iq1.x) * invs, (o.f.y - iq1.y) * invs};
        o.D[1] = {(Pq.x - E1.x + iq1.x) * invs, (Pq.y - E1.y + iq1.y) * invs};
        o.D[2] = {(P.x - Pq.x - o.f.x) * invs, (P.y - Pq.y - o.f.y) * invs};
        o.p1 = vmin ? 0 : (vmax ? 2 : 1);
        o.plo = vmin ? 1 : 0;
        o.phi = vmax ? 1 : 2;
        o.ab = a <= b;
    }
}

template <class R>
__device__ __forceinline__ R sel3(int k, R t0, R t1, R t2) {
    return k == 0 ? t0 : (k == 1 ? t1 : t2);
}

}  // namespace dm
