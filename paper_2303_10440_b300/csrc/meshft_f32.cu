// FP32 mixed-precision mesh Fourier transform (Eq. 5, 7-8) and its adjoint (Eq. 6, 9-10).
//
// Both sums are bound by instruction issue, so each thread evaluates two
// (frequency, triangle) terms at once ("lanes" A and B) with paired FP32
// instructions (__ffma2_rn / __fadd2_rn / __fmul2_rn on float2 = (A, B)); MUFU
// ops, comparisons and selects stay per lane.
//
// Per term, in the frame of the triangle's middle vertex (the one whose phase lies
// between the other two): with the node gaps d1 = phi_m - phi_lo, d2 = phi_hi - phi_m,
// s = d1 + d2, E(d) = (1 - e^{-id})/(id), q(d) = (E(d) - 1)/d, r(d) = -i E(d) - q(d):
//   f_T          = e^{-i phi_m} i (E(d2) - conj E(d1)) / s                    (Eq. 8)
//   df/dphi_lo   = e^{-i phi_m} (f_m + i conj r(d1)) / s
//   df/dphi_mid  = e^{-i phi_m} i (q(d2) + conj q(d1)) / s                    (Eq. 10)
//   df/dphi_hi   = e^{-i phi_m} (i r(d2) - f_m) / s
// (f_m = i (E(d2) - conj E(d1)) / s). E and q switch to their Taylor series for
// gaps below TG; terms whose three phases lie within TS of each other replace f_m
// and the derivatives by their series in the same frame (series_f / series_adj),
// so every term shares the vertex mapping. phi_m = phi_1 + (phi_m - phi_1), where phi_1
// comes from exact integer reduction (n . U mod 2^32) and the offset from the
// FP32 edge projections.
//
// Forward: a thread holds two band frequencies in registers; the block walks a slice
// of the triangle list (slices sized so that the launch has ~112 units per SM) in
// tiles bulk-copied (TMA) into a ring of shared-memory stages with full/empty
// mbarriers. FP32 sums within a tile, Kahan across tiles; slices are summed
// afterwards in a fixed order (compensated FP32).
// Adjoint: a thread holds one triangle; the block walks a chunk of the band in
// tiles of frequency-pair records bulk-copied the same way, summing the triangle's
// 10 (surface) or 12 (volume) terms of a tile in registers and carrying the running
// sums in shared memory; chunks are summed afterwards in FP64 in a fixed order
// (deterministic).
#include "dm_kernels.cuh"
#include "meshft_math.cuh"

namespace dm {

namespace {

constexpr float kTwoPiOver2p32 = 1.4629180792671596e-09f;  // 2 pi / 2^32
constexpr float TS = MathCfg<float>::TS;
constexpr float TG = MathCfg<float>::TG;

constexpr int kFwdStages = 4, kFwdTile = 64;  // forward: 4 stages x 64 triangle records (24 KB)
constexpr int kAdjStages = 4;                 // adjoint: 4 stages x 128 frequency pairs (32 KB)
static_assert(FWD_TILE % kFwdTile == 0, "triangle padding must cover whole forward tiles");

typedef float2 F2;
__device__ __forceinline__ F2 mk(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ F2 mul2(F2 a, F2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ F2 fma2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ F2 sub2(F2 a, F2 b) { return __ffma2_rn(b, mk(-1.f, -1.f), a); }  // a - b
__device__ __forceinline__ F2 fms2(F2 a, F2 b, F2 c) { return __ffma2_rn(a, b, mk(-c.x, -c.y)); }  // a*b - c
__device__ __forceinline__ F2 sel2(bool ca, bool cb, F2 t, F2 f) { return mk(ca ? t.x : f.x, cb ? t.y : f.y); }

// Taylor polynomials pr(t), pi(t) of meshft_math.cuh (t = d^2) for a pair of gaps.
__device__ __forceinline__ void taylor2(F2 t, F2& pr, F2& pi) {
    const F2 nt = mk(-t.x, -t.y);
    pr = fma2(mk((float)inv_fact(7), (float)inv_fact(7)), nt, mk((float)inv_fact(5), (float)inv_fact(5)));
    pr = fma2(pr, t, mk(-(float)inv_fact(3), -(float)inv_fact(3)));
    pi = fma2(mk((float)inv_fact(8), (float)inv_fact(8)), nt, mk((float)inv_fact(6), (float)inv_fact(6)));
    pi = fma2(pi, nt, mk((float)inv_fact(4), (float)inv_fact(4)));
    pi = fma2(pi, nt, mk((float)inv_fact(2), (float)inv_fact(2)));
    pi = mk(-pi.x, -pi.y);
}
static_assert(MathCfg<float>::NPR == 3 && MathCfg<float>::NPI == 4, "taylor2 is written for these orders");

__device__ __forceinline__ void kahan_add(float& s, float& c, float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Node ordering of (0, a, b) for one lane: lo, mid, hi and the vertex-identity flags.
struct Order {
    float lo, mid, hi;
    bool lo1, hi1, ab;  // vertex 1 is lowest / highest; a <= b
};
__device__ __forceinline__ Order order3(float a, float b) {
    Order o;
    const float mn = fminf(a, b), mx = fmaxf(a, b);
    o.lo = fminf(mn, 0.f);
    o.hi = fmaxf(mx, 0.f);
    o.mid = fmaxf(mn, fminf(mx, 0.f));
    o.lo1 = 0.f <= mn;
    o.hi1 = mx <= 0.f;
    o.ab = a <= b;
    return o;
}

// Reciprocal by the PTX approximate instruction (one MUFU op; arguments here are >= TG or >= TS,
// never subnormal). __fdividef(1, x) adds range handling that measurably costs issue slots.
__device__ __forceinline__ float rcpa(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

// Adjoint gap functions for both lanes of both gaps: E(d1), E(d2), q(d1), q(d2) and 1/s.
// Since s = d1 + d2 >= TS >= 2 TG here, at most one gap per lane is below TG, so a single
// Taylor evaluation on min(d1, d2) serves whichever gap needs it.
static_assert(MathCfg<float>::TS >= 2.0f * MathCfg<float>::TG, "one Taylor evaluation per term needs TS >= 2 TG");
struct Gaps {
    F2 E1x, E1y, E2x, E2y;
    F2 q1x, q1y, q2x, q2y;
    F2 invs;
};
__device__ __forceinline__ void gaps2(F2 d1, F2 d2, F2 s, Gaps& g) {
    float s1a, c1a, s1b, c1b, s2a, c2a, s2b, c2b;
    __sincosf(d1.x, &s1a, &c1a);
    __sincosf(d1.y, &s1b, &c1b);
    __sincosf(d2.x, &s2a, &c2a);
    __sincosf(d2.y, &s2b, &c2b);
    const bool m1a = d1.x < TG, m1b = d1.y < TG, m2a = d2.x < TG, m2b = d2.y < TG;
    // reciprocals on the MUFU pipe (the FP32 pipe is the busier one); 1/d is only used for
    // d >= TG, so the inf / NaN of a zero gap never leaves the unselected lane value
    const F2 inv1 = mk(rcpa(d1.x), rcpa(d1.y));
    const F2 inv2 = mk(rcpa(d2.x), rcpa(d2.y));
    g.invs = mk(rcpa(s.x), rcpa(s.y));  // inf when s = 0; such lanes take the series below
    const F2 dm = mk(fminf(d1.x, d2.x), fminf(d1.y, d2.y));
    const F2 tm = mul2(dm, dm);
    F2 pr, pi;
    taylor2(tm, pr, pi);
    const F2 mone = mk(-1.f, -1.f);
    // Taylor: Re E = 1 + d^2 pr, Im E = d pi ; direct: E = sin d / d - i (1 - cos d) / d
    const F2 Etx = fma2(tm, pr, mk(1.f, 1.f)), Ety = mul2(dm, pi);
    const F2 E1xd = mul2(mk(s1a, s1b), inv1), E1yd = mul2(add2(mk(c1a, c1b), mone), inv1);
    const F2 E2xd = mul2(mk(s2a, s2b), inv2), E2yd = mul2(add2(mk(c2a, c2b), mone), inv2);
    g.E1x = sel2(m1a, m1b, Etx, E1xd);
    g.E1y = sel2(m1a, m1b, Ety, E1yd);
    g.E2x = sel2(m2a, m2b, Etx, E2xd);
    g.E2y = sel2(m2a, m2b, Ety, E2yd);
    {
        // Taylor: Re q = d pr, Im q = pi ; direct: q = (E - 1)/d
        const F2 qtx = mul2(dm, pr);
        g.q1x = sel2(m1a, m1b, qtx, mul2(add2(E1xd, mone), inv1));
        g.q1y = sel2(m1a, m1b, pi, mul2(E1yd, inv1));
        g.q2x = sel2(m2a, m2b, qtx, mul2(add2(E2xd, mone), inv2));
        g.q2y = sel2(m2a, m2b, pi, mul2(E2yd, inv2));
    }
}

// Forward middle-frame value f_m = i (E(d2) - conj E(d1)) / s (both lanes) over one common
// denominator. With N = d E = (sin d, cos d - 1) and c = d for a gap >= TG, and N = E (Taylor),
// c = 1 for the (at most one) gap below TG: E(d2) - conj E(d1) = (c1 N2 - c2 conj N1) / (c1 c2), so
// f_m = i (c1 N2 - c2 conj N1) / (c1 c2 s) takes one reciprocal per lane instead of three. The
// denominator is >= TG^2 TS where the lane keeps this value (s >= TS); lanes with s < TS are
// replaced by the series. Returns f_m = -fmr + i fmi.
__device__ __forceinline__ void fm_closed(F2 d1, F2 d2, F2 s, F2& fmr, F2& fmi) {
    float s1a, c1a, s1b, c1b, s2a, c2a, s2b, c2b;
    __sincosf(d1.x, &s1a, &c1a);
    __sincosf(d1.y, &s1b, &c1b);
    __sincosf(d2.x, &s2a, &c2a);
    __sincosf(d2.y, &s2b, &c2b);
    const bool m1a = d1.x < TG, m1b = d1.y < TG, m2a = d2.x < TG, m2b = d2.y < TG;
    const F2 dm = mk(fminf(d1.x, d2.x), fminf(d1.y, d2.y));
    const F2 tm = mul2(dm, dm);
    F2 pr, pi;
    taylor2(tm, pr, pi);
    const F2 one = mk(1.f, 1.f), mone = mk(-1.f, -1.f);
    const F2 Etx = fma2(tm, pr, one), Ety = mul2(dm, pi);
    const F2 c1 = sel2(m1a, m1b, one, d1), c2 = sel2(m2a, m2b, one, d2);
    const F2 N1x = sel2(m1a, m1b, Etx, mk(s1a, s1b)), N1y = sel2(m1a, m1b, Ety, add2(mk(c1a, c1b), mone));
    const F2 N2x = sel2(m2a, m2b, Etx, mk(s2a, s2b)), N2y = sel2(m2a, m2b, Ety, add2(mk(c2a, c2b), mone));
    const F2 den = mul2(mul2(c1, c2), s);
    const F2 R = mk(rcpa(den.x), rcpa(den.y));
    // c1 N2 - c2 conj N1 = (c1 N2x - c2 N1x) + i (c1 N2y + c2 N1y); times i R
    const F2 nx = fms2(c1, N2x, mul2(c2, N1x)), ny = fma2(c1, N2y, mul2(c2, N1y));
    fmr = mul2(ny, R);
    fmi = mul2(nx, R);
}

// Middle-frame series for terms whose three phases lie within TS (s < TS). With the nodes
// (-d1, 0, d2) relative to the middle phase and F(x) = -e^{-ix}, the divided differences are
// sums over the complete homogeneous symmetric polynomials h_k of the nonzero nodes:
//   f_m  = DD2[F](-d1, 0, d2)      = sum_k (-i)^k h_k(-d1, d2) / (k+2)!
//   D_mid = DD3[F](-d1, 0, 0, d2)  = sum_k (-i)^(k+1) h_k(-d1, d2) / (k+3)!
//   D_lo  = DD3[F](-d1, -d1, 0, d2) = sum_k (-i)^(k+1) h_k(-d1, -d1, d2) / (k+3)!
//   D_hi  = -(i f_m + D_lo + D_mid)     (the three phase derivatives sum to -i f_m)
// h_k(-d1, d2) = (d2 - d1) h_{k-1} + d1 d2 h_{k-2}; h_k(-d1, -d1, d2) = e1 h_{k-1} - e2 h_{k-2}
// + e3 h_{k-3} with e1 = d2 - 2 d1, e2 = d1^2 - 2 d1 d2, e3 = d1^2 d2. With s < 0.5 the terms fall
// below 1e-7 of the sum by k = 7, so KS = 8 terms serve FP32. Both lanes at once.
constexpr int KS = 8;

// (-i)^j = sign * (1 or i): real for even j; sign + for j mod 4 in {0, 3}.
__host__ __device__ constexpr float isign(int j) { return (j % 4 == 0 || j % 4 == 3) ? 1.f : -1.f; }

__device__ __forceinline__ void series_f(F2 d1, F2 d2, F2& fr, F2& fi) {
    const F2 del = sub2(d2, d1), pr = mul2(d1, d2);
    F2 hm2 = mk(1.f, 1.f), hm1 = del;
    fr = mk((float)inv_fact(2), (float)inv_fact(2));
    fi = mul2(del, mk(-(float)inv_fact(3), -(float)inv_fact(3)));
#pragma unroll
    for (int k = 2; k < KS; ++k) {
        const F2 h = fma2(del, hm1, mul2(pr, hm2));
        const float c = isign(k) * (float)inv_fact(k + 2);
        if (k % 2 == 0)
            fr = fma2(h, mk(c, c), fr);
        else
            fi = fma2(h, mk(c, c), fi);
        hm2 = hm1;
        hm1 = h;
    }
}

__device__ __forceinline__ void series_adj(F2 d1, F2 d2, F2& fr, F2& fi, F2& lr, F2& li, F2& mr, F2& mi) {
    const F2 del = sub2(d2, d1), pr = mul2(d1, d2);
    const F2 d1s = mul2(d1, d1);
    const F2 e1 = sub2(del, d1);                        // d2 - 2 d1
    const F2 e2 = fma2(pr, mk(-2.f, -2.f), d1s);        // d1^2 - 2 d1 d2
    const F2 e3 = mul2(d1s, d2);                        // d1^2 d2
    // k = 0, 1
    fr = mk((float)inv_fact(2), (float)inv_fact(2));
    fi = mul2(del, mk(-(float)inv_fact(3), -(float)inv_fact(3)));
    mi = mk(-(float)inv_fact(3), -(float)inv_fact(3));  // j = 1: -i h_0 / 3!
    mr = mul2(del, mk(-(float)inv_fact(4), -(float)inv_fact(4)));  // j = 2: -h_1 / 4!
    li = mi;
    lr = mul2(e1, mk(-(float)inv_fact(4), -(float)inv_fact(4)));
    F2 hm2 = mk(1.f, 1.f), hm1 = del;               // h(-d1, d2)
    F2 gm3 = mk(0.f, 0.f), gm2 = mk(1.f, 1.f), gm1 = e1;  // h(-d1, -d1, d2)
#pragma unroll
    for (int k = 2; k < KS; ++k) {
        const F2 h = fma2(del, hm1, mul2(pr, hm2));
        const F2 g = fma2(e3, gm3, fms2(e1, gm1, mul2(e2, gm2)));
        const float cf = isign(k) * (float)inv_fact(k + 2);
        const float cd = isign(k + 1) * (float)inv_fact(k + 3);
        if (k % 2 == 0) {
            fr = fma2(h, mk(cf, cf), fr);
            mi = fma2(h, mk(cd, cd), mi);
            li = fma2(g, mk(cd, cd), li);
        } else {
            fi = fma2(h, mk(cf, cf), fi);
            mr = fma2(h, mk(cd, cd), mr);
            lr = fma2(g, mk(cd, cd), lr);
        }
        hm2 = hm1;
        hm1 = h;
        gm3 = gm2;
        gm2 = gm1;
        gm1 = g;
    }
}

// ------------------------------------------------------------------------------------- forward
// One forward block: band frequencies [bidx * 512, bidx * 512 + 512) against n_tiles tiles of
// triangle records, of which the last holds `last` real triangles (the rest is padding, skipped).
// Returns false (without touching the barriers) when the block lies beyond the band.
template <int MODE, bool EXPLICIT>
__device__ __forceinline__ bool fwd_block(const TriF32* __restrict__ tris, int n_tiles, int last, const FreqSrc& fs,
                                          float tpx,
                                          float tpy, float tpz, const double* __restrict__ d_vol,
                                          float2* __restrict__ S, int* __restrict__ err, int64_t bidx,
                                          TriF32 (*stage)[kFwdTile], uint64_t* full, uint64_t* empty,
                                          bool vol_term = true) {
    constexpr int PER_BLOCK = 2 * FWD_THREADS;
    const int tid = threadIdx.x;
    const int64_t M = fs.dM ? *fs.dM : fs.M;
    if (bidx * PER_BLOCK >= M) return false;  // whole block beyond the band (uniform)
    const int64_t m0 = bidx * PER_BLOCK + 2 * tid;
    const bool actA = m0 < M, actB = m0 + 1 < M;

    int n[2][3] = {{0, 0, 0}, {0, 0, 0}};
#pragma unroll
    for (int l = 0; l < 2; ++l) {
        const int64_t m = m0 + l;
        if (m < M) {
            if (EXPLICIT) {
                n[l][0] = fs.nlist[3 * m];
                n[l][1] = fs.nlist[3 * m + 1];
                n[l][2] = fs.nlist[3 * m + 2];
            } else {
                const int64_t idx = fs.idx ? (int64_t)fs.idx[m] : m;
                decode_h(idx, fs, n[l][0], n[l][1], n[l][2]);
            }
        }
    }
    const F2 X = mk((float)n[0][0] * tpx, (float)n[1][0] * tpx);
    const F2 Y = mk((float)n[0][1] * tpy, (float)n[1][1] * tpy);
    const F2 Z = mk((float)n[0][2] * tpz, (float)n[1][2] * tpz);
    const uint32_t uA0 = (uint32_t)n[0][0], uA1 = (uint32_t)n[0][1], uA2 = (uint32_t)n[0][2];
    const uint32_t uB0 = (uint32_t)n[1][0], uB1 = (uint32_t)n[1][1], uB2 = (uint32_t)n[1][2];

    F2 SX = mk(0.f, 0.f), SY = mk(0.f, 0.f), CX = mk(0.f, 0.f), CY = mk(0.f, 0.f);
    int tile_no = 0;  // tiles arrive in order
    const auto consume = [&](const TriF32* tile) {
        const int cnt = ++tile_no == n_tiles ? last : kFwdTile;
        F2 PX = mk(0.f, 0.f), PY = mk(0.f, 0.f);
        #pragma unroll 1
        for (int j = 0; j < cnt; ++j) {
            const TriF32& T = tile[j];
            const uint32_t PA = uA0 * T.U[0] + uA1 * T.U[1] + uA2 * T.U[2];
            const uint32_t PB = uB0 * T.U[0] + uB1 * T.U[1] + uB2 * T.U[2];
            const F2 ph = mul2(mk((float)(int32_t)PA, (float)(int32_t)PB), mk(kTwoPiOver2p32, kTwoPiOver2p32));
            const F2 a = fma2(Z, T.e21z, fma2(Y, T.e21y, mul2(X, T.e21x)));
            const F2 b = fma2(Z, T.e31z, fma2(Y, T.e31y, mul2(X, T.e31x)));
            const F2 w = MODE == 0 ? T.w0 : fma2(Z, T.w2, fma2(Y, T.w1, mul2(X, T.w0)));
            const Order oA = order3(a.x, b.x), oB = order3(a.y, b.y);
            const F2 lo = mk(oA.lo, oB.lo), hi = mk(oA.hi, oB.hi), mid = mk(oA.mid, oB.mid);
            const F2 s = sub2(hi, lo);
            const F2 d1 = sub2(mid, lo), d2 = sub2(hi, mid);
            const F2 phm = add2(ph, mid);
            F2 fmr, fmi;
            fm_closed(d1, d2, s, fmr, fmi);
            float sma, cma, smb, cmb;
            __sincosf(phm.x, &sma, &cma);
            __sincosf(phm.y, &smb, &cmb);
            const F2 sm = mk(sma, smb), cm = mk(cma, cmb);
            if (s.x < TS || s.y < TS) {
                // three phases within TS: the series in the same frame (warp-divergent, rare)
                F2 sr, si;
                series_f(d1, d2, sr, si);
                const bool ta = s.x < TS, tb = s.y < TS;
                fmr = sel2(ta, tb, mk(-sr.x, -sr.y), fmr);
                fmi = sel2(ta, tb, si, fmi);
            }
            // f = e^{-i phi_m} f_m = (cm - i sm)(-fmr + i fmi)
            const F2 fx = fms2(sm, fmi, mul2(cm, fmr));
            const F2 fy = fma2(cm, fmi, mul2(sm, fmr));
            PX = fma2(w, fx, PX);
            PY = fma2(w, fy, PY);
        }
        kahan_add(SX.x, CX.x, PX.x);
        kahan_add(SX.y, CX.y, PX.y);
        kahan_add(SY.x, CY.x, PY.x);
        kahan_add(SY.y, CY.y, PY.y);
    };
    run_tile_pipeline<kFwdStages, kFwdTile>(tris, n_tiles, stage, full, empty, err, consume);
    float sx[2] = {SX.x, SX.y}, sy[2] = {SY.x, SY.y};
    if (MODE == 1) {
        // volume: S = (i / |xi|^2) sum_T (xi . n_T) f_T, and the enclosed volume at xi = 0
        const float xs[2] = {X.x, X.y}, ys[2] = {Y.x, Y.y}, zs[2] = {Z.x, Z.y};
#pragma unroll
        for (int l = 0; l < 2; ++l) {
            if (n[l][0] == 0 && n[l][1] == 0 && n[l][2] == 0) {
                sx[l] = vol_term ? (float)*d_vol : 0.f;  // added once when the triangles are split
                sy[l] = 0.f;
            } else {
                const float ik2 = 1.0f / (xs[l] * xs[l] + ys[l] * ys[l] + zs[l] * zs[l]);
                const float tx = -sy[l] * ik2, ty = sx[l] * ik2;
                sx[l] = tx;
                sy[l] = ty;
            }
        }
    }
    if (actA && actB && (reinterpret_cast<uintptr_t>(S + m0) & 15) == 0) {
        *reinterpret_cast<float4*>(S + m0) = make_float4(sx[0], sy[0], sx[1], sy[1]);
    } else {
        if (actA) S[m0] = make_float2(sx[0], sy[0]);
        if (actB) S[m0 + 1] = make_float2(sx[1], sy[1]);
    }
    return true;
}

// Work units of the forward: (frequency block, triangle split). A small band splits the triangle list so
// that enough blocks run; the split count follows from the band size on the device (dM), identically
// in the sums and in the reduction below.
__device__ __forceinline__ void fwd_units(const FreqSrc& fs, int n_tiles, int target, int64_t& M, int64_t& fb,
                                          int& splits) {
    M = fs.dM ? *fs.dM : fs.M;
    fb = (M + FWD_BLOCK_FREQS - 1) / FWD_BLOCK_FREQS;
    splits = fwd_splits(fb, (n_tiles + 3) / 4, target);  // at least ~4 triangle tiles per split
}

template <int MODE, bool EXPLICIT>
__global__ void __launch_bounds__(FWD_THREADS, 4) k_fwd_f32(const TriF32* __restrict__ tris, int n_tiles, int last,
                                                         FreqSrc fs,
                                                         float tpx, float tpy, float tpz,
                                                         const double* __restrict__ d_vol, float2* __restrict__ S,
                                                         float2* __restrict__ S_part, int target,
                                                         int* __restrict__ err) {
    __shared__ __align__(128) TriF32 stage[kFwdStages][kFwdTile];
    __shared__ __align__(8) uint64_t full[kFwdStages], empty[kFwdStages];
    int64_t M, fb;
    int splits;
    fwd_units(fs, n_tiles, S_part ? target : 0, M, fb, splits);
    const int64_t u = blockIdx.x;
    if (u >= fb * splits) return;  // uniform per block
    const int64_t b = u / splits;
    const int ts = (int)(u - b * splits);
    const int t0 = (int)((int64_t)n_tiles * ts / splits), t1 = (int)((int64_t)n_tiles * (ts + 1) / splits);
    float2* out = splits == 1 ? S : S_part + (int64_t)ts * M;
    fwd_block<MODE, EXPLICIT>(tris + (int64_t)t0 * kFwdTile, t1 - t0, t1 == n_tiles ? last : kFwdTile, fs, tpx, tpy,
                              tpz, d_vol, out, err, b, stage, full, empty, ts == 0);
}

// S[m] = sum over the triangle splits of the partial spectra (fixed order, compensated); nothing when
// unsplit.
// fixed_splits > 0: that many splits (a served job's own count) instead of the band-derived one.
__global__ void __launch_bounds__(256) k_fwd_reduce(FreqSrc fs, int n_tiles, int target, int fixed_splits,
                                                    const float2* __restrict__ S_part, float2* __restrict__ S) {
    int64_t M, fb;
    int splits;
    fwd_units(fs, n_tiles, target, M, fb, splits);
    if (fixed_splits > 0) splits = fixed_splits;
    if (splits == 1) return;
    for (int64_t m = (int64_t)blockIdx.x * 256 + threadIdx.x; m < M; m += (int64_t)gridDim.x * 256) {
        // compensated FP32 sums (B300's FP64 adds are slow); the result is rounded to FP32 anyway
        float sx = 0.f, cx = 0.f, sy = 0.f, cy = 0.f;
        for (int ts = 0; ts < splits; ++ts) {
            const float2 v = S_part[(int64_t)ts * M + m];
            kahan_add(sx, cx, v.x);
            kahan_add(sy, cy, v.y);
        }
        S[m] = make_float2(sx, sy);
    }
}

// ------------------------------------------------------------------------------------- adjoint
constexpr int kAdjPairs = ADJ_FTILE / 2;

// One adjoint block: triangles [tblock * 128, tblock * 128 + 128) against frequency tiles [f0, f1);
// writes the block's sums to out[k * n_t_pad + t] (k < 10 or 12). Returns whether the barriers were used.
template <int MODE>
__device__ __forceinline__ bool adj_block(const TriF32* __restrict__ tris, int64_t n_t, int64_t n_t_pad,
                                          const FreqPairF32* __restrict__ fr, int f0, int f1, int64_t tblock,
                                          float* __restrict__ out_chunk, int* __restrict__ err,
                                          FreqPairF32 (*stage)[kAdjPairs], uint64_t* full, uint64_t* empty,
                                          float* acc_s) {
    constexpr int NACC = MODE == 0 ? NACC_SURF : NACC_VOL;
    constexpr int PAIRS = kAdjPairs;
    const int tid = threadIdx.x;
    const int64_t t = tblock * ADJ_THREADS + tid;

    // A padding lane evaluates the block's first triangle (its sums are dropped), so a part-padded
    // warp branches like its real lanes; a warp of padding only skips the tiles.
    const TriF32 T = tris[t < n_t ? t : tblock * ADJ_THREADS];
    const bool idle = tblock * ADJ_THREADS + (tid & ~31) >= n_t;
    // edge vectors held once per thread (the record stores each field twice for paired loads from
    // shared memory; in registers the pairs are rebuilt at each use, which needs fewer registers)
    const float e21[3] = {T.e21x.x, T.e21y.x, T.e21z.x}, e31[3] = {T.e31x.x, T.e31y.x, T.e31z.x};
    // the triangle's running sums and their compensations live in shared memory (each thread its
    // own column), touched once per tile, leaving the registers to the frequency loop
    float* tot = acc_s + tid;
    float* comp = acc_s + NACC * ADJ_THREADS + tid;
#pragma unroll
    for (int k = 0; k < NACC; ++k) tot[k * ADJ_THREADS] = comp[k * ADJ_THREADS] = 0.f;

    if (f1 > f0) {
        const auto consume = [&](const FreqPairF32* tile) {
            if (idle) return;
            F2 part[NACC];
            #pragma unroll
            for (int k = 0; k < NACC; ++k) part[k] = mk(0.f, 0.f);
            #pragma unroll 2
            for (int j = 0; j < PAIRS; ++j) {
            const FreqPairF32& R = tile[j];
            const uint32_t PA = (uint32_t)R.nA[0] * T.U[0] + (uint32_t)R.nA[1] * T.U[1] + (uint32_t)R.nA[2] * T.U[2];
            const uint32_t PB = (uint32_t)R.nB[0] * T.U[0] + (uint32_t)R.nB[1] * T.U[1] + (uint32_t)R.nB[2] * T.U[2];
            const F2 ph = mul2(mk((float)(int32_t)PA, (float)(int32_t)PB), mk(kTwoPiOver2p32, kTwoPiOver2p32));
            const F2 X = R.x, Y = R.y, Z = R.z;
            const F2 a = fma2(Z, mk(e21[2], e21[2]), fma2(Y, mk(e21[1], e21[1]), mul2(X, mk(e21[0], e21[0]))));
            const F2 b = fma2(Z, mk(e31[2], e31[2]), fma2(Y, mk(e31[1], e31[1]), mul2(X, mk(e31[0], e31[0]))));
            const Order oA = order3(a.x, b.x), oB = order3(a.y, b.y);
            const F2 lo = mk(oA.lo, oB.lo), hi = mk(oA.hi, oB.hi), mid = mk(oA.mid, oB.mid);
            const F2 s = sub2(hi, lo);
            F2 rf, tv1, tv2, tv3;
            {
                const F2 d1 = sub2(mid, lo), d2 = sub2(hi, mid);
                const F2 phm = add2(ph, mid);
                Gaps g;
                gaps2(d1, d2, s, g);
                float sma, cma, smb, cmb;
                __sincosf(phm.x, &sma, &cma);
                __sincosf(phm.y, &smb, &cmb);
                const F2 sm = mk(sma, smb), cm = mk(cma, cmb);
                // w = conj(Gw) e^{-i phi_m} = h - i k (h = Gr cm - Gi sm, k = Gr sm + Gi cm) and
                // Re(w z) = h z.x + k z.y. With s f_m = i (E2 - conj E1) = (-gy, gx) and r = -i E - q,
                // the unscaled derivatives s D_lo = f_m + i conj r1, s D_mid = i (q2 + conj q1),
                // s D_hi = i r2 - f_m contract to
                //   Re(w i conj r1) = k (E1y - q1x) - h (E1x + q1y)
                //   Re(w i (q2 + conj q1)) = h (q1y - q2y) + k (q1x + q2x)
                //   Re(w i r2) = h (E2x + q2y) + k (E2y - q2x)
                const F2 h = fms2(R.Gr, cm, mul2(R.Gi, sm));
                const F2 k = fma2(R.Gr, sm, mul2(R.Gi, cm));
                const F2 gx = sub2(g.E2x, g.E1x), gy = add2(g.E2y, g.E1y);
                rf = mul2(fms2(k, gx, mul2(h, gy)), g.invs);  // Re(w f_m)
                const F2 c1 = fms2(k, sub2(g.E1y, g.q1x), mul2(h, add2(g.E1x, g.q1y)));
                const F2 cm_ = fma2(h, sub2(g.q1y, g.q2y), mul2(k, add2(g.q1x, g.q2x)));
                const F2 c2 = fma2(h, add2(g.E2x, g.q2y), mul2(k, sub2(g.E2y, g.q2x)));
                F2 tlo = mul2(add2(rf, c1), g.invs);
                F2 tmd = mul2(cm_, g.invs);
                F2 thi = mul2(sub2(c2, rf), g.invs);
                if (s.x < TS || s.y < TS) {
                    // three phases within TS: the series in the same frame gives f_m and the true
                    // derivatives, contracted here for those lanes (warp-divergent, rare)
                    F2 fr, fi, lr, li, mr, mi;
                    series_adj(d1, d2, fr, fi, lr, li, mr, mi);
                    const F2 hr = sub2(sub2(fi, lr), mr);                      // D_hi = -(i f_m + D_lo + D_mid)
                    const F2 hi_ = mk(-fr.x - li.x - mi.x, -fr.y - li.y - mi.y);
                    const bool ta = s.x < TS, tb = s.y < TS;
                    rf = sel2(ta, tb, fma2(h, fr, mul2(k, fi)), rf);
                    tlo = sel2(ta, tb, fma2(h, lr, mul2(k, li)), tlo);
                    tmd = sel2(ta, tb, fma2(h, mr, mul2(k, mi)), tmd);
                    thi = sel2(ta, tb, fma2(h, hr, mul2(k, hi_)), thi);
                }
                // vertex 1 = 0, vertex 2 = a, vertex 3 = b
                const F2 tmn = sel2(oA.lo1, oB.lo1, tmd, tlo), tmx = sel2(oA.hi1, oB.hi1, tmd, thi);
                tv1 = sel2(oA.lo1, oB.lo1, tlo, sel2(oA.hi1, oB.hi1, thi, tmd));
                tv2 = sel2(oA.ab, oB.ab, tmn, tmx);
                tv3 = sel2(oA.ab, oB.ab, tmx, tmn);
            }
            constexpr int B = MODE == 0 ? 1 : 3;
            if (MODE == 0) {
                part[0] = add2(part[0], rf);
            } else {
                const F2 wn = fma2(Z, T.w2, fma2(Y, T.w1, mul2(X, T.w0)));  // xi . n_T
                part[0] = fma2(rf, X, part[0]);
                part[1] = fma2(rf, Y, part[1]);
                part[2] = fma2(rf, Z, part[2]);
                tv1 = mul2(tv1, wn);
                tv2 = mul2(tv2, wn);
                tv3 = mul2(tv3, wn);
            }
            part[B + 0] = fma2(tv1, X, part[B + 0]);
            part[B + 1] = fma2(tv1, Y, part[B + 1]);
            part[B + 2] = fma2(tv1, Z, part[B + 2]);
            part[B + 3] = fma2(tv2, X, part[B + 3]);
            part[B + 4] = fma2(tv2, Y, part[B + 4]);
            part[B + 5] = fma2(tv2, Z, part[B + 5]);
            part[B + 6] = fma2(tv3, X, part[B + 6]);
            part[B + 7] = fma2(tv3, Y, part[B + 7]);
            part[B + 8] = fma2(tv3, Z, part[B + 8]);
            }
            #pragma unroll
            for (int k = 0; k < NACC; ++k) {
                float sk = tot[k * ADJ_THREADS], ck = comp[k * ADJ_THREADS];
                kahan_add(sk, ck, part[k].x + part[k].y);
                tot[k * ADJ_THREADS] = sk;
                comp[k * ADJ_THREADS] = ck;
            }
        };
        run_tile_pipeline<kAdjStages, kAdjPairs>(fr + (int64_t)f0 * PAIRS, f1 - f0, stage, full, empty, err, consume);
    }
    if (t < n_t_pad) {
        float* out = out_chunk + t;
#pragma unroll
        for (int k = 0; k < NACC; ++k) out[(int64_t)k * n_t_pad] = t < n_t ? tot[k * ADJ_THREADS] : 0.f;
    }
    return f1 > f0;
}

template <int MODE>
__global__ void __launch_bounds__(ADJ_THREADS, MODE == 0 ? 5 : 4) k_adj_f32(const TriF32* __restrict__ tris, int64_t n_t,
                                                         int64_t n_t_pad, const FreqPairF32* __restrict__ fr,
                                                         const int64_t* __restrict__ dM, int64_t M_max,
                                                         float* __restrict__ partial, int* __restrict__ err) {
    constexpr int NACC = MODE == 0 ? NACC_SURF : NACC_VOL;
    __shared__ __align__(128) FreqPairF32 stage[kAdjStages][kAdjPairs];
    __shared__ __align__(8) uint64_t full[kAdjStages], empty[kAdjStages];
    const int64_t M = dM ? *dM : M_max;
    const int n_ftiles = (int)((M + ADJ_FTILE - 1) / ADJ_FTILE);
    // the chunks share the band's tiles as it is on the device (a narrow band still uses every chunk)
    const int tpc = (n_ftiles + (int)gridDim.y - 1) / (int)gridDim.y;
    const int f0 = blockIdx.y * tpc;
    const int f1 = min(f0 + tpc, n_ftiles);
    __shared__ float acc_s[2 * NACC * ADJ_THREADS];
    // a chunk past the band's last tile writes zeros, which the chunk reduction leaves out
    adj_block<MODE>(tris, n_t, n_t_pad, fr, f0, f1, blockIdx.x, partial + (int64_t)blockIdx.y * NACC * n_t_pad, err,
                    stage, full, empty, acc_s);
}

// ------------------------------------------------------------------------------------- batched
__device__ __forceinline__ void inval_barriers(uint64_t* full, uint64_t* empty, int n) {
    for (int s = 0; s < n; ++s) {
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&full[s])) : "memory");
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_u32(&empty[s])) : "memory");
    }
}

// Persistent forward over the units of several jobs of one label (MODE): each block repeatedly
// takes the next unit (job, frequency block) from an atomic counter. A unit's result does not
// depend on which block runs it or on the other jobs in the batch. One instantiation per label
// keeps each at its own register count (a kernel holding both paths takes the larger).
template <int MODE>
__global__ void __launch_bounds__(FWD_THREADS, MODE == 0 ? 4 : 3) k_fwd_batch_f32(const BatchFwdJob* __restrict__ jobs,
                                                               const BatchUnit* __restrict__ units, int n_units,
                                                               int* __restrict__ counter, int* __restrict__ err) {
    __shared__ __align__(128) TriF32 stage[kFwdStages][kFwdTile];
    __shared__ __align__(8) uint64_t full[kFwdStages], empty[kFwdStages];
    __shared__ int s_u;
    while (true) {
        if (threadIdx.x == 0) s_u = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_u;
        __syncthreads();
        if (u >= n_units) break;
        const BatchUnit U = units[u];
        const BatchFwdJob& J = jobs[U.job];
        const int t0 = (int)((int64_t)J.n_tiles * U.b / J.splits), t1 = (int)((int64_t)J.n_tiles * (U.b + 1) / J.splits);
        float2* out = J.S;
        if (J.splits > 1) out = J.S_part + (int64_t)U.b * (J.fs.dM ? *J.fs.dM : J.fs.M);
        const bool used = fwd_block<MODE, false>(J.tris + (int64_t)t0 * kFwdTile, t1 - t0,
                                                 t1 == J.n_tiles ? J.last : kFwdTile, J.fs, J.tp[0], J.tp[1], J.tp[2],
                                                 J.d_vol, out, err, U.a, stage, full, empty, U.b == 0);
        __syncthreads();
        if (used && threadIdx.x == 0) inval_barriers(full, empty, kFwdStages);
        __syncthreads();
    }
}

// Persistent adjoint over units (job, triangle block, frequency chunk of chunk_tiles tiles) of one label.
template <int MODE>
__global__ void __launch_bounds__(ADJ_THREADS, MODE == 0 ? 5 : 4) k_adj_batch_f32(const BatchAdjJob* __restrict__ jobs,
                                                               const BatchUnit* __restrict__ units, int n_units,
                                                               int* __restrict__ counter, int* __restrict__ err) {
    constexpr int NACC = MODE == 0 ? NACC_SURF : NACC_VOL;
    __shared__ __align__(128) FreqPairF32 stage[kAdjStages][kAdjPairs];
    __shared__ __align__(8) uint64_t full[kAdjStages], empty[kAdjStages];
    __shared__ int s_u;
    __shared__ float acc_s[2 * NACC * ADJ_THREADS];
    while (true) {
        if (threadIdx.x == 0) s_u = atomicAdd(counter, 1);
        __syncthreads();
        const int u = s_u;
        __syncthreads();
        if (u >= n_units) break;
        const BatchUnit U = units[u];
        const BatchAdjJob& J = jobs[U.job];
        const int64_t M = J.dM ? *J.dM : J.M_max;
        const int n_ftiles = (int)((M + ADJ_FTILE - 1) / ADJ_FTILE);
        const int f0 = U.b * J.chunk_tiles;
        const int f1 = min(f0 + J.chunk_tiles, n_ftiles);
        float* out = J.partial + (int64_t)U.b * NACC * J.n_t_pad;
        const bool used = adj_block<MODE>(J.tris, J.n_t, J.n_t_pad, J.fr, f0, f1, U.a, out, err, stage, full, empty,
                                          acc_s);
        __syncthreads();
        if (used && threadIdx.x == 0) inval_barriers(full, empty, kAdjStages);
        __syncthreads();
    }
}

}  // namespace

// Work units of the forward: at least ~112 per SM (28 per resident block). Units are equal in cost
// and handed out as blocks free up, so the SMs finish within about one unit of each other: with
// 8 units per SM the last, partly filled round of blocks cost 6% of the 128^3 forward; 56 and 112
// per SM took it from 11.9 to 11.1 and 11.05 ms (224 was slower again: each unit then covers few
// triangle tiles). The triangle splits this makes are summed in a fixed order.
int fwd_target_units(int sm_count) { return 112 * sm_count; }

size_t fwd_partial_elems(int64_t M_max, int sm_count) {
    const int64_t fb = (M_max + FWD_BLOCK_FREQS - 1) / FWD_BLOCK_FREQS;
    return (size_t)(fwd_target_units(sm_count) + fb) * FWD_BLOCK_FREQS;
}

cudaError_t launch_fwd_f32(int mode, const TriF32* tris, int64_t n_t, const FreqSrc& fs, const Geom& g,
                           const double* d_vol, float2* S, float2* S_part, int sm_count, int* d_err, cudaStream_t st) {
    const int n_tiles = (int)((n_t + kFwdTile - 1) / kFwdTile);
    const int last = (int)(n_t - (int64_t)(n_tiles - 1) * kFwdTile);
    const float tpx = (float)(2.0 * M_PI / g.L[0]), tpy = (float)(2.0 * M_PI / g.L[1]),
                tpz = (float)(2.0 * M_PI / g.L[2]);
    const int64_t fb_max = (fs.M + FWD_BLOCK_FREQS - 1) / FWD_BLOCK_FREQS;
    if (fb_max <= 0 || n_tiles <= 0) return cudaSuccess;
    // enough blocks for any band size up to fs.M: fb * splits <= target + fb
    const int target = fwd_target_units(sm_count);
    const int64_t blocks = S_part ? fb_max + target : fb_max;
    const dim3 grid((unsigned)blocks);
    const bool ex = fs.nlist != nullptr;
    if (mode == 0 && !ex)
        k_fwd_f32<0, false><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, last, fs, tpx, tpy, tpz, d_vol, S, S_part,
                                                          target, d_err);
    if (mode == 0 && ex)
        k_fwd_f32<0, true><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, last, fs, tpx, tpy, tpz, d_vol, S, S_part,
                                                         target, d_err);
    if (mode == 1 && !ex)
        k_fwd_f32<1, false><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, last, fs, tpx, tpy, tpz, d_vol, S, S_part,
                                                          target, d_err);
    if (mode == 1 && ex)
        k_fwd_f32<1, true><<<grid, FWD_THREADS, 0, st>>>(tris, n_tiles, last, fs, tpx, tpy, tpz, d_vol, S, S_part,
                                                         target, d_err);
    if (S_part) k_fwd_reduce<<<4 * sm_count, 256, 0, st>>>(fs, n_tiles, target, 0, S_part, S);
    return cudaGetLastError();
}

int adj_chunks_f32(int64_t n_t, int64_t M_max, int sm_count) {
    const int64_t tblocks = (n_t + ADJ_THREADS - 1) / ADJ_THREADS;
    const int64_t ftiles = (M_max + ADJ_FTILE - 1) / ADJ_FTILE;
    // ~128 (triangle block, frequency chunk) units per SM, so that the SMs finish within a small
    // fraction of the launch of each other (8 per SM left 10% of the 128^3 adjoint in the last,
    // partly filled round of blocks: 20.9 -> 18.3 ms at 128 per SM); the chunks' partial sums are
    // added afterwards in a fixed order
    const int64_t target = (int64_t)sm_count * 128;
    int64_t c = (target + tblocks - 1) / tblocks;
    if (c < 1) c = 1;
    if (c > ftiles) c = ftiles;
    if (c > 65535) c = 65535;
    return (int)(c < 1 ? 1 : c);
}

cudaError_t launch_adj_f32(int mode, const TriF32* tris, int64_t n_t, int64_t n_t_pad, const FreqF32* fr,
                           const int64_t* dM, int64_t M_max, float* partial, int n_chunks, int* d_err, cudaStream_t st) {
    const dim3 grid((unsigned)(n_t_pad / ADJ_THREADS), (unsigned)n_chunks);
    if (mode == 0)
        k_adj_f32<0><<<grid, ADJ_THREADS, 0, st>>>(tris, n_t, n_t_pad, fr, dM, M_max, partial, d_err);
    else
        k_adj_f32<1><<<grid, ADJ_THREADS, 0, st>>>(tris, n_t, n_t_pad, fr, dM, M_max, partial, d_err);
    return cudaGetLastError();
}

int batch_blocks_per_sm_fwd(int mode) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mode == 0 ? k_fwd_batch_f32<0> : k_fwd_batch_f32<1>,
                                                  FWD_THREADS, 0);
    return n > 0 ? n : 1;
}
int batch_blocks_per_sm_adj(int mode) {
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, mode == 0 ? k_adj_batch_f32<0> : k_adj_batch_f32<1>,
                                                  ADJ_THREADS, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_fwd_batch_f32(int mode, const BatchFwdJob* jobs, const BatchUnit* units, int n_units, int* counter,
                                 int grid, int* d_err, cudaStream_t st) {
    if (n_units <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (mode == 0)
        k_fwd_batch_f32<0><<<grid, FWD_THREADS, 0, st>>>(jobs, units, n_units, counter, d_err);
    else
        k_fwd_batch_f32<1><<<grid, FWD_THREADS, 0, st>>>(jobs, units, n_units, counter, d_err);
    return cudaGetLastError();
}

cudaError_t launch_fwd_reduce_splits(const FreqSrc& fs, int splits, const float2* S_part, float2* S, int sm_count,
                                     cudaStream_t st) {
    if (splits <= 1) return cudaSuccess;
    k_fwd_reduce<<<4 * sm_count, 256, 0, st>>>(fs, 1, 0, splits, S_part, S);
    return cudaGetLastError();
}

cudaError_t launch_adj_batch_f32(int mode, const BatchAdjJob* jobs, const BatchUnit* units, int n_units, int* counter,
                                 int grid, int* d_err, cudaStream_t st) {
    if (n_units <= 0) return cudaSuccess;
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    if (mode == 0)
        k_adj_batch_f32<0><<<grid, ADJ_THREADS, 0, st>>>(jobs, units, n_units, counter, d_err);
    else
        k_adj_batch_f32<1><<<grid, ADJ_THREADS, 0, st>>>(jobs, units, n_units, counter, d_err);
    return cudaGetLastError();
}

}  // namespace dm
