// kernels3d.cuh -- device routines of the 3D query (Algorithm 1, query half).
//
// leaf3_eval: exact GWN of one trimmed leaf (Section 3.3) by a Stokes
//   reduction of Eq. 2.  With a unit vector s, the potential
//       A_s(r) = (s x r) / (|r| (|r| + s . r))
//   satisfies curl A_s = r / |r|^3 off the half line {q - t s, t > 0}, so
//       w = (1/4pi) sum_c mult_c int A_s(x_c(t) - q) . x_c'(t) dt  -  sum_hits wind sign(s . n)
//   where x_c are the leaf's boundary curves (trims composed with the surface,
//   built by build3d.cpp) and the hits are crossings of the half line with the
//   visible surface.
//   * q outside the sphere around the leaf's box (radius 1.1 x half diagonal):
//     s points from q to the box centre.  The half line then leaves the box
//     behind (no hits), and every boundary point is seen at more than 90 degrees
//     from the half line, so the integrand is smooth.
//   * otherwise s is the leaf's mean normal, oriented so that the half line
//     points away from the leaf's mid-plane.  The leaf is a graph along its mean
//     normal (normal cone below 55 degrees, enforced by the build), so the half
//     line meets it at most once: the foot point is found by Newton's method on
//     the two tangential components, and counted if it lies on the half line
//     and inside the leaf's visible region (winding number of its local 2D
//     boundary).
//   The line integral uses Gauss-Legendre panels (4 points in FP32, 8 in FP64),
//   bisected (stackless, by level and index) until each panel is shorter than
//   a ratio (kRatio*) times its distance to q and to the string.  FP32 stops at
//   kLevel32 bisections; a leaf that needs more, or whose foot point is too
//   close to call in FP32, is evaluated again in FP64: the near-boundary band
//   (one warp per pair, leaf3_warp64).
// far3: the order-2 Taylor expansion of Eq. 3 in folded form (gwn_internal.h).
#pragma once

#include "gwn_internal.h"
#include "kernels2d.cuh"
#include "../../include/gwn.h"

namespace gwn {

constexpr int kLevel32 = 10;
constexpr float kInfF = 3.0e38f;  // below it: a finite panel length in a node table
constexpr int kLevel64 = 30;
// panel length / distance-to-q bound of the 8-point rule: the quadrature error
// of an analytic integrand decays like rho^-16 with rho the Bernstein-ellipse
// parameter, ~3.0 at 1.5 and ~6 at 0.75.  The FP32 bulk takes 4-point panels
// at 0.75 (error ~6^-8); the FP64 near band that completes it 8-point panels
// at 1.5 (FP64 is needed there for the geometry, not for the quadrature); the
// repair 1.0 (measured ~1e-7 against the oracle); the all-FP64 precision mode
// 0.5 (~1e-8).
constexpr float kRatio32 = 0.75f;
constexpr double kRatio64Band = 1.5;
constexpr double kRatio64Repair = 1.0;
constexpr double kRatio64Exact = 0.5;
// the warp evaluator (leaf3_warp64<4>) takes 4-point panels at half these ratios,
// which keeps the same Bernstein-ellipse margin per panel with half the nodes
constexpr double kRatio64BandW4 = 0.75;
constexpr double kRatio64RepairW4 = 0.5;

// binomial coefficients and the 8-point Gauss-Legendre rule on [0, 1]: device
// constant memory, with host mirrors for host-side execution
__constant__ float c_binom[kMaxC3Deg + 1][kMaxC3Deg + 1];
__constant__ double c_glx8[8];
__constant__ double c_glw8[8];
__constant__ float c_glx4f[4];
__constant__ float c_glw4f[4];
__constant__ double c_glx4d[4];
__constant__ double c_glw4d[4];
static float h_binom[kMaxC3Deg + 1][kMaxC3Deg + 1];
static double h_glx8[8], h_glw8[8];
static float h_glx4f[4], h_glw4f[4];
static double h_glx4d[4], h_glw4d[4];
#if defined(__CUDA_ARCH__)
#define GWN_BINOM(d, i) c_binom[d][i]
#define GWN_GLX(k) c_glx8[k]
#define GWN_GLW(k) c_glw8[k]
#define GWN_GLXF(k) c_glx4f[k]
#define GWN_GLWF(k) c_glw4f[k]
#define GWN_GLX4D(k) c_glx4d[k]
#define GWN_GLW4D(k) c_glw4d[k]
#else
#define GWN_BINOM(d, i) h_binom[d][i]
#define GWN_GLX(k) h_glx8[k]
#define GWN_GLW(k) h_glw8[k]
#define GWN_GLXF(k) h_glx4f[k]
#define GWN_GLWF(k) h_glw4f[k]
#define GWN_GLX4D(k) h_glx4d[k]
#define GWN_GLW4D(k) h_glw4d[k]
#endif

// accessors of one leaf's geometry, in FP32 (relative to the leaf centre) or FP64 (absolute)
struct Geo32 {
    static constexpr int kPtStride = 1;  // array elements per curve point
    const float4* net;
    const float4* pts;
    GWN_HD inline void net_pt(int k, float h[4]) const {
        float4 v = GWN_LDG(net + k);
        h[0] = v.x; h[1] = v.y; h[2] = v.z; h[3] = v.w;
    }
    GWN_HD inline void pt(int k, float h[4]) const {
        float4 v = GWN_LDG(pts + k);
        h[0] = v.x; h[1] = v.y; h[2] = v.z; h[3] = v.w;
    }
};
struct Geo64 {
    static constexpr int kPtStride = 4;
    const double* net;
    const double* pts;
    GWN_HD inline void net_pt(int k, double h[4]) const {
        for (int c = 0; c < 4; ++c) h[c] = net[k * 4 + c];
    }
    GWN_HD inline void pt(int k, double h[4]) const {
        for (int c = 0; c < 4; ++c) h[c] = pts[k * 4 + c];
    }
};

// value and derivative (homogeneous) of a degree-D Bernstein curve by Horner's
// rule in r = a / (1 - a), a = min(t, 1 - t) (the curve is read backwards when
// t > 1/2), with the binomial-scaled points P_i = C(D,i) c_i and derivative
// points Q_i = C(D-1,i) (c_{i+1} - c_i) stored by the build:
//   X(t)  = (1 - a)^D     sum_i P_i r^i
//   X'(t) = D (1 - a)^(D-1) sum_i Q_i r^i
template <typename T, typename G>
GWN_HD inline void bern4(const G& g0, int D, T t, T X[4], T dX[4]) {
    const bool rev = t > T(0.5);
    const T a = rev ? T(1) - t : t;
    const T b = T(1) - a;
    const T r = a * Num<T>::rcp_fast(b);
    G g = g0;
    if (rev) g.pts += (size_t)(2 * D + 1) * G::kPtStride;  // the reversed copy
    T acc[4], dacc[4], h[4];
    g.pt(D, acc);
    for (int i = D - 1; i >= 0; --i) {
        g.pt(i, h);
        for (int c = 0; c < 4; ++c) acc[c] = acc[c] * r + h[c];
    }
    g.pt(D + 1 + D - 1, dacc);
    for (int i = D - 2; i >= 0; --i) {
        g.pt(D + 1 + i, h);
        for (int c = 0; c < 4; ++c) dacc[c] = dacc[c] * r + h[c];
    }
    // b^(D-1) by repeated squaring
    T pw = T(1), base = b;
    int e = D - 1;
    while (e > 0) {
        if (e & 1) pw *= base;
        base *= base;
        e >>= 1;
    }
    for (int c = 0; c < 4; ++c) {
        X[c] = acc[c] * pw * b;
        dX[c] = T(D) * dacc[c] * pw;
    }
}

// the same for a degree known at compile time (the loops unroll and the point
// loads become independent); FP32 takes the hardware reciprocal for r
template <int D, typename T, typename G>
GWN_HD inline void bern4_fixed(const G& g0, T t, T X[4], T dX[4]) {
    const bool rev = t > T(0.5);
    const T a = rev ? T(1) - t : t;
    const T b = T(1) - a;
    const T r = a * Num<T>::rcp_fast(b);
    G g = g0;
    if (rev) g.pts += (size_t)(2 * D + 1) * G::kPtStride;  // the reversed copy
    T acc[4], dacc[4], h[4];
    g.pt(D, acc);
#pragma unroll
    for (int i = D - 1; i >= 0; --i) {
        g.pt(i, h);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = acc[c] * r + h[c];
    }
    g.pt(D + 1 + D - 1, dacc);
#pragma unroll
    for (int i = D - 2; i >= 0; --i) {
        g.pt(D + 1 + i, h);
#pragma unroll
        for (int c = 0; c < 4; ++c) dacc[c] = dacc[c] * r + h[c];
    }
    T pw = T(1);
#pragma unroll
    for (int e = 0; e < D - 1; ++e) pw *= b;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        X[c] = acc[c] * pw * b;
        dX[c] = T(D) * dacc[c] * pw;
    }
}

// Gauss-Legendre rules on [0, 1] of the panels: 4 points in FP32 (relative
// error ~rho^-8 ~ 6e-7 per panel at the FP32 panel ratio 0.75, rho ~ 6), 8 in
// FP64; span = fraction of the panel between the first and the last node
template <typename T> struct Gl8;
template <> struct Gl8<float> {
    static constexpr int K = 4;
    static constexpr float span_inv = 1.17f;  // nodes span 86 % of the panel
    static GWN_HD inline float x(int k) { return GWN_GLXF(k); }
    static GWN_HD inline float w(int k) { return GWN_GLWF(k); }
};
template <> struct Gl8<double> {
    static constexpr int K = 8;
    static constexpr double span_inv = 1.1;  // nodes span 96 % of the panel
    static GWN_HD inline double x(int k) { return GWN_GLX(k); }
    static GWN_HD inline double w(int k) { return GWN_GLW(k); }
};

// the integrand A_s(x(t) - q) . x'(t) at parameter t of one boundary curve;
// also the point x(t) and min(|r|^2, 2 |r| (|r| + s.r)): the integrand is
// singular at q and along the string {q - t s}, and near the string
// |r| (|r| + s.r) ~ (distance to the string)^2 / 2, so a panel must be short
// relative to both distances
template <int DF, typename T, typename G>
GWN_HD inline T gl_node(const G& g, int D, T t, const T q[3], const T s[3], T x[3], T* dm2) {
    T X[4], dX[4];
    if (DF > 0) bern4_fixed<(DF > 0 ? DF : 1), T>(g, t, X, dX);
    else bern4<T>(g, D, t, X, dX);
    T iw = Num<T>::rcp_fast(X[3]);
    T x0 = X[0] * iw, x1 = X[1] * iw, x2 = X[2] * iw;
    T d0 = (dX[0] - x0 * dX[3]) * iw, d1 = (dX[1] - x1 * dX[3]) * iw, d2 = (dX[2] - x2 * dX[3]) * iw;
    T r0 = x0 - q[0], r1 = x1 - q[1], r2 = x2 - q[2];
    T rr = r0 * r0 + r1 * r1 + r2 * r2;
    T rn = Num<T>::sqrt_fast(rr);
    T sr = s[0] * r0 + s[1] * r1 + s[2] * r2;
    T c0 = s[1] * r2 - s[2] * r1, c1 = s[2] * r0 - s[0] * r2, c2 = s[0] * r1 - s[1] * r0;
    T den = rn * (rn + sr);
    x[0] = x0; x[1] = x1; x[2] = x2;
    *dm2 = fmin(rr, T(2) * den);
    return (c0 * d0 + c1 * d1 + c2 * d2) * Num<T>::rcp_fast(den);
}

// gl_node with the degree dispatched to the unrolled evaluators of the common
// composed degrees (6 d for local pieces of degree d = 1, 2, 3; edges of the
// leaf rectangle are degree-1 pieces)
template <typename T, typename G>
GWN_HD inline T gl_node_any(const G& g, int D, T t, const T q[3], const T s[3], T x[3], T* dm2) {
    switch (D) {
        case 6: return gl_node<6, T>(g, D, t, q, s, x, dm2);
        case 12: return gl_node<12, T>(g, D, t, q, s, x, dm2);
        case 18: return gl_node<18, T>(g, D, t, q, s, x, dm2);
        default: return gl_node<0, T>(g, D, t, q, s, x, dm2);
    }
}

// int A_s(x(t) - q) . x'(t) dt over the panels of one boundary curve below panel
// (level0, idx0) (panel idx of level L spans [idx, idx + 1] / 2^L), adaptive:
// a panel is bisected until its length is at most `ratio` times its distance to
// q and to the string; sets deep if the level limit was hit.
template <int DF, typename T, typename G>
GWN_HD T panel_subtree_d(const G& g, int D, const T q[3], const T s[3], int level0, unsigned idx0, int maxlevel, T ratio,
                         bool& deep, WorkLocal* wl) {
    const T ratio2 = ratio * ratio;
    T acc = 0;
    int level = level0;
    unsigned idx = idx0;  // panel index at `level` (levels stay below 32)
    while (true) {
        const T h = T(1) / T(1u << level);
        const T a = T(idx) * h;
        T psum = 0, dmin2 = T(1e30), len = 0;
        T px = 0, py = 0, pz = 0;
        // FP32 with a fixed degree: nodes unrolled by two (independent evaluations, ILP)
#pragma unroll(DF > 0 && sizeof(T) == 4 ? 2 : 1)
        for (int k = 0; k < Gl8<T>::K; ++k) {
            T x[3], dm2;
            T f = gl_node<DF, T>(g, D, a + h * Gl8<T>::x(k), q, s, x, &dm2);
            psum += Gl8<T>::w(k) * f;
            dmin2 = fmin(dmin2, dm2);
            if (k > 0) {
                T e0 = x[0] - px, e1 = x[1] - py, e2 = x[2] - pz;
                len += Num<T>::sqrt_fast(e0 * e0 + e1 * e1 + e2 * e2);
            }
            px = x[0]; py = x[1]; pz = x[2];
        }
        if (wl) {
            wl->v[kWorkGlNodes] += Gl8<T>::K;
            wl->v[kWorkGlDeg] += (unsigned long long)Gl8<T>::K * (unsigned long long)D;
        }
        len *= T(Gl8<T>::span_inv);
        bool refine = len * len > ratio2 * dmin2;
        if (refine && level < maxlevel) {
            ++level;
            idx <<= 1;
            continue;
        }
        if (refine) deep = true;
        acc += psum * h;
        while (level > level0 && (idx & 1u)) {
            idx >>= 1;
            --level;
        }
        if (level == level0) break;
        ++idx;
    }
    return acc;
}

template <typename T, typename G>
GWN_HD T panel_subtree(const G& g, int D, const T q[3], const T s[3], int level0, unsigned idx0, int maxlevel, T ratio,
                       bool& deep, WorkLocal* wl = nullptr) {
    switch (D) {
        case 6: return panel_subtree_d<6, T>(g, D, q, s, level0, idx0, maxlevel, ratio, deep, wl);
        case 12: return panel_subtree_d<12, T>(g, D, q, s, level0, idx0, maxlevel, ratio, deep, wl);
        case 18: return panel_subtree_d<18, T>(g, D, q, s, level0, idx0, maxlevel, ratio, deep, wl);
        default: return panel_subtree_d<0, T>(g, D, q, s, level0, idx0, maxlevel, ratio, deep, wl);
    }
}

// the whole curve, starting from the 2^min_level panels of level min_level
template <typename T, typename G>
GWN_HD T curve_line_integral(const G& g, int D, const T q[3], const T s[3], int maxlevel, T ratio, bool& deep,
                             WorkLocal* wl = nullptr, int min_level = 0) {
    if (min_level <= 0) return panel_subtree<T>(g, D, q, s, 0, 0u, maxlevel, ratio, deep, wl);
    T acc = 0;
    for (unsigned idx = 0; idx < (1u << min_level); ++idx)
        acc += panel_subtree<T>(g, D, q, s, min_level, idx, maxlevel, ratio, deep, wl);
    return acc;
}



// S, S_u, S_v of the leaf's bicubic net at local (u, v)
template <typename T, typename G>
GWN_HD void net_eval3(const G& g, T u, T v, T S[3], T Su[3], T Sv[3]) {
    T su = T(1) - u, sv = T(1) - v;
    T Bu[4] = {su * su * su, T(3) * u * su * su, T(3) * u * u * su, u * u * u};
    T Bv[4] = {sv * sv * sv, T(3) * v * sv * sv, T(3) * v * v * sv, v * v * v};
    T dBu[4] = {T(-3) * su * su, T(3) * su * su - T(6) * u * su, T(6) * u * su - T(3) * u * u, T(3) * u * u};
    T dBv[4] = {T(-3) * sv * sv, T(3) * sv * sv - T(6) * v * sv, T(6) * v * sv - T(3) * v * v, T(3) * v * v};
    T H[4] = {0, 0, 0, 0}, Hu[4] = {0, 0, 0, 0}, Hv[4] = {0, 0, 0, 0};
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            T h[4];
            g.net_pt(i * 4 + j, h);
            T b = Bu[i] * Bv[j], bu = dBu[i] * Bv[j], bv = Bu[i] * dBv[j];
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                H[c] += b * h[c];
                Hu[c] += bu * h[c];
                Hv[c] += bv * h[c];
            }
        }
    T iw = T(1) / H[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        S[c] = H[c] * iw;
        Su[c] = (Hu[c] - S[c] * Hu[3]) * iw;
        Sv[c] = (Hv[c] - S[c] * Hv[3]) * iw;
    }
}

enum { kHitNone = 0, kHitOk = 1, kHitUnsure = 2 };

// winding number of the leaf's local 2D boundary around (u, v); returns false if
// (u, v) is too close to the boundary to decide at this precision
template <typename T>
GWN_HD bool local_winding(const DevTree& t, const Leaf3Info& I, T u, T v, int maxlevel, int* wind) {
    T acc = 0;
    for (int c = 0; c < I.c2_cnt; ++c) {
        T H[4][3];
        int k = I.c2_off + c;
        if (sizeof(T) == 4) {
            const float4* C = t.c2 + (size_t)k * kC2Vec;
            float4 a = GWN_LDG(C), b = GWN_LDG(C + 1), d = GWN_LDG(C + 2);
            float f[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, d.x, d.y, d.z, d.w};
            for (int i = 0; i < 4; ++i) {
                H[i][0] = (T)f[3 * i] - u * (T)f[3 * i + 2];
                H[i][1] = (T)f[3 * i + 1] - v * (T)f[3 * i + 2];
                H[i][2] = (T)f[3 * i + 2];
            }
        } else {
            const double* C = t.c2_64 + (size_t)k * 12;
            for (int i = 0; i < 4; ++i) {
                H[i][0] = (T)C[3 * i] - u * (T)C[3 * i + 2];
                H[i][1] = (T)C[3 * i + 1] - v * (T)C[3 * i + 2];
                H[i][2] = (T)C[3 * i + 2];
            }
        }
        T a;
        if (!curve_angle<T>(H, maxlevel, &a)) return false;
        acc += (T)t.c2mult[k] * a;
    }
    *wind = (int)round(acc * Num<T>::inv2pi);
    return true;
}

// crossing of the half line {q + tau sig n, tau > 0} with the leaf: *contrib =
// wind * sign(s . N) with s = -sig n, to be subtracted from the line integral
template <typename T, typename G>
GWN_HD int leaf_hit(const DevTree& t, const Leaf3Info& I, const G& g, const T q[3], const T nrm[3], T sig, T diag,
                        T* contrib, int maxlevel) {
    *contrib = 0;
    // tangent basis
    T e1[3], e2[3];
    {
        T ax = fabs(nrm[0]) < T(0.9) ? T(1) : T(0), ay = T(1) - ax;
        // e1 = normalize(a x n) with a = x or y axis
        T a[3] = {ax, ay, 0};
        e1[0] = a[1] * nrm[2] - a[2] * nrm[1];
        e1[1] = a[2] * nrm[0] - a[0] * nrm[2];
        e1[2] = a[0] * nrm[1] - a[1] * nrm[0];
        T l = Num<T>::rsqrt_(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
        e1[0] *= l; e1[1] *= l; e1[2] *= l;
        e2[0] = nrm[1] * e1[2] - nrm[2] * e1[1];
        e2[1] = nrm[2] * e1[0] - nrm[0] * e1[2];
        e2[2] = nrm[0] * e1[1] - nrm[1] * e1[0];
    }
    // quick rejects from the convex hull of the control points (positive
    // weights): q's projection outside the projected control-net box, or the
    // whole net behind q along the half line (every hull point has a height
    // sig n . (P - q) below -tau_eps, so no crossing exists and q is not near
    // the leaf's surface either)
    const T tau_eps = sizeof(T) == 4 ? T(1e-4) * diag : T(1e-12) * diag;
    T mn1 = T(1e30), mx1 = T(-1e30), mn2 = T(1e30), mx2 = T(-1e30), mxh = T(-1e30);
    for (int k = 0; k < 16; ++k) {
        T h[4];
        g.net_pt(k, h);
        T iw = T(1) / h[3];
        T d0 = h[0] * iw - q[0], d1 = h[1] * iw - q[1], d2 = h[2] * iw - q[2];
        T p1 = d0 * e1[0] + d1 * e1[1] + d2 * e1[2];
        T p2 = d0 * e2[0] + d1 * e2[1] + d2 * e2[2];
        T ph = sig * (d0 * nrm[0] + d1 * nrm[1] + d2 * nrm[2]);
        mn1 = fmin(mn1, p1); mx1 = fmax(mx1, p1);
        mn2 = fmin(mn2, p2); mx2 = fmax(mx2, p2);
        mxh = fmax(mxh, ph);
    }
    if (mn1 > 0 || mx1 < 0 || mn2 > 0 || mx2 < 0) return kHitNone;
    if (mxh < -tau_eps) return kHitNone;
    // exact test: winding number of the projected domain boundary (the net's
    // four edge curves, rational cubics) around q's projection.  Zero means the
    // line along the normal misses the leaf's rectangle altogether.
    {
        T acc = 0;
        for (int e = 0; e < 4; ++e) {
            T H[4][3];
            for (int k = 0; k < 4; ++k) {
                // bottom (v=0, u up), right (u=1, v up), top (v=1, u down), left (u=0, v down)
                int i = e == 0 ? k : (e == 1 ? 3 : (e == 2 ? 3 - k : 0));
                int j = e == 0 ? 0 : (e == 1 ? k : (e == 2 ? 3 : 3 - k));
                T h[4];
                g.net_pt(i * 4 + j, h);
                T dx = h[0] - q[0] * h[3], dy = h[1] - q[1] * h[3], dz = h[2] - q[2] * h[3];
                H[k][0] = e1[0] * dx + e1[1] * dy + e1[2] * dz;
                H[k][1] = e2[0] * dx + e2[1] * dy + e2[2] * dz;
                H[k][2] = h[3];
            }
            T a;
            if (!curve_angle<T>(H, maxlevel, &a)) return kHitUnsure;  // q over the rectangle's edge
            acc += a;
        }
        if (fabs(acc) < T(3.14159265)) return kHitNone;  // winding number 0
    }
    T u = T(0.5), v = T(0.5);
    bool conv = false;
    T S[3], Su[3], Sv[3];
    const T tol = sizeof(T) == 4 ? T(1e-6) : T(1e-14);
    for (int it = 0; it < 40; ++it) {
        net_eval3<T>(g, u, v, S, Su, Sv);
        T d[3] = {S[0] - q[0], S[1] - q[1], S[2] - q[2]};
        T F1 = e1[0] * d[0] + e1[1] * d[1] + e1[2] * d[2];
        T F2 = e2[0] * d[0] + e2[1] * d[1] + e2[2] * d[2];
        T J00 = e1[0] * Su[0] + e1[1] * Su[1] + e1[2] * Su[2];
        T J01 = e1[0] * Sv[0] + e1[1] * Sv[1] + e1[2] * Sv[2];
        T J10 = e2[0] * Su[0] + e2[1] * Su[1] + e2[2] * Su[2];
        T J11 = e2[0] * Sv[0] + e2[1] * Sv[1] + e2[2] * Sv[2];
        T det = J00 * J11 - J01 * J10;
        if (!(fabs(det) > T(0))) break;
        T du = (J11 * F1 - J01 * F2) / det, dv = (J00 * F2 - J10 * F1) / det;
        u -= du;
        v -= dv;
        u = fmin(fmax(u, T(-0.5)), T(1.5));
        v = fmin(fmax(v, T(-0.5)), T(1.5));
        if (fabs(du) + fabs(dv) < tol) {
            conv = true;
            break;
        }
    }
    if (!conv) return kHitUnsure;
    const T eps = sizeof(T) == 4 ? T(1e-5) : T(1e-12);
    if (u < -eps || u > T(1) + eps || v < -eps || v > T(1) + eps) return kHitNone;
    net_eval3<T>(g, u, v, S, Su, Sv);
    T tau = sig * (nrm[0] * (S[0] - q[0]) + nrm[1] * (S[1] - q[1]) + nrm[2] * (S[2] - q[2]));
    if (fabs(tau) < tau_eps) return kHitUnsure;  // q too close to the surface to decide here
    if (u < eps || u > T(1) - eps || v < eps || v > T(1) - eps) return kHitUnsure;  // on the leaf's rectangle edge
    if (tau < 0) return kHitNone;
    int wind = 0;
    if (!local_winding<T>(t, I, u, v, maxlevel, &wind)) return kHitUnsure;
    if (wind == 0) return kHitNone;
    T N[3] = {Su[1] * Sv[2] - Su[2] * Sv[1], Su[2] * Sv[0] - Su[0] * Sv[2], Su[0] * Sv[1] - Su[1] * Sv[0]};
    // s = -sig nrm; the crossing enters the Stokes identity as wind * sign(s . N)
    T sn = -sig * (nrm[0] * N[0] + nrm[1] * N[1] + nrm[2] * N[2]);
    *contrib = (T)wind * (sn > 0 ? T(1) : T(-1));
    return kHitOk;
}

// the leaf's mean normal as a unit vector in precision T.  It is stored in
// float, so in double it is a unit vector only to ~6e-8; the string potential
// A_s has curl r / |r|^3 only for |s| = 1, and a string of length 1 + e shifts
// the line integral by about e times the leaf's solid angle, so the FP64
// evaluations renormalise it in double
template <typename T>
GWN_HD inline void unit_normal(const Leaf3Info& I, T nrm[3]) {
    nrm[0] = (T)I.nrm[0];
    nrm[1] = (T)I.nrm[1];
    nrm[2] = (T)I.nrm[2];
    if (sizeof(T) == 8) {
        const T l = T(1) / sqrt(nrm[0] * nrm[0] + nrm[1] * nrm[1] + nrm[2] * nrm[2]);
        nrm[0] *= l;
        nrm[1] *= l;
        nrm[2] *= l;
    }
}

// GWN of leaf li at q (q relative to the leaf geometry's origin); false if the
// precision of T could not resolve it
template <typename T, typename G>
GWN_HD bool leaf3_core(const DevTree& t, const Leaf3Info& I, const G& g, const T q[3], T* out, int maxlevel, T ratio,
                       WorkLocal* wl = nullptr) {
    if (wl) wl->v[kWorkLeaves] += 1;
    T nrm[3];
    unit_normal<T>(I, nrm);
    T cen[3];
    if (sizeof(T) == 4) {
        cen[0] = cen[1] = cen[2] = T(0);
    } else {
        cen[0] = (T)I.cen[0]; cen[1] = (T)I.cen[1]; cen[2] = (T)I.cen[2];
    }
    T dq[3] = {q[0] - cen[0], q[1] - cen[1], q[2] - cen[2]};
    T d2 = dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2];
    T rfar = T(1.1) * (T)I.rad;
    T s[3];
    T hits = 0;
    if (d2 > rfar * rfar) {
        T l = Num<T>::rsqrt_(d2);
        s[0] = -dq[0] * l; s[1] = -dq[1] * l; s[2] = -dq[2] * l;
    } else {
        T sig = (dq[0] * nrm[0] + dq[1] * nrm[1] + dq[2] * nrm[2]) >= 0 ? T(1) : T(-1);
        s[0] = -sig * nrm[0]; s[1] = -sig * nrm[1]; s[2] = -sig * nrm[2];
        if (wl) wl->v[kWorkHits] += 1;
        int hr = leaf_hit<T>(t, I, g, q, nrm, sig, (T)I.diag, &hits, sizeof(T) == 4 ? kNear32 : kMaxLevel64);
        if (hr == kHitUnsure) return false;
    }
    T acc = 0;
    bool deep = false;
    for (int c = 0; c < I.c3_cnt; ++c) {
        Curve3Info ci = t.c3[I.c3_off + c];
        G gc = g;
        if (sizeof(T) == 4) gc.pts = reinterpret_cast<decltype(gc.pts)>(t.c3pts + ci.ctrl_off);
        else gc.pts = reinterpret_cast<decltype(gc.pts)>(t.c3pts64 + (size_t)ci.ctrl_off * 4);
        // the 4-point FP32 rule starts at the curve's own minimum level; the 8-point
        // FP64 rule resolves the parametrisation from level 0
        acc += (T)ci.mult * curve_line_integral<T>(gc, ci.deg, q, s, maxlevel, ratio, deep, wl,
                                                   sizeof(T) == 4 ? ci.min_level : 0);
    }
    if (deep) return false;
    *out = acc * T(0.07957747154594767) - hits;  // 1 / (4 pi)
    return true;
}

GWN_HD inline double leaf3_eval64(const DevTree& t, int li, double qx, double qy, double qz, uint32_t& st,
                                  double ratio = kRatio64Exact) {
    Leaf3Info I = t.leaf3[li];
    Geo64 g{t.net3_64 + (size_t)li * 64, nullptr};
    double q[3] = {qx, qy, qz};
    double w = 0;
    if (!leaf3_core<double>(t, I, g, q, &w, kLevel64, ratio)) st |= GWN_QS_UNRESOLVED;
    return w;
}

// One panel of 4 Gauss-Legendre nodes read from a node table (6 float4: x, y,
// z, dx/dt, dy/dt, dz/dt per node): the weighted sum of the string potential's
// integrand A_s(x - q) . x' and the minimum over the nodes of
// min(|r|^2, 2 |r| (|r| + s.r)), the distance measure of the panel test.
// Per node: 3 subtractions, 12 multiply-adds, a square root and a reciprocal.
GWN_HD inline void fast_panel(const float4* P, const float q[3], const float s[3], float& psum, float& dmin2) {
    float f[24];
#pragma unroll
    for (int v = 0; v < 6; ++v) {
        const float4 a = GWN_LDG(P + v);
        f[4 * v] = a.x; f[4 * v + 1] = a.y; f[4 * v + 2] = a.z; f[4 * v + 3] = a.w;
    }
    psum = 0.f;
    dmin2 = 1e30f;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const float* n = f + 6 * k;
        const float r0 = n[0] - q[0], r1 = n[1] - q[1], r2 = n[2] - q[2];
        const float rr = r0 * r0 + r1 * r1 + r2 * r2;
        const float rn = Num<float>::sqrt_fast(rr);
        const float sr = s[0] * r0 + s[1] * r1 + s[2] * r2;
        const float c0 = s[1] * r2 - s[2] * r1, c1 = s[2] * r0 - s[0] * r2, c2 = s[0] * r1 - s[1] * r0;
        const float den = rn * (rn + sr);
        psum += GWN_GLWF(k) * (c0 * n[3] + c1 * n[4] + c2 * n[5]) * Num<float>::rcp_fast(den);
        dmin2 = fminf(dmin2, fminf(rr, 2.f * den));
    }
}

// FP32 exact leaf from the node tables, for a point outside the sphere of
// radius 1.1 x the leaf's half diagonal (q relative to the leaf centre, d2 =
// |q|^2): the string points from q away from the leaf, so there is no crossing
// to count, and every panel that the adaptive rule of leaf3_core would stop at
// level 0 or 1 is read from the table.  Same rule, ratio and node positions as
// leaf3_core<float> (the table's positions are rounded once from FP64).
// Returns false if some curve needs a panel below level 1 (or starts below
// it); the caller then evaluates the pair with leaf3_core.
GWN_HD inline bool leaf3_fast32(const DevTree& t, const Leaf3Info& I, const float q[3], float d2, float* out,
                                WorkLocal* wl = nullptr) {
    const float l = Num<float>::rsqrt_(d2);
    const float s[3] = {-q[0] * l, -q[1] * l, -q[2] * l};
    const float ratio2 = kRatio32 * kRatio32;
    float acc = 0.f;
    int nodes = 0;
    for (int c = 0; c < I.c3_cnt; ++c) {
        const float4* H = t.c3n + (size_t)(I.c3_off + c) * kC3NodeVec;
        // len0, len1a, len1b, mult; an infinite length marks a panel below the
        // curve's minimum level (level 0: skipped; level 1: the full evaluator)
        const float4 hd = GWN_LDG(H);
        if (hd.x < kInfF) {
            float psum, dmin2;
            fast_panel(H + 1, q, s, psum, dmin2);
            nodes += 4;
            if (hd.x * hd.x <= ratio2 * dmin2) {
                acc += hd.w * psum;
                continue;
            }
        }
        float pa, da, pb, db;
        fast_panel(H + 7, q, s, pa, da);
        fast_panel(H + 13, q, s, pb, db);
        nodes += 8;
        if (!(hd.y * hd.y <= ratio2 * da && hd.z * hd.z <= ratio2 * db)) return false;
        acc += hd.w * 0.5f * (pa + pb);
    }
    if (wl) wl->v[kWorkFastNodes] += (unsigned long long)nodes;  // kWorkLeaves counts the full evaluations
    *out = acc * 0.07957747154594767f;  // 1 / (4 pi)
    return true;
}

// FP32 evaluation only; false if the leaf needs the FP64 near band.  With
// try_fast, a point outside the leaf's 1.1-radius sphere first tries the
// node tables (leaf3_fast32).
GWN_HD inline bool leaf3_try32(const DevTree& t, int li, float qx, float qy, float qz, float* w,
                               WorkLocal* wl = nullptr, bool try_fast = true) {
    Leaf3Info I = t.leaf3[li];
    float q[3] = {qx - I.cen[0], qy - I.cen[1], qz - I.cen[2]};
    *w = 0.f;
    if (try_fast && t.c3n) {
        const float d2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2];
        const float rfar = 1.1f * I.rad;
        if (d2 > rfar * rfar && leaf3_fast32(t, I, q, d2, w, wl)) return true;
    }
    Geo32 g{t.net3 + (size_t)li * kNet3Vec, nullptr};
    return leaf3_core<float>(t, I, g, q, w, kLevel32, kRatio32, wl);
}

GWN_HD inline float leaf3_eval32(const DevTree& t, int li, float qx, float qy, float qz, uint32_t& st) {
    float w;
    if (leaf3_try32(t, li, qx, qy, qz, &w)) return w;
    st |= GWN_QS_NEAR;
    return (float)leaf3_eval64(t, li, (double)qx, (double)qy, (double)qz, st, kRatio64Band);
}

// ---- FP64 exact leaf from the FP64 node tables (the repair's far pairs).
// q (absolute) outside the sphere of radius 1.1 x the leaf's half diagonal:
// the string points from q away from the leaf (no crossing), and every curve
// whose 8-point panels stop at level 0 or 1 at panel ratio `ratio` is read from
// its table.  Same rule and node positions as leaf3_core<double>'s first two
// levels.  node64 adds one node: weight x A_s(x - q) . x' and the panel test's
// distance measure min(|r|^2, 2 |r| (|r| + s.r)).
GWN_HD inline void node64(const double* n, const double q[3], const double s[3], double wk, double& f, double& dm) {
    const double r0 = n[0] - q[0], r1 = n[1] - q[1], r2 = n[2] - q[2];
    const double rr = r0 * r0 + r1 * r1 + r2 * r2;
    const double rn = sqrt(rr);
    const double sr = s[0] * r0 + s[1] * r1 + s[2] * r2;
    const double c0 = s[1] * r2 - s[2] * r1, c1 = s[2] * r0 - s[0] * r2, c2 = s[0] * r1 - s[1] * r0;
    const double den = rn * (rn + sr);
    f += wk * (c0 * n[3] + c1 * n[4] + c2 * n[5]) / den;
    dm = fmin(dm, fmin(rr, 2.0 * den));
}

// the string direction of a far pair: from q towards the leaf centre, unit in FP64
GWN_HD inline double far_string64(const Leaf3Info& I, const double q[3], double s[3]) {
    const double dq[3] = {q[0] - (double)I.cen[0], q[1] - (double)I.cen[1], q[2] - (double)I.cen[2]};
    const double d2 = dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2];
    const double l = 1.0 / sqrt(d2);
    s[0] = -dq[0] * l;
    s[1] = -dq[1] * l;
    s[2] = -dq[2] * l;
    return d2;
}

// one thread (host execution and tests); false where leaf3_core<double> is needed
GWN_HD inline bool leaf3_fast64(const DevTree& t, int li, const double q[3], double ratio, double* out) {
    const Leaf3Info I = t.leaf3[li];
    double s[3];
    const double d2 = far_string64(I, q, s);
    const double rfar = 1.1 * (double)I.rad;
    if (!t.c3n64 || !(d2 > rfar * rfar)) return false;
    const double ratio2 = ratio * ratio;
    double acc = 0;
    for (int c = 0; c < I.c3_cnt; ++c) {
        const double* H = t.c3n64 + (size_t)(I.c3_off + c) * kC3Node64;
        double f = 0, dm = 1e300;
        for (int k = 0; k < 8; ++k) node64(H + 4 + 6 * k, q, s, GWN_GLW(k), f, dm);
        if (H[0] * H[0] <= ratio2 * dm) {
            acc += H[3] * f;
            continue;
        }
        double fa = 0, da = 1e300, fb = 0, db = 1e300;
        for (int k = 0; k < 8; ++k) {
            node64(H + 52 + 6 * k, q, s, GWN_GLW(k), fa, da);
            node64(H + 100 + 6 * k, q, s, GWN_GLW(k), fb, db);
        }
        if (H[1] * H[1] > ratio2 * da || H[2] * H[2] > ratio2 * db) return false;
        acc += H[3] * 0.5 * (fa + fb);
    }
    *out = acc * 0.07957747154594767;  // 1 / (4 pi)
    return true;
}

#if defined(__CUDACC__)
// the same spread over a warp: 4 curves at a time, 8 lanes per curve (one
// node each), panel sums and distance measures reduced within the 8 lanes
__device__ inline bool leaf3_fast64_warp(const DevTree& t, int li, const double q[3], double ratio, double* out) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, grp = lane >> 3, k = lane & 7;
    const Leaf3Info I = t.leaf3[li];
    double s[3];
    const double d2 = far_string64(I, q, s);
    const double rfar = 1.1 * (double)I.rad;
    if (!t.c3n64 || !(d2 > rfar * rfar)) return false;
    const double ratio2 = ratio * ratio;
    const double wk = GWN_GLW(k);
    double acc = 0;
    bool deep = false;
    for (int c0 = 0; c0 < I.c3_cnt; c0 += 4) {
        const int c = c0 + grp;
        const bool act = c < I.c3_cnt;
        const double* H = t.c3n64 + (size_t)(I.c3_off + (act ? c : 0)) * kC3Node64;
        double f = 0, dm = 1e300;
        if (act) node64(H + 4 + 6 * k, q, s, wk, f, dm);
        for (int off = 1; off < 8; off <<= 1) {
            f += __shfl_xor_sync(full, f, off);
            dm = fmin(dm, __shfl_xor_sync(full, dm, off));
        }
        const bool need1 = act && H[0] * H[0] > ratio2 * dm;
        double val = f;
        if (__any_sync(full, need1)) {
            double fa = 0, da = 1e300, fb = 0, db = 1e300;
            if (need1) {
                node64(H + 52 + 6 * k, q, s, wk, fa, da);
                node64(H + 100 + 6 * k, q, s, wk, fb, db);
            }
            for (int off = 1; off < 8; off <<= 1) {
                fa += __shfl_xor_sync(full, fa, off);
                fb += __shfl_xor_sync(full, fb, off);
                da = fmin(da, __shfl_xor_sync(full, da, off));
                db = fmin(db, __shfl_xor_sync(full, db, off));
            }
            if (need1) {
                if (H[1] * H[1] > ratio2 * da || H[2] * H[2] > ratio2 * db) deep = true;
                val = 0.5 * (fa + fb);
            }
        }
        if (act && k == 0) acc += H[3] * val;
    }
    if (__any_sync(full, deep)) return false;
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(full, acc, off);
    *out = acc * 0.07957747154594767;  // 1 / (4 pi)
    return true;
}
#endif

// ---- One FP64 leaf evaluation spread over a warp (near band and repair).
// In one thread, an evaluation close to a boundary curve runs hundreds of
// Gauss-Legendre nodes one after another at FP64 latency, and such a single
// pair bounds the duration of its whole launch.  Here lane 0 does the crossing
// test, then the warp works through the adaptive panels of all boundary curves
// as a shared list (in shared memory, `stk`, kQuadStack entries): 32 / K panels
// per step, one Gauss-Legendre node per lane, the K lanes of a panel reducing
// its sum, distance and length with shuffles.  A panel that fails the length
// test pushes its two halves; when the list is full its group's leader
// integrates the panel's subtree alone.  Same arithmetic as leaf3_core<double>
// up to the order of the additions.  Returns false (w undefined) where
// leaf3_core would.
constexpr int kQuadStack = 256;

#if defined(__CUDACC__)
template <int K>
__device__ inline bool leaf3_warp64(const DevTree& t, int li, const double q[3], double ratio, int maxlevel, int2* stk,
                                    double* out) {
    static_assert(K == 4 || K == 8, "4 or 8 nodes per panel");
    constexpr int kPanels = 32 / K;                    // panels per step
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, grp = lane / K, k = lane % K;
    const Leaf3Info I = t.leaf3[li];
    const Geo64 g{t.net3_64 + (size_t)li * 64, nullptr};
    double nrm[3];
    unit_normal<double>(I, nrm);
    const double dq[3] = {q[0] - (double)I.cen[0], q[1] - (double)I.cen[1], q[2] - (double)I.cen[2]};
    const double d2 = dq[0] * dq[0] + dq[1] * dq[1] + dq[2] * dq[2];
    const double rfar = 1.1 * (double)I.rad;
    double s[3];
    double hits = 0;
    if (d2 > rfar * rfar) {
        double l = Num<double>::rsqrt_(d2);
        s[0] = -dq[0] * l; s[1] = -dq[1] * l; s[2] = -dq[2] * l;
    } else {
        double sig = (dq[0] * nrm[0] + dq[1] * nrm[1] + dq[2] * nrm[2]) >= 0 ? 1.0 : -1.0;
        s[0] = -sig * nrm[0]; s[1] = -sig * nrm[1]; s[2] = -sig * nrm[2];
        int hr = kHitNone;
        if (lane == 0) hr = leaf_hit<double>(t, I, g, q, nrm, sig, (double)I.diag, &hits, kMaxLevel64);
        hr = __shfl_sync(full, hr, 0);
        hits = __shfl_sync(full, hits, 0);
        if (hr == kHitUnsure) return false;
    }
    const double ratio2 = ratio * ratio;
    double acc = 0;
    bool deep = false;
    int sp = 0, next_curve = 0;
    __syncwarp();
    while (true) {
        // curves not started yet enter the list while it has room
        const int add = min(kQuadStack - sp, I.c3_cnt - next_curve);
        for (int j = lane; j < add; j += 32) stk[sp + j] = make_int2(next_curve + j, 0);
        sp += add;
        next_curve += add;
        __syncwarp();
        if (sp == 0) break;
        const int take = min(sp, kPanels);
        int2 task = make_int2(-1, 0);
        if (grp < take) task = stk[sp - 1 - grp];
        sp -= take;
        __syncwarp();
        const bool act = task.x >= 0;
        int level = 0, cidx = 0;
        unsigned idx = 0;
        double h = 1, f = 0, dm2 = 1e300, x[3] = {0, 0, 0};
        Curve3Info ci{};
        Geo64 gc = g;
        if (act) {
            cidx = task.x & 0xffff;
            level = task.x >> 16;
            idx = (unsigned)task.y;
            ci = t.c3[I.c3_off + cidx];
            gc.pts = t.c3pts64 + (size_t)ci.ctrl_off * 4;
            h = 1.0 / double(1u << level);
            const double xk = K == 8 ? Gl8<double>::x(k) : GWN_GLX4D(k);
            f = gl_node_any<double>(gc, ci.deg, double(idx) * h + h * xk, q, s, x, &dm2);
        }
        const double p0 = __shfl_up_sync(full, x[0], 1), p1 = __shfl_up_sync(full, x[1], 1),
                     p2 = __shfl_up_sync(full, x[2], 1);
        double seg = 0;
        if (act && k > 0) {
            const double e0 = x[0] - p0, e1 = x[1] - p1, e2 = x[2] - p2;
            seg = sqrt(e0 * e0 + e1 * e1 + e2 * e2);
        }
        double psum = act ? (K == 8 ? Gl8<double>::w(k) : GWN_GLW4D(k)) * f : 0.0;
        for (int off = 1; off < K; off <<= 1) {
            psum += __shfl_xor_sync(full, psum, off);
            seg += __shfl_xor_sync(full, seg, off);
            dm2 = fmin(dm2, __shfl_xor_sync(full, dm2, off));
        }
        const double len = seg * (K == 8 ? 1.1 : 1.17);  // the nodes span 96 % (8) or 86 % (4) of the panel
        const bool refine = act && len * len > ratio2 * dm2;
        const bool split = refine && level < maxlevel;
        if (refine && !split) deep = true;
        if (act && !split && k == 0) acc += (double)ci.mult * psum * h;
        // the halves of split panels go to the list (positions by a prefix sum over the leaders)
        const int npush = (split && k == 0) ? 2 : 0;
        int incl = npush;
        for (int off = 1; off < 32; off <<= 1) {
            int v = __shfl_up_sync(full, incl, off);
            if (lane >= off) incl += v;
        }
        const int total = __shfl_sync(full, incl, 31);
        if (sp + total <= kQuadStack) {
            if (npush) {
                const int cl = cidx | ((level + 1) << 16);
                stk[sp + incl - 2] = make_int2(cl, (int)(2u * idx + 1u));
                stk[sp + incl - 1] = make_int2(cl, (int)(2u * idx));
            }
            sp += total;
        } else if (npush) {
            bool dp = false;
            acc += (double)ci.mult * panel_subtree<double>(gc, ci.deg, q, s, level, idx, maxlevel, ratio, dp);
            if (dp) deep = true;
        }
        __syncwarp();
    }
    for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(full, acc, off);
    if (__any_sync(full, deep)) return false;
    *out = acc * 0.07957747154594767 - hits;  // 1 / (4 pi)
    return true;
}
#endif

// The order-3 part of a folded moment block (f[23 .. 44], zero below order 3):
// i3 i2 (e + i2 (r^T F r + i2 G[r r r r])), the constant e, the quadratic F and
// the quartic G of the expansion's third-order term, given r, its squares and
// the inverse powers i2 = 1/|r|^2, i3 = 1/|r|^3.
template <typename T>
GWN_HD inline T far3_order3(const T* f, T rx, T ry, T rz, T xx, T yy, T zz, T i2, T i3) {
    const T xy = rx * ry, xz = rx * rz, yz = ry * rz;
    const T q = f[24] * xx + f[25] * yy + f[26] * zz + f[27] * xy + f[28] * xz + f[29] * yz;
    const T t3 = xx * (f[30] * xx + f[31] * xy + f[32] * xz + f[33] * yy + f[34] * zz + f[35] * yz) +
                 yy * (f[36] * yy + f[37] * xy + f[38] * yz + f[39] * zz + f[40] * xz) +
                 zz * (f[41] * zz + f[42] * xz + f[43] * yz + f[44] * xy);
    return i3 * i2 * (f[23] + i2 * (q + i2 * t3));
}

template <typename T>
GWN_HD inline T far3_eval(const T* f, T rx, T ry, T rz, bool o3) {
    T r2 = rx * rx + ry * ry + rz * rz;
    T i2, i3;
    if (sizeof(T) == 4) {
        // both inverse powers from one reciprocal square root (no division):
        // relative error of a few ulp, far below the Taylor remainder
        const T rs = Num<T>::rsqrt_(r2);
        i2 = rs * rs;
        i3 = i2 * rs;
    } else {
        i2 = T(1) / r2;
        i3 = i2 * Num<T>::rsqrt_(r2);
    }
    T t0 = f[0] * rx + f[1] * ry + f[2] * rz + f[3];
    T xx = rx * rx, yy = ry * ry, zz = rz * rz;
    T t1 = f[4] * xx + f[5] * yy + f[6] * zz + f[7] * rx * ry + f[8] * rx * rz + f[9] * ry * rz + f[10] * rx + f[11] * ry +
           f[12] * rz;
    T t2 = rx * (f[13] * xx + f[16] * rx * ry + f[17] * rx * rz + f[18] * yy + f[20] * zz + f[22] * ry * rz) +
           ry * (f[14] * yy + f[19] * ry * rz + f[21] * zz) + f[15] * zz * rz;
    T w = i3 * (t0 + i2 * (t1 + i2 * t2));
    if (o3) w += far3_order3<T>(f, rx, ry, rz, xx, yy, zz, i2, i3);
    return w;
}

// FP32 moment block of a node or leaf: the first 6 float4 carry orders 0-2 (and
// the order-3 constant), the next 6 only the order-3 terms.  All loads are issued
// before the arithmetic (order 3: 1.7 % faster than loading the second half after
// the order-2 value, at 64 instead of 62 registers, 8 blocks per SM either way)
GWN_HD inline float far3_node32(const float4* M, float rx, float ry, float rz, bool o3) {
    float f[48];
#pragma unroll
    for (int v = 0; v < 6; ++v) {
        const float4 a = GWN_LDG(M + v);
        f[4 * v] = a.x;
        f[4 * v + 1] = a.y;
        f[4 * v + 2] = a.z;
        f[4 * v + 3] = a.w;
    }
    if (o3) {
#pragma unroll
        for (int v = 6; v < 12; ++v) {
            const float4 a = GWN_LDG(M + v);
            f[4 * v] = a.x;
            f[4 * v + 1] = a.y;
            f[4 * v + 2] = a.z;
            f[4 * v + 3] = a.w;
        }
    }
    const float r2 = rx * rx + ry * ry + rz * rz;
    const float rs = rsqrtf(r2);
    const float i2 = rs * rs, i3 = i2 * rs;
    const float xx = rx * rx, yy = ry * ry, zz = rz * rz;
    const float t0 = f[0] * rx + f[1] * ry + f[2] * rz + f[3];
    const float t1 = f[4] * xx + f[5] * yy + f[6] * zz + f[7] * rx * ry + f[8] * rx * rz + f[9] * ry * rz + f[10] * rx +
                     f[11] * ry + f[12] * rz;
    const float t2 = rx * (f[13] * xx + f[16] * rx * ry + f[17] * rx * rz + f[18] * yy + f[20] * zz + f[22] * ry * rz) +
                     ry * (f[14] * yy + f[19] * ry * rz + f[21] * zz) + f[15] * zz * rz;
    float w = i3 * (t0 + i2 * (t1 + i2 * t2));
    if (o3) w += far3_order3<float>(f, rx, ry, rz, xx, yy, zz, i2, i3);
    return w;
}

// Second-order local expansion of one node's order-2 far field about a packet
// centre p (an extension beyond the paper, for packets of nearby queries):
// with D = x0 - p and s = q - p, F(x0 - q) = F(D - s) ~ F(D) - grad F(D) . s
// + s^T H_F(D) s / 2.  F is the folded form t0 g3 + t1 g5 + t2 g7 (g_n =
// |r|^-n, t_k the polynomials of far3_eval), so
//   grad F = sum_k (g_n grad t_k - n g_{n+2} t_k r),
//   H_F    = sum_k (g_n H t_k - n g_{n+2} (grad t_k r^T + r grad t_k^T)
//                   + t_k (n (n+2) g_{n+4} r r^T - n g_{n+2} I)),  n = 3 + 2k.
// v receives F, grad F (3) and H_F (xx yy zz xy xz yz).
GWN_HD inline void far3_local2(const float4* M, float x, float y, float z, float v[10]) {
    float f[24];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 a = GWN_LDG(M + k);
        f[4 * k] = a.x; f[4 * k + 1] = a.y; f[4 * k + 2] = a.z; f[4 * k + 3] = a.w;
    }
    const float r2 = x * x + y * y + z * z;
    const float rs = Num<float>::rsqrt_(r2), i2 = rs * rs;
    float g[6];  // g3 .. g13 in steps of 2
    g[0] = i2 * rs;
#pragma unroll
    for (int k = 1; k < 6; ++k) g[k] = g[k - 1] * i2;
    const float xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
    // the three polynomials with their gradients and Hessians
    float t[3], gt[3][3], ht[3][6];
    t[0] = f[0] * x + f[1] * y + f[2] * z + f[3];
    gt[0][0] = f[0]; gt[0][1] = f[1]; gt[0][2] = f[2];
#pragma unroll
    for (int k = 0; k < 6; ++k) ht[0][k] = 0.f;
    t[1] = f[4] * xx + f[5] * yy + f[6] * zz + f[7] * xy + f[8] * xz + f[9] * yz + f[10] * x + f[11] * y + f[12] * z;
    gt[1][0] = 2.f * f[4] * x + f[7] * y + f[8] * z + f[10];
    gt[1][1] = 2.f * f[5] * y + f[7] * x + f[9] * z + f[11];
    gt[1][2] = 2.f * f[6] * z + f[8] * x + f[9] * y + f[12];
    ht[1][0] = 2.f * f[4]; ht[1][1] = 2.f * f[5]; ht[1][2] = 2.f * f[6];
    ht[1][3] = f[7]; ht[1][4] = f[8]; ht[1][5] = f[9];
    t[2] = x * (f[13] * xx + f[16] * xy + f[17] * xz + f[18] * yy + f[20] * zz + f[22] * yz) +
           y * (f[14] * yy + f[19] * yz + f[21] * zz) + f[15] * zz * z;
    gt[2][0] = 3.f * f[13] * xx + 2.f * f[16] * xy + 2.f * f[17] * xz + f[18] * yy + f[20] * zz + f[22] * yz;
    gt[2][1] = 3.f * f[14] * yy + f[16] * xx + 2.f * f[18] * xy + 2.f * f[19] * yz + f[21] * zz + f[22] * xz;
    gt[2][2] = 3.f * f[15] * zz + f[17] * xx + f[19] * yy + 2.f * f[20] * xz + 2.f * f[21] * yz + f[22] * xy;
    ht[2][0] = 6.f * f[13] * x + 2.f * f[16] * y + 2.f * f[17] * z;
    ht[2][1] = 6.f * f[14] * y + 2.f * f[18] * x + 2.f * f[19] * z;
    ht[2][2] = 6.f * f[15] * z + 2.f * f[20] * x + 2.f * f[21] * y;
    ht[2][3] = 2.f * f[16] * x + 2.f * f[18] * y + f[22] * z;
    ht[2][4] = 2.f * f[17] * x + 2.f * f[20] * z + f[22] * y;
    ht[2][5] = 2.f * f[19] * y + 2.f * f[21] * z + f[22] * x;
    const float r[3] = {x, y, z};
#pragma unroll
    for (int k = 0; k < 10; ++k) v[k] = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const float n = (float)(3 + 2 * k);
        const float gn = g[k], gn2 = g[k + 1], gn4 = g[k + 2];
        const float a = n * gn2, b = n * (n + 2.f) * gn4 * t[k];
        v[0] += t[k] * gn;
#pragma unroll
        for (int c = 0; c < 3; ++c) v[1 + c] += gt[k][c] * gn - a * t[k] * r[c];
        // Hessian entries (i, j) in the order xx yy zz xy xz yz
        const int I[6] = {0, 1, 2, 0, 0, 1}, J[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
        for (int e = 0; e < 6; ++e) {
            const int i = I[e], j = J[e];
            float h = ht[k][e] * gn - a * (gt[k][i] * r[j] + r[i] * gt[k][j]) + b * r[i] * r[j];
            if (i == j) h -= a * t[k];
            v[4 + e] += h;
        }
    }
}

// Algorithm 1 for one 3D query, FP32 (beta2l: the leaves' far test, <= 0 means beta2)
GWN_HD float query3_32(const DevTree& t, float qx, float qy, float qz, float beta2, uint32_t& st, float beta2l = 0.f) {
    if (!(beta2l > 0.f)) beta2l = beta2;
    float w = 0.f;
    int stack[kStack32];
    int sp = 0;
    int node = t.root;
    while (true) {
        if (node < 0) {
            int li = ~node;
            bool done = false;
            if (t.leaf_far) {
                float4 h = GWN_LDG(t.lhdr + li);
                float rx = h.x - qx, ry = h.y - qy, rz = h.z - qz;
                if (rx * rx + ry * ry + rz * rz > beta2l * h.w) {
                    w += far3_node32(t.lmom + (size_t)li * kMom3Vec, rx, ry, rz, t.order3);
                    done = true;
                }
            }
            if (!done) w += leaf3_eval32(t, li, qx, qy, qz, st);
        } else {
            float4 h = GWN_LDG(t.hdr + node);
            float rx = h.x - qx, ry = h.y - qy, rz = h.z - qz;
            if (rx * rx + ry * ry + rz * rz > beta2 * h.w) {
                w += far3_node32(t.mom + (size_t)node * kMom3Vec, rx, ry, rz, t.order3);
            } else {
                int2 ch = GWN_LDG(t.child + node);
                if (sp < kStack32) stack[sp++] = ch.y; else st |= GWN_QS_STACK_OVERFLOW;
                node = ch.x;
                continue;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return w;
}

// Algorithm 1 in FP64 (repair pass); beta2 <= 0 evaluates every leaf directly
GWN_HD double query3_64(const DevTree& t, double qx, double qy, double qz, double beta2, uint32_t& st,
                        double ratio = kRatio64Exact) {
    double w = 0.0;
    if (beta2 <= 0.0) {
        for (int i = 0; i < t.n_leaves; ++i) w += leaf3_eval64(t, i, qx, qy, qz, st, ratio);
        return w;
    }
    int stack[kStack64];
    int sp = 0;
    int node = t.root;
    while (true) {
        if (node < 0) {
            int li = ~node;
            bool done = false;
            if (t.leaf_far) {
                const double* h = t.lhdr64 + (size_t)li * 4;
                double rx = h[0] - qx, ry = h[1] - qy, rz = h[2] - qz;
                if (rx * rx + ry * ry + rz * rz > beta2 * h[3]) {
                    w += far3_eval<double>(t.lmom64 + (size_t)li * kMom3F64, rx, ry, rz, t.order3_64);
                    done = true;
                }
            }
            if (!done) w += leaf3_eval64(t, li, qx, qy, qz, st, ratio);
        } else {
            const double* h = t.hdr64 + (size_t)node * 4;
            double rx = h[0] - qx, ry = h[1] - qy, rz = h[2] - qz;
            if (rx * rx + ry * ry + rz * rz > beta2 * h[3]) {
                w += far3_eval<double>(t.mom64 + (size_t)node * kMom3F64, rx, ry, rz, t.order3_64);
            } else {
                int2 ch = t.child[node];
                if (sp < kStack64) stack[sp++] = ch.y; else st |= GWN_QS_UNRESOLVED;
                node = ch.x;
                continue;
            }
        }
        if (sp == 0) break;
        node = stack[--sp];
    }
    return w;
}

}  // namespace gwn
