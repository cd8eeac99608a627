// kernels2d.cuh -- device routines of the 2D query (Algorithm 1, query half).
//
// leaf2_eval: exact GWN of one cubic rational Bezier leaf (Section 3.3).  If q
//   lies outside the control-point box, the curve's GWN equals the angle its
//   chord subtends at q (the closed loop curve + reversed chord lies in the
//   convex hull, so it cannot wind around q); that angle is one atan2 of the
//   chord's cross and dot products, without normalisation.  Otherwise the curve
//   is bisected, depth first, until q is outside each piece's box.  The
//   traversal is stackless: a piece is identified by (level, index) and its
//   control points are recomputed from the leaf by two de Casteljau splits.
//   FP32 stops at level kNear32; a leaf that needs more is evaluated again in
//   FP64 -- the near-boundary band, i.e. q within ~2^-kNear32 of the leaf's
//   extent from the curve.
// far2: the order-2 Taylor expansion of Eq. 3 in folded form (gwn_internal.h).
// query2: the stack traversal of Algorithm 1.
#pragma once

#include "gwn_internal.h"
#include "../../include/gwn.h"

namespace gwn {

constexpr int kNear32 = 8;      // FP32 bisection levels before the FP64 near band
constexpr int kMaxLevel64 = 52; // FP64 bisection limit (then GWN_QS_UNRESOLVED)
constexpr int kStack32 = 64;
constexpr int kStack64 = 96;

template <typename T> struct Num;
template <> struct Num<float> {
    static GWN_HD inline float atan2_(float y, float x) { return atan2f(y, x); }
#if defined(__CUDA_ARCH__)
    static GWN_HD inline float inv_(float x) { return __frcp_rn(x); }
    static GWN_HD inline float rsqrt_(float x) { return rsqrtf(x); }
    // approximate reciprocal and square root (a few ulp) for the FP32 bulk of the
    // quadrature, whose error budget is 1e-4; sqrt_fast(0) is NaN
    static GWN_HD inline float rcp_fast(float x) { return __fdividef(1.0f, x); }
    static GWN_HD inline float sqrt_fast(float x) { return x * rsqrtf(x); }
#else
    static GWN_HD inline float inv_(float x) { return 1.0f / x; }
    static GWN_HD inline float rsqrt_(float x) { return 1.0f / sqrtf(x); }
    static GWN_HD inline float rcp_fast(float x) { return 1.0f / x; }
    static GWN_HD inline float sqrt_fast(float x) { return sqrtf(x); }
#endif
    static constexpr float inv2pi = 0.15915494309189535f;
};
template <> struct Num<double> {
    static GWN_HD inline double atan2_(double y, double x) { return atan2(y, x); }
    static GWN_HD inline double inv_(double x) { return 1.0 / x; }
    static GWN_HD inline double rcp_fast(double x) { return 1.0 / x; }
    static GWN_HD inline double sqrt_fast(double x) { return sqrt(x); }
#if defined(__CUDA_ARCH__)
    static GWN_HD inline double rsqrt_(double x) { return rsqrt(x); }
#else
    static GWN_HD inline double rsqrt_(double x) { return 1.0 / sqrt(x); }
#endif
    static constexpr double inv2pi = 0.15915494309189533577;
};

// split a cubic (3 homogeneous components) at t; keep the part selected by `left`
template <typename T>
GWN_HD inline void cubic_part(T (&h)[4][3], T t, bool left) {
    T a[3], b[3], c[3], d[3], e[3], f[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        a[k] = h[0][k] + t * (h[1][k] - h[0][k]);
        b[k] = h[1][k] + t * (h[2][k] - h[1][k]);
        c[k] = h[2][k] + t * (h[3][k] - h[2][k]);
        d[k] = a[k] + t * (b[k] - a[k]);
        e[k] = b[k] + t * (c[k] - b[k]);
        f[k] = d[k] + t * (e[k] - d[k]);
    }
    if (left) {
#pragma unroll
        for (int k = 0; k < 3; ++k) { h[1][k] = a[k]; h[2][k] = d[k]; h[3][k] = f[k]; }
    } else {
#pragma unroll
        for (int k = 0; k < 3; ++k) { h[0][k] = f[k]; h[1][k] = e[k]; h[2][k] = c[k]; }
    }
}

// Exact GWN (times 2 pi) of the cubic rational curve with homogeneous control
// points H (coordinates relative to q).  Returns false if more than maxlevel
// bisection levels would be needed.
template <typename T>
GWN_HD bool curve_angle(const T (&H)[4][3], int maxlevel, T* out) {
    T acc = 0;
    int level = 0;
    unsigned long long idx = 0;
    bool ok = true;
    while (true) {
        T h[4][3];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) h[i][k] = H[i][k];
        if (level > 0) {
            T sc = T(1) / T(1ull << level);   // exact power of two (level <= 62)
            T t0 = T(idx) * sc, t1 = T(idx + 1) * sc;
            if (t1 < T(1)) cubic_part(h, t1, true);
            if (t0 > T(0)) cubic_part(h, t0 / t1, false);
        }
        T ex[4], ey[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            T iw = Num<T>::inv_(h[i][2]);
            ex[i] = h[i][0] * iw;
            ey[i] = h[i][1] * iw;
        }
        T mnx = fmin(fmin(ex[0], ex[1]), fmin(ex[2], ex[3]));
        T mxx = fmax(fmax(ex[0], ex[1]), fmax(ex[2], ex[3]));
        T mny = fmin(fmin(ey[0], ey[1]), fmin(ey[2], ey[3]));
        T mxy = fmax(fmax(ey[0], ey[1]), fmax(ey[2], ey[3]));
        bool inside = mnx <= T(0) && mxx >= T(0) && mny <= T(0) && mxy >= T(0);
        if (inside && level < maxlevel) {
            ++level;
            idx <<= 1;
            continue;
        }
        if (inside) ok = false;
        acc += Num<T>::atan2_(ex[0] * ey[3] - ey[0] * ex[3], ex[0] * ex[3] + ey[0] * ey[3]);
        while (idx & 1ull) {
            idx >>= 1;
            --level;
        }
        if (level == 0) break;
        ++idx;
    }
    *out = acc;
    return ok;
}

// GWN of 2D leaf `li` at q; FP32 with the FP64 near band.
GWN_HD inline float leaf2_eval32(const DevTree& t, int li, float qx, float qy, uint32_t& st) {
    const float4* L = t.leaf2 + (size_t)li * kLeaf2Vec;
    float4 v0 = GWN_LDG(L + 0), v1 = GWN_LDG(L + 1), v2 = GWN_LDG(L + 2), v3 = GWN_LDG(L + 3);
    // q relative to the leaf centre, then control points relative to q
    float rx = qx - v3.x, ry = qy - v3.y;
    float px[4] = {v0.x - rx, v0.z - rx, v1.x - rx, v1.z - rx};
    float py[4] = {v0.y - ry, v0.w - ry, v1.y - ry, v1.w - ry};
    float mnx = fminf(fminf(px[0], px[1]), fminf(px[2], px[3]));
    float mxx = fmaxf(fmaxf(px[0], px[1]), fmaxf(px[2], px[3]));
    float mny = fminf(fminf(py[0], py[1]), fminf(py[2], py[3]));
    float mxy = fmaxf(fmaxf(py[0], py[1]), fmaxf(py[2], py[3]));
    if (mnx > 0.f || mxx < 0.f || mny > 0.f || mxy < 0.f)
        return atan2f(px[0] * py[3] - py[0] * px[3], px[0] * px[3] + py[0] * py[3]) * Num<float>::inv2pi;
    float H[4][3];
    float w[4] = {v2.x, v2.y, v2.z, v2.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        H[i][0] = w[i] * px[i];
        H[i][1] = w[i] * py[i];
        H[i][2] = w[i];
    }
    float a;
    if (curve_angle<float>(H, kNear32, &a)) return a * Num<float>::inv2pi;
    // near band: the whole leaf again in FP64
    st |= GWN_QS_NEAR;
    const double* D = t.leaf2_64 + (size_t)li * kLeaf2F64;
    double Hd[4][3];
    for (int i = 0; i < 4; ++i) {
        double wi = D[8 + i];
        Hd[i][0] = wi * (D[2 * i] - (double)qx);
        Hd[i][1] = wi * (D[2 * i + 1] - (double)qy);
        Hd[i][2] = wi;
    }
    double ad;
    if (!curve_angle<double>(Hd, kMaxLevel64, &ad)) st |= GWN_QS_UNRESOLVED;
    return (float)(ad * Num<double>::inv2pi);
}

GWN_HD inline double leaf2_eval64(const DevTree& t, int li, double qx, double qy, uint32_t& st) {
    const double* D = t.leaf2_64 + (size_t)li * kLeaf2F64;
    double Hd[4][3];
    double mnx = 1e300, mxx = -1e300, mny = 1e300, mxy = -1e300;
    for (int i = 0; i < 4; ++i) {
        double wi = D[8 + i];
        double px = D[2 * i] - qx, py = D[2 * i + 1] - qy;
        mnx = fmin(mnx, px); mxx = fmax(mxx, px);
        mny = fmin(mny, py); mxy = fmax(mxy, py);
        Hd[i][0] = wi * px;
        Hd[i][1] = wi * py;
        Hd[i][2] = wi;
    }
    if (mnx > 0 || mxx < 0 || mny > 0 || mxy < 0) {
        double x0 = D[0] - qx, y0 = D[1] - qy, x3 = D[6] - qx, y3 = D[7] - qy;
        return atan2(x0 * y3 - y0 * x3, x0 * x3 + y0 * y3) * Num<double>::inv2pi;
    }
    double ad;
    if (!curve_angle<double>(Hd, kMaxLevel64, &ad)) st |= GWN_QS_UNRESOLVED;
    return ad * Num<double>::inv2pi;
}

template <typename T>
GWN_HD inline T far2_eval(const T* f, T rx, T ry) {
    T r2 = rx * rx + ry * ry;
    T i2 = Num<T>::inv_(r2);
    T t0 = f[0] * rx + f[1] * ry + f[2];
    T t1 = (f[3] * rx + f[4] * ry + f[6]) * rx + (f[5] * ry + f[7]) * ry;
    T t2 = ((f[8] * rx + f[9] * ry) * rx + f[10] * ry * ry) * rx + f[11] * ry * ry * ry;
    return i2 * (t0 + i2 * (t1 + i2 * t2));
}

// Algorithm 1 for one 2D query, FP32.
GWN_HD float query2_32(const DevTree& t, float qx, float qy, float beta2, uint32_t& st, WorkLocal* wl = nullptr) {
    float w = 0.f;
    int stack[kStack32];
    int sp = 0;
    int node = t.root;
    while (true) {
        if (node < 0) {
            if (wl) wl->v[kWorkLeaves] += 1;
            w += leaf2_eval32(t, ~node, qx, qy, st);
        } else {
            if (wl) wl->v[kWorkNodes] += 1;
            float4 h = GWN_LDG(t.hdr + node);
            float rx = h.x - qx, ry = h.y - qy;
            if (rx * rx + ry * ry > beta2 * h.w) {
                if (wl) wl->v[kWorkFar] += 1;
                const float4* M = t.mom + (size_t)node * kMom2Vec;
                float4 a = GWN_LDG(M), b = GWN_LDG(M + 1), c = GWN_LDG(M + 2);
                float f[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
                w += far2_eval<float>(f, rx, ry);
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

// Algorithm 1 in FP64 (repair pass); beta2 <= 0 evaluates every leaf directly.
GWN_HD double query2_64(const DevTree& t, double qx, double qy, double beta2, uint32_t& st) {
    double w = 0.0;
    if (beta2 <= 0.0) {
        for (int i = 0; i < t.n_leaves; ++i) w += leaf2_eval64(t, i, qx, qy, st);
        return w;
    }
    int stack[kStack64];
    int sp = 0;
    int node = t.root;
    while (true) {
        if (node < 0) {
            w += leaf2_eval64(t, ~node, qx, qy, st);
        } else {
            const double* h = t.hdr64 + (size_t)node * 4;
            double rx = h[0] - qx, ry = h[1] - qy;
            if (rx * rx + ry * ry > beta2 * h[3]) {
                w += far2_eval<double>(t.mom64 + (size_t)node * kMom2F64, rx, ry);
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
