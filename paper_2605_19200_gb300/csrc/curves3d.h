// curves3d.h -- the per-leaf arithmetic of the 3D build (Section 3.1 leaf
// moments, and the boundary curves the near field integrates), written once
// for the host build (build3d.cpp) and for the device build stage
// (build_device.cu).  Both compile the same operations in the same order
// without fused multiply-adds (the host files with -ffp-contract=off, which
// g++ does not default to on aarch64; the device file with -fmad=false), with
// IEEE division and square root on both sides, so the two stages produce the
// same bits.
#pragma once

#include <cmath>
#include <cstdint>

#include "gwn_internal.h"

namespace gwn {

#if defined(__CUDACC__)
// device copy of the binomial table (filled by build_device.cu before its kernels run)
static __constant__ double c_binom64[40][40];
#endif

// binomial coefficients C(n, k), n < 40, from Pascal's rule in FP64 (the
// host table; device code reads the same numbers from c_binom64)
inline double binom64_host(int n, int k) {
    struct Table {
        double T[40][40];
        Table() {
            for (int a = 0; a < 40; ++a) {
                for (int b = 0; b < 40; ++b) T[a][b] = 0.0;
                T[a][0] = T[a][a] = 1.0;
                for (int b = 1; b < a; ++b) T[a][b] = T[a - 1][b - 1] + T[a - 1][b];
            }
        }
    };
    static const Table table;  // thread-safe one-time initialisation
    return table.T[n][k];
}
// The curve routines that pack_curve calls run out of line in device code,
// each in its own stack frame: inlined, nvcc 13.0 at -O3 gave the working
// array of bez4_eval the stack slot of pack_curve's composed points X, so the
// evaluations in curve_min_level overwrote X.
#if defined(__CUDA_ARCH__)
#define GWN_OUTLINE __noinline__
#else
#define GWN_OUTLINE
#endif

#if defined(__CUDA_ARCH__)
#define GWN_BINOM64(n, k) c_binom64[n][k]
#else
#define GWN_BINOM64(n, k) binom64_host(n, k)
#endif

struct TP {  // rational Bezier piece in (u, v), homogeneous (w u, w v, w), degree <= 3
    int deg;
    double h[4][3];
};

struct Net {  // bicubic rational Bezier net, [i_u][i_v] homogeneous (w x, w y, w z, w)
    double h[4][4][4];
};

// product of Bernstein polynomials a (degree m) and b (degree n)
GWN_HD inline void bmul(const double* a, int m, const double* b, int n, double* c) {
    for (int k = 0; k <= m + n; ++k) c[k] = 0;
    for (int i = 0; i <= m; ++i)
        for (int j = 0; j <= n; ++j)
            c[i + j] += GWN_BINOM64(m, i) * GWN_BINOM64(n, j) / GWN_BINOM64(m + n, i + j) * a[i] * b[j];
}

// point (and derivative) of a piece at t, by de Casteljau
GWN_HD inline void tp_eval(const TP& p, double t, double* x, double* dx) {
    double T[4][3];
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 3; ++k) T[i][k] = p.h[i][k];
    int n = p.deg;
    double D[3] = {0, 0, 0};
    for (int r = 1; r <= n; ++r) {
        if (r == n && dx)
            for (int k = 0; k < 3; ++k) D[k] = n * (T[1][k] - T[0][k]);
        for (int i = 0; i <= n - r; ++i)
            for (int k = 0; k < 3; ++k) T[i][k] = (1 - t) * T[i][k] + t * T[i + 1][k];
    }
    x[0] = T[0][0] / T[0][2];
    x[1] = T[0][1] / T[0][2];
    if (dx) {
        dx[0] = (D[0] - x[0] * D[2]) / T[0][2];
        dx[1] = (D[1] - x[1] * D[2]) / T[0][2];
    }
}

// degree elevation to a cubic (the local 2D curves of the trim membership test)
GWN_HD inline TP tp_elevate3(const TP& p) {
    TP q = p;
    while (q.deg < 3) {
        TP r;
        int n = q.deg;
        r.deg = n + 1;
        for (int k = 0; k < 3; ++k) {
            r.h[0][k] = q.h[0][k];
            r.h[n + 1][k] = q.h[n][k];
        }
        for (int i = 1; i <= n; ++i) {
            double a = (double)i / (n + 1);
            for (int k = 0; k < 3; ++k) r.h[i][k] = a * q.h[i - 1][k] + (1 - a) * q.h[i][k];
        }
        q = r;
    }
    return q;
}

// S, S_u, S_v of a net at local (u, v)
GWN_HD inline void net_eval(const Net& N, double u, double v, double* S, double* Su, double* Sv) {
    double Bu[4], Bv[4], dBu[4], dBv[4];
    {
        double s = 1 - u;
        Bu[0] = s * s * s; Bu[1] = 3 * u * s * s; Bu[2] = 3 * u * u * s; Bu[3] = u * u * u;
        dBu[0] = -3 * s * s; dBu[1] = 3 * s * s - 6 * u * s; dBu[2] = 6 * u * s - 3 * u * u; dBu[3] = 3 * u * u;
    }
    {
        double s = 1 - v;
        Bv[0] = s * s * s; Bv[1] = 3 * v * s * s; Bv[2] = 3 * v * v * s; Bv[3] = v * v * v;
        dBv[0] = -3 * s * s; dBv[1] = 3 * s * s - 6 * v * s; dBv[2] = 6 * v * s - 3 * v * v; dBv[3] = 3 * v * v;
    }
    double H[4] = {0, 0, 0, 0}, Hu[4] = {0, 0, 0, 0}, Hv[4] = {0, 0, 0, 0};
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 4; ++k) {
                double h = N.h[i][j][k];
                H[k] += Bu[i] * Bv[j] * h;
                Hu[k] += dBu[i] * Bv[j] * h;
                Hv[k] += Bu[i] * dBv[j] * h;
            }
    for (int k = 0; k < 3; ++k) S[k] = H[k] / H[3];
    if (Su)
        for (int k = 0; k < 3; ++k) {
            Su[k] = (Hu[k] - S[k] * Hu[3]) / H[3];
            Sv[k] = (Hv[k] - S[k] * Hv[3]) / H[3];
        }
}

// Leaf moments by Green's theorem on the leaf's local boundary (Section 3.1):
// int_D f du dv = oint F dv with F(u, v) = int_0^u f(s, v) ds, both integrals
// with the n-point Gauss-Legendre rule (gx, gw on [0, 1]).  mom receives the
// uncentred moments about xref, int n (3), int x n (9), int x x n (27) and
// int x x x n (81, for the order-3 far field); area = int |n|, ax = int x |n|
// (absolute x).
GWN_HD inline void leaf_moments_core(const Net& net, const TP* bnd, const double* mult, int nb, const double* xref,
                                     const double* gx, const double* gw, int n, double* mom, double* area,
                                     double* ax) {
    for (int k = 0; k < kLeafMom3; ++k) mom[k] = 0.0;
    *area = 0;
    ax[0] = ax[1] = ax[2] = 0;
    for (int pi = 0; pi < nb; ++pi) {
        const TP& P = bnd[pi];
        const double m = mult[pi];
        for (int a = 0; a < n; ++a) {
            double uv[2], duv[2];
            tp_eval(P, gx[a], uv, duv);
            double wo = m * gw[a] * duv[1];
            if (wo == 0.0) continue;
            for (int b = 0; b < n; ++b) {
                double s = uv[0] * gx[b];
                double wt = wo * uv[0] * gw[b];
                double S[3], Su[3], Sv[3];
                net_eval(net, s, uv[1], S, Su, Sv);
                double N[3] = {Su[1] * Sv[2] - Su[2] * Sv[1], Su[2] * Sv[0] - Su[0] * Sv[2], Su[0] * Sv[1] - Su[1] * Sv[0]};
                double nl = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
                double x[3] = {S[0] - xref[0], S[1] - xref[1], S[2] - xref[2]};
                for (int k = 0; k < 3; ++k) mom[k] += wt * N[k];
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) mom[3 + i * 3 + k] += wt * x[i] * N[k];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double xx = wt * x[i] * x[j];
                        for (int k = 0; k < 3; ++k) mom[12 + (i * 3 + j) * 3 + k] += xx * N[k];
                        for (int l = 0; l < 3; ++l) {
                            double xxx = xx * x[l];
                            for (int k = 0; k < 3; ++k) mom[39 + ((i * 3 + j) * 3 + l) * 3 + k] += xxx * N[k];
                        }
                    }
                *area += wt * nl;
                for (int k = 0; k < 3; ++k) ax[k] += wt * nl * S[k];
            }
        }
    }
}

// Compose a local (u, v) piece of degree d with the bicubic net: the rational
// Bezier space curve of degree 6 d, exactly,
//     X(t) = sum_ij C(3,i) C(3,j) U^i (W - U)^(3-i) V^j (W - V)^(3-j) h_ij,
// X holds (6 d + 1) homogeneous points of 4 doubles.
GWN_HD GWN_OUTLINE inline void compose(const TP& p, const Net& N, double* X) {
    int d = p.deg;
    double U[4], V[4], W[4], WU[4], WV[4];
    for (int i = 0; i <= d; ++i) {
        U[i] = p.h[i][0];
        V[i] = p.h[i][1];
        W[i] = p.h[i][2];
        WU[i] = W[i] - U[i];
        WV[i] = W[i] - V[i];
    }
    // Up[i] = U^i (W - U)^(3 - i), Vp[i] likewise, degree 3 d
    double Up[4][13], Vp[4][13], tmp[13];
    for (int i = 0; i < 4; ++i) {
        double cur[13] = {1.0};
        int deg = 0;
        for (int k = 0; k < 3; ++k) {
            bmul(cur, deg, k < i ? U : WU, d, tmp);
            deg += d;
            for (int c = 0; c <= deg; ++c) cur[c] = tmp[c];
        }
        for (int c = 0; c <= deg; ++c) Up[i][c] = cur[c];
        double cv[13] = {1.0};
        deg = 0;
        for (int k = 0; k < 3; ++k) {
            bmul(cv, deg, k < i ? V : WV, d, tmp);
            deg += d;
            for (int c = 0; c <= deg; ++c) cv[c] = tmp[c];
        }
        for (int c = 0; c <= deg; ++c) Vp[i][c] = cv[c];
    }
    const int D = 6 * d;
    for (int t = 0; t < (D + 1) * 4; ++t) X[t] = 0.0;
    double prod[19];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            bmul(Up[i], 3 * d, Vp[j], 3 * d, prod);
            double c = GWN_BINOM64(3, i) * GWN_BINOM64(3, j);
            for (int t = 0; t <= D; ++t)
                for (int k = 0; k < 4; ++k) X[t * 4 + k] += c * prod[t] * N.h[i][j][k];
        }
}

// homogeneous point and derivative of a degree-D Bezier curve (D + 1 points of
// 4 doubles in X) at t, by de Casteljau: the two points of the last-but-one
// level give the derivative D (b1 - b0) and the point (1 - t) b0 + t b1
GWN_HD GWN_OUTLINE inline void bez4_eval(const double* X, int D, double t, double P[4], double dP[4]) {
    double b[kMaxC3Deg + 1][4];
    for (int i = 0; i <= D; ++i)
        for (int c = 0; c < 4; ++c) b[i][c] = X[i * 4 + c];
    for (int r = 1; r < D; ++r)
        for (int i = 0; i <= D - r; ++i)
            for (int c = 0; c < 4; ++c) b[i][c] = (1 - t) * b[i][c] + t * b[i + 1][c];
    for (int c = 0; c < 4; ++c) {
        dP[c] = D * (b[1][c] - b[0][c]);
        P[c] = (1 - t) * b[0][c] + t * b[1][c];
    }
}

// position and tangent of the composed curve at t
GWN_HD inline void curve_point(const double* X, int D, double t, double x[3], double dx[3]) {
    double P[4], dP[4];
    bez4_eval(X, D, t, P, dP);
    for (int c = 0; c < 3; ++c) {
        x[c] = P[c] / P[3];
        dx[c] = (dP[c] - x[c] * dP[3]) / P[3];
    }
}

// Panel level from which the 4-point Gauss-Legendre rule of the FP32 line
// integral resolves the curve's own rational parametrisation.  The integrand
// carries the tangent x'(t) = (X' W - X W') / W^2, whose poles (the complex
// zeros of the weight W(t)) bound the rule's convergence: its error on a panel
// falls like rho^-8, rho the Bernstein-ellipse parameter of the nearest pole.
// On every panel of the returned level the rule must integrate x' itself --
// whose exact integral is the chord x(b) - x(a) -- to 1e-6 of the panel's arc
// length.  A quarter circle (weights 1, 1/sqrt 2, 1) composed with a bicubic
// net has its poles at t = 1/2 +- 1.21 i: rho ~ 5 on [0, 1], ~ 10 on its halves.
GWN_HD GWN_OUTLINE inline int curve_min_level(const double* X, int D, const double* x4, const double* w4) {
    for (int L = 0; L < kMaxMinLevel; ++L) {
        const int np = 1 << L;
        const double h = 1.0 / np;
        bool ok = true;
        for (int p = 0; p < np && ok; ++p) {
            double a[3], b[3], d[3], I[3] = {0, 0, 0}, arc = 0;
            curve_point(X, D, h * p, a, d);
            curve_point(X, D, h * (p + 1), b, d);
            for (int k = 0; k < 4; ++k) {
                double x[3];
                curve_point(X, D, h * (p + x4[k]), x, d);
                for (int c = 0; c < 3; ++c) I[c] += h * w4[k] * d[c];
                arc += h * w4[k] * sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            }
            const double e = sqrt((I[0] - (b[0] - a[0])) * (I[0] - (b[0] - a[0])) +
                                  (I[1] - (b[1] - a[1])) * (I[1] - (b[1] - a[1])) +
                                  (I[2] - (b[2] - a[2])) * (I[2] - (b[2] - a[2])));
            ok = e <= 1e-6 * arc;
        }
        if (ok) return L;
    }
    return kMaxMinLevel;
}

// the FP32 node table of one boundary curve (kC3NodeVec in gwn_internal.h):
// positions relative to the leaf centre and tangents at the 4 Gauss-Legendre
// nodes of the level-0 panel and of the two level-1 panels, and each panel's
// length estimate (chords between the nodes x the FP32 rule's span factor 1.17,
// as the kernels compute it).  A panel below the curve's minimum level gets an
// infinite length, so the table itself tells the kernel to skip it (level 0)
// or to leave the curve to the full evaluator (level 1).
GWN_HD GWN_OUTLINE inline void node_table(const double* X, int D, const float cen[3], float mult, int min_level, const double* x4,
                              float4 out[kC3NodeVec]) {
    const double a0[3] = {0.0, 0.0, 0.5}, hh[3] = {1.0, 0.5, 0.5};
    float len[3];
    for (int p = 0; p < 3; ++p) {
        float f[24];
        double prev[3] = {0, 0, 0}, L = 0;
        for (int k = 0; k < 4; ++k) {
            double x[3], dx[3];
            curve_point(X, D, a0[p] + hh[p] * x4[k], x, dx);
            for (int c = 0; c < 3; ++c) {
                f[6 * k + c] = (float)(x[c] - (double)cen[c]);
                f[6 * k + 3 + c] = (float)dx[c];
            }
            if (k > 0) L += sqrt((x[0] - prev[0]) * (x[0] - prev[0]) + (x[1] - prev[1]) * (x[1] - prev[1]) +
                                 (x[2] - prev[2]) * (x[2] - prev[2]));
            for (int c = 0; c < 3; ++c) prev[c] = x[c];
        }
        len[p] = (float)(1.17 * L);
        for (int v = 0; v < 6; ++v) {
            out[1 + 6 * p + v].x = f[4 * v];
            out[1 + 6 * p + v].y = f[4 * v + 1];
            out[1 + 6 * p + v].z = f[4 * v + 2];
            out[1 + 6 * p + v].w = f[4 * v + 3];
        }
    }
    out[0].x = min_level >= 1 ? INFINITY : len[0];
    out[0].y = min_level >= 2 ? INFINITY : len[1];
    out[0].z = min_level >= 2 ? INFINITY : len[2];
    out[0].w = mult;
}

// the FP64 node table of one boundary curve (kC3Node64 in gwn_internal.h):
// absolute positions and tangents at the 8 Gauss-Legendre nodes of the level-0
// panel and of the two level-1 panels, and the panels' length estimates with
// the 8-point rule's span factor 1.1 (as the FP64 kernels compute them)
GWN_HD GWN_OUTLINE inline void node_table64(const double* X, int D, double mult, const double* x8, double* out) {
    const double a0[3] = {0.0, 0.0, 0.5}, hh[3] = {1.0, 0.5, 0.5};
    for (int p = 0; p < 3; ++p) {
        double* nodes = out + 4 + 48 * p;
        double prev[3] = {0, 0, 0}, L = 0;
        for (int k = 0; k < 8; ++k) {
            curve_point(X, D, a0[p] + hh[p] * x8[k], nodes + 6 * k, nodes + 6 * k + 3);
            const double* x = nodes + 6 * k;
            if (k > 0) L += sqrt((x[0] - prev[0]) * (x[0] - prev[0]) + (x[1] - prev[1]) * (x[1] - prev[1]) +
                                 (x[2] - prev[2]) * (x[2] - prev[2]));
            for (int c = 0; c < 3; ++c) prev[c] = x[c];
        }
        out[p] = 1.1 * L;
    }
    out[3] = mult;
}

// The curve-point copies of one composed curve (Curve3Info in gwn_internal.h):
// D + 1 points scaled by C(D, i), then the D derivative points C(D-1, i)
// (c_{i+1} - c_i), then the same 2 D + 1 points of the reversed curve (read
// for t > 1/2); pts32 relative to the leaf centre (2 (2 D + 1) float4), pts64
// absolute (2 (2 D + 1) x 4 doubles)
GWN_HD GWN_OUTLINE inline void curve_points(const double* X, int D, const float cen[3], float4* pts32, double* pts64) {
    const int n = 2 * D + 1;
    double rel[(kMaxC3Deg + 1) * 4];
    for (int t = 0; t <= D; ++t) {
        const double* h = X + t * 4;
        double r4[4] = {h[0] - cen[0] * h[3], h[1] - cen[1] * h[3], h[2] - cen[2] * h[3], h[3]};
        for (int k = 0; k < 4; ++k) rel[t * 4 + k] = r4[k];
        double c = GWN_BINOM64(D, t);
        pts32[t].x = (float)(c * r4[0]);
        pts32[t].y = (float)(c * r4[1]);
        pts32[t].z = (float)(c * r4[2]);
        pts32[t].w = (float)(c * r4[3]);
        for (int k = 0; k < 4; ++k) pts64[t * 4 + k] = c * h[k];
    }
    for (int t = 0; t < D; ++t) {
        double c = GWN_BINOM64(D - 1, t);
        float f[4];
        for (int k = 0; k < 4; ++k) {
            f[k] = (float)(c * (rel[(t + 1) * 4 + k] - rel[t * 4 + k]));
            pts64[(D + 1 + t) * 4 + k] = c * (X[(t + 1) * 4 + k] - X[t * 4 + k]);
        }
        pts32[D + 1 + t].x = f[0];
        pts32[D + 1 + t].y = f[1];
        pts32[D + 1 + t].z = f[2];
        pts32[D + 1 + t].w = f[3];
    }
    // reversed copy: R_i = P_{D-i}, RQ_i = Q_{D-1-i}
    for (int t = 0; t <= D; ++t) {
        pts32[n + t] = pts32[D - t];
        for (int k = 0; k < 4; ++k) pts64[(n + t) * 4 + k] = pts64[(D - t) * 4 + k];
    }
    for (int t = 0; t < D; ++t) {
        pts32[n + D + 1 + t] = pts32[D + 1 + D - 1 - t];
        for (int k = 0; k < 4; ++k) pts64[(n + D + 1 + t) * 4 + k] = pts64[(D + 1 + D - 1 - t) * 4 + k];
    }
}

// everything the query kernels keep for one boundary piece of a leaf: its
// Curve3Info (ctrl_off filled in by the caller), point copies, node tables and
// the cubic local 2D curve of the trim membership test
GWN_HD inline void pack_curve(const TP& piece, double mult, const Net& net, const float cen[3], const double* x4,
                              const double* w4, const double* x8, Curve3Info* ci, float4* pts32, double* pts64,
                              float4* tab32, double* tab64, float4* c2, double* c2_64, float* c2mult) {
    double X[(kMaxC3Deg + 1) * 4];
    compose(piece, net, X);
    const int D = 6 * piece.deg;
    ci->deg = D;
    ci->mult = (float)mult;
    ci->min_level = curve_min_level(X, D, x4, w4);
    node_table(X, D, cen, ci->mult, ci->min_level, x4, tab32);
    node_table64(X, D, mult, x8, tab64);
    curve_points(X, D, cen, pts32, pts64);
    TP e3 = tp_elevate3(piece);
    float f[12];
    for (int t = 0; t < 4; ++t)
        for (int k = 0; k < 3; ++k) {
            f[t * 3 + k] = (float)e3.h[t][k];
            c2_64[t * 3 + k] = e3.h[t][k];
        }
    for (int v = 0; v < 3; ++v) {
        c2[v].x = f[4 * v];
        c2[v].y = f[4 * v + 1];
        c2[v].z = f[4 * v + 2];
        c2[v].w = f[4 * v + 3];
    }
    *c2mult = (float)mult;
}

}  // namespace gwn
