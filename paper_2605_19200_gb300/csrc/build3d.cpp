// build3d.cpp -- 3D preprocessing of Algorithm 1 for trimmed NURBS patches.
//
// Leaves.  Every patch is split at its knot lines into rational Bezier spans
// (degree-elevated to bicubic), and every span's parameter rectangle is
// bisected -- across the direction of larger physical extent of its control
// net -- until the net's box diagonal is below max_aabb_frac times the shape's
// box diagonal (Section 3.2) and its normals stay within a cone of half-angle
// kMaxConeDeg around their mean (so that a line along the mean normal meets
// the leaf at most once; the near-field evaluator relies on it).  A leaf keeps
// the visible part D cap R of its rectangle R: the trimming curves clipped to R
// plus the pieces of R's edges inside D, each counted with the trims' winding
// number there.  Leaves with an empty visible part are dropped.
//
// Moments (Section 3.1, Figure 3).  The uncentred moments int n, int x n,
// int x x n, the area int |n| and int x |n| of a leaf are integrated with
// Green's theorem on its visible region in local (u, v):
//     int_D f du dv = oint_{dD} F dv,   F(u, v) = int_0^u f(s, v) ds,
// both integrals with n-point Gauss-Legendre rules (n = quad_nodes, 10 by
// default) that reuse the same nodes for every integrand.
//
// Near-field data.  Each boundary piece of a leaf (a rational Bezier curve of
// degree d in local (u, v)) is composed with the leaf's bicubic net into a
// rational Bezier space curve of degree 6 d, exactly:
//     X(t) = sum_ij C(3,i) C(3,j) U^i (W - U)^(3-i) V^j (W - V)^(3-j) h_ij
// with (U, V, W) the piece's homogeneous coordinates.  The query kernels
// integrate the string potential along these curves (kernels3d.cuh).
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <thread>

#include "build.h"

namespace gwn {

namespace {

constexpr double kMaxConeDeg = 55.0;
constexpr int kMaxSplitDepth = 14;

struct BinomTable {
    double T[40][40];
    BinomTable() {
        for (int a = 0; a < 40; ++a) {
            for (int b = 0; b < 40; ++b) T[a][b] = 0.0;
            T[a][0] = T[a][a] = 1.0;
            for (int b = 1; b < a; ++b) T[a][b] = T[a - 1][b - 1] + T[a - 1][b];
        }
    }
};

double binom(int n, int k) {
    static const BinomTable table;  // thread-safe one-time initialisation
    return table.T[n][k];
}

// product of Bernstein polynomials a (degree m) and b (degree n)
void bmul(const double* a, int m, const double* b, int n, double* c) {
    for (int k = 0; k <= m + n; ++k) c[k] = 0;
    for (int i = 0; i <= m; ++i)
        for (int j = 0; j <= n; ++j) c[i + j] += binom(m, i) * binom(n, j) / binom(m + n, i + j) * a[i] * b[j];
}

// ---------------------------------------------------------------- 2D pieces

struct TP {  // rational Bezier piece in (u, v), homogeneous (w u, w v, w)
    int deg;
    double h[4][3];
};

void tp_eval(const TP& p, double t, double* x, double* dx) {
    double T[4][3];
    std::memcpy(T, p.h, sizeof(T));
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

void tp_split(const TP& p, double t, TP* L, TP* R) {
    double T[4][3];
    std::memcpy(T, p.h, sizeof(T));
    int n = p.deg;
    L->deg = R->deg = n;
    for (int k = 0; k < 3; ++k) { L->h[0][k] = T[0][k]; R->h[n][k] = T[n][k]; }
    for (int j = 1; j <= n; ++j) {
        for (int i = 0; i <= n - j; ++i)
            for (int k = 0; k < 3; ++k) T[i][k] = (1 - t) * T[i][k] + t * T[i + 1][k];
        for (int k = 0; k < 3; ++k) { L->h[j][k] = T[0][k]; R->h[n - j][k] = T[n - j][k]; }
    }
}

TP tp_sub(const TP& p, double a, double b) {
    TP L, R, out = p;
    if (b < 1.0) { tp_split(out, b, &L, &R); out = L; }
    if (a > 0.0) { tp_split(out, a / b, &L, &R); out = R; }
    return out;
}

TP tp_line(double u0, double v0, double u1, double v1) {
    TP p;
    p.deg = 1;
    p.h[0][0] = u0; p.h[0][1] = v0; p.h[0][2] = 1;
    p.h[1][0] = u1; p.h[1][1] = v1; p.h[1][2] = 1;
    return p;
}

TP tp_elevate3(const TP& p) {
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

// roots in [0, 1] of sum B_i(t) cf_i, isolated by halving: no sign change in
// the coefficients (zeros skipped) means no root inside; exactly one means one
// simple root, refined by bisection.  Roots at the ends are reported as well.
void bern_roots_rec(const double* cf, int n, double a, double b, int depth, std::vector<double>* out) {
    bool allz = true;
    for (int i = 0; i <= n; ++i) allz = allz && cf[i] == 0.0;
    if (allz) return;  // the piece runs along the line: no transversal crossing
    int var = 0, prev = 0;
    for (int i = 0; i <= n; ++i) {
        int sg = (cf[i] > 0) - (cf[i] < 0);
        if (sg != 0) {
            if (prev != 0 && sg != prev) ++var;
            prev = sg;
        }
    }
    if (var == 0) {
        if (cf[0] == 0) out->push_back(a);
        if (cf[n] == 0) out->push_back(b);
        return;
    }
    if (var == 1 && cf[0] != 0 && cf[n] != 0) {
        double lo = 0, hi = 1, flo = cf[0];
        for (int it = 0; it < 100; ++it) {
            double m = 0.5 * (lo + hi);
            double T[4];
            std::memcpy(T, cf, sizeof(double) * (n + 1));
            for (int r = 1; r <= n; ++r)
                for (int i = 0; i <= n - r; ++i) T[i] = (1 - m) * T[i] + m * T[i + 1];
            if (T[0] == 0) { lo = hi = m; break; }
            if ((T[0] < 0) == (flo < 0)) { lo = m; flo = T[0]; } else hi = m;
        }
        out->push_back(a + (b - a) * 0.5 * (lo + hi));
        return;
    }
    if (depth > 50 || b - a < 1e-15) {
        out->push_back(0.5 * (a + b));  // cluster of roots (tangency)
        return;
    }
    double T[4], Lc[4], Rc[4];
    std::memcpy(T, cf, sizeof(double) * (n + 1));
    Lc[0] = T[0];
    Rc[n] = T[n];
    for (int j = 1; j <= n; ++j) {
        for (int i = 0; i <= n - j; ++i) T[i] = 0.5 * (T[i] + T[i + 1]);
        Lc[j] = T[0];
        Rc[n - j] = T[n - j];
    }
    double m = 0.5 * (a + b);
    bern_roots_rec(Lc, n, a, m, depth + 1, out);
    bern_roots_rec(Rc, n, m, b, depth + 1, out);
}

void tp_cross(const TP& p, int axis, double c, std::vector<double>* roots) {
    double cf[4];
    for (int i = 0; i <= p.deg; ++i) cf[i] = p.h[i][axis] - c * p.h[i][2];
    bern_roots_rec(cf, p.deg, 0.0, 1.0, 0, roots);
}

// angle (radians) swept by the piece seen from x, by chord angles after
// bisecting while x is inside the control-point box
double tp_angle(const TP& p, const double* x, int depth) {
    double lo[2] = {1e300, 1e300}, hi[2] = {-1e300, -1e300};
    double e[4][2];
    for (int i = 0; i <= p.deg; ++i) {
        e[i][0] = p.h[i][0] / p.h[i][2] - x[0];
        e[i][1] = p.h[i][1] / p.h[i][2] - x[1];
        for (int k = 0; k < 2; ++k) {
            lo[k] = std::min(lo[k], e[i][k]);
            hi[k] = std::max(hi[k], e[i][k]);
        }
    }
    bool inside = lo[0] <= 0 && hi[0] >= 0 && lo[1] <= 0 && hi[1] >= 0;
    if (!inside || depth > 48) {
        const double* a = e[0];
        const double* b = e[p.deg];
        return std::atan2(a[0] * b[1] - a[1] * b[0], a[0] * b[0] + a[1] * b[1]);
    }
    TP L, R;
    tp_split(p, 0.5, &L, &R);
    return tp_angle(L, x, depth + 1) + tp_angle(R, x, depth + 1);
}

int winding(const std::vector<TP>& pcs, const double* x) {
    double acc = 0;
    for (auto& p : pcs) acc += tp_angle(p, x, 0);
    return (int)std::lround(acc / (2 * M_PI));
}

// ---------------------------------------------------------------- bicubic nets

struct Net {
    double h[4][4][4];  // [i_u][i_v] homogeneous (w x, w y, w z, w)
};

void net_eval(const Net& N, double u, double v, double* S, double* Su, double* Sv) {
    double Bu[4], Bv[4], dBu[4], dBv[4];
    auto bern = [](double t, double* B, double* dB) {
        double s = 1 - t;
        B[0] = s * s * s; B[1] = 3 * t * s * s; B[2] = 3 * t * t * s; B[3] = t * t * t;
        dB[0] = -3 * s * s; dB[1] = 3 * s * s - 6 * t * s; dB[2] = 6 * t * s - 3 * t * t; dB[3] = 3 * t * t;
    };
    bern(u, Bu, dBu);
    bern(v, Bv, dBv);
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

// restrict a bicubic net to [u0,u1] x [v0,v1] of its own [0,1]^2 domain
Net net_sub(const Net& N, double u0, double u1, double v0, double v1) {
    auto sub1 = [](double (*P)[4], double a, double b) {  // 4 points of 4 comps
        auto split = [](double (*Q)[4], double t, bool left) {
            double T[4][4];
            std::memcpy(T, Q, sizeof(T));
            double Lh[4][4], Rh[4][4];
            for (int k = 0; k < 4; ++k) { Lh[0][k] = T[0][k]; Rh[3][k] = T[3][k]; }
            for (int j = 1; j <= 3; ++j) {
                for (int i = 0; i <= 3 - j; ++i)
                    for (int k = 0; k < 4; ++k) T[i][k] = (1 - t) * T[i][k] + t * T[i + 1][k];
                for (int k = 0; k < 4; ++k) { Lh[j][k] = T[0][k]; Rh[3 - j][k] = T[3 - j][k]; }
            }
            std::memcpy(Q, left ? Lh : Rh, sizeof(T));
        };
        if (b < 1.0) split(P, b, true);
        if (a > 0.0) split(P, a / b, false);
    };
    Net out = N;
    for (int j = 0; j < 4; ++j) {
        double P[4][4];
        for (int i = 0; i < 4; ++i) std::memcpy(P[i], out.h[i][j], sizeof(P[i]));
        sub1(P, u0, u1);
        for (int i = 0; i < 4; ++i) std::memcpy(out.h[i][j], P[i], sizeof(P[i]));
    }
    for (int i = 0; i < 4; ++i) {
        double P[4][4];
        for (int j = 0; j < 4; ++j) std::memcpy(P[j], out.h[i][j], sizeof(P[j]));
        sub1(P, v0, v1);
        for (int j = 0; j < 4; ++j) std::memcpy(out.h[i][j], P[j], sizeof(P[j]));
    }
    return out;
}

void net_box(const Net& N, double* lo, double* hi) {
    for (int k = 0; k < 3; ++k) { lo[k] = 1e300; hi[k] = -1e300; }
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j)
            for (int k = 0; k < 3; ++k) {
                double x = N.h[i][j][k] / N.h[i][j][3];
                lo[k] = std::min(lo[k], x);
                hi[k] = std::max(hi[k], x);
            }
}

double dist3(const double* a, const double* b) {
    return std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
}

// ---------------------------------------------------------------- leaves

struct Rect {
    double u0, u1, v0, v1;
};

struct Leaf {
    int64_t prim;
    Rect R;              // global parameter rectangle
    Net net;             // bicubic net on R, local [0,1]^2
    std::vector<TP> bnd; // visible boundary in local coordinates
    std::vector<double> mult;
    double lo[3], hi[3];
    double mom[39];      // uncentred moments about xref
    double area, ax[3];  // int |n|, int x |n| (absolute x)
    double nrm[3];
};

struct PatchWork {
    int64_t prim;
    std::vector<std::pair<Rect, Net>> spans;  // span rectangles (global) with their bicubic nets
    std::vector<TP> trims;                    // global (u, v) pieces
    bool untrimmed;
};

// boundary of (visible region) cap R, in global (u, v), with multiplicities
void clip_boundary(const PatchWork& P, const Rect& R, std::vector<TP>* out, std::vector<double>* mult) {
    out->clear();
    mult->clear();
    if (P.untrimmed) {
        out->push_back(tp_line(R.u0, R.v0, R.u1, R.v0));
        out->push_back(tp_line(R.u1, R.v0, R.u1, R.v1));
        out->push_back(tp_line(R.u1, R.v1, R.u0, R.v1));
        out->push_back(tp_line(R.u0, R.v1, R.u0, R.v0));
        mult->assign(4, 1.0);
        return;
    }
    const double eu = 1e-13 * (R.u1 - R.u0), ev = 1e-13 * (R.v1 - R.v0);
    for (const TP& T : P.trims) {
        std::vector<double> r;
        tp_cross(T, 0, R.u0, &r);
        tp_cross(T, 0, R.u1, &r);
        tp_cross(T, 1, R.v0, &r);
        tp_cross(T, 1, R.v1, &r);
        r.push_back(0.0);
        r.push_back(1.0);
        std::sort(r.begin(), r.end());
        for (size_t k = 0; k + 1 < r.size(); ++k) {
            double a = std::max(0.0, r[k]), b = std::min(1.0, r[k + 1]);
            if (b - a < 1e-13) continue;
            double mid[2];
            tp_eval(T, 0.5 * (a + b), mid, nullptr);
            if (mid[0] > R.u0 + eu && mid[0] < R.u1 - eu && mid[1] > R.v0 + ev && mid[1] < R.v1 - ev) {
                out->push_back(tp_sub(T, a, b));
                mult->push_back(1.0);
            }
        }
    }
    // the rectangle's edges, counter-clockwise, weighted by the trims' winding number
    double C[5][2] = {{R.u0, R.v0}, {R.u1, R.v0}, {R.u1, R.v1}, {R.u0, R.v1}, {R.u0, R.v0}};
    for (int e = 0; e < 4; ++e) {
        const double* A = C[e];
        const double* B = C[e + 1];
        int axis = (e % 2 == 0) ? 1 : 0;  // bottom/top: v constant; right/left: u constant
        double cval = A[axis];
        int other = 1 - axis;
        std::vector<double> s = {0.0, 1.0};
        for (const TP& T : P.trims) {
            std::vector<double> r;
            tp_cross(T, axis, cval, &r);
            for (double t : r) {
                double x[2];
                tp_eval(T, t, x, nullptr);
                double lam = (x[other] - A[other]) / (B[other] - A[other]);
                if (lam > 0 && lam < 1) s.push_back(lam);
            }
        }
        std::sort(s.begin(), s.end());
        for (size_t k = 0; k + 1 < s.size(); ++k) {
            double a = s[k], b = s[k + 1];
            if (b - a < 1e-13) continue;
            double m = 0.5 * (a + b);
            double x[2] = {A[0] + m * (B[0] - A[0]), A[1] + m * (B[1] - A[1])};
            int w = winding(P.trims, x);
            if (w != 0) {
                out->push_back(tp_line(A[0] + a * (B[0] - A[0]), A[1] + a * (B[1] - A[1]), A[0] + b * (B[0] - A[0]),
                                       A[1] + b * (B[1] - A[1])));
                mult->push_back((double)w);
            }
        }
    }
}

// global (u, v) piece -> local coordinates of rectangle R
TP to_local(const TP& p, const Rect& R) {
    TP q = p;
    double du = R.u1 - R.u0, dv = R.v1 - R.v0;
    for (int i = 0; i <= p.deg; ++i) {
        q.h[i][0] = (p.h[i][0] - R.u0 * p.h[i][2]) / du;
        q.h[i][1] = (p.h[i][1] - R.v0 * p.h[i][2]) / dv;
    }
    return q;
}

bool cone_ok(const Net& N, double* nrm) {
    double acc[3] = {0, 0, 0};
    double ns[5][5][3];
    bool ok = true;
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) {
            double S[3], Su[3], Sv[3];
            net_eval(N, a / 4.0, b / 4.0, S, Su, Sv);
            double n[3] = {Su[1] * Sv[2] - Su[2] * Sv[1], Su[2] * Sv[0] - Su[0] * Sv[2], Su[0] * Sv[1] - Su[1] * Sv[0]};
            double l = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (!(l > 0)) ok = false;
            for (int k = 0; k < 3; ++k) {
                ns[a][b][k] = l > 0 ? n[k] / l : 0.0;
                acc[k] += ns[a][b][k];
            }
        }
    double l = std::sqrt(acc[0] * acc[0] + acc[1] * acc[1] + acc[2] * acc[2]);
    if (!(l > 0)) {
        nrm[0] = 0; nrm[1] = 0; nrm[2] = 1;
        return false;
    }
    for (int k = 0; k < 3; ++k) nrm[k] = acc[k] / l;
    double cmin = std::cos(kMaxConeDeg * M_PI / 180.0);
    for (int a = 0; a < 5; ++a)
        for (int b = 0; b < 5; ++b) {
            double c = ns[a][b][0] * nrm[0] + ns[a][b][1] * nrm[1] + ns[a][b][2] * nrm[2];
            if (c < cmin) ok = false;
        }
    return ok;
}

// moments by Green's theorem on the leaf's local boundary
void leaf_moments(Leaf& L, const double* xref, const std::vector<double>& gx, const std::vector<double>& gw) {
    std::fill(L.mom, L.mom + 39, 0.0);
    L.area = 0;
    L.ax[0] = L.ax[1] = L.ax[2] = 0;
    const int n = (int)gx.size();
    for (size_t pi = 0; pi < L.bnd.size(); ++pi) {
        const TP& P = L.bnd[pi];
        const double m = L.mult[pi];
        for (int a = 0; a < n; ++a) {
            double uv[2], duv[2];
            tp_eval(P, gx[a], uv, duv);
            double wo = m * gw[a] * duv[1];
            if (wo == 0.0) continue;
            for (int b = 0; b < n; ++b) {
                double s = uv[0] * gx[b];
                double wt = wo * uv[0] * gw[b];
                double S[3], Su[3], Sv[3];
                net_eval(L.net, s, uv[1], S, Su, Sv);
                double N[3] = {Su[1] * Sv[2] - Su[2] * Sv[1], Su[2] * Sv[0] - Su[0] * Sv[2], Su[0] * Sv[1] - Su[1] * Sv[0]};
                double nl = std::sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
                double x[3] = {S[0] - xref[0], S[1] - xref[1], S[2] - xref[2]};
                for (int k = 0; k < 3; ++k) L.mom[k] += wt * N[k];
                for (int i = 0; i < 3; ++i)
                    for (int k = 0; k < 3; ++k) L.mom[3 + i * 3 + k] += wt * x[i] * N[k];
                for (int i = 0; i < 3; ++i)
                    for (int j = 0; j < 3; ++j) {
                        double xx = wt * x[i] * x[j];
                        for (int k = 0; k < 3; ++k) L.mom[12 + (i * 3 + j) * 3 + k] += xx * N[k];
                    }
                L.area += wt * nl;
                for (int k = 0; k < 3; ++k) L.ax[k] += wt * nl * S[k];
            }
        }
    }
}

void gauss_legendre01(int n, std::vector<double>* x, std::vector<double>* w) {
    x->resize(n);
    w->resize(n);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 1;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1, p2 = 0;
            for (int j = 1; j <= n; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = n * (z * p1 - p2) / (z * z - 1);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        (*x)[i] = 0.5 * (1 - z);
        (*w)[i] = 1.0 / ((1 - z * z) * pp * pp);
    }
}

// homogeneous point and derivative of a degree-D Bezier curve (D + 1 points of
// 4 doubles in X) at t, by de Casteljau: the two points of the last-but-one
// level give the derivative D (b1 - b0) and the point (1 - t) b0 + t b1
void bez4_eval(const std::vector<double>& X, int D, double t, double P[4], double dP[4]) {
    double b[kMaxC3Deg + 1][4];
    for (int i = 0; i <= D; ++i)
        for (int c = 0; c < 4; ++c) b[i][c] = X[(size_t)i * 4 + c];
    for (int r = 1; r < D; ++r)
        for (int i = 0; i <= D - r; ++i)
            for (int c = 0; c < 4; ++c) b[i][c] = (1 - t) * b[i][c] + t * b[i + 1][c];
    for (int c = 0; c < 4; ++c) {
        dP[c] = D * (b[1][c] - b[0][c]);
        P[c] = (1 - t) * b[0][c] + t * b[1][c];
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
int curve_min_level(const std::vector<double>& X, int D, const std::vector<double>& x4, const std::vector<double>& w4) {
    auto point = [&](double t, double x[3], double dx[3]) {
        double P[4], dP[4];
        bez4_eval(X, D, t, P, dP);
        for (int c = 0; c < 3; ++c) {
            x[c] = P[c] / P[3];
            dx[c] = (dP[c] - x[c] * dP[3]) / P[3];
        }
    };
    for (int L = 0; L < kMaxMinLevel; ++L) {
        const int np = 1 << L;
        const double h = 1.0 / np;
        bool ok = true;
        for (int p = 0; p < np && ok; ++p) {
            double a[3], b[3], d[3], I[3] = {0, 0, 0}, arc = 0;
            point(h * p, a, d);
            point(h * (p + 1), b, d);
            for (size_t k = 0; k < x4.size(); ++k) {
                double x[3];
                point(h * (p + x4[k]), x, d);
                for (int c = 0; c < 3; ++c) I[c] += h * w4[k] * d[c];
                arc += h * w4[k] * std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            }
            const double e = std::sqrt((I[0] - (b[0] - a[0])) * (I[0] - (b[0] - a[0])) +
                                       (I[1] - (b[1] - a[1])) * (I[1] - (b[1] - a[1])) +
                                       (I[2] - (b[2] - a[2])) * (I[2] - (b[2] - a[2])));
            ok = e <= 1e-6 * arc;
        }
        if (ok) return L;
    }
    return kMaxMinLevel;
}

// the node table of one boundary curve (Curve3Info / kC3NodeVec in
// gwn_internal.h): positions relative to the leaf centre and derivatives at
// the 4 Gauss-Legendre nodes of the level-0 panel and of the two level-1
// panels, and each panel's length estimate (chords between the nodes x the
// FP32 rule's span factor 1.17, as the kernels compute it)
void node_table(const std::vector<double>& X, int D, const float cen[3], float mult, const std::vector<double>& x4,
                float4 out[kC3NodeVec]) {
    const double a0[3] = {0.0, 0.0, 0.5}, hh[3] = {1.0, 0.5, 0.5};
    float len[3];
    for (int p = 0; p < 3; ++p) {
        float f[24];
        double prev[3] = {0, 0, 0}, L = 0;
        for (int k = 0; k < 4; ++k) {
            double P[4], dP[4];
            bez4_eval(X, D, a0[p] + hh[p] * x4[k], P, dP);
            double x[3];
            for (int c = 0; c < 3; ++c) {
                x[c] = P[c] / P[3];
                f[6 * k + c] = (float)(x[c] - (double)cen[c]);
                f[6 * k + 3 + c] = (float)((dP[c] - x[c] * dP[3]) / P[3]);
            }
            if (k > 0) L += std::sqrt((x[0] - prev[0]) * (x[0] - prev[0]) + (x[1] - prev[1]) * (x[1] - prev[1]) +
                                      (x[2] - prev[2]) * (x[2] - prev[2]));
            for (int c = 0; c < 3; ++c) prev[c] = x[c];
        }
        len[p] = (float)(1.17 * L);
        for (int v = 0; v < 6; ++v) out[1 + 6 * p + v] = float4{f[4 * v], f[4 * v + 1], f[4 * v + 2], f[4 * v + 3]};
    }
    out[0] = float4{len[0], len[1], len[2], mult};
}

// the FP64 node table of one boundary curve (kC3Node64 in gwn_internal.h):
// absolute positions and tangents at the 8 Gauss-Legendre nodes of the level-0
// panel and of the two level-1 panels, and the panels' length estimates with
// the 8-point rule's span factor 1.1 (as the FP64 kernels compute them)
void node_table64(const std::vector<double>& X, int D, double mult, const std::vector<double>& x8, double* out) {
    const double a0[3] = {0.0, 0.0, 0.5}, hh[3] = {1.0, 0.5, 0.5};
    for (int p = 0; p < 3; ++p) {
        double* nodes = out + 4 + 48 * p;
        double prev[3] = {0, 0, 0}, L = 0;
        for (int k = 0; k < 8; ++k) {
            double P[4], dP[4];
            bez4_eval(X, D, a0[p] + hh[p] * x8[k], P, dP);
            for (int c = 0; c < 3; ++c) {
                const double x = P[c] / P[3];
                nodes[6 * k + c] = x;
                nodes[6 * k + 3 + c] = (dP[c] - x * dP[3]) / P[3];
            }
            const double* x = nodes + 6 * k;
            if (k > 0) L += std::sqrt((x[0] - prev[0]) * (x[0] - prev[0]) + (x[1] - prev[1]) * (x[1] - prev[1]) +
                                      (x[2] - prev[2]) * (x[2] - prev[2]));
            for (int c = 0; c < 3; ++c) prev[c] = x[c];
        }
        out[p] = 1.1 * L;
    }
    out[3] = mult;
}

// compose a local (u, v) piece with the bicubic net: 4D rational Bezier of degree 6 deg
void compose(const TP& p, const Net& N, std::vector<double>* X) {
    int d = p.deg;
    double U[4], V[4], W[4], WU[4], WV[4];
    for (int i = 0; i <= d; ++i) {
        U[i] = p.h[i][0];
        V[i] = p.h[i][1];
        W[i] = p.h[i][2];
        WU[i] = W[i] - U[i];
        WV[i] = W[i] - V[i];
    }
    // Upow[i] = U^i (W - U)^(3 - i), degree 3 d
    double Up[4][13], Vp[4][13], tmp[13], tmp2[13];
    for (int i = 0; i < 4; ++i) {
        double cur[13] = {1.0};
        int deg = 0;
        for (int k = 0; k < i; ++k) { bmul(cur, deg, U, d, tmp); deg += d; std::memcpy(cur, tmp, sizeof(double) * (deg + 1)); }
        for (int k = i; k < 3; ++k) { bmul(cur, deg, WU, d, tmp); deg += d; std::memcpy(cur, tmp, sizeof(double) * (deg + 1)); }
        std::memcpy(Up[i], cur, sizeof(double) * (deg + 1));
        double cv[13] = {1.0};
        deg = 0;
        for (int k = 0; k < i; ++k) { bmul(cv, deg, V, d, tmp2); deg += d; std::memcpy(cv, tmp2, sizeof(double) * (deg + 1)); }
        for (int k = i; k < 3; ++k) { bmul(cv, deg, WV, d, tmp2); deg += d; std::memcpy(cv, tmp2, sizeof(double) * (deg + 1)); }
        std::memcpy(Vp[i], cv, sizeof(double) * (deg + 1));
    }
    const int D = 6 * d;
    X->assign((size_t)(D + 1) * 4, 0.0);
    double prod[19];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            bmul(Up[i], 3 * d, Vp[j], 3 * d, prod);
            double c = binom(3, i) * binom(3, j);
            for (int t = 0; t <= D; ++t)
                for (int k = 0; k < 4; ++k) (*X)[t * 4 + k] += c * prod[t] * N.h[i][j][k];
        }
}

void make_leaves(const PatchWork& P, const gwn_build_opts& o, double sdiag, const double* xref,
                 const std::vector<double>& gx, const std::vector<double>& gw, std::vector<Leaf>* out) {
    const double lim = o.max_aabb_frac > 0 ? o.max_aabb_frac * sdiag : 1e300;
    struct Item {
        Rect R;        // global
        Rect loc;      // within the span's [0,1]^2
        int span;
        int depth;
    };
    std::vector<Item> st;
    for (int s = 0; s < (int)P.spans.size(); ++s) st.push_back({P.spans[s].first, {0, 1, 0, 1}, s, 0});
    std::vector<TP> bnd;
    std::vector<double> mult;
    while (!st.empty()) {
        Item it = st.back();
        st.pop_back();
        Net net = net_sub(P.spans[it.span].second, it.loc.u0, it.loc.u1, it.loc.v0, it.loc.v1);
        clip_boundary(P, it.R, &bnd, &mult);
        if (bnd.empty()) continue;  // invisible
        double lo[3], hi[3], nrm[3];
        net_box(net, lo, hi);
        bool cone = cone_ok(net, nrm);
        bool big = dist3(lo, hi) >= lim;
        if ((big || !cone) && it.depth < kMaxSplitDepth) {
            // split across the direction of larger physical extent of the net
            double eu = 0, ev = 0;
            for (int j = 0; j < 4; ++j) {
                double a[3], b[3], c[3];
                for (int k = 0; k < 3; ++k) {
                    a[k] = net.h[0][j][k] / net.h[0][j][3];
                    b[k] = net.h[3][j][k] / net.h[3][j][3];
                }
                eu += dist3(a, b);
                for (int k = 0; k < 3; ++k) {
                    a[k] = net.h[j][0][k] / net.h[j][0][3];
                    c[k] = net.h[j][3][k] / net.h[j][3][3];
                }
                ev += dist3(a, c);
            }
            if (eu >= ev) {
                double gm = 0.5 * (it.R.u0 + it.R.u1), lm = 0.5 * (it.loc.u0 + it.loc.u1);
                st.push_back({{it.R.u0, gm, it.R.v0, it.R.v1}, {it.loc.u0, lm, it.loc.v0, it.loc.v1}, it.span, it.depth + 1});
                st.push_back({{gm, it.R.u1, it.R.v0, it.R.v1}, {lm, it.loc.u1, it.loc.v0, it.loc.v1}, it.span, it.depth + 1});
            } else {
                double gm = 0.5 * (it.R.v0 + it.R.v1), lm = 0.5 * (it.loc.v0 + it.loc.v1);
                st.push_back({{it.R.u0, it.R.u1, it.R.v0, gm}, {it.loc.u0, it.loc.u1, it.loc.v0, lm}, it.span, it.depth + 1});
                st.push_back({{it.R.u0, it.R.u1, gm, it.R.v1}, {it.loc.u0, it.loc.u1, lm, it.loc.v1}, it.span, it.depth + 1});
            }
            continue;
        }
        Leaf L;
        L.prim = P.prim;
        L.R = it.R;
        L.net = net;
        for (auto& b : bnd) L.bnd.push_back(to_local(b, it.R));
        L.mult = mult;
        std::memcpy(L.lo, lo, sizeof(lo));
        std::memcpy(L.hi, hi, sizeof(hi));
        std::memcpy(L.nrm, nrm, sizeof(nrm));
        leaf_moments(L, xref, gx, gw);
        out->push_back(std::move(L));
    }
}

std::string validate_curve(const gwn_curve2d& C, double U0, double U1, double V0, double V1) {
    if (C.degree < 1 || C.degree > 3) return "trim degree must be 1..3";
    if (C.n_ctrl < C.degree + 1) return "trim has too few control points";
    if (!C.ctrl || !C.knots) return "trim has NULL control points or knots";
    std::string e = check_knots(C.degree, C.n_ctrl, C.knots);
    if (!e.empty()) return "trim: " + e;
    double tu = 1e-9 * (U1 - U0), tv = 1e-9 * (V1 - V0);
    for (int i = 0; i < C.n_ctrl; ++i) {
        double w = C.weights ? C.weights[i] : 1.0;
        double u = C.ctrl[2 * i], v = C.ctrl[2 * i + 1];
        if (!(w > 0) || !std::isfinite(w) || !std::isfinite(u) || !std::isfinite(v)) return "trim: bad point or weight";
        if (u < U0 - tu || u > U1 + tu || v < V0 - tv || v > V1 + tv) return "trim outside the parameter domain";
    }
    return "";
}

}  // namespace

// The boundary data of one leaf (curves composed with its net, their point
// copies, node tables and local 2D curves), packed on its own so that leaves
// are packed in parallel; ctrl_off counts from the leaf's first curve point.
struct LeafPack {
    std::vector<Curve3Info> c3;
    std::vector<float4> c3pts;
    std::vector<double> c3pts64;
    std::vector<float4> c3n;
    std::vector<double> c3n64;
    std::vector<float4> c2;
    std::vector<double> c2_64;
    std::vector<float> c2mult;
};

void pack_leaf(const Leaf& L, const float cen[3], const std::vector<double>& g4x, const std::vector<double>& g4w,
               const std::vector<double>& g8x, LeafPack* P) {
    std::vector<double> X;
    for (size_t b = 0; b < L.bnd.size(); ++b) {
        compose(L.bnd[b], L.net, &X);
        int D = 6 * L.bnd[b].deg;
        Curve3Info ci;
        ci.ctrl_off = (int32_t)P->c3pts.size();
        ci.deg = D;
        ci.mult = (float)L.mult[b];
        ci.min_level = curve_min_level(X, D, g4x, g4w);
        P->c3.push_back(ci);
        {
            float4 tab[kC3NodeVec];
            node_table(X, D, cen, ci.mult, g4x, tab);
            P->c3n.insert(P->c3n.end(), tab, tab + kC3NodeVec);
            double tab64[kC3Node64];
            node_table64(X, D, (double)L.mult[b], g8x, tab64);
            P->c3n64.insert(P->c3n64.end(), tab64, tab64 + kC3Node64);
        }
        // D + 1 points scaled by C(D, i), then D derivative points C(D-1, i) (c_{i+1} - c_i),
        // then the same 2 D + 1 points of the reversed curve (evaluation for t > 1/2);
        // float copies relative to the leaf centre, double copies absolute
        std::vector<double> rel((size_t)(D + 1) * 4);
        for (int t = 0; t <= D; ++t) {
            const double* h = &X[(size_t)t * 4];
            double r4[4] = {h[0] - cen[0] * h[3], h[1] - cen[1] * h[3], h[2] - cen[2] * h[3], h[3]};
            for (int k = 0; k < 4; ++k) rel[(size_t)t * 4 + k] = r4[k];
            double c = binom(D, t);
            P->c3pts.push_back(float4{(float)(c * r4[0]), (float)(c * r4[1]), (float)(c * r4[2]), (float)(c * r4[3])});
            for (int k = 0; k < 4; ++k) P->c3pts64.push_back(c * h[k]);
        }
        for (int t = 0; t < D; ++t) {
            double c = binom(D - 1, t);
            float f[4];
            for (int k = 0; k < 4; ++k) {
                f[k] = (float)(c * (rel[(size_t)(t + 1) * 4 + k] - rel[(size_t)t * 4 + k]));
                P->c3pts64.push_back(c * (X[(size_t)(t + 1) * 4 + k] - X[(size_t)t * 4 + k]));
            }
            P->c3pts.push_back(float4{f[0], f[1], f[2], f[3]});
        }
        {
            // reversed copy: R_i = P_{D-i}, RQ_i = Q_{D-1-i}
            const size_t f0 = (size_t)ci.ctrl_off, d0 = (size_t)ci.ctrl_off * 4;
            for (int t = 0; t <= D; ++t) {
                P->c3pts.push_back(P->c3pts[f0 + (size_t)(D - t)]);
                for (int k = 0; k < 4; ++k) P->c3pts64.push_back(P->c3pts64[d0 + (size_t)(D - t) * 4 + k]);
            }
            for (int t = 0; t < D; ++t) {
                P->c3pts.push_back(P->c3pts[f0 + (size_t)(D + 1 + D - 1 - t)]);
                for (int k = 0; k < 4; ++k)
                    P->c3pts64.push_back(P->c3pts64[d0 + (size_t)(D + 1 + D - 1 - t) * 4 + k]);
            }
        }
        TP e3 = tp_elevate3(L.bnd[b]);
        float f[12];
        for (int t = 0; t < 4; ++t)
            for (int k = 0; k < 3; ++k) {
                f[t * 3 + k] = (float)e3.h[t][k];
                P->c2_64.push_back(e3.h[t][k]);
            }
        P->c2.push_back(float4{f[0], f[1], f[2], f[3]});
        P->c2.push_back(float4{f[4], f[5], f[6], f[7]});
        P->c2.push_back(float4{f[8], f[9], f[10], f[11]});
        P->c2mult.push_back((float)L.mult[b]);
    }
}

std::string build_model_3d(const gwn_patch3d* patches, size_t n, const gwn_build_opts& o, HostModel* out,
                           gwn_status* code) {
    *code = GWN_ERR_INVALID_ARG;
    if (n == 0) return "no patches";
    if (!patches) return "patches is NULL";
    std::vector<PatchWork> work(n);
    double slo[3] = {1e300, 1e300, 1e300}, shi[3] = {-1e300, -1e300, -1e300};
    std::vector<double> H, pu, bu, pv, bv;
    for (size_t pi = 0; pi < n; ++pi) {
        const gwn_patch3d& P = patches[pi];
        std::string where = "patch " + std::to_string(pi) + ": ";
        *code = GWN_ERR_INVALID_ARG;
        if (P.deg_u < 1 || P.deg_u > 3 || P.deg_v < 1 || P.deg_v > 3) return where + "degrees must be 1..3";
        if (P.n_u < P.deg_u + 1 || P.n_v < P.deg_v + 1) return where + "too few control points";
        if (!P.ctrl || !P.knots_u || !P.knots_v) return where + "NULL control points or knots";
        if (P.n_trims < 0 || (P.n_trims > 0 && !P.trims)) return where + "bad trim array";
        *code = GWN_ERR_INVALID_GEOMETRY;
        std::string e = check_knots(P.deg_u, P.n_u, P.knots_u);
        if (e.empty()) e = check_knots(P.deg_v, P.n_v, P.knots_v);
        if (!e.empty()) return where + e;
        const int nu = P.n_u, nv = P.n_v, du = P.deg_u, dv = P.deg_v;
        // homogeneous control points, u-major
        H.assign((size_t)nu * nv * 4, 0.0);
        for (int i = 0; i < nu * nv; ++i) {
            double w = P.weights ? P.weights[i] : 1.0;
            if (!(w > 0) || !std::isfinite(w)) return where + "weight <= 0 or not finite";
            for (int k = 0; k < 3; ++k) {
                double x = P.ctrl[3 * i + k];
                if (!std::isfinite(x)) return where + "control point not finite";
                H[(size_t)i * 4 + k] = w * x;
                slo[k] = std::min(slo[k], x);
                shi[k] = std::max(shi[k], x);
            }
            H[(size_t)i * 4 + 3] = w;
        }
        PatchWork& W = work[pi];
        W.prim = (int64_t)pi;
        // spans: decompose along u (points = whole v-rows), then along v
        int su = decompose(du, nu, P.knots_u, 4 * nv, H.data(), &pu, &bu);
        std::vector<std::vector<double>> vrows;
        int sv = -1;
        std::vector<double> bvv;
        const int nu2 = su * (du + 1);
        std::vector<double> all;  // [row][v-point][4]
        for (int r = 0; r < nu2; ++r) {
            std::vector<double> seg, brk;
            int s = decompose(dv, nv, P.knots_v, 4, &pu[(size_t)r * 4 * nv], &seg, &brk);
            if (sv < 0) { sv = s; bvv = brk; all.resize((size_t)nu2 * s * (dv + 1) * 4); }
            std::memcpy(&all[(size_t)r * sv * (dv + 1) * 4], seg.data(), sizeof(double) * seg.size());
        }
        const double U0 = P.knots_u[0], U1 = P.knots_u[nu + du], V0 = P.knots_v[0], V1 = P.knots_v[nv + dv];
        for (int a = 0; a < su; ++a)
            for (int b = 0; b < sv; ++b) {
                // span net of degree (du, dv) -> bicubic by elevation in both directions
                double net[4][4][4];
                double cur[4][4][4];
                for (int i = 0; i <= du; ++i)
                    for (int j = 0; j <= dv; ++j)
                        for (int k = 0; k < 4; ++k)
                            cur[i][j][k] = all[(((size_t)(a * (du + 1) + i)) * sv * (dv + 1) + (size_t)b * (dv + 1) + j) * 4 + k];
                int cu = du, cv = dv;
                while (cu < 3) {
                    double nx[4][4][4];
                    for (int j = 0; j <= cv; ++j) {
                        for (int k = 0; k < 4; ++k) { nx[0][j][k] = cur[0][j][k]; nx[cu + 1][j][k] = cur[cu][j][k]; }
                        for (int i = 1; i <= cu; ++i) {
                            double al = (double)i / (cu + 1);
                            for (int k = 0; k < 4; ++k) nx[i][j][k] = al * cur[i - 1][j][k] + (1 - al) * cur[i][j][k];
                        }
                    }
                    std::memcpy(cur, nx, sizeof(cur));
                    ++cu;
                }
                while (cv < 3) {
                    double nx[4][4][4];
                    for (int i = 0; i <= cu; ++i) {
                        for (int k = 0; k < 4; ++k) { nx[i][0][k] = cur[i][0][k]; nx[i][cv + 1][k] = cur[i][cv][k]; }
                        for (int j = 1; j <= cv; ++j) {
                            double al = (double)j / (cv + 1);
                            for (int k = 0; k < 4; ++k) nx[i][j][k] = al * cur[i][j - 1][k] + (1 - al) * cur[i][j][k];
                        }
                    }
                    std::memcpy(cur, nx, sizeof(cur));
                    ++cv;
                }
                std::memcpy(net, cur, sizeof(net));
                Net N;
                std::memcpy(N.h, net, sizeof(net));
                W.spans.push_back({Rect{bu[a], bu[a + 1], bvv[b], bvv[b + 1]}, N});
            }
        W.untrimmed = P.n_trims == 0;
        for (int t = 0; t < P.n_trims; ++t) {
            const gwn_curve2d& C = P.trims[t];
            e = validate_curve(C, U0, U1, V0, V1);
            if (!e.empty()) {
                *code = (e.find("degree") != std::string::npos || e.find("NULL") != std::string::npos)
                            ? GWN_ERR_INVALID_ARG : GWN_ERR_INVALID_GEOMETRY;
                return where + e;
            }
            std::vector<double> th((size_t)C.n_ctrl * 3), seg, brk;
            for (int i = 0; i < C.n_ctrl; ++i) {
                double w = C.weights ? C.weights[i] : 1.0;
                th[i * 3 + 0] = w * C.ctrl[2 * i];
                th[i * 3 + 1] = w * C.ctrl[2 * i + 1];
                th[i * 3 + 2] = w;
            }
            int np = decompose(C.degree, C.n_ctrl, C.knots, 3, th.data(), &seg, &brk);
            for (int k = 0; k < np; ++k) {
                TP tp;
                tp.deg = C.degree;
                for (int i = 0; i <= C.degree; ++i)
                    for (int c = 0; c < 3; ++c) tp.h[i][c] = seg[((size_t)k * (C.degree + 1) + i) * 3 + c];
                W.trims.push_back(tp);
            }
        }
    }
    double sdiag = dist3(slo, shi);
    double xref[3];
    for (int k = 0; k < 3; ++k) xref[k] = 0.5 * (slo[k] + shi[k]);
    std::vector<double> gx, gw;
    gauss_legendre01(o.quad_nodes, &gx, &gw);

    // leaves of every patch, in parallel over patches
    int nt = o.n_threads > 0 ? o.n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    nt = std::min<int>(nt, (int)n);
    std::vector<std::vector<Leaf>> per(n);
    std::atomic<size_t> next{0};
    auto worker = [&]() {
        for (size_t i; (i = next.fetch_add(1)) < n;) make_leaves(work[i], o, sdiag, xref, gx, gw, &per[i]);
    };
    std::vector<std::thread> th;
    for (int t = 1; t < nt; ++t) th.emplace_back(worker);
    worker();
    for (auto& t : th) t.join();
    std::vector<Leaf> leaves;
    for (auto& v : per)
        for (auto& L : v) leaves.push_back(std::move(L));
    if (leaves.empty()) {
        *code = GWN_ERR_INVALID_GEOMETRY;
        return "no visible surface";
    }

    const int nl = (int)leaves.size();
    LeafSet S;
    S.dim = 3;
    std::memcpy(S.xref, xref, sizeof(xref));
    S.box.resize((size_t)nl * 6);
    S.mom.resize((size_t)nl * 39);
    S.wsum.resize(nl);
    S.wx.resize((size_t)nl * 3);
    for (int i = 0; i < nl; ++i) {
        const Leaf& L = leaves[i];
        for (int k = 0; k < 3; ++k) {
            S.box[i * 6 + k] = L.lo[k];
            S.box[i * 6 + 3 + k] = L.hi[k];
            S.wx[i * 3 + k] = L.ax[k];
        }
        std::memcpy(&S.mom[(size_t)i * 39], L.mom, sizeof(L.mom));
        S.wsum[i] = L.area;
    }
    std::vector<int> perm;
    build_tree(S, o.order, out, &perm, o.adaptive_beta);
    for (int k = 0; k < 3; ++k) { out->lo[k] = slo[k]; out->hi[k] = shi[k]; }

    // pack leaves in BVH order
    out->leaf_prim.resize(nl);
    out->leaf_param.resize((size_t)nl * 4);
    out->leaf3.resize(nl);
    out->net3.resize((size_t)nl * kNet3Vec);
    out->net3_64.resize((size_t)nl * 64);
    std::vector<double> g4x, g4w, g8x, g8w;  // the FP32 rule (tables, minimum levels) and the FP64 rule
    gauss_legendre01(4, &g4x, &g4w);
    gauss_legendre01(8, &g8x, &g8w);
    // every leaf's boundary data on its own, in parallel over leaves (composing
    // the curves and tabulating their nodes is most of the build), then the
    // pieces are concatenated in BVH order
    std::vector<LeafPack> packs(nl);
    {
        std::atomic<int> next_leaf{0};
        auto pack_worker = [&]() {
            for (int i; (i = next_leaf.fetch_add(1)) < nl;) {
                const Leaf& L = leaves[perm[i]];
                out->leaf_prim[i] = L.prim;
                out->leaf_param[i * 4 + 0] = L.R.u0;
                out->leaf_param[i * 4 + 1] = L.R.u1;
                out->leaf_param[i * 4 + 2] = L.R.v0;
                out->leaf_param[i * 4 + 3] = L.R.v1;
                Leaf3Info I;
                float cen[3];
                for (int k = 0; k < 3; ++k) {
                    cen[k] = (float)(0.5 * (L.lo[k] + L.hi[k]));
                    I.cen[k] = cen[k];
                    I.nrm[k] = (float)L.nrm[k];
                }
                double dg = dist3(L.lo, L.hi);
                I.diag = (float)dg;
                I.rad = (float)(0.5 * dg);
                for (int a = 0; a < 4; ++a)
                    for (int b = 0; b < 4; ++b) {
                        const double* h = L.net.h[a][b];
                        out->net3[(size_t)i * kNet3Vec + a * 4 + b] =
                            float4{(float)(h[0] - cen[0] * h[3]), (float)(h[1] - cen[1] * h[3]),
                                   (float)(h[2] - cen[2] * h[3]), (float)h[3]};
                        for (int k = 0; k < 4; ++k) out->net3_64[(size_t)i * 64 + (a * 4 + b) * 4 + k] = h[k];
                    }
                I.c3_cnt = (int32_t)L.bnd.size();
                I.c2_cnt = (int32_t)L.bnd.size();
                out->leaf3[i] = I;  // offsets follow when the pieces are concatenated
                pack_leaf(L, cen, g4x, g4w, g8x, &packs[i]);
            }
        };
        std::vector<std::thread> pth;
        for (int t = 1; t < nt; ++t) pth.emplace_back(pack_worker);
        pack_worker();
        for (auto& t : pth) t.join();
    }
    for (int i = 0; i < nl; ++i) {
        LeafPack& P = packs[i];
        Leaf3Info& I = out->leaf3[i];
        I.c3_off = (int32_t)out->c3.size();
        I.c2_off = (int32_t)(out->c2.size() / kC2Vec);
        const int32_t base = (int32_t)out->c3pts.size();
        for (Curve3Info ci : P.c3) {
            ci.ctrl_off += base;
            out->c3.push_back(ci);
        }
        out->c3pts.insert(out->c3pts.end(), P.c3pts.begin(), P.c3pts.end());
        out->c3pts64.insert(out->c3pts64.end(), P.c3pts64.begin(), P.c3pts64.end());
        out->c3n.insert(out->c3n.end(), P.c3n.begin(), P.c3n.end());
        out->c3n64.insert(out->c3n64.end(), P.c3n64.begin(), P.c3n64.end());
        out->c2.insert(out->c2.end(), P.c2.begin(), P.c2.end());
        out->c2_64.insert(out->c2_64.end(), P.c2_64.begin(), P.c2_64.end());
        out->c2mult.insert(out->c2mult.end(), P.c2mult.begin(), P.c2mult.end());
        P = LeafPack();  // release as we go
    }
    *code = GWN_OK;
    return "";
}

}  // namespace gwn
