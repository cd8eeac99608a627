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
#include "build_device.h"
#include "curves3d.h"

namespace gwn {

namespace {

constexpr double kMaxConeDeg = 55.0;
constexpr int kMaxSplitDepth = 14;

// ---------------------------------------------------------------- 2D pieces


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
    double mom[kLeafMom3];  // uncentred moments about xref (orders 0-3)
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

// moments by Green's theorem on the leaf's local boundary (leaf_moments_core)
void leaf_moments(Leaf& L, const double* xref, const std::vector<double>& gx, const std::vector<double>& gw) {
    leaf_moments_core(L.net, L.bnd.data(), L.mult.data(), (int)L.bnd.size(), xref, gx.data(), gw.data(), (int)gx.size(),
                      L.mom, &L.area, L.ax);
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

// leaves of one patch; with `moments` their moments too (else the device
// stage computes them)
void make_leaves(const PatchWork& P, const gwn_build_opts& o, double sdiag, const double* xref,
                 const std::vector<double>& gx, const std::vector<double>& gw, bool moments, std::vector<Leaf>* out) {
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
        if (moments) leaf_moments(L, xref, gx, gw);
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
    const size_t nb = L.bnd.size();
    P->c3.resize(nb);
    P->c3n.resize(nb * kC3NodeVec);
    P->c3n64.resize(nb * kC3Node64);
    P->c2.resize(nb * kC2Vec);
    P->c2_64.resize(nb * 12);
    P->c2mult.resize(nb);
    size_t npts = 0;
    for (size_t b = 0; b < nb; ++b) npts += 2 * (2 * 6 * (size_t)L.bnd[b].deg + 1);
    P->c3pts.resize(npts);
    P->c3pts64.resize(npts * 4);
    size_t off = 0;
    for (size_t b = 0; b < nb; ++b) {
        Curve3Info& ci = P->c3[b];
        ci.ctrl_off = (int32_t)off;
        pack_curve(L.bnd[b], L.mult[b], L.net, cen, g4x.data(), g4w.data(), g8x.data(), &ci, &P->c3pts[off],
                   &P->c3pts64[off * 4], &P->c3n[b * kC3NodeVec], &P->c3n64[b * kC3Node64], &P->c2[b * kC2Vec],
                   &P->c2_64[b * 12], &P->c2mult[b]);
        off += 2 * (2 * (size_t)ci.deg + 1);
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
    // the per-leaf stage (moments, boundary curves) on the model's GPU, unless
    // the build is host-only or asks for the host stage
    const bool dev = o.device_build != 0 && o.device != GWN_DEVICE_HOST_ONLY;

    // leaves of every patch, in parallel over patches
    int nt = o.n_threads > 0 ? o.n_threads : (int)std::max(1u, std::thread::hardware_concurrency());
    nt = std::min<int>(nt, (int)n);
    std::vector<std::vector<Leaf>> per(n);
    std::atomic<size_t> next{0};
    auto worker = [&]() {
        for (size_t i; (i = next.fetch_add(1)) < n;) make_leaves(work[i], o, sdiag, xref, gx, gw, !dev, &per[i]);
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
    if (dev) {
        // leaf moments on the device, one thread per leaf
        std::vector<Net> nets(nl);
        std::vector<TP> pieces;
        std::vector<double> mult, mom, area_ax;
        std::vector<int> off(nl + 1, 0);
        for (int i = 0; i < nl; ++i) {
            nets[i] = leaves[i].net;
            pieces.insert(pieces.end(), leaves[i].bnd.begin(), leaves[i].bnd.end());
            mult.insert(mult.end(), leaves[i].mult.begin(), leaves[i].mult.end());
            off[i + 1] = (int)pieces.size();
        }
        std::string e = device_leaf_moments(nets, pieces, mult, off, xref, gx, gw, &mom, &area_ax);
        if (!e.empty()) {
            *code = GWN_ERR_CUDA;
            return e;
        }
        for (int i = 0; i < nl; ++i) {
            Leaf& L = leaves[i];
            std::memcpy(L.mom, &mom[(size_t)i * kLeafMom3], sizeof(L.mom));
            L.area = area_ax[(size_t)i * 4];
            for (int k = 0; k < 3; ++k) L.ax[k] = area_ax[(size_t)i * 4 + 1 + k];
        }
    }
    LeafSet S;
    S.dim = 3;
    std::memcpy(S.xref, xref, sizeof(xref));
    S.box.resize((size_t)nl * 6);
    S.mom.resize((size_t)nl * kLeafMom3);
    S.wsum.resize(nl);
    S.wx.resize((size_t)nl * 3);
    for (int i = 0; i < nl; ++i) {
        const Leaf& L = leaves[i];
        for (int k = 0; k < 3; ++k) {
            S.box[i * 6 + k] = L.lo[k];
            S.box[i * 6 + 3 + k] = L.hi[k];
            S.wx[i * 3 + k] = L.ax[k];
        }
        std::memcpy(&S.mom[(size_t)i * kLeafMom3], L.mom, sizeof(L.mom));
        S.wsum[i] = L.area;
    }
    std::vector<int> perm;
    build_tree(S, o.order, out, &perm, o.adaptive_beta, o.tree_builder);
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
                if (!dev) pack_leaf(L, cen, g4x, g4w, g8x, &packs[i]);
            }
        };
        std::vector<std::thread> pth;
        for (int t = 1; t < nt; ++t) pth.emplace_back(pack_worker);
        pack_worker();
        for (auto& t : pth) t.join();
    }
    if (dev) {
        // the boundary curves on the device, one thread per curve, in BVH order
        std::vector<Net> nets(nl);
        std::vector<float> cen((size_t)nl * 3);
        std::vector<TP> pieces;
        std::vector<double> mult;
        std::vector<int> cleaf;
        std::vector<int32_t> coff;
        size_t npts = 0;
        for (int i = 0; i < nl; ++i) {
            const Leaf& L = leaves[perm[i]];
            Leaf3Info& I = out->leaf3[i];
            nets[i] = L.net;
            for (int k = 0; k < 3; ++k) cen[(size_t)i * 3 + k] = I.cen[k];
            I.c3_off = (int32_t)pieces.size();
            I.c2_off = I.c3_off;
            for (size_t b = 0; b < L.bnd.size(); ++b) {
                pieces.push_back(L.bnd[b]);
                mult.push_back(L.mult[b]);
                cleaf.push_back(i);
                coff.push_back((int32_t)npts);
                npts += 2 * (2 * 6 * (size_t)L.bnd[b].deg + 1);
            }
        }
        const size_t nc = pieces.size();
        out->c3.resize(nc);
        out->c3pts.resize(npts);
        out->c3pts64.resize(npts * 4);
        out->c3n.resize(nc * kC3NodeVec);
        out->c3n64.resize(nc * kC3Node64);
        out->c2.resize(nc * kC2Vec);
        out->c2_64.resize(nc * 12);
        out->c2mult.resize(nc);
        std::string e = device_pack_curves(nets, cen, pieces, mult, cleaf, coff, g4x, g4w, g8x, out);
        if (!e.empty()) {
            *code = GWN_ERR_CUDA;
            return e;
        }
        *code = GWN_OK;
        return "";
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
