// build.cpp -- generic BVH construction (top-down sweep or Karras LBVH) with
// moment up-sweep and centring, and the 2D preprocessing of Algorithm 1.
//
// 2D leaves (Section 3.2): every NURBS curve is split into rational Bezier
// pieces, then each piece is bisected until the diagonal of its control-point
// box is below max_aabb_frac times the diagonal of the whole shape's box.
// Leaf moments (Section 3.1) are those of the leaf's chord, which has the same
// GWN as the curve at any point outside the curve's convex hull; with
// beta >= 2 the far test only accepts such points.  For a chord a -> b with
// e = b - a and normal N = (e_y, -e_x) the uncentred moments are exact:
//   int n       = N
//   int x n     = (a + e/2) (x) N
//   int x x n   = (a a + (a e + e a)/2 + e e / 3) (x) N
#include "build.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <numeric>
#include <stdexcept>
#include <thread>

namespace gwn {

static inline bool finite(double x) { return std::isfinite(x); }

std::string check_knots(int degree, int n_ctrl, const double* U) {
    int m = n_ctrl + degree + 1;
    for (int i = 0; i < m; ++i)
        if (!finite(U[i])) return "knot is not finite";
    for (int i = 0; i + 1 < m; ++i)
        if (U[i + 1] < U[i]) return "knots decrease";
    for (int i = 1; i <= degree; ++i)
        if (U[i] != U[0] || U[m - 1 - i] != U[m - 1]) return "knot vector is not clamped";
    if (!(U[m - 1] > U[0])) return "empty parameter range";
    // interior multiplicities must not exceed the degree
    for (int i = degree + 1; i < n_ctrl;) {
        int j = i;
        while (j < n_ctrl && U[j] == U[i]) ++j;
        if (j - i > degree) return "interior knot multiplicity exceeds the degree";
        i = j;
    }
    return "";
}

// Bezier decomposition in one left-to-right sweep: for each interior knot the
// current segment is completed by raising that knot's multiplicity to the
// degree; the points computed for the next segment are carried over.
int decompose(int p, int n, const double* U, int hd, const double* P, std::vector<double>* out,
              std::vector<double>* brk) {
    const int m = n + p;  // index of the last knot
    std::vector<double> cur((p + 1) * hd), nxt((p + 1) * hd), alpha(p + 1);
    out->clear();
    brk->clear();
    for (int i = 0; i <= p; ++i) std::memcpy(&cur[i * hd], &P[i * hd], sizeof(double) * hd);
    int a = p, b = p + 1;
    brk->push_back(U[p]);
    while (b < m) {
        int i0 = b;
        while (b < m && U[b + 1] == U[b]) ++b;
        int mult = b - i0 + 1;
        if (mult < p) {
            double numer = U[b] - U[a];
            for (int j = p; j > mult; --j) alpha[j - mult - 1] = numer / (U[a + j] - U[a]);
            int rr = p - mult;
            for (int j = 1; j <= rr; ++j) {
                int save = rr - j, s = mult + j;
                for (int k = p; k >= s; --k) {
                    double al = alpha[k - s];
                    for (int d = 0; d < hd; ++d)
                        cur[k * hd + d] = al * cur[k * hd + d] + (1.0 - al) * cur[(k - 1) * hd + d];
                }
                if (b < m)
                    for (int d = 0; d < hd; ++d) nxt[save * hd + d] = cur[p * hd + d];
            }
        }
        out->insert(out->end(), cur.begin(), cur.end());
        brk->push_back(U[b]);
        if (b < m) {
            for (int i = p - mult; i <= p; ++i)
                for (int d = 0; d < hd; ++d) nxt[i * hd + d] = P[(b - p + i) * hd + d];
            std::swap(cur, nxt);
            a = b;
            ++b;
        }
    }
    if (brk->size() == 1) {  // a single span: no interior knots were visited
        out->insert(out->end(), cur.begin(), cur.end());
        brk->push_back(U[n]);
    }
    return (int)brk->size() - 1;
}

// ------------------------------------------------------------------ BVH

static inline int clz64(uint64_t x) { return x ? __builtin_clzll(x) : 64; }

static uint64_t spread2(uint32_t x) {  // 32 bits -> even bits of 64
    uint64_t v = x;
    v = (v | (v << 16)) & 0x0000FFFF0000FFFFull;
    v = (v | (v << 8)) & 0x00FF00FF00FF00FFull;
    v = (v | (v << 4)) & 0x0F0F0F0F0F0F0F0Full;
    v = (v | (v << 2)) & 0x3333333333333333ull;
    v = (v | (v << 1)) & 0x5555555555555555ull;
    return v;
}
static uint64_t spread3(uint32_t x) {  // 21 bits -> every third bit of 63
    uint64_t v = x & 0x1FFFFF;
    v = (v | (v << 32)) & 0x1F00000000FFFFull;
    v = (v | (v << 16)) & 0x1F0000FF0000FFull;
    v = (v | (v << 8)) & 0x100F00F00F00F00Full;
    v = (v | (v << 4)) & 0x10C30C30C30C30C3ull;
    v = (v | (v << 2)) & 0x1249249249249249ull;
    return v;
}

namespace {
struct Karras {
    const std::vector<uint64_t>& key;
    int n;
    int delta(int i, int j) const {
        if (j < 0 || j >= n) return -1;
        uint64_t x = key[i] ^ key[j];
        if (x) return clz64(x);
        return 64 + __builtin_clz((uint32_t)(i ^ j));  // equal codes: order by index (i != j)
    }
};
}  // namespace

// uncentred moments per leaf or node: orders 0-2 in 2D, 0-3 in 3D
static int momn(int d) { return d == 2 ? 2 + 4 + 8 : kLeafMom3; }

// Folded polynomial coefficients of the order-`order` Taylor expansion (Eq. 3)
// for moments centred at x0, as evaluated by the kernels.
static void fold_moments_2d(const double* m, int order, double* f) {
    const double* m0 = m;
    const double* m1 = m + 2;
    const double* m2 = m + 6;   // m2[(i*2 + j)*2 + k]
    const double c = 1.0 / (2.0 * M_PI);
    auto M2 = [&](int i, int j, int k) { return m2[(i * 2 + j) * 2 + k]; };
    double a[2], b[2];
    for (int k = 0; k < 2; ++k) a[k] = M2(0, 0, k) + M2(1, 1, k);
    for (int j = 0; j < 2; ++j) b[j] = M2(0, j, 0) + M2(1, j, 1);
    std::fill(f, f + kMom2F64, 0.0);
    f[0] = c * m0[0];
    f[1] = c * m0[1];
    if (order >= 1) {
        f[2] = c * (m1[0] + m1[3]);                 // tr M1
        f[3] = -2.0 * c * m1[0];                     // Bxx
        f[4] = -2.0 * c * (m1[1] + m1[2]);           // Bxy (both orders)
        f[5] = -2.0 * c * m1[3];                     // Byy
    }
    if (order >= 2) {
        f[6] = -c * (a[0] + 2.0 * b[0]);
        f[7] = -c * (a[1] + 2.0 * b[1]);
        f[8] = 4.0 * c * M2(0, 0, 0);
        f[9] = 4.0 * c * (M2(0, 0, 1) + M2(0, 1, 0) + M2(1, 0, 0));
        f[10] = 4.0 * c * (M2(0, 1, 1) + M2(1, 0, 1) + M2(1, 1, 0));
        f[11] = 4.0 * c * M2(1, 1, 1);
    }
}

static void fold_moments_3d(const double* m, int order, double* f) {
    const double* m0 = m;
    const double* m1 = m + 3;   // m1[i*3 + j]
    const double* m2 = m + 12;  // m2[(i*3 + j)*3 + k]
    const double c = 1.0 / (4.0 * M_PI);
    auto M1 = [&](int i, int j) { return m1[i * 3 + j]; };
    auto M2 = [&](int i, int j, int k) { return m2[(i * 3 + j) * 3 + k]; };
    // fully symmetrised sum over the index permutations of (i, j, k)
    auto S3 = [&](int i, int j, int k) {
        int idx[3] = {i, j, k};
        std::sort(idx, idx + 3);
        double s = 0;
        do { s += M2(idx[0], idx[1], idx[2]); } while (std::next_permutation(idx, idx + 3));
        return s;
    };
    std::fill(f, f + kMom3F64, 0.0);
    f[0] = c * m0[0];
    f[1] = c * m0[1];
    f[2] = c * m0[2];
    if (order >= 1) {
        f[3] = c * (M1(0, 0) + M1(1, 1) + M1(2, 2));
        f[4] = -3.0 * c * M1(0, 0);
        f[5] = -3.0 * c * M1(1, 1);
        f[6] = -3.0 * c * M1(2, 2);
        f[7] = -3.0 * c * (M1(0, 1) + M1(1, 0));
        f[8] = -3.0 * c * (M1(0, 2) + M1(2, 0));
        f[9] = -3.0 * c * (M1(1, 2) + M1(2, 1));
    }
    if (order >= 2) {
        double a[3], b[3];
        for (int k = 0; k < 3; ++k) a[k] = M2(0, 0, k) + M2(1, 1, k) + M2(2, 2, k);
        for (int j = 0; j < 3; ++j) b[j] = M2(0, j, 0) + M2(1, j, 1) + M2(2, j, 2);
        for (int k = 0; k < 3; ++k) f[10 + k] = -1.5 * c * (a[k] + 2.0 * b[k]);
        const double e = 7.5 * c;
        // S3 sums the distinct permutations of the sorted index triple, which
        // is exactly the coefficient of the monomial r_i r_j r_k
        f[13] = e * S3(0, 0, 0);
        f[14] = e * S3(1, 1, 1);
        f[15] = e * S3(2, 2, 2);
        f[16] = e * S3(0, 0, 1);
        f[17] = e * S3(0, 0, 2);
        f[18] = e * S3(0, 1, 1);
        f[19] = e * S3(1, 1, 2);
        f[20] = e * S3(0, 2, 2);
        f[21] = e * S3(1, 2, 2);
        f[22] = e * S3(0, 1, 2);
    }
    if (order >= 3) {
        // The order-3 term (1/6) sum d_i d_j d_l K_k(r) M3_ijlk of the same
        // expansion, K(v) = v / |v|^3, M3_ijlk = int y_i y_j y_l n_k.  With
        // d_ijl K_k = -3 (d_jk d_il + d_ij d_kl + d_ik d_jl) / |r|^5
        //             + 15 (d_jk r_i r_l + d_ij r_k r_l + d_ik r_j r_l
        //                   + d_il r_j r_k + d_jl r_i r_k + d_kl r_i r_j) / |r|^7
        //             - 105 r_i r_j r_l r_k / |r|^9
        // and M3 symmetric in its first three indices it is
        //   -1.5 T / |r|^5 + 7.5 r^T (Q + R) r / |r|^7 - 17.5 M3[r r r r] / |r|^9,
        // T = sum_ik M3_iikk, Q_ab = sum_j M3_abjj, R_lk = sum_i M3_iilk.
        const double* m3 = m + 39;  // m3[((i*3 + j)*3 + l)*3 + k]
        auto M3 = [&](int i, int j, int l, int k) { return m3[((i * 3 + j) * 3 + l) * 3 + k]; };
        auto S4 = [&](int i, int j, int l, int k) {
            int idx[4] = {i, j, l, k};
            std::sort(idx, idx + 4);
            double s = 0;
            do { s += M3(idx[0], idx[1], idx[2], idx[3]); } while (std::next_permutation(idx, idx + 4));
            return s;
        };
        double T = 0, P[3][3];
        for (int i = 0; i < 3; ++i)
            for (int k = 0; k < 3; ++k) T += M3(i, i, k, k);
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                double q = 0, r = 0;
                for (int j = 0; j < 3; ++j) {
                    q += M3(a, b, j, j);
                    r += M3(j, j, a, b);
                }
                P[a][b] = q + r;
            }
        f[23] = -1.5 * c * T;
        const double g = 7.5 * c;
        f[24] = g * P[0][0];
        f[25] = g * P[1][1];
        f[26] = g * P[2][2];
        f[27] = g * (P[0][1] + P[1][0]);
        f[28] = g * (P[0][2] + P[2][0]);
        f[29] = g * (P[1][2] + P[2][1]);
        // quartic monomials in the kernels' grouping: x^2 (x^2 xy xz y^2 z^2 yz),
        // y^2 (y^2 xy yz z^2 xz), z^2 (z^2 xz yz xy)
        const int quart[15][4] = {{0, 0, 0, 0}, {0, 0, 0, 1}, {0, 0, 0, 2}, {0, 0, 1, 1}, {0, 0, 2, 2},
                                  {0, 0, 1, 2}, {1, 1, 1, 1}, {0, 1, 1, 1}, {1, 1, 1, 2}, {1, 1, 2, 2},
                                  {0, 1, 1, 2}, {2, 2, 2, 2}, {0, 2, 2, 2}, {1, 2, 2, 2}, {0, 1, 2, 2}};
        const double h = -17.5 * c;
        for (int k = 0; k < 15; ++k) f[30 + k] = h * S4(quart[k][0], quart[k][1], quart[k][2], quart[k][3]);
    }
}

// Centroid (weighted, or the box centre when the weight is zero), radius (half
// the box diagonal) and the moments centred at the centroid: the moment
// transform of Section 3.1,
//   int (x - x0) n         = int x n - x0 (x) int n
//   int (x - x0)(x - x0) n = int x x n - x0 (x) int x n - (int x n with x0 in the
//                            second slot) + x0 (x) x0 (x) int n,
// in 3D also the third-order moments by the same binomial expansion, with the
// uncentred moments m taken about the reference point xref.
static void centre_block(int d, const double* box, double w, const double* wx, const double* m, const double* xref,
                         double* x0, double* radius, double* c) {
    double rr = 0;
    for (int k = 0; k < d; ++k) {
        double e = box[d + k] - box[k];
        rr += e * e;
        x0[k] = w > 0 ? wx[k] / w : 0.5 * (box[k] + box[d + k]);
    }
    *radius = 0.5 * std::sqrt(rr);
    double y[3] = {0, 0, 0};
    for (int k = 0; k < d; ++k) y[k] = x0[k] - xref[k];
    const double* m0 = m;
    const double* m1 = m + d;
    const double* m2 = m + d + d * d;
    double* c0 = c;
    double* c1 = c + d;
    double* c2 = c + d + d * d;
    for (int k = 0; k < d; ++k) c0[k] = m0[k];
    for (int i = 0; i < d; ++i)
        for (int k = 0; k < d; ++k) c1[i * d + k] = m1[i * d + k] - y[i] * m0[k];
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j)
            for (int k = 0; k < d; ++k)
                c2[(i * d + j) * d + k] =
                    m2[(i * d + j) * d + k] - y[i] * m1[j * d + k] - y[j] * m1[i * d + k] + y[i] * y[j] * m0[k];
    if (d == 3) {
        // int (x - x0)_i (x - x0)_j (x - x0)_l n_k from the uncentred moments
        const double* m3 = m + 39;
        double* c3 = c + 39;
        auto M2 = [&](int a, int b, int k) { return m2[(a * 3 + b) * 3 + k]; };
        auto M1 = [&](int a, int k) { return m1[a * 3 + k]; };
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                for (int l = 0; l < 3; ++l)
                    for (int k = 0; k < 3; ++k) {
                        const int o = ((i * 3 + j) * 3 + l) * 3 + k;
                        c3[o] = m3[o] - y[i] * M2(j, l, k) - y[j] * M2(i, l, k) - y[l] * M2(i, j, k) +
                                y[i] * y[j] * M1(l, k) + y[i] * y[l] * M1(j, k) + y[j] * y[l] * M1(i, k) -
                                y[i] * y[j] * y[l] * m0[k];
                    }
    }
}

// Karras LBVH (Section 3.1): leaves sorted by the Morton codes of their box
// centres (stable, by index on equal codes), internal node i spanning the range
// whose codes share the longest prefix, split where the next bit changes.
static void karras_tree(const LeafSet& L, std::vector<int>* perm, std::vector<int2>* child) {
    const int d = L.dim;
    const int n = (int)L.wsum.size();
    const int ni = std::max(0, n - 1);
    // scene box of the leaf boxes for Morton quantisation
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int i = 0; i < n; ++i)
        for (int k = 0; k < d; ++k) {
            lo[k] = std::min(lo[k], L.box[i * 2 * d + k]);
            hi[k] = std::max(hi[k], L.box[i * 2 * d + d + k]);
        }
    std::vector<uint64_t> code(n);
    for (int i = 0; i < n; ++i) {
        uint32_t g[3] = {0, 0, 0};
        for (int k = 0; k < d; ++k) {
            double c = 0.5 * (L.box[i * 2 * d + k] + L.box[i * 2 * d + d + k]);
            double ext = hi[k] - lo[k];
            double t = ext > 0 ? (c - lo[k]) / ext : 0.5;
            double cells = (d == 2) ? 4294967295.0 : 2097151.0;
            g[k] = (uint32_t)std::min(cells, std::max(0.0, std::floor(t * cells)));
        }
        code[i] = (d == 2) ? (spread2(g[0]) | (spread2(g[1]) << 1))
                           : (spread3(g[0]) | (spread3(g[1]) << 1) | (spread3(g[2]) << 2));
    }
    perm->resize(n);
    std::iota(perm->begin(), perm->end(), 0);
    std::stable_sort(perm->begin(), perm->end(), [&](int a, int b) { return code[a] < code[b]; });
    std::vector<uint64_t> key(n);
    for (int i = 0; i < n; ++i) key[i] = code[(*perm)[i]];

    child->assign(ni, int2{0, 0});
    Karras K{key, n};
    for (int i = 0; i < ni; ++i) {
        int dir = (K.delta(i, i + 1) - K.delta(i, i - 1)) >= 0 ? 1 : -1;
        int dmin = K.delta(i, i - dir);
        int lmax = 2;
        while (K.delta(i, i + lmax * dir) > dmin) lmax *= 2;
        int l = 0;
        for (int t = lmax / 2; t >= 1; t /= 2)
            if (K.delta(i, i + (l + t) * dir) > dmin) l += t;
        int j = i + l * dir;
        int dnode = K.delta(i, j);
        int s = 0;
        for (int t = (l + 1) / 2;; t = (t + 1) / 2) {
            if (K.delta(i, i + (s + t) * dir) > dnode) s += t;
            if (t == 1) break;
        }
        int gamma = i + s * dir + std::min(dir, 0);
        int left = (std::min(i, j) == gamma) ? ~gamma : gamma;
        int right = (std::max(i, j) == gamma + 1) ? ~(gamma + 1) : gamma + 1;
        (*child)[i] = int2{left, right};
    }
}

// Top-down sweep builder.  The leaves of a node (a range of perm) are split
// where k |D_L|^2 + (m - k) |D_R|^2 is least, D the diagonal of each side's box
// union and k the leaves on the left, over the three axes with the leaves
// sorted by box centre along the axis (prefix and suffix unions give every
// split of an axis in one pass).  A node is visited when a query comes within
// beta r of it, so small radii over many leaves cut the visits per query;
// weighting each side by its leaf count keeps the split from peeling off
// single leaves.  Internal nodes are numbered in preorder (root 0, left child
// = parent + 1), leaves are ~(position in perm), as the Karras build numbers
// them.
static void topdown_tree(const LeafSet& L, std::vector<int>* perm, std::vector<int2>* child) {
    const int d = L.dim;
    const int n = (int)L.wsum.size();
    perm->resize(n);
    std::iota(perm->begin(), perm->end(), 0);
    child->assign(std::max(0, n - 1), int2{0, 0});
    if (n < 2) return;
    auto lo = [&](int i, int k) { return L.box[(size_t)i * 2 * d + k]; };
    auto hi = [&](int i, int k) { return L.box[(size_t)i * 2 * d + d + k]; };
    struct Task {
        int b, e, parent, side;
    };
    std::vector<Task> st{{0, n, -1, 0}};
    std::vector<int> ord, best_ord;
    std::vector<double> suf;  // suffix diagonal^2
    int next = 0;
    while (!st.empty()) {
        const Task t = st.back();
        st.pop_back();
        const int id = next++;
        if (t.parent >= 0) (t.side ? (*child)[t.parent].y : (*child)[t.parent].x) = id;
        const int m = t.e - t.b;
        double best = 1e300;
        int best_k = m / 2;
        best_ord.assign(perm->begin() + t.b, perm->begin() + t.e);
        for (int ax = 0; ax < d; ++ax) {
            ord.assign(perm->begin() + t.b, perm->begin() + t.e);
            std::sort(ord.begin(), ord.end(), [&](int a, int b) {
                const double ca = lo(a, ax) + hi(a, ax), cb = lo(b, ax) + hi(b, ax);
                return ca < cb || (ca == cb && a < b);
            });
            suf.assign(m + 1, 0.0);
            double blo[3] = {1e300, 1e300, 1e300}, bhi[3] = {-1e300, -1e300, -1e300};
            for (int j = m - 1; j >= 1; --j) {
                double dd = 0;
                for (int k = 0; k < d; ++k) {
                    blo[k] = std::min(blo[k], lo(ord[j], k));
                    bhi[k] = std::max(bhi[k], hi(ord[j], k));
                    dd += (bhi[k] - blo[k]) * (bhi[k] - blo[k]);
                }
                suf[j] = dd;
            }
            double plo[3] = {1e300, 1e300, 1e300}, phi[3] = {-1e300, -1e300, -1e300};
            bool improved = false;
            for (int j = 0; j < m - 1; ++j) {
                double dd = 0;
                for (int k = 0; k < d; ++k) {
                    plo[k] = std::min(plo[k], lo(ord[j], k));
                    phi[k] = std::max(phi[k], hi(ord[j], k));
                    dd += (phi[k] - plo[k]) * (phi[k] - plo[k]);
                }
                const double cost = (j + 1) * dd + (m - j - 1) * suf[j + 1];
                // equal costs (coincident boxes) go to the more balanced split,
                // so that duplicated leaves do not form a chain
                const bool tie = cost <= best * (1.0 + 1e-12) && cost >= best * (1.0 - 1e-12);
                if ((cost < best && !tie) || (tie && std::abs(2 * (j + 1) - m) < std::abs(2 * best_k - m))) {
                    best = cost;
                    best_k = j + 1;
                    improved = true;
                }
            }
            if (improved) best_ord = ord;
        }
        std::copy(best_ord.begin(), best_ord.end(), perm->begin() + t.b);
        const int mid = t.b + best_k;
        // right first, so that the left subtree takes the next preorder numbers
        if (t.e - mid == 1) (*child)[id].y = ~mid;
        else st.push_back({mid, t.e, id, 1});
        if (mid - t.b == 1) (*child)[id].x = ~t.b;
        else st.push_back({t.b, mid, id, 0});
    }
}

void build_tree(const LeafSet& L, int order, HostModel* out, std::vector<int>* perm, int adaptive_beta,
                int tree_builder) {
    const int d = L.dim;
    const int n = (int)L.wsum.size();
    const int M = momn(d);
    out->dim = d;
    out->n_leaves = n;
    const int ni = std::max(0, n - 1);
    if (tree_builder != 0) {
        topdown_tree(L, perm, &out->child);
    } else {
        karras_tree(L, perm, &out->child);
    }

    // up-sweep in post-order (children before parents)
    std::vector<double> nbox(ni * 2 * d), nmom((size_t)ni * M), nw(ni), nwx(ni * d);
    auto leaf_box = [&](int li) { return &L.box[(size_t)(*perm)[li] * 2 * d]; };
    std::vector<int> order_post;
    order_post.reserve(ni);
    std::vector<int> depth(ni, 0);
    int maxdepth = 0;
    if (ni > 0) {
        std::vector<std::pair<int, int>> st;  // (node, state)
        st.push_back({0, 0});
        while (!st.empty()) {
            auto [node, state] = st.back();
            st.pop_back();
            if (state == 0) {
                st.push_back({node, 1});
                int2 c = out->child[node];
                for (int cc : {c.x, c.y}) {
                    if (cc >= 0) {
                        depth[cc] = depth[node] + 1;
                        st.push_back({cc, 0});
                    } else {
                        maxdepth = std::max(maxdepth, depth[node] + 1);
                    }
                }
            } else {
                order_post.push_back(node);
            }
        }
    }
    out->max_depth = maxdepth;
    for (int node : order_post) {
        double* bx = &nbox[node * 2 * d];
        for (int k = 0; k < d; ++k) { bx[k] = 1e300; bx[d + k] = -1e300; }
        double* mm = &nmom[(size_t)node * M];
        std::fill(mm, mm + M, 0.0);
        nw[node] = 0;
        for (int k = 0; k < d; ++k) nwx[node * d + k] = 0;
        int2 c = out->child[node];
        for (int cc : {c.x, c.y}) {
            const double *cb, *cm, *cwx;
            double cw;
            if (cc < 0) {
                int li = (*perm)[~cc];
                cb = &L.box[(size_t)li * 2 * d];
                cm = &L.mom[(size_t)li * M];
                cw = L.wsum[li];
                cwx = &L.wx[(size_t)li * d];
            } else {
                cb = &nbox[cc * 2 * d];
                cm = &nmom[(size_t)cc * M];
                cw = nw[cc];
                cwx = &nwx[cc * d];
            }
            for (int k = 0; k < d; ++k) {
                bx[k] = std::min(bx[k], cb[k]);
                bx[d + k] = std::max(bx[d + k], cb[d + k]);
            }
            for (int k = 0; k < M; ++k) mm[k] += cm[k];
            nw[node] += cw;
            for (int k = 0; k < d; ++k) nwx[node * d + k] += cwx[k];
        }
    }
    (void)leaf_box;

    // far-field data of every leaf (moments centred at the leaf's own centroid)
    {
        const int fv = d == 2 ? kMom2Vec : kMom3Vec;
        const int ff = d == 2 ? kMom2F64 : kMom3F64;
        out->lhdr.assign(n, float4{0, 0, 0, 0});
        out->lhdr64.assign((size_t)n * 4, 0.0);
        out->lmom.assign((size_t)n * fv, float4{0, 0, 0, 0});
        out->lmom64.assign((size_t)n * ff, 0.0);
        std::vector<double> c(M);
        for (int i = 0; i < n; ++i) {
            int li = (*perm)[i];
            double x0[3] = {0, 0, 0}, radius;
            centre_block(d, &L.box[(size_t)li * 2 * d], L.wsum[li], &L.wx[(size_t)li * d], &L.mom[(size_t)li * M],
                         L.xref, x0, &radius, c.data());
            double f[kMom3F64];
            if (d == 2) fold_moments_2d(c.data(), order, f); else fold_moments_3d(c.data(), order, f);
            for (int k = 0; k < ff; ++k) out->lmom64[(size_t)i * ff + k] = f[k];
            float* fp = reinterpret_cast<float*>(&out->lmom[(size_t)i * fv]);
            for (int k = 0; k < 4 * fv; ++k) fp[k] = k < ff ? (float)f[k] : 0.0f;
            out->lhdr[i] = float4{(float)x0[0], (float)x0[1], (float)x0[2], (float)(radius * radius)};
            for (int k = 0; k < 3; ++k) out->lhdr64[i * 4 + k] = x0[k];
            out->lhdr64[i * 4 + 3] = radius * radius;
        }
    }

    // centre in place and pack
    out->x0.assign((size_t)ni * d, 0.0);
    out->r.assign(ni, 0.0);
    out->mom_c.assign((size_t)ni * M, 0.0);
    out->hdr.assign(ni, float4{0, 0, 0, 0});
    out->hdr64.assign((size_t)ni * 4, 0.0);
    const int fv = d == 2 ? kMom2Vec : kMom3Vec;
    const int ff = d == 2 ? kMom2F64 : kMom3F64;
    out->mom.assign((size_t)ni * fv, float4{0, 0, 0, 0});
    out->mom64.assign((size_t)ni * ff, 0.0);
    for (int node = 0; node < ni; ++node) {
        double x0[3] = {0, 0, 0}, radius;
        double* c = &out->mom_c[(size_t)node * M];
        centre_block(d, &nbox[node * 2 * d], nw[node], &nwx[node * d], &nmom[(size_t)node * M], L.xref, x0, &radius, c);
        for (int k = 0; k < d; ++k) out->x0[node * d + k] = x0[k];
        out->r[node] = radius;
        double f[kMom3F64];
        if (d == 2) fold_moments_2d(c, order, f); else fold_moments_3d(c, order, f);
        for (int k = 0; k < ff; ++k) out->mom64[(size_t)node * ff + k] = f[k];
        float* fp = reinterpret_cast<float*>(&out->mom[(size_t)node * fv]);
        for (int k = 0; k < 4 * fv; ++k) fp[k] = k < ff ? (float)f[k] : 0.0f;
        out->hdr[node] = float4{(float)x0[0], (float)x0[1], (float)x0[2], (float)(radius * radius)};
        for (int k = 0; k < 3; ++k) out->hdr64[node * 4 + k] = x0[k];
        out->hdr64[node * 4 + 3] = radius * radius;
    }
    if (adaptive_beta && ni > 1) {
        // geometry-aware far test: the order-p remainder of a cluster of fill
        // a = (total curve length or area) / r^(d-1) grows like a * beta^-(p+d), so
        // a cluster denser than the median is approximated only beyond
        // beta * s * r, s = (a / a_median)^(1 / (p + d)) in [1, 4]; the far test
        // compares |x0 - q|^2 with beta^2 * hdr.w, so hdr.w carries s^2 r^2
        std::vector<double> fill(ni);
        for (int node = 0; node < ni; ++node) {
            const double r = std::max(out->r[node], 1e-300);
            fill[node] = nw[node] / (d == 2 ? r : r * r);
        }
        std::vector<double> sorted = fill;
        std::nth_element(sorted.begin(), sorted.begin() + ni / 2, sorted.end());
        const double med = std::max(sorted[ni / 2], 1e-300);
        for (int node = 0; node < ni; ++node) {
            const double s = std::min(4.0, std::max(1.0, std::pow(fill[node] / med, 1.0 / (order + d))));
            const double r2 = out->r[node] * out->r[node] * s * s;
            out->hdr[node].w = (float)r2;
            out->hdr64[node * 4 + 3] = r2;
        }
    }
}

// ------------------------------------------------------------------ 2D

namespace {
struct Piece2 {  // cubic rational Bezier, homogeneous (w x, w y, w)
    double h[4][3];
    int64_t prim;
    double t0, t1;
};

void elevate_to_cubic(int p, const double* H, double out[4][3]) {
    // exact degree elevation in homogeneous coordinates
    double cur[4][3];
    for (int i = 0; i <= p; ++i)
        for (int k = 0; k < 3; ++k) cur[i][k] = H[i * 3 + k];
    for (int q = p; q < 3; ++q) {
        double nxt[4][3];
        for (int k = 0; k < 3; ++k) {
            nxt[0][k] = cur[0][k];
            nxt[q + 1][k] = cur[q][k];
        }
        for (int i = 1; i <= q; ++i) {
            double a = (double)i / (q + 1);
            for (int k = 0; k < 3; ++k) nxt[i][k] = a * cur[i - 1][k] + (1 - a) * cur[i][k];
        }
        std::memcpy(cur, nxt, sizeof(cur));
    }
    std::memcpy(out, cur, sizeof(cur));
}

void split_half(const Piece2& P, Piece2* L, Piece2* R) {
    double T[4][3];
    std::memcpy(T, P.h, sizeof(T));
    L->prim = R->prim = P.prim;
    double tm = 0.5 * (P.t0 + P.t1);
    L->t0 = P.t0; L->t1 = tm;
    R->t0 = tm; R->t1 = P.t1;
    for (int k = 0; k < 3; ++k) { L->h[0][k] = T[0][k]; R->h[3][k] = T[3][k]; }
    for (int j = 1; j <= 3; ++j) {
        for (int i = 0; i <= 3 - j; ++i)
            for (int k = 0; k < 3; ++k) T[i][k] = 0.5 * (T[i][k] + T[i + 1][k]);
        for (int k = 0; k < 3; ++k) { L->h[j][k] = T[0][k]; R->h[3 - j][k] = T[3 - j][k]; }
    }
}

void piece_box(const Piece2& P, double* lo, double* hi) {
    lo[0] = lo[1] = 1e300;
    hi[0] = hi[1] = -1e300;
    for (int i = 0; i < 4; ++i)
        for (int k = 0; k < 2; ++k) {
            double x = P.h[i][k] / P.h[i][2];
            lo[k] = std::min(lo[k], x);
            hi[k] = std::max(hi[k], x);
        }
}
}  // namespace

std::string build_model_2d(const gwn_curve2d* curves, size_t n, const gwn_build_opts& o, HostModel* out,
                           gwn_status* code) {
    *code = GWN_ERR_INVALID_ARG;
    if (n == 0) return "no curves";
    if (!curves) return "curves is NULL";
    std::vector<Piece2> pieces;
    double slo[2] = {1e300, 1e300}, shi[2] = {-1e300, -1e300};
    std::vector<double> H, seg, brk;
    for (size_t c = 0; c < n; ++c) {
        const gwn_curve2d& C = curves[c];
        std::string where = "curve " + std::to_string(c) + ": ";
        if (C.degree < 1 || C.degree > 3) return where + "degree must be 1..3";
        if (C.n_ctrl < C.degree + 1) return where + "too few control points";
        if (!C.ctrl || !C.knots) return where + "NULL control points or knots";
        *code = GWN_ERR_INVALID_GEOMETRY;
        std::string e = check_knots(C.degree, C.n_ctrl, C.knots);
        if (!e.empty()) return where + e;
        H.resize((size_t)C.n_ctrl * 3);
        for (int i = 0; i < C.n_ctrl; ++i) {
            double w = C.weights ? C.weights[i] : 1.0;
            double x = C.ctrl[2 * i], y = C.ctrl[2 * i + 1];
            if (!(w > 0) || !finite(w) || !finite(x) || !finite(y)) return where + "non-finite point or weight <= 0";
            H[i * 3 + 0] = w * x;
            H[i * 3 + 1] = w * y;
            H[i * 3 + 2] = w;
            slo[0] = std::min(slo[0], x); slo[1] = std::min(slo[1], y);
            shi[0] = std::max(shi[0], x); shi[1] = std::max(shi[1], y);
        }
        *code = GWN_ERR_INVALID_ARG;
        int np = decompose(C.degree, C.n_ctrl, C.knots, 3, H.data(), &seg, &brk);
        for (int k = 0; k < np; ++k) {
            Piece2 P;
            elevate_to_cubic(C.degree, &seg[(size_t)k * (C.degree + 1) * 3], P.h);
            P.prim = (int64_t)c;
            P.t0 = brk[k];
            P.t1 = brk[k + 1];
            pieces.push_back(P);
        }
    }
    double sdiag = std::hypot(shi[0] - slo[0], shi[1] - slo[1]);
    // adaptive subdivision (Section 3.2)
    std::vector<Piece2> leaves;
    if (o.max_aabb_frac > 0 && sdiag > 0) {
        double lim = o.max_aabb_frac * sdiag;
        std::vector<std::pair<Piece2, int>> stack;
        for (auto& P : pieces) stack.push_back({P, 0});
        while (!stack.empty()) {
            auto [P, depth] = stack.back();
            stack.pop_back();
            double lo[2], hi[2];
            piece_box(P, lo, hi);
            if (std::hypot(hi[0] - lo[0], hi[1] - lo[1]) >= lim && depth < 30) {
                Piece2 L, R;
                split_half(P, &L, &R);
                stack.push_back({R, depth + 1});
                stack.push_back({L, depth + 1});
            } else {
                leaves.push_back(P);
            }
        }
    } else {
        leaves = pieces;
    }
    const int nl = (int)leaves.size();
    LeafSet S;
    S.dim = 2;
    S.xref[0] = 0.5 * (slo[0] + shi[0]);
    S.xref[1] = 0.5 * (slo[1] + shi[1]);
    S.box.resize((size_t)nl * 4);
    S.mom.resize((size_t)nl * 14);
    S.wsum.resize(nl);
    S.wx.resize((size_t)nl * 2);
    for (int i = 0; i < nl; ++i) {
        const Piece2& P = leaves[i];
        double lo[2], hi[2];
        piece_box(P, lo, hi);
        S.box[i * 4 + 0] = lo[0]; S.box[i * 4 + 1] = lo[1];
        S.box[i * 4 + 2] = hi[0]; S.box[i * 4 + 3] = hi[1];
        double a[2] = {P.h[0][0] / P.h[0][2] - S.xref[0], P.h[0][1] / P.h[0][2] - S.xref[1]};
        double b[2] = {P.h[3][0] / P.h[3][2] - S.xref[0], P.h[3][1] / P.h[3][2] - S.xref[1]};
        double e[2] = {b[0] - a[0], b[1] - a[1]};
        double N[2] = {e[1], -e[0]};
        double* m = &S.mom[(size_t)i * 14];
        m[0] = N[0];
        m[1] = N[1];
        for (int ii = 0; ii < 2; ++ii)
            for (int k = 0; k < 2; ++k) m[2 + ii * 2 + k] = (a[ii] + 0.5 * e[ii]) * N[k];
        for (int ii = 0; ii < 2; ++ii)
            for (int j = 0; j < 2; ++j) {
                double s = a[ii] * a[j] + 0.5 * (a[ii] * e[j] + e[ii] * a[j]) + e[ii] * e[j] / 3.0;
                for (int k = 0; k < 2; ++k) m[6 + (ii * 2 + j) * 2 + k] = s * N[k];
            }
        double len = std::hypot(e[0], e[1]);
        S.wsum[i] = len;
        S.wx[i * 2 + 0] = len * (0.5 * (a[0] + b[0]) + S.xref[0]);
        S.wx[i * 2 + 1] = len * (0.5 * (a[1] + b[1]) + S.xref[1]);
    }
    std::vector<int> perm;
    build_tree(S, o.order, out, &perm, o.adaptive_beta, o.tree_builder);
    out->lo[0] = slo[0]; out->lo[1] = slo[1];
    out->hi[0] = shi[0]; out->hi[1] = shi[1];
    out->leaf_prim.resize(nl);
    out->leaf_param.assign((size_t)nl * 4, 0.0);
    out->leaf2.resize((size_t)nl * kLeaf2Vec);
    out->leaf2_64.resize((size_t)nl * kLeaf2F64);
    for (int i = 0; i < nl; ++i) {
        const Piece2& P = leaves[perm[i]];
        out->leaf_prim[i] = P.prim;
        out->leaf_param[i * 4 + 0] = P.t0;
        out->leaf_param[i * 4 + 1] = P.t1;
        double x[4], y[4], w[4];
        for (int k = 0; k < 4; ++k) {
            w[k] = P.h[k][2];
            x[k] = P.h[k][0] / w[k];
            y[k] = P.h[k][1] / w[k];
        }
        // float centre, then offsets measured from that exact float value
        float cx = (float)(0.25 * (x[0] + x[1] + x[2] + x[3]));
        float cy = (float)(0.25 * (y[0] + y[1] + y[2] + y[3]));
        out->leaf2[i * 4 + 0] = float4{(float)(x[0] - cx), (float)(y[0] - cy), (float)(x[1] - cx), (float)(y[1] - cy)};
        out->leaf2[i * 4 + 1] = float4{(float)(x[2] - cx), (float)(y[2] - cy), (float)(x[3] - cx), (float)(y[3] - cy)};
        out->leaf2[i * 4 + 2] = float4{(float)w[0], (float)w[1], (float)w[2], (float)w[3]};
        out->leaf2[i * 4 + 3] = float4{cx, cy, 0.0f, 0.0f};
        double* d64 = &out->leaf2_64[(size_t)i * 12];
        double v[12] = {x[0], y[0], x[1], y[1], x[2], y[2], x[3], y[3], w[0], w[1], w[2], w[3]};
        std::memcpy(d64, v, sizeof(v));
    }
    *code = GWN_OK;
    return "";
}

}  // namespace gwn
