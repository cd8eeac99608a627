// Host execution of the query routines of the CUDA path (test harness).
//
// The leaf evaluators and the traversal of kernels2d.cuh / kernels3d.cuh are
// host-device functions; this file runs them on the CPU against models built
// by the library's own host build, so that the CPU test suite can compare the
// CUDA path's arithmetic with the FP64 oracle without a GPU.  It is test
// infrastructure: nothing in the package loads it.
#include <cmath>
#include <cstring>
#include <string>

#include "../../paper_2605_19200_gb300/csrc/build.h"
#include "../../paper_2605_19200_gb300/csrc/kernels3d.cuh"

using namespace gwn;

namespace {

// n-point Gauss-Legendre rule on [0, 1] (Newton on the Legendre polynomial)
void gauss01(int n, double* x, double* w) {
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
        x[i] = 0.5 * (1 - z);
        w[i] = 1.0 / ((1 - z * z) * pp * pp);
    }
}

void init_tables() {
    for (int a = 0; a <= kMaxC3Deg; ++a) {
        for (int b = 0; b <= kMaxC3Deg; ++b) h_binom[a][b] = 0.f;
        h_binom[a][0] = h_binom[a][a] = 1.f;
        for (int b = 1; b < a; ++b) h_binom[a][b] = h_binom[a - 1][b - 1] + h_binom[a - 1][b];
    }
    gauss01(8, h_glx8, h_glw8);
    gauss01(4, h_glx4d, h_glw4d);
    for (int i = 0; i < 4; ++i) {
        h_glx4f[i] = (float)h_glx4d[i];
        h_glw4f[i] = (float)h_glw4d[i];
    }
}

DevTree host_tree(const HostModel& H, int leaf_far, int order = 2) {
    DevTree t{};
    t.dim = H.dim;
    t.n_leaves = H.n_leaves;
    t.n_internal = H.n_leaves - 1;
    t.root = H.n_leaves > 1 ? 0 : ~0;
    t.leaf_far = leaf_far;
    t.order3 = H.dim == 3 && order >= 3 ? 1 : 0;
    t.order3_64 = t.order3;
    t.lhdr = H.lhdr.data();
    t.lmom = H.lmom.data();
    t.lhdr64 = H.lhdr64.data();
    t.lmom64 = H.lmom64.data();
    t.hdr = H.hdr.data();
    t.child = H.child.data();
    t.mom = H.mom.data();
    t.hdr64 = H.hdr64.data();
    t.mom64 = H.mom64.data();
    t.leaf2 = H.leaf2.data();
    t.leaf2_64 = H.leaf2_64.data();
    t.leaf3 = H.leaf3.data();
    t.net3 = H.net3.data();
    t.net3_64 = H.net3_64.data();
    t.c3 = H.c3.data();
    t.c3pts = H.c3pts.data();
    t.c3pts64 = H.c3pts64.data();
    t.c3n = H.c3n.empty() ? nullptr : H.c3n.data();
    t.c3n64 = H.c3n64.empty() ? nullptr : H.c3n64.data();
    t.c2 = H.c2.data();
    t.c2_64 = H.c2_64.data();
    t.c2mult = H.c2mult.data();
    return t;
}

}  // namespace

// For each query: the direct sums over every leaf in FP32 (with the FP64 near
// band) and in FP64, and the FP32 traversal with far-field factors beta and
// beta_leaf.  Returns the number of leaves, or -1 if the build failed.
extern "C" int hx_query3(const gwn_patch3d* patches, size_t n, const gwn_build_opts* o, const double* q, int nq,
                         double beta, double beta_leaf, double* direct32, double* direct64, double* bvh32,
                         unsigned* status) {
    init_tables();
    HostModel H;
    gwn_status code;
    if (!build_model_3d(patches, n, *o, &H, &code).empty()) return -1;
    const DevTree t = host_tree(H, 1, o->order);
    for (int i = 0; i < nq; ++i) {
        const float qx = (float)q[3 * i], qy = (float)q[3 * i + 1], qz = (float)q[3 * i + 2];
        uint32_t s32 = 0, s64 = 0, sb = 0;
        double a = 0, b = 0;
        for (int l = 0; l < t.n_leaves; ++l) {
            a += leaf3_eval32(t, l, qx, qy, qz, s32);
            b += leaf3_eval64(t, l, q[3 * i], q[3 * i + 1], q[3 * i + 2], s64);
        }
        direct32[i] = a;
        direct64[i] = b;
        bvh32[i] = query3_32(t, qx, qy, qz, (float)(beta * beta), sb, (float)(beta_leaf * beta_leaf));
        status[i] = s32 | s64 | sb;
    }
    return t.n_leaves;
}

// work[0..2] receive the traversal's totals: internal nodes visited, Taylor
// evaluations, exact leaf evaluations (may be NULL)
extern "C" int hx_query2(const gwn_curve2d* curves, size_t n, const gwn_build_opts* o, const double* q, int nq,
                         double beta, double* direct32, double* direct64, double* bvh32, unsigned* status,
                         long long* work) {
    init_tables();
    HostModel H;
    gwn_status code;
    if (!build_model_2d(curves, n, *o, &H, &code).empty()) return -1;
    const DevTree t = host_tree(H, 0);
    for (int i = 0; i < nq; ++i) {
        const float qx = (float)q[2 * i], qy = (float)q[2 * i + 1];
        uint32_t s32 = 0, s64 = 0, sb = 0;
        double a = 0, b = 0;
        for (int l = 0; l < t.n_leaves; ++l) {
            a += leaf2_eval32(t, l, qx, qy, s32);
            b += leaf2_eval64(t, l, q[2 * i], q[2 * i + 1], s64);
        }
        direct32[i] = a;
        direct64[i] = b;
        WorkLocal wl = {};
        bvh32[i] = query2_32(t, qx, qy, (float)(beta * beta), sb, &wl);
        status[i] = s32 | s64 | sb;
        if (work) {
            work[0] += (long long)wl.v[kWorkNodes];
            work[1] += (long long)wl.v[kWorkFar];
            work[2] += (long long)wl.v[kWorkLeaves];
        }
    }
    return t.n_leaves;
}

// Per (query, leaf) pair of a direct sum: the FP32 value from the node tables
// (fast32, NaN where leaf3_fast32 declines: the point is near the leaf or a
// curve needs panels below level 1), the full FP32 evaluation (full32, NaN
// where it needs the FP64 near band) and the FP64 evaluation (exact64).
// Arrays hold nq x n_leaves values.  Returns the number of leaves.
extern "C" int hx_leaf_paths3(const gwn_patch3d* patches, size_t n, const gwn_build_opts* o, const double* q, int nq,
                              double* fast32, double* full32, double* exact64, int max_leaves) {
    init_tables();
    HostModel H;
    gwn_status code;
    if (!build_model_3d(patches, n, *o, &H, &code).empty()) return -1;
    const DevTree t = host_tree(H, 1, o->order);
    if (t.n_leaves > max_leaves) return -2;
    for (int i = 0; i < nq; ++i)
        for (int l = 0; l < t.n_leaves; ++l) {
            const size_t k = (size_t)i * t.n_leaves + l;
            const Leaf3Info I = t.leaf3[l];
            const float qf[3] = {(float)q[3 * i], (float)q[3 * i + 1], (float)q[3 * i + 2]};
            const float qr[3] = {qf[0] - I.cen[0], qf[1] - I.cen[1], qf[2] - I.cen[2]};
            const float d2 = qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2];
            const float rfar = 1.1f * I.rad;
            float v = 0.f;
            fast32[k] = (d2 > rfar * rfar && leaf3_fast32(t, I, qr, d2, &v)) ? (double)v : NAN;
            full32[k] = leaf3_try32(t, l, qf[0], qf[1], qf[2], &v, nullptr, false) ? (double)v : NAN;
            uint32_t st = 0;
            exact64[k] = leaf3_eval64(t, l, (double)qf[0], (double)qf[1], (double)qf[2], st);
        }
    return t.n_leaves;
}

// Per (query, leaf) pair: the FP64 value from the FP64 node tables at the
// repair's panel ratio (fast64, NaN where leaf3_fast64 declines) and the full
// FP64 evaluation (exact64).  Arrays hold nq x n_leaves values.
extern "C" int hx_leaf_paths64(const gwn_patch3d* patches, size_t n, const gwn_build_opts* o, const double* q, int nq,
                               double* fast64, double* exact64, int max_leaves) {
    init_tables();
    HostModel H;
    gwn_status code;
    if (!build_model_3d(patches, n, *o, &H, &code).empty()) return -1;
    const DevTree t = host_tree(H, 1, o->order);
    if (t.n_leaves > max_leaves) return -2;
    for (int i = 0; i < nq; ++i)
        for (int l = 0; l < t.n_leaves; ++l) {
            const size_t k = (size_t)i * t.n_leaves + l;
            double v = 0;
            fast64[k] = leaf3_fast64(t, l, q + 3 * i, kRatio64Repair, &v) ? v : NAN;
            uint32_t st = 0;
            exact64[k] = leaf3_eval64(t, l, q[3 * i], q[3 * i + 1], q[3 * i + 2], st);
        }
    return t.n_leaves;
}

// The packet local expansion of internal node `node` about the point p
// (far3_local2) evaluated at p + s[k], and the node's own FP32 Taylor term at
// the same points (far3_node32), for ns offsets.  Returns the node count, or -1.
extern "C" int hx_local2(const gwn_patch3d* patches, size_t n, const gwn_build_opts* o, int node, const double* p,
                         const double* s, int ns, double* local, double* direct) {
    init_tables();
    HostModel H;
    gwn_status code;
    if (!build_model_3d(patches, n, *o, &H, &code).empty()) return -1;
    const DevTree t = host_tree(H, 1, o->order);
    if (node < 0 || node >= t.n_internal) return -1;
    const float4 h = t.hdr[node];
    const float4* M = t.mom + (size_t)node * kMom3Vec;
    const float D[3] = {h.x - (float)p[0], h.y - (float)p[1], h.z - (float)p[2]};
    float v[10];
    far3_local2(M, D[0], D[1], D[2], v);
    for (int k = 0; k < ns; ++k) {
        const float sx = (float)s[3 * k], sy = (float)s[3 * k + 1], sz = (float)s[3 * k + 2];
        local[k] = v[0] - (v[1] * sx + v[2] * sy + v[3] * sz) + 0.5f * (v[4] * sx * sx + v[5] * sy * sy + v[6] * sz * sz) +
                   v[7] * sx * sy + v[8] * sx * sz + v[9] * sy * sz;
        direct[k] = far3_node32(M, D[0] - sx, D[1] - sy, D[2] - sz, false);
    }
    return t.n_internal;
}

// The FP64 traversal (query3_64, the repair's far field) at factor beta with the
// model's Taylor order, and the exact FP64 sum over every leaf, for nq points.
extern "C" int hx_query3_64(const gwn_patch3d* patches, size_t n, const gwn_build_opts* o, const double* q, int nq,
                            double beta, double* bvh64, double* direct64) {
    init_tables();
    HostModel H;
    gwn_status code;
    if (!build_model_3d(patches, n, *o, &H, &code).empty()) return -1;
    const DevTree t = host_tree(H, 1, o->order);
    for (int i = 0; i < nq; ++i) {
        uint32_t s = 0;
        bvh64[i] = query3_64(t, q[3 * i], q[3 * i + 1], q[3 * i + 2], beta * beta, s);
        direct64[i] = query3_64(t, q[3 * i], q[3 * i + 1], q[3 * i + 2], 0.0, s);
    }
    return t.n_leaves;
}
