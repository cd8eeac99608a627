// gwn_internal.h -- data layouts shared by the host build and the CUDA kernels.
//
// A model is a BVH (Section 3.1; top-down sweep or Karras LBVH, numbered alike)
// over leaf primitives.  Internal node k (0 <= k < n_leaves - 1) stores its
// centroid x0 and squared radius r^2 (radius
// = half the diagonal of the node's control-point box, Section 3), its two
// children (>= 0: internal node, < 0: leaf ~i), and the Taylor coefficients
// of Eq. 3 (order 2; order 3 in 3D as an extension) folded into the polynomial
// form evaluated by the kernels (see fold_moments_2d / fold_moments_3d in
// build.cpp):
//
//   2D  w = i2 (A0.r + a1 + i2 (r^T B r + c.r + i2 D[r r r])),  i2 = 1/|r|^2
//   3D  w = i3 (A0.r + a1 + i2 (r^T B r + c.r + e + i2 (D[r r r] + r^T F r
//                + i2 G[r r r r]))),                             i3 = 1/|r|^3
//
// with r = x0 - q (e, F, G: the order-3 terms, zero below order 3).  Every array is a structure of arrays indexed by node or
// leaf so that a node visit reads one 16-byte header, and the moment block is
// read only when the far test passes.
#pragma once

#include <cstdint>

#ifdef __CUDACC__
#include <cuda_runtime.h>
#else
struct alignas(16) float4 { float x, y, z, w; };
struct alignas(8) int2 { int x, y; };
#endif

// Device routines are also compiled for the host (GWN_HD) so that they can be
// exercised on a CPU; GWN_LDG is a read-only cached load on the device.
#ifdef __CUDACC__
#define GWN_HD __host__ __device__
#else
#define GWN_HD
#endif
#if defined(__CUDA_ARCH__)
#define GWN_LDG(p) __ldg(p)
#else
#define GWN_LDG(p) (*(p))
#endif

namespace gwn {

constexpr int kMom2Vec = 3;    // float4 per 2D moment block (12 floats)
constexpr int kMom3Vec = 12;   // float4 per 3D moment block (45 floats + pad; the first 6 hold order <= 2)
constexpr int kMom2F64 = 12;   // doubles per 2D moment block
constexpr int kMom3F64 = 48;   // doubles per 3D moment block
constexpr int kLeafMom3 = 120; // uncentred 3D moments of a leaf: 3 + 9 + 27 + 81
// 2D leaf: cubic rational Bezier stored as a centre c (float) plus offsets of
// the control points from c, so that near queries lose no precision to the
// absolute magnitude of the coordinates:
//   (o0 o1) (o2 o3) (w0 w1 w2 w3) (c.x c.y 0 0)
constexpr int kLeaf2Vec = 4;
constexpr int kLeaf2F64 = 12;  // absolute (x0 y0 x1 y1 x2 y2 x3 y3 w0 w1 w2 w3)

// 3D leaf: local [0,1]^2 rational bicubic Bezier net (16 homogeneous points),
// box, mean normal, and ranges into the boundary-curve tables.
constexpr int kNet3Vec = 16;   // float4 (w x, w y, w z, w) per leaf
struct Leaf3Info {
    float cen[3];              // leaf centre; float geometry of the leaf is stored relative to it
    float rad;                 // half the box diagonal
    float nrm[3];              // unit mean normal (string direction for near queries)
    float diag;                // box diagonal
    int32_t c3_off, c3_cnt;    // 3D boundary curves (composition of trims with the surface)
    int32_t c2_off, c2_cnt;    // 2D boundary curves in local (u, v) for the trim membership test
};

// A 3D boundary curve: rational Bezier of degree D = deg (<= kMaxC3Deg) stored
// from ctrl_off in the curve-point array as D + 1 homogeneous points scaled by
// their binomial coefficients C(D, i) c_i, followed by the D derivative points
// C(D-1, i) (c_{i+1} - c_i), then the same 2 D + 1 points of the reversed
// curve (evaluation for t > 1/2 reads them in forward order), and counted `mult`
// times (winding multiplicity of a clipped rectangle edge).  min_level: the
// FP32 line integral starts with 2^min_level panels, the level at which the
// 4-point rule resolves the curve's own rational parametrisation (the complex
// zeros of its weight polynomial; a quarter circle needs level 1).
constexpr int kMaxC3Deg = 18;
constexpr int kMaxMinLevel = 8;
struct Curve3Info {
    int32_t ctrl_off;
    int32_t deg;
    float mult;
    int32_t min_level;
};

// Query-independent node table of one boundary curve (same index as its
// Curve3Info), kC3NodeVec float4:
//   [0]       (len0, len1a, len1b, mult): the length estimate of the level-0
//             panel and of the two level-1 panels (sum of the chords between
//             the 4 Gauss-Legendre nodes x the rule's span factor), and mult
//   [1..6]    level-0 panel: 4 nodes x (x, y, z, dx/dt, dy/dt, dz/dt)
//   [7..12]   level-1 panel [0, 1/2], same layout
//   [13..18]  level-1 panel [1/2, 1]
// with positions relative to the leaf centre.  A far (point, leaf) pair whose
// panels stop at level 0 or 1 evaluates the line integral from this table
// alone (leaf3_fast32): no curve evaluation per query.
constexpr int kC3NodeVec = 19;
// FP64 node table of one boundary curve for the FP64 repair (8-point
// Gauss-Legendre rule, absolute coordinates), kC3Node64 doubles:
//   [0..3]      (len0, len1a, len1b, mult), lengths with the 8-point rule's span factor
//   [4..51]     level-0 panel: 8 nodes x (x, y, z, dx/dt, dy/dt, dz/dt)
//   [52..99]    level-1 panel [0, 1/2]
//   [100..147]  level-1 panel [1/2, 1]
constexpr int kC3Node64 = 148;

// FP32 flops of one node read from a table (fast_panel in kernels3d.cuh): 3
// subtractions and 31 multiply/add operations, plus a square root and a
// reciprocal on the special-function unit
constexpr double kFastNodeFlops = 34.0;

// 2D boundary curve in local (u, v): rational cubic, 4 homogeneous points.
constexpr int kC2Vec = 3;      // float4 per 2D local curve: (h0 h1 h2 h3) as 12 floats, multiplicity kept in Curve2Mult

struct DevTree {
    int dim;
    int n_leaves;
    int n_internal;
    int root;                  // 0, or ~0 when the model has a single leaf
    int leaf_far;              // 1: leaves also take the far test (their own moments)
    int order3;                // 1: the FP32 traversal evaluates the order-3 terms
    int order3_64;             // 1: the FP64 evaluations (repair, FP64 precision) evaluate them: every
                               // model built with order 3, whatever order its FP32 bulk evaluates
    // per-leaf far-field data (same layout as the nodes)
    const float4* lhdr;
    const float4* lmom;
    const double* lhdr64;
    const double* lmom64;
    // internal nodes
    const float4* hdr;         // (x0.x, x0.y, x0.z, r^2)
    const int2* child;
    const float4* chdr;        // 3D: 2 per internal node, the headers of its two children (hdr or lhdr)
    const float4* mom;         // kMom2Vec or kMom3Vec per node
    const double* hdr64;       // 4 per node
    const double* mom64;       // kMom2F64 or kMom3F64 per node
    // 2D leaves
    const float4* leaf2;       // kLeaf2Vec per leaf
    const double* leaf2_64;    // kLeaf2F64 per leaf
    // 3D leaves
    const Leaf3Info* leaf3;
    const float4* net3;        // kNet3Vec per leaf
    const double* net3_64;     // 64 per leaf
    const Curve3Info* c3;
    const float4* c3pts;
    const double* c3pts64;     // 4 per point
    const float4* c3n;         // kC3NodeVec per boundary curve
    const double* c3n64;       // kC3Node64 per boundary curve
    const float4* c2;          // kC2Vec per local curve
    const double* c2_64;       // 12 per local curve
    const float* c2mult;
};

// Work counters (only when QueryParams::work != nullptr): the algorithmic
// units counted by the kernels, from which the benchmark forms the flops of
// its roofline numerator (per Gauss-Legendre node 28 D + 70, per Taylor term
// 72, per far test 10, per foot-point search 2000).
enum {
    kWorkNodes = 0,      // internal nodes visited (far test)
    kWorkLeafTests = 1,  // leaves visited (far test or direct)
    kWorkFar = 2,        // Taylor evaluations (nodes and leaves)
    kWorkLeaves = 3,     // exact leaf evaluations
    kWorkGlNodes = 4,    // Gauss-Legendre nodes of 3D boundary integrals
    kWorkGlDeg = 5,      // sum over those nodes of the curve degree D
    kWorkHits = 6,       // foot-point searches (3D near leaves)
    kWorkChords = 7,     // chord angles (2D leaf pieces)
    kWorkFastNodes = 8,  // Gauss-Legendre nodes read from the node tables (leaf3_fast32)
    kWorkLocal = 9,      // nodes and leaves taken by a packet's local expansion (k_trav3)
    kWorkCount = 10
};

struct WorkLocal {
    unsigned long long v[kWorkCount];
};

struct QueryParams {
    unsigned long long* work;  // nullptr: no counting
    float beta2;               // beta^2 of the FP32 pass (internal nodes)
    float beta2_leaf;          // beta^2 of the leaves' own far test (3D)
    double beta2_repair;       // beta^2 of the FP64 repair pass; <= 0: direct sum
    double beta2_repair_leaf;  // beta^2 of the repair's leaf far test (3D)
    float band;                // repair band around half-integers
    float kappa2;              // (packet local expansion ratio)^2; 0: off
    int mode;                  // GWN_MODE_*
    int precision;             // GWN_PREC_*
};

constexpr long long kRepairPairCap = 1ll << 22;  // FP64 repair pairs per repair pass
constexpr int kCounterCount = 16;                // device counters of one chunk

// The points of one FP64 repair pass and its scratch.  The list holds point
// indices into the arrays the repair kernels are given; count may exceed cap
// (entries past cap were not stored and are not repaired by this pass).
struct RepairList {
    const int* idx;
    const int* count;
    int cap;
    double* rw;         // FP64 sum per entry (3D: far field and in-place leaves, then the pairs)
    uint32_t* rst;      // status bits per entry (3D)
    int2* pairs;        // FP64 (entry, leaf) pairs (3D), kRepairPairCap
    int* npairs;        // their count
    int2* pairs2;       // those the FP64 node tables left to the full evaluator, kRepairPairCap
    int* npairs2;       // their count
};

// Scratch of one in-flight query (one chunk of points), carved from one
// device allocation (see workspace_layout in gwn_api.cu).
struct Workspace {
    int2* pairs64;    // near-band pairs (capacity n)
    int2* rpairs;     // FP64 repair pairs (kRepairPairCap, 3D)
    int2* rpairs2;    // of which the full FP64 evaluator takes (kRepairPairCap, 3D)
    double* rw;       // FP64 repair accumulators (n)
    int* perm;        // n
    int* key;         // n: Morton cell of each point (binning)
    int* hist;        // max(cells, n_leaves) + 1: binning histogram, then the pair sort's
    float* wacc;      // n
    uint32_t* st;     // n
    int2* pairs;      // pair capacity: (point, leaf) pairs of the traversal, in runs of one leaf;
                      // then those the node tables left to the full evaluator
    int2* pairs2;     // pair capacity: the pairs sorted by leaf
    int* counters;    // [0] pairs, [1] repair count, [2] near-band pairs, [3] overflowed points, [4] repair pairs,
                      // [5] overflowed points of the current round (list input), [6] total overflow,
                      // [7] pairs of finished rounds, [8] pairs left to the full evaluator this round,
                      // [9] the same over finished rounds, [10] repair pairs the FP64 tables left
    int* olist;       // n: points whose pairs did not fit (rounds alternate with olist2)
    int* olist2;      // n
    unsigned long long* work;  // kWorkCount counters
    unsigned long long* acc;   // per-query totals of the counters over all chunks
    int* rlist;       // n: points of this chunk to repair that did not fit the query's list
    int* rlist_g;     // n: the query's points to repair (indices into the whole query), one pass after its last chunk
    uint32_t* rst;    // n: status bits per repair-list entry
    int* gcount;      // [0] entries of rlist_g, [1] FP64 pairs of its pass, [2] of which the full evaluator
                      // takes (cleared once per query)
    unsigned* bbox;   // 8: the chunk's bounding box as order-preserving keys (k_bbox)
    int rcap;         // entries of rlist_g (= the points a workspace holds)
    long long pair_cap;
};

}  // namespace gwn
