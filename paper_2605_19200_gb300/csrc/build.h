// build.h -- host-side (FP64) model construction: the preprocessing half of
// Algorithm 1 (AdaptiveSubdivision, ComputeUncenteredMoments, ConstructBVH,
// SumUncenteredMomentsUpTree, CenterMomentsInPlace).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/gwn.h"
#include "gwn_internal.h"

namespace gwn {

// Everything a model needs on the device, in host memory, already in BVH order.
struct HostModel {
    int dim = 0;
    int n_leaves = 0;
    int max_depth = 0;
    double lo[3] = {0, 0, 0}, hi[3] = {0, 0, 0};
    // internal nodes (n_leaves - 1)
    std::vector<int2> child;
    std::vector<float4> hdr;
    std::vector<float4> mom;
    std::vector<double> hdr64;
    std::vector<double> mom64;
    // per-leaf far-field data (BVH order), used when leaves take the far test
    std::vector<float4> lhdr;
    std::vector<float4> lmom;
    std::vector<double> lhdr64;
    std::vector<double> lmom64;
    std::vector<double> x0;        // dim per node, absolute coordinates
    std::vector<double> r;         // radius per node
    std::vector<double> mom_c;     // centred moments per node (d + d^2 + d^3)
    // leaves in BVH order
    std::vector<int64_t> leaf_prim;
    std::vector<double> leaf_param;  // 4 per leaf
    // 2D leaf payload
    std::vector<float4> leaf2;
    std::vector<double> leaf2_64;
    // 3D leaf payload
    std::vector<Leaf3Info> leaf3;
    std::vector<float4> net3;
    std::vector<double> net3_64;
    std::vector<Curve3Info> c3;
    std::vector<float4> c3pts;
    std::vector<double> c3pts64;
    std::vector<float4> c3n;       // kC3NodeVec per boundary curve
    std::vector<double> c3n64;     // kC3Node64 per boundary curve
    std::vector<float4> c2;
    std::vector<double> c2_64;
    std::vector<float> c2mult;
};

// Leaf-level inputs of the generic tree build, in input (leaf) order.
struct LeafSet {
    int dim = 2;
    std::vector<double> box;    // 2 * dim per leaf: lo, hi
    std::vector<double> mom;    // uncentred moments about xref: d + d^2 + d^3 per leaf
    std::vector<double> wsum;   // centroid weight (chord length or area) per leaf
    std::vector<double> wx;     // weight * centroid (absolute), dim per leaf
    double xref[3] = {0, 0, 0}; // reference point of the uncentred moments
};

// Returns an empty string on success, else a message; *code receives the status.
std::string build_model_2d(const gwn_curve2d* curves, size_t n, const gwn_build_opts& o, HostModel* out,
                           gwn_status* code);
std::string build_model_3d(const gwn_patch3d* patches, size_t n, const gwn_build_opts& o, HostModel* out,
                           gwn_status* code);

// Hierarchy (tree_builder 0: Karras LBVH; else the top-down sweep, see
// gwn_build_opts::tree_builder) + up-sweep + centring + packing of the node
// arrays.  perm receives the BVH leaf order (perm[i] = input leaf index of BVH
// leaf i).  adaptive_beta: scale each cluster's far-test radius by its fill
// (see gwn_build_opts::adaptive_beta).
void build_tree(const LeafSet& L, int order, HostModel* out, std::vector<int>* perm, int adaptive_beta = 0,
                int tree_builder = 1);

// Validation of a clamped NURBS knot vector; returns "" when valid.
std::string check_knots(int degree, int n_ctrl, const double* knots);

// Bezier decomposition of a clamped NURBS in homogeneous coordinates of
// dimension hd (points of hd doubles).  Returns pieces * (degree + 1) points in
// `pieces` and the breakpoints in `brk` (pieces + 1 values).
int decompose(int degree, int n_ctrl, const double* knots, int hd, const double* hpts, std::vector<double>* pieces,
              std::vector<double>* brk);

}  // namespace gwn
