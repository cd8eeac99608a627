// build_device.h -- the device stage of the 3D build (build_device.cu): the
// per-leaf work that dominates the build -- leaf moments and the packing of the
// leaves' boundary curves -- one thread per leaf or per curve, with the same
// arithmetic as the host stage (curves3d.h), so the model is the same either way.
#pragma once

#include <string>
#include <vector>

#include "build.h"
#include "curves3d.h"

namespace gwn {

// Leaf moments (leaf_moments_core) of nl leaves: nets[i], the pieces
// [off[i], off[i + 1]) of `pieces` with multiplicities `mult`, the n-point
// rule (gx, gw).  mom receives kLeafMom3 (120) doubles per leaf, area_ax 4 (area, ax).
// Runs on the current CUDA device; returns "" or an error message.
std::string device_leaf_moments(const std::vector<Net>& nets, const std::vector<TP>& pieces,
                                const std::vector<double>& mult, const std::vector<int>& off, const double* xref,
                                const std::vector<double>& gx, const std::vector<double>& gw, std::vector<double>* mom,
                                std::vector<double>* area_ax);

// Packing (pack_curve) of nc boundary curves into the arrays of `out`, which
// the caller has sized: curve g is pieces[g] with multiplicity mult[g] on leaf
// curve_leaf[g] (nets[leaf], centre cen[3 leaf ..]), its points at ctrl_off[g].
// x4, w4: the 4-point rule; x8: the 8-point rule.  Returns "" or a message.
std::string device_pack_curves(const std::vector<Net>& nets, const std::vector<float>& cen,
                               const std::vector<TP>& pieces, const std::vector<double>& mult,
                               const std::vector<int>& curve_leaf, const std::vector<int32_t>& ctrl_off,
                               const std::vector<double>& x4, const std::vector<double>& w4,
                               const std::vector<double>& x8, HostModel* out);

}  // namespace gwn
