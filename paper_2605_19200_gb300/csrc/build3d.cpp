// build3d.cpp -- 3D preprocessing of Algorithm 1 (trimmed NURBS patches).
#include "build.h"

namespace gwn {

std::string build_model_3d(const gwn_patch3d* patches, size_t n, const gwn_build_opts& o, HostModel* out,
                           gwn_status* code) {
    (void)patches; (void)n; (void)o; (void)out;
    *code = GWN_ERR_INVALID_ARG;
    return "3D models are not available in this build";
}

}  // namespace gwn
