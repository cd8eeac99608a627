// kernels3d.cuh -- device routines of the 3D query (Algorithm 1, query half).
#pragma once

#include "gwn_internal.h"
#include "../../include/gwn.h"

namespace gwn {

__device__ __forceinline__ float leaf3_eval32(const DevTree& t, int li, float qx, float qy, float qz, uint32_t& st) {
    (void)t; (void)li; (void)qx; (void)qy; (void)qz;
    st |= GWN_QS_UNRESOLVED;
    return 0.f;
}
__device__ __forceinline__ double leaf3_eval64(const DevTree& t, int li, double qx, double qy, double qz, uint32_t& st) {
    (void)t; (void)li; (void)qx; (void)qy; (void)qz;
    st |= GWN_QS_UNRESOLVED;
    return 0.0;
}
__device__ __forceinline__ float query3_32(const DevTree& t, float qx, float qy, float qz, float beta2, uint32_t& st) {
    (void)t; (void)qx; (void)qy; (void)qz; (void)beta2;
    st |= GWN_QS_UNRESOLVED;
    return 0.f;
}
__device__ __forceinline__ double query3_64(const DevTree& t, double qx, double qy, double qz, double beta2, uint32_t& st) {
    (void)t; (void)qx; (void)qy; (void)qz; (void)beta2;
    st |= GWN_QS_UNRESOLVED;
    return 0.0;
}

}  // namespace gwn
