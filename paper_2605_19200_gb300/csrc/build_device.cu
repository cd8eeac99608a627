// build_device.cu -- the device stage of the 3D build (build_device.h).
//
// The host stage subdivides the patches and clips their trims (branchy,
// cheap); the per-leaf arithmetic that dominates the build runs here: the
// leaf moments of Section 3.1 (Green's theorem, n-point Gauss-Legendre rules;
// one thread per leaf) and the boundary curves of the near field (composition
// with the leaf's net, point copies, FP32/FP64 node tables, minimum panel
// levels; one thread per curve).  The routines are those of curves3d.h, and
// this file is compiled without fused multiply-adds (-fmad=false), so the
// device stage writes the same bits as the host stage.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>
#include <vector>

#include "build_device.h"

namespace gwn {
namespace {

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() {
        if (p) cudaFree(p);
    }
};

template <typename T>
bool to_device(DevBuf& b, const T* src, size_t n) {
    if (n == 0) n = 1;
    if (cudaMalloc(&b.p, n * sizeof(T)) != cudaSuccess) return false;
    return src == nullptr || cudaMemcpy(b.p, src, n * sizeof(T), cudaMemcpyHostToDevice) == cudaSuccess;
}

bool ensure_binomials() {
    double T[40][40];
    for (int a = 0; a < 40; ++a)
        for (int b = 0; b < 40; ++b) T[a][b] = binom64_host(a, b);
    return cudaMemcpyToSymbol(c_binom64, T, sizeof(T)) == cudaSuccess;
}

struct Rule {
    double x[32], w[32];
    int n;
};

__global__ void k_leaf_moments(int nl, const Net* nets, const TP* pieces, const double* mult, const int* off,
                               double3 xref, Rule rule, double* mom, double* area_ax) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nl) return;
    const double xr[3] = {xref.x, xref.y, xref.z};
    double area, ax[3];
    leaf_moments_core(nets[i], pieces + off[i], mult + off[i], off[i + 1] - off[i], xr, rule.x, rule.w, rule.n,
                      mom + (size_t)i * kLeafMom3, &area, ax);
    area_ax[(size_t)i * 4] = area;
    for (int k = 0; k < 3; ++k) area_ax[(size_t)i * 4 + 1 + k] = ax[k];
}

struct Rules48 {
    double x4[4], w4[4], x8[8];
};

__global__ void k_pack_curves(int nc, const Net* nets, const float* cen, const TP* pieces, const double* mult,
                              const int* curve_leaf, const int32_t* ctrl_off, Rules48 r, Curve3Info* c3,
                              float4* pts32, double* pts64, float4* tab32, double* tab64, float4* c2, double* c2_64,
                              float* c2mult) {
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nc) return;
    const int leaf = curve_leaf[g];
    const float c[3] = {cen[3 * leaf], cen[3 * leaf + 1], cen[3 * leaf + 2]};
    const size_t o = (size_t)ctrl_off[g];
    Curve3Info ci;
    ci.ctrl_off = ctrl_off[g];
    pack_curve(pieces[g], mult[g], nets[leaf], c, r.x4, r.w4, r.x8, &ci, pts32 + o, pts64 + o * 4,
               tab32 + (size_t)g * kC3NodeVec, tab64 + (size_t)g * kC3Node64, c2 + (size_t)g * kC2Vec,
               c2_64 + (size_t)g * 12, c2mult + g);
    c3[g] = ci;
}

std::string cuda_msg(const char* what) {
    return std::string("device build stage: ") + what + ": " + cudaGetErrorString(cudaGetLastError());
}

}  // namespace

std::string device_leaf_moments(const std::vector<Net>& nets, const std::vector<TP>& pieces,
                                const std::vector<double>& mult, const std::vector<int>& off, const double* xref,
                                const std::vector<double>& gx, const std::vector<double>& gw, std::vector<double>* mom,
                                std::vector<double>* area_ax) {
    const int nl = (int)nets.size();
    Rule rule{};
    rule.n = (int)gx.size();
    if (rule.n > 32) return "device build stage: at most 32 quadrature nodes";
    for (int k = 0; k < rule.n; ++k) {
        rule.x[k] = gx[k];
        rule.w[k] = gw[k];
    }
    mom->assign((size_t)nl * kLeafMom3, 0.0);
    area_ax->assign((size_t)nl * 4, 0.0);
    if (nl == 0) return "";
    if (!ensure_binomials()) return cuda_msg("binomial table");
    DevBuf dn, dp, dm, doff, dmom, da;
    if (!to_device(dn, nets.data(), nets.size()) || !to_device(dp, pieces.data(), pieces.size()) ||
        !to_device(dm, mult.data(), mult.size()) || !to_device(doff, off.data(), off.size()) ||
        !to_device<double>(dmom, nullptr, mom->size()) || !to_device<double>(da, nullptr, area_ax->size()))
        return cuda_msg("upload");
    const int B = 64;
    k_leaf_moments<<<(nl + B - 1) / B, B>>>(nl, (const Net*)dn.p, (const TP*)dp.p, (const double*)dm.p,
                                            (const int*)doff.p, make_double3(xref[0], xref[1], xref[2]), rule,
                                            (double*)dmom.p, (double*)da.p);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return cuda_msg("k_leaf_moments");
    if (cudaMemcpy(mom->data(), dmom.p, mom->size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(area_ax->data(), da.p, area_ax->size() * sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
        return cuda_msg("download");
    return "";
}

std::string device_pack_curves(const std::vector<Net>& nets, const std::vector<float>& cen,
                               const std::vector<TP>& pieces, const std::vector<double>& mult,
                               const std::vector<int>& curve_leaf, const std::vector<int32_t>& ctrl_off,
                               const std::vector<double>& x4, const std::vector<double>& w4,
                               const std::vector<double>& x8, HostModel* out) {
    const int nc = (int)pieces.size();
    if (nc == 0) return "";
    Rules48 r{};
    for (int k = 0; k < 4; ++k) {
        r.x4[k] = x4[k];
        r.w4[k] = w4[k];
    }
    for (int k = 0; k < 8; ++k) r.x8[k] = x8[k];
    if (!ensure_binomials()) return cuda_msg("binomial table");
    DevBuf dn, dc, dp, dm, dl, dof, d3, dp32, dp64, dt32, dt64, dc2, dc2d, dc2m;
    if (!to_device(dn, nets.data(), nets.size()) || !to_device(dc, cen.data(), cen.size()) ||
        !to_device(dp, pieces.data(), pieces.size()) || !to_device(dm, mult.data(), mult.size()) ||
        !to_device(dl, curve_leaf.data(), curve_leaf.size()) || !to_device(dof, ctrl_off.data(), ctrl_off.size()) ||
        !to_device<Curve3Info>(d3, nullptr, out->c3.size()) || !to_device<float4>(dp32, nullptr, out->c3pts.size()) ||
        !to_device<double>(dp64, nullptr, out->c3pts64.size()) || !to_device<float4>(dt32, nullptr, out->c3n.size()) ||
        !to_device<double>(dt64, nullptr, out->c3n64.size()) || !to_device<float4>(dc2, nullptr, out->c2.size()) ||
        !to_device<double>(dc2d, nullptr, out->c2_64.size()) || !to_device<float>(dc2m, nullptr, out->c2mult.size()))
        return cuda_msg("upload");
    const int B = 64;
    k_pack_curves<<<(nc + B - 1) / B, B>>>(nc, (const Net*)dn.p, (const float*)dc.p, (const TP*)dp.p,
                                           (const double*)dm.p, (const int*)dl.p, (const int32_t*)dof.p, r,
                                           (Curve3Info*)d3.p, (float4*)dp32.p, (double*)dp64.p, (float4*)dt32.p,
                                           (double*)dt64.p, (float4*)dc2.p, (double*)dc2d.p, (float*)dc2m.p);
    if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) return cuda_msg("k_pack_curves");
    auto down = [](void* dst, const DevBuf& b, size_t bytes) {
        return bytes == 0 || cudaMemcpy(dst, b.p, bytes, cudaMemcpyDeviceToHost) == cudaSuccess;
    };
    if (!down(out->c3.data(), d3, out->c3.size() * sizeof(Curve3Info)) ||
        !down(out->c3pts.data(), dp32, out->c3pts.size() * sizeof(float4)) ||
        !down(out->c3pts64.data(), dp64, out->c3pts64.size() * sizeof(double)) ||
        !down(out->c3n.data(), dt32, out->c3n.size() * sizeof(float4)) ||
        !down(out->c3n64.data(), dt64, out->c3n64.size() * sizeof(double)) ||
        !down(out->c2.data(), dc2, out->c2.size() * sizeof(float4)) ||
        !down(out->c2_64.data(), dc2d, out->c2_64.size() * sizeof(double)) ||
        !down(out->c2mult.data(), dc2m, out->c2mult.size() * sizeof(float)))
        return cuda_msg("download");
    return "";
}

}  // namespace gwn
