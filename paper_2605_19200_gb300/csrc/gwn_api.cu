// gwn_api.cu -- the C ABI (include/gwn.h): model construction, device upload,
// batched queries and inspection.
//
// Query pipeline for one call (Algorithm 1, "threaded batched query", one CUDA
// thread per query point):
//   1. k_query_*  : FP32 traversal (or FP32 direct sum).  Each thread writes
//                   its value, label and status and, when the value lies within
//                   `repair_band` of a half-integer or the traversal flagged a
//                   problem, appends its index to the model's repair list.
//   2. k_repair_* : persistent grid over the repair list; FP64 traversal with
//                   beta_repair (or the FP64 direct sum when beta_repair == 0).
// Both launches are on the caller's stream; the repair count lives in device
// memory, so no host synchronisation happens between them.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include <sys/stat.h>

#include "../../include/gwn.h"
#include "build.h"
#include "gwn_internal.h"
#include "kernels2d.cuh"
#include "kernels3d.cuh"
#include "query_pipeline.cuh"
#include "model.h"

using namespace gwn;

namespace {
thread_local std::string g_err;

gwn_status fail(gwn_status s, const std::string& msg) {
    g_err = msg;
    return s;
}

#define GWN_CUDA_TRY(call)                                                                    \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess) return fail(GWN_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    bool changed = false;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (dev >= 0 && dev != prev) {
            cudaSetDevice(dev);
            changed = true;
        }
    }
    ~DeviceGuard() {
        if (changed) cudaSetDevice(prev);
    }
};
}  // namespace



namespace {

template <typename V>
gwn_status upload(gwn_model_s* m, const std::vector<V>& v, const V** out) {
    *out = nullptr;
    if (v.empty()) return GWN_OK;
    void* p = nullptr;
    size_t bytes = v.size() * sizeof(V);
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) return fail(GWN_ERR_OOM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
    m->allocs.push_back(p);
    m->device_bytes += bytes;
    GWN_CUDA_TRY(cudaMemcpy(p, v.data(), bytes, cudaMemcpyHostToDevice));
    *out = reinterpret_cast<const V*>(p);
    return GWN_OK;
}

void free_model_memory(gwn_model_s* m) {
    for (void* p : m->allocs) cudaFree(p);
    m->allocs.clear();
    if (m->ws_mem) cudaFree(m->ws_mem);
    if (m->stage) cudaFree(m->stage);
    for (auto& row : m->ev)
        for (auto& e : row)
            if (e) cudaEventDestroy(e), e = nullptr;
    if (m->last) cudaEventDestroy(m->last);
    m->last = nullptr;
    m->last_recorded = false;
    m->ws_mem = nullptr;
    m->ws_bytes = 0;
    m->ws_n = 0;
    m->stage = nullptr;
    m->stage_cap = 0;
}

// constant tables of the 3D kernels (binomial coefficients, 8-point
// Gauss-Legendre rule on [0, 1]); uploaded once per device
std::mutex g_const_mu;
bool g_const_ready[256];

gwn_status init_constants(int dev) {
    std::lock_guard<std::mutex> lk(g_const_mu);
    if (dev < 0 || dev >= 256) return fail(GWN_ERR_INVALID_ARG, "device ordinal out of range");
    if (g_const_ready[dev]) return GWN_OK;
    float bin[kMaxC3Deg + 1][kMaxC3Deg + 1] = {};
    for (int a = 0; a <= kMaxC3Deg; ++a) {
        bin[a][0] = bin[a][a] = 1.f;
        for (int b = 1; b < a; ++b) bin[a][b] = bin[a - 1][b - 1] + bin[a - 1][b];
    }
    // n-point Gauss-Legendre nodes and weights on [0, 1]: Newton's method on the
    // Legendre polynomial P_n from the standard cosine initial guesses
    auto gauss = [](int n, double* x, double* w) {
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
    };
    double x[8], w[8], x4[4], w4[4];
    gauss(8, x, w);
    gauss(4, x4, w4);
    float xf[4], wf[4];
    for (int i = 0; i < 4; ++i) {
        xf[i] = (float)x4[i];
        wf[i] = (float)w4[i];
    }
    std::memcpy(h_binom, bin, sizeof(bin));
    std::memcpy(h_glx8, x, sizeof(x));
    std::memcpy(h_glw8, w, sizeof(w));
    std::memcpy(h_glx4f, xf, sizeof(xf));
    std::memcpy(h_glw4f, wf, sizeof(wf));
    std::memcpy(h_glx4d, x4, sizeof(x4));
    std::memcpy(h_glw4d, w4, sizeof(w4));
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_glx4d, x4, sizeof(x4)));
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_glw4d, w4, sizeof(w4)));
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_glx4f, xf, sizeof(xf)));
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_glw4f, wf, sizeof(wf)));
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_binom, bin, sizeof(bin)));
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_glx8, x, sizeof(x)));
    GWN_CUDA_TRY(cudaMemcpyToSymbol(c_glw8, w, sizeof(w)));
    g_const_ready[dev] = true;
    return GWN_OK;
}

gwn_status upload_model(gwn_model_s* m) {
    {
        int dev = 0;
        cudaGetDevice(&dev);
        gwn_status cs = init_constants(dev);
        if (cs != GWN_OK) return cs;
    }
    const HostModel& H = m->host;
    DevTree& t = m->tree;
    t.dim = H.dim;
    t.n_leaves = H.n_leaves;
    t.n_internal = H.n_leaves - 1;
    t.root = H.n_leaves > 1 ? 0 : ~0;
    gwn_status s;
#define UP(vec, field) if ((s = upload(m, H.vec, &t.field)) != GWN_OK) return s
    t.leaf_far = m->leaf_far;
    t.order3 = H.dim == 3 && m->eval_order >= 3 ? 1 : 0;
    t.order3_64 = H.dim == 3 && m->opts.order >= 3 ? 1 : 0;
    UP(lhdr, lhdr);
    UP(lmom, lmom);
    UP(lhdr64, lhdr64);
    UP(lmom64, lmom64);
    UP(hdr, hdr);
    UP(child, child);
    {
        // both children's headers beside each internal node (3D traversal): the
        // child indices and the headers load together instead of one after the other
        std::vector<float4> chdr;
        if (H.dim == 3) {
            chdr.resize(H.child.size() * 2);
            for (size_t k = 0; k < H.child.size(); ++k) {
                const int c[2] = {H.child[k].x, H.child[k].y};
                for (int j = 0; j < 2; ++j) chdr[2 * k + j] = c[j] < 0 ? H.lhdr[~c[j]] : H.hdr[c[j]];
            }
        }
        if ((s = upload(m, chdr, &t.chdr)) != GWN_OK) return s;
    }
    UP(mom, mom);
    UP(hdr64, hdr64);
    UP(mom64, mom64);
    UP(leaf2, leaf2);
    UP(leaf2_64, leaf2_64);
    UP(leaf3, leaf3);
    UP(net3, net3);
    UP(net3_64, net3_64);
    UP(c3, c3);
    UP(c3pts, c3pts);
    UP(c3pts64, c3pts64);
    UP(c3n, c3n);
    UP(c3n64, c3n64);
    UP(c2, c2);
    UP(c2_64, c2_64);
    UP(c2mult, c2mult);
#undef UP
    return GWN_OK;
}

gwn_status finish_build(gwn_model_s* m, gwn_model* out) {
    // the packet traversal's warp stack holds the pending second children along
    // one root-to-leaf path: sized from the tree's depth (deeper paths overflow,
    // are flagged and repaired)
    const int need = m->host.max_depth + 8;
    m->stack_depth = need <= 64 ? 64 : need <= 96 ? 96 : 128;
    gwn_status s = upload_model(m);
    if (s != GWN_OK) {
        free_model_memory(m);
        delete m;
        return s;
    }
    *out = m;
    return GWN_OK;
}

gwn_status check_opts(const gwn_build_opts& o, int dim) {
    if (!(o.beta == 0.0 || o.beta >= 2.0) || !std::isfinite(o.beta)) return fail(GWN_ERR_INVALID_ARG, "beta must be 0 (autotune) or >= 2");
    if (!(o.beta_leaf == 0.0 || o.beta_leaf >= 2.0)) return fail(GWN_ERR_INVALID_ARG, "beta_leaf must be 0 or >= 2");
    if (o.order < 0 || o.order > (dim == 3 ? 3 : 2))
        return fail(GWN_ERR_INVALID_ARG, dim == 3 ? "order must be 0, 1, 2 or 3" : "order must be 0, 1 or 2");
    if (o.adaptive_beta != 0 && o.adaptive_beta != 1) return fail(GWN_ERR_INVALID_ARG, "adaptive_beta must be 0 or 1");
    if (o.device_build < -1 || o.device_build > 1) return fail(GWN_ERR_INVALID_ARG, "device_build must be -1, 0 or 1");
    if (o.tree_builder < -1 || o.tree_builder > 1) return fail(GWN_ERR_INVALID_ARG, "tree_builder must be -1, 0 or 1");
    if (!(o.local_ratio <= 0.0 || (o.local_ratio >= 4.0 && o.local_ratio < 1e6)))
        return fail(GWN_ERR_INVALID_ARG, "local_ratio must be <= 0 or in [4, 1e6)");
    if (!(o.beta_repair <= 0.0 || o.beta_repair >= 2.0)) return fail(GWN_ERR_INVALID_ARG, "beta_repair must be <= 0 or >= 2");
    if (!(o.repair_band >= 0.0 && o.repair_band < 0.5)) return fail(GWN_ERR_INVALID_ARG, "repair_band must be in [0, 0.5)");
    if (o.quad_nodes < 1 || o.quad_nodes > 32) return fail(GWN_ERR_INVALID_ARG, "quad_nodes must be 1..32");
    if (o.precision < 0 || o.precision > 2) return fail(GWN_ERR_INVALID_ARG, "unknown precision");
    return GWN_OK;
}

// ------------------------------------------------------------------ kernels

__device__ __forceinline__ void load_point(const void* pts, int dtype, int dim, long long i, double* q) {
    if (dtype == GWN_F32) {
        const float* p = reinterpret_cast<const float*>(pts) + i * dim;
        for (int k = 0; k < dim; ++k) q[k] = (double)p[k];
    } else {
        const double* p = reinterpret_cast<const double*>(pts) + i * dim;
        for (int k = 0; k < dim; ++k) q[k] = p[k];
    }
}

__device__ __forceinline__ bool near_half(double w, float band) {
    double fr = w - floor(w);
    return fabs(fr - 0.5) < (double)band;
}

template <int DIM>
__global__ void __launch_bounds__(128) k_query32(DevTree t, const void* pts, int dtype, long long n, QueryParams p,
                                                 double* out_w, int* out_label, uint32_t* out_status, int* rlist,
                                                 int* rcount) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double qd[3];
    load_point(pts, dtype, DIM, i, qd);
    uint32_t st = 0;
    // the direct sum adds one FP32 value per leaf (thousands per query): the
    // running sum is kept in FP64 so that its rounding stays below the leaves' own
    double wd = 0.0;
    if (DIM == 2) {
        if (p.mode == GWN_MODE_DIRECT) {
            for (int l = 0; l < t.n_leaves; ++l) wd += (double)leaf2_eval32(t, l, (float)qd[0], (float)qd[1], st);
        } else {
            wd = (double)query2_32(t, (float)qd[0], (float)qd[1], p.beta2, st);
        }
    } else {
        if (p.mode == GWN_MODE_DIRECT) {
            for (int l = 0; l < t.n_leaves; ++l)
                wd += (double)leaf3_eval32(t, l, (float)qd[0], (float)qd[1], (float)qd[2], st);
        } else {
            wd = (double)query3_32(t, (float)qd[0], (float)qd[1], (float)qd[2], p.beta2, st);
        }
    }
    if (p.precision == GWN_PREC_FP32_REPAIR &&
        (near_half(wd, p.band) || (st & (GWN_QS_STACK_OVERFLOW | GWN_QS_UNRESOLVED)))) {
        int slot = atomicAdd(rcount, 1);
        rlist[slot] = (int)i;
    }
    out_w[i] = wd;
    if (out_label) out_label[i] = (int)round(wd);
    if (out_status) out_status[i] = st;
}

template <int DIM>
__device__ double query64(const DevTree& t, const double* q, double beta2, int mode, uint32_t& st,
                          double ratio = kRatio64Exact) {
    double b2 = (mode == GWN_MODE_DIRECT) ? 0.0 : beta2;
    if (DIM == 2) return query2_64(t, q[0], q[1], b2, st);
    return query3_64(t, q[0], q[1], q[2], b2, st, ratio);
}

// FP64 pass over every query (precision GWN_PREC_FP64)
template <int DIM>
__global__ void __launch_bounds__(128) k_query64(DevTree t, const void* pts, int dtype, long long n, QueryParams p,
                                                 double* out_w, int* out_label, uint32_t* out_status) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double q[3];
    load_point(pts, dtype, DIM, i, q);
    uint32_t st = 0;
    double w = query64<DIM>(t, q, p.mode == GWN_MODE_DIRECT ? 0.0 : (double)p.beta2, p.mode, st);
    out_w[i] = w;
    if (out_label) out_label[i] = (int)round(w);
    if (out_status) out_status[i] = st;
}

__global__ void k_iota(int n, int* list, int* count) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) list[i] = i;
    if (i == 0) *count = n;
}

// FP64 repair of the listed queries (persistent grid over the device-side
// count).  With beta_repair > 0 each thread re-runs the traversal in FP64;
// with beta_repair == 0 (exact direct sum) a whole warp shares one query, its
// lanes striding over the leaves, so that few repaired queries still fill the
// FP64 pipes.
template <int DIM>
__device__ __forceinline__ double leaf64(const DevTree& t, int l, const double* q, uint32_t& st, double ratio) {
    if (DIM == 2) return leaf2_eval64(t, l, q[0], q[1], st);
    return leaf3_eval64(t, l, q[0], q[1], q[2], st, ratio);
}

template <int DIM>
__global__ void __launch_bounds__(128) k_repair(DevTree t, const void* pts, int dtype, QueryParams p, double* out_w,
                                                int* out_label, uint32_t* out_status, const int* rlist,
                                                const int* rcount, int cap = 0x7fffffff) {
    int cnt = min(*rcount, cap);
    bool direct = p.mode == GWN_MODE_DIRECT || !(p.beta2_repair > 0);
    // the all-FP64 precision mode integrates to ~1e-8, the repair to ~1e-7
    const double ratio = p.precision == GWN_PREC_FP64 ? kRatio64Exact : kRatio64Repair;
    if (!direct) {
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
            int i = rlist[k];
            double q[3];
            load_point(pts, dtype, DIM, i, q);
            uint32_t st = 0;
            double w = query64<DIM>(t, q, p.beta2_repair, GWN_MODE_BVH, st, ratio);
            out_w[i] = w;
            if (out_label) out_label[i] = (int)round(w);
            if (out_status) out_status[i] = (out_status[i] | st | GWN_QS_REPAIRED);
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int nwarps = (gridDim.x * blockDim.x) >> 5;
    for (int k = warp; k < cnt; k += nwarps) {
        int i = rlist[k];
        double q[3];
        load_point(pts, dtype, DIM, i, q);
        uint32_t st = 0;
        double w = 0.0;
        for (int l = lane; l < t.n_leaves; l += 32) w += leaf64<DIM>(t, l, q, st, ratio);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, off);
            st |= __shfl_xor_sync(0xffffffffu, st, off);
        }
        if (lane == 0) {
            out_w[i] = w;
            if (out_label) out_label[i] = (int)round(w);
            if (out_status) out_status[i] = (p.precision == GWN_PREC_FP64 ? 0u : out_status[i]) | st | GWN_QS_REPAIRED;
        }
    }
}

// Bytes of the query workspace for n points of model m, and its layout.
// dim 0 lays out a workspace that serves both 2D and 3D models.
size_t workspace_layout(int dim, int n_leaves, size_t n, char* base, Workspace* ws) {
    const long long cap = dim != 2 ? (long long)n * 96 + 65536 : 0;
    const size_t cells = kMaxBinCells;  // the finest binning of either dimension
    const size_t hist = std::max(cells, (size_t)n_leaves) + 1;
    const size_t keyn = n;
    size_t off = 0;
    auto carve = [&](size_t bytes) {
        char* p = base ? base + off : nullptr;
        off += (bytes + 255) & ~size_t(255);
        return p;
    };
    Workspace w{};
    w.perm = (int*)carve(n * sizeof(int));
    w.key = (int*)carve(keyn * sizeof(int));
    w.hist = (int*)carve(hist * sizeof(int));
    w.wacc = (float*)carve(n * sizeof(float));
    w.st = (uint32_t*)carve(n * sizeof(uint32_t));
    w.pairs = (int2*)carve((size_t)cap * sizeof(int2));
    w.pairs2 = (int2*)carve((size_t)cap * sizeof(int2));  // pairs left to the full evaluator
    w.counters = (int*)carve(kCounterCount * sizeof(int));
    w.rpairs = (int2*)carve((dim != 2 ? (size_t)kRepairPairCap : 0) * sizeof(int2));
    w.rpairs2 = (int2*)carve((dim != 2 ? (size_t)kRepairPairCap : 0) * sizeof(int2));
    w.rw = (double*)carve(n * sizeof(double));
    w.pairs64 = (int2*)carve((dim != 2 ? n : 0) * sizeof(int2));
    w.rlist = (int*)carve(n * sizeof(int));
    w.rlist_g = (int*)carve(n * sizeof(int));
    w.rst = (uint32_t*)carve(n * sizeof(uint32_t));
    w.gcount = (int*)carve(8 * sizeof(int));
    w.bbox = (unsigned*)carve(8 * sizeof(unsigned));
    w.rcap = (int)n;
    w.olist = (int*)carve((dim != 2 ? n : 0) * sizeof(int));
    w.olist2 = (int*)carve((dim != 2 ? n : 0) * sizeof(int));
    w.work = (unsigned long long*)carve(kWorkCount * sizeof(unsigned long long));
    w.acc = (unsigned long long*)carve(kCounterCount * sizeof(unsigned long long));
    w.pair_cap = cap;
    if (ws) *ws = w;
    return off;
}

constexpr size_t kChunk = (size_t)1 << 20;  // points per pass of the query pipeline
constexpr int kQueryStats = 20;              // entries of gwn_last_query_stats

// beta of the FP64 repair when the build leaves it automatic: the exact sum over
// every leaf for small models, else the traversal at (by default) 3 beta, whose
// order-2 remainder is 3^-4 = 1/81 of the bulk's (Eq. 3's remainder falls like
// beta^-4); the autotuner may lower the factor (repair_node_factor)
double auto_beta_repair(const gwn_model_s* m, double beta) {
    return m->host.n_leaves <= 512 ? 0.0 : m->repair_node_factor * beta;
}

gwn_status ensure_workspace(gwn_model_s* m, size_t n, size_t stage_bytes) {
    n = std::min(n, kChunk);
    if (n > m->ws_n || !m->ws_mem) {
        size_t want = std::max<size_t>(n, 4096);
        size_t bytes = workspace_layout(m->dim, m->host.n_leaves, want, nullptr, nullptr);
        if (m->ws_mem) cudaFree(m->ws_mem);
        m->ws_mem = nullptr;
        cudaError_t e = cudaMalloc(&m->ws_mem, bytes);
        if (e != cudaSuccess) { m->ws_n = 0; m->ws_bytes = 0; return fail(GWN_ERR_OOM, "query workspace allocation failed"); }
        m->ws_bytes = bytes;
        m->ws_n = want;
        workspace_layout(m->dim, m->host.n_leaves, want, reinterpret_cast<char*>(m->ws_mem), &m->ws);
    }
    if (stage_bytes > m->stage_cap) {
        if (m->stage) cudaFree(m->stage);
        m->stage = nullptr;
        cudaError_t e = cudaMalloc(&m->stage, stage_bytes);
        if (e != cudaSuccess) { m->stage_cap = 0; return fail(GWN_ERR_OOM, "staging allocation failed"); }
        m->stage_cap = stage_bytes;
    }
    return GWN_OK;
}

}  // namespace

// Morton-cell bits per axis of the 3D binning of a chunk of n points: about
// ppc points per cell, 3..6 bits
static int bin_bits3(size_t n, int ppc) {
    const double cells = std::max(1.0, (double)n / std::max(1, ppc));
    const int b = (int)std::lround(std::log2(cells) / 3.0);
    return std::min(6, std::max(3, b));
}

// the kernels' parameters of one query
static QueryParams query_params(const gwn_model_s* m, const gwn_query_opts& qo, const Workspace& ws) {
    QueryParams p;
    p.work = qo.count_work ? ws.work : nullptr;
    double beta = qo.beta > 0 ? qo.beta : m->opts.beta;
    p.beta2 = (float)(beta * beta);
    double beta_leaf = qo.beta_leaf > 0 ? qo.beta_leaf : (m->opts.beta_leaf > 0 ? m->opts.beta_leaf : beta);
    p.beta2_leaf = (float)(beta_leaf * beta_leaf);
    double br = m->opts.beta_repair;
    const bool automatic = br < 0;
    if (automatic) br = auto_beta_repair(m, beta);
    p.beta2_repair = br > 0 ? br * br : 0.0;
    // the repair's leaves: the automatic factor times beta_leaf, or, with a given
    // beta_repair, the bulk's ratio beta_leaf / beta
    const double brl = br > 0 ? (automatic ? m->repair_leaf_factor * beta_leaf : br * beta_leaf / beta) : 0.0;
    p.beta2_repair_leaf = brl > 0 ? brl * brl : 0.0;
    p.band = (float)(qo.repair_band > 0 ? qo.repair_band : m->opts.repair_band);
    // packet local expansion (3D, order-2 evaluation): the query's ratio, else the model's; < 0 off
    const double kap = qo.local_ratio != 0.0 ? qo.local_ratio : m->local_ratio;
    p.kappa2 = m->dim == 3 && !m->tree.order3 && kap > 0 ? (float)(kap * kap) : 0.f;
    p.mode = qo.mode;
    p.precision = qo.precision >= 0 ? qo.precision : m->opts.precision;
    return p;
}

static int device_sms() {
    int dev = 0, sms = 152;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

// FP64 re-evaluation (GWN_PREC_FP32_REPAIR) of the points in list R, whose
// indices address pts and the outputs.  3D always goes through the warp
// traversal and the FP64 pair list: with beta_repair = 0 or in direct mode
// (exact sum over every leaf) every leaf becomes a pair, and the pairs of all
// repaired points spread over the whole GPU instead of one warp walking all
// leaves per point.
static gwn_status enqueue_repair(gwn_model_s* m, const QueryParams& p, const void* pts, int dtype, const RepairList& R,
                                 double* out_w, int* out_label, uint32_t* out_status, cudaStream_t st, int sms) {
    const int B = 128;
    const unsigned rb = (unsigned)(sms * 8);
    const unsigned wb = (unsigned)(sms * 4);  // blocks of kRepairWarps warps, one warp per repaired point
    if (m->dim == 2 && (p.mode == GWN_MODE_DIRECT || !(p.beta2_repair > 0))) {
        k_repair<2><<<rb, B, 0, st>>>(m->tree, pts, dtype, p, out_w, out_label, out_status, R.idx, R.count, R.cap);
    } else if (m->dim == 2) {
        k_rtrav_warp<2><<<wb, 32 * kRepairWarps, 0, st>>>(m->tree, pts, dtype, p.beta2_repair, R, out_w, out_label,
                                                         out_status);
    } else {
        const bool direct = p.mode == GWN_MODE_DIRECT;
        k_rtrav_warp<3><<<wb, 32 * kRepairWarps, 0, st>>>(m->tree, pts, dtype, direct ? 0.0 : p.beta2_repair, R,
                                                         out_w, out_label, out_status,
                                                         direct ? 0.0 : p.beta2_repair_leaf);
        k_rpairs3_fast<<<(unsigned)(sms * 8), B, 0, st>>>(m->tree, pts, dtype, R);
        k_rpairs3_warp<<<(unsigned)(sms * 8), B, 0, st>>>(m->tree, pts, dtype, R);
        k_rfinish<<<(unsigned)(sms * 2), B, 0, st>>>(R, out_w, out_label, out_status);
    }
    GWN_CUDA_TRY(cudaGetLastError());
    return GWN_OK;
}

// Enqueue the query kernels of one chunk (points off .. off + n - 1 of the
// query; pts and the outputs point at the chunk) on `st`, using workspace
// `ws` (sized for at least n points).  Shared with the batched and serving
// entry points through gwn_enqueue_device.
static gwn_status enqueue_chunk(gwn_model_s* m, const void* pts, int dtype, size_t n, size_t off, double* out_w,
                                int* out_label, uint32_t* out_status, const gwn_query_opts& qo, cudaStream_t st,
                                const Workspace& ws) {
    const QueryParams p = query_params(m, qo, ws);
    const int pc = m->prof_chunks;
    const bool prof = qo.profile != 0 && pc < gwn_model_s::kMaxProfChunks;
    cudaEvent_t* ev = prof ? m->ev[pc] : nullptr;
    if (prof) {
        if (!ev[0])
            for (int k = 0; k < 5; ++k) GWN_CUDA_TRY(cudaEventCreate(&ev[k]));
        m->prof_chunks = pc + 1;
    }
    const int B = 128;
    const int ni = (int)n;
    const unsigned nb = (unsigned)((n + B - 1) / B);
    const int sms = device_sms();
    if (p.precision == GWN_PREC_FP64) {
        if (p.mode == GWN_MODE_DIRECT) {
            // exact FP64 direct sum, one warp per point (lanes stride over the leaves)
            k_iota<<<nb, B, 0, st>>>(ni, ws.rlist, ws.counters + 1);
            unsigned rb = (unsigned)std::min<long long>(((long long)n * 32 + B - 1) / B, (long long)sms * 16);
            QueryParams pd = p;
            pd.beta2_repair = 0.0;
            if (m->dim == 2) k_repair<2><<<rb, B, 0, st>>>(m->tree, pts, dtype, pd, out_w, out_label, out_status, ws.rlist, ws.counters + 1);
            else k_repair<3><<<rb, B, 0, st>>>(m->tree, pts, dtype, pd, out_w, out_label, out_status, ws.rlist, ws.counters + 1);
        } else {
            if (m->dim == 2) k_query64<2><<<nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status);
            else k_query64<3><<<nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status);
        }
        GWN_CUDA_TRY(cudaGetLastError());
        return GWN_OK;
    }
    int* rcount = ws.counters + 1;
    GWN_CUDA_TRY(cudaMemsetAsync(ws.counters, 0, kCounterCount * sizeof(int), st));
    if (p.mode == GWN_MODE_DIRECT) {
        if (m->dim == 2)
            k_query32<2><<<nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status, ws.rlist, rcount);
        else
            k_query32<3><<<nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status, ws.rlist, rcount);
        GWN_CUDA_TRY(cudaGetLastError());
    } else {
        // 1. spatial binning of the points (counting sort by Morton cell)
        const int* perm = nullptr;
        if (n >= 2048) {
            const int bits = m->dim == 2 ? kBinBits2 : bin_bits3(n, m->bin_ppc);
            const int cells = 1 << (m->dim * bits);
            GWN_CUDA_TRY(cudaMemsetAsync(ws.hist, 0, (size_t)cells * sizeof(int), st));
            GWN_CUDA_TRY(cudaMemsetAsync(ws.bbox, 0, 8 * sizeof(unsigned), st));
            const unsigned bb = (unsigned)std::min<long long>(nb, (long long)sms * 4);
            if (m->dim == 2) {
                k_bbox<2><<<bb, B, 0, st>>>(pts, dtype, ni, ws.bbox);
                k_bin<2><<<nb, B, 0, st>>>(pts, dtype, ni, ws.bbox, bits, ws.key, ws.hist);
            } else {
                k_bbox<3><<<bb, B, 0, st>>>(pts, dtype, ni, ws.bbox);
                k_bin<3><<<nb, B, 0, st>>>(pts, dtype, ni, ws.bbox, bits, ws.key, ws.hist);
            }
            k_scan<<<1, 1024, 0, st>>>(ws.hist, cells);
            k_scatter_perm<<<nb, B, 0, st>>>(ni, ws.key, ws.hist, ws.perm);
            GWN_CUDA_TRY(cudaGetLastError());
            perm = ws.perm;
        }
        // 2. traversal
        if (prof) GWN_CUDA_TRY(cudaEventRecord(ev[0], st));
        if (m->dim == 2) {
            k_trav2<<<nb, B, 0, st>>>(m->tree, pts, dtype, ni, perm, p.beta2, ws, p.work);
            if (prof) {
                GWN_CUDA_TRY(cudaEventRecord(ev[1], st));
                GWN_CUDA_TRY(cudaEventRecord(ev[2], st));
                GWN_CUDA_TRY(cudaEventRecord(ev[4], st));
                GWN_CUDA_TRY(cudaEventRecord(ev[3], st));
            }
        } else {
            // rounds: round 0 over all points; rounds 1, 2 over the points whose
            // (point, leaf) pairs did not fit the list in the previous round
            for (int round = 0; round < 3; ++round) {
                const int* list = round == 0 ? perm : (round == 1 ? ws.olist : ws.olist2);
                int* olist_out = round == 1 ? ws.olist2 : ws.olist;
                const int* ndev = round == 0 ? nullptr : ws.counters + 5;
                // instance by warp-stack size, by whether the order-3 terms are evaluated,
                // and by whether packets take far nodes by local expansion (order 2 only)
                if (!m->tree.order3 && p.kappa2 > 0.f) {
                    auto trav = m->stack_depth <= 64 ? k_trav3_local<64>
                                                     : m->stack_depth <= 96 ? k_trav3_local<96> : k_trav3_local<128>;
                    trav<<<nb, B, 0, st>>>(m->tree, pts, dtype, ni, list, p.beta2, p.beta2_leaf, ws, p.work, ndev,
                                           olist_out, p.kappa2);
                } else {
                    const bool o3 = m->tree.order3 != 0;
                    auto trav = m->stack_depth <= 64   ? (o3 ? k_trav3<64, true> : k_trav3<64, false>)
                                : m->stack_depth <= 96 ? (o3 ? k_trav3<96, true> : k_trav3<96, false>)
                                                       : (o3 ? k_trav3<128, true> : k_trav3<128, false>);
                    trav<<<nb, B, 0, st>>>(m->tree, pts, dtype, ni, list, p.beta2, p.beta2_leaf, ws, p.work, ndev,
                                           olist_out);
                }
                if (prof && round == 0) GWN_CUDA_TRY(cudaEventRecord(ev[1], st));
                GWN_CUDA_TRY(cudaGetLastError());
                // 3. exact leaves, sorted by leaf (one atomic per run of a leaf); far
                // pairs from the node tables, the rest, in leaf order, to the full
                // evaluator (ws.pairs is free again once the sorted copy exists)
                GWN_CUDA_TRY(cudaMemsetAsync(ws.hist, 0, (size_t)m->host.n_leaves * sizeof(int), st));
                k_pair_hist<<<(unsigned)(sms * 16), B, 0, st>>>(ws.pair_cap, ws.counters, ws.pairs, ws.hist);
                k_scan<<<1, 1024, 0, st>>>(ws.hist, m->host.n_leaves);
                k_pair_sort<<<(unsigned)(sms * 16), B, 0, st>>>(ws.pair_cap, ws.counters, ws.pairs, ws.hist, ws.pairs2);
                if (prof && round == 0) GWN_CUDA_TRY(cudaEventRecord(ev[2], st));
                k_pair_fast<<<(unsigned)(sms * 16), B, 0, st>>>(m->tree, pts, dtype, ws.pair_cap, ws.counters,
                                                                ws.pairs2, ws.wacc, ws.st, ws.pairs, p.work);
                if (prof && round == 0) GWN_CUDA_TRY(cudaEventRecord(ev[4], st));
                k_pair_eval<<<(unsigned)(sms * 8), B, 0, st>>>(m->tree, pts, dtype, ws.pair_cap, ws.counters + 8,
                                                               ws.counters, ws.pairs, ws.wacc, ws.st, ws.pairs64, ni,
                                                               p.work);
                if (prof && round == 0) GWN_CUDA_TRY(cudaEventRecord(ev[3], st));
                if (round < 2) k_next_round<<<1, 32, 0, st>>>(ws);
            }
            // the near band of all rounds in one launch: a round only re-traverses
            // points whose pairs overflowed, and those never enter the near band,
            // so every listed point's FP32 sum is final here
            k_pair_eval64_warp<<<(unsigned)(sms * 2), B, 0, st>>>(m->tree, pts, dtype, ni, ws.counters, ws.pairs64,
                                                                  ws.wacc, ws.st);
            k_overflow3<<<(unsigned)(sms * 2), B, 0, st>>>(m->tree, pts, dtype, p.beta2, ws, ws.olist);
        }
        GWN_CUDA_TRY(cudaGetLastError());
        // 4. outputs and the repair list
        k_finish<<<nb, B, 0, st>>>(ni, ws.wacc, ws.st, p.precision, p.band, out_w, out_label, out_status, ws.rlist,
                                   rcount, (int)off, ws.rlist_g, ws.gcount, ws.rcap);
        GWN_CUDA_TRY(cudaGetLastError());
    }
    if (p.precision == GWN_PREC_FP32_REPAIR) {
        // points of this chunk that did not fit the query's repair list (normally
        // none: the list holds as many points as a chunk), repaired right away;
        // direct mode, whose k_query32 lists every point locally, too
        const RepairList R{ws.rlist, rcount, ws.rcap, ws.rw, ws.rst, ws.rpairs, ws.counters + 4, ws.rpairs2,
                           ws.counters + 10};
        gwn_status s = enqueue_repair(m, p, pts, dtype, R, out_w, out_label, out_status, st, sms);
        if (s != GWN_OK) return s;
    }
    k_accum<<<1, 32, 0, st>>>(ws);
    GWN_CUDA_TRY(cudaGetLastError());
    return GWN_OK;
}

// Enqueue a query on `st` for device-resident points and outputs, in chunks of
// at most kChunk points (the workspace holds one chunk), or of max_chunk when
// smaller: the serving loop takes shorter kernels so that requests on other
// slots interleave.
gwn_status gwn_enqueue_device(gwn_model_s* m, const void* pts, int dtype, size_t n, double* out_w, int* out_label,
                              uint32_t* out_status, const gwn_query_opts& qo, cudaStream_t st, const Workspace& ws,
                              size_t max_chunk) {
    const size_t chunk = max_chunk > 0 ? std::min(max_chunk, kChunk) : kChunk;
    const size_t esz = (dtype == GWN_F32 ? sizeof(float) : sizeof(double)) * m->dim;
    GWN_CUDA_TRY(cudaMemsetAsync(ws.acc, 0, kCounterCount * sizeof(unsigned long long), st));
    if (qo.count_work) GWN_CUDA_TRY(cudaMemsetAsync(ws.work, 0, kWorkCount * sizeof(unsigned long long), st));
    m->prof_chunks = 0;
    m->profiled = qo.profile != 0;
    GWN_CUDA_TRY(cudaMemsetAsync(ws.gcount, 0, 8 * sizeof(int), st));
    for (size_t off = 0; off < n; off += chunk) {
        size_t c = std::min(chunk, n - off);
        gwn_status s = enqueue_chunk(m, reinterpret_cast<const char*>(pts) + off * esz, dtype, c, off, out_w + off,
                                     out_label ? out_label + off : nullptr, out_status ? out_status + off : nullptr,
                                     qo, st, ws);
        if (s != GWN_OK) return s;
    }
    // one FP64 repair pass over the points that every chunk listed (indices into
    // the whole query), so that the repair fills the GPU instead of running a
    // few warps after each chunk
    const QueryParams p = query_params(m, qo, ws);
    if (p.precision == GWN_PREC_FP32_REPAIR && p.mode == GWN_MODE_BVH) {
        const RepairList R{ws.rlist_g, ws.gcount, ws.rcap, ws.rw, ws.rst, ws.rpairs, ws.gcount + 1, ws.rpairs2,
                           ws.gcount + 2};
        gwn_status s = enqueue_repair(m, p, pts, dtype, R, out_w, out_label, out_status, st, device_sms());
        if (s != GWN_OK) return s;
        k_accum_repair<<<1, 32, 0, st>>>(ws);
        GWN_CUDA_TRY(cudaGetLastError());
    }
    return GWN_OK;
}

extern "C" {

void gwn_default_build_opts(gwn_build_opts* o) {
    if (!o) return;
    o->tolerance = 1e-4;
    o->max_aabb_frac = 0.1;
    o->order = 2;
    o->beta = 2.0;
    o->beta_repair = -1.0;
    o->repair_band = 1e-3;
    o->quad_nodes = 10;
    o->precision = GWN_PREC_FP32_REPAIR;
    o->device = -1;
    o->n_threads = 0;
    o->leaf_far = -1;
    o->beta_leaf = 0.0;
    o->adaptive_beta = 0;
    o->device_build = -1;
    o->tree_builder = -1;
    o->local_ratio = 0.0;
}

void gwn_default_query_opts(gwn_query_opts* q) {
    if (!q) return;
    q->mode = GWN_MODE_BVH;
    q->precision = -1;
    q->beta = 0.0;
    q->count_work = 0;
    q->profile = 0;
    q->beta_leaf = 0.0;
    q->repair_band = 0.0;
    q->local_ratio = 0.0;
}

// ---------------------------------------------------------------- autotuner
//
// Picks the far-field factors (beta for internal nodes, beta_leaf for 3D
// leaves) of a model, and for a 3D model built with order 3 the Taylor order
// the queries evaluate (3, or 2 from the same coefficients): validation points
// -- uniform in the model's box, plus points a little off the surface at
// random leaf centroids -- are evaluated exactly (FP64 direct sum on the
// device), then with the FP32 path for every candidate.  The candidates whose
// max |dGWN| stays below half the tolerance are ranked by counted work (flops
// per point) and the cheapest few of each order are timed (below).

__global__ void k_err(int n, const double* a, const double* b, double* out) {
    __shared__ double smax[128];
    double m = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = fmax(m, fabs(a[i] - b[i]));
    smax[threadIdx.x] = m;
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long*>(out), __double_as_longlong(smax[0]));
}

// max |a - b| over the points whose status carries GWN_QS_REPAIRED, and their count
__global__ void k_err_repaired(int n, const double* a, const double* b, const uint32_t* st, double* out, int* cnt) {
    __shared__ double smax[128];
    double m = 0;
    int c = 0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
        if (st[i] & GWN_QS_REPAIRED) {
            m = fmax(m, fabs(a[i] - b[i]));
            ++c;
        }
    smax[threadIdx.x] = m;
    atomicAdd(cnt, c);
    __syncthreads();
    for (int o = 64; o > 0; o >>= 1) {
        if (threadIdx.x < o) smax[threadIdx.x] = fmax(smax[threadIdx.x], smax[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) atomicMax(reinterpret_cast<unsigned long long*>(out), __double_as_longlong(smax[0]));
}

static gwn_status autotune(gwn_model_s* m) {
    const int d = m->dim;
    const HostModel& H = m->host;
    const int nu = 768, nn = 256, nv = nu + nn;
    std::vector<float> pts((size_t)nv * d);
    uint64_t seed = 0x9e3779b97f4a7c15ull ^ (uint64_t)H.n_leaves;
    auto rnd = [&]() {  // splitmix64
        seed += 0x9e3779b97f4a7c15ull;
        uint64_t z = seed;
        z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
        z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
        z ^= z >> 31;
        return (double)(z >> 11) * (1.0 / 9007199254740992.0);
    };
    for (int i = 0; i < nu; ++i)
        for (int k = 0; k < d; ++k) pts[(size_t)i * d + k] = (float)(H.lo[k] + rnd() * (H.hi[k] - H.lo[k]));
    double diag = 0;
    for (int k = 0; k < d; ++k) diag += (H.hi[k] - H.lo[k]) * (H.hi[k] - H.lo[k]);
    diag = std::sqrt(diag);
    for (int i = nu; i < nv; ++i) {
        int li = (int)(rnd() * H.n_leaves) % std::max(1, H.n_leaves);
        for (int k = 0; k < d; ++k) {
            double c = d == 3 ? (double)H.lhdr64[(size_t)li * 4 + k] : H.lhdr64[(size_t)li * 4 + k];
            pts[(size_t)i * d + k] = (float)(c + (rnd() - 0.5) * 0.02 * diag);
        }
    }
    float* dp = nullptr;
    double *ref = nullptr, *w = nullptr, *err = nullptr;
    GWN_CUDA_TRY(cudaMalloc(&dp, pts.size() * sizeof(float)));
    GWN_CUDA_TRY(cudaMalloc(&ref, nv * sizeof(double)));
    GWN_CUDA_TRY(cudaMalloc(&w, nv * sizeof(double)));
    GWN_CUDA_TRY(cudaMalloc(&err, sizeof(double)));
    GWN_CUDA_TRY(cudaMemcpy(dp, pts.data(), pts.size() * sizeof(float), cudaMemcpyHostToDevice));
    gwn_status s = ensure_workspace(m, nv, 0);
    gwn_query_opts qo;
    gwn_default_query_opts(&qo);
    qo.mode = GWN_MODE_DIRECT;
    qo.precision = GWN_PREC_FP64;
    if (s == GWN_OK) s = gwn_enqueue_device(m, dp, GWN_F32, nv, ref, nullptr, nullptr, qo, 0, m->ws);
    const double betas[] = {3.0, 3.5, 4.0, 4.5, 5.0, 5.5, 6.0, 7.0, 8.0, 10.0, 12.0, 16.0};
    // 2D leaves have no separate factor (0 = beta); 3D leaves: per-level factors
    const double leafb[] = {0.0, 2.0, 2.5, 2.75, 3.0, 3.25, 3.5, 4.0, 5.0};
    double best_cost = 1e300, best_b = 0, best_bl = 0;
    int best_o = m->eval_order;
    std::vector<std::tuple<double, double, double, int>> ok_cands;  // (counted flops, beta, beta_leaf, order)
    double fb_err = 1e300, fb_b = 0, fb_bl = 0;  // fallback: smallest error seen
    int fb_o = m->eval_order;
    const double tol = 0.5 * m->opts.tolerance;
    std::vector<int> orders{m->eval_order};
    if (d == 3 && m->opts.order >= 3) orders = {3, 2};
    for (int ord : orders)
    for (double b : betas) {
        m->tree.order3 = ord >= 3 ? 1 : 0;
        bool any_ok = false;
        for (double bl : leafb) {
            if (s != GWN_OK) break;
            if (d == 2 && bl != 0.0) continue;
            if (d == 3 && bl == 0.0) continue;
            if (bl > b) continue;
            double blv = bl == 0.0 ? b : bl;
            gwn_query_opts q2;
            gwn_default_query_opts(&q2);
            q2.precision = GWN_PREC_FP32;
            q2.beta = b;
            q2.beta_leaf = blv;
            q2.count_work = 1;
            s = gwn_enqueue_device(m, dp, GWN_F32, nv, w, nullptr, nullptr, q2, 0, m->ws);
            if (s != GWN_OK) break;
            cudaMemset(err, 0, sizeof(double));
            k_err<<<4, 128>>>(nv, ref, w, err);
            double e = 0;
            unsigned long long wk[kWorkCount] = {}, acc[kCounterCount] = {};
            if (cudaMemcpy(&e, err, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(wk, m->ws.work, sizeof(wk), cudaMemcpyDeviceToHost) != cudaSuccess ||
                cudaMemcpy(acc, m->ws.acc, sizeof(acc), cudaMemcpyDeviceToHost) != cudaSuccess) {
                s = fail(GWN_ERR_CUDA, "autotune readback failed");
                break;
            }
            // a candidate whose exact-leaf pairs overflow the work list is rejected:
            // its overflow path is slow and not counted
            if (acc[3] + acc[6] > 0) continue;
            if (e < fb_err) {
                fb_err = e;
                fb_b = b;
                fb_bl = blv;
                fb_o = ord;
            }
            double cost = 10.0 * (wk[kWorkNodes] + wk[kWorkLeafTests]) + (ord >= 3 ? 120.0 : 72.0) * wk[kWorkFar] +
                          28.0 * wk[kWorkGlDeg] + 70.0 * wk[kWorkGlNodes] + 2000.0 * wk[kWorkHits] +
                          kFastNodeFlops * wk[kWorkFastNodes] +
                          (d == 2 ? 60.0 * wk[kWorkLeaves] : 30.0 * wk[kWorkLeaves]);
            if (std::getenv("GWN_AUTOTUNE_VERBOSE"))
                std::fprintf(stderr,
                             "[gwn autotune] leaves=%d order=%d beta=%.1f beta_leaf=%.1f max|dGWN|=%.3g flops/pt=%.3g\n",
                             H.n_leaves, ord, b, blv, e, cost / nv);
            if (e <= tol) {
                any_ok = true;
                ok_cands.push_back({cost, b, blv, ord});
                if (cost < best_cost) {
                    best_cost = cost;
                    best_b = b;
                    best_bl = blv;
                    best_o = ord;
                }
            }
        }
        if (any_ok && b >= 8.0) break;  // larger beta only costs more
    }
    struct Free {
        std::vector<void*> p;
        ~Free() {
            for (void* q : p) cudaFree(q);
        }
    } frees{{ref, w, err, dp}};
    if (s != GWN_OK) return s;
    if (best_b == 0) {  // nothing met the tolerance: the most accurate candidate tried
        best_b = fb_b > 0 ? fb_b : 8.0;
        best_bl = fb_b > 0 ? fb_bl : 8.0;
        best_o = fb_o;
    }
    m->opts.beta = best_b;
    m->opts.beta_leaf = d == 3 ? best_bl : 0.0;
    m->eval_order = best_o;
    m->tree.order3 = d == 3 && best_o >= 3 ? 1 : 0;
    // Counted flops do not weigh the kernels alike (the traversal's far tests and
    // Taylor terms issue about twice the instructions per counted flop of the
    // node-table leaves), so among the accurate candidates the cheapest four by
    // count of each order are timed on one chunk of points uniform in the model's
    // box (binned and paired as a large query is: smaller samples bin and pair
    // differently and flipped the choice between close candidates from run to
    // run), and
    // the fastest is kept; then the binning's target points per cell is timed
    // the same way (the sample is binned at the resolution its size gives, as a
    // query is).
    if (ok_cands.size() > 1 || d == 3) {
        std::sort(ok_cands.begin(), ok_cands.end());
        {
            std::vector<std::tuple<double, double, double, int>> keep;
            int per_order[4] = {0, 0, 0, 0};
            for (const auto& c : ok_cands)
                if (per_order[std::get<3>(c)]++ < 4) keep.push_back(c);
            ok_cands.swap(keep);
        }
        const int nt = (int)kChunk;  // one full chunk: binned and paired as a large query is
        std::vector<float> tp((size_t)nt * d);
        for (int i = 0; i < nt; ++i)
            for (int k = 0; k < d; ++k) tp[(size_t)i * d + k] = (float)(H.lo[k] + rnd() * (H.hi[k] - H.lo[k]));
        float* dt = nullptr;
        double* wt = nullptr;
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        bool ok = cudaMalloc(&dt, tp.size() * sizeof(float)) == cudaSuccess &&
                  cudaMalloc(&wt, (size_t)nt * sizeof(double)) == cudaSuccess &&
                  cudaMemcpy(dt, tp.data(), tp.size() * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
                  cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess &&
                  ensure_workspace(m, nt, 0) == GWN_OK;
        // best of two timed runs after one untimed run (microseconds)
        auto timed = [&](double b, double bl) -> double {
            gwn_query_opts q3;
            gwn_default_query_opts(&q3);
            q3.beta = b;
            q3.beta_leaf = bl;
            float best = 1e30f;
            for (int rep = 0; rep < 3 && ok; ++rep) {
                ok = cudaEventRecord(e0, 0) == cudaSuccess &&
                     gwn_enqueue_device(m, dt, GWN_F32, nt, wt, nullptr, nullptr, q3, 0, m->ws) == GWN_OK &&
                     cudaEventRecord(e1, 0) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
                float ms = 0;
                if (ok && rep > 0 && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess) best = std::min(best, ms);
            }
            return 1e3 * best;
        };
        double best_t = 1e300;
        if (ok_cands.size() > 1) {
            for (const auto& c : ok_cands) {
                m->tree.order3 = d == 3 && std::get<3>(c) >= 3 ? 1 : 0;
                const double tus = timed(std::get<1>(c), std::get<2>(c));
                if (std::getenv("GWN_AUTOTUNE_VERBOSE"))
                    std::fprintf(stderr, "[gwn autotune] order=%d beta=%.1f beta_leaf=%.1f: %.1f us for %d points\n",
                                 std::get<3>(c), std::get<1>(c), std::get<2>(c), tus, nt);
                if (ok && tus < best_t) {
                    best_t = tus;
                    m->opts.beta = std::get<1>(c);
                    m->opts.beta_leaf = d == 3 ? std::get<2>(c) : 0.0;
                    m->eval_order = std::get<3>(c);
                }
            }
            m->tree.order3 = d == 3 && m->eval_order >= 3 ? 1 : 0;
        }
        if (d == 3 && ok) {
            const double bl = m->opts.beta_leaf > 0 ? m->opts.beta_leaf : m->opts.beta;
            int best_ppc = m->bin_ppc;
            double bt = 1e300;
            for (int ppc : {4, 8, 16, 32, 64}) {
                m->bin_ppc = ppc;
                const double tus = timed(m->opts.beta, bl);
                if (ok && tus < bt) {
                    bt = tus;
                    best_ppc = ppc;
                }
            }
            m->bin_ppc = best_ppc;
        }
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        cudaFree(dt);
        cudaFree(wt);
        if (!ok) return fail(GWN_ERR_CUDA, "autotune timing failed");
    }
    // The automatic FP64 repair (more than 512 leaves): every validation point
    // whose value is fractional is sent through the repair (band 0.4999), and the
    // node and leaf factors are lowered from 3 while its values stay within 1e-7
    // of the FP64 direct sum; fewer FP64 pairs per repaired point.
    if (d == 3 && m->opts.beta_repair < 0 && H.n_leaves > 512 && m->opts.precision == GWN_PREC_FP32_REPAIR) {
        const double facs[][2] = {{3.0, 3.0}, {2.5, 2.5}, {2.5, 2.0}, {2.0, 2.0}, {2.0, 1.5}, {1.5, 1.5}};
        uint32_t* dst = nullptr;
        int* dcnt = nullptr;
        bool ok = cudaMalloc(&dst, nv * sizeof(uint32_t)) == cudaSuccess && cudaMalloc(&dcnt, sizeof(int)) == cudaSuccess;
        double keep_n = m->repair_node_factor, keep_l = m->repair_leaf_factor;
        for (const auto& f : facs) {
            if (!ok) break;
            m->repair_node_factor = f[0];
            m->repair_leaf_factor = f[1];
            gwn_query_opts qr;
            gwn_default_query_opts(&qr);
            qr.repair_band = 0.4999;
            double e = 0;
            int cnt = 0;
            ok = gwn_enqueue_device(m, dp, GWN_F32, nv, w, nullptr, dst, qr, 0, m->ws) == GWN_OK &&
                 cudaMemset(err, 0, sizeof(double)) == cudaSuccess && cudaMemset(dcnt, 0, sizeof(int)) == cudaSuccess;
            if (ok) k_err_repaired<<<4, 128>>>(nv, ref, w, dst, err, dcnt);
            ok = ok && cudaMemcpy(&e, err, sizeof(double), cudaMemcpyDeviceToHost) == cudaSuccess &&
                 cudaMemcpy(&cnt, dcnt, sizeof(int), cudaMemcpyDeviceToHost) == cudaSuccess;
            if (std::getenv("GWN_AUTOTUNE_VERBOSE"))
                std::fprintf(stderr, "[gwn autotune] repair factors %.1f / %.1f: max|dGWN| %.3g over %d repaired\n",
                             f[0], f[1], e, cnt);
            if (!ok || e > 1e-7) break;
            keep_n = f[0];
            keep_l = f[1];
        }
        m->repair_node_factor = keep_n;
        m->repair_leaf_factor = keep_l;
        if (dst) cudaFree(dst);
        if (dcnt) cudaFree(dcnt);
        if (!ok) return fail(GWN_ERR_CUDA, "autotune of the repair failed");
    }
    // the tuning workspace is not the model's: the first query sizes its own
    if (m->ws_mem) {
        cudaFree(m->ws_mem);
        m->ws_mem = nullptr;
        m->ws_n = 0;
        m->ws_bytes = 0;
    }
    return GWN_OK;
}

static gwn_status build_common(int dim, const void* prims, size_t n, const gwn_build_opts* opts, gwn_model* out) {
    if (!out) return fail(GWN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    gwn_build_opts o;
    gwn_default_build_opts(&o);
    if (opts) o = *opts;
    gwn_status s = check_opts(o, dim);
    if (s != GWN_OK) return s;
    auto t0 = std::chrono::steady_clock::now();
    gwn_model_s* m = new (std::nothrow) gwn_model_s();
    if (!m) return fail(GWN_ERR_OOM, "host allocation failed");
    m->dim = dim;
    m->opts = o;
    m->eval_order = o.order;
    m->local_ratio = o.local_ratio > 0 ? o.local_ratio : 0.0;
    m->leaf_far = o.leaf_far < 0 ? (dim == 3 ? 1 : 0) : (o.leaf_far ? 1 : 0);
    m->n_primitives = (int64_t)n;
    gwn_status code = GWN_OK;
    std::string err;
    // the device stage of the 3D build runs on the model's device
    DeviceGuard dg(o.device == GWN_DEVICE_HOST_ONLY ? -1 : o.device);
    try {
        if (dim == 2) err = build_model_2d(reinterpret_cast<const gwn_curve2d*>(prims), n, o, &m->host, &code);
        else err = build_model_3d(reinterpret_cast<const gwn_patch3d*>(prims), n, o, &m->host, &code);
    } catch (const std::bad_alloc&) {
        delete m;
        return fail(GWN_ERR_OOM, "host allocation failed during build");
    } catch (const std::exception& e) {
        delete m;
        return fail(GWN_ERR_INTERNAL, e.what());
    }
    if (!err.empty()) {
        delete m;
        return fail(code == GWN_OK ? GWN_ERR_INTERNAL : code, err);
    }
    if (o.device == GWN_DEVICE_HOST_ONLY) {  // inspection only: no device upload
        m->device = GWN_DEVICE_HOST_ONLY;
        m->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
        *out = m;
        return GWN_OK;
    }
    DeviceGuard g(o.device);
    cudaGetDevice(&m->device);
    bool tune = o.beta == 0.0;
    if (tune) m->opts.beta = 2.0;
    s = finish_build(m, out);
    if (s != GWN_OK) return s;
    if (tune) {
        s = autotune(m);
        if (s != GWN_OK) {
            gwn_release(m);
            *out = nullptr;
            return s;
        }
    }
    m->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return GWN_OK;
}

gwn_status gwn_build_2d(const gwn_curve2d* curves, size_t n, const gwn_build_opts* opts, gwn_model* out) {
    return build_common(2, curves, n, opts, out);
}

gwn_status gwn_build_3d(const gwn_patch3d* patches, size_t n, const gwn_build_opts* opts, gwn_model* out) {
    return build_common(3, patches, n, opts, out);
}

gwn_status gwn_query(gwn_model m, const void* points, int32_t dtype, int32_t mem, size_t n, double* out_w,
                     int32_t* out_label, uint32_t* out_status, const gwn_query_opts* qopts, void* stream) {
    if (!m) return fail(GWN_ERR_INVALID_ARG, "model is NULL");
    if (m->device == GWN_DEVICE_HOST_ONLY) return fail(GWN_ERR_INVALID_ARG, "model was built host-only");
    if (n == 0) return GWN_OK;
    if (!points || !out_w) return fail(GWN_ERR_INVALID_ARG, "points and out_w are required");
    if (dtype != GWN_F32 && dtype != GWN_F64) return fail(GWN_ERR_INVALID_ARG, "unknown points dtype");
    if (mem != GWN_MEM_DEVICE && mem != GWN_MEM_HOST) return fail(GWN_ERR_INVALID_ARG, "unknown memory kind");
    if (n > (size_t)0x7fffffff) return fail(GWN_ERR_INVALID_ARG, "at most 2^31 - 1 points per call");
    gwn_query_opts qo;
    gwn_default_query_opts(&qo);
    if (qopts) qo = *qopts;
    if (qo.mode != GWN_MODE_BVH && qo.mode != GWN_MODE_DIRECT) return fail(GWN_ERR_INVALID_ARG, "unknown mode");
    if (qo.precision < -1 || qo.precision > 2) return fail(GWN_ERR_INVALID_ARG, "unknown precision");
    if (qo.beta != 0.0 && !(qo.beta >= 2.0)) return fail(GWN_ERR_INVALID_ARG, "beta must be >= 2");
    if (qo.beta_leaf != 0.0 && !(qo.beta_leaf >= 2.0)) return fail(GWN_ERR_INVALID_ARG, "beta_leaf must be >= 2");
    if (!(qo.repair_band >= 0.0 && qo.repair_band < 0.5)) return fail(GWN_ERR_INVALID_ARG, "repair_band must be in [0, 0.5)");
    if (!(qo.local_ratio <= 0.0 || (qo.local_ratio >= 4.0 && qo.local_ratio < 1e6)))
        return fail(GWN_ERR_INVALID_ARG, "local_ratio must be <= 0 or in [4, 1e6)");
    DeviceGuard g(m->device);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    size_t esz = dtype == GWN_F32 ? sizeof(float) : sizeof(double);
    size_t pbytes = n * m->dim * esz;
    size_t obytes = n * (sizeof(double) + sizeof(int32_t) + sizeof(uint32_t));
    gwn_status s = ensure_workspace(m, n, mem == GWN_MEM_HOST ? pbytes + obytes + 64 : 0);
    if (s != GWN_OK) return s;
    // calls on other streams share the model's workspace: start after the previous call's work
    if (!m->last) GWN_CUDA_TRY(cudaEventCreateWithFlags(&m->last, cudaEventDisableTiming));
    if (m->last_recorded) GWN_CUDA_TRY(cudaStreamWaitEvent(st, m->last, 0));
    // the end of whatever this call enqueued, also when a later enqueue fails:
    // the next call must not reuse the workspace under kernels already queued
    auto mark_last = [&]() {
        if (cudaEventRecord(m->last, st) == cudaSuccess) m->last_recorded = true;
    };
    if (mem == GWN_MEM_DEVICE) {
        s = gwn_enqueue_device(m, points, dtype, n, out_w, out_label, (uint32_t*)out_status, qo, st, m->ws);
        mark_last();
        return s;
    }
    // host buffers: stage through model-owned device memory
    char* base = reinterpret_cast<char*>(m->stage);
    void* dp = base;
    double* dw = reinterpret_cast<double*>(base + ((pbytes + 15) & ~size_t(15)));
    int32_t* dl = reinterpret_cast<int32_t*>(dw + n);
    uint32_t* ds = reinterpret_cast<uint32_t*>(dl + n);
    GWN_CUDA_TRY(cudaMemcpyAsync(dp, points, pbytes, cudaMemcpyHostToDevice, st));
    s = gwn_enqueue_device(m, dp, dtype, n, dw, out_label ? dl : nullptr, out_status ? ds : nullptr, qo, st, m->ws);
    if (s != GWN_OK) {
        mark_last();
        return s;
    }
    GWN_CUDA_TRY(cudaMemcpyAsync(out_w, dw, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (out_label) GWN_CUDA_TRY(cudaMemcpyAsync(out_label, dl, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (out_status) GWN_CUDA_TRY(cudaMemcpyAsync(out_status, ds, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GWN_CUDA_TRY(cudaEventRecord(m->last, st));
    m->last_recorded = true;
    GWN_CUDA_TRY(cudaStreamSynchronize(st));
    return GWN_OK;
}

}  // extern "C"

// ---------------------------------------------------------------- query without allocation
//
// gwn_query_noalloc runs the FP32 traversal with FP64 repair without asking the
// CUDA runtime for memory: its only scratch -- the list of points to repair
// and its counter -- is the file-scope device array below, which every GPU
// that loads this library holds until the process exits.  Host code cannot
// use g_noalloc_scratch's name as a device address; the address comes from
// cudaGetSymbolAddress, once per device, on the first call made with that
// device current.

static constexpr size_t kNoAllocMaxPoints = (size_t)1 << 20;   // points per call
static constexpr int kNoAllocHeader = 64;                      // counter, padded to 256 bytes
static __device__ __align__(256) int g_noalloc_scratch[kNoAllocHeader + kNoAllocMaxPoints];

namespace {
std::mutex g_noalloc_mu;
int* g_noalloc_addr[256] = {};
int g_noalloc_sms[256] = {};

// the array's device address and the device's SM count, looked up once per
// device (with that device current) and cached
gwn_status noalloc_scratch(int dev, int** out, int* sms) {
    std::lock_guard<std::mutex> lk(g_noalloc_mu);
    if (dev < 0 || dev >= 256) return fail(GWN_ERR_INVALID_ARG, "device ordinal out of range");
    if (!g_noalloc_addr[dev]) {
        void* p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(GWN_ERR_CUDA, std::string("cudaGetSymbolAddress(no-alloc scratch): ") + cudaGetErrorString(e));
        int n_sm = 0;
        e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess || n_sm <= 0)
            return fail(GWN_ERR_CUDA, std::string("cudaDeviceGetAttribute(SM count): ") + cudaGetErrorString(e));
        g_noalloc_sms[dev] = n_sm;
        g_noalloc_addr[dev] = reinterpret_cast<int*>(p);
    }
    *out = g_noalloc_addr[dev];
    *sms = g_noalloc_sms[dev];
    return GWN_OK;
}

// one thread per point: Algorithm 1 in FP32 with every leaf evaluated in place;
// points near a half-integer or flagged go to the repair list
template <int DIM>
__global__ void __launch_bounds__(128) k_query_noalloc(DevTree t, const void* pts, int dtype, long long n, QueryParams p,
                                                       double* out_w, int* out_label, uint32_t* out_status, int* rlist,
                                                       int* rcount) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double qd[3];
    load_point(pts, dtype, DIM, i, qd);
    uint32_t st = 0;
    float w = DIM == 2 ? query2_32(t, (float)qd[0], (float)qd[1], p.beta2, st)
                       : query3_32(t, (float)qd[0], (float)qd[1], (float)qd[2], p.beta2, st, p.beta2_leaf);
    double wd = (double)w;
    if (near_half(wd, p.band) || (st & (GWN_QS_STACK_OVERFLOW | GWN_QS_UNRESOLVED))) rlist[atomicAdd(rcount, 1)] = (int)i;
    out_w[i] = wd;
    if (out_label) out_label[i] = (int)round(wd);
    if (out_status) out_status[i] = st;
}
}  // namespace

extern "C" gwn_status gwn_query_noalloc(gwn_model m, const void* points, int32_t dtype, size_t n, double* out_w,
                                        int32_t* out_label, uint32_t* out_status, void* stream) {
    if (!m) return fail(GWN_ERR_INVALID_ARG, "model is NULL");
    if (m->device == GWN_DEVICE_HOST_ONLY) return fail(GWN_ERR_INVALID_ARG, "model was built host-only");
    if (n == 0) return GWN_OK;
    if (!points || !out_w) return fail(GWN_ERR_INVALID_ARG, "points and out_w are required");
    if (dtype != GWN_F32 && dtype != GWN_F64) return fail(GWN_ERR_INVALID_ARG, "unknown points dtype");
    if (n > kNoAllocMaxPoints)
        return fail(GWN_ERR_INVALID_ARG, "gwn_query_noalloc takes at most " + std::to_string(kNoAllocMaxPoints) +
                                             " points per call (its scratch array has a fixed size); split the batch");
    DeviceGuard g(m->device);
    int* scratch = nullptr;
    int sms = 0;
    gwn_status s = noalloc_scratch(m->device, &scratch, &sms);
    if (s != GWN_OK) return s;
    int* rcount = scratch;
    int* rlist = scratch + kNoAllocHeader;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    QueryParams p{};
    p.work = nullptr;
    const double beta = m->opts.beta;
    const double beta_leaf = m->opts.beta_leaf > 0 ? m->opts.beta_leaf : beta;
    p.beta2 = (float)(beta * beta);
    p.beta2_leaf = (float)(beta_leaf * beta_leaf);
    double br = m->opts.beta_repair;
    if (br < 0) br = auto_beta_repair(m, beta);
    p.beta2_repair = br > 0 ? br * br : 0.0;
    p.band = (float)m->opts.repair_band;
    p.mode = GWN_MODE_BVH;
    p.precision = GWN_PREC_FP32_REPAIR;
    // the array keeps the previous call's contents: the counter must start at zero
    GWN_CUDA_TRY(cudaMemsetAsync(rcount, 0, sizeof(int), st));
    const int B = 128;
    const unsigned nb = (unsigned)((n + B - 1) / B);
    const unsigned rb = (unsigned)std::min<long long>(std::max<long long>(nb, sms * 4), (long long)sms * 8);
    if (m->dim == 2) {
        k_query_noalloc<2><<<nb, B, 0, st>>>(m->tree, points, dtype, (long long)n, p, out_w, out_label, out_status, rlist, rcount);
        k_repair<2><<<rb, B, 0, st>>>(m->tree, points, dtype, p, out_w, out_label, out_status, rlist, rcount);
    } else {
        k_query_noalloc<3><<<nb, B, 0, st>>>(m->tree, points, dtype, (long long)n, p, out_w, out_label, out_status, rlist, rcount);
        k_repair<3><<<rb, B, 0, st>>>(m->tree, points, dtype, p, out_w, out_label, out_status, rlist, rcount);
    }
    GWN_CUDA_TRY(cudaGetLastError());
    return GWN_OK;
}

extern "C" {

gwn_status gwn_last_query_stats(gwn_model m, int64_t* out) {
    if (!m || !out) return fail(GWN_ERR_INVALID_ARG, "NULL argument");
    DeviceGuard g(m->device);
    std::lock_guard<std::mutex> lk(m->mu);
    unsigned long long c[kCounterCount] = {};
    unsigned long long wk[kWorkCount] = {};
    if (m->ws_mem) {
        GWN_CUDA_TRY(cudaDeviceSynchronize());
        GWN_CUDA_TRY(cudaMemcpy(c, m->ws.acc, sizeof(c), cudaMemcpyDeviceToHost));
        GWN_CUDA_TRY(cudaMemcpy(wk, m->ws.work, sizeof(wk), cudaMemcpyDeviceToHost));
    }
    for (int k = 0; k < kQueryStats; ++k) out[k] = 0;
    for (int k = 0; k < 4; ++k) out[k] = (int64_t)c[k];
    out[0] = (int64_t)(c[0] + c[7]);  // pairs over all rounds
    out[2] = (int64_t)c[2];           // near-band (FP64) pairs over all rounds
    out[3] = (int64_t)(c[6] + c[3]);  // points whose pairs overflowed in any round
    for (int k = 0; k < 8; ++k) out[4 + k] = (int64_t)wk[k];
    out[14] = (int64_t)(c[8] + c[9]);  // pairs the full evaluator took (the rest came from the node tables)
    out[15] = (int64_t)wk[kWorkFastNodes];
    out[18] = (int64_t)wk[kWorkLocal];
    if (m->profiled) {
        double a = 0, b = 0, f = 0;
        for (int ch = 0; ch < m->prof_chunks; ++ch) {
            float x = 0, y = 0, z = 0;
            GWN_CUDA_TRY(cudaEventSynchronize(m->ev[ch][3]));
            GWN_CUDA_TRY(cudaEventElapsedTime(&x, m->ev[ch][0], m->ev[ch][1]));
            GWN_CUDA_TRY(cudaEventElapsedTime(&y, m->ev[ch][2], m->ev[ch][3]));
            GWN_CUDA_TRY(cudaEventElapsedTime(&z, m->ev[ch][2], m->ev[ch][4]));
            a += x;
            b += y;
            f += z;
        }
        out[12] = (int64_t)(a * 1000.0);
        out[13] = (int64_t)(b * 1000.0);
        out[16] = (int64_t)(f * 1000.0);
        out[17] = (int64_t)((b - f) * 1000.0);
    }
    return GWN_OK;
}

gwn_status gwn_model_info(gwn_model m, gwn_model_stats* s) {
    if (!m || !s) return fail(GWN_ERR_INVALID_ARG, "NULL argument");
    std::memset(s, 0, sizeof(*s));
    s->dim = m->dim;
    s->n_primitives = m->n_primitives;
    s->n_leaves = m->host.n_leaves;
    s->n_nodes = std::max(0, m->host.n_leaves - 1);
    s->max_depth = m->host.max_depth;
    s->device_bytes = (int64_t)m->device_bytes;
    s->build_ms = m->build_ms;
    s->beta = m->opts.beta;
    s->beta_repair = m->opts.beta_repair < 0 ? auto_beta_repair(m, m->opts.beta) : m->opts.beta_repair;
    s->repair_band = m->opts.repair_band;
    s->order = m->opts.order;
    s->eval_order = m->eval_order;
    s->local_ratio = m->dim == 3 ? m->local_ratio : 0.0;
    for (int k = 0; k < 3; ++k) {
        s->lo[k] = m->host.lo[k];
        s->hi[k] = m->host.hi[k];
    }
    s->beta_leaf = m->opts.beta_leaf > 0 ? m->opts.beta_leaf : m->opts.beta;
    s->device = m->device;
    s->bin_points_per_cell = m->dim == 3 ? m->bin_ppc : 0;
    s->stack_depth = m->stack_depth;
    {
        const double bl = m->opts.beta_leaf > 0 ? m->opts.beta_leaf : m->opts.beta;
        const double br = s->beta_repair;
        s->beta_repair_leaf = br > 0 ? (m->opts.beta_repair < 0 ? m->repair_leaf_factor * bl : br * bl / m->opts.beta)
                                     : 0.0;
    }
    return GWN_OK;
}

gwn_status gwn_model_leaves(gwn_model m, int64_t* prim, double* param) {
    if (!m) return fail(GWN_ERR_INVALID_ARG, "model is NULL");
    if (prim) std::memcpy(prim, m->host.leaf_prim.data(), m->host.leaf_prim.size() * sizeof(int64_t));
    if (param) std::memcpy(param, m->host.leaf_param.data(), m->host.leaf_param.size() * sizeof(double));
    return GWN_OK;
}

gwn_status gwn_model_tree(gwn_model m, int32_t* child, double* x0, double* r, double* mom) {
    if (!m) return fail(GWN_ERR_INVALID_ARG, "model is NULL");
    const HostModel& H = m->host;
    int ni = std::max(0, H.n_leaves - 1);
    if (child)
        for (int k = 0; k < ni; ++k) {
            child[2 * k] = H.child[k].x;
            child[2 * k + 1] = H.child[k].y;
        }
    if (x0) std::memcpy(x0, H.x0.data(), H.x0.size() * sizeof(double));
    if (r) std::memcpy(r, H.r.data(), H.r.size() * sizeof(double));
    if (mom) std::memcpy(mom, H.mom_c.data(), H.mom_c.size() * sizeof(double));
    return GWN_OK;
}

// ---------------------------------------------------------------- checkpoint
//
// A model file holds everything the device upload needs, so that a serving
// process can load a model without rebuilding it: a header (magic, format
// version, dimension, leaf mode, primitive count, build options after
// autotuning) and every host array of the model, each as a 64-bit element
// count followed by the raw elements.  Files are written and read on
// little-endian hosts (x86-64, aarch64) with the same struct layouts.

}  // extern "C"

namespace {
constexpr char kModelMagic[8] = {'G', 'W', 'N', 'M', 'O', 'D', 'E', 'L'};
constexpr uint32_t kModelVersion = 7;

template <typename V>
bool write_vec(FILE* f, const std::vector<V>& v) {
    const uint64_t n = v.size();
    return std::fwrite(&n, sizeof(n), 1, f) == 1 && (n == 0 || std::fwrite(v.data(), sizeof(V), n, f) == n);
}

// reads one array; `left` is the number of bytes of the file not read yet, so a
// corrupt count can neither allocate more than the file holds nor read past it
template <typename V>
bool read_vec(FILE* f, std::vector<V>* v, uint64_t* left) {
    uint64_t n = 0;
    if (*left < sizeof(n) || std::fread(&n, sizeof(n), 1, f) != 1) return false;
    *left -= sizeof(n);
    if (n > *left / sizeof(V)) return false;
    v->resize((size_t)n);
    if (n != 0 && std::fread(v->data(), sizeof(V), (size_t)n, f) != n) return false;
    *left -= n * sizeof(V);
    return true;
}

// Every array has the size the build gives it for the model's dimension and
// leaf count, every child index names a node or a leaf, each node and leaf
// except the root has exactly one parent (so the traversal ends), and every
// leaf's and boundary curve's ranges stay inside their tables.
bool host_model_consistent(const HostModel& H, int dim) {
    if (H.dim != dim || H.n_leaves < 1) return false;
    const size_t nl = (size_t)H.n_leaves, ni = nl - 1, d = (size_t)dim;
    const size_t fv = dim == 2 ? kMom2Vec : kMom3Vec, ff = dim == 2 ? kMom2F64 : kMom3F64;
    const size_t M = dim == 2 ? 2 + 4 + 8 : kLeafMom3;
    if (H.child.size() != ni || H.hdr.size() != ni || H.mom.size() != ni * fv || H.hdr64.size() != ni * 4 ||
        H.mom64.size() != ni * ff || H.lhdr.size() != nl || H.lmom.size() != nl * fv || H.lhdr64.size() != nl * 4 ||
        H.lmom64.size() != nl * ff || H.x0.size() != ni * d || H.r.size() != ni || H.mom_c.size() != ni * M ||
        H.leaf_prim.size() != nl || H.leaf_param.size() != nl * 4)
        return false;
    std::vector<unsigned char> parents(ni + nl, 0);
    for (size_t k = 0; k < ni; ++k)
        for (int c : {H.child[k].x, H.child[k].y}) {
            size_t slot;
            if (c >= 0) {
                if ((size_t)c >= ni || c == 0) return false;  // node 0 is the root
                slot = (size_t)c;
            } else {
                const long long li = ~(long long)c;
                if (li >= (long long)nl) return false;
                slot = ni + (size_t)li;
            }
            if (parents[slot]++) return false;
        }
    for (size_t k = 1; k < ni + nl; ++k)
        if (parents[k] != 1 && !(ni == 0 && k == 0)) return false;
    if (dim == 2) return H.leaf2.size() == nl * kLeaf2Vec && H.leaf2_64.size() == nl * kLeaf2F64;
    if (H.leaf3.size() != nl || H.net3.size() != nl * kNet3Vec || H.net3_64.size() != nl * 64 ||
        H.c3pts64.size() != H.c3pts.size() * 4 || H.c3n.size() != H.c3.size() * kC3NodeVec ||
        H.c3n64.size() != H.c3.size() * kC3Node64 ||
        H.c2.size() != H.c2mult.size() * kC2Vec ||
        H.c2_64.size() != H.c2mult.size() * 12)
        return false;
    for (const Curve3Info& c : H.c3)
        if (c.deg < 1 || c.deg > kMaxC3Deg || c.ctrl_off < 0 || c.min_level < 0 || c.min_level > kMaxMinLevel ||
            (size_t)c.ctrl_off + 2 * (2 * (size_t)c.deg + 1) > H.c3pts.size())
            return false;
    for (const Leaf3Info& I : H.leaf3)
        if (I.c3_off < 0 || I.c3_cnt < 0 || (size_t)I.c3_off + (size_t)I.c3_cnt > H.c3.size() || I.c2_off < 0 ||
            I.c2_cnt < 0 || (size_t)I.c2_off + (size_t)I.c2_cnt > H.c2mult.size())
            return false;
    return true;
}

// apply f to every array of the host model, in file order
template <typename F>
bool each_array(HostModel& H, F f) {
    return f(H.child) && f(H.hdr) && f(H.mom) && f(H.hdr64) && f(H.mom64) && f(H.lhdr) && f(H.lmom) &&
           f(H.lhdr64) && f(H.lmom64) && f(H.x0) && f(H.r) && f(H.mom_c) && f(H.leaf_prim) && f(H.leaf_param) &&
           f(H.leaf2) && f(H.leaf2_64) && f(H.leaf3) && f(H.net3) && f(H.net3_64) && f(H.c3) && f(H.c3pts) &&
           f(H.c3pts64) && f(H.c3n) && f(H.c3n64) && f(H.c2) && f(H.c2_64) && f(H.c2mult);
}
}  // namespace

extern "C" {

gwn_status gwn_model_save(gwn_model m, const char* path) {
    if (!m || !path) return fail(GWN_ERR_INVALID_ARG, "model and path are required");
    FILE* f = std::fopen(path, "wb");
    if (!f) return fail(GWN_ERR_INVALID_ARG, std::string("cannot open for writing: ") + path);
    const int32_t hdr[4] = {(int32_t)kModelVersion, m->dim, m->leaf_far, (int32_t)sizeof(gwn_build_opts)};
    const HostModel& H = m->host;
    const int32_t hm[5] = {H.dim, H.n_leaves, H.max_depth, m->bin_ppc, m->eval_order};
    const double rf[3] = {m->repair_node_factor, m->repair_leaf_factor, m->local_ratio};
    bool ok = std::fwrite(kModelMagic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(hdr), 1, f) == 1 &&
              std::fwrite(&m->n_primitives, sizeof(m->n_primitives), 1, f) == 1 &&
              std::fwrite(&m->opts, sizeof(gwn_build_opts), 1, f) == 1 && std::fwrite(hm, sizeof(hm), 1, f) == 1 &&
              std::fwrite(rf, sizeof(rf), 1, f) == 1 &&
              std::fwrite(H.lo, sizeof(H.lo), 1, f) == 1 && std::fwrite(H.hi, sizeof(H.hi), 1, f) == 1 &&
              each_array(const_cast<HostModel&>(H), [&](auto& v) { return write_vec(f, v); });
    ok = (std::fclose(f) == 0) && ok;
    return ok ? GWN_OK : fail(GWN_ERR_INTERNAL, std::string("write failed: ") + path);
}

gwn_status gwn_model_load(const char* path, int32_t device, gwn_model* out) {
    if (!path || !out) return fail(GWN_ERR_INVALID_ARG, "path and out are required");
    *out = nullptr;
    FILE* f = std::fopen(path, "rb");
    if (!f) return fail(GWN_ERR_INVALID_ARG, std::string("cannot open for reading: ") + path);
    gwn_model_s* m = new (std::nothrow) gwn_model_s();
    if (!m) {
        std::fclose(f);
        return fail(GWN_ERR_OOM, "host allocation failed");
    }
    char magic[8] = {};
    int32_t hdr[4] = {}, hm[5] = {};
    double rf[3] = {};
    bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, kModelMagic, 8) == 0 &&
              std::fread(hdr, sizeof(hdr), 1, f) == 1 && hdr[0] == (int32_t)kModelVersion &&
              (hdr[1] == 2 || hdr[1] == 3) && hdr[3] == (int32_t)sizeof(gwn_build_opts) &&
              std::fread(&m->n_primitives, sizeof(m->n_primitives), 1, f) == 1 &&
              std::fread(&m->opts, sizeof(gwn_build_opts), 1, f) == 1 && std::fread(hm, sizeof(hm), 1, f) == 1 &&
              std::fread(rf, sizeof(rf), 1, f) == 1 &&
              std::fread(m->host.lo, sizeof(m->host.lo), 1, f) == 1 &&
              std::fread(m->host.hi, sizeof(m->host.hi), 1, f) == 1;
    try {
        // no array may hold more elements than the rest of the file has bytes
        long pos = ok ? std::ftell(f) : -1;
        struct stat sb;
        ok = ok && pos >= 0 && fstat(fileno(f), &sb) == 0 && (uint64_t)sb.st_size >= (uint64_t)pos;
        uint64_t left = ok ? (uint64_t)sb.st_size - (uint64_t)pos : 0;
        ok = ok && each_array(m->host, [&](auto& v) { return read_vec(f, &v, &left); });
        ok = ok && left == 0;  // nothing may follow the last array
    } catch (const std::bad_alloc&) {
        ok = false;
    }
    std::fclose(f);
    HostModel& H = m->host;
    if (ok) {
        m->dim = hdr[1];
        m->leaf_far = hdr[2] ? 1 : 0;
        H.dim = hm[0];
        H.n_leaves = hm[1];
        H.max_depth = hm[2];
        m->bin_ppc = hm[3];
        m->eval_order = hm[4];
        m->repair_node_factor = rf[0];
        m->repair_leaf_factor = rf[1];
        m->local_ratio = rf[2];
        ok = hm[3] >= 1 && hm[3] <= 4096 && rf[0] >= 1.0 && rf[0] <= 16.0 && rf[1] >= 1.0 && rf[1] <= 16.0 &&
             hm[4] >= 0 && hm[4] <= m->opts.order && (rf[2] == 0.0 || (rf[2] >= 4.0 && rf[2] < 1e6));
        // consistency of the arrays the kernels index
        ok = ok && host_model_consistent(H, m->dim);
    }
    if (!ok || check_opts(m->opts, m->dim) != GWN_OK) {
        delete m;
        return fail(GWN_ERR_INVALID_ARG, std::string("not a model file of this library version: ") + path);
    }
    m->opts.device = device;
    if (device == GWN_DEVICE_HOST_ONLY) {
        m->device = GWN_DEVICE_HOST_ONLY;
        *out = m;
        return GWN_OK;
    }
    auto t0 = std::chrono::steady_clock::now();
    DeviceGuard g(device);
    cudaGetDevice(&m->device);
    const bool tune = m->opts.beta == 0.0;  // saved from a host-only build: tune now
    if (tune) m->opts.beta = 2.0;
    gwn_status s = finish_build(m, out);
    if (s != GWN_OK) return s;
    if (tune) {
        s = autotune(m);
        if (s != GWN_OK) {
            gwn_release(m);
            *out = nullptr;
            return s;
        }
    }
    m->build_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return GWN_OK;
}

gwn_status gwn_release(gwn_model m) {
    if (!m) return GWN_OK;
    if (m->device != GWN_DEVICE_HOST_ONLY) {
        DeviceGuard g(m->device);
        std::lock_guard<std::mutex> lk(m->mu);
        free_model_memory(m);
    }
    delete m;
    return GWN_OK;
}

const char* gwn_last_error(void) { return g_err.c_str(); }

const char* gwn_version(void) { return "gwn-gb300 0.1 (sm_103a)"; }

}  // extern "C"

gwn_status gwn_fail(gwn_status s, const std::string& msg) { return fail(s, msg); }

size_t gwn_workspace_bytes(int dim, int n_leaves, char* base, gwn::Workspace* ws) {
    return workspace_layout(dim, n_leaves, kChunk, base, ws);
}

size_t gwn_chunk_points() { return kChunk; }
