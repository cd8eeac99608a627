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
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/gwn.h"
#include "build.h"
#include "gwn_internal.h"
#include "kernels2d.cuh"
#include "kernels3d.cuh"

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

struct gwn_model_s {
    int dim = 2;
    int leaf_far = 0;
    int device = 0;
    int64_t n_primitives = 0;
    gwn_build_opts opts{};
    double build_ms = 0;
    HostModel host;       // host copy (inspection)
    DevTree tree{};
    std::vector<void*> allocs;
    size_t device_bytes = 0;
    // scratch: repair list + counter, host staging
    std::mutex mu;
    int* rlist = nullptr;
    int* rcount = nullptr;
    size_t rcap = 0;
    void* stage = nullptr;
    size_t stage_cap = 0;
};

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
    if (m->rlist) cudaFree(m->rlist);
    if (m->rcount) cudaFree(m->rcount);
    if (m->stage) cudaFree(m->stage);
    m->rlist = nullptr;
    m->rcount = nullptr;
    m->stage = nullptr;
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
    double x[8], w[8];
    for (int i = 0; i < 8; ++i) {
        double z = std::cos(M_PI * (i + 0.75) / 8.5), pp = 1;
        for (int it = 0; it < 100; ++it) {
            double p1 = 1, p2 = 0;
            for (int j = 1; j <= 8; ++j) {
                double p3 = p2;
                p2 = p1;
                p1 = ((2.0 * j - 1) * z * p2 - (j - 1.0) * p3) / j;
            }
            pp = 8 * (z * p1 - p2) / (z * z - 1);
            double dz = p1 / pp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) break;
        }
        x[i] = 0.5 * (1 - z);
        w[i] = 1.0 / ((1 - z * z) * pp * pp);
    }
    std::memcpy(h_binom, bin, sizeof(bin));
    std::memcpy(h_glx8, x, sizeof(x));
    std::memcpy(h_glw8, w, sizeof(w));
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
    UP(lhdr, lhdr);
    UP(lmom, lmom);
    UP(lhdr64, lhdr64);
    UP(lmom64, lmom64);
    UP(hdr, hdr);
    UP(child, child);
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
    UP(c2, c2);
    UP(c2_64, c2_64);
    UP(c2mult, c2mult);
#undef UP
    return GWN_OK;
}

gwn_status finish_build(gwn_model_s* m, gwn_model* out) {
    gwn_status s = upload_model(m);
    if (s != GWN_OK) {
        free_model_memory(m);
        delete m;
        return s;
    }
    *out = m;
    return GWN_OK;
}

gwn_status check_opts(const gwn_build_opts& o) {
    if (!(o.beta >= 2.0) || !std::isfinite(o.beta)) return fail(GWN_ERR_INVALID_ARG, "beta must be >= 2");
    if (o.order < 0 || o.order > 2) return fail(GWN_ERR_INVALID_ARG, "order must be 0, 1 or 2");
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
    float w = 0.f;
    if (DIM == 2) {
        if (p.mode == GWN_MODE_DIRECT) {
            for (int l = 0; l < t.n_leaves; ++l) w += leaf2_eval32(t, l, (float)qd[0], (float)qd[1], st);
        } else {
            w = query2_32(t, (float)qd[0], (float)qd[1], p.beta2, st);
        }
    } else {
        if (p.mode == GWN_MODE_DIRECT) {
            for (int l = 0; l < t.n_leaves; ++l) w += leaf3_eval32(t, l, (float)qd[0], (float)qd[1], (float)qd[2], st);
        } else {
            w = query3_32(t, (float)qd[0], (float)qd[1], (float)qd[2], p.beta2, st);
        }
    }
    double wd = (double)w;
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
__device__ double query64(const DevTree& t, const double* q, double beta2, int mode, uint32_t& st) {
    double b2 = (mode == GWN_MODE_DIRECT) ? 0.0 : beta2;
    if (DIM == 2) return query2_64(t, q[0], q[1], b2, st);
    return query3_64(t, q[0], q[1], q[2], b2, st);
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

// FP64 repair of the listed queries (persistent grid over the device-side
// count).  With beta_repair > 0 each thread re-runs the traversal in FP64;
// with beta_repair == 0 (exact direct sum) a whole warp shares one query, its
// lanes striding over the leaves, so that few repaired queries still fill the
// FP64 pipes.
template <int DIM>
__device__ __forceinline__ double leaf64(const DevTree& t, int l, const double* q, uint32_t& st) {
    if (DIM == 2) return leaf2_eval64(t, l, q[0], q[1], st);
    return leaf3_eval64(t, l, q[0], q[1], q[2], st);
}

template <int DIM>
__global__ void __launch_bounds__(128) k_repair(DevTree t, const void* pts, int dtype, QueryParams p, double* out_w,
                                                int* out_label, uint32_t* out_status, const int* rlist,
                                                const int* rcount) {
    int cnt = *rcount;
    bool direct = p.mode == GWN_MODE_DIRECT || !(p.beta2_repair > 0);
    if (!direct) {
        for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
            int i = rlist[k];
            double q[3];
            load_point(pts, dtype, DIM, i, q);
            uint32_t st = 0;
            double w = query64<DIM>(t, q, p.beta2_repair, GWN_MODE_BVH, st);
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
        for (int l = lane; l < t.n_leaves; l += 32) w += leaf64<DIM>(t, l, q, st);
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            w += __shfl_xor_sync(0xffffffffu, w, off);
            st |= __shfl_xor_sync(0xffffffffu, st, off);
        }
        if (lane == 0) {
            out_w[i] = w;
            if (out_label) out_label[i] = (int)round(w);
            if (out_status) out_status[i] = (out_status[i] | st | GWN_QS_REPAIRED);
        }
    }
}

gwn_status ensure_scratch(gwn_model_s* m, size_t n, size_t stage_bytes) {
    if (n > m->rcap) {
        if (m->rlist) cudaFree(m->rlist);
        m->rlist = nullptr;
        size_t cap = std::max<size_t>(n, 1024);
        cudaError_t e = cudaMalloc(&m->rlist, cap * sizeof(int));
        if (e != cudaSuccess) { m->rcap = 0; return fail(GWN_ERR_OOM, "repair list allocation failed"); }
        m->rcap = cap;
    }
    if (!m->rcount) {
        cudaError_t e = cudaMalloc(&m->rcount, sizeof(int) * 4);
        if (e != cudaSuccess) return fail(GWN_ERR_OOM, "repair counter allocation failed");
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

// Enqueue the query kernels on `st` for device-resident points/outputs.
// Shared with the batched and serving entry points.
gwn_status gwn_enqueue_device(gwn_model_s* m, const void* pts, int dtype, size_t n, double* out_w, int* out_label,
                              uint32_t* out_status, const gwn_query_opts& qo, cudaStream_t st, int* rlist,
                              int* rcount) {
    QueryParams p;
    double beta = qo.beta > 0 ? qo.beta : m->opts.beta;
    p.beta2 = (float)(beta * beta);
    double br = m->opts.beta_repair;
    if (br < 0) br = m->host.n_leaves <= 4096 ? 0.0 : 4.0 * beta;  // automatic choice
    p.beta2_repair = br > 0 ? br * br : 0.0;
    p.band = (float)m->opts.repair_band;
    p.mode = qo.mode;
    p.precision = qo.precision >= 0 ? qo.precision : m->opts.precision;
    const int B = 128;
    long long nb = ((long long)n + B - 1) / B;
    if (p.precision == GWN_PREC_FP64) {
        if (m->dim == 2) k_query64<2><<<(unsigned)nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status);
        else k_query64<3><<<(unsigned)nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status);
        GWN_CUDA_TRY(cudaGetLastError());
        return GWN_OK;
    }
    GWN_CUDA_TRY(cudaMemsetAsync(rcount, 0, sizeof(int), st));
    if (m->dim == 2)
        k_query32<2><<<(unsigned)nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status, rlist, rcount);
    else
        k_query32<3><<<(unsigned)nb, B, 0, st>>>(m->tree, pts, dtype, (long long)n, p, out_w, out_label, out_status, rlist, rcount);
    GWN_CUDA_TRY(cudaGetLastError());
    if (p.precision == GWN_PREC_FP32_REPAIR) {
        int dev = 0, sms = 152;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        unsigned rb = (unsigned)std::min<long long>(std::max<long long>(nb, sms * 4), (long long)sms * 8);
        if (rb == 0) rb = 1;
        if (m->dim == 2) k_repair<2><<<rb, B, 0, st>>>(m->tree, pts, dtype, p, out_w, out_label, out_status, rlist, rcount);
        else k_repair<3><<<rb, B, 0, st>>>(m->tree, pts, dtype, p, out_w, out_label, out_status, rlist, rcount);
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
}

void gwn_default_query_opts(gwn_query_opts* q) {
    if (!q) return;
    q->mode = GWN_MODE_BVH;
    q->precision = -1;
    q->beta = 0.0;
}

static gwn_status build_common(int dim, const void* prims, size_t n, const gwn_build_opts* opts, gwn_model* out) {
    if (!out) return fail(GWN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    gwn_build_opts o;
    gwn_default_build_opts(&o);
    if (opts) o = *opts;
    gwn_status s = check_opts(o);
    if (s != GWN_OK) return s;
    auto t0 = std::chrono::steady_clock::now();
    gwn_model_s* m = new (std::nothrow) gwn_model_s();
    if (!m) return fail(GWN_ERR_OOM, "host allocation failed");
    m->dim = dim;
    m->opts = o;
    m->leaf_far = o.leaf_far < 0 ? (dim == 3 ? 1 : 0) : (o.leaf_far ? 1 : 0);
    m->n_primitives = (int64_t)n;
    gwn_status code = GWN_OK;
    std::string err;
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
    s = finish_build(m, out);
    if (s != GWN_OK) return s;
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
    DeviceGuard g(m->device);
    std::lock_guard<std::mutex> lk(m->mu);
    cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
    size_t esz = dtype == GWN_F32 ? sizeof(float) : sizeof(double);
    size_t pbytes = n * m->dim * esz;
    size_t obytes = n * (sizeof(double) + sizeof(int32_t) + sizeof(uint32_t));
    gwn_status s = ensure_scratch(m, n, mem == GWN_MEM_HOST ? pbytes + obytes + 64 : 0);
    if (s != GWN_OK) return s;
    if (mem == GWN_MEM_DEVICE)
        return gwn_enqueue_device(m, points, dtype, n, out_w, out_label, (uint32_t*)out_status, qo, st, m->rlist, m->rcount);
    // host buffers: stage through model-owned device memory
    char* base = reinterpret_cast<char*>(m->stage);
    void* dp = base;
    double* dw = reinterpret_cast<double*>(base + ((pbytes + 15) & ~size_t(15)));
    int32_t* dl = reinterpret_cast<int32_t*>(dw + n);
    uint32_t* ds = reinterpret_cast<uint32_t*>(dl + n);
    GWN_CUDA_TRY(cudaMemcpyAsync(dp, points, pbytes, cudaMemcpyHostToDevice, st));
    s = gwn_enqueue_device(m, dp, dtype, n, dw, out_label ? dl : nullptr, out_status ? ds : nullptr, qo, st, m->rlist,
                           m->rcount);
    if (s != GWN_OK) return s;
    GWN_CUDA_TRY(cudaMemcpyAsync(out_w, dw, n * sizeof(double), cudaMemcpyDeviceToHost, st));
    if (out_label) GWN_CUDA_TRY(cudaMemcpyAsync(out_label, dl, n * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    if (out_status) GWN_CUDA_TRY(cudaMemcpyAsync(out_status, ds, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, st));
    GWN_CUDA_TRY(cudaStreamSynchronize(st));
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
    s->beta_repair = m->opts.beta_repair;
    s->repair_band = m->opts.repair_band;
    s->order = m->opts.order;
    for (int k = 0; k < 3; ++k) {
        s->lo[k] = m->host.lo[k];
        s->hi[k] = m->host.hi[k];
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
