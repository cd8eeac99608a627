// gwn_batch.cu -- many models and point sets in one launch (gwn_query_batch in gwn.h).
//
// A batch plan owns a pool of CUDA streams, each with its own query workspace.
// gwn_query_batch spreads the items over the streams (largest first, each to
// the stream with the least work so far), so the pipelines of different
// models run concurrently on the GPU: small models fill the SMs that a large
// one leaves idle, and the latency-bound FP64 tails of one item overlap the
// bulk of another.  An item longer than one chunk of the query pipeline is
// planned as chunk-aligned pieces, so that a large model's chunks also run on
// several streams instead of one after the other at the end of the batch;
// the pieces bin and evaluate their points exactly as the whole item would.  The whole fork/join is captured once into a CUDA graph
// (every stage of the query pipeline is driven by device-side counters, with
// no host synchronisation, so it can be captured) and later calls with the
// same items replay that graph with one cudaGraphLaunch on the caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "../../include/gwn.h"
#include "model.h"

#define BATCH_CUDA_TRY(call)                                                                        \
    do {                                                                                            \
        cudaError_t e_ = (call);                                                                    \
        if (e_ != cudaSuccess) return gwn_fail(GWN_ERR_CUDA, std::string(#call ": ") + cudaGetErrorString(e_)); \
    } while (0)

struct gwn_batch_s {
    int device = 0;
    std::mutex mu;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> done;   // one per stream (join)
    cudaEvent_t fork = nullptr;
    cudaEvent_t last = nullptr;      // end of the previous launch (launches share the workspaces)
    bool last_recorded = false;
    std::vector<void*> ws_mem;
    std::vector<gwn::Workspace> ws;
    int ws_leaves = 0;               // workspaces are laid out for this many leaves
    size_t ws_bytes = 0;
    // device copies of host items' points and outputs (gwn_query_batch_host)
    void* stage = nullptr;
    size_t stage_bytes = 0;
    // captured graph and the items it was captured for
    std::vector<gwn_query_item> key;
    bool key_host = false;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t launches = 0, captures = 0;
};

namespace {

// field by field: the struct has padding, which callers need not initialise
bool same_items(const std::vector<gwn_query_item>& a, const gwn_query_item* b, size_t n) {
    if (a.size() != n) return false;
    for (size_t i = 0; i < n; ++i) {
        const gwn_query_item &x = a[i], &y = b[i];
        if (x.model != y.model || x.points != y.points || x.points_dtype != y.points_dtype || x.n != y.n ||
            x.out_w != y.out_w || x.out_label != y.out_label || x.out_status != y.out_status)
            return false;
    }
    return true;
}

void drop_graph(gwn_batch_s* B) {
    if (B->exec) cudaGraphExecDestroy(B->exec);
    if (B->graph) cudaGraphDestroy(B->graph);
    B->exec = nullptr;
    B->graph = nullptr;
    B->key.clear();
}

gwn_status ensure_workspaces(gwn_batch_s* B, int leaves) {
    if (leaves <= B->ws_leaves && !B->ws_mem.empty() && B->ws_mem[0]) return GWN_OK;
    for (void* p : B->ws_mem)
        if (p) cudaFree(p);
    const size_t bytes = gwn_workspace_bytes(0, leaves, nullptr, nullptr);
    for (size_t k = 0; k < B->streams.size(); ++k) {
        B->ws_mem[k] = nullptr;
        if (cudaMalloc(&B->ws_mem[k], bytes) != cudaSuccess) {
            for (size_t j = 0; j < k; ++j) cudaFree(B->ws_mem[j]), B->ws_mem[j] = nullptr;
            B->ws_leaves = 0;
            return gwn_fail(GWN_ERR_OOM, "batch: stream workspaces");
        }
        gwn_workspace_bytes(0, leaves, reinterpret_cast<char*>(B->ws_mem[k]), &B->ws[k]);
    }
    B->ws_leaves = leaves;
    B->ws_bytes = bytes;
    drop_graph(B);  // the captured graph points at the old workspaces
    return GWN_OK;
}

}  // namespace

extern "C" {

gwn_status gwn_batch_create(int32_t n_streams, int32_t device, gwn_batch* out) {
    if (!out) return gwn_fail(GWN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (n_streams < 1 || n_streams > 32) return gwn_fail(GWN_ERR_INVALID_ARG, "n_streams must be 1..32");
    if (device >= 0 && cudaSetDevice(device) != cudaSuccess) return gwn_fail(GWN_ERR_CUDA, "cudaSetDevice failed");
    auto* B = new (std::nothrow) gwn_batch_s();
    if (!B) return gwn_fail(GWN_ERR_OOM, "host allocation failed");
    cudaGetDevice(&B->device);
    B->streams.assign(n_streams, nullptr);
    B->done.assign(n_streams, nullptr);
    B->ws_mem.assign(n_streams, nullptr);
    B->ws.assign(n_streams, gwn::Workspace{});
    bool ok = cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) == cudaSuccess &&
              cudaEventCreateWithFlags(&B->last, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < n_streams; ++k)
        ok = cudaStreamCreateWithFlags(&B->streams[k], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&B->done[k], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) {
        gwn_batch_release(B);
        return gwn_fail(GWN_ERR_CUDA, "batch: stream/event creation failed");
    }
    *out = B;
    return GWN_OK;
}

}  // extern "C"

namespace {

// checks every item against the plan; *leaves receives the largest model's leaf count
gwn_status check_items(const gwn_batch_s* B, const gwn_query_item* items, size_t n_items, int* leaves) {
    *leaves = 1;
    for (size_t i = 0; i < n_items; ++i) {
        const gwn_query_item& it = items[i];
        if (!it.model) return gwn_fail(GWN_ERR_INVALID_ARG, "item without a model");
        if (it.model->device == GWN_DEVICE_HOST_ONLY) return gwn_fail(GWN_ERR_INVALID_ARG, "model was built host-only");
        if (it.model->device != B->device) return gwn_fail(GWN_ERR_INVALID_ARG, "model lives on another device");
        if (it.n > 0 && (!it.points || !it.out_w)) return gwn_fail(GWN_ERR_INVALID_ARG, "points and out_w are required");
        if (it.points_dtype != GWN_F32 && it.points_dtype != GWN_F64)
            return gwn_fail(GWN_ERR_INVALID_ARG, "unknown points dtype");
        if (it.n > (size_t)0x7fffffff) return gwn_fail(GWN_ERR_INVALID_ARG, "at most 2^31 - 1 points per item");
        *leaves = std::max(*leaves, it.model->host.n_leaves);
    }
    return GWN_OK;
}

size_t point_bytes(const gwn_query_item& it) {
    return it.n * (size_t)it.model->dim * (it.points_dtype == GWN_F32 ? sizeof(float) : sizeof(double));
}

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// device buffers for the points and outputs of host items: `dev` receives the
// items with their pointers moved into the plan's staging memory
gwn_status stage_items(gwn_batch_s* B, const gwn_query_item* items, size_t n_items, std::vector<gwn_query_item>* dev) {
    size_t need = 0;
    for (size_t i = 0; i < n_items; ++i) {
        const gwn_query_item& it = items[i];
        need += align256(point_bytes(it)) + align256(it.n * sizeof(double));
        if (it.out_label) need += align256(it.n * sizeof(int32_t));
        if (it.out_status) need += align256(it.n * sizeof(uint32_t));
    }
    if (need > B->stage_bytes) {
        if (B->stage) cudaFree(B->stage);
        B->stage = nullptr;
        B->stage_bytes = 0;
        drop_graph(B);  // a captured graph may point at the old staging memory
        if (cudaMalloc(&B->stage, std::max<size_t>(need, 256)) != cudaSuccess) {
            B->stage = nullptr;
            return gwn_fail(GWN_ERR_OOM, "batch: staging memory for host items");
        }
        B->stage_bytes = std::max<size_t>(need, 256);
    }
    char* p = reinterpret_cast<char*>(B->stage);
    dev->assign(items, items + n_items);
    for (size_t i = 0; i < n_items; ++i) {
        gwn_query_item& d = (*dev)[i];
        const gwn_query_item& it = items[i];
        d.points = p;
        p += align256(point_bytes(it));
        d.out_w = reinterpret_cast<double*>(p);
        p += align256(it.n * sizeof(double));
        if (it.out_label) {
            d.out_label = reinterpret_cast<int32_t*>(p);
            p += align256(it.n * sizeof(int32_t));
        }
        if (it.out_status) {
            d.out_status = reinterpret_cast<uint32_t*>(p);
            p += align256(it.n * sizeof(uint32_t));
        }
    }
    return GWN_OK;
}

// Issue the items on the plan's streams: largest item first, each to the least
// loaded stream; the streams fork from and join into streams[0].  With `host`
// the items' host buffers are copied in before and out after each query (one
// cudaMemcpyAsync per buffer on the item's stream); `dev` holds the items as
// the kernels see them.
// points per piece of a long item: the query pipeline's chunk (gwn_api.cu)
constexpr size_t kPiece = (size_t)1 << 20;

// item i restricted to its points [off, off + n): the same arrays, offset
gwn_query_item piece_of(const gwn_query_item& it, size_t off, size_t n) {
    gwn_query_item p = it;
    const size_t pb = n ? point_bytes(it) / it.n : 0;  // bytes per point
    p.points = static_cast<const char*>(it.points) + off * pb;
    p.n = n;
    p.out_w = it.out_w + off;
    if (it.out_label) p.out_label = it.out_label + off;
    if (it.out_status) p.out_status = it.out_status + off;
    return p;
}

gwn_status issue_plan(gwn_batch_s* B, const gwn_query_item* items_dev, const gwn_query_item* items_host,
                      size_t n_items) {
    // chunk-aligned pieces of the items (device and, for host buffers, host views)
    std::vector<gwn_query_item> pd, ph;
    for (size_t i = 0; i < n_items; ++i)
        for (size_t off = 0; off < items_dev[i].n || (off == 0 && items_dev[i].n == 0); off += kPiece) {
            const size_t n = std::min(kPiece, items_dev[i].n - off);
            pd.push_back(piece_of(items_dev[i], off, n));
            if (items_host) ph.push_back(piece_of(items_host[i], off, n));
            if (items_dev[i].n == 0) break;
        }
    const gwn_query_item* dev = pd.data();
    const gwn_query_item* host = items_host ? ph.data() : nullptr;
    const size_t n_pieces = pd.size();
    std::vector<size_t> order(n_pieces);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return dev[a].n > dev[b].n; });
    const size_t ns = B->streams.size();
    std::vector<double> load(ns, 0.0);
    std::vector<std::vector<size_t>> plan(ns);
    for (size_t i : order) {
        size_t k = std::min_element(load.begin(), load.end()) - load.begin();
        plan[k].push_back(i);
        load[k] += (double)dev[i].n + 65536.0;  // fixed cost per piece
    }
    cudaStream_t origin = B->streams[0];
    BATCH_CUDA_TRY(cudaEventRecord(B->fork, origin));
    for (size_t k = 1; k < ns; ++k) BATCH_CUDA_TRY(cudaStreamWaitEvent(B->streams[k], B->fork, 0));
    gwn_query_opts qo;
    gwn_default_query_opts(&qo);
    for (size_t k = 0; k < ns; ++k) {
        cudaStream_t s = B->streams[k];
        for (size_t i : plan[k]) {
            const gwn_query_item& it = dev[i];
            if (it.n == 0) continue;
            if (host)
                BATCH_CUDA_TRY(cudaMemcpyAsync(const_cast<void*>(it.points), host[i].points, point_bytes(it),
                                               cudaMemcpyHostToDevice, s));
            gwn_status es = gwn_enqueue_device(it.model, it.points, it.points_dtype, it.n, it.out_w, it.out_label,
                                               it.out_status, qo, s, B->ws[k]);
            if (es != GWN_OK) return es;
            if (host) {
                BATCH_CUDA_TRY(cudaMemcpyAsync(host[i].out_w, it.out_w, it.n * sizeof(double),
                                               cudaMemcpyDeviceToHost, s));
                if (it.out_label)
                    BATCH_CUDA_TRY(cudaMemcpyAsync(host[i].out_label, it.out_label, it.n * sizeof(int32_t),
                                                   cudaMemcpyDeviceToHost, s));
                if (it.out_status)
                    BATCH_CUDA_TRY(cudaMemcpyAsync(host[i].out_status, it.out_status, it.n * sizeof(uint32_t),
                                                   cudaMemcpyDeviceToHost, s));
            }
        }
        if (k > 0) {
            BATCH_CUDA_TRY(cudaEventRecord(B->done[k], s));
            BATCH_CUDA_TRY(cudaStreamWaitEvent(origin, B->done[k], 0));
        }
    }
    return GWN_OK;
}

// capture issue_plan into the plan's graph (B->exec) for `key`
gwn_status capture_plan(gwn_batch_s* B, const gwn_query_item* key, const gwn_query_item* dev,
                        const gwn_query_item* host, size_t n_items) {
    drop_graph(B);
    cudaStream_t cap = B->streams[0];
    BATCH_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    gwn_status es = issue_plan(B, dev, host, n_items);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cap, &g);
    if (es != GWN_OK) {
        if (g) cudaGraphDestroy(g);
        return es;
    }
    if (ee != cudaSuccess || !g) {
        if (g) cudaGraphDestroy(g);
        return gwn_fail(GWN_ERR_CUDA, std::string("batch capture failed: ") + cudaGetErrorString(ee));
    }
    cudaGraphExec_t ex = nullptr;
    cudaError_t ce = cudaGraphInstantiate(&ex, g, 0);
    if (ce != cudaSuccess) {
        cudaGraphDestroy(g);
        return gwn_fail(GWN_ERR_CUDA, std::string("batch graph instantiation failed: ") + cudaGetErrorString(ce));
    }
    B->graph = g;
    B->exec = ex;
    B->key.assign(key, key + n_items);
    B->key_host = host != nullptr;
    B->captures += 1;
    return GWN_OK;
}

struct DeviceSwitch {
    int prev = -1;
    explicit DeviceSwitch(int dev) {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != dev) {
            prev = cur;
            cudaSetDevice(dev);
        }
    }
    ~DeviceSwitch() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

// page-locked host memory (cudaHostAlloc or cudaHostRegister) can be captured
// in a graph's copies; pageable memory cannot
bool page_locked(const void* p) {
    if (!p) return true;
    cudaPointerAttributes a{};
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();  // clear the sticky-free error of an unknown pointer
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace

extern "C" {

gwn_status gwn_query_batch(gwn_batch B, const gwn_query_item* items, size_t n_items, void* stream) {
    if (!B) return gwn_fail(GWN_ERR_INVALID_ARG, "batch is NULL");
    if (n_items == 0) return GWN_OK;
    if (!items) return gwn_fail(GWN_ERR_INVALID_ARG, "items is NULL");
    int leaves = 1;
    gwn_status s = check_items(B, items, n_items, &leaves);
    if (s != GWN_OK) return s;
    std::lock_guard<std::mutex> lk(B->mu);
    DeviceSwitch dsw(B->device);
    s = ensure_workspaces(B, leaves);
    if (s != GWN_OK) return s;
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    if (!B->exec || B->key_host || !same_items(B->key, items, n_items)) {
        s = capture_plan(B, items, items, nullptr, n_items);
        if (s != GWN_OK) return s;
    }
    // launches on different caller streams would share the workspaces: order
    // each after the previous one
    if (B->last_recorded) BATCH_CUDA_TRY(cudaStreamWaitEvent(caller, B->last, 0));
    BATCH_CUDA_TRY(cudaGraphLaunch(B->exec, caller));
    BATCH_CUDA_TRY(cudaEventRecord(B->last, caller));
    B->last_recorded = true;
    B->launches += 1;
    return GWN_OK;
}

gwn_status gwn_query_batch_host(gwn_batch B, const gwn_query_item* items, size_t n_items, void* stream) {
    if (!B) return gwn_fail(GWN_ERR_INVALID_ARG, "batch is NULL");
    if (n_items == 0) return GWN_OK;
    if (!items) return gwn_fail(GWN_ERR_INVALID_ARG, "items is NULL");
    int leaves = 1;
    gwn_status s = check_items(B, items, n_items, &leaves);
    if (s != GWN_OK) return s;
    std::lock_guard<std::mutex> lk(B->mu);
    DeviceSwitch dsw(B->device);
    s = ensure_workspaces(B, leaves);
    if (s != GWN_OK) return s;
    std::vector<gwn_query_item> dev;
    s = stage_items(B, items, n_items, &dev);
    if (s != GWN_OK) return s;
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    bool locked = true;
    for (size_t i = 0; i < n_items && locked; ++i)
        locked = page_locked(items[i].points) && page_locked(items[i].out_w) && page_locked(items[i].out_label) &&
                 page_locked(items[i].out_status);
    if (B->last_recorded) BATCH_CUDA_TRY(cudaStreamWaitEvent(caller, B->last, 0));
    if (locked) {
        if (!B->exec || !B->key_host || !same_items(B->key, items, n_items)) {
            s = capture_plan(B, items, dev.data(), items, n_items);
            if (s != GWN_OK) return s;
        }
        BATCH_CUDA_TRY(cudaGraphLaunch(B->exec, caller));
        B->launches += 1;
    } else {
        // pageable buffers: the same copies and kernels, issued directly
        BATCH_CUDA_TRY(cudaEventRecord(B->fork, caller));
        BATCH_CUDA_TRY(cudaStreamWaitEvent(B->streams[0], B->fork, 0));
        s = issue_plan(B, dev.data(), items, n_items);
        if (s != GWN_OK) return s;
        BATCH_CUDA_TRY(cudaEventRecord(B->done[0], B->streams[0]));
        BATCH_CUDA_TRY(cudaStreamWaitEvent(caller, B->done[0], 0));
    }
    BATCH_CUDA_TRY(cudaEventRecord(B->last, caller));
    B->last_recorded = true;
    BATCH_CUDA_TRY(cudaStreamSynchronize(caller));
    return GWN_OK;
}

gwn_status gwn_batch_info(gwn_batch B, int64_t* graph_launches, int64_t* captures, int64_t* workspace_bytes) {
    if (!B) return gwn_fail(GWN_ERR_INVALID_ARG, "batch is NULL");
    std::lock_guard<std::mutex> lk(B->mu);
    if (graph_launches) *graph_launches = B->launches;
    if (captures) *captures = B->captures;
    if (workspace_bytes) *workspace_bytes = (int64_t)(B->ws_bytes * B->streams.size() + B->stage_bytes);
    return GWN_OK;
}

gwn_status gwn_batch_release(gwn_batch B) {
    if (!B) return GWN_OK;
    {
        std::lock_guard<std::mutex> lk(B->mu);
        for (cudaStream_t s : B->streams)
            if (s) cudaStreamSynchronize(s);
        drop_graph(B);
        for (void* p : B->ws_mem)
            if (p) cudaFree(p);
        if (B->stage) cudaFree(B->stage);
        for (cudaEvent_t e : B->done)
            if (e) cudaEventDestroy(e);
        if (B->fork) cudaEventDestroy(B->fork);
        if (B->last) cudaEventDestroy(B->last);
        for (cudaStream_t s : B->streams)
            if (s) cudaStreamDestroy(s);
    }
    delete B;
    return GWN_OK;
}

}  // extern "C"
