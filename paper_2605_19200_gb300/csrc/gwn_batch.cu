// gwn_batch.cu -- many models and point sets in one launch (gwn_query_batch in gwn.h).
//
// A batch plan owns a pool of CUDA streams, each with its own query workspace.
// gwn_query_batch spreads the items over the streams (largest first, each to
// the stream with the least work so far), so the pipelines of different
// models run concurrently on the GPU: small models fill the SMs that a large
// one leaves idle, and the latency-bound FP64 tails of one item overlap the
// bulk of another.  The whole fork/join is captured once into a CUDA graph
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
    // captured graph and the items it was captured for
    std::vector<gwn_query_item> key;
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

gwn_status gwn_query_batch(gwn_batch B, const gwn_query_item* items, size_t n_items, void* stream) {
    if (!B) return gwn_fail(GWN_ERR_INVALID_ARG, "batch is NULL");
    if (n_items == 0) return GWN_OK;
    if (!items) return gwn_fail(GWN_ERR_INVALID_ARG, "items is NULL");
    int leaves = 1;
    for (size_t i = 0; i < n_items; ++i) {
        const gwn_query_item& it = items[i];
        if (!it.model) return gwn_fail(GWN_ERR_INVALID_ARG, "item without a model");
        if (it.model->device == GWN_DEVICE_HOST_ONLY) return gwn_fail(GWN_ERR_INVALID_ARG, "model was built host-only");
        if (it.model->device != B->device) return gwn_fail(GWN_ERR_INVALID_ARG, "model lives on another device");
        if (it.n > 0 && (!it.points || !it.out_w)) return gwn_fail(GWN_ERR_INVALID_ARG, "points and out_w are required");
        if (it.points_dtype != GWN_F32 && it.points_dtype != GWN_F64)
            return gwn_fail(GWN_ERR_INVALID_ARG, "unknown points dtype");
        if (it.n > (size_t)0x7fffffff) return gwn_fail(GWN_ERR_INVALID_ARG, "at most 2^31 - 1 points per item");
        leaves = std::max(leaves, it.model->host.n_leaves);
    }
    std::lock_guard<std::mutex> lk(B->mu);
    int prev = -1;
    cudaGetDevice(&prev);
    if (prev != B->device) cudaSetDevice(B->device);
    struct Restore {
        int d;
        ~Restore() {
            if (d >= 0) cudaSetDevice(d);
        }
    } restore{prev != B->device ? prev : -1};
    gwn_status s = ensure_workspaces(B, leaves);
    if (s != GWN_OK) return s;
    cudaStream_t caller = reinterpret_cast<cudaStream_t>(stream);
    if (!B->exec || !same_items(B->key, items, n_items)) {
        drop_graph(B);
        // largest item first, each to the least loaded stream
        std::vector<size_t> order(n_items);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(), [&](size_t a, size_t b) { return items[a].n > items[b].n; });
        const size_t ns = B->streams.size();
        std::vector<double> load(ns, 0.0);
        std::vector<std::vector<size_t>> plan(ns);
        for (size_t i : order) {
            size_t k = std::min_element(load.begin(), load.end()) - load.begin();
            plan[k].push_back(i);
            load[k] += (double)items[i].n + 65536.0;  // fixed cost per item
        }
        cudaStream_t cap = B->streams[0];
        BATCH_CUDA_TRY(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
        gwn_status es = GWN_OK;
        cudaError_t ce = cudaEventRecord(B->fork, cap);
        for (size_t k = 1; k < ns && ce == cudaSuccess; ++k) ce = cudaStreamWaitEvent(B->streams[k], B->fork, 0);
        gwn_query_opts qo;
        gwn_default_query_opts(&qo);
        for (size_t k = 0; k < ns && ce == cudaSuccess && es == GWN_OK; ++k) {
            for (size_t i : plan[k]) {
                const gwn_query_item& it = items[i];
                if (it.n == 0) continue;
                es = gwn_enqueue_device(it.model, it.points, it.points_dtype, it.n, it.out_w, it.out_label,
                                        it.out_status, qo, B->streams[k], B->ws[k]);
                if (es != GWN_OK) break;
            }
            if (k > 0 && es == GWN_OK) {
                ce = cudaEventRecord(B->done[k], B->streams[k]);
                if (ce == cudaSuccess) ce = cudaStreamWaitEvent(cap, B->done[k], 0);
            }
        }
        cudaGraph_t g = nullptr;
        cudaError_t ee = cudaStreamEndCapture(cap, &g);
        if (es != GWN_OK) {
            if (g) cudaGraphDestroy(g);
            return es;
        }
        if (ce != cudaSuccess || ee != cudaSuccess || !g) {
            if (g) cudaGraphDestroy(g);
            return gwn_fail(GWN_ERR_CUDA, std::string("batch capture failed: ") +
                                              cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        cudaGraphExec_t ex = nullptr;
        ce = cudaGraphInstantiate(&ex, g, 0);
        if (ce != cudaSuccess) {
            cudaGraphDestroy(g);
            return gwn_fail(GWN_ERR_CUDA, std::string("batch graph instantiation failed: ") + cudaGetErrorString(ce));
        }
        B->graph = g;
        B->exec = ex;
        B->key.assign(items, items + n_items);
        B->captures += 1;
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

gwn_status gwn_batch_info(gwn_batch B, int64_t* graph_launches, int64_t* captures, int64_t* workspace_bytes) {
    if (!B) return gwn_fail(GWN_ERR_INVALID_ARG, "batch is NULL");
    std::lock_guard<std::mutex> lk(B->mu);
    if (graph_launches) *graph_launches = B->launches;
    if (captures) *captures = B->captures;
    if (workspace_bytes) *workspace_bytes = (int64_t)(B->ws_bytes * B->streams.size());
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
