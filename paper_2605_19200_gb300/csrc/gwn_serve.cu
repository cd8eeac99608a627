// gwn_serve.cu -- request loop over device-resident models (gwn_serve_* in gwn.h).
//
// Continuous batching: requests are queued by gwn_serve_submit; a worker thread
// admits them in arrival order whenever a slot (a CUDA stream with its own
// query workspace and pinned staging) is free and the request's device memory
// (points + outputs, allocated stream-ordered) fits the remaining budget.  An
// admitted request is copied to the device, queried and copied back on its
// slot's stream, so requests in different slots overlap on the GPU; the
// worker polls the slots' completion events and frees their memory, which
// admits the next requests.  Every wait is bounded.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <vector>

#include "../../include/gwn.h"
#include "model.h"

namespace {

using clk = std::chrono::steady_clock;

struct Request {
    uint64_t id = 0;
    int model = 0;
    int dtype = GWN_F32;
    size_t n = 0;
    std::vector<char> points;  // host copy taken at submit
    std::vector<double> w;     // results
    std::vector<int32_t> label;
    clk::time_point t_submit, t_done;
    bool done = false;
    gwn_status status = GWN_OK;
    std::string error;
    size_t dev_bytes = 0;
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    cudaEvent_t t0 = nullptr, t1 = nullptr;  // timing: the current request's device work begins / ends
    void* ws_mem = nullptr;
    gwn::Workspace ws{};
    size_t ws_bytes = 0;
    void* pin_in = nullptr;  // pinned staging of points
    void* pin_out = nullptr; // pinned staging of outputs (w then label)
    size_t pin_cap = 0;      // bytes of each staging buffer
    char* dev = nullptr;     // device buffer of the current request
    std::shared_ptr<Request> cur;
};

}  // namespace

struct gwn_server_s {
    gwn_serve_opts opts{};
    int device = 0;
    std::vector<gwn_model_s*> models;
    int max_leaves = 1;
    std::vector<Slot> slots;
    std::mutex mu;
    std::condition_variable cv;
    std::deque<std::shared_ptr<Request>> queue;
    std::map<uint64_t, std::shared_ptr<Request>> reqs;
    std::vector<double> latencies_ms;
    // device windows of completed requests (ms since `ref`): evidence that the
    // work of requests in different slots overlaps on the GPU
    cudaEvent_t ref = nullptr;
    std::vector<std::pair<double, double>> windows;
    int64_t max_in_flight = 0;
    uint64_t next_id = 1;
    int64_t submitted = 0, completed = 0, points_done = 0;
    clk::time_point t_first{}, t_last{};
    bool have_first = false;
    size_t budget_used = 0;
    std::atomic<bool> stop{false};
    std::thread worker;
    std::string fatal;
};

namespace {

size_t point_bytes(const gwn_server_s* s, const Request& r) {
    const int dim = s->models[r.model]->dim;
    return r.n * dim * (r.dtype == GWN_F32 ? sizeof(float) : sizeof(double));
}

size_t request_dev_bytes(const gwn_server_s* s, const Request& r) {
    size_t pb = (point_bytes(s, r) + 255) & ~size_t(255);
    return pb + r.n * (sizeof(double) + sizeof(int32_t)) + 512;
}

gwn_status ensure_slot(gwn_server_s* S, Slot& sl, size_t pin_bytes) {
    if (!sl.stream) {
        if (cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreate(&sl.t0) != cudaSuccess || cudaEventCreate(&sl.t1) != cudaSuccess)
            return gwn_fail(GWN_ERR_CUDA, "serve: stream/event creation failed");
    }
    if (!sl.ws_mem) {
        size_t bytes = gwn_workspace_bytes(0, S->max_leaves, nullptr, nullptr);
        if (cudaMalloc(&sl.ws_mem, bytes) != cudaSuccess) return gwn_fail(GWN_ERR_OOM, "serve: slot workspace");
        sl.ws_bytes = bytes;
        gwn_workspace_bytes(0, S->max_leaves, reinterpret_cast<char*>(sl.ws_mem), &sl.ws);
    }
    if (pin_bytes > sl.pin_cap) {
        if (sl.pin_in) cudaFreeHost(sl.pin_in);
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
        sl.pin_in = sl.pin_out = nullptr;
        sl.pin_cap = 0;
        if (cudaHostAlloc(&sl.pin_in, pin_bytes, cudaHostAllocDefault) != cudaSuccess ||
            cudaHostAlloc(&sl.pin_out, pin_bytes, cudaHostAllocDefault) != cudaSuccess)
            return gwn_fail(GWN_ERR_OOM, "serve: pinned staging");
        sl.pin_cap = pin_bytes;
    }
    return GWN_OK;
}

// launch request r on slot sl (called by the worker, lock not held)
gwn_status launch(gwn_server_s* S, Slot& sl, Request& r) {
    const size_t pb = point_bytes(S, r);
    const size_t ob = r.n * (sizeof(double) + sizeof(int32_t));
    gwn_status st = ensure_slot(S, sl, std::max(pb, ob));
    if (st != GWN_OK) return st;
    sl.dev = nullptr;
    if (cudaMallocAsync(reinterpret_cast<void**>(&sl.dev), r.dev_bytes, sl.stream) != cudaSuccess) {
        sl.dev = nullptr;
        return gwn_fail(GWN_ERR_OOM, "serve: request buffer");
    }
    char* dpts = sl.dev;
    double* dw = reinterpret_cast<double*>(sl.dev + ((pb + 255) & ~size_t(255)));
    int32_t* dl = reinterpret_cast<int32_t*>(dw + r.n);
    std::memcpy(sl.pin_in, r.points.data(), pb);
    if (cudaEventRecord(sl.t0, sl.stream) != cudaSuccess ||
        cudaMemcpyAsync(dpts, sl.pin_in, pb, cudaMemcpyHostToDevice, sl.stream) != cudaSuccess)
        return gwn_fail(GWN_ERR_CUDA, "serve: copy in");
    gwn_query_opts qo;
    gwn_default_query_opts(&qo);
    // chunks of 2^19 points: shorter kernels let the other slots' requests interleave
    // (with full 2^20-point chunks the p99 at 0.9 of saturation doubled)
    st = gwn_enqueue_device(S->models[r.model], dpts, r.dtype, r.n, dw, dl, nullptr, qo, sl.stream, sl.ws,
                            (size_t)1 << 19);
    if (st != GWN_OK) return st;
    if (cudaMemcpyAsync(sl.pin_out, dw, ob, cudaMemcpyDeviceToHost, sl.stream) != cudaSuccess ||
        cudaFreeAsync(sl.dev, sl.stream) != cudaSuccess)
        return gwn_fail(GWN_ERR_CUDA, "serve: copy out");
    sl.dev = nullptr;
    if (cudaEventRecord(sl.t1, sl.stream) != cudaSuccess || cudaEventRecord(sl.done, sl.stream) != cudaSuccess)
        return gwn_fail(GWN_ERR_CUDA, "serve: event");
    return GWN_OK;
}

void finish(gwn_server_s* S, Slot& sl) {
    Request& r = *sl.cur;
    float a = -1.f, b = -1.f;
    if (r.status == GWN_OK) {
        r.w.resize(r.n);
        r.label.resize(r.n);
        std::memcpy(r.w.data(), sl.pin_out, r.n * sizeof(double));
        std::memcpy(r.label.data(), reinterpret_cast<char*>(sl.pin_out) + r.n * sizeof(double), r.n * sizeof(int32_t));
        if (S->ref && (cudaEventElapsedTime(&a, S->ref, sl.t0) != cudaSuccess ||
                       cudaEventElapsedTime(&b, S->ref, sl.t1) != cudaSuccess))
            a = b = -1.f;
    }
    std::lock_guard<std::mutex> lk(S->mu);
    if (a >= 0.f && b >= a) S->windows.push_back({(double)a, (double)b});
    r.t_done = clk::now();
    r.done = true;
    r.points.clear();
    r.points.shrink_to_fit();
    S->budget_used -= r.dev_bytes;
    S->completed += 1;
    S->points_done += (int64_t)r.n;
    S->latencies_ms.push_back(std::chrono::duration<double, std::milli>(r.t_done - r.t_submit).count());
    S->t_last = r.t_done;
    sl.cur.reset();
    S->cv.notify_all();
}

void worker_loop(gwn_server_s* S) {
    cudaSetDevice(S->device);
    // the time origin of the requests' device windows
    if (cudaEventCreate(&S->ref) != cudaSuccess || cudaEventRecord(S->ref, 0) != cudaSuccess ||
        cudaEventSynchronize(S->ref) != cudaSuccess) {
        if (S->ref) cudaEventDestroy(S->ref);
        S->ref = nullptr;  // windows are then not recorded
    }
    while (true) {
        std::vector<std::pair<Slot*, std::shared_ptr<Request>>> todo;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->stop && S->queue.empty()) {
                bool busy = false;
                for (auto& sl : S->slots) busy = busy || sl.cur != nullptr;
                if (!busy) return;
            }
            // admission: arrival order, while a slot is free and the head fits the budget
            for (auto& sl : S->slots) {
                if (sl.cur || S->queue.empty()) continue;
                auto& head = S->queue.front();
                // when nothing is in flight budget_used is 0, and every queued request
                // fits on its own (checked at submit), so the head always starts
                if (S->budget_used + head->dev_bytes > (size_t)S->opts.mem_budget_bytes) break;
                S->budget_used += head->dev_bytes;
                sl.cur = head;
                todo.push_back({&sl, head});
                S->queue.pop_front();
            }
            int64_t busy = 0;
            for (auto& sl : S->slots) busy += sl.cur ? 1 : 0;
            S->max_in_flight = std::max(S->max_in_flight, busy);
        }
        for (auto& [sl, r] : todo) {
            gwn_status st = launch(S, *sl, *r);
            if (st != GWN_OK) {
                r->status = st;
                r->error = gwn_last_error();
                if (sl->dev) cudaFreeAsync(sl->dev, sl->stream);
                cudaStreamSynchronize(sl->stream);
                finish(S, *sl);
            }
        }
        bool any = false;
        for (auto& sl : S->slots) {
            if (!sl.cur) continue;
            any = true;
            cudaError_t e = cudaEventQuery(sl.done);
            if (e == cudaSuccess) {
                finish(S, sl);
            } else if (e != cudaErrorNotReady) {
                sl.cur->status = GWN_ERR_CUDA;
                sl.cur->error = cudaGetErrorString(e);
                finish(S, sl);
            }
        }
        std::unique_lock<std::mutex> lk(S->mu);
        if (!any && S->queue.empty() && !S->stop)
            S->cv.wait_for(lk, std::chrono::milliseconds(5));
        else if (any)
            S->cv.wait_for(lk, std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

void gwn_default_serve_opts(gwn_serve_opts* o) {
    if (!o) return;
    o->mem_budget_bytes = (int64_t)40 << 30;
    o->n_slots = 4;
    o->device = -1;
}

gwn_status gwn_serve_create(const gwn_serve_opts* opts, gwn_server* out) {
    if (!out) return gwn_fail(GWN_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    gwn_serve_opts o;
    gwn_default_serve_opts(&o);
    if (opts) o = *opts;
    if (o.n_slots < 1 || o.n_slots > 64) return gwn_fail(GWN_ERR_INVALID_ARG, "n_slots must be 1..64");
    if (o.mem_budget_bytes <= 0) return gwn_fail(GWN_ERR_INVALID_ARG, "mem_budget_bytes must be > 0");
    auto* S = new (std::nothrow) gwn_server_s();
    if (!S) return gwn_fail(GWN_ERR_OOM, "host allocation failed");
    S->opts = o;
    if (o.device >= 0) cudaSetDevice(o.device);
    cudaGetDevice(&S->device);
    S->slots.resize(o.n_slots);
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return GWN_OK;
}

gwn_status gwn_serve_add_model(gwn_server S, gwn_model m, int32_t* model_id) {
    if (!S || !m || !model_id) return gwn_fail(GWN_ERR_INVALID_ARG, "NULL argument");
    if (m->device == GWN_DEVICE_HOST_ONLY) return gwn_fail(GWN_ERR_INVALID_ARG, "model was built host-only");
    std::lock_guard<std::mutex> lk(S->mu);
    for (auto& sl : S->slots)
        if (sl.cur) return gwn_fail(GWN_ERR_BUSY, "add models before submitting requests");
    // slot workspaces are sized for the largest model: drop existing ones (idle)
    if (m->host.n_leaves > S->max_leaves) {
        S->max_leaves = m->host.n_leaves;
        for (auto& sl : S->slots)
            if (sl.ws_mem) {
                cudaFree(sl.ws_mem);
                sl.ws_mem = nullptr;
            }
    }
    S->models.push_back(m);
    *model_id = (int32_t)S->models.size() - 1;
    return GWN_OK;
}

gwn_status gwn_serve_submit(gwn_server S, int32_t model_id, const void* points, int32_t dtype, size_t n,
                            uint64_t* request_id) {
    if (!S || !request_id) return gwn_fail(GWN_ERR_INVALID_ARG, "NULL argument");
    if (dtype != GWN_F32 && dtype != GWN_F64) return gwn_fail(GWN_ERR_INVALID_ARG, "unknown points dtype");
    if (n == 0 || !points) return gwn_fail(GWN_ERR_INVALID_ARG, "empty request");
    auto r = std::make_shared<Request>();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (model_id < 0 || model_id >= (int)S->models.size()) return gwn_fail(GWN_ERR_NOT_FOUND, "unknown model id");
        r->model = model_id;
    }
    r->dtype = dtype;
    r->n = n;
    r->dev_bytes = request_dev_bytes(S, *r);
    if (r->dev_bytes > (size_t)S->opts.mem_budget_bytes)
        return gwn_fail(GWN_ERR_INVALID_ARG, "request larger than the memory budget");
    const size_t pb = point_bytes(S, *r);
    r->points.resize(pb);
    std::memcpy(r->points.data(), points, pb);
    r->t_submit = clk::now();
    std::lock_guard<std::mutex> lk(S->mu);
    r->id = S->next_id++;
    if (!S->have_first) {
        S->t_first = r->t_submit;
        S->have_first = true;
    }
    S->submitted += 1;
    S->reqs[r->id] = r;
    S->queue.push_back(r);
    *request_id = r->id;
    S->cv.notify_all();
    return GWN_OK;
}

gwn_status gwn_serve_poll(gwn_server S, uint64_t request_id, double* out_w, int32_t* out_label, int32_t timeout_ms) {
    if (!S) return gwn_fail(GWN_ERR_INVALID_ARG, "server is NULL");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->reqs.find(request_id);
    if (it == S->reqs.end()) return gwn_fail(GWN_ERR_NOT_FOUND, "unknown request id");
    std::shared_ptr<Request> r = it->second;
    auto deadline = clk::now() + std::chrono::milliseconds(std::max(0, timeout_ms));
    while (!r->done) {
        if (S->cv.wait_until(lk, deadline) == std::cv_status::timeout && !r->done)
            return gwn_fail(GWN_ERR_TIMEOUT, "request not finished within the timeout");
    }
    S->reqs.erase(it);
    lk.unlock();
    if (r->status != GWN_OK) return gwn_fail(r->status, r->error);
    if (out_w) std::memcpy(out_w, r->w.data(), r->n * sizeof(double));
    if (out_label) std::memcpy(out_label, r->label.data(), r->n * sizeof(int32_t));
    return GWN_OK;
}

gwn_status gwn_serve_stats(gwn_server S, gwn_server_stats* st) {
    if (!S || !st) return gwn_fail(GWN_ERR_INVALID_ARG, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    std::memset(st, 0, sizeof(*st));
    st->submitted = S->submitted;
    st->completed = S->completed;
    st->queued = (int64_t)S->queue.size();
    for (auto& sl : S->slots) st->in_flight += sl.cur ? 1 : 0;
    st->points_completed = S->points_done;
    std::vector<double> l = S->latencies_ms;
    if (!l.empty()) {
        std::sort(l.begin(), l.end());
        auto q = [&](double f) { return l[std::min(l.size() - 1, (size_t)(f * (l.size() - 1) + 0.5))]; };
        st->p50_ms = q(0.50);
        st->p99_ms = q(0.99);
        double s = 0;
        for (double x : l) s += x;
        st->mean_ms = s / l.size();
        double span = std::chrono::duration<double>(S->t_last - S->t_first).count();
        st->queries_per_s = span > 0 ? S->points_done / span : 0.0;
    }
    st->budget_used_bytes = (int64_t)S->budget_used;
    st->max_in_flight = S->max_in_flight;
    // largest number of completed requests whose device windows overlapped
    // (sweep over the window endpoints; an end sorts before a start at the same time)
    std::vector<std::pair<double, int>> ev;
    ev.reserve(S->windows.size() * 2);
    for (auto& w : S->windows) {
        ev.push_back({w.first, +1});
        ev.push_back({w.second, -1});
    }
    std::sort(ev.begin(), ev.end());
    int64_t cur = 0;
    for (auto& e : ev) {
        cur += e.second;
        st->max_gpu_overlap = std::max(st->max_gpu_overlap, cur);
    }
    return GWN_OK;
}

gwn_status gwn_serve_destroy(gwn_server S) {
    if (!S) return GWN_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->cv.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (auto& sl : S->slots) {
        if (sl.stream) cudaStreamSynchronize(sl.stream);
        if (sl.ws_mem) cudaFree(sl.ws_mem);
        if (sl.pin_in) cudaFreeHost(sl.pin_in);
        if (sl.pin_out) cudaFreeHost(sl.pin_out);
        if (sl.done) cudaEventDestroy(sl.done);
        if (sl.t0) cudaEventDestroy(sl.t0);
        if (sl.t1) cudaEventDestroy(sl.t1);
        if (sl.stream) cudaStreamDestroy(sl.stream);
    }
    if (S->ref) cudaEventDestroy(S->ref);
    delete S;
    return GWN_OK;
}

}  // extern "C"
