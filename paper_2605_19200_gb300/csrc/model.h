// model.h -- the model object behind gwn_model and the host functions the
// serving loop shares with the query entry points.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <string>
#include <vector>

#include "../../include/gwn.h"
#include "build.h"
#include "gwn_internal.h"

struct gwn_model_s {
    int dim = 2;
    int leaf_far = 0;
    int device = 0;
    int64_t n_primitives = 0;
    gwn_build_opts opts{};
    // launch parameters of the 3D query: the spatial binning aims at this many
    // points per Morton cell (a chunk of n points gets 3 log2(n / ppc) / 3 bits,
    // 3..6 per axis; picked by the autotuner from 4, 8, 16, 32, 64 by measured time),
    // and the packet traversal's warp stack (64, 96 or 128 entries, from the
    // tree depth)
    int bin_ppc = 16;
    int stack_depth = 96;
    // Taylor order the queries evaluate: the build's order, except that a 3D
    // model built with order 3 may be evaluated at order 2 when the autotuner
    // finds that faster at the tolerance (the order-2 coefficients are the same)
    int eval_order = 2;
    // packet local expansion of the 3D traversal: nodes beyond this many packet
    // radii (and far for the whole packet box) are taken by a second-order local
    // expansion about the packet's centre; 0: off (the default)
    double local_ratio = 0.0;
    // automatic FP64 repair (beta_repair < 0, more than 512 leaves): its far
    // tests at these multiples of beta (nodes) and beta_leaf (leaves); the
    // autotuner lowers them while the repaired values stay within 1e-7
    double repair_node_factor = 3.0;
    double repair_leaf_factor = 3.0;
    double build_ms = 0;
    gwn::HostModel host;       // host copy (inspection)
    gwn::DevTree tree{};
    std::vector<void*> allocs;
    size_t device_bytes = 0;
    // scratch owned by the model: query workspace and host staging
    std::mutex mu;
    void* ws_mem = nullptr;
    size_t ws_bytes = 0;
    size_t ws_n = 0;
    gwn::Workspace ws{};
    static constexpr int kMaxProfChunks = 32;
    // per chunk: before and after the traversal, before the table kernel,
    // after the full evaluator, between the two (round 0 of each chunk)
    cudaEvent_t ev[kMaxProfChunks][5] = {};
    int prof_chunks = 0;
    bool profiled = false;
    void* stage = nullptr;
    size_t stage_cap = 0;
    // end of the last gwn_query's work: the next call, possibly on another
    // stream, waits for it before it reuses the workspace
    cudaEvent_t last = nullptr;
    bool last_recorded = false;
};

// Record an error message for gwn_last_error() and return the status.
gwn_status gwn_fail(gwn_status s, const std::string& msg);

// Enqueue a query (device-resident points and outputs) on `st` using workspace `ws`,
// in chunks of at most max_chunk points (0: the workspace's full chunk).
gwn_status gwn_enqueue_device(gwn_model_s* m, const void* pts, int dtype, size_t n, double* out_w, int* out_label,
                              uint32_t* out_status, const gwn_query_opts& qo, cudaStream_t st, const gwn::Workspace& ws,
                              size_t max_chunk = 0);

// Bytes of a query workspace for `dim` (0 = either dimension) and `n_leaves`;
// when base != nullptr also lays it out in the allocation at base.
size_t gwn_workspace_bytes(int dim, int n_leaves, char* base, gwn::Workspace* ws);

// Points one workspace (one chunk of a query) holds.
size_t gwn_chunk_points();
