/*
 * gwn.h -- C ABI of the GB300 generalized-winding-number (GWN) library.
 *
 * The library answers batched containment queries against collections of
 * NURBS curves (2D) and trimmed NURBS patches (3D) with the agglomerated
 * evaluation of "Spatially Accelerated Winding Numbers for Curved Geometry"
 * (Algorithm 1): adaptive subdivision (Section 3.2), uncentred moments summed
 * up a BVH (top-down sweep or Karras LBVH) and centred in place (Section 3.1, Eq. 3 and the moment
 * transform), and a per-query traversal that evaluates the order-0/1/2 Taylor
 * expansion of Eq. 3 (order 3 in 3D as an extension) for clusters that pass
 * the far test of Section 3 and the
 * exact GWN (Section 3.3) for the leaves it reaches.
 *
 * Conventions shared by every call
 *   - Every function returns gwn_status; nothing throws across the ABI.
 *     gwn_last_error() returns a thread-local message for the last failure.
 *   - GWN normalisation follows Eq. 2: a counter-clockwise closed curve, or a
 *     closed shell with outward normals S_u x S_v, has winding number 1 inside.
 *   - Curves and patches use clamped knot vectors (first and last knot repeated
 *     degree + 1 times), positive weights, and degree 1..3 in each direction.
 *   - Trimming curves of a patch are closed loops in its (u, v) domain; the
 *     visible region is counted with the loops' winding number (outer loops
 *     counter-clockwise, holes clockwise).  A patch with n_trims == 0 is
 *     untrimmed: its boundary is the parameter rectangle.
 *   - A gwn_model owns all device memory it allocates until gwn_release();
 *     the build functions deep-copy their inputs, so the caller may free them
 *     when the call returns.  Output buffers always belong to the caller.
 */
#ifndef GWN_H
#define GWN_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    GWN_OK = 0,
    GWN_ERR_INVALID_ARG = 1,      /* bad pointer, size, option or unsupported degree */
    GWN_ERR_INVALID_GEOMETRY = 2, /* non-clamped knots, weights <= 0, NaN/Inf, trims outside the domain */
    GWN_ERR_OOM = 3,              /* device or host allocation failed */
    GWN_ERR_CUDA = 4,             /* a CUDA runtime call failed */
    GWN_ERR_TIMEOUT = 5,          /* a bounded device or host wait ran out */
    GWN_ERR_BUSY = 6,             /* not admitted yet (memory budget); retry later */
    GWN_ERR_INTERNAL = 7,
    GWN_ERR_NOT_FOUND = 8         /* unknown request or model id */
} gwn_status;

typedef struct gwn_model_s* gwn_model;

/* A NURBS curve in the plane.  ctrl: n_ctrl x 2 (x, y), weights: n_ctrl or
 * NULL (all ones), knots: n_ctrl + degree + 1, clamped and non-decreasing. */
typedef struct {
    int32_t degree;
    int32_t n_ctrl;
    const double* ctrl;
    const double* weights;
    const double* knots;
} gwn_curve2d;

/* A trimmed tensor-product NURBS patch.  ctrl: n_u x n_v x 3 with the v index
 * fastest ((i_u * n_v + i_v) * 3), weights: n_u x n_v or NULL, knots_u:
 * n_u + deg_u + 1, knots_v: n_v + deg_v + 1.  trims: n_trims curves in (u, v)
 * that must lie inside the parameter rectangle. */
typedef struct {
    int32_t deg_u, deg_v;
    int32_t n_u, n_v;
    const double* ctrl;
    const double* weights;
    const double* knots_u;
    const double* knots_v;
    int32_t n_trims;
    const gwn_curve2d* trims;
} gwn_patch3d;

enum {
    GWN_PREC_FP32_REPAIR = 0, /* FP32 traversal, FP64 re-evaluation near half-integers and for flagged queries */
    GWN_PREC_FP32 = 1,        /* FP32 only (no repair) */
    GWN_PREC_FP64 = 2         /* every query evaluated in FP64 */
};

enum {
    GWN_MODE_BVH = 0,    /* Algorithm 1: BVH traversal with Taylor far field */
    GWN_MODE_DIRECT = 1  /* plain direct sum: every leaf evaluated exactly for every query */
};

enum { GWN_F32 = 0, GWN_F64 = 1 };              /* point dtypes */
enum { GWN_DEVICE_HOST_ONLY = -2 };
enum { GWN_MEM_DEVICE = 0, GWN_MEM_HOST = 1 };  /* where points and outputs live */

/* Per-query status bits written to out_status. */
enum {
    GWN_QS_REPAIRED = 1u,       /* value re-evaluated in FP64 */
    GWN_QS_NEAR = 2u,           /* a leaf of this query went to the FP64 near band (query very near the boundary) */
    GWN_QS_STACK_OVERFLOW = 4u, /* traversal stack overflow in the FP32 pass (value repaired) */
    GWN_QS_UNRESOLVED = 8u      /* FP64 pass also hit a refinement or stack limit: value may be inexact */
};

typedef struct {
    double tolerance;     /* target max |dGWN| for the FP32 path (default 1e-4) */
    double max_aabb_frac; /* subdivide until a leaf's box diagonal < frac * shape diagonal (0.1); <= 0: no subdivision */
    int32_t order;        /* Taylor order 0, 1 or 2 of Eq. 3 (default 2); 3D models also take 3, the next
                             term of the same expansion (third-order moments int y y y n), beyond the
                             paper: its remainder falls one power of r/|x0 - q| faster, so the same
                             tolerance holds at a smaller beta and beta_leaf.  The FP64 evaluations (the
                             repair, GWN_PREC_FP64) then always take the order-3 terms; the FP32 bulk
                             takes them where the autotuner finds that faster (gwn_model_stats.eval_order) */
    double beta;          /* far test ||q - c|| > beta * r, r = half box diagonal; >= 2, or 0 = autotune:
                             among the (beta, beta_leaf) pairs whose FP32 error on validation points
                             (FP64 direct sum on the device) stays below tolerance / 2, the fastest on
                             a timed uniform sample, then the binning's points per cell by measured
                             time (default 2) */
    double beta_repair;   /* beta of the FP64 repair traversal; 0 = exact direct sum over all leaves;
                             < 0 = automatic: direct sum up to 512 leaves, else 3 x beta for nodes and
                             3 x beta_leaf for leaves, factors the autotuner lowers (to 2 and 1.5 at
                             least) while the repaired values of its validation points stay within
                             1e-7 of the FP64 direct sum (default -1) */
    double repair_band;   /* re-evaluate in FP64 when |w - round(w) +- 1/2| < band (default 1e-3) */
    int32_t quad_nodes;   /* Gauss-Legendre nodes per rule for 3D moments (default 10) */
    int32_t precision;    /* GWN_PREC_* (default GWN_PREC_FP32_REPAIR) */
    int32_t device;       /* CUDA device ordinal, -1 = current (default -1); GWN_DEVICE_HOST_ONLY
                             builds the host-side tree only (inspection, no queries) */
    int32_t n_threads;    /* host threads for the build, 0 = all (default 0) */
    int32_t leaf_far;     /* 1: a leaf that passes the far test is approximated by its own moments
                             (only leaves containing the query are evaluated exactly); 0: every
                             leaf reached is evaluated exactly; -1: 1 in 3D, 0 in 2D (default) */
    double beta_leaf;     /* far-test factor of the leaves themselves when leaf_far is on; 0 = beta (default 0) */
    int32_t adaptive_beta; /* 1: geometry-aware far test per cluster (the per-cluster beta Section 5 names):
                              a cluster of fill a = (curve length or area) / r^(d-1) is approximated only
                              beyond beta * s * r with s = clamp((a / median a)^(1 / (order + d)), 1, 4),
                              since its order-p remainder grows like a * beta^-(p + d); dense clusters are
                              opened earlier, the others keep beta.  0 = off (default 0) */
    int32_t device_build;  /* 3D: the per-leaf stage of the build -- leaf moments (Section 3.1) and the
                              packing of the leaves' boundary curves for the near field -- on the model's
                              GPU, one thread per leaf or curve (1), or on the host threads (0); both give
                              the same model bit for bit.  -1 = on the GPU unless the build is host-only
                              (default -1) */
    int32_t tree_builder;  /* the hierarchy over the leaves: 0 = Karras LBVH over the Morton codes of the
                              leaf-box centres (Section 3.1); 1 = top-down sweep that splits each node
                              where (leaves x radius^2) summed over the two children is least, over the
                              three axes, so that far tests accept clusters earlier (fewer node visits
                              per query); -1 = 1 (default -1).  Both give the same node layout */
    double local_ratio;    /* 3D: the model's packet local-expansion ratio (gwn_query_opts.local_ratio),
                              >= 4; <= 0 = off (default 0) */
} gwn_build_opts;

/* Fills *opts with the defaults listed above. */
void gwn_default_build_opts(gwn_build_opts* opts);

typedef struct {
    int32_t mode;       /* GWN_MODE_* (default GWN_MODE_BVH) */
    int32_t precision;  /* GWN_PREC_*, or -1 = the model's (default -1) */
    double beta;        /* 0 = the model's */
    int32_t count_work; /* 1: count algorithmic work units (slower; see gwn_last_query_stats) */
    int32_t profile;    /* 1: time the traversal and exact-leaf kernels with CUDA events on the stream */
    double beta_leaf;   /* 0 = the model's */
    double repair_band; /* > 0: re-evaluate in FP64 when |w - round(w) +- 1/2| < this band instead of the
                           model's (GWN_PREC_FP32_REPAIR only); 0 = the model's (default 0) */
    double local_ratio; /* 3D, order-2 evaluation: a cluster that every query of a warp's packet (32 binned
                           queries) reaches, that is far for the packet's whole box and lies beyond this
                           many packet radii is taken by a second-order local expansion about the
                           packet's centre -- one expansion per cluster for the warp instead of one Taylor
                           term per query (a local-expansion far field; the paper evaluates every term per
                           query).  Its remainder falls like (1/ratio)^3 of the cluster's term, and the
                           remainders of the clusters a packet takes add up: with ~700 clusters per
                           packet, ratio 16 moved values by up to 7.6e-5 and 32 keeps them within 2e-5.  It pays
                           only where a packet's 32 queries are close together next to the clusters the
                           traversal accepts: on queries uniform in a CAD model's box at 1.2M points it
                           took 3 of 787 terms per query and slowed the traversal.  0 = the model's;
                           < 0 = off; >= 4 = this ratio (default 0) */
} gwn_query_opts;

void gwn_default_query_opts(gwn_query_opts* opts);

/* Build a 2D model from n NURBS curves (Algorithm 1, preprocessing):
 * Bezier extraction and adaptive subdivision (Section 3.2), chord moments
 * (Section 3.1: far from a curve its GWN equals that of its chord), BVH
 * (Section 3.1, Karras), moment up-sweep and centring.  On success *out holds
 * a device-resident model.  Errors: INVALID_ARG, INVALID_GEOMETRY, OOM, CUDA. */
gwn_status gwn_build_2d(const gwn_curve2d* curves, size_t n, const gwn_build_opts* opts, gwn_model* out);

/* Build a 3D model from n trimmed NURBS patches (Algorithm 1,
 * preprocessing): adaptive subdivision of the parameter rectangle with trims
 * clipped to every leaf (Section 3.2), leaf moments and centroid by
 * Gauss-Legendre quadrature over the trimmed region via Green's theorem
 * (Section 3.1, Figure 3), BVH, up-sweep and centring.  Same errors. */
gwn_status gwn_build_3d(const gwn_patch3d* patches, size_t n, const gwn_build_opts* opts, gwn_model* out);

/* GWN at n points (Algorithm 1, batched query).
 *   points    : n x 2 (2D model) or n x 3 (3D model), dtype GWN_F32 or GWN_F64
 *   mem       : GWN_MEM_DEVICE -- points and outputs are device pointers and the
 *               call is asynchronous on `stream`; GWN_MEM_HOST -- host pointers,
 *               staged through model-owned device buffers, synchronous.
 *   out_w     : n doubles (required); out_label: n int32 = round(w) (nullable);
 *   out_status: n uint32 GWN_QS_* bits (nullable).
 *   stream    : a cudaStream_t, or NULL for the default stream.
 * Calls on the same model share its scratch buffers: each call's work starts
 * after the previous call's (an event, also across streams), and calls from
 * several host threads are serialised by the model's lock.  n == 0 is a no-op. */
gwn_status gwn_query(gwn_model model, const void* points, int32_t points_dtype, int32_t mem, size_t n,
                     double* out_w, int32_t* out_label, uint32_t* out_status, const gwn_query_opts* qopts,
                     void* stream);

/* Query without any device allocation (the paper has no counterpart; this is
 * an interface for callers that cannot allocate).
 *
 * gwn_query may call cudaMalloc: the first query on a model, and any query
 * larger than the model's workspace, grow the workspace.  Some callers cannot
 * allow that: real-time loops that must never stall on an allocation
 * (cudaMalloc can synchronise the whole device), programs whose device memory
 * is entirely owned by another allocator or a fixed budget decided at start-up,
 * and code that must not change the process's device footprint after set-up.
 * gwn_query_noalloc serves them: it runs the FP32
 * traversal (every leaf evaluated in place, no spatial binning) and the FP64
 * repair of GWN_PREC_FP32_REPAIR with the model's beta, and its only scratch
 * is a file-scope device array of 4 MiB + 256 B that every GPU which loads
 * the library keeps until the process exits.  It calls no cudaMalloc or
 * cudaFree and no allocating library routine.
 *   points, out_w, out_label, out_status: device pointers as in gwn_query
 *     with GWN_MEM_DEVICE (out_label, out_status nullable); the call is
 *     asynchronous on `stream`.
 *   n <= 1,048,576 per call; larger n fails with GWN_ERR_INVALID_ARG.
 *   The first call on each device looks up the array's device address
 *   (cudaGetSymbolAddress) with that device current; make that first call
 *   before any stream capture.
 *   Every call shares the one array: calls whose work overlaps on the GPU
 *   (concurrent streams, or threads that do not serialise their streams)
 *   race and must not be issued.
 *   The model itself must have been built beforehand (gwn_build_* allocates). */
gwn_status gwn_query_noalloc(gwn_model model, const void* points, int32_t points_dtype, size_t n, double* out_w,
                             int32_t* out_label, uint32_t* out_status, void* stream);

typedef struct {
    int32_t dim;
    int64_t n_primitives;   /* curves or patches given to the build */
    int64_t n_leaves;       /* after Bezier extraction and subdivision */
    int64_t n_nodes;        /* internal nodes = n_leaves - 1 */
    int32_t max_depth;      /* deepest leaf */
    int64_t device_bytes;   /* device memory owned by the model */
    double build_ms;        /* wall time of the build */
    double beta, beta_repair, repair_band;
    int32_t order;
    double lo[3], hi[3];    /* box of all control points */
    double beta_leaf;       /* far-test factor of the leaves (3D; equals beta unless set or tuned) */
    int32_t device;         /* CUDA ordinal holding the model, or GWN_DEVICE_HOST_ONLY */
    int32_t bin_points_per_cell; /* 3D: points per Morton cell the query's spatial binning aims at (a chunk
                               of n points is binned with round(log2(n / this) / 3) bits per axis, 3..6);
                               picked by the autotuner from 4, 8, 16, 32, 64 by measured time (default 16).
                               2D: 0 (9 bits per axis) */
    int32_t stack_depth;    /* warp-stack entries of the packet traversal (from the tree depth) */
    double beta_repair_leaf; /* far-test factor of the FP64 repair's leaves (0: exact sum over every leaf) */
    int32_t eval_order;     /* Taylor order the queries evaluate: `order`, or 2 for a 3D model built with
                               order 3 whose autotuner found order 2 faster at the tolerance */
    double local_ratio;     /* 3D: the model's packet local-expansion ratio (gwn_query_opts.local_ratio);
                               0 = off */
} gwn_model_stats;

gwn_status gwn_model_info(gwn_model model, gwn_model_stats* stats);

/* Work counters of the last gwn_query on this model (synchronises the
 * device).  out holds 20 int64:
 *   out[0] exact-leaf (point, leaf) pairs of the 3D traversal
 *   out[1] points re-evaluated in FP64 (repair)
 *   out[2] 3D leaf evaluations moved to the FP64 near band
 *   out[3] points whose pairs did not fit the work list
 *   out[4..11] with count_work: internal nodes visited, leaves visited, Taylor
 *     evaluations, exact leaf evaluations, Gauss-Legendre nodes, sum of curve
 *     degrees over those nodes, foot-point searches, 2D chord angles
 *   out[12..13] with profile: traversal and exact-leaf kernel time in
 *     microseconds (CUDA events on the query's stream)
 *   out[14] exact-leaf pairs evaluated by the full evaluator (the others were
 *     read from the boundary curves' node tables)
 *   out[15] with count_work: Gauss-Legendre nodes read from the node tables
 *   out[16..17] with profile: the exact-leaf time split into the node-table
 *     kernel and the full evaluator (microseconds)
 *   out[18] with count_work: clusters taken by packets' local expansions
 *   out[19] zero (reserved) */
gwn_status gwn_last_query_stats(gwn_model model, int64_t* out);

/* Copy per-leaf records to host memory for inspection (used by the tests).
 * For each leaf i in BVH order: prim[i] = input primitive index and
 * param[4 i .. 4 i + 3] = (t0, t1, 0, 0) for curves or (u0, u1, v0, v1) for
 * patches.  Either pointer may be NULL; arrays hold n_leaves entries. */
gwn_status gwn_model_leaves(gwn_model model, int64_t* prim, double* param);

/* Copy the FP64 tree to host memory (used by the tests): for internal node k,
 * child[2k], child[2k+1] (>= 0: internal node, < 0: leaf ~index), centroid
 * x0[dim k ..], radius r[k], and the centred moments mom[k * M ..] laid out as
 * m0[d], m1[d][d], m2[d][d][d] with m1_ij = int (x - x0)_i n_j and
 * m2_ijk = int (x - x0)_i (x - x0)_j n_k (M = 14 in 2D), followed in 3D by
 * m3[3][3][3][3], m3_ijlk = int (x - x0)_i (x - x0)_j (x - x0)_l n_k (M = 120).
 * Any pointer may be NULL. */
gwn_status gwn_model_tree(gwn_model model, int32_t* child, double* x0, double* r, double* mom);

/* Checkpoint: write a built model (its host arrays: tree, moments, leaf
 * geometry, and its build options after autotuning) to `path`, so that a
 * serving process can restore it with gwn_model_load instead of rebuilding
 * (the paper has no counterpart).  Errors: INVALID_ARG (cannot open),
 * INTERNAL (write failed). */
gwn_status gwn_model_save(gwn_model model, const char* path);

/* Read a model written by gwn_model_save and upload it to `device` (-1 =
 * current, GWN_DEVICE_HOST_ONLY = host copy only).  A model saved from a
 * host-only build with beta = 0 is autotuned on load.  Errors: INVALID_ARG
 * (cannot open, not a model file of this library version, inconsistent
 * arrays), OOM, CUDA. */
gwn_status gwn_model_load(const char* path, int32_t device, gwn_model* out);

/* ---------------------------------------------------------------- batches
 * Many models and point sets in one launch.  Algorithm 1 is stated for one
 * model; a batch runs the query of each item (its own model, points and
 * outputs, all device memory) through the same pipeline as gwn_query with the
 * model's build options, the items spread over a pool of CUDA streams so that
 * their work overlaps on the GPU (an item of more than 2^20 points is spread
 * as chunk-aligned pieces, each with its own FP64 repair pass, so that one
 * large model does not run its chunks one after another at the end; the values
 * are those of the whole item).  The first call with a given item list
 * captures the whole fork/join into a CUDA graph; later calls with an
 * identical list (same models, pointers and sizes) replay it with a single
 * graph launch on the caller's stream.  Asynchronous: outputs are ready when
 * the caller's stream reaches the launch. */
typedef struct gwn_batch_s* gwn_batch;

typedef struct {
    gwn_model model;
    const void* points;    /* device, n x dim, points_dtype (GWN_F32 or GWN_F64) */
    int32_t points_dtype;
    size_t n;              /* may be 0 (item skipped) */
    double* out_w;         /* device, n values */
    int32_t* out_label;    /* device, n, nullable */
    uint32_t* out_status;  /* device, n, nullable (GWN_QS_* bits) */
} gwn_query_item;

/* A batch plan with n_streams streams (1..32), each owning a query workspace
 * sized for the largest model it has seen; on `device` (-1 = current).
 * Errors: INVALID_ARG, CUDA, OOM. */
gwn_status gwn_batch_create(int32_t n_streams, int32_t device, gwn_batch* out);

/* Enqueue the items on `stream` (cudaStream_t or NULL).  Models must have been
 * built on the plan's device and must outlive the plan's captured graph (the
 * next call with other items, or gwn_batch_release).  Errors: INVALID_ARG (bad
 * item), OOM (workspaces), CUDA (capture or launch). */
gwn_status gwn_query_batch(gwn_batch batch, const gwn_query_item* items, size_t n_items, void* stream);

/* The same batch with every item's points and outputs in HOST memory (the
 * call an application makes when its data lives on the CPU).  For each item
 * the library copies the points into device memory owned by the plan, runs
 * the item's query as gwn_query_batch does, and copies the values (and the
 * labels and status words, when requested) back, with one cudaMemcpyAsync
 * per buffer on the item's stream, so one item's copies overlap other items'
 * kernels.  When every host buffer is page-locked (cudaHostAlloc or
 * cudaHostRegister) the copies are captured with the kernels into the plan's
 * CUDA graph, and a later call with an identical item list replays it with a
 * single graph launch; pageable buffers are staged by the CUDA runtime and
 * the work is issued without a graph.  Synchronous: on return the outputs are
 * in the caller's host buffers.  The plan keeps device memory for the largest
 * item list it has staged (points + outputs) until gwn_batch_release.
 * Errors: as gwn_query_batch; OOM if the staging memory cannot be allocated. */
gwn_status gwn_query_batch_host(gwn_batch batch, const gwn_query_item* items, size_t n_items, void* stream);

/* Graph launches so far, graph captures so far, bytes of the stream workspaces
 * and of the staging memory of host items. */
gwn_status gwn_batch_info(gwn_batch batch, int64_t* graph_launches, int64_t* captures, int64_t* workspace_bytes);

/* Wait for the plan's streams and free it.  NULL is a no-op. */
gwn_status gwn_batch_release(gwn_batch batch);

/* ---------------------------------------------------------------- serving
 * A request loop over device-resident models with continuous batching (the
 * paper has no serving layer; this runs Algorithm 1's batched query per
 * request).  Requests are queued by gwn_serve_submit and admitted in arrival
 * order by a worker thread whenever one of n_slots slots (a CUDA stream with
 * its own query workspace) is free and the request's device memory (points +
 * outputs) fits the budget; requests in different slots run concurrently on
 * the GPU.  Models must outlive the server and are not released by it. */
typedef struct gwn_server_s* gwn_server;

typedef struct {
    int64_t mem_budget_bytes; /* device memory for the buffers (points + outputs) of the requests in
                                 flight (default 40 GiB); the slots' query workspaces, one per slot
                                 sized for the largest model, come on top */
    int32_t n_slots;          /* requests in flight at once (default 4) */
    int32_t device;           /* -1 = current */
} gwn_serve_opts;

void gwn_default_serve_opts(gwn_serve_opts* opts);

/* Start a server (spawns its worker thread).  Errors: INVALID_ARG, OOM. */
gwn_status gwn_serve_create(const gwn_serve_opts* opts, gwn_server* out);

/* Register a model; *model_id receives its id.  Only while no request is in
 * flight (else GWN_ERR_BUSY). */
gwn_status gwn_serve_add_model(gwn_server server, gwn_model model, int32_t* model_id);

/* Queue a request: n host points (n x dim, dtype GWN_F32 or GWN_F64), copied
 * before the call returns.  *request_id identifies it.  Errors: NOT_FOUND
 * (model id), INVALID_ARG (empty, or larger than the memory budget). */
gwn_status gwn_serve_submit(gwn_server server, int32_t model_id, const void* points, int32_t dtype, size_t n,
                            uint64_t* request_id);

/* Wait up to timeout_ms for a request; on success copy its n values
 * (out_w, FP64) and labels (out_label, nullable) and forget the request.
 * GWN_ERR_TIMEOUT if it has not finished (it stays queued); NOT_FOUND for an
 * unknown or already collected id. */
gwn_status gwn_serve_poll(gwn_server server, uint64_t request_id, double* out_w, int32_t* out_label,
                          int32_t timeout_ms);

typedef struct {
    int64_t submitted, completed, in_flight, queued;
    int64_t points_completed;
    double p50_ms, p99_ms, mean_ms;  /* submit -> results ready, over completed requests */
    double queries_per_s;            /* points completed / (last completion - first submit) */
    int64_t budget_used_bytes;
    int64_t max_in_flight;           /* most slots occupied at once (admitted, not finished) */
    int64_t max_gpu_overlap;         /* most completed requests whose device work windows (copy in .. copy
                                        out, CUDA events on their slots' streams) overlapped in time */
} gwn_server_stats;

gwn_status gwn_serve_stats(gwn_server server, gwn_server_stats* stats);

/* Finish the requests already admitted or queued, stop the worker and free
 * the server's memory.  NULL is a no-op. */
gwn_status gwn_serve_destroy(gwn_server server);

/* Release a model and all its device memory.  NULL is a no-op. */
gwn_status gwn_release(gwn_model model);

/* Thread-local description of the last error (never NULL). */
const char* gwn_last_error(void);

/* Library version string. */
const char* gwn_version(void);

#ifdef __cplusplus
}
#endif

#endif /* GWN_H */
