// query_pipeline.cuh -- the batched query as a sequence of kernels on one stream.
//
//  1. Spatial binning: each point gets the Morton code of its cell in a
//     2^kBinBits-per-axis grid over the model's box; a counting sort by cell
//     yields a permutation, so the 32 points of a warp are neighbours.
//  2. Traversal (Algorithm 1), one packet per warp: the warp's points walk the
//     tree together; far nodes (and, in 3D, far leaves) add their Taylor term
//     (Eq. 3) to each point's accumulator.  2D leaves are evaluated in place
//     (one atan2 unless the point is inside the leaf's box).  3D leaves that
//     need the exact evaluation are not evaluated in the traversal: the
//     (point, leaf) pairs are appended to a work list through a per-warp
//     shared-memory buffer, one atomic per 128 pairs;
//     points whose pairs do not fit are traversed again in up to two more
//     rounds.
//  3. 3D only: the work list is counting-sorted by leaf (one atomic per run of
//     a leaf, as the traversal writes them), and one thread per pair evaluates
//     the leaf in FP32 and adds it to the point's accumulator.  Consecutive
//     threads share the leaf, so a warp reads one set of boundary curves.  Far pairs whose panels stop at level 0 or 1 (nearly
//     all) read the curves' query-independent node tables (k_pair_fast); the
//     rest take the full evaluation (k_pair_eval: foot-point search, adaptive
//     panels from the Bernstein form).  Pairs FP32 cannot resolve go to the
//     FP64 near band (one warp per pair).
//  4. Finish: value, label and status per point; points whose value lies within
//     the repair band of a half-integer, or that were flagged, are appended to
//     the FP64 repair list (warp traversal + FP64 pairs, one warp per pair).
#pragma once

#include "gwn_internal.h"
#include "kernels2d.cuh"
#include "kernels3d.cuh"

namespace gwn {

constexpr int kBinBits2 = 9;   // 512 x 512 cells in 2D
constexpr int kBinBits3 = 5;   // 32^3 cells in 3D (default; the autotuner picks 4, 5 or 6 per model)
constexpr int kMaxBinCells = 1 << 18;  // 2^(2 x 9) = 2^(3 x 6)
constexpr uint32_t kPairOverflow = 0x100u;  // internal status bit: the point's pairs did not fit



__device__ __forceinline__ uint32_t spread_bits2(uint32_t x) {
    x &= 0x0000ffffu;
    x = (x | (x << 8)) & 0x00ff00ffu;
    x = (x | (x << 4)) & 0x0f0f0f0fu;
    x = (x | (x << 2)) & 0x33333333u;
    x = (x | (x << 1)) & 0x55555555u;
    return x;
}
__device__ __forceinline__ uint32_t spread_bits3(uint32_t x) {
    x &= 0x000003ffu;
    x = (x | (x << 16)) & 0xff0000ffu;
    x = (x | (x << 8)) & 0x0300f00fu;
    x = (x | (x << 4)) & 0x030c30c3u;
    x = (x | (x << 2)) & 0x09249249u;
    return x;
}

__device__ __forceinline__ void flush_work(const WorkLocal& wl, unsigned long long* work) {
    for (int k = 0; k < kWorkCount; ++k)
        if (wl.v[k]) atomicAdd(&work[k], wl.v[k]);
}

__device__ __forceinline__ void load_point_f(const void* pts, int dtype, int dim, long long i, float* q) {
    if (dtype == GWN_F32) {
        const float* p = reinterpret_cast<const float*>(pts) + i * dim;
        for (int k = 0; k < dim; ++k) q[k] = p[k];
    } else {
        const double* p = reinterpret_cast<const double*>(pts) + i * dim;
        for (int k = 0; k < dim; ++k) q[k] = (float)p[k];
    }
}

// order-preserving integer key of a float (larger float, larger key) and back
__device__ __forceinline__ unsigned float_key(float f) {
    const unsigned u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float key_float(unsigned k) {
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7fffffffu) : ~k);
}

// bounding box of the n points: box[0..2] receive the complemented keys of the
// minima and box[3..5] the keys of the maxima (box zeroed beforehand, so that
// atomicMax serves both), one atomic per block and coordinate
template <int DIM>
__global__ void __launch_bounds__(128) k_bbox(const void* pts, int dtype, int n, unsigned* box) {
    __shared__ unsigned sk[4][6];
    const unsigned full = 0xffffffffu;
    unsigned kmin[3] = {0u, 0u, 0u}, kmax[3] = {0u, 0u, 0u};  // complemented minima, maxima
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        float q[3] = {0, 0, 0};
        load_point_f(pts, dtype, DIM, i, q);
        for (int k = 0; k < DIM; ++k) {
            if (q[k] != q[k]) continue;  // NaN: no cell of its own
            const unsigned key = float_key(q[k]);
            kmin[k] = max(kmin[k], ~key);
            kmax[k] = max(kmax[k], key);
        }
    }
    for (int k = 0; k < 3; ++k)
        for (int off = 16; off > 0; off >>= 1) {
            kmin[k] = max(kmin[k], __shfl_xor_sync(full, kmin[k], off));
            kmax[k] = max(kmax[k], __shfl_xor_sync(full, kmax[k], off));
        }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
        for (int k = 0; k < 3; ++k) {
            sk[warp][k] = kmin[k];
            sk[warp][3 + k] = kmax[k];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        unsigned v = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) v = max(v, sk[w][threadIdx.x]);
        if (v) atomicMax(&box[threadIdx.x], v);
    }
}

template <int DIM>
__global__ void k_bin(const void* pts, int dtype, int n, const unsigned* box, int bits, int* key, int* hist) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float q[3] = {0, 0, 0};
    load_point_f(pts, dtype, DIM, i, q);
    const float cells = (float)(1 << bits);
    // the grid spans the chunk's own box (k_bbox), so that points gathered in a
    // small part of the model's box still fall into many cells
    float l[3] = {0.f, 0.f, 0.f}, s[3] = {0.f, 0.f, 0.f};
    for (int k = 0; k < DIM; ++k) {
        l[k] = key_float(~box[k]);
        const float e = key_float(box[3 + k]) - l[k];
        s[k] = e > 0.f ? 1.f / e : 0.f;
    }
    uint32_t c[3];
    for (int k = 0; k < DIM; ++k) {
        float t = (q[k] - l[k]) * s[k] * cells;
        t = fminf(fmaxf(t, 0.f), cells - 1.f);
        c[k] = (uint32_t)t;
    }
    int code = DIM == 2 ? (int)(spread_bits2(c[0]) | (spread_bits2(c[1]) << 1))
                        : (int)(spread_bits3(c[0]) | (spread_bits3(c[1]) << 1) | (spread_bits3(c[2]) << 2));
    key[i] = code;
    atomicAdd(&hist[code], 1);
}

// exclusive scan of hist[0..K) in place by one block
__global__ void k_scan(int* hist, int K) {
    __shared__ int part[1024];
    __shared__ int carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int base = 0; base < K; base += 1024) {
        int i = base + threadIdx.x;
        int v = i < K ? hist[i] : 0;
        part[threadIdx.x] = v;
        __syncthreads();
        for (int off = 1; off < 1024; off <<= 1) {
            int t = threadIdx.x >= off ? part[threadIdx.x - off] : 0;
            __syncthreads();
            part[threadIdx.x] += t;
            __syncthreads();
        }
        if (i < K) hist[i] = carry + part[threadIdx.x] - v;
        __syncthreads();
        if (threadIdx.x == 1023) carry += part[1023];
        __syncthreads();
    }
}

__global__ void k_scatter_perm(int n, const int* key, int* cursor, int* perm) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int pos = atomicAdd(&cursor[key[i]], 1);
    perm[pos] = i;
}

constexpr int kPairBuf = 128;  // (point, leaf) pairs buffered per warp in shared memory

// write a warp's buffered pairs (n of them, warp-uniform) to the pair list with
// one atomic and coalesced stores.  If the list is full, the lanes that own the
// entries which did not fit are added to `ovf` (every lane gets the same mask);
// their points skip the pair pass and are traversed again in the next round.
__device__ __forceinline__ void flush_warp_pairs(const int2* buf, const unsigned char* own, int n, const Workspace& ws,
                                                 unsigned& ovf) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int base = 0;
    if (lane == 0 && n > 0) base = atomicAdd(&ws.counters[0], n);
    base = __shfl_sync(full, base, 0);
    unsigned lost = 0;
    for (int j = lane; j < n; j += 32) {
        const long long pos = (long long)base + j;
        if (pos < ws.pair_cap) ws.pairs[pos] = buf[j];
        else lost |= 1u << own[j];
    }
    for (int off = 16; off > 0; off >>= 1) lost |= __shfl_xor_sync(full, lost, off);
    ovf |= lost;
}

// traversal with deferred 3D leaves, one packet per warp: the 32 queries of a
// warp (neighbours in the binned order) walk the tree together.  The warp
// holds one internal node and the mask of its lanes for which that node was
// near; an iteration tests both children of the node for those lanes: far
// lanes add the child's Taylor term, and for a leaf the lanes that need it
// exactly write their pairs, for an internal child the lanes for which it is
// near need its subtree.  The walk goes on into a near child and keeps the
// other (if it is near too) on a warp stack in shared memory.  Node and moment
// loads are the same address for the whole warp, and lanes never wait on each
// other's different branches.  Binned queries share most of their paths (the
// union of a warp's visits is ~1.05x the longest single path), so the packet
// costs little extra work; testing the children inline makes one loop
// iteration and at most one stack entry per near node, not one per node
// tested.  Exact 3D leaves go to the pair list: at a leaf, the lanes that need
// it exactly write their (point, leaf) pairs next to each other into the
// warp's shared-memory buffer, which is flushed to the list with one atomic
// when full, so the list comes out in runs of one leaf (the pair kernels read a
// leaf's data once per run, with no sort by leaf).  Every thread of the grid
// reaches the flushes (lanes past the end of the list take part with an empty
// mask).
// n_dev != nullptr: the point list `perm` holds *n_dev entries (a later round
// over the points whose pairs overflowed; their indices go to `olist_out`)
// STACK: entries of the warp stack (pending near siblings along the packet's
// path), chosen per model from its tree depth (64, 96 or 128).  O3: the model
// evaluates the order-3 terms (a separate instance, so that order-2 models do
// not pay its registers)
constexpr int kPacketStack = 96;  // entries per warp of the 2D traversal

template <int STACK, bool O3>
__global__ void __launch_bounds__(128) k_trav3(DevTree t, const void* pts, int dtype, int n, const int* perm,
                                               float beta2, float beta2l, Workspace ws, unsigned long long* work,
                                               const int* n_dev, int* olist_out) {
    __shared__ int2 sstk[4][STACK];
    __shared__ int2 sbuf[4][kPairBuf];
    __shared__ unsigned char sown[4][kPairBuf];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int2* stk = sstk[threadIdx.x >> 5];
    int2* buf = sbuf[threadIdx.x >> 5];
    unsigned char* own = sown[threadIdx.x >> 5];
    WorkLocal wl = {};
    if (n_dev) n = *n_dev;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (n_dev && blockIdx.x * blockDim.x >= n) return;  // whole block past the list
    const bool active = i < n;
    int qi = active ? (perm ? perm[i] : i) : 0;
    float q[3] = {0, 0, 0};
    if (active) load_point_f(pts, dtype, 3, qi, q);
    float w = 0.f;
    uint32_t st = 0;
    int bcnt = 0;                      // warp-uniform: entries in buf
    unsigned ovf = 0;                  // lanes with pairs that did not fit the list
    int sp = 0;                        // warp-uniform

    // Test node or leaf c for the lanes of `msk` (warp-uniform c and msk):
    // Taylor terms for the far lanes, pairs for the lanes that need a leaf
    // exactly; returns the lanes for which an internal c is near.
    auto test = [&](int c, unsigned msk, const float4& h) -> unsigned {
        const bool mine = (msk >> lane) & 1u;
        if (c < 0) {
            const int li = ~c;
            const float rx = h.x - q[0], ry = h.y - q[1], rz = h.z - q[2];
            const bool far = mine && t.leaf_far && rx * rx + ry * ry + rz * rz > beta2l * h.w;
            if (work && mine) wl.v[kWorkLeafTests] += 1;
            if (far) {
                if (work) wl.v[kWorkFar] += 1;
                w += far3_node32(t.lmom + (size_t)li * kMom3Vec, rx, ry, rz, O3);
            }
            const unsigned need = __ballot_sync(full, mine && !far);
            if (need) {
                const int nn = __popc(need);
                if (bcnt + nn > kPairBuf) {
                    __syncwarp();
                    flush_warp_pairs(buf, own, bcnt, ws, ovf);
                    bcnt = 0;
                    __syncwarp();
                }
                if ((need >> lane) & 1u) {
                    const int pos = bcnt + __popc(need & ((1u << lane) - 1u));
                    buf[pos] = make_int2(qi, li);
                    own[pos] = (unsigned char)lane;
                }
                bcnt += nn;
            }
            return 0u;
        }
        const float rx = h.x - q[0], ry = h.y - q[1], rz = h.z - q[2];
        const bool far = mine && rx * rx + ry * ry + rz * rz > beta2 * h.w;
        if (work && mine) wl.v[kWorkNodes] += 1;
        if (far) {
            if (work) wl.v[kWorkFar] += 1;
            w += far3_node32(t.mom + (size_t)c * kMom3Vec, rx, ry, rz, O3);
        }
        return __ballot_sync(full, mine && !far);
    };

    int node = t.root;  // warp-uniform
    unsigned mask = __ballot_sync(full, active);
    if (mask) mask = test(node, mask, node < 0 ? GWN_LDG(t.lhdr + ~node) : GWN_LDG(t.hdr + node));  // the root
    while (mask) {
        // the child indices and both children's headers, loaded together
        const int2 ch = GWN_LDG(t.child + node);
        const float4 ha = GWN_LDG(t.chdr + 2 * node), hb = GWN_LDG(t.chdr + 2 * node + 1);
        const unsigned na = test(ch.x, mask, ha);
        const unsigned nb = test(ch.y, mask, hb);
        if (na) {
            if (nb) {
                if (sp < STACK) {
                    if (lane == 0) stk[sp] = make_int2(ch.y, (int)nb);
                    ++sp;
                } else if ((nb >> lane) & 1u) {
                    st |= GWN_QS_STACK_OVERFLOW;  // the second subtree is dropped for these lanes
                }
                __syncwarp();
            }
            node = ch.x;
            mask = na;
        } else if (nb) {
            node = ch.y;
            mask = nb;
        } else {
            if (sp == 0) break;
            --sp;
            const int2 e = stk[sp];
            node = e.x;
            mask = (unsigned)e.y;
            __syncwarp();
        }
    }
    __syncwarp();
    flush_warp_pairs(buf, own, bcnt, ws, ovf);
    if ((ovf >> lane) & 1u) st |= kPairOverflow;
    if (active) {
        ws.wacc[qi] = w;
        ws.st[qi] = st;
        if (st & kPairOverflow) olist_out[atomicAdd(&ws.counters[3], 1)] = qi;
    }
    if (work) flush_work(wl, work);
}

// k_trav3 with the packet local expansion (order-2 models, query option
// local_ratio; a local-expansion far field beyond the paper): the same walk,
// and a node or leaf that every active lane of the packet needs, that passes
// the far test for every point of the packet's box (|x0 - p| > beta r + rho,
// p and rho the box's centre and half diagonal) and lies beyond kappa rho
// (kappa2 = kappa^2) is not evaluated per lane: it goes to a per-warp list,
// and 32 of them at a time each lane forms one node's second-order local
// expansion about p (far3_local2), summed over the warp; every lane evaluates
// the summed expansion at its own point at the end.  A kernel of its own:
// sharing k_trav3's body cost the plain traversal 4 % (9.16 -> 9.51 ms on a
// 2M-query model) at the same register count.
template <int STACK>
__global__ void __launch_bounds__(128) k_trav3_local(DevTree t, const void* pts, int dtype, int n, const int* perm,
                                               float beta2, float beta2l, Workspace ws, unsigned long long* work,
                                               const int* n_dev, int* olist_out, float kappa2) {
    __shared__ int2 sstk[4][STACK];
    __shared__ int2 sbuf[4][kPairBuf];
    __shared__ unsigned char sown[4][kPairBuf];
    __shared__ int slocal[4][32];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int2* stk = sstk[threadIdx.x >> 5];
    int2* buf = sbuf[threadIdx.x >> 5];
    unsigned char* own = sown[threadIdx.x >> 5];
    int* lst = slocal[threadIdx.x >> 5];
    WorkLocal wl = {};
    if (n_dev) n = *n_dev;
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (n_dev && blockIdx.x * blockDim.x >= n) return;  // whole block past the list
    const bool active = i < n;
    int qi = active ? (perm ? perm[i] : i) : 0;
    float q[3] = {0, 0, 0};
    if (active) load_point_f(pts, dtype, 3, qi, q);
    float w = 0.f;
    uint32_t st = 0;
    int bcnt = 0;                      // warp-uniform: entries in buf
    unsigned ovf = 0;                  // lanes with pairs that did not fit the list
    int sp = 0;                        // warp-uniform
    const unsigned amask = __ballot_sync(full, active);

    // packet box of the active lanes (centre p, half diagonal rho) and the
    // local expansion's coefficients (F, grad F, Hessian), the same in all lanes
    float pc[3] = {0.f, 0.f, 0.f}, rho = 0.f, lc[10];
    int lcnt = 0;  // warp-uniform: entries in lst
    {
        float d2 = 0.f;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float lo = active ? q[k] : 3.0e38f, hi = active ? q[k] : -3.0e38f;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                lo = fminf(lo, __shfl_xor_sync(full, lo, off));
                hi = fmaxf(hi, __shfl_xor_sync(full, hi, off));
            }
            pc[k] = 0.5f * (lo + hi);
            d2 += (hi - lo) * (hi - lo);
        }
        rho = 0.5f * sqrtf(d2);
#pragma unroll
        for (int k = 0; k < 10; ++k) lc[k] = 0.f;
    }
    // every lane takes one listed node's expansion, and the warp sums them
    auto flush_local = [&]() {
        float v[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) v[k] = 0.f;
        __syncwarp();
        if (lane < lcnt) {
            const int c = lst[lane];
            const float4 h = c < 0 ? GWN_LDG(t.lhdr + ~c) : GWN_LDG(t.hdr + c);
            const float4* M = c < 0 ? t.lmom + (size_t)(~c) * kMom3Vec : t.mom + (size_t)c * kMom3Vec;
            far3_local2(M, h.x - pc[0], h.y - pc[1], h.z - pc[2], v);
        }
#pragma unroll
        for (int k = 0; k < 10; ++k) {
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) v[k] += __shfl_xor_sync(full, v[k], off);
            lc[k] += v[k];
        }
        lcnt = 0;
        __syncwarp();
    };
    // c is far for the whole packet box and beyond kappa rho: list it (true)
    auto packet_far = [&](int c, unsigned msk, const float4& h, float b2) -> bool {
        if (msk != amask) return false;
        const float dx = h.x - pc[0], dy = h.y - pc[1], dz = h.z - pc[2];
        const float dd = dx * dx + dy * dy + dz * dz;
        const float lim = sqrtf(b2 * h.w) + rho;
        if (!(dd > kappa2 * rho * rho && dd > lim * lim)) return false;
        if (lane == 0) lst[lcnt] = c;
        if (work && ((amask >> lane) & 1u)) wl.v[kWorkLocal] += 1;
        if (++lcnt == 32) flush_local();
        return true;
    };

    // Test node or leaf c for the lanes of `msk` (warp-uniform c and msk):
    // Taylor terms for the far lanes, pairs for the lanes that need a leaf
    // exactly; returns the lanes for which an internal c is near.
    auto test = [&](int c, unsigned msk) -> unsigned {
        const bool mine = (msk >> lane) & 1u;
        if (c < 0) {
            const int li = ~c;
            const float4 h = GWN_LDG(t.lhdr + li);
            if (work && mine) wl.v[kWorkLeafTests] += 1;
            if (t.leaf_far && packet_far(c, msk, h, beta2l)) return 0u;
            const float rx = h.x - q[0], ry = h.y - q[1], rz = h.z - q[2];
            const bool far = mine && t.leaf_far && rx * rx + ry * ry + rz * rz > beta2l * h.w;
            if (far) {
                if (work) wl.v[kWorkFar] += 1;
                w += far3_node32(t.lmom + (size_t)li * kMom3Vec, rx, ry, rz, false);
            }
            const unsigned need = __ballot_sync(full, mine && !far);
            if (need) {
                const int nn = __popc(need);
                if (bcnt + nn > kPairBuf) {
                    __syncwarp();
                    flush_warp_pairs(buf, own, bcnt, ws, ovf);
                    bcnt = 0;
                    __syncwarp();
                }
                if ((need >> lane) & 1u) {
                    const int pos = bcnt + __popc(need & ((1u << lane) - 1u));
                    buf[pos] = make_int2(qi, li);
                    own[pos] = (unsigned char)lane;
                }
                bcnt += nn;
            }
            return 0u;
        }
        const float4 h = GWN_LDG(t.hdr + c);
        if (work && mine) wl.v[kWorkNodes] += 1;
        if (packet_far(c, msk, h, beta2)) return 0u;
        const float rx = h.x - q[0], ry = h.y - q[1], rz = h.z - q[2];
        const bool far = mine && rx * rx + ry * ry + rz * rz > beta2 * h.w;
        if (far) {
            if (work) wl.v[kWorkFar] += 1;
            w += far3_node32(t.mom + (size_t)c * kMom3Vec, rx, ry, rz, false);
        }
        return __ballot_sync(full, mine && !far);
    };

    int node = t.root;  // warp-uniform
    unsigned mask = __ballot_sync(full, active);
    if (mask) mask = test(node, mask);  // the root itself (a leaf when the model has one)
    while (mask) {
        const int2 ch = GWN_LDG(t.child + node);
        const unsigned na = test(ch.x, mask);
        const unsigned nb = test(ch.y, mask);
        if (na) {
            if (nb) {
                if (sp < STACK) {
                    if (lane == 0) stk[sp] = make_int2(ch.y, (int)nb);
                    ++sp;
                } else if ((nb >> lane) & 1u) {
                    st |= GWN_QS_STACK_OVERFLOW;  // the second subtree is dropped for these lanes
                }
                __syncwarp();
            }
            node = ch.x;
            mask = na;
        } else if (nb) {
            node = ch.y;
            mask = nb;
        } else {
            if (sp == 0) break;
            --sp;
            const int2 e = stk[sp];
            node = e.x;
            mask = (unsigned)e.y;
            __syncwarp();
        }
    }
    {
        if (lcnt > 0) flush_local();
        // F(D - s) ~ F - grad F . s + s^T H s / 2, s = q - p
        const float sx = q[0] - pc[0], sy = q[1] - pc[1], sz = q[2] - pc[2];
        w += lc[0] - (lc[1] * sx + lc[2] * sy + lc[3] * sz) +
             0.5f * (lc[4] * sx * sx + lc[5] * sy * sy + lc[6] * sz * sz) + lc[7] * sx * sy + lc[8] * sx * sz +
             lc[9] * sy * sz;
    }
    __syncwarp();
    flush_warp_pairs(buf, own, bcnt, ws, ovf);
    if ((ovf >> lane) & 1u) st |= kPairOverflow;
    if (active) {
        ws.wacc[qi] = w;
        ws.st[qi] = st;
        if (st & kPairOverflow) olist_out[atomicAdd(&ws.counters[3], 1)] = qi;
    }
    if (work) flush_work(wl, work);
}

// points whose pairs still overflowed after the last round: whole traversal
// again, leaves in place
__global__ void __launch_bounds__(128) k_overflow3(DevTree t, const void* pts, int dtype, float beta2, Workspace ws,
                                                   const int* list) {
    int cnt = ws.counters[3];
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        int qi = list[k];
        float q[3];
        load_point_f(pts, dtype, 3, qi, q);
        uint32_t st = 0;
        ws.wacc[qi] = query3_32(t, q[0], q[1], q[2], beta2, st);
        ws.st[qi] = st;
    }
}

// Counting sort of the pair list by leaf, one run at a time: the traversal
// writes each leaf's pairs of a warp in one run, so the lanes of a warp that
// hold the same leaf (__match_any_sync) take one atomic for their run, in the
// histogram pass and in the scatter pass.  Sorted, a leaf's pairs from every
// warp are contiguous and the pair kernels read its tables once for many warps.
__global__ void k_pair_hist(long long npair_cap, const int* counters, const int2* pairs, int* hist) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long np = min((long long)counters[0], npair_cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < np; base += stride) {
        const long long k = base + threadIdx.x;
        const int leaf = k < np ? pairs[k].y : -1;
        const unsigned m = __match_any_sync(full, leaf);
        if (leaf >= 0 && lane == __ffs(m) - 1) atomicAdd(&hist[leaf], __popc(m));
    }
}

__global__ void k_pair_sort(long long npair_cap, const int* counters, const int2* pairs, int* cursor, int2* out) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const long long np = min((long long)counters[0], npair_cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < np; base += stride) {
        const long long k = base + threadIdx.x;
        const int2 pr = k < np ? pairs[k] : make_int2(0, -1);
        const unsigned m = __match_any_sync(full, pr.y);
        const int leader = __ffs(m) - 1;
        int start = 0;
        if (pr.y >= 0 && lane == leader) start = atomicAdd(&cursor[pr.y], __popc(m));
        start = __shfl_sync(full, start, leader);
        if (pr.y >= 0) out[start + __popc(m & ((1u << lane) - 1u))] = pr;
    }
}

// exact 3D leaves from the node tables, one thread per (point, leaf) pair in
// leaf order (the 32 pairs of a warp mostly share one leaf, so its table is
// read once for the warp, and consecutive warps reuse it from L1): pairs whose point lies outside the leaf's
// 1.1-radius sphere and whose panels stop at level 0 or 1 add their value
// here (leaf3_fast32).  The others -- points near the leaf, whose string needs
// the foot-point search, and curves that need deeper panels -- are appended in
// order to `slow` (counter [8]) for k_pair_eval.  Every thread of a block runs
// the same iterations, so a warp appends with a single atomic.
__global__ void __launch_bounds__(128) k_pair_fast(DevTree t, const void* pts, int dtype, long long npair_cap,
                                                   int* counters, const int2* pairs, float* wacc, const uint32_t* st,
                                                   int2* slow, unsigned long long* work) {
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    WorkLocal wl = {};
    const long long np = min((long long)counters[0], npair_cap);
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long base = (long long)blockIdx.x * blockDim.x; base < np; base += stride) {
        const long long k = base + threadIdx.x;
        bool to_slow = false;
        int2 pr = make_int2(0, 0);
        if (k < np) {
            pr = pairs[k];
            if (!(st[pr.x] & kPairOverflow)) {  // overflowed points are recomputed by k_overflow3
                float q[3];
                load_point_f(pts, dtype, 3, pr.x, q);
                const Leaf3Info I = t.leaf3[pr.y];
                const float qr[3] = {q[0] - I.cen[0], q[1] - I.cen[1], q[2] - I.cen[2]};
                const float d2 = qr[0] * qr[0] + qr[1] * qr[1] + qr[2] * qr[2];
                const float rfar = 1.1f * I.rad;
                float v;
                if (d2 > rfar * rfar && leaf3_fast32(t, I, qr, d2, &v, work ? &wl : nullptr))
                    atomicAdd(&wacc[pr.x], v);
                else
                    to_slow = true;
            }
        }
        const unsigned m = __ballot_sync(full, to_slow);
        if (m) {
            const int leader = __ffs(m) - 1;
            int slot0 = 0;
            if (lane == leader) slot0 = atomicAdd(&counters[8], __popc(m));
            slot0 = __shfl_sync(full, slot0, leader);
            if (to_slow) slow[slot0 + __popc(m & ((1u << lane) - 1u))] = pr;
        }
    }
    if (work) flush_work(wl, work);
}

// the pairs that k_pair_fast left (count *count): the full FP32 evaluation
// (foot-point search, adaptive panels from the curves' Bernstein form); pairs
// FP32 cannot resolve go to the FP64 near band
__global__ void __launch_bounds__(128, 5) k_pair_eval(DevTree t, const void* pts, int dtype, long long npair_cap,
                                                   const int* count, int* counters, const int2* pairs, float* wacc,
                                                   uint32_t* st, int2* pairs64, int npair64_cap,
                                                   unsigned long long* work) {
    WorkLocal wl = {};
    long long np = min((long long)*count, npair_cap);
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < np; k += (long long)gridDim.x * blockDim.x) {
        int2 pr = pairs[k];
        if (st[pr.x] & kPairOverflow) continue;  // recomputed by k_overflow3
        float q[3];
        load_point_f(pts, dtype, 3, pr.x, q);
        float v;
        if (leaf3_try32(t, pr.y, q[0], q[1], q[2], &v, work ? &wl : nullptr, false)) {
            atomicAdd(&wacc[pr.x], v);
        } else {
            int slot = atomicAdd(&counters[2], 1);
            if (slot < npair64_cap) pairs64[slot] = pr;
            atomicOr(&st[pr.x], slot < npair64_cap ? GWN_QS_NEAR : GWN_QS_STACK_OVERFLOW);
        }
    }
    if (work) flush_work(wl, work);
}

// 4-point FP64 panels are used for leaves whose boundary curves all have degree
// <= 6 (pieces of degree 1 composed with the bicubic net); curves of higher
// degree (rational trims) take 8-point panels, whose error does not depend on
// how close the rational parametrisation's poles come to the panel
__device__ __forceinline__ bool leaf_fits_w4(const DevTree& t, int li) {
    const Leaf3Info I = t.leaf3[li];
    int dmax = 0;
    for (int c = threadIdx.x & 31; c < I.c3_cnt; c += 32) dmax = max(dmax, t.c3[I.c3_off + c].deg);
    for (int off = 16; off > 0; off >>= 1) dmax = max(dmax, __shfl_xor_sync(0xffffffffu, dmax, off));
    return dmax <= 6;
}

// the near band with one warp per pair (leaf3_warp64)
__global__ void __launch_bounds__(128) k_pair_eval64_warp(DevTree t, const void* pts, int dtype, int npair64_cap,
                                                          const int* counters, const int2* pairs64, float* wacc,
                                                          uint32_t* st) {
    __shared__ int2 sstk[4][kQuadStack];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int np = min(counters[2], npair64_cap);
    for (int k = blockIdx.x * 4 + wid; k < np; k += gridDim.x * 4) {
        const int2 pr = pairs64[k];
        double q[3];
        if (dtype == GWN_F32) {
            const float* p = reinterpret_cast<const float*>(pts) + (size_t)pr.x * 3;
            q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
        } else {
            const double* p = reinterpret_cast<const double*>(pts) + (size_t)pr.x * 3;
            q[0] = (double)(float)p[0]; q[1] = (double)(float)p[1]; q[2] = (double)(float)p[2];
        }
        double v = 0;
        const bool ok = leaf_fits_w4(t, pr.y) ? leaf3_warp64<4>(t, pr.y, q, kRatio64BandW4, kLevel64, sstk[wid], &v)
                                              : leaf3_warp64<8>(t, pr.y, q, kRatio64Band, kLevel64, sstk[wid], &v);
        if (lane == 0) {
            atomicAdd(&wacc[pr.x], ok ? (float)v : 0.f);
            if (!ok) atomicOr(&st[pr.x], GWN_QS_UNRESOLVED);
        }
        __syncwarp();
    }
}

// 2D traversal in binned order, one packet per warp as in k_trav3 (node + lane
// mask, second children on a shared-memory warp stack); 2D leaves are
// evaluated in place by the lanes that reach them (an exact 2D leaf costs a
// chord angle, see leaf2_eval32)
__global__ void __launch_bounds__(128) k_trav2(DevTree t, const void* pts, int dtype, int n, const int* perm,
                                               float beta2, Workspace ws, unsigned long long* work) {
    __shared__ int2 sstk[4][kPacketStack];
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    int2* stk = sstk[threadIdx.x >> 5];
    WorkLocal wl = {};
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const bool active = i < n;
    const int qi = active ? (perm ? perm[i] : i) : 0;
    float q[2] = {0, 0};
    if (active) load_point_f(pts, dtype, 2, qi, q);
    float w = 0.f;
    uint32_t st = 0;
    int sp = 0;                        // warp-uniform
    int node = t.root;                 // warp-uniform
    unsigned mask = __ballot_sync(full, active);
    while (mask) {
        const bool mine = (mask >> lane) & 1u;
        bool descend = false;
        if (node < 0) {
            if (mine) {
                if (work) wl.v[kWorkLeaves] += 1;
                w += leaf2_eval32(t, ~node, q[0], q[1], st);
            }
        } else {
            const float4 h = GWN_LDG(t.hdr + node);
            const float rx = h.x - q[0], ry = h.y - q[1];
            const bool far = mine && rx * rx + ry * ry > beta2 * h.w;
            if (work && mine) wl.v[kWorkNodes] += 1;
            if (far) {
                if (work) wl.v[kWorkFar] += 1;
                const float4* M = t.mom + (size_t)node * kMom2Vec;
                const float4 a = GWN_LDG(M), b = GWN_LDG(M + 1), c = GWN_LDG(M + 2);
                const float f[12] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w, c.x, c.y, c.z, c.w};
                w += far2_eval<float>(f, rx, ry);
            }
            const unsigned near = __ballot_sync(full, mine && !far);
            if (near) {
                const int2 ch = GWN_LDG(t.child + node);
                if (sp < kPacketStack) {
                    if (lane == 0) stk[sp] = make_int2(ch.y, (int)near);
                    ++sp;
                } else if ((near >> lane) & 1u) {
                    st |= GWN_QS_STACK_OVERFLOW;  // the second subtree is dropped for these lanes
                }
                __syncwarp();
                node = ch.x;
                mask = near;
                descend = true;
            }
        }
        if (!descend) {
            if (sp == 0) break;
            --sp;
            const int2 e = stk[sp];
            node = e.x;
            mask = (unsigned)e.y;
            __syncwarp();
        }
    }
    if (active) {
        ws.wacc[qi] = w;
        ws.st[qi] = st;
    }
    if (work) flush_work(wl, work);
}

// outputs of one chunk (points off .. off + n - 1 of the query); points to
// repair go to the query's list (index off + i) while it has room, else to the
// chunk's own list (index i), repaired right after the chunk
__global__ void k_finish(int n, const float* wacc, const uint32_t* stv, int precision, float band, double* out_w,
                         int* out_label, uint32_t* out_status, int* rlist, int* rcount, int off, int* rlist_g,
                         int* gcount, int gcap) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double w = (double)wacc[i];
    uint32_t st = stv[i];
    if (precision == GWN_PREC_FP32_REPAIR) {
        double fr = w - floor(w);
        if (fabs(fr - 0.5) < (double)band || (st & (GWN_QS_STACK_OVERFLOW | GWN_QS_UNRESOLVED))) {
            int slot = atomicAdd(gcount, 1);
            if (slot < gcap) {
                rlist_g[slot] = off + i;
            } else {
                slot = atomicAdd(rcount, 1);
                rlist[slot] = i;
            }
        }
    }
    out_w[i] = w;
    if (out_label) out_label[i] = (int)round(w);
    if (out_status) out_status[i] = st;
}

}  // namespace gwn

namespace gwn {

__device__ __forceinline__ void load_point_d(const void* pts, int dtype, long long i, double q[3]) {
    if (dtype == GWN_F32) {
        const float* p = reinterpret_cast<const float*>(pts) + (size_t)i * 3;
        q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
    } else {
        const double* p = reinterpret_cast<const double*>(pts) + (size_t)i * 3;
        q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
    }
}

// FP64 repair pairs from the FP64 node tables, one warp per pair
// (leaf3_fast64_warp: far pairs whose 8-point panels stop at level 0 or 1, at
// the repair ratio); the others go to the second list for k_rpairs3_warp
__global__ void __launch_bounds__(128) k_rpairs3_fast(DevTree t, const void* pts, int dtype, RepairList R) {
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long np = min((long long)*R.npairs, kRepairPairCap);
    for (long long j = (long long)blockIdx.x * 4 + wid; j < np; j += (long long)gridDim.x * 4) {
        const int2 pr = R.pairs[j];
        double q[3];
        load_point_d(pts, dtype, R.idx[pr.x], q);
        double v = 0;
        const bool ok = leaf3_fast64_warp(t, pr.y, q, kRatio64Repair, &v);
        if (lane == 0) {
            if (ok) atomicAdd(&R.rw[pr.x], v);
            else R.pairs2[atomicAdd(R.npairs2, 1)] = pr;
        }
        __syncwarp();
    }
}

// FP64 repair pairs with one warp per pair (leaf3_warp64): those the tables left
__global__ void __launch_bounds__(128) k_rpairs3_warp(DevTree t, const void* pts, int dtype, RepairList R) {
    __shared__ int2 sstk[4][kQuadStack];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long np = min((long long)*R.npairs2, kRepairPairCap);
    for (long long j = (long long)blockIdx.x * 4 + wid; j < np; j += (long long)gridDim.x * 4) {
        const int2 pr = R.pairs2[j];
        const int qi = R.idx[pr.x];
        double q[3];
        if (dtype == GWN_F32) {
            const float* p = reinterpret_cast<const float*>(pts) + (size_t)qi * 3;
            q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
        } else {
            const double* p = reinterpret_cast<const double*>(pts) + (size_t)qi * 3;
            q[0] = p[0]; q[1] = p[1]; q[2] = p[2];
        }
        double v = 0;
        const bool ok = leaf_fits_w4(t, pr.y) ? leaf3_warp64<4>(t, pr.y, q, kRatio64RepairW4, kLevel64, sstk[wid], &v)
                                              : leaf3_warp64<8>(t, pr.y, q, kRatio64Repair, kLevel64, sstk[wid], &v);
        if (lane == 0) {
            if (ok) atomicAdd(&R.rw[pr.x], v);
            else atomicOr(&R.rst[pr.x], GWN_QS_UNRESOLVED);
        }
        __syncwarp();
    }
}

// between rounds: the overflow list just written becomes the next round's
// input list, and the pair list is emptied
__global__ void k_next_round(Workspace ws) {
    if (threadIdx.x == 0) {
        ws.counters[5] = ws.counters[3];
        ws.counters[6] += ws.counters[3];
        ws.counters[7] += ws.counters[0];  // pairs of the finished round
        ws.counters[9] += ws.counters[8];  // of which the full evaluator took
        ws.counters[3] = 0;
        ws.counters[0] = 0;  // the near-band list (counters[2]) spans all rounds
        ws.counters[8] = 0;
    }
}

__global__ void k_accum(Workspace ws) {
    if (threadIdx.x < kCounterCount) ws.acc[threadIdx.x] += (unsigned long long)ws.counters[threadIdx.x];
}

// the query-wide repair pass in the totals: repaired points and FP64 pairs
__global__ void k_accum_repair(Workspace ws) {
    if (threadIdx.x == 0) {
        ws.acc[1] += (unsigned long long)min(ws.gcount[0], ws.rcap);
        ws.acc[4] += (unsigned long long)ws.gcount[1];
    }
}

// repaired values, labels and status (the FP32 status bits k_finish wrote are kept)
__global__ void k_rfinish(RepairList R, double* out_w, int* out_label, uint32_t* out_status) {
    const int cnt = min(*R.count, R.cap);
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < cnt; k += gridDim.x * blockDim.x) {
        int qi = R.idx[k];
        double w = R.rw[k];
        out_w[qi] = w;
        if (out_label) out_label[qi] = (int)round(w);
        if (out_status) out_status[qi] |= R.rst[k] | GWN_QS_REPAIRED;
    }
}

}  // namespace gwn

namespace gwn {

// ---- Warp-cooperative FP64 repair traversal.  One warp per repaired point:
// the warp keeps a node stack in shared memory and each step the lanes take up
// to 32 nodes from its top, apply the far test in FP64 and push the children
// of the nodes that fail it (positions by a warp prefix sum).  This spreads one
// point's traversal over 32 lanes, which matters because FP64 issue is slow
// and latency-bound when a single thread walks the tree.  Exact leaves: 2D in
// place (FP64), 3D appended to the FP64 pair list (k_rpairs3_warp).
constexpr int kWarpStack = 2048;
constexpr int kRepairWarps = 4;  // warps per block

template <int DIM>
__global__ void __launch_bounds__(32 * kRepairWarps) k_rtrav_warp(DevTree t, const void* pts, int dtype, double beta2r,
                                                                  RepairList R, double* out_w, int* out_label,
                                                                  uint32_t* out_status, double beta2rl = -1.0) {
    if (beta2rl < 0) beta2rl = beta2r;  // leaves' far test (3D): default the nodes' factor
    __shared__ int sstack[kRepairWarps][kWarpStack];
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int gw = blockIdx.x * kRepairWarps + wid;
    const int nw = gridDim.x * kRepairWarps;
    const int cnt = min(*R.count, R.cap);
    int* stk = sstack[wid];
    for (int k = gw; k < cnt; k += nw) {
        const int qi = R.idx[k];
        double q[3] = {0, 0, 0};
        if (dtype == GWN_F32) {
            const float* p = reinterpret_cast<const float*>(pts) + (size_t)qi * DIM;
            for (int c = 0; c < DIM; ++c) q[c] = p[c];
        } else {
            const double* p = reinterpret_cast<const double*>(pts) + (size_t)qi * DIM;
            for (int c = 0; c < DIM; ++c) q[c] = p[c];
        }
        double acc = 0.0;
        uint32_t st = 0;
        if (lane == 0) stk[0] = t.root;
        int sp = 1;
        __syncwarp();
        while (sp > 0) {
            const int take = min(sp, 32);
            const int node = lane < take ? stk[sp - 1 - lane] : 0;
            sp -= take;
            __syncwarp();
            int c0 = 0, c1 = 0, npush = 0;
            if (lane < take) {
                if (node < 0) {
                    const int li = ~node;
                    if (DIM == 2) {
                        acc += leaf2_eval64(t, li, q[0], q[1], st);
                    } else {
                        const double* h = t.lhdr64 + (size_t)li * 4;
                        double rx = h[0] - q[0], ry = h[1] - q[1], rz = h[2] - q[2];
                        if (beta2rl > 0 && t.leaf_far && rx * rx + ry * ry + rz * rz > beta2rl * h[3]) {
                            acc += far3_eval<double>(t.lmom64 + (size_t)li * kMom3F64, rx, ry, rz, t.order3_64);
                        } else {
                            int slot = atomicAdd(R.npairs, 1);
                            if (slot < kRepairPairCap) R.pairs[slot] = make_int2(k, li);
                            else acc += leaf3_eval64(t, li, q[0], q[1], q[2], st, kRatio64Repair);
                        }
                    }
                } else {
                    const double* h = t.hdr64 + (size_t)node * 4;
                    double rx = h[0] - q[0], ry = h[1] - q[1], rz = DIM == 3 ? h[2] - q[2] : 0.0;
                    double d2 = rx * rx + ry * ry + rz * rz;
                    if (beta2r > 0 && d2 > beta2r * h[3]) {
                        if (DIM == 2) acc += far2_eval<double>(t.mom64 + (size_t)node * kMom2F64, rx, ry);
                        else acc += far3_eval<double>(t.mom64 + (size_t)node * kMom3F64, rx, ry, rz, t.order3_64);
                    } else {
                        int2 ch = t.child[node];
                        c0 = ch.x;
                        c1 = ch.y;
                        npush = 2;
                    }
                }
            }
            // warp prefix sum of the pushes
            int incl = npush;
            for (int off = 1; off < 32; off <<= 1) {
                int v = __shfl_up_sync(0xffffffffu, incl, off);
                if (lane >= off) incl += v;
            }
            const int total = __shfl_sync(0xffffffffu, incl, 31);
            if (sp + total > kWarpStack) {
                st |= GWN_QS_UNRESOLVED;  // stack full: those subtrees are dropped (flagged)
            } else if (npush) {
                stk[sp + incl - 2] = c1;
                stk[sp + incl - 1] = c0;
            }
            if (sp + total <= kWarpStack) sp += total;
            __syncwarp();
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc += __shfl_xor_sync(0xffffffffu, acc, off);
            st |= __shfl_xor_sync(0xffffffffu, st, off);
        }
        if (lane == 0) {
            if (DIM == 2) {
                out_w[qi] = acc;
                if (out_label) out_label[qi] = (int)round(acc);
                if (out_status) out_status[qi] |= st | GWN_QS_REPAIRED;
            } else {
                R.rw[k] = acc;
                R.rst[k] = st;
            }
        }
        __syncwarp();
    }
}

}  // namespace gwn
