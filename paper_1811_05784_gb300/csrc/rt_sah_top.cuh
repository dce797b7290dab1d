// rt_sah_top.cuh -- surface-area-heuristic top levels over Morton cells
// (included by rt_build.cu after its BuildMeta and f2ord / ord2f).
//
// The linear BVH splits every node at the highest differing bit of its
// Morton codes, which ignores how much surface a split leaves on either
// side.  This stage keeps the LBVH below "cells" -- the sets of triangles
// whose codes share their top CELL_BITS bits -- and rebuilds the tree above
// them top-down with the surface area heuristic (MacDonald & Booth 1990;
// the binned form of Wald 2007), the hybrid of Garanzha et al. 2011 with
// cells in place of their clusters:
//   cost(split) = A(left box) N_left + A(right box) N_right,
// A the box surface area, N the triangle count of a side.
//
// Why it fits into the existing build without moving anything:
//   * the triangles of a cell are contiguous in Morton order and form one
//     subtree of the Karras hierarchy; its root has the cell's range, and
//     since a Karras node's range starts or ends at its own index, that root
//     is node a or node b of the cell [a, b] (a single-triangle cell is the
//     leaf itself);
//   * the Karras nodes whose ranges span more than one cell are exactly the
//     C - 1 internal nodes of a binary tree over the C cells.  Their indices
//     (node 0, the root, among them) are reused for the new top nodes, so the
//     arrays keep their size and the root stays node 0;
//   * a top node's (first, last) become (0, M - 1), so every top node is
//     kept as an inner node by the 4-wide collapse (a node joining two
//     single-triangle cells then becomes a small 4-wide node instead of a
//     leaf of two), and the collapse and emission work unchanged.
//
// Node ids need no counter.  In a binary tree over an ordered sequence,
// number every left child by the position of its last element, every right
// child by the position of its first, and the root 0: a left child ending at
// q and a right child starting at q would overlap without nesting, which a
// tree excludes, so this is a bijection of the C - 1 inner nodes onto
// [0, C - 2] (the numbering of Karras 2012, for any tree).  Positions are
// those of the cells after the partitions, which every segment knows.
//
// Construction, with no host synchronisation:
//   * in the first WIDE_LEVELS levels, a segment of more than WIDE_MIN cells
//     is split by the whole grid (k_wide_*, at the end of this file);
//   * SAH_LEVELS launches of k_sah_level for the others, one thread block per
//     segment of more than SAH_SMALL cells (blocks of SAH_THREADS, or of
//     SAH_MID_THREADS for segments of at most SAH_MID cells, so that the
//     many small segments of the deep levels find blocks to run on): the
//     block bins the cells' box centres
//     (SAH_BINS bins per axis over the centre bounds; counts and boxes in
//     shared memory, combined per warp first; a segment of more than
//     SAH_SAMPLE cells bins that many evenly spaced ones and counts its left
//     side afterwards), evaluates the SAH at every bin boundary of the three
//     axes, and partitions the segment stably into two (ping-pong between two
//     record arrays, so every segment keeps Morton order);
//   * one launch of k_sah_small, one warp per remaining segment: split by a
//     sweep of the SAH along the Morton order (each lane one cell; prefix and
//     suffix boxes by warp scans), or in the middle while a segment has more
//     than 32 cells or the node is SAH_MAX_DEPTH deep.
// Cells travel as 32-byte records in segment order (box, subtree root,
// triangle count), so every pass over a segment is one coalesced stream.
// Each top node writes its own entries of the binary arrays (children, parent
// links of its children, box, range).  A cell whose root is not where the
// Karras construction puts it, or counts that disagree, are reported through
// BuildMeta::sah_error and fail the build; every write checks its index.
//
// Measured on one GB300 against rt_build_tree: the theatre (436,796
// triangles) visits 15.7 instead of 19.6 nodes per query and its bounce loop
// takes 2.4 instead of 2.9 ms; the closed L-room 12.5 instead of 14.7 and
// 10.4 instead of 15.4 ms.  The build takes 1.7-2.6 ms instead of 0.3-0.8
// (one block per top-level segment: 2.0-4.2 ms): the latency of the deep
// levels' many small segments is what remains.
// With one block per top-level segment, cells of 21 bits built in 1.6-1.8 ms
// but left 16.3 and 12.6 nodes per query; cells of 27 bits took 4.8 ms for
// the theatre and left no fewer nodes than 24 bits.

#pragma once

namespace rr {

static constexpr int CELL_BITS = 24;      // 8 bits per axis: 256^3 cells
static constexpr int SAH_BINS = 16;       // per axis
static constexpr int SAH_SMALL = 32;      // segments up to this size go to the warp kernel
static constexpr int SAH_LEVELS = 14;     // block-per-segment levels
static constexpr int SAH_SAMPLE = 4096;   // larger segments bin this many evenly spaced cells
static constexpr int SAH_MAX_DEPTH = 26;  // from this depth of the top part on, only middle splits
static constexpr int SAH_THREADS = 256;   // blocks for segments of more than SAH_MID cells
static constexpr int SAH_MID = 1024;      // segments up to this size run on blocks of SAH_MID_THREADS
static constexpr int SAH_MID_THREADS = 64;
static constexpr int SAH_UNROLL = 4;      // records in flight per thread and pass
static constexpr int SAH_GRID = 1216;     // 8 blocks per SM on 152 SMs; blocks loop over segments
static constexpr int SAH_MID_GRID = 4864; // 32 blocks per SM

// a cell in segment order: box, its subtree root (lo.w), its triangle count (hi.w)
struct CellRec {
    float4 lo, hi;
};

struct SahSeg {
    uint32_t begin, end;  // cells [begin, end) of the record array `buf` (= their final positions)
    int32_t node;         // top node id (0 = root; see the numbering above)
    int16_t depth, buf;
};

// counts[0..SAH_LEVELS - 1]: segments of more than SAH_MID cells per level;
// counts[SAH_LEVELS]: segments of at most SAH_SMALL; counts_mid: the others
struct SahLists {
    SahSeg *seg_in, *seg_next, *seg_small;
    uint32_t* counts;
    CellRec *rec0, *rec1;
    SahSeg *mid_in, *mid_next;
    uint32_t* counts_mid;
};

// queues a segment of at least two cells for the next level (by its size) or the warp kernel
__device__ __forceinline__ void sah_queue(const SahLists& li, int level, bool last_level, const SahSeg& c) {
    const uint32_t m = c.end - c.begin;
    if (last_level || m <= (uint32_t)SAH_SMALL)
        li.seg_small[atomicAdd(&li.counts[SAH_LEVELS], 1u)] = c;
    else if (m > (uint32_t)SAH_MID)
        li.seg_next[atomicAdd(&li.counts[level + 1], 1u)] = c;
    else
        li.mid_next[atomicAdd(&li.counts_mid[level + 1], 1u)] = c;
}

__device__ __forceinline__ uint32_t cell_key(uint64_t code) { return (uint32_t)(code >> (48 - CELL_BITS)); }

// 1 where a new cell starts in the sorted codes
__global__ void k_cell_flags(const uint64_t* __restrict__ keys, int64_t M, uint32_t* __restrict__ flag) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    flag[j] = (j == 0 || cell_key(keys[j]) != cell_key(keys[j - 1])) ? 1u : 0u;
}

// cell_first[cid[j]] = j where flag[j] (cid the exclusive scan of flag); cell_first[C] = M
__global__ void k_cell_first(const uint32_t* __restrict__ flag, const uint32_t* __restrict__ cid, int64_t M,
                             uint32_t* __restrict__ cell_first) {
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    if (flag[j]) cell_first[cid[j]] = (uint32_t)j;
    if (j == M - 1) cell_first[cid[j] + flag[j]] = (uint32_t)M;
}

// per cell, in Morton order: its record (box, subtree root, triangle count)
__global__ void k_cell_records(const uint32_t* __restrict__ cell_first, const uint32_t* __restrict__ n_cells_p,
                               int64_t M, const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                               const float4* __restrict__ leaf_box, const float4* __restrict__ node_box,
                               CellRec* __restrict__ rec, BuildMeta* meta) {
    const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= (int64_t)*n_cells_p) return;
    const int32_t a = (int32_t)cell_first[c], b = (int32_t)cell_first[c + 1] - 1;
    int32_t ref;
    float4 lo, hi;
    if (a == b) {
        ref = ~a;
        lo = leaf_box[2 * (int64_t)a];
        hi = leaf_box[2 * (int64_t)a + 1];
    } else {
        if ((int64_t)a < M - 1 && first[a] == a && last[a] == b) {
            ref = a;
        } else if ((int64_t)b < M - 1 && first[b] == a && last[b] == b) {
            ref = b;
        } else {  // not a Karras subtree: cannot happen for a valid hierarchy
            atomicAdd(&meta->sah_error, 1u);
            ref = a < M - 1 ? a : 0;
        }
        lo = node_box[2 * (int64_t)ref];
        hi = node_box[2 * (int64_t)ref + 1];
    }
    lo.w = __int_as_float(ref);
    hi.w = __int_as_float(b - a + 1);
    rec[c].lo = lo;
    rec[c].hi = hi;
}

// 1 for the internal nodes whose range spans more than one cell
__global__ void k_top_flags(const uint64_t* __restrict__ keys, int64_t NI, const int32_t* __restrict__ first,
                            const int32_t* __restrict__ last, uint32_t* __restrict__ is_top) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NI) return;
    is_top[i] = cell_key(keys[first[i]]) != cell_key(keys[last[i]]) ? 1u : 0u;
}

// top_idx[t] = index of the t-th top node (ascending, so top_idx[0] = 0)
__global__ void k_top_compact(const uint32_t* __restrict__ is_top, const uint32_t* __restrict__ pos, int64_t NI,
                              uint32_t* __restrict__ top_idx) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NI) return;
    if (is_top[i]) top_idx[pos[i]] = (uint32_t)i;
}

__device__ __forceinline__ float box_area(float lx, float ly, float lz, float hx, float hy, float hz) {
    const float dx = hx - lx, dy = hy - ly, dz = hz - lz;
    return (dx < 0.f || dy < 0.f || dz < 0.f) ? 0.f : 2.f * (dx * dy + dy * dz + dz * dx);
}

__device__ __forceinline__ float warp_min(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// inclusive prefix (lanes <= l: box pl/ph, sums pt, pc) and suffix (lanes >= l:
// box ql/qh, sum qt) over the 32 lanes; empty lanes carry +inf / -inf boxes
__device__ __forceinline__ void warp_prefix_suffix(int lane, float* pl, float* ph, unsigned int& pt, unsigned int& pc,
                                                   float* ql, float* qh, unsigned int& qt) {
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned int ut = __shfl_up_sync(0xffffffffu, pt, o), uc = __shfl_up_sync(0xffffffffu, pc, o);
        const unsigned int dt = __shfl_down_sync(0xffffffffu, qt, o);
        float ul[3], uh[3], dl[3], dh[3];
        for (int d = 0; d < 3; d++) {
            ul[d] = __shfl_up_sync(0xffffffffu, pl[d], o), uh[d] = __shfl_up_sync(0xffffffffu, ph[d], o);
            dl[d] = __shfl_down_sync(0xffffffffu, ql[d], o), dh[d] = __shfl_down_sync(0xffffffffu, qh[d], o);
        }
        if (lane >= o) {
            pt += ut, pc += uc;
            for (int d = 0; d < 3; d++) pl[d] = fminf(pl[d], ul[d]), ph[d] = fmaxf(ph[d], uh[d]);
        }
        if (lane + o < 32) {
            qt += dt;
            for (int d = 0; d < 3; d++) ql[d] = fminf(ql[d], dl[d]), qh[d] = fmaxf(qh[d], dh[d]);
        }
    }
}

// Links the child [b, e) of the top node with binary index parent_i and
// returns its reference: a single cell is its subtree root (from its record,
// `single`), a larger side the top node numbered by its position (last cell
// of a left child, first of a right one).  Indices are checked before use.
__device__ __forceinline__ int32_t sah_link(bool is_left, uint32_t b, uint32_t e, int parent_i, int32_t single,
                                            const uint32_t* top_idx, uint32_t n_top, int64_t M, int32_t* pint,
                                            int32_t* pleaf, BuildMeta* meta) {
    int32_t ref;
    if (e - b == 1) {
        ref = single;
    } else {
        const uint32_t id = is_left ? e - 1 : b;
        if (id >= n_top) {
            atomicAdd(&meta->sah_error, 1u);
            return -1;
        }
        ref = (int32_t)top_idx[id];
    }
    if (ref >= 0 ? (int64_t)ref < M - 1 : (int64_t)~ref < M) {
        if (ref >= 0)
            pint[ref] = parent_i;
        else
            pleaf[~ref] = parent_i;
    } else {  // cannot happen for consistent records: reported, not written
        atomicAdd(&meta->sah_error, 1u);
    }
    return ref;
}

__device__ __forceinline__ int sah_bin(float c, float lo, float scale) {
    return min(SAH_BINS - 1, max(0, (int)((c - lo) * scale)));
}

// shared-memory state of one block's binned SAH
struct SahBins {
    unsigned int lo[3][SAH_BINS][3], hi[3][SAH_BINS][3];  // bin boxes, order-preserving bits
    unsigned int tri[3][SAH_BINS], cel[3][SAH_BINS];
    float cost[3];
    int split[3];
    unsigned int nl[3];
};

// Bins the centres of the cells [begin, begin + n) of rin -- an even sample of
// SAH_SAMPLE of them when n is larger -- and picks the SAH split: the axis (-1
// when every centre is equal), the last bin of the left side, and the left
// side's cell count (exact when nothing was sampled).  Every thread of a block
// of T threads calls it with the same centre bounds (clo, ext, scale).
template <int T>
__device__ __forceinline__ void sah_choose(SahBins& sb, const CellRec* __restrict__ rin, uint32_t begin, uint32_t n,
                                           const float* clo, const float* ext, const float* scale, int& axis,
                                           int& split, uint32_t& nl) {
    constexpr int U = SAH_UNROLL;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int t = tid; t < 3 * SAH_BINS; t += T) {  // empty bins
        const int k = t / SAH_BINS, b = t % SAH_BINS;
        sb.tri[k][b] = sb.cel[k][b] = 0u;
        for (int d = 0; d < 3; d++) sb.lo[k][b][d] = f2ord(INFINITY), sb.hi[k][b][d] = f2ord(-INFINITY);
    }
    __syncthreads();
    // bins of the three axes (triangles for the cost, cells for the
    // partition).  Cells in Morton order are neighbours, so a warp's cells
    // mostly share bins: the lanes of one bin combine their values first
    // and one of them updates the bin.
    const bool sampled = n > (uint32_t)SAH_SAMPLE;
    const uint32_t nb = sampled ? (uint32_t)SAH_SAMPLE : n;
    for (uint32_t i0 = tid; i0 < nb + (uint32_t)tid; i0 += T * U) {
        float4 lo[U], hi[U];
#pragma unroll
        for (int u = 0; u < U; u++) {
            const uint32_t i = i0 + u * T;
            const uint32_t k = begin + (sampled ? (uint32_t)(((uint64_t)i * n) / SAH_SAMPLE) : i);
            if (i < nb) lo[u] = rin[k].lo, hi[u] = rin[k].hi;
        }
#pragma unroll
        for (int u = 0; u < U; u++) {
            const bool inr = i0 + u * T < nb;
            const unsigned int act = __ballot_sync(0xffffffffu, inr);
            if (!inr) continue;
            const float cen[3] = {0.5f * (lo[u].x + hi[u].x), 0.5f * (lo[u].y + hi[u].y),
                                  0.5f * (lo[u].z + hi[u].z)};
            const unsigned int nt = (unsigned int)__float_as_int(hi[u].w);
            const unsigned int o[6] = {f2ord(lo[u].x), f2ord(lo[u].y), f2ord(lo[u].z),
                                       f2ord(hi[u].x), f2ord(hi[u].y), f2ord(hi[u].z)};
            for (int a = 0; a < 3; a++) {
                if (!(ext[a] > 0.f)) continue;  // the same for every lane
                const int b = sah_bin(cen[a], clo[a], scale[a]);
                const unsigned int grp = __match_any_sync(act, b);
                const unsigned int tsum = __reduce_add_sync(grp, nt);
                unsigned int r[6];
                for (int d = 0; d < 3; d++)
                    r[d] = __reduce_min_sync(grp, o[d]), r[3 + d] = __reduce_max_sync(grp, o[3 + d]);
                if (lane == __ffs(grp) - 1) {
                    atomicAdd(&sb.tri[a][b], tsum);
                    atomicAdd(&sb.cel[a][b], (unsigned int)__popc(grp));
                    for (int d = 0; d < 3; d++) atomicMin(&sb.lo[a][b][d], r[d]), atomicMax(&sb.hi[a][b][d], r[3 + d]);
                }
            }
        }
    }
    __syncthreads();
    // SAH at the bin boundaries: a warp evaluates an axis, lane l the boundary after bin l
    for (int a = warp; a < 3; a += T / 32) {
        const bool in = lane < SAH_BINS && ext[a] > 0.f;
        float pl[3], ph[3], ql[3], qh[3];
        unsigned int pt = 0u, pc = 0u, qt = 0u;
        for (int d = 0; d < 3; d++) {
            pl[d] = in ? ord2f(sb.lo[a][lane][d]) : INFINITY;
            ph[d] = in ? ord2f(sb.hi[a][lane][d]) : -INFINITY;
            ql[d] = pl[d];
            qh[d] = ph[d];
        }
        if (in) pt = qt = sb.tri[a][lane], pc = sb.cel[a][lane];
        warp_prefix_suffix(lane, pl, ph, pt, pc, ql, qh, qt);
        // the right side of boundary l is the suffix from bin l + 1
        const unsigned int rt = __shfl_down_sync(0xffffffffu, qt, 1);
        float rl[3], rh[3];
        for (int d = 0; d < 3; d++)
            rl[d] = __shfl_down_sync(0xffffffffu, ql[d], 1), rh[d] = __shfl_down_sync(0xffffffffu, qh[d], 1);
        float cost = INFINITY;
        if (in && lane < SAH_BINS - 1 && pt > 0u && rt > 0u)
            cost = box_area(pl[0], pl[1], pl[2], ph[0], ph[1], ph[2]) * (float)pt +
                   box_area(rl[0], rl[1], rl[2], rh[0], rh[1], rh[2]) * (float)rt;
        const float best = warp_min(cost);
        const unsigned int at = __ballot_sync(0xffffffffu, cost == best && best < INFINITY);
        const int bl = at ? __ffs(at) - 1 : -1;
        const unsigned int left_cells = __shfl_sync(0xffffffffu, pc, bl < 0 ? 0 : bl);
        if (lane == 0) {
            sb.cost[a] = bl < 0 ? INFINITY : best;
            sb.split[a] = bl;
            sb.nl[a] = left_cells;
        }
    }
    __syncthreads();
    axis = -1;
    float bc = INFINITY;
    for (int a = 0; a < 3; a++)
        if (sb.split[a] >= 0 && sb.cost[a] < bc) bc = sb.cost[a], axis = a;
    split = axis < 0 ? 0 : sb.split[axis];
    nl = axis < 0 ? n / 2 : sb.nl[axis];  // all centres equal: split in the middle
}

// one level: one block per segment (T threads: segments of more than SAH_MID
// cells, or of SAH_SMALL + 1 to SAH_MID cells when MID)
template <int T, bool MID>
__global__ void __launch_bounds__(T)
    k_sah_level(int level, bool last_level, SahLists li, const uint32_t* __restrict__ top_idx,
                const uint32_t* __restrict__ n_top_p, int64_t M, int32_t* __restrict__ left,
                int32_t* __restrict__ right, int32_t* __restrict__ first, int32_t* __restrict__ last,
                int32_t* __restrict__ pint, int32_t* __restrict__ pleaf, float4* __restrict__ node_box,
                BuildMeta* meta) {
    constexpr int NW = T / 32, U = SAH_UNROLL;
    __shared__ SahBins sb;
    __shared__ float s_red[NW][12];
    __shared__ float s_b[12];  // node box lo, hi; centre bounds lo, hi
    __shared__ unsigned int s_wl[U][NW], s_wr[U][NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n_seg = MID ? li.counts_mid[level] : li.counts[level];
    const SahSeg* seg_in = MID ? li.mid_in : li.seg_in;
    const uint32_t n_top = *n_top_p;
    for (uint32_t si = blockIdx.x; si < n_seg; si += gridDim.x) {
        const SahSeg sg = seg_in[si];
        const CellRec* rin = sg.buf ? li.rec1 : li.rec0;
        CellRec* rout = sg.buf ? li.rec0 : li.rec1;
        const uint32_t n = sg.end - sg.begin;
        const int parent_i = (int)top_idx[sg.node];
        // pass 1: the node's box and the bounds of the cell centres
        float v[12];
        for (int k = 0; k < 3; k++) v[k] = v[6 + k] = INFINITY, v[3 + k] = v[9 + k] = -INFINITY;
        for (uint32_t k0 = sg.begin + tid; k0 < sg.end; k0 += T * U) {
            float4 lo[U], hi[U];
#pragma unroll
            for (int u = 0; u < U; u++)
                if (k0 + u * T < sg.end) lo[u] = rin[k0 + u * T].lo, hi[u] = rin[k0 + u * T].hi;
#pragma unroll
            for (int u = 0; u < U; u++) {
                if (k0 + u * T >= sg.end) break;
                const float cx = 0.5f * (lo[u].x + hi[u].x), cy = 0.5f * (lo[u].y + hi[u].y),
                            cz = 0.5f * (lo[u].z + hi[u].z);
                v[0] = fminf(v[0], lo[u].x), v[1] = fminf(v[1], lo[u].y), v[2] = fminf(v[2], lo[u].z);
                v[3] = fmaxf(v[3], hi[u].x), v[4] = fmaxf(v[4], hi[u].y), v[5] = fmaxf(v[5], hi[u].z);
                v[6] = fminf(v[6], cx), v[7] = fminf(v[7], cy), v[8] = fminf(v[8], cz);
                v[9] = fmaxf(v[9], cx), v[10] = fmaxf(v[10], cy), v[11] = fmaxf(v[11], cz);
            }
        }
        for (int k = 0; k < 12; k++) v[k] = (k % 6) < 3 ? warp_min(v[k]) : warp_max(v[k]);
        if (lane == 0)
            for (int k = 0; k < 12; k++) s_red[warp][k] = v[k];
        __syncthreads();
        if (tid < 12) {
            float r = s_red[0][tid];
            for (int w = 1; w < NW; w++) r = (tid % 6) < 3 ? fminf(r, s_red[w][tid]) : fmaxf(r, s_red[w][tid]);
            s_b[tid] = r;
        }
        __syncthreads();
        float clo[3], ext[3], scale[3];
        for (int k = 0; k < 3; k++) {
            clo[k] = s_b[6 + k];
            ext[k] = s_b[9 + k] - s_b[6 + k];
            scale[k] = ext[k] > 0.f ? (float)SAH_BINS / ext[k] : 0.f;
        }
        if (tid == 0) {
            node_box[2 * (int64_t)parent_i] = make_float4(s_b[0], s_b[1], s_b[2], 0.f);
            node_box[2 * (int64_t)parent_i + 1] = make_float4(s_b[3], s_b[4], s_b[5], 0.f);
            first[parent_i] = 0;  // kept by the 4-wide collapse
            last[parent_i] = (int32_t)(M - 1);
        }
        const bool sampled = n > (uint32_t)SAH_SAMPLE;
        int axis, split;
        uint32_t nL;
        sah_choose<T>(sb, rin, sg.begin, n, clo, ext, scale, axis, split, nL);
        const float alo = axis < 0 ? 0.f : clo[axis], asc = axis < 0 ? 0.f : scale[axis];
        // the left side's cells: from the bins, or counted when they held a sample
        if (sampled && axis >= 0) {
            uint32_t cnt = 0;
            for (uint32_t k0 = sg.begin + tid; k0 < sg.end; k0 += T * U) {
                float4 lo[U], hi[U];
#pragma unroll
                for (int u = 0; u < U; u++)
                    if (k0 + u * T < sg.end) lo[u] = rin[k0 + u * T].lo, hi[u] = rin[k0 + u * T].hi;
#pragma unroll
                for (int u = 0; u < U; u++) {
                    if (k0 + u * T >= sg.end) break;
                    const float cen = axis == 0 ? 0.5f * (lo[u].x + hi[u].x)
                                                : (axis == 1 ? 0.5f * (lo[u].y + hi[u].y) : 0.5f * (lo[u].z + hi[u].z));
                    cnt += sah_bin(cen, alo, asc) <= split ? 1u : 0u;
                }
            }
            cnt = __reduce_add_sync(0xffffffffu, cnt);
            if (lane == 0) s_wl[0][warp] = cnt;
            __syncthreads();
            nL = 0;
            for (int w = 0; w < NW; w++) nL += s_wl[0][w];
            __syncthreads();
        }
        // pass 3: stable partition into the other record array, U chunks of T cells per round
        uint32_t lbase = 0, rbase = 0;
        for (uint32_t k0 = sg.begin; k0 < sg.end; k0 += T * U) {
            CellRec r[U];
            bool pred[U], isr[U];
#pragma unroll
            for (int u = 0; u < U; u++) {
                const uint32_t k = k0 + u * T + tid;
                const bool inr = k < sg.end;
                if (inr) r[u].lo = rin[k].lo, r[u].hi = rin[k].hi;
                bool p = false;
                if (inr) {
                    if (axis < 0) {
                        p = k - sg.begin < nL;
                    } else {
                        const float cen = axis == 0 ? 0.5f * (r[u].lo.x + r[u].hi.x)
                                                    : (axis == 1 ? 0.5f * (r[u].lo.y + r[u].hi.y)
                                                                 : 0.5f * (r[u].lo.z + r[u].hi.z));
                        p = sah_bin(cen, alo, asc) <= split;
                    }
                }
                pred[u] = p;
                isr[u] = inr && !p;
                const unsigned int wl = __ballot_sync(0xffffffffu, pred[u]), wr = __ballot_sync(0xffffffffu, isr[u]);
                if (lane == 0) s_wl[u][warp] = __popc(wl), s_wr[u][warp] = __popc(wr);
            }
            __syncthreads();
            const unsigned int below = (1u << lane) - 1u;
#pragma unroll
            for (int u = 0; u < U; u++) {
                uint32_t offl = 0, offr = 0, totl = 0, totr = 0;
                for (int w = 0; w < NW; w++) {
                    if (w < warp) offl += s_wl[u][w], offr += s_wr[u][w];
                    totl += s_wl[u][w], totr += s_wr[u][w];
                }
                const unsigned int wl = __ballot_sync(0xffffffffu, pred[u]), wr = __ballot_sync(0xffffffffu, isr[u]);
                // each side stays inside its part of the segment even if the
                // counts disagreed (reported below)
                const uint32_t dl = sg.begin + lbase + offl + __popc(wl & below);
                const uint32_t dr = sg.begin + nL + rbase + offr + __popc(wr & below);
                if (pred[u] && dl < sg.begin + nL) rout[dl] = r[u];
                if (isr[u] && dr < sg.end) rout[dr] = r[u];
                lbase += totl;
                rbase += totr;
            }
            __syncthreads();
        }
        if (tid == 0) {
            const bool bad = lbase != nL || lbase + rbase != n || nL == 0 || nL == n;
            if (bad) {
                atomicAdd(&meta->sah_error, 1u);
            } else {
                const int32_t sl = __float_as_int(rout[sg.begin].lo.w), sr = __float_as_int(rout[sg.begin + nL].lo.w);
                left[parent_i] = sah_link(true, sg.begin, sg.begin + nL, parent_i, sl, top_idx, n_top, M, pint, pleaf,
                                          meta);
                right[parent_i] = sah_link(false, sg.begin + nL, sg.end, parent_i, sr, top_idx, n_top, M, pint, pleaf,
                                           meta);
                SahSeg c;
                c.depth = (int16_t)(sg.depth + 1);
                c.buf = (int16_t)(1 - sg.buf);
                for (int side = 0; side < 2; side++) {
                    c.begin = side ? sg.begin + nL : sg.begin;
                    c.end = side ? sg.end : sg.begin + nL;
                    if (c.end - c.begin < 2) continue;  // a single cell: linked above
                    c.node = (int32_t)(side ? c.begin : c.end - 1);
                    if ((uint32_t)c.node >= n_top) continue;  // reported by sah_link
                    sah_queue(li, level, last_level, c);
                }
            }
        }
        __syncthreads();
    }
}

// a segment of at most 32 cells, one per lane, loaded once: every node of its
// subtree is a range of lanes [lb, le), split by the SAH along the Morton
// order (or in the middle from SAH_MAX_DEPTH on); the stack of lane ranges
// (with node ids, fixed when their parent split) is alike in every lane, the
// smaller child on top
__device__ __forceinline__ void sah_lanes(const SahSeg& root, int lane, const CellRec* __restrict__ rec,
                                          const uint32_t* __restrict__ top_idx, uint32_t n_top, int64_t M,
                                          int32_t* left, int32_t* right, int32_t* first, int32_t* last, int32_t* pint,
                                          int32_t* pleaf, float4* node_box, BuildMeta* meta) {
    const int n = (int)(root.end - root.begin);
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    unsigned int nt = 0u;
    int32_t w = 0;
    if (lane < n) {
        const float4 l4 = rec[root.begin + lane].lo, h4 = rec[root.begin + lane].hi;
        lo[0] = l4.x, lo[1] = l4.y, lo[2] = l4.z, hi[0] = h4.x, hi[1] = h4.y, hi[2] = h4.z;
        w = __float_as_int(l4.w);
        nt = (unsigned int)__float_as_int(h4.w);
    }
    int sb[32], se[32], sd[32], sn[32];
    int sp = 1;
    sb[0] = 0, se[0] = n, sd[0] = root.depth, sn[0] = root.node;
    for (int it = 0; sp > 0 && it < n; it++) {
        --sp;
        const int lb = sb[sp], le = se[sp], dep = sd[sp], id = sn[sp];
        const int pi = (int)top_idx[id];
        const bool in = lane >= lb && lane < le;
        float bl[3], bh[3];
        for (int d = 0; d < 3; d++) bl[d] = warp_min(in ? lo[d] : INFINITY), bh[d] = warp_max(in ? hi[d] : -INFINITY);
        if (lane == 0) {
            node_box[2 * (int64_t)pi] = make_float4(bl[0], bl[1], bl[2], 0.f);
            node_box[2 * (int64_t)pi + 1] = make_float4(bh[0], bh[1], bh[2], 0.f);
            first[pi] = 0;  // kept by the 4-wide collapse
            last[pi] = (int32_t)(M - 1);
        }
        int m = lb + (le - lb) / 2;
        if (dep < SAH_MAX_DEPTH) {
            float pl[3], ph[3], ql[3], qh[3];
            for (int d = 0; d < 3; d++) {
                pl[d] = ql[d] = in ? lo[d] : INFINITY;
                ph[d] = qh[d] = in ? hi[d] : -INFINITY;
            }
            unsigned int pt = in ? nt : 0u, qt = pt, pc = 0u;
            warp_prefix_suffix(lane, pl, ph, pt, pc, ql, qh, qt);
            const unsigned int rt = __shfl_down_sync(0xffffffffu, qt, 1);
            float rl[3], rh[3];
            for (int d = 0; d < 3; d++)
                rl[d] = __shfl_down_sync(0xffffffffu, ql[d], 1), rh[d] = __shfl_down_sync(0xffffffffu, qh[d], 1);
            const bool cand = in && lane + 1 < le;
            const float cost = cand ? box_area(pl[0], pl[1], pl[2], ph[0], ph[1], ph[2]) * (float)pt +
                                          box_area(rl[0], rl[1], rl[2], rh[0], rh[1], rh[2]) * (float)rt
                                    : INFINITY;
            const float best = warp_min(cost);
            const unsigned int at = __ballot_sync(0xffffffffu, cand && cost == best);
            if (at) m = __ffs(at);  // split after the lowest best lane
        }
        // children [lb, m) and [m, le); ids by position (alike in every lane)
        const int32_t wl = __shfl_sync(0xffffffffu, w, lb & 31), wr = __shfl_sync(0xffffffffu, w, m & 31);
        const uint32_t idl = root.begin + (uint32_t)m - 1u, idr = root.begin + (uint32_t)m;
        const bool morel = m - lb >= 2, morer = le - m >= 2;
        if ((morel && idl >= n_top) || (morer && idr >= n_top) || sp + 2 > 32) {
            if (lane == 0) atomicAdd(&meta->sah_error, 1u);
            return;
        }
        if (lane == 0) {
            left[pi] = sah_link(true, root.begin + lb, root.begin + m, pi, wl, top_idx, n_top, M, pint, pleaf, meta);
            right[pi] = sah_link(false, root.begin + m, root.begin + le, pi, wr, top_idx, n_top, M, pint, pleaf, meta);
        }
        const bool left_larger = m - lb >= le - m;
        if (morel && morer) {
            if (left_larger) {
                sb[sp] = lb, se[sp] = m, sd[sp] = dep + 1, sn[sp] = (int)idl, sp++;
                sb[sp] = m, se[sp] = le, sd[sp] = dep + 1, sn[sp] = (int)idr, sp++;
            } else {
                sb[sp] = m, se[sp] = le, sd[sp] = dep + 1, sn[sp] = (int)idr, sp++;
                sb[sp] = lb, se[sp] = m, sd[sp] = dep + 1, sn[sp] = (int)idl, sp++;
            }
        } else if (morel) {
            sb[sp] = lb, se[sp] = m, sd[sp] = dep + 1, sn[sp] = (int)idl, sp++;
        } else if (morer) {
            sb[sp] = m, se[sp] = le, sd[sp] = dep + 1, sn[sp] = (int)idr, sp++;
        }
    }
    if (sp > 0 && lane == 0) atomicAdd(&meta->sah_error, 1u);  // iteration bound reached
}

// the rest of the top part: one warp per queued segment.  Segments of at
// most 32 cells go through sah_lanes; longer ones (left over after the last
// block level) are split in the middle until their parts are that short.
__global__ void __launch_bounds__(256)
    k_sah_small(SahLists li, const uint32_t* __restrict__ top_idx, const uint32_t* __restrict__ n_top_p, int64_t M,
                int32_t* __restrict__ left, int32_t* __restrict__ right, int32_t* __restrict__ first,
                int32_t* __restrict__ last, int32_t* __restrict__ pint, int32_t* __restrict__ pleaf,
                float4* __restrict__ node_box, BuildMeta* meta) {
    const int lane = threadIdx.x & 31;
    const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t n_small = li.counts[SAH_LEVELS];
    const uint32_t n_top = *n_top_p;
    for (int64_t si = wid; si < (int64_t)n_small; si += nw) {
        const SahSeg root = li.seg_small[si];
        const CellRec* rec = root.buf ? li.rec1 : li.rec0;
        SahSeg stack[32];
        int sp = 0;
        stack[sp++] = root;
        for (uint32_t it = 0; sp > 0 && it < root.end - root.begin; it++) {
            const SahSeg g = stack[--sp];
            const uint32_t n = g.end - g.begin;
            if (n <= 32u) {
                sah_lanes(g, lane, rec, top_idx, n_top, M, left, right, first, last, pint, pleaf, node_box, meta);
                continue;
            }
            const int pi = (int)top_idx[g.node];
            const uint32_t m = g.begin + n / 2;
            float bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
            for (uint32_t k = g.begin + lane; k < g.end; k += 32) {
                const float4 lo = rec[k].lo, hi = rec[k].hi;
                bl[0] = fminf(bl[0], lo.x), bl[1] = fminf(bl[1], lo.y), bl[2] = fminf(bl[2], lo.z);
                bh[0] = fmaxf(bh[0], hi.x), bh[1] = fmaxf(bh[1], hi.y), bh[2] = fmaxf(bh[2], hi.z);
            }
            for (int d = 0; d < 3; d++) bl[d] = warp_min(bl[d]), bh[d] = warp_max(bh[d]);
            if (sp + 2 > 32 || m >= n_top) {
                if (lane == 0) atomicAdd(&meta->sah_error, 1u);
                break;
            }
            if (lane == 0) {
                node_box[2 * (int64_t)pi] = make_float4(bl[0], bl[1], bl[2], 0.f);
                node_box[2 * (int64_t)pi + 1] = make_float4(bh[0], bh[1], bh[2], 0.f);
                first[pi] = 0;
                last[pi] = (int32_t)(M - 1);
                // both halves hold more than 16 cells: two top nodes
                left[pi] = sah_link(true, g.begin, m, pi, 0, top_idx, n_top, M, pint, pleaf, meta);
                right[pi] = sah_link(false, m, g.end, pi, 0, top_idx, n_top, M, pint, pleaf, meta);
            }
            SahSeg L, R;
            L.begin = g.begin, L.end = m, L.node = (int32_t)(m - 1u);
            R.begin = m, R.end = g.end, R.node = (int32_t)m;
            L.depth = R.depth = (int16_t)(g.depth + 1);
            L.buf = R.buf = g.buf;
            stack[sp++] = R;  // equal halves up to one cell
            stack[sp++] = L;
        }
        if (sp > 0 && lane == 0) atomicAdd(&meta->sah_error, 1u);  // iteration bound reached
    }
}

// ---------------------------------------------------------------------------
// Wide segments.  The first levels hold few segments of many cells, which one
// block each would stream through one SM.  A segment of more than WIDE_MIN
// cells in the first WIDE_LEVELS levels is split by the whole grid instead,
// in chunks of WIDE_CHUNK cells: its bounds (ordered atomics per segment),
// its split (one block per segment, on the sample sah_choose takes), the
// left count of every chunk, a stable scatter whose offsets sum the counts of
// the segment's earlier chunks, and its children (one thread per segment).
// ---------------------------------------------------------------------------
static constexpr int WIDE_MIN = 16384;
static constexpr int WIDE_LEVELS = 5;
static constexpr int WIDE_CHUNK = 4096;
static constexpr int WIDE_THREADS = 256;

struct SahWide {
    SahSeg *in, *next;          // this level's wide segments, the next level's
    uint32_t* counts;           // [WIDE_LEVELS + 1] wide segments per level
    unsigned int *bin, *bnext;  // [cap][12] bounds of this level's and of the next level's segments:
                                // box lo, box hi, centre lo, centre hi (order-preserving bits)
    int4* split;                // [cap] axis, split bin, centre lo on the axis, bin scale (float bits)
    uint32_t* chunk_left;       // [chunks] left cells of every chunk of this level
    uint32_t cap;               // entries of in, next, bin, bnext, split
};

__device__ __forceinline__ void wide_bounds_init(unsigned int* b) {
    for (int k = 0; k < 12; k++) b[k] = (k % 6) < 3 ? f2ord(INFINITY) : f2ord(-INFINITY);
}

// the wide segment holding global chunk g, the index of its first chunk and
// the chunk's first cell; false past the last chunk of the level
__device__ __forceinline__ bool wide_chunk(const SahSeg* in, uint32_t n_wide, uint32_t g, uint32_t& s,
                                           uint32_t& first_chunk, uint32_t& c0) {
    uint32_t acc = 0;
    for (uint32_t k = 0; k < n_wide; k++) {
        const uint32_t nch = (in[k].end - in[k].begin + WIDE_CHUNK - 1) / WIDE_CHUNK;
        if (g < acc + nch) {
            s = k;
            first_chunk = acc;
            c0 = in[k].begin + (g - acc) * WIDE_CHUNK;
            return true;
        }
        acc += nch;
    }
    return false;
}

// the side a cell goes to: by its centre's bin, or by position when every centre is equal
__device__ __forceinline__ bool wide_left(const int4& sp, const CellRec& r, uint32_t k, const SahSeg& sg) {
    if (sp.x < 0) return k - sg.begin < (sg.end - sg.begin) / 2;
    const float cen = sp.x == 0 ? 0.5f * (r.lo.x + r.hi.x) : (sp.x == 1 ? 0.5f * (r.lo.y + r.hi.y) : 0.5f * (r.lo.z + r.hi.z));
    return sah_bin(cen, __int_as_float(sp.z), __int_as_float(sp.w)) <= sp.y;
}

// bounds of every wide segment, one block per chunk
__global__ void __launch_bounds__(WIDE_THREADS)
    k_wide_bounds(int level, SahWide w, const CellRec* __restrict__ rec0, const CellRec* __restrict__ rec1) {
    constexpr int NW = WIDE_THREADS / 32;
    __shared__ float s_red[NW][12];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n_wide = w.counts[level];
    for (uint32_t g = blockIdx.x;; g += gridDim.x) {
        uint32_t s, fc, c0;
        if (!wide_chunk(w.in, n_wide, g, s, fc, c0)) break;  // the same for the whole block
        const SahSeg sg = w.in[s];
        const CellRec* rin = sg.buf ? rec1 : rec0;
        const uint32_t c1 = min(c0 + (uint32_t)WIDE_CHUNK, sg.end);
        float v[12];
        for (int k = 0; k < 3; k++) v[k] = v[6 + k] = INFINITY, v[3 + k] = v[9 + k] = -INFINITY;
        for (uint32_t k = c0 + tid; k < c1; k += WIDE_THREADS) {
            const float4 lo = rin[k].lo, hi = rin[k].hi;
            const float cx = 0.5f * (lo.x + hi.x), cy = 0.5f * (lo.y + hi.y), cz = 0.5f * (lo.z + hi.z);
            v[0] = fminf(v[0], lo.x), v[1] = fminf(v[1], lo.y), v[2] = fminf(v[2], lo.z);
            v[3] = fmaxf(v[3], hi.x), v[4] = fmaxf(v[4], hi.y), v[5] = fmaxf(v[5], hi.z);
            v[6] = fminf(v[6], cx), v[7] = fminf(v[7], cy), v[8] = fminf(v[8], cz);
            v[9] = fmaxf(v[9], cx), v[10] = fmaxf(v[10], cy), v[11] = fmaxf(v[11], cz);
        }
        for (int k = 0; k < 12; k++) v[k] = (k % 6) < 3 ? warp_min(v[k]) : warp_max(v[k]);
        if (lane == 0)
            for (int k = 0; k < 12; k++) s_red[warp][k] = v[k];
        __syncthreads();
        if (tid < 12) {
            float r = s_red[0][tid];
            for (int q = 1; q < NW; q++) r = (tid % 6) < 3 ? fminf(r, s_red[q][tid]) : fmaxf(r, s_red[q][tid]);
            if ((tid % 6) < 3)
                atomicMin(&w.bin[12 * s + tid], f2ord(r));
            else
                atomicMax(&w.bin[12 * s + tid], f2ord(r));
        }
        __syncthreads();
    }
}

// the split of every wide segment, one block per segment (its SAH_SAMPLE
// samples in one round of loads); writes the node's box
static constexpr int WIDE_DECIDE_THREADS = 1024;
__global__ void __launch_bounds__(WIDE_DECIDE_THREADS)
    k_wide_decide(int level, SahWide w, const CellRec* __restrict__ rec0, const CellRec* __restrict__ rec1,
                  const uint32_t* __restrict__ top_idx, int64_t M, int32_t* __restrict__ first,
                  int32_t* __restrict__ last, float4* __restrict__ node_box) {
    __shared__ SahBins sb;
    const uint32_t n_wide = w.counts[level];
    for (uint32_t si = blockIdx.x; si < n_wide; si += gridDim.x) {
        const SahSeg sg = w.in[si];
        const CellRec* rin = sg.buf ? rec1 : rec0;
        const unsigned int* b = w.bin + 12 * si;
        float clo[3], ext[3], scale[3];
        for (int k = 0; k < 3; k++) {
            clo[k] = ord2f(b[6 + k]);
            ext[k] = ord2f(b[9 + k]) - clo[k];
            scale[k] = ext[k] > 0.f ? (float)SAH_BINS / ext[k] : 0.f;
        }
        const int pi = (int)top_idx[sg.node];
        if (threadIdx.x == 0) {
            node_box[2 * (int64_t)pi] = make_float4(ord2f(b[0]), ord2f(b[1]), ord2f(b[2]), 0.f);
            node_box[2 * (int64_t)pi + 1] = make_float4(ord2f(b[3]), ord2f(b[4]), ord2f(b[5]), 0.f);
            first[pi] = 0;  // kept by the 4-wide collapse
            last[pi] = (int32_t)(M - 1);
        }
        int axis, split;
        uint32_t nl;
        sah_choose<WIDE_DECIDE_THREADS>(sb, rin, sg.begin, sg.end - sg.begin, clo, ext, scale, axis, split, nl);
        if (threadIdx.x == 0)
            w.split[si] = make_int4(axis, split, __float_as_int(axis < 0 ? 0.f : clo[axis]),
                                    __float_as_int(axis < 0 ? 0.f : scale[axis]));
        __syncthreads();
    }
}

// the left cells of every chunk
__global__ void __launch_bounds__(WIDE_THREADS)
    k_wide_count(int level, SahWide w, const CellRec* __restrict__ rec0, const CellRec* __restrict__ rec1) {
    constexpr int NW = WIDE_THREADS / 32;
    __shared__ uint32_t s_cnt[NW];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n_wide = w.counts[level];
    for (uint32_t g = blockIdx.x;; g += gridDim.x) {
        uint32_t s, fc, c0;
        if (!wide_chunk(w.in, n_wide, g, s, fc, c0)) break;
        const SahSeg sg = w.in[s];
        const CellRec* rin = sg.buf ? rec1 : rec0;
        const int4 sp = w.split[s];
        const uint32_t c1 = min(c0 + (uint32_t)WIDE_CHUNK, sg.end);
        uint32_t cnt = 0;
        for (uint32_t k = c0 + tid; k < c1; k += WIDE_THREADS) {
            const CellRec r = rin[k];
            cnt += wide_left(sp, r, k, sg) ? 1u : 0u;
        }
        cnt = __reduce_add_sync(0xffffffffu, cnt);
        if (lane == 0) s_cnt[warp] = cnt;
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
            for (int q = 0; q < NW; q++) t += s_cnt[q];
            w.chunk_left[g] = t;
        }
        __syncthreads();
    }
}

// stable partition of every wide segment into the other record array, one
// block per chunk: its left cells follow the left cells of the segment's
// earlier chunks, its right cells those of their right cells
__global__ void __launch_bounds__(WIDE_THREADS)
    k_wide_scatter(int level, SahWide w, CellRec* __restrict__ rec0, CellRec* __restrict__ rec1, BuildMeta* meta) {
    constexpr int NW = WIDE_THREADS / 32;
    __shared__ uint32_t s_wl[NW], s_wr[NW];
    __shared__ uint32_t s_base[2];  // left cells of the earlier chunks, of the whole segment
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t n_wide = w.counts[level];
    for (uint32_t g = blockIdx.x;; g += gridDim.x) {
        uint32_t s, fc, c0;
        if (!wide_chunk(w.in, n_wide, g, s, fc, c0)) break;
        const SahSeg sg = w.in[s];
        const CellRec* rin = sg.buf ? rec1 : rec0;
        CellRec* rout = sg.buf ? rec0 : rec1;
        const int4 sp = w.split[s];
        const uint32_t c1 = min(c0 + (uint32_t)WIDE_CHUNK, sg.end);
        if (tid == 0) {
            const uint32_t nch = (sg.end - sg.begin + WIDE_CHUNK - 1) / WIDE_CHUNK;
            uint32_t before = 0, total = 0;
            for (uint32_t j = 0; j < nch; j++) {
                const uint32_t c = w.chunk_left[fc + j];
                if (fc + j < g) before += c;
                total += c;
            }
            s_base[0] = before;
            s_base[1] = total;
        }
        __syncthreads();
        const uint32_t nL = s_base[1];
        uint32_t lb = sg.begin + s_base[0];                        // next left slot
        uint32_t rb = sg.begin + nL + (c0 - sg.begin) - s_base[0];  // next right slot
        for (uint32_t r0 = c0; r0 < c1; r0 += WIDE_THREADS) {
            const uint32_t k = r0 + tid;
            const bool inr = k < c1;
            CellRec r;
            bool p = false;
            if (inr) {
                r = rin[k];
                p = wide_left(sp, r, k, sg);
            }
            const bool q = inr && !p;
            const unsigned int wl = __ballot_sync(0xffffffffu, p), wr = __ballot_sync(0xffffffffu, q);
            if (lane == 0) s_wl[warp] = __popc(wl), s_wr[warp] = __popc(wr);
            __syncthreads();
            uint32_t offl = 0, offr = 0, totl = 0, totr = 0;
            for (int x = 0; x < NW; x++) {
                if (x < warp) offl += s_wl[x], offr += s_wr[x];
                totl += s_wl[x], totr += s_wr[x];
            }
            const unsigned int below = (1u << lane) - 1u;
            const uint32_t dl = lb + offl + __popc(wl & below), dr = rb + offr + __popc(wr & below);
            // each side stays inside its part of the segment even if a count disagreed
            if (p) {
                if (dl < sg.begin + nL)
                    rout[dl] = r;
                else
                    atomicAdd(&meta->sah_error, 1u);
            }
            if (q) {
                if (dr >= sg.begin + nL && dr < sg.end)
                    rout[dr] = r;
                else
                    atomicAdd(&meta->sah_error, 1u);
            }
            lb += totl;
            rb += totr;
            __syncthreads();
        }
    }
}

// the children of every wide segment, one thread per segment: links, and the
// queues of the next level (wide or not) or of the warp kernel
__global__ void k_wide_children(int level, SahWide w, SahLists li, const uint32_t* __restrict__ top_idx,
                                const uint32_t* __restrict__ n_top_p, int64_t M, int32_t* __restrict__ left,
                                int32_t* __restrict__ right, int32_t* __restrict__ pint, int32_t* __restrict__ pleaf,
                                BuildMeta* meta) {
    const uint32_t n_wide = w.counts[level];
    const uint32_t n_top = *n_top_p;
    uint32_t fc = 0;
    for (uint32_t si = 0; si < n_wide; si++) {  // one thread: few segments, and fc runs through them
        const SahSeg sg = w.in[si];
        const uint32_t n = sg.end - sg.begin, nch = (n + WIDE_CHUNK - 1) / WIDE_CHUNK;
        uint32_t nL = 0;
        for (uint32_t j = 0; j < nch; j++) nL += w.chunk_left[fc + j];
        fc += nch;
        if (nL == 0 || nL >= n) {
            atomicAdd(&meta->sah_error, 1u);
            continue;
        }
        const CellRec* rout = sg.buf ? li.rec0 : li.rec1;
        const int pi = (int)top_idx[sg.node];
        const int32_t sl = __float_as_int(rout[sg.begin].lo.w), sr = __float_as_int(rout[sg.begin + nL].lo.w);
        left[pi] = sah_link(true, sg.begin, sg.begin + nL, pi, sl, top_idx, n_top, M, pint, pleaf, meta);
        right[pi] = sah_link(false, sg.begin + nL, sg.end, pi, sr, top_idx, n_top, M, pint, pleaf, meta);
        SahSeg c;
        c.depth = (int16_t)(sg.depth + 1);
        c.buf = (int16_t)(1 - sg.buf);
        for (int side = 0; side < 2; side++) {
            c.begin = side ? sg.begin + nL : sg.begin;
            c.end = side ? sg.end : sg.begin + nL;
            if (c.end - c.begin < 2) continue;  // a single cell: linked above
            c.node = (int32_t)(side ? c.begin : c.end - 1);
            if ((uint32_t)c.node >= n_top) continue;  // reported by sah_link
            const uint32_t m = c.end - c.begin;
            if (m > (uint32_t)WIDE_MIN && level + 1 < WIDE_LEVELS) {
                const uint32_t slot = atomicAdd(&w.counts[level + 1], 1u);
                if (slot >= w.cap) {
                    atomicAdd(&meta->sah_error, 1u);
                    continue;
                }
                w.next[slot] = c;
                wide_bounds_init(w.bnext + 12 * slot);
            } else {
                sah_queue(li, level, false, c);
            }
        }
    }
}


// the root segment when there are at least two cells (queued for the grid-wide
// kernels when it has more than WIDE_MIN cells); a top-node count other than
// C - 1 is reported and nothing is built
__global__ void k_sah_init(const uint32_t* __restrict__ n_cells_p, const uint32_t* __restrict__ n_top_p,
                           SahLists li, SahWide w, BuildMeta* meta) {
    const uint32_t C = *n_cells_p;
    if (C < 2) return;
    if (*n_top_p != C - 1) {
        atomicAdd(&meta->sah_error, 1u);
        return;
    }
    SahSeg s;
    s.begin = 0;
    s.end = C;
    s.node = 0;
    s.depth = 0;
    s.buf = 0;
    if (C > (uint32_t)WIDE_MIN) {
        w.in[0] = s;
        w.counts[0] = 1u;
        wide_bounds_init(w.bin);
    } else if (C > (uint32_t)SAH_MID) {
        li.seg_in[0] = s;
        li.counts[0] = 1u;
    } else if (C > (uint32_t)SAH_SMALL) {
        li.mid_in[0] = s;
        li.counts_mid[0] = 1u;
    } else {
        li.seg_small[0] = s;
        li.counts[SAH_LEVELS] = 1u;
    }
}

}  // namespace rr
