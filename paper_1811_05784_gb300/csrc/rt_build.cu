// rt_build.cu -- rt_build_tree: mesh ingest and device LBVH construction.
//
// The paper accelerates the nearest-element search with a binary tree:
// mother box, split along the largest dimension at the median, recursively,
// one element per leaf (Sec. 2.2).  On the GPU the tree is a linear BVH
// (Karras 2012, "Maximizing parallelism in the construction of BVHs, octrees
// and k-d trees"): 48-bit Morton codes of triangle centroids are sorted with
// the device radix sort, every internal node finds its key range and split
// independently, boxes are refitted bottom-up with one atomic flag per node
// (the second child to arrive computes the union and climbs on), and
// subtrees of at most RR_LEAF_MAX triangles collapse into leaves.  The binary
// tree is then stored 4-wide: every kept node at even depth holds its
// grandchildren, which halves the traversal steps of a query.
//
// Layout in HBM (see also rt_internal.cuh):
//   nodes   : 128 B per 4-wide node = 8 x float4 = child boxes as SoA
//             (lo.x[4] lo.y[4] lo.z[4] hi.x[4] hi.y[4] hi.z[4]), refs[4], count
//   tris    : 48 B per triangle in tree order = 3 x float4 (v0|id, v1|surface, v2)
//   tri_nrm : 16 B per triangle by id = float32 unit normal + surface id
//   planes  : 32 B per surface, FP64 (n, d) for image-source mirroring
#include "rt_internal.cuh"

#include <algorithm>
#include <climits>
#include <cmath>
#include <map>
#include <tuple>

namespace rr {

struct BuildMeta {
    unsigned int cmin[3], cmax[3];  // centroid bounds, order-preserving float bits
    int max_surf, min_surf, max_mat, min_mat;
    unsigned int bad_index, non_finite, degenerate, mixed_material;
    int depth;
    unsigned int sah_error;  // inconsistencies found by the SAH top levels (none expected)
};

__device__ __forceinline__ unsigned int f2ord(float f) {
    unsigned int b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int o) {
    unsigned int b = (o & 0x80000000u) ? (o & 0x7FFFFFFFu) : ~o;
    return __uint_as_float(b);
}

// pass 1: validate, convert to float32, per-triangle normal, bounds, id ranges.
// Bounds and id ranges are reduced within each warp, then within the block
// (one atomic per block and quantity instead of one per triangle).
static constexpr int TRI_PREP_THREADS = 256;

__global__ void __launch_bounds__(TRI_PREP_THREADS) k_tri_prep(const double* __restrict__ V, int64_t nV, const int32_t* __restrict__ T, int64_t M,
                           const int32_t* __restrict__ mat, const int32_t* __restrict__ surf,
                           float4* __restrict__ tv, float4* __restrict__ nrm, BuildMeta* meta) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool in = t < M;
    unsigned int cmin[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, cmax[3] = {0u, 0u, 0u};
    int smax = INT_MIN, smin = INT_MAX, mmax = INT_MIN, mmin = INT_MAX;
    if (in) {
        int32_t ia = T[3 * t], ib = T[3 * t + 1], ic = T[3 * t + 2];
        if (ia < 0 || ib < 0 || ic < 0 || ia >= nV || ib >= nV || ic >= nV) {
            atomicAdd(&meta->bad_index, 1u);
            ia = ib = ic = 0;
        }
        double a[3], b[3], c[3];
        for (int k = 0; k < 3; k++) {
            a[k] = V[3 * (int64_t)ia + k];
            b[k] = V[3 * (int64_t)ib + k];
            c[k] = V[3 * (int64_t)ic + k];
        }
        bool finite = true;
        for (int k = 0; k < 3; k++) finite = finite && isfinite(a[k]) && isfinite(b[k]) && isfinite(c[k]);
        if (!finite) {
            atomicAdd(&meta->non_finite, 1u);
            for (int k = 0; k < 3; k++) a[k] = b[k] = c[k] = 0.0;
        }
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
        double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                       e1[0] * e2[1] - e1[1] * e2[0]};
        double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (!(len > 0.0)) {
            atomicAdd(&meta->degenerate, 1u);
            len = 1.0;
        }
        const int32_t s = surf[t], m = mat[t];
        const double il = 1.0 / len;  // one FP64 division instead of three (FP64 division is costly)
        nrm[t] = make_float4((float)(n[0] * il), (float)(n[1] * il), (float)(n[2] * il), __int_as_float(s));
        float4 fa = make_float4((float)a[0], (float)a[1], (float)a[2], __int_as_float((int)t));
        float4 fb = make_float4((float)b[0], (float)b[1], (float)b[2], __int_as_float(s));
        float4 fc = make_float4((float)c[0], (float)c[1], (float)c[2], 0.f);
        tv[3 * t] = fa;
        tv[3 * t + 1] = fb;
        tv[3 * t + 2] = fc;
        const float cx = (fa.x + fb.x + fc.x) * (1.0f / 3.0f), cy = (fa.y + fb.y + fc.y) * (1.0f / 3.0f),
                    cz = (fa.z + fb.z + fc.z) * (1.0f / 3.0f);
        cmin[0] = cmax[0] = f2ord(cx);
        cmin[1] = cmax[1] = f2ord(cy);
        cmin[2] = cmax[2] = f2ord(cz);
        smax = smin = s;
        mmax = mmin = m;
    }
    const unsigned int full = 0xffffffffu;
    for (int k = 0; k < 3; k++) {
        cmin[k] = __reduce_min_sync(full, cmin[k]);
        cmax[k] = __reduce_max_sync(full, cmax[k]);
    }
    smax = __reduce_max_sync(full, smax);
    smin = __reduce_min_sync(full, smin);
    mmax = __reduce_max_sync(full, mmax);
    mmin = __reduce_min_sync(full, mmin);
    // then across the block: one atomic per block and quantity
    __shared__ unsigned int s_u[TRI_PREP_THREADS / 32][6];
    __shared__ int s_i[TRI_PREP_THREADS / 32][4];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        for (int k = 0; k < 3; k++) s_u[warp][k] = cmin[k], s_u[warp][3 + k] = cmax[k];
        s_i[warp][0] = smax, s_i[warp][1] = smin, s_i[warp][2] = mmax, s_i[warp][3] = mmin;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = TRI_PREP_THREADS / 32;
        if (lane < 3) {
            unsigned int lo = s_u[0][lane], hi = s_u[0][3 + lane];
            for (int w = 1; w < nw; w++) lo = min(lo, s_u[w][lane]), hi = max(hi, s_u[w][3 + lane]);
            atomicMin(&meta->cmin[lane], lo);
            atomicMax(&meta->cmax[lane], hi);
        } else if (lane < 7) {
            const int q = lane - 3;
            int v = s_i[0][q];
            for (int w = 1; w < nw; w++) v = (q & 1) ? min(v, s_i[w][q]) : max(v, s_i[w][q]);
            if (q == 0) atomicMax(&meta->max_surf, v);
            if (q == 1) atomicMin(&meta->min_surf, v);
            if (q == 2) atomicMax(&meta->max_mat, v);
            if (q == 3) atomicMin(&meta->min_mat, v);
        }
    }
}

// Surface tables.  They run on the raw input before it has been validated
// on the host, so every id and index is checked before it is used: surface
// ids outside [0, cap) and vertex indices outside [0, nV) are skipped (the
// host then reports them from the build's own checks).
// lowest triangle id per surface (first[] starts at 0x7F7F7F7F >= M)
// (lanes of a warp holding the same surface send one atomic: the lowest lane's
// triangle, the lowest id among them)
__global__ void k_surf_first(const int32_t* __restrict__ surf, int64_t M, int64_t cap, int32_t* __restrict__ first) {
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int32_t sid = t < M ? surf[t] : -1;
    const unsigned int peers = __match_any_sync(0xffffffffu, sid);
    if (sid >= 0 && sid < cap && (peers & ((1u << lane) - 1u)) == 0) atomicMin(&first[sid], (int32_t)t);
}

// FP64 plane of each surface from its lowest-id triangle; its material
__global__ void k_planes(const double* __restrict__ V, int64_t nV, const int32_t* __restrict__ T, int64_t M,
                         const int32_t* __restrict__ mat, const int32_t* __restrict__ first, int64_t S,
                         Plane* __restrict__ planes, int32_t* __restrict__ mat_of_surf) {
    int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= S) return;
    int32_t t = first[s];
    int32_t ia = 0, ib = 0, ic = 0;
    if (t >= 0 && t < M) ia = T[3 * (int64_t)t], ib = T[3 * (int64_t)t + 1], ic = T[3 * (int64_t)t + 2];
    if (t < 0 || t >= M || ia < 0 || ib < 0 || ic < 0 || ia >= nV || ib >= nV || ic >= nV) {
        planes[s] = Plane{0.0, 0.0, 0.0, 0.0};  // unused surface id, or input the host rejects
        mat_of_surf[s] = t >= 0 && t < M ? mat[t] : 0;
        return;
    }
    const double* a = V + 3 * (int64_t)ia;
    const double* b = V + 3 * (int64_t)ib;
    const double* c = V + 3 * (int64_t)ic;
    double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]};
    double e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    if (!(len > 0.0)) len = 1.0;
    n[0] /= len;
    n[1] /= len;
    n[2] /= len;
    planes[s] = Plane{n[0], n[1], n[2], n[0] * a[0] + n[1] * a[1] + n[2] * a[2]};
    mat_of_surf[s] = mat[t];
}

__global__ void k_surf_check(const int32_t* __restrict__ surf, const int32_t* __restrict__ mat, int64_t M,
                             int64_t cap, const int32_t* __restrict__ mat_of_surf, BuildMeta* meta) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    const int32_t sid = surf[t];
    if (sid >= 0 && sid < cap && mat[t] != mat_of_surf[sid]) atomicAdd(&meta->mixed_material, 1u);
}

// Morton code of the float32 centroid within the centroid bounds: 48 bits
// (16 per axis, cells of 1/65536 of the bounds) sort in 6 radix passes instead
// of the 8 of 63-bit codes; equal codes are ordered by index, as in Karras's
// construction
static constexpr int MORTON_BITS_PER_AXIS = 16;

__global__ void k_morton(const float4* __restrict__ tv, int64_t M, const BuildMeta* meta,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= M) return;
    float4 a = tv[3 * t], b = tv[3 * t + 1], c = tv[3 * t + 2];
    float cen[3] = {(a.x + b.x + c.x) * (1.0f / 3.0f), (a.y + b.y + c.y) * (1.0f / 3.0f),
                    (a.z + b.z + c.z) * (1.0f / 3.0f)};
    uint32_t q[3];
    for (int k = 0; k < 3; k++) {
        float lo = ord2f(meta->cmin[k]), hi = ord2f(meta->cmax[k]);
        float ext = hi - lo;
        float x = ext > 0.f ? (cen[k] - lo) / ext : 0.f;
        float s = x * 65536.0f;  // 2^16 cells per axis
        uint32_t v = s <= 0.f ? 0u : (s >= 65535.0f ? 65535u : (uint32_t)s);
        q[k] = v;
    }
    uint64_t code = 0;
    for (int bit = 0; bit < MORTON_BITS_PER_AXIS; bit++) {
        code |= (uint64_t)((q[0] >> bit) & 1u) << (3 * bit + 2);
        code |= (uint64_t)((q[1] >> bit) & 1u) << (3 * bit + 1);
        code |= (uint64_t)((q[2] >> bit) & 1u) << (3 * bit);
    }
    keys[t] = code;
    vals[t] = (uint32_t)t;
}

// Karras delta: common prefix length of (code, index) keys; -1 outside [0, M)
__device__ __forceinline__ int kdelta(const uint64_t* __restrict__ codes, int64_t M, int64_t i, int64_t j) {
    if (j < 0 || j >= M) return -1;
    uint64_t a = codes[i], b = codes[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz((int)((uint32_t)i ^ (uint32_t)j));
}

// one thread per internal node i in [0, M-1): its key range and split
__global__ void k_karras(const uint64_t* __restrict__ codes, int64_t M, int32_t* __restrict__ left,
                         int32_t* __restrict__ right, int32_t* __restrict__ first, int32_t* __restrict__ last,
                         int32_t* __restrict__ parent_int, int32_t* __restrict__ parent_leaf) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= M - 1) return;
    int d = (kdelta(codes, M, i, i + 1) - kdelta(codes, M, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = kdelta(codes, M, i, i - d);
    int64_t lmax = 2;
    while (lmax < 2 * M && kdelta(codes, M, i, i + lmax * d) > dmin) lmax *= 2;
    int64_t l = 0;
    for (int64_t t = lmax / 2; t >= 1; t /= 2)
        if (kdelta(codes, M, i, i + (l + t) * d) > dmin) l += t;
    int64_t j = i + l * d;
    int dnode = kdelta(codes, M, i, j);
    int64_t s = 0;
    int64_t div = 2;
    for (int it = 0; it < 64; it++) {
        int64_t t = (l + div - 1) / div;
        if (kdelta(codes, M, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
        div *= 2;
    }
    int64_t gamma = i + s * d + (d < 0 ? -1 : 0);
    int64_t lo = i < j ? i : j, hi = i < j ? j : i;
    int32_t lc, rc;
    if (lo == gamma) {
        lc = ~(int32_t)gamma;
        parent_leaf[gamma] = (int32_t)i;
    } else {
        lc = (int32_t)gamma;
        parent_int[gamma] = (int32_t)i;
    }
    if (hi == gamma + 1) {
        rc = ~(int32_t)(gamma + 1);
        parent_leaf[gamma + 1] = (int32_t)i;
    } else {
        rc = (int32_t)(gamma + 1);
        parent_int[gamma + 1] = (int32_t)i;
    }
    left[i] = lc;
    right[i] = rc;
    first[i] = (int32_t)lo;
    last[i] = (int32_t)hi;
}

struct Box {
    float lo[3], hi[3];
};

__device__ __forceinline__ Box tri_box(const float4* __restrict__ tv, int64_t t) {
    float4 a = tv[3 * t], b = tv[3 * t + 1], c = tv[3 * t + 2];
    Box r;
    r.lo[0] = fminf(a.x, fminf(b.x, c.x));
    r.lo[1] = fminf(a.y, fminf(b.y, c.y));
    r.lo[2] = fminf(a.z, fminf(b.z, c.z));
    r.hi[0] = fmaxf(a.x, fmaxf(b.x, c.x));
    r.hi[1] = fmaxf(a.y, fmaxf(b.y, c.y));
    r.hi[2] = fmaxf(a.z, fmaxf(b.z, c.z));
    return r;
}

// leaf boxes in sorted order
// ---------------------------------------------------------------------------
// The paper's tree (Sec. 2.2): the box of a node's triangles is split along
// its largest extent at the median, recursively, down to one triangle.  Its
// shape depends on M alone -- every node [s, e] gives its first
// ceil(count / 2) triangles to the left child -- so the topology is written
// directly, with internal node ids = split positions (the root relabelled
// to 0); only the order of the triangles depends on the geometry.  Level L
// sorts every node of depth L by centroid along its box's largest extent
// (segmented, as one radix sort of (node start, coordinate) keys).
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ int64_t msplit(int64_t s, int64_t e) { return s + (e - s + 2) / 2 - 1; }

__device__ __forceinline__ int32_t median_id(int64_t g, int64_t root) {
    return (int32_t)(g == root ? 0 : (g == 0 ? root : g));
}

// the node of depth L that holds position p (or the leaf it reached earlier)
__device__ __forceinline__ void median_segment(int64_t M, int64_t p, int L, int64_t& s, int64_t& e) {
    s = 0;
    e = M - 1;
    for (int l = 0; l < L && e > s; l++) {
        const int64_t m = msplit(s, e);
        if (p <= m)
            e = m;
        else
            s = m + 1;
    }
}

__global__ void k_iota(int64_t n, uint32_t* __restrict__ v) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

__global__ void k_median_boxes(const float4* __restrict__ tv, const uint32_t* __restrict__ order, int64_t M, int L,
                               unsigned int* __restrict__ seg_lo, unsigned int* __restrict__ seg_hi) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    int64_t s, e;
    median_segment(M, p, L, s, e);
    if (e == s) return;
    const Box b = tri_box(tv, order[p]);
    for (int k = 0; k < 3; k++) {
        atomicMin(&seg_lo[3 * s + k], f2ord(b.lo[k]));
        atomicMax(&seg_hi[3 * s + k], f2ord(b.hi[k]));
    }
}

__global__ void k_median_keys(const float4* __restrict__ tv, const uint32_t* __restrict__ order, int64_t M, int L,
                              const unsigned int* __restrict__ seg_lo, const unsigned int* __restrict__ seg_hi,
                              uint64_t* __restrict__ keys) {
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= M) return;
    int64_t s, e;
    median_segment(M, p, L, s, e);
    uint32_t c = 0;
    if (e > s) {
        float ext[3];
        for (int k = 0; k < 3; k++) ext[k] = ord2f(seg_hi[3 * s + k]) - ord2f(seg_lo[3 * s + k]);
        const int ax = (ext[0] >= ext[1] && ext[0] >= ext[2]) ? 0 : (ext[1] >= ext[2] ? 1 : 2);
        const int64_t t = order[p];
        const float4 a = tv[3 * t], b = tv[3 * t + 1], d = tv[3 * t + 2];
        const float ca = ax == 0 ? a.x : (ax == 1 ? a.y : a.z);
        const float cb = ax == 0 ? b.x : (ax == 1 ? b.y : b.z);
        const float cd = ax == 0 ? d.x : (ax == 1 ? d.y : d.z);
        c = f2ord((ca + cb + cd) * (1.0f / 3.0f));
    }
    keys[p] = ((uint64_t)s << 32) | c;
}

__global__ void k_median_topology(int64_t M, int32_t* __restrict__ left, int32_t* __restrict__ right,
                                  int32_t* __restrict__ first, int32_t* __restrict__ last,
                                  int32_t* __restrict__ parent_int, int32_t* __restrict__ parent_leaf) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= M - 1) return;
    const int64_t root = msplit(0, M - 1);
    int64_t s = 0, e = M - 1;
    int32_t parent = -1;
    for (int guard = 0; guard < 64; guard++) {  // depth <= ceil(log2 M) < 64
        const int64_t m = msplit(s, e);
        if (m == g) break;
        parent = median_id(m, root);
        if (g < m)
            e = m;
        else
            s = m + 1;
    }
    const int32_t id = median_id(g, root);
    first[id] = (int32_t)s;
    last[id] = (int32_t)e;
    parent_int[id] = parent;
    if (s == g) {
        left[id] = ~(int32_t)s;
        parent_leaf[s] = id;
    } else {
        left[id] = median_id(msplit(s, g), root);
    }
    if (g + 1 == e) {
        right[id] = ~(int32_t)e;
        parent_leaf[e] = id;
    } else {
        right[id] = median_id(msplit(g + 1, e), root);
    }
}

__global__ void k_leaf_boxes(const float4* __restrict__ tv, const uint32_t* __restrict__ order, int64_t M,
                             float4* __restrict__ leaf_box) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    Box b = tri_box(tv, order[j]);
    leaf_box[2 * j] = make_float4(b.lo[0], b.lo[1], b.lo[2], 0.f);
    leaf_box[2 * j + 1] = make_float4(b.hi[0], b.hi[1], b.hi[2], 0.f);
}

__device__ __forceinline__ void child_box(int32_t c, const float4* leaf_box, const float4* node_box, float4& lo,
                                          float4& hi) {
    if (c < 0) {
        lo = leaf_box[2 * (int64_t)(~c)];
        hi = leaf_box[2 * (int64_t)(~c) + 1];
    } else {
        lo = __ldcg(node_box + 2 * (int64_t)c);
        hi = __ldcg(node_box + 2 * (int64_t)c + 1);
    }
}

// bottom-up refit: the second child to reach a node computes its box.  The
// thread carries the box of the subtree it comes from, so it loads only the
// sibling's box, and it reads the node's children and parent before its
// atomic so that those loads overlap the atomic's round trip.
__global__ void k_refit(int64_t M, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                        const int32_t* __restrict__ parent_int, const int32_t* __restrict__ parent_leaf,
                        const float4* __restrict__ leaf_box, float4* node_box, unsigned int* flags) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    int32_t p = parent_leaf[j];
    int32_t from = ~(int32_t)j;  // child reference of the subtree this thread carries
    float4 clo = leaf_box[2 * j], chi = leaf_box[2 * j + 1];
    for (int64_t step = 0; p >= 0 && step < M; step++) {
        const int32_t l = left[p], r = right[p], pp = parent_int[p];
        __threadfence();
        unsigned int old = atomicAdd(&flags[p], 1u);
        if (old == 0) return;
        __threadfence();
        float4 sl, sh;
        child_box(l == from ? r : l, leaf_box, node_box, sl, sh);
        clo = make_float4(fminf(clo.x, sl.x), fminf(clo.y, sl.y), fminf(clo.z, sl.z), 0.f);
        chi = make_float4(fmaxf(chi.x, sh.x), fmaxf(chi.y, sh.y), fmaxf(chi.z, sh.z), 0.f);
        __stcg(node_box + 2 * (int64_t)p, clo);
        __stcg(node_box + 2 * (int64_t)p + 1, chi);
        from = p;
        p = pp;
    }
}

__global__ void k_depth(int64_t M, const int32_t* __restrict__ parent_int, const int32_t* __restrict__ parent_leaf,
                        BuildMeta* meta) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    int depth = 1;
    int32_t p = parent_leaf[j];
    while (p >= 0 && depth < 100000) {
        depth++;
        p = parent_int[p];
    }
    atomicMax(&meta->depth, depth);
}

__global__ void k_keep(int64_t n_int, const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                       uint32_t* __restrict__ keep) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    keep[i] = (i == 0 || (last[i] - first[i] + 1) > RR_LEAF_MAX) ? 1u : 0u;
}

// A kept binary node at even depth becomes a 4-wide node whose children are
// its binary grandchildren (children where a child is a leaf).  Kept nodes
// form a connected top part of the tree (a parent holds more triangles than
// its child), so every kept odd-depth node is opened by its parent.
__global__ void k_keep4(int64_t n_int, const int32_t* __restrict__ parent_int, const uint32_t* __restrict__ keep,
                        uint32_t* __restrict__ keep4) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    if (!keep[i]) {
        keep4[i] = 0u;
        return;
    }
    int depth = 0;
    int32_t p = parent_int[i];
    while (p >= 0 && depth < 100000) {
        depth++;
        p = parent_int[p];
    }
    keep4[i] = (depth & 1) ? 0u : 1u;
}

// leaf reference: ~(first triangle << 3 | count), count <= RR_LEAF_MAX
__device__ __forceinline__ int32_t leaf_ref(int32_t first, int32_t count) { return ~((first << 3) | count); }

struct WideChild {
    float4 lo, hi;
    int32_t ref;
};

// binary child c as a wide child: a single-triangle leaf (c < 0), a leaf of
// a non-kept subtree, or a kept node's 4-wide index
__device__ __forceinline__ WideChild wide_child(int32_t c, const uint32_t* keep, const uint32_t* newidx,
                                                const int32_t* first, const int32_t* last, const float4* leaf_box,
                                                const float4* node_box) {
    WideChild w;
    if (c < 0) {
        w.lo = leaf_box[2 * (int64_t)(~c)];
        w.hi = leaf_box[2 * (int64_t)(~c) + 1];
        w.ref = leaf_ref(~c, 1);
    } else {
        w.lo = node_box[2 * (int64_t)c];
        w.hi = node_box[2 * (int64_t)c + 1];
        w.ref = keep[c] ? (int32_t)newidx[c] : leaf_ref(first[c], last[c] - first[c] + 1);
    }
    return w;
}

// 4-wide node layout (128 B): float4 0..5 = lo.x[4], lo.y[4], lo.z[4],
// hi.x[4], hi.y[4], hi.z[4]; float4 6 = child refs; float4 7 = child count.
// An empty slot has lo = hi = +inf, which every ray misses (entry at +inf or
// an empty interval) and ref = leaf_ref(0, 0).
__device__ __forceinline__ void store_wide(float4* n, const WideChild* c, int nc) {
    float v[6][4];
    int32_t r[4];
    for (int k = 0; k < 4; k++) {
        const bool ok = k < nc;
        v[0][k] = ok ? c[k].lo.x : INFINITY;
        v[1][k] = ok ? c[k].lo.y : INFINITY;
        v[2][k] = ok ? c[k].lo.z : INFINITY;
        v[3][k] = ok ? c[k].hi.x : INFINITY;
        v[4][k] = ok ? c[k].hi.y : INFINITY;
        v[5][k] = ok ? c[k].hi.z : INFINITY;
        r[k] = ok ? c[k].ref : leaf_ref(0, 0);
    }
    for (int j = 0; j < 6; j++) n[j] = make_float4(v[j][0], v[j][1], v[j][2], v[j][3]);
    n[6] = make_float4(__int_as_float(r[0]), __int_as_float(r[1]), __int_as_float(r[2]), __int_as_float(r[3]));
    n[7] = make_float4(__int_as_float(nc), 0.f, 0.f, 0.f);
}

__global__ void k_emit_wide(int64_t n_int, const int32_t* __restrict__ left, const int32_t* __restrict__ right,
                            const int32_t* __restrict__ first, const int32_t* __restrict__ last,
                            const uint32_t* __restrict__ keep, const uint32_t* __restrict__ keep4,
                            const uint32_t* __restrict__ newidx, const float4* __restrict__ leaf_box,
                            const float4* __restrict__ node_box, float4* __restrict__ nodes) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int || !keep4[i]) return;
    WideChild c[4];
    int nc = 0;
    if (i == 0 && (last[0] - first[0] + 1) <= RR_LEAF_MAX) {
        // the whole mesh fits one leaf
        c[0].lo = node_box[0];
        c[0].hi = node_box[1];
        c[0].ref = leaf_ref(0, last[0] - first[0] + 1);
        nc = 1;
    } else {
        const int32_t kids[2] = {left[i], right[i]};
        for (int k = 0; k < 2; k++) {
            const int32_t b = kids[k];
            if (b >= 0 && keep[b]) {  // a kept odd-depth node: open it
                c[nc++] = wide_child(left[b], keep, newidx, first, last, leaf_box, node_box);
                c[nc++] = wide_child(right[b], keep, newidx, first, last, leaf_box, node_box);
            } else {
                c[nc++] = wide_child(b, keep, newidx, first, last, leaf_box, node_box);
            }
        }
    }
    store_wide(nodes + 8 * (int64_t)newidx[i], c, nc);
}

// single-triangle mesh: one 4-wide node holding one leaf
__global__ void k_single(const float4* __restrict__ tv, float4* __restrict__ nodes, float4* __restrict__ tris,
                         int32_t* __restrict__ pos_of) {
    Box b = tri_box(tv, 0);
    WideChild c;
    c.lo = make_float4(b.lo[0], b.lo[1], b.lo[2], 0.f);
    c.hi = make_float4(b.hi[0], b.hi[1], b.hi[2], 0.f);
    c.ref = leaf_ref(0, 1);
    store_wide(nodes, &c, 1);
    pos_of[0] = 0;
    tris[0] = tv[0];
    tris[1] = tv[1];
    tris[2] = tv[2];
}

__global__ void k_reorder(const float4* __restrict__ tv, const uint32_t* __restrict__ order, int64_t M,
                          float4* __restrict__ tris, int32_t* __restrict__ pos_of) {
    int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= M) return;
    int64_t t = order[j];
    pos_of[t] = (int32_t)j;
    tris[3 * j] = tv[3 * t];
    tris[3 * j + 1] = tv[3 * t + 1];
    tris[3 * j + 2] = tv[3 * t + 2];
}

static unsigned grid_of(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace rr

#include "rt_sah_top.cuh"

namespace rr {

// SAH top levels over the Morton cells of an LBVH whose boxes are refitted
// (rt_sah_top.cuh); rewrites the top nodes' entries of the binary arrays
static rt_status sah_top(const uint64_t* keys, int64_t M, int32_t* left, int32_t* right, int32_t* first,
                         int32_t* last, int32_t* pint, int32_t* pleaf, const float4* leaf_box, float4* node_box,
                         BuildMeta* meta, Arena& tmp, cudaStream_t s) {
    const int64_t NI = M - 1;
    uint32_t *cflag, *cid, *cell_first, *n_cells, *is_top, *top_pos, *n_top, *top_idx, *counts;
    CellRec *rec0, *rec1;
    SahSeg *seg_a, *seg_b, *seg_small;
    RR_TRY(tmp.alloc(&cflag, M));
    RR_TRY(tmp.alloc(&cid, M));
    RR_TRY(tmp.alloc(&cell_first, M + 1));
    RR_TRY(tmp.alloc(&n_cells, 1));
    RR_TRY(tmp.alloc(&is_top, NI));
    RR_TRY(tmp.alloc(&top_pos, NI));
    RR_TRY(tmp.alloc(&n_top, 1));
    RR_TRY(tmp.alloc(&top_idx, NI));
    RR_TRY(tmp.alloc(&counts, SAH_LEVELS + 1));
    RR_TRY(tmp.alloc(&rec0, M));
    RR_TRY(tmp.alloc(&rec1, M));
    RR_TRY(tmp.alloc(&seg_a, M));
    RR_TRY(tmp.alloc(&seg_b, M));
    RR_TRY(tmp.alloc(&seg_small, M));
    SahSeg *mid_a, *mid_b;
    uint32_t* counts_mid;
    RR_TRY(tmp.alloc(&mid_a, M));
    RR_TRY(tmp.alloc(&mid_b, M));
    RR_TRY(tmp.alloc(&counts_mid, SAH_LEVELS));
    // the grid-wide first levels: at most C / WIDE_MIN segments of more than WIDE_MIN cells
    const int64_t wcap = M / WIDE_MIN + 2, wchunks = (M + WIDE_CHUNK - 1) / WIDE_CHUNK + wcap;
    SahSeg *wseg_a, *wseg_b;
    uint32_t *wcounts, *chunk_left;
    unsigned int *wbin_a, *wbin_b;
    int4* wsplit;
    RR_TRY(tmp.alloc(&wseg_a, wcap));
    RR_TRY(tmp.alloc(&wseg_b, wcap));
    RR_TRY(tmp.alloc(&wcounts, WIDE_LEVELS + 1));
    RR_TRY(tmp.alloc(&wbin_a, 12 * wcap));
    RR_TRY(tmp.alloc(&wbin_b, 12 * wcap));
    RR_TRY(tmp.alloc(&wsplit, wcap));
    RR_TRY(tmp.alloc(&chunk_left, wchunks));
    void* scan_tmp;
    RR_TRY(tmp.alloc((char**)&scan_tmp, scan_temp_bytes(M)));
    // cells and their records (boxes from the refit)
    RR_LAUNCH(k_cell_flags, grid_of(M, 256), 256, 0, s, keys, M, cflag);
    RR_TRY(exclusive_scan_u32(cflag, cid, M, n_cells, scan_tmp, s));
    RR_LAUNCH(k_cell_first, grid_of(M, 256), 256, 0, s, cflag, cid, M, cell_first);
    RR_LAUNCH(k_cell_records, grid_of(M, 256), 256, 0, s, cell_first, n_cells, M, first, last, leaf_box, node_box,
              rec0, meta);
    // the Karras nodes above the cells give the top nodes their indices
    RR_LAUNCH(k_top_flags, grid_of(NI, 256), 256, 0, s, keys, NI, first, last, is_top);
    RR_CUDA(cudaGetLastError());
    RR_TRY(exclusive_scan_u32(is_top, top_pos, NI, n_top, scan_tmp, s));
    RR_LAUNCH(k_top_compact, grid_of(NI, 256), 256, 0, s, is_top, top_pos, NI, top_idx);
    RR_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * (SAH_LEVELS + 1), s));
    RR_CUDA(cudaMemsetAsync(wcounts, 0, sizeof(uint32_t) * (WIDE_LEVELS + 1), s));
    RR_CUDA(cudaMemsetAsync(counts_mid, 0, sizeof(uint32_t) * SAH_LEVELS, s));
    SahLists li{seg_a, seg_b, seg_small, counts, rec0, rec1, mid_a, mid_b, counts_mid};
    SahWide wi{wseg_a, wseg_b, wcounts, wbin_a, wbin_b, wsplit, chunk_left, (uint32_t)wcap};
    RR_LAUNCH(k_sah_init, 1, 1, 0, s, n_cells, n_top, li, wi, meta);
    const unsigned wgrid = (unsigned)std::min<int64_t>(wchunks, SAH_GRID);
    for (int L = 0; L < SAH_LEVELS; L++) {
        SahLists ll = li;
        ll.seg_in = (L & 1) ? seg_b : seg_a;
        ll.seg_next = (L & 1) ? seg_a : seg_b;
        ll.mid_in = (L & 1) ? mid_b : mid_a;
        ll.mid_next = (L & 1) ? mid_a : mid_b;
        if (L < WIDE_LEVELS) {  // this level's wide segments, split by the whole grid
            SahWide wl = wi;
            wl.in = (L & 1) ? wseg_b : wseg_a;
            wl.next = (L & 1) ? wseg_a : wseg_b;
            wl.bin = (L & 1) ? wbin_b : wbin_a;
            wl.bnext = (L & 1) ? wbin_a : wbin_b;
            RR_LAUNCH(k_wide_bounds, wgrid, WIDE_THREADS, 0, s, L, wl, rec0, rec1);
            RR_LAUNCH(k_wide_decide, (unsigned)std::min<int64_t>(wcap, 152), WIDE_DECIDE_THREADS, 0, s, L, wl, rec0, rec1,
                      top_idx, M, first, last, node_box);
            RR_LAUNCH(k_wide_count, wgrid, WIDE_THREADS, 0, s, L, wl, rec0, rec1);
            RR_LAUNCH(k_wide_scatter, wgrid, WIDE_THREADS, 0, s, L, wl, rec0, rec1, meta);
            RR_LAUNCH(k_wide_children, 1, 1, 0, s, L, wl, ll, top_idx, n_top, M, left, right, pint, pleaf, meta);
        }
        RR_LAUNCH((k_sah_level<SAH_THREADS, false>), SAH_GRID, SAH_THREADS, 0, s, L, L == SAH_LEVELS - 1, ll, top_idx,
                  n_top, M, left, right, first, last, pint, pleaf, node_box, meta);
        RR_LAUNCH((k_sah_level<SAH_MID_THREADS, true>), SAH_MID_GRID, SAH_MID_THREADS, 0, s, L, L == SAH_LEVELS - 1, ll,
                  top_idx, n_top, M, left, right, first, last, pint, pleaf, node_box, meta);
    }
    RR_LAUNCH(k_sah_small, SAH_GRID, 256, 0, s, li, top_idx, n_top, M, left, right, first, last, pint, pleaf,
              node_box, meta);
    RR_CUDA(cudaGetLastError());
    return RT_OK;
}

// host grouping of triangles into surfaces by (material, plane) when the
// caller gives no surface ids
static std::vector<int32_t> group_surfaces(const double* V, const int32_t* T, const int32_t* mat, int64_t M) {
    std::map<std::tuple<int32_t, long long, long long, long long, long long>, int32_t> ids;
    std::vector<int32_t> out((size_t)M);
    for (int64_t t = 0; t < M; t++) {
        const double *a = V + 3 * (int64_t)T[3 * t], *b = V + 3 * (int64_t)T[3 * t + 1],
                     *c = V + 3 * (int64_t)T[3 * t + 2];
        double e1[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, e2[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
        double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
        double len = std::sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        if (len > 0) {
            n[0] /= len, n[1] /= len, n[2] /= len;
        }
        // canonical orientation: first non-zero component positive
        int k = std::fabs(n[0]) > 1e-12 ? 0 : (std::fabs(n[1]) > 1e-12 ? 1 : 2);
        if (n[k] < 0) n[0] = -n[0], n[1] = -n[1], n[2] = -n[2];
        double d = n[0] * a[0] + n[1] * a[1] + n[2] * a[2];
        auto key = std::make_tuple(mat[t], std::llround(n[0] * 1e7), std::llround(n[1] * 1e7),
                                   std::llround(n[2] * 1e7), std::llround(d * 1e5));
        auto it = ids.find(key);
        if (it == ids.end()) it = ids.emplace(key, (int32_t)ids.size()).first;
        out[(size_t)t] = it->second;
    }
    return out;
}

enum BuildKind { BUILD_LBVH = 0, BUILD_MEDIAN = 1, BUILD_SAH_TOP = 2 };

static rt_status build_impl(const rt_mesh* mesh, cudaStream_t s, rt_tree** out, BuildKind kind = BUILD_LBVH) {
    const bool median = kind == BUILD_MEDIAN;
    if (!mesh || !out) {
        set_error("rt_build_tree: null argument");
        return RT_ERR_INVALID_ARG;
    }
    *out = nullptr;
    const int64_t M = mesh->n_tris, nV = mesh->n_vertices;
    if (M < 1 || nV < 3 || !mesh->vertices || !mesh->tris || !mesh->material_id) {
        set_error("rt_build_tree: need n_tris >= 1, n_vertices >= 3 and non-null arrays");
        return RT_ERR_INVALID_ARG;
    }
    if (M >= ((int64_t)1 << 28)) {
        set_error("rt_build_tree: %lld triangles exceed the 32-bit index range", (long long)M);
        return RT_ERR_INVALID_ARG;
    }
    if (mesh->memory != RT_MEM_HOST && mesh->memory != RT_MEM_DEVICE) {
        set_error("rt_build_tree: bad memory kind");
        return RT_ERR_INVALID_ARG;
    }
    if (!mesh->surface_id && mesh->memory != RT_MEM_HOST) {
        set_error("rt_build_tree: surface_id may be NULL only for host meshes");
        return RT_ERR_INVALID_ARG;
    }
    Arena tmp(s), keep_arena(s);
    const double* dV = mesh->vertices;
    const int32_t *dT = mesh->tris, *dmat = mesh->material_id, *dsurf = mesh->surface_id;
    std::vector<int32_t> host_surf;
    if (mesh->memory == RT_MEM_HOST) {
        double* v;
        int32_t *t, *m, *sf;
        RR_TRY(tmp.alloc(&v, 3 * nV));
        RR_TRY(tmp.alloc(&t, 3 * M));
        RR_TRY(tmp.alloc(&m, M));
        RR_TRY(tmp.alloc(&sf, M));
        const int32_t* hs = mesh->surface_id;
        if (!hs) {
            for (int64_t k = 0; k < 3 * M; k++) {
                if (mesh->tris[k] < 0 || mesh->tris[k] >= nV) {
                    set_error("rt_build_tree: vertex index out of range");
                    return RT_ERR_INVALID_ARG;
                }
            }
            host_surf = group_surfaces(mesh->vertices, mesh->tris, mesh->material_id, M);
            hs = host_surf.data();
        }
        RR_CUDA(cudaMemcpyAsync(v, mesh->vertices, sizeof(double) * 3 * nV, cudaMemcpyHostToDevice, s));
        RR_CUDA(cudaMemcpyAsync(t, mesh->tris, sizeof(int32_t) * 3 * M, cudaMemcpyHostToDevice, s));
        RR_CUDA(cudaMemcpyAsync(m, mesh->material_id, sizeof(int32_t) * M, cudaMemcpyHostToDevice, s));
        RR_CUDA(cudaMemcpyAsync(sf, hs, sizeof(int32_t) * M, cudaMemcpyHostToDevice, s));
        dV = v, dT = t, dmat = m, dsurf = sf;
    }
    rt_tree* tree = new rt_tree();
    struct Guard {
        rt_tree*& t;
        ~Guard() {
            if (t) {
                for (void* p : t->owned) dev_free(p, t->stream);
                delete t;
            }
        }
    } guard{tree};
    tree->stream = s;
    tree->n_tris = M;

    BuildMeta* meta;
    RR_TRY(tmp.alloc(&meta, 1));
    BuildMeta hm;
    for (int k = 0; k < 3; k++) hm.cmin[k] = 0xFFFFFFFFu, hm.cmax[k] = 0u;
    hm.max_surf = INT_MIN, hm.min_surf = INT_MAX, hm.max_mat = INT_MIN, hm.min_mat = INT_MAX;
    hm.bad_index = hm.non_finite = hm.degenerate = hm.mixed_material = 0;
    hm.depth = 0;
    hm.sah_error = 0;
    RR_CUDA(cudaMemcpyAsync(meta, &hm, sizeof hm, cudaMemcpyHostToDevice, s));

    float4 *tv, *tri_nrm;
    RR_TRY(tmp.alloc(&tv, 3 * M));
    RR_TRY(keep_arena.alloc(&tri_nrm, M));
    RR_LAUNCH(k_tri_prep, grid_of(M, TRI_PREP_THREADS), TRI_PREP_THREADS, 0, s, dV, nV, dT, M, dmat, dsurf, tv,
              tri_nrm, meta);
    RR_CUDA(cudaGetLastError());
    // Everything up to the 4-wide nodes depends only on M, so it is queued
    // before the first synchronisation; invalid input (reported below) was
    // made harmless by k_tri_prep (indices clamped, coordinates zeroed).

    // Morton codes, sort
    uint64_t *keys, *keys_alt;
    uint32_t *vals, *vals_alt;
    RR_TRY(tmp.alloc(&keys, M));
    RR_TRY(tmp.alloc(&keys_alt, M));
    RR_TRY(tmp.alloc(&vals, M));
    RR_TRY(tmp.alloc(&vals_alt, M));
    void* sort_tmp;
    RR_TRY(tmp.alloc((char**)&sort_tmp, sort_temp_bytes(M)));
    if (!median) {
        RR_LAUNCH(k_morton, grid_of(M, 256), 256, 0, s, tv, M, meta, keys, vals);
        RR_CUDA(cudaGetLastError());
        RR_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, M, 0, 3 * MORTON_BITS_PER_AXIS, sort_tmp, s));
    } else {
        // identity order, then one segmented sort per level
        RR_LAUNCH(k_iota, grid_of(M, 256), 256, 0, s, M, vals);
        unsigned int *seg_lo, *seg_hi;
        RR_TRY(tmp.alloc(&seg_lo, 3 * M));
        RR_TRY(tmp.alloc(&seg_hi, 3 * M));
        int levels = 0;
        while ((int64_t)1 << levels < M) levels++;
        for (int L = 0; L < levels; L++) {
            RR_CUDA(cudaMemsetAsync(seg_lo, 0xFF, sizeof(unsigned int) * 3 * M, s));
            RR_CUDA(cudaMemsetAsync(seg_hi, 0x00, sizeof(unsigned int) * 3 * M, s));
            RR_LAUNCH(k_median_boxes, grid_of(M, 256), 256, 0, s, tv, vals, M, L, seg_lo, seg_hi);
            RR_LAUNCH(k_median_keys, grid_of(M, 256), 256, 0, s, tv, vals, M, L, seg_lo, seg_hi, keys);
            RR_CUDA(cudaGetLastError());
            RR_TRY(radix_sort_pairs(keys, vals, keys_alt, vals_alt, M, 0, 64, sort_tmp, s));
        }
    }

    float4* tris;
    RR_TRY(keep_arena.alloc(&tris, 3 * M));
    int32_t* pos_of;
    RR_TRY(keep_arena.alloc(&pos_of, M));
    float4* nodes;
    uint32_t* total = nullptr;
    if (M == 1) {
        RR_TRY(keep_arena.alloc(&nodes, 8));
        RR_LAUNCH(k_single, 1, 1, 0, s, tv, nodes, tris, pos_of);
        RR_CUDA(cudaGetLastError());
    } else {
        const int64_t NI = M - 1;
        int32_t *left, *right, *first, *last, *pint, *pleaf;
        float4 *leaf_box, *node_box;
        unsigned int* flags;
        uint32_t *keep, *keep4, *newidx;
        RR_TRY(tmp.alloc(&left, NI));
        RR_TRY(tmp.alloc(&right, NI));
        RR_TRY(tmp.alloc(&first, NI));
        RR_TRY(tmp.alloc(&last, NI));
        RR_TRY(tmp.alloc(&pint, NI));
        RR_TRY(tmp.alloc(&pleaf, M));
        RR_TRY(tmp.alloc(&leaf_box, 2 * M));
        RR_TRY(tmp.alloc(&node_box, 2 * NI));
        RR_TRY(tmp.alloc(&flags, NI));
        RR_TRY(tmp.alloc(&keep, NI));
        RR_TRY(tmp.alloc(&keep4, NI));
        RR_TRY(tmp.alloc(&newidx, NI));
        RR_TRY(tmp.alloc(&total, 1));
        void* scan_tmp;
        RR_TRY(tmp.alloc((char**)&scan_tmp, scan_temp_bytes(NI)));
        RR_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned int) * NI, s));
        RR_CUDA(cudaMemsetAsync(pint, 0xFF, sizeof(int32_t) * NI, s));  // root keeps -1
        if (!median)
            RR_LAUNCH(k_karras, grid_of(NI, 256), 256, 0, s, keys, M, left, right, first, last, pint, pleaf);
        else
            RR_LAUNCH(k_median_topology, grid_of(NI, 256), 256, 0, s, M, left, right, first, last, pint, pleaf);
        RR_LAUNCH(k_leaf_boxes, grid_of(M, 256), 256, 0, s, tv, vals, M, leaf_box);
        RR_LAUNCH(k_refit, grid_of(M, 256), 256, 0, s, M, left, right, pint, pleaf, leaf_box, node_box, flags);
        if (kind == BUILD_SAH_TOP)
            RR_TRY(sah_top(keys, M, left, right, first, last, pint, pleaf, leaf_box, node_box, meta, tmp, s));
        RR_LAUNCH(k_depth, grid_of(M, 256), 256, 0, s, M, pint, pleaf, meta);
        RR_LAUNCH(k_keep, grid_of(NI, 256), 256, 0, s, NI, first, last, keep);
        RR_LAUNCH(k_keep4, grid_of(NI, 256), 256, 0, s, NI, pint, keep, keep4);
        RR_CUDA(cudaGetLastError());
        RR_TRY(exclusive_scan_u32(keep4, newidx, NI, total, scan_tmp, s));
        // at most NI 4-wide nodes (one per kept binary node): allocate that
        // instead of reading the count back first
        RR_TRY(keep_arena.alloc(&nodes, 8 * NI));
        RR_LAUNCH(k_emit_wide, grid_of(NI, 256), 256, 0, s, NI, left, right, first, last, keep, keep4, newidx,
                  leaf_box, node_box, nodes);
        RR_LAUNCH(k_reorder, grid_of(M, 256), 256, 0, s, tv, vals, M, tris, pos_of);
        RR_CUDA(cudaGetLastError());
    }
    // surface tables, sized for ids below M (the usual dense numbering), queued
    // before the synchronisation as well; sparse ids larger than that are
    // handled after it
    int32_t *mat_of_surf = nullptr, *surf_of = nullptr;
    Plane* planes = nullptr;
    RR_TRY(keep_arena.alloc(&surf_of, M));
    RR_CUDA(cudaMemcpyAsync(surf_of, dsurf, sizeof(int32_t) * M, cudaMemcpyDeviceToDevice, s));
    auto surface_tables = [&](int64_t cap) -> rt_status {
        int32_t* sfirst;
        RR_TRY(tmp.alloc(&sfirst, cap));
        RR_TRY(keep_arena.alloc(&mat_of_surf, cap));
        RR_TRY(keep_arena.alloc(&planes, cap));
        RR_CUDA(cudaMemsetAsync(sfirst, 0x7F, sizeof(int32_t) * cap, s));
        RR_CUDA(cudaMemsetAsync(&meta->mixed_material, 0, sizeof(unsigned int), s));
        RR_LAUNCH(k_surf_first, grid_of(M, 256), 256, 0, s, dsurf, M, cap, sfirst);
        RR_LAUNCH(k_planes, grid_of(cap, 128), 128, 0, s, dV, nV, dT, M, dmat, sfirst, cap, planes, mat_of_surf);
        RR_LAUNCH(k_surf_check, grid_of(M, 256), 256, 0, s, dsurf, dmat, M, cap, mat_of_surf, meta);
        RR_CUDA(cudaGetLastError());
        return RT_OK;
    };
    RR_TRY(surface_tables(M));
    uint32_t nn = 1;
    if (total) RR_CUDA(cudaMemcpyAsync(&nn, total, sizeof nn, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaMemcpyAsync(&hm, meta, sizeof hm, cudaMemcpyDeviceToHost, s));
    RR_CUDA(cudaStreamSynchronize(s));
    const int64_t n_nodes = nn;
    if (M == 1) hm.depth = 1;
    if (hm.bad_index) {
        set_error("rt_build_tree: %u triangles index vertices out of range", hm.bad_index);
        return RT_ERR_INVALID_ARG;
    }
    if (hm.sah_error) {
        set_error("rt_build_tree_sah: %u inconsistencies in the top levels", hm.sah_error);
        return RT_ERR_INTERNAL;
    }
    if (hm.non_finite) {
        set_error("rt_build_tree: %u triangles have non-finite coordinates", hm.non_finite);
        return RT_ERR_INVALID_ARG;
    }
    if (hm.degenerate) {
        set_error("rt_build_tree: %u triangles have zero area", hm.degenerate);
        return RT_ERR_DEGENERATE_MESH;
    }
    if (hm.min_surf < 0 || hm.min_mat < 0 || hm.max_surf >= (1 << 30)) {
        set_error("rt_build_tree: surface or material ids out of range");
        return RT_ERR_INVALID_ARG;
    }
    const int S = hm.max_surf + 1;
    tree->n_surfaces = S;
    tree->n_materials = hm.max_mat + 1;

    unsigned int mixed = hm.mixed_material;
    if (S > M) {  // sparse surface ids: the tables again, at their full size
        RR_TRY(surface_tables(S));
        RR_CUDA(cudaMemcpyAsync(&mixed, &meta->mixed_material, sizeof mixed, cudaMemcpyDeviceToHost, s));
        RR_CUDA(cudaStreamSynchronize(s));
    }
    if (mixed) {
        set_error("rt_build_tree: %u triangles differ in material from their surface", mixed);
        return RT_ERR_INVALID_ARG;
    }
    if (((uintptr_t)nodes | (uintptr_t)tris) & 31u) {  // the traversal reads them in 32-byte sectors
        set_error("rt_build_tree: the device allocator returned memory that is not 32-byte aligned");
        return RT_ERR_INVALID_ARG;
    }
    tree->depth = hm.depth;
    tree->n_nodes = n_nodes;
    tree->nodes = nodes;
    tree->tris = tris;
    tree->tri_nrm = tri_nrm;
    tree->surf_of = surf_of;
    tree->pos_of = pos_of;
    tree->mat_of_surf = mat_of_surf;
    tree->planes = planes;
    float lo[3], hi[3];
    for (int k = 0; k < 3; k++) {
        unsigned int a = hm.cmin[k], b = hm.cmax[k];
        unsigned int ba = (a & 0x80000000u) ? (a & 0x7FFFFFFFu) : ~a;
        unsigned int bb = (b & 0x80000000u) ? (b & 0x7FFFFFFFu) : ~b;
        memcpy(&lo[k], &ba, 4);
        memcpy(&hi[k], &bb, 4);
    }
    double dd = 0;
    for (int k = 0; k < 3; k++) dd += (double)(hi[k] - lo[k]) * (hi[k] - lo[k]);
    tree->diameter = std::sqrt(dd) > 0 ? std::sqrt(dd) : 1.0;
    tree->owned = keep_arena.release();
    *out = tree;
    tree = nullptr;  // disarm the guard
    return RT_OK;
}

}  // namespace rr

extern "C" rt_status rt_build_tree(const rt_mesh* mesh, void* stream, rt_tree** out) {
    rr::NvtxRange nvtx_range("rt_build_tree");
    rr::clear_error();
    return rr::build_impl(mesh, (cudaStream_t)stream, out);
}

extern "C" rt_status rt_build_tree_median(const rt_mesh* mesh, void* stream, rt_tree** out) {
    rr::NvtxRange nvtx_range("rt_build_tree_median");
    rr::clear_error();
    return rr::build_impl(mesh, (cudaStream_t)stream, out, rr::BUILD_MEDIAN);
}

extern "C" rt_status rt_build_tree_sah(const rt_mesh* mesh, void* stream, rt_tree** out) {
    rr::NvtxRange nvtx_range("rt_build_tree_sah");
    rr::clear_error();
    return rr::build_impl(mesh, (cudaStream_t)stream, out, rr::BUILD_SAH_TOP);
}

extern "C" void rt_tree_free(rt_tree* tree) {
    if (!tree) return;
    for (void* p : tree->owned) rr::dev_free(p, tree->stream);
    delete tree;
}

extern "C" rt_status rt_tree_info(const rt_tree* tree, int64_t* n_nodes, int64_t* n_tris, int32_t* depth,
                                  int32_t* n_surfaces) {
    if (!tree) {
        rr::set_error("rt_tree_info: null tree");
        return RT_ERR_INVALID_ARG;
    }
    if (n_nodes) *n_nodes = tree->n_nodes;
    if (n_tris) *n_tris = tree->n_tris;
    if (depth) *depth = tree->depth;
    if (n_surfaces) *n_surfaces = tree->n_surfaces;
    return RT_OK;
}
