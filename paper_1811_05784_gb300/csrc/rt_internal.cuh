// rt_internal.cuh -- shared definitions of the roomrays CUDA library.
//
// Handles (rt_tree, rt_image_sources, rt_rir), device allocation, error
// reporting and the generic device primitives (radix sort, scan) used by the
// build, trace and histogram stages.
#pragma once

#include <nvtx3/nvToolsExt.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <utility>
#include <vector>

#include "../../include/roomrays.h"

namespace rr {

// NVTX range over one call of the C ABI, for timeline tools (nsys, ncu's
// range filters); without a tool attached the push and pop do nothing.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};


// ---------------------------------------------------------------------------
// errors
// ---------------------------------------------------------------------------
void set_error(const char* fmt, ...);
void clear_error();

struct Failure {
    rt_status status;
};

// Throw-free control flow inside the library: helpers return rt_status and
// the RR_TRY macro propagates it.
#define RR_TRY(expr)                        \
    do {                                    \
        rt_status _s = (expr);              \
        if (_s != RT_OK) return _s;         \
    } while (0)

rt_status cuda_status(cudaError_t e, const char* what);
#define RR_CUDA(call) RR_TRY(::rr::cuda_status((call), #call))

// ---------------------------------------------------------------------------
// device memory
// ---------------------------------------------------------------------------
void* dev_alloc(size_t bytes, cudaStream_t s);
// true if the last dev_alloc on this thread failed because the caller's
// allocator returned a block that is not 256-byte aligned
bool last_alloc_misaligned();
void dev_free(void* p, cudaStream_t s);

// Owns device allocations made during one call; frees them on scope exit
// unless released to a handle.
struct Arena {
    cudaStream_t stream;
    std::vector<void*> ptrs;
    explicit Arena(cudaStream_t s) : stream(s) {}
    ~Arena() {
        for (void* p : ptrs) dev_free(p, stream);
    }
    template <class T>
    rt_status alloc(T** out, size_t count) {
        size_t bytes = count * sizeof(T);
        if (bytes == 0) bytes = 16;
        void* p = dev_alloc(bytes, stream);
        if (!p) {
            if (last_alloc_misaligned())
                set_error("device allocation of %zu bytes failed: the allocator's block is not 256-byte aligned",
                          bytes);
            else
                set_error("device allocation of %zu bytes failed", bytes);
            return RT_ERR_OOM;
        }
        ptrs.push_back(p);
        *out = static_cast<T*>(p);
        return RT_OK;
    }
    // hand every allocation over to a handle (which frees them later)
    std::vector<void*> release() {
        std::vector<void*> v;
        v.swap(ptrs);
        return v;
    }
};

// Several arrays carved out of one allocation (256-byte aligned slices): fewer
// allocator calls, and blocks of the same size from one call to the next, so
// the stream-ordered pool reuses them instead of growing.
struct Carve {
    size_t total = 0;
    std::vector<std::pair<size_t, void*>> parts;  // offset, address of the caller's pointer
    std::vector<void (*)(void*, unsigned char*)> setters;
    template <class T>
    void add(T** out, size_t count) {
        const size_t off = (total + 255) & ~(size_t)255;
        total = off + std::max<size_t>(count * sizeof(T), 16);
        parts.emplace_back(off, (void*)out);
        setters.push_back([](void* o, unsigned char* p) { *static_cast<T**>(o) = reinterpret_cast<T*>(p); });
    }
    rt_status alloc(Arena& ar) {
        unsigned char* base;
        RR_TRY(ar.alloc(&base, total));
        for (size_t k = 0; k < parts.size(); k++) setters[k](parts[k].second, base + parts[k].first);
        return RT_OK;
    }
};

// ---------------------------------------------------------------------------
// device primitives
// ---------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs on key bits [begin_bit, end_bit).
// keys/vals hold the input; alt buffers are scratch of the same size.  The
// sorted pairs end up in keys/vals.  temp: scratch of sort_temp_bytes(n).
size_t sort_temp_bytes(int64_t n);
rt_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt,
                           int64_t n, int begin_bit, int end_bit, void* temp, cudaStream_t s);

// Exclusive prefix sum of n uint32 values (in may equal out); the total is
// written to *total_dev (device pointer) when not null.
size_t scan_temp_bytes(int64_t n);
rt_status exclusive_scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* total_dev, void* temp,
                             cudaStream_t s);

int device_sm_count();

// process-wide count of kernel launches made by the library
void note_launch();
long long launch_count();

}  // namespace rr

#define RR_LAUNCH(kernel, grid, block, smem, stream, ...)               \
    do {                                                                \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__);     \
        ::rr::note_launch();                                            \
    } while (0)

// FP64 plane n.x = d of a surface (unit normal n)
struct alignas(32) Plane {
    double x, y, z, w;
};

// ---------------------------------------------------------------------------
// handles
// ---------------------------------------------------------------------------
struct rt_tree {
    int64_t n_tris = 0;
    int64_t n_nodes = 0;
    int32_t n_surfaces = 0;
    int32_t depth = 0;
    int32_t n_materials = 0;      // max material id + 1
    double diameter = 1.0;
    // device arrays
    float4* nodes = nullptr;      // [n_nodes][8]: four child boxes (SoA) + refs + count (128 B / node)
    float4* tris = nullptr;       // [n_tris][3] tree order: v0 (w = id), v1 (w = surface id), v2
    float4* tri_nrm = nullptr;    // [n_tris] by id: unit normal (float32 of FP64), w = surface id bits
    int32_t* surf_of = nullptr;   // [n_tris] by id
    int32_t* pos_of = nullptr;    // [n_tris] by id: position of the triangle in tree order
    int32_t* mat_of_surf = nullptr;  // [n_surfaces]
    Plane* planes = nullptr;      // [n_surfaces] FP64 plane n.x = d
    std::vector<void*> owned;
    cudaStream_t stream = nullptr;
};

struct rt_image_sources {
    rt_is_view v{};
    int32_t n_rcv = 0;
    double c = 343.2;
    std::vector<void*> owned;
    cudaStream_t stream = nullptr;
};

struct rt_response {
    rt_response_view v{};
    std::vector<void*> owned;
    cudaStream_t stream = nullptr;
};

// Node reference encoding shared by the build and the traversal.
//   ref >= 0 : internal node index
//   ref <  0 : leaf, first triangle (tree order) = ~ref, count in the node's cnt field
#define RR_LEAF_MAX 2
