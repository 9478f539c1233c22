// gm_internal.cuh -- internal types and helpers of libgazemap (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/gazemap.h"

// ------------------------------------------------------------------------------------------
// error state (thread-local message, see gm_last_error)
// ------------------------------------------------------------------------------------------
gm_status gm_set_error(gm_status st, const std::string& msg);
gm_status gm_cuda_error(cudaError_t e, const char* what);

#define GM_TRY_CUDA(expr)                                                  \
    do {                                                                   \
        cudaError_t _e = (expr);                                           \
        if (_e != cudaSuccess) return gm_cuda_error(_e, #expr);            \
    } while (0)

#define GM_TRY(expr)                                                       \
    do {                                                                   \
        gm_status _s = (expr);                                             \
        if (_s != GM_OK) return _s;                                        \
    } while (0)

// Device-side fault codes written to gm_ctx::dev_err (first writer wins).
enum { GM_DEV_OK = 0, GM_DEV_STACK_OVERFLOW = 1, GM_DEV_BAD_INDEX = 2, GM_DEV_WAIT_TIMEOUT = 4,
       GM_DEV_TOO_MANY_SAMPLES = 8 };

struct gm_ctx {
    int device = 0;
    int n_sm = 0;
    int* dev_err = nullptr;      // one int in device memory, zero when healthy
    unsigned long long launches = 0;  // kernels launched through this context (host count)
    void* noalloc_scratch = nullptr;  // device address of the allocation-free entry point's array
};

struct gm_scene {
    gm_ctx* ctx = nullptr;
    uint32_t n_tris = 0;
    uint32_t n_meshes = 0;
    float4* tri_canon = nullptr;     // n_tris x 3 float4 (v0, v1, v2), stored (mesh) order
    uint32_t* tri_mesh = nullptr;    // n_tris mesh index
    uint32_t* mesh_object = nullptr; // n_meshes object id
    double* mesh_inv = nullptr;      // n_meshes x 12: world -> local affine map (row-major 3x4)
    bool mesh_inv_ok = true;         // every mesh transform was invertible
    float4* tri_local = nullptr;     // n_tris x 3 float4 mesh-local vertices (scenes built dynamic only)
    uint64_t zb_pairs_per_fix = 0;   // z-buffer path: raster pairs per fixation seen last (capacity hint)
    float4* nodes = nullptr;         // (n_tris - 1) x 4 float4: child boxes + child links
    float4* bvh_tris = nullptr;      // n_tris x 3 float4 in leaf order, v0.w = global tri id
    uint32_t depth = 0;
    // 4-wide collapse of the binary tree: the binary nodes at even depth, each holding up to four
    // children (its grandchildren) as 8 float4: lo.x[4] hi.x[4] lo.y[4] hi.y[4] lo.z[4] hi.z[4]
    // links[4] (int bits; >= 0 node, < 0 leaf ~slot, INT_MIN empty) and one spare float4
    float4* nodes4 = nullptr;
    uint32_t n4 = 0;
    float box_lo[3], box_hi[3];      // world bounds of all vertices
};

enum { GM_SAMPLES_PHILOX = 0, GM_SAMPLES_GRID = 1, GM_SAMPLES_POINTS = 2 };

struct gm_samples {
    gm_scene* scene = nullptr;
    uint64_t n = 0;
    float4* pos = nullptr;           // n: (x, y, z, global tri id as bits), stored order
    float2* bary = nullptr;          // n: (b1, b2); null for explicit points
    int64_t* tri_offset = nullptr;   // n_tris + 1; null for explicit points
    int kind = 0;                    // GM_SAMPLES_PHILOX, GM_SAMPLES_GRID or GM_SAMPLES_POINTS
    uint2 key{0u, 0u};               // Philox key (seed) of a Philox sample set
    uint32_t session = 0;            // Philox counter word of a Philox sample set
    uint32_t* res = nullptr;         // n_tris grid resolutions of a grid sample set
    // spatial work order for the accumulation (Morton order of the sample positions)
    float4* work_pos = nullptr;      // n, work order
    uint32_t* work_idx = nullptr;    // n, stored index of each work-order sample
};

struct gm_map {
    gm_ctx* ctx = nullptr;
    uint32_t W = 1;
    uint64_t ns = 0;
    float* values = nullptr;           // W x ns
    unsigned int* max_bits = nullptr;  // W (bit pattern of a non-negative float)
    unsigned long long* counters = nullptr;  // [0] in_cone [1] visible [2] debug cursor [3] fixations used
                                             // [4] BVH nodes visited [5] triangles tested
                                             // [6] next warp tile of the persistent kernel
    uint32_t* dbg_sample = nullptr;
    uint32_t* dbg_fix = nullptr;
    uint8_t* dbg_vis = nullptr;
    float* dbg_g = nullptr;
    uint64_t dbg_cap = 0;
    gm_map_stats stats{};
    bool timing = false;
    bool zbuffer = false;                    // made by gm_accumulate_zbuffer: 16 counters, [8..11] its own
    cudaEvent_t ev[6] = {};
    cudaStream_t stream = nullptr;
};

// ------------------------------------------------------------------------------------------
// host helpers
// ------------------------------------------------------------------------------------------
bool gm_is_device_ptr(const void* p);
// Make `src` (host or device, `bytes` long) available on the device: returns src itself when
// it already is device memory, else a fresh stream-ordered allocation holding a copy
// (*owned set; free with cudaFreeAsync on the same stream).
gm_status gm_stage_to_device(const void* src, size_t bytes, cudaStream_t s, void** dev, bool* owned);
gm_status gm_copy_out(void* dst, const void* dev_src, size_t bytes, cudaStream_t s);
gm_status gm_alloc(void** p, size_t bytes, cudaStream_t s);

// ------------------------------------------------------------------------------------------
// sort / scan (gm_sort.cu)
// ------------------------------------------------------------------------------------------
// Stable LSD radix sort of (key, value) pairs on `bits` low key bits. keys/vals are sorted in
// place (ping-pong through temporaries allocated on `s`).
gm_status gm_radix_sort_u64(uint64_t* keys, uint32_t* vals, uint32_t n, int bits, cudaStream_t s,
                            int* launches);
gm_status gm_radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t n, int bits, cudaStream_t s,
                            int* launches);
// The same sort with caller-provided temporaries: tmp_keys/tmp_vals of n entries and a histogram
// table of gm_radix_sort_u32_hist_words(n) words. Allocates nothing (usable under graph capture).
size_t gm_radix_sort_u32_hist_words(uint32_t n);
gm_status gm_radix_sort_u32_prealloc(uint32_t* keys, uint32_t* vals, uint32_t n, int bits, uint32_t* tmp_keys,
                                     uint32_t* tmp_vals, uint32_t* hist, cudaStream_t s, int* launches);
// Inclusive prefix sum of int64 values in place.
gm_status gm_inclusive_scan_i64(int64_t* data, uint32_t n, cudaStream_t s, int* launches);

// ------------------------------------------------------------------------------------------
// device helpers
// ------------------------------------------------------------------------------------------
__device__ __forceinline__ unsigned int gm_lanemask_lt() {
    unsigned int m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

static inline uint32_t gm_div_up(uint64_t a, uint64_t b) { return (uint32_t)((a + b - 1) / b); }
