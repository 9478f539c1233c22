// gm_eyegrid.cuh -- the eye grid (per-fixation angular cell lists for the occlusion test): the
// cell mapping shared by its build and its query, and the host interface of gm_eyegrid.cu.
#pragma once

#include <vector>

#include "gm_internal.cuh"

// Grid cell coordinate of x/w along one axis (clamped; NaN goes to 0). Monotone in x/w, so a
// point inside a margin-expanded box always falls in one of the box's cells.
static __device__ __forceinline__ int eg_cell_coord(float xw, float s, int R) {
    return (int)floorf(fminf(fmaxf(fmaf(xw, s, 0.5f * (float)R), 0.f), (float)R - 0.5f));
}

struct EyeGrid {
    uint32_t R = 0;             // cells per side (64 or 128)
    float T = 0.f;              // half width of the grid square in x/w and y/w
    float s = 0.f;              // R / (2 T)
    uint32_t nf = 0;            // fixations in the sorted list
    uint32_t n_valid = 0;       // of which valid (the first n_valid)
    uint32_t n_blocks = 0;      // runs of 256 leaf-order triangles
    float4* spheres = nullptr;  // n_blocks bounding spheres
    float4* basis = nullptr;    // 2 per fixation: (u, 0), (v, 0)
    uint32_t* totals = nullptr; // entries per fixation
    uint32_t* cells = nullptr;  // per fixation of a chunk: R*R + 2 offsets
    uint2* ent = nullptr;       // entries of a chunk
    uint32_t* base = nullptr;   // per fixation of a chunk: its first entry
    std::vector<uint32_t> h_tot, h_base;
    std::vector<uint32_t> chunk;   // chunk boundaries over [0, n_valid)
    uint64_t max_entries = 0;
    uint32_t max_fix = 0;
};

// Frames, spheres and entry counts of every fixation of the sorted, packed list `fix` (nf
// fixations, *n_valid_dev valid), then (host) the chunks: at most `entry_budget` entries each.
// Synchronises the stream once (to read the counts).
gm_status eg_prepare(gm_scene* sc, const float4* fix, const uint32_t* n_valid_dev, uint32_t nf, float tan_phi,
                     uint32_t R, uint64_t entry_budget, cudaStream_t s, EyeGrid* g, int* launches);
// The cell lists of chunk k.
gm_status eg_build_chunk(gm_scene* sc, const float4* fix, EyeGrid* g, uint32_t k, cudaStream_t s, int* launches);
void eg_free(EyeGrid* g, cudaStream_t s);
