// gm_eyegrid.cu -- the eye grid: per-fixation angular cell lists for the occlusion test.
//
// Every occlusion segment of fixation f starts at its eye e and stays inside its 4 sigma cone, so
// in the fixation's gaze frame (axis r^, lateral axes u, v) the whole segment maps to the single
// point (x/w, y/w) of its sample, w = (q - e).r^. A triangle can block the segment only if its
// image in that frame covers the point and part of it lies nearer than the sample. The grid is an
// R x R array of cells over the square |x/w|, |y/w| <= T (T = cutoff tan(theta), enlarged by
// 1e-4); each cell lists the triangles whose image box (expanded by a rounding margin) meets the
// cell, with a lower bound of their depth w, sorted by that bound. A ray then tests only the
// triangles of its own cell, nearest first, and stops at the first hit or at the first entry that
// lies wholly beyond its sample. The test itself is the BVH path's watertight triangle test, and
// every triangle that test can report is in the list, so the visibility decisions -- and the maps
// -- are the same as with the BVH.
//
// Rounding: vertex depths carry a bound 2^-21 |q - e|_1 (three FMA roundings of a unit-vector dot
// product); image coordinates X = x/w a margin 2^-18 (1 + |X| + |Y|)^2, which bounds the FP32
// error of X on either side (vertex and sample) plus the watertight test's own angular slack
// (about 1e-7 rad) with room to spare. Triangles with a vertex nearer than W0 along the gaze are
// clipped at w = W0 in FP64 (the part nearer than W0 lies outside the cone unless the triangle
// comes within RNEAR of the eye); a triangle within RNEAR of the eye, or one whose image box covers
// more than EG_BIG_CELLS cells, goes to the fixation's all-rays list (cell R*R), walked by every ray
// of the fixation.
//
// Stages: k_eg_spheres (bounding sphere of each run of 256 leaf-order triangles), k_eg_count (one
// block per fixation: cone test of the spheres, then of their triangles, cell counts in shared
// memory; the fixation's total), then per chunk of fixations k_eg_build (the counts again, a
// block-wide scan into the chunk's offset table, the fill, a depth sort of every cell in batches
// staged in shared memory). The host
// reads the totals once to size the chunks (memory) and their entry offsets.
#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "gm_internal.cuh"
#include "gm_scan.cuh"
#include "gm_eyegrid.cuh"

namespace {

constexpr int EG_THREADS = 512;
constexpr int EG_BATCH = 2048;       // surviving 256-triangle blocks handled per round
constexpr int EG_BLOCK = 256;        // leaf-order triangles per bounding sphere
constexpr float EG_W0 = 0.02f;       // clip depth (metres) for triangles reaching toward the eye plane
constexpr int EG_BIG_CELLS = 1024;   // triangles whose box covers more cells go to the all-rays list

struct EgFix {
    float3 e, r, u, v;
};

struct EgGeom {
    float T;      // half width of the grid square in x/w and y/w
    float s;      // R / (2 T)
    float rnear;  // triangles nearer than this to the eye go to the near list
};

__device__ __forceinline__ float3 eg_sub(float4 a, float3 e) { return make_float3(a.x - e.x, a.y - e.y, a.z - e.z); }
__device__ __forceinline__ float eg_dot(float3 a, float3 b) { return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z)); }

// The gaze frame of a fixation: u = unit(r x a) with a the coordinate axis least aligned with r,
// v = r x u.
__device__ void eg_frame(float3 r, float3& u, float3& v) {
    const float ax = fabsf(r.x), ay = fabsf(r.y), az = fabsf(r.z);
    float3 a = (ax <= ay && ax <= az) ? make_float3(1.f, 0.f, 0.f)
                                      : (ay <= az ? make_float3(0.f, 1.f, 0.f) : make_float3(0.f, 0.f, 1.f));
    float3 c = make_float3(r.y * a.z - r.z * a.y, r.z * a.x - r.x * a.z, r.x * a.y - r.y * a.x);
    const float n = rsqrtf(c.x * c.x + c.y * c.y + c.z * c.z);
    u = make_float3(c.x * n, c.y * n, c.z * n);
    v = make_float3(r.y * u.z - r.z * u.y, r.z * u.x - r.x * u.z, r.x * u.y - r.y * u.x);
}

// True when a sphere (centre, radius; radius < 0: empty) cannot meet the cone of half-angle
// atan(T) around the gaze (the conservative test of the accumulation's warp-tile spheres).
__device__ __forceinline__ bool eg_sphere_misses(float4 S, const EgFix& F, float T) {
    if (S.w < 0.f) return true;
    const float qx = S.x - F.e.x, qy = S.y - F.e.y, qz = S.z - F.e.z;
    const float d1c = fmaf(qx, F.r.x, fmaf(qy, F.r.y, qz * F.r.z));
    const float ux = fmaf(qy, F.r.z, -qz * F.r.y);
    const float uy = fmaf(qz, F.r.x, -qx * F.r.z);
    const float uz = fmaf(qx, F.r.y, -qy * F.r.x);
    const float margin = 1e-4f * (fabsf(qx) + fabsf(qy) + fabsf(qz) + S.w);
    const float reach = d1c + S.w;
    const float lim = S.w + fmaf(T, fmaxf(reach, 0.f), margin);
    return reach <= -margin || fmaf(ux, ux, fmaf(uy, uy, uz * uz)) > lim * lim;
}

__device__ __forceinline__ void eg_grow(float X, float Y, float& X0, float& X1, float& Y0, float& Y1) {
    const float q = 1.f + fabsf(X) + fabsf(Y);
    const float m = 3.8146973e-6f * q * q;   // 2^-18 (1 + |X| + |Y|)^2
    X0 = fminf(X0, X - m);
    X1 = fmaxf(X1, X + m);
    Y0 = fminf(Y0, Y - m);
    Y1 = fmaxf(Y1, Y + m);
}

// Image box of the part of the triangle at depth >= EG_W0, in FP64 (Sutherland-Hodgman against
// one plane). False when no part is that deep.
__device__ bool eg_clip_box(float4 a, float4 b, float4 c, const EgFix& F, float& X0, float& X1, float& Y0, float& Y1) {
    const float4 V[3] = {a, b, c};
    double w[3], x[3], y[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const double dx = (double)V[k].x - (double)F.e.x, dy = (double)V[k].y - (double)F.e.y,
                     dz = (double)V[k].z - (double)F.e.z;
        w[k] = dx * F.r.x + dy * F.r.y + dz * F.r.z;
        x[k] = dx * F.u.x + dy * F.u.y + dz * F.u.z;
        y[k] = dx * F.v.x + dy * F.v.y + dz * F.v.z;
    }
    const double w0 = (double)EG_W0;
    bool any = false;
    for (int i = 0; i < 3; ++i) {
        const int j = i == 2 ? 0 : i + 1;
        const bool in_i = w[i] >= w0, in_j = w[j] >= w0;
        if (in_i) {
            eg_grow((float)(x[i] / w[i]), (float)(y[i] / w[i]), X0, X1, Y0, Y1);
            any = true;
        }
        if (in_i != in_j) {
            const double t = (w0 - w[i]) / (w[j] - w[i]);
            eg_grow((float)((x[i] + t * (x[j] - x[i])) / w0), (float)((y[i] + t * (y[j] - y[i])) / w0), X0, X1, Y0,
                    Y1);
            any = true;
        }
    }
    return any;
}

// Which cells of the fixation's grid a triangle can block rays in. False: none (it cannot meet
// the cone, or lies wholly at or behind the eye plane). near: the triangle comes within rnear of
// the eye (it goes to the near list). wlo: a lower bound of its depth along the gaze.
template <int R>
__device__ bool eg_classify(const EgFix& F, const EgGeom& G, float4 a, float4 b, float4 c, int& cx0, int& cx1,
                            int& cy0, int& cy1, bool& near, float& wlo) {
    const float3 D[3] = {eg_sub(a, F.e), eg_sub(b, F.e), eg_sub(c, F.e)};
    float w[3];
    float wl = INFINITY, wh = -INFINITY;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        w[k] = eg_dot(D[k], F.r);
        const float er = 4.7683716e-7f * (fabsf(D[k].x) + fabsf(D[k].y) + fabsf(D[k].z));   // 2^-21 |D|_1
        wl = fminf(wl, w[k] - er);
        wh = fmaxf(wh, w[k] + er);
    }
    if (!(wh > 0.f)) return false;
    wlo = wl;
    // a lower bound of the distance from the eye: the box of the three offsets
    const float lx = fminf(fminf(D[0].x, D[1].x), D[2].x), hx = fmaxf(fmaxf(D[0].x, D[1].x), D[2].x);
    const float ly = fminf(fminf(D[0].y, D[1].y), D[2].y), hy = fmaxf(fmaxf(D[0].y, D[1].y), D[2].y);
    const float lz = fminf(fminf(D[0].z, D[1].z), D[2].z), hz = fmaxf(fmaxf(D[0].z, D[1].z), D[2].z);
    const float cxx = 0.5f * (lx + hx), cyy = 0.5f * (ly + hy), czz = 0.5f * (lz + hz);
    const float rad = 0.5f * sqrtf((hx - lx) * (hx - lx) + (hy - ly) * (hy - ly) + (hz - lz) * (hz - lz));
    const float cen = sqrtf(cxx * cxx + cyy * cyy + czz * czz);
    if (cen - rad * 1.0001f - 1e-5f * (cen + rad) <= G.rnear) {
        near = true;
        return true;
    }
    near = false;
    float X0 = INFINITY, X1 = -INFINITY, Y0 = INFINITY, Y1 = -INFINITY;
    if (wl >= EG_W0) {
#pragma unroll
        for (int k = 0; k < 3; ++k)
            eg_grow(__fdividef(eg_dot(D[k], F.u), w[k]), __fdividef(eg_dot(D[k], F.v), w[k]), X0, X1, Y0, Y1);
    } else if (!eg_clip_box(a, b, c, F, X0, X1, Y0, Y1)) {
        return false;
    }
    if (!(X1 >= -G.T && X0 <= G.T && Y1 >= -G.T && Y0 <= G.T)) return false;
    const float dx = fmaxf(fmaxf(X0, -X1), 0.f), dy = fmaxf(fmaxf(Y0, -Y1), 0.f);
    if (dx * dx + dy * dy > G.T * G.T) return false;
    cx0 = eg_cell_coord(X0, G.s, R);
    cx1 = eg_cell_coord(X1, G.s, R);
    cy0 = eg_cell_coord(Y0, G.s, R);
    cy1 = eg_cell_coord(Y1, G.s, R);
    return true;
}

// A cell can hold an in-cone ray only if its nearest point to the axis is within T: with cell
// bounds at (k - R/2) / s this is an integer test.
template <int R>
__device__ __forceinline__ bool eg_cell_in_disk(int cx, int cy) {
    const int a = max(0, max(cx - R / 2, R / 2 - 1 - cx));
    const int b = max(0, max(cy - R / 2, R / 2 - 1 - cy));
    return a * a + b * b <= (R / 2) * (R / 2);
}

// Both passes over the fixation's candidate triangles. FILL = false: cnt[cell] += 1 per covered
// cell. FILL = true: cnt holds each cell's next position (relative to the fixation's first
// entry); the entry (leaf slot, depth bound) is written there. Cell R*R is the near list.
template <int R, bool FILL>
__device__ void eg_pass(const EgFix& F, const EgGeom& G, const float4* __restrict__ spheres, uint32_t n_blocks,
                        const float4* __restrict__ tris, uint32_t nt, uint32_t* cnt, uint32_t* blist,
                        uint32_t* nsurv, uint2* __restrict__ ent, uint32_t tot, int* __restrict__ err) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (uint32_t b0 = 0; b0 < n_blocks; b0 += EG_BATCH) {
        if (threadIdx.x == 0) *nsurv = 0;
        __syncthreads();
        const uint32_t b1 = min(n_blocks, b0 + (uint32_t)EG_BATCH);
        for (uint32_t bk = b0 + threadIdx.x; bk < b1; bk += EG_THREADS)
            if (!eg_sphere_misses(__ldg(&spheres[bk]), F, G.T)) blist[atomicAdd(nsurv, 1u)] = bk;
        __syncthreads();
        const uint32_t m = *nsurv;
        for (uint32_t q = warp; q < m; q += EG_THREADS / 32) {
            const uint32_t t0 = blist[q] * (uint32_t)EG_BLOCK;
            const uint32_t t1 = min(nt, t0 + (uint32_t)EG_BLOCK);
            for (uint32_t t = t0 + lane; t < t1; t += 32) {
                const float4 a = __ldg(&tris[3 * t]), b = __ldg(&tris[3 * t + 1]), c = __ldg(&tris[3 * t + 2]);
                int cx0, cx1, cy0, cy1;
                bool near;
                float wlo;
                if (!eg_classify<R>(F, G, a, b, c, cx0, cx1, cy0, cy1, near, wlo)) continue;
                const uint2 rec = make_uint2(t, __float_as_uint(wlo));
                // a triangle near the eye, or one whose box covers many cells, goes to the list
                // every ray of the fixation walks (cell R*R) instead of into each of its cells
                if (near || (cx1 - cx0 + 1) * (cy1 - cy0 + 1) > EG_BIG_CELLS) {
                    const uint32_t p = atomicAdd(&cnt[R * R], 1u);
                    if (FILL) {
                        if (p < tot) ent[p] = rec;
                        else atomicCAS(err, 0, GM_DEV_BAD_INDEX);
                    }
                    continue;
                }
                for (int cy = cy0; cy <= cy1; ++cy)
                    for (int cx = cx0; cx <= cx1; ++cx) {
                        if (!eg_cell_in_disk<R>(cx, cy)) continue;
                        const uint32_t p = atomicAdd(&cnt[cy * R + cx], 1u);
                        if (FILL) {
                            if (p < tot) ent[p] = rec;
                            else atomicCAS(err, 0, GM_DEV_BAD_INDEX);
                        }
                    }
            }
        }
        __syncthreads();
    }
}

__device__ __forceinline__ EgFix eg_load_fix(const float4* __restrict__ fix, const float4* basis, uint32_t f) {
    const float4 F0 = fix[2 * f], F1 = fix[2 * f + 1];
    EgFix F;
    F.e = make_float3(F0.x, F0.y, F0.z);
    F.r = make_float3(F1.x, F1.y, F1.z);
    if (basis) {
        const float4 U = basis[2 * f], V = basis[2 * f + 1];
        F.u = make_float3(U.x, U.y, U.z);
        F.v = make_float3(V.x, V.y, V.z);
    } else {
        eg_frame(F.r, F.u, F.v);
    }
    return F;
}

// Bounding sphere (box centre, half diagonal) of each run of EG_BLOCK leaf-order triangles.
__global__ void k_eg_spheres(const float4* __restrict__ tris, uint32_t nt, uint32_t n_blocks, float4* __restrict__ out) {
    const uint32_t bk = blockIdx.x * blockDim.x + threadIdx.x;
    if (bk >= n_blocks) return;
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    const uint32_t t1 = min(nt, (bk + 1) * (uint32_t)EG_BLOCK);
    for (uint32_t t = bk * (uint32_t)EG_BLOCK; t < t1; ++t)
        for (int k = 0; k < 3; ++k) {
            const float4 p = tris[3 * t + k];
            lo[0] = fminf(lo[0], p.x), lo[1] = fminf(lo[1], p.y), lo[2] = fminf(lo[2], p.z);
            hi[0] = fmaxf(hi[0], p.x), hi[1] = fmaxf(hi[1], p.y), hi[2] = fmaxf(hi[2], p.z);
        }
    out[bk] = lo[0] <= hi[0]
                  ? make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]),
                                0.5f * sqrtf((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                             (hi[2] - lo[2]) * (hi[2] - lo[2])) * 1.0001f)
                  : make_float4(0.f, 0.f, 0.f, -1.f);
}

// One block per fixation of the sorted list: its gaze frame into basis, its entry count (cells
// and near list) into totals. Fixations past the valid count get 0.
template <int R>
__global__ void __launch_bounds__(EG_THREADS) k_eg_count(const float4* __restrict__ fix,
                                                         const uint32_t* __restrict__ n_valid,
                                                         const float4* __restrict__ spheres, uint32_t n_blocks,
                                                         const float4* __restrict__ tris, uint32_t nt, EgGeom G,
                                                         float4* __restrict__ basis, uint32_t* __restrict__ totals,
                                                         int* __restrict__ err) {
    extern __shared__ uint32_t eg_sm[];
    uint32_t* cnt = eg_sm;
    uint32_t* blist = eg_sm + R * R + 1;
    __shared__ uint32_t nsurv;
    const uint32_t f = blockIdx.x;
    if (f >= *n_valid) {
        if (threadIdx.x == 0) totals[f] = 0;
        return;
    }
    const EgFix F = eg_load_fix(fix, nullptr, f);
    if (threadIdx.x == 0) {
        basis[2 * f] = make_float4(F.u.x, F.u.y, F.u.z, 0.f);
        basis[2 * f + 1] = make_float4(F.v.x, F.v.y, F.v.z, 0.f);
    }
    for (int c = threadIdx.x; c <= R * R; c += EG_THREADS) cnt[c] = 0;
    __syncthreads();
    eg_pass<R, false>(F, G, spheres, n_blocks, tris, nt, cnt, blist, &nsurv, nullptr, 0, err);
    uint32_t s = 0;
    for (int c = threadIdx.x; c <= R * R; c += EG_THREADS) s += cnt[c];
    uint32_t tot;
    block_excl_scan<uint32_t, EG_THREADS>(s, &tot);
    if (threadIdx.x == 0) totals[f] = tot;
}

constexpr int EG_STAGE = 4096;       // entries staged in shared memory for the per-cell sorts

// In-place shell sort of one cell's entries by depth bound, one thread (gaps 701 ... 1: plain
// insertion sort for the short lists that are the rule).
__device__ void eg_sort(uint2* a, uint32_t n) {
    const uint32_t gaps[8] = {701, 301, 132, 57, 23, 10, 4, 1};
#pragma unroll 1
    for (int gi = 0; gi < 8; ++gi) {
        const uint32_t g = gaps[gi];
        if (g >= n) continue;
        for (uint32_t i = g; i < n; ++i) {
            const uint2 t = a[i];
            const float k = __uint_as_float(t.y);
            uint32_t j = i;
            while (j >= g && __uint_as_float(a[j - g].y) > k) {
                a[j] = a[j - g];
                j -= g;
            }
            a[j] = t;
        }
    }
}

// One block per fixation [f0, f0 + gridDim.x): offsets (R*R + 2 per fixation: cell starts, the
// near list's start, its end) into cells, entries from base[f - f0] on into ent, sorted by depth
// bound within every cell.
template <int R>
__global__ void __launch_bounds__(EG_THREADS) k_eg_build(const float4* __restrict__ fix, uint32_t f0,
                                                         const float4* __restrict__ spheres, uint32_t n_blocks,
                                                         const float4* __restrict__ tris, uint32_t nt, EgGeom G,
                                                         const float4* __restrict__ basis,
                                                         const uint32_t* __restrict__ base,
                                                         const uint32_t* __restrict__ totals,
                                                         uint32_t* __restrict__ cells, uint2* __restrict__ ent,
                                                         int* __restrict__ err) {
    extern __shared__ uint32_t eg_sm[];
    uint32_t* cnt = eg_sm;
    uint32_t* blist = eg_sm + R * R + 1;
    __shared__ uint32_t nsurv;
    constexpr int NC = R * R + 1;                       // cells + near list
    constexpr int PER = (NC + EG_THREADS - 1) / EG_THREADS;
    const uint32_t fl = blockIdx.x, f = f0 + fl;
    const EgFix F = eg_load_fix(fix, basis, f);
    const uint32_t b = base[fl], tot = totals[f];
    uint32_t* my = cells + (size_t)fl * (R * R + 2);
    uint2* e = ent + b;
    for (int c = threadIdx.x; c < NC; c += EG_THREADS) cnt[c] = 0;
    __syncthreads();
    eg_pass<R, false>(F, G, spheres, n_blocks, tris, nt, cnt, blist, &nsurv, nullptr, 0, err);
    // exclusive scan of the counts: thread t owns cells [t PER, (t + 1) PER)
    uint32_t s = 0;
    const int c0 = threadIdx.x * PER;
#pragma unroll 1
    for (int k = 0; k < PER; ++k)
        if (c0 + k < NC) s += cnt[c0 + k];
    uint32_t all;
    uint32_t run = block_excl_scan<uint32_t, EG_THREADS>(s, &all);
#pragma unroll 1
    for (int k = 0; k < PER; ++k) {
        const int c = c0 + k;
        if (c < NC) {
            const uint32_t n = cnt[c];
            cnt[c] = run;
            my[c] = b + run;
            run += n;
        }
    }
    if (threadIdx.x == 0) {
        my[NC] = b + all;
        if (all != tot) atomicCAS(err, 0, GM_DEV_BAD_INDEX);   // the two passes must agree
    }
    __syncthreads();
    eg_pass<R, true>(F, G, spheres, n_blocks, tris, nt, cnt, blist, &nsurv, e, min(all, tot), err);
    __syncthreads();
    // after the fill cnt[c] is the end of cell c, i.e. the start of cell c + 1. The cells are sorted
    // in batches of consecutive cells staged in shared memory (their entries are contiguous): one
    // thread per cell, insertion or shell sort; a cell longer than the stage is sorted in place
    uint2* stage = reinterpret_cast<uint2*>(eg_sm + (((size_t)R * R + 1 + EG_BATCH + 1) & ~(size_t)1));
    __shared__ int s_c1;
    for (int c0 = 0; c0 < NC;) {
        const uint32_t st0 = c0 == 0 ? 0u : cnt[c0 - 1];
        if (threadIdx.x == 0) {
            // the last cell c1 - 1 whose end is within EG_STAGE entries of st0 (binary search; ends
            // are non-decreasing), at least one cell
            int lo = c0, hi = NC - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (cnt[mid] - st0 <= (uint32_t)EG_STAGE) lo = mid;
                else hi = mid - 1;
            }
            s_c1 = lo + 1;
        }
        __syncthreads();
        const int c1 = s_c1;
        const uint32_t en1 = min(cnt[c1 - 1], all);
        if (en1 - st0 > (uint32_t)EG_STAGE) {   // one cell longer than the stage
            if (threadIdx.x == 0) eg_sort(e + st0, en1 - st0);
        } else {
            for (uint32_t k = threadIdx.x; k < en1 - st0; k += EG_THREADS) stage[k] = e[st0 + k];
            __syncthreads();
            for (int c = c0 + threadIdx.x; c < c1; c += EG_THREADS) {
                const uint32_t a = (c == 0 ? 0u : cnt[c - 1]) - st0, b = min(cnt[c], all) - st0;
                if (b > a + 1) eg_sort(stage + a, b - a);
            }
            __syncthreads();
            for (uint32_t k = threadIdx.x; k < en1 - st0; k += EG_THREADS) e[st0 + k] = stage[k];
        }
        __syncthreads();
        c0 = c1;
    }
}

// counts (R*R + 1), the surviving-block list, and (build only) the sort stage
template <int R>
size_t eg_smem(bool build) {
    const size_t b = sizeof(uint32_t) * ((size_t)R * R + 1 + EG_BATCH);
    return build ? ((b + 7) & ~(size_t)7) + sizeof(uint2) * EG_STAGE : b;
}

template <int R>
gm_status eg_configure(int device) {
    static int done = -1;
    if (done == device) return GM_OK;
    GM_TRY_CUDA(cudaFuncSetAttribute(k_eg_count<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eg_smem<R>(false)));
    GM_TRY_CUDA(cudaFuncSetAttribute(k_eg_build<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)eg_smem<R>(true)));
    done = device;
    return GM_OK;
}

EgGeom eg_geom(const EyeGrid& g) {
    EgGeom G;
    G.T = g.T;
    G.s = g.s;
    G.rnear = EG_W0 * std::sqrt(1.f + 2.f * g.T * g.T) * 1.001f + 1e-6f;
    return G;
}

}  // namespace

gm_status eg_prepare(gm_scene* sc, const float4* fix, const uint32_t* n_valid_dev, uint32_t nf, float tan_phi,
                     uint32_t R, uint64_t entry_budget, cudaStream_t s, EyeGrid* g, int* launches) {
    if (R != 64 && R != 128) return gm_set_error(GM_ERR_INVALID_ARG, "eye grid: resolution must be 64 or 128");
    g->R = R;
    g->T = tan_phi * 1.0001f;
    g->s = (float)R / (2.f * g->T);
    g->nf = nf;
    const uint32_t nt = sc->n_tris;
    g->n_blocks = gm_div_up(nt, EG_BLOCK);
    if (R == 64) GM_TRY(eg_configure<64>(sc->ctx->device));
    else GM_TRY(eg_configure<128>(sc->ctx->device));
    GM_TRY(gm_alloc((void**)&g->spheres, sizeof(float4) * std::max<uint32_t>(1, g->n_blocks), s));
    GM_TRY(gm_alloc((void**)&g->basis, sizeof(float4) * 2 * std::max<uint32_t>(1, nf), s));
    GM_TRY(gm_alloc((void**)&g->totals, sizeof(uint32_t) * std::max<uint32_t>(1, nf), s));
    const EgGeom G = eg_geom(*g);
    if (g->n_blocks > 0) {
        k_eg_spheres<<<gm_div_up(g->n_blocks, 128), 128, 0, s>>>(sc->bvh_tris, nt, g->n_blocks, g->spheres);
        ++*launches;
    }
    if (nf > 0) {
        if (R == 64)
            k_eg_count<64><<<nf, EG_THREADS, eg_smem<64>(false), s>>>(fix, n_valid_dev, g->spheres, g->n_blocks,
                                                                  sc->bvh_tris, nt, G, g->basis, g->totals,
                                                                  sc->ctx->dev_err);
        else
            k_eg_count<128><<<nf, EG_THREADS, eg_smem<128>(false), s>>>(fix, n_valid_dev, g->spheres, g->n_blocks,
                                                                    sc->bvh_tris, nt, G, g->basis, g->totals,
                                                                    sc->ctx->dev_err);
        ++*launches;
    }
    GM_TRY_CUDA(cudaGetLastError());
    // the host sizes the chunks: one read of the valid count and the per-fixation totals
    uint32_t nv = 0;
    g->h_tot.assign(nf, 0u);
    GM_TRY_CUDA(cudaMemcpyAsync(&nv, n_valid_dev, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    if (nf > 0) GM_TRY_CUDA(cudaMemcpyAsync(g->h_tot.data(), g->totals, sizeof(uint32_t) * nf, cudaMemcpyDeviceToHost, s));
    GM_TRY_CUDA(cudaStreamSynchronize(s));
    g->n_valid = nv;
    // chunks: at most 1 GiB of offset tables and `entry_budget` entries (and 2^31 - 1) each
    const uint64_t per_fix = (uint64_t)R * R + 2;
    const uint64_t fix_cap = std::max<uint64_t>(1, (1ull << 30) / (per_fix * sizeof(uint32_t)));
    const uint64_t ent_cap = std::min<uint64_t>(entry_budget, 0x7fffffffull);
    g->chunk.assign(1, 0u);
    g->h_base.assign(nv, 0u);
    uint64_t acc = 0;
    uint32_t c_begin = 0;
    g->max_entries = 0;
    g->max_fix = 0;
    for (uint32_t f = 0; f < nv; ++f) {
        const uint64_t t = g->h_tot[f];
        if (t > 0x7fffffffull)
            return gm_set_error(GM_ERR_UNSUPPORTED, "eye grid: one fixation needs " + std::to_string(t) +
                                                        " entries (limit 2^31 - 1)");
        // a chunk holds at least one fixation, however large
        if (f > c_begin && (acc + t > ent_cap || f - c_begin >= fix_cap)) {
            g->chunk.push_back(f);
            g->max_entries = std::max(g->max_entries, acc);
            g->max_fix = std::max(g->max_fix, f - c_begin);
            c_begin = f;
            acc = 0;
        }
        g->h_base[f] = (uint32_t)acc;
        acc += t;
    }
    if (nv > 0) {
        g->chunk.push_back(nv);
        g->max_entries = std::max(g->max_entries, acc);
        g->max_fix = std::max(g->max_fix, nv - c_begin);
    }
    if (nv > 0) {
        GM_TRY(gm_alloc((void**)&g->cells, sizeof(uint32_t) * per_fix * g->max_fix, s));
        GM_TRY(gm_alloc((void**)&g->ent, sizeof(uint2) * std::max<uint64_t>(1, g->max_entries), s));
        GM_TRY(gm_alloc((void**)&g->base, sizeof(uint32_t) * g->max_fix, s));
    }
    return GM_OK;
}

gm_status eg_build_chunk(gm_scene* sc, const float4* fix, EyeGrid* g, uint32_t k, cudaStream_t s, int* launches) {
    const uint32_t f0 = g->chunk[k], f1 = g->chunk[k + 1];
    if (f1 <= f0) return GM_OK;
    // per chunk fixation: its first entry in the chunk's buffer (pageable source: the copy has
    // consumed it when the call returns)
    GM_TRY_CUDA(cudaMemcpyAsync(g->base, g->h_base.data() + f0, sizeof(uint32_t) * (f1 - f0), cudaMemcpyHostToDevice, s));
    const EgGeom G = eg_geom(*g);
    if (g->R == 64)
        k_eg_build<64><<<f1 - f0, EG_THREADS, eg_smem<64>(true), s>>>(fix, f0, g->spheres, g->n_blocks, sc->bvh_tris,
                                                                   sc->n_tris, G, g->basis, g->base, g->totals,
                                                                   g->cells, g->ent, sc->ctx->dev_err);
    else
        k_eg_build<128><<<f1 - f0, EG_THREADS, eg_smem<128>(true), s>>>(fix, f0, g->spheres, g->n_blocks, sc->bvh_tris,
                                                                     sc->n_tris, G, g->basis, g->base, g->totals,
                                                                     g->cells, g->ent, sc->ctx->dev_err);
    ++*launches;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

void eg_free(EyeGrid* g, cudaStream_t s) {
    for (void* p : {(void*)g->spheres, (void*)g->basis, (void*)g->totals, (void*)g->cells, (void*)g->ent,
                    (void*)g->base})
        if (p) cudaFreeAsync(p, s);
    *g = EyeGrid();
}
