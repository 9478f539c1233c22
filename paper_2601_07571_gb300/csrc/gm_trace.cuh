// gm_trace.cuh -- device code shared by the single-map and the batched accumulation kernels:
// the occlusion queries (binary and 4-wide BVH, or the per-fixation eye grid; one watertight
// triangle test for all of them) and the per-warp tile body that runs the cone test, the ray
// queue, the Gaussian and the compensated sums for 32*SPT consecutive work-order samples over a
// range of the fixation list.
#pragma once

#include "gm_internal.cuh"
#include "gm_eyegrid.cuh"

namespace {

constexpr int ACC_THREADS = 256;
constexpr int SPT = 4;            // samples per thread
constexpr int STACK = 64;         // binary traversal stack (the build refuses trees deeper than 64)
constexpr int STACK4 = 96;        // 4-wide traversal stack: at most 3 pushes per level, <= 32 levels
constexpr int LINK_EMPTY = (int)0x80000000;

struct AccParams {
    float C2;     // log2(e) / (2 tan^2 theta)
    float K;      // (cutoff tan theta)^2
    float tmax;   // 1 - eps_rel
    uint32_t ns;
    uint32_t W;
    uint32_t nt;
    uint64_t dbg_cap;
    // warp tile t covers samples base(t) + k * stride + lane (k < SPT) with group G:
    // base = (t / G) * WARP_TILE * G + (t % G) * 32, stride = 32 * G. G = 1: 128 consecutive
    // work-order samples; G = 8: four runs of 32, spread over 1024 samples shared by 8 tiles.
    uint32_t group = 1;
    uint32_t tile_cull = 1;   // skip fixations whose cone misses the warp tile's bounding sphere
    float tanphi = 0.f;       // cutoff tan theta, slightly enlarged (the sphere test's cone)
    // fixations [f0, min(f1, n_valid)) of the sorted list are processed by this launch; with
    // carry_in the sums start from `carry` (and the window of fixation f0 - 1 is still open),
    // with carry_out they are saved there instead of being flushed at the end
    uint32_t f0 = 0, f1 = 0xffffffffu;
    uint32_t carry_in = 0, carry_out = 0;
    float2* carry = nullptr;  // per work-order sample: (sum, compensation)
    // eye grid of the fixations [f0, f1) (occlusion by cell lists instead of the BVH)
    const float4* eg_basis = nullptr;   // per fixation (global index): (u, 0), (v, 0)
    const uint32_t* eg_cells = nullptr; // per fixation of the launch: R*R + 2 entry offsets
    const uint2* eg_ent = nullptr;      // (leaf slot, depth lower bound bits), depth-sorted per cell
    uint32_t eg_R = 0;
    float eg_s = 0.f;                   // cells per unit of x/w: R / (2 T)
};

struct DebugOut {
    uint32_t* sample;
    uint32_t* fix;
    uint8_t* vis;
    float* g;
    const uint32_t* fix_orig;
};

// ------------------------------------------------------------------------------------------
// occlusion: BVH any-hit with a watertight segment/triangle test
// ------------------------------------------------------------------------------------------
struct Ray {
    float3 o, d;
    float3 idir, oidir;   // slab test: t = lo * idir - o * idir
    float tmax, tmax_box;
    int kx, ky, kz;
    float Sx, Sy, Sz;
};

__device__ __forceinline__ float comp(const float3& v, int k) { return k == 0 ? v.x : (k == 1 ? v.y : v.z); }

__device__ __forceinline__ void make_ray(Ray& R, float3 o, float3 d, float tmax) {
    R.o = o;
    R.d = d;
    R.tmax = tmax;
    R.tmax_box = tmax * 1.0001f;
    const float tiny = 1e-20f;
    float dx = fabsf(d.x) < tiny ? copysignf(tiny, d.x) : d.x;
    float dy = fabsf(d.y) < tiny ? copysignf(tiny, d.y) : d.y;
    float dz = fabsf(d.z) < tiny ? copysignf(tiny, d.z) : d.z;
    R.idir = make_float3(1.f / dx, 1.f / dy, 1.f / dz);
    R.oidir = make_float3(o.x * R.idir.x, o.y * R.idir.y, o.z * R.idir.z);
    float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = (ax > ay) ? (ax > az ? 0 : 2) : (ay > az ? 1 : 2);
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (comp(d, kz) < 0.f) {
        int t = kx;
        kx = ky;
        ky = t;
    }
    R.kx = kx;
    R.ky = ky;
    R.kz = kz;
    float dkz = comp(d, kz);
    R.Sx = comp(d, kx) / dkz;
    R.Sy = comp(d, ky) / dkz;
    R.Sz = 1.0f / dkz;
}

__device__ __forceinline__ float fmax3(float a, float b, float c) {
    float r;
    asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}
__device__ __forceinline__ float fmin3(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Entry distance of the segment into the box, or +inf when it misses (three-input min/max).
__device__ __forceinline__ float slab(const Ray& R, float lx, float ly, float lz, float hx, float hy, float hz) {
    const float t0x = fmaf(lx, R.idir.x, -R.oidir.x), t1x = fmaf(hx, R.idir.x, -R.oidir.x);
    const float t0y = fmaf(ly, R.idir.y, -R.oidir.y), t1y = fmaf(hy, R.idir.y, -R.oidir.y);
    const float t0z = fmaf(lz, R.idir.z, -R.oidir.z), t1z = fmaf(hz, R.idir.z, -R.oidir.z);
    const float tn = fmax3(fminf(t0x, t1x), fminf(t0y, t1y), fmaxf(fminf(t0z, t1z), 0.f));
    const float tf = fmin3(fmaxf(t0x, t1x), fmaxf(t0y, t1y), fminf(fmaxf(t0z, t1z), R.tmax_box));
    return tn <= tf ? tn : INFINITY;
}

// Woop, Benthin, Wald, "Watertight ray/triangle intersection", JCGT 2(1), 2013. Edge functions
// are evaluated without fused multiply-add so that a shared edge gives exactly opposite values
// in its two triangles (no ray slips between them).
__device__ __forceinline__ bool tri_hit(const Ray& R, float4 a, float4 b, float4 c) {
    float3 A = make_float3(a.x - R.o.x, a.y - R.o.y, a.z - R.o.z);
    float3 B = make_float3(b.x - R.o.x, b.y - R.o.y, b.z - R.o.z);
    float3 C = make_float3(c.x - R.o.x, c.y - R.o.y, c.z - R.o.z);
    float Akz = comp(A, R.kz), Bkz = comp(B, R.kz), Ckz = comp(C, R.kz);
    float Ax = __fsub_rn(comp(A, R.kx), __fmul_rn(R.Sx, Akz));
    float Ay = __fsub_rn(comp(A, R.ky), __fmul_rn(R.Sy, Akz));
    float Bx = __fsub_rn(comp(B, R.kx), __fmul_rn(R.Sx, Bkz));
    float By = __fsub_rn(comp(B, R.ky), __fmul_rn(R.Sy, Bkz));
    float Cx = __fsub_rn(comp(C, R.kx), __fmul_rn(R.Sx, Ckz));
    float Cy = __fsub_rn(comp(C, R.ky), __fmul_rn(R.Sy, Ckz));
    float U = __fsub_rn(__fmul_rn(Cx, By), __fmul_rn(Cy, Bx));
    float V = __fsub_rn(__fmul_rn(Ax, Cy), __fmul_rn(Ay, Cx));
    float W = __fsub_rn(__fmul_rn(Bx, Ay), __fmul_rn(By, Ax));
    if ((U < 0.f || V < 0.f || W < 0.f) && (U > 0.f || V > 0.f || W > 0.f)) return false;
    float det = U + V + W;
    if (det == 0.f) return false;
    float T = U * (R.Sz * Akz) + V * (R.Sz * Bkz) + W * (R.Sz * Ckz);
    return det > 0.f ? (T > 0.f && T < R.tmax * det) : (T < 0.f && T > R.tmax * det);
}

__device__ __forceinline__ bool leaf_hit(const Ray& R, const float4* __restrict__ tris, int slot, uint32_t own,
                                         uint32_t& n_tri) {
    ++n_tri;
    float4 a = __ldg(&tris[3 * slot]);
    if (__float_as_uint(a.w) == own) return false;
    return tri_hit(R, a, __ldg(&tris[3 * slot + 1]), __ldg(&tris[3 * slot + 2]));
}

// Any-hit traversal of the segment: stack of deferred subtrees, nearer child first (an occluder
// between the eye and the sample is met sooner), leaves tested as soon as they are reached.
__device__ bool occluded(const Ray& R, uint32_t own, const float4* __restrict__ nodes,
                         const float4* __restrict__ tris, uint32_t nt, int* __restrict__ err, uint32_t& n_node,
                         uint32_t& n_tri, int& hit_slot) {
    if (nt < 2) {
        const bool h = nt == 1 && leaf_hit(R, tris, 0, own, n_tri);
        if (h) hit_slot = 0;
        return h;
    }
    int stack[STACK];
    int sp = 0;
    int node = 0;
    for (;;) {
        ++n_node;
        const float4 n3 = __ldg(&nodes[4 * node + 3]);
        const float4 n0 = __ldg(&nodes[4 * node + 0]);
        const float4 n1 = __ldg(&nodes[4 * node + 1]);
        const float4 n2 = __ldg(&nodes[4 * node + 2]);
        const int cl = __float_as_int(n3.x), cr = __float_as_int(n3.y);
        float tl = slab(R, n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
        float tr = slab(R, n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
        if (tl < INFINITY && cl < 0) {
            if (leaf_hit(R, tris, ~cl, own, n_tri)) {
                hit_slot = ~cl;
                return true;
            }
            tl = INFINITY;
        }
        if (tr < INFINITY && cr < 0) {
            if (leaf_hit(R, tris, ~cr, own, n_tri)) {
                hit_slot = ~cr;
                return true;
            }
            tr = INFINITY;
        }
        if (tl < INFINITY && tr < INFINITY) {
            if (sp >= STACK) {
                atomicCAS(err, 0, GM_DEV_STACK_OVERFLOW);
                return true;
            }
            const bool left_first = tl <= tr;
            stack[sp++] = left_first ? cr : cl;
            node = left_first ? cl : cr;
        } else if (tl < INFINITY) {
            node = cl;
        } else if (tr < INFINITY) {
            node = cr;
        } else {
            if (sp == 0) return false;
            node = stack[--sp];
        }
    }
}

__device__ __forceinline__ void cswap(float& ta, int& la, float& tb, int& lb) {
    const bool sw = tb < ta;
    const float t = sw ? tb : ta;
    const int l = sw ? lb : la;
    tb = sw ? ta : tb;
    lb = sw ? la : lb;
    ta = t;
    la = l;
}

// Any-hit traversal of the 4-wide tree: one 128-byte node fetch tests four child boxes; leaf
// children are tested at once; internal children are visited nearest first (a five-exchange
// sorting network on the entry distances), the others pushed far-to-near.
__device__ bool occluded4(const Ray& R, uint32_t own, const float4* __restrict__ nodes4,
                          const float4* __restrict__ tris, int* __restrict__ err, uint32_t& n_node,
                          uint32_t& n_tri, int& hit_slot) {
    int stack[STACK4];
    int sp = 0;
    int node = 0;
    for (;;) {
        ++n_node;
        const float4* N = nodes4 + 8 * node;
        const float4 lx = __ldg(N + 0), hx = __ldg(N + 1), ly = __ldg(N + 2), hy = __ldg(N + 3);
        const float4 lz = __ldg(N + 4), hz = __ldg(N + 5), L = __ldg(N + 6);
        float t0 = slab(R, lx.x, ly.x, lz.x, hx.x, hy.x, hz.x);
        float t1 = slab(R, lx.y, ly.y, lz.y, hx.y, hy.y, hz.y);
        float t2 = slab(R, lx.z, ly.z, lz.z, hx.z, hy.z, hz.z);
        float t3 = slab(R, lx.w, ly.w, lz.w, hx.w, hy.w, hz.w);
        int c0 = __float_as_int(L.x), c1 = __float_as_int(L.y), c2 = __float_as_int(L.z), c3 = __float_as_int(L.w);
        if (t0 < INFINITY && c0 < 0) { if (c0 != LINK_EMPTY && leaf_hit(R, tris, ~c0, own, n_tri)) { hit_slot = ~c0; return true; } t0 = INFINITY; }
        if (t1 < INFINITY && c1 < 0) { if (c1 != LINK_EMPTY && leaf_hit(R, tris, ~c1, own, n_tri)) { hit_slot = ~c1; return true; } t1 = INFINITY; }
        if (t2 < INFINITY && c2 < 0) { if (c2 != LINK_EMPTY && leaf_hit(R, tris, ~c2, own, n_tri)) { hit_slot = ~c2; return true; } t2 = INFINITY; }
        if (t3 < INFINITY && c3 < 0) { if (c3 != LINK_EMPTY && leaf_hit(R, tris, ~c3, own, n_tri)) { hit_slot = ~c3; return true; } t3 = INFINITY; }
        cswap(t0, c0, t1, c1);
        cswap(t2, c2, t3, c3);
        cswap(t0, c0, t2, c2);
        cswap(t1, c1, t3, c3);
        cswap(t1, c1, t2, c2);
        if (t0 == INFINITY) {
            if (sp == 0) return false;
            node = stack[--sp];
            continue;
        }
        const int np = (t1 < INFINITY) + (t2 < INFINITY) + (t3 < INFINITY);
        if (sp + np > STACK4) {
            atomicCAS(err, 0, GM_DEV_STACK_OVERFLOW);
            return true;
        }
        if (t3 < INFINITY) stack[sp++] = c3;
        if (t2 < INFINITY) stack[sp++] = c2;
        if (t1 < INFINITY) stack[sp++] = c1;
        node = c0;
    }
}

// Any-hit query of the segment through the eye grid of its fixation: the triangles binned in the
// ray's cell (and the fixation's near list, cell R*R) are every triangle the segment can meet,
// stored with a lower bound of their depth along the gaze and sorted by it; the walk stops at
// the first hit or at the first entry that lies wholly beyond the sample (wlim).
__device__ __forceinline__ bool eg_list_hit(const Ray& R, uint32_t own, uint32_t b, uint32_t e, float wlim,
                                            const uint2* __restrict__ ent, const float4* __restrict__ tris,
                                            uint32_t& n_ent, uint32_t& n_tri, int& hit_slot) {
    // two entries per step: both triangles' loads are in flight before either is tested
    for (uint32_t k = b; k < e; k += 2) {
        const uint2 t0 = __ldg(&ent[k]);
        const bool two = k + 1 < e;
        const uint2 t1 = two ? __ldg(&ent[k + 1]) : make_uint2(0u, 0x7f800000u);
        const bool u0 = __uint_as_float(t0.y) <= wlim, u1 = two && __uint_as_float(t1.y) <= wlim;
        n_ent += two ? 2 : 1;
        if (!u0) break;
        const float4* p0 = tris + 3 * (size_t)t0.x;
        const float4* p1 = tris + 3 * (size_t)(u1 ? t1.x : t0.x);
        const float4 a0 = __ldg(p0), b0 = __ldg(p0 + 1), c0 = __ldg(p0 + 2);
        const float4 a1 = __ldg(p1), b1 = __ldg(p1 + 1), c1 = __ldg(p1 + 2);
        ++n_tri;
        if (__float_as_uint(a0.w) != own && tri_hit(R, a0, b0, c0)) {
            hit_slot = (int)t0.x;
            return true;
        }
        if (!u1) break;
        ++n_tri;
        if (__float_as_uint(a1.w) != own && tri_hit(R, a1, b1, c1)) {
            hit_slot = (int)t1.x;
            return true;
        }
    }
    return false;
}

__device__ __forceinline__ bool occluded_grid(const Ray& R, uint32_t own, float w_s, int cell, int R2,
                                              const uint32_t* __restrict__ cs, const uint2* __restrict__ ent,
                                              const float4* __restrict__ tris, uint32_t& n_ent, uint32_t& n_tri,
                                              int& hit_slot) {
    // a triangle can hold the hit only if part of it lies nearer than the sample (t < 1); the
    // stored bounds are conservative and 1e-5 covers the rounding of the sample's own depth
    const float wlim = w_s * 1.00001f;
    const uint32_t nb = __ldg(&cs[R2]), ne = __ldg(&cs[R2 + 1]);
    const uint32_t cb = __ldg(&cs[cell]), ce = __ldg(&cs[cell + 1]);
    if (nb < ne && eg_list_hit(R, own, nb, ne, wlim, ent, tris, n_ent, n_tri, hit_slot)) return true;
    return eg_list_hit(R, own, cb, ce, wlim, ent, tris, n_ent, n_tri, hit_slot);
}

__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Whether the cone of fixation (F0: eye; F1: unit gaze r^) with half-angle tan(phi) = tanphi can
// reach the sphere bs (centre, radius; a negative radius: no sphere, always true). A point
// p = q + u with |u| <= R has d1 <= d1c + R and |p x r^| >= |q x r^| - R; it is in the cone only
// if |p x r^| <= tan(phi) d1. Compared squared (both sides are non-negative); the margin, from the
// L1 norm of q, covers FP32 rounding on both sides.
__device__ __forceinline__ bool cone_reaches_sphere(const float4 bs, const float4 F0, const float4 F1,
                                                    const float tanphi) {
    if (bs.w < 0.f) return true;
    const float bR = bs.w;
    const float qx = bs.x - F0.x, qy = bs.y - F0.y, qz = bs.z - F0.z;
    const float d1c = fmaf(qx, F1.x, fmaf(qy, F1.y, qz * F1.z));
    const float ux = fmaf(qy, F1.z, -qz * F1.y);
    const float uy = fmaf(qz, F1.x, -qx * F1.z);
    const float uz = fmaf(qx, F1.y, -qy * F1.x);
    const float margin = 1e-4f * (fabsf(qx) + fabsf(qy) + fabsf(qz) + bR);
    const float reach = d1c + bR;
    const float lim = bR + fmaf(tanphi, fmaxf(reach, 0.f), margin);
    return !(reach <= -margin || fmaf(ux, ux, fmaf(uy, uy, uz * uz)) > lim * lim);
}

// The bounding sphere of a warp's points (centre of their box, half its diagonal, enlarged by
// 1e-4 relative), the same in every lane; radius -1 when no lane holds a point.
__device__ __forceinline__ float4 warp_bounding_sphere(const bool has, const float x, const float y, const float z) {
    float lo[3] = {has ? x : INFINITY, has ? y : INFINITY, has ? z : INFINITY};
    float hi[3] = {has ? x : -INFINITY, has ? y : -INFINITY, has ? z : -INFINITY};
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    }
    if (!(lo[0] <= hi[0])) return make_float4(0.f, 0.f, 0.f, -1.f);
    return make_float4(0.5f * (lo[0] + hi[0]), 0.5f * (lo[1] + hi[1]), 0.5f * (lo[2] + hi[2]),
                       0.5f * sqrtf((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                    (hi[2] - lo[2]) * (hi[2] - lo[2])) * 1.0001f);
}

constexpr int WARP_TILE = 32 * SPT;   // samples per warp tile

// Compensated addition of g into a sample's (sum, compensation) slot.
__device__ __forceinline__ void kahan_slot(float2* wacc, int slot, float g) {
    float2 a = wacc[slot];
    const float y = g - a.y;
    const float t = a.x + y;
    a.y = (t - a.x) - y;
    a.x = t;
    wacc[slot] = a;
}

struct AccParams;
struct DebugOut;

struct TileStats {
    unsigned long long n_in = 0, n_vis = 0;
    uint32_t n_node = 0, n_tri = 0;
    unsigned long long n_tested = 0;   // sample x fixation cone tests evaluated (not skipped by a tile sphere)
};

// Debug record of one traced pair (sample index in stored order, fixation in input order).
__device__ __forceinline__ void record_pair(unsigned long long* cursor, const DebugOut& dbg, const AccParams& P,
                                            const uint32_t* __restrict__ sidx, uint32_t base0, uint32_t stride, int slot,
                                            uint32_t fi, bool vis, float g) {
    const unsigned long long q = atomicAdd(cursor, 1ull);
    if (q < P.dbg_cap) {
        dbg.sample[q] = sidx[base0 + (slot >> 5) * stride + (slot & 31)];
        dbg.fix[q] = dbg.fix_orig[fi];
        dbg.vis[q] = vis ? 1 : 0;
        dbg.g[q] = g;
    }
}

// One warp processes the S x 32 work-order samples of warp tile `tile` (see AccParams::group) against
// fixations [P.f0, min(P.f1, nf)) of `fix` (packed (e, w), (r^, window), sorted by window). Sums are
// written to out[window * P.ns + sidx[j]] when a window ends; each window's maximum is folded into
// max_bits[window] with one atomicMax per warp. Eye-grid kernels only: with P.carry_in the
// compensated sums start from P.carry and the window of fixation f0 - 1 continues; with
// P.carry_out the open sums are saved to P.carry at the end instead of being written (a later
// launch continues them); the BVH kernels take the whole list [0, nf). The warp's
// shared-memory regions (WARP_TILE entries each) are used only when COMPACT. Occlusion: the BVH
// (binary or, WIDE, 4-wide) or, GRID, the eye grid of P (COMPACT only). No block-wide
// synchronisation. *tested counts the sample x fixation cone tests actually evaluated. FSM: the
// fixations are staged 32 at a time in the warp's slot wfix (64 float4) instead of being read
// one by one through L1.
template <bool DEBUG, bool COMPACT, bool WIDE, bool GRID = false, int S = SPT, bool FSM = false>
__device__ __forceinline__ void warp_tile(uint32_t tile, const float4* __restrict__ spos,
                                          const uint32_t* __restrict__ sidx, const float4* __restrict__ fix,
                                          uint32_t nf, const float4* __restrict__ nodes,
                                          const float4* __restrict__ tris, const AccParams& P,
                                          float* __restrict__ out, unsigned int* __restrict__ max_bits,
                                          float4* wsmp, float2* wacc, uint16_t* qslot, float* qg, float4* wbox,
                                          unsigned long long* __restrict__ dbg_cursor, const DebugOut& dbg,
                                          int* __restrict__ err, TileStats& st, float4* wfix = nullptr) {
    static_assert(!GRID || COMPACT, "the eye grid traces from the ray queue");
    static_assert(!(GRID && FSM), "staged fixations are a form of the BVH kernels");
    // fixation ranges and sums carried across launches exist for the eye grid's chunks only; the
    // BVH kernels cover the whole list in one launch and keep none of that code
    constexpr bool CH = GRID;
    const int lane = threadIdx.x & 31;
    const uint32_t G = P.group;
    const uint32_t stride = 32u * G;
    const uint32_t base0 = (tile / G) * (uint32_t)(32 * S) * G + (tile % G) * 32u;
    const uint32_t base = base0 + lane;
    const uint32_t i_end = CH ? min(nf, P.f1) : nf;
    float sx[S], sy[S], sz[S], sum[S], cmp[S];
    uint32_t own[S];
    float blo[3] = {INFINITY, INFINITY, INFINITY}, bhi[3] = {-INFINITY, -INFINITY, -INFINITY};
    uint32_t live = 0;
#pragma unroll
    for (int k = 0; k < S; ++k) {
        const uint32_t j = base + k * stride;
        // padding lanes hold NaN positions: every cone test on them is false
        const float4 p = j < P.ns ? spos[j]
                                  : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, __uint_as_float(0xffffffffu));
        if (j < P.ns) {
            ++live;
            blo[0] = fminf(blo[0], p.x);
            blo[1] = fminf(blo[1], p.y);
            blo[2] = fminf(blo[2], p.z);
            bhi[0] = fmaxf(bhi[0], p.x);
            bhi[1] = fmaxf(bhi[1], p.y);
            bhi[2] = fmaxf(bhi[2], p.z);
        }
        const float2 c0 = (CH && P.carry_in && j < P.ns) ? P.carry[j] : make_float2(0.f, 0.f);
        sum[k] = c0.x;
        cmp[k] = c0.y;
        if (COMPACT) {
            wsmp[k * 32 + lane] = p;
            wacc[k * 32 + lane] = c0;
        } else {
            sx[k] = p.x;
            sy[k] = p.y;
            sz[k] = p.z;
            own[k] = __float_as_uint(p.w);
        }
    }
    __syncwarp();
    // the tile's bounding sphere (centre of its box, half the box diagonal): a fixation whose cone
    // cannot reach the sphere is skipped without per-sample tests, which leaves every in-cone pair
    // and every sum as it is
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            blo[c] = fminf(blo[c], __shfl_xor_sync(0xffffffffu, blo[c], o));
            bhi[c] = fmaxf(bhi[c], __shfl_xor_sync(0xffffffffu, bhi[c], o));
        }
    }
    // the sphere stays in the warp's shared-memory slot (registers are the traversal's)
    const bool tile_box = P.tile_cull && blo[0] <= bhi[0];
    if (lane == 0)
        *wbox = make_float4(0.5f * (blo[0] + bhi[0]), 0.5f * (blo[1] + bhi[1]), 0.5f * (blo[2] + bhi[2]),
                            tile_box ? 0.5f * sqrtf((bhi[0] - blo[0]) * (bhi[0] - blo[0]) +
                                                    (bhi[1] - blo[1]) * (bhi[1] - blo[1]) +
                                                    (bhi[2] - blo[2]) * (bhi[2] - blo[2])) * 1.0001f
                                     : -1.f);
    __syncwarp();
    // the open window: none, or (continuing a previous launch) the window of fixation f0 - 1
    uint32_t cur = 0xffffffffu;
    if (CH && P.carry_in && P.f0 > 0) cur = __float_as_uint(__ldg(&fix[2 * (P.f0 - 1) + 1]).w);

    auto flush = [&](uint32_t w) {
        float m = 0.f;
        if (COMPACT) __syncwarp();
#pragma unroll
        for (int k = 0; k < S; ++k) {
            if (COMPACT) {
                sum[k] = wacc[k * 32 + lane].x;
                wacc[k * 32 + lane] = make_float2(0.f, 0.f);
            }
            const uint32_t j = base + k * stride;
            if (j < P.ns && (P.W == 1 || sum[k] != 0.f)) out[(size_t)w * P.ns + sidx[j]] = sum[k];
            m = fmaxf(m, sum[k]);
            sum[k] = 0.f;
            cmp[k] = 0.f;
        }
        if (COMPACT) __syncwarp();
        m = warp_max(m);
        if (lane == 0 && m > 0.f) atomicMax(&max_bits[w], __float_as_uint(m));
    };

    const uint32_t i_beg = CH ? P.f0 : 0u;
    float4 nF0 = !FSM && i_beg < i_end ? __ldg(&fix[2 * i_beg]) : make_float4(0.f, 0.f, 0.f, 0.f);
    float4 nF1 = !FSM && i_beg < i_end ? __ldg(&fix[2 * i_beg + 1]) : make_float4(0.f, 0.f, 0.f, 0.f);
    // whether fixation (F0, F1)'s cone can reach the tile's bounding sphere (always, without one)
    auto sphere_reach = [&](const float4 F0, const float4 F1) -> bool {
        return cone_reaches_sphere(*wbox, F0, F1, P.tanphi);
    };
    // the work of one fixation (window change, tile sphere test unless `reached` says it was
    // passed, cone tests, ray queue)
    auto per_fixation = [&](const uint32_t i, const float4 F0, const float4 F1, const bool reached) {
        const uint32_t win = __float_as_uint(F1.w);
        if (win != cur) {
            if (cur != 0xffffffffu) flush(cur);
            cur = win;
        }
        if (!reached && !sphere_reach(F0, F1)) return;
        st.n_tested += live;
        if (COMPACT) {
            int tot = 0;
#pragma unroll
            for (int k = 0; k < S; ++k) {
                // the tile's samples are read from shared memory (they are there for the ray queue
                // anyway), which keeps 4 x 4 registers free for occupancy
                const float4 q = wsmp[k * 32 + lane];
                const float px = q.x - F0.x, py = q.y - F0.y, pz = q.z - F0.z;
                const float d1 = fmaf(px, F1.x, fmaf(py, F1.y, pz * F1.z));
                const float cx = fmaf(py, F1.z, -pz * F1.y);
                const float cy = fmaf(pz, F1.x, -px * F1.z);
                const float cz = fmaf(px, F1.y, -py * F1.x);
                const float c2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
                const float d1s = d1 * d1;
                const bool in = d1 > 0.f && c2 <= P.K * d1s;
                const unsigned m = __ballot_sync(0xffffffffu, in);
                if (in) {
                    const int pos = tot + __popc(m & gm_lanemask_lt());
                    qslot[pos] = (uint16_t)(k * 32 + lane);
                    // the weight is rounded on its own (never fused into the compensated sum), so
                    // both tracing forms add exactly the same value
                    qg[pos] = __fmul_rn(F0.w, ex2_approx(-P.C2 * __fdividef(c2, d1s)));
                }
                tot += __popc(m);
            }
            if (tot == 0) return;
            __syncwarp();
            // the eye grid of this fixation (warp-uniform): its gaze frame and its cell offsets
            float4 gU = make_float4(0.f, 0.f, 0.f, 0.f), gV = gU;
            const uint32_t* cs = nullptr;
            if (GRID) {
                gU = __ldg(&P.eg_basis[2 * i]);
                gV = __ldg(&P.eg_basis[2 * i + 1]);
                cs = P.eg_cells + (size_t)(i - P.f0) * (P.eg_R * P.eg_R + 2u);
            }
            // the queue is traced 32 rays at a time: rays of one batch leave one eye toward neighbouring
            // samples and walk the tree nearly in step (node fetches are shared); a queue-refill
            // variant that let lanes run out of phase measured 28 % slower
            for (int b = 0; b < tot; b += 32) {
                const int e = b + lane;
                if (e < tot) {
                    const int slot = qslot[e];
                    const float4 sp = wsmp[slot];
                    const float g = qg[e];
                    ++st.n_in;
                    Ray R;
                    const float3 d = make_float3(sp.x - F0.x, sp.y - F0.y, sp.z - F0.z);
                    make_ray(R, make_float3(F0.x, F0.y, F0.z), d, P.tmax);
                    int hit = -1;
                    bool vis;
                    if (GRID) {
                        // the ray's cell: its direction in the fixation's gaze frame
                        const float w_s = fmaf(d.x, F1.x, fmaf(d.y, F1.y, d.z * F1.z));
                        const float xs = __fdividef(fmaf(d.x, gU.x, fmaf(d.y, gU.y, d.z * gU.z)), w_s);
                        const float ys = __fdividef(fmaf(d.x, gV.x, fmaf(d.y, gV.y, d.z * gV.z)), w_s);
                        const int RR = (int)P.eg_R;
                        const int cell = eg_cell_coord(ys, P.eg_s, RR) * RR + eg_cell_coord(xs, P.eg_s, RR);
                        vis = !occluded_grid(R, __float_as_uint(sp.w), w_s, cell, RR * RR, cs, P.eg_ent, tris,
                                             st.n_node, st.n_tri, hit);
                    } else {
                        vis = WIDE ? !occluded4(R, __float_as_uint(sp.w), nodes, tris, err, st.n_node, st.n_tri, hit)
                                   : !occluded(R, __float_as_uint(sp.w), nodes, tris, P.nt, err, st.n_node,
                                               st.n_tri, hit);
                    }
                    if (vis) {
                        ++st.n_vis;
                        kahan_slot(wacc, slot, g);
                    }
                    if (DEBUG) record_pair(dbg_cursor, dbg, P, sidx, base0, stride, slot, i, vis, g);
                }
            }
            __syncwarp();
        } else {
#pragma unroll
            for (int k = 0; k < S; ++k) {
                const float px = sx[k] - F0.x, py = sy[k] - F0.y, pz = sz[k] - F0.z;
                const float d1 = fmaf(px, F1.x, fmaf(py, F1.y, pz * F1.z));
                const float cx = fmaf(py, F1.z, -pz * F1.y);
                const float cy = fmaf(pz, F1.x, -px * F1.z);
                const float cz = fmaf(px, F1.y, -py * F1.x);
                const float c2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
                const float d1s = d1 * d1;
                if (d1 > 0.f && c2 <= P.K * d1s) {
                    ++st.n_in;
                    Ray R;
                    make_ray(R, make_float3(F0.x, F0.y, F0.z), make_float3(px, py, pz), P.tmax);
                    int hit = -1;
                    const bool vis = WIDE ? !occluded4(R, own[k], nodes, tris, err, st.n_node, st.n_tri, hit)
                                          : !occluded(R, own[k], nodes, tris, P.nt, err, st.n_node, st.n_tri, hit);
                    const float g = __fmul_rn(F0.w, ex2_approx(-P.C2 * __fdividef(c2, d1s)));
                    if (vis) {
                        ++st.n_vis;
                        const float y = g - cmp[k];
                        const float t = sum[k] + y;
                        cmp[k] = (t - sum[k]) - y;
                        sum[k] = t;
                    }
                    if (DEBUG) {
                        const unsigned long long q = atomicAdd(dbg_cursor, 1ull);
                        if (q < P.dbg_cap) {
                            dbg.sample[q] = sidx[base + k * stride];
                            dbg.fix[q] = dbg.fix_orig[i];
                            dbg.vis[q] = vis ? 1 : 0;
                            dbg.g[q] = g;
                        }
                    }
                }
            }
        }
        };
    if (FSM) {
        // fixations staged 32 at a time in the warp's shared-memory slot (one coalesced load per
        // lane); each lane tests its fixation against the tile's sphere, and the warp then visits
        // only the fixations that reach it, in list order. Skipping a fixation never changes a
        // sum; a window is written when the next visited fixation opens another one, or at the
        // end, which writes the same values as writing it at the first fixation of the next window.
        for (uint32_t c0 = i_beg; c0 < i_end; c0 += 32) {
            const uint32_t m = min(32u, i_end - c0);
            __syncwarp();
            bool pass = false;
            if ((uint32_t)lane < m) {
                const float4 a = __ldg(&fix[2 * (c0 + lane)]), b = __ldg(&fix[2 * (c0 + lane) + 1]);
                wfix[2 * lane] = a;
                wfix[2 * lane + 1] = b;
                pass = sphere_reach(a, b);
            }
            unsigned pm = __ballot_sync(0xffffffffu, pass);
            __syncwarp();
            while (pm) {
                const int k = __ffs(pm) - 1;
                pm &= pm - 1u;
                per_fixation(c0 + k, wfix[2 * k], wfix[2 * k + 1], true);
            }
        }
    } else {
        // fixations read through L1 as warp-wide broadcasts, the next one in flight
        for (uint32_t i = i_beg; i < i_end; ++i) {
            const float4 F0 = nF0, F1 = nF1;
            if (i + 1 < i_end) {
                nF0 = __ldg(&fix[2 * (i + 1)]);
                nF1 = __ldg(&fix[2 * (i + 1) + 1]);
            }
            per_fixation(i, F0, F1, false);
        }
    }
    if (CH && P.carry_out) {
        // the window goes on in the next launch: keep the open sums
        if (COMPACT) __syncwarp();
#pragma unroll
        for (int k = 0; k < S; ++k) {
            const uint32_t j = base + k * stride;
            if (j < P.ns) P.carry[j] = COMPACT ? wacc[k * 32 + lane] : make_float2(sum[k], cmp[k]);
        }
        if (COMPACT) __syncwarp();
        return;
    }
    if (cur != 0xffffffffu) flush(cur);
    else if (P.W == 1) flush(0);   // no fixation at all: window 0 is written as zeros
}

// Sum a warp's tile statistics into counters [0] in-cone, [1] visible, [4] nodes, [5] triangles.
__device__ __forceinline__ void warp_stats_commit(TileStats st, unsigned long long* __restrict__ counters) {
    unsigned long long a = st.n_in, b = st.n_vis, c = st.n_node, d = st.n_tri, t = st.n_tested;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
        d += __shfl_xor_sync(0xffffffffu, d, o);
        t += __shfl_xor_sync(0xffffffffu, t, o);
    }
    if ((threadIdx.x & 31) == 0) {
        if (a | b) {
            atomicAdd(&counters[0], a);
            atomicAdd(&counters[1], b);
            atomicAdd(&counters[4], c);
            atomicAdd(&counters[5], d);
        }
        if (t) atomicAdd(&counters[7], t);
    }
}

}  // namespace
