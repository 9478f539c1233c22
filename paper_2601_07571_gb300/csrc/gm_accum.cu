// gm_accum.cu -- gm_accumulate_fixations: Section 3.2 of the paper on one GPU.
//
// Per fixation (prep kernel): r^ = r / |r|, weight t / (sigma sqrt(2 pi)), window id
// floor((ts - t_begin) / window_s); fixations outside [t_begin, t_end) are dropped and the
// rest are stably sorted by window (radix sort on the window id), so every window is one
// contiguous run of the fixation list.
//
// Accumulation (one fused kernel, sample-stationary): every thread owns SPT samples taken in
// spatial (Morton) work order and keeps their compensated FP32 sums in registers. The block
// streams the fixation list through shared memory in tiles; for each fixation every thread
// runs the 4-sigma cone test on its samples (p = s - e, d1 = p.r^, c = p x r^,
// in-cone <=> d1 > 0 and |c|^2 <= (cutoff tan theta)^2 d1^2, about 20 FP32 instructions per
// pair) and, for in-cone pairs only, traces the occlusion segment e -> e + (1 - eps) p (any-hit,
// early exit, the sample's own triangle skipped) with the watertight ray/triangle test of Woop,
// Benthin and Wald (JCGT 2013), through the BVH or, with GM_F_EYE_GRID, over the triangles of the
// segment's cell in the fixation's eye grid (gm_eyegrid.cu). With more fixations than one eye-grid
// chunk holds, the kernel runs once per chunk and the compensated sums carry over. A visible pair adds
// g = w exp(-(|c|/d1)^2 / (2 tan^2 theta)), i.e. the paper's t/(sigma sqrt(2 pi)) *
// exp(-sigma_k^2 / (2 sigma^2)) with sigma_k = d2 / d1, d2 = |c|, in fixation order (Kahan).
// When the window id of the next fixation changes (block-uniform), the block stores its sums
// for the finished window and folds its maximum into that window's max with one atomicMax on
// the float's bit pattern (values are >= 0) -- the paper keeps this running maximum under a
// mutex (Section 3.3.1); here no lock is needed.
// Normalisation (Section 3.2.3) is a separate streaming kernel: v / max per window.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "gm_internal.cuh"

#include "gm_trace.cuh"

namespace {

// ------------------------------------------------------------------------------------------
// fixation prep
// ------------------------------------------------------------------------------------------
__global__ void k_fix_keys(const double* __restrict__ ts, const float* __restrict__ eye,
                           const float* __restrict__ gaze, const float* __restrict__ dur, uint32_t nf,
                           double t_begin, double t_end, double window_s, uint32_t W, uint32_t only,
                           uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                           uint32_t* __restrict__ n_valid, int* __restrict__ err) {
    uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    double t = ts[f];
    uint32_t key = W;
    if (t >= t_begin && t < t_end) {
        // the window bucket of a FP64 timestamp (one division per fixation)
        double w = window_s > 0.0 ? floor((t - t_begin) / window_s) : 0.0;
        if (w >= 0.0 && w < (double)W) key = (uint32_t)w;
        if (only != 0xffffffffu && key != only) key = W;   // one window of a dynamic scene at a time
    }
    float gx = gaze[3 * f], gy = gaze[3 * f + 1], gz = gaze[3 * f + 2];
    float ex = eye[3 * f], ey = eye[3 * f + 1], ez = eye[3 * f + 2];
    float d = dur[f];
    bool finite = isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(ex) && isfinite(ey) && isfinite(ez) &&
                  isfinite(d) && (gx != 0.f || gy != 0.f || gz != 0.f);
    if (!finite || !(d >= 0.f) || isnan(t)) {
        atomicCAS(err, 0, 3);
        key = W;
    }
    keys[f] = key;
    vals[f] = f;
    if (key < W) atomicAdd(n_valid, 1u);
}

__global__ void k_fix_pack(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                           const float* __restrict__ eye, const float* __restrict__ gaze,
                           const float* __restrict__ dur, uint32_t nf, float wnorm,
                           float4* __restrict__ packed, uint32_t* __restrict__ orig) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    uint32_t f = vals[i];
    float rx = gaze[3 * f], ry = gaze[3 * f + 1], rz = gaze[3 * f + 2];
    float rn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry)), __fmul_rn(rz, rz)));
    rx = __fdiv_rn(rx, rn);
    ry = __fdiv_rn(ry, rn);
    rz = __fdiv_rn(rz, rn);
    packed[2 * i + 0] = make_float4(eye[3 * f], eye[3 * f + 1], eye[3 * f + 2], __fmul_rn(dur[f], wnorm));
    packed[2 * i + 1] = make_float4(rx, ry, rz, __uint_as_float(keys[i]));
    orig[i] = f;
}

// Persistent: every warp pulls warp tiles (WARP_TILE consecutive work-order samples, see
// warp_tile) from a device counter until all n_tiles are done, so tiles that see many in-cone
// rays (densely gazed patches) spread over the whole run instead of forming a tail. MINB is the
// minimum number of resident blocks per SM the register allocation must allow (3: up to 80
// registers, 4: up to 64).
template <bool DEBUG, bool COMPACT, bool WIDE, int MINB, int NT = ACC_THREADS, bool GRID = false, int S = SPT,
          bool FSM = false>
__global__ void __launch_bounds__(NT, MINB) k_accumulate(
    const float4* __restrict__ spos, const uint32_t* __restrict__ sidx, const float4* __restrict__ fix,
    const uint32_t* __restrict__ n_fix_dev, const float4* __restrict__ nodes, const float4* __restrict__ tris,
    AccParams P, uint32_t n_tiles, int persistent, float* __restrict__ out, unsigned int* __restrict__ max_bits,
    unsigned long long* __restrict__ counters, int* __restrict__ err, DebugOut dbg) {
    constexpr int QN = COMPACT ? NT * S : 1;
    __shared__ float4 wsmp[QN];     // per warp: its WARP_TILE samples (x, y, z, own triangle)
    __shared__ float2 wacc[QN];     // per warp: (sum, compensation) of each sample
    __shared__ float4 wbox[NT / 32];   // per warp: its tile's bounding sphere
    __shared__ uint16_t qslot[QN];  // per warp: queue of in-cone sample slots
    __shared__ float qg[QN];        // per warp: their weights
    __shared__ float4 wfix[FSM ? (NT / 32) * 64 : 1];   // per warp: 32 staged fixations
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int wb = COMPACT ? warp * 32 * S : 0;
    const uint32_t nf = *n_fix_dev;
    unsigned int* next = reinterpret_cast<unsigned int*>(&counters[6]);
    TileStats st;
    for (uint32_t round = 0;; ++round) {
        uint32_t tile = 0;
        if (persistent) {
            if (lane == 0) tile = atomicAdd(next, 1u);
            tile = __shfl_sync(0xffffffffu, tile, 0);
        } else {
            if (round > 0) break;
            tile = blockIdx.x * (NT / 32) + warp;
        }
        if (tile >= n_tiles) break;
        warp_tile<DEBUG, COMPACT, WIDE, GRID, S, FSM>(tile, spos, sidx, fix, nf, nodes, tris, P, out, max_bits,
                                                          wsmp + wb, wacc + wb, qslot + wb, qg + wb, wbox + warp,
                                                          &counters[2], dbg, err, st, FSM ? wfix + warp * 64 : nullptr);
    }
    warp_stats_commit(st, counters);
}

// (The driver's default shared-memory carveout is kept: preferring the largest L1 leaves room for
// fewer blocks per SM and measured 316 vs 253 ms at the paper scene.)
template <bool D, bool Cm, bool Wd, int Mb, int NT = ACC_THREADS, bool Gr = false, int S = SPT, bool Fs = false>
int acc_occupancy() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_accumulate<D, Cm, Wd, Mb, NT, Gr, S, Fs>, NT, 0);
    return b > 0 ? b : 1;
}

// v / max for every window, windows whose maximum is 0 left as they are (0). A persistent grid
// (every resident block slot once) walks work items (window, chunk of NORM_ITEM float4): each
// thread moves NORM_UNROLL float4 of the chunk, all its loads issued before the first division.
// 32 registers a thread, so 8 blocks of 256 fit an SM. A window whose start is not
// 16-byte aligned (W > 1, ns not a multiple of 4) has up to 3 head floats before its float4 body
// and up to 3 tail floats after it; the window's first item does those one by one.
constexpr int NORM_THREADS = 256;
constexpr int NORM_UNROLL = 4;
constexpr uint64_t NORM_ITEM = (uint64_t)NORM_THREADS * NORM_UNROLL;

__global__ void __launch_bounds__(NORM_THREADS, 8) k_normalize(float* __restrict__ v, uint64_t ns,
                                                            const unsigned int* __restrict__ max_bits, uint64_t W,
                                                            uint64_t items_per_win) {
    const uint64_t n_items = W * items_per_win;
    for (uint64_t it = blockIdx.x; it < n_items; it += gridDim.x) {
        const uint64_t win = it / items_per_win;
        const uint64_t c = it - win * items_per_win;
        const float m = __uint_as_float(max_bits[win]);
        if (!(m > 0.f)) continue;
        float* w = v + win * ns;
        const uint64_t mis = ((16u - (reinterpret_cast<uintptr_t>(w) & 15u)) & 15u) / 4u;
        const uint64_t head = mis < ns ? mis : ns;
        const uint64_t n4 = (ns - head) / 4;
        float4* w4 = reinterpret_cast<float4*>(w + head);
        const uint64_t i0 = c * NORM_ITEM + threadIdx.x;
        float4 x[NORM_UNROLL];
#pragma unroll
        for (int u = 0; u < NORM_UNROLL; ++u) {
            const uint64_t i = i0 + (uint64_t)u * NORM_THREADS;
            if (i < n4) x[u] = w4[i];
        }
#pragma unroll
        for (int u = 0; u < NORM_UNROLL; ++u) {
            const uint64_t i = i0 + (uint64_t)u * NORM_THREADS;
            if (i < n4) {
                x[u].x = __fdiv_rn(x[u].x, m);
                x[u].y = __fdiv_rn(x[u].y, m);
                x[u].z = __fdiv_rn(x[u].z, m);
                x[u].w = __fdiv_rn(x[u].w, m);
                w4[i] = x[u];
            }
        }
        if (c == 0 && threadIdx.x < 8) {
            // threads 0..3: the head floats; threads 4..7: the floats after the float4 body
            const uint64_t k = threadIdx.x < 4 ? threadIdx.x : head + 4 * n4 + (threadIdx.x - 4);
            if (threadIdx.x < 4 ? k < head : k < ns) w[k] = __fdiv_rn(w[k], m);
        }
    }
}

__global__ void k_iota(uint32_t* p, uint32_t n) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = i;
}

__global__ void k_gather_values(const float* __restrict__ v, uint64_t ns, uint32_t w, const uint32_t* __restrict__ idx,
                                uint64_t n, float* __restrict__ out, int* __restrict__ err) {
    uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t j = idx[i];
    if (j >= ns) {
        atomicCAS(err, 0, GM_DEV_BAD_INDEX);
        out[i] = 0.f;
        return;
    }
    out[i] = v[(size_t)w * ns + j];
}

__global__ void k_add_valid(unsigned long long* __restrict__ c, const uint32_t* __restrict__ n_valid) {
    c[0] += *n_valid;
}

// v / max for every window of a map (windows whose maximum is 0 stay 0); returns launches.
int launch_normalize(gm_map* mp, int n_sm, cudaStream_t s) {
    const uint64_t ns = mp->ns, W = mp->W;
    if (ns == 0) return 0;
    const uint64_t items_per_win = std::max<uint64_t>(1, gm_div_up(ns / 4, NORM_ITEM));
    // every resident block slot once, never more blocks than items
    static const int per_sm = [] {
        int b = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_normalize, NORM_THREADS, 0);
        return b > 0 ? b : 1;
    }();
    const uint64_t grid = std::min<uint64_t>((uint64_t)n_sm * per_sm, W * items_per_win);
    k_normalize<<<(uint32_t)grid, NORM_THREADS, 0, s>>>(mp->values, ns, mp->max_bits, W, items_per_win);
    return 1;
}

gm_status n_windows_of(const gm_params* prm, uint64_t* W_out) {
    uint64_t W = 1;
    if (prm->window_s > 0.0) {
        if (!std::isfinite(prm->t_begin) || !std::isfinite(prm->t_end) || !std::isfinite(prm->window_s))
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: windows need a finite interval");
        W = (uint64_t)std::ceil((prm->t_end - prm->t_begin) / prm->window_s);
        if (W == 0) W = 1;
        if (W > (1u << 24)) return gm_set_error(GM_ERR_UNSUPPORTED, "gm_accumulate_fixations: more than 2^24 windows");
    }
    *W_out = W;
    return GM_OK;
}

// The accumulation of one fixation set. into == nullptr: a new map (returned in *out) over all
// windows. into != nullptr: adds the fixations of window `only_window` to that existing map
// (no normalisation, no stage timing), for dynamic scenes posed window by window.
gm_status accumulate_impl(gm_scene* sc, gm_samples* sm, const gm_fixations* fx, const gm_params* prm,
                          gm_stream stream, gm_map* into, int64_t only_window, gm_map** out) {
    if (!sc || !sm || !fx || !prm || (!out && !into))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: null argument");
    if (out) *out = nullptr;
    if (sm->scene != sc) return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: samples belong to another scene");
    if (!(prm->theta_rad > 0.f) || !(prm->theta_rad < 1.5f))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: theta must be in (0, 1.5) rad");
    if (!(prm->cutoff_sigmas > 0.f) || !std::isfinite(prm->cutoff_sigmas))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: cutoff must be > 0");
    if (!(prm->eps_rel >= 0.f && prm->eps_rel < 1.f))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: eps_rel must be in [0, 1)");
    if (std::isnan(prm->t_begin) || std::isnan(prm->t_end) || !(prm->t_begin < prm->t_end))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: need t_begin < t_end");
    if (fx->n > 0 && (!fx->eye_xyz || !fx->gaze_xyz || !fx->duration_s || !fx->timestamp_s))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: null fixation array");
    uint64_t W = 1;
    GM_TRY(n_windows_of(prm, &W));
    if (into && (into->W != W || into->ns != sm->n))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: map does not match windows or samples");
    const bool debug = into ? ((prm->flags & GM_F_DEBUG_PAIRS) && into->dbg_cap > 0)
                            : ((prm->flags & GM_F_DEBUG_PAIRS) && prm->debug_pair_cap > 0);
    cudaStream_t s = (cudaStream_t)stream;
    gm_ctx* ctx = sc->ctx;
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    const uint64_t ns = sm->n;
    const uint32_t nf = fx->n;

    gm_map* mp = into ? into : new gm_map();
    if (!into) {
        mp->ctx = ctx;
        mp->W = (uint32_t)W;
        mp->ns = ns;
        mp->stream = s;
        mp->timing = (prm->flags & GM_F_TIMING) != 0;
        mp->stats.n_windows = (uint32_t)W;
    }
    std::vector<void*> tmp;
    EyeGrid* egp = nullptr;   // set once the eye grid exists, freed with the temporaries
    auto fail = [&](gm_status st) {
        for (void* p : tmp) cudaFreeAsync(p, s);
        if (egp) eg_free(egp, s);
        if (!into) gm_map_free(mp);
        return st;
    };
    gm_status st;
#define TMP_ALLOC(ptr, bytes)                                                          \
    do {                                                                               \
        if ((st = gm_alloc((void**)&(ptr), (bytes), s)) != GM_OK) return fail(st);     \
        tmp.push_back((void*)(ptr));                                                   \
    } while (0)
#define MAP_ALLOC(ptr, bytes) \
    if ((st = gm_alloc((void**)&(ptr), (bytes), s)) != GM_OK) return fail(st)

    const bool timing = mp->timing && !into;
    if (timing) {
        for (int i = 0; i < 6; ++i) {
            cudaError_t e = cudaEventCreate(&mp->ev[i]);
            if (e != cudaSuccess) return fail(gm_cuda_error(e, "cudaEventCreate"));
        }
        cudaEventRecord(mp->ev[0], s);
    }
    if (into) {
        // the persistent kernel's tile counter starts from 0 on every launch
        GM_TRY_CUDA(cudaMemsetAsync(&mp->counters[6], 0, sizeof(unsigned long long), s));
    } else {
        MAP_ALLOC(mp->values, sizeof(float) * W * ns);
        MAP_ALLOC(mp->max_bits, sizeof(unsigned int) * W);
        MAP_ALLOC(mp->counters, sizeof(unsigned long long) * 8);
        GM_TRY_CUDA(cudaMemsetAsync(mp->max_bits, 0, sizeof(unsigned int) * W, s));
        GM_TRY_CUDA(cudaMemsetAsync(mp->counters, 0, sizeof(unsigned long long) * 8, s));
        if (W > 1) GM_TRY_CUDA(cudaMemsetAsync(mp->values, 0, sizeof(float) * W * ns, s));
    }
    if (debug && !into) {
        mp->dbg_cap = prm->debug_pair_cap;
        MAP_ALLOC(mp->dbg_sample, sizeof(uint32_t) * mp->dbg_cap);
        MAP_ALLOC(mp->dbg_fix, sizeof(uint32_t) * mp->dbg_cap);
        MAP_ALLOC(mp->dbg_vis, mp->dbg_cap);
        MAP_ALLOC(mp->dbg_g, sizeof(float) * mp->dbg_cap);
    }
    int launches = 0;

    // ---- fixation prep --------------------------------------------------------------------
    void *d_eye = nullptr, *d_gaze = nullptr, *d_dur = nullptr, *d_ts = nullptr;
    bool o1, o2, o3, o4;
    if ((st = gm_stage_to_device(fx->eye_xyz, sizeof(float) * 3 * (size_t)nf, s, &d_eye, &o1)) != GM_OK) return fail(st);
    if (o1) tmp.push_back(d_eye);
    if ((st = gm_stage_to_device(fx->gaze_xyz, sizeof(float) * 3 * (size_t)nf, s, &d_gaze, &o2)) != GM_OK) return fail(st);
    if (o2) tmp.push_back(d_gaze);
    if ((st = gm_stage_to_device(fx->duration_s, sizeof(float) * (size_t)nf, s, &d_dur, &o3)) != GM_OK) return fail(st);
    if (o3) tmp.push_back(d_dur);
    if ((st = gm_stage_to_device(fx->timestamp_s, sizeof(double) * (size_t)nf, s, &d_ts, &o4)) != GM_OK) return fail(st);
    if (o4) tmp.push_back(d_ts);
    uint32_t *keys = nullptr, *vals = nullptr, *n_valid = nullptr, *orig = nullptr;
    float4* packed = nullptr;
    TMP_ALLOC(keys, sizeof(uint32_t) * (nf ? nf : 1));
    TMP_ALLOC(vals, sizeof(uint32_t) * (nf ? nf : 1));
    TMP_ALLOC(orig, sizeof(uint32_t) * (nf ? nf : 1));
    TMP_ALLOC(packed, sizeof(float4) * 2 * (nf ? nf : 1));
    MAP_ALLOC(n_valid, sizeof(uint32_t));
    tmp.push_back(n_valid);
    GM_TRY_CUDA(cudaMemsetAsync(n_valid, 0, sizeof(uint32_t), s));
    const double tan_t = std::tan((double)prm->theta_rad);
    const float wnorm = (float)(1.0 / (tan_t * std::sqrt(2.0 * 3.14159265358979323846)));
    if (nf > 0) {
        k_fix_keys<<<gm_div_up(nf, 256), 256, 0, s>>>((const double*)d_ts, (const float*)d_eye, (const float*)d_gaze,
                                                      (const float*)d_dur, nf, prm->t_begin, prm->t_end,
                                                      prm->window_s > 0.0 ? prm->window_s : 0.0, (uint32_t)W,
                                                      only_window >= 0 ? (uint32_t)only_window : 0xffffffffu, keys,
                                                      vals, n_valid, ctx->dev_err);
        ++launches;
        int bits = 1;
        while (bits < 32 && (1ull << bits) <= W) ++bits;
        if ((st = gm_radix_sort_u32(keys, vals, nf, bits, s, &launches)) != GM_OK) return fail(st);
        k_fix_pack<<<gm_div_up(nf, 256), 256, 0, s>>>(keys, vals, (const float*)d_eye, (const float*)d_gaze,
                                                      (const float*)d_dur, nf, wnorm, packed, orig);
        ++launches;
    }
    if (timing) cudaEventRecord(mp->ev[1], s);

    // ---- accumulate -----------------------------------------------------------------------
    AccParams P;
    P.C2 = (float)(1.4426950408889634 / (2.0 * tan_t * tan_t));
    P.K = (float)((double)prm->cutoff_sigmas * tan_t * (double)prm->cutoff_sigmas * tan_t);
    P.tmax = 1.0f - prm->eps_rel;
    P.ns = (uint32_t)ns;
    P.W = (uint32_t)W;
    P.nt = sc->n_tris;
    P.dbg_cap = mp->dbg_cap;
    DebugOut dbg{mp->dbg_sample, mp->dbg_fix, mp->dbg_vis, mp->dbg_g, orig};
    EyeGrid eg;
    egp = &eg;
    float2* carry = nullptr;
    const bool reorder = !(prm->flags & GM_F_NO_REORDER) && sm->work_pos;
    uint32_t* ident = nullptr;
    const float4* spos = reorder ? sm->work_pos : sm->pos;
    const uint32_t* sidx = reorder ? sm->work_idx : nullptr;
    if (!sidx) TMP_ALLOC(ident, sizeof(uint32_t) * (ns ? ns : 1));
    if (ns > 0) {
        if (!sidx) {
            k_iota<<<gm_div_up(ns, 256), 256, 0, s>>>(ident, (uint32_t)ns);
            ++launches;
            sidx = ident;
        }
        P.group = (prm->flags & GM_F_TILE_CONSECUTIVE) ? 1u : 8u;
        P.tile_cull = (prm->flags & GM_F_NO_TILE_CULL) ? 0u : 1u;
        P.tanphi = (float)(std::sqrt((double)P.K) * 1.00001);
        const uint32_t n_tiles = gm_div_up(ns, (uint64_t)WARP_TILE * P.group) * P.group;
        const int persistent = (prm->flags & GM_F_STATIC_TILES) ? 0 : 1;
        const bool compact = !(prm->flags & GM_F_NO_COMPACT);
        const bool wide = (prm->flags & GM_F_WIDE_BVH) && sc->nodes4;
        const bool occ4 = (prm->flags & GM_F_REGCAP64) != 0;
        const bool b128 = (prm->flags & GM_F_BLOCK128) != 0;
        // the eye grid (opt-in) traces from the ray queue; the in-place, 4-wide and 64-register
        // variants keep the tree
        const bool grid = (prm->flags & GM_F_EYE_GRID) && compact && !wide && !occ4 && nf > 0;
        const float4* tree = wide ? sc->nodes4 : sc->nodes;
        const int code = (compact ? 1 : 0) | (wide ? 2 : 0) | (occ4 ? 4 : 0);
        // persistent grid: every resident block slot once, never more blocks than tiles need
#define GM_LAUNCH_ACC_F(D, Cm, Wd, Mb, NT, Gr, S_, Fs)                                                           \
    do {                                                                                                          \
        const uint32_t nt_s = gm_div_up(ns, (uint64_t)32 * (S_) * P.group) * P.group;                             \
        const uint32_t all = gm_div_up(nt_s, NT / 32);                                                            \
        const uint32_t grd = persistent ? std::min<uint32_t>(                                                     \
                                              (uint32_t)ctx->n_sm * acc_occupancy<D, Cm, Wd, Mb, NT, Gr, S_, Fs>(), \
                                              all)                                                                \
                                        : all;                                                                    \
        k_accumulate<D, Cm, Wd, Mb, NT, Gr, S_, Fs><<<grd, NT, 0, s>>>(spos, sidx, packed, n_valid, tree,          \
                                                                       sc->bvh_tris, P, nt_s, persistent,         \
                                                                       mp->values, mp->max_bits, mp->counters,    \
                                                                       ctx->dev_err, dbg);                        \
    } while (0)
#define GM_LAUNCH_ACC_S(D, Cm, Wd, Mb, NT, Gr, S_) GM_LAUNCH_ACC_F(D, Cm, Wd, Mb, NT, Gr, S_, false)
#define GM_LAUNCH_ACC_NT(D, Cm, Wd, Mb, NT, Gr) GM_LAUNCH_ACC_S(D, Cm, Wd, Mb, NT, Gr, SPT)
#define GM_LAUNCH_ACC(D, Cm, Wd, Mb) GM_LAUNCH_ACC_NT(D, Cm, Wd, Mb, ACC_THREADS, false)
        if (grid) {
            const uint32_t R = (prm->flags & GM_F_GRID64) ? 64u : 128u;
            size_t fr = 0, tot = 0;
            GM_TRY_CUDA(cudaMemGetInfo(&fr, &tot));
            // entries of one chunk: at most a third of the free memory (8 bytes each), or fewer when
            // GM_EYEGRID_CHUNK_ENTRIES says so (smaller chunks: tighter memory, more launches)
            uint64_t budget = std::max<uint64_t>(1u << 20, (uint64_t)fr / 3 / sizeof(uint2));
            if (const char* env = std::getenv("GM_EYEGRID_CHUNK_ENTRIES")) {
                const unsigned long long v = std::strtoull(env, nullptr, 10);
                if (v > 0) budget = std::min<uint64_t>(budget, v);
            }
            if ((st = eg_prepare(sc, packed, n_valid, nf, (float)std::sqrt((double)P.K), R, budget, s, &eg,
                                 &launches)) != GM_OK)
                return fail(st);
            const uint32_t nchunk = (uint32_t)eg.chunk.size() - 1;
            // accumulation launches: within a build chunk, runs of fixations holding at most
            // GM_EYEGRID_L2_ENTRIES entries (default: the whole chunk in one launch; L2-sized runs
            // measured slower, each launch waiting on its slowest warp tile); the sums carry over
            uint64_t l2_entries = ~0ull;   // measured: one launch per chunk beats L2-sized runs
            if (const char* env = std::getenv("GM_EYEGRID_L2_ENTRIES")) {
                const unsigned long long v = std::strtoull(env, nullptr, 10);
                if (v > 0) l2_entries = v;
            }
            std::vector<std::pair<uint32_t, uint32_t>> runs;   // [a, b) per launch
            std::vector<uint32_t> run_chunk;
            for (uint32_t k = 0; k < nchunk; ++k) {
                uint32_t a = eg.chunk[k];
                uint64_t acc = 0;
                for (uint32_t f = eg.chunk[k]; f < eg.chunk[k + 1]; ++f) {
                    if (f > a && acc + eg.h_tot[f] > l2_entries) {
                        runs.emplace_back(a, f);
                        run_chunk.push_back(k);
                        a = f;
                        acc = 0;
                    }
                    acc += eg.h_tot[f];
                }
                runs.emplace_back(a, eg.chunk[k + 1]);
                run_chunk.push_back(k);
            }
            if (runs.size() > 1) TMP_ALLOC(carry, sizeof(float2) * ns);
            P.carry = carry;
            P.eg_basis = eg.basis;
            P.eg_ent = eg.ent;
            P.eg_R = R;
            P.eg_s = eg.s;
            if (timing) cudaEventRecord(mp->ev[4], s);
            const size_t per_fix = (size_t)R * R + 2;
            for (size_t q = 0; q < std::max<size_t>(1, runs.size()); ++q) {
                if (!runs.empty()) {
                    const uint32_t k = run_chunk[q];
                    if (q == 0 || run_chunk[q - 1] != k)
                        if ((st = eg_build_chunk(sc, packed, &eg, k, s, &launches)) != GM_OK) return fail(st);
                    P.f0 = runs[q].first;
                    P.f1 = runs[q].second;
                    P.eg_cells = eg.cells + (size_t)(runs[q].first - eg.chunk[k]) * per_fix;
                    P.carry_in = q > 0;
                    P.carry_out = q + 1 < runs.size();
                }
                if (timing && q == 0) cudaEventRecord(mp->ev[5], s);
                if (q > 0) GM_TRY_CUDA(cudaMemsetAsync(&mp->counters[6], 0, sizeof(unsigned long long), s));
                // shape: samples per thread (GM_F_SPT1 / GM_F_SPT2, else 4) and block size
                // (GM_F_BLOCK128 / GM_F_BLOCK512, else 256); 80 registers a thread in every shape
                const int spt = (prm->flags & GM_F_SPT1) ? 1 : (prm->flags & GM_F_SPT2) ? 2 : 4;   // default 4
                const int nth = b128 ? 128 : (prm->flags & GM_F_BLOCK512) ? 512 : 256;
                if (debug) GM_LAUNCH_ACC_S(true, true, false, 3, 256, true, 4);
                else if (nth == 256 && spt == 4) GM_LAUNCH_ACC_S(false, true, false, 3, 256, true, 4);
                else if (nth == 256 && spt == 2) GM_LAUNCH_ACC_S(false, true, false, 3, 256, true, 2);
                else if (nth == 256) GM_LAUNCH_ACC_S(false, true, false, 3, 256, true, 1);
                else if (nth == 128 && spt == 4) GM_LAUNCH_ACC_S(false, true, false, 6, 128, true, 4);
                else if (nth == 128 && spt == 2) GM_LAUNCH_ACC_S(false, true, false, 6, 128, true, 2);
                else if (nth == 128) GM_LAUNCH_ACC_S(false, true, false, 6, 128, true, 1);
                else if (spt == 1) GM_LAUNCH_ACC_S(false, true, false, 1, 512, true, 1);
                else GM_LAUNCH_ACC_S(false, true, false, 1, 512, true, 2);   // 512 x 4 exceeds static shared memory
                ++launches;
            }
            mp->stats.grid_chunks = std::max<uint32_t>(1u, nchunk);
            mp->stats.grid_launches = (uint32_t)std::max<size_t>(1, runs.size());
        } else {
            if (timing) {
                cudaEventRecord(mp->ev[4], s);
                cudaEventRecord(mp->ev[5], s);
            }
            if (debug) {
                switch (code & 3) {
                    case 0: GM_LAUNCH_ACC(true, false, false, 3); break;
                    case 1: GM_LAUNCH_ACC(true, true, false, 3); break;
                    case 2: GM_LAUNCH_ACC(true, false, true, 3); break;
                    default: GM_LAUNCH_ACC(true, true, true, 3); break;
                }
            } else {
                // the ray-queue binary-tree kernels: samples per thread 1 (the default), 2 or 4; the
                // one-sample tiles fit 64 registers (4 blocks per SM) and stage their fixations in
                // shared memory
                const int qspt = (prm->flags & GM_F_SPT4) ? 4 : (prm->flags & GM_F_SPT2) ? 2 : 1;
                const bool b512 = (prm->flags & GM_F_BLOCK512) != 0;
                if ((code == 1 || code == 5) && qspt == 1) {
                    if (b128) GM_LAUNCH_ACC_F(false, true, false, 8, 128, false, 1, true);
                    else if (b512) GM_LAUNCH_ACC_F(false, true, false, 2, 512, false, 1, true);
                    else if (prm->flags & GM_F_FIX_L1) GM_LAUNCH_ACC_F(false, true, false, 4, 256, false, 1, false);
                    else GM_LAUNCH_ACC_F(false, true, false, 4, 256, false, 1, true);
                } else if ((code == 0 || code == 4) && (prm->flags & GM_F_SPT1)) {
                    // one-sample tiles traced in place: a lane traces its own sample's ray
                    GM_LAUNCH_ACC_F(false, false, false, 4, 256, false, 1, true);
                } else if ((code == 1 || code == 5) && qspt == 2) {
                    if (code == 5) GM_LAUNCH_ACC_F(false, true, false, 4, 256, false, 2, true);
                    else GM_LAUNCH_ACC_F(false, true, false, 3, 256, false, 2, true);
                } else if (b128 && code == 1) GM_LAUNCH_ACC_NT(false, true, false, 7, 128, false);
                else if (b128 && code == 5) GM_LAUNCH_ACC_NT(false, true, false, 8, 128, false);
                else switch (code) {
                    case 0: GM_LAUNCH_ACC(false, false, false, 3); break;
                    case 1:   // 4 samples per thread: fixations staged in shared memory (GM_F_FIX_L1: through L1)
                        if (prm->flags & GM_F_FIX_L1) GM_LAUNCH_ACC(false, true, false, 3);
                        else GM_LAUNCH_ACC_F(false, true, false, 3, 256, false, SPT, true);
                        break;
                    case 2: GM_LAUNCH_ACC(false, false, true, 3); break;
                    case 3: GM_LAUNCH_ACC(false, true, true, 3); break;
                    case 4: GM_LAUNCH_ACC(false, false, false, 4); break;
                    case 5:
                        if (prm->flags & GM_F_SPT1) GM_LAUNCH_ACC_F(false, true, false, 4, 256, false, 1, true);
                        else if (prm->flags & GM_F_SPT2) GM_LAUNCH_ACC_F(false, true, false, 4, 256, false, 2, true);
                        else GM_LAUNCH_ACC(false, true, false, 4);
                        break;
                    case 6: GM_LAUNCH_ACC(false, false, true, 4); break;
                    default: GM_LAUNCH_ACC(false, true, true, 4); break;
                }
            }
            ++launches;
        }
#undef GM_LAUNCH_ACC
#undef GM_LAUNCH_ACC_NT
#undef GM_LAUNCH_ACC_S
#undef GM_LAUNCH_ACC_F
    }
    if (timing) cudaEventRecord(mp->ev[2], s);
    if (prm->normalize && !into) launches += launch_normalize(mp, ctx->n_sm, s) > 0 ? 1 : 0;
    if (timing) cudaEventRecord(mp->ev[3], s);
    // keep the valid-fixation count with the map for gm_map_info
    if (into) {
        k_add_valid<<<1, 1, 0, s>>>(&mp->counters[3], n_valid);
        ++launches;
    } else {
        GM_TRY_CUDA(cudaMemcpyAsync(&mp->counters[3], n_valid, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_accumulate_fixations launch"));
    for (void* p : tmp) cudaFreeAsync(p, s);
    eg_free(&eg, s);
    mp->stats.launches = (into ? mp->stats.launches : 0) + (uint32_t)launches;
    ctx->launches += launches;
    if (out) *out = mp;
    return GM_OK;
#undef TMP_ALLOC
#undef MAP_ALLOC
}

}  // namespace

extern "C" gm_status gm_accumulate_fixations(gm_scene* sc, gm_samples* sm, const gm_fixations* fx,
                                             const gm_params* prm, gm_stream stream, gm_map** out) {
    if (!out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: null argument");
    return accumulate_impl(sc, sm, fx, prm, stream, nullptr, -1, out);
}

extern "C" gm_status gm_accumulate_dynamic(gm_scene* sc, gm_samples* sm, const gm_fixations* fx, const gm_params* prm,
                                           const double* window_transforms, gm_stream stream, gm_map** out) {
    if (!sc || !sm || !fx || !prm || !window_transforms || !out)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_dynamic: null argument");
    *out = nullptr;
    if (sm->scene != sc) return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_dynamic: samples belong to another scene");
    if (!sc->tri_local)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_dynamic: the scene was not built with gm_build_opts.dynamic");
    if (sm->kind == GM_SAMPLES_POINTS)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_dynamic: explicit points do not follow the meshes");
    uint64_t W = 1;
    GM_TRY(n_windows_of(prm, &W));
    gm_params p = *prm;
    p.normalize = 0;
    p.flags &= ~(int32_t)GM_F_TIMING;
    gm_map* mp = nullptr;
    for (uint64_t k = 0; k < W; ++k) {
        gm_status st = gm_scene_pose(sc, window_transforms + 16 * (size_t)sc->n_meshes * k, stream);
        if (st == GM_OK) st = gm_samples_follow(sm, stream);
        if (st == GM_OK) st = accumulate_impl(sc, sm, fx, &p, stream, mp, (int64_t)k, k == 0 ? &mp : nullptr);
        if (st != GM_OK) {
            gm_map_free(mp);
            return st;
        }
    }
    if (prm->normalize) {
        const int l = launch_normalize(mp, sc->ctx->n_sm, (cudaStream_t)stream);
        sc->ctx->launches += l;
        mp->stats.launches += (uint32_t)l;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) {
            gm_map_free(mp);
            return gm_cuda_error(e, "gm_accumulate_dynamic normalise");
        }
    }
    *out = mp;
    return GM_OK;
}

extern "C" gm_status gm_map_info(gm_map* mp, uint32_t* n_windows, uint64_t* n_samples, gm_map_stats* stats) {
    if (!mp) return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_info: null map");
    GM_TRY_CUDA(cudaStreamSynchronize(mp->stream));
    int err = 0;
    unsigned long long c[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    GM_TRY_CUDA(cudaMemcpy(&err, mp->ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost));
    GM_TRY_CUDA(cudaMemcpy(c, mp->counters, sizeof(c), cudaMemcpyDeviceToHost));
    if (err) {
        cudaMemset(mp->ctx->dev_err, 0, sizeof(int));
        if (err == 3) return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_fixations: non-finite fixation, zero gaze or negative duration");
        if (err == GM_DEV_STACK_OVERFLOW) return gm_set_error(GM_ERR_INTERNAL, "BVH traversal stack overflow");
        return gm_set_error(GM_ERR_INTERNAL, "device consistency check failed (" + std::to_string(err) + ")");
    }
    uint32_t nvalid = (uint32_t)(c[3] & 0xffffffffu);
    mp->stats.in_cone = c[0];
    mp->stats.visible = c[1];
    mp->stats.n_fixations_used = nvalid;
    mp->stats.pairs = (uint64_t)nvalid * mp->ns;
    mp->stats.nodes_visited = c[4];
    mp->stats.tris_tested = c[5];
    mp->stats.pairs_tested = c[7];
    if (mp->timing) {
        float a = 0, b = 0, d = 0, g = 0;
        cudaEventElapsedTime(&a, mp->ev[0], mp->ev[1]);
        if (mp->ev[4] && mp->ev[5]) {
            // ev[1] .. ev[4]: eye-grid frames and counts; ev[4] .. ev[5]: the first chunk's build
            float g0 = 0, g1 = 0;
            cudaEventElapsedTime(&g0, mp->ev[1], mp->ev[4]);
            cudaEventElapsedTime(&g1, mp->ev[4], mp->ev[5]);
            g = g0 + g1;
            cudaEventElapsedTime(&b, mp->ev[5], mp->ev[2]);
        } else {
            cudaEventElapsedTime(&b, mp->ev[1], mp->ev[2]);
        }
        cudaEventElapsedTime(&d, mp->ev[2], mp->ev[3]);
        mp->stats.prep_ms = a;
        mp->stats.grid_ms = g;
        mp->stats.accumulate_ms = b;
        mp->stats.normalize_ms = d;
    }
    if (n_windows) *n_windows = mp->W;
    if (n_samples) *n_samples = mp->ns;
    if (stats) *stats = mp->stats;
    // any window whose maximum is 0 -> warning
    std::vector<unsigned int> mx(mp->W);
    GM_TRY_CUDA(cudaMemcpy(mx.data(), mp->max_bits, sizeof(unsigned int) * mp->W, cudaMemcpyDeviceToHost));
    for (unsigned int m : mx)
        if (m == 0) return GM_WARN_EMPTY;
    return GM_OK;
}

extern "C" gm_status gm_map_copy(const gm_map* mp, uint32_t window, float* dst, float* max_out, gm_stream stream) {
    if (!mp || !dst) return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_copy: null argument");
    if (window >= mp->W) return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_copy: window out of range");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY(gm_copy_out(dst, mp->values + (size_t)window * mp->ns, sizeof(float) * mp->ns, s));
    if (max_out) {
        unsigned int b = 0;
        GM_TRY_CUDA(cudaMemcpyAsync(&b, mp->max_bits + window, sizeof(b), cudaMemcpyDeviceToHost, s));
        GM_TRY_CUDA(cudaStreamSynchronize(s));
        memcpy(max_out, &b, sizeof(float));
    }
    return GM_OK;
}

extern "C" const float* gm_map_device_values(const gm_map* mp) { return mp ? mp->values : nullptr; }

extern "C" gm_status gm_map_max(const gm_map* mp, float* out, gm_stream stream) {
    if (!mp || !out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_max: null argument");
    // the maxima are kept as the bit patterns of non-negative floats: the bytes are the floats
    return gm_copy_out(out, mp->max_bits, sizeof(float) * mp->W, (cudaStream_t)stream);
}

extern "C" gm_status gm_map_normalize(gm_map* mp, const float* maxima, gm_stream stream) {
    if (!mp) return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_normalize: null map");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(mp->ctx->device));
    if (maxima) {
        if (!gm_is_device_ptr(maxima)) {
            for (uint32_t w = 0; w < mp->W; ++w)
                if (!(maxima[w] >= 0.f) || !std::isfinite(maxima[w]))
                    return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_normalize: maxima must be finite and >= 0");
        }
        GM_TRY_CUDA(cudaMemcpyAsync(mp->max_bits, maxima, sizeof(float) * mp->W, cudaMemcpyDefault, s));
    }
    const int l = launch_normalize(mp, mp->ctx->n_sm, s);
    mp->ctx->launches += l;
    mp->stats.launches += (uint32_t)l;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

extern "C" gm_status gm_map_debug_pairs(const gm_map* mp, uint32_t* sample, uint32_t* fix, uint8_t* vis, float* g,
                                        uint64_t cap, uint64_t* n) {
    if (!mp || !n) return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_debug_pairs: null argument");
    GM_TRY_CUDA(cudaStreamSynchronize(mp->stream));
    unsigned long long cnt = 0;
    if (mp->counters) GM_TRY_CUDA(cudaMemcpy(&cnt, &mp->counters[2], sizeof(cnt), cudaMemcpyDeviceToHost));
    *n = cnt;
    uint64_t k = std::min<uint64_t>(std::min<uint64_t>(cnt, cap), mp->dbg_cap);
    if (k == 0) return GM_OK;
    if (!sample || !fix || !vis || !g) return gm_set_error(GM_ERR_INVALID_ARG, "gm_map_debug_pairs: null output");
    GM_TRY_CUDA(cudaMemcpy(sample, mp->dbg_sample, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
    GM_TRY_CUDA(cudaMemcpy(fix, mp->dbg_fix, sizeof(uint32_t) * k, cudaMemcpyDeviceToHost));
    GM_TRY_CUDA(cudaMemcpy(vis, mp->dbg_vis, k, cudaMemcpyDeviceToHost));
    GM_TRY_CUDA(cudaMemcpy(g, mp->dbg_g, sizeof(float) * k, cudaMemcpyDeviceToHost));
    return GM_OK;
}

extern "C" void gm_map_free(gm_map* mp) {
    if (!mp) return;
    cudaFree(mp->values);
    cudaFree(mp->max_bits);
    cudaFree(mp->counters);
    cudaFree(mp->dbg_sample);
    cudaFree(mp->dbg_fix);
    cudaFree(mp->dbg_vis);
    cudaFree(mp->dbg_g);
    for (auto& e : mp->ev)
        if (e) cudaEventDestroy(e);
    delete mp;
}

extern "C" gm_status gm_query_density(const gm_map* mp, const gm_field* field, gm_query_mode mode, uint32_t window,
                                      const uint32_t* sample_idx, const float* xyz, uint64_t n, float* out,
                                      gm_stream stream) {
    if (!out && n > 0) return gm_set_error(GM_ERR_INVALID_ARG, "gm_query_density: null output");
    cudaStream_t s = (cudaStream_t)stream;
    if (mode == GM_Q_SAMPLE) {
        if (!mp || (!sample_idx && n > 0)) return gm_set_error(GM_ERR_INVALID_ARG, "gm_query_density: map and indices required");
        if (window >= mp->W) return gm_set_error(GM_ERR_INVALID_ARG, "gm_query_density: window out of range");
        if (n == 0) return GM_OK;
        void* di = nullptr;
        bool oi = false;
        GM_TRY(gm_stage_to_device(sample_idx, sizeof(uint32_t) * n, s, &di, &oi));
        bool dev_out = gm_is_device_ptr(out);
        float* dout = out;
        if (!dev_out) GM_TRY(gm_alloc((void**)&dout, sizeof(float) * n, s));
        k_gather_values<<<gm_div_up(n, 256), 256, 0, s>>>(mp->values, mp->ns, window, (const uint32_t*)di, n, dout,
                                                          mp->ctx->dev_err);
        mp->ctx->launches += 1;
        gm_status st = GM_OK;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = gm_cuda_error(e, "gm_query_density launch");
        if (!dev_out) {
            if (st == GM_OK) st = gm_copy_out(out, dout, sizeof(float) * n, s);
            cudaFreeAsync(dout, s);
        }
        if (oi) cudaFreeAsync(di, s);
        return st;
    }
    if (mode == GM_Q_PLAIN)
        return gm_set_error(GM_ERR_INVALID_ARG,
                            "gm_query_density: GM_Q_PLAIN points are accumulated with gm_samples_from_points + "
                            "gm_accumulate_fixations");
    if (mode == GM_Q_FIELD) {
        if (!field) return gm_set_error(GM_ERR_INVALID_ARG, "gm_query_density: GM_Q_FIELD needs a field");
        return gm_field_query(field, xyz, n, out, stream);
    }
    return gm_set_error(GM_ERR_INVALID_ARG, "gm_query_density: unknown mode");
}
