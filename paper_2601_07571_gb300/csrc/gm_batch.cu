// gm_batch.cu -- many independent sessions in one persistent, CUDA-graph-captured launch, and
// the autotuner that picks the accumulation variant.
//
// A session is (scene, samples, fixations); all sessions share the generation parameters. At
// plan creation every session's fixations are staged into one device buffer and a work list
// of warp tiles (session, 32*SPT consecutive work-order samples) is built on the host: sessions
// grouped into three size buckets by triangle count, within a bucket ordered by decreasing cost
// (fixations per tile, i.e. longest processing time first). The plan then captures into one
// CUDA graph: the counter resets, the batched fixation prep (window keys per session, one stable
// radix sort, packing), one persistent accumulation launch per bucket on forked streams (its
// warps pull the bucket's work items from the bucket's counter; each bucket has its own kernel
// variant and events around its launch; a bucket's tail overlaps the next one's start), and the
// batched normalisation. gm_batch_run replays the graph: no
// host work and one graph launch per call.
//
// Autotuning: the candidates are the accumulation variants (per-warp ray queue on/off, binary
// or 4-wide tree, 80- or 64-register cap). Each is timed on every bucket's own launch and each
// bucket keeps its fastest; results are cached per bucket and size (log2 of samples, fixations,
// triangles) in memory and in the JSON file named by GM_TUNE_CACHE, if set.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <fstream>
#include <map>
#include <mutex>
#include <numeric>
#include <sstream>
#include <string>
#include <vector>

#include "gm_trace.cuh"

namespace {

struct SessionDev {
    const float4* spos;
    const uint32_t* sidx;
    const float4* fix;        // this session's packed fixations (sorted by window)
    const uint32_t* n_fix;    // number of valid fixations (device)
    const float4* nodes;
    const float4* tris;
    float* out;
    unsigned int* max_bits;
    unsigned long long* counters;
    uint32_t ns, nt, W, pad;
};

__global__ void k_bfix_keys(const double* __restrict__ ts, const float* __restrict__ eye,
                            const float* __restrict__ gaze, const float* __restrict__ dur,
                            const uint32_t* __restrict__ sess_of, uint32_t nf, double t_begin, double t_end,
                            double window_s, uint32_t W, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                            uint32_t* __restrict__ n_valid, int* __restrict__ err) {
    const uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const uint32_t s = sess_of[f];
    const double t = ts[f];
    uint32_t w = W;
    if (t >= t_begin && t < t_end) {
        const double x = window_s > 0.0 ? floor((t - t_begin) / window_s) : 0.0;
        if (x >= 0.0 && x < (double)W) w = (uint32_t)x;
    }
    const float gx = gaze[3 * f], gy = gaze[3 * f + 1], gz = gaze[3 * f + 2];
    const bool ok = isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(eye[3 * f]) && isfinite(eye[3 * f + 1]) &&
                    isfinite(eye[3 * f + 2]) && isfinite(dur[f]) && dur[f] >= 0.f && (gx != 0.f || gy != 0.f || gz != 0.f) &&
                    !isnan(t);
    if (!ok) {
        atomicCAS(err, 0, 3);
        w = W;
    }
    keys[f] = s * (W + 1) + w;
    vals[f] = f;
    if (w < W) atomicAdd(&n_valid[s], 1u);
}

__global__ void k_bfix_pack(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                            const float* __restrict__ eye, const float* __restrict__ gaze,
                            const float* __restrict__ dur, uint32_t nf, uint32_t W, float wnorm,
                            float4* __restrict__ packed) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    const uint32_t f = vals[i];
    float rx = gaze[3 * f], ry = gaze[3 * f + 1], rz = gaze[3 * f + 2];
    const float rn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry)), __fmul_rn(rz, rz)));
    rx = __fdiv_rn(rx, rn);
    ry = __fdiv_rn(ry, rn);
    rz = __fdiv_rn(rz, rn);
    packed[2 * i + 0] = make_float4(eye[3 * f], eye[3 * f + 1], eye[3 * f + 2], __fmul_rn(dur[f], wnorm));
    packed[2 * i + 1] = make_float4(rx, ry, rz, __uint_as_float(keys[i] % (W + 1)));
}

struct AccConst {
    float C2, K, tmax;
};

// Warp tiles of the batch use the spread layout (four 32-sample runs over 1024 samples).
constexpr uint32_t BATCH_GROUP = 8;
constexpr int BATCH_BUCKETS = 3;   // sessions of < 2^14, < 2^17 and more triangles

int bucket_of_tris(uint32_t nt) { return nt < (1u << 14) ? 0 : nt < (1u << 17) ? 1 : 2; }

// Warp-tile sizes of the batched kernels, by tile index: 4, 2 or 1 samples per thread.
constexpr int BATCH_TILES = 3;
constexpr int BATCH_TILE_SPT[BATCH_TILES] = {4, 2, 1};

// Persistent: every warp pulls work items (session, warp tile of 32 S samples per run) from `work`
// until none is left. FSM: fixations staged in the warp's shared memory.
template <bool COMPACT, bool WIDE, int MINB, int S = SPT, bool FSM = false>
__global__ void __launch_bounds__(ACC_THREADS, MINB) k_accumulate_batch(const SessionDev* __restrict__ sess,
                                                                        const uint2* __restrict__ items,
                                                                        uint32_t n_items, unsigned int* __restrict__ work,
                                                                        AccConst C, int* __restrict__ err) {
    constexpr int QN = COMPACT ? ACC_THREADS * S : 1;
    __shared__ float4 wsmp[QN];
    __shared__ float2 wacc[QN];
    __shared__ float4 wbox[ACC_THREADS / 32];
    __shared__ uint16_t qslot[QN];
    __shared__ float qg[QN];
    __shared__ float4 wfix[FSM ? (ACC_THREADS / 32) * 64 : 1];
    const int lane = threadIdx.x & 31;
    const int wb = COMPACT ? (threadIdx.x >> 5) * 32 * S : 0;
    const DebugOut dbg{nullptr, nullptr, nullptr, nullptr, nullptr};
    for (;;) {
        uint32_t it = 0;
        if (lane == 0) it = atomicAdd(work, 1u);
        it = __shfl_sync(0xffffffffu, it, 0);
        if (it >= n_items) break;
        const uint2 wi = items[it];
        const SessionDev Sd = sess[wi.x];
        AccParams P;
        P.C2 = C.C2;
        P.K = C.K;
        P.tmax = C.tmax;
        P.ns = Sd.ns;
        P.W = Sd.W;
        P.nt = Sd.nt;
        P.dbg_cap = 0;
        P.group = BATCH_GROUP;
        P.tanphi = sqrtf(C.K) * 1.00001f;
        TileStats st;
        warp_tile<false, COMPACT, WIDE, false, S, FSM>(wi.y, Sd.spos, Sd.sidx, Sd.fix, *Sd.n_fix, Sd.nodes, Sd.tris, P,
                                                       Sd.out, Sd.max_bits, wsmp + wb, wacc + wb, qslot + wb, qg + wb,
                                                       wbox + (threadIdx.x >> 5), nullptr, dbg, err, st,
                                                       FSM ? wfix + (threadIdx.x >> 5) * 64 : nullptr);
        warp_stats_commit(st, Sd.counters);
    }
}

__global__ void k_bnormalize(const SessionDev* __restrict__ sess) {
    const SessionDev S = sess[blockIdx.y];
    const uint64_t total = (uint64_t)S.ns * S.W;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x) {
        const float m = __uint_as_float(S.max_bits[i / S.ns]);
        S.out[i] = m > 0.f ? __fdiv_rn(S.out[i], m) : 0.f;
    }
}

// Each map keeps its session's valid-fixation count in counters[3] (read by gm_map_info).
__global__ void k_bcount(const SessionDev* __restrict__ sess, uint32_t n) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) sess[i].counters[3] = *sess[i].n_fix;
}

template <bool Cm, bool Wd, int Mb, int S = SPT, bool Fs = false>
int occupancy_of() {
    int b = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_accumulate_batch<Cm, Wd, Mb, S, Fs>, ACC_THREADS, 0);
    return std::max(b, 1);
}

// Variant codes: bits 0-2 the kernel (ray queue, 4-wide tree, 64-register cap), 8 x the tile index
// (ray-queue binary tree only: 2 samples per thread with fixations staged in shared memory, or 1,
// which also takes 64 registers).
void launch_batch(int code, int grid, cudaStream_t s, const SessionDev* sess, const uint2* items, uint32_t n_items,
                  unsigned int* work, AccConst C, int* err) {
#define GM_B(Cm, Wd, Mb, S_, Fs) \
    k_accumulate_batch<Cm, Wd, Mb, S_, Fs><<<grid, ACC_THREADS, 0, s>>>(sess, items, n_items, work, C, err)
    const int t = code >> 3;
    if (t == 2) GM_B(true, false, 4, 1, true);
    else if (t == 1 && (code & 7) == 5) GM_B(true, false, 4, 2, true);
    else if (t == 1) GM_B(true, false, 3, 2, true);
    else switch (code & 7) {
        case 0: GM_B(false, false, 3, SPT, false); break;
        case 1: GM_B(true, false, 3, SPT, false); break;
        case 2: GM_B(false, true, 3, SPT, false); break;
        case 3: GM_B(true, true, 3, SPT, false); break;
        case 4: GM_B(false, false, 4, SPT, false); break;
        case 5: GM_B(true, false, 4, SPT, false); break;
        case 6: GM_B(false, true, 4, SPT, false); break;
        default: GM_B(true, true, 4, SPT, false); break;
    }
#undef GM_B
}

int batch_occupancy(int code) {
    const int t = code >> 3;
    if (t == 2) return occupancy_of<true, false, 4, 1, true>();
    if (t == 1) return (code & 7) == 5 ? occupancy_of<true, false, 4, 2, true>() : occupancy_of<true, false, 3, 2, true>();
    switch (code & 7) {
        case 0: return occupancy_of<false, false, 3>();
        case 1: return occupancy_of<true, false, 3>();
        case 2: return occupancy_of<false, true, 3>();
        case 3: return occupancy_of<true, true, 3>();
        case 4: return occupancy_of<false, false, 4>();
        case 5: return occupancy_of<true, false, 4>();
        case 6: return occupancy_of<false, true, 4>();
        default: return occupancy_of<true, true, 4>();
    }
}

// variant code <-> GM_F_* flags (the ray-queue binary tree takes 1 sample per thread by default)
int code_of_flags(int flags) {
    const int base =
        ((flags & GM_F_NO_COMPACT) ? 0 : 1) | ((flags & GM_F_WIDE_BVH) ? 2 : 0) | ((flags & GM_F_REGCAP64) ? 4 : 0);
    if ((base & 3) != 1) return base;
    if (flags & GM_F_SPT4) return base;
    if (flags & GM_F_SPT2) return base + 8;
    return 1 + 16;
}
int flags_of_code(int code) {
    const int t = code >> 3, base = code & 7;
    return ((base & 1) ? 0 : GM_F_NO_COMPACT) | ((base & 2) ? GM_F_WIDE_BVH : 0) | ((base & 4) ? GM_F_REGCAP64 : 0) |
           ((base & 3) == 1 ? (t == 0 ? GM_F_SPT4 : t == 1 ? GM_F_SPT2 : 0) : 0);
}
// the codes the batched autotuner times
constexpr int BATCH_CODES[] = {0, 1, 2, 3, 4, 5, 6, 7, 9, 13, 17};
int tile_of_code(int code) { return code >> 3; }
constexpr int VARIANT_MASK = GM_F_NO_COMPACT | GM_F_WIDE_BVH | GM_F_REGCAP64 | GM_F_SPT1 | GM_F_SPT2 | GM_F_SPT4;

// ---- tuning cache ------------------------------------------------------------------------------
std::mutex g_tune_mutex;
std::map<std::string, int> g_tune;
bool g_tune_loaded = false;

std::string bucket_key(const char* kind, uint64_t ns, uint64_t nf, uint64_t nt) {
    auto lg = [](uint64_t v) { return v ? (int)std::floor(std::log2((double)v)) : -1; };
    std::ostringstream o;
    o << kind << ":" << lg(ns) << ":" << lg(nf) << ":" << lg(nt);
    return o.str();
}

void tune_load_locked() {
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char* path = std::getenv("GM_TUNE_CACHE");
    if (!path) return;
    std::ifstream in(path);
    std::string line;
    // one entry per line: "key": flags,
    while (std::getline(in, line)) {
        size_t a = line.find('"'), b = line.find('"', a + 1), c = line.find(':', b);
        if (a == std::string::npos || b == std::string::npos || c == std::string::npos) continue;
        g_tune[line.substr(a + 1, b - a - 1)] = std::atoi(line.c_str() + c + 1);
    }
}

void tune_store_locked() {
    const char* path = std::getenv("GM_TUNE_CACHE");
    if (!path) return;
    std::ofstream out(path);
    out << "{\n";
    size_t i = 0;
    for (auto& kv : g_tune) out << "  \"" << kv.first << "\": " << kv.second << (++i < g_tune.size() ? ",\n" : "\n");
    out << "}\n";
}

}  // namespace

struct gm_batch {
    gm_ctx* ctx = nullptr;
    uint32_t n = 0;
    gm_params prm{};
    int flags = 0;
    uint32_t W = 1;
    uint32_t nf_total = 0;
    uint64_t pairs = 0;
    std::vector<gm_map*> maps;
    std::vector<const gm_scene*> scenes;
    std::vector<uint32_t> fix_off;
    std::vector<SessionDev> host_sess;
    SessionDev* sess = nullptr;
    uint2* items[BATCH_TILES] = {};   // the work list for each warp-tile size
    uint32_t n_items[BATCH_TILES] = {};
    unsigned int* work = nullptr;
    uint32_t* n_valid = nullptr;
    float *eye = nullptr, *gaze = nullptr, *dur = nullptr;
    double* ts = nullptr;
    uint32_t* sess_of = nullptr;
    uint32_t *keys = nullptr, *vals = nullptr, *tkeys = nullptr, *tvals = nullptr, *hist = nullptr;
    float4* packed = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    int launches_per_run = 0;
    // size buckets (by triangles): each a contiguous run of the work list, its own counter, its
    // own kernel variant and its own persistent launch, timed by events recorded in the graph
    uint32_t bucket_begin[BATCH_TILES][BATCH_BUCKETS + 1] = {};
    uint32_t bucket_sessions[BATCH_BUCKETS] = {};
    int bflags[BATCH_BUCKETS] = {};
    cudaEvent_t bev[BATCH_BUCKETS][2] = {};
    cudaStream_t bs[BATCH_BUCKETS] = {};       // capture-time fork streams of the bucket launches
    cudaEvent_t fork = nullptr, join[BATCH_BUCKETS] = {};
};

// work items of bucket k in the work list of its variant's tile size
static uint32_t bucket_items(const gm_batch* b, int k) {
    const int tk = tile_of_code(code_of_flags(b->bflags[k]));
    return b->bucket_begin[tk][k + 1] - b->bucket_begin[tk][k];
}
// whether bucket k holds any sample (the same for every tile size)
static bool bucket_busy(const gm_batch* b, int k) { return b->bucket_begin[0][k + 1] > b->bucket_begin[0][k]; }

static void batch_release_graph(gm_batch* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
}

// Capture the whole batched call into a graph with the variants in b->bflags. concurrent: the
// buckets' launches run on forked streams (one bucket's tail overlaps the next one's start);
// else one after another (the autotuner times each bucket alone).
static gm_status batch_capture(gm_batch* b, bool concurrent = true) {
    batch_release_graph(b);
    // the session table points at the tree its bucket's variant traverses
    for (uint32_t i = 0; i < b->n; ++i) {
        const gm_scene* sc = b->scenes[i];
        const int f = b->bflags[bucket_of_tris(sc->n_tris)];
        b->host_sess[i].nodes = (f & GM_F_WIDE_BVH) && sc->nodes4 ? sc->nodes4 : sc->nodes;
    }
    GM_TRY_CUDA(cudaMemcpy(b->sess, b->host_sess.data(), sizeof(SessionDev) * b->n, cudaMemcpyHostToDevice));
    cudaStream_t cs;
    GM_TRY_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
    int launches = 0;
    const double tan_t = std::tan((double)b->prm.theta_rad);
    gm_status st = GM_OK;
    if (e == cudaSuccess) {
        cudaMemsetAsync(b->work, 0, sizeof(unsigned int) * BATCH_BUCKETS, cs);
        cudaMemsetAsync(b->n_valid, 0, sizeof(uint32_t) * b->n, cs);
        for (uint32_t i = 0; i < b->n; ++i) {
            gm_map* m = b->maps[i];
            cudaMemsetAsync(m->max_bits, 0, sizeof(unsigned int) * m->W, cs);
            cudaMemsetAsync(m->counters, 0, sizeof(unsigned long long) * 8, cs);
            if (m->W > 1 && m->ns) cudaMemsetAsync(m->values, 0, sizeof(float) * m->W * m->ns, cs);
        }
        if (b->nf_total > 0) {
            k_bfix_keys<<<gm_div_up(b->nf_total, 256), 256, 0, cs>>>(
                b->ts, b->eye, b->gaze, b->dur, b->sess_of, b->nf_total, b->prm.t_begin, b->prm.t_end,
                b->prm.window_s > 0.0 ? b->prm.window_s : 0.0, b->W, b->keys, b->vals, b->n_valid, b->ctx->dev_err);
            ++launches;
            const uint64_t kmax = (uint64_t)b->n * (b->W + 1);
            int bits = 1;
            while (bits < 32 && (1ull << bits) <= kmax) ++bits;
            st = gm_radix_sort_u32_prealloc(b->keys, b->vals, b->nf_total, bits, b->tkeys, b->tvals, b->hist, cs,
                                            &launches);
            const float wnorm = (float)(1.0 / (tan_t * std::sqrt(2.0 * 3.14159265358979323846)));
            k_bfix_pack<<<gm_div_up(b->nf_total, 256), 256, 0, cs>>>(b->keys, b->vals, b->eye, b->gaze, b->dur,
                                                                      b->nf_total, b->W, wnorm, b->packed);
            ++launches;
        }
        if (b->n_items[0] > 0) {
            AccConst C;
            C.C2 = (float)(1.4426950408889634 / (2.0 * tan_t * tan_t));
            C.K = (float)((double)b->prm.cutoff_sigmas * tan_t * (double)b->prm.cutoff_sigmas * tan_t);
            C.tmax = 1.0f - b->prm.eps_rel;
            if (concurrent) {
                cudaEventRecord(b->fork, cs);   // (inside the capture: an ordering edge only)
                for (int k = 0; k < BATCH_BUCKETS; ++k) cudaStreamWaitEvent(b->bs[k], b->fork, 0);
            }
            for (int k = 0; k < BATCH_BUCKETS; ++k) {
                const int code = code_of_flags(b->bflags[k]);
                const int tk = tile_of_code(code);
                const uint32_t i0 = b->bucket_begin[tk][k], i1 = b->bucket_begin[tk][k + 1];
                cudaStream_t ks = concurrent ? b->bs[k] : cs;
                if (i1 > i0) {
                    const int grid = (int)std::min<uint64_t>((uint64_t)b->ctx->n_sm * batch_occupancy(code),
                                                             gm_div_up(i1 - i0, ACC_THREADS / 32));
                    // external event records: the graph records them when it runs (a plain record in
                    // a capture only orders the work)
                    cudaEventRecordWithFlags(b->bev[k][0], ks, cudaEventRecordExternal);
                    launch_batch(code, grid, ks, b->sess, b->items[tk] + i0, i1 - i0, b->work + k, C, b->ctx->dev_err);
                    cudaEventRecordWithFlags(b->bev[k][1], ks, cudaEventRecordExternal);
                    ++launches;
                }
                if (concurrent) {
                    cudaEventRecord(b->join[k], ks);
                    cudaStreamWaitEvent(cs, b->join[k], 0);
                }
            }
        }
        if (b->prm.normalize) {
            dim3 g(std::max(1, b->ctx->n_sm * 8 / (int)std::max<uint32_t>(1, b->n)), b->n);
            k_bnormalize<<<g, 256, 0, cs>>>(b->sess);
            ++launches;
        }
        k_bcount<<<gm_div_up(b->n, 256), 256, 0, cs>>>(b->sess, b->n);
        ++launches;
        e = cudaStreamEndCapture(cs, &b->graph);
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    cudaStreamDestroy(cs);
    if (st != GM_OK) return st;
    if (e != cudaSuccess) return gm_cuda_error(e, "gm_batch: graph capture");
    b->launches_per_run = launches;
    return GM_OK;
}

extern "C" void gm_batch_free(gm_batch* b) {
    if (b) {
        for (int k = 0; k < BATCH_BUCKETS; ++k) {
            for (int q = 0; q < 2; ++q)
                if (b->bev[k][q]) cudaEventDestroy(b->bev[k][q]);
            if (b->join[k]) cudaEventDestroy(b->join[k]);
            if (b->bs[k]) cudaStreamDestroy(b->bs[k]);
        }
        if (b->fork) cudaEventDestroy(b->fork);
    }
    if (!b) return;
    batch_release_graph(b);
    for (gm_map* m : b->maps) gm_map_free(m);
    cudaFree(b->sess);
    for (int t = 0; t < BATCH_TILES; ++t) cudaFree(b->items[t]);
    cudaFree(b->work);
    cudaFree(b->n_valid);
    cudaFree(b->eye);
    cudaFree(b->gaze);
    cudaFree(b->dur);
    cudaFree(b->ts);
    cudaFree(b->sess_of);
    cudaFree(b->keys);
    cudaFree(b->vals);
    cudaFree(b->tkeys);
    cudaFree(b->tvals);
    cudaFree(b->hist);
    cudaFree(b->packed);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
}

extern "C" gm_status gm_batch_create(gm_ctx* ctx, const gm_session_desc* ss, uint32_t n, const gm_params* prm,
                                     gm_stream stream, gm_batch** out) {
    if (!ctx || !ss || !prm || !out || n == 0) return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_create: null argument");
    *out = nullptr;
    if (!(prm->theta_rad > 0.f) || !(prm->theta_rad < 1.5f) || !(prm->cutoff_sigmas > 0.f) ||
        !(prm->eps_rel >= 0.f && prm->eps_rel < 1.f) || std::isnan(prm->t_begin) || std::isnan(prm->t_end) ||
        !(prm->t_begin < prm->t_end))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_create: invalid parameters");
    uint64_t W = 1;
    if (prm->window_s > 0.0) {
        if (!std::isfinite(prm->t_begin) || !std::isfinite(prm->t_end) || !std::isfinite(prm->window_s))
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_create: windows need a finite interval");
        W = std::max<uint64_t>(1, (uint64_t)std::ceil((prm->t_end - prm->t_begin) / prm->window_s));
        if (W > (1u << 20)) return gm_set_error(GM_ERR_UNSUPPORTED, "gm_batch_create: more than 2^20 windows");
    }
    for (uint32_t i = 0; i < n; ++i) {
        if (!ss[i].scene || !ss[i].samples || ss[i].samples->scene != ss[i].scene)
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_create: session " + std::to_string(i) + " is incomplete");
        if (ss[i].fix.n > 0 && (!ss[i].fix.eye_xyz || !ss[i].fix.gaze_xyz || !ss[i].fix.duration_s || !ss[i].fix.timestamp_s))
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_create: null fixation array");
        if ((uint64_t)n * (W + 1) > 0xffffffffull)
            return gm_set_error(GM_ERR_UNSUPPORTED, "gm_batch_create: sessions x windows exceed 2^32");
    }
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    gm_batch* b = new gm_batch();
    b->ctx = ctx;
    b->n = n;
    b->prm = *prm;
    b->W = (uint32_t)W;
    b->flags = prm->flags & VARIANT_MASK;
    for (int k = 0; k < BATCH_BUCKETS; ++k) b->bflags[k] = b->flags;
    auto fail = [&](gm_status st) {
        cudaStreamSynchronize(s);
        gm_batch_free(b);
        return st;
    };
    gm_status st;
    // per-session maps
    b->fix_off.resize(n + 1, 0);
    for (uint32_t i = 0; i < n; ++i) {
        b->fix_off[i + 1] = b->fix_off[i] + ss[i].fix.n;
        gm_map* m = new gm_map();
        m->ctx = ctx;
        m->W = b->W;
        m->ns = ss[i].samples->n;
        m->stream = s;
        m->stats.n_windows = b->W;
        b->maps.push_back(m);
        if ((st = gm_alloc((void**)&m->values, sizeof(float) * m->W * (m->ns ? m->ns : 1), s)) != GM_OK) return fail(st);
        if ((st = gm_alloc((void**)&m->max_bits, sizeof(unsigned int) * m->W, s)) != GM_OK) return fail(st);
        if ((st = gm_alloc((void**)&m->counters, sizeof(unsigned long long) * 8, s)) != GM_OK) return fail(st);
        b->pairs += (uint64_t)ss[i].fix.n * m->ns;
    }
    b->nf_total = b->fix_off[n];
    const uint32_t nf = b->nf_total;
    const size_t nfa = nf ? nf : 1;
    if ((st = gm_alloc((void**)&b->eye, sizeof(float) * 3 * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->gaze, sizeof(float) * 3 * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->dur, sizeof(float) * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->ts, sizeof(double) * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->sess_of, sizeof(uint32_t) * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->keys, sizeof(uint32_t) * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->vals, sizeof(uint32_t) * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->tkeys, sizeof(uint32_t) * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->tvals, sizeof(uint32_t) * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->hist, sizeof(uint32_t) * gm_radix_sort_u32_hist_words(nf ? nf : 1), s)) != GM_OK ||
        (st = gm_alloc((void**)&b->packed, sizeof(float4) * 2 * nfa, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->n_valid, sizeof(uint32_t) * n, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->work, sizeof(unsigned int) * BATCH_BUCKETS, s)) != GM_OK ||
        (st = gm_alloc((void**)&b->sess, sizeof(SessionDev) * n, s)) != GM_OK)
        return fail(st);
    // stage fixations (host or device sources) into the concatenated buffers
    std::vector<uint32_t> sess_of(nfa, 0);
    cudaError_t e = cudaSuccess;
    for (uint32_t i = 0; i < n && e == cudaSuccess; ++i) {
        const gm_fixations& f = ss[i].fix;
        const uint32_t o = b->fix_off[i];
        for (uint32_t k = 0; k < f.n; ++k) sess_of[o + k] = i;
        if (f.n == 0) continue;
        e = cudaMemcpyAsync(b->eye + 3 * o, f.eye_xyz, sizeof(float) * 3 * f.n, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->gaze + 3 * o, f.gaze_xyz, sizeof(float) * 3 * f.n, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->dur + o, f.duration_s, sizeof(float) * f.n, cudaMemcpyDefault, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(b->ts + o, f.timestamp_s, sizeof(double) * f.n, cudaMemcpyDefault, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->sess_of, sess_of.data(), sizeof(uint32_t) * nfa, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_batch_create: staging"));
    // session table
    b->host_sess.resize(n);
    for (uint32_t i = 0; i < n; ++i) {
        gm_samples* sm = ss[i].samples;
        gm_scene* sc = ss[i].scene;
        SessionDev& d = b->host_sess[i];
        b->scenes.push_back(sc);
        d.spos = sm->work_pos ? sm->work_pos : sm->pos;
        d.sidx = sm->work_idx;
        d.fix = b->packed + 2 * (size_t)b->fix_off[i];
        d.n_fix = b->n_valid + i;
        d.nodes = (b->flags & GM_F_WIDE_BVH) && sc->nodes4 ? sc->nodes4 : sc->nodes;
        d.tris = sc->bvh_tris;
        d.out = b->maps[i]->values;
        d.max_bits = b->maps[i]->max_bits;
        d.counters = b->maps[i]->counters;
        d.ns = (uint32_t)sm->n;
        d.nt = sc->n_tris;
        d.W = b->W;
        d.pad = 0;
        if (sm->n > 0 && !sm->work_idx)
            return fail(gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_create: samples without a work order"));
    }
    e = cudaMemcpyAsync(b->sess, b->host_sess.data(), sizeof(SessionDev) * n, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_batch_create: session table"));
    // work list: by size bucket, within a bucket longest processing time first
    std::vector<uint32_t> order(n);
    std::iota(order.begin(), order.end(), 0u);
    std::stable_sort(order.begin(), order.end(), [&](uint32_t a, uint32_t c) {
        const int ba = bucket_of_tris(ss[a].scene->n_tris), bc = bucket_of_tris(ss[c].scene->n_tris);
        return ba != bc ? ba < bc : ss[a].fix.n > ss[c].fix.n;
    });
    for (uint32_t i : order) ++b->bucket_sessions[bucket_of_tris(ss[i].scene->n_tris)];
    std::vector<uint2> items[BATCH_TILES];
    for (int tk = 0; tk < BATCH_TILES; ++tk) {
        const uint64_t per_tile = 32ull * BATCH_TILE_SPT[tk] * BATCH_GROUP;
        for (uint32_t i : order) {
            const int k = bucket_of_tris(ss[i].scene->n_tris);
            const uint32_t tiles = (uint32_t)(gm_div_up(ss[i].samples->n, per_tile) * BATCH_GROUP);
            for (uint32_t t = 0; t < tiles; ++t) items[tk].push_back(make_uint2(i, t));
            for (int q = k + 1; q <= BATCH_BUCKETS; ++q) b->bucket_begin[tk][q] = (uint32_t)items[tk].size();
        }
        b->n_items[tk] = (uint32_t)items[tk].size();
        const size_t nb = sizeof(uint2) * (items[tk].empty() ? 1 : items[tk].size());
        if ((st = gm_alloc((void**)&b->items[tk], nb, s)) != GM_OK) return fail(st);
        if (!items[tk].empty()) {
            e = cudaMemcpyAsync(b->items[tk], items[tk].data(), sizeof(uint2) * items[tk].size(),
                                cudaMemcpyHostToDevice, s);
            if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_batch_create: work list"));
        }
    }
    if ((e = cudaEventCreate(&b->ev0)) != cudaSuccess || (e = cudaEventCreate(&b->ev1)) != cudaSuccess)
        return fail(gm_cuda_error(e, "gm_batch_create: events"));
    for (int k = 0; k < BATCH_BUCKETS; ++k) {
        for (int q = 0; q < 2; ++q)
            if ((e = cudaEventCreate(&b->bev[k][q])) != cudaSuccess)
                return fail(gm_cuda_error(e, "gm_batch_create: events"));
        if ((e = cudaEventCreateWithFlags(&b->join[k], cudaEventDisableTiming)) != cudaSuccess ||
            (e = cudaStreamCreateWithFlags(&b->bs[k], cudaStreamNonBlocking)) != cudaSuccess)
            return fail(gm_cuda_error(e, "gm_batch_create: streams"));
    }
    if ((e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming)) != cudaSuccess)
        return fail(gm_cuda_error(e, "gm_batch_create: events"));
    // everything above is stream-ordered on s; the graph replays on any stream after it
    if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return fail(gm_cuda_error(e, "gm_batch_create"));
    if ((st = batch_capture(b)) != GM_OK) return fail(st);
    *out = b;
    return GM_OK;
}

extern "C" gm_status gm_batch_run(gm_batch* b, gm_stream stream) {
    if (!b) return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_run: null batch");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(b->ctx->device));
    GM_TRY_CUDA(cudaEventRecord(b->ev0, s));
    GM_TRY_CUDA(cudaGraphLaunch(b->exec, s));
    GM_TRY_CUDA(cudaEventRecord(b->ev1, s));
    for (gm_map* m : b->maps) m->stream = s;
    b->ctx->launches += b->launches_per_run;
    return GM_OK;
}

extern "C" gm_status gm_batch_info(gm_batch* b, uint32_t* n_sessions, uint64_t* n_items, uint64_t* pairs,
                                   float* last_ms, int32_t* variant_flags) {
    if (!b) return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_info: null batch");
    if (n_sessions) *n_sessions = b->n;
    if (n_items) {
        *n_items = 0;
        for (int k = 0; k < BATCH_BUCKETS; ++k) *n_items += bucket_items(b, k);
    }
    if (pairs) *pairs = b->pairs;
    if (variant_flags) {
        // the variant of the bucket with the most samples
        int kb = 0;
        for (int k = 1; k < BATCH_BUCKETS; ++k)
            if (b->bucket_begin[0][k + 1] - b->bucket_begin[0][k] > b->bucket_begin[0][kb + 1] - b->bucket_begin[0][kb])
                kb = k;
        *variant_flags = b->bflags[kb];
    }
    if (last_ms) {
        *last_ms = 0.f;
        if (cudaEventQuery(b->ev1) != cudaErrorNotReady) {
            GM_TRY_CUDA(cudaEventSynchronize(b->ev1));
            cudaError_t e = cudaEventElapsedTime(last_ms, b->ev0, b->ev1);
            if (e != cudaSuccess) {
                cudaGetLastError();
                *last_ms = 0.f;
            }
        }
    }
    return GM_OK;
}

extern "C" gm_status gm_batch_map(gm_batch* b, uint32_t i, gm_map** out) {
    if (!b || !out || i >= b->n) return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_map: bad session index");
    *out = b->maps[i];
    return GM_OK;
}

extern "C" gm_status gm_accumulate_batch(gm_ctx* ctx, const gm_session_desc* ss, uint32_t n, const gm_params* prm,
                                         gm_stream stream, gm_map** out_per_session) {
    if (!out_per_session) return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_batch: null output");
    gm_batch* b = nullptr;
    GM_TRY(gm_batch_create(ctx, ss, n, prm, stream, &b));
    gm_status st = gm_batch_run(b, stream);
    if (st == GM_OK) {
        cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
        if (e != cudaSuccess) st = gm_cuda_error(e, "gm_accumulate_batch");
    }
    if (st != GM_OK) {
        gm_batch_free(b);
        return st;
    }
    for (uint32_t i = 0; i < n; ++i) out_per_session[i] = b->maps[i];
    b->maps.clear();  // ownership passes to the caller
    gm_batch_free(b);
    return GM_OK;
}

// ---- autotuning ---------------------------------------------------------------------------------

extern "C" gm_status gm_batch_autotune(gm_batch* b, gm_stream stream, int32_t* best_flags, float* best_ms) {
    if (!b) return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_autotune: null batch");
    // per bucket: its totals for the cache key, then every variant timed on its own launch (events
    // recorded in the graph around each bucket's launch), the fastest kept
    uint64_t ns_k[BATCH_BUCKETS] = {}, nf_k[BATCH_BUCKETS] = {}, nt_k[BATCH_BUCKETS] = {};
    for (uint32_t i = 0; i < b->n; ++i) {
        const int k = bucket_of_tris(b->host_sess[i].nt);
        ns_k[k] += b->host_sess[i].ns;
        nf_k[k] += b->fix_off[i + 1] - b->fix_off[i];
        nt_k[k] += b->host_sess[i].nt;
    }
    int best[BATCH_BUCKETS];
    float best_t[BATCH_BUCKETS];
    bool todo = false;
    std::string keys[BATCH_BUCKETS];
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_load_locked();
        for (int k = 0; k < BATCH_BUCKETS; ++k) {
            keys[k] = bucket_key(("batch" + std::to_string(k)).c_str(), ns_k[k], nf_k[k], nt_k[k]);
            auto it = g_tune.find(keys[k]);
            best[k] = it != g_tune.end() ? it->second : -1;
            best_t[k] = 1e30f;
            todo |= best[k] < 0 && bucket_busy(b, k);
        }
    }
    if (todo) {
        for (const int code : BATCH_CODES) {
            for (int k = 0; k < BATCH_BUCKETS; ++k) b->bflags[k] = flags_of_code(code);
            GM_TRY(batch_capture(b, false));   // buckets one after another: each timed alone
            float t[BATCH_BUCKETS] = {1e30f, 1e30f, 1e30f};
            for (int rep = 0; rep < 2; ++rep) {
                GM_TRY(gm_batch_run(b, stream));
                GM_TRY_CUDA(cudaEventSynchronize(b->ev1));
                for (int k = 0; k < BATCH_BUCKETS; ++k) {
                    if (!bucket_busy(b, k)) continue;
                    float ms = 0.f;
                    const cudaError_t e = cudaEventElapsedTime(&ms, b->bev[k][0], b->bev[k][1]);
                    if (e != cudaSuccess) {
                        cudaGetLastError();   // leave no error behind for the next launch check
                        return gm_cuda_error(e, "gm_batch_autotune: bucket timing");
                    }
                    t[k] = std::min(t[k], ms);
                }
            }
            for (int k = 0; k < BATCH_BUCKETS; ++k)
                if (t[k] < best_t[k]) {
                    best_t[k] = t[k];
                    best[k] = flags_of_code(code);
                }
        }
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        for (int k = 0; k < BATCH_BUCKETS; ++k)
            if (bucket_busy(b, k)) g_tune[keys[k]] = best[k];
        tune_store_locked();
    }
    for (int k = 0; k < BATCH_BUCKETS; ++k) b->bflags[k] = best[k] >= 0 ? best[k] : b->flags;
    GM_TRY(batch_capture(b));
    // the whole replay with the chosen variants
    float total = 0.f;
    GM_TRY(gm_batch_run(b, stream));
    GM_TRY_CUDA(cudaEventSynchronize(b->ev1));
    GM_TRY_CUDA(cudaEventElapsedTime(&total, b->ev0, b->ev1));
    if (best_flags) GM_TRY(gm_batch_info(b, nullptr, nullptr, nullptr, nullptr, best_flags));
    if (best_ms) *best_ms = total;
    return GM_OK;
}

extern "C" gm_status gm_batch_buckets(gm_batch* b, uint32_t* n_buckets, int32_t* flags, uint32_t* sessions,
                                      uint32_t* work_items, float* last_ms) {
    if (!b) return gm_set_error(GM_ERR_INVALID_ARG, "gm_batch_buckets: null batch");
    if (n_buckets) *n_buckets = BATCH_BUCKETS;
    bool done = last_ms && cudaEventQuery(b->ev1) != cudaErrorNotReady;
    if (done) GM_TRY_CUDA(cudaEventSynchronize(b->ev1));
    for (int k = 0; k < BATCH_BUCKETS; ++k) {
        if (flags) flags[k] = b->bflags[k];
        if (sessions) sessions[k] = b->bucket_sessions[k];
        if (work_items) work_items[k] = bucket_items(b, k);
        if (last_ms) {
            last_ms[k] = 0.f;
            if (done && bucket_busy(b, k) &&
                cudaEventElapsedTime(&last_ms[k], b->bev[k][0], b->bev[k][1]) != cudaSuccess) {
                cudaGetLastError();
                last_ms[k] = 0.f;
            }
        }
    }
    return GM_OK;
}

extern "C" gm_status gm_autotune_accumulate(gm_scene* sc, gm_samples* sm, const gm_fixations* fx, const gm_params* prm,
                                            gm_stream stream, int32_t* best_flags, float* best_ms) {
    if (!sc || !sm || !fx || !prm || !best_flags)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_autotune_accumulate: null argument");
    const std::string key = bucket_key("plain", sm->n, fx->n, sc->n_tris);
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        tune_load_locked();
        auto it = g_tune.find(key);
        if (it != g_tune.end()) {
            *best_flags = it->second;
            if (best_ms) *best_ms = 0.f;
            return GM_OK;
        }
    }
    // Candidates are ranked on a prefix of the fixations (a sixteenth, at least 256), by the time
    // of the whole call (fixation prep, eye grid, accumulation); the two best are then timed on the
    // full list and the faster is kept, so a prefix that ranks them wrongly costs nothing.
    gm_fixations sub = *fx;
    sub.n = std::min<uint32_t>(fx->n, std::max<uint32_t>(256, fx->n / 16));
    constexpr int kTileFlags = GM_F_TILE_CONSECUTIVE | GM_F_STATIC_TILES;
    constexpr int kShapeFlags = GM_F_BLOCK128 | GM_F_BLOCK512 | GM_F_SPT1 | GM_F_SPT2 | GM_F_SPT4 | GM_F_GRID64 |
                                GM_F_EYE_GRID | GM_F_FIX_L1;
    std::vector<int> cand;
    // BVH: the eight kernel variants (in place or ray queue, binary or 4-wide tree, 80- or
    // 64-register cap), the ray-queue binary tree with 4, 2 or 1 samples per thread (1 takes 64
    // registers either way) and the in-place binary tree also with 1, times the warp-tile shape
    // (spread runs or consecutive samples) and the scheduling (persistent or one tile per warp);
    // then 128-thread blocks of the ray-queue binary tree (4 samples per thread with either cap,
    // or 1) and 512-thread blocks (1 sample per thread)
    for (int shape = 0; shape < 4; ++shape) {
        const int sf = ((shape & 1) ? GM_F_TILE_CONSECUTIVE : 0) | ((shape & 2) ? GM_F_STATIC_TILES : 0);
        for (int v = 0; v < 8; ++v) {
            const int vf = ((v & 1) ? 0 : GM_F_NO_COMPACT) | ((v & 2) ? GM_F_WIDE_BVH : 0) | ((v & 4) ? GM_F_REGCAP64 : 0);
            if ((v & 3) != 1) {
                cand.push_back(vf | sf);
                if (v == 0) cand.push_back(vf | sf | GM_F_SPT1);   // one-sample tiles traced in place
                continue;
            }
            cand.push_back(vf | sf | GM_F_SPT4);
            cand.push_back(vf | sf | GM_F_SPT2);
            if (v == 1) cand.push_back(vf | sf);
        }
        cand.push_back(sf | GM_F_BLOCK128 | GM_F_SPT4);
        cand.push_back(sf | GM_F_BLOCK128 | GM_F_SPT4 | GM_F_REGCAP64);
        cand.push_back(sf | GM_F_BLOCK128);
        cand.push_back(sf | GM_F_BLOCK512);
    }
    // eye grid: 128 or 64 cells a side, samples per thread and block size, spread or consecutive tiles
    const int grid_shapes[7] = {0, GM_F_SPT2, GM_F_SPT1, GM_F_BLOCK128, GM_F_BLOCK128 | GM_F_SPT2,
                                GM_F_BLOCK512 | GM_F_SPT2, GM_F_BLOCK512 | GM_F_SPT1};
    for (int res = 0; res < 2; ++res)
        for (int sh = 0; sh < 7; ++sh)
            for (int tl = 0; tl < 2; ++tl)
                cand.push_back(GM_F_EYE_GRID | (res ? GM_F_GRID64 : 0) | grid_shapes[sh] |
                               (tl ? GM_F_TILE_CONSECUTIVE : 0));
    auto time_of = [&](int f, const gm_fixations* fs, float* out_ms) -> gm_status {
        gm_params p = *prm;
        p.flags = (prm->flags & ~VARIANT_MASK & ~kTileFlags & ~kShapeFlags & ~GM_F_DEBUG_PAIRS) | f | GM_F_TIMING;
        p.normalize = 0;
        float t = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            gm_map* m = nullptr;
            GM_TRY(gm_accumulate_fixations(sc, sm, fs, &p, stream, &m));
            gm_map_stats stt;
            gm_status st = gm_map_info(m, nullptr, nullptr, &stt);
            gm_map_free(m);
            if (st != GM_OK && st != GM_WARN_EMPTY) return st;
            t = std::min(t, stt.prep_ms + stt.grid_ms + stt.accumulate_ms);
        }
        *out_ms = t;
        return GM_OK;
    };
    int b1 = cand[0], b2 = cand[0];
    float t1 = 1e30f, t2 = 1e30f;
    for (int f : cand) {
        float t;
        GM_TRY(time_of(f, &sub, &t));
        if (t < t1) {
            b2 = b1, t2 = t1;
            b1 = f, t1 = t;
        } else if (t < t2) {
            b2 = f, t2 = t;
        }
    }
    int best = b1;
    float best_t = t1;
    if (sub.n < fx->n) {
        float f1, f2 = 1e30f;
        GM_TRY(time_of(b1, fx, &f1));
        if (b2 != b1) GM_TRY(time_of(b2, fx, &f2));
        best = f2 < f1 ? b2 : b1;
        best_t = std::min(f1, f2);
    }
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tune[key] = best;
        tune_store_locked();
    }
    *best_flags = best;
    if (best_ms) *best_ms = best_t;
    return GM_OK;
}
