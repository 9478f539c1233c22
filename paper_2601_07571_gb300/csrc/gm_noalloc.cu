// gm_noalloc.cu -- gm_tri_offsets_noalloc: the per-triangle sample offsets of gm_sample_surface
// for callers that cannot allocate device memory.
//
// Some callers cannot call cudaMalloc at the moment they need this step: an engine plugin whose
// host application owns every byte of device memory through its own allocator, or a real-time
// (per-frame) thread on which an allocation may stall or fail. This entry point computes the
// same offsets as gm_sample_surface (FP64 area per triangle, rint(k A 2^32) in 32.32 fixed
// point, inclusive int64 prefix, rounded starts) from buffers the caller already owns, and
// allocates nothing: the caller passes the inputs and the output, the output array doubles as
// the prefix buffer, and the one scratch buffer -- the per-block partial sums of the prefix --
// is the file-scope device array below, which every GPU that loads this library holds until the
// process exits.
//
// The 32.32 fixed-point prefix is an int64 and would wrap once the scene needs about 2^31 samples;
// each scan block therefore also sums its k A in FP64, and when a block or the whole scene
// exceeds 2^31 - 16 expected samples every partial sum is marked negative, every offset is written
// as 0 and the device error word reports it (gm_sync: GM_ERR_UNSUPPORTED).
#include <cmath>
#include <mutex>
#include <string>

#include "gm_internal.cuh"
#include "gm_scan.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 8;
constexpr int NA_TILE = NA_THREADS * NA_ITEMS;       // triangles per scan block
constexpr uint32_t NA_MAX_BLOCKS = 65536;            // 512 KiB of partial sums

}  // namespace

// One partial sum per scan block; shared by every call in the process on this device.
static __device__ __align__(256) int64_t g_noalloc_scan_part[NA_MAX_BLOCKS];

namespace {

std::mutex g_setup_mutex;

// Expected samples (FP64 sum of k A) above which the int64 prefix could wrap: the FP64 sums are
// within a few samples of the exact ones, and (2^31 - 16 + 4) 2^32 + n_tris / 2 < 2^63.
constexpr double NA_MAX_EXPECTED = 2147483632.0;

// q_i = rint(k_i A_i 2^32) into off[i + 1]; then the partial sum of each tile, or -1 when the
// tile's FP64 sum of k A is too large for the int64 sum.
__global__ void __launch_bounds__(NA_THREADS) na_counts_reduce(const float* __restrict__ tri,
                                                               const double* __restrict__ dens, uint32_t nt,
                                                               int64_t* __restrict__ off, int64_t* __restrict__ part,
                                                               int* __restrict__ err) {
    const uint32_t base = blockIdx.x * (uint32_t)NA_TILE;
    uint64_t s = 0;   // unsigned: a tile that is too large may wrap it (it is then marked, not used)
    double ks = 0.0;
#pragma unroll
    for (int it = 0; it < NA_ITEMS; ++it) {
        const uint32_t i = base + it * NA_THREADS + threadIdx.x;
        if (i >= nt) continue;
        const float* t = tri + 9 * (size_t)i;
        double e1x = __dsub_rn(t[3], t[0]), e1y = __dsub_rn(t[4], t[1]), e1z = __dsub_rn(t[5], t[2]);
        double e2x = __dsub_rn(t[6], t[0]), e2y = __dsub_rn(t[7], t[1]), e2z = __dsub_rn(t[8], t[2]);
        double cx = __dsub_rn(__dmul_rn(e1y, e2z), __dmul_rn(e1z, e2y));
        double cy = __dsub_rn(__dmul_rn(e1z, e2x), __dmul_rn(e1x, e2z));
        double cz = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
        double n2 = __dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz));
        double k = __dmul_rn(dens[i], __dmul_rn(0.5, __dsqrt_rn(n2)));
        if (!(k >= 0.0) || k >= 2147483648.0) {
            atomicCAS(err, 0, GM_DEV_BAD_INDEX);
            k = 0.0;
        }
        const int64_t q = __double2ll_rn(__dmul_rn(k, 4294967296.0));
        off[i + 1] = q;
        s += (uint64_t)q;
        ks += k;
    }
    double ktot;
    block_excl_scan<double, NA_THREADS>(ks, &ktot);
    uint64_t tot;
    block_excl_scan<uint64_t, NA_THREADS>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = ktot <= NA_MAX_EXPECTED ? (int64_t)tot : (int64_t)-1;
}

// Exclusive scan of the partial sums (one block). First the FP64 total of the partials: when a
// partial is marked or the total exceeds the limit, every partial becomes -1 and the error word
// is set; else the exact int64 scan (no partial prefix can then reach 2^63).
__global__ void __launch_bounds__(1024) na_scan_parts(int64_t* __restrict__ part, uint32_t nb, int* __restrict__ err) {
    __shared__ int64_t carry;
    double acc = 0.0;
    int bad = 0;
    for (uint32_t i = threadIdx.x; i < nb; i += 1024) {
        const int64_t v = part[i];
        bad |= v < 0;
        acc += (double)v;
    }
    double total;
    block_excl_scan<double, 1024>(acc, &total);
    if (__syncthreads_or(bad) || !(total <= NA_MAX_EXPECTED * 4294967296.0)) {
        for (uint32_t i = threadIdx.x; i < nb; i += 1024) part[i] = -1;
        if (threadIdx.x == 0) atomicCAS(err, 0, GM_DEV_TOO_MANY_SAMPLES);
        return;
    }
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nb; b0 += 1024) {
        const uint32_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? part[i] : 0;
        int64_t tot;
        const int64_t ex = block_excl_scan<int64_t, 1024>(v, &tot);
        if (i < nb) part[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

// Inclusive prefix inside each tile plus the tile's offset, then start = (S + 2^31) >> 32.
__global__ void __launch_bounds__(NA_THREADS) na_scan_down(int64_t* __restrict__ off, uint32_t nt,
                                                           const int64_t* __restrict__ part) {
    __shared__ int64_t tile[NA_TILE];
    const uint32_t base = blockIdx.x * (uint32_t)NA_TILE;
    if (blockIdx.x == 0 && threadIdx.x == 0) off[0] = 0;
    if (part[blockIdx.x] < 0) {
        // the scene needs too many samples: no offsets (the error word says why)
        for (uint32_t i = base + threadIdx.x; i < nt && i < base + NA_TILE; i += NA_THREADS) off[i + 1] = 0;
        return;
    }
#pragma unroll
    for (int it = 0; it < NA_ITEMS; ++it) {
        const uint32_t i = base + it * NA_THREADS + threadIdx.x;
        tile[it * NA_THREADS + threadIdx.x] = i < nt ? off[i + 1] : 0;
    }
    __syncthreads();
    int64_t v[NA_ITEMS], s = 0;
#pragma unroll
    for (int it = 0; it < NA_ITEMS; ++it) {
        s += tile[threadIdx.x * NA_ITEMS + it];
        v[it] = s;
    }
    int64_t tot;
    const int64_t ex = block_excl_scan<int64_t, NA_THREADS>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int it = 0; it < NA_ITEMS; ++it) tile[threadIdx.x * NA_ITEMS + it] = v[it] + ex;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < NA_ITEMS; ++it) {
        const uint32_t i = base + it * NA_THREADS + threadIdx.x;
        if (i < nt) off[i + 1] = (tile[it * NA_THREADS + threadIdx.x] + ((int64_t)1 << 31)) >> 32;
    }
}

}  // namespace

extern "C" gm_status gm_tri_offsets_noalloc(gm_ctx* ctx, const float* tri_xyz, const double* density_per_tri,
                                            uint32_t n_tris, int64_t* offsets, gm_stream stream) {
    if (!ctx || !offsets || (n_tris > 0 && (!tri_xyz || !density_per_tri)))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_tri_offsets_noalloc: null argument");
    const uint64_t nb = (n_tris + (uint64_t)NA_TILE - 1) / NA_TILE;
    if (nb > NA_MAX_BLOCKS)
        return gm_set_error(GM_ERR_UNSUPPORTED,
                            "gm_tri_offsets_noalloc: " + std::to_string(n_tris) + " triangles exceed the limit of " +
                                std::to_string((uint64_t)NA_MAX_BLOCKS * NA_TILE) + " (fixed scratch of " +
                                std::to_string(NA_MAX_BLOCKS) + " partial sums)");
    if (!gm_is_device_ptr(offsets) || (n_tris > 0 && (!gm_is_device_ptr(tri_xyz) || !gm_is_device_ptr(density_per_tri))))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_tri_offsets_noalloc: every buffer must be device memory");
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    int64_t* part = nullptr;
    {
        // once per context, with its device current: the device address of the scratch array. A
        // context made after a reset of the device (cudaDeviceReset) looks it up again.
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!ctx->noalloc_scratch) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scan_part);
            if (e != cudaSuccess) return gm_cuda_error(e, "gm_tri_offsets_noalloc: cudaGetSymbolAddress");
            ctx->noalloc_scratch = p;
        }
        part = static_cast<int64_t*>(ctx->noalloc_scratch);
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n_tris == 0) {
        GM_TRY_CUDA(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
        return GM_OK;
    }
    na_counts_reduce<<<(uint32_t)nb, NA_THREADS, 0, s>>>(tri_xyz, density_per_tri, n_tris, offsets, part, ctx->dev_err);
    na_scan_parts<<<1, 1024, 0, s>>>(part, (uint32_t)nb, ctx->dev_err);
    na_scan_down<<<(uint32_t)nb, NA_THREADS, 0, s>>>(offsets, n_tris, part);
    ctx->launches += 3;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}
