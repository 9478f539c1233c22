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
#include <cmath>
#include <mutex>
#include <string>

#include "gm_internal.cuh"

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_ITEMS = 8;
constexpr int NA_TILE = NA_THREADS * NA_ITEMS;       // triangles per scan block
constexpr uint32_t NA_MAX_BLOCKS = 65536;            // 512 KiB of partial sums

}  // namespace

// One partial sum per scan block; shared by every call in the process on this device.
static __device__ __align__(256) int64_t g_noalloc_scan_part[NA_MAX_BLOCKS];

namespace {

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_setup_mutex;
int64_t* g_part_addr[NA_MAX_DEVICES] = {};

template <typename T>
__device__ __forceinline__ T na_warp_incl(T v) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T u = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += u;
    }
    return v;
}

template <typename T, int NT>
__device__ __forceinline__ T na_block_excl(T v, T* total) {
    __shared__ T warp_tot[NT / 32];
    __shared__ T tot_sh;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    T inc = na_warp_incl(v);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T w = lane < NT / 32 ? warp_tot[lane] : T(0);
        T wi = na_warp_incl(w);
        if (lane < NT / 32) warp_tot[lane] = wi - w;
        if (lane == NT / 32 - 1) tot_sh = wi;
    }
    __syncthreads();
    T res = warp_tot[warp] + inc - v;
    *total = tot_sh;
    __syncthreads();
    return res;
}

// q_i = rint(k_i A_i 2^32) into off[i + 1]; then the partial sum of each tile.
__global__ void __launch_bounds__(NA_THREADS) na_counts_reduce(const float* __restrict__ tri,
                                                               const double* __restrict__ dens, uint32_t nt,
                                                               int64_t* __restrict__ off, int64_t* __restrict__ part,
                                                               int* __restrict__ err) {
    const uint32_t base = blockIdx.x * (uint32_t)NA_TILE;
    int64_t s = 0;
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
        s += q;
    }
    int64_t tot;
    na_block_excl<int64_t, NA_THREADS>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

// Exclusive scan of the partial sums (one block).
__global__ void __launch_bounds__(1024) na_scan_parts(int64_t* __restrict__ part, uint32_t nb) {
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t b0 = 0; b0 < nb; b0 += 1024) {
        const uint32_t i = b0 + threadIdx.x;
        const int64_t v = i < nb ? part[i] : 0;
        int64_t tot;
        const int64_t ex = na_block_excl<int64_t, 1024>(v, &tot);
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
    const int64_t ex = na_block_excl<int64_t, NA_THREADS>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int it = 0; it < NA_ITEMS; ++it) tile[threadIdx.x * NA_ITEMS + it] = v[it] + ex;
    __syncthreads();
#pragma unroll
    for (int it = 0; it < NA_ITEMS; ++it) {
        const uint32_t i = base + it * NA_THREADS + threadIdx.x;
        if (i < nt) off[i + 1] = (tile[it * NA_THREADS + threadIdx.x] + ((int64_t)1 << 31)) >> 32;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) off[0] = 0;
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
    if (ctx->device < 0 || ctx->device >= NA_MAX_DEVICES)
        return gm_set_error(GM_ERR_UNSUPPORTED, "gm_tri_offsets_noalloc: device ordinal too large");
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    int64_t* part = nullptr;
    {
        // once per device, with that device current: the device address of the scratch array
        std::lock_guard<std::mutex> lock(g_setup_mutex);
        if (!g_part_addr[ctx->device]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scan_part);
            if (e != cudaSuccess) return gm_cuda_error(e, "gm_tri_offsets_noalloc: cudaGetSymbolAddress");
            g_part_addr[ctx->device] = static_cast<int64_t*>(p);
        }
        part = g_part_addr[ctx->device];
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n_tris == 0) {
        GM_TRY_CUDA(cudaMemsetAsync(offsets, 0, sizeof(int64_t), s));
        return GM_OK;
    }
    na_counts_reduce<<<(uint32_t)nb, NA_THREADS, 0, s>>>(tri_xyz, density_per_tri, n_tris, offsets, part, ctx->dev_err);
    na_scan_parts<<<1, 1024, 0, s>>>(part, (uint32_t)nb);
    na_scan_down<<<(uint32_t)nb, NA_THREADS, 0, s>>>(offsets, n_tris, part);
    ctx->launches += 3;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}
