// gm_sort.cu -- stable LSD radix sort (8-bit digits) and an int64 inclusive scan.
//
// Used by the BVH build (Morton keys of triangle centroids), the spatial work order of the
// samples, the window sort of fixations, and the fixed-point prefix of per-triangle counts.
// Three kernels per radix pass: per-tile digit histograms, one exclusive scan over the
// digit-major histogram table, then a stable scatter in which every 256-key round ranks its
// keys with warp match + per-warp digit counts. No spin-waits anywhere.
#include <algorithm>

#include "gm_internal.cuh"
#include "gm_scan.cuh"

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_ITEMS = 16;
constexpr int RS_TILE = RS_THREADS * RS_ITEMS;
constexpr int RS_WARPS = RS_THREADS / 32;

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) rs_hist(const K* __restrict__ keys, uint32_t n, int shift,
                                                      uint32_t* __restrict__ hist, uint32_t nblocks) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint32_t base = blockIdx.x * (uint32_t)RS_TILE;
#pragma unroll 4
    for (int i = 0; i < RS_ITEMS; ++i) {
        uint32_t idx = base + i * RS_THREADS + threadIdx.x;
        uint32_t d = idx < n ? (uint32_t)((keys[idx] >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        if (d < 256u && (peers & gm_lanemask_lt()) == 0) atomicAdd(&h[d], (uint32_t)__popc(peers));
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * nblocks + blockIdx.x] = h[threadIdx.x];
}

// Exclusive scan of `total` uint32 entries in place, one block of 1024 threads.
__global__ void __launch_bounds__(1024) rs_scan(uint32_t* __restrict__ a, uint32_t total) {
    constexpr int PER = 4;
    __shared__ uint32_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < total; base += 1024 * PER) {
        uint32_t v[PER], s = 0;
        uint32_t i0 = base + threadIdx.x * PER;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            v[k] = (i0 + k < total) ? a[i0 + k] : 0u;
            s += v[k];
        }
        uint32_t tot;
        uint32_t ex = block_excl_scan<uint32_t, 1024>(s, &tot);
        uint32_t run = carry + ex;
#pragma unroll
        for (int k = 0; k < PER; ++k) {
            if (i0 + k < total) a[i0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

template <typename K>
__global__ void __launch_bounds__(RS_THREADS) rs_scatter(const K* __restrict__ kin, const uint32_t* __restrict__ vin,
                                                         K* __restrict__ kout, uint32_t* __restrict__ vout,
                                                         uint32_t n, int shift,
                                                         const uint32_t* __restrict__ hist, uint32_t nblocks) {
    __shared__ uint32_t base_off[256];
    __shared__ uint32_t wcount[RS_WARPS][256];
    const int tid = threadIdx.x, warp = tid >> 5;
    base_off[tid] = hist[(size_t)tid * nblocks + blockIdx.x];
    const uint32_t tile = blockIdx.x * (uint32_t)RS_TILE;
    for (int round = 0; round < RS_ITEMS; ++round) {
        for (int i = tid; i < RS_WARPS * 256; i += RS_THREADS) (&wcount[0][0])[i] = 0;
        __syncthreads();
        uint32_t idx = tile + round * RS_THREADS + tid;
        bool valid = idx < n;
        K k = valid ? kin[idx] : K(0);
        uint32_t v = valid ? vin[idx] : 0u;
        uint32_t d = valid ? (uint32_t)((k >> shift) & 255u) : 256u;
        unsigned peers = __match_any_sync(0xffffffffu, d);
        uint32_t rank = __popc(peers & gm_lanemask_lt());
        if (valid && rank == 0) wcount[warp][d] = __popc(peers);
        __syncthreads();
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < RS_WARPS; ++w) {
            uint32_t c = wcount[w][tid];
            wcount[w][tid] = run;
            run += c;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = base_off[d] + wcount[warp][d] + rank;
            kout[pos] = k;
            vout[pos] = v;
        }
        __syncthreads();
        base_off[tid] += run;
    }
}

// The passes proper, with caller-provided temporaries (n keys, n values, 256 * tiles counters).
template <typename K>
cudaError_t radix_passes(K* keys, uint32_t* vals, uint32_t n, int bits, K* k2, uint32_t* v2, uint32_t* hist,
                         cudaStream_t s, int* launches) {
    if (n <= 1 || bits <= 0) return cudaSuccess;
    const uint32_t nb = gm_div_up(n, RS_TILE);
    K *ka = keys, *kb = k2;
    uint32_t *va = vals, *vb = v2;
    int passes = 0;
    for (int shift = 0; shift < bits; shift += 8, ++passes) {
        rs_hist<K><<<nb, RS_THREADS, 0, s>>>(ka, n, shift, hist, nb);
        rs_scan<<<1, 1024, 0, s>>>(hist, 256u * nb);
        rs_scatter<K><<<nb, RS_THREADS, 0, s>>>(ka, va, kb, vb, n, shift, hist, nb);
        std::swap(ka, kb);
        std::swap(va, vb);
    }
    if (launches) *launches += 3 * passes;
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess && ka != keys) {
        e = cudaMemcpyAsync(keys, ka, sizeof(K) * n, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(vals, va, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s);
    }
    return e;
}

template <typename K>
gm_status radix_sort(K* keys, uint32_t* vals, uint32_t n, int bits, cudaStream_t s, int* launches) {
    if (n <= 1 || bits <= 0) return GM_OK;
    const uint32_t nb = gm_div_up(n, RS_TILE);
    K* k2 = nullptr;
    uint32_t *v2 = nullptr, *hist = nullptr;
    gm_status st = gm_alloc((void**)&k2, sizeof(K) * n, s);
    if (st == GM_OK) st = gm_alloc((void**)&v2, sizeof(uint32_t) * n, s);
    if (st == GM_OK) st = gm_alloc((void**)&hist, sizeof(uint32_t) * 256 * (size_t)nb, s);
    if (st != GM_OK) {
        if (k2) cudaFreeAsync(k2, s);
        if (v2) cudaFreeAsync(v2, s);
        return st;
    }
    cudaError_t e = radix_passes<K>(keys, vals, n, bits, k2, v2, hist, s, launches);
    cudaFreeAsync(k2, s);
    cudaFreeAsync(v2, s);
    cudaFreeAsync(hist, s);
    if (e != cudaSuccess) return gm_cuda_error(e, "radix sort");
    return GM_OK;
}

// ---- int64 inclusive scan: tile reduce, scan of tile sums, tile scan + offset ----------------
constexpr int SC_THREADS = 256;
constexpr int SC_ITEMS = 8;
constexpr int SC_TILE = SC_THREADS * SC_ITEMS;

__global__ void __launch_bounds__(SC_THREADS) scan_reduce(const int64_t* __restrict__ a, uint32_t n,
                                                          int64_t* __restrict__ part) {
    const uint32_t base = blockIdx.x * (uint32_t)SC_TILE;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        uint32_t idx = base + i * SC_THREADS + threadIdx.x;
        if (idx < n) s += a[idx];
    }
    int64_t tot;
    block_excl_scan<int64_t, SC_THREADS>(s, &tot);
    if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(1024) scan_parts(int64_t* __restrict__ part, uint32_t nb) {
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (uint32_t base = 0; base < nb; base += 1024) {
        uint32_t i = base + threadIdx.x;
        int64_t v = i < nb ? part[i] : 0;
        int64_t tot;
        int64_t ex = block_excl_scan<int64_t, 1024>(v, &tot);
        if (i < nb) part[i] = carry + ex;
        __syncthreads();
        if (threadIdx.x == 0) carry += tot;
        __syncthreads();
    }
}

__global__ void __launch_bounds__(SC_THREADS) scan_down(int64_t* __restrict__ a, uint32_t n,
                                                        const int64_t* __restrict__ part) {
    __shared__ int64_t tile[SC_TILE];
    const uint32_t base = blockIdx.x * (uint32_t)SC_TILE;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        uint32_t idx = base + i * SC_THREADS + threadIdx.x;
        tile[i * SC_THREADS + threadIdx.x] = idx < n ? a[idx] : 0;
    }
    __syncthreads();
    int64_t v[SC_ITEMS], s = 0;
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        v[i] = tile[threadIdx.x * SC_ITEMS + i];
        s += v[i];
        v[i] = s;
    }
    int64_t tot;
    int64_t ex = block_excl_scan<int64_t, SC_THREADS>(s, &tot) + part[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) tile[threadIdx.x * SC_ITEMS + i] = v[i] + ex;
    __syncthreads();
#pragma unroll
    for (int i = 0; i < SC_ITEMS; ++i) {
        uint32_t idx = base + i * SC_THREADS + threadIdx.x;
        if (idx < n) a[idx] = tile[i * SC_THREADS + threadIdx.x];
    }
}

}  // namespace

gm_status gm_radix_sort_u64(uint64_t* keys, uint32_t* vals, uint32_t n, int bits, cudaStream_t s, int* launches) {
    return radix_sort<uint64_t>(keys, vals, n, bits, s, launches);
}

gm_status gm_radix_sort_u32(uint32_t* keys, uint32_t* vals, uint32_t n, int bits, cudaStream_t s, int* launches) {
    return radix_sort<uint32_t>(keys, vals, n, std::min(bits, 32), s, launches);
}

size_t gm_radix_sort_u32_hist_words(uint32_t n) { return 256 * (size_t)gm_div_up(n, RS_TILE); }

gm_status gm_radix_sort_u32_prealloc(uint32_t* keys, uint32_t* vals, uint32_t n, int bits, uint32_t* tmp_keys,
                                     uint32_t* tmp_vals, uint32_t* hist, cudaStream_t s, int* launches) {
    cudaError_t e = radix_passes<uint32_t>(keys, vals, n, std::min(bits, 32), tmp_keys, tmp_vals, hist, s, launches);
    if (e != cudaSuccess) return gm_cuda_error(e, "radix sort");
    return GM_OK;
}

gm_status gm_inclusive_scan_i64(int64_t* data, uint32_t n, cudaStream_t s, int* launches) {
    if (n == 0) return GM_OK;
    const uint32_t nb = gm_div_up(n, SC_TILE);
    int64_t* part = nullptr;
    GM_TRY(gm_alloc((void**)&part, sizeof(int64_t) * nb, s));
    scan_reduce<<<nb, SC_THREADS, 0, s>>>(data, n, part);
    scan_parts<<<1, 1024, 0, s>>>(part, nb);
    scan_down<<<nb, SC_THREADS, 0, s>>>(data, n, part);
    if (launches) *launches += 3;
    cudaError_t e = cudaGetLastError();
    cudaFreeAsync(part, s);
    if (e != cudaSuccess) return gm_cuda_error(e, "int64 scan");
    return GM_OK;
}
