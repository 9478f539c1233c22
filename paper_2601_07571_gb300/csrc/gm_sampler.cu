// gm_sampler.cu -- area-weighted surface sampling (Section 3.1) and sample export.
//
// Section 3.1.2 asks for #p / A = k on every triangle. Counts here are area-weighted exactly:
//   A_i   = 1/2 |(v1 - v0) x (v2 - v0)| in FP64 from the FP32 world vertices, evaluated as
//           ((cx^2 + cy^2) + cz^2) with correctly rounded, unfused operations so the value is
//           bit-identical to an FP64 CPU evaluation in the same order;
//   q_i   = rint(k A_i 2^32) (int64, 32.32 fixed point); S = inclusive int64 prefix of q;
//   start_i = (S_{i-1} + 2^31) >> 32, count_i = start_{i+1} - start_i,
// so |count_i - k A_i| < 1 and the total is round(k sum A). FP64 is used on the GPU for these
// two steps only. Sample j (global index) takes Philox4x32-10(key = seed, ctr = (j lo, j hi,
// session, 0)) words w0, w1 -> u = ((w >> 9) + 1/2) 2^-23 (exact in FP32), barycentrics
// (1 - sqrt u1, sqrt u1 (1 - u2), sqrt u1 u2) (uniform over the triangle, Osada et al. 2002),
// and world position b0 v0 + b1 v1 + b2 v2 in FP32.
#include <cmath>
#include <string>

#include "gm_internal.cuh"

namespace {

// q_i = rint(k_i A_i 2^32) per triangle. The int64 prefix of the q_i wraps once the scene needs
// about 2^31 samples in total, so every block also adds its FP64 sum of k_i A_i into *ksum (one
// atomic per block); the host refuses the scene when that sum exceeds 2^31 - 16 before it trusts
// the prefix.
__global__ void __launch_bounds__(256) k_tri_counts(const float4* __restrict__ tri, const uint32_t* __restrict__ tri_mesh,
                                                   const double* __restrict__ dens, uint32_t nt,
                                                   int64_t* __restrict__ q, double* __restrict__ ksum,
                                                   int* __restrict__ err) {
    __shared__ double wsum[8];
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    double k = 0.0;
    if (i < nt) {
        float4 a = tri[3 * i], b = tri[3 * i + 1], c = tri[3 * i + 2];
        double e1x = __dsub_rn(b.x, a.x), e1y = __dsub_rn(b.y, a.y), e1z = __dsub_rn(b.z, a.z);
        double e2x = __dsub_rn(c.x, a.x), e2y = __dsub_rn(c.y, a.y), e2z = __dsub_rn(c.z, a.z);
        double cx = __dsub_rn(__dmul_rn(e1y, e2z), __dmul_rn(e1z, e2y));
        double cy = __dsub_rn(__dmul_rn(e1z, e2x), __dmul_rn(e1x, e2z));
        double cz = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
        double n2 = __dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz));
        double A = __dmul_rn(0.5, __dsqrt_rn(n2));
        k = __dmul_rn(dens[tri_mesh[i]], A);
        if (!(k >= 0.0) || k >= 2147483648.0) {
            atomicCAS(err, 0, GM_DEV_BAD_INDEX);
            k = 0.0;
        }
        q[i] = __double2ll_rn(__dmul_rn(k, 4294967296.0));
    }
    double v = k;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += wsum[w];
        if (b > 0.0) atomicAdd(ksum, b);
    }
}

__global__ void k_offsets(const int64_t* __restrict__ S, uint32_t nt, int64_t* __restrict__ off) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) off[0] = 0;
    if (i < nt) off[i + 1] = (S[i] + ((int64_t)1 << 31)) >> 32;
}

// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, round multipliers 0xD2511F53 and
// 0xCD9E8D57, key increments 0x9E3779B9 and 0xBB67AE85.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        uint32_t hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        uint32_t hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += 0x9E3779B9u;
        k.y += 0xBB67AE85u;
    }
    return c;
}

__device__ __forceinline__ float unit23(uint32_t w) {
    // ((w >> 9) + 1/2) / 2^23 == (2 (w >> 9) + 1) / 2^24: an odd integer below 2^24, exact in FP32
    return __uint2float_rn(((w >> 9) << 1) | 1u) * (1.0f / 16777216.0f);
}

__global__ void k_expand(const int64_t* __restrict__ off, uint32_t nt, uint32_t n, const float4* __restrict__ tri,
                         uint2 key, uint32_t session, float4* __restrict__ pos, float2* __restrict__ bary) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    // last triangle whose start is <= j (empty triangles share their successor's start)
    uint32_t lo = 0, hi = nt;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= (int64_t)j) lo = mid; else hi = mid;
    }
    uint4 w = philox4x32_10(make_uint4(j, 0u, session, 0u), key);
    float u1 = unit23(w.x), u2 = unit23(w.y);
    float su = __fsqrt_rn(u1);
    float b0 = __fsub_rn(1.0f, su);
    float b1 = __fmul_rn(su, __fsub_rn(1.0f, u2));
    float b2 = __fmul_rn(su, u2);
    float4 a = tri[3 * lo], b = tri[3 * lo + 1], c = tri[3 * lo + 2];
    float x = fmaf(b2, c.x, fmaf(b1, b.x, b0 * a.x));
    float y = fmaf(b2, c.y, fmaf(b1, b.y, b0 * a.y));
    float z = fmaf(b2, c.z, fmaf(b1, b.z, b0 * a.z));
    pos[j] = make_float4(x, y, z, __uint_as_float(lo));
    bary[j] = make_float2(b1, b2);
}

// ---- the paper's grid sampler (Section 3.1) ---------------------------------------------------
// Resolution r_i (Section 3.1.2): D = 1 + 8 k A (FP64, same unfused order as the FP64 reference),
// r = 1 when D < 25, else rint((-3 + sqrt(D)) / 2); count (r + 1)(r + 2) / 2 (Eq. 1).
__global__ void k_grid_counts(const float4* __restrict__ tri, const uint32_t* __restrict__ tri_mesh,
                              const double* __restrict__ dens, uint32_t nt, int64_t* __restrict__ cnt,
                              uint32_t* __restrict__ res, int* __restrict__ err) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    float4 a = tri[3 * i], b = tri[3 * i + 1], c = tri[3 * i + 2];
    double e1x = __dsub_rn(b.x, a.x), e1y = __dsub_rn(b.y, a.y), e1z = __dsub_rn(b.z, a.z);
    double e2x = __dsub_rn(c.x, a.x), e2y = __dsub_rn(c.y, a.y), e2z = __dsub_rn(c.z, a.z);
    double cx = __dsub_rn(__dmul_rn(e1y, e2z), __dmul_rn(e1z, e2y));
    double cy = __dsub_rn(__dmul_rn(e1z, e2x), __dmul_rn(e1x, e2z));
    double cz = __dsub_rn(__dmul_rn(e1x, e2y), __dmul_rn(e1y, e2x));
    double n2 = __dadd_rn(__dadd_rn(__dmul_rn(cx, cx), __dmul_rn(cy, cy)), __dmul_rn(cz, cz));
    double A = __dmul_rn(0.5, __dsqrt_rn(n2));
    double D = __dadd_rn(1.0, __dmul_rn(__dmul_rn(8.0, dens[tri_mesh[i]]), A));
    long long r = 1;
    if (!(D < 25.0)) {
        const double rr = __dmul_rn(__dadd_rn(-3.0, __dsqrt_rn(D)), 0.5);
        if (!(rr < 65535.0)) {
            atomicCAS(err, 0, GM_DEV_BAD_INDEX);
            r = 1;
        } else {
            r = __double2ll_rn(rr);
        }
    }
    if (r < 1) r = 1;
    res[i] = (uint32_t)r;
    cnt[i] = (int64_t)((r + 1) * (r + 2) / 2);
}

__global__ void k_excl_from_incl(const int64_t* __restrict__ S, uint32_t nt, int64_t* __restrict__ off) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) off[0] = 0;
    if (i < nt) off[i + 1] = S[i];
}

// Sample j: triangle by binary search, local index idx -> row = max m with m(m+1)/2 <= idx,
// col = idx - row(row+1)/2 (Eq. 2); weights (col/r, 1 - row/r, (row - col)/r) (Eq. 3, third
// weight read as 1 - w1 - w2) of (v0, v1, v2).
__global__ void k_grid_expand(const int64_t* __restrict__ off, const uint32_t* __restrict__ res, uint32_t nt,
                              uint32_t n, const float4* __restrict__ tri, float4* __restrict__ pos,
                              float2* __restrict__ bary) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t lo = 0, hi = nt;
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) >> 1;
        if (off[mid] <= (int64_t)j) lo = mid; else hi = mid;
    }
    const long long idx = (long long)j - off[lo];
    long long m = (long long)((sqrtf((float)(8 * idx + 1)) - 1.f) * 0.5f);
    while (m > 0 && m * (m + 1) / 2 > idx) --m;
    while ((m + 1) * (m + 2) / 2 <= idx) ++m;
    const long long col = idx - m * (m + 1) / 2;
    const float r = (float)res[lo];
    const float w1 = __fdiv_rn((float)col, r);
    const float w2 = __fsub_rn(1.0f, __fdiv_rn((float)m, r));
    const float w3 = __fdiv_rn((float)(m - col), r);
    const float4 a = tri[3 * lo], b = tri[3 * lo + 1], c = tri[3 * lo + 2];
    const float x = fmaf(w3, c.x, fmaf(w2, b.x, w1 * a.x));
    const float y = fmaf(w3, c.y, fmaf(w2, b.y, w1 * a.y));
    const float z = fmaf(w3, c.z, fmaf(w2, b.z, w1 * a.z));
    pos[j] = make_float4(x, y, z, __uint_as_float(lo));
    bary[j] = make_float2(w2, w3);
}

// ---- spatial work order: 30-bit Morton code of each sample position in the scene box -------
__device__ __forceinline__ uint32_t spread3_10(uint32_t v) {
    v &= 0x3ffu;
    v = (v | (v << 16)) & 0x030000ffu;
    v = (v | (v << 8)) & 0x0300f00fu;
    v = (v | (v << 4)) & 0x030c30c3u;
    v = (v | (v << 2)) & 0x09249249u;
    return v;
}

__global__ void k_sample_morton(const float4* __restrict__ pos, uint32_t n, float3 lo, float3 inv_ext,
                                uint32_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float4 p = pos[j];
    uint32_t qx = (uint32_t)fminf(fmaxf((p.x - lo.x) * inv_ext.x, 0.f), 1023.f);
    uint32_t qy = (uint32_t)fminf(fmaxf((p.y - lo.y) * inv_ext.y, 0.f), 1023.f);
    uint32_t qz = (uint32_t)fminf(fmaxf((p.z - lo.z) * inv_ext.z, 0.f), 1023.f);
    keys[j] = (spread3_10(qx) << 2) | (spread3_10(qy) << 1) | spread3_10(qz);
    vals[j] = j;
}

__global__ void k_gather_work(const float4* __restrict__ pos, const uint32_t* __restrict__ idx, uint32_t n,
                              float4* __restrict__ work) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) work[j] = pos[idx[j]];
}

__global__ void k_points(const float* __restrict__ xyz, const uint32_t* __restrict__ tri, uint32_t n,
                         uint32_t nt, float4* __restrict__ pos, int* __restrict__ err) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    uint32_t t = tri[j];
    if (t >= nt) atomicCAS(err, 0, GM_DEV_BAD_INDEX);
    pos[j] = make_float4(xyz[3 * j], xyz[3 * j + 1], xyz[3 * j + 2], __uint_as_float(t));
}

gm_status build_work_order(gm_samples* sm, cudaStream_t s, int* launches) {
    const uint32_t n = (uint32_t)sm->n;
    GM_TRY(gm_alloc((void**)&sm->work_pos, sizeof(float4) * n, s));
    GM_TRY(gm_alloc((void**)&sm->work_idx, sizeof(uint32_t) * n, s));
    if (n == 0) return GM_OK;
    uint32_t* keys = nullptr;
    GM_TRY(gm_alloc((void**)&keys, sizeof(uint32_t) * n, s));
    const gm_scene* sc = sm->scene;
    float3 lo = make_float3(sc->box_lo[0], sc->box_lo[1], sc->box_lo[2]);
    float ex = fmaxf(fmaxf(sc->box_hi[0] - sc->box_lo[0], sc->box_hi[1] - sc->box_lo[1]),
                     sc->box_hi[2] - sc->box_lo[2]);
    float inv = ex > 0.f ? 1024.f / ex : 0.f;
    k_sample_morton<<<gm_div_up(n, 256), 256, 0, s>>>(sm->pos, n, lo, make_float3(inv, inv, inv), keys, sm->work_idx);
    gm_status st = gm_radix_sort_u32(keys, sm->work_idx, n, 30, s, launches);
    if (st == GM_OK) k_gather_work<<<gm_div_up(n, 256), 256, 0, s>>>(sm->pos, sm->work_idx, n, sm->work_pos);
    *launches += 2;
    cudaFreeAsync(keys, s);
    if (st != GM_OK) return st;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

}  // namespace

extern "C" gm_status gm_sample_surface(gm_scene* sc, const double* density_per_mesh, uint64_t seed,
                                       uint32_t session, gm_stream stream, gm_samples** out) {
    if (!sc || !density_per_mesh || !out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_sample_surface: null argument");
    *out = nullptr;
    for (uint32_t m = 0; m < sc->n_meshes; ++m)
        if (!(density_per_mesh[m] >= 0.0) || !std::isfinite(density_per_mesh[m]))
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_sample_surface: density must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(sc->ctx->device));
    const uint32_t nt = sc->n_tris;
    gm_samples* sm = new gm_samples();
    sm->scene = sc;
    double* dens = nullptr;
    int64_t* q = nullptr;
    auto fail = [&](gm_status st) {
        if (dens) cudaFreeAsync(dens, s);
        if (q) cudaFreeAsync(q, s);
        gm_samples_free(sm);
        return st;
    };
    gm_status st;
    // dens[0 .. n_meshes) the per-mesh densities, dens[n_meshes] the FP64 sum of k A over triangles
    if ((st = gm_alloc((void**)&dens, sizeof(double) * (sc->n_meshes + 1), s)) != GM_OK) return fail(st);
    if ((st = gm_alloc((void**)&q, sizeof(int64_t) * nt, s)) != GM_OK) return fail(st);
    if ((st = gm_alloc((void**)&sm->tri_offset, sizeof(int64_t) * (nt + 1), s)) != GM_OK) return fail(st);
    cudaError_t e = cudaMemcpyAsync(dens, density_per_mesh, sizeof(double) * sc->n_meshes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "density upload"));
    if ((e = cudaMemsetAsync(dens + sc->n_meshes, 0, sizeof(double), s)) != cudaSuccess)
        return fail(gm_cuda_error(e, "gm_sample_surface"));
    int launches = 0;
    k_tri_counts<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->tri_canon, sc->tri_mesh, dens, nt, q, dens + sc->n_meshes,
                                                    sc->ctx->dev_err);
    if ((st = gm_inclusive_scan_i64(q, nt, s, &launches)) != GM_OK) return fail(st);
    k_offsets<<<gm_div_up(nt, 256), 256, 0, s>>>(q, nt, sm->tri_offset);
    launches += 2;
    int64_t total = 0;
    double ksum = 0.0;
    int herr = 0;
    if ((e = cudaMemcpyAsync(&total, sm->tri_offset + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&ksum, dens + sc->n_meshes, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&herr, sc->ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(gm_cuda_error(e, "gm_sample_surface"));
    cudaFreeAsync(q, s);
    q = nullptr;
    cudaFreeAsync(dens, s);
    dens = nullptr;
    if (herr) {
        cudaMemsetAsync(sc->ctx->dev_err, 0, sizeof(int), s);
        return fail(gm_set_error(GM_ERR_UNSUPPORTED, "gm_sample_surface: a triangle needs 2^31 or more samples"));
    }
    // The FP64 sum is within 4 samples of the exact one (at most 2^24 block atomics of relative
    // error 2^-53 on a sum below 2^31), so sum k A <= 2^31 - 16 keeps the 32.32 prefix below
    // (2^31 - 12) 2^32 + n_tris / 2 < 2^63: no wrap. Beyond it the prefix may have wrapped and
    // the sum decides.
    if (!(ksum <= 2147483632.0) || total < 0 || total > 0x7fffffffLL)
        return fail(gm_set_error(GM_ERR_UNSUPPORTED, "gm_sample_surface: more than 2^31-1 samples"));
    sm->n = (uint64_t)total;
    const uint32_t n = (uint32_t)total;
    if ((st = gm_alloc((void**)&sm->pos, sizeof(float4) * n, s)) != GM_OK) return fail(st);
    if ((st = gm_alloc((void**)&sm->bary, sizeof(float2) * n, s)) != GM_OK) return fail(st);
    sm->kind = GM_SAMPLES_PHILOX;
    sm->key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    sm->session = session;
    if (n > 0)
        k_expand<<<gm_div_up(n, 256), 256, 0, s>>>(sm->tri_offset, nt, n, sc->tri_canon, sm->key, session, sm->pos,
                                                  sm->bary);
    if (n > 0) ++launches;
    if ((st = build_work_order(sm, s, &launches)) != GM_OK) return fail(st);
    sc->ctx->launches += launches;
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_sample_surface launch"));
    *out = sm;
    return GM_OK;
}

extern "C" gm_status gm_sample_surface_grid(gm_scene* sc, const double* density_per_mesh, gm_stream stream,
                                            gm_samples** out) {
    if (!sc || !density_per_mesh || !out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_sample_surface_grid: null argument");
    *out = nullptr;
    for (uint32_t m = 0; m < sc->n_meshes; ++m)
        if (!(density_per_mesh[m] >= 0.0) || !std::isfinite(density_per_mesh[m]))
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_sample_surface_grid: density must be finite and >= 0");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(sc->ctx->device));
    const uint32_t nt = sc->n_tris;
    gm_samples* sm = new gm_samples();
    sm->scene = sc;
    double* dens = nullptr;
    int64_t* cnt = nullptr;
    uint32_t* res = nullptr;
    auto fail = [&](gm_status st) {
        if (dens) cudaFreeAsync(dens, s);
        if (cnt) cudaFreeAsync(cnt, s);
        if (res) cudaFreeAsync(res, s);
        gm_samples_free(sm);
        return st;
    };
    gm_status st;
    if ((st = gm_alloc((void**)&dens, sizeof(double) * sc->n_meshes, s)) != GM_OK) return fail(st);
    if ((st = gm_alloc((void**)&cnt, sizeof(int64_t) * nt, s)) != GM_OK) return fail(st);
    if ((st = gm_alloc((void**)&res, sizeof(uint32_t) * nt, s)) != GM_OK) return fail(st);
    if ((st = gm_alloc((void**)&sm->tri_offset, sizeof(int64_t) * (nt + 1), s)) != GM_OK) return fail(st);
    cudaError_t e = cudaMemcpyAsync(dens, density_per_mesh, sizeof(double) * sc->n_meshes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "density upload"));
    int launches = 0;
    k_grid_counts<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->tri_canon, sc->tri_mesh, dens, nt, cnt, res, sc->ctx->dev_err);
    if ((st = gm_inclusive_scan_i64(cnt, nt, s, &launches)) != GM_OK) return fail(st);
    k_excl_from_incl<<<gm_div_up(nt, 256), 256, 0, s>>>(cnt, nt, sm->tri_offset);
    launches += 2;
    int64_t total = 0;
    int herr = 0;
    if ((e = cudaMemcpyAsync(&total, sm->tri_offset + nt, sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&herr, sc->ctx->dev_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(gm_cuda_error(e, "gm_sample_surface_grid"));
    if (herr) {
        cudaMemsetAsync(sc->ctx->dev_err, 0, sizeof(int), s);
        return fail(gm_set_error(GM_ERR_UNSUPPORTED, "gm_sample_surface_grid: a triangle needs a resolution of 65535 or more"));
    }
    if (total > 0x7fffffffLL) return fail(gm_set_error(GM_ERR_UNSUPPORTED, "gm_sample_surface_grid: more than 2^31-1 samples"));
    sm->n = (uint64_t)total;
    const uint32_t n = (uint32_t)total;
    if ((st = gm_alloc((void**)&sm->pos, sizeof(float4) * n, s)) != GM_OK) return fail(st);
    if ((st = gm_alloc((void**)&sm->bary, sizeof(float2) * n, s)) != GM_OK) return fail(st);
    if (n > 0) {
        k_grid_expand<<<gm_div_up(n, 256), 256, 0, s>>>(sm->tri_offset, res, nt, n, sc->tri_canon, sm->pos, sm->bary);
        ++launches;
    }
    if ((st = build_work_order(sm, s, &launches)) != GM_OK) return fail(st);
    sc->ctx->launches += launches;
    cudaFreeAsync(dens, s);
    cudaFreeAsync(cnt, s);
    sm->kind = GM_SAMPLES_GRID;
    sm->res = res;   // kept: a dynamic scene re-places the grid samples on every pose
    dens = nullptr;
    cnt = nullptr;
    res = nullptr;
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_sample_surface_grid launch"));
    *out = sm;
    return GM_OK;
}

extern "C" gm_status gm_samples_from_points(gm_scene* sc, const float* xyz, const uint32_t* tri, uint64_t n,
                                            gm_stream stream, gm_samples** out) {
    if (!sc || !out || (n > 0 && (!xyz || !tri)))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_from_points: null argument");
    if (n > 0x7fffffffULL) return gm_set_error(GM_ERR_UNSUPPORTED, "gm_samples_from_points: more than 2^31-1 points");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(sc->ctx->device));
    gm_samples* sm = new gm_samples();
    sm->scene = sc;
    sm->n = n;
    sm->kind = GM_SAMPLES_POINTS;
    void *dx = nullptr, *dt = nullptr;
    bool ox = false, ot = false;
    auto fail = [&](gm_status st) {
        if (ox) cudaFreeAsync(dx, s);
        if (ot) cudaFreeAsync(dt, s);
        gm_samples_free(sm);
        return st;
    };
    gm_status st;
    if ((st = gm_alloc((void**)&sm->pos, sizeof(float4) * n, s)) != GM_OK) return fail(st);
    if (n > 0) {
        if ((st = gm_stage_to_device(xyz, sizeof(float) * 3 * n, s, &dx, &ox)) != GM_OK) return fail(st);
        if ((st = gm_stage_to_device(tri, sizeof(uint32_t) * n, s, &dt, &ot)) != GM_OK) return fail(st);
        k_points<<<gm_div_up(n, 256), 256, 0, s>>>((const float*)dx, (const uint32_t*)dt, (uint32_t)n, sc->n_tris,
                                                   sm->pos, sc->ctx->dev_err);
    }
    int launches = n > 0 ? 1 : 0;
    if ((st = build_work_order(sm, s, &launches)) != GM_OK) return fail(st);
    sc->ctx->launches += launches;
    if (ox) cudaFreeAsync(dx, s);
    if (ot) cudaFreeAsync(dt, s);
    ox = ot = false;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_samples_from_points launch"));
    *out = sm;
    return GM_OK;
}

extern "C" gm_status gm_samples_info(const gm_samples* sm, uint64_t* n) {
    if (!sm) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_info: null samples");
    if (n) *n = sm->n;
    return GM_OK;
}

extern "C" gm_status gm_samples_offsets(const gm_samples* sm, int64_t* dst, gm_stream stream) {
    if (!sm || !dst) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_offsets: null argument");
    if (!sm->tri_offset) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_offsets: samples were given as points");
    return gm_copy_out(dst, sm->tri_offset, sizeof(int64_t) * (sm->scene->n_tris + 1), (cudaStream_t)stream);
}

namespace {
__global__ void k_export(const float4* __restrict__ pos, const float2* __restrict__ bary,
                         const uint32_t* __restrict__ tri_mesh, const uint32_t* __restrict__ mesh_obj, uint32_t n,
                         uint32_t nt, float* __restrict__ xyz, uint32_t* __restrict__ tri, float* __restrict__ b2,
                         uint32_t* __restrict__ obj) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float4 p = pos[j];
    uint32_t t = __float_as_uint(p.w);
    if (xyz) { xyz[3 * j] = p.x; xyz[3 * j + 1] = p.y; xyz[3 * j + 2] = p.z; }
    if (tri) tri[j] = t;
    if (b2) {
        float2 b = bary ? bary[j] : make_float2(0.f, 0.f);
        b2[2 * j] = b.x;
        b2[2 * j + 1] = b.y;
    }
    if (obj) obj[j] = t < nt ? mesh_obj[tri_mesh[t]] : 0xffffffffu;
}
}  // namespace

extern "C" gm_status gm_samples_copy(const gm_samples* sm, float* xyz, uint32_t* tri, float* bary2, uint32_t* obj,
                                     gm_stream stream) {
    if (!sm) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_copy: null samples");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)sm->n;
    if (n == 0) return GM_OK;
    void* outs[4] = {xyz, tri, bary2, obj};
    size_t sizes[4] = {sizeof(float) * 3 * (size_t)n, sizeof(uint32_t) * (size_t)n, sizeof(float) * 2 * (size_t)n,
                       sizeof(uint32_t) * (size_t)n};
    void* dev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool owned[4] = {false, false, false, false};
    gm_status st = GM_OK;
    for (int k = 0; k < 4 && st == GM_OK; ++k) {
        if (!outs[k]) continue;
        if (gm_is_device_ptr(outs[k])) dev[k] = outs[k];
        else if ((st = gm_alloc(&dev[k], sizes[k], s)) == GM_OK) owned[k] = true;
    }
    if (st == GM_OK) {
        k_export<<<gm_div_up(n, 256), 256, 0, s>>>(sm->pos, sm->bary, sm->scene->tri_mesh, sm->scene->mesh_object, n,
                                                  sm->scene->n_tris,
                                                  (float*)dev[0], (uint32_t*)dev[1], (float*)dev[2], (uint32_t*)dev[3]);
        sm->scene->ctx->launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = gm_cuda_error(e, "gm_samples_copy launch");
    }
    for (int k = 0; k < 4; ++k) {
        if (owned[k]) {
            if (st == GM_OK) st = gm_copy_out(outs[k], dev[k], sizes[k], s);
            cudaFreeAsync(dev[k], s);
        }
    }
    return st;
}

namespace {
__global__ void k_export_record(const float4* __restrict__ pos, const float2* __restrict__ bary,
                                const uint32_t* __restrict__ tri_mesh, const uint32_t* __restrict__ mesh_obj,
                                const double* __restrict__ inv, const float* __restrict__ values, uint32_t n,
                                uint32_t nt, float* __restrict__ value, uint32_t* __restrict__ obj,
                                uint32_t* __restrict__ tri, float* __restrict__ b3, float* __restrict__ local,
                                float* __restrict__ world) {
    uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const float4 p = pos[j];
    const uint32_t t = __float_as_uint(p.w);
    const uint32_t m = t < nt ? tri_mesh[t] : 0u;
    if (value) value[j] = values[j];
    if (obj) obj[j] = t < nt ? mesh_obj[m] : 0xffffffffu;
    if (tri) tri[j] = t;
    if (b3) {
        const float2 b = bary ? bary[j] : make_float2(0.f, 0.f);
        b3[3 * j] = 1.f - b.x - b.y;
        b3[3 * j + 1] = b.x;
        b3[3 * j + 2] = b.y;
    }
    if (world) {
        world[3 * j] = p.x;
        world[3 * j + 1] = p.y;
        world[3 * j + 2] = p.z;
    }
    if (local) {
        const double* A = inv + 12 * m;
        for (int r = 0; r < 3; ++r)
            local[3 * j + r] = (float)(A[4 * r] * p.x + A[4 * r + 1] * p.y + A[4 * r + 2] * p.z + A[4 * r + 3]);
    }
}
}  // namespace

extern "C" gm_status gm_samples_export(const gm_samples* sm, const gm_map* mp, uint32_t window,
                                       const gm_export_dst* dst, gm_stream stream) {
    if (!sm || !mp || !dst) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_export: null argument");
    if (mp->ns != sm->n || window >= mp->W)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_export: map does not match samples or bad window");
    if (dst->local_xyz && !sm->scene->mesh_inv_ok)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_export: a mesh transform is singular (no local frame)");
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t n = (uint32_t)sm->n;
    if (n == 0) return GM_OK;
    void* outs[6] = {dst->value, dst->object_id, dst->triangle, dst->bary3, dst->local_xyz, dst->world_xyz};
    const size_t sizes[6] = {4ull * n, 4ull * n, 4ull * n, 12ull * n, 12ull * n, 12ull * n};
    void* dev[6] = {};
    bool owned[6] = {};
    gm_status st = GM_OK;
    for (int k = 0; k < 6 && st == GM_OK; ++k) {
        if (!outs[k]) continue;
        if (gm_is_device_ptr(outs[k])) dev[k] = outs[k];
        else if ((st = gm_alloc(&dev[k], sizes[k], s)) == GM_OK) owned[k] = true;
    }
    if (st == GM_OK) {
        const gm_scene* sc = sm->scene;
        k_export_record<<<gm_div_up(n, 256), 256, 0, s>>>(sm->pos, sm->bary, sc->tri_mesh, sc->mesh_object, sc->mesh_inv,
                                                         mp->values + (size_t)window * mp->ns, n, sc->n_tris,
                                                         (float*)dev[0], (uint32_t*)dev[1], (uint32_t*)dev[2],
                                                         (float*)dev[3], (float*)dev[4], (float*)dev[5]);
        sc->ctx->launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = gm_cuda_error(e, "gm_samples_export launch");
    }
    for (int k = 0; k < 6; ++k) {
        if (owned[k]) {
            if (st == GM_OK) st = gm_copy_out(outs[k], dev[k], sizes[k], s);
            cudaFreeAsync(dev[k], s);
        }
    }
    return st;
}

extern "C" gm_status gm_samples_follow(gm_samples* sm, gm_stream stream) {
    if (!sm) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_follow: null samples");
    if (sm->kind == GM_SAMPLES_POINTS)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_follow: explicit points are not attached to a triangle frame");
    const gm_scene* sc = sm->scene;
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(sc->ctx->device));
    const uint32_t n = (uint32_t)sm->n;
    if (n == 0) return GM_OK;
    // the same expansion as at sampling time, on the posed triangles: same counts, same
    // barycentrics, new positions
    if (sm->kind == GM_SAMPLES_PHILOX)
        k_expand<<<gm_div_up(n, 256), 256, 0, s>>>(sm->tri_offset, sc->n_tris, n, sc->tri_canon, sm->key, sm->session,
                                                  sm->pos, sm->bary);
    else
        k_grid_expand<<<gm_div_up(n, 256), 256, 0, s>>>(sm->tri_offset, sm->res, sc->n_tris, n, sc->tri_canon, sm->pos,
                                                       sm->bary);
    // the work order of the first pose is kept (it only groups samples into warp tiles)
    k_gather_work<<<gm_div_up(n, 256), 256, 0, s>>>(sm->pos, sm->work_idx, n, sm->work_pos);
    sc->ctx->launches += 2;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

extern "C" gm_status gm_samples_slice(const gm_samples* src, uint64_t begin, uint64_t end, gm_stream stream,
                                      gm_samples** out) {
    if (!src || !out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_slice: null argument");
    *out = nullptr;
    if (begin > end || end > src->n) return gm_set_error(GM_ERR_INVALID_ARG, "gm_samples_slice: range outside the set");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(src->scene->ctx->device));
    gm_samples* sm = new gm_samples();
    sm->scene = src->scene;
    sm->n = end - begin;
    sm->kind = GM_SAMPLES_POINTS;   // fixed points: no offsets of their own, they do not follow poses
    auto fail = [&](gm_status st) {
        gm_samples_free(sm);
        return st;
    };
    gm_status st;
    const size_t n = (size_t)sm->n;
    if ((st = gm_alloc((void**)&sm->pos, sizeof(float4) * n, s)) != GM_OK) return fail(st);
    cudaError_t e = n ? cudaMemcpyAsync(sm->pos, src->pos + begin, sizeof(float4) * n, cudaMemcpyDeviceToDevice, s)
                      : cudaSuccess;
    if (e == cudaSuccess && src->bary && n) {
        if ((st = gm_alloc((void**)&sm->bary, sizeof(float2) * n, s)) != GM_OK) return fail(st);
        e = cudaMemcpyAsync(sm->bary, src->bary + begin, sizeof(float2) * n, cudaMemcpyDeviceToDevice, s);
    }
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_samples_slice"));
    int launches = 0;
    if ((st = build_work_order(sm, s, &launches)) != GM_OK) return fail(st);
    sm->scene->ctx->launches += launches;
    *out = sm;
    return GM_OK;
}

extern "C" void gm_samples_free(gm_samples* sm) {
    if (!sm) return;
    cudaFree(sm->pos);
    cudaFree(sm->bary);
    cudaFree(sm->res);
    cudaFree(sm->tri_offset);
    cudaFree(sm->work_pos);
    cudaFree(sm->work_idx);
    delete sm;
}
