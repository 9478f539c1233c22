// gm_field.cu -- the neural density field: a Fourier-feature MLP trained on the maps the plain
// method produces, answering density queries at arbitrary surface points (not in the paper).
//
// Definition (64 features, 4 hidden layers of 64, softplus output):
//   x~ = (x - c) / h  (c: centre, h: half the largest side of the scene box)
//   f = [x~, sin(2^k pi x~), cos(2^k pi x~) for k = 0..9, 0]      (3 + 60 + 1 = 64 features)
//   h0 = bf16(f); h_l = bf16(relu(h_{l-1} bf16(W_l)^T + b_l))  l = 1..4  (FP32 accumulation)
//   out = softplus(h4 . w5 + b5)                                       (FP32)
// Training minimises the mean squared error to the normalised map with Adam (FP32 master
// weights and moments), one fused kernel per step for the forward and backward passes plus one
// update kernel. Both the queries and the training have two kernels: the default runs every
// hidden-layer product on the 5th-generation tensor cores (tcgen05.mma, accumulators in tensor
// memory; k_field_query_tc, k_field_train_tc), the other on warp-level BF16 mma.sync.m16n8k16 with
// FP32 accumulation (k_field_query, k_field_train).
//
// Warp-level data flow: a warp owns 16 points. Its activations stay in registers between
// layers: the FP32 accumulator fragments of two adjacent n8 tiles, rounded to bf16, are exactly
// the A fragment of the next k16 step. Weights live in shared memory as bf16 rows of 72 entries
// (64 + 8 padding), which makes every B-fragment load bank-conflict free. In training, the
// forward activations are also written transposed to shared memory so that the weight gradients
// dW_l = dZ_l^T H_{l-1} of the block's 128 points are block-level tensor-core products.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "gm_internal.cuh"

namespace {

constexpr int FW = 64;               // width (features and hidden units)
constexpr int FD = 4;                // hidden layers
constexpr int FOCT = 10;             // octaves
constexpr int WS = 72;               // bf16 row stride of weights in shared memory
constexpr int TS = 136;              // bf16 row stride of transposed activations (128 points + 8)
constexpr int NPAR = FD * (FW * FW + FW) + FW + 1;   // 16 705
constexpr int NPAR_PAD = (NPAR + 3) & ~3;            // partial-sum slices, 16-byte aligned
static_assert(NPAR_PAD > NPAR, "the slices need a padding slot for the loss");
constexpr int TRAIN_PTS = 128;       // points per training block (8 warps x 16)

__host__ __device__ constexpr int w_off(int l) { return l * (FW * FW + FW); }
__host__ __device__ constexpr int b_off(int l) { return l * (FW * FW + FW) + FW * FW; }
constexpr int W5_OFF = FD * (FW * FW + FW);
constexpr int B5_OFF = W5_OFF + FW;

struct FieldBox {
    float cx, cy, cz, inv_h;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

// bf16(relu(lo)), bf16(relu(hi)) packed (lo in the low half) by one conversion instruction: rounding
// to nearest is monotone and keeps 0, so clamping before or after it gives the same value.
__device__ __forceinline__ uint32_t pack_bf16_relu(float lo, float hi) {
    uint32_t r;
    asm("cvt.rn.relu.bf16x2.f32 %0, %1, %2;" : "=r"(r) : "f"(hi), "f"(lo));
    return r;
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Feature `col` of a normalised position. y = 2^k x~ is exact; y - 2 rint(y / 2) is an exact
// reduction to [-1, 1] (sin and cos of pi y have period 2 in y), after which the hardware sine
// and cosine are accurate to ~1e-6 -- far below the bf16 rounding that follows.
__device__ __forceinline__ float feature(const float xt[3], int col) {
    if (col < 3) return xt[col];
    if (col >= 63) return 0.f;
    const int c = col - 3, k = c / 6, r = c % 6;
    float y = ldexpf(xt[r % 3], k);
    y = y - 2.f * rintf(0.5f * y);
    const float a = 3.14159265358979f * y;
    return r < 3 ? __sinf(a) : __cosf(a);
}

// A fragments (4 k16 chunks) of the 64 features of rows g and g + 8 of a 16-point group.
__device__ __forceinline__ void encode_frags(const float xa[3], const float xb[3], int t, uint32_t a[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
        a[kk][0] = pack_bf16(feature(xa, c0), feature(xa, c0 + 1));
        a[kk][1] = pack_bf16(feature(xb, c0), feature(xb, c0 + 1));
        a[kk][2] = pack_bf16(feature(xa, c1), feature(xa, c1 + 1));
        a[kk][3] = pack_bf16(feature(xb, c1), feature(xb, c1 + 1));
    }
}

// acc[j] (n tile j: outputs 8j..8j+7) = bias + A x W^T, W rows in shared memory (stride WS).
__device__ __forceinline__ void layer_mma(const uint32_t a[4][4], const __nv_bfloat16* __restrict__ W,
                                          const float* __restrict__ bias, int g, int t, float acc[8][4]) {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        const float b0 = bias[8 * j + 2 * t], b1 = bias[8 * j + 2 * t + 1];
        acc[j][0] = b0;
        acc[j][1] = b1;
        acc[j][2] = b0;
        acc[j][3] = b1;
    }
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            const __nv_bfloat16* row = W + (8 * j + g) * WS + 16 * kk + 2 * t;
            const uint32_t b0 = *reinterpret_cast<const uint32_t*>(row);
            const uint32_t b1 = *reinterpret_cast<const uint32_t*>(row + 8);
            mma16816(acc[j], a[kk], b0, b1);
        }
    }
}

// relu, round to bf16 and repack the accumulators as the next layer's A fragments.
__device__ __forceinline__ void relu_to_frags(const float acc[8][4], uint32_t a[4][4]) {
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const float* p = acc[2 * kk];
        const float* q = acc[2 * kk + 1];
        a[kk][0] = pack_bf16(fmaxf(p[0], 0.f), fmaxf(p[1], 0.f));
        a[kk][1] = pack_bf16(fmaxf(p[2], 0.f), fmaxf(p[3], 0.f));
        a[kk][2] = pack_bf16(fmaxf(q[0], 0.f), fmaxf(q[1], 0.f));
        a[kk][3] = pack_bf16(fmaxf(q[2], 0.f), fmaxf(q[3], 0.f));
    }
}

__device__ __forceinline__ float frag_elem(const uint32_t a[4][4], int kk, int r, int hi) {
    const uint32_t v = a[kk][r];
    const unsigned short s = hi ? (unsigned short)(v >> 16) : (unsigned short)(v & 0xffffu);
    return __bfloat162float(__ushort_as_bfloat16(s));
}

// Output layer: z5 of rows g (zr[0]) and g + 8 (zr[1]) from the h4 fragments, all four lanes of
// a quad end with the full sums.
__device__ __forceinline__ void output_dot(const uint32_t h[4][4], const float* __restrict__ w5, float b5, int t,
                                           float zr[2]) {
    float s0 = 0.f, s1 = 0.f;
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
        s0 = fmaf(frag_elem(h, kk, 0, 0), w5[c0], s0);
        s0 = fmaf(frag_elem(h, kk, 0, 1), w5[c0 + 1], s0);
        s0 = fmaf(frag_elem(h, kk, 2, 0), w5[c1], s0);
        s0 = fmaf(frag_elem(h, kk, 2, 1), w5[c1 + 1], s0);
        s1 = fmaf(frag_elem(h, kk, 1, 0), w5[c0], s1);
        s1 = fmaf(frag_elem(h, kk, 1, 1), w5[c0 + 1], s1);
        s1 = fmaf(frag_elem(h, kk, 3, 0), w5[c1], s1);
        s1 = fmaf(frag_elem(h, kk, 3, 1), w5[c1 + 1], s1);
    }
    s0 += __shfl_xor_sync(0xffffffffu, s0, 1);
    s0 += __shfl_xor_sync(0xffffffffu, s0, 2);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 1);
    s1 += __shfl_xor_sync(0xffffffffu, s1, 2);
    zr[0] = s0 + b5;
    zr[1] = s1 + b5;
}

__device__ __forceinline__ float softplusf(float z) { return z > 30.f ? z : log1pf(expf(z)); }
__device__ __forceinline__ float sigmoidf_(float z) { return 1.f / (1.f + expf(-z)); }

__device__ __forceinline__ void load_xt(const float* __restrict__ xyz, uint64_t i, uint64_t n, FieldBox B, float xt[3]) {
    if (i < n) {
        xt[0] = (xyz[3 * i] - B.cx) * B.inv_h;
        xt[1] = (xyz[3 * i + 1] - B.cy) * B.inv_h;
        xt[2] = (xyz[3 * i + 2] - B.cz) * B.inv_h;
    } else {
        xt[0] = xt[1] = xt[2] = 0.f;
    }
}

// ---- parameter maintenance --------------------------------------------------------------------
// bf16 copies of the hidden-layer weights: W (row = output) and W^T (row = input), dense 64x64.
__global__ void k_field_cast(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wbf,
                             __nv_bfloat16* __restrict__ wtbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= FD * FW * FW) return;
    const int l = i / (FW * FW), r = (i / FW) % FW, c = i % FW;
    const __nv_bfloat16 v = __float2bfloat16_rn(theta[w_off(l) + r * FW + c]);
    wbf[i] = v;
    wtbf[l * FW * FW + c * FW + r] = v;
}

__global__ void k_field_adam(float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v,
                             float* __restrict__ grad, float lr, float bc1, float bc2,
                             __nv_bfloat16* __restrict__ wbf, __nv_bfloat16* __restrict__ wtbf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= NPAR) return;
    const float g = grad[i];
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    theta[i] = th;
    grad[i] = 0.f;
    // keep the bf16 copies of the hidden weights current
    const int l = i / (FW * FW + FW), o = i % (FW * FW + FW);
    if (l < FD && o < FW * FW) {
        const int r = o / FW, c = o % FW;
        const __nv_bfloat16 b = __float2bfloat16_rn(th);
        wbf[l * FW * FW + r * FW + c] = b;
        wtbf[l * FW * FW + c * FW + r] = b;
    }
}

// Stage bf16 weights (dense 64 x 64 per layer) into shared memory rows of stride WS.
__device__ __forceinline__ void stage_weights(const __nv_bfloat16* __restrict__ src, __nv_bfloat16* dst) {
    for (int i = threadIdx.x; i < FD * FW * FW / 2; i += blockDim.x) {
        const int e = 2 * i, l = e / (FW * FW), r = (e / FW) % FW, c = e % FW;
        *reinterpret_cast<uint32_t*>(dst + l * FW * WS + r * WS + c) = reinterpret_cast<const uint32_t*>(src)[i];
    }
}

// ---- inference --------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_field_query(const float* __restrict__ xyz, uint64_t n,
                                                     const __nv_bfloat16* __restrict__ wbf,
                                                     const float* __restrict__ theta, FieldBox B,
                                                     float* __restrict__ out) {
    __shared__ __align__(16) __nv_bfloat16 sW[FD * FW * WS];
    __shared__ float sb[FD * FW];
    __shared__ float sw5[FW + 1];
    stage_weights(wbf, sW);
    for (int i = threadIdx.x; i < FD * FW; i += blockDim.x) sb[i] = theta[b_off(i / FW) + i % FW];
    for (int i = threadIdx.x; i <= FW; i += blockDim.x) sw5[i] = theta[W5_OFF + i];
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const uint64_t groups = (n + 15) / 16;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t grp = warp0; grp < groups; grp += nwarps) {
        const uint64_t ra = grp * 16 + g, rb = ra + 8;
        float xa[3], xb[3];
        load_xt(xyz, ra, n, B, xa);
        load_xt(xyz, rb, n, B, xb);
        uint32_t a[4][4];
        encode_frags(xa, xb, t, a);
        float acc[8][4];
#pragma unroll 1
        for (int l = 0; l < FD; ++l) {
            layer_mma(a, sW + l * FW * WS, sb + l * FW, g, t, acc);
            relu_to_frags(acc, a);
        }
        float z[2];
        output_dot(a, sw5, sw5[FW], t, z);
        if (t == 0) {
            if (ra < n) out[ra] = softplusf(z[0]);
            if (rb < n) out[rb] = softplusf(z[1]);
        }
    }
}


// ---- inference on the 5th-generation tensor cores ---------------------------------------------
// Blocks of 256 threads, persistent; each half (128 threads, its own named barrier) runs its own
// pipeline over tiles of 128 points (the MMA's M), so two tiles per block -- and those of the other
// resident blocks -- overlap one tile's tensor-core products with another's epilogue, while the
// weights are staged once per block. Per tile: the point coordinates arrive by a bulk asynchronous
// copy (double-buffered, the next tile's copy in flight while this one computes; plain loads when
// the input is not 16-byte aligned or the tile is the ragged tail); thread t of the half encodes
// point t's 64 features into row t of its A tile (bf16, K-major core-matrix layout: 8 x 8 blocks
// of 128 bytes); per layer one thread issues four tcgen05.mma (M 128, N 64, K 16, bf16 x bf16 ->
// FP32 in tensor memory, columns 64 h .. 64 h + 63 for half h) and commits them to the half's
// mbarrier; every thread then reads its row of the accumulator with tcgen05.ld, adds the bias,
// applies ReLU, rounds to bf16 and writes the next A row. The output layer is
// a fifth product with N = 16 whose B rows are the three bf16 parts of w5. Waits are bounded: on a
// timeout the block records GM_DEV_WAIT_TIMEOUT, drains its own copies, frees its tensor memory and
// returns.
constexpr int TQ = 128;                       // points per tile (threads per half)
constexpr int TQ_THREADS = 2 * TQ;
constexpr uint32_t TQ_TMEM_COLS = 128;        // two FP32 accumulators of N = 64
constexpr int TQ_WAIT_ITERS = 1 << 22;

struct QuerySmem {
    alignas(1024) __nv_bfloat16 A[2][TQ * FW];    // 2 x 16 KB
    alignas(1024) __nv_bfloat16 W[FD][FW * FW];   // 32 KB
    alignas(1024) __nv_bfloat16 W5[16 * FW];      // output layer as B (N = 16): w5 = hi + mid + lo in rows 0..2
    alignas(16) float bias[FD * FW];
    float w5[FW + 1];
    alignas(16) float xyz[2][2][TQ * 3];          // [half][buffer]
    alignas(8) uint64_t mbar_mma[2];
    uint64_t mbar_ld[2][2];
    uint32_t tmem;
    int abort;
};

__device__ __forceinline__ uint32_t smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor, no swizzle: start address, the byte offset between core
// matrices along K (leading) and along M or N (stride), descriptor version 1.
__device__ __forceinline__ uint64_t umma_desc(uint32_t addr, uint32_t lead, uint32_t stride) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lead >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((stride >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, N = 64, M = 128.
constexpr uint32_t kQueryIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kQueryIdescN16 = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

// The three bf16 parts of an FP32 value: hi = bf16(w), mid = bf16(w - hi), lo = w - hi - mid. Each
// difference is exact in FP32 and lo needs at most 8 significant bits, so hi + mid + lo = w exactly;
// a product with a bf16 activation is then three exact products summed in FP32.
__device__ __forceinline__ void split3_bf16(float w, __nv_bfloat16 part[3]) {
    part[0] = __float2bfloat16_rn(w);
    const float r1 = w - __bfloat162float(part[0]);
    part[1] = __float2bfloat16_rn(r1);
    part[2] = __float2bfloat16_rn(r1 - __bfloat162float(part[1]));
}

// Bounded wait on an mbarrier phase: false after `iters` polls without completion.
__device__ __forceinline__ bool mbar_wait_n(uint32_t addr, uint32_t parity, uint32_t iters) {
    for (uint32_t it = 0; it < iters; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity) {
    for (int it = 0; it < TQ_WAIT_ITERS; ++it) {
        uint32_t done;
        asm volatile(
            "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

__device__ __forceinline__ void bulk_load(float* dst, const float* src, uint32_t bytes, uint64_t* mbar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(mbar)), "r"(bytes) : "memory");
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(mbar))
        : "memory");
}

__device__ __forceinline__ void half_sync(int h) {
    if (h == 0) asm volatile("bar.sync 1, 128;" ::: "memory");
    else asm volatile("bar.sync 2, 128;" ::: "memory");
}

// Row t of an A tile: 64 values as bf16, eight 16-byte stores into the core-matrix layout.
__device__ __forceinline__ void store_a_row(__nv_bfloat16* A, int t, const float* v) {
#pragma unroll
    for (int kg = 0; kg < 8; ++kg) {
        uint4 q;
        q.x = pack_bf16(v[8 * kg + 0], v[8 * kg + 1]);
        q.y = pack_bf16(v[8 * kg + 2], v[8 * kg + 3]);
        q.z = pack_bf16(v[8 * kg + 4], v[8 * kg + 5]);
        q.w = pack_bf16(v[8 * kg + 6], v[8 * kg + 7]);
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(A) + kg * 2048 + (t >> 3) * 128 + (t & 7) * 16) = q;
    }
}

// The 64 features of one point for the tensor-core kernel: sine and cosine of 2^k pi x~ from an
// exact reduction and the hardware sincos at octaves 0, 3, 6 and 9, and by the double-angle
// formulas (sin 2a = 2 sin a cos a, cos 2a = cos^2 a - sin^2 a) for the two octaves after each;
// two doublings keep the error within a few 1e-6, far under the bf16 rounding that follows.
__device__ __forceinline__ void features_fast(const float xt[3], float* v) {
    v[0] = xt[0];
    v[1] = xt[1];
    v[2] = xt[2];
    v[63] = 0.f;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        float sn = 0.f, cs = 1.f;
#pragma unroll
        for (int k = 0; k < FOCT; ++k) {
            if (k % 3 == 0) {
                float y = ldexpf(xt[r], k);
                y = y - 2.f * rintf(0.5f * y);
                __sincosf(3.14159265358979f * y, &sn, &cs);
            } else {
                const float s2 = 2.f * (sn * cs);
                const float c2 = fmaf(cs, cs, -(sn * sn));
                sn = s2;
                cs = c2;
            }
            v[3 + 6 * k + r] = sn;
            v[6 + 6 * k + r] = cs;
        }
    }
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

__global__ void __launch_bounds__(TQ_THREADS, 3) k_field_query_tc(const float* __restrict__ xyz, uint64_t n,
                                                              const __nv_bfloat16* __restrict__ wbf,
                                                              const float* __restrict__ theta, FieldBox B, int bulk,
                                                              float* __restrict__ out, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char q_smem_raw[];
    QuerySmem& S = *reinterpret_cast<QuerySmem*>(q_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int h = tid / TQ, t = tid % TQ;   // half and row within the half's tile
    // weights in the core-matrix layout: (n, k) at (k / 8) * 1024 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2
    for (int i = tid; i < FD * FW * 8; i += TQ_THREADS) {
        const int l = i / (FW * 8), nn = (i / 8) % FW, kg = i % 8;
        const uint4 q = reinterpret_cast<const uint4*>(wbf + (size_t)l * FW * FW + nn * FW)[kg];
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.W[l]) + kg * 1024 + (nn >> 3) * 128 + (nn & 7) * 16) = q;
    }
    // the output layer as a 16 x 64 B operand: rows 0..2 the three bf16 parts of w5, the rest zero;
    // (n, k) at (k / 8) * 256 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2
    for (int e = tid; e < 16 * FW; e += TQ_THREADS) {
        const int nn = e / FW, k = e % FW;
        __nv_bfloat16 part[3];
        split3_bf16(theta[W5_OFF + k], part);
        const __nv_bfloat16 v = nn < 3 ? part[nn] : __float2bfloat16_rn(0.f);
        *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<char*>(S.W5) + (k >> 3) * 256 + (nn >> 3) * 128 +
                                          (nn & 7) * 16 + (k & 7) * 2) = v;
    }
    for (int i = tid; i < FD * FW; i += TQ_THREADS) S.bias[i] = theta[b_off(i / FW) + i % FW];
    for (int i = tid; i <= FW; i += TQ_THREADS) S.w5[i] = theta[W5_OFF + i];
    if (tid == 0) {
        S.abort = 0;
        for (int k = 0; k < 2; ++k) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar_mma[k])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar_ld[k][0])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar_ld[k][1])));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem)),
                     "r"(TQ_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem_h = S.tmem + (uint32_t)(h * FW);         // this half's accumulator columns
    const uint32_t row_addr = tmem_h + ((uint32_t)((warp & 3) * 32) << 16);
    __nv_bfloat16* A = S.A[h];
    const uint32_t a_addr = smem_addr(A);
    const uint64_t ntiles = (n + TQ - 1) / TQ;
    const uint64_t pipes = 2ull * gridDim.x, pipe = 2ull * blockIdx.x + h;
    uint32_t pm = 0, pl[2] = {0, 0};
    bool pending[2] = {false, false};   // row 0 of the half: a bulk copy into this buffer is in flight
    auto full_tile = [&](uint64_t tile) { return (tile + 1) * TQ <= n; };
    uint64_t tile = pipe;
    if (t == 0 && bulk && tile < ntiles && full_tile(tile)) {
        bulk_load(S.xyz[h][0], xyz + tile * TQ * 3, TQ * 12, &S.mbar_ld[h][0]);
        pending[0] = true;
    }
    bool stop = false;
    for (int it = 0; tile < ntiles && !stop; ++it, tile += pipes) {
        const int buf = it & 1;
        const uint64_t next = tile + pipes;
        if (t == 0 && bulk && next < ntiles && full_tile(next)) {
            bulk_load(S.xyz[h][buf ^ 1], xyz + next * TQ * 3, TQ * 12, &S.mbar_ld[h][buf ^ 1]);
            pending[buf ^ 1] = true;
        }
        const uint64_t i = tile * TQ + t;
        float x[3] = {0.f, 0.f, 0.f};
        if (bulk && full_tile(tile)) {
            if (!mbar_wait(smem_addr(&S.mbar_ld[h][buf]), pl[buf])) S.abort = 1;
            pl[buf] ^= 1;
            if (t == 0) pending[buf] = false;
            x[0] = S.xyz[h][buf][3 * t];
            x[1] = S.xyz[h][buf][3 * t + 1];
            x[2] = S.xyz[h][buf][3 * t + 2];
        } else if (i < n) {
            x[0] = xyz[3 * i];
            x[1] = xyz[3 * i + 1];
            x[2] = xyz[3 * i + 2];
        }
        float xt[3] = {(x[0] - B.cx) * B.inv_h, (x[1] - B.cy) * B.inv_h, (x[2] - B.cz) * B.inv_h};
        float v[FW];
        features_fast(xt, v);
        store_a_row(A, t, v);
        // four hidden layers, then the output layer (l == FD) as one more product: A = h4, B = the
        // three parts of w5, so z5 - b5 is the sum of the first three accumulator columns. Each
        // product starts a fresh accumulator (the previous tile's last read is complete); the bias
        // is added to the 64 sums as they are read back.
        for (int l = 0; l <= FD; ++l) {
            asm volatile("fence.proxy.async.shared::cta;");   // this thread's A row, visible to the MMA
            asm volatile("tcgen05.fence::before_thread_sync;");
            half_sync(h);
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (S.abort) {
                stop = true;
                break;
            }
            if (t == 0) {
                if (l < FD) {
                    const uint32_t w_addr = smem_addr(S.W[l]);
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const uint64_t da = umma_desc(a_addr + s * 4096, 2048, 128);
                        const uint64_t db = umma_desc(w_addr + s * 2048, 1024, 128);
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_h),
                            "l"(da), "l"(db), "r"(kQueryIdesc), "r"(s > 0 ? 1u : 0u));
                    }
                } else {
                    const uint32_t w5_addr = smem_addr(S.W5);
#pragma unroll
                    for (int s = 0; s < 4; ++s) {
                        const uint64_t da = umma_desc(a_addr + s * 4096, 2048, 128);
                        const uint64_t db = umma_desc(w5_addr + s * 512, 256, 128);
                        asm volatile(
                            "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
                            " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem_h),
                            "l"(da), "l"(db), "r"(kQueryIdescN16), "r"(s > 0 ? 1u : 0u));
                    }
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&S.mbar_mma[h])));
            }
            if (!mbar_wait(smem_addr(&S.mbar_mma[h]), pm)) S.abort = 1;
            pm ^= 1;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (l == FD) {
                float v[16];
                tmem_ld16(row_addr, v);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                if (i < n) out[i] = softplusf(((v[0] + v[1]) + v[2]) + S.w5[FW]);
                break;
            }
            // 32 columns at a time: read, add the bias, ReLU and round to bf16, write the next A row
            const float* bl = S.bias + l * FW;
#pragma unroll
            for (int c0 = 0; c0 < FW; c0 += 32) {
                float va[32];
                tmem_ld16(row_addr + c0, va);
                tmem_ld16(row_addr + c0 + 16, va + 16);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                uint32_t pk[16];
#pragma unroll
                for (int c = 0; c < 32; c += 4) {
                    const float4 b4 = *reinterpret_cast<const float4*>(bl + c0 + c);   // one 16-byte broadcast
                    pk[c / 2] = pack_bf16_relu(va[c] + b4.x, va[c + 1] + b4.y);
                    pk[c / 2 + 1] = pack_bf16_relu(va[c + 2] + b4.z, va[c + 3] + b4.w);
                }
#pragma unroll
                for (int g = 0; g < 4; ++g) {
                    const int kg = c0 / 8 + g;
                    *reinterpret_cast<uint4*>(reinterpret_cast<char*>(A) + kg * 2048 + (t >> 3) * 128 + (t & 7) * 16) =
                        make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
                }
            }
        }
    }
    if (S.abort && t == 0) {
        atomicCAS(err, 0, GM_DEV_WAIT_TIMEOUT);
        for (int b = 0; b < 2; ++b)
            if (pending[b]) mbar_wait(smem_addr(&S.mbar_ld[h][b]), pl[b]);   // drain this half's own copies
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(S.tmem), "r"(TQ_TMEM_COLS));
}

// ---- training: forward + backward of 128 points per block -------------------------------------
struct TrainSmem {
    __nv_bfloat16 W[FD * FW * WS];     // W_l rows (output) for the forward products
    __nv_bfloat16 WT[FD * FW * WS];    // W_l^T rows (input) for dH = dZ W
    __nv_bfloat16 HT[FD * FW * TS];    // H_0..H_3 transposed (feature rows, point columns)
    __nv_bfloat16 DZT[FW * TS];        // dZ_l transposed (output rows, point columns)
    float b[FD * FW];
    float w5[FW + 1];
    float gw5[FW];
    float gb[FW];
};

__device__ __forceinline__ void store_frags_T(const uint32_t a[4][4], __nv_bfloat16* T, int p0, int g, int t) {
    // fragment (rows = points p0 + g, p0 + g + 8; cols = features) -> T[feature][point]
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
        const uint32_t* v = a[kk];
        auto put = [&](int col, int row, uint32_t w) {
            T[col * TS + row] = __ushort_as_bfloat16((unsigned short)(w & 0xffffu));
            T[(col + 1) * TS + row] = __ushort_as_bfloat16((unsigned short)(w >> 16));
        };
        put(c0, p0 + g, v[0]);
        put(c0, p0 + g + 8, v[1]);
        put(c1, p0 + g, v[2]);
        put(c1, p0 + g + 8, v[3]);
    }
}

// dW (64 x 64, rows = outputs) += DZT x HT^T over the block's 128 points; each warp one m16 row
// slab and four n8 tiles; results go to the global gradient with atomics.
__device__ __forceinline__ void block_weight_grad(const __nv_bfloat16* DZT, const __nv_bfloat16* HTl,
                                                  float* __restrict__ gW, int warp, int g, int t) {
    const int m0 = 16 * (warp >> 1), n0 = 32 * (warp & 1);
    float acc[4][4];
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
#pragma unroll
    for (int ks = 0; ks < TRAIN_PTS / 16; ++ks) {
        const int k0 = 16 * ks + 2 * t;
        uint32_t a[4];
        a[0] = *reinterpret_cast<const uint32_t*>(DZT + (m0 + g) * TS + k0);
        a[1] = *reinterpret_cast<const uint32_t*>(DZT + (m0 + g + 8) * TS + k0);
        a[2] = *reinterpret_cast<const uint32_t*>(DZT + (m0 + g) * TS + k0 + 8);
        a[3] = *reinterpret_cast<const uint32_t*>(DZT + (m0 + g + 8) * TS + k0 + 8);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const __nv_bfloat16* row = HTl + (n0 + 8 * j + g) * TS + k0;
            mma16816(acc[j], a, *reinterpret_cast<const uint32_t*>(row), *reinterpret_cast<const uint32_t*>(row + 8));
        }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const int c = n0 + 8 * j + 2 * t;
        atomicAdd(&gW[(m0 + g) * FW + c], acc[j][0]);
        atomicAdd(&gW[(m0 + g) * FW + c + 1], acc[j][1]);
        atomicAdd(&gW[(m0 + g + 8) * FW + c], acc[j][2]);
        atomicAdd(&gW[(m0 + g + 8) * FW + c + 1], acc[j][3]);
    }
}

__device__ __forceinline__ uint32_t philox_x(uint32_t c0, uint32_t c1, uint32_t k0, uint32_t k1) {
    uint32_t c2 = 0, c3 = 0;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
        const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c1 = lo1;
        c3 = lo0;
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return c0;
}

// One block: 128 batch points. `pts` are float4 (x, y, z, -) positions or, when stride is 3,
// packed xyz; targets are FP32. Batch entries come from `idx` or, if null, from Philox
// (key = seed, counter = (step, i)) modulo n.
__global__ void __launch_bounds__(256, 1) k_field_train(const float* __restrict__ pts, int stride,
                                                        const float* __restrict__ target, uint64_t n,
                                                        const uint32_t* __restrict__ idx, uint32_t batch,
                                                        uint32_t step, uint2 seed, FieldBox B,
                                                        const __nv_bfloat16* __restrict__ wbf,
                                                        const __nv_bfloat16* __restrict__ wtbf,
                                                        const float* __restrict__ theta, float* __restrict__ grad,
                                                        float* __restrict__ loss_sum) {
    extern __shared__ __align__(16) unsigned char smraw[];
    TrainSmem& S = *reinterpret_cast<TrainSmem*>(smraw);
    stage_weights(wbf, S.W);
    stage_weights(wtbf, S.WT);
    for (int i = threadIdx.x; i < FD * FW; i += blockDim.x) S.b[i] = theta[b_off(i / FW) + i % FW];
    for (int i = threadIdx.x; i <= FW; i += blockDim.x) S.w5[i] = theta[W5_OFF + i];
    for (int i = threadIdx.x; i < FW; i += blockDim.x) {
        S.gw5[i] = 0.f;
        S.gb[i] = 0.f;
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
    const int p0 = 16 * warp;                               // this warp's first point in the block
    const uint32_t e0 = blockIdx.x * TRAIN_PTS + p0 + g, e1 = e0 + 8;   // batch entries
    auto draw = [&](uint32_t e) -> uint64_t {
        if (e >= batch) return n;                           // padding row
        if (idx) return idx[e];
        return philox_x(step, e, seed.x, seed.y) % (uint32_t)n;
    };
    const uint64_t ia = draw(e0), ib = draw(e1);
    float xa[3], xb[3];
    auto load = [&](uint64_t i, float x[3]) {
        if (i < n) {
            x[0] = (pts[stride * i] - B.cx) * B.inv_h;
            x[1] = (pts[stride * i + 1] - B.cy) * B.inv_h;
            x[2] = (pts[stride * i + 2] - B.cz) * B.inv_h;
        } else {
            x[0] = x[1] = x[2] = 0.f;
        }
    };
    load(ia, xa);
    load(ib, xb);
    // forward, keeping every layer's bf16 input fragments
    uint32_t h[FD + 1][4][4];
    encode_frags(xa, xb, t, h[0]);
    float acc[8][4];
#pragma unroll
    for (int l = 0; l < FD; ++l) {
        store_frags_T(h[l], S.HT + l * FW * TS, p0, g, t);
        layer_mma(h[l], S.W + l * FW * WS, S.b + l * FW, g, t, acc);
        relu_to_frags(acc, h[l + 1]);
    }
    float z[2];
    output_dot(h[FD], S.w5, S.w5[FW], t, z);
    const float inv_b = 1.f / (float)batch;
    float dz5[2];
    {
        const float ya = ia < n ? target[ia] : 0.f, yb = ib < n ? target[ib] : 0.f;
        const float fa = softplusf(z[0]), fb = softplusf(z[1]);
        const float ra = e0 < batch ? fa - ya : 0.f, rb = e1 < batch ? fb - yb : 0.f;
        dz5[0] = 2.f * ra * inv_b * sigmoidf_(z[0]);
        dz5[1] = 2.f * rb * inv_b * sigmoidf_(z[1]);
        float l2 = t == 0 ? ra * ra + rb * rb : 0.f;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) l2 += __shfl_xor_sync(0xffffffffu, l2, o);
        if (lane == 0) atomicAdd(loss_sum, l2);
    }
    // output layer gradients and dz4 = dz5 w5 (.) [h4 > 0]
    uint32_t dz[4][4];
    {
        float gb5 = t == 0 ? dz5[0] + dz5[1] : 0.f;
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
            const int cols[4] = {c0, c0 + 1, c1, c1 + 1};
            float d0[4], d1[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r0 = q < 2 ? 0 : 2, hi = q & 1;
                const float ha = frag_elem(h[FD], kk, r0, hi), hb = frag_elem(h[FD], kk, r0 + 1, hi);
                float gsum = dz5[0] * ha + dz5[1] * hb;
                gsum += __shfl_xor_sync(0xffffffffu, gsum, 4);
                gsum += __shfl_xor_sync(0xffffffffu, gsum, 8);
                gsum += __shfl_xor_sync(0xffffffffu, gsum, 16);
                if (g == 0) atomicAdd(&S.gw5[cols[q]], gsum);
                d0[q] = ha > 0.f ? dz5[0] * S.w5[cols[q]] : 0.f;
                d1[q] = hb > 0.f ? dz5[1] * S.w5[cols[q]] : 0.f;
            }
            dz[kk][0] = pack_bf16(d0[0], d0[1]);
            dz[kk][1] = pack_bf16(d1[0], d1[1]);
            dz[kk][2] = pack_bf16(d0[2], d0[3]);
            dz[kk][3] = pack_bf16(d1[2], d1[3]);
        }
        gb5 += __shfl_xor_sync(0xffffffffu, gb5, 4);
        gb5 += __shfl_xor_sync(0xffffffffu, gb5, 8);
        gb5 += __shfl_xor_sync(0xffffffffu, gb5, 16);
        if (lane == 0) atomicAdd(&grad[B5_OFF], gb5);
    }
#pragma unroll
    for (int l = FD - 1; l >= 0; --l) {
        // bias gradient of layer l+1 (index l) and dZ_l^T into shared memory
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const int c0 = 16 * kk + 2 * t, c1 = c0 + 8;
            const int cols[4] = {c0, c0 + 1, c1, c1 + 1};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int r0 = q < 2 ? 0 : 2, hi = q & 1;
                float s = frag_elem(dz, kk, r0, hi) + frag_elem(dz, kk, r0 + 1, hi);
                s += __shfl_xor_sync(0xffffffffu, s, 4);
                s += __shfl_xor_sync(0xffffffffu, s, 8);
                s += __shfl_xor_sync(0xffffffffu, s, 16);
                if (g == 0) atomicAdd(&S.gb[cols[q]], s);
            }
        }
        store_frags_T(dz, S.DZT, p0, g, t);
        __syncthreads();
        block_weight_grad(S.DZT, S.HT + l * FW * TS, grad + w_off(l), warp, g, t);
        for (int i = threadIdx.x; i < FW; i += blockDim.x) {
            atomicAdd(&grad[b_off(l) + i], S.gb[i]);
            S.gb[i] = 0.f;
        }
        if (l > 0) {
            // dH_{l-1} = dZ_l W_l, then the relu mask of h_l (the input of this layer)
            float dh[8][4];
#pragma unroll
            for (int j = 0; j < 8; ++j) dh[j][0] = dh[j][1] = dh[j][2] = dh[j][3] = 0.f;
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    const __nv_bfloat16* row = S.WT + l * FW * WS + (8 * j + g) * WS + 16 * kk + 2 * t;
                    mma16816(dh[j], dz[kk], *reinterpret_cast<const uint32_t*>(row),
                             *reinterpret_cast<const uint32_t*>(row + 8));
                }
            }
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {
                const float* p = dh[2 * kk];
                const float* q = dh[2 * kk + 1];
                const float m00 = frag_elem(h[l], kk, 0, 0) > 0.f, m01 = frag_elem(h[l], kk, 0, 1) > 0.f;
                const float m10 = frag_elem(h[l], kk, 1, 0) > 0.f, m11 = frag_elem(h[l], kk, 1, 1) > 0.f;
                const float m20 = frag_elem(h[l], kk, 2, 0) > 0.f, m21 = frag_elem(h[l], kk, 2, 1) > 0.f;
                const float m30 = frag_elem(h[l], kk, 3, 0) > 0.f, m31 = frag_elem(h[l], kk, 3, 1) > 0.f;
                dz[kk][0] = pack_bf16(p[0] * m00, p[1] * m01);
                dz[kk][1] = pack_bf16(p[2] * m10, p[3] * m11);
                dz[kk][2] = pack_bf16(q[0] * m20, q[1] * m21);
                dz[kk][3] = pack_bf16(q[2] * m30, q[3] * m31);
            }
        }
        __syncthreads();
    }
    for (int i = threadIdx.x; i < FW; i += blockDim.x) atomicAdd(&grad[W5_OFF + i], S.gw5[i]);
}

// ---- training on the 5th-generation tensor cores ----------------------------------------------
// Persistent blocks of 256 threads, one per SM; two threads per point (accumulator row): thread
// (quarter q, half c) owns point 32 q + lane and the columns [32 c, 32 c + 32). Per tile of 128
// batch points, every product of the hidden layers is a tcgen05.mma (bf16 x bf16, FP32 in tensor
// memory):
//   forward   Z_l = H_l W_l^T + b_l        A = H_l rows (K = inputs),   B = W_l   (N = outputs)
//   backward  dH_l = dZ_l W_l              A = dZ_l rows (K = outputs), B = W_l^T (N = inputs)
//             gW_l += dZ_l^T H_l           A = dZ_l^T (K = points),     B = H_l^T (N = inputs)
//             gb_l += dZ_l^T 1             A = dZ_l^T,                  B = a 16 x 128 block whose row 0 is ones
// The weight and bias gradients accumulate in tensor memory over all tiles of the block and leave
// it once, into the block's own slice of a partial-sum buffer that the update kernel reduces in a
// fixed order (deterministic, no atomics on the gradient). The point-major operands (dZ^T, H^T)
// are written one 2-byte element per (row, point) into a no-swizzle K-major layout whose core
// matrices sit 144 bytes apart along the points, so that the 32 lanes of a warp (32 consecutive
// points) store into 32 different banks. The gradient products have 64 real rows (outputs); the
// MMA runs with M = 128 and rows 64..127 read the next buffer and are never read back. The output
// layer (w5, b5) and the loss stay in FP32 on the CUDA cores: w5's gradient is a warp transpose-sum.
// Waits are bounded; on a timeout the block records GM_DEV_WAIT_TIMEOUT, frees its tensor memory
// and returns.
constexpr int TT = 128;                        // points per tile
constexpr int TT_CW = 32;                      // accumulator columns per thread (16: 53.9 vs 49.8 us a step)
constexpr int TT_GROUPS = FW / TT_CW;          // threads per point
constexpr int TT_THREADS = TT * TT_GROUPS;
constexpr uint32_t TT_TMEM_COLS = 512;
constexpr uint32_t TT_COL_ACC = 0;             // forward / dH accumulator (64 columns)
constexpr uint32_t TT_COL_GW = 64;             // weight gradients, 64 columns per layer
constexpr uint32_t TT_COL_GB = 320;            // bias gradients, 16 columns per layer (column 0 used)
constexpr int T_LBO = 144;                     // point-major operands: core matrices along the points
constexpr int T_SBO = 16 * T_LBO;              // ... and along the rows
constexpr int T_BYTES = 8 * T_SBO;             // 64 rows x 128 points

struct TrainTcSmem {
    alignas(1024) __nv_bfloat16 A[TT * FW];        // rows = points: H_l (forward) or dZ_l (backward)
    alignas(1024) __nv_bfloat16 W[FD][FW * FW];    // W_l, rows = outputs
    alignas(1024) __nv_bfloat16 WT[FD][FW * FW];   // W_l^T, rows = inputs
    alignas(1024) unsigned char DZT[T_BYTES];      // dZ_l^T; rows 64..127 of its M = 128 read HT[0]
    alignas(1024) unsigned char HT[FD][T_BYTES];   // H_l^T, l = 0..3
    alignas(1024) unsigned char ONES[2 * T_SBO];   // 16 rows x 128 points, row 0 = 1
    alignas(16) float bias[FD * FW];
    float w5[FW + 1];
    float gw5w[TT_THREADS / 32][32];   // per warp: w5-gradient sums of its columns
    float zpart[TT_GROUPS][TT];
    float gb5w[4], lossw[4];           // per warp of the first column half
    alignas(8) uint64_t mbar;
    uint32_t tmem;
    int abort;
};

// Byte offset of element (row, point) of a point-major operand.
__device__ __forceinline__ int tp_off(int row, int k) {
    return (k >> 3) * T_LBO + (row >> 3) * T_SBO + (row & 7) * 16 + (k & 7) * 2;
}

constexpr uint32_t kIdescN64 = (1u << 4) | (1u << 7) | (1u << 10) | ((64u >> 3) << 17) | ((128u >> 4) << 24);
constexpr uint32_t kIdescN16 = (1u << 4) | (1u << 7) | (1u << 10) | ((16u >> 3) << 17) | ((128u >> 4) << 24);

__device__ __forceinline__ void umma_bf16(uint32_t d, uint64_t da, uint64_t db, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
        "l"(da), "l"(db), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void tmem_st_cw(uint32_t taddr, const float* v) {
#pragma unroll
    for (int c0 = 0; c0 < TT_CW; c0 += 16)
        asm volatile(
            "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::
                "r"(taddr + c0),
            "f"(v[c0]), "f"(v[c0 + 1]), "f"(v[c0 + 2]), "f"(v[c0 + 3]), "f"(v[c0 + 4]), "f"(v[c0 + 5]),
            "f"(v[c0 + 6]), "f"(v[c0 + 7]), "f"(v[c0 + 8]), "f"(v[c0 + 9]), "f"(v[c0 + 10]), "f"(v[c0 + 11]),
            "f"(v[c0 + 12]), "f"(v[c0 + 13]), "f"(v[c0 + 14]), "f"(v[c0 + 15]));
}

// This thread's part of a row (columns c0 .. c0 + TT_CW - 1 as packed bf16 pairs) into the K-major
// A tile and into column p of a point-major operand.
__device__ __forceinline__ void store_part(__nv_bfloat16* A, unsigned char* T, int p, int c0, const uint32_t* pk) {
#pragma unroll
    for (int g = 0; g < TT_CW / 8; ++g) {
        const int kg = c0 / 8 + g;
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(A) + kg * 2048 + (p >> 3) * 128 + (p & 7) * 16) =
            make_uint4(pk[4 * g], pk[4 * g + 1], pk[4 * g + 2], pk[4 * g + 3]);
    }
#pragma unroll
    for (int j = 0; j < TT_CW; j += 2) {
        *reinterpret_cast<uint16_t*>(T + tp_off(c0 + j, p)) = (uint16_t)(pk[j / 2] & 0xffffu);
        *reinterpret_cast<uint16_t*>(T + tp_off(c0 + j + 1, p)) = (uint16_t)(pk[j / 2] >> 16);
    }
}

__device__ __forceinline__ float bf_lo(uint32_t v) { return __uint_as_float(v << 16); }
__device__ __forceinline__ float bf_hi(uint32_t v) { return __uint_as_float(v & 0xffff0000u); }

// Lane L ends with the sum over the warp's 32 lanes of v[L mod TT_CW].
__device__ __forceinline__ float warp_transpose_sum(float v[TT_CW]) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 16; o >= TT_CW; o >>= 1) {
#pragma unroll
        for (int j = 0; j < TT_CW; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], o);
    }
#pragma unroll
    for (int o = TT_CW / 2; o >= 1; o >>= 1) {
        const bool up = (lane & o) != 0;
#pragma unroll
        for (int j = 0; j < o; ++j) {
            const float send = up ? v[j] : v[j + o];
            const float keep = up ? v[j + o] : v[j];
            v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
        }
    }
    return v[0];
}

__global__ void __launch_bounds__(TT_THREADS, 1) k_field_train_tc(
    const float* __restrict__ pts, int stride, const float* __restrict__ target, uint64_t n,
    const uint32_t* __restrict__ idx, uint32_t batch, uint32_t step, uint2 seed, FieldBox B,
    const __nv_bfloat16* __restrict__ wbf, const __nv_bfloat16* __restrict__ wtbf, const float* __restrict__ theta,
    float* __restrict__ partial, int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char t_smem_raw[];
    TrainTcSmem& S = *reinterpret_cast<TrainTcSmem*>(t_smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = warp & 3, c = warp >> 2;
    const int p = 32 * q + lane, c0 = TT_CW * c;
    // weights in the core-matrix layout: (n, k) at (k / 8) * 1024 + (n / 8) * 128 + (n % 8) * 16 + (k % 8) * 2
    for (int i = tid; i < FD * FW * 8; i += TT_THREADS) {
        const int l = i / (FW * 8), nn = (i / 8) % FW, kg = i % 8;
        const size_t src = (size_t)l * FW * FW + nn * FW;
        const int dst = kg * 1024 + (nn >> 3) * 128 + (nn & 7) * 16;
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.W[l]) + dst) = reinterpret_cast<const uint4*>(wbf + src)[kg];
        *reinterpret_cast<uint4*>(reinterpret_cast<char*>(S.WT[l]) + dst) =
            reinterpret_cast<const uint4*>(wtbf + src)[kg];
    }
    for (int i = tid; i < 2 * T_SBO / 16; i += TT_THREADS) reinterpret_cast<uint4*>(S.ONES)[i] = make_uint4(0, 0, 0, 0);
    for (int i = tid; i < FD * FW; i += TT_THREADS) S.bias[i] = theta[b_off(i / FW) + i % FW];
    for (int i = tid; i <= FW; i += TT_THREADS) S.w5[i] = theta[W5_OFF + i];
    S.gw5w[warp][lane] = 0.f;
    if (tid == 0) {
        S.abort = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&S.mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&S.tmem)),
                     "r"(TT_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    __syncthreads();
    if (tid < TT) *reinterpret_cast<uint16_t*>(S.ONES + tp_off(0, tid)) = 0x3F80;   // bf16 1.0
    asm volatile("fence.proxy.async.shared::cta;");
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tm = S.tmem;
    const uint32_t row_acc = tm + ((uint32_t)(32 * q) << 16) + TT_COL_ACC + c0;
    const uint32_t a_addr = smem_addr(S.A), dzt_addr = smem_addr(S.DZT), ones_addr = smem_addr(S.ONES);
    const uint32_t ntiles = (batch + TT - 1) / TT;
    const float inv_b = 1.f / (float)batch;
    uint32_t ph = 0;
    bool first = true, stop = false;
    float loss_acc = 0.f, gb5_acc = 0.f;
    // bounded wait on the block's MMA barrier; every thread takes part
    auto sync_mma = [&]() {
        if (!mbar_wait(smem_addr(&S.mbar), ph)) S.abort = 1;
        ph ^= 1;
        asm volatile("tcgen05.fence::after_thread_sync;");
    };
    auto block_sync = [&]() {
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        return S.abort != 0;
    };
    // the batch entry of this thread's point in a tile, its position and target; issued one tile
    // ahead so that the random gathers are in flight while the previous tile computes
    uint32_t ne = 0;
    uint64_t ni = n;
    float nx[3] = {0.f, 0.f, 0.f}, ny = 0.f;
    auto prefetch = [&](uint32_t t) {
        ne = t * TT + p;
        ni = n;
        if (t < ntiles && ne < batch)
            ni = idx ? (uint64_t)idx[ne] : (uint64_t)(philox_x(step, ne, seed.x, seed.y) % (uint32_t)n);
        if (ni < n) {
            nx[0] = pts[stride * ni];
            nx[1] = pts[stride * ni + 1];
            nx[2] = pts[stride * ni + 2];
            ny = target[ni];
        }
    };
    prefetch(blockIdx.x);
    for (uint32_t tile = blockIdx.x; tile < ntiles && !stop; tile += gridDim.x) {
        const uint32_t e = ne;
        const uint64_t i = ni;
        float xt[3] = {0.f, 0.f, 0.f};
        if (i < n) {
            xt[0] = (nx[0] - B.cx) * B.inv_h;
            xt[1] = (nx[1] - B.cy) * B.inv_h;
            xt[2] = (nx[2] - B.cz) * B.inv_h;
        }
        const float y = i < n ? ny : 0.f;
        prefetch(tile + gridDim.x);
        uint32_t pk[TT_CW / 2];
        {
            float v[FW];
            features_fast(xt, v);
#pragma unroll
            for (int g = 0; g < TT_GROUPS; ++g)   // static indices keep v in registers
                if (g == c) {
#pragma unroll
                    for (int j = 0; j < TT_CW; j += 2) pk[j / 2] = pack_bf16(v[g * TT_CW + j], v[g * TT_CW + j + 1]);
                }
        }
        store_part(S.A, S.HT[0], p, c0, pk);
        uint32_t mask[FD];
        float zp = 0.f;
#pragma unroll
        for (int l = 0; l < FD; ++l) {
            tmem_st_cw(row_acc, S.bias + l * FW + c0);
            asm volatile("tcgen05.wait::st.sync.aligned;");
            if (block_sync()) {
                stop = true;
                break;
            }
            if (tid == 0) {
                const uint32_t w_addr = smem_addr(S.W[l]);
#pragma unroll
                for (int s = 0; s < 4; ++s)
                    umma_bf16(tm + TT_COL_ACC, umma_desc(a_addr + s * 4096, 2048, 128),
                              umma_desc(w_addr + s * 2048, 1024, 128), kIdescN64, 1u);
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&S.mbar)));
            }
            sync_mma();
            float z[TT_CW];
#pragma unroll
            for (int j = 0; j < TT_CW; j += 16) tmem_ld16(row_acc + j, z + j);
            asm volatile("tcgen05.wait::ld.sync.aligned;");
            uint32_t m = 0;
#pragma unroll
            for (int j = 0; j < TT_CW; j += 2) {
                pk[j / 2] = pack_bf16_relu(z[j], z[j + 1]);
                m |= (z[j] > 0.f ? 1u : 0u) << j;
                m |= (z[j + 1] > 0.f ? 1u : 0u) << (j + 1);
            }
            mask[l] = m;
            if (l + 1 < FD) {
                store_part(S.A, S.HT[l + 1], p, c0, pk);
            } else {
#pragma unroll
                for (int j = 0; j < TT_CW; j += 2) {
                    zp = fmaf(bf_lo(pk[j / 2]), S.w5[c0 + j], zp);
                    zp = fmaf(bf_hi(pk[j / 2]), S.w5[c0 + j + 1], zp);
                }
            }
        }
        if (stop) break;
        // output layer: both halves form z5 in the same order
        S.zpart[c][p] = zp;
        __syncthreads();
        float z5 = S.zpart[0][p];
#pragma unroll
        for (int g = 1; g < TT_GROUPS; ++g) z5 += S.zpart[g][p];
        z5 += S.w5[FW];
        const float r = e < batch ? softplusf(z5) - y : 0.f;
        const float dz5 = 2.f * r * inv_b * sigmoidf_(z5);
        if (c == 0) {
            loss_acc = fmaf(r, r, loss_acc);
            gb5_acc += dz5;
        }
        {
            float gv[TT_CW];
#pragma unroll
            for (int j = 0; j < TT_CW; j += 2) {
                gv[j] = dz5 * bf_lo(pk[j / 2]);
                gv[j + 1] = dz5 * bf_hi(pk[j / 2]);
            }
            S.gw5w[warp][lane] += warp_transpose_sum(gv);
        }
        // dZ_3 = bf16(dz5 w5 . [z_3 > 0])
#pragma unroll
        for (int j = 0; j < TT_CW; j += 2) {
            const float d0 = (mask[FD - 1] >> j) & 1u ? dz5 * S.w5[c0 + j] : 0.f;
            const float d1 = (mask[FD - 1] >> (j + 1)) & 1u ? dz5 * S.w5[c0 + j + 1] : 0.f;
            pk[j / 2] = pack_bf16(d0, d1);
        }
        store_part(S.A, S.DZT, p, c0, pk);
#pragma unroll
        for (int l = FD - 1; l >= 0; --l) {
            if (block_sync()) {
                stop = true;
                break;
            }
            if (tid == 0) {
                const uint32_t ht_addr = smem_addr(S.HT[l]);
#pragma unroll
                for (int s = 0; s < 8; ++s) {
                    const uint32_t acc = (!first || s > 0) ? 1u : 0u;
                    const uint64_t da = umma_desc(dzt_addr + s * 2 * T_LBO, T_LBO, T_SBO);
                    umma_bf16(tm + TT_COL_GW + 64 * l, da, umma_desc(ht_addr + s * 2 * T_LBO, T_LBO, T_SBO),
                              kIdescN64, acc);
                    umma_bf16(tm + TT_COL_GB + 16 * l, da, umma_desc(ones_addr + s * 2 * T_LBO, T_LBO, T_SBO),
                              kIdescN16, acc);
                }
                if (l > 0) {
                    const uint32_t wt_addr = smem_addr(S.WT[l]);
#pragma unroll
                    for (int s = 0; s < 4; ++s)
                        umma_bf16(tm + TT_COL_ACC, umma_desc(a_addr + s * 4096, 2048, 128),
                                  umma_desc(wt_addr + s * 2048, 1024, 128), kIdescN64, s > 0 ? 1u : 0u);
                }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_addr(&S.mbar)));
            }
            sync_mma();
            if (l > 0) {
                // dZ_{l-1} = bf16(dH_l . [z_{l-1} > 0])
                float dh[TT_CW];
#pragma unroll
                for (int j = 0; j < TT_CW; j += 16) tmem_ld16(row_acc + j, dh + j);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
                for (int j = 0; j < TT_CW; j += 2) {
                    const float d0 = (mask[l - 1] >> j) & 1u ? dh[j] : 0.f;
                    const float d1 = (mask[l - 1] >> (j + 1)) & 1u ? dh[j + 1] : 0.f;
                    pk[j / 2] = pack_bf16(d0, d1);
                }
                store_part(S.A, S.DZT, p, c0, pk);
            }
        }
        first = false;
    }
    // the block's sums into its slice of the partial-sum buffer
    if (c == 0) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            loss_acc += __shfl_xor_sync(0xffffffffu, loss_acc, o);
            gb5_acc += __shfl_xor_sync(0xffffffffu, gb5_acc, o);
        }
        if (lane == 0) {
            S.lossw[q] = loss_acc;
            S.gb5w[q] = gb5_acc;
        }
    }
    const bool ok = !block_sync() && !stop;
    float* P = partial + (size_t)blockIdx.x * NPAR_PAD;
    if (ok && q < 2) {
        // accumulator rows 0..63 are the outputs of each layer
#pragma unroll 1
        for (int l = 0; l < FD; ++l) {
            float v[TT_CW];
            const uint32_t ra = tm + ((uint32_t)(32 * q) << 16) + TT_COL_GW + 64 * l + c0;
            if (first) {
#pragma unroll
                for (int j = 0; j < TT_CW; ++j) v[j] = 0.f;
            } else {
#pragma unroll
                for (int j = 0; j < TT_CW; j += 16) tmem_ld16(ra + j, v + j);
                asm volatile("tcgen05.wait::ld.sync.aligned;");
            }
            float4* dst = reinterpret_cast<float4*>(P + w_off(l) + p * FW + c0);
#pragma unroll
            for (int j = 0; j < TT_CW / 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
            if (c == 0) {
                float gb[16];
                if (first) gb[0] = 0.f;
                else {
                    tmem_ld16(tm + ((uint32_t)(32 * q) << 16) + TT_COL_GB + 16 * l, gb);
                    asm volatile("tcgen05.wait::ld.sync.aligned;");
                }
                P[b_off(l) + p] = gb[0];
            }
        }
    }
    if (ok) {
        // warps in a fixed order: the block's sums do not depend on scheduling
        if (tid < FW) {
            const int g = tid / TT_CW, j = tid % TT_CW;   // column group and column within it
            P[W5_OFF + tid] = ((S.gw5w[4 * g][j] + S.gw5w[4 * g + 1][j]) + S.gw5w[4 * g + 2][j]) + S.gw5w[4 * g + 3][j];
        }
        if (tid == 0) {
            P[B5_OFF] = ((S.gb5w[0] + S.gb5w[1]) + S.gb5w[2]) + S.gb5w[3];
            P[NPAR] = ((S.lossw[0] + S.lossw[1]) + S.lossw[2]) + S.lossw[3];   // the padding slot
        }
    }
    if (S.abort && tid == 0) atomicCAS(err, 0, GM_DEV_WAIT_TIMEOUT);
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(TT_TMEM_COLS));
}

// Gradient = the fixed-order sum of the blocks' partial sums; then either that gradient is
// stored (grad_out) or one Adam step is taken (and the bf16 copies of the weights refreshed).
// A block of 8 warps handles 32 consecutive entries: warp w adds the slices b = w, w + 8, ... in
// order, then the eight warp sums are added in warp order. Entry NPAR of every slice (padding)
// holds a block's squared-error sum; its total goes to loss_sum.
constexpr int UPD_WARPS = 8;
__global__ void __launch_bounds__(32 * UPD_WARPS) k_field_update(
    const float* __restrict__ partial, int nblk, float* __restrict__ loss_sum, float* __restrict__ grad_out,
    float* __restrict__ theta, float* __restrict__ m, float* __restrict__ v, float lr, float bc1, float bc2,
    __nv_bfloat16* __restrict__ wbf, __nv_bfloat16* __restrict__ wtbf) {
    __shared__ float red[UPD_WARPS][32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * 32 + lane;
    float g = 0.f;
    if (i <= NPAR) {
#pragma unroll 4
        for (int b = w; b < nblk; b += UPD_WARPS) g += partial[(size_t)b * NPAR_PAD + i];
    }
    red[w][lane] = g;
    __syncthreads();
    if (w != 0 || i > NPAR) return;
    g = red[0][lane];
#pragma unroll
    for (int k = 1; k < UPD_WARPS; ++k) g += red[k][lane];
    if (i == NPAR) {
        *loss_sum = g;
        return;
    }
    if (grad_out) {
        grad_out[i] = g;
        return;
    }
    const float mi = 0.9f * m[i] + 0.1f * g;
    const float vi = 0.999f * v[i] + 0.001f * g * g;
    m[i] = mi;
    v[i] = vi;
    const float th = theta[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + 1e-8f);
    theta[i] = th;
    const int l = i / (FW * FW + FW), o = i % (FW * FW + FW);
    if (l < FD && o < FW * FW) {
        const int r = o / FW, cc = o % FW;
        const __nv_bfloat16 b = __float2bfloat16_rn(th);
        wbf[l * FW * FW + r * FW + cc] = b;
        wtbf[l * FW * FW + cc * FW + r] = b;
    }
}

}  // namespace

struct gm_field {
    gm_ctx* ctx = nullptr;
    FieldBox box{};
    float box_lo[3], box_hi[3];
    float *theta = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr, *loss = nullptr;
    __nv_bfloat16 *wbf = nullptr, *wtbf = nullptr;
    uint32_t t = 0;   // Adam steps taken
    float last_loss = 0.f;
    float train_ms = 0.f;
    int32_t query_kernel = GM_FIELD_QUERY_TCGEN05;
    int32_t train_kernel = GM_FIELD_QUERY_TCGEN05;
    float* partial = nullptr;   // per-block gradient sums of the tensor-core training kernel
    int nblk = 0;               // blocks of the last tensor-core gradient launch
};

static const size_t kTrainSmem = sizeof(TrainSmem);
static const size_t kTrainTcSmem = sizeof(TrainTcSmem);
static const int kUpdateGrid = (NPAR + 1 + 31) / 32;   // entries 0..NPAR (the last is the loss)

extern "C" gm_status gm_field_create(gm_ctx* ctx, const float* box_lo, const float* box_hi, const float* init_params,
                                     gm_stream stream, gm_field** out) {
    if (!ctx || !box_lo || !box_hi || !init_params || !out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_create: null argument");
    *out = nullptr;
    float ext = 0.f;
    for (int k = 0; k < 3; ++k) {
        if (!std::isfinite(box_lo[k]) || !std::isfinite(box_hi[k]) || box_hi[k] < box_lo[k])
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_create: invalid box");
        ext = std::max(ext, box_hi[k] - box_lo[k]);
    }
    if (!(ext > 0.f)) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_create: empty box");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    gm_field* f = new gm_field();
    f->ctx = ctx;
    for (int k = 0; k < 3; ++k) {
        f->box_lo[k] = box_lo[k];
        f->box_hi[k] = box_hi[k];
    }
    f->box = FieldBox{0.5f * (box_lo[0] + box_hi[0]), 0.5f * (box_lo[1] + box_hi[1]), 0.5f * (box_lo[2] + box_hi[2]),
                      2.f / ext};
    gm_status st;
    auto fail = [&](gm_status e) {
        gm_field_free(f);
        return e;
    };
    if ((st = gm_alloc((void**)&f->theta, sizeof(float) * NPAR, s)) != GM_OK ||
        (st = gm_alloc((void**)&f->m, sizeof(float) * NPAR, s)) != GM_OK ||
        (st = gm_alloc((void**)&f->v, sizeof(float) * NPAR, s)) != GM_OK ||
        (st = gm_alloc((void**)&f->grad, sizeof(float) * NPAR, s)) != GM_OK ||
        (st = gm_alloc((void**)&f->loss, sizeof(float) * 4, s)) != GM_OK ||
        (st = gm_alloc((void**)&f->wbf, sizeof(__nv_bfloat16) * FD * FW * FW, s)) != GM_OK ||
        (st = gm_alloc((void**)&f->wtbf, sizeof(__nv_bfloat16) * FD * FW * FW, s)) != GM_OK ||
        (st = gm_alloc((void**)&f->partial, sizeof(float) * NPAR_PAD * (size_t)std::max(1, ctx->n_sm), s)) != GM_OK)
        return fail(st);
    cudaError_t e = cudaMemcpyAsync(f->theta, init_params, sizeof(float) * NPAR, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->m, 0, sizeof(float) * NPAR, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->v, 0, sizeof(float) * NPAR, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(f->grad, 0, sizeof(float) * NPAR, s);
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_field_create"));
    k_field_cast<<<gm_div_up(FD * FW * FW, 256), 256, 0, s>>>(f->theta, f->wbf, f->wtbf);
    ctx->launches += 1;
    e = cudaFuncSetAttribute(k_field_train, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_field_train_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTrainTcSmem);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_field_create"));
    *out = f;
    return GM_OK;
}

static gm_status field_grad(gm_field* f, const float* pts, int stride, const float* target, uint64_t n,
                            const uint32_t* idx, uint32_t batch, uint32_t step, uint64_t seed, cudaStream_t s) {
    if (f->train_kernel == GM_FIELD_QUERY_TCGEN05) {   // the update kernel writes the loss
        const uint32_t ntiles = (batch + TT - 1) / TT;
        const int grid = (int)std::min<uint32_t>((uint32_t)std::max(1, f->ctx->n_sm), ntiles);
        k_field_train_tc<<<grid, TT_THREADS, kTrainTcSmem, s>>>(
            pts, stride, target, n, idx, batch, step, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), f->box,
            f->wbf, f->wtbf, f->theta, f->partial, f->ctx->dev_err);
        f->nblk = grid;
        f->ctx->launches += 1;
        GM_TRY_CUDA(cudaGetLastError());
        return GM_OK;
    }
    GM_TRY_CUDA(cudaMemsetAsync(f->loss, 0, sizeof(float), s));
    k_field_train<<<gm_div_up(batch, TRAIN_PTS), 256, kTrainSmem, s>>>(
        pts, stride, target, n, idx, batch, step, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)), f->box, f->wbf,
        f->wtbf, f->theta, f->grad, f->loss);
    f->ctx->launches += 1;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

static gm_status field_adam(gm_field* f, float lr, cudaStream_t s) {
    f->t += 1;
    const float bc1 = (float)(1.0 - std::pow(0.9, (double)f->t));
    const float bc2 = (float)(1.0 - std::pow(0.999, (double)f->t));
    if (f->train_kernel == GM_FIELD_QUERY_TCGEN05)
        k_field_update<<<kUpdateGrid, 32 * UPD_WARPS, 0, s>>>(f->partial, f->nblk, f->loss, nullptr, f->theta, f->m,
                                                               f->v, lr, bc1, bc2, f->wbf, f->wtbf);
    else
        k_field_adam<<<gm_div_up(NPAR, 256), 256, 0, s>>>(f->theta, f->m, f->v, f->grad, lr, bc1, bc2, f->wbf,
                                                          f->wtbf);
    f->ctx->launches += 1;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

extern "C" gm_status gm_field_loss_grad(gm_field* f, const float* xyz, const float* target, uint64_t n,
                                        const uint32_t* batch_idx, uint32_t batch, float* grad_out, float* loss_out,
                                        gm_stream stream) {
    if (!f || !xyz || !target || !batch_idx || batch == 0 || n == 0)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_loss_grad: null argument or empty batch");
    if (!gm_is_device_ptr(xyz) || !gm_is_device_ptr(target) || !gm_is_device_ptr(batch_idx))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_loss_grad: inputs must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY(field_grad(f, xyz, 3, target, n, batch_idx, batch, 0, 0, s));
    if (f->train_kernel == GM_FIELD_QUERY_TCGEN05) {
        k_field_update<<<kUpdateGrid, 32 * UPD_WARPS, 0, s>>>(f->partial, f->nblk, f->loss, f->grad, nullptr,
                                                               nullptr, nullptr, 0.f, 1.f, 1.f, nullptr, nullptr);
        f->ctx->launches += 1;
        GM_TRY_CUDA(cudaGetLastError());
    }
    if (grad_out) GM_TRY(gm_copy_out(grad_out, f->grad, sizeof(float) * NPAR, s));
    if (loss_out) {
        float l = 0.f;
        GM_TRY(gm_copy_out(&l, f->loss, sizeof(float), s));
        *loss_out = l / (float)batch;
    }
    GM_TRY_CUDA(cudaMemsetAsync(f->grad, 0, sizeof(float) * NPAR, s));
    return GM_OK;
}

extern "C" gm_status gm_field_step(gm_field* f, const float* xyz, const float* target, uint64_t n,
                                   const uint32_t* batch_idx, uint32_t batch, float lr, gm_stream stream) {
    if (!f || !xyz || !target || batch == 0 || n == 0) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_step: bad argument");
    if (!gm_is_device_ptr(xyz) || !gm_is_device_ptr(target) || (batch_idx && !gm_is_device_ptr(batch_idx)))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_step: inputs must be device memory");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY(field_grad(f, xyz, 3, target, n, batch_idx, batch, f->t, 0, s));
    return field_adam(f, lr, s);
}

extern "C" gm_status gm_field_train(gm_field* f, const gm_samples* sm, const gm_map* mp, uint32_t window,
                                    const gm_field_cfg* cfg, gm_stream stream, float* final_loss) {
    if (!f || !sm || !mp || !cfg) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_train: null argument");
    if (mp->ns != sm->n || window >= mp->W) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_train: map does not match samples");
    if (cfg->batch == 0 || cfg->steps == 0 || !(cfg->lr > 0.f) || !(cfg->lr_min >= 0.f) || sm->n == 0)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_train: empty configuration");
    cudaStream_t s = (cudaStream_t)stream;
    cudaEvent_t e0, e1;
    GM_TRY_CUDA(cudaEventCreate(&e0));
    GM_TRY_CUDA(cudaEventCreate(&e1));
    cudaEventRecord(e0, s);
    const float* targets = mp->values + (size_t)window * mp->ns;
    gm_status st = GM_OK;
    for (uint32_t k = 0; k < cfg->steps && st == GM_OK; ++k) {
        const double lr = cfg->steps > 1 ? cfg->lr_min + 0.5 * (cfg->lr - cfg->lr_min) *
                                                             (1.0 + std::cos(3.14159265358979323846 * k / (cfg->steps - 1)))
                                         : cfg->lr;
        st = field_grad(f, reinterpret_cast<const float*>(sm->pos), 4, targets, sm->n, nullptr, cfg->batch, f->t,
                        cfg->seed, s);
        if (st == GM_OK) st = field_adam(f, (float)lr, s);
    }
    cudaEventRecord(e1, s);
    if (st == GM_OK) {
        float l = 0.f;
        st = gm_copy_out(&l, f->loss, sizeof(float), s);
        f->last_loss = l / (float)cfg->batch;
        cudaEventElapsedTime(&f->train_ms, e0, e1);
        if (final_loss) *final_loss = f->last_loss;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return st;
}

extern "C" gm_status gm_field_query(const gm_field* f, const float* xyz, uint64_t n, float* out, gm_stream stream) {
    if (!f || (n > 0 && (!xyz || !out))) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_query: null argument");
    if (n == 0) return GM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    void* dx = nullptr;
    bool ox = false;
    GM_TRY(gm_stage_to_device(xyz, sizeof(float) * 3 * n, s, &dx, &ox));
    const bool dev_out = gm_is_device_ptr(out);
    float* dout = out;
    gm_status st = GM_OK;
    if (!dev_out) st = gm_alloc((void**)&dout, sizeof(float) * n, s);
    if (st == GM_OK && f->query_kernel == GM_FIELD_QUERY_TCGEN05) {
        static int configured_device = -1;   // the attribute is per device and per function
        const int smem = (int)sizeof(QuerySmem);
        if (configured_device != f->ctx->device) {
            cudaError_t e = cudaFuncSetAttribute(k_field_query_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) st = gm_cuda_error(e, "gm_field_query (shared memory)");
            else configured_device = f->ctx->device;
        }
        // blocks per SM from the shared memory each one holds (the occupancy query reports one block
        // for this kernel; the hardware runs as many as their shared memory and tensor-memory
        // columns allow, here 3 x 128 of 512 columns)
        int per_sm = 1;
        if (st == GM_OK) {
            int smem_sm = 0;
            cudaError_t e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, f->ctx->device);
            if (e != cudaSuccess) st = gm_cuda_error(e, "gm_field_query (shared memory per SM)");
            else per_sm = std::max(1, std::min(8, smem_sm / (smem + 1024)));
        }
        if (st == GM_OK) {
            const uint64_t ntiles = (n + TQ - 1) / TQ;
            const uint32_t grid = (uint32_t)std::min<uint64_t>(
                (ntiles + 1) / 2, (uint64_t)f->ctx->n_sm * (uint64_t)std::max(1, per_sm));
            const int bulk = (reinterpret_cast<uintptr_t>(dx) % 16) == 0;
            k_field_query_tc<<<grid, TQ_THREADS, smem, s>>>((const float*)dx, n, f->wbf, f->theta, f->box, bulk,
                                                            dout, f->ctx->dev_err);
            f->ctx->launches += 1;
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) st = gm_cuda_error(e, "gm_field_query");
        }
        if (!dev_out) {
            if (st == GM_OK) st = gm_copy_out(out, dout, sizeof(float) * n, s);
            cudaFreeAsync(dout, s);
        }
    } else if (st == GM_OK) {
        const uint64_t groups = (n + 15) / 16;
        const uint32_t grid = (uint32_t)std::min<uint64_t>((groups + 7) / 8, (uint64_t)f->ctx->n_sm * 8);
        k_field_query<<<grid, 256, 0, s>>>((const float*)dx, n, f->wbf, f->theta, f->box, dout);
        f->ctx->launches += 1;
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = gm_cuda_error(e, "gm_field_query");
        if (!dev_out) {
            if (st == GM_OK) st = gm_copy_out(out, dout, sizeof(float) * n, s);
            cudaFreeAsync(dout, s);
        }
    }
    if (ox) cudaFreeAsync(dx, s);
    return st;
}

// One block waits, with the field kernels' bounded wait, on an mbarrier that nothing completes (no
// thread arrives, no copy is issued): the wait gives up after `iters` polls and the block records
// the timeout in the error word, as the field kernels do.
__global__ void k_wait_timeout(uint32_t iters, int* __restrict__ err) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0)
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar)), "r"(1u) : "memory");
    __syncthreads();
    const bool ok = mbar_wait_n(smem_addr(&bar), 0u, iters);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (!ok) atomicCAS(err, 0, GM_DEV_WAIT_TIMEOUT);
        asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(smem_addr(&bar)) : "memory");
    }
}

extern "C" gm_status gm_debug_wait_timeout(gm_ctx* ctx, uint32_t iterations, gm_stream stream) {
    if (!ctx) return gm_set_error(GM_ERR_INVALID_ARG, "gm_debug_wait_timeout: null context");
    if (iterations == 0 || iterations > (1u << 16))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_debug_wait_timeout: iterations must be in [1, 2^16]");
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    k_wait_timeout<<<1, 32, 0, (cudaStream_t)stream>>>(iterations, ctx->dev_err);
    ctx->launches += 1;
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

extern "C" gm_status gm_field_get_state(const gm_field* f, float* theta, float* m, float* v, uint32_t* steps,
                                        gm_stream stream) {
    if (!f) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_get_state: null field");
    cudaStream_t s = (cudaStream_t)stream;
    if (theta) GM_TRY(gm_copy_out(theta, f->theta, sizeof(float) * NPAR, s));
    if (m) GM_TRY(gm_copy_out(m, f->m, sizeof(float) * NPAR, s));
    if (v) GM_TRY(gm_copy_out(v, f->v, sizeof(float) * NPAR, s));
    if (steps) *steps = f->t;
    return GM_OK;
}

extern "C" gm_status gm_field_set_state(gm_field* f, const float* theta, const float* m, const float* v,
                                        uint32_t steps, gm_stream stream) {
    if (!f || !theta || !m || !v) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_set_state: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    GM_TRY_CUDA(cudaMemcpyAsync(f->theta, theta, sizeof(float) * NPAR, cudaMemcpyDefault, s));
    GM_TRY_CUDA(cudaMemcpyAsync(f->m, m, sizeof(float) * NPAR, cudaMemcpyDefault, s));
    GM_TRY_CUDA(cudaMemcpyAsync(f->v, v, sizeof(float) * NPAR, cudaMemcpyDefault, s));
    // the bf16 copies the kernels read follow the restored parameters
    k_field_cast<<<gm_div_up(FD * FW * FW, 256), 256, 0, s>>>(f->theta, f->wbf, f->wtbf);
    f->ctx->launches += 1;
    GM_TRY_CUDA(cudaGetLastError());
    f->t = steps;
    return GM_OK;
}

extern "C" gm_status gm_field_query_kernel(gm_field* f, int32_t kernel) {
    if (!f) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_query_kernel: null field");
    if (kernel != GM_FIELD_QUERY_TCGEN05 && kernel != GM_FIELD_QUERY_MMA_SYNC)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_query_kernel: unknown kernel");
    f->query_kernel = kernel;
    return GM_OK;
}

extern "C" gm_status gm_field_train_kernel(gm_field* f, int32_t kernel) {
    if (!f) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_train_kernel: null field");
    if (kernel != GM_FIELD_QUERY_TCGEN05 && kernel != GM_FIELD_QUERY_MMA_SYNC)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_train_kernel: unknown kernel");
    f->train_kernel = kernel;
    return GM_OK;
}

extern "C" gm_status gm_field_params(const gm_field* f, float* out, gm_stream stream) {
    if (!f || !out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_params: null argument");
    return gm_copy_out(out, f->theta, sizeof(float) * NPAR, (cudaStream_t)stream);
}

extern "C" gm_status gm_field_info(const gm_field* f, uint32_t* n_params, uint32_t* steps_taken, float* last_loss,
                                   float* train_ms) {
    if (!f) return gm_set_error(GM_ERR_INVALID_ARG, "gm_field_info: null field");
    if (n_params) *n_params = NPAR;
    if (steps_taken) *steps_taken = f->t;
    if (last_loss) *last_loss = f->last_loss;
    if (train_ms) *train_ms = f->train_ms;
    return GM_OK;
}

extern "C" void gm_field_free(gm_field* f) {
    if (!f) return;
    cudaFree(f->theta);
    cudaFree(f->m);
    cudaFree(f->v);
    cudaFree(f->grad);
    cudaFree(f->loss);
    cudaFree(f->wbf);
    cudaFree(f->wtbf);
    cudaFree(f->partial);
    delete f;
}
