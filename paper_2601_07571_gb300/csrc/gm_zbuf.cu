// gm_zbuf.cu -- the paper's own occlusion path as CUDA kernels (Sections 3.2.2 and 3.3.2,
// Appendix A): per fixation a camera at the eye, the near-plane crop window of the 4 sigma cone,
// a software z-buffer of that window and the +-eps depth comparison in each sample's pixel.
//
// Stages, per chunk of fixations (sorted by window like the ray path):
//   k_zb_frustum   one thread per fixation, FP64: camera basis from the head's forward and up
//                  hints, the gaze in camera space, the exact crop window (tangent planes through
//                  the eye; Appendix A centres its window on the gaze point E, which is not the
//                  centre of an oblique conic section) and the pixel mapping
//   k_zb_cull      one thread per triangle, frusta staged in shared memory: a triangle is kept for
//                  a fixation unless all three vertices lie outside one frustum plane; survivors
//                  are appended as (fixation, triangle) pairs with one atomic per warp
//   k_zb_raster    one thread per pair: near-plane clipping, projection, point sampling at pixel
//                  centres with edge functions evaluated in a canonical vertex order (a shared
//                  edge gives exactly opposite values, no cracks), perspective-correct 1/w, and
//                  atomicMin of the linear depth w (positive floats order as their bits); pairs
//                  covering more than RASTER_THREAD_PIXELS pixels go to k_zb_raster_warp (one warp
//                  each, lanes over pixels), more than RASTER_WARP_PIXELS to k_zb_raster_big (one
//                  block each): lanes of a warp no longer wait for one lane's large triangle
//   k_zb_accumulate one thread per work-order sample over the chunk's fixations: the exact cone
//                  test and Gaussian of the ray path, visibility |w - zbuf| <= eps, compensated
//                  sums carried across chunks, per-window writes and maxima; optionally the exact
//                  ray test beside it, counting the pairs on which the two disagree
#include "gm_trace.cuh"

#include <algorithm>
#include <cmath>
#include <vector>

namespace {

constexpr int ZB_THREADS = 256;
constexpr int ZB_SMEM_FRUSTA = 64;            // frusta staged per pass of the cull kernel
constexpr int RASTER_THREAD_PIXELS = 64;      // larger pixel boxes go to the warp rasteriser,
constexpr int RASTER_WARP_PIXELS = 1024;      // and larger ones still to the block rasteriser
constexpr uint32_t ZB_EMPTY = 0xffffffffu;    // cleared z-buffer word (above every finite depth)
constexpr uint32_t NO_WINDOW = 0xffffffffu;

struct ZbFrustum {
    float e[3], rgt[3], up[3], fwd[3];
    float n, f;
    float sx, ox, sy, oy;   // pixel coordinates: u = sx x / w + ox, v = sy y / w + oy
    int ok;
    int pad;
};

struct PairFT {
    uint32_t fix, tri;
};

// ---- fixation prep (window keys, stable sort by window, packing) --------------------------
__global__ void k_zb_keys(const double* __restrict__ ts, const float* __restrict__ eye, const float* __restrict__ gaze,
                          const float* __restrict__ dur, uint32_t nf, double t_begin, double t_end, double window_s,
                          uint32_t W, uint32_t* __restrict__ keys, uint32_t* __restrict__ vals,
                          uint32_t* __restrict__ n_valid, int* __restrict__ err) {
    uint32_t f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    double t = ts[f];
    uint32_t key = W;
    if (t >= t_begin && t < t_end) {
        double w = window_s > 0.0 ? floor((t - t_begin) / window_s) : 0.0;
        if (w >= 0.0 && w < (double)W) key = (uint32_t)w;
    }
    float gx = gaze[3 * f], gy = gaze[3 * f + 1], gz = gaze[3 * f + 2];
    bool finite = isfinite(gx) && isfinite(gy) && isfinite(gz) && isfinite(eye[3 * f]) && isfinite(eye[3 * f + 1]) &&
                  isfinite(eye[3 * f + 2]) && isfinite(dur[f]) && (gx != 0.f || gy != 0.f || gz != 0.f);
    if (!finite || !(dur[f] >= 0.f) || isnan(t)) {
        atomicCAS(err, 0, 3);
        key = W;
    }
    keys[f] = key;
    vals[f] = f;
    if (key < W) atomicAdd(n_valid, 1u);
}

// Same packing as the ray path: (e, t * 1/(sigma sqrt(2 pi))), (r^, window bits).
__global__ void k_zb_pack(const uint32_t* __restrict__ keys, const uint32_t* __restrict__ vals,
                          const float* __restrict__ eye, const float* __restrict__ gaze, const float* __restrict__ dur,
                          uint32_t nf, float wnorm, float4* __restrict__ packed, uint32_t* __restrict__ orig) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nf) return;
    uint32_t f = vals[i];
    float rx = gaze[3 * f], ry = gaze[3 * f + 1], rz = gaze[3 * f + 2];
    float rn = __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry)), __fmul_rn(rz, rz)));
    packed[2 * i + 0] = make_float4(eye[3 * f], eye[3 * f + 1], eye[3 * f + 2], __fmul_rn(dur[f], wnorm));
    packed[2 * i + 1] = make_float4(__fdiv_rn(rx, rn), __fdiv_rn(ry, rn), __fdiv_rn(rz, rn), __uint_as_float(keys[i]));
    orig[i] = f;
}

// ---- frustum (FP64) ------------------------------------------------------------------------
__device__ __forceinline__ void d_cross(const double a[3], const double b[3], double o[3]) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
__device__ __forceinline__ double d_dot(const double a[3], const double b[3]) {
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}
__device__ __forceinline__ bool d_unit(double a[3]) {
    const double l = sqrt(d_dot(a, a));
    if (!(l > 0.0) || !isfinite(l)) return false;
    a[0] /= l;
    a[1] /= l;
    a[2] /= l;
    return true;
}

// Fixation k of the list (orig[k] in the input arrays when orig is given): camera basis
// fwd = unit(forward hint or gaze), right = unit(fwd x up hint) (world z, then x, when the hint
// is parallel), up = right x fwd; gaze rc in camera space (x right, y up, z back); crop window
// on z = -n bounded by the planes through the eye tangent to the cone of half-angle
// phi = atan(cutoff tan theta): (rc_z^2 - s^2) c^2 + 2 rc_q rc_z c + rc_q^2 - s^2 = 0, bound = n c.
// A cone reaching behind the camera (rc_z >= 0 or rc_z^2 <= s^2) has no window: ok = 0.
__global__ void k_zb_frustum(uint32_t nfix, const uint32_t* __restrict__ orig, const float* __restrict__ eye,
                             const float* __restrict__ gaze, const float* __restrict__ cam_fwd,
                             const float* __restrict__ cam_up, double theta, double cutoff, double near_m,
                             double far_m, uint32_t res, ZbFrustum* __restrict__ out, double* __restrict__ crop,
                             unsigned long long* __restrict__ skipped) {
    uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nfix) return;
    const uint32_t i = orig ? orig[k] : k;
    ZbFrustum F;
    F.ok = 0;
    F.pad = 0;
    double f[3], u[3], g[3] = {gaze[3 * i], gaze[3 * i + 1], gaze[3 * i + 2]};
    for (int c = 0; c < 3; ++c) {
        f[c] = cam_fwd ? (double)cam_fwd[3 * i + c] : g[c];
        u[c] = cam_up ? (double)cam_up[3 * i + c] : (c == 1 ? 1.0 : 0.0);
    }
    double r[3], bnd[4] = {NAN, NAN, NAN, NAN};
    bool ok = d_unit(f) && d_unit(g);
    if (ok) {
        d_cross(f, u, r);
        const double lu = sqrt(d_dot(u, u));
        if (!(sqrt(d_dot(r, r)) > 1e-6 * lu)) {
            const double z[3] = {0.0, 0.0, 1.0};
            d_cross(f, z, r);
            if (!(sqrt(d_dot(r, r)) > 1e-6)) {
                const double x[3] = {1.0, 0.0, 0.0};
                d_cross(f, x, r);
            }
        }
        d_unit(r);
        d_cross(r, f, u);
        double rc[3] = {d_dot(g, r), d_dot(g, u), -d_dot(g, f)};
        d_unit(rc);
        const double phi = atan(cutoff * tan(theta));
        const double s = sin(phi);
        const double A = rc[2] * rc[2] - s * s;
        ok = rc[2] < 0.0 && A > 0.0;
        if (ok) {
            for (int q = 0; q < 2; ++q) {
                const double disc = s * sqrt(rc[q] * rc[q] + rc[2] * rc[2] - s * s);
                const double c1 = (-rc[q] * rc[2] - disc) / A, c2 = (-rc[q] * rc[2] + disc) / A;
                bnd[2 * q] = near_m * fmin(c1, c2);
                bnd[2 * q + 1] = near_m * fmax(c1, c2);
            }
            ok = bnd[1] > bnd[0] && bnd[3] > bnd[2];
        }
        for (int c = 0; c < 3; ++c) {
            F.e[c] = eye[3 * i + c];
            F.rgt[c] = (float)r[c];
            F.up[c] = (float)u[c];
            F.fwd[c] = (float)f[c];
        }
    }
    F.n = (float)near_m;
    F.f = (float)far_m;
    if (ok) {
        const double wx = bnd[1] - bnd[0], wy = bnd[3] - bnd[2];
        F.sx = (float)(near_m * res / wx);
        F.ox = (float)(-bnd[0] * res / wx);
        F.sy = (float)(near_m * res / wy);
        F.oy = (float)(-bnd[2] * res / wy);
        F.ok = 1;
    } else {
        F.sx = F.ox = F.sy = F.oy = 0.f;
        if (skipped) atomicAdd(skipped, 1ull);
    }
    out[k] = F;
    if (crop)
        for (int c = 0; c < 4; ++c) crop[4 * k + c] = ok ? bnd[c] : NAN;
}

__device__ __forceinline__ void to_camera(const ZbFrustum& F, float px, float py, float pz, float& x, float& y,
                                          float& w) {
    const float dx = px - F.e[0], dy = py - F.e[1], dz = pz - F.e[2];
    x = fmaf(dx, F.rgt[0], fmaf(dy, F.rgt[1], dz * F.rgt[2]));
    y = fmaf(dx, F.up[0], fmaf(dy, F.up[1], dz * F.up[2]));
    w = fmaf(dx, F.fwd[0], fmaf(dy, F.fwd[1], dz * F.fwd[2]));
}

// ---- cull: (fixation, triangle) pairs whose triangle may meet the fixation's frustum ---------
// Frustum planes as linear forms through the eye (u in [-1, res + 1] pixels: one pixel of slack),
// plus near/far with 1e-5 relative slack. FP32; the slack keeps it conservative.
// True when a sphere (centre c, radius r) lies wholly outside a frustum: beyond its near or far
// plane or one of its four side planes (these pass through the eye; unit normals in camera
// coordinates from the pixel mapping with one pixel of slack). The slack covers FP32 rounding.
__device__ __forceinline__ bool sphere_outside(const ZbFrustum& F, float cx, float cy, float cz, float r, float R) {
    float xc, yc, wc;
    to_camera(F, cx, cy, cz, xc, yc, wc);
    const float slack = r + 1e-4f * (fabsf(xc) + fabsf(yc) + fabsf(wc) + r);
    const float l0 = F.ox + 1.f, l1 = R + 1.f - F.ox, b0 = F.oy + 1.f, b1 = R + 1.f - F.oy;
    return wc < F.n - slack || wc > F.f + slack ||
           fmaf(F.sx, xc, l0 * wc) < -slack * sqrtf(fmaf(F.sx, F.sx, l0 * l0)) ||
           fmaf(-F.sx, xc, l1 * wc) < -slack * sqrtf(fmaf(F.sx, F.sx, l1 * l1)) ||
           fmaf(F.sy, yc, b0 * wc) < -slack * sqrtf(fmaf(F.sy, F.sy, b0 * b0)) ||
           fmaf(-F.sy, yc, b1 * wc) < -slack * sqrtf(fmaf(F.sy, F.sy, b1 * b1));
}

__global__ void __launch_bounds__(ZB_THREADS) k_zb_cull(const float4* __restrict__ tris, uint32_t nt,
                                                        const ZbFrustum* __restrict__ frusta, uint32_t nfix,
                                                        uint32_t res, PairFT* __restrict__ pairs, uint64_t cap,
                                                        unsigned long long* __restrict__ count) {
    __shared__ ZbFrustum sF[ZB_SMEM_FRUSTA];
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < nt;
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f), b = a, c = a;
    if (valid) {   // leaf order: a warp's 32 triangles are neighbours in space; v0.w = triangle id
        a = tris[3 * t];
        b = tris[3 * t + 1];
        c = tris[3 * t + 2];
    }
    const uint32_t id = __float_as_uint(a.w);
    const int lane = threadIdx.x & 31;
    const float R = (float)res;
    // the warp's triangles in one sphere (box centre, half diagonal), tested against each frustum
    // before the per-triangle tests
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (valid) {
        lo[0] = fminf(fminf(a.x, b.x), c.x);
        lo[1] = fminf(fminf(a.y, b.y), c.y);
        lo[2] = fminf(fminf(a.z, b.z), c.z);
        hi[0] = fmaxf(fmaxf(a.x, b.x), c.x);
        hi[1] = fmaxf(fmaxf(a.y, b.y), c.y);
        hi[2] = fmaxf(fmaxf(a.z, b.z), c.z);
    }
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[q] = fminf(lo[q], __shfl_xor_sync(0xffffffffu, lo[q], o));
            hi[q] = fmaxf(hi[q], __shfl_xor_sync(0xffffffffu, hi[q], o));
        }
    }
    const bool wbox = lo[0] <= hi[0];
    const float wx = 0.5f * (lo[0] + hi[0]), wy = 0.5f * (lo[1] + hi[1]), wz = 0.5f * (lo[2] + hi[2]);
    const float wR = wbox ? 0.5f * sqrtf((hi[0] - lo[0]) * (hi[0] - lo[0]) + (hi[1] - lo[1]) * (hi[1] - lo[1]) +
                                         (hi[2] - lo[2]) * (hi[2] - lo[2])) * 1.0001f
                          : 0.f;
    // the block's 256 triangles (also neighbours in leaf order) in one sphere: a frustum that
    // misses it is skipped by every warp of the block without its own sphere test
    __shared__ float sBox[ZB_THREADS / 32][6];
    __shared__ float4 sBlk;
    __shared__ unsigned sMask[ZB_SMEM_FRUSTA / 32];
    const int warp = threadIdx.x >> 5;
    if (lane == 0) {
        sBox[warp][0] = lo[0], sBox[warp][1] = lo[1], sBox[warp][2] = lo[2];
        sBox[warp][3] = hi[0], sBox[warp][4] = hi[1], sBox[warp][5] = hi[2];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float bl[3] = {INFINITY, INFINITY, INFINITY}, bh[3] = {-INFINITY, -INFINITY, -INFINITY};
        for (int w = 0; w < ZB_THREADS / 32; ++w)
            for (int q = 0; q < 3; ++q) {
                bl[q] = fminf(bl[q], sBox[w][q]);
                bh[q] = fmaxf(bh[q], sBox[w][3 + q]);
            }
        sBlk = bl[0] <= bh[0]
                   ? make_float4(0.5f * (bl[0] + bh[0]), 0.5f * (bl[1] + bh[1]), 0.5f * (bl[2] + bh[2]),
                                 0.5f * sqrtf((bh[0] - bl[0]) * (bh[0] - bl[0]) + (bh[1] - bl[1]) * (bh[1] - bl[1]) +
                                              (bh[2] - bl[2]) * (bh[2] - bl[2])) * 1.0001f)
                   : make_float4(0.f, 0.f, 0.f, -1.f);
    }
    // blockIdx.y picks a group of fixations (one shared-memory load of their frusta); the blocks of
    // one group run together, so the pairs they emit -- and the raster's atomics -- stay on a few
    // z-buffers that fit in L2
    for (uint32_t f0 = blockIdx.y * ZB_SMEM_FRUSTA; f0 < nfix; f0 += gridDim.y * ZB_SMEM_FRUSTA) {
        const uint32_t m = min((uint32_t)ZB_SMEM_FRUSTA, nfix - f0);
        __syncthreads();
        for (uint32_t k = threadIdx.x; k < m; k += blockDim.x) sF[k] = frusta[f0 + k];
        __syncthreads();
        if (threadIdx.x < ZB_SMEM_FRUSTA) {   // whole warps: ZB_SMEM_FRUSTA is a multiple of 32
            const uint32_t k = threadIdx.x;
            const float4 bs = sBlk;
            const bool reach = k < m && sF[k].ok && bs.w >= 0.f && !sphere_outside(sF[k], bs.x, bs.y, bs.z, bs.w, R);
            const unsigned bits = __ballot_sync(0xffffffffu, reach);
            if (lane == 0) sMask[k >> 5] = bits;
        }
        __syncthreads();
        for (uint32_t k = 0; k < m; ++k) {
            if (!((sMask[k >> 5] >> (k & 31)) & 1u)) continue;
            const ZbFrustum& F = sF[k];
            if (!wbox || sphere_outside(F, wx, wy, wz, wR, R)) continue;
            bool keep = false;
            if (valid) {
                float x[3], y[3], w[3];
                to_camera(F, a.x, a.y, a.z, x[0], y[0], w[0]);
                to_camera(F, b.x, b.y, b.z, x[1], y[1], w[1]);
                to_camera(F, c.x, c.y, c.z, x[2], y[2], w[2]);
                int o0 = 0, o1 = 0, o2 = 0, o3 = 0, o4 = 0, o5 = 0;
#pragma unroll
                for (int v = 0; v < 3; ++v) {
                    const float U = fmaf(F.sx, x[v], F.ox * w[v]), V = fmaf(F.sy, y[v], F.oy * w[v]);
                    o0 += U < -w[v];
                    o1 += U > (R + 1.f) * w[v];
                    o2 += V < -w[v];
                    o3 += V > (R + 1.f) * w[v];
                    o4 += w[v] < F.n * (1.f - 1e-5f);
                    o5 += w[v] > F.f * (1.f + 1e-5f);
                }
                keep = o0 < 3 && o1 < 3 && o2 < 3 && o3 < 3 && o4 < 3 && o5 < 3;
            }
            const unsigned msk = __ballot_sync(0xffffffffu, keep);
            if (msk) {
                unsigned long long base = 0;
                if (lane == __ffs(msk) - 1) base = atomicAdd(count, (unsigned long long)__popc(msk));
                base = __shfl_sync(0xffffffffu, base, __ffs(msk) - 1);
                if (keep) {
                    const unsigned long long q = base + __popc(msk & gm_lanemask_lt());
                    if (q < cap) pairs[q] = PairFT{f0 + k, id};
                }
            }
        }
    }
}

// ---- raster --------------------------------------------------------------------------------
struct ClipPoly {
    float u[4], v[4], iw[4];
    int n;
};

// Camera-space triangle clipped to w >= n (Sutherland-Hodgman against one plane), projected to
// pixel coordinates with 1/w per vertex.
__device__ __forceinline__ void clip_project(const ZbFrustum& F, float4 a, float4 b, float4 c, ClipPoly& P) {
    float x[3], y[3], w[3];
    to_camera(F, a.x, a.y, a.z, x[0], y[0], w[0]);
    to_camera(F, b.x, b.y, b.z, x[1], y[1], w[1]);
    to_camera(F, c.x, c.y, c.z, x[2], y[2], w[2]);
    float cx[4], cy[4], cw[4];
    int n = 0;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const int j = k == 2 ? 0 : k + 1;
        const bool ik = w[k] >= F.n, ij = w[j] >= F.n;
        if (ik) {
            cx[n] = x[k];
            cy[n] = y[k];
            cw[n] = w[k];
            ++n;
        }
        if (ik != ij) {
            const float s = (F.n - w[k]) / (w[j] - w[k]);
            cx[n] = fmaf(s, x[j] - x[k], x[k]);
            cy[n] = fmaf(s, y[j] - y[k], y[k]);
            cw[n] = F.n;
            ++n;
        }
    }
    P.n = n;
    for (int k = 0; k < n; ++k) {
        const float iw = 1.0f / cw[k];
        P.u[k] = fmaf(F.sx, cx[k] * iw, F.ox);
        P.v[k] = fmaf(F.sy, cy[k] * iw, F.oy);
        P.iw[k] = iw;
    }
}

// Edge function of p against the directed edge a -> b, evaluated with the endpoints in a
// canonical (lexicographic) order and the sign restored, so that the two triangles sharing an
// edge get exactly opposite values.
__device__ __forceinline__ float edge_fn(float ax, float ay, float bx, float by, float px, float py) {
    const bool swap = (bx < ax) || (bx == ax && by < ay);
    const float x0 = swap ? bx : ax, y0 = swap ? by : ay, x1 = swap ? ax : bx, y1 = swap ? ay : by;
    const float e = __fsub_rn(__fmul_rn(x1 - x0, py - y0), __fmul_rn(y1 - y0, px - x0));
    return swap ? -e : e;
}

__device__ __forceinline__ void poly_bbox(const ClipPoly& P, int res, int& x0, int& x1, int& y0, int& y1) {
    float umin = P.u[0], umax = P.u[0], vmin = P.v[0], vmax = P.v[0];
    for (int k = 1; k < P.n; ++k) {
        umin = fminf(umin, P.u[k]);
        umax = fmaxf(umax, P.u[k]);
        vmin = fminf(vmin, P.v[k]);
        vmax = fmaxf(vmax, P.v[k]);
    }
    // pixel centres px + 1/2 within [umin, umax], widened by 1/100 pixel for the rounding of the
    // edge functions (an FP32 error of a few 1e-4 pixels at these coordinates)
    constexpr float e = 0.01f;
    x0 = max(0, (int)ceilf(fmaxf(umin, -2.f) - 0.5f - e));
    x1 = min(res - 1, (int)floorf(fminf(umax, (float)res + 2.f) - 0.5f + e));
    y0 = max(0, (int)ceilf(fmaxf(vmin, -2.f) - 0.5f - e));
    y1 = min(res - 1, (int)floorf(fminf(vmax, (float)res + 2.f) - 0.5f + e));
}

// Depth test of one pixel against the fan triangles of the polygon.
__device__ __forceinline__ void shade_pixel(const ClipPoly& P, int px, int py, float n, float f,
                                            uint32_t* __restrict__ zb, int res) {
    const float cx = px + 0.5f, cy = py + 0.5f;
    for (int k = 1; k + 1 < P.n; ++k) {
        const float ax = P.u[0], ay = P.v[0], bx = P.u[k], by = P.v[k], qx = P.u[k + 1], qy = P.v[k + 1];
        const float e0 = edge_fn(bx, by, qx, qy, cx, cy);
        const float e1 = edge_fn(qx, qy, ax, ay, cx, cy);
        const float e2 = edge_fn(ax, ay, bx, by, cx, cy);
        const bool in = (e0 >= 0.f && e1 >= 0.f && e2 >= 0.f) || (e0 <= 0.f && e1 <= 0.f && e2 <= 0.f);
        const float area = e0 + e1 + e2;
        if (!in || area == 0.f) continue;
        const float iw = (e0 * P.iw[0] + e1 * P.iw[k] + e2 * P.iw[k + 1]) / area;
        const float w = 1.0f / iw;
        if (w >= n * (1.f - 1e-6f) && w <= f && w > 0.f) atomicMin(zb + (size_t)py * res + px, __float_as_uint(w));
    }
}

// Append `value` to a list for every lane that wants to, with one atomic per warp. All 32 lanes call it.
__device__ __forceinline__ void warp_push(bool want, uint32_t value, uint32_t* __restrict__ list, uint64_t cap,
                                          unsigned long long* __restrict__ counter) {
    const unsigned m = __ballot_sync(0xffffffffu, want);
    if (!m) return;
    const int lane = threadIdx.x & 31, leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) {
        const unsigned long long q = base + __popc(m & gm_lanemask_lt());
        if (q < cap) list[q] = value;
    }
}

__global__ void __launch_bounds__(ZB_THREADS) k_zb_raster(const PairFT* __restrict__ pairs, uint64_t n_pairs,
                                                          const ZbFrustum* __restrict__ frusta,
                                                          const float4* __restrict__ tris, uint32_t res,
                                                          uint32_t* __restrict__ zbuf, uint32_t* __restrict__ big,
                                                          uint32_t* __restrict__ mid, uint64_t list_cap,
                                                          unsigned long long* __restrict__ n_lists) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    PairFT pr{0u, 0u};
    ZbFrustum F;
    ClipPoly P;
    P.n = 0;
    int x0 = 0, x1 = -1, y0 = 0, y1 = -1;
    if (i < n_pairs) {
        pr = pairs[i];
        F = frusta[pr.fix];
        clip_project(F, tris[3 * pr.tri], tris[3 * pr.tri + 1], tris[3 * pr.tri + 2], P);
        if (P.n >= 3) poly_bbox(P, (int)res, x0, x1, y0, y1);
    }
    const int npx = (P.n >= 3 && x1 >= x0 && y1 >= y0) ? (x1 - x0 + 1) * (y1 - y0 + 1) : 0;
    const bool to_big = npx > RASTER_WARP_PIXELS, to_mid = npx > RASTER_THREAD_PIXELS && !to_big;
    warp_push(to_big, (uint32_t)i, big, list_cap, &n_lists[0]);
    warp_push(to_mid, (uint32_t)i, mid, list_cap, &n_lists[1]);
    if (npx == 0 || to_big || to_mid) return;
    uint32_t* zb = zbuf + (size_t)pr.fix * res * res;
    for (int py = y0; py <= y1; ++py)
        for (int px = x0; px <= x1; ++px) shade_pixel(P, px, py, F.n, F.f, zb, (int)res);
}

__global__ void __launch_bounds__(ZB_THREADS) k_zb_raster_warp(const uint32_t* __restrict__ mid, uint64_t n_mid,
                                                               const PairFT* __restrict__ pairs,
                                                               const ZbFrustum* __restrict__ frusta,
                                                               const float4* __restrict__ tris, uint32_t res,
                                                               uint32_t* __restrict__ zbuf) {
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const int lane = threadIdx.x & 31;
    for (uint64_t q = warp0; q < n_mid; q += nwarps) {
        const PairFT pr = pairs[mid[q]];
        const ZbFrustum F = frusta[pr.fix];
        ClipPoly P;
        clip_project(F, tris[3 * pr.tri], tris[3 * pr.tri + 1], tris[3 * pr.tri + 2], P);
        if (P.n < 3) continue;
        int x0, x1, y0, y1;
        poly_bbox(P, (int)res, x0, x1, y0, y1);
        if (x1 < x0 || y1 < y0) continue;
        const int wdt = x1 - x0 + 1, cnt = wdt * (y1 - y0 + 1);
        uint32_t* zb = zbuf + (size_t)pr.fix * res * res;
        for (int k = lane; k < cnt; k += 32) shade_pixel(P, x0 + k % wdt, y0 + k / wdt, F.n, F.f, zb, (int)res);
    }
}

__global__ void __launch_bounds__(ZB_THREADS) k_zb_raster_big(const uint32_t* __restrict__ big,
                                                              const PairFT* __restrict__ pairs,
                                                              const ZbFrustum* __restrict__ frusta,
                                                              const float4* __restrict__ tris, uint32_t res,
                                                              uint32_t* __restrict__ zbuf) {
    const PairFT pr = pairs[big[blockIdx.x]];
    const ZbFrustum F = frusta[pr.fix];
    ClipPoly P;
    clip_project(F, tris[3 * pr.tri], tris[3 * pr.tri + 1], tris[3 * pr.tri + 2], P);
    if (P.n < 3) return;
    int x0, x1, y0, y1;
    poly_bbox(P, (int)res, x0, x1, y0, y1);
    if (x1 < x0 || y1 < y0) return;
    const int wdt = x1 - x0 + 1, cnt = wdt * (y1 - y0 + 1);
    uint32_t* zb = zbuf + (size_t)pr.fix * res * res;
    for (int k = threadIdx.x; k < cnt; k += blockDim.x) shade_pixel(P, x0 + k % wdt, y0 + k / wdt, F.n, F.f, zb, (int)res);
}

// ---- accumulate -----------------------------------------------------------------------------
struct ZbAccParams {
    float C2, K, tmax, eps;
    uint32_t ns, W, nt, res;
    uint64_t dbg_cap;
    float tanphi;   // cutoff tan theta, slightly enlarged (the warp-sphere test's cone)
};

// Visibility of a point in fixation F's z-buffer: inside the crop frustum (the NDC filter of
// Section 3.3.2) and |w - zbuf| <= eps (Section 3.2.2).
__device__ __forceinline__ bool zb_visible(const ZbFrustum& F, float px, float py, float pz,
                                           const uint32_t* __restrict__ zb, uint32_t res, float eps) {
    float x, y, w;
    to_camera(F, px, py, pz, x, y, w);
    if (!(w >= F.n && w <= F.f)) return false;
    const float u = fmaf(F.sx, __fdiv_rn(x, w), F.ox), v = fmaf(F.sy, __fdiv_rn(y, w), F.oy);
    const float R = (float)res;
    if (!(u >= 0.f && u <= R && v >= 0.f && v <= R)) return false;
    const int ix = min((int)u, (int)res - 1), iy = min((int)v, (int)res - 1);
    const uint32_t bits = __ldg(zb + (size_t)iy * res + ix);
    if (bits >= 0x7f800000u) return false;
    return fabsf(w - __uint_as_float(bits)) <= eps;
}

template <bool COMPARE, bool DEBUG>
__global__ void __launch_bounds__(ZB_THREADS) k_zb_accumulate(
    const float4* __restrict__ spos, const uint32_t* __restrict__ sidx, const float4* __restrict__ fix, uint32_t f0,
    uint32_t f1, const ZbFrustum* __restrict__ frusta, const uint32_t* __restrict__ zbuf, ZbAccParams P,
    float* __restrict__ out, unsigned int* __restrict__ max_bits, float2* __restrict__ state, uint32_t cur_in,
    int last, unsigned long long* __restrict__ counters, const float4* __restrict__ nodes,
    const float4* __restrict__ tris, int* __restrict__ err, DebugOut dbg) {
    const uint32_t j = blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = j < P.ns;
    const int lane = threadIdx.x & 31;
    const float4 s = valid ? spos[j] : make_float4(__int_as_float(0x7fc00000), 0.f, 0.f, 0.f);
    float sum = 0.f, cmp = 0.f;
    if (valid && cur_in != NO_WINDOW) {
        const float2 st = state[j];
        sum = st.x;
        cmp = st.y;
    }
    uint32_t cur = cur_in;
    unsigned long long n_in = 0, n_vis = 0, flip_v = 0, flip_h = 0;
    uint32_t n_node = 0, n_tri = 0;
    auto flush = [&](uint32_t w) {
        if (valid && sum != 0.f) out[(size_t)w * P.ns + sidx[j]] = sum;
        const float m = warp_max(valid ? sum : 0.f);
        if (lane == 0 && m > 0.f) atomicMax(&max_bits[w], __float_as_uint(m));
        sum = 0.f;
        cmp = 0.f;
    };
    // the warp's 32 samples (consecutive in the work order) as one sphere: each lane tests one of
    // 32 fixations against it, and the warp visits, in list order, only the fixations whose cone
    // reaches it; a skipped fixation changes no sum, and a window is written when the next visited
    // fixation opens another one
    const float4 bs = warp_bounding_sphere(valid, s.x, s.y, s.z);
    __shared__ float4 wf[ZB_THREADS / 32][64];
    float4* myf = wf[threadIdx.x >> 5];
    for (uint32_t c0 = f0; c0 < f1; c0 += 32) {
      const uint32_t m = min(32u, f1 - c0);
      bool pass = false;
      __syncwarp();
      if ((uint32_t)lane < m) {
          const float4 a = __ldg(&fix[2 * (c0 + lane)]), b = __ldg(&fix[2 * (c0 + lane) + 1]);
          myf[2 * lane] = a;
          myf[2 * lane + 1] = b;
          pass = cone_reaches_sphere(bs, a, b, P.tanphi);
      }
      unsigned pm = __ballot_sync(0xffffffffu, pass);
      __syncwarp();
      while (pm) {
        const int kk = __ffs(pm) - 1;
        pm &= pm - 1u;
        const uint32_t i = c0 + kk;
        const float4 F0 = myf[2 * kk], F1 = myf[2 * kk + 1];
        const uint32_t win = __float_as_uint(F1.w);
        if (win != cur) {
            if (cur != NO_WINDOW) flush(cur);
            cur = win;
        }
        const float px = s.x - F0.x, py = s.y - F0.y, pz = s.z - F0.z;
        const float d1 = fmaf(px, F1.x, fmaf(py, F1.y, pz * F1.z));
        const float cx = fmaf(py, F1.z, -pz * F1.y);
        const float cy = fmaf(pz, F1.x, -px * F1.z);
        const float cz = fmaf(px, F1.y, -py * F1.x);
        const float c2 = fmaf(cx, cx, fmaf(cy, cy, cz * cz));
        const float d1s = d1 * d1;
        if (!(d1 > 0.f && c2 <= P.K * d1s)) continue;
        const ZbFrustum& Fr = frusta[i - f0];
        if (!Fr.ok) continue;   // no crop window: the fixation is skipped (counted at set-up)
        ++n_in;
        const float g = F0.w * ex2_approx(-P.C2 * __fdividef(c2, d1s));
        const bool vis = zb_visible(Fr, s.x, s.y, s.z, zbuf + (size_t)(i - f0) * P.res * P.res, P.res, P.eps);
        if (vis) {
            ++n_vis;
            const float y = g - cmp;
            const float t = sum + y;
            cmp = (t - sum) - y;
            sum = t;
        }
        if (COMPARE) {
            Ray R;
            make_ray(R, make_float3(F0.x, F0.y, F0.z), make_float3(px, py, pz), P.tmax);
            int hit = -1;
            const bool ray_vis = !occluded(R, __float_as_uint(s.w), nodes, tris, P.nt, err, n_node, n_tri, hit);
            flip_v += vis && !ray_vis;
            flip_h += !vis && ray_vis;
        }
        if (DEBUG) {
            const unsigned long long q = atomicAdd(&counters[2], 1ull);
            if (q < P.dbg_cap) {
                dbg.sample[q] = sidx[j];
                dbg.fix[q] = dbg.fix_orig[i];
                dbg.vis[q] = vis ? 1 : 0;
                dbg.g[q] = g;
            }
        }
      }
    }
    if (last) {
        if (cur != NO_WINDOW) flush(cur);
    } else {
        // the next chunk continues the window of fixation f1 - 1: sums of an earlier window (its
        // last fixations were skipped here) are written now
        if (f1 > f0) {
            const uint32_t wl = __float_as_uint(__ldg(&fix[2 * (f1 - 1) + 1]).w);
            if (cur != wl && cur != NO_WINDOW) flush(cur);
        }
        if (valid) state[j] = make_float2(sum, cmp);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n_in += __shfl_xor_sync(0xffffffffu, n_in, o);
        n_vis += __shfl_xor_sync(0xffffffffu, n_vis, o);
        flip_v += __shfl_xor_sync(0xffffffffu, flip_v, o);
        flip_h += __shfl_xor_sync(0xffffffffu, flip_h, o);
    }
    if (lane == 0) {
        if (n_in) atomicAdd(&counters[0], n_in);
        if (n_vis) atomicAdd(&counters[1], n_vis);
        if (flip_v) atomicAdd(&counters[9], flip_v);
        if (flip_h) atomicAdd(&counters[10], flip_h);
    }
}

__global__ void k_zb_normalize(float* __restrict__ v, uint64_t ns, const unsigned int* __restrict__ max_bits,
                               uint32_t w0) {
    const uint32_t w = w0 + blockIdx.y;
    const float m = __uint_as_float(max_bits[w]);
    float* p = v + (size_t)w * ns;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ns; i += (uint64_t)gridDim.x * blockDim.x)
        p[i] = m > 0.f ? __fdiv_rn(p[i], m) : 0.f;
}

__global__ void k_zb_export(const uint32_t* __restrict__ zb, uint64_t n, float* __restrict__ out) {
    const uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = zb[i] >= 0x7f800000u ? INFINITY : __uint_as_float(zb[i]);
}

__global__ void k_zb_set_valid(unsigned long long* __restrict__ c, const uint32_t* __restrict__ n_valid) {
    c[3] = *n_valid;
}

// Render the z-buffers of frusta [0, nfix) into zbuf (nfix x res^2 words, cleared here). The pair
// list grows (and the chunk is redone) when the cull finds more pairs than it holds.
struct RasterBuffers {
    PairFT* pairs = nullptr;
    uint32_t* big = nullptr;
    uint32_t* mid = nullptr;
    uint64_t cap = 0;
    unsigned long long* counts = nullptr;   // [0] pairs [1] big [2] mid
};

gm_status rb_alloc(RasterBuffers& rb, uint64_t cap, cudaStream_t s) {
    rb.cap = cap;
    GM_TRY(gm_alloc((void**)&rb.pairs, sizeof(PairFT) * cap, s));
    GM_TRY(gm_alloc((void**)&rb.big, sizeof(uint32_t) * cap, s));
    GM_TRY(gm_alloc((void**)&rb.mid, sizeof(uint32_t) * cap, s));
    return GM_OK;
}

void rb_free(RasterBuffers& rb, cudaStream_t s) {
    if (rb.pairs) cudaFreeAsync(rb.pairs, s);
    if (rb.big) cudaFreeAsync(rb.big, s);
    if (rb.mid) cudaFreeAsync(rb.mid, s);
    rb.pairs = nullptr;
    rb.big = rb.mid = nullptr;
}

gm_status render_zbuffers(gm_ctx* ctx, gm_scene* sc, const ZbFrustum* frusta, uint32_t nfix, uint32_t res,
                          uint32_t* zbuf, RasterBuffers& rb, cudaStream_t s, int* launches,
                          unsigned long long* raster_pairs) {
    const size_t npx = (size_t)res * res;
    for (int attempt = 0; attempt < 3; ++attempt) {
        static_assert(ZB_EMPTY == 0xffffffffu, "a byte-wise 0xff clear writes ZB_EMPTY");
        GM_TRY_CUDA(cudaMemsetAsync(zbuf, 0xff, sizeof(uint32_t) * npx * nfix, s));
        GM_TRY_CUDA(cudaMemsetAsync(rb.counts, 0, sizeof(unsigned long long) * 3, s));
        const dim3 cgrid(gm_div_up(sc->n_tris, ZB_THREADS), std::min<uint32_t>(gm_div_up(nfix, ZB_SMEM_FRUSTA), 65535));
        k_zb_cull<<<cgrid, ZB_THREADS, 0, s>>>(sc->bvh_tris, sc->n_tris, frusta, nfix,
                                                                          res, rb.pairs, rb.cap, &rb.counts[0]);
        ++*launches;
        unsigned long long np = 0;
        GM_TRY_CUDA(cudaMemcpyAsync(&np, &rb.counts[0], sizeof(np), cudaMemcpyDeviceToHost, s));
        GM_TRY_CUDA(cudaStreamSynchronize(s));
        if (np > rb.cap) {
            rb_free(rb, s);
            GM_TRY(rb_alloc(rb, np + np / 4, s));
            continue;
        }
        if (raster_pairs) *raster_pairs += np;
        // the next call on this scene starts with room for this density of pairs
        sc->zb_pairs_per_fix = std::max<uint64_t>(sc->zb_pairs_per_fix, np / nfix + 1);
        if (np > 0) {
            if (np > 0xffffffffull) return gm_set_error(GM_ERR_UNSUPPORTED, "z-buffer: more than 2^32 raster pairs");
            k_zb_raster<<<(uint32_t)((np + ZB_THREADS - 1) / ZB_THREADS), ZB_THREADS, 0, s>>>(
                rb.pairs, np, frusta, sc->tri_canon, res, zbuf, rb.big, rb.mid, rb.cap, &rb.counts[1]);
            ++*launches;
            unsigned long long nl[2] = {0, 0};
            GM_TRY_CUDA(cudaMemcpyAsync(nl, &rb.counts[1], sizeof(nl), cudaMemcpyDeviceToHost, s));
            GM_TRY_CUDA(cudaStreamSynchronize(s));
            const unsigned long long nb = std::min<unsigned long long>(nl[0], rb.cap);
            const unsigned long long nm = std::min<unsigned long long>(nl[1], rb.cap);
            if (nm > 0) {
                const uint32_t wblocks = (uint32_t)std::min<unsigned long long>((nm + 7) / 8, (uint64_t)ctx->n_sm * 16);
                k_zb_raster_warp<<<wblocks, ZB_THREADS, 0, s>>>(rb.mid, nm, rb.pairs, frusta, sc->tri_canon, res, zbuf);
                ++*launches;
            }
            for (unsigned long long b0 = 0; b0 < nb; b0 += 1u << 30) {
                const uint32_t nblk = (uint32_t)std::min<unsigned long long>(nb - b0, 1u << 30);
                k_zb_raster_big<<<nblk, ZB_THREADS, 0, s>>>(rb.big + b0, rb.pairs, frusta, sc->tri_canon, res, zbuf);
                ++*launches;
            }
        }
        GM_TRY_CUDA(cudaGetLastError());
        return GM_OK;
    }
    return gm_set_error(GM_ERR_INTERNAL, "z-buffer: raster pair list did not settle");
}

gm_status check_zb_params(const gm_zbuffer_params* zp) {
    if (!zp) return gm_set_error(GM_ERR_INVALID_ARG, "z-buffer: null parameters");
    if (zp->res < 1 || zp->res > 8192) return gm_set_error(GM_ERR_INVALID_ARG, "z-buffer: res must be in [1, 8192]");
    if (!(zp->near_m > 0.f) || !(zp->far_m > zp->near_m) || !std::isfinite(zp->far_m))
        return gm_set_error(GM_ERR_INVALID_ARG, "z-buffer: need 0 < near < far < inf");
    if (!(zp->eps_m >= 0.f) || !std::isfinite(zp->eps_m))
        return gm_set_error(GM_ERR_INVALID_ARG, "z-buffer: eps must be finite and >= 0");
    return GM_OK;
}

}  // namespace

extern "C" gm_status gm_zbuffer_render(gm_scene* sc, const float* eye, const float* gaze, const float* cam_forward,
                                       const float* cam_up, uint32_t n, float theta_rad, float cutoff_sigmas,
                                       const gm_zbuffer_params* zp, float* zbuf_out, double* crop_out,
                                       gm_stream stream) {
    if (!sc || (n > 0 && (!eye || !gaze || !zbuf_out)))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_zbuffer_render: null argument");
    GM_TRY(check_zb_params(zp));
    if (!(theta_rad > 0.f && theta_rad < 1.5f) || !(cutoff_sigmas > 0.f))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_zbuffer_render: bad theta or cutoff");
    if (n == 0) return GM_OK;
    cudaStream_t s = (cudaStream_t)stream;
    gm_ctx* ctx = sc->ctx;
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    const size_t npx = (size_t)zp->res * zp->res;
    std::vector<std::pair<void*, bool>> staged;
    std::vector<void*> tmp;
    auto done = [&](gm_status st) {
        for (auto& p : staged)
            if (p.second) cudaFreeAsync(p.first, s);
        for (void* p : tmp) cudaFreeAsync(p, s);
        return st;
    };
    auto stage = [&](const float* src, size_t nfl, const float** dst) -> gm_status {
        if (!src) {
            *dst = nullptr;
            return GM_OK;
        }
        void* d = nullptr;
        bool owned = false;
        GM_TRY(gm_stage_to_device(src, sizeof(float) * nfl, s, &d, &owned));
        staged.push_back({d, owned});
        *dst = (const float*)d;
        return GM_OK;
    };
    const float *d_eye, *d_gaze, *d_fwd, *d_up;
    gm_status st;
    if ((st = stage(eye, 3 * (size_t)n, &d_eye)) != GM_OK || (st = stage(gaze, 3 * (size_t)n, &d_gaze)) != GM_OK ||
        (st = stage(cam_forward, 3 * (size_t)n, &d_fwd)) != GM_OK || (st = stage(cam_up, 3 * (size_t)n, &d_up)) != GM_OK)
        return done(st);
    ZbFrustum* fr = nullptr;
    double* crop = nullptr;
    uint32_t* zb = nullptr;
    float* zf = nullptr;
    RasterBuffers rb;
    rb.cap = std::max<uint64_t>(1u << 16, (uint64_t)n * std::max<uint64_t>(4096, sc->zb_pairs_per_fix * 5 / 4));
#define ZB_TMP(ptr, bytes)                                                          \
    do {                                                                            \
        if ((st = gm_alloc((void**)&(ptr), (bytes), s)) != GM_OK) return done(st);  \
        tmp.push_back((void*)(ptr));                                                \
    } while (0)
    ZB_TMP(fr, sizeof(ZbFrustum) * n);
    ZB_TMP(crop, sizeof(double) * 4 * n);
    ZB_TMP(zb, sizeof(uint32_t) * npx * n);
    ZB_TMP(rb.counts, sizeof(unsigned long long) * 3);
    if ((st = rb_alloc(rb, rb.cap, s)) != GM_OK) {
        rb_free(rb, s);
        return done(st);
    }
    int launches = 0;
    k_zb_frustum<<<gm_div_up(n, 128), 128, 0, s>>>(n, nullptr, d_eye, d_gaze, d_fwd, d_up, (double)theta_rad,
                                                   (double)cutoff_sigmas, (double)zp->near_m, (double)zp->far_m,
                                                   zp->res, fr, crop, nullptr);
    ++launches;
    st = render_zbuffers(ctx, sc, fr, n, zp->res, zb, rb, s, &launches, nullptr);
    if (st == GM_OK && gm_is_device_ptr(zbuf_out)) {
        k_zb_export<<<gm_div_up(npx * n, 256), 256, 0, s>>>(zb, npx * n, zbuf_out);
        ++launches;
    } else if (st == GM_OK) {
        if ((st = gm_alloc((void**)&zf, sizeof(float) * npx * n, s)) == GM_OK) {
            k_zb_export<<<gm_div_up(npx * n, 256), 256, 0, s>>>(zb, npx * n, zf);
            ++launches;
            st = gm_copy_out(zbuf_out, zf, sizeof(float) * npx * n, s);
            cudaFreeAsync(zf, s);
        }
    }
    if (st == GM_OK && crop_out) st = gm_copy_out(crop_out, crop, sizeof(double) * 4 * n, s);
    rb_free(rb, s);
    ctx->launches += launches;
    if (st == GM_OK) {
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) st = gm_cuda_error(e, "gm_zbuffer_render");
    }
    if (st == GM_OK) {
        cudaError_t e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) st = gm_cuda_error(e, "gm_zbuffer_render");
    }
    return done(st);
#undef ZB_TMP
}

extern "C" gm_status gm_accumulate_zbuffer(gm_scene* sc, gm_samples* sm, const gm_fixations* fx,
                                           const float* cam_forward, const float* cam_up, const gm_params* prm,
                                           const gm_zbuffer_params* zp, gm_stream stream, gm_map** out) {
    if (!sc || !sm || !fx || !prm || !out) return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: null argument");
    *out = nullptr;
    if (sm->scene != sc) return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: samples belong to another scene");
    GM_TRY(check_zb_params(zp));
    if (!(prm->theta_rad > 0.f) || !(prm->theta_rad < 1.5f))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: theta must be in (0, 1.5) rad");
    if (!(prm->cutoff_sigmas > 0.f) || !std::isfinite(prm->cutoff_sigmas))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: cutoff must be > 0");
    if (!(prm->eps_rel >= 0.f && prm->eps_rel < 1.f))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: eps_rel must be in [0, 1)");
    if (std::isnan(prm->t_begin) || std::isnan(prm->t_end) || !(prm->t_begin < prm->t_end))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: need t_begin < t_end");
    if (fx->n > 0 && (!fx->eye_xyz || !fx->gaze_xyz || !fx->duration_s || !fx->timestamp_s))
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: null fixation array");
    uint64_t W = 1;
    if (prm->window_s > 0.0) {
        if (!std::isfinite(prm->t_begin) || !std::isfinite(prm->t_end) || !std::isfinite(prm->window_s))
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_accumulate_zbuffer: windows need a finite interval");
        W = (uint64_t)std::ceil((prm->t_end - prm->t_begin) / prm->window_s);
        if (W == 0) W = 1;
        if (W > (1u << 24)) return gm_set_error(GM_ERR_UNSUPPORTED, "gm_accumulate_zbuffer: more than 2^24 windows");
    }
    const bool debug = (prm->flags & GM_F_DEBUG_PAIRS) && prm->debug_pair_cap > 0;
    const bool compare = zp->compare != 0;
    cudaStream_t s = (cudaStream_t)stream;
    gm_ctx* ctx = sc->ctx;
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    const uint64_t ns = sm->n;
    const uint32_t nf = fx->n;
    const uint32_t res = zp->res;
    const size_t npx = (size_t)res * res;

    gm_map* mp = new gm_map();
    mp->ctx = ctx;
    mp->W = (uint32_t)W;
    mp->ns = ns;
    mp->stream = s;
    mp->stats.n_windows = (uint32_t)W;
    mp->zbuffer = true;
    std::vector<void*> tmp;
    RasterBuffers rb;
    auto fail = [&](gm_status st) {
        for (void* p : tmp) cudaFreeAsync(p, s);
        rb_free(rb, s);
        gm_map_free(mp);
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
    MAP_ALLOC(mp->values, sizeof(float) * W * (ns ? ns : 1));
    MAP_ALLOC(mp->max_bits, sizeof(unsigned int) * W);
    MAP_ALLOC(mp->counters, sizeof(unsigned long long) * 16);
    GM_TRY_CUDA(cudaMemsetAsync(mp->values, 0, sizeof(float) * W * (ns ? ns : 1), s));
    GM_TRY_CUDA(cudaMemsetAsync(mp->max_bits, 0, sizeof(unsigned int) * W, s));
    GM_TRY_CUDA(cudaMemsetAsync(mp->counters, 0, sizeof(unsigned long long) * 16, s));
    if (debug) {
        mp->dbg_cap = prm->debug_pair_cap;
        MAP_ALLOC(mp->dbg_sample, sizeof(uint32_t) * mp->dbg_cap);
        MAP_ALLOC(mp->dbg_fix, sizeof(uint32_t) * mp->dbg_cap);
        MAP_ALLOC(mp->dbg_vis, mp->dbg_cap);
        MAP_ALLOC(mp->dbg_g, sizeof(float) * mp->dbg_cap);
    }
    int launches = 0;

    // ---- fixation prep --------------------------------------------------------------------
    void *d_eye = nullptr, *d_gaze = nullptr, *d_dur = nullptr, *d_ts = nullptr, *d_fwd = nullptr, *d_up = nullptr;
    bool o[6] = {};
    if ((st = gm_stage_to_device(fx->eye_xyz, sizeof(float) * 3 * (size_t)nf, s, &d_eye, &o[0])) != GM_OK) return fail(st);
    if (o[0]) tmp.push_back(d_eye);
    if ((st = gm_stage_to_device(fx->gaze_xyz, sizeof(float) * 3 * (size_t)nf, s, &d_gaze, &o[1])) != GM_OK) return fail(st);
    if (o[1]) tmp.push_back(d_gaze);
    if ((st = gm_stage_to_device(fx->duration_s, sizeof(float) * (size_t)nf, s, &d_dur, &o[2])) != GM_OK) return fail(st);
    if (o[2]) tmp.push_back(d_dur);
    if ((st = gm_stage_to_device(fx->timestamp_s, sizeof(double) * (size_t)nf, s, &d_ts, &o[3])) != GM_OK) return fail(st);
    if (o[3]) tmp.push_back(d_ts);
    if (cam_forward) {
        if ((st = gm_stage_to_device(cam_forward, sizeof(float) * 3 * (size_t)nf, s, &d_fwd, &o[4])) != GM_OK) return fail(st);
        if (o[4]) tmp.push_back(d_fwd);
    }
    if (cam_up) {
        if ((st = gm_stage_to_device(cam_up, sizeof(float) * 3 * (size_t)nf, s, &d_up, &o[5])) != GM_OK) return fail(st);
        if (o[5]) tmp.push_back(d_up);
    }
    uint32_t *keys = nullptr, *vals = nullptr, *n_valid = nullptr, *orig = nullptr;
    float4* packed = nullptr;
    TMP_ALLOC(keys, sizeof(uint32_t) * (nf ? nf : 1));
    TMP_ALLOC(vals, sizeof(uint32_t) * (nf ? nf : 1));
    TMP_ALLOC(orig, sizeof(uint32_t) * (nf ? nf : 1));
    TMP_ALLOC(packed, sizeof(float4) * 2 * (nf ? nf : 1));
    TMP_ALLOC(n_valid, sizeof(uint32_t));
    GM_TRY_CUDA(cudaMemsetAsync(n_valid, 0, sizeof(uint32_t), s));
    const double tan_t = std::tan((double)prm->theta_rad);
    const float wnorm = (float)(1.0 / (tan_t * std::sqrt(2.0 * 3.14159265358979323846)));
    if (nf > 0) {
        k_zb_keys<<<gm_div_up(nf, 256), 256, 0, s>>>((const double*)d_ts, (const float*)d_eye, (const float*)d_gaze,
                                                     (const float*)d_dur, nf, prm->t_begin, prm->t_end,
                                                     prm->window_s > 0.0 ? prm->window_s : 0.0, (uint32_t)W, keys, vals,
                                                     n_valid, ctx->dev_err);
        ++launches;
        int bits = 1;
        while (bits < 32 && (1ull << bits) <= W) ++bits;
        if ((st = gm_radix_sort_u32(keys, vals, nf, bits, s, &launches)) != GM_OK) return fail(st);
        k_zb_pack<<<gm_div_up(nf, 256), 256, 0, s>>>(keys, vals, (const float*)d_eye, (const float*)d_gaze,
                                                     (const float*)d_dur, nf, wnorm, packed, orig);
        ++launches;
    }
    uint32_t nv = 0;
    GM_TRY_CUDA(cudaMemcpyAsync(&nv, n_valid, sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
    GM_TRY_CUDA(cudaStreamSynchronize(s));
    k_zb_set_valid<<<1, 1, 0, s>>>(mp->counters, n_valid);
    ++launches;

    // ---- frusta, then z-buffers and accumulation chunk by chunk ---------------------------
    ZbFrustum* frusta = nullptr;
    TMP_ALLOC(frusta, sizeof(ZbFrustum) * (nv ? nv : 1));
    if (nv > 0) {
        k_zb_frustum<<<gm_div_up(nv, 128), 128, 0, s>>>(nv, orig, (const float*)d_eye, (const float*)d_gaze,
                                                        (const float*)d_fwd, (const float*)d_up, (double)prm->theta_rad,
                                                        (double)prm->cutoff_sigmas, (double)zp->near_m,
                                                        (double)zp->far_m, res, frusta, nullptr, &mp->counters[8]);
        ++launches;
    }
    const uint64_t budget = zp->zbuffer_bytes ? zp->zbuffer_bytes : (2ull << 30);
    const uint32_t chunk = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(nv ? nv : 1, budget / (npx * 4)));
    uint32_t* zbuf = nullptr;
    float2* state = nullptr;
    TMP_ALLOC(zbuf, sizeof(uint32_t) * npx * chunk);
    if (chunk < nv) TMP_ALLOC(state, sizeof(float2) * (ns ? ns : 1));
    rb.cap = std::max<uint64_t>(1u << 20, (uint64_t)chunk * std::max<uint64_t>(2048, sc->zb_pairs_per_fix * 5 / 4));
    TMP_ALLOC(rb.counts, sizeof(unsigned long long) * 3);
    if ((st = rb_alloc(rb, rb.cap, s)) != GM_OK) return fail(st);

    ZbAccParams P;
    P.C2 = (float)(1.4426950408889634 / (2.0 * tan_t * tan_t));
    P.K = (float)((double)prm->cutoff_sigmas * tan_t * (double)prm->cutoff_sigmas * tan_t);
    P.tmax = 1.0f - prm->eps_rel;
    P.eps = zp->eps_m;
    P.ns = (uint32_t)ns;
    P.W = (uint32_t)W;
    P.nt = sc->n_tris;
    P.res = res;
    P.dbg_cap = mp->dbg_cap;
    P.tanphi = (float)(std::sqrt((double)P.K) * 1.00001);
    DebugOut dbg{mp->dbg_sample, mp->dbg_fix, mp->dbg_vis, mp->dbg_g, orig};
    const bool reorder = sm->work_pos != nullptr;
    uint32_t* ident = nullptr;
    const float4* spos = reorder ? sm->work_pos : sm->pos;
    const uint32_t* sidx = reorder ? sm->work_idx : nullptr;
    if (!sidx && ns > 0) {
        std::vector<uint32_t> h(ns);
        for (uint64_t k = 0; k < ns; ++k) h[k] = (uint32_t)k;
        TMP_ALLOC(ident, sizeof(uint32_t) * ns);
        GM_TRY_CUDA(cudaMemcpyAsync(ident, h.data(), sizeof(uint32_t) * ns, cudaMemcpyHostToDevice, s));
        GM_TRY_CUDA(cudaStreamSynchronize(s));
        sidx = ident;
    }
    std::vector<uint32_t> win_of(nv);
    if (nv > 0) {
        std::vector<float4> hp(2 * (size_t)nv);
        GM_TRY_CUDA(cudaMemcpyAsync(hp.data(), packed, sizeof(float4) * 2 * nv, cudaMemcpyDeviceToHost, s));
        GM_TRY_CUDA(cudaStreamSynchronize(s));
        for (uint32_t i = 0; i < nv; ++i) {
            uint32_t b;
            memcpy(&b, &hp[2 * (size_t)i + 1].w, 4);
            win_of[i] = b;
        }
    }
    unsigned long long raster_pairs = 0;
    for (uint32_t f0 = 0; f0 < nv; f0 += chunk) {
        const uint32_t f1 = std::min(nv, f0 + chunk);
        if ((st = render_zbuffers(ctx, sc, frusta + f0, f1 - f0, res, zbuf, rb, s, &launches, &raster_pairs)) != GM_OK)
            return fail(st);
        if (ns > 0) {
            const uint32_t cur_in = f0 == 0 ? NO_WINDOW : win_of[f0 - 1];
            const int last = f1 == nv;
            const uint32_t grid = gm_div_up(ns, ZB_THREADS);
#define ZB_ACC(C, D)                                                                                          \
    k_zb_accumulate<C, D><<<grid, ZB_THREADS, 0, s>>>(spos, sidx, packed, f0, f1, frusta + f0, zbuf, P, mp->values, \
                                                      mp->max_bits, state, cur_in, last, mp->counters, sc->nodes,  \
                                                      sc->bvh_tris, ctx->dev_err, dbg)
            if (compare) {
                if (debug) ZB_ACC(true, true);
                else ZB_ACC(true, false);
            } else {
                if (debug) ZB_ACC(false, true);
                else ZB_ACC(false, false);
            }
#undef ZB_ACC
            ++launches;
        }
    }
    if (prm->normalize && ns > 0) {
        const uint32_t per_win = std::max<uint32_t>(1, std::min<uint32_t>(gm_div_up(ns, 256), 64));
        for (uint64_t w0 = 0; w0 < W; w0 += 65535) {
            dim3 grid(per_win, (uint32_t)std::min<uint64_t>(65535, W - w0));
            k_zb_normalize<<<grid, 256, 0, s>>>(mp->values, ns, mp->max_bits, (uint32_t)w0);
            ++launches;
        }
    }
    GM_TRY_CUDA(cudaMemcpyAsync(&mp->counters[11], &raster_pairs, sizeof(raster_pairs), cudaMemcpyHostToDevice, s));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_accumulate_zbuffer launch"));
    GM_TRY_CUDA(cudaStreamSynchronize(s));   // raster_pairs and the host vectors above are host temporaries
    for (void* p : tmp) cudaFreeAsync(p, s);
    rb_free(rb, s);
    mp->stats.launches = (uint32_t)launches;
    ctx->launches += launches;
    *out = mp;
    return GM_OK;
#undef TMP_ALLOC
#undef MAP_ALLOC
}

extern "C" gm_status gm_zbuffer_stats(const gm_map* mp, uint64_t* skipped_fixations, uint64_t* flips_to_visible,
                                      uint64_t* flips_to_hidden, uint64_t* raster_pairs) {
    if (!mp || !mp->counters) return gm_set_error(GM_ERR_INVALID_ARG, "gm_zbuffer_stats: null map");
    if (!mp->zbuffer) return gm_set_error(GM_ERR_INVALID_ARG, "gm_zbuffer_stats: the map was not made by gm_accumulate_zbuffer");
    unsigned long long c[16] = {};
    GM_TRY_CUDA(cudaStreamSynchronize(mp->stream));
    GM_TRY_CUDA(cudaMemcpy(c, mp->counters, sizeof(c), cudaMemcpyDeviceToHost));
    if (skipped_fixations) *skipped_fixations = c[8];
    if (flips_to_visible) *flips_to_visible = c[9];
    if (flips_to_hidden) *flips_to_hidden = c[10];
    if (raster_pairs) *raster_pairs = c[11];
    return GM_OK;
}
