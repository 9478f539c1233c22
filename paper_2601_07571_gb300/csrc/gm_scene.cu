// gm_scene.cu -- gm_build_scene: meshes -> world triangles -> BVH; gm_scene_pose: re-posed meshes.
//
// The paper tests occlusion with a z-buffer rendered per point of view (Section 3.2.2); here
// occlusion is an exact segment test against every triangle, accelerated by a binary BVH built
// on the GPU in data-parallel steps:
//   1. world vertices: FP64 transform per vertex, rounded to FP32 (same operation order as
//      the FP64 reference: ((m0 x + m1 y) + m2 z) + m3, no fused multiply-add);
//   2. 63-bit Morton code of each triangle centroid in the centroid bounds;
//   3. stable radix sort of the codes (leaf order);
//   4. the hierarchy, by one of two builders:
//      PLOC (default; Meister & Bittner, "Parallel locally-ordered clustering for bounding volume
//      hierarchy construction", TVCG 2018): rounds of nearest-neighbour search by union-box
//      surface area within +-8 positions of the Morton order, merging of mutual pairs and
//      compaction, until one cluster is left;
//      LBVH (Karras, "Maximizing parallelism in the construction of BVHs, octrees, and k-d
//      trees", HPG 2012): one thread per internal node finds its key range and split, then a
//      bottom-up refit in which the second child to arrive writes the node's union box;
//   5. internal nodes renumbered in depth-first order (a parent's nearer child is often in the
//      next 64 bytes).
// Node layout (64 B): the boxes of both children plus the two child links, so one node fetch
// decides both children. A child link >= 0 is an internal node, < 0 is leaf ~link (one
// triangle). Boxes are widened by 2^-19 of the scene's largest coordinate so that the FP32
// slab test never rejects a triangle the watertight triangle test would hit.
// Dynamic scenes keep the mesh-local triangles; gm_scene_pose recomputes the world triangles for
// new transforms and refits every box bottom-up over the unchanged hierarchy.
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "gm_internal.cuh"

namespace {

// Store internal nodes in depth-first order (see k_dfs_index).
constexpr bool kDfsLayout = true;
// Clustering radius of the PLOC builder: 8 neighbours on each side traced the paper scene in
// 244 ms against 257 ms for 16 (34.2 vs 34.1 nodes per ray; the depth-first layout of the
// smaller-radius tree caches better), and builds faster.
constexpr int kPlocRadius = 8;

struct Mat16 {
    double m[16];
};

__global__ void k_transform(const float* __restrict__ v, uint32_t nv, Mat16 M, float* __restrict__ out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    double x = v[3 * i], y = v[3 * i + 1], z = v[3 * i + 2];
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        double s = __dadd_rn(__dmul_rn(M.m[4 * r + 0], x), __dmul_rn(M.m[4 * r + 1], y));
        s = __dadd_rn(s, __dmul_rn(M.m[4 * r + 2], z));
        s = __dadd_rn(s, M.m[4 * r + 3]);
        out[3 * i + r] = __double2float_rn(s);
    }
}

__device__ __forceinline__ unsigned int f2ord(float f) {
    unsigned int b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(unsigned int o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// bounds layout (ordered-uint encoded floats): [0..2] centroid min, [3..5] centroid max,
// [6..8] vertex min, [9..11] vertex max.
__global__ void k_bounds_init(unsigned int* b) {
    int i = threadIdx.x;
    if (i < 12) b[i] = ((i / 3) % 2 == 0) ? 0xffffffffu : 0u;
}

__global__ void k_gather(const float* __restrict__ wv, const uint32_t* __restrict__ idx, uint32_t nt,
                         uint32_t nv, uint32_t tri_base, uint32_t mesh, float4* __restrict__ tri_canon,
                         uint32_t* __restrict__ tri_mesh, unsigned int* __restrict__ bounds,
                         int* __restrict__ err) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[6], hi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { lo[c] = INFINITY; hi[c] = -INFINITY; }
    if (t < nt) {
        float3 v[3];
        bool bad = false;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint32_t vi = idx[3 * t + k];
            if (vi >= nv) { bad = true; vi = 0; }
            v[k] = make_float3(wv[3 * vi], wv[3 * vi + 1], wv[3 * vi + 2]);
        }
        if (bad) atomicCAS(err, 0, GM_DEV_BAD_INDEX);
        uint32_t g = tri_base + t;
        tri_canon[3 * g + 0] = make_float4(v[0].x, v[0].y, v[0].z, 0.f);
        tri_canon[3 * g + 1] = make_float4(v[1].x, v[1].y, v[1].z, 0.f);
        tri_canon[3 * g + 2] = make_float4(v[2].x, v[2].y, v[2].z, 0.f);
        tri_mesh[g] = mesh;
        float c[3] = {(v[0].x + v[1].x + v[2].x) * (1.f / 3.f), (v[0].y + v[1].y + v[2].y) * (1.f / 3.f),
                      (v[0].z + v[1].z + v[2].z) * (1.f / 3.f)};
        const float* vf = &v[0].x;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = hi[a] = c[a];
            lo[3 + a] = fminf(fminf(vf[a], vf[3 + a]), vf[6 + a]);
            hi[3 + a] = fmaxf(fmaxf(vf[a], vf[3 + a]), vf[6 + a]);
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    }
    if ((threadIdx.x & 31) == 0 && blockIdx.x * blockDim.x + (threadIdx.x & ~31u) < nt) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bounds[a], f2ord(lo[a]));
            atomicMax(&bounds[3 + a], f2ord(hi[a]));
            atomicMin(&bounds[6 + a], f2ord(lo[3 + a]));
            atomicMax(&bounds[9 + a], f2ord(hi[3 + a]));
        }
    }
}

__device__ __forceinline__ uint64_t spread3_21(uint32_t v) {
    uint64_t x = v & 0x1fffffu;
    x = (x | x << 32) & 0x1f00000000ffffull;
    x = (x | x << 16) & 0x1f0000ff0000ffull;
    x = (x | x << 8) & 0x100f00f00f00f00full;
    x = (x | x << 4) & 0x10c30c30c30c30c3ull;
    x = (x | x << 2) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t quant21(float c, float lo, float hi) {
    float ext = hi - lo;
    if (!(ext > 0.f)) return 0u;
    float q = (c - lo) / ext * 2097152.f;
    q = fminf(fmaxf(q, 0.f), 2097151.f);
    return (uint32_t)q;
}

__global__ void k_morton(const float4* __restrict__ tri, uint32_t nt, const unsigned int* __restrict__ bounds,
                         uint64_t* __restrict__ keys, uint32_t* __restrict__ vals) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    float4 a = tri[3 * t], b = tri[3 * t + 1], c = tri[3 * t + 2];
    float cx = (a.x + b.x + c.x) * (1.f / 3.f), cy = (a.y + b.y + c.y) * (1.f / 3.f),
          cz = (a.z + b.z + c.z) * (1.f / 3.f);
    uint32_t qx = quant21(cx, ord2f(bounds[0]), ord2f(bounds[3]));
    uint32_t qy = quant21(cy, ord2f(bounds[1]), ord2f(bounds[4]));
    uint32_t qz = quant21(cz, ord2f(bounds[2]), ord2f(bounds[5]));
    keys[t] = (spread3_21(qx) << 2) | (spread3_21(qy) << 1) | spread3_21(qz);
    vals[t] = t;
}

__device__ __forceinline__ int lcp(const uint64_t* __restrict__ keys, int n, int i, int j) {
    if (j < 0 || j >= n) return -1;
    uint64_t a = keys[i], b = keys[j];
    if (a != b) return __clzll((long long)(a ^ b));
    return 64 + __clz(i ^ j);
}

__global__ void k_hierarchy(const uint64_t* __restrict__ keys, int n, float4* __restrict__ nodes,
                            int* __restrict__ parent_node, int* __restrict__ parent_leaf) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    int d = (lcp(keys, n, i, i + 1) - lcp(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    int dmin = lcp(keys, n, i, i - d);
    int lmax = 2;
    while (lcp(keys, n, i, i + lmax * d) > dmin) lmax <<= 1;
    int l = 0;
    for (int t = lmax >> 1; t >= 1; t >>= 1)
        if (lcp(keys, n, i, i + (l + t) * d) > dmin) l += t;
    int j = i + l * d;
    int dnode = lcp(keys, n, i, j);
    int s = 0, t = l;
    do {
        t = (t + 1) >> 1;
        if (lcp(keys, n, i, i + (s + t) * d) > dnode) s += t;
    } while (t > 1);
    int split = i + s * d + min(d, 0);
    int lo = min(i, j), hi = max(i, j);
    int left = (lo == split) ? ~split : split;
    int right = (hi == split + 1) ? ~(split + 1) : split + 1;
    nodes[4 * i + 3] = make_float4(__int_as_float(left), __int_as_float(right), 0.f, 0.f);
    if (left < 0) parent_leaf[~left] = i; else parent_node[left] = i;
    if (right < 0) parent_leaf[~right] = i; else parent_node[right] = i;
    if (i == 0) parent_node[0] = -1;
}

__device__ __forceinline__ void store_child_box(float* node, int side, const float lo[3], const float hi[3]) {
    // side 0: floats 0..5 = Lmin xyz, Lmax xyz; side 1: floats 6..11 = Rmin xyz, Rmax xyz
    float* p = node + 6 * side;
    p[0] = lo[0]; p[1] = lo[1]; p[2] = lo[2];
    p[3] = hi[0]; p[4] = hi[1]; p[5] = hi[2];
}

__global__ void k_refit(const float4* __restrict__ tri_canon, const uint32_t* __restrict__ order, int n,
                        float4* __restrict__ nodes, const int* __restrict__ parent_node,
                        const int* __restrict__ parent_leaf, unsigned int* __restrict__ flags,
                        const unsigned int* __restrict__ bounds, float4* __restrict__ bvh_tris) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t t = order[i];
    float4 a = tri_canon[3 * t], b = tri_canon[3 * t + 1], c = tri_canon[3 * t + 2];
    bvh_tris[3 * i + 0] = make_float4(a.x, a.y, a.z, __uint_as_float(t));
    bvh_tris[3 * i + 1] = b;
    bvh_tris[3 * i + 2] = c;
    if (n == 1) return;
    float big = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) big = fmaxf(big, fmaxf(fabsf(ord2f(bounds[6 + k])), fabsf(ord2f(bounds[9 + k]))));
    const float margin = big * (1.0f / 524288.0f) + 1e-30f;
    float lo[3] = {fminf(fminf(a.x, b.x), c.x) - margin, fminf(fminf(a.y, b.y), c.y) - margin,
                   fminf(fminf(a.z, b.z), c.z) - margin};
    float hi[3] = {fmaxf(fmaxf(a.x, b.x), c.x) + margin, fmaxf(fmaxf(a.y, b.y), c.y) + margin,
                   fmaxf(fmaxf(a.z, b.z), c.z) + margin};
    int p = parent_leaf[i];
    int self = ~i;
    while (p >= 0) {
        float* node = reinterpret_cast<float*>(nodes + 4 * p);
        int left = __float_as_int(node[12]);
        store_child_box(node, left == self ? 0 : 1, lo, hi);
        __threadfence();
        if (atomicAdd(&flags[p], 1u) == 0u) return;  // the sibling finishes this node
        __threadfence();
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            lo[k] = fminf(__ldcg(node + k), __ldcg(node + 6 + k));
            hi[k] = fmaxf(__ldcg(node + 3 + k), __ldcg(node + 9 + k));
        }
        self = p;
        p = parent_node[p];
    }
}

__global__ void k_depth(const int* __restrict__ parent_node, const int* __restrict__ parent_leaf, int n,
                        unsigned int* __restrict__ depth) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || n < 2) return;
    unsigned int d = 1;
    int p = parent_leaf[i];
    while (p > 0 && d < 4096u) {
        p = parent_node[p];
        ++d;
    }
    atomicMax(depth, d);
}

// Depth of every internal node (root 0); even-depth nodes become 4-wide nodes.
__global__ void k_node_depth(const int* __restrict__ parent_node, int n_int, int64_t* __restrict__ flag) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    int d = 0, p = i;
    while (p > 0 && d < 4096) {
        p = parent_node[p];
        ++d;
    }
    flag[i] = (d & 1) == 0 ? 1 : 0;
}

constexpr int LINK_EMPTY = (int)0x80000000;

__device__ __forceinline__ void child_box(const float* node, int side, float lo[3], float hi[3]) {
    const float* p = node + 6 * side;
    lo[0] = p[0]; lo[1] = p[1]; lo[2] = p[2];
    hi[0] = p[3]; hi[1] = p[4]; hi[2] = p[5];
}

__global__ void k_collapse4(const float4* __restrict__ nodes, int n_int, const int64_t* __restrict__ incl,
                            float4* __restrict__ nodes4) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_int) return;
    const int64_t before = i > 0 ? incl[i - 1] : 0;
    if (incl[i] == before) return;                    // odd depth: absorbed by its parent
    const int j = (int)before;                        // index of this 4-wide node
    const float* bn = reinterpret_cast<const float*>(nodes + 4 * i);
    float lo[4][3], hi[4][3];
    int link[4];
    int m = 0;
    for (int side = 0; side < 2; ++side) {
        const int c = __float_as_int(bn[12 + side]);
        if (c < 0) {
            child_box(bn, side, lo[m], hi[m]);
            link[m++] = c;
        } else {
            const float* cn = reinterpret_cast<const float*>(nodes + 4 * c);
            for (int s2 = 0; s2 < 2; ++s2) {
                const int g = __float_as_int(cn[12 + s2]);
                child_box(cn, s2, lo[m], hi[m]);
                link[m++] = g < 0 ? g : (int)(g > 0 ? incl[g - 1] : 0);
            }
        }
    }
    for (; m < 4; ++m) {
        for (int k = 0; k < 3; ++k) lo[m][k] = hi[m][k] = 1e30f;   // a box no segment reaches
        link[m] = LINK_EMPTY;
    }
    float4* o = nodes4 + 8 * (size_t)j;
    o[0] = make_float4(lo[0][0], lo[1][0], lo[2][0], lo[3][0]);
    o[1] = make_float4(hi[0][0], hi[1][0], hi[2][0], hi[3][0]);
    o[2] = make_float4(lo[0][1], lo[1][1], lo[2][1], lo[3][1]);
    o[3] = make_float4(hi[0][1], hi[1][1], hi[2][1], hi[3][1]);
    o[4] = make_float4(lo[0][2], lo[1][2], lo[2][2], lo[3][2]);
    o[5] = make_float4(hi[0][2], hi[1][2], hi[2][2], hi[3][2]);
    o[6] = make_float4(__int_as_float(link[0]), __int_as_float(link[1]), __int_as_float(link[2]),
                       __int_as_float(link[3]));
    o[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// ---- PLOC: parallel locally-ordered clustering (Meister & Bittner, TVCG 2018) ----------------
// Clusters start as the Morton-ordered leaves. Each round, every cluster finds the cluster within
// +-R positions whose union box has the smallest surface area; mutual nearest neighbours merge
// into a new node (the lower position keeps the merged cluster), and the array is compacted.
// Node indices are handed out downwards from n - 2, so the last merge -- the root -- is node 0.

struct Box6 {
    float lo[3], hi[3];
};

__device__ __forceinline__ float union_area(const float4 al, const float4 ah, const float4 bl, const float4 bh) {
    const float dx = fmaxf(ah.x, bh.x) - fminf(al.x, bl.x);
    const float dy = fmaxf(ah.y, bh.y) - fminf(al.y, bl.y);
    const float dz = fmaxf(ah.z, bh.z) - fminf(al.z, bl.z);
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_ploc_init(const float4* __restrict__ tri_canon, const uint32_t* __restrict__ order, int n,
                            const unsigned int* __restrict__ bounds, int* __restrict__ cid, float4* __restrict__ blo,
                            float4* __restrict__ bhi, float4* __restrict__ bvh_tris) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t t = order[i];
    float4 a = tri_canon[3 * t], b = tri_canon[3 * t + 1], c = tri_canon[3 * t + 2];
    bvh_tris[3 * i + 0] = make_float4(a.x, a.y, a.z, __uint_as_float(t));
    bvh_tris[3 * i + 1] = b;
    bvh_tris[3 * i + 2] = c;
    float big = 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k) big = fmaxf(big, fmaxf(fabsf(ord2f(bounds[6 + k])), fabsf(ord2f(bounds[9 + k]))));
    const float margin = big * (1.0f / 524288.0f) + 1e-30f;
    blo[i] = make_float4(fminf(fminf(a.x, b.x), c.x) - margin, fminf(fminf(a.y, b.y), c.y) - margin,
                         fminf(fminf(a.z, b.z), c.z) - margin, 0.f);
    bhi[i] = make_float4(fmaxf(fmaxf(a.x, b.x), c.x) + margin, fmaxf(fmaxf(a.y, b.y), c.y) + margin,
                         fmaxf(fmaxf(a.z, b.z), c.z) + margin, 0.f);
    cid[i] = ~i;
}

template <int R>
__global__ void __launch_bounds__(256) k_ploc_nn(const float4* __restrict__ blo, const float4* __restrict__ bhi,
                                                 int m, int* __restrict__ nn) {
    __shared__ float4 sl[256 + 2 * R], sh[256 + 2 * R];
    const int b0 = blockIdx.x * 256;
    for (int k = threadIdx.x; k < 256 + 2 * R; k += 256) {
        const int g = b0 - R + k;
        if (g >= 0 && g < m) {
            sl[k] = blo[g];
            sh[k] = bhi[g];
        }
    }
    __syncthreads();
    const int i = b0 + threadIdx.x;
    if (i >= m) return;
    const float4 al = sl[threadIdx.x + R], ah = sh[threadIdx.x + R];
    float best = INFINITY;
    int bj = -1;
    for (int d = -R; d <= R; ++d) {
        const int j = i + d;
        if (d == 0 || j < 0 || j >= m) continue;
        const float a = union_area(al, ah, sl[threadIdx.x + R + d], sh[threadIdx.x + R + d]);
        if (a < best || (a == best && j < bj)) {
            best = a;
            bj = j;
        }
    }
    nn[i] = bj;
}

__global__ void k_ploc_merge(int m, const int* __restrict__ nn, int* __restrict__ cid, float4* __restrict__ blo,
                             float4* __restrict__ bhi, int64_t* __restrict__ keep, int* __restrict__ counter,
                             float4* __restrict__ nodes, int* __restrict__ parent_node, int* __restrict__ parent_leaf) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int j = nn[i];
    const bool mutual = j >= 0 && nn[j] == i;
    if (!mutual) {
        keep[i] = 1;
        return;
    }
    if (i > j) {   // the lower position builds the node and keeps the merged cluster
        keep[i] = 0;
        return;
    }
    const int k = atomicSub(counter, 1) - 1;
    const float4 al = blo[i], ah = bhi[i], bl = blo[j], bh = bhi[j];
    const int ci = cid[i], cj = cid[j];
    float* node = reinterpret_cast<float*>(nodes + 4 * k);
    node[0] = al.x; node[1] = al.y; node[2] = al.z; node[3] = ah.x; node[4] = ah.y; node[5] = ah.z;
    node[6] = bl.x; node[7] = bl.y; node[8] = bl.z; node[9] = bh.x; node[10] = bh.y; node[11] = bh.z;
    nodes[4 * k + 3] = make_float4(__int_as_float(ci), __int_as_float(cj), 0.f, 0.f);
    if (ci < 0) parent_leaf[~ci] = k; else parent_node[ci] = k;
    if (cj < 0) parent_leaf[~cj] = k; else parent_node[cj] = k;
    // position j is only read by its own thread (which returns above), so i may be rewritten here
    cid[i] = k;
    blo[i] = make_float4(fminf(al.x, bl.x), fminf(al.y, bl.y), fminf(al.z, bl.z), 0.f);
    bhi[i] = make_float4(fmaxf(ah.x, bh.x), fmaxf(ah.y, bh.y), fmaxf(ah.z, bh.z), 0.f);
    keep[i] = 1;
}

__global__ void k_ploc_compact(int m, const int64_t* __restrict__ incl, const int* __restrict__ cid,
                               const float4* __restrict__ blo, const float4* __restrict__ bhi, int* __restrict__ cid2,
                               float4* __restrict__ blo2, float4* __restrict__ bhi2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const int64_t before = i > 0 ? incl[i - 1] : 0;
    if (incl[i] == before) return;
    cid2[before] = cid[i];
    blo2[before] = blo[i];
    bhi2[before] = bhi[i];
}

// ---- depth-first node layout ------------------------------------------------------------------
// Renumber the internal nodes in depth-first order (a node, then its left subtree, then its right
// subtree), so that a node's left child directly follows it in memory and often shares its
// cache line. leaves[v] = number of leaves below v (bottom-up); the index of v is the sum, over
// the path from the root, of 1 per step plus the left sibling's internal-node count when the
// step goes right.
// Leaves under every internal node, bottom-up: the second of a node's two children to arrive
// sums the children's counts and climbs on (one atomic per node, as in the box refit).
__global__ void k_leaf_counts(const int* __restrict__ parent_leaf, const int* __restrict__ parent_node,
                              const float4* __restrict__ nodes, int n, unsigned int* __restrict__ leaves,
                              unsigned int* __restrict__ flags) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int p = parent_leaf[i];
    int guard = 0;
    while (p >= 0 && guard++ < 4096) {
        __threadfence();
        if (atomicAdd(&flags[p], 1u) == 0u) return;   // the sibling finishes this node
        __threadfence();
        const float4 l = nodes[4 * p + 3];
        const int a = __float_as_int(l.x), b = __float_as_int(l.y);
        const unsigned int ca = a >= 0 ? __ldcg(&leaves[a]) : 1u;
        const unsigned int cb = b >= 0 ? __ldcg(&leaves[b]) : 1u;
        leaves[p] = ca + cb;
        p = p > 0 ? parent_node[p] : -1;
    }
}

__global__ void k_dfs_index(const float4* __restrict__ nodes, const int* __restrict__ parent_node,
                            const unsigned int* __restrict__ leaves, int n_int, int* __restrict__ dfs) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_int) return;
    int idx = 0, u = v, guard = 0;
    while (u > 0 && guard++ < 4096) {
        const int p = parent_node[u];
        const float4 l = nodes[4 * p + 3];
        const int left = __float_as_int(l.x);
        idx += 1;
        if (left != u) idx += left >= 0 ? (int)leaves[left] - 1 : 0;   // internal nodes of the left subtree
        u = p;
    }
    dfs[v] = idx;
}

__global__ void k_dfs_remap(const float4* __restrict__ nodes, const int* __restrict__ dfs, int n_int,
                            float4* __restrict__ out) {
    int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_int) return;
    const int d = dfs[v];
    out[4 * d + 0] = nodes[4 * v + 0];
    out[4 * d + 1] = nodes[4 * v + 1];
    out[4 * d + 2] = nodes[4 * v + 2];
    const float4 l = nodes[4 * v + 3];
    const int a = __float_as_int(l.x), b = __float_as_int(l.y);
    out[4 * d + 3] = make_float4(__int_as_float(a >= 0 ? dfs[a] : a), __int_as_float(b >= 0 ? dfs[b] : b), 0.f, 0.f);
}

// ---- dynamic scenes: re-pose every mesh, refit the boxes over the unchanged topology ----------
// Mesh-local triangle vertices in stored (mesh) order, kept for re-posing.
__global__ void k_gather_local(const float* __restrict__ v, const uint32_t* __restrict__ idx, uint32_t nt,
                               uint32_t nv, uint32_t tri_base, float4* __restrict__ tri_local) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        uint32_t vi = idx[3 * t + k];
        if (vi >= nv) vi = 0;   // the world gather of the same mesh reports the bad index
        tri_local[3 * (tri_base + t) + k] = make_float4(v[3 * vi], v[3 * vi + 1], v[3 * vi + 2], 0.f);
    }
}

// World triangles of a new pose: the transform of k_transform (same FP64 operation order, so a
// pose equal to the build's transforms reproduces the built triangles bit for bit), one thread
// per triangle; scene bounds as in k_gather (centroid box in [0, 6), vertex box in [6, 12)).
__global__ void k_pose(const float4* __restrict__ tri_local, const uint32_t* __restrict__ tri_mesh,
                       const double* __restrict__ xf, uint32_t nt, float4* __restrict__ tri_canon,
                       unsigned int* __restrict__ bounds) {
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float lo[6], hi[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) { lo[c] = INFINITY; hi[c] = -INFINITY; }
    if (t < nt) {
        const double* M = xf + 12 * tri_mesh[t];
        float w[9];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 p = tri_local[3 * t + k];
            const double x = p.x, y = p.y, z = p.z;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                double a = __dadd_rn(__dmul_rn(M[4 * r + 0], x), __dmul_rn(M[4 * r + 1], y));
                a = __dadd_rn(a, __dmul_rn(M[4 * r + 2], z));
                a = __dadd_rn(a, M[4 * r + 3]);
                w[3 * k + r] = __double2float_rn(a);
            }
            tri_canon[3 * t + k] = make_float4(w[3 * k], w[3 * k + 1], w[3 * k + 2], 0.f);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            lo[a] = hi[a] = (w[a] + w[3 + a] + w[6 + a]) * (1.f / 3.f);
            lo[3 + a] = fminf(fminf(w[a], w[3 + a]), w[6 + a]);
            hi[3 + a] = fmaxf(fmaxf(w[a], w[3 + a]), w[6 + a]);
        }
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) {
        for (int o = 16; o > 0; o >>= 1) {
            lo[c] = fminf(lo[c], __shfl_xor_sync(0xffffffffu, lo[c], o));
            hi[c] = fmaxf(hi[c], __shfl_xor_sync(0xffffffffu, hi[c], o));
        }
    }
    if ((threadIdx.x & 31) == 0 && blockIdx.x * blockDim.x + (threadIdx.x & ~31u) < nt) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(&bounds[a], f2ord(lo[a]));
            atomicMax(&bounds[3 + a], f2ord(hi[a]));
            atomicMin(&bounds[6 + a], f2ord(lo[3 + a]));
            atomicMax(&bounds[9 + a], f2ord(hi[3 + a]));
        }
    }
}

// Triangle id of every leaf slot (v0.w of the leaf-order copy).
__global__ void k_leaf_order(const float4* __restrict__ bvh_tris, uint32_t n, uint32_t* __restrict__ order) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) order[i] = __float_as_uint(bvh_tris[3 * i].w);
}

// Parents in the final node layout, from the child links (root: -1 from the memset).
__global__ void k_final_parents(const float4* __restrict__ nodes, int n_int, int n_leaves,
                                int* __restrict__ parent_node, int* __restrict__ parent_leaf) {
    int p = blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n_int) return;
    const float4 l = nodes[4 * p + 3];
    const int c[2] = {__float_as_int(l.x), __float_as_int(l.y)};
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        if (c[k] >= 0) {
            if (c[k] < n_int) parent_node[c[k]] = p;
        } else if (~c[k] < n_leaves) {
            parent_leaf[~c[k]] = p;
        }
    }
}

}  // namespace

// Inverse affine maps (world -> mesh-local, row-major 3 x 4) of row-major 4 x 4 transforms, by the
// adjugate in FP64; false if any transform is singular (its rows are left zero).
static bool mesh_inverses(const double* xf, uint32_t n_meshes, std::vector<double>& inv) {
    inv.assign(12 * (size_t)n_meshes, 0.0);
    bool ok = true;
    for (uint32_t m = 0; m < n_meshes; ++m) {
        const double* M = xf + 16 * m;
        const double a = M[0], b = M[1], c = M[2], d = M[4], e2 = M[5], f = M[6], g = M[8], h = M[9], k = M[10];
        const double det = a * (e2 * k - f * h) - b * (d * k - f * g) + c * (d * h - e2 * g);
        if (!(std::fabs(det) > 1e-300) || !std::isfinite(det)) {
            ok = false;
            continue;
        }
        const double r[9] = {(e2 * k - f * h) / det, (c * h - b * k) / det, (b * f - c * e2) / det,
                             (f * g - d * k) / det,  (a * k - c * g) / det,  (c * d - a * f) / det,
                             (d * h - e2 * g) / det, (b * g - a * h) / det,  (a * e2 - b * d) / det};
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) inv[12 * m + 4 * i + j] = r[3 * i + j];
            inv[12 * m + 4 * i + 3] = -(r[3 * i] * M[3] + r[3 * i + 1] * M[7] + r[3 * i + 2] * M[11]);
        }
    }
    return ok;
}

static gm_status build_scene(gm_ctx* ctx, const gm_mesh_desc* meshes, uint32_t n_meshes, int builder,
                             bool dynamic, int ploc_radius, gm_stream stream, gm_scene** out) {
    if (!ctx || !meshes || !out || n_meshes == 0)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene: null argument or no meshes");
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    uint64_t nt64 = 0;
    for (uint32_t m = 0; m < n_meshes; ++m) {
        const gm_mesh_desc& d = meshes[m];
        if (d.n_tris > 0 && (!d.vertices || !d.indices || d.n_verts == 0))
            return gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene: mesh " + std::to_string(m) + " has triangles but no vertices/indices");
        for (int k = 0; k < 16; ++k)
            if (!std::isfinite(d.transform[k]))
                return gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene: non-finite transform");
        nt64 += d.n_tris;
    }
    if (nt64 == 0) return gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene: the scene has no triangles");
    if (nt64 > 0x7fffffffu) return gm_set_error(GM_ERR_UNSUPPORTED, "gm_build_scene: more than 2^31-1 triangles");
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    const uint32_t nt = (uint32_t)nt64;

    gm_scene* sc = new gm_scene();
    sc->ctx = ctx;
    sc->n_tris = nt;
    sc->n_meshes = n_meshes;
    std::vector<void*> tmp;
    auto fail = [&](gm_status st) {
        for (void* p : tmp) cudaFreeAsync(p, s);
        gm_scene_free(sc);
        return st;
    };
    gm_status st;
#define SC_ALLOC(ptr, bytes) \
    if ((st = gm_alloc((void**)&(ptr), (bytes), s)) != GM_OK) return fail(st)
#define TMP_ALLOC(ptr, bytes)                                          \
    do {                                                               \
        if ((st = gm_alloc((void**)&(ptr), (bytes), s)) != GM_OK) return fail(st); \
        tmp.push_back((void*)(ptr));                                   \
    } while (0)

    SC_ALLOC(sc->tri_canon, sizeof(float4) * 3 * (size_t)nt);
    SC_ALLOC(sc->tri_mesh, sizeof(uint32_t) * (size_t)nt);
    SC_ALLOC(sc->mesh_object, sizeof(uint32_t) * n_meshes);
    SC_ALLOC(sc->bvh_tris, sizeof(float4) * 3 * (size_t)nt);
    if (dynamic) SC_ALLOC(sc->tri_local, sizeof(float4) * 3 * (size_t)nt);
    if (nt > 1) SC_ALLOC(sc->nodes, sizeof(float4) * 4 * (size_t)(nt - 1));
    unsigned int* bounds = nullptr;
    int* err = nullptr;
    TMP_ALLOC(bounds, sizeof(unsigned int) * 16);
    err = ctx->dev_err;
    k_bounds_init<<<1, 32, 0, s>>>(bounds);
    int launches = 1;

    std::vector<uint32_t> objs(n_meshes);
    uint32_t base = 0;
    for (uint32_t m = 0; m < n_meshes; ++m) {
        const gm_mesh_desc& d = meshes[m];
        objs[m] = d.object_id;
        if (d.n_tris == 0) continue;
        void *dv = nullptr, *di = nullptr;
        bool ov = false, oi = false;
        if ((st = gm_stage_to_device(d.vertices, sizeof(float) * 3 * (size_t)d.n_verts, s, &dv, &ov)) != GM_OK) return fail(st);
        if (ov) tmp.push_back(dv);
        if ((st = gm_stage_to_device(d.indices, sizeof(uint32_t) * 3 * (size_t)d.n_tris, s, &di, &oi)) != GM_OK) return fail(st);
        if (oi) tmp.push_back(di);
        float* wv = nullptr;
        TMP_ALLOC(wv, sizeof(float) * 3 * (size_t)d.n_verts);
        Mat16 M;
        memcpy(M.m, d.transform, sizeof(M.m));
        k_transform<<<gm_div_up(d.n_verts, 256), 256, 0, s>>>((const float*)dv, d.n_verts, M, wv);
        k_gather<<<gm_div_up(d.n_tris, 256), 256, 0, s>>>(wv, (const uint32_t*)di, d.n_tris, d.n_verts, base, m,
                                                          sc->tri_canon, sc->tri_mesh, bounds, err);
        launches += 2;
        if (dynamic) {
            k_gather_local<<<gm_div_up(d.n_tris, 256), 256, 0, s>>>((const float*)dv, (const uint32_t*)di, d.n_tris,
                                                                    d.n_verts, base, sc->tri_local);
            ++launches;
        }
        base += d.n_tris;
    }
    GM_TRY_CUDA(cudaMemcpyAsync(sc->mesh_object, objs.data(), sizeof(uint32_t) * n_meshes, cudaMemcpyHostToDevice, s));
    // world -> mesh-local maps for the export format (affine inverse in FP64)
    {
        std::vector<double> xf(16 * (size_t)n_meshes);
        for (uint32_t m = 0; m < n_meshes; ++m) memcpy(&xf[16 * m], meshes[m].transform, sizeof(double) * 16);
        std::vector<double> inv;
        sc->mesh_inv_ok = mesh_inverses(xf.data(), n_meshes, inv);
        SC_ALLOC(sc->mesh_inv, sizeof(double) * 12 * n_meshes);
        GM_TRY_CUDA(cudaMemcpyAsync(sc->mesh_inv, inv.data(), sizeof(double) * 12 * n_meshes, cudaMemcpyHostToDevice, s));
        GM_TRY_CUDA(cudaStreamSynchronize(s));   // inv is a host temporary
    }

    uint64_t* keys = nullptr;
    uint32_t* order = nullptr;
    int *parent_node = nullptr, *parent_leaf = nullptr;
    unsigned int *flags = nullptr, *depth = nullptr;
    TMP_ALLOC(keys, sizeof(uint64_t) * nt);
    TMP_ALLOC(order, sizeof(uint32_t) * nt);
    TMP_ALLOC(parent_leaf, sizeof(int) * nt);
    TMP_ALLOC(parent_node, sizeof(int) * (nt > 1 ? nt - 1 : 1));
    TMP_ALLOC(flags, sizeof(unsigned int) * (nt > 1 ? nt - 1 : 1));
    TMP_ALLOC(depth, sizeof(unsigned int));
    GM_TRY_CUDA(cudaMemsetAsync(flags, 0, sizeof(unsigned int) * (nt > 1 ? nt - 1 : 1), s));
    // -1 everywhere: a link the hierarchy step did not write stops the refit instead of escaping
    GM_TRY_CUDA(cudaMemsetAsync(parent_leaf, 0xff, sizeof(int) * nt, s));
    GM_TRY_CUDA(cudaMemsetAsync(parent_node, 0xff, sizeof(int) * (nt > 1 ? nt - 1 : 1), s));
    GM_TRY_CUDA(cudaMemsetAsync(depth, 0, sizeof(unsigned int), s));
    k_morton<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->tri_canon, nt, bounds, keys, order);
    if ((st = gm_radix_sort_u64(keys, order, nt, 63, s, &launches)) != GM_OK) return fail(st);
    if (builder == GM_BUILD_PLOC && nt > 1) {
        int *cid = nullptr, *cid2 = nullptr, *nn = nullptr, *counter = nullptr;
        float4 *blo = nullptr, *bhi = nullptr, *blo2 = nullptr, *bhi2 = nullptr;
        int64_t* keep = nullptr;
        TMP_ALLOC(cid, sizeof(int) * nt);
        TMP_ALLOC(cid2, sizeof(int) * nt);
        TMP_ALLOC(nn, sizeof(int) * nt);
        TMP_ALLOC(counter, sizeof(int));
        TMP_ALLOC(blo, sizeof(float4) * nt);
        TMP_ALLOC(bhi, sizeof(float4) * nt);
        TMP_ALLOC(blo2, sizeof(float4) * nt);
        TMP_ALLOC(bhi2, sizeof(float4) * nt);
        TMP_ALLOC(keep, sizeof(int64_t) * nt);
        k_ploc_init<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->tri_canon, order, (int)nt, bounds, cid, blo, bhi,
                                                       sc->bvh_tris);
        const int first = (int)nt - 1;
        GM_TRY_CUDA(cudaMemcpyAsync(counter, &first, sizeof(int), cudaMemcpyHostToDevice, s));
        launches += 1;
        int m = (int)nt;
        int64_t* m_host = nullptr;
        GM_TRY_CUDA(cudaMallocHost(&m_host, sizeof(int64_t)));
        int rounds = 0;
        while (m > 1 && rounds < 4096) {
            ++rounds;
            switch (ploc_radius) {
                case 4: k_ploc_nn<4><<<gm_div_up(m, 256), 256, 0, s>>>(blo, bhi, m, nn); break;
                case 16: k_ploc_nn<16><<<gm_div_up(m, 256), 256, 0, s>>>(blo, bhi, m, nn); break;
                case 32: k_ploc_nn<32><<<gm_div_up(m, 256), 256, 0, s>>>(blo, bhi, m, nn); break;
                case 64: k_ploc_nn<64><<<gm_div_up(m, 256), 256, 0, s>>>(blo, bhi, m, nn); break;
                default: k_ploc_nn<8><<<gm_div_up(m, 256), 256, 0, s>>>(blo, bhi, m, nn); break;
            }
            k_ploc_merge<<<gm_div_up(m, 256), 256, 0, s>>>(m, nn, cid, blo, bhi, keep, counter, sc->nodes, parent_node,
                                                           parent_leaf);
            if ((st = gm_inclusive_scan_i64(keep, (uint32_t)m, s, &launches)) != GM_OK) {
                cudaFreeHost(m_host);
                return fail(st);
            }
            k_ploc_compact<<<gm_div_up(m, 256), 256, 0, s>>>(m, keep, cid, blo, bhi, cid2, blo2, bhi2);
            launches += 3;
            std::swap(cid, cid2);
            std::swap(blo, blo2);
            std::swap(bhi, bhi2);
            cudaError_t ce = cudaMemcpyAsync(m_host, keep + (m - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) {
                cudaFreeHost(m_host);
                return fail(gm_cuda_error(ce, "gm_build_scene (clustering)"));
            }
            if (*m_host >= m) {   // no mutual pair: cannot happen with consistent tie-breaking
                cudaFreeHost(m_host);
                return fail(gm_set_error(GM_ERR_INTERNAL, "gm_build_scene: clustering made no progress"));
            }
            m = (int)*m_host;
        }
        cudaFreeHost(m_host);
    } else {
        if (nt > 1) k_hierarchy<<<gm_div_up(nt - 1, 256), 256, 0, s>>>(keys, (int)nt, sc->nodes, parent_node, parent_leaf);
        k_refit<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->tri_canon, order, (int)nt, sc->nodes, parent_node, parent_leaf,
                                                    flags, bounds, sc->bvh_tris);
        launches += (nt > 1 ? 2 : 1);
    }
    k_depth<<<gm_div_up(nt, 256), 256, 0, s>>>(parent_node, parent_leaf, (int)nt, depth);
    launches += 2;
    ctx->launches += launches;
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_build_scene launch"));
    unsigned int hb[16] = {0};
    unsigned int hdepth = 0;
    int herr = 0;
    if ((e = cudaMemcpyAsync(hb, bounds, sizeof(unsigned int) * 12, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&hdepth, depth, sizeof(unsigned int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return fail(gm_cuda_error(e, "gm_build_scene"));
    int* parent_node_keep = parent_node;
    if (herr == GM_DEV_BAD_INDEX) {
        cudaMemsetAsync(ctx->dev_err, 0, sizeof(int), s);
        return fail(gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene: a vertex index is out of range"));
    }
    auto dec = [](unsigned int o) {
        unsigned int b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
        float f;
        memcpy(&f, &b, 4);
        return f;
    };
    for (int k = 0; k < 3; ++k) {
        sc->box_lo[k] = dec(hb[6 + k]);
        sc->box_hi[k] = dec(hb[9 + k]);
        if (!std::isfinite(sc->box_lo[k]) || !std::isfinite(sc->box_hi[k]))
            return fail(gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene: non-finite vertex"));
    }
    sc->depth = nt > 1 ? hdepth : 0;
    if (sc->depth > 64)
        return fail(gm_set_error(GM_ERR_UNSUPPORTED, "gm_build_scene: BVH deeper than 64 levels (" +
                                                         std::to_string(sc->depth) + ")"));
    if (nt > 1) {
        const uint32_t n_int = nt - 1;
        int64_t* incl = nullptr;
        TMP_ALLOC(incl, sizeof(int64_t) * n_int);
        k_node_depth<<<gm_div_up(n_int, 256), 256, 0, s>>>(parent_node_keep, (int)n_int, incl);
        launches = 1;
        if ((st = gm_inclusive_scan_i64(incl, n_int, s, &launches)) != GM_OK) return fail(st);
        int64_t n4 = 0;
        if ((e = cudaMemcpyAsync(&n4, incl + (n_int - 1), sizeof(int64_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
            (e = cudaStreamSynchronize(s)) != cudaSuccess)
            return fail(gm_cuda_error(e, "gm_build_scene (4-wide count)"));
        sc->n4 = (uint32_t)n4;
        SC_ALLOC(sc->nodes4, sizeof(float4) * 8 * (size_t)sc->n4);
        k_collapse4<<<gm_div_up(n_int, 256), 256, 0, s>>>(sc->nodes, (int)n_int, incl, sc->nodes4);
        ++launches;
        ctx->launches += launches;
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_build_scene collapse"));
    }
    if (kDfsLayout && nt > 2) {
        const int n_int = (int)nt - 1;
        unsigned int* leaves = nullptr;
        int* dfs = nullptr;
        unsigned int* arrived = nullptr;
        float4* reordered = nullptr;
        TMP_ALLOC(leaves, sizeof(unsigned int) * n_int);
        TMP_ALLOC(dfs, sizeof(int) * n_int);
        TMP_ALLOC(arrived, sizeof(unsigned int) * n_int);
        GM_TRY_CUDA(cudaMemsetAsync(leaves, 0, sizeof(unsigned int) * n_int, s));
        GM_TRY_CUDA(cudaMemsetAsync(arrived, 0, sizeof(unsigned int) * n_int, s));
        if ((st = gm_alloc((void**)&reordered, sizeof(float4) * 4 * (size_t)n_int, s)) != GM_OK) return fail(st);
        k_leaf_counts<<<gm_div_up(nt, 256), 256, 0, s>>>(parent_leaf, parent_node_keep, sc->nodes, (int)nt, leaves,
                                                         arrived);
        k_dfs_index<<<gm_div_up(n_int, 256), 256, 0, s>>>(sc->nodes, parent_node_keep, leaves, n_int, dfs);
        k_dfs_remap<<<gm_div_up(n_int, 256), 256, 0, s>>>(sc->nodes, dfs, n_int, reordered);
        ctx->launches += 3;
        cudaFreeAsync(sc->nodes, s);
        sc->nodes = reordered;
        e = cudaGetLastError();
        if (e != cudaSuccess) return fail(gm_cuda_error(e, "gm_build_scene layout"));
    }
    for (void* p : tmp) cudaFreeAsync(p, s);
    tmp.clear();
    *out = sc;
    return GM_OK;
#undef SC_ALLOC
#undef TMP_ALLOC
}

extern "C" gm_status gm_build_scene(gm_ctx* ctx, const gm_mesh_desc* meshes, uint32_t n_meshes, gm_stream stream,
                                    gm_scene** out) {
    return build_scene(ctx, meshes, n_meshes, GM_BUILD_DEFAULT, false, kPlocRadius, stream, out);
}

extern "C" gm_status gm_build_scene_opts(gm_ctx* ctx, const gm_mesh_desc* meshes, uint32_t n_meshes,
                                         const gm_build_opts* opts, gm_stream stream, gm_scene** out) {
    const int b = opts ? opts->builder : GM_BUILD_DEFAULT;
    if (b != GM_BUILD_LBVH && b != GM_BUILD_PLOC)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene_opts: unknown builder");
    const int r = opts && opts->ploc_radius ? opts->ploc_radius : kPlocRadius;
    if (r != 4 && r != 8 && r != 16 && r != 32 && r != 64)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_build_scene_opts: ploc_radius must be 4, 8, 16, 32 or 64");
    return build_scene(ctx, meshes, n_meshes, b, opts && opts->dynamic != 0, r, stream, out);
}

extern "C" gm_status gm_scene_pose(gm_scene* sc, const double* transforms, gm_stream stream) {
    if (!sc || !transforms) return gm_set_error(GM_ERR_INVALID_ARG, "gm_scene_pose: null argument");
    if (!sc->tri_local)
        return gm_set_error(GM_ERR_INVALID_ARG, "gm_scene_pose: the scene was not built with gm_build_opts.dynamic");
    const uint32_t nm = sc->n_meshes, nt = sc->n_tris;
    for (size_t k = 0; k < 16 * (size_t)nm; ++k)
        if (!std::isfinite(transforms[k])) return gm_set_error(GM_ERR_INVALID_ARG, "gm_scene_pose: non-finite transform");
    cudaStream_t s = (cudaStream_t)stream;
    gm_ctx* ctx = sc->ctx;
    GM_TRY_CUDA(cudaSetDevice(ctx->device));
    std::vector<double> xf12(12 * (size_t)nm);
    for (uint32_t m = 0; m < nm; ++m) memcpy(&xf12[12 * m], transforms + 16 * m, sizeof(double) * 12);
    std::vector<double> inv;
    const bool inv_ok = mesh_inverses(transforms, nm, inv);
    std::vector<void*> tmp;
    auto done = [&](gm_status st) {
        for (void* p : tmp) cudaFreeAsync(p, s);
        return st;
    };
    gm_status st;
#define POSE_TMP(ptr, bytes)                                                          \
    do {                                                                              \
        if ((st = gm_alloc((void**)&(ptr), (bytes), s)) != GM_OK) return done(st);    \
        tmp.push_back((void*)(ptr));                                                  \
    } while (0)
    double* d_xf = nullptr;
    unsigned int* bounds = nullptr;
    uint32_t* order = nullptr;
    int *parent_node = nullptr, *parent_leaf = nullptr;
    unsigned int* flags = nullptr;
    const uint32_t n_int = nt > 1 ? nt - 1 : 1;
    POSE_TMP(d_xf, sizeof(double) * 12 * nm);
    POSE_TMP(bounds, sizeof(unsigned int) * 16);
    POSE_TMP(order, sizeof(uint32_t) * nt);
    POSE_TMP(parent_node, sizeof(int) * n_int);
    POSE_TMP(parent_leaf, sizeof(int) * nt);
    POSE_TMP(flags, sizeof(unsigned int) * n_int);
#undef POSE_TMP
    cudaError_t e;
    if ((e = cudaMemcpyAsync(d_xf, xf12.data(), sizeof(double) * 12 * nm, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(sc->mesh_inv, inv.data(), sizeof(double) * 12 * nm, cudaMemcpyHostToDevice, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(parent_node, 0xff, sizeof(int) * n_int, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(parent_leaf, 0xff, sizeof(int) * nt, s)) != cudaSuccess ||
        (e = cudaMemsetAsync(flags, 0, sizeof(unsigned int) * n_int, s)) != cudaSuccess)
        return done(gm_cuda_error(e, "gm_scene_pose"));
    k_bounds_init<<<1, 32, 0, s>>>(bounds);
    k_pose<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->tri_local, sc->tri_mesh, d_xf, nt, sc->tri_canon, bounds);
    k_leaf_order<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->bvh_tris, nt, order);
    int launches = 3;
    if (nt > 1) {
        k_final_parents<<<gm_div_up(nt - 1, 256), 256, 0, s>>>(sc->nodes, (int)(nt - 1), (int)nt, parent_node,
                                                               parent_leaf);
        ++launches;
    }
    // leaf-order triangles rewritten from the posed ones, then the boxes bottom-up (the
    // hierarchy and its depth are unchanged)
    k_refit<<<gm_div_up(nt, 256), 256, 0, s>>>(sc->tri_canon, order, (int)nt, sc->nodes, parent_node, parent_leaf,
                                                flags, bounds, sc->bvh_tris);
    ++launches;
    unsigned int hb[12] = {0};
    if ((e = cudaGetLastError()) != cudaSuccess ||
        (e = cudaMemcpyAsync(hb, bounds, sizeof(hb), cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return done(gm_cuda_error(e, "gm_scene_pose"));
    ctx->launches += launches;
    auto dec = [](unsigned int o) {
        unsigned int b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
        float f;
        memcpy(&f, &b, 4);
        return f;
    };
    for (int k = 0; k < 3; ++k) {
        sc->box_lo[k] = dec(hb[6 + k]);
        sc->box_hi[k] = dec(hb[9 + k]);
    }
    sc->mesh_inv_ok = inv_ok;
    // the 4-wide collapse holds the old boxes: drop it (the binary tree serves every variant)
    if (sc->nodes4) {
        cudaFreeAsync(sc->nodes4, s);
        sc->nodes4 = nullptr;
        sc->n4 = 0;
    }
    for (int k = 0; k < 3; ++k)
        if (!std::isfinite(sc->box_lo[k]) || !std::isfinite(sc->box_hi[k]))
            return done(gm_set_error(GM_ERR_INVALID_ARG, "gm_scene_pose: non-finite vertex"));
    return done(GM_OK);
}

extern "C" gm_status gm_scene_info(const gm_scene* sc, uint32_t* n_tris, uint32_t* bvh_depth) {
    if (!sc) return gm_set_error(GM_ERR_INVALID_ARG, "gm_scene_info: null scene");
    if (n_tris) *n_tris = sc->n_tris;
    if (bvh_depth) *bvh_depth = sc->depth;
    return GM_OK;
}

namespace {
__global__ void k_unpack_tris(const float4* __restrict__ t, uint32_t nt, float* __restrict__ out) {
    uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        float4 v = t[3 * i + k];
        out[9 * i + 3 * k + 0] = v.x;
        out[9 * i + 3 * k + 1] = v.y;
        out[9 * i + 3 * k + 2] = v.z;
    }
}
}  // namespace

extern "C" gm_status gm_scene_triangles(const gm_scene* sc, float* dst, gm_stream stream) {
    if (!sc || !dst) return gm_set_error(GM_ERR_INVALID_ARG, "gm_scene_triangles: null argument");
    cudaStream_t s = (cudaStream_t)stream;
    size_t bytes = sizeof(float) * 9 * (size_t)sc->n_tris;
    bool dev = gm_is_device_ptr(dst);
    float* tmp = dst;
    if (!dev) GM_TRY(gm_alloc((void**)&tmp, bytes, s));
    k_unpack_tris<<<gm_div_up(sc->n_tris, 256), 256, 0, s>>>(sc->tri_canon, sc->n_tris, tmp);
    sc->ctx->launches += 1;
    if (!dev) {
        gm_status st = gm_copy_out(dst, tmp, bytes, s);
        cudaFreeAsync(tmp, s);
        return st;
    }
    GM_TRY_CUDA(cudaGetLastError());
    return GM_OK;
}

extern "C" void gm_scene_free(gm_scene* sc) {
    if (!sc) return;
    cudaFree(sc->tri_canon);
    cudaFree(sc->tri_mesh);
    cudaFree(sc->mesh_object);
    cudaFree(sc->mesh_inv);
    cudaFree(sc->nodes);
    cudaFree(sc->nodes4);
    cudaFree(sc->bvh_tris);
    cudaFree(sc->tri_local);
    delete sc;
}
