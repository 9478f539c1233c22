/*
 * gm_oracle.c -- plain, slow, FP64 CPU oracle for surface-based gaze mapping
 * (Javerliat & Lavoue, "GPU accelerated surface-based gaze mapping for XR experiences").
 *
 * TEST INFRASTRUCTURE ONLY. This file is the reference that the CUDA library is checked
 * against. Only the tests, the package's smoke check and the benchmark's CPU-baseline leg
 * load it; the library never does. It shares no code, header, table or constant generator
 * with the CUDA path.
 *
 * Every step is written in the order the method defines it, with no blocking, fusion or
 * acceleration structure: areas and counts per triangle, one Philox evaluation per sample,
 * and for every sample x fixation pair the cone test, a brute-force occlusion test against
 * every triangle of the scene, and the duration-weighted Gaussian.
 *
 * Readings taken where the paper is silent (stated once here, used below):
 *  - area is measured in world space, after the mesh transform;
 *  - counts come from an exact fixed-point prefix of k*A (area-weighted count within one
 *    sample of k*A per triangle) instead of the integer grid resolution of Section 3.1.2;
 *  - sample positions are uniform in the triangle (Osada et al. 2002 map) from
 *    Philox4x32-10 (Salmon et al., SC'11) words;
 *  - d2 = |p x r^| (the scalar rejection of p from r in 3-D);
 *  - a pair contributes only when d1 > 0 and sigma_k <= 4 sigma (the 4 sigma cut-off of
 *    Fig. 4 and Section 3.3.2), inclusive;
 *  - occlusion is exact: the segment from the eye to (1 - eps_rel) of the way to the sample
 *    must not meet any triangle other than the sample's own (replaces the z-buffer +-eps
 *    comparison of Section 3.2.2);
 *  - duration t is in seconds; the normalising constant 1/(sigma sqrt(2 pi)) is kept as
 *    printed; a map whose maximum is 0 normalises to all zeros.
 *
 * Build: cc -O2 -std=c11 -ffp-contract=off -fno-fast-math -fPIC -shared -pthread.
 * -ffp-contract=off matters: the world transform and the FP64 areas must be the exact
 * sequence of correctly rounded operations written below.
 */
#define _POSIX_C_SOURCE 200809L
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORA_PI 3.14159265358979323846

/* ------------------------------------------------------------------------------------ */
/* World vertices: FP64 row-major 4x4 transform applied to FP32 mesh-local vertices,     */
/* rounded to FP32.  out = ((m0*x + m1*y) + m2*z) + m3 per row.                           */
/* ------------------------------------------------------------------------------------ */
void ora_world_vertices(const float* v, int64_t nv, const double* m, float* out)
{
    for (int64_t i = 0; i < nv; ++i) {
        double x = v[3 * i], y = v[3 * i + 1], z = v[3 * i + 2];
        for (int r = 0; r < 3; ++r) {
            double a = m[4 * r + 0] * x;
            double b = m[4 * r + 1] * y;
            double s = a + b;
            double c = m[4 * r + 2] * z;
            s = s + c;
            s = s + m[4 * r + 3];
            out[3 * i + r] = (float)s;
        }
    }
}

/* Gather world triangles (9 floats each) for several meshes concatenated in order.
 * verts/idx: all meshes' local vertices and (mesh-local) indices, back to back;
 * xf: 16 doubles per mesh. Returns 0, or -1 if an index is out of range. */
int ora_world_triangles(const float* verts, const uint32_t* idx, const double* xf,
                        const int64_t* n_verts, const int64_t* n_tris, int32_t n_meshes,
                        float* tri_out)
{
    int64_t voff = 0, toff = 0;
    for (int32_t mi = 0; mi < n_meshes; ++mi) {
        float* w = (float*)malloc(sizeof(float) * 3 * (size_t)(n_verts[mi] > 0 ? n_verts[mi] : 1));
        if (!w) return -2;
        ora_world_vertices(verts + 3 * voff, n_verts[mi], xf + 16 * mi, w);
        for (int64_t t = 0; t < n_tris[mi]; ++t) {
            for (int k = 0; k < 3; ++k) {
                uint32_t vi = idx[3 * (toff + t) + k];
                if ((int64_t)vi >= n_verts[mi]) { free(w); return -1; }
                for (int c = 0; c < 3; ++c) tri_out[9 * (toff + t) + 3 * k + c] = w[3 * vi + c];
            }
        }
        free(w);
        voff += n_verts[mi];
        toff += n_tris[mi];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Triangle area (Section 3.1.2). Primary: half the norm of the cross product of two     */
/* edges, FP64, in this exact order. Cross-check: Heron's formula as the paper prints it  */
/* (edge lengths a, b, c; semi-perimeter s; A = sqrt(s(s-a)(s-b)(s-c))).                 */
/* ------------------------------------------------------------------------------------ */
void ora_tri_areas(const float* tri, int64_t nt, double* area)
{
    for (int64_t i = 0; i < nt; ++i) {
        const float* t = tri + 9 * i;
        double e1x = (double)t[3] - (double)t[0], e1y = (double)t[4] - (double)t[1], e1z = (double)t[5] - (double)t[2];
        double e2x = (double)t[6] - (double)t[0], e2y = (double)t[7] - (double)t[1], e2z = (double)t[8] - (double)t[2];
        double cx = e1y * e2z - e1z * e2y;
        double cy = e1z * e2x - e1x * e2z;
        double cz = e1x * e2y - e1y * e2x;
        double n2 = (cx * cx + cy * cy) + cz * cz;
        area[i] = 0.5 * sqrt(n2);
    }
}

void ora_tri_areas_heron(const float* tri, int64_t nt, double* area)
{
    for (int64_t i = 0; i < nt; ++i) {
        const float* t = tri + 9 * i;
        double v0[3] = {t[0], t[1], t[2]}, v1[3] = {t[3], t[4], t[5]}, v2[3] = {t[6], t[7], t[8]};
        double a = sqrt((v1[0] - v0[0]) * (v1[0] - v0[0]) + (v1[1] - v0[1]) * (v1[1] - v0[1]) + (v1[2] - v0[2]) * (v1[2] - v0[2]));
        double b = sqrt((v2[0] - v1[0]) * (v2[0] - v1[0]) + (v2[1] - v1[1]) * (v2[1] - v1[1]) + (v2[2] - v1[2]) * (v2[2] - v1[2]));
        double c = sqrt((v2[0] - v0[0]) * (v2[0] - v0[0]) + (v2[1] - v0[1]) * (v2[1] - v0[1]) + (v2[2] - v0[2]) * (v2[2] - v0[2]));
        double s = (a + b + c) / 2.0;
        double p = s * (s - a) * (s - b) * (s - c);
        area[i] = p > 0 ? sqrt(p) : 0.0;
    }
}

/* ------------------------------------------------------------------------------------ */
/* Per-triangle sample counts (Section 3.1.2 asks #p / A = k per triangle). The count of  */
/* triangle i is the difference of rounded running totals of k*A in 32.32 fixed point:    */
/*   q_i = rint(k_i A_i 2^32),  S_i = q_0 + ... + q_i,  start_i = (S_{i-1} + 2^31) >> 32. */
/* Returns 0, or -1 if a count would overflow.                                           */
/* ------------------------------------------------------------------------------------ */
int ora_tri_offsets(const double* area, const double* density, int64_t nt, int64_t* offsets)
{
    int64_t S = 0;
    offsets[0] = 0;
    for (int64_t i = 0; i < nt; ++i) {
        double c = density[i] * area[i];
        if (!(c >= 0.0) || c >= 2147483648.0) return -1;
        int64_t q = llrint(c * 4294967296.0);
        if (S > INT64_MAX - q) return -1;
        S += q;
        offsets[i + 1] = (S + ((int64_t)1 << 31)) >> 32;
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as easy as       */
/* 1, 2, 3", SC'11): ten rounds of two 32x32->64 multiplies with the round multipliers,  */
/* the key bumped by the Weyl constants between rounds.                                   */
/* ------------------------------------------------------------------------------------ */
void ora_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t n0 = (uint32_t)(p1 >> 32) ^ c1 ^ k0;
        uint32_t n1 = (uint32_t)p1;
        uint32_t n2 = (uint32_t)(p0 >> 32) ^ c3 ^ k1;
        uint32_t n3 = (uint32_t)p0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A Philox word to a uniform in (0, 1): the top 23 bits, centred: (w>>9 + 1/2) / 2^23. */
static double unit_from_word(uint32_t w) { return ((double)(w >> 9) + 0.5) / 8388608.0; }

/* ------------------------------------------------------------------------------------ */
/* Sample expansion. Global sample j lives in the triangle i with                         */
/* offsets[i] <= j < offsets[i+1]; its position is drawn from Philox4x32-10 with          */
/* key = (seed lo, seed hi) and counter = (j lo, j hi, session, 0): u1, u2 from the first */
/* two words, barycentrics (1 - sqrt u1, sqrt u1 (1 - u2), sqrt u1 u2), all in FP64.     */
/* ------------------------------------------------------------------------------------ */
int ora_samples(const float* tri, const int64_t* offsets, int64_t nt, uint64_t seed, uint32_t session,
                const int64_t* which, int64_t n, int64_t* tri_out, uint32_t* words_out,
                double* bary_out, double* xyz_out)
{
    uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = which[k];
        if (j < 0 || j >= offsets[nt]) return -1;
        /* plain binary search for the last i with offsets[i] <= j */
        int64_t lo = 0, hi = nt;           /* invariant: offsets[lo] <= j < offsets[hi] */
        while (hi - lo > 1) {
            int64_t mid = lo + (hi - lo) / 2;
            if (offsets[mid] <= j) lo = mid; else hi = mid;
        }
        uint32_t ctr[4] = {(uint32_t)j, (uint32_t)((uint64_t)j >> 32), session, 0u}, w[4];
        ora_philox4x32_10(ctr, key, w);
        double u1 = unit_from_word(w[0]), u2 = unit_from_word(w[1]);
        double su = sqrt(u1);
        double b0 = 1.0 - su, b1 = su * (1.0 - u2), b2 = su * u2;
        const float* t = tri + 9 * lo;
        tri_out[k] = lo;
        if (words_out) { words_out[2 * k] = w[0]; words_out[2 * k + 1] = w[1]; }
        if (bary_out) { bary_out[3 * k] = b0; bary_out[3 * k + 1] = b1; bary_out[3 * k + 2] = b2; }
        for (int c = 0; c < 3; ++c)
            xyz_out[3 * k + c] = b0 * (double)t[c] + b1 * (double)t[3 + c] + b2 * (double)t[6 + c];
    }
    return 0;
}

/* ------------------------------------------------------------------------------------ */
/* The Gaussian projection of Section 3.2.1 for one sample and one fixation.               */
/* p = s - e; d1 = p.r/|r|; d2 = |p x r|/|r|; sigma = tan(theta); d = d1 tan(theta);      */
/* sigma_k = (d2/d) sigma (0 if d = 0); g = t/(sigma sqrt(2 pi)) exp(-sigma_k^2/(2 sigma^2)). */
/* Returns 1 if the pair is inside the cut-off cone (d1 > 0, sigma_k <= cutoff*sigma).     */
/* *edge is set when sigma_k is within rel_band of the cut-off (either side).             */
/* ------------------------------------------------------------------------------------ */
typedef struct { double g, d1, d2, sk; int edge; } pair_eval;

static int gaussian_pair(const double s[3], const double e[3], const double r[3], double t,
                         double theta, double cutoff, double rel_band, pair_eval* pe)
{
    double p[3] = {s[0] - e[0], s[1] - e[1], s[2] - e[2]};
    double rn = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double rh[3] = {r[0] / rn, r[1] / rn, r[2] / rn};
    double d1 = p[0] * rh[0] + p[1] * rh[1] + p[2] * rh[2];
    double cx = p[1] * rh[2] - p[2] * rh[1];
    double cy = p[2] * rh[0] - p[0] * rh[2];
    double cz = p[0] * rh[1] - p[1] * rh[0];
    double d2 = sqrt(cx * cx + cy * cy + cz * cz);
    double sigma = tan(theta);
    double d = d1 * sigma;
    pe->d1 = d1; pe->d2 = d2;
    pe->edge = 0;
    if (!(d1 > 0.0)) { pe->g = 0.0; pe->sk = INFINITY; return 0; }
    double sk = (d == 0.0) ? 0.0 : (d2 / d) * sigma;
    pe->sk = sk;
    pe->g = t / (sigma * sqrt(2.0 * ORA_PI)) * exp(-(sk * sk) / (2.0 * sigma * sigma));
    double lim = cutoff * sigma;
    pe->edge = fabs(sk - lim) <= rel_band * lim;
    return sk <= lim;
}

int ora_pair_weight(const double* s, const double* e, const double* r, double t, double theta,
                    double cutoff, double* g_out)
{
    pair_eval pe;
    int in = gaussian_pair(s, e, r, t, theta, cutoff, 0.0, &pe);
    *g_out = pe.g;
    return in;
}

/* ------------------------------------------------------------------------------------ */
/* Segment / triangle test, Moller & Trumbore (1997), FP64. The segment is o + t d,        */
/* 0 < t < tmax. Returns 1 for an exact hit. *robust is set when the hit holds with a     */
/* margin of delta (metres) on every edge and on both ends of the segment; *near when the */
/* decision could flip under a perturbation of delta (a grazing case).                    */
/* ------------------------------------------------------------------------------------ */
static int seg_tri(const double o[3], const double d[3], double tmax, const float* T,
                   double delta, int* robust, int* near)
{
    double v0[3] = {T[0], T[1], T[2]}, v1[3] = {T[3], T[4], T[5]}, v2[3] = {T[6], T[7], T[8]};
    double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    double n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    double area2 = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    *robust = 0; *near = 0;
    if (area2 == 0.0) return 0;                       /* a zero-area triangle cannot occlude */
    double dl = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double cosinc = fabs(n[0] * d[0] + n[1] * d[1] + n[2] * d[2]) / (area2 * dl);
    double P[3] = {d[1] * e2[2] - d[2] * e2[1], d[2] * e2[0] - d[0] * e2[2], d[0] * e2[1] - d[1] * e2[0]};
    double det = e1[0] * P[0] + e1[1] * P[1] + e1[2] * P[2];
    if (cosinc < 1e-9 || det == 0.0) {
        /* (nearly) parallel: only a segment lying within delta of the plane is in doubt */
        double h = fabs(n[0] * (o[0] - v0[0]) + n[1] * (o[1] - v0[1]) + n[2] * (o[2] - v0[2])) / area2;
        *near = h <= delta + 1e-9 * dl;
        return 0;
    }
    double Tv[3] = {o[0] - v0[0], o[1] - v0[1], o[2] - v0[2]};
    double u = (Tv[0] * P[0] + Tv[1] * P[1] + Tv[2] * P[2]) / det;
    double Q[3] = {Tv[1] * e1[2] - Tv[2] * e1[1], Tv[2] * e1[0] - Tv[0] * e1[2], Tv[0] * e1[1] - Tv[1] * e1[0]};
    double v = (d[0] * Q[0] + d[1] * Q[1] + d[2] * Q[2]) / det;
    double t = (e2[0] * Q[0] + e2[1] * Q[1] + e2[2] * Q[2]) / det;
    double b[3] = {1.0 - u - v, u, v};
    int hit = b[0] >= 0.0 && b[1] >= 0.0 && b[2] >= 0.0 && t > 0.0 && t < tmax;
    /* signed distance of the plane hit point to each edge line = barycentric x altitude */
    double l12 = sqrt((v2[0] - v1[0]) * (v2[0] - v1[0]) + (v2[1] - v1[1]) * (v2[1] - v1[1]) + (v2[2] - v1[2]) * (v2[2] - v1[2]));
    double l02 = sqrt(e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
    double l01 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    double md = b[0] * (area2 / l12);
    double m1 = b[1] * (area2 / l02);
    double m2 = b[2] * (area2 / l01);
    if (m1 < md) md = m1;
    if (m2 < md) md = m2;
    double de = delta / cosinc, dt = delta / (cosinc * dl);
    *robust = md > de && t > dt && t < tmax - dt;
    *near = !*robust && md > -de && t > -dt && t < tmax + dt;
    return hit;
}

/* ------------------------------------------------------------------------------------ */
/* Accumulation (Section 3.2) over every sample x fixation pair, then per-window sums.     */
/* ------------------------------------------------------------------------------------ */
typedef struct {
    double theta, cutoff, eps_rel, t_begin, t_end, window_s;
    double delta_abs;       /* grazing margin (metres) for the ambiguity bookkeeping */
    double cone_band;       /* relative band around the cut-off for the ambiguity bookkeeping */
    int32_t n_windows;
    int32_t nthreads;
} ora_params;

typedef struct {
    int64_t pairs, in_cone, rays, visible, ambiguous, cone_edge;
} ora_stats;

enum { PF_IN_CONE = 1, PF_VISIBLE = 2, PF_VIS_AMBIG = 4, PF_CONE_EDGE = 8 };

typedef struct {
    const float* tri; int64_t nt;
    const double* sxyz; const int64_t* stri; int64_t s0, s1, ns;
    const float *eye, *gaze, *dur; const int32_t* win; int64_t nf;
    const ora_params* prm;
    double *density, *amb, *sens;
    ora_stats st;
    int record;
    int64_t *ps; int32_t* pf; uint8_t* pflag; double* pg; int64_t np, cap;
    int err;
} ora_job;

static void push_pair(ora_job* J, int64_t s, int32_t f, uint8_t flag, double g)
{
    if (J->np == J->cap) {
        int64_t nc = J->cap ? 2 * J->cap : 1024;
        int64_t* a = (int64_t*)realloc(J->ps, sizeof(int64_t) * nc);
        int32_t* b = (int32_t*)realloc(J->pf, sizeof(int32_t) * nc);
        uint8_t* c = (uint8_t*)realloc(J->pflag, nc);
        double* d = (double*)realloc(J->pg, sizeof(double) * nc);
        if (a) J->ps = a;
        if (b) J->pf = b;
        if (c) J->pflag = c;
        if (d) J->pg = d;
        if (!a || !b || !c || !d) { J->err = -2; return; }
        J->cap = nc;
    }
    J->ps[J->np] = s; J->pf[J->np] = f; J->pflag[J->np] = flag; J->pg[J->np] = g; J->np++;
}

static void* accumulate_range(void* arg)
{
    ora_job* J = (ora_job*)arg;
    const ora_params* P = J->prm;
    double tan_t = tan(P->theta);
    for (int64_t s = J->s0; s < J->s1; ++s) {
        const double* sp = J->sxyz + 3 * s;
        int64_t own = J->stri[s];
        for (int64_t f = 0; f < J->nf; ++f) {
            int32_t w = J->win[f];
            if (w < 0) continue;
            J->st.pairs++;
            double e[3] = {J->eye[3 * f], J->eye[3 * f + 1], J->eye[3 * f + 2]};
            double r[3] = {J->gaze[3 * f], J->gaze[3 * f + 1], J->gaze[3 * f + 2]};
            pair_eval pe;
            int in = gaussian_pair(sp, e, r, (double)J->dur[f], P->theta, P->cutoff, P->cone_band, &pe);
            if (!in && !pe.edge) continue;
            /* occlusion: segment e -> e + (1 - eps) (s - e), every triangle but the sample's own */
            double d[3] = {sp[0] - e[0], sp[1] - e[1], sp[2] - e[2]};
            double tmax = 1.0 - P->eps_rel;
            int blocked = 0, any_robust = 0, any_near = 0;
            for (int64_t j = 0; j < J->nt; ++j) {
                if (j == own) continue;
                int rob, nr;
                blocked |= seg_tri(e, d, tmax, J->tri + 9 * j, P->delta_abs, &rob, &nr);
                any_robust |= rob;
                any_near |= nr;
                if (any_robust) break;
            }
            int amb_vis = !any_robust && any_near;
            size_t o = (size_t)w * (size_t)J->ns + (size_t)s;
            uint8_t flag = (uint8_t)((in ? PF_IN_CONE : 0) | (blocked ? 0 : PF_VISIBLE)
                                     | (amb_vis ? PF_VIS_AMBIG : 0) | (pe.edge ? PF_CONE_EDGE : 0));
            if (in) {
                J->st.in_cone++;
                J->st.rays++;
                if (!blocked) {
                    J->st.visible++;
                    J->density[o] += pe.g;
                    if (J->sens)
                        J->sens[o] += pe.g * (pe.d2 / (pe.d1 * pe.d1)) * (1.0 + pe.d2 / pe.d1) / (tan_t * tan_t);
                }
            }
            if (amb_vis || pe.edge) {
                if (J->amb) J->amb[o] += pe.g;
                J->st.ambiguous += amb_vis;
                J->st.cone_edge += pe.edge;
            }
            if (J->record) push_pair(J, s, (int32_t)f, flag, pe.g);
        }
    }
    return NULL;
}

/* Window of each fixation: floor((ts - t_begin) / window_s) when window_s > 0, else 0;
 * -1 when the timestamp is outside [t_begin, t_end) or past the last window (Section 3.3.4
 * lists the time interval of the fixations among the generation parameters). */
void ora_fixation_windows(const double* ts, int64_t nf, double t_begin, double t_end,
                          double window_s, int32_t n_windows, int32_t* win)
{
    for (int64_t f = 0; f < nf; ++f) {
        double t = ts[f];
        if (!(t >= t_begin && t < t_end)) { win[f] = -1; continue; }
        int64_t w = window_s > 0.0 ? (int64_t)floor((t - t_begin) / window_s) : 0;
        win[f] = (w >= 0 && w < n_windows) ? (int32_t)w : -1;
    }
}

/*
 * density, amb, sens: n_windows * ns doubles each (window-major), zeroed here.
 * amb[s]  = sum of g over the sample's pairs whose cone or visibility decision is within the
 *           bookkeeping margins (the CUDA path may decide those either way);
 * sens[s] = sum over visible in-cone pairs of g * |d ln g / d position| (1/m), a first-order
 *           bound of how the sample's value moves when its position moves.
 * Pairs (in cone, or at the cone edge) are recorded in sample-major, fixation-minor order
 * when rec_cap >= 0; *n_rec returns how many exist (only min(n, rec_cap) are copied).
 */
int ora_accumulate(const float* tri, int64_t nt, const double* sxyz, const int64_t* stri, int64_t ns,
                   const float* eye, const float* gaze, const float* dur, const double* ts, int64_t nf,
                   const ora_params* prm, double* density, double* amb, double* sens, ora_stats* st,
                   int64_t rec_cap, int64_t* rec_s, int32_t* rec_f, uint8_t* rec_flag, double* rec_g,
                   int64_t* n_rec)
{
    int32_t* win = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
    if (!win) return -2;
    ora_fixation_windows(ts, nf, prm->t_begin, prm->t_end, prm->window_s, prm->n_windows, win);
    size_t nout = (size_t)prm->n_windows * (size_t)ns;
    memset(density, 0, sizeof(double) * nout);
    if (amb) memset(amb, 0, sizeof(double) * nout);
    if (sens) memset(sens, 0, sizeof(double) * nout);
    int nth = prm->nthreads > 0 ? prm->nthreads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nth < 1) nth = 1;
    if (nth > ns) nth = ns > 0 ? (int)ns : 1;
    ora_job* jobs = (ora_job*)calloc((size_t)nth, sizeof(ora_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nth, sizeof(pthread_t));
    if (!jobs || !th) { free(win); free(jobs); free(th); return -2; }
    for (int i = 0; i < nth; ++i) {
        ora_job* J = &jobs[i];
        J->tri = tri; J->nt = nt; J->sxyz = sxyz; J->stri = stri; J->ns = ns;
        J->s0 = ns * i / nth; J->s1 = ns * (i + 1) / nth;
        J->eye = eye; J->gaze = gaze; J->dur = dur; J->win = win; J->nf = nf;
        J->prm = prm; J->density = density; J->amb = amb; J->sens = sens;
        J->record = rec_cap >= 0;
    }
    for (int i = 1; i < nth; ++i) pthread_create(&th[i], NULL, accumulate_range, &jobs[i]);
    accumulate_range(&jobs[0]);
    for (int i = 1; i < nth; ++i) pthread_join(th[i], NULL);
    int err = 0;
    ora_stats tot = {0, 0, 0, 0, 0, 0};
    int64_t nrec = 0;
    for (int i = 0; i < nth; ++i) {
        ora_job* J = &jobs[i];
        if (J->err) err = J->err;
        tot.pairs += J->st.pairs; tot.in_cone += J->st.in_cone; tot.rays += J->st.rays;
        tot.visible += J->st.visible; tot.ambiguous += J->st.ambiguous; tot.cone_edge += J->st.cone_edge;
        for (int64_t k = 0; k < J->np; ++k, ++nrec) {
            if (nrec < rec_cap) {
                rec_s[nrec] = J->ps[k]; rec_f[nrec] = J->pf[k];
                rec_flag[nrec] = J->pflag[k]; rec_g[nrec] = J->pg[k];
            }
        }
        free(J->ps); free(J->pf); free(J->pflag); free(J->pg);
    }
    if (st) *st = tot;
    if (n_rec) *n_rec = nrec;
    free(jobs); free(th); free(win);
    return err;
}

/* Normalisation (Section 3.2.3): divide by the maximum so every value is in [0, 1].
 * Returns the maximum; a map whose maximum is 0 becomes all zeros. */
double ora_normalize(const double* v, int64_t n, double* out)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i) if (v[i] > m) m = v[i];
    for (int64_t i = 0; i < n; ++i) out[i] = m > 0.0 ? v[i] / m : 0.0;
    return m;
}

/* Philox4x32-10 over many counters (n x 4 words in, n x 4 words out), one key. */
void ora_philox_batch(const uint32_t* ctr, int64_t n, const uint32_t key[2], uint32_t* out)
{
    for (int64_t i = 0; i < n; ++i) ora_philox4x32_10(ctr + 4 * i, key, out + 4 * i);
}

/* ------------------------------------------------------------------------------------ */
/* The paper's own sampler (Section 3.1): every triangle is subdivided with an integer     */
/* resolution r and holds #p = f(r) = (r+1)(r+2)/2 samples on its barycentric grid.       */
/* Adaptive resolution (Section 3.1.2): with D = 1 + 8 k A, r = 1 when D < 25, else the    */
/* positive root (-3 + sqrt(D)) / 2 of r^2 + 3r + 2 - 2kA = 0, rounded to the nearest      */
/* integer (ties to even; the rounding is not stated).                                    */
/* ------------------------------------------------------------------------------------ */
void ora_grid_resolution(const double* area, const double* density, int64_t nt, int64_t* r_out, double* r_real)
{
    for (int64_t i = 0; i < nt; ++i) {
        double D = 1.0 + 8.0 * density[i] * area[i];
        double r = D < 25.0 ? 1.0 : (-3.0 + sqrt(D)) / 2.0;
        if (r_real) r_real[i] = r;
        int64_t ri = D < 25.0 ? 1 : (int64_t)nearbyint(r);
        r_out[i] = ri < 1 ? 1 : ri;
    }
}

/* Offsets of the grid samples: offsets[i+1] - offsets[i] = (r_i + 1)(r_i + 2) / 2. */
void ora_grid_offsets(const int64_t* r, int64_t nt, int64_t* offsets)
{
    offsets[0] = 0;
    for (int64_t i = 0; i < nt; ++i) offsets[i + 1] = offsets[i] + (r[i] + 1) * (r[i] + 2) / 2;
}

/* Sample idx of a triangle of resolution r: row = the largest m with m(m+1)/2 <= idx (the
 * integer form of Eq. 2's ceil((-3 + sqrt(8 idx + 9)) / 2)), col = idx - row(row+1)/2;
 * barycentrics (Eq. 3) w1 = col / r, w2 = 1 - row / r, w3 = 1 - w1 - w2 = (row - col) / r
 * (the printed third coordinate does not sum to one); position w1 v0 + w2 v1 + w3 v2. */
void ora_grid_index(int64_t idx, int64_t* row, int64_t* col)
{
    int64_t m = 0;
    while ((m + 1) * (m + 2) / 2 <= idx) ++m;
    *row = m;
    *col = idx - m * (m + 1) / 2;
}

int ora_grid_samples(const float* tri, const int64_t* offsets, const int64_t* r, int64_t nt, const int64_t* which,
                     int64_t n, int64_t* tri_out, int64_t* rowcol_out, double* bary_out, double* xyz_out)
{
    for (int64_t k = 0; k < n; ++k) {
        int64_t j = which[k];
        if (j < 0 || j >= offsets[nt]) return -1;
        int64_t lo = 0, hi = nt;
        while (hi - lo > 1) {
            int64_t mid = lo + (hi - lo) / 2;
            if (offsets[mid] <= j) lo = mid; else hi = mid;
        }
        int64_t row, col;
        ora_grid_index(j - offsets[lo], &row, &col);
        double rr = (double)r[lo];
        double w1 = col / rr, w2 = 1.0 - row / rr, w3 = (row - col) / rr;
        const float* t = tri + 9 * lo;
        tri_out[k] = lo;
        if (rowcol_out) { rowcol_out[2 * k] = row; rowcol_out[2 * k + 1] = col; }
        if (bary_out) { bary_out[3 * k] = w1; bary_out[3 * k + 1] = w2; bary_out[3 * k + 2] = w3; }
        for (int c = 0; c < 3; ++c)
            xyz_out[3 * k + c] = w1 * (double)t[c] + w2 * (double)t[3 + c] + w3 * (double)t[6 + c];
    }
    return 0;
}
