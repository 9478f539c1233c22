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

/* ==================================================================================== */
/* The paper's own occlusion path (Sections 3.2.2 and 3.3.2, Appendix A): per fixation a  */
/* camera at the eye, the near-plane crop window of the 4 sigma cone, a z-buffer of that  */
/* window and the +-eps depth comparison. Readings (the paper leaves these open):         */
/*  - camera: x right, y up, looking down -z; forward and up hints per fixation (the head */
/*    pose); the gaze r is a direction in that frame;                                     */
/*  - the z-buffer stores linear view depth w = (p - e).forward (metres), the +-eps test  */
/*    compares it with the sample's w; a pixel holds the nearest surface that covers its  */
/*    centre (point sampling), with geometry clipped to n <= w <= f; triangles two-sided; */
/*  - the crop window used for filtering is the exact bounding box of the cone's section */
/*    (tangent planes through the eye); the printed construction (E-centred ellipse with */
/*    quaternion-rotated rays) is kept below as ora_crop_paper for comparison, since the */
/*    centre of an oblique conic section is not the gaze point E;                        */
/*  - samples keep the exact 4 sigma cone test of the ray path; the crop is a filter.    */
/* ==================================================================================== */

static void v3_cross(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double v3_dot(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static int v3_unit(double a[3])
{
    double l = sqrt(v3_dot(a, a));
    if (!(l > 0.0) || !isfinite(l)) return -1;
    a[0] /= l; a[1] /= l; a[2] /= l;
    return 0;
}

/* Camera basis from a forward and an up hint: fwd = unit(forward), right = unit(fwd x up),
 * up = right x fwd. An up hint within 1e-6 of parallel to forward is replaced by world z.
 * Returns 0, or -1 for a zero forward. */
int ora_camera_basis(const double fwd_in[3], const double up_in[3], double right[3], double up[3], double fwd[3])
{
    double f[3] = {fwd_in[0], fwd_in[1], fwd_in[2]}, u[3] = {up_in[0], up_in[1], up_in[2]};
    if (v3_unit(f)) return -1;
    double r[3];
    v3_cross(f, u, r);
    double lu = sqrt(v3_dot(u, u));
    if (!(sqrt(v3_dot(r, r)) > 1e-6 * lu)) {
        double z[3] = {0.0, 0.0, 1.0};
        v3_cross(f, z, r);
        if (!(sqrt(v3_dot(r, r)) > 1e-6)) { double x[3] = {1.0, 0.0, 0.0}; v3_cross(f, x, r); }
    }
    v3_unit(r);
    v3_cross(r, f, u);
    for (int k = 0; k < 3; ++k) { right[k] = r[k]; up[k] = u[k]; fwd[k] = f[k]; }
    return 0;
}

/* Hamilton product helpers for the rotation q v q^-1 of Appendix A. */
static void quat_rotate(const double axis[3], double ang, const double v[3], double out[3])
{
    double c = cos(0.5 * ang), s = sin(0.5 * ang);
    double q[4] = {c, s * axis[0], s * axis[1], s * axis[2]};        /* w, x, y, z */
    double qi[4] = {c, -q[1], -q[2], -q[3]};
    double p[4] = {0.0, v[0], v[1], v[2]};
    double t[4], r[4];
    /* t = q p */
    t[0] = q[0] * p[0] - q[1] * p[1] - q[2] * p[2] - q[3] * p[3];
    t[1] = q[0] * p[1] + q[1] * p[0] + q[2] * p[3] - q[3] * p[2];
    t[2] = q[0] * p[2] - q[1] * p[3] + q[2] * p[0] + q[3] * p[1];
    t[3] = q[0] * p[3] + q[1] * p[2] - q[2] * p[1] + q[3] * p[0];
    /* r = t qi */
    r[0] = t[0] * qi[0] - t[1] * qi[1] - t[2] * qi[2] - t[3] * qi[3];
    r[1] = t[0] * qi[1] + t[1] * qi[0] + t[2] * qi[3] - t[3] * qi[2];
    r[2] = t[0] * qi[2] - t[1] * qi[3] + t[2] * qi[0] + t[3] * qi[1];
    r[3] = t[0] * qi[3] + t[1] * qi[2] - t[2] * qi[1] + t[3] * qi[0];
    out[0] = r[1]; out[1] = r[2]; out[2] = r[3];
}

/* The crop window as Appendix A constructs it, for a unit gaze direction rc in camera space
 * (x right, y up, z back) and the cone half-angle phi = atan(cutoff tan theta): rays rotated
 * by -+phi about u1 = rc x i and u2 = rc x u1 (i = the forward axis (0, 0, -1); both axes
 * normalised) meet the near plane z = -n at A0, A1, B0, B1; a = |A1 - A0| / 2, b = |B1 - B0| / 2,
 * E = the gaze ray's point on the plane, alpha = acos(j . unit(E - M)) with j = (1, 0, 0) and
 * M = (0, 0, -n); bounds E -+ sqrt(a^2 cos^2 alpha + b^2 sin^2 alpha) in x and
 * E -+ sqrt(a^2 sin^2 alpha + b^2 cos^2 alpha) in y. When rc is along the forward axis u1 is
 * undefined: the section is a circle, a = b = n tan phi, alpha = 0.
 * out: l, r, b, t, E_x, E_y, a, b, alpha. Returns -1 if a rotated ray does not reach the plane. */
int ora_crop_paper(const double rc_in[3], double phi, double n, double* out)
{
    double rc[3] = {rc_in[0], rc_in[1], rc_in[2]};
    if (v3_unit(rc)) return -1;
    if (!(rc[2] < 0.0)) return -1;
    double Ex = -n / rc[2] * rc[0], Ey = -n / rc[2] * rc[1];
    double i_ax[3] = {0.0, 0.0, -1.0};
    double u1[3], u2[3];
    v3_cross(rc, i_ax, u1);
    double a, b, alpha;
    if (sqrt(v3_dot(u1, u1)) < 1e-12) {
        a = b = n * tan(phi);
        alpha = 0.0;
    } else {
        v3_unit(u1);
        v3_cross(rc, u1, u2);
        v3_unit(u2);
        double a0[3], a1[3], b0[3], b1[3];
        quat_rotate(u1, -phi, rc, a0);
        quat_rotate(u1, phi, rc, a1);
        quat_rotate(u2, -phi, rc, b0);
        quat_rotate(u2, phi, rc, b1);
        if (!(a0[2] < 0.0 && a1[2] < 0.0 && b0[2] < 0.0 && b1[2] < 0.0)) return -1;
        a = 0.5 * n * sqrt(pow(a0[0] / a0[2] - a1[0] / a1[2], 2) + pow(a0[1] / a0[2] - a1[1] / a1[2], 2));
        b = 0.5 * n * sqrt(pow(b0[0] / b0[2] - b1[0] / b1[2], 2) + pow(b0[1] / b0[2] - b1[1] / b1[2], 2));
        double me[3] = {Ex, Ey, 0.0};
        v3_unit(me);
        double c = me[0];
        if (c > 1.0) c = 1.0;
        if (c < -1.0) c = -1.0;
        alpha = acos(c);
    }
    double hx = sqrt(a * a * cos(alpha) * cos(alpha) + b * b * sin(alpha) * sin(alpha));
    double hy = sqrt(a * a * sin(alpha) * sin(alpha) + b * b * cos(alpha) * cos(alpha));
    out[0] = Ex - hx; out[1] = Ex + hx; out[2] = Ey - hy; out[3] = Ey + hy;
    out[4] = Ex; out[5] = Ey; out[6] = a; out[7] = b; out[8] = alpha;
    return 0;
}

/* The exact crop window: the cone of half-angle phi about the unit direction rc (camera
 * space) meets the near plane z = -n in a conic whose x-extent is bounded by the two planes
 * through the eye, x + c z = 0, tangent to the cone: |(1, 0, c) . rc| = sin(phi) sqrt(1 + c^2),
 * i.e. (rc_z^2 - s^2) c^2 + 2 rc_x rc_z c + (rc_x^2 - s^2) = 0 with s = sin(phi); the plane
 * meets z = -n at x = c n. The same with y. Needs the whole cone in front of the camera
 * (rc_z < 0 and rc_z^2 > s^2); returns -1 otherwise. out: l, r, b, t. */
int ora_crop_exact(const double rc_in[3], double phi, double n, double* out)
{
    double rc[3] = {rc_in[0], rc_in[1], rc_in[2]};
    if (v3_unit(rc)) return -1;
    double s = sin(phi);
    double A = rc[2] * rc[2] - s * s;
    if (!(rc[2] < 0.0) || !(A > 0.0)) return -1;
    for (int k = 0; k < 2; ++k) {
        double q = rc[k];
        double disc = s * sqrt(q * q + rc[2] * rc[2] - s * s);
        double c1 = (-q * rc[2] - disc) / A, c2 = (-q * rc[2] + disc) / A;
        out[2 * k] = n * (c1 < c2 ? c1 : c2);
        out[2 * k + 1] = n * (c1 < c2 ? c2 : c1);
    }
    return 0;
}

/* Ray o + t d (t > 0) against one triangle, FP64 Moller-Trumbore. Returns 1 on a hit and its
 * t; *near is set when the point is within delta (metres, in the triangle's plane) of an edge,
 * on either side (a coverage decision an FP32 rasteriser may take the other way). */
static int ray_tri_t(const double o[3], const double d[3], const float* T, double delta, double* t_out, int* near,
                     double* t_plane)
{
    double v0[3] = {T[0], T[1], T[2]}, v1[3] = {T[3], T[4], T[5]}, v2[3] = {T[6], T[7], T[8]};
    double e1[3] = {v1[0] - v0[0], v1[1] - v0[1], v1[2] - v0[2]};
    double e2[3] = {v2[0] - v0[0], v2[1] - v0[1], v2[2] - v0[2]};
    double nrm[3];
    v3_cross(e1, e2, nrm);
    double area2 = sqrt(v3_dot(nrm, nrm));
    *near = 0;
    *t_plane = INFINITY;
    if (area2 == 0.0) return 0;
    double P[3];
    v3_cross(d, e2, P);
    double det = v3_dot(e1, P);
    double dl = sqrt(v3_dot(d, d));
    double cosinc = fabs(v3_dot(nrm, d)) / (area2 * dl);
    if (det == 0.0 || cosinc < 1e-9) return 0;
    double Tv[3] = {o[0] - v0[0], o[1] - v0[1], o[2] - v0[2]};
    double u = v3_dot(Tv, P) / det;
    double Q[3];
    v3_cross(Tv, e1, Q);
    double v = v3_dot(d, Q) / det;
    double t = v3_dot(e2, Q) / det;
    *t_plane = t;
    double b[3] = {1.0 - u - v, u, v};
    double l12 = sqrt(pow(v2[0] - v1[0], 2) + pow(v2[1] - v1[1], 2) + pow(v2[2] - v1[2], 2));
    double l02 = sqrt(v3_dot(e2, e2)), l01 = sqrt(v3_dot(e1, e1));
    double md = b[0] * (area2 / l12), m1 = b[1] * (area2 / l02), m2 = b[2] * (area2 / l01);
    if (m1 < md) md = m1;
    if (m2 < md) md = m2;
    double de = delta / cosinc;
    *near = t > 0.0 && fabs(md) <= de;
    if (b[0] >= 0.0 && b[1] >= 0.0 && b[2] >= 0.0 && t > 0.0) {
        *t_out = t;
        return 1;
    }
    return 0;
}

typedef struct {
    double e[3], right[3], up[3], fwd[3];
    double n, f, l, r, b, t;
    int32_t ok;
} ora_frustum;

/* Frustum of one fixation: camera basis, gaze in camera space, exact crop window. */
int ora_zb_frustum(const float* eye, const float* gaze, const float* cam_fwd, const float* cam_up, double theta,
                   double cutoff, double n, double f, ora_frustum* F)
{
    double fw[3] = {cam_fwd[0], cam_fwd[1], cam_fwd[2]}, uh[3] = {cam_up[0], cam_up[1], cam_up[2]};
    memset(F, 0, sizeof(*F));
    for (int k = 0; k < 3; ++k) F->e[k] = eye[k];
    F->n = n; F->f = f;
    if (ora_camera_basis(fw, uh, F->right, F->up, F->fwd)) return -1;
    double g[3] = {gaze[0], gaze[1], gaze[2]};
    if (v3_unit(g)) return -1;
    double rc[3] = {v3_dot(g, F->right), v3_dot(g, F->up), -v3_dot(g, F->fwd)};
    double phi = atan(cutoff * tan(theta));
    double bnd[4];
    if (ora_crop_exact(rc, phi, n, bnd)) return -1;
    F->l = bnd[0]; F->r = bnd[1]; F->b = bnd[2]; F->t = bnd[3];
    F->ok = 1;
    return 0;
}

/* Z-buffer of one frustum: res x res pixels over the crop window; pixel (px, py) has its centre
 * at x = l + (px + 1/2)(r - l)/res, y = b + (py + 1/2)(t - b)/res on the near plane; its depth
 * is the smallest w = t n over triangles that the ray e + t (x right + y up + n fwd) meets with
 * n <= w <= f (+inf when none). amb[p] is set when a triangle whose edge passes within delta_px
 * pixels of the centre (at its own depth) lies no deeper than the pixel's depth (plus 1e-6
 * relative), or a hit lies within zb_depth_band of a clip plane: a clipper that computes camera
 * depths in FP32 may place the clip edge that far from the exact plane. zbuf and amb: res * res. */
/* How far a camera depth w = (p - e).fwd evaluated in FP32 (from FP32 p and e, an FP32 copy of
 * fwd: one subtraction and three multiply-adds per coordinate) can lie from the exact one: six
 * units of 2^-24 of ||p - e||_1; doubled here to cover a clip point interpolated between two such
 * depths. Absolute (metres), so it grows with the distance of the geometry, not of the plane. */
static double zb_depth_band(const double q[3], const double e[3])
{
    return 12.0 * 5.9604644775390625e-8 * (fabs(q[0] - e[0]) + fabs(q[1] - e[1]) + fabs(q[2] - e[2]));
}

static void zb_pixel(const float* tri, int64_t nt, const ora_frustum* F, int32_t res, double delta_px, int32_t px,
                     int32_t py, double* depth, uint8_t* amb_out)
{
    double pxw = (F->r - F->l) / res, pxh = (F->t - F->b) / res;
    {
        {
            double x = F->l + (px + 0.5) * pxw, y = F->b + (py + 0.5) * pxh;
            double d[3];
            for (int k = 0; k < 3; ++k) d[k] = x * F->right[k] + y * F->up[k] + F->n * F->fwd[k];
            double best = INFINITY, near_best = INFINITY;
            int clip_amb = 0;
            for (int64_t j = 0; j < nt; ++j) {
                double t, tp;
                int nr;
                /* delta in metres at this depth: delta_px pixels of width (r - l)/res at the near plane */
                double dw = delta_px * pxw / F->n;
                int hit = ray_tri_t(F->e, d, tri + 9 * j, 0.0, &t, &nr, &tp);
                double w = hit ? t * F->n : INFINITY;
                double wp = tp * F->n;
                /* edge proximity measured at the plane hit depth */
                int nr2;
                double tt, tp2;
                ray_tri_t(F->e, d, tri + 9 * j, dw * (wp > 0.0 ? wp : 0.0), &tt, &nr2, &tp2);
                if (hit) {
                    const float* T = tri + 9 * j;
                    double band = 0.0;
                    for (int k = 0; k < 3; ++k) {
                        const double v[3] = {T[3 * k], T[3 * k + 1], T[3 * k + 2]};
                        const double bk = zb_depth_band(v, F->e);
                        if (bk > band) band = bk;
                    }
                    if (fabs(w - F->n) <= band || fabs(w - F->f) <= band) clip_amb = 1;
                    if (w >= F->n && w <= F->f && w < best) best = w;
                }
                if (nr2 && wp >= F->n * (1.0 - 1e-9) && wp <= F->f * (1.0 + 1e-9) && wp < near_best) near_best = wp;
            }
            *depth = best;
            *amb_out = (uint8_t)(clip_amb || (isfinite(near_best) && near_best <= best * (1.0 + 1e-6)));
        }
    }
}

int ora_zb_render(const float* tri, int64_t nt, const ora_frustum* F, int32_t res, double delta_px, double* zbuf,
                  uint8_t* amb)
{
    if (!F->ok || res <= 0) return -1;
    for (int32_t py = 0; py < res; ++py)
        for (int32_t px = 0; px < res; ++px)
            zb_pixel(tri, nt, F, res, delta_px, px, py, &zbuf[(size_t)py * res + px], &amb[(size_t)py * res + px]);
    return 0;
}

typedef struct {
    int32_t res;
    double n, f;              /* clip planes (metres) */
    double eps;               /* +-eps depth tolerance (metres) */
    double delta_px;          /* pixel-position margin of the ambiguity bookkeeping (pixels) */
    double delta_w_rel;       /* depth margin of the ambiguity bookkeeping (relative) */
} ora_zb_params;

typedef struct {
    int64_t in_cone, visible, ambiguous, skipped_fixations;
} ora_zb_stats;

typedef struct {
    const float* tri; int64_t nt;
    const ora_frustum* F; const double* Z; const uint8_t* A; int32_t res;
    int64_t f0, f1;
    const ora_zb_params* zp;
    int err;
} ora_render_job;

static void* render_range(void* arg)
{
    ora_render_job* J = (ora_render_job*)arg;
    size_t px = (size_t)J->res * (size_t)J->res;
    for (int64_t f = J->f0; f < J->f1; ++f) {
        if (!J->F[f].ok) continue;
        if (ora_zb_render(J->tri, J->nt, &J->F[f], J->res, J->zp->delta_px, (double*)J->Z + px * f,
                          (uint8_t*)J->A + px * f))
            J->err = -1;
    }
    return NULL;
}

typedef struct {
    const float* tri; int64_t nt;
    const double* sxyz; int64_t s0, s1, ns;
    const float *eye, *gaze, *dur; const int32_t* win; int64_t nf;
    const ora_frustum* F; const double* Z; const uint8_t* A;
    const ora_params* prm; const ora_zb_params* zp;
    double *density, *amb, *sens;
    ora_zb_stats st;
    int record;
    int64_t *ps; int32_t* pf; uint8_t* pflag; double* pg; int64_t np, cap;
    int err;
} ora_zb_job;

/* The z-buffer visibility of sample sp in frustum F, with the ambiguity bookkeeping: pixel depths
 * come from `look` (a stored z-buffer, or pixels cast on demand). */
typedef void (*zb_lookup_fn)(void* ctx, int32_t px, int32_t py, double* depth, uint8_t* amb);

static void zb_decide(const ora_frustum* F, const double sp[3], const ora_zb_params* zp, zb_lookup_fn look, void* ctx,
                      int* vis_out, int* amb_out)
{
    const int32_t res = zp->res;
    double v[3] = {sp[0] - F->e[0], sp[1] - F->e[1], sp[2] - F->e[2]};
    double x = v3_dot(v, F->right), y = v3_dot(v, F->up), w = v3_dot(v, F->fwd);
    int vis = 0, amb_vis = 0;
    {
        const double band = zb_depth_band(sp, F->e);   /* the sample's own FP32 camera depth */
        if (fabs(w - F->n) <= band || fabs(w - F->f) <= band) amb_vis = 1;
    }
    if (w >= F->n && w <= F->f) {
        double u = (F->n * x / w - F->l) / (F->r - F->l) * res;
        double q = (F->n * y / w - F->b) / (F->t - F->b) * res;
        double dp = zp->delta_px;
        if (u < dp || u > res - dp || q < dp || q > res - dp) {
            /* on the crop border: inside or filtered out depending on rounding */
            if (!(u < -dp || u > res + dp || q < -dp || q > res + dp)) amb_vis = 1;
        }
        if (u >= 0.0 && u <= res && q >= 0.0 && q <= res) {
            int32_t cx[2], cy[2];
            cx[0] = (int32_t)floor(u - dp); cx[1] = (int32_t)floor(u + dp);
            cy[0] = (int32_t)floor(q - dp); cy[1] = (int32_t)floor(q + dp);
            for (int k = 0; k < 2; ++k) {
                if (cx[k] < 0) cx[k] = 0;
                if (cx[k] > res - 1) cx[k] = res - 1;
                if (cy[k] < 0) cy[k] = 0;
                if (cy[k] > res - 1) cy[k] = res - 1;
            }
            int32_t px = (int32_t)floor(u), py = (int32_t)floor(q);
            if (px > res - 1) px = res - 1;
            if (py > res - 1) py = res - 1;
            double z0;
            uint8_t a0;
            look(ctx, px, py, &z0, &a0);
            vis = isfinite(z0) && fabs(w - z0) <= zp->eps;
            double dw = zp->delta_w_rel * w;
            for (int a = 0; a < 2; ++a) {
                for (int b = 0; b < 2; ++b) {
                    double z;
                    uint8_t am;
                    look(ctx, cx[a], cy[b], &z, &am);
                    if (am) amb_vis = 1;
                    if ((isfinite(z) && fabs(w - z) <= zp->eps) != vis) amb_vis = 1;
                    if (isfinite(z) && fabs(fabs(w - z) - zp->eps) <= dw) amb_vis = 1;
                }
            }
        }
    }
    *vis_out = vis;
    *amb_out = amb_vis;
}

typedef struct { const double* Z; const uint8_t* A; int32_t res; } zb_stored;

static void zb_lookup_stored(void* ctx, int32_t px, int32_t py, double* depth, uint8_t* amb)
{
    const zb_stored* S = (const zb_stored*)ctx;
    size_t p = (size_t)py * S->res + px;
    *depth = S->Z[p];
    *amb = S->A[p];
}

static void* zb_accumulate_range(void* arg)
{
    ora_zb_job* J = (ora_zb_job*)arg;
    const ora_params* P = J->prm;
    const ora_zb_params* zp = J->zp;
    const int32_t res = zp->res;
    const size_t npx = (size_t)res * (size_t)res;
    double tan_t = tan(P->theta);
    for (int64_t s = J->s0; s < J->s1; ++s) {
        const double* sp = J->sxyz + 3 * s;
        for (int64_t f = 0; f < J->nf; ++f) {
            int32_t wi = J->win[f];
            if (wi < 0 || !J->F[f].ok) continue;
            double e[3] = {J->eye[3 * f], J->eye[3 * f + 1], J->eye[3 * f + 2]};
            double r[3] = {J->gaze[3 * f], J->gaze[3 * f + 1], J->gaze[3 * f + 2]};
            pair_eval pe;
            int in = gaussian_pair(sp, e, r, (double)J->dur[f], P->theta, P->cutoff, P->cone_band, &pe);
            if (!in && !pe.edge) continue;
            const ora_frustum* F = &J->F[f];
            zb_stored S = {J->Z + npx * f, J->A + npx * f, res};
            int vis = 0, amb_vis = 0;
            zb_decide(F, sp, zp, zb_lookup_stored, &S, &vis, &amb_vis);
            size_t o = (size_t)wi * (size_t)J->ns + (size_t)s;
            uint8_t flag = (uint8_t)((in ? PF_IN_CONE : 0) | (vis ? PF_VISIBLE : 0) | (amb_vis ? PF_VIS_AMBIG : 0)
                                     | (pe.edge ? PF_CONE_EDGE : 0));
            if (in) {
                J->st.in_cone++;
                if (vis) {
                    J->st.visible++;
                    J->density[o] += pe.g;
                    if (J->sens)
                        J->sens[o] += pe.g * (pe.d2 / (pe.d1 * pe.d1)) * (1.0 + pe.d2 / pe.d1) / (tan_t * tan_t);
                }
            }
            if (amb_vis || pe.edge) {
                if (J->amb) J->amb[o] += pe.g;
                J->st.ambiguous += amb_vis;
            }
            if (J->record) {
                ora_job tmp;
                memset(&tmp, 0, sizeof(tmp));
                tmp.ps = J->ps; tmp.pf = J->pf; tmp.pflag = J->pflag; tmp.pg = J->pg; tmp.np = J->np; tmp.cap = J->cap;
                push_pair(&tmp, s, (int32_t)f, flag, pe.g);
                J->ps = tmp.ps; J->pf = tmp.pf; J->pflag = tmp.pflag; J->pg = tmp.pg; J->np = tmp.np; J->cap = tmp.cap;
                if (tmp.err) J->err = tmp.err;
            }
        }
    }
    return NULL;
}

/* The z-buffer form of the accumulation (Sections 3.2.2 and 3.3.2): for every fixation its
 * frustum and z-buffer, then for every sample x fixation pair the exact 4 sigma cone test, the
 * crop-window filter and the +-eps depth comparison in the sample's pixel; visible in-cone
 * pairs add the same Gaussian as the ray form. Fixations whose cone is not entirely in front
 * of their camera are skipped (counted). frusta_out (nf) and zbuf_out / amb_out (nf * res^2)
 * may be NULL. Arguments otherwise as ora_accumulate. */
int ora_zb_accumulate(const float* tri, int64_t nt, const double* sxyz, int64_t ns, const float* eye,
                      const float* gaze, const float* dur, const double* ts, const float* cam_fwd,
                      const float* cam_up, int64_t nf, const ora_params* prm, const ora_zb_params* zp,
                      double* density, double* amb, double* sens, ora_zb_stats* st, int64_t rec_cap,
                      int64_t* rec_s, int32_t* rec_f, uint8_t* rec_flag, double* rec_g, int64_t* n_rec,
                      ora_frustum* frusta_out, double* zbuf_out, uint8_t* amb_out)
{
    size_t npx = (size_t)zp->res * (size_t)zp->res;
    int32_t* win = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
    ora_frustum* F = (ora_frustum*)calloc((size_t)(nf > 0 ? nf : 1), sizeof(ora_frustum));
    double* Z = zbuf_out ? zbuf_out : (double*)malloc(sizeof(double) * npx * (size_t)(nf > 0 ? nf : 1));
    uint8_t* A = amb_out ? amb_out : (uint8_t*)malloc(npx * (size_t)(nf > 0 ? nf : 1));
    if (!win || !F || !Z || !A) return -2;
    ora_fixation_windows(ts, nf, prm->t_begin, prm->t_end, prm->window_s, prm->n_windows, win);
    ora_zb_stats tot = {0, 0, 0, 0};
    for (int64_t f = 0; f < nf; ++f) {
        if (ora_zb_frustum(eye + 3 * f, gaze + 3 * f, cam_fwd + 3 * f, cam_up + 3 * f, prm->theta, prm->cutoff, zp->n,
                           zp->f, &F[f]))
            F[f].ok = 0;
        if (!F[f].ok && win[f] >= 0) tot.skipped_fixations++;
    }
    int nth = prm->nthreads > 0 ? prm->nthreads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nth < 1) nth = 1;
    int err = 0;
    {
        int nr = nth < nf ? nth : (nf > 0 ? (int)nf : 1);
        ora_render_job* rj = (ora_render_job*)calloc((size_t)nr, sizeof(ora_render_job));
        pthread_t* th = (pthread_t*)calloc((size_t)nr, sizeof(pthread_t));
        for (int i = 0; i < nr; ++i) {
            rj[i].tri = tri; rj[i].nt = nt; rj[i].F = F; rj[i].Z = Z; rj[i].A = A; rj[i].res = zp->res;
            rj[i].f0 = nf * i / nr; rj[i].f1 = nf * (i + 1) / nr; rj[i].zp = zp;
        }
        for (int i = 1; i < nr; ++i) pthread_create(&th[i], NULL, render_range, &rj[i]);
        render_range(&rj[0]);
        for (int i = 1; i < nr; ++i) pthread_join(th[i], NULL);
        for (int i = 0; i < nr; ++i) if (rj[i].err) err = rj[i].err;
        free(rj); free(th);
    }
    size_t nout = (size_t)prm->n_windows * (size_t)ns;
    memset(density, 0, sizeof(double) * nout);
    if (amb) memset(amb, 0, sizeof(double) * nout);
    if (sens) memset(sens, 0, sizeof(double) * nout);
    if (nth > ns) nth = ns > 0 ? (int)ns : 1;
    ora_zb_job* jobs = (ora_zb_job*)calloc((size_t)nth, sizeof(ora_zb_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nth, sizeof(pthread_t));
    for (int i = 0; i < nth; ++i) {
        ora_zb_job* J = &jobs[i];
        J->tri = tri; J->nt = nt; J->sxyz = sxyz; J->ns = ns; J->s0 = ns * i / nth; J->s1 = ns * (i + 1) / nth;
        J->eye = eye; J->gaze = gaze; J->dur = dur; J->win = win; J->nf = nf;
        J->F = F; J->Z = Z; J->A = A; J->prm = prm; J->zp = zp;
        J->density = density; J->amb = amb; J->sens = sens; J->record = rec_cap >= 0;
    }
    for (int i = 1; i < nth; ++i) pthread_create(&th[i], NULL, zb_accumulate_range, &jobs[i]);
    zb_accumulate_range(&jobs[0]);
    for (int i = 1; i < nth; ++i) pthread_join(th[i], NULL);
    int64_t nrec = 0;
    for (int i = 0; i < nth; ++i) {
        ora_zb_job* J = &jobs[i];
        if (J->err) err = J->err;
        tot.in_cone += J->st.in_cone; tot.visible += J->st.visible; tot.ambiguous += J->st.ambiguous;
        for (int64_t k = 0; k < J->np; ++k, ++nrec) {
            if (nrec < rec_cap) {
                rec_s[nrec] = J->ps[k]; rec_f[nrec] = J->pf[k]; rec_flag[nrec] = J->pflag[k]; rec_g[nrec] = J->pg[k];
            }
        }
        free(J->ps); free(J->pf); free(J->pflag); free(J->pg);
    }
    if (st) *st = tot;
    if (n_rec) *n_rec = nrec;
    if (frusta_out) memcpy(frusta_out, F, sizeof(ora_frustum) * (size_t)nf);
    free(jobs); free(th); free(win); free(F);
    if (!zbuf_out) free(Z);
    if (!amb_out) free(A);
    return err;
}

/* Sampled form of the z-buffer decision for full-size scenes: for each given (sample, fixation)
 * pair, the fixation's frustum and only the pixels the decision reads, each cast against every
 * triangle as ora_zb_render does. vis/amb per pair; frustum_ok 0 when the fixation has no crop
 * window. Threads over pairs. */
typedef struct {
    const float* tri; int64_t nt; const ora_frustum* F; int32_t res; double delta_px;
    int32_t cx[5], cy[5]; double cz[5]; uint8_t ca[5]; int nc;   /* pixels already cast for this pair */
} zb_cast;

static void zb_lookup_cast(void* ctx, int32_t px, int32_t py, double* depth, uint8_t* amb)
{
    zb_cast* C = (zb_cast*)ctx;
    for (int k = 0; k < C->nc; ++k)
        if (C->cx[k] == px && C->cy[k] == py) { *depth = C->cz[k]; *amb = C->ca[k]; return; }
    zb_pixel(C->tri, C->nt, C->F, C->res, C->delta_px, px, py, depth, amb);
    if (C->nc < 5) { C->cx[C->nc] = px; C->cy[C->nc] = py; C->cz[C->nc] = *depth; C->ca[C->nc] = *amb; ++C->nc; }
}

typedef struct {
    const float* tri; int64_t nt; const double* sxyz; const float *eye, *gaze, *fwd, *up;
    double theta, cutoff; const ora_zb_params* zp; int8_t *vis, *amb, *ok; int64_t p0, p1;
} zb_pairs_job;

static void* zb_pairs_range(void* arg)
{
    zb_pairs_job* J = (zb_pairs_job*)arg;
    for (int64_t k = J->p0; k < J->p1; ++k) {
        ora_frustum F;
        if (ora_zb_frustum(J->eye + 3 * k, J->gaze + 3 * k, J->fwd + 3 * k, J->up + 3 * k, J->theta, J->cutoff,
                           J->zp->n, J->zp->f, &F) || !F.ok) {
            J->ok[k] = 0; J->vis[k] = 0; J->amb[k] = 0;
            continue;
        }
        zb_cast C;
        memset(&C, 0, sizeof(C));
        C.tri = J->tri; C.nt = J->nt; C.F = &F; C.res = J->zp->res; C.delta_px = J->zp->delta_px;
        int vis, amb;
        zb_decide(&F, J->sxyz + 3 * k, J->zp, zb_lookup_cast, &C, &vis, &amb);
        J->ok[k] = 1; J->vis[k] = (int8_t)vis; J->amb[k] = (int8_t)amb;
    }
    return NULL;
}

int ora_zb_pairs(const float* tri, int64_t nt, int64_t n, const double* sxyz, const float* eye, const float* gaze,
                 const float* fwd, const float* up, double theta, double cutoff, const ora_zb_params* zp,
                 int8_t* vis, int8_t* amb, int8_t* ok, int32_t nthreads)
{
    int nth = nthreads > 0 ? nthreads : (int)sysconf(_SC_NPROCESSORS_ONLN);
    if (nth < 1) nth = 1;
    if (nth > n) nth = n > 0 ? (int)n : 1;
    zb_pairs_job* jobs = (zb_pairs_job*)calloc((size_t)nth, sizeof(zb_pairs_job));
    pthread_t* th = (pthread_t*)calloc((size_t)nth, sizeof(pthread_t));
    if (!jobs || !th) { free(jobs); free(th); return -2; }
    for (int i = 0; i < nth; ++i) {
        zb_pairs_job* J = &jobs[i];
        J->tri = tri; J->nt = nt; J->sxyz = sxyz; J->eye = eye; J->gaze = gaze; J->fwd = fwd; J->up = up;
        J->theta = theta; J->cutoff = cutoff; J->zp = zp; J->vis = vis; J->amb = amb; J->ok = ok;
        J->p0 = n * i / nth; J->p1 = n * (i + 1) / nth;
    }
    for (int i = 1; i < nth; ++i) pthread_create(&th[i], NULL, zb_pairs_range, &jobs[i]);
    zb_pairs_range(&jobs[0]);
    for (int i = 1; i < nth; ++i) pthread_join(th[i], NULL);
    free(jobs); free(th);
    return 0;
}
