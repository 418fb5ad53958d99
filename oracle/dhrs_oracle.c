/*
 * dhrs_oracle.c -- CPU oracle for the DHR+S server hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and the
 * cpu_baseline / reference legs of bench.py may load this library.  It shares
 * no code, header, table or constant generator with the CUDA library; the two
 * meet only through the seeded inputs of the `workloads` package and through
 * the written specification of the sampling formulas.
 *
 * What it computes, and where each part comes from:
 *   - primary visibility (G-buffer from pixel-centre rays): stands in for the
 *     client rasteriser of Section 1 / Section 3.3 (depth, normal, mesh id);
 *   - soft shadow: one shadow ray per light whose direction is jittered
 *     uniformly over the light's cone (Section 3.1, Fig. 1);
 *   - ambient occlusion: cosine-weighted hemisphere rays bounded by radius r,
 *     O = N_unoccluded / N (Section 3.2, Eqs. 1-3);
 *   - modified SVGF: temporal reprojection + exponential moving average,
 *     moment variance with a 7x7 depth/normal-weighted spatial fallback, and
 *     edge-stopping a-trous iterations (Section 3.3);
 *   - selective shadow rays: a shadow map per light and the classification
 *     of each receiver as lit, umbra or to be ray traced (Section 5).
 *
 * Precision: geometry, intersection and filtering run in double.  Where a
 * floating-point value decides an integer (disk-sample rejection, validity
 * of reprojected history taps) the decision is taken in binary32 with every
 * operation written out and correctly rounded, so that a binary32 GPU kernel
 * can take the same decision.  The reprojection decision is also written as
 * its plain definition in double (reproject_f64, orc_reproject_check); the
 * two must agree wherever the double decision is not within a small margin
 * of a threshold.  Compile with -ffp-contract=off and without -ffast-math.
 *
 * Intersection is brute force over every triangle (Moller-Trumbore in double);
 * there is no acceleration structure here.
 *
 * Parity pins: see tests/test_oracle_*.py.  Every exported function below is
 * pinned by at least one closed form, invariant or independent library
 * routine there.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAX_LIGHTS 8
#define ORC_BACKGROUND 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Structures (ctypes mirrors live in oracle/__init__.py)                   */
/* ------------------------------------------------------------------------ */
typedef struct {
    float pos[3], fwd[3], right[3], up[3];
    float tan_half_fov_y;
    int32_t width, height;
} orc_camera;

typedef struct {
    int32_t n_lights;
    float light_dir[ORC_MAX_LIGHTS][3];   /* unit, pointing toward the light */
    float cone_half_angle[ORC_MAX_LIGHTS];/* radians */
    float ao_radius;
    int32_t ao_spp;
    uint32_t frame;
    uint32_t seed;
} orc_trace_params;

typedef struct {
    double eps_abs;   /* world-space tolerance for the grazing classification */
    double eps_rel;   /* ... plus eps_rel * (|origin|_inf + distance along the ray) */
} orc_margin;

typedef struct {
    int64_t n;
    double *v0, *e1, *e2;    /* [n][3] */
    double *inv_h;           /* [n][3]: 1 / (distance of vertex k to the opposite edge) */
    double *nrm;             /* [n][3] unit geometric normal (e1 x e2) */
    uint32_t *mesh;
    double extent;           /* largest |coordinate| of any vertex */
    double bmin[3], bmax[3]; /* bounds of the triangles' vertices (0 without triangles) */
} orc_scene;

typedef struct {
    double alpha, sigma_z, sigma_n, sigma_l, eps_z, eps_l;
    int32_t ao_spp, levels, fixed_alpha, wl_in_atrous;
    int32_t kernel_width;    /* 5 (or 0): B3-spline taps; 3: (1/4, 1/2, 1/4) */
} orc_svgf_params;

/* per-pixel record of the temporal step (used by the adjoint) */
typedef struct {
    int fg, valid, n, spatial;
    int x0, y0, ok;        /* bilinear taps (x0 + (k&1), y0 + (k>>1)), valid bits */
    double a;              /* effective alpha */
    double beta[4];        /* normalised weights of the valid taps */
} orc_trec;

/* ======================================================================== */
/* 1. Random numbers: pcg4d of Jarzynski & Olano, "Hash Functions for GPU   */
/*    Rendering", JCGT 9(3), 2020.  The paper only says the jitter is       */
/*    random (Section 3.1) and that AO rays are shot at random (Section     */
/*    3.3); this counter-based hash is the chosen generator.                */
/* ======================================================================== */
void orc_pcg4d(uint32_t v[4])
{
    /* linear congruential step on each lane */
    for (int k = 0; k < 4; ++k) v[k] = v[k] * 1664525u + 1013904223u;
    /* cross-lane mixing, shift, mixing again */
    v[0] += v[1] * v[3];
    v[1] += v[2] * v[0];
    v[2] += v[0] * v[1];
    v[3] += v[1] * v[2];
    for (int k = 0; k < 4; ++k) v[k] ^= v[k] >> 16;
    v[0] += v[1] * v[3];
    v[1] += v[2] * v[0];
    v[2] += v[0] * v[1];
    v[3] += v[1] * v[2];
}

/* top 24 bits of a hash word -> exact float in [0, 1) */
float orc_u24(uint32_t h) { return (float)(h >> 8) * (1.0f / 16777216.0f); }

/* Hash input for one sample: (px, py, frame ^ seed, stream) with
 * stream = ray_type << 24 | (sample & 0xFFFF) << 8 | call. */
static void hash_call(uint32_t px, uint32_t py, uint32_t frame, uint32_t seed,
                      uint32_t ray_type, uint32_t sample, uint32_t call, uint32_t out[4])
{
    out[0] = px;
    out[1] = py;
    out[2] = frame ^ seed;
    out[3] = (ray_type << 24) | ((sample & 0xFFFFu) << 8) | (call & 0xFFu);
    orc_pcg4d(out);
}

/* Uniform point on the unit disk by rejection: up to 8 candidates, two per
 * hash call (u0,u1) then (u2,u3); the test x*x + y*y < 1 is taken in
 * binary32.  Returns the index of the accepted candidate, 8 if all were
 * rejected (then the point is the centre). */
int orc_disk_point(uint32_t px, uint32_t py, uint32_t frame, uint32_t seed,
                   uint32_t ray_type, uint32_t sample, float xy[2])
{
    for (uint32_t call = 0; call < 4; ++call) {
        uint32_t h[4];
        hash_call(px, py, frame, seed, ray_type, sample, call, h);
        for (int half = 0; half < 2; ++half) {
            volatile float x = 2.0f * orc_u24(h[2 * half]) - 1.0f;
            volatile float y = 2.0f * orc_u24(h[2 * half + 1]) - 1.0f;
            volatile float xx = x * x;
            volatile float yy = y * y;
            volatile float s = xx + yy;
            if (s < 1.0f) {
                xy[0] = x;
                xy[1] = y;
                return (int)(2 * call + half);
            }
        }
    }
    xy[0] = 0.0f;
    xy[1] = 0.0f;
    return 8;
}

/* Orthonormal basis (T, B) around unit n: the branch-free construction of
 * Duff et al., "Building an Orthonormal Basis, Revisited", JCGT 6(1), 2017.
 * binary32 version, one rounding per written operation. */
void orc_onb_f32(const float n[3], float T[3], float B[3])
{
    volatile float sgn = copysignf(1.0f, n[2]);
    volatile float den = sgn + n[2];
    volatile float a = -1.0f / den;
    volatile float nxny = n[0] * n[1];
    volatile float b = nxny * a;
    volatile float snx = sgn * n[0];
    volatile float snxnx = snx * n[0];
    volatile float t0 = snxnx * a;
    T[0] = 1.0f + t0;
    T[1] = sgn * b;
    T[2] = -(sgn * n[0]);
    volatile float nyny = n[1] * n[1];
    volatile float b1 = nyny * a;
    B[0] = b;
    B[1] = sgn + b1;
    B[2] = -n[1];
}

/* Cosine-weighted direction about n (Malley's method: a uniform disk point
 * lifted to the hemisphere); Section 3.2 samples AO directions with a
 * cosine-weighted pdf.  binary32: d = (x T + y B) + z n. */
void orc_ao_dir_f32(const float n[3], float x, float y, float d[3])
{
    float T[3], B[3];
    orc_onb_f32(n, T, B);
    volatile float xx = x * x, yy = y * y;
    volatile float s = xx + yy;
    volatile float om = 1.0f - s;
    volatile float z = sqrtf(om > 0.0f ? om : 0.0f);
    for (int k = 0; k < 3; ++k) {
        volatile float a = x * T[k];
        volatile float b = y * B[k];
        volatile float c = z * n[k];
        volatile float ab = a + b;
        d[k] = ab + c;
    }
}

/* Soft-shadow direction, Section 3.1 / Fig. 1b: the direction toward the
 * light is offset by a bounded random amount inside the cone of half angle
 * theta and renormalised to unit length (its length does not change).
 * Disk form: q = l + tan(theta) (x T_l + y B_l), d = q / |q|.  binary32. */
void orc_cone_dir_f32(const float l[3], float tan_theta, float x, float y, float d[3])
{
    float T[3], B[3];
    orc_onb_f32(l, T, B);
    float q[3];
    for (int k = 0; k < 3; ++k) {
        volatile float a = x * T[k];
        volatile float b = y * B[k];
        volatile float ab = a + b;
        volatile float o = tan_theta * ab;
        q[k] = l[k] + o;
    }
    volatile float q0 = q[0] * q[0], q1 = q[1] * q[1], q2 = q[2] * q[2];
    volatile float s01 = q0 + q1;
    volatile float s = s01 + q2;
    volatile float len = sqrtf(s);
    for (int k = 0; k < 3; ++k) d[k] = q[k] / len;
}


/* Batch form used by the bit-exactness test: for each (pixel, sample) the
 * accepted disk point and both binary32 directions. */
void orc_sample_batch_f32(int64_t n, const uint32_t* px, const uint32_t* py, uint32_t frame,
                          uint32_t seed, uint32_t sample, const float* normals /*[n][3]*/,
                          const float* light /*[3]*/, float tan_theta,
                          float* disk_ao /*[n][2]*/, float* dir_ao /*[n][3]*/,
                          float* disk_sh /*[n][2]*/, float* dir_sh /*[n][3]*/)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        orc_disk_point(px[i], py[i], frame, seed, 1u, sample, disk_ao + 2 * i);
        orc_ao_dir_f32(normals + 3 * i, disk_ao[2 * i], disk_ao[2 * i + 1], dir_ao + 3 * i);
        orc_disk_point(px[i], py[i], frame, seed, 0u, sample, disk_sh + 2 * i);
        orc_cone_dir_f32(light, tan_theta, disk_sh[2 * i], disk_sh[2 * i + 1], dir_sh + 3 * i);
    }
}

/* ======================================================================== */
/* 2. Scene and brute-force ray casting (double)                            */
/* ======================================================================== */
static inline void sub3(const double* a, const double* b, double* o)
{ o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline void cross3(const double* a, const double* b, double* o)
{ o[0] = a[1] * b[2] - a[2] * b[1]; o[1] = a[2] * b[0] - a[0] * b[2]; o[2] = a[0] * b[1] - a[1] * b[0]; }
static inline double dot3(const double* a, const double* b)
{ return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline double norm3(const double* a) { return sqrt(dot3(a, a)); }

orc_scene* orc_scene_create(const float* verts, const uint32_t* idx, const uint32_t* mesh,
                            int64_t n_vertices, int64_t n_tris)
{
    orc_scene* s = (orc_scene*)calloc(1, sizeof(orc_scene));
    s->n = n_tris;
    s->v0 = (double*)malloc(sizeof(double) * 3 * (size_t)n_tris);
    s->e1 = (double*)malloc(sizeof(double) * 3 * (size_t)n_tris);
    s->e2 = (double*)malloc(sizeof(double) * 3 * (size_t)n_tris);
    s->inv_h = (double*)malloc(sizeof(double) * 3 * (size_t)n_tris);
    s->nrm = (double*)malloc(sizeof(double) * 3 * (size_t)n_tris);
    s->mesh = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)n_tris);
    double ext = 0.0;
    for (int64_t v = 0; v < n_vertices * 3; ++v) ext = fmax(ext, fabs((double)verts[v]));
    s->extent = ext;
    for (int c = 0; c < 3; ++c) {
        s->bmin[c] = n_tris > 0 ? INFINITY : 0.0;
        s->bmax[c] = n_tris > 0 ? -INFINITY : 0.0;
    }
    for (int64_t i = 0; i < n_tris; ++i) {
        double p[3][3];
        for (int k = 0; k < 3; ++k)
            for (int c = 0; c < 3; ++c) {
                p[k][c] = (double)verts[3 * (int64_t)idx[3 * i + k] + c];
                s->bmin[c] = fmin(s->bmin[c], p[k][c]);
                s->bmax[c] = fmax(s->bmax[c], p[k][c]);
            }
        double *v0 = s->v0 + 3 * i, *e1 = s->e1 + 3 * i, *e2 = s->e2 + 3 * i;
        memcpy(v0, p[0], sizeof(double) * 3);
        sub3(p[1], p[0], e1);
        sub3(p[2], p[0], e2);
        double c[3];
        cross3(e1, e2, c);
        double a2 = norm3(c);                      /* twice the area */
        double e12[3];
        sub3(p[2], p[1], e12);
        double len_opp[3] = {norm3(e12), norm3(e2), norm3(e1)};  /* edges opposite v0, v1, v2 */
        for (int k = 0; k < 3; ++k) {
            double h = (a2 > 0.0 && len_opp[k] > 0.0) ? a2 / len_opp[k] : 0.0;
            s->inv_h[3 * i + k] = h > 0.0 ? 1.0 / h : 0.0;
            s->nrm[3 * i + k] = a2 > 0.0 ? c[k] / a2 : 0.0;
        }
        s->mesh[i] = mesh ? mesh[i] : 0u;
    }
    return s;
}

void orc_scene_destroy(orc_scene* s)
{
    if (!s) return;
    free(s->v0); free(s->e1); free(s->e2); free(s->inv_h); free(s->nrm); free(s->mesh);
    free(s);
}

/* Moller & Trumbore, "Fast, Minimum Storage Ray/Triangle Intersection"
 * (JGT 1997), double precision.  Returns 0 when the ray is parallel to the
 * plane; otherwise the ray parameter t of the plane crossing and its
 * barycentrics (u on v1, v on v2; 1-u-v on v0). */
static inline int mt_plane(const orc_scene* s, int64_t i, const double* o, const double* d,
                           double* t, double* u, double* v)
{
    const double *v0 = s->v0 + 3 * i, *e1 = s->e1 + 3 * i, *e2 = s->e2 + 3 * i;
    double pv[3], tv[3], qv[3];
    cross3(d, e2, pv);
    double det = dot3(e1, pv);
    if (det == 0.0) return 0;
    double inv = 1.0 / det;
    sub3(o, v0, tv);
    *u = dot3(tv, pv) * inv;
    cross3(tv, e1, qv);
    *v = dot3(d, qv) * inv;
    *t = dot3(e2, qv) * inv;
    return 1;
}

/* signed world distance from the plane crossing to the triangle boundary
 * (positive inside) */
static inline double edge_margin(const orc_scene* s, int64_t i, double u, double v)
{
    const double* ih = s->inv_h + 3 * i;
    double w = 1.0 - u - v;
    double m0 = ih[0] > 0.0 ? w / ih[0] : -INFINITY;
    double m1 = ih[1] > 0.0 ? u / ih[1] : -INFINITY;
    double m2 = ih[2] > 0.0 ? v / ih[2] : -INFINITY;
    return fmin(m0, fmin(m1, m2));
}

static inline double inf_norm3(const double* a)
{ return fmax(fabs(a[0]), fmax(fabs(a[1]), fabs(a[2]))); }

typedef struct {
    int hit;              /* exact outcome */
    int ambiguous;        /* outcome may flip under a perturbation within the margin */
    double t;             /* closest: hit distance (ray parameter) */
    int64_t tri;          /* closest: triangle index (ties: smaller index) */
    double u, v;
} cast_result;

/* Closest hit with t in (tmin, tmax).  Ambiguity flags a silhouette, an
 * edge crossing or a near-tie between surfaces within the margin. */
static cast_result cast_closest(const orc_scene* s, const double* o, const double* d,
                                double tmin, double tmax, const orc_margin* mg)
{
    cast_result r = {0, 0, INFINITY, -1, 0, 0};
    double dl = norm3(d);
    double oinf = inf_norm3(o);
    for (int64_t i = 0; i < s->n; ++i) {
        double t, u, v;
        if (!mt_plane(s, i, o, d, &t, &u, &v)) continue;
        if (!(t > tmin && t < tmax)) continue;
        if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
            if (t < r.t || (t == r.t && i < r.tri)) {
                r.t = t; r.tri = i; r.u = u; r.v = v; r.hit = 1;
            }
        }
    }
    /* ambiguity pass */
    double t_ref = r.hit ? r.t : tmax;
    for (int64_t i = 0; i < s->n; ++i) {
        double t, u, v;
        if (!mt_plane(s, i, o, d, &t, &u, &v)) continue;
        if (!(t > tmin)) continue;
        double tw = t * dl;
        double eps = mg->eps_abs + mg->eps_rel * (oinf + tw);
        double cosang = fabs(dot3(d, s->nrm + 3 * i)) / dl;
        double eps_t = eps / fmax(cosang, 1e-3);
        double m = edge_margin(s, i, u, v);
        if (i == r.tri) {
            if (m < eps) r.ambiguous = 1;          /* hit close to an edge */
            continue;
        }
        if (m >= -eps && tw < t_ref * dl + eps_t && t < tmax) {
            r.ambiguous = 1;                       /* another surface within the margin in front */
            break;
        }
    }
    return r;
}

/* Any hit with t in (tmin, tmax) (occlusion test).  The outcome is
 * ambiguous when a perturbation of the ray within the margin could change
 * it: a surface near a triangle edge, near tmax, or crossing the ray within
 * four binary32 units in the last place of the origin's largest coordinate
 * behind it (the origin of a secondary ray is derived from a hit point that
 * each implementation rounds in its own precision, so a surface that close
 * may lie on either side of it; the hit surface itself lies 16 such units
 * behind and is not counted). */
static cast_result cast_any(const orc_scene* s, const double* o, const double* d,
                            double tmin, double tmax, const orc_margin* mg)
{
    cast_result r = {0, 0, INFINITY, -1, 0, 0};
    double dl = norm3(d);
    double oinf = inf_norm3(o);
    int loose = 0, strict = 0;
    double tmax_w = tmax * dl, tmin_w = tmin * dl;
    double eps_o = 4.0 * ldexp(fmax(oinf, 0x1p-20), -23);
    for (int64_t i = 0; i < s->n; ++i) {
        double t, u, v;
        if (!mt_plane(s, i, o, d, &t, &u, &v)) continue;
        double tw = t * dl;
        double eps = mg->eps_abs + mg->eps_rel * (oinf + fmin(fabs(tw), 4.0 * s->extent));
        double cosang = fabs(dot3(d, s->nrm + 3 * i)) / dl;
        double eps_t = eps / fmax(cosang, 1e-3);
        double m = edge_margin(s, i, u, v);
        if (!(t > tmin)) {
            /* behind the origin: a surface within the rounding of it */
            if (m >= -eps && tw > tmin_w - eps_o / fmax(cosang, 1e-3)) loose = 1;
            continue;
        }
        if (m >= 0.0 && t < tmax) {
            r.hit = 1;
            if (r.tri < 0) { r.tri = i; r.t = t; }
        }
        if (m >= -eps && tw < tmax_w + eps_t) loose = 1;
        if (m >= eps && tw > eps_t && tw < tmax_w - eps_t) strict = 1;
        if (r.hit && strict) break;                /* certain occlusion */
    }
    r.ambiguous = (loose != strict);
    return r;
}

/* Public single-ray entry points (unit tests) */
void orc_cast(const orc_scene* s, const double* o, const double* d, double tmin, double tmax,
              int any_hit, const orc_margin* mg, int32_t* hit, int32_t* ambiguous,
              double* t, int64_t* tri, double* uv)
{
    cast_result r = any_hit ? cast_any(s, o, d, tmin, tmax, mg) : cast_closest(s, o, d, tmin, tmax, mg);
    *hit = r.hit; *ambiguous = r.ambiguous; *t = r.t; *tri = r.tri;
    if (uv) { uv[0] = r.u; uv[1] = r.v; }
}

/* Pixel-centre camera ray, unnormalised: D = f + sx r + sy u, so that the
 * ray parameter of a hit equals its linear view depth (dot(D, f) = 1 for an
 * orthonormal basis).  Image row 0 is the top row. */
static void camera_ray(const orc_camera* c, int x, int y, double o[3], double D[3])
{
    double W = c->width, H = c->height;
    double sx = (2.0 * (x + 0.5) / W - 1.0) * c->tan_half_fov_y * (W / H);
    double sy = (1.0 - 2.0 * (y + 0.5) / H) * c->tan_half_fov_y;
    for (int k = 0; k < 3; ++k) {
        o[k] = c->pos[k];
        D[k] = (double)c->fwd[k] + sx * c->right[k] + sy * c->up[k];
    }
}

/* Unit normal of triangle i in binary32 with a written operation order (the
 * specification shared with the GPU kernel, each step rounded once, no
 * fused multiply-add): a = v1 - v0, b = v2 - v0, c = a x b component by
 * component as (a_y b_z - a_z b_y, a_z b_x - a_x b_z, a_x b_y - a_y b_x),
 * l = sqrt((c_x^2 + c_y^2) + c_z^2) correctly rounded, n = c / l.  The
 * sample frame of the AO rays is built from it: a frame built from a
 * normal's sign bits (Duff et al.) switches where a component is zero, so
 * both sides must hold the same bits. */
static void normal_f32(const orc_scene* s, int64_t i, float n[3])
{
    const double *v0 = s->v0 + 3 * i, *e1 = s->e1 + 3 * i, *e2 = s->e2 + 3 * i;
    volatile float a[3], b[3];
    for (int k = 0; k < 3; ++k) {
        /* v1 - v0 rounded once: the double difference of two binary32 values is exact */
        a[k] = (float)e1[k];
        b[k] = (float)e2[k];
    }
    (void)v0;
    volatile float p0 = a[1] * b[2], q0 = a[2] * b[1];
    volatile float p1 = a[2] * b[0], q1 = a[0] * b[2];
    volatile float p2 = a[0] * b[1], q2 = a[1] * b[0];
    volatile float cx = p0 - q0, cy = p1 - q1, cz = p2 - q2;
    volatile float xx = cx * cx, yy = cy * cy, zz = cz * cz;
    volatile float xy = xx + yy;
    volatile float q = xy + zz;
    volatile float l = sqrtf(q);
    n[0] = cx / l;
    n[1] = cy / l;
    n[2] = cz / l;
}

/* 16 units in the last place of a binary32 value of magnitude m (m taken
 * as at least 2^-20): 16 * 2^(floor(log2 m) - 23), an exact power of two. */
static double surface_offset(double m)
{
    int ex;
    if (m < 0x1p-20) m = 0x1p-20;
    frexp(m, &ex);                   /* m = f 2^ex, f in [0.5, 1) */
    return ldexp(16.0, ex - 1 - 23);
}

/*
 * Trace pixels: G-buffer (closest hit of the pixel-centre ray), one
 * cone-jittered shadow ray per light, ao_spp cosine-weighted AO rays of
 * length r (Section 3.1, Section 3.2 Eqs. 1-3).
 *
 * Per pixel outputs: depth = dot(X - eye, forward) (+inf on a miss),
 * normal = unit geometric normal facing the eye, pos = X, tri and mesh id
 * (0xFFFFFFFF on a miss), shadow_mask bit k = light k unoccluded (all bits
 * set on a miss; 0 when the jittered direction points below the surface,
 * n . d <= 0, which the surface itself blocks), ao_count = N_unoccluded
 * (ao_spp on a miss).  Ambiguity
 * outputs: amb_primary, amb_shadow (bit per light), amb_ao (count of AO
 * rays whose outcome is within the margin).
 * Secondary rays start at X moved along n by 16 binary32 ulps of the hit
 * triangle's largest vertex coordinate and accept hits with t > 0.
 */
void orc_trace(const orc_scene* s, const orc_camera* cam, const orc_trace_params* tp,
               const orc_margin* mg, const int32_t* pixels /*[np][2] (x, y)*/, int64_t np,
               double* depth, double* normal, double* pos, int64_t* tri, uint32_t* mesh,
               uint8_t* shadow_mask, uint8_t* ao_count,
               uint8_t* amb_primary, uint8_t* amb_shadow, uint8_t* amb_ao)
{
    float tan_f[ORC_MAX_LIGHTS];       /* tan of each cone half angle, in double rounded once */
    for (int k = 0; k < tp->n_lights; ++k) tan_f[k] = (float)tan((double)tp->cone_half_angle[k]);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < np; ++i) {
        int x = pixels[2 * i], y = pixels[2 * i + 1];
        double o[3], D[3];
        camera_ray(cam, x, y, o, D);
        cast_result pr = cast_closest(s, o, D, 0.0, INFINITY, mg);
        amb_primary[i] = (uint8_t)pr.ambiguous;
        amb_shadow[i] = 0;
        amb_ao[i] = 0;
        if (!pr.hit) {
            depth[i] = INFINITY;
            for (int k = 0; k < 3; ++k) { normal[3 * i + k] = 0.0; pos[3 * i + k] = 0.0; }
            tri[i] = -1;
            mesh[i] = ORC_BACKGROUND;
            shadow_mask[i] = (uint8_t)((1u << tp->n_lights) - 1u);
            ao_count[i] = (uint8_t)tp->ao_spp;
            continue;
        }
        double X[3], n[3];
        float n32[3];
        for (int k = 0; k < 3; ++k) X[k] = o[k] + pr.t * D[k];
        /* the binary32 normal, facing the eye; a facing decision within
         * rounding of the grazing angle is ambiguous */
        const double* gn = s->nrm + 3 * pr.tri;
        double facing_eye = dot3(gn, D) / norm3(D);
        double side = facing_eye > 0.0 ? -1.0 : 1.0;
        if (fabs(facing_eye) < 1e-6) amb_primary[i] = 1;
        normal_f32(s, pr.tri, n32);
        for (int k = 0; k < 3; ++k) {
            n32[k] = (float)side * n32[k];
            n[k] = n32[k];
        }
        double f[3] = {cam->fwd[0], cam->fwd[1], cam->fwd[2]};
        double rel[3];
        sub3(X, o, rel);
        depth[i] = dot3(rel, f);
        for (int k = 0; k < 3; ++k) { normal[3 * i + k] = n[k]; pos[3 * i + k] = X[k]; }
        tri[i] = pr.tri;
        mesh[i] = s->mesh[pr.tri];
        /* secondary rays start at X moved along n by 16 ulps (binary32) of
         * the largest vertex coordinate of the hit triangle; t > 0 */
        double O[3];
        {
            double m = 0.0;
            const double *v0 = s->v0 + 3 * pr.tri, *e1 = s->e1 + 3 * pr.tri, *e2 = s->e2 + 3 * pr.tri;
            for (int k = 0; k < 3; ++k) {
                m = fmax(m, fabs(v0[k]));
                m = fmax(m, fabs(v0[k] + e1[k]));
                m = fmax(m, fabs(v0[k] + e2[k]));
            }
            double delta = surface_offset(m);
            for (int k = 0; k < 3; ++k) O[k] = X[k] + delta * n[k];
        }
        double tmin = 0.0;
        /* shadow rays, one per light */
        uint8_t m = 0, am = 0;
        for (int k = 0; k < tp->n_lights; ++k) {
            float xy[2];
            orc_disk_point((uint32_t)x, (uint32_t)y, tp->frame, tp->seed, 0u, (uint32_t)k, xy);
            /* the binary32 sample direction of the specification */
            float d32[3];
            orc_cone_dir_f32(tp->light_dir[k], tan_f[k], xy[0], xy[1], d32);
            double d[3] = {d32[0], d32[1], d32[2]};
            /* a direction below the surface is blocked by the surface itself */
            double facing = dot3(d, n);
            if (fabs(facing) < 1e-6) am |= (uint8_t)(1u << k);
            if (facing <= 0.0) continue;
            cast_result sr = cast_any(s, O, d, tmin, INFINITY, mg);
            if (!sr.hit) m |= (uint8_t)(1u << k);
            if (sr.ambiguous) am |= (uint8_t)(1u << k);
        }
        shadow_mask[i] = m;
        amb_shadow[i] = am;
        /* ambient occlusion rays, Eq. 3: count unoccluded rays of length r */
        int cnt = 0, amb = 0;
        for (int j = 0; j < tp->ao_spp; ++j) {
            float xy[2];
            orc_disk_point((uint32_t)x, (uint32_t)y, tp->frame, tp->seed, 1u, (uint32_t)j, xy);
            float d32[3];
            orc_ao_dir_f32(n32, xy[0], xy[1], d32);
            double d[3] = {d32[0], d32[1], d32[2]};
            cast_result ar = cast_any(s, O, d, tmin, (double)tp->ao_radius, mg);
            if (!ar.hit) ++cnt;
            if (ar.ambiguous) ++amb;
        }
        ao_count[i] = (uint8_t)cnt;
        amb_ao[i] = (uint8_t)amb;
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ======================================================================== */
/* 3. Modified SVGF (Section 3.3), double precision                         */
/* ======================================================================== */
/* Buffers: zn = [H][W][4] binary32 (linear depth, unit normal), mesh =
 * [H][W]; background pixels have depth +inf and mesh id 0xFFFFFFFF.
 * illum = [H][W][4] double (colour AO, colour shadow, variance AO,
 * variance shadow). */

static inline int is_fg(const float* zn, int64_t p) { return isfinite(zn[4 * p]); }

/* Temporal reprojection decision in binary32 (Section 3.3: back-project the
 * pixel's world position into the previous frame; discard history samples
 * inconsistent in projected depth, normal or mesh id).  Depth consistency:
 * |z_prev(q) - z'| <= 0.01 z' + 2 max(|dz/dx|, |dz/dy|), the slope term
 * covering the one-pixel footprint of a bilinear tap on surfaces seen at
 * grazing angles.  The written order of
 * operations is the specification shared with the GPU kernel; each
 * intermediate is rounded to binary32.
 * Returns 1 with the four bilinear taps (valid flags and weights, history
 * length of the valid taps) or 0 when no valid history exists. */
typedef struct {
    int valid;
    int tx[4], ty[4], ok[4];
    float w[4];
    float sumw;
    int histlen_min;
} reproj_t;

/* binary32 depth slope along each axis from the one-sided differences
 * toward the foreground neighbours: with both, the one of smaller magnitude
 * when they have the same sign and 0 when their signs differ or one is 0
 * (minmod, continuous in the depths); with one, its difference; with none,
 * 0.  As used by the history decision; returns max(|gx|, |gy|). */
static float depth_slope_f32(int W, int H, const float* zn, int x, int y)
{
    int64_t p = (int64_t)y * W + x;
    float zp = zn[4 * p];
    float g[2];
    for (int ax = 0; ax < 2; ++ax) {
        int has_p = 0, has_m = 0;
        volatile float dp = 0.0f, dm = 0.0f;
        int xp = x + (ax == 0), yp = y + (ax == 1);
        int xm = x - (ax == 0), ym = y - (ax == 1);
        if (xp < W && yp < H) {
            int64_t q = (int64_t)yp * W + xp;
            if (is_fg(zn, q)) { dp = zn[4 * q] - zp; has_p = 1; }
        }
        if (xm >= 0 && ym >= 0) {
            int64_t q = (int64_t)ym * W + xm;
            if (is_fg(zn, q)) { dm = zp - zn[4 * q]; has_m = 1; }
        }
        if (has_p && has_m)
            g[ax] = ((dp > 0.0f && dm > 0.0f) || (dp < 0.0f && dm < 0.0f)) ? ((fabsf(dm) < fabsf(dp)) ? dm : dp)
                                                                           : 0.0f;
        else if (has_p) g[ax] = dp;
        else if (has_m) g[ax] = dm;
        else g[ax] = 0.0f;
    }
    return fmaxf(fabsf(g[0]), fabsf(g[1]));
}

static reproj_t reproject_f32(int W, int H, int x, int y, const float* znp, uint32_t mp,
                              const orc_camera* cc, const orc_camera* cp,
                              const float* zn_prev, const uint32_t* mesh_prev, const int32_t* hist,
                              float slope)
{
    reproj_t r;
    memset(&r, 0, sizeof(r));
    volatile float Wf = (float)W, Hf = (float)H;
    volatile float aspect = Wf / Hf;
    volatile float fx = (float)x + 0.5f, fy = (float)y + 0.5f;
    volatile float t2x = 2.0f * fx, t2y = 2.0f * fy;
    volatile float qx = t2x / Wf, qy = t2y / Hf;
    volatile float ndx = qx - 1.0f, ndy = 1.0f - qy;
    volatile float sxa = ndx * cc->tan_half_fov_y;
    volatile float sx = sxa * aspect;
    volatile float sy = ndy * cc->tan_half_fov_y;
    float z = znp[0];
    float X[3];
    for (int k = 0; k < 3; ++k) {
        volatile float a = sx * cc->right[k];
        volatile float b = sy * cc->up[k];
        volatile float fa = cc->fwd[k] + a;
        volatile float D = fa + b;
        volatile float zd = z * D;
        X[k] = cc->pos[k] + zd;
    }
    float rr[3];
    for (int k = 0; k < 3; ++k) rr[k] = X[k] - cp->pos[k];
    volatile float f0 = rr[0] * cp->fwd[0], f1 = rr[1] * cp->fwd[1], f2 = rr[2] * cp->fwd[2];
    volatile float f01 = f0 + f1;
    volatile float zp = f01 + f2;
    volatile float r0 = rr[0] * cp->right[0], r1 = rr[1] * cp->right[1], r2 = rr[2] * cp->right[2];
    volatile float r01 = r0 + r1;
    volatile float rx = r01 + r2;
    volatile float u0 = rr[0] * cp->up[0], u1 = rr[1] * cp->up[1], u2 = rr[2] * cp->up[2];
    volatile float u01 = u0 + u1;
    volatile float ry = u01 + u2;
    if (!(zp > 0.0f)) return r;
    volatile float zt = zp * cp->tan_half_fov_y;
    volatile float zta = zt * aspect;
    volatile float su = rx / zta;
    volatile float sv = ry / zt;
    volatile float pu = su + 1.0f, pv = 1.0f - sv;
    volatile float hu = pu * 0.5f, hv = pv * 0.5f;
    volatile float pxc = hu * Wf, pyc = hv * Hf;
    volatile float gx = pxc - 0.5f, gy = pyc - 0.5f;
    if (!(gx > -1.0f && gx < Wf && gy > -1.0f && gy < Hf)) return r;
    float x0f = floorf(gx), y0f = floorf(gy);
    volatile float ax = gx - x0f, ay = gy - y0f;
    volatile float bx = 1.0f - ax, by = 1.0f - ay;
    volatile float w00 = bx * by, w10 = ax * by, w01 = bx * ay, w11 = ax * ay;
    float wt[4] = {w00, w10, w01, w11};
    int x0 = (int)x0f, y0 = (int)y0f;
    int dxs[4] = {0, 1, 0, 1}, dys[4] = {0, 0, 1, 1};
    volatile float sumw = 0.0f;
    int hmin = 1 << 30;
    /* projected depths agree within 1 % plus two pixels of the local depth slope */
    volatile float zrel = 0.01f * zp;
    volatile float zsl = 2.0f * slope;
    volatile float zlim = zrel + zsl;
    for (int k = 0; k < 4; ++k) {
        int qx2 = x0 + dxs[k], qy2 = y0 + dys[k];
        r.tx[k] = qx2; r.ty[k] = qy2; r.w[k] = wt[k]; r.ok[k] = 0;
        if (qx2 < 0 || qy2 < 0 || qx2 >= W || qy2 >= H) continue;
        int64_t q = (int64_t)qy2 * W + qx2;
        if (mesh_prev[q] != mp) continue;
        volatile float dz = zn_prev[4 * q] - zp;
        if (!(fabsf(dz) <= zlim)) continue;
        volatile float n0 = znp[1] * zn_prev[4 * q + 1];
        volatile float n1 = znp[2] * zn_prev[4 * q + 2];
        volatile float n2 = znp[3] * zn_prev[4 * q + 3];
        volatile float n01 = n0 + n1;
        volatile float nd = n01 + n2;
        if (!(nd >= 0.9f)) continue;
        r.ok[k] = 1;
        sumw = sumw + wt[k];
        if (hist[q] < hmin) hmin = hist[q];
    }
    r.sumw = sumw;
    r.valid = (sumw >= 1e-4f);
    r.histlen_min = r.valid ? hmin : 0;
    return r;
}

static void depth_grad(int W, int H, const float* zn, int x, int y, double g[2]);

/*
 * The same back-projection as its plain definition in double (Section 3.3),
 * written independently of the binary32 operation order above: the world
 * position of pixel p is X = eye + z D(p) with D the pixel-centre direction
 * of camera_ray; z' = (X - eye') . f' is its depth in the previous camera
 * and (u', v') its continuous pixel position there; the taps are the 2x2
 * pixels around (u' - 1/2, v' - 1/2) with bilinear weights; a tap is valid
 * when it lies in the image, carries the same mesh id, its depth is within
 * 0.01 z' + 2 max(|dz/dx|, |dz/dy|) of z' (one-sided differences of smaller
 * magnitude) and its normal has cosine >= 0.9 with p's; history exists
 * when the valid weights sum to at least 1e-4.
 *
 * Besides the decision it reports how near each of its comparisons came to
 * flipping: m_px = distance in pixels of (u' - 1/2, v' - 1/2) to the image
 * bounds and to the integer grid (where floor() changes), m_z = smallest
 * | |z_prev(q) - z'| - limit | / z' over in-image taps of p's mesh, m_n =
 * smallest |cos - 0.9| over taps that passed the depth test, m_w =
 * |sum of valid weights - 1e-4|.
 */
typedef struct {
    int valid, x0, y0, ok;   /* ok: bit k = tap k (00, 10, 01, 11) valid */
    double m_px, m_z, m_n, m_w;
} reproj64_t;

static reproj64_t reproject_f64(int W, int H, int x, int y, const float* zn, const uint32_t* mesh,
                                const orc_camera* cc, const orc_camera* cp,
                                const float* zn_prev, const uint32_t* mesh_prev)
{
    reproj64_t r;
    memset(&r, 0, sizeof(r));
    r.m_px = r.m_z = r.m_n = r.m_w = INFINITY;
    int64_t p = (int64_t)y * W + x;
    double o[3], D[3], X[3], rel[3];
    camera_ray(cc, x, y, o, D);
    double z = zn[4 * p];
    for (int k = 0; k < 3; ++k) { X[k] = o[k] + z * D[k]; rel[k] = X[k] - cp->pos[k]; }
    double fp[3] = {cp->fwd[0], cp->fwd[1], cp->fwd[2]};
    double rp[3] = {cp->right[0], cp->right[1], cp->right[2]};
    double up[3] = {cp->up[0], cp->up[1], cp->up[2]};
    double zq = dot3(rel, fp);
    r.m_z = fabs(zq) / fmax(z, 1e-300);
    if (!(zq > 0.0)) return r;
    double t = cp->tan_half_fov_y, aspect = (double)W / (double)H;
    double u = (dot3(rel, rp) / (zq * t * aspect) + 1.0) * 0.5 * W - 0.5;
    double v = (1.0 - dot3(rel, up) / (zq * t)) * 0.5 * H - 0.5;
    r.m_px = fmin(fmin(fabs(u + 1.0), fabs(u - W)), fmin(fabs(v + 1.0), fabs(v - H)));
    if (!(u > -1.0 && u < W && v > -1.0 && v < H)) return r;
    r.m_px = fmin(r.m_px, fmin(fabs(u - nearbyint(u)), fabs(v - nearbyint(v))));
    double fu = floor(u), fv = floor(v);
    r.x0 = (int)fu;
    r.y0 = (int)fv;
    double au = u - fu, av = v - fv;
    double wt[4] = {(1 - au) * (1 - av), au * (1 - av), (1 - au) * av, au * av};
    double g[2];
    depth_grad(W, H, zn, x, y, g);
    double lim = 0.01 * zq + 2.0 * fmax(fabs(g[0]), fabs(g[1]));
    double sumw = 0.0;
    for (int k = 0; k < 4; ++k) {
        int qx = r.x0 + (k & 1), qy = r.y0 + (k >> 1);
        if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
        int64_t q = (int64_t)qy * W + qx;
        if (mesh_prev[q] != mesh[p]) continue;
        double dz = fabs((double)zn_prev[4 * q] - zq);
        r.m_z = fmin(r.m_z, fabs(dz - lim) / zq);
        if (!(dz <= lim)) continue;
        double c = (double)zn[4 * p + 1] * zn_prev[4 * q + 1] + (double)zn[4 * p + 2] * zn_prev[4 * q + 2]
                   + (double)zn[4 * p + 3] * zn_prev[4 * q + 3];
        r.m_n = fmin(r.m_n, fabs(c - 0.9));
        if (!(c >= 0.9)) continue;
        r.ok |= 1 << k;
        sumw += wt[k];
    }
    r.m_w = fabs(sumw - 1e-4);
    r.valid = sumw >= 1e-4;
    return r;
}

/* Both reprojection decisions for every foreground pixel of a frame:
 * dec32, dec64 [H][W][4] = (valid, x0, y0, ok bits), zero on background
 * or without history; margin [H][W][4] = (m_px, m_z, m_n, m_w) of the
 * double decision (+inf where a comparison was not reached). */
void orc_reproject_check(int W, int H, const float* zn, const uint32_t* mesh,
                         const float* zn_prev, const uint32_t* mesh_prev,
                         const orc_camera* cam, const orc_camera* cam_prev,
                         int32_t* dec32, int32_t* dec64, double* margin)
{
    int32_t* hist = (int32_t*)calloc((size_t)W * H, sizeof(int32_t));
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            for (int k = 0; k < 4; ++k) { dec32[4 * p + k] = 0; dec64[4 * p + k] = 0; margin[4 * p + k] = INFINITY; }
            if (!is_fg(zn, p)) continue;
            reproj_t a = reproject_f32(W, H, x, y, zn + 4 * p, mesh[p], cam, cam_prev, zn_prev, mesh_prev,
                                       hist, depth_slope_f32(W, H, zn, x, y));
            if (a.valid) {
                dec32[4 * p] = 1;
                dec32[4 * p + 1] = a.tx[0];
                dec32[4 * p + 2] = a.ty[0];
                for (int k = 0; k < 4; ++k) dec32[4 * p + 3] |= a.ok[k] << k;
            }
            reproj64_t b = reproject_f64(W, H, x, y, zn, mesh, cam, cam_prev, zn_prev, mesh_prev);
            if (b.valid) {
                dec64[4 * p] = 1;
                dec64[4 * p + 1] = b.x0;
                dec64[4 * p + 2] = b.y0;
                dec64[4 * p + 3] = b.ok;
            }
            margin[4 * p] = b.m_px; margin[4 * p + 1] = b.m_z;
            margin[4 * p + 2] = b.m_n; margin[4 * p + 3] = b.m_w;
        }
    }
    free(hist);
}

/* depth gradient at p: per axis the minmod of the one-sided differences
 * toward the foreground neighbours (the smaller magnitude when both share a
 * sign, 0 when the signs differ or one is 0; one neighbour: its difference;
 * none: 0) */
static void depth_grad(int W, int H, const float* zn, int x, int y, double g[2])
{
    int64_t p = (int64_t)y * W + x;
    double zp = zn[4 * p];
    for (int ax = 0; ax < 2; ++ax) {
        int has_p = 0, has_m = 0;
        double dp = 0.0, dm = 0.0;
        int xp = x + (ax == 0), yp = y + (ax == 1);
        int xm = x - (ax == 0), ym = y - (ax == 1);
        if (xp < W && yp < H) {
            int64_t q = (int64_t)yp * W + xp;
            if (is_fg(zn, q)) { dp = (double)zn[4 * q] - zp; has_p = 1; }
        }
        if (xm >= 0 && ym >= 0) {
            int64_t q = (int64_t)ym * W + xm;
            if (is_fg(zn, q)) { dm = zp - (double)zn[4 * q]; has_m = 1; }
        }
        if (has_p && has_m)
            g[ax] = ((dp > 0.0 && dm > 0.0) || (dp < 0.0 && dm < 0.0)) ? ((fabs(dm) < fabs(dp)) ? dm : dp) : 0.0;
        else if (has_p) g[ax] = dp;
        else if (has_m) g[ax] = dm;
        else g[ax] = 0.0;
    }
}

/* depth edge-stopping weight for offset (ox, oy) = p - q in pixels */
static inline double w_depth(double zp, double zq, const double g[2], double ox, double oy,
                             const orc_svgf_params* P)
{
    double den = P->sigma_z * fabs(g[0] * ox + g[1] * oy) + P->eps_z;
    return exp(-fabs(zp - zq) / den);
}

/* normal edge-stopping weight max(0, n_p . n_q)^sigma_n */
static inline double w_normal(const float* a, const float* b, double sigma_n)
{
    double d = (double)a[0] * b[0] + (double)a[1] * b[1] + (double)a[2] * b[2];
    d = fmax(0.0, d);
    return pow(d, sigma_n);
}

/* noisy signals of the current frame: AO = N_unoccluded / N (Eq. 3),
 * shadow = visibility bit of light 0 */
static inline void noisy(const uint8_t* mask, const uint8_t* ao, int64_t p, int spp, double s[2])
{
    s[0] = (double)ao[p] / (double)spp;
    s[1] = (mask[p] & 1u) ? 1.0 : 0.0;
}

/*
 * Temporal accumulation + variance estimation (Section 3.3).
 * In:  current G-buffer, previous G-buffer (NULL: no history), cameras,
 *      noisy inputs, history (col_hist [H][W][2], mom [H][W][4] = mu1 AO,
 *      mu1 shadow, mu2 AO, mu2 shadow, histlen [H][W]).
 * Out: illum [H][W][4]; new moments mom_out and histlen_out.
 * Exponential moving average with alpha_eff = max(alpha, 1/n) (or alpha
 * when fixed_alpha; 1 without history); n = min(histlen + 1, 255).
 * Variance = max(0, mu2 - mu1^2) when n >= 4, else a 7x7 spatial estimate
 * of the current frame's signal weighted by depth and normal only (the
 * paper's modification: no luminance term), whose mean is also the colour.
 */
static void temporal_core(int W, int H, const float* zn, const uint32_t* mesh,
                          const float* zn_prev, const uint32_t* mesh_prev,
                          const orc_camera* cam, const orc_camera* cam_prev,
                          const double* sig, const orc_svgf_params* P,
                          const double* col_hist, const double* mom_in, const int32_t* hist_in,
                          double* mom_out, int32_t* hist_out, double* illum,
                          int32_t* valid_out, orc_trec* rec)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            if (rec) memset(rec + p, 0, sizeof(orc_trec));
            if (!is_fg(zn, p)) {
                illum[4 * p + 0] = 1.0; illum[4 * p + 1] = 1.0;
                illum[4 * p + 2] = 0.0; illum[4 * p + 3] = 0.0;
                for (int k = 0; k < 4; ++k) mom_out[4 * p + k] = 1.0;
                hist_out[p] = 0;
                if (valid_out) valid_out[p] = 0;
                continue;
            }
            double s[2] = {sig[2 * p], sig[2 * p + 1]};
            double ch[2] = {0, 0}, mh[4] = {0, 0, 0, 0};
            int n = 1, valid = 0;
            if (zn_prev) {
                reproj_t r = reproject_f32(W, H, x, y, zn + 4 * p, mesh[p], cam, cam_prev,
                                           zn_prev, mesh_prev, hist_in,
                                           depth_slope_f32(W, H, zn, x, y));
                if (r.valid) {
                    valid = 1;
                    /* weighted mean over the valid taps: (sum w v) / (sum w) */
                    double sw = 0.0;
                    for (int k = 0; k < 4; ++k) {
                        if (!r.ok[k]) continue;
                        int64_t q = (int64_t)r.ty[k] * W + r.tx[k];
                        double w = (double)r.w[k];
                        sw += w;
                        ch[0] += w * col_hist[2 * q]; ch[1] += w * col_hist[2 * q + 1];
                        for (int c = 0; c < 4; ++c) mh[c] += w * mom_in[4 * q + c];
                    }
                    ch[0] /= sw; ch[1] /= sw;
                    for (int c = 0; c < 4; ++c) mh[c] /= sw;
                    if (rec) {
                        rec[p].x0 = r.tx[0]; rec[p].y0 = r.ty[0];
                        for (int k = 0; k < 4; ++k) {
                            rec[p].ok |= r.ok[k] << k;
                            rec[p].beta[k] = r.ok[k] ? (double)r.w[k] / sw : 0.0;
                        }
                    }
                    n = r.histlen_min + 1;
                    if (n > 255) n = 255;
                }
            }
            if (valid_out) valid_out[p] = valid;
            double a = valid ? (P->fixed_alpha ? P->alpha : fmax(P->alpha, 1.0 / n)) : 1.0;
            if (rec) {
                rec[p].fg = 1; rec[p].valid = valid; rec[p].n = n; rec[p].a = a;
                rec[p].spatial = n < 4;
            }
            /* exponential moving average, written h + a (s - h) */
            double c[2], m[4];
            for (int k = 0; k < 2; ++k) {
                c[k] = ch[k] + a * (s[k] - ch[k]);
                m[k] = mh[k] + a * (s[k] - mh[k]);
                m[2 + k] = mh[2 + k] + a * (s[k] * s[k] - mh[2 + k]);
            }
            for (int k = 0; k < 4; ++k) mom_out[4 * p + k] = m[k];
            hist_out[p] = n;
            if (n >= 4) {
                illum[4 * p + 0] = c[0];
                illum[4 * p + 1] = c[1];
                illum[4 * p + 2] = fmax(0.0, m[2] - m[0] * m[0]);
                illum[4 * p + 3] = fmax(0.0, m[3] - m[1] * m[1]);
            } else {
                double g[2];
                depth_grad(W, H, zn, x, y, g);
                double sw = 0.0, s1[2] = {0, 0}, s2[2] = {0, 0};
                for (int dy = -3; dy <= 3; ++dy) {
                    for (int dx = -3; dx <= 3; ++dx) {
                        int qx = x + dx, qy = y + dy;
                        if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                        int64_t q = (int64_t)qy * W + qx;
                        if (!is_fg(zn, q)) continue;
                        double w = 1.0;
                        if (dx || dy)
                            w = w_depth(zn[4 * p], zn[4 * q], g, -dx, -dy, P)
                                * w_normal(zn + 4 * p + 1, zn + 4 * q + 1, P->sigma_n);
                        double sq[2] = {sig[2 * q], sig[2 * q + 1]};
                        sw += w;
                        for (int k = 0; k < 2; ++k) { s1[k] += w * sq[k]; s2[k] += w * sq[k] * sq[k]; }
                    }
                }
                for (int k = 0; k < 2; ++k) {
                    double m1 = s1[k] / sw, m2 = s2[k] / sw;
                    illum[4 * p + k] = m1;
                    illum[4 * p + 2 + k] = fmax(0.0, m2 - m1 * m1);
                }
            }
        }
    }
}

static double* signals_from_counts(int64_t n, const uint8_t* mask, const uint8_t* ao, int spp)
{
    double* sig = (double*)malloc(sizeof(double) * 2 * (size_t)n);
    for (int64_t p = 0; p < n; ++p) noisy(mask, ao, p, spp, sig + 2 * p);
    return sig;
}

void orc_svgf_temporal(int W, int H, const float* zn, const uint32_t* mesh,
                       const float* zn_prev, const uint32_t* mesh_prev,
                       const orc_camera* cam, const orc_camera* cam_prev,
                       const uint8_t* mask, const uint8_t* ao, const orc_svgf_params* P,
                       const double* col_hist, const double* mom_in, const int32_t* hist_in,
                       double* mom_out, int32_t* hist_out, double* illum,
                       int32_t* valid_out /* optional [H][W] */)
{
    double* sig = signals_from_counts((int64_t)W * H, mask, ao, P->ao_spp);
    temporal_core(W, H, zn, mesh, zn_prev, mesh_prev, cam, cam_prev, sig, P, col_hist, mom_in, hist_in,
                  mom_out, hist_out, illum, valid_out, NULL);
    free(sig);
}

/*
 * One edge-stopping a-trous iteration with step h (Section 3.3: the filter
 * is repeated several times, each pass working on the previous pass's
 * output): 5x5 B3-spline taps (1/16, 1/4, 3/8, 1/4, 1/16) at offsets
 * h*{-2..2}, weights k * w_z * w_n * w_l; w_l uses a 3x3 Gaussian of the
 * variance at p.  colour' = sum w c / sum w, variance' = sum w^2 var / (sum w)^2.
 * kernel_width = 3 takes the smaller kernel of the lightweight denoiser
 * Section 3.3 proposes: 3x3 taps (1/4, 1/2, 1/4) at offsets h*{-1..1}.
 */
void orc_svgf_atrous(int W, int H, const float* zn, const double* in, int step,
                     const orc_svgf_params* P, double* out)
{
    static const double b3[5] = {1.0 / 16, 1.0 / 4, 3.0 / 8, 1.0 / 4, 1.0 / 16};
    static const double k3[3] = {1.0 / 4, 1.0 / 2, 1.0 / 4};
    const int R = P->kernel_width == 3 ? 1 : 2;
    const double* k5 = R == 2 ? b3 : k3;     /* taps k5[i + R], i in -R..R */
#pragma omp parallel for schedule(dynamic, 4)
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            if (!is_fg(zn, p)) {
                out[4 * p + 0] = 1.0; out[4 * p + 1] = 1.0;
                out[4 * p + 2] = 0.0; out[4 * p + 3] = 0.0;
                continue;
            }
            /* 3x3 Gaussian of the variance, renormalised over foreground taps */
            double gv[2] = {0, 0}, gw = 0.0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                    int64_t q = (int64_t)qy * W + qx;
                    if (!is_fg(zn, q)) continue;
                    double k = k3[dx + 1] * k3[dy + 1];
                    gw += k;
                    gv[0] += k * in[4 * q + 2];
                    gv[1] += k * in[4 * q + 3];
                }
            gv[0] /= gw; gv[1] /= gw;
            double g[2];
            depth_grad(W, H, zn, x, y, g);
            double sw[2] = {0, 0}, sc[2] = {0, 0}, sv[2] = {0, 0};
            for (int j = -R; j <= R; ++j) {
                for (int i = -R; i <= R; ++i) {
                    int qx = x + i * step, qy = y + j * step;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                    int64_t q = (int64_t)qy * W + qx;
                    if (!is_fg(zn, q)) continue;
                    double k = k5[i + R] * k5[j + R];
                    for (int ch = 0; ch < 2; ++ch) {
                        double w = k;
                        if (i || j) {
                            double wz = w_depth(zn[4 * p], zn[4 * q], g, -(double)i * step,
                                                -(double)j * step, P);
                            double wn = w_normal(zn + 4 * p + 1, zn + 4 * q + 1, P->sigma_n);
                            double wl = 1.0;
                            if (P->wl_in_atrous)
                                wl = exp(-fabs(in[4 * p + ch] - in[4 * q + ch])
                                         / (P->sigma_l * sqrt(fmax(0.0, gv[ch])) + P->eps_l));
                            w = k * wz * wn * wl;
                        }
                        sw[ch] += w;
                        sc[ch] += w * in[4 * q + ch];
                        sv[ch] += w * w * in[4 * q + 2 + ch];
                    }
                }
            }
            for (int ch = 0; ch < 2; ++ch) {
                out[4 * p + ch] = sc[ch] / sw[ch];
                out[4 * p + 2 + ch] = sv[ch] / (sw[ch] * sw[ch]);
            }
        }
    }
}

/*
 * One full frame of the modified SVGF: temporal + variance, then `levels`
 * a-trous iterations with steps 1, 2, 4, ...; the first iteration's colour
 * becomes next frame's colour history (the SVGF design the paper adopts);
 * the last iteration's colour is the output.
 * State (in/out): col_hist [H][W][2], mom [H][W][4], hist [H][W].
 * levels_out (optional): [levels][H][W][4]; illum_out (optional): [H][W][4].
 */
void orc_svgf_frame(int W, int H, const float* zn, const uint32_t* mesh,
                    const float* zn_prev, const uint32_t* mesh_prev,
                    const orc_camera* cam, const orc_camera* cam_prev,
                    const uint8_t* mask, const uint8_t* ao, const orc_svgf_params* P,
                    double* col_hist, double* mom, int32_t* hist,
                    double* illum_out, double* levels_out, double* ao_out, double* sh_out)
{
    int64_t n = (int64_t)W * H;
    double* a = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    double* b = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    double* mom2 = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    int32_t* hist2 = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* sig = signals_from_counts(n, mask, ao, P->ao_spp);
    temporal_core(W, H, zn, mesh, zn_prev, mesh_prev, cam, cam_prev, sig, P,
                  col_hist, mom, hist, mom2, hist2, a, NULL, NULL);
    free(sig);
    memcpy(mom, mom2, sizeof(double) * 4 * (size_t)n);
    memcpy(hist, hist2, sizeof(int32_t) * (size_t)n);
    if (illum_out) memcpy(illum_out, a, sizeof(double) * 4 * (size_t)n);
    if (P->levels == 0)
        for (int64_t p = 0; p < n; ++p) { col_hist[2 * p] = a[4 * p]; col_hist[2 * p + 1] = a[4 * p + 1]; }
    for (int l = 0; l < P->levels; ++l) {
        orc_svgf_atrous(W, H, zn, a, 1 << l, P, b);
        if (l == 0)
            for (int64_t p = 0; p < n; ++p) { col_hist[2 * p] = b[4 * p]; col_hist[2 * p + 1] = b[4 * p + 1]; }
        if (levels_out) memcpy(levels_out + 4 * n * l, b, sizeof(double) * 4 * (size_t)n);
        double* t = a; a = b; b = t;
    }
    for (int64_t p = 0; p < n; ++p) { ao_out[p] = a[4 * p]; sh_out[p] = a[4 * p + 1]; }
    free(a); free(b); free(mom2); free(hist2);
}

/* ======================================================================== */
/* 4. Adjoint of the modified SVGF over a sequence of frames (double)       */
/*                                                                          */
/* Loss gradient g_out = dL/d(filtered colour) per frame.  Returned: dL/ds  */
/* for the per-pixel noisy signals s (AO and shadow) of every frame and     */
/* dL/d(sigma_z, sigma_n, sigma_l).  The temporal recursion is not cut:     */
/* frame f's level-0 colour and moments feed frame f+1.  The reprojection   */
/* taps, validity and history lengths depend only on G-buffers and cameras  */
/* and are constants.  Conventions: d|x|/dx = sign(x) with sign(0) = 0;     */
/* d max(0, x)/dx = [x > 0]; d sqrt(g)/dg = 0 at g = 0; d w_n/d sigma_n =   */
/* w_n ln(n.n') where n.n' > 0, else 0.  Written in scatter form: every     */
/* output pixel pushes its contributions to the inputs it read.             */
/* ======================================================================== */
static inline double sgn(double x) { return x > 0.0 ? 1.0 : (x < 0.0 ? -1.0 : 0.0); }

/* backward of one a-trous iteration.  in: the iteration's input (colour x2,
 * variance x2); gc_out, gv_out: dL/d its output colour and variance
 * ([N][2] each).  Adds dL/d input into gc_in, gv_in ([N][2]) and the sigma
 * gradients into gsig[3]. */
static void atrous_backward(int W, int H, const float* zn, const double* in, int step,
                            const orc_svgf_params* P, const double* gc_out, const double* gv_out,
                            double* gc_in, double* gv_in, double* gsig)
{
    static const double k5[5] = {1.0 / 16, 1.0 / 4, 3.0 / 8, 1.0 / 4, 1.0 / 16};
    static const double k3[3] = {1.0 / 4, 1.0 / 2, 1.0 / 4};
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            if (!is_fg(zn, p)) continue;
            /* forward quantities at p */
            double gv[2] = {0, 0}, gw = 0.0;
            for (int dy = -1; dy <= 1; ++dy)
                for (int dx = -1; dx <= 1; ++dx) {
                    int qx = x + dx, qy = y + dy;
                    if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                    int64_t q = (int64_t)qy * W + qx;
                    if (!is_fg(zn, q)) continue;
                    double k = k3[dx + 1] * k3[dy + 1];
                    gw += k;
                    gv[0] += k * in[4 * q + 2];
                    gv[1] += k * in[4 * q + 3];
                }
            gv[0] /= gw; gv[1] /= gw;
            double gz[2];
            depth_grad(W, H, zn, x, y, gz);
            for (int ch = 0; ch < 2; ++ch) {
                double root = sqrt(fmax(0.0, gv[ch]));
                double il = 1.0 / (P->sigma_l * root + P->eps_l);
                /* pass 1: W, A, B */
                double Wsum = 0.0, A = 0.0, B = 0.0;
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        int qx = x + i * step, qy = y + j * step;
                        if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                        int64_t q = (int64_t)qy * W + qx;
                        if (!is_fg(zn, q)) continue;
                        double k = k5[i + 2] * k5[j + 2], w = k;
                        if (i || j) {
                            double wz = w_depth(zn[4 * p], zn[4 * q], gz, -(double)i * step,
                                                -(double)j * step, P);
                            double wn = w_normal(zn + 4 * p + 1, zn + 4 * q + 1, P->sigma_n);
                            double wl = P->wl_in_atrous
                                ? exp(-fabs(in[4 * p + ch] - in[4 * q + ch]) * il) : 1.0;
                            w = k * wz * wn * wl;
                        }
                        Wsum += w;
                        A += w * in[4 * q + ch];
                        B += w * w * in[4 * q + 2 + ch];
                    }
                double cp_out = A / Wsum, vp_out = B / (Wsum * Wsum);
                double Gc = gc_out[2 * p + ch], Gv = gv_out[2 * p + ch];
                double Gil = 0.0;
                /* pass 2: push gradients to the taps */
                for (int j = -2; j <= 2; ++j)
                    for (int i = -2; i <= 2; ++i) {
                        int qx = x + i * step, qy = y + j * step;
                        if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                        int64_t q = (int64_t)qy * W + qx;
                        if (!is_fg(zn, q)) continue;
                        double k = k5[i + 2] * k5[j + 2], w = k;
                        double wz = 1.0, wn = 1.0, wl = 1.0, a_off = 0.0, D = 1.0, dlt = 0.0;
                        double nd = 1.0;
                        if (i || j) {
                            a_off = fabs(gz[0] * (-(double)i * step) + gz[1] * (-(double)j * step));
                            D = P->sigma_z * a_off + P->eps_z;
                            wz = exp(-fabs((double)zn[4 * p] - (double)zn[4 * q]) / D);
                            const float* np_ = zn + 4 * p + 1;
                            const float* nq_ = zn + 4 * q + 1;
                            nd = (double)np_[0] * nq_[0] + (double)np_[1] * nq_[1] + (double)np_[2] * nq_[2];
                            wn = w_normal(np_, nq_, P->sigma_n);
                            dlt = in[4 * p + ch] - in[4 * q + ch];
                            if (P->wl_in_atrous) wl = exp(-fabs(dlt) * il);
                            w = k * wz * wn * wl;
                        }
                        double cq = in[4 * q + ch], vq = in[4 * q + 2 + ch];
                        /* direct dependence of the output on the tap values */
                        gc_in[2 * q + ch] += Gc * w / Wsum;
                        gv_in[2 * q + ch] += Gv * w * w / (Wsum * Wsum);
                        if (!(i || j)) continue;          /* centre weight is a constant */
                        /* dependence through the weight */
                        double Gw = Gc * (cq - cp_out) / Wsum
                                    + Gv * (2.0 * w * vq / (Wsum * Wsum) - 2.0 * vp_out / Wsum);
                        if (P->wl_in_atrous) {
                            double dwdc = w * il * sgn(dlt);            /* dw/dc_q; dw/dc_p = -dwdc */
                            gc_in[2 * q + ch] += Gw * dwdc;
                            gc_in[2 * p + ch] -= Gw * dwdc;
                            Gil += Gw * (-w * fabs(dlt));
                        }
                        double dz = fabs((double)zn[4 * p] - (double)zn[4 * q]);
                        gsig[0] += Gw * w * dz * a_off / (D * D);
                        if (nd > 0.0) gsig[1] += Gw * w * log(nd);
                    }
                /* il = 1 / (sigma_l sqrt(g) + eps_l) */
                if (P->wl_in_atrous) {
                    gsig[2] += Gil * (-il * il * root);
                    if (gv[ch] > 1e-12) {       /* d sqrt(g)/dg taken as 0 below g = 1e-12 */
                        double Gg = Gil * (-il * il * P->sigma_l * 0.5 / root);
                        for (int dy = -1; dy <= 1; ++dy)
                            for (int dx = -1; dx <= 1; ++dx) {
                                int qx = x + dx, qy = y + dy;
                                if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                                int64_t q = (int64_t)qy * W + qx;
                                if (!is_fg(zn, q)) continue;
                                gv_in[2 * q + ch] += Gg * k3[dx + 1] * k3[dy + 1] / gw;
                            }
                    }
                }
            }
        }
    }
}

/* backward of the temporal step of one frame.  gc, gv: dL/d illum colour
 * and variance ([N][2]); gmom: dL/d this frame's moments output ([N][4]).
 * Adds dL/ds into gsig_s ([N][2]), dL/d the previous frame's colour history
 * and moments into gcol_prev ([N][2]), gmom_prev ([N][4]), sigma gradients
 * of the spatial estimate into gsig[0..1]. */
static void temporal_backward(int W, int H, const float* zn, const double* sig, const double* mom,
                              const orc_trec* rec, const orc_svgf_params* P, const double* gc,
                              const double* gv, const double* gmom, double* gsig_s,
                              double* gcol_prev, double* gmom_prev, double* gsig)
{
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            const orc_trec* r = rec + p;
            if (!r->fg) continue;
            double a = r->a;
            double Gc_ema[2] = {0, 0}, Gm[4];
            for (int k = 0; k < 4; ++k) Gm[k] = gmom[4 * p + k];
            if (!r->spatial) {
                for (int ch = 0; ch < 2; ++ch) {
                    Gc_ema[ch] = gc[2 * p + ch];
                    double mu1 = mom[4 * p + ch], mu2 = mom[4 * p + 2 + ch];
                    if (mu2 - mu1 * mu1 > 0.0) {            /* var = max(0, mu2 - mu1^2) */
                        Gm[2 + ch] += gv[2 * p + ch];
                        Gm[ch] += -2.0 * mu1 * gv[2 * p + ch];
                    }
                }
            } else {
                /* colour = m1, var = max(0, m2 - m1^2), m_k = sum w s^k / sum w
                 * over the 7x7 window with w = w_z w_n (centre 1) */
                double gz[2];
                depth_grad(W, H, zn, x, y, gz);
                double sw = 0.0, s1[2] = {0, 0}, s2[2] = {0, 0};
                for (int pass = 0; pass < 2; ++pass) {
                    double m1[2], m2[2], Gm1[2], Gm2[2];
                    if (pass == 1) {
                        for (int ch = 0; ch < 2; ++ch) {
                            m1[ch] = s1[ch] / sw;
                            m2[ch] = s2[ch] / sw;
                            double var = m2[ch] - m1[ch] * m1[ch];
                            Gm1[ch] = gc[2 * p + ch] - (var > 0.0 ? 2.0 * m1[ch] * gv[2 * p + ch] : 0.0);
                            Gm2[ch] = var > 0.0 ? gv[2 * p + ch] : 0.0;
                        }
                    }
                    for (int dy = -3; dy <= 3; ++dy)
                        for (int dx = -3; dx <= 3; ++dx) {
                            int qx = x + dx, qy = y + dy;
                            if (qx < 0 || qy < 0 || qx >= W || qy >= H) continue;
                            int64_t q = (int64_t)qy * W + qx;
                            if (!is_fg(zn, q)) continue;
                            double w = 1.0, a_off = 0.0, D = 1.0, nd = 1.0;
                            if (dx || dy) {
                                a_off = fabs(gz[0] * (double)(-dx) + gz[1] * (double)(-dy));
                                D = P->sigma_z * a_off + P->eps_z;
                                nd = (double)zn[4 * p + 1] * zn[4 * q + 1] + (double)zn[4 * p + 2] * zn[4 * q + 2]
                                     + (double)zn[4 * p + 3] * zn[4 * q + 3];
                                w = w_depth(zn[4 * p], zn[4 * q], gz, -dx, -dy, P)
                                    * w_normal(zn + 4 * p + 1, zn + 4 * q + 1, P->sigma_n);
                            }
                            if (pass == 0) {
                                sw += w;
                                for (int ch = 0; ch < 2; ++ch) {
                                    s1[ch] += w * sig[2 * q + ch];
                                    s2[ch] += w * sig[2 * q + ch] * sig[2 * q + ch];
                                }
                                continue;
                            }
                            double Gw = 0.0;
                            for (int ch = 0; ch < 2; ++ch) {
                                double sq = sig[2 * q + ch];
                                gsig_s[2 * q + ch] += Gm1[ch] * w / sw + Gm2[ch] * 2.0 * sq * w / sw;
                                Gw += Gm1[ch] * (sq - m1[ch]) / sw + Gm2[ch] * (sq * sq - m2[ch]) / sw;
                            }
                            if (dx || dy) {
                                double dz = fabs((double)zn[4 * p] - (double)zn[4 * q]);
                                gsig[0] += Gw * w * dz * a_off / (D * D);
                                if (nd > 0.0) gsig[1] += Gw * w * log(nd);
                            }
                        }
                }
            }
            /* moving averages c = c_h + a (s - c_h), mu1 likewise, mu2 with s^2 */
            for (int ch = 0; ch < 2; ++ch) {
                double sv = sig[2 * p + ch];
                gsig_s[2 * p + ch] += a * Gc_ema[ch] + a * Gm[ch] + 2.0 * a * sv * Gm[2 + ch];
            }
            if (!r->valid) continue;
            double Gch[2] = {(1.0 - a) * Gc_ema[0], (1.0 - a) * Gc_ema[1]};
            double Gmh[4];
            for (int k = 0; k < 4; ++k) Gmh[k] = (1.0 - a) * Gm[k];
            for (int t = 0; t < 4; ++t) {
                if (!(r->ok & (1 << t))) continue;
                int64_t q = (int64_t)(r->y0 + (t >> 1)) * W + (r->x0 + (t & 1));
                double b = r->beta[t];
                gcol_prev[2 * q] += b * Gch[0];
                gcol_prev[2 * q + 1] += b * Gch[1];
                for (int k = 0; k < 4; ++k) gmom_prev[4 * q + k] += b * Gmh[k];
            }
        }
    }
}

/*
 * Forward and adjoint of the modified SVGF over F consecutive frames that
 * start without history.  zn [F][H][W][4], mesh [F][H][W], cams [F],
 * sig [F][H][W][2] (noisy AO and shadow in [0, 1]), g_out [F][H][W][2]
 * (dL/d filtered colour).  Outputs out [F][H][W][2], g_sig [F][H][W][2],
 * g_sigma[3] = dL/d(sigma_z, sigma_n, sigma_l).
 */
void orc_svgf_seq_grad(int F, int W, int H, const float* zn, const uint32_t* mesh,
                       const orc_camera* cams, const double* sig, const orc_svgf_params* P,
                       const double* g_out, double* out, double* g_sig, double* g_sigma)
{
    int64_t N = (int64_t)W * H;
    int L = P->levels;
    /* recordings */
    double* lev = (double*)calloc((size_t)F * (L + 1) * N * 4, sizeof(double));
    double* mom = (double*)calloc((size_t)F * N * 4, sizeof(double));
    orc_trec* rec = (orc_trec*)calloc((size_t)F * N, sizeof(orc_trec));
    double* col = (double*)calloc((size_t)N * 2, sizeof(double));
    double* mom_prev = (double*)calloc((size_t)N * 4, sizeof(double));
    int32_t* hist = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    int32_t* hist2 = (int32_t*)calloc((size_t)N, sizeof(int32_t));
    for (int f = 0; f < F; ++f) {
        const float* znf = zn + (size_t)f * N * 4;
        const float* znp = f ? zn + (size_t)(f - 1) * N * 4 : NULL;
        const uint32_t* mp = f ? mesh + (size_t)(f - 1) * N : NULL;
        double* illum = lev + ((size_t)f * (L + 1)) * N * 4;
        double* momf = mom + (size_t)f * N * 4;
        temporal_core(W, H, znf, mesh + (size_t)f * N, znp, mp, cams + f, f ? cams + f - 1 : cams + f,
                      sig + (size_t)f * N * 2, P, col, mom_prev, hist, momf, hist2, illum, NULL,
                      rec + (size_t)f * N);
        memcpy(mom_prev, momf, sizeof(double) * 4 * (size_t)N);
        memcpy(hist, hist2, sizeof(int32_t) * (size_t)N);
        for (int l = 0; l < L; ++l)
            orc_svgf_atrous(W, H, znf, illum + (size_t)l * N * 4, 1 << l, P, illum + (size_t)(l + 1) * N * 4);
        const double* first = illum + (size_t)(L ? 1 : 0) * N * 4;
        const double* last = illum + (size_t)L * N * 4;
        for (int64_t p = 0; p < N; ++p) {
            col[2 * p] = first[4 * p];
            col[2 * p + 1] = first[4 * p + 1];
            out[(size_t)f * N * 2 + 2 * p] = last[4 * p];
            out[(size_t)f * N * 2 + 2 * p + 1] = last[4 * p + 1];
        }
    }
    /* backward */
    double* gc = (double*)calloc((size_t)N * 2, sizeof(double));
    double* gv = (double*)calloc((size_t)N * 2, sizeof(double));
    double* gc2 = (double*)calloc((size_t)N * 2, sizeof(double));
    double* gv2 = (double*)calloc((size_t)N * 2, sizeof(double));
    double* gcol_next = (double*)calloc((size_t)N * 2, sizeof(double));
    double* gmom_next = (double*)calloc((size_t)N * 4, sizeof(double));
    double* gcol_prev = (double*)calloc((size_t)N * 2, sizeof(double));
    double* gmom_prev = (double*)calloc((size_t)N * 4, sizeof(double));
    memset(g_sig, 0, sizeof(double) * (size_t)F * N * 2);
    g_sigma[0] = g_sigma[1] = g_sigma[2] = 0.0;
    for (int f = F - 1; f >= 0; --f) {
        const float* znf = zn + (size_t)f * N * 4;
        double* illum = lev + ((size_t)f * (L + 1)) * N * 4;
        memcpy(gc, g_out + (size_t)f * N * 2, sizeof(double) * 2 * (size_t)N);
        memset(gv, 0, sizeof(double) * 2 * (size_t)N);
        for (int l = L - 1; l >= 0; --l) {
            if (l == 0)   /* level-0 colour is also next frame's colour history */
                for (int64_t i = 0; i < 2 * N; ++i) gc[i] += gcol_next[i];
            memset(gc2, 0, sizeof(double) * 2 * (size_t)N);
            memset(gv2, 0, sizeof(double) * 2 * (size_t)N);
            atrous_backward(W, H, znf, illum + (size_t)l * N * 4, 1 << l, P, gc, gv, gc2, gv2, g_sigma);
            memcpy(gc, gc2, sizeof(double) * 2 * (size_t)N);
            memcpy(gv, gv2, sizeof(double) * 2 * (size_t)N);
        }
        if (L == 0)
            for (int64_t i = 0; i < 2 * N; ++i) gc[i] += gcol_next[i];
        memset(gcol_prev, 0, sizeof(double) * 2 * (size_t)N);
        memset(gmom_prev, 0, sizeof(double) * 4 * (size_t)N);
        temporal_backward(W, H, znf, sig + (size_t)f * N * 2, mom + (size_t)f * N * 4, rec + (size_t)f * N, P,
                          gc, gv, gmom_next, g_sig + (size_t)f * N * 2, gcol_prev, gmom_prev, g_sigma);
        memcpy(gcol_next, gcol_prev, sizeof(double) * 2 * (size_t)N);
        memcpy(gmom_next, gmom_prev, sizeof(double) * 4 * (size_t)N);
    }
    free(lev); free(mom); free(rec); free(col); free(mom_prev); free(hist); free(hist2);
    free(gc); free(gv); free(gc2); free(gv2); free(gcol_next); free(gmom_next); free(gcol_prev);
    free(gmom_prev);
}

/* ======================================================================== */
/* 5. Delay reprojection (Section 4.1, Fig. 5: camera data reaches the       */
/*    server late; the result is shown at a newer pose)                     */
/* ======================================================================== */
/* Each pixel of the target pose (G-buffer zn_t, mesh_t, camera cam_t) takes
 * the value of the nearest valid pixel of the source pose: the history-tap
 * rule of the temporal step (binary32 decision, reproject_f32), nearest =
 * largest bilinear weight among the valid taps (ties: first tap).  Without
 * a valid tap, or on background, the value is 1 and valid = 0. */
void orc_delay_warp(int W, int H, const float* zn_t, const uint32_t* mesh_t, const orc_camera* cam_t,
                    const float* zn_s, const uint32_t* mesh_s, const orc_camera* cam_s,
                    const double* src_ao, const double* src_sh, double* out_ao, double* out_sh,
                    int32_t* valid)
{
    int32_t* zero_hist = (int32_t*)calloc((size_t)W * H, sizeof(int32_t));
    for (int y = 0; y < H; ++y) {
        for (int x = 0; x < W; ++x) {
            int64_t p = (int64_t)y * W + x;
            out_ao[p] = 1.0;
            out_sh[p] = 1.0;
            valid[p] = 0;
            if (!is_fg(zn_t, p)) continue;
            reproj_t r = reproject_f32(W, H, x, y, zn_t + 4 * p, mesh_t[p], cam_t, cam_s, zn_s, mesh_s,
                                       zero_hist, depth_slope_f32(W, H, zn_t, x, y));
            if (!r.valid) continue;
            int best = -1;
            float bw = -1.0f;
            for (int k = 0; k < 4; ++k)
                if (r.ok[k] && r.w[k] > bw) { bw = r.w[k]; best = k; }
            int64_t q = (int64_t)r.ty[best] * W + r.tx[best];
            out_ao[p] = src_ao[q];
            out_sh[p] = src_sh[q];
            valid[p] = 1;
        }
    }
    free(zero_hist);
}

/* ======================================================================== */
/* 8. Selective shadow rays (Section 5: the shadow-map ray mask of          */
/*    Lauterbach and Manocha that the paper plans to adopt)                 */
/* ======================================================================== */
/*
 * The method: a shadow map from the light marks the pixels whose shadow
 * verdict it cannot give reliably; those pixels, widened by a radius set by
 * the light's angular size and the distance to the occluder, form a ray
 * mask.  Masked pixels are ray traced; the others take the shadow map's
 * verdict (lit, or umbra).  The reading written out here (gather form):
 *
 * Map frame, in double, from the unit light direction L (toward the light)
 * and the bounds [bmin, bmax] of the triangles' vertices:
 *   helper a = (0, 1, 0) if |L.y| < 0.9 else (1, 0, 0);
 *   eu = (a x L) / |a x L|, ev = L x eu;
 *   u, v, t = eu.c, ev.c, L.c over the 8 bound corners c -> [umin, umax],
 *   [vmin, vmax], tmax; E = max(umax - umin, vmax - vmin) (1 if not > 0);
 *   texel size w = E (1 + 2^-10) / R; the R x R map is centred on the
 *   projected bounds: u0 = (umin + umax) / 2 - w R / 2 (v0 alike);
 *   light plane h = tmax + E / 64; depth of a point x is h - L.x.
 * Map S[j][i] (texel i along eu, j along ev): depth of the closest surface
 *   met by the ray from h L + (u0 + (i + 1/2) w) eu + (v0 + (j + 1/2) w) ev
 *   along -L, +inf when it meets none.
 * Classification of a pixel (hit point X, unit normal n) for a light whose
 *   cone has half angle theta (tau = tan theta):
 *   1. g = sin theta + 0.05.  n.L < -g: the whole cone is below the
 *      surface -> UMBRA; n.L <= g: the cone grazes the surface -> TRACE.
 *   2. a = (eu.X - u0) / w - 1/2, b = (ev.X - v0) / w - 1/2 (texel
 *      coordinates, centres at integers), z = h - L.X.
 *   3. Occluder bound: a cone ray that has moved r texels sideways is at
 *      least r w / tau closer to the light, so no occluder above
 *      zmin = min S can be met beyond r0 = max(0, (z - zmin) tau / w)
 *      texels.  The texel range [floor(a - r0), ceil(a + r0)] (and b
 *      alike), clamped to the map, spans s texels; at the smallest level
 *      l with 2^l >= s the range meets at most 2 x 2 cells of 2^l x 2^l
 *      texels, and zocc = min S over those cells.
 *   4. Penumbra radius r = max(0, (z - zocc) tau / w) texels (the light's
 *      angular size times the distance to the nearest possible occluder).
 *      r + 1 > 4 -> TRACE (footprint wider than the 9 x 9 window).
 *   5. Window: texels i in [ceil(a - r - 1), floor(a + r + 1)] (and j
 *      alike), clamped to the map.  Texel (i, j) is occluded when
 *      S[j][i] < z + ((i - a) n.eu + (j - b) n.ev) w / n.L - w, i.e. a
 *      surface lies more than one texel size above the receiver's tangent
 *      plane there.  All free -> LIT; all occluded -> UMBRA; else TRACE.
 * The ray mask is the set of TRACE pixels; they take the ray-traced bit of
 * the full method, LIT pixels bit 1, UMBRA pixels bit 0.
 */
#define ORC_SMAP_WINDOW 4           /* largest window radius r + 1, texels */
#define ORC_SMAP_GRAZE 0.05         /* margin of n.L over sin theta */
#define ORC_CLS_TRACE 0
#define ORC_CLS_LIT 1
#define ORC_CLS_UMBRA 2

typedef struct {
    int32_t res;               /* R, a power of two */
    double L[3], eu[3], ev[3];
    double u0, v0, w, h;
} orc_smap_frame;

void orc_smap_frame_make(const orc_scene* s, const float light[3], int32_t res, orc_smap_frame* f)
{
    double l[3] = {light[0], light[1], light[2]};
    double ln = norm3(l);
    for (int k = 0; k < 3; ++k) f->L[k] = l[k] / ln;
    double a[3] = {0.0, 0.0, 0.0};
    if (fabs(f->L[1]) < 0.9) a[1] = 1.0; else a[0] = 1.0;
    double c[3];
    cross3(a, f->L, c);
    double cn = norm3(c);
    for (int k = 0; k < 3; ++k) f->eu[k] = c[k] / cn;
    cross3(f->L, f->eu, f->ev);
    double umin = INFINITY, umax = -INFINITY, vmin = INFINITY, vmax = -INFINITY, tmax = -INFINITY;
    for (int k = 0; k < 8; ++k) {
        double p[3] = {(k & 1) ? s->bmax[0] : s->bmin[0], (k & 2) ? s->bmax[1] : s->bmin[1],
                       (k & 4) ? s->bmax[2] : s->bmin[2]};
        double u = dot3(f->eu, p), v = dot3(f->ev, p), t = dot3(f->L, p);
        umin = fmin(umin, u); umax = fmax(umax, u);
        vmin = fmin(vmin, v); vmax = fmax(vmax, v);
        tmax = fmax(tmax, t);
    }
    double E = fmax(umax - umin, vmax - vmin);
    if (!(E > 0.0)) E = 1.0;
    f->res = res;
    f->w = E * (1.0 + 1.0 / 1024.0) / res;
    f->u0 = 0.5 * (umin + umax) - 0.5 * f->w * res;
    f->v0 = 0.5 * (vmin + vmax) - 0.5 * f->w * res;
    f->h = tmax + E / 64.0;
}

/* Depth of texels (i, j) = texels[2k], texels[2k + 1] (all R x R texels in
 * row-major order when texels is NULL), with the closest-hit ambiguity flag. */
void orc_smap_render(const orc_scene* s, const orc_smap_frame* f, const orc_margin* mg,
                     const int32_t* texels, int64_t n, double* depth, uint8_t* amb)
{
    int64_t R = f->res;
    if (!texels) n = R * R;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = texels ? texels[2 * k] : k % R, j = texels ? texels[2 * k + 1] : k / R;
        double u = f->u0 + ((double)i + 0.5) * f->w, v = f->v0 + ((double)j + 0.5) * f->w;
        double o[3], d[3];
        for (int c = 0; c < 3; ++c) {
            o[c] = f->h * f->L[c] + u * f->eu[c] + v * f->ev[c];
            d[c] = -f->L[c];
        }
        cast_result r = cast_closest(s, o, d, 0.0, INFINITY, mg);
        depth[k] = r.hit ? r.t : INFINITY;
        amb[k] = (uint8_t)r.ambiguous;
    }
}

static int near_integer(double x, double tol) { return fabs(x - nearbyint(x)) < tol; }

static int64_t clampi(int64_t x, int64_t lo, int64_t hi) { return x < lo ? lo : (x > hi ? hi : x); }

/* Classify np pixels (pos, nrm: [np][3]; fg[i] = 0 skips background) for a
 * light of cone half angle theta against a full map S ([R][R], S_amb its
 * ambiguity flags).  cls: ORC_CLS_*; amb = 1 where a decision of the
 * classification lies within tol_t texels (integer bounds, the window cap)
 * or tol_z world units (texel tests, grazing test in units of n.L) of
 * flipping, or reads an ambiguous texel. */
void orc_smap_classify(const orc_smap_frame* f, const double* S, const uint8_t* S_amb, double theta,
                       int64_t np, const double* pos, const double* nrm, const uint8_t* fg,
                       double tol_t, double tol_z, uint8_t* cls, uint8_t* amb)
{
    const int64_t R = f->res;
    const double tau = tan(theta), g = sin(theta) + ORC_SMAP_GRAZE;
    double zmin = INFINITY, zmin_sure = INFINITY;
    for (int64_t k = 0; k < R * R; ++k) {
        zmin = fmin(zmin, S[k]);
        if (!S_amb[k]) zmin_sure = fmin(zmin_sure, S[k]);
    }
    const int zmin_amb = zmin != zmin_sure;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t p = 0; p < np; ++p) {
        cls[p] = ORC_CLS_LIT;
        amb[p] = 0;
        if (fg && !fg[p]) continue;
        const double* X = pos + 3 * p;
        const double* n = nrm + 3 * p;
        int am = zmin_amb;
        double nL = dot3(n, f->L);
        if (fabs(nL - g) < 1e-5 || fabs(nL + g) < 1e-5) am = 1;
        if (nL < -g) { cls[p] = ORC_CLS_UMBRA; amb[p] = (uint8_t)am; continue; }
        if (nL <= g) { cls[p] = ORC_CLS_TRACE; amb[p] = (uint8_t)am; continue; }
        double a = (dot3(f->eu, X) - f->u0) / f->w - 0.5;
        double b = (dot3(f->ev, X) - f->v0) / f->w - 0.5;
        double z = f->h - dot3(f->L, X);
        /* 3. occluder bound over the pyramid cells */
        double r0 = fmax(0.0, (z - zmin) * tau / f->w);
        if (near_integer(a - r0, tol_t) || near_integer(a + r0, tol_t) || near_integer(b - r0, tol_t) ||
            near_integer(b + r0, tol_t))
            am = 1;
        int64_t ilo = clampi((int64_t)floor(a - r0), 0, R - 1), ihi = clampi((int64_t)ceil(a + r0), 0, R - 1);
        int64_t jlo = clampi((int64_t)floor(b - r0), 0, R - 1), jhi = clampi((int64_t)ceil(b + r0), 0, R - 1);
        int64_t span = (ihi - ilo > jhi - jlo ? ihi - ilo : jhi - jlo) + 1;
        int lv = 0;
        while (((int64_t)1 << lv) < span) ++lv;
        int64_t ci0 = (ilo >> lv) << lv, ci1 = ((ihi >> lv) + 1) << lv;
        int64_t cj0 = (jlo >> lv) << lv, cj1 = ((jhi >> lv) + 1) << lv;
        double zocc = INFINITY;
        for (int64_t j = cj0; j < cj1; ++j)
            for (int64_t i = ci0; i < ci1; ++i) {
                zocc = fmin(zocc, S[j * R + i]);
                if (S_amb[j * R + i]) am = 1;
            }
        /* 4. penumbra radius */
        double r = fmax(0.0, (z - zocc) * tau / f->w);
        if (fabs(r + 1.0 - ORC_SMAP_WINDOW) < tol_t) am = 1;
        if (r + 1.0 > ORC_SMAP_WINDOW) { cls[p] = ORC_CLS_TRACE; amb[p] = (uint8_t)am; continue; }
        /* 5. window of tangent-plane shadow tests */
        if (near_integer(a - r - 1.0, tol_t) || near_integer(a + r + 1.0, tol_t) ||
            near_integer(b - r - 1.0, tol_t) || near_integer(b + r + 1.0, tol_t))
            am = 1;
        int64_t wi0 = clampi((int64_t)ceil(a - r - 1.0), 0, R - 1), wi1 = clampi((int64_t)floor(a + r + 1.0), 0, R - 1);
        int64_t wj0 = clampi((int64_t)ceil(b - r - 1.0), 0, R - 1), wj1 = clampi((int64_t)floor(b + r + 1.0), 0, R - 1);
        double gu = dot3(n, f->eu) / nL * f->w, gv = dot3(n, f->ev) / nL * f->w;
        double tz = tol_z + tol_t * (fabs(gu) + fabs(gv));
        int occ = 0, fre = 0;
        for (int64_t j = wj0; j <= wj1; ++j)
            for (int64_t i = wi0; i <= wi1; ++i) {
                double plane = z + ((double)i - a) * gu + ((double)j - b) * gv - f->w;
                double sv = S[j * R + i];
                if (S_amb[j * R + i] || fabs(sv - plane) < tz) am = 1;
                if (sv < plane) occ = 1; else fre = 1;
            }
        cls[p] = (uint8_t)(occ && fre ? ORC_CLS_TRACE : (occ ? ORC_CLS_UMBRA : ORC_CLS_LIT));
        amb[p] = (uint8_t)am;
    }
}
