/*
 * FP64 CPU oracle for voxel-grid NeRF rendering and sparse radiance warping (SpaRW).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or call this file:
 * it is used by tests/, by __graft_entry__.smoke() and by the CPU-baseline leg of bench.py.
 * It shares no code, header, table or constant generator with the CUDA library.
 *
 * Everything here is the plain definition, one ray (or one pixel) at a time, in the order the
 * paper states it:
 *   - Indexing, Feature Gathering, Feature Computation and accumulation       Sec. II-B
 *   - SpaRW target rendering: point cloud (Eq. 1), transform (Eq. 2),
 *     re-projection (Eq. 3), sparse rendering of the holes (Eq. 4),
 *     the void depth test and the warp-angle heuristic phi                    Sec. III-B, III-C
 * Values are computed in FP64.  Integer decisions that the GPU takes in FP32 (which voxel a
 * sample falls in, whether it is inside the box or an occupied cell, which target pixel a
 * warped point lands on, which point wins the depth test) are taken here in FP32 with the
 * same operation order and no contraction (the file is built with -ffp-contract=off), so they
 * agree bit for bit given identical float inputs.  The early-stop decision depends on
 * transcendental functions and is taken in FP64; rays whose transmittance lies within a
 * relative 1e-4 of the threshold are flagged and their other outcome is returned as well.
 *
 * Readings where the paper is silent (camera axes, sample placement, activation, positional
 * encoding, background, depth definition, void rule, splat footprint, tie-break) are stated at
 * each function below.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_AMBIG_REL 1e-4
#define OR_MAX_HIDDEN 256
#define OR_MAX_IN 96

/* Multiresolution hash encoding (the hash-grid workload, Instant-NGP-like): `levels` levels of
 * `feat` features.  Level l divides the grid box into res[l] cells per axis; its (res+1)^3
 * vertices are stored densely, at x + (res+1) (y + (res+1) z), when they fit the level's table of
 * T = 2^log2_size entries, otherwise at the spatial hash (x * 1) xor (y * 2654435761) xor
 * (z * 805459861) mod T of 32-bit unsigned integers.  A level's features are the trilinear
 * interpolation of its 8 corner entries; the levels are concatenated (feature l * feat + c). */
typedef struct {
    int levels, feat, log2_size;
    int res[16];
    int dtype;             /* storage of the table: 1 f32, 2 f16 bits */
    const void *table;     /* [levels][T][feat] */
} or_hash;

typedef struct {
    int n[3];              /* vertices along x, y, z */
    int C;                 /* feature channels (levels * feat with a hash encoding) */
    float aabb_min[3], aabb_max[3];
    double act_shift;      /* density activation shift (-4) */
    int dtype;             /* storage of density/features: 0 f64, 1 f32, 2 f16 bits */
    const void *density;   /* [z][y][x] */
    const void *features;  /* [z][y][x][C] */
    const uint8_t *occ;    /* [R][R][R] or NULL */
    int occ_res;
    const or_hash *hash;   /* NULL: features from the dense grid; else from the hash encoding */
} or_grid;

typedef struct {
    int in_dim, hidden, n_freq;
    int dtype;             /* 0 f64, 1 f32 */
    const void *w1, *b1, *w2, *b2, *w3, *b3;  /* row-major [out][in] */
} or_mlp;

typedef struct {
    float near_t, far_t;
    int n_samples;
    float step;            /* 0: n_samples midpoints in [near, far]; >0: march from box entry */
    float t_stop;          /* early stop when transmittance < t_stop (0: never) */
    float bg[3];
    float void_acc;        /* depth is +inf when the accumulated opacity is below this */
} or_sampling;

typedef struct {
    int kind;              /* 0: pinhole camera pixels, 1: explicit rays */
    int width, height;
    float f, cx, cy;
    float c2w[12];         /* row-major 3x4, OpenCV axes */
    const int32_t *pix;    /* optional pixel list (camera kind); NULL = every pixel */
    int n_pix;
    const float *o, *d;    /* explicit kind: [R][3] each */
    int n_rays;
} or_rays;

/* ------------------------------------------------------------------------------------------
 * input decoding */

static double f16_to_f64(uint16_t h) {
    int s = (h >> 15) & 1, e = (h >> 10) & 31, m = h & 1023;
    double v;
    if (e == 0) v = ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = ldexp((double)(m | 1024), e - 25);
    return s ? -v : v;
}

static double grid_val(const or_grid *g, const void *base, size_t i) {
    if (g->dtype == 0) return ((const double *)base)[i];
    if (g->dtype == 1) return (double)((const float *)base)[i];
    return f16_to_f64(((const uint16_t *)base)[i]);
}

static double mlp_w(const or_mlp *m, const void *base, size_t i) {
    return m->dtype == 0 ? ((const double *)base)[i] : (double)((const float *)base)[i];
}

static int n_rays_of(const or_rays *r) {
    if (r->kind == 1) return r->n_rays;
    return r->pix ? r->n_pix : r->width * r->height;
}

/* ------------------------------------------------------------------------------------------
 * Ray generation (Sec. II-B, Indexing: one ray per pixel).  Pixel p = j*W + i has its centre at
 * (i + 0.5, j + 0.5); the camera-space direction is ((u - cx)/f, (v - cy)/f, 1) (the pinhole
 * model of Eq. 1 and Eq. 3), rotated by the camera-to-world rotation and normalised.  */

static void ray_f32(const or_rays *r, int k, float o[3], float d[3]) {
    if (r->kind == 1) {
        for (int a = 0; a < 3; a++) { o[a] = r->o[3 * k + a]; d[a] = r->d[3 * k + a]; }
        return;
    }
    int p = r->pix ? r->pix[k] : k;
    int i = p % r->width, j = p / r->width;
    float u = (float)i + 0.5f, v = (float)j + 0.5f;
    float dx = (u - r->cx) / r->f;
    float dy = (v - r->cy) / r->f;
    const float *M = r->c2w;
    float w[3];
    for (int a = 0; a < 3; a++) w[a] = (M[4 * a] * dx + M[4 * a + 1] * dy) + M[4 * a + 2];
    float n = sqrtf((w[0] * w[0] + w[1] * w[1]) + w[2] * w[2]);
    for (int a = 0; a < 3; a++) { d[a] = w[a] / n; o[a] = M[4 * a + 3]; }
}

static void ray_f64(const or_rays *r, int k, double o[3], double d[3]) {
    if (r->kind == 1) {
        for (int a = 0; a < 3; a++) { o[a] = r->o[3 * k + a]; d[a] = r->d[3 * k + a]; }
        return;
    }
    int p = r->pix ? r->pix[k] : k;
    int i = p % r->width, j = p / r->width;
    double dx = ((double)i + 0.5 - (double)r->cx) / (double)r->f;
    double dy = ((double)j + 0.5 - (double)r->cy) / (double)r->f;
    const float *M = r->c2w;
    double w[3];
    for (int a = 0; a < 3; a++) w[a] = (double)M[4 * a] * dx + (double)M[4 * a + 1] * dy + (double)M[4 * a + 2];
    double n = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    for (int a = 0; a < 3; a++) { d[a] = w[a] / n; o[a] = (double)M[4 * a + 3]; }
}

/* ------------------------------------------------------------------------------------------
 * Sample placement (Sec. II-B: every ray takes a set of point samples along its direction).
 * step == 0: slot k sits at near + (k + 1/2) * (far - near) / S (midpoint rule), S slots.
 * step  > 0: the slab test gives the entry t_in and exit t_out of the box; slot k sits at
 *            t_in + (k + 1/2) * step while k < S and the slot is before t_out.
 * The FP32 variant fixes the slot count and positions used for decisions; the FP64 variant
 * gives the positions used for values. */

typedef struct { int n_slots; float t0, dt; } slots32;     /* t_k = t0 + (k + 0.5) * dt */

static int slab_f32(const or_grid *g, const float o[3], const float d[3], float tn, float tf,
                    float *tin, float *tout) {
    float lo = tn, hi = tf;
    for (int a = 0; a < 3; a++) {
        if (d[a] == 0.0f) {
            if (o[a] < g->aabb_min[a] || o[a] > g->aabb_max[a]) return 0;
            continue;
        }
        float t0 = (g->aabb_min[a] - o[a]) / d[a];
        float t1 = (g->aabb_max[a] - o[a]) / d[a];
        if (t0 > t1) { float s = t0; t0 = t1; t1 = s; }
        if (t0 > lo) lo = t0;
        if (t1 < hi) hi = t1;
    }
    *tin = lo; *tout = hi;
    return lo < hi;
}

static double slab_entry_f64(const or_grid *g, const double o[3], const double d[3], double tn) {
    double lo = tn;
    for (int a = 0; a < 3; a++) {
        if (d[a] == 0.0) continue;
        double t0 = ((double)g->aabb_min[a] - o[a]) / d[a];
        double t1 = ((double)g->aabb_max[a] - o[a]) / d[a];
        if (t0 > t1) t0 = t1;
        if (t0 > lo) lo = t0;
    }
    return lo;
}

static slots32 place_f32(const or_grid *g, const or_sampling *s, const float o[3], const float d[3]) {
    slots32 r;
    if (s->step <= 0.0f) {
        r.n_slots = s->n_samples;
        r.t0 = s->near_t;
        r.dt = (s->far_t - s->near_t) / (float)s->n_samples;
        return r;
    }
    float tin, tout;
    r.t0 = 0.0f; r.dt = s->step; r.n_slots = 0;
    if (!slab_f32(g, o, d, s->near_t, s->far_t, &tin, &tout)) return r;
    r.t0 = tin;
    int k = 0;
    while (k < s->n_samples && (tin + ((float)k + 0.5f) * s->step) < tout) k++;
    r.n_slots = k;
    return r;
}

static float slot_t_f32(const slots32 *sl, int k) { return sl->t0 + ((float)k + 0.5f) * sl->dt; }

/* ------------------------------------------------------------------------------------------
 * Indexing (Sec. II-B): the voxel that holds a sample.  Vertices sit on the box corners, so
 * the continuous vertex coordinate is g = (p - min) * (N - 1) / (max - min).  A sample counts
 * only when 0 <= g <= N - 1 on every axis (and its occupancy cell is set, when a mask is
 * given); its voxel is i0 = min(floor(g), N - 2).  Taken in FP32 (decision). */

typedef struct { int inside; int i0[3]; int cell[3]; } index32;

static index32 index_f32(const or_grid *g, const float p[3]) {
    index32 r;
    r.inside = 1;
    for (int a = 0; a < 3; a++) {
        float inv_h = (float)(g->n[a] - 1) / (g->aabb_max[a] - g->aabb_min[a]);
        float ga = (p[a] - g->aabb_min[a]) * inv_h;
        if (!(ga >= 0.0f && ga <= (float)(g->n[a] - 1))) { r.inside = 0; return r; }
        int i = (int)floorf(ga);
        if (i > g->n[a] - 2) i = g->n[a] - 2;
        r.i0[a] = i;
        if (g->occ) {
            float sc = (float)g->occ_res / (float)(g->n[a] - 1);
            int c = (int)floorf(ga * sc);
            if (c > g->occ_res - 1) c = g->occ_res - 1;
            r.cell[a] = c;
        }
    }
    if (g->occ) {
        int R = g->occ_res;
        if (!g->occ[((size_t)r.cell[2] * R + r.cell[1]) * R + r.cell[0]]) r.inside = 0;
    }
    return r;
}

/* Feature Gathering (Sec. II-B): the eight vertices of the voxel, trilinearly weighted. */
static void trilinear(const or_grid *g, const int i0[3], const double f[3], double *raw, double *feat) {
    int C = g->C;
    if (raw) *raw = 0.0;
    if (feat) for (int c = 0; c < C; c++) feat[c] = 0.0;
    for (int dz = 0; dz < 2; dz++)
        for (int dy = 0; dy < 2; dy++)
            for (int dx = 0; dx < 2; dx++) {
                double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                size_t v = ((size_t)(i0[2] + dz) * g->n[1] + (size_t)(i0[1] + dy)) * g->n[0] + (size_t)(i0[0] + dx);
                if (raw) *raw += w * grid_val(g, g->density, v);
                if (feat) for (int c = 0; c < C; c++) feat[c] += w * grid_val(g, g->features, v * C + c);
            }
}

static uint32_t hash_index(const or_hash *h, int l, uint32_t x, uint32_t y, uint32_t z) {
    const uint32_t n = (uint32_t)h->res[l] + 1u;
    const uint64_t T = 1ull << h->log2_size;
    if ((uint64_t)n * n * n <= T) return x + n * (y + n * z);
    return (x * 1u ^ y * 2654435761u ^ z * 805459861u) & (uint32_t)(T - 1);
}

/* Features of the hash encoding at world position p (FP64). */
static void hash_features(const or_grid *g, const double p[3], double *feat) {
    const or_hash *h = g->hash;
    const size_t T = (size_t)1 << h->log2_size;
    double pn[3];
    for (int a = 0; a < 3; a++) {
        double u = (p[a] - (double)g->aabb_min[a]) / ((double)g->aabb_max[a] - (double)g->aabb_min[a]);
        pn[a] = u < 0.0 ? 0.0 : (u > 1.0 ? 1.0 : u);
    }
    for (int l = 0; l < h->levels; l++) {
        const int N = h->res[l];
        int i0[3];
        double f[3];
        for (int a = 0; a < 3; a++) {
            double gx = pn[a] * N;
            int i = (int)floor(gx);
            if (i > N - 1) i = N - 1;
            i0[a] = i;
            f[a] = gx - i;
        }
        for (int c = 0; c < h->feat; c++) feat[l * h->feat + c] = 0.0;
        for (int dz = 0; dz < 2; dz++)
            for (int dy = 0; dy < 2; dy++)
                for (int dx = 0; dx < 2; dx++) {
                    double w = (dx ? f[0] : 1.0 - f[0]) * (dy ? f[1] : 1.0 - f[1]) * (dz ? f[2] : 1.0 - f[2]);
                    size_t e = ((size_t)l * T + hash_index(h, l, i0[0] + dx, i0[1] + dy, i0[2] + dz)) * h->feat;
                    for (int c = 0; c < h->feat; c++) {
                        double v = h->dtype == 1 ? (double)((const float *)h->table)[e + c]
                                                 : f16_to_f64(((const uint16_t *)h->table)[e + c]);
                        feat[l * h->feat + c] += w * v;
                    }
                }
    }
}

static double softplus(double x) { return x > 30.0 ? x + log1p(exp(-x)) : log1p(exp(x)); }
static double sigm(double x) { return 1.0 / (1.0 + exp(-x)); }

/* ------------------------------------------------------------------------------------------
 * Feature Computation (Sec. II-B, a small MLP whose shape the paper does not give).  Input x = [features (C), d (3),
 * then for k = 0..n_freq-1: sin(2^k d_x), sin(2^k d_y), sin(2^k d_z), cos(2^k d_x),
 * cos(2^k d_y), cos(2^k d_z)]; h1 = relu(W1 x + b1); h2 = relu(W2 h1 + b2);
 * c = sigmoid(W3 h2 + b3). */

static void encode(const or_mlp *m, int C, const double *feat, const double d[3], double *x) {
    for (int c = 0; c < C; c++) x[c] = feat[c];
    for (int a = 0; a < 3; a++) x[C + a] = d[a];
    for (int k = 0; k < m->n_freq; k++) {
        double s = ldexp(1.0, k);
        for (int a = 0; a < 3; a++) {
            x[C + 3 + 6 * k + a] = sin(s * d[a]);
            x[C + 3 + 6 * k + 3 + a] = cos(s * d[a]);
        }
    }
}

typedef struct { double pre1[OR_MAX_HIDDEN], h1[OR_MAX_HIDDEN], pre2[OR_MAX_HIDDEN], h2[OR_MAX_HIDDEN], z3[3], c[3]; } mlp_state;

static void mlp_fwd(const or_mlp *m, const double *x, mlp_state *st) {
    int I = m->in_dim, H = m->hidden;
    for (int o = 0; o < H; o++) {
        double s = mlp_w(m, m->b1, o);
        for (int i = 0; i < I; i++) s += mlp_w(m, m->w1, (size_t)o * I + i) * x[i];
        st->pre1[o] = s; st->h1[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < H; o++) {
        double s = mlp_w(m, m->b2, o);
        for (int i = 0; i < H; i++) s += mlp_w(m, m->w2, (size_t)o * H + i) * st->h1[i];
        st->pre2[o] = s; st->h2[o] = s > 0.0 ? s : 0.0;
    }
    for (int o = 0; o < 3; o++) {
        double s = mlp_w(m, m->b3, o);
        for (int i = 0; i < H; i++) s += mlp_w(m, m->w3, (size_t)o * H + i) * st->h2[i];
        st->z3[o] = s; st->c[o] = sigm(s);
    }
}

/* ------------------------------------------------------------------------------------------
 * One ray, front to back (accumulation, Sec. II-B: the samples of a ray are summed along it,
 * here with the standard emission-absorption quadrature):
 *   sigma_k = softplus(trilinear(density) + shift),  alpha_k = 1 - exp(-sigma_k * delta),
 *   T_0 = 1; before slot k: stop if T_k < t_stop; w_k = T_k alpha_k; T_{k+1} = T_k (1 - alpha_k)
 *   rgb = sum w_k c_k + T_end bg,  acc = sum w_k,  depth = sum w_k t_k / acc  (+inf if acc < void_acc)
 * flip_level >= 0 inverts the stop decisions taken while exactly flip_level samples with
 * alpha > 0 have been composited (the other outcome of an ambiguous decision). */

typedef struct {
    double rgb[3], depth, acc, T_end;
    int n_steps;
    int amb_level;   /* first ambiguous level, or -1 */
} ray_out;

typedef struct {
    int slot; double t, delta; int i0[3]; double f[3]; double raw, sigma, alpha, T, w;
    mlp_state st; double x[OR_MAX_IN];
} sample_rec;

static void march_ray(const or_grid *g, const or_mlp *m, const or_rays *rays, const or_sampling *s,
                      int r, int flip_level, ray_out *out, sample_rec *recs, int *n_recs) {
    float o32[3], d32[3];
    double o[3], d[3];
    ray_f32(rays, r, o32, d32);
    ray_f64(rays, r, o, d);
    slots32 sl = place_f32(g, s, o32, d32);
    double t0, dt;
    if (s->step <= 0.0f) { t0 = s->near_t; dt = ((double)s->far_t - (double)s->near_t) / s->n_samples; }
    else { t0 = slab_entry_f64(g, o, d, s->near_t); dt = s->step; }

    double T = 1.0, acc = 0.0, dsum = 0.0, rgb[3] = {0, 0, 0};
    double feat[OR_MAX_IN], x[OR_MAX_IN];
    int level = 0, k, nr = 0;
    out->amb_level = -1;
    for (k = 0; k < sl.n_slots; k++) {
        if (s->t_stop > 0.0f) {
            int stop = T < (double)s->t_stop;
            if (fabs(T - (double)s->t_stop) <= OR_AMBIG_REL * (double)s->t_stop && out->amb_level < 0)
                out->amb_level = level;
            if (level == flip_level) stop = !stop;
            if (stop) break;
        }
        float tk = slot_t_f32(&sl, k);
        float p32[3];
        for (int a = 0; a < 3; a++) p32[a] = o32[a] + tk * d32[a];
        index32 ix = index_f32(g, p32);
        if (!ix.inside) continue;
        double t = t0 + ((double)k + 0.5) * dt;
        double f[3];
        for (int a = 0; a < 3; a++) {
            double ga = (o[a] + t * d[a] - (double)g->aabb_min[a]) * (double)(g->n[a] - 1) /
                        ((double)g->aabb_max[a] - (double)g->aabb_min[a]);
            f[a] = ga - ix.i0[a];
        }
        double raw;
        trilinear(g, ix.i0, f, &raw, g->hash ? NULL : feat);
        if (g->hash) {
            double p[3];
            for (int a = 0; a < 3; a++) p[a] = o[a] + t * d[a];
            hash_features(g, p, feat);
        }
        double sigma = softplus(raw + g->act_shift);
        double alpha = -expm1(-sigma * dt);
        double w = T * alpha;
        encode(m, g->C, feat, d, x);
        mlp_state st;
        mlp_fwd(m, x, &st);
        for (int c = 0; c < 3; c++) rgb[c] += w * st.c[c];
        acc += w;
        dsum += w * t;
        if (recs) {
            sample_rec *q = &recs[nr];
            q->slot = k; q->t = t; q->delta = dt;
            memcpy(q->i0, ix.i0, sizeof q->i0);
            memcpy(q->f, f, sizeof q->f);
            q->raw = raw; q->sigma = sigma; q->alpha = alpha; q->T = T; q->w = w;
            q->st = st;
            memcpy(q->x, x, sizeof(double) * m->in_dim);
        }
        nr++;
        T *= (1.0 - alpha);
        level++;
    }
    for (int c = 0; c < 3; c++) out->rgb[c] = rgb[c] + T * (double)s->bg[c];
    out->acc = acc;
    out->T_end = T;
    out->depth = acc >= (double)s->void_acc ? dsum / acc : INFINITY;
    out->n_steps = k;
    if (n_recs) *n_recs = nr;
}

/* Render every ray.  rgb [R][3], depth/acc [R], n_steps/amb [R]; the *_alt arrays (may be NULL)
 * receive the other outcome of an ambiguous early-stop decision (a copy of the primary result
 * when the ray is not ambiguous). */
int or_render(const or_grid *g, const or_mlp *m, const or_rays *rays, const or_sampling *s,
              double *rgb, double *depth, double *acc, int32_t *n_steps, int32_t *amb,
              double *rgb_alt, double *depth_alt, double *acc_alt, int32_t *n_steps_alt, int nthreads) {
    int R = n_rays_of(rays);
    if (m->in_dim != g->C + 3 + 6 * m->n_freq || m->hidden > OR_MAX_HIDDEN || m->in_dim > OR_MAX_IN) return -1;
#ifdef _OPENMP
    const int nt = nthreads > 0 ? nthreads : omp_get_max_threads();  /* this call only */
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt)
#endif
    for (int r = 0; r < R; r++) {
        ray_out a, b;
        march_ray(g, m, rays, s, r, -1, &a, NULL, NULL);
        b = a;
        if (a.amb_level >= 0) march_ray(g, m, rays, s, r, a.amb_level, &b, NULL, NULL);
        for (int c = 0; c < 3; c++) rgb[3 * r + c] = a.rgb[c];
        if (depth) depth[r] = a.depth;
        if (acc) acc[r] = a.acc;
        if (n_steps) n_steps[r] = a.n_steps;
        if (amb) amb[r] = a.amb_level >= 0;
        if (rgb_alt) for (int c = 0; c < 3; c++) rgb_alt[3 * r + c] = b.rgb[c];
        if (depth_alt) depth_alt[r] = b.depth;
        if (acc_alt) acc_alt[r] = b.acc;
        if (n_steps_alt) n_steps_alt[r] = b.n_steps;
    }
    return 0;
}

/* The samples that reach Feature Gathering, in ray order then slot order, with the brick
 * ("MVoxel", Sec. IV-A) of B^3 voxels that holds each one: brick (bx, by, bz) = i0 / B and
 * id = (bz * nby + by) * nbx + bx with nb = ceil((N - 1) / B).  This is the content of the
 * Ray Index Table before it is grouped by brick.  voxel_of (may be NULL) receives the voxel i0 of
 * each sample as (i0z * Ny + i0y) * Nx + i0x.  Returns the number of samples (or -1 if `cap` is
 * too small); n_steps/amb as in or_render. */
long or_active_samples(const or_grid *g, const or_rays *rays, const or_sampling *s, int B,
                       int32_t *ray_of, int32_t *slot_of, int32_t *brick_of, int32_t *voxel_of, long cap,
                       int32_t *n_steps, int32_t *amb) {
    int R = n_rays_of(rays);
    int nb[3];
    for (int a = 0; a < 3; a++) nb[a] = (g->n[a] - 2) / B + 1;
    /* the stop decision needs the density; run the full march per ray (MLP skipped below) */
    or_mlp dummy;
    memset(&dummy, 0, sizeof dummy);
    long cnt = 0;
    for (int r = 0; r < R; r++) {
        float o32[3], d32[3];
        double o[3], d[3];
        ray_f32(rays, r, o32, d32);
        ray_f64(rays, r, o, d);
        slots32 sl = place_f32(g, s, o32, d32);
        double t0, dt;
        if (s->step <= 0.0f) { t0 = s->near_t; dt = ((double)s->far_t - (double)s->near_t) / s->n_samples; }
        else { t0 = slab_entry_f64(g, o, d, s->near_t); dt = s->step; }
        double T = 1.0;
        int k, am = 0;
        for (k = 0; k < sl.n_slots; k++) {
            if (s->t_stop > 0.0f) {
                if (fabs(T - (double)s->t_stop) <= OR_AMBIG_REL * (double)s->t_stop) am = 1;
                if (T < (double)s->t_stop) break;
            }
            float tk = slot_t_f32(&sl, k);
            float p32[3];
            for (int a = 0; a < 3; a++) p32[a] = o32[a] + tk * d32[a];
            index32 ix = index_f32(g, p32);
            if (!ix.inside) continue;
            double t = t0 + ((double)k + 0.5) * dt, f[3], raw;
            for (int a = 0; a < 3; a++)
                f[a] = (o[a] + t * d[a] - (double)g->aabb_min[a]) * (double)(g->n[a] - 1) /
                       ((double)g->aabb_max[a] - (double)g->aabb_min[a]) - ix.i0[a];
            trilinear(g, ix.i0, f, &raw, NULL);
            double alpha = -expm1(-softplus(raw + g->act_shift) * dt);
            if (cnt >= cap) return -1;
            ray_of[cnt] = r;
            slot_of[cnt] = k;
            brick_of[cnt] = ((ix.i0[2] / B) * nb[1] + ix.i0[1] / B) * nb[0] + ix.i0[0] / B;
            if (voxel_of) voxel_of[cnt] = (ix.i0[2] * g->n[1] + ix.i0[1]) * g->n[0] + ix.i0[0];
            cnt++;
            T *= 1.0 - alpha;
        }
        if (n_steps) n_steps[r] = k;
        if (amb) amb[r] = am;
    }
    return cnt;
}

/* ------------------------------------------------------------------------------------------
 * Pieces exposed for pin tests. */

/* Trilinear sample of density and features at FP64 points (i0 = min(floor(g), N - 2)). */
void or_sample_grid(const or_grid *g, const double *p, int n, double *raw, double *feat) {
    for (int k = 0; k < n; k++) {
        int i0[3];
        double f[3];
        for (int a = 0; a < 3; a++) {
            double ga = (p[3 * k + a] - (double)g->aabb_min[a]) * (double)(g->n[a] - 1) /
                        ((double)g->aabb_max[a] - (double)g->aabb_min[a]);
            int i = (int)floor(ga);
            if (i > g->n[a] - 2) i = g->n[a] - 2;
            if (i < 0) i = 0;
            i0[a] = i;
            f[a] = ga - i;
        }
        trilinear(g, i0, f, raw ? &raw[k] : NULL, feat ? &feat[(size_t)k * g->C] : NULL);
    }
}

/* The MLP on M encoded inputs x [M][in_dim] -> c [M][3]. */
void or_mlp_eval(const or_mlp *m, const double *x, int M, double *c) {
    for (int k = 0; k < M; k++) {
        mlp_state st;
        mlp_fwd(m, &x[(size_t)k * m->in_dim], &st);
        for (int a = 0; a < 3; a++) c[3 * k + a] = st.c[a];
    }
}

/* The MLP input for given features [M][C] and directions [M][3]. */
void or_encode(const or_mlp *m, int C, const double *feat, const double *d, int M, double *x) {
    for (int k = 0; k < M; k++) encode(m, C, &feat[(size_t)k * C], &d[3 * k], &x[(size_t)k * m->in_dim]);
}

/* ------------------------------------------------------------------------------------------
 * SpaRW target frame (Sec. III-B).  Reference pixel q = (i, j) with ray distance D:
 *   Eq. 1  z-depth Z = D / |((u - cx)/f, (v - cy)/f, 1)|,  P = Z ((u - cx)/f, (v - cy)/f, 1)
 *   Eq. 2  P' = R_rel P + t_rel, [R_rel | t_rel] = inverse(c2w_tgt) c2w_ref, formed in FP64
 *          from the float poses (R_tgt^T R_ref, R_tgt^T (t_ref - t_tgt)) and rounded to FP32
 *   Eq. 3  u' = f' X'/Z' + cx', v' = f' Y'/Z' + cy'; target pixel (floor(u'), floor(v'))
 * Points with Z' <= 1e-6 or outside the target image are dropped.  A reference pixel with
 * D = +inf (void) is a point at infinity: its direction is rotated and projected and it keeps
 * depth +inf.  Depth test: the smallest key (float bits of Z' << 32 | q) wins, i.e. the nearest
 * point, ties to the lower reference index.  With phi < 180 deg a point is kept only when the
 * angle between its reference ray and its target ray (theta in the paper's figure on the warping intuition) is below phi;
 * points at infinity have theta = 0.
 * Target pixels: a winner copies its reference colour (mask 0).  A pixel with no winner is a
 * hole; with a void grid given, a hole whose ray has no sample inside the box (and in an
 * occupied cell) is void (mask 2: background colour, depth +inf, skipped - the paper's depth
 * test: pixels at infinite depth are not rendered); the rest (mask 1) are listed in ascending pixel
 * order for sparse rendering (Eq. 4).  warped_depth (may be NULL) is |P'| for warped pixels. */

typedef struct { int width, height; float f, cx, cy; float c2w[12]; } or_cam;

static void rel_pose(const or_cam *ref, const or_cam *tgt, float Rr[9], float tr[3]) {
    double Ra[9], Rb[9], ta[3], tb[3];
    for (int a = 0; a < 3; a++) {
        for (int b = 0; b < 3; b++) { Ra[3 * a + b] = ref->c2w[4 * a + b]; Rb[3 * a + b] = tgt->c2w[4 * a + b]; }
        ta[a] = ref->c2w[4 * a + 3]; tb[a] = tgt->c2w[4 * a + 3];
    }
    for (int i = 0; i < 3; i++) {
        for (int j = 0; j < 3; j++) {
            double s = Rb[0 * 3 + i] * Ra[0 * 3 + j];
            s = s + Rb[1 * 3 + i] * Ra[1 * 3 + j];
            s = s + Rb[2 * 3 + i] * Ra[2 * 3 + j];
            Rr[3 * i + j] = (float)s;
        }
        double s = Rb[0 * 3 + i] * (ta[0] - tb[0]);
        s = s + Rb[1 * 3 + i] * (ta[1] - tb[1]);
        s = s + Rb[2 * 3 + i] * (ta[2] - tb[2]);
        tr[i] = (float)s;
    }
}

typedef struct { int ok; int px, py; float X, Y, Z; float zkey; } splat;

static splat splat_point(const or_cam *ref, const or_cam *tgt, const float Rr[9], const float tr[3],
                         float cos_phi, int use_phi, const float *ref_depth, int q) {
    splat s;
    s.ok = 0;
    int i = q % ref->width, j = q / ref->width;
    float u = (float)i + 0.5f, v = (float)j + 0.5f;
    float dx = (u - ref->cx) / ref->f;
    float dy = (v - ref->cy) / ref->f;
    float D = ref_depth[q];
    float P[3];
    int at_inf = isinf(D) && D > 0.0f;
    if (at_inf) {
        P[0] = dx; P[1] = dy; P[2] = 1.0f;
    } else {
        if (!(D > 0.0f)) return s;   /* NaN or non-positive depth: nothing to warp */
        float nrm = sqrtf((dx * dx + dy * dy) + 1.0f);
        float Z = D / nrm;
        P[0] = dx * Z; P[1] = dy * Z; P[2] = Z;
    }
    float Q[3];
    for (int a = 0; a < 3; a++) {
        float acc = (Rr[3 * a] * P[0] + Rr[3 * a + 1] * P[1]) + Rr[3 * a + 2] * P[2];
        Q[a] = at_inf ? acc : acc + tr[a];
    }
    if (!(Q[2] > 1e-6f)) return s;
    float up = (tgt->f * Q[0]) / Q[2] + tgt->cx;
    float vp = (tgt->f * Q[1]) / Q[2] + tgt->cy;
    if (!(up >= 0.0f && up < (float)tgt->width && vp >= 0.0f && vp < (float)tgt->height)) return s;
    if (use_phi && !at_inf) {
        float A[3] = {Q[0] - tr[0], Q[1] - tr[1], Q[2] - tr[2]};
        float dot = (A[0] * Q[0] + A[1] * Q[1]) + A[2] * Q[2];
        float na = sqrtf((A[0] * A[0] + A[1] * A[1]) + A[2] * A[2]);
        float nq = sqrtf((Q[0] * Q[0] + Q[1] * Q[1]) + Q[2] * Q[2]);
        if (!(dot > cos_phi * (na * nq))) return s;
    }
    s.ok = 1;
    s.px = (int)floorf(up);
    s.py = (int)floorf(vp);
    s.X = Q[0]; s.Y = Q[1]; s.Z = Q[2];
    s.zkey = at_inf ? INFINITY : Q[2];
    return s;
}

static uint64_t key_of(float z, int q) {
    uint32_t b;
    memcpy(&b, &z, 4);
    return ((uint64_t)b << 32) | (uint32_t)q;
}

/* Void depth test for a hole: does the target ray have any sample inside the box (and in an
 * occupied cell)?  Same FP32 slot placement and indexing as rendering. */
static int ray_has_sample(const or_grid *g, const or_sampling *s, const or_cam *tgt, int p) {
    or_rays rr;
    memset(&rr, 0, sizeof rr);
    rr.kind = 0; rr.width = tgt->width; rr.height = tgt->height;
    rr.f = tgt->f; rr.cx = tgt->cx; rr.cy = tgt->cy;
    memcpy(rr.c2w, tgt->c2w, sizeof rr.c2w);
    float o[3], d[3];
    ray_f32(&rr, p, o, d);
    slots32 sl = place_f32(g, s, o, d);
    for (int k = 0; k < sl.n_slots; k++) {
        float tk = slot_t_f32(&sl, k), p32[3];
        for (int a = 0; a < 3; a++) p32[a] = o[a] + tk * d[a];
        if (index_f32(g, p32).inside) return 1;
    }
    return 0;
}

static void resolve(const or_cam *ref, const or_cam *tgt, const float Rr[9], const float tr[3],
                    float cos_phi, int use_phi, const float *ref_rgb, const float *ref_depth,
                    const uint64_t *zbuf, const or_grid *vg, const or_sampling *vs,
                    float *warped_rgb, float *warped_depth, uint8_t *mask, int32_t *hole_idx, int32_t *n_holes) {
    int NT = tgt->width * tgt->height, nh = 0;
    for (int p = 0; p < NT; p++) {
        uint64_t key = zbuf[p];
        if (key != ~(uint64_t)0) {
            int q = (int)(key & 0xffffffffu);
            for (int c = 0; c < 3; c++) warped_rgb[3 * p + c] = ref_rgb[3 * q + c];
            if (warped_depth) {
                splat s = splat_point(ref, tgt, Rr, tr, cos_phi, use_phi, ref_depth, q);
                warped_depth[p] = isinf(s.zkey) ? INFINITY : sqrtf((s.X * s.X + s.Y * s.Y) + s.Z * s.Z);
            }
            mask[p] = 0;
        } else if (vg && !ray_has_sample(vg, vs, tgt, p)) {
            for (int c = 0; c < 3; c++) warped_rgb[3 * p + c] = vs->bg[c];
            if (warped_depth) warped_depth[p] = INFINITY;
            mask[p] = 2;
        } else {
            for (int c = 0; c < 3; c++) warped_rgb[3 * p + c] = 0.0f;
            if (warped_depth) warped_depth[p] = 0.0f;
            mask[p] = 1;
            hole_idx[nh++] = p;
        }
    }
    *n_holes = nh;
}

static float cos_of_deg(float deg) { return (float)cos((double)deg * 3.14159265358979323846 / 180.0); }

int or_warp(const float *ref_rgb, const float *ref_depth, const or_cam *ref, const or_cam *tgt,
            float max_angle_deg, const or_grid *void_grid, const or_sampling *void_s,
            float *warped_rgb, float *warped_depth, uint8_t *mask, int32_t *hole_idx, int32_t *n_holes,
            int32_t *src_of) {
    float Rr[9], tr[3];
    rel_pose(ref, tgt, Rr, tr);
    int use_phi = max_angle_deg < 180.0f;
    float cphi = use_phi ? cos_of_deg(max_angle_deg) : -1.0f;
    int NR = ref->width * ref->height, NT = tgt->width * tgt->height;
    uint64_t *zbuf = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)NT);
    if (!zbuf) return -1;
    for (int p = 0; p < NT; p++) zbuf[p] = ~(uint64_t)0;
    for (int q = 0; q < NR; q++) {
        splat s = splat_point(ref, tgt, Rr, tr, cphi, use_phi, ref_depth, q);
        if (!s.ok) continue;
        int p = s.py * tgt->width + s.px;
        uint64_t k = key_of(s.zkey, q);
        if (k < zbuf[p]) zbuf[p] = k;
    }
    if (src_of)
        for (int p = 0; p < NT; p++) src_of[p] = zbuf[p] == ~(uint64_t)0 ? -1 : (int32_t)(zbuf[p] & 0xffffffffu);
    resolve(ref, tgt, Rr, tr, cphi, use_phi, ref_rgb, ref_depth, zbuf, void_grid, void_s,
            warped_rgb, warped_depth, mask, hole_idx, n_holes);
    free(zbuf);
    return 0;
}

/* Brute-force depth test: for every target pixel, search all reference points for the smallest
 * key directly (no depth buffer).  src_of[p] = winning reference index or -1. */
void or_warp_bruteforce(const float *ref_depth, const or_cam *ref, const or_cam *tgt,
                        float max_angle_deg, int32_t *src_of) {
    float Rr[9], tr[3];
    rel_pose(ref, tgt, Rr, tr);
    int use_phi = max_angle_deg < 180.0f;
    float cphi = use_phi ? cos_of_deg(max_angle_deg) : -1.0f;
    int NR = ref->width * ref->height, NT = tgt->width * tgt->height;
    for (int p = 0; p < NT; p++) {
        uint64_t best = ~(uint64_t)0;
        for (int q = 0; q < NR; q++) {
            splat s = splat_point(ref, tgt, Rr, tr, cphi, use_phi, ref_depth, q);
            if (!s.ok || s.py * tgt->width + s.px != p) continue;
            uint64_t k = key_of(s.zkey, q);
            if (k < best) best = k;
        }
        src_of[p] = best == ~(uint64_t)0 ? -1 : (int32_t)(best & 0xffffffffu);
    }
}

/* The relative pose [R_rel | t_rel] as rounded to FP32 (row-major 3x4). */
void or_rel_pose(const or_cam *ref, const or_cam *tgt, float *out12) {
    float Rr[9], tr[3];
    rel_pose(ref, tgt, Rr, tr);
    for (int a = 0; a < 3; a++) {
        for (int b = 0; b < 3; b++) out12[4 * a + b] = Rr[3 * a + b];
        out12[4 * a + 3] = tr[a];
    }
}

/* ------------------------------------------------------------------------------------------
 * Gradient of a loss L(rgb) with respect to the grid (and optionally the MLP), given
 * d_rgb = dL/drgb [R][3].  Early stop is a fixed truncation (the primary decision).  For a ray
 * with composited samples k:
 *   dL/dc_k     = w_k g
 *   dL/dsigma_k = delta (T_{k+1} g.c_k - g.R_k),  R_k = sum_{j>k} w_j c_j + T_end bg
 *   dL/draw_k   = dL/dsigma_k * sigmoid(raw_k + shift)          (softplus' = sigmoid)
 * then the MLP chain rule (relu'(0) = 0) down to the feature inputs, and the trilinear adjoint
 * into the eight vertices.  d_mlp (may be NULL) is [W1, b1, W2, b2, W3, b3] flattened.
 * Accumulates into the output arrays (zero them first).  Single-threaded, FP64. */
int or_backward(const or_grid *g, const or_mlp *m, const or_rays *rays, const or_sampling *s,
                const double *d_rgb, double *d_density, double *d_features, double *d_mlp) {
    int R = n_rays_of(rays), C = g->C, I = m->in_dim, H = m->hidden;
    if (m->in_dim != C + 3 + 6 * m->n_freq || H > OR_MAX_HIDDEN || I > OR_MAX_IN) return -1;
    if (g->hash) return -3;  /* the gradient of the hash encoding is not defined here */
    int maxs = s->n_samples;
    sample_rec *recs = (sample_rec *)malloc(sizeof(sample_rec) * (size_t)(maxs > 0 ? maxs : 1));
    if (!recs) return -2;
    double *dW1 = NULL, *db1 = NULL, *dW2 = NULL, *db2 = NULL, *dW3 = NULL, *db3 = NULL;
    if (d_mlp) {
        dW1 = d_mlp; db1 = dW1 + (size_t)H * I; dW2 = db1 + H; db2 = dW2 + (size_t)H * H;
        dW3 = db2 + H; db3 = dW3 + 3 * H;
    }
    for (int r = 0; r < R; r++) {
        ray_out out;
        int nr = 0;
        march_ray(g, m, rays, s, r, -1, &out, recs, &nr);
        const double *gr = &d_rgb[3 * r];
        double Rk[3];
        for (int c = 0; c < 3; c++) Rk[c] = out.T_end * (double)s->bg[c];
        for (int q = nr - 1; q >= 0; q--) {
            sample_rec *e = &recs[q];
            double Tn = e->T * (1.0 - e->alpha);
            double gc = 0.0, gR = 0.0;
            for (int c = 0; c < 3; c++) { gc += gr[c] * e->st.c[c]; gR += gr[c] * Rk[c]; }
            double dsig = e->delta * (Tn * gc - gR);
            double draw = dsig * sigm(e->raw + g->act_shift);
            for (int c = 0; c < 3; c++) Rk[c] += e->w * e->st.c[c];
            /* MLP backward */
            double dz3[3], dh2[OR_MAX_HIDDEN], dh1[OR_MAX_HIDDEN], dx[OR_MAX_IN];
            for (int c = 0; c < 3; c++) dz3[c] = e->w * gr[c] * e->st.c[c] * (1.0 - e->st.c[c]);
            for (int i = 0; i < H; i++) {
                double a = 0.0;
                for (int c = 0; c < 3; c++) a += mlp_w(m, m->w3, (size_t)c * H + i) * dz3[c];
                dh2[i] = e->st.pre2[i] > 0.0 ? a : 0.0;
            }
            for (int i = 0; i < H; i++) {
                double a = 0.0;
                for (int o = 0; o < H; o++) a += mlp_w(m, m->w2, (size_t)o * H + i) * dh2[o];
                dh1[i] = e->st.pre1[i] > 0.0 ? a : 0.0;
            }
            for (int i = 0; i < C; i++) {
                double a = 0.0;
                for (int o = 0; o < H; o++) a += mlp_w(m, m->w1, (size_t)o * I + i) * dh1[o];
                dx[i] = a;
            }
            if (d_mlp) {
                for (int c = 0; c < 3; c++) {
                    for (int i = 0; i < H; i++) dW3[(size_t)c * H + i] += dz3[c] * e->st.h2[i];
                    db3[c] += dz3[c];
                }
                for (int o = 0; o < H; o++) {
                    for (int i = 0; i < H; i++) dW2[(size_t)o * H + i] += dh2[o] * e->st.h1[i];
                    db2[o] += dh2[o];
                }
                for (int o = 0; o < H; o++) {
                    for (int i = 0; i < I; i++) dW1[(size_t)o * I + i] += dh1[o] * e->x[i];
                    db1[o] += dh1[o];
                }
            }
            /* trilinear adjoint */
            for (int dz = 0; dz < 2; dz++)
                for (int dy = 0; dy < 2; dy++)
                    for (int dxv = 0; dxv < 2; dxv++) {
                        double w = (dxv ? e->f[0] : 1.0 - e->f[0]) * (dy ? e->f[1] : 1.0 - e->f[1]) *
                                   (dz ? e->f[2] : 1.0 - e->f[2]);
                        size_t v = ((size_t)(e->i0[2] + dz) * g->n[1] + (size_t)(e->i0[1] + dy)) * g->n[0] +
                                   (size_t)(e->i0[0] + dxv);
                        d_density[v] += w * draw;
                        for (int c = 0; c < C; c++) d_features[v * C + c] += w * dx[c];
                    }
        }
    }
    free(recs);
    return 0;
}

/* Pre-activations of every composited sample (for the ReLU-kink guard of finite-difference
 * tests): writes min over hidden units of |pre1|, |pre2| per ray into kink[R]. */
void or_relu_margin(const or_grid *g, const or_mlp *m, const or_rays *rays, const or_sampling *s, double *kink) {
    int R = n_rays_of(rays), H = m->hidden;
    sample_rec *recs = (sample_rec *)malloc(sizeof(sample_rec) * (size_t)(s->n_samples > 0 ? s->n_samples : 1));
    for (int r = 0; r < R; r++) {
        ray_out out;
        int nr = 0;
        march_ray(g, m, rays, s, r, -1, &out, recs, &nr);
        double mn = INFINITY;
        for (int q = 0; q < nr; q++)
            for (int i = 0; i < H; i++) {
                double a = fabs(recs[q].st.pre1[i]), b = fabs(recs[q].st.pre2[i]);
                if (a < mn) mn = a;
                if (b < mn) mn = b;
            }
        kink[r] = mn;
    }
    free(recs);
}

/* The rays of a ray set (Sec. II-B Indexing; pinhole of Eq. 1 / Eq. 3): origin and unit
 * direction of every ray, both the FP32 rays that take the integer decisions and the FP64 rays
 * that carry the values.  o32, d32, o64, d64: [n_rays][3]; any of them may be NULL. */
void or_rays_of(const or_rays *rays, float *o32, float *d32, double *o64, double *d64) {
    const int R = n_rays_of(rays);
    for (int k = 0; k < R; k++) {
        float of[3], df[3];
        double od[3], dd[3];
        ray_f32(rays, k, of, df);
        ray_f64(rays, k, od, dd);
        for (int a = 0; a < 3; a++) {
            if (o32) o32[3 * k + a] = of[a];
            if (d32) d32[3 * k + a] = df[a];
            if (o64) o64[3 * k + a] = od[a];
            if (d64) d64[3 * k + a] = dd[a];
        }
    }
}

/* Features of the hash encoding at n world positions p [n][3] -> feat [n][levels * feat]. */
void or_hash_features(const or_grid *g, const double *p, int n, double *feat) {
    for (int i = 0; i < n; i++) hash_features(g, p + 3 * i, feat + (size_t)i * g->C);
}

int or_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
