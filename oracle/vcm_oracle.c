/*
 * vcm_oracle.c -- plain CPU oracle for the visibility color map.
 *
 * TEST INFRASTRUCTURE ONLY (see vcm_oracle.h).  Written for a reader to check
 * against the paper by eye: no culling, no blocking, no reordering beyond the
 * definitions.  Occlusion is the OR over all boxes of an exact segment/box
 * predicate; the visibility is a float64 Neumaier sum over patches.
 */
#include "vcm_oracle.h"

#include <math.h>
#include <pthread.h>
#include <stdlib.h>
#include <string.h>

#define UNITS_PER_M 1024.0
#define VO_PI 3.14159265358979323846
#define COORD_LIMIT ((int64_t)1 << 24)

static int axis_index(int32_t code) { return code >> 1; }
static int64_t axis_sign(int32_t code) { return (code & 1) ? -1 : 1; }

/* Nearest integer to num/den (den > 0), halves rounded away from zero. */
static int64_t round_half_away(int64_t num, int64_t den)
{
    if (num >= 0)
        return (2 * num + den) / (2 * den);
    return -((2 * (-num) + den) / (2 * den));
}

static int in_limit(int64_t x) { return x >= -COORD_LIMIT && x <= COORD_LIMIT; }

static int vo_check_scene(const vo_scene *s, int dims)
{
    if (!s)
        return 0;
    if (s->dims != dims || s->n_boxes < 0 || (s->n_boxes > 0 && (!s->lo || !s->hi)))
        return -1;
    for (int64_t i = 0; i < s->n_boxes; ++i)
        for (int k = 0; k < s->dims; ++k) {
            int64_t lo = s->lo[3 * i + k], hi = s->hi[3 * i + k];
            if (lo > hi || !in_limit(lo) || !in_limit(hi))
                return -1;
        }
    return 0;
}

int vo_check(const vo_scene *s, const vo_request *r)
{
    if (!r || (r->dims != 2 && r->dims != 3))
        return -1;
    if (r->mode < VO_PARTIAL || r->mode > VO_VIEWER)
        return -1;
    if (r->mode == VO_VIEWER) {
        if (r->width <= 0 || r->grid_nx < 1 || r->grid_ny < 1 || (r->dims == 3 && (r->n_layers < 1 || !r->layer_z)))
            return -1;
        for (int k = 0; k < 3; ++k)
            if (!in_limit(r->center[k]))
                return -1;
        return vo_check_scene(s, r->dims);
    }
    if (r->axis_u < 0 || r->axis_u > 5 || r->normal < 0 || r->normal > 5)
        return -1;
    if ((r->two_sided != 0 && r->two_sided != 1) || !isfinite(r->fov_deg) || r->fov_deg < 0.0f)
        return -1;
    for (int k = 0; k < 3; ++k)
        if (!isfinite(r->gaze[k]))
            return -1;
    if (r->dims == 3) {
        if (r->axis_w < 0 || r->axis_w > 5)
            return -1;
        int a = axis_index(r->axis_u), b = axis_index(r->axis_w), c = axis_index(r->normal);
        if (a == b || a == c || b == c)
            return -1;
        if (r->patches_w < 1 || r->height <= 0 || r->n_layers < 1 || !r->layer_z)
            return -1;
    } else {
        if (axis_index(r->axis_u) > 1 || axis_index(r->normal) > 1 ||
            axis_index(r->axis_u) == axis_index(r->normal))
            return -1;
    }
    if (r->patches_u < 1 || r->width <= 0 || r->grid_nx < 1 || r->grid_ny < 1)
        return -1;
    return vo_check_scene(s, r->dims);
}

/* Patch centre: c + ((i + 1/2)/N - 1/2) * W along u (and likewise along w),
 * i.e. the centre of each of the N equal parts (cell centre as the cell's
 * representative, Section III-A end), rounded to the lattice. */
int vo_patch_centres(const vo_request *r, int64_t *out)
{
    int nw = (r->dims == 3) ? r->patches_w : 1;
    int au = axis_index(r->axis_u), aw = axis_index(r->axis_w);
    int64_t su = axis_sign(r->axis_u), sw = axis_sign(r->axis_w);
    int64_t Nu = r->patches_u, Nw = nw;
    for (int iw = 0; iw < nw; ++iw)
        for (int iu = 0; iu < r->patches_u; ++iu) {
            int64_t *p = out + 3 * ((int64_t)iw * r->patches_u + iu);
            p[0] = r->center[0];
            p[1] = r->center[1];
            p[2] = (r->dims == 3) ? r->center[2] : 0;
            /* exact coordinate times 2N, then rounded */
            int64_t num_u = 2 * Nu * r->center[au] + su * (2 * iu + 1 - Nu) * r->width;
            p[au] = round_half_away(num_u, 2 * Nu);
            if (r->dims == 3) {
                int64_t num_w = 2 * Nw * r->center[aw] + sw * (2 * iw + 1 - Nw) * r->height;
                p[aw] = round_half_away(num_w, 2 * Nw);
            }
            for (int k = 0; k < 3; ++k)
                if (!in_limit(p[k]))
                    return -1;
        }
    return 0;
}

double vo_patch_measure(const vo_request *r)
{
    double len_u = (double)r->width / UNITS_PER_M / (double)r->patches_u;
    if (r->dims == 2)
        return len_u;
    return len_u * ((double)r->height / UNITS_PER_M / (double)r->patches_w);
}

/* Viewpoint = centre of grid cell (ix, iy) on layer z, rounded to the lattice. */
int vo_viewpoint(const vo_request *r, int64_t index, int64_t out[3])
{
    int64_t nx = r->grid_nx, ny = r->grid_ny;
    int64_t ix = index % nx;
    int64_t iy = (index / nx) % ny;
    int64_t layer = index / (nx * ny);
    out[0] = round_half_away(2 * r->grid_origin[0] + (2 * ix + 1) * r->grid_step[0], 2);
    out[1] = round_half_away(2 * r->grid_origin[1] + (2 * iy + 1) * r->grid_step[1], 2);
    out[2] = (r->dims == 3) ? r->layer_z[layer] : 0;
    for (int k = 0; k < 3; ++k)
        if (!in_limit(out[k]))
            return -1;
    return 0;
}

/* Point-to-point visibility (Def. 2) against one box, with touching counted
 * as blocking (Def. 4).  The segment is q + t (p - q), t in [0, 1].  Along
 * each axis the points inside the slab [lo, hi] form a t-interval; the
 * segment meets the box iff the intersection of those intervals with [0, 1]
 * is non-empty.  Interval ends are kept as fractions n/d with d > 0 and
 * compared by cross-multiplication; all values are below 2^26 in magnitude,
 * so every product fits easily in int64 and the answer is exact. */
int vo_segment_hits_box(int dims, const int64_t q[3], const int64_t p[3],
                        const int64_t lo[3], const int64_t hi[3])
{
    int64_t lower_n[4], lower_d[4], upper_n[4], upper_d[4];
    int n_lower = 0, n_upper = 0;
    lower_n[n_lower] = 0; lower_d[n_lower++] = 1;   /* t >= 0 */
    upper_n[n_upper] = 1; upper_d[n_upper++] = 1;   /* t <= 1 */
    for (int k = 0; k < dims; ++k) {
        int64_t d = p[k] - q[k];
        int64_t a = lo[k] - q[k];
        int64_t b = hi[k] - q[k];
        if (d == 0) {
            /* the segment runs parallel to this slab: inside it or never */
            if (a > 0 || b < 0)
                return 0;
            continue;
        }
        if (d > 0) {
            lower_n[n_lower] = a;  lower_d[n_lower++] = d;
            upper_n[n_upper] = b;  upper_d[n_upper++] = d;
        } else {
            lower_n[n_lower] = -b; lower_d[n_lower++] = -d;
            upper_n[n_upper] = -a; upper_d[n_upper++] = -d;
        }
    }
    for (int i = 0; i < n_lower; ++i)
        for (int j = 0; j < n_upper; ++j)
            if (lower_n[i] * upper_d[j] > upper_n[j] * lower_d[i])
                return 0;
    return 1;
}

static int patch_blocked(const vo_scene *s, const int64_t q[3], const int64_t p[3])
{
    for (int64_t b = 0; b < s->n_boxes; ++b)
        if (vo_segment_hits_box(s->dims, q, p, s->lo + 3 * b, s->hi + 3 * b))
            return 1;
    return 0;
}

/* Viewer-centric value of one grid cell (Section IV-B; VO_VIEWER above). */
static double viewer_value(const vo_scene *s, const vo_request *r, const int64_t q[3], uint32_t *bits)
{
    int64_t v[3] = {r->center[0], r->center[1], (r->dims == 3) ? r->center[2] : 0};
    int blocked = patch_blocked(s, q, v);
    if (bits)
        bits[0] = blocked ? 1u : 0u;
    double dx = (double)(q[0] - v[0]) / UNITS_PER_M, dy = (double)(q[1] - v[1]) / UNITS_PER_M;
    double dz = (double)(q[2] - v[2]) / UNITS_PER_M;
    double D = sqrt(dx * dx + dy * dy + dz * dz);
    if (blocked || !(D > 0.0))
        return 0.0;
    double S = (double)r->width / UNITS_PER_M;
    if (r->dims == 2)
        return 2.0 * atan(S / (2.0 * D));              /* Eq. 1 */
    return 4.0 * asin(S * S / (S * S + 4.0 * D * D));  /* S x S square facing the viewer */
}

/* Field of view (vcm_oracle.h): the cosine c of the cone's half-angle and
 * its unit axis a, in float64, or 0 when there is no cone. */
static int fov_setup(const vo_request *r, double *c, double a[3])
{
    if (!(r->fov_deg > 0.0f) || r->fov_deg >= 360.0f)
        return 0;
    *c = cos((double)r->fov_deg * VO_PI / 360.0);
    double g[3] = {r->gaze[0], r->gaze[1], r->dims == 3 ? r->gaze[2] : 0.0f};
    if (g[0] == 0.0 && g[1] == 0.0 && g[2] == 0.0)
        g[axis_index(r->normal)] = (double)axis_sign(r->normal);
    double len = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
    for (int k = 0; k < 3; ++k)
        a[k] = g[k] / len;
    return 1;
}

/* The cone test in float64 (Section III-B, Table II): q lies in the cone of
 * patch p iff the angle between r = q - p and the axis a is at most half the
 * field of view, i.e. a.r >= c |r| (|a.r| for a two-sided target).  The
 * differences are exact (lattice values), so the only roundings are those
 * of the dot product, the norm and the product, about 1e-15 |r|.  Returns
 * the decision; *margin gets (a.r - c |r|) / |r| (0 when q = p). */
static int in_fov(const int64_t q[3], const int64_t p[3], double c, const double a[3], int two_sided,
                  double *margin)
{
    double rk[3];
    for (int k = 0; k < 3; ++k)
        rk[k] = (double)(q[k] - p[k]) / UNITS_PER_M;
    double d = a[0] * rk[0] + a[1] * rk[1] + a[2] * rk[2];
    if (two_sided)
        d = fabs(d);
    double len = sqrt(rk[0] * rk[0] + rk[1] * rk[1] + rk[2] * rk[2]);
    double m = d - c * len;
    *margin = len > 0.0 ? m / len : 0.0;
    return m >= 0.0;
}

int vo_fov_test(const vo_request *r, const int64_t q[3], const int64_t p[3], double *margin)
{
    double c = 0.0, a[3] = {0.0, 0.0, 0.0}, m = 0.0;
    if (!fov_setup(r, &c, a))
        return -1;
    int in = in_fov(q, p, c, a, r->two_sided, &m);
    if (margin)
        *margin = m;
    return in;
}

double vo_visibility_ex(const vo_scene *s, const vo_request *r, int64_t index, uint32_t *bits, double band[3])
{
    int64_t q[3];
    if (band)
        band[0] = band[1] = band[2] = 0.0;
    if (vo_viewpoint(r, index, q) != 0)
        return NAN;
    if (r->mode == VO_VIEWER)
        return viewer_value(s, r, q, bits);
    int64_t P = (int64_t)r->patches_u * ((r->dims == 3) ? r->patches_w : 1);
    int64_t *pc = (int64_t *)malloc(sizeof(int64_t) * 3 * P);
    if (!pc || vo_patch_centres(r, pc) != 0) {
        free(pc);
        return NAN;
    }
    int64_t words = (P + 31) / 32;
    if (bits)
        memset(bits, 0, sizeof(uint32_t) * words);
    int an = axis_index(r->normal);
    double sn = (double)axis_sign(r->normal);
    double measure = vo_patch_measure(r);
    double fov_c = 0.0, fov_a[3] = {0.0, 0.0, 0.0};
    int cone = fov_setup(r, &fov_c, fov_a);
    double sum = 0.0, comp = 0.0;   /* Neumaier running sum and compensation */
    double b_pairs = 0.0, b_in = 0.0, b_out = 0.0;
    int any_blocked = 0;
    for (int64_t j = 0; j < P; ++j) {
        const int64_t *p = pc + 3 * j;
        /* cos(theta) * |r| = n . (q - p): positive in front of the target;
         * a two-sided target is seen from either side */
        double cos_r = sn * (double)(q[an] - p[an]) / UNITS_PER_M;
        if (r->two_sided)
            cos_r = fabs(cos_r);
        int blocked = 0;
        if (bits || cos_r > 0.0 || r->mode == VO_STRICT)
            blocked = patch_blocked(s, q, p);
        any_blocked |= blocked;
        if (bits && blocked)
            bits[j >> 5] |= 1u << (j & 31);
        if (blocked || !(cos_r > 0.0))
            continue;
        double rx = (double)(q[0] - p[0]) / UNITS_PER_M;
        double ry = (double)(q[1] - p[1]) / UNITS_PER_M;
        double rz = (double)(q[2] - p[2]) / UNITS_PER_M;
        double d2 = rx * rx + ry * ry + rz * rz;
        double term;
        if (r->dims == 3)
            term = measure * cos_r / (d2 * sqrt(d2));   /* A cos(theta) / d^2 */
        else
            term = measure * cos_r / d2;                /* len cos(theta) / d */
        if (cone) {
            double margin;
            int in = in_fov(q, p, fov_c, fov_a, r->two_sided, &margin);
            if (fabs(margin) <= VO_FOV_BAND) {
                /* a float32 evaluation of the cone may decide this pair
                 * either way */
                b_pairs += 1.0;
                if (in)
                    b_in += term;
                else
                    b_out += term;
            }
            if (!in)
                continue;   /* outside the target's field of view */
        }
        double t = sum + term;
        if (fabs(sum) >= fabs(term))
            comp += (sum - t) + term;
        else
            comp += (term - t) + sum;
        sum = t;
    }
    free(pc);
    if (r->mode == VO_STRICT && any_blocked)
        return 0.0;   /* not completely visible: obstructed region */
    if (band) {
        band[0] = b_pairs;
        band[1] = b_in;
        band[2] = b_out;
    }
    return sum + comp;
}

double vo_visibility(const vo_scene *s, const vo_request *r, int64_t index, uint32_t *bits)
{
    return vo_visibility_ex(s, r, index, bits, NULL);
}

typedef struct {
    const vo_scene *s;
    const vo_request *r;
    const int64_t *indices;
    int64_t n;
    double *v_out;
    uint32_t *bits_out;
    double *band_out;
    int64_t words;
    int tid, threads;
} vo_job;

static void *vo_worker(void *arg)
{
    vo_job *job = (vo_job *)arg;
    for (int64_t i = job->tid; i < job->n; i += job->threads) {
        uint32_t *bits = job->bits_out ? job->bits_out + i * job->words : NULL;
        double *band = job->band_out ? job->band_out + 3 * i : NULL;
        job->v_out[i] = vo_visibility_ex(job->s, job->r, job->indices[i], bits, band);
    }
    return NULL;
}

int vo_run_ex(const vo_scene *s, const vo_request *r, const int64_t *indices, int64_t n,
              double *v_out, uint32_t *bits_out, double *band_out, int threads)
{
    if (vo_check(s, r) != 0)
        return -1;
    int64_t nvp = (int64_t)r->grid_nx * r->grid_ny * ((r->dims == 3) ? r->n_layers : 1);
    for (int64_t i = 0; i < n; ++i)
        if (indices[i] < 0 || indices[i] >= nvp)
            return -1;
    int64_t P = (r->mode == VO_VIEWER) ? 1 : (int64_t)r->patches_u * ((r->dims == 3) ? r->patches_w : 1);
    if (threads < 1)
        threads = 1;
    if (threads > 256)
        threads = 256;
    pthread_t tids[256];
    vo_job jobs[256];
    for (int t = 0; t < threads; ++t) {
        jobs[t] = (vo_job){s, r, indices, n, v_out, bits_out, band_out, (P + 31) / 32, t, threads};
        pthread_create(&tids[t], NULL, vo_worker, &jobs[t]);
    }
    for (int t = 0; t < threads; ++t)
        pthread_join(tids[t], NULL);
    for (int64_t i = 0; i < n; ++i)
        if (isnan(v_out[i]))
            return -1;
    return 0;
}

int vo_run(const vo_scene *s, const vo_request *r, const int64_t *indices, int64_t n,
           double *v_out, uint32_t *bits_out, int threads)
{
    return vo_run_ex(s, r, indices, n, v_out, bits_out, NULL, threads);
}

double vo_max(const double *v, int64_t n)
{
    double m = 0.0;
    for (int64_t i = 0; i < n; ++i)
        if (v[i] > m)
            m = v[i];
    return m;
}

/* Colors normalised to [0,1] (Def. 1) in L levels; zero visibility keeps
 * level 0 (obstructed regions take color zero, Section III-C). */
int vo_quantise(const double *v, int64_t n, double v_ref, int levels, uint8_t *color_out)
{
    if (levels < 2 || levels > 256)
        return -1;
    for (int64_t i = 0; i < n; ++i) {
        if (!(v[i] > 0.0) || !(v_ref > 0.0)) {
            color_out[i] = 0;
            continue;
        }
        double x = floor((double)(levels - 1) * v[i] / v_ref);
        if (x > (double)(levels - 2))
            x = (double)(levels - 2);
        color_out[i] = (uint8_t)(1 + (int)x);
    }
    return 0;
}
