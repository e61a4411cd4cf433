/*
 * vcm_oracle.h -- plain, slow CPU oracle for the visibility color map (VCM).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The GPU library shares no
 * code, header, table or helper with it.
 *
 * What it computes (target-centric VCM, Def. 1 of Section II-A):
 *   - the target is an axis-aligned rectangle (3D) or segment (2D) split into
 *     patches_u x patches_w patches whose centres are the sample points
 *     (a cell is represented by its centre, Section III-A end);
 *   - a viewpoint q sees patch centre p iff the closed segment qp meets no
 *     obstacle box (point-to-point visibility, Def. 2 of Section II-B.2; a
 *     segment that only touches a box is blocked, Def. 4 of Section III-B);
 *   - the visibility is the sum over visible patches of A*cos(theta)/d^2 (3D,
 *     the solid angle of the visible part) or len*cos(theta)/d (2D, the
 *     subtended angle, which reduces to Eq. 1 of Section II-B.1 for an
 *     unobstructed target seen head-on);
 *   - colors are the visibility normalised to [0,1] (Def. 1) and cut into
 *     L levels, with level 0 reserved for zero visibility (Section III-C).
 *
 * Lengths are integer lattice units of 2^-10 m; every coordinate must satisfy
 * |x| <= 2^24 units.  Occlusion is decided in exact int64 arithmetic; the
 * measure is summed in float64 with Neumaier compensation.
 *
 * Axis codes: 0 = +x, 1 = -x, 2 = +y, 3 = -y, 4 = +z, 5 = -z.
 */
#ifndef VCM_ORACLE_H
#define VCM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int32_t dims;        /* 2 or 3 */
    int64_t n_boxes;
    const int64_t *lo;   /* [n_boxes][3], lattice units (z ignored in 2D) */
    const int64_t *hi;   /* [n_boxes][3] */
} vo_scene;

typedef struct {
    int32_t dims;
    int64_t center[3];
    int32_t axis_u, axis_w, normal;   /* axis codes; axis_w unused in 2D */
    int64_t width, height;            /* along u and w, lattice units */
    int32_t patches_u, patches_w;     /* patches_w = 1 in 2D */
    int64_t grid_origin[2];           /* corner of the viewpoint grid (x, y) */
    int64_t grid_step[2];
    int32_t grid_nx, grid_ny;
    int32_t n_layers;
    const int64_t *layer_z;           /* [n_layers]; ignored in 2D */
    int32_t mode;                     /* VO_PARTIAL, VO_STRICT or VO_VIEWER */
    int32_t two_sided;                /* 1: the target counts from both faces */
    float fov_deg;                    /* field of view of the target; 0 or >= 360: none */
    float gaze[3];                    /* axis of the field of view (world); 0,0,0: the normal */
} vo_request;

/* Modes.
 * VO_PARTIAL: the sum over the unblocked patches (above).
 * VO_STRICT:  the viewpoint keeps the whole target's measure only if no
 *             patch is blocked, else 0 (the visible region holds the points
 *             from which the target is completely visible, Def. 3 and the
 *             end of Section III-B).
 * VO_VIEWER:  viewer-centric VCM (Section IV-B): `center` is the viewer and
 *             `width` the size S of an object placed at each grid cell and
 *             facing the viewer; a cell's value is the object's visual angle
 *             2 atan(S / 2D) (2D, Eq. 1) or the solid angle of an S x S
 *             square 4 asin(S^2 / (S^2 + 4 D^2)) (3D), D the distance to the
 *             viewer, and 0 if the segment to the viewer is blocked or D = 0.
 *             One occlusion bit per cell. */
enum { VO_PARTIAL = 0, VO_STRICT = 1, VO_VIEWER = 2 };

/* Sides and field of view (target-centric modes only).
 * two_sided = 0: a patch counts only from the side its normal faces,
 *   s = n.(q - p) > 0 (one-sided target; nothing counts from behind).
 * two_sided = 1: both faces count; the term uses |s| and s = 0 gives 0.
 * fov_deg in (0, 360): the target sees only a cone of half-angle fov/2
 *   around the gaze axis a (Section III-B sets up the visible region as the
 *   part of space inside the field of view, 120 degrees by default, Table II;
 *   Section IV-C turns the gaze).  A patch p counts for q only when q lies in
 *   p's cone, that is when the angle between r = q - p and a is at most
 *   fov/2:  a.r >= cos(fov/2) |r|  (|a.r| for a two-sided target), with
 *   a = g / |g| (g = gaze, or the target's normal if gaze is 0).  The oracle
 *   decides this in float64 on the exact differences r.
 *   A float32 evaluation of the same inequality (one rounding per operation,
 *   as the GPU path makes it) errs in the margin a.r - c |r| by at most
 *   about 10.5 u |r| (u = 2^-24): 5 u from the rounded r, axis, products and
 *   two sums of the dot product, 5.5 u from the rounded squares, sums, square
 *   root, cosine and product of the right-hand side.  So it can decide a
 *   pair differently only where |a.r - c |r|| <= VO_FOV_BAND |r|; those
 *   pairs are reported by vo_visibility_ex.
 * Strict mode with a cone: 0 if any patch is blocked, else the sum over the
 * patches inside the cone. */

/* Relative cone margin within which a float32 evaluation of the cone test
 * may differ from the exact one (more than twice the 10.5 u bound above). */
#define VO_FOV_BAND 1e-6

/* 0 on success, -1 on an invalid request. */
int vo_check(const vo_scene *s, const vo_request *r);

/* Patch centres, [patches_w * patches_u][3] units, index j = iw*patches_u + iu. */
int vo_patch_centres(const vo_request *r, int64_t *out);

/* Area (3D, m^2) or length (2D, m) of one patch. */
double vo_patch_measure(const vo_request *r);

/* Viewpoint centre of grid index ((layer*ny)+iy)*nx+ix, in units. */
int vo_viewpoint(const vo_request *r, int64_t index, int64_t out[3]);

/* 1 iff the closed segment q-p meets the closed box [lo, hi] (exact). */
int vo_segment_hits_box(int dims, const int64_t q[3], const int64_t p[3],
                        const int64_t lo[3], const int64_t hi[3]);

/* Visibility of the target from viewpoint `index`.  If bits != NULL, the
 * occlusion bit of every patch is written (ceil(P/32) words, bit j set iff
 * patch j is blocked). */
double vo_visibility(const vo_scene *s, const vo_request *r, int64_t index, uint32_t *bits);

/* The same; if band != NULL it also receives, over the unblocked patches in
 * front (those with a term) whose cone margin lies within VO_FOV_BAND of the
 * cone's edge: band[0] their number, band[1] the sum of the terms of those
 * counted (inside the cone), band[2] the sum of those left out.  A float32
 * evaluation of the cone therefore gives a value in
 * [v - band[1], v + band[2]].  All zero without a cone, and in strict mode
 * when a patch is blocked (the value is 0 whatever the cone decides). */
double vo_visibility_ex(const vo_scene *s, const vo_request *r, int64_t index, uint32_t *bits, double band[3]);

/* The cone test for one pair (q, p), in units: 1 inside, 0 outside, -1 if
 * the request has no cone; *margin (optional) gets (a.r - c |r|) / |r|. */
int vo_fov_test(const vo_request *r, const int64_t q[3], const int64_t p[3], double *margin);

/* Visibility for n viewpoint indices on `threads` POSIX threads.
 * bits_out (optional) holds n * ceil(P/32) words.  Returns 0 or -1. */
int vo_run(const vo_scene *s, const vo_request *r, const int64_t *indices, int64_t n,
           double *v_out, uint32_t *bits_out, int threads);

/* The same, with band_out (optional) holding n * 3 doubles of
 * vo_visibility_ex's band output. */
int vo_run_ex(const vo_scene *s, const vo_request *r, const int64_t *indices, int64_t n,
              double *v_out, uint32_t *bits_out, double *band_out, int threads);

/* Largest value of v[0..n). */
double vo_max(const double *v, int64_t n);

/* color = 0 if v == 0 else 1 + min(L-2, floor((L-1) * v / v_ref)). */
int vo_quantise(const double *v, int64_t n, double v_ref, int levels, uint8_t *color_out);

#ifdef __cplusplus
}
#endif
#endif
