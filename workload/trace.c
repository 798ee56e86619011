/*
 * Closest-hit ray casting against axis-aligned boxes, for the seeded
 * synthetic workloads.  This stands in for the hardware ray tracing of the
 * paper (Section 4: any caster that returns the hit point will do); it is
 * input generation, not part of the radiance-caching method, and both the
 * oracle and the CUDA path consume its output unchanged.
 *
 * Acceleration: a uniform grid over the scene bounds, traversed with a 3D
 * DDA (Amanatides & Woo 1987).  Arithmetic is plain IEEE float32; build with
 * -ffp-contract=off so x86 and Arm hosts produce the same bits.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef struct {
    float lo[3], cell, inv_cell;
    int dim[3];
    int *start; /* dim0*dim1*dim2 + 1 offsets into idx */
    int *idx;
} grid_t;

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static void grid_build(grid_t *g, const float *bmin, const float *bmax, int nb) {
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int b = 0; b < nb; ++b)
        for (int a = 0; a < 3; ++a) {
            if (bmin[3 * b + a] < lo[a]) lo[a] = bmin[3 * b + a];
            if (bmax[3 * b + a] > hi[a]) hi[a] = bmax[3 * b + a];
        }
    double ext[3], vol = 1.0;
    for (int a = 0; a < 3; ++a) {
        ext[a] = (double)hi[a] - (double)lo[a];
        if (ext[a] < 1e-3) ext[a] = 1e-3;
        vol *= ext[a];
    }
    double target = 4.0 * (double)(nb > 1 ? nb : 1);
    double cell = cbrt(vol / target);
    for (int a = 0; a < 3; ++a) {
        g->lo[a] = lo[a];
        int d = (int)ceil(ext[a] / cell);
        g->dim[a] = clampi(d, 1, 256);
    }
    /* one cubic cell size that covers every axis */
    double c = 0.0;
    for (int a = 0; a < 3; ++a) {
        double ca = ext[a] / g->dim[a];
        if (ca > c) c = ca;
    }
    g->cell = (float)(c * 1.0001);
    g->inv_cell = 1.0f / g->cell;
    int ncell = g->dim[0] * g->dim[1] * g->dim[2];
    g->start = (int *)calloc((size_t)ncell + 1, sizeof(int));
    /* count pass */
    for (int pass = 0; pass < 2; ++pass) {
        int *fill = NULL;
        if (pass == 1) {
            for (int i = 0; i < ncell; ++i) g->start[i + 1] += g->start[i];
            g->idx = (int *)malloc(sizeof(int) * (size_t)(g->start[ncell] > 0 ? g->start[ncell] : 1));
            fill = (int *)calloc((size_t)ncell, sizeof(int));
        }
        for (int b = 0; b < nb; ++b) {
            int c0[3], c1[3];
            for (int a = 0; a < 3; ++a) {
                c0[a] = clampi((int)floorf((bmin[3 * b + a] - g->lo[a]) * g->inv_cell), 0, g->dim[a] - 1);
                c1[a] = clampi((int)floorf((bmax[3 * b + a] - g->lo[a]) * g->inv_cell), 0, g->dim[a] - 1);
            }
            for (int z = c0[2]; z <= c1[2]; ++z)
                for (int y = c0[1]; y <= c1[1]; ++y)
                    for (int x = c0[0]; x <= c1[0]; ++x) {
                        int ci = (z * g->dim[1] + y) * g->dim[0] + x;
                        if (pass == 0)
                            g->start[ci + 1]++;
                        else
                            g->idx[g->start[ci] + fill[ci]++] = b;
                    }
        }
        free(fill);
    }
}

static void grid_free(grid_t *g) {
    free(g->start);
    free(g->idx);
}

/* Slab test.  Returns 1 and the entering distance/face when the ray enters the
 * box at t in (tmin, tmax]; a ray starting inside a box does not hit it. */
static int ray_box(const float *lo, const float *hi, const float o[3], const float inv[3],
                   float tmin, float tmax, float *t_hit, int *face) {
    float t0 = tmin, t1 = tmax;
    int f = -1;
    for (int a = 0; a < 3; ++a) {
        float ta = (lo[a] - o[a]) * inv[a];
        float tb = (hi[a] - o[a]) * inv[a];
        float tn, tf;
        int fn;
        if (inv[a] >= 0.0f) {
            tn = ta; tf = tb; fn = 2 * a + 0; /* enters through the min face: normal -e_a */
        } else {
            tn = tb; tf = ta; fn = 2 * a + 1; /* enters through the max face: normal +e_a */
        }
        if (tn > t0) { t0 = tn; f = fn; }
        if (tf < t1) t1 = tf;
        if (t0 > t1) return 0;
    }
    if (f < 0) return 0;
    *t_hit = t0;
    *face = f;
    return 1;
}

static void trace_one(const grid_t *g, const float *bmin, const float *bmax, const float o[3],
                      const float d_in[3], float tmax, float *t_out, int *box_out, int *face_out) {
    float d[3], inv[3];
    for (int a = 0; a < 3; ++a) {
        d[a] = d_in[a];
        if (d[a] == 0.0f) d[a] = signbit(d_in[a]) ? -1e-30f : 1e-30f;
        inv[a] = 1.0f / d[a];
    }
    /* clip the ray to the grid bounds */
    float t0 = 0.0f, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        float glo = g->lo[a], ghi = g->lo[a] + g->cell * (float)g->dim[a];
        float ta = (glo - o[a]) * inv[a], tb = (ghi - o[a]) * inv[a];
        float tn = ta < tb ? ta : tb, tf = ta < tb ? tb : ta;
        if (tn > t0) t0 = tn;
        if (tf < t1) t1 = tf;
    }
    *t_out = INFINITY;
    *box_out = -1;
    *face_out = -1;
    if (!(t0 <= t1)) return;
    int c[3], step[3];
    float tnext[3], tdelta[3];
    for (int a = 0; a < 3; ++a) {
        float p = o[a] + d[a] * t0;
        c[a] = clampi((int)floorf((p - g->lo[a]) * g->inv_cell), 0, g->dim[a] - 1);
        step[a] = d[a] >= 0.0f ? 1 : -1;
        float bound = g->lo[a] + g->cell * (float)(c[a] + (d[a] >= 0.0f ? 1 : 0));
        tnext[a] = (bound - o[a]) * inv[a];
        tdelta[a] = g->cell * fabsf(inv[a]);
    }
    float best = tmax;
    int best_box = -1, best_face = -1;
    for (;;) {
        int ci = (c[2] * g->dim[1] + c[1]) * g->dim[0] + c[0];
        for (int k = g->start[ci]; k < g->start[ci + 1]; ++k) {
            int b = g->idx[k];
            float th;
            int fh;
            if (ray_box(bmin + 3 * b, bmax + 3 * b, o, inv, 0.0f, best, &th, &fh)) {
                if (th < best || (th == best && b < best_box)) {
                    best = th; best_box = b; best_face = fh;
                }
            }
        }
        int ax = tnext[0] < tnext[1] ? (tnext[0] < tnext[2] ? 0 : 2) : (tnext[1] < tnext[2] ? 1 : 2);
        float texit = tnext[ax];
        if (best_box >= 0 && best <= texit) break;
        if (texit > t1) break;
        c[ax] += step[ax];
        if (c[ax] < 0 || c[ax] >= g->dim[ax]) break;
        tnext[ax] += tdelta[ax];
    }
    if (best_box >= 0) {
        *t_out = best;
        *box_out = best_box;
        *face_out = best_face;
    }
}

/*
 * Trace n rays (origins o[3n], unit directions d[3n]) against nb boxes.
 * Outputs per ray: hit distance (INFINITY on a miss), box index (-1 on a
 * miss) and entering face (2*axis + (1 if the normal is +e_axis)).
 */
int wl_trace(const float *bmin, const float *bmax, int nb, const float *o, const float *d, long n,
             float tmax, float *t_out, int *box_out, int *face_out, int nthreads) {
    if (nb <= 0 || n < 0) return -1;
    grid_t g;
    memset(&g, 0, sizeof g);
    grid_build(&g, bmin, bmax, nb);
#pragma omp parallel for schedule(dynamic, 4096) num_threads(nthreads)
    for (long i = 0; i < n; ++i)
        trace_one(&g, bmin, bmax, o + 3 * i, d + 3 * i, tmax, t_out + i, box_out + i, face_out + i);
    grid_free(&g);
    return 0;
}
