/*
 * Uniform-grid candidate cull for the synthetic hair-patch workload.
 *
 * This is input generation, not part of the intersection method: the paper
 * treats the top-level structure that finds candidate (ray, fiber) pairs as
 * orthogonal to the intersector (Sec. 2, last paragraph; Sec. 4).  Each
 * segment's control-hull AABB, dilated by its largest control radius, is
 * binned into a uniform grid; each ray walks the grid with a 3-D DDA
 * (Amanatides & Woo) and collects the de-duplicated ids of every segment
 * registered in the cells it crosses, in the order the walk first meets them
 * (front to back along the ray; by id within a cell).  The result is a CSR
 * list per ray.
 *
 * Host C only; the same source builds on x86-64 and aarch64.  Output does not
 * depend on the thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
    float lo[3], hi[3], cs[3];
    int n[3];
    int64_t ncell;
    int32_t *cell_ptr; /* ncell + 1 */
    int32_t *cell_seg;
} grid_t;

static void seg_aabb(const float *cp, float lo[3], float hi[3])
{
    float rmax = 0.f;
    for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int k = 0; k < 4; ++k) {
        for (int a = 0; a < 3; ++a) {
            float v = cp[4 * k + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
        if (cp[4 * k + 3] > rmax) rmax = cp[4 * k + 3];
    }
    for (int a = 0; a < 3; ++a) { lo[a] -= rmax; hi[a] += rmax; }
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

static int grid_build(grid_t *g, const float *cps, int64_t n_seg, int nx, int ny, int nz)
{
    g->n[0] = nx; g->n[1] = ny; g->n[2] = nz;
    for (int a = 0; a < 3; ++a) { g->lo[a] = INFINITY; g->hi[a] = -INFINITY; }
    for (int64_t s = 0; s < n_seg; ++s) {
        float lo[3], hi[3];
        seg_aabb(cps + 16 * s, lo, hi);
        for (int a = 0; a < 3; ++a) {
            if (lo[a] < g->lo[a]) g->lo[a] = lo[a];
            if (hi[a] > g->hi[a]) g->hi[a] = hi[a];
        }
    }
    for (int a = 0; a < 3; ++a) {
        float ext = g->hi[a] - g->lo[a];
        if (!(ext > 0.f)) ext = 1e-6f;
        g->hi[a] = g->lo[a] + ext;
        g->cs[a] = ext / (float)g->n[a];
    }
    g->ncell = (int64_t)nx * ny * nz;
    g->cell_ptr = (int32_t *)calloc((size_t)g->ncell + 1, sizeof(int32_t));
    if (!g->cell_ptr) return -1;
    int *box = (int *)malloc(sizeof(int) * 6 * (size_t)(n_seg > 0 ? n_seg : 1));
    if (!box) return -1;
    for (int64_t s = 0; s < n_seg; ++s) {
        float lo[3], hi[3];
        seg_aabb(cps + 16 * s, lo, hi);
        for (int a = 0; a < 3; ++a) {
            box[6 * s + a] = clampi((int)floorf((lo[a] - g->lo[a]) / g->cs[a]), 0, g->n[a] - 1);
            box[6 * s + 3 + a] = clampi((int)floorf((hi[a] - g->lo[a]) / g->cs[a]), 0, g->n[a] - 1);
        }
        for (int z = box[6 * s + 2]; z <= box[6 * s + 5]; ++z)
            for (int y = box[6 * s + 1]; y <= box[6 * s + 4]; ++y)
                for (int x = box[6 * s + 0]; x <= box[6 * s + 3]; ++x)
                    g->cell_ptr[((int64_t)z * ny + y) * nx + x + 1]++;
    }
    for (int64_t c = 0; c < g->ncell; ++c) g->cell_ptr[c + 1] += g->cell_ptr[c];
    int64_t total = g->cell_ptr[g->ncell];
    g->cell_seg = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
    int32_t *fill = (int32_t *)malloc(sizeof(int32_t) * (size_t)g->ncell);
    if (!g->cell_seg || !fill) { free(box); free(fill); return -1; }
    memcpy(fill, g->cell_ptr, sizeof(int32_t) * (size_t)g->ncell);
    for (int64_t s = 0; s < n_seg; ++s)
        for (int z = box[6 * s + 2]; z <= box[6 * s + 5]; ++z)
            for (int y = box[6 * s + 1]; y <= box[6 * s + 4]; ++y)
                for (int x = box[6 * s + 0]; x <= box[6 * s + 3]; ++x)
                    g->cell_seg[fill[((int64_t)z * ny + y) * nx + x]++] = (int32_t)s;
    free(fill);
    free(box);
    return 0;
}

/* Walks one ray through the grid; appends unseen segment ids to buf. */
static int64_t walk_ray(const grid_t *g, const float *ray, int32_t stamp_id, int32_t *stamp,
                        int32_t **buf, int64_t *cap)
{
    double o[3] = {ray[0], ray[1], ray[2]}, w[3] = {ray[4], ray[5], ray[6]};
    double tmax = ray[3];
    double t0 = 0.0, t1 = tmax;
    for (int a = 0; a < 3; ++a) {
        if (w[a] == 0.0) {
            if (o[a] < g->lo[a] || o[a] > g->hi[a]) return 0;
            continue;
        }
        double ta = (g->lo[a] - o[a]) / w[a], tb = (g->hi[a] - o[a]) / w[a];
        if (ta > tb) { double tt = ta; ta = tb; tb = tt; }
        if (ta > t0) t0 = ta;
        if (tb < t1) t1 = tb;
    }
    if (t0 > t1) return 0;
    int c[3], step[3];
    double tnext[3], tdelta[3];
    for (int a = 0; a < 3; ++a) {
        double pa = o[a] + t0 * w[a];
        c[a] = clampi((int)floor((pa - g->lo[a]) / g->cs[a]), 0, g->n[a] - 1);
        if (w[a] > 0.0) {
            step[a] = 1;
            tnext[a] = (g->lo[a] + (c[a] + 1) * (double)g->cs[a] - o[a]) / w[a];
            tdelta[a] = g->cs[a] / w[a];
        } else if (w[a] < 0.0) {
            step[a] = -1;
            tnext[a] = (g->lo[a] + c[a] * (double)g->cs[a] - o[a]) / w[a];
            tdelta[a] = -g->cs[a] / w[a];
        } else {
            step[a] = 0;
            tnext[a] = INFINITY;
            tdelta[a] = INFINITY;
        }
    }
    int64_t n = 0;
    for (;;) {
        int64_t cell = ((int64_t)c[2] * g->n[1] + c[1]) * g->n[0] + c[0];
        for (int32_t k = g->cell_ptr[cell]; k < g->cell_ptr[cell + 1]; ++k) {
            int32_t s = g->cell_seg[k];
            if (stamp[s] == stamp_id) continue;
            stamp[s] = stamp_id;
            if (n == *cap) {
                *cap *= 2;
                *buf = (int32_t *)realloc(*buf, sizeof(int32_t) * (size_t)*cap);
            }
            (*buf)[n++] = s;
        }
        int a = 0;
        if (tnext[1] < tnext[a]) a = 1;
        if (tnext[2] < tnext[a]) a = 2;
        if (tnext[a] > t1) break;
        c[a] += step[a];
        if (c[a] < 0 || c[a] >= g->n[a]) break;
        tnext[a] += tdelta[a];
    }
    return n;
}

/*
 * Counts (seg_idx == NULL) or fills the candidate CSR.
 * cps: n_seg x 4 x (x, y, z, r) float; rays: n_ray x 8 float {o, tmax, w, 0}.
 * row_ptr: n_ray + 1 entries, written in both passes.  Returns the number of
 * pairs, or -1 on allocation failure / -2 if cap is too small.
 */
int64_t gc_cull(const float *cps, int64_t n_seg, const float *rays, int64_t n_ray,
                int nx, int ny, int nz, int nthreads,
                int32_t *row_ptr, int32_t *seg_idx, int64_t cap)
{
    grid_t g;
    memset(&g, 0, sizeof(g));
    if (grid_build(&g, cps, n_seg, nx, ny, nz) != 0) return -1;
    int32_t *counts = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_ray > 0 ? n_ray : 1));
    int err = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
    if (!seg_idx) {
#pragma omp parallel
        {
            int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_seg > 0 ? n_seg : 1));
            int64_t bcap = 1024;
            int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)bcap);
            for (int64_t s = 0; s < n_seg; ++s) stamp[s] = -1;
#pragma omp for schedule(dynamic, 512)
            for (int64_t r = 0; r < n_ray; ++r)
                counts[r] = (int32_t)walk_ray(&g, rays + 8 * r, (int32_t)r, stamp, &buf, &bcap);
            free(stamp);
            free(buf);
        }
        row_ptr[0] = 0;
        int64_t acc = 0;
        for (int64_t r = 0; r < n_ray; ++r) {
            acc += counts[r];
            row_ptr[r + 1] = (int32_t)acc;
        }
    } else {
        if (row_ptr[n_ray] > cap) err = 1;
        if (!err) {
#pragma omp parallel
            {
                int32_t *stamp = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n_seg > 0 ? n_seg : 1));
                int64_t bcap = 1024;
                int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)bcap);
                for (int64_t s = 0; s < n_seg; ++s) stamp[s] = -1;
#pragma omp for schedule(dynamic, 512)
                for (int64_t r = 0; r < n_ray; ++r) {
                    int64_t n = walk_ray(&g, rays + 8 * r, (int32_t)r, stamp, &buf, &bcap);
                    memcpy(seg_idx + row_ptr[r], buf, sizeof(int32_t) * (size_t)n);
                }
                free(stamp);
                free(buf);
            }
        }
    }
    int64_t total = row_ptr[n_ray];
    free(counts);
    free(g.cell_ptr);
    free(g.cell_seg);
    return err ? -2 : total;
}
