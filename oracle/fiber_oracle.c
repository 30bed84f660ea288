/*
 * fiber_oracle.c -- plain, slow FP64 reference of the ray / cubic-fiber
 * intersection of Binder & Keller, "Fast, High Precision Ray/Fiber
 * Intersection using Tight, Disjoint Bounding Volumes" (arXiv 1811.03374).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the package smoke check and
 * the CPU-baseline / reference leg of the benchmark may load this file.  It
 * shares no code, header, table or helper with the CUDA library and includes
 * nothing from it.
 *
 * Every function follows one passage of the paper, cited in its comment, and
 * is written in the paper's notation: control points p0..p3 with the radius as
 * fourth component (Sec. 3.3), the (p, d, t0, t1) representation and its
 * subdivision rules (Sec. 3.1), the partitioned bounding cylinder (Sec. 3.2,
 * Fig. 5), the unit-ray cylinder / plane tests (Sec. 3.3, App. A), the
 * bit-string traversal (Sec. 3.3) and the curve constraints (Sec. 3.4,
 * App. B.2).  Where the paper is silent or garbled, the reading taken is
 * stated at the place it is used.
 *
 * Parity of each exported function is pinned by the oracle test suite
 * (closed forms, brute force over leaves, golden values from the paper's
 * figures, invariants).  Precision: double throughout; u intervals are exact
 * dyadics start * 2^-23.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ROOT_SIZE (1u << 23) /* parametric domain [0,1] in units of 2^-23 */
#define U_UNIT (1.0 / 8388608.0)

typedef struct { double x, y, z, w; } v4;

/* (p, d, t0, t1): p = p0, d = p3 - p0, t0 = p1 - p0, t1 = p3 - p2 (Sec. 3.1) */
typedef struct { v4 p, d, t0, t1; } node_t;

typedef struct {
    double t, u;       /* distance along the unit ray, curve parameter */
    int32_t hit;       /* 1 if a hit closer than the ray's t_max was found */
    int32_t leaf;      /* start of the hit leaf in units of 2^-23 */
    int32_t nodes;     /* node (pruning) tests performed */
    int32_t descents;  /* partition + subdivide steps */
    int32_t backtracks;/* jump_up + recompute steps */
    int32_t pad;
} orc_hit;

/* ---------------------------------------------------------------- vectors */

static v4 V(double x, double y, double z, double w) { v4 r = {x, y, z, w}; return r; }
static v4 add4(v4 a, v4 b) { return V(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w); }
static v4 sub4(v4 a, v4 b) { return V(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w); }
static v4 mul4(double s, v4 a) { return V(s * a.x, s * a.y, s * a.z, s * a.w); }
static double dot3(v4 a, v4 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static double dmax(double a, double b) { return a > b ? a : b; }
static double dmin(double a, double b) { return a < b ? a : b; }

static v4 load_cp(const double *cp, int k) { return V(cp[4 * k], cp[4 * k + 1], cp[4 * k + 2], cp[4 * k + 3]); }

/* ------------------------------------------------------- Bezier evaluation */

/* Cubic Bezier point c(u) in Bernstein form (all four components). */
static v4 bez_eval(const v4 P[4], double u)
{
    double v = 1.0 - u;
    return add4(add4(mul4(v * v * v, P[0]), mul4(3.0 * u * v * v, P[1])),
                add4(mul4(3.0 * u * u * v, P[2]), mul4(u * u * u, P[3])));
}

/* c'(u) / 3: the scaled derivative the paper evaluates (App. C). */
static v4 bez_deriv3(const v4 P[4], double u)
{
    double v = 1.0 - u;
    return add4(add4(mul4(v * v, sub4(P[1], P[0])), mul4(2.0 * u * v, sub4(P[2], P[1]))),
                mul4(u * u, sub4(P[3], P[2])));
}

/* c''(u). */
static v4 bez_deriv2(const v4 P[4], double u)
{
    v4 a = sub4(add4(P[2], P[0]), mul4(2.0, P[1]));
    v4 b = sub4(add4(P[3], P[1]), mul4(2.0, P[2]));
    return mul4(6.0, add4(mul4(1.0 - u, a), mul4(u, b)));
}

/* ------------------------------------------------------------ ray frame */

/*
 * Orthonormal frame (e1, e2, w) around the unit direction w.  Sec. 3.3 uses
 * Duff et al.'s construction; any orthonormal completion gives the same
 * result, because every quantity the method uses (a_x p_y - a_y p_x,
 * a_x^2 + a_y^2, dot products, z components) is invariant under rotation
 * about the ray.  This one is Gram-Schmidt against the least aligned axis.
 */
static void ray_frame(const double w[3], double e1[3], double e2[3])
{
    double a[3] = {0.0, 0.0, 0.0};
    double ax = fabs(w[0]), ay = fabs(w[1]), az = fabs(w[2]);
    if (ax <= ay && ax <= az) a[0] = 1.0;
    else if (ay <= az) a[1] = 1.0;
    else a[2] = 1.0;
    double k = a[0] * w[0] + a[1] * w[1] + a[2] * w[2];
    double q[3] = {a[0] - k * w[0], a[1] - k * w[1], a[2] - k * w[2]};
    double n = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    for (int i = 0; i < 3; ++i) e1[i] = q[i] / n;
    e2[0] = w[1] * e1[2] - w[2] * e1[1];
    e2[1] = w[2] * e1[0] - w[0] * e1[2];
    e2[2] = w[0] * e1[1] - w[1] * e1[0];
}

typedef struct { double o[3], w[3], e1[3], e2[3], tmax; } ray_t;

/* Ray from 8 floats {o, t_max, w, 0}; the direction is normalised (unit ray, Sec. 3.3). */
static ray_t make_ray_f(const float *r8)
{
    ray_t r;
    double n = sqrt((double)r8[4] * r8[4] + (double)r8[5] * r8[5] + (double)r8[6] * r8[6]);
    for (int i = 0; i < 3; ++i) { r.o[i] = r8[i]; r.w[i] = r8[4 + i] / n; }
    r.tmax = r8[3];
    ray_frame(r.w, r.e1, r.e2);
    return r;
}

static ray_t make_ray_d(const double *r7)
{
    ray_t r;
    double n = sqrt(r7[3] * r7[3] + r7[4] * r7[4] + r7[5] * r7[5]);
    for (int i = 0; i < 3; ++i) { r.o[i] = r7[i]; r.w[i] = r7[3 + i] / n; }
    r.tmax = r7[6];
    ray_frame(r.w, r.e1, r.e2);
    return r;
}

/* Control points in the ray-centric frame: the ray starts at the origin and
 * runs along +z; the radius is carried unchanged (Sec. 3.3). */
static void to_ray_frame(const ray_t *r, const double *cp, v4 Q[4])
{
    for (int k = 0; k < 4; ++k) {
        double q[3] = {cp[4 * k] - r->o[0], cp[4 * k + 1] - r->o[1], cp[4 * k + 2] - r->o[2]};
        Q[k].x = q[0] * r->e1[0] + q[1] * r->e1[1] + q[2] * r->e1[2];
        Q[k].y = q[0] * r->e2[0] + q[1] * r->e2[1] + q[2] * r->e2[2];
        Q[k].z = q[0] * r->w[0] + q[1] * r->w[1] + q[2] * r->w[2];
        Q[k].w = cp[4 * k + 3];
    }
}

/* ---------------------------------------------------------- primitives */

/* Unit ray against the plane through p with normal n: t = <n, p> / n_z
 * (Sec. 3.3).  Returns 0 when n_z == 0 (plane parallel to the ray). */
static int plane_t(v4 p, v4 n, double *t)
{
    if (n.z == 0.0) return 0;
    *t = dot3(n, p) / n.z;
    return 1;
}

/*
 * Unit ray against the infinite cylinder of radius r through p along a
 * (App. A): g = a_x^2 + a_y^2, squared distance (a_x p_y - a_y p_x)^2 / g,
 * t_cpa = p_z - a_z (a_x p_x + a_y p_y) / g, s = sqrt((r^2 - d^2)(a_z^2 + g) / g),
 * hits at t_cpa -+ s.  Axis parallel to the ray (g == 0): inside gives
 * (-inf, +inf), outside is a miss.  Returns 0 on a miss.
 */
static int cylinder(v4 p, v4 a, double r, double *c0, double *c1)
{
    double g = a.x * a.x + a.y * a.y;
    if (g == 0.0) {
        if (p.x * p.x + p.y * p.y < r * r) { *c0 = -INFINITY; *c1 = INFINITY; return 1; }
        return 0;
    }
    double cr = a.x * p.y - a.y * p.x;
    double e = r * r - cr * cr / g;
    if (e < 0.0) return 0;
    double tcpa = p.z - a.z * (a.x * p.x + a.y * p.y) / g;
    double s = sqrt(e * (a.z * a.z + g) / g);
    *c0 = tcpa - s;
    *c1 = tcpa + s;
    return 1;
}

/*
 * Conservative radius of the bounding cylinder along (p, p + d): the larger
 * distance of the two inner control points from the axis plus the largest
 * control radius (Sec. 3.3, convex hull property).  Inner points relative to p
 * are t0 and d - t1, whose distances from the axis equal those of t0 and t1.
 * Zero-length axis: distance from p (reading).
 */
static double cons_radius(const node_t *c)
{
    double dd = dot3(c->d, c->d), m;
    if (dd > 0.0) {
        double b0 = dot3(c->t0, c->d) / dd, b1 = dot3(c->t1, c->d) / dd;
        v4 q0 = sub4(c->t0, mul4(b0, c->d)), q1 = sub4(c->t1, mul4(b1, c->d));
        m = dmax(dot3(q0, q0), dot3(q1, q1));
    } else {
        m = dmax(dot3(c->t0, c->t0), dot3(c->t1, c->t1));
    }
    /* radii of the control points: r0 = p.w, r1 = p.w + t0.w, r3 = p.w + d.w,
       r2 = r3 - t1.w */
    double rmax = c->p.w + dmax(dmax(0.0, c->t0.w), dmax(c->d.w, c->d.w - c->t1.w));
    return sqrt(m) + rmax;
}

/*
 * t-interval of the region between the cropping planes: the start plane
 * through p with normal t0 (kept side <x - p, t0> >= 0) and the end plane
 * through p + d with normal t1 (kept side <x - p - d, t1> <= 0), clipped to
 * [0, ray_tmax] (Sec. 3.3).  A plane parallel to the ray either leaves the
 * interval alone or, if the ray lies on its excluded side, empties it.
 * Returns 0 for an empty interval.
 */
static int slab(const node_t *c, double ray_tmax, double *tmin, double *tmax)
{
    double lo = 0.0, hi = ray_tmax, t;
    if (plane_t(c->p, c->t0, &t)) {
        if (c->t0.z > 0.0) lo = dmax(lo, t);
        else hi = dmin(hi, t);
    } else if (-dot3(c->p, c->t0) < 0.0) {
        lo = INFINITY;
    }
    v4 q = add4(c->p, c->d);
    if (plane_t(q, c->t1, &t)) {
        if (c->t1.z < 0.0) lo = dmax(lo, t);
        else hi = dmin(hi, t);
    } else if (-dot3(q, c->t1) > 0.0) {
        lo = INFINITY;
    }
    *tmin = lo;
    *tmax = hi;
    return lo <= hi;
}

/* Subdivision of (p, d, t0, t1) at the domain centre (Sec. 3.1):
 * dp = 3/8 t0 + 1/2 d - 3/8 t1, tc = -1/8 t0 + 1/4 d - 1/8 t1;
 * left = (p, dp, t0/2, tc), right = (p + dp, d - dp, tc, t1/2). */
static void split_terms(const node_t *c, v4 *dp, v4 *tc)
{
    *dp = add4(add4(mul4(0.375, c->t0), mul4(0.5, c->d)), mul4(-0.375, c->t1));
    *tc = add4(add4(mul4(-0.125, c->t0), mul4(0.25, c->d)), mul4(-0.125, c->t1));
}

static void subdivide(node_t *c, int go_right, v4 dp, v4 tc)
{
    if (go_right) {
        c->p = add4(c->p, dp);
        c->d = sub4(c->d, dp);
        c->t0 = tc;
        c->t1 = mul4(0.5, c->t1);
    } else {
        c->d = dp;
        c->t0 = mul4(0.5, c->t0);
        c->t1 = tc;
    }
}

/* Node of the sub-interval [u0, u1] (start, size in units of 2^-23),
 * recomputed from the curve after backtracking (Sec. 3.3):
 * p = c(u0), d = c(u1) - c(u0), t0,1 = (u1 - u0) c'(u0,1) / 3. */
static void node_at(const v4 Q[4], uint32_t start, uint32_t size, node_t *c)
{
    double u0 = start * U_UNIT, u1 = (double)(start + size) * U_UNIT;
    v4 a = bez_eval(Q, u0), b = bez_eval(Q, u1);
    c->p = a;
    c->d = sub4(b, a);
    c->t0 = mul4(u1 - u0, bez_deriv3(Q, u0));
    c->t1 = mul4(u1 - u0, bez_deriv3(Q, u1));
}

/* Conversion {p0, p1, p2, p3} -> {p, d, t0, t1} (Sec. 3.1). */
static void node_of_points(const v4 Q[4], node_t *c)
{
    c->p = Q[0];
    c->d = sub4(Q[3], Q[0]);
    c->t0 = sub4(Q[1], Q[0]);
    c->t1 = sub4(Q[3], Q[2]);
}

/* ------------------------------------------------ FP32-band probe */

/*
 * Decisions within the FP32 band (used only by orc_ray_counts_amb; the
 * traversal's own decisions are unchanged).  A decision is "in the band" of
 * a ray when moving the ray sideways by up to delta could flip it: each probe
 * below re-evaluates a decision with the node translated in the ray frame by
 * delta in 8 directions of the xy plane (a sideways shift of the ray by
 * delta is a shift of everything else by -delta), or compares the margin of
 * a comparison along the ray with delta.  The first such decision of a ray
 * sets its flag.  NULL context: no probing.
 */
typedef struct { double delta; int amb; } probe_t;
static _Thread_local probe_t *g_probe = NULL;

static node_t shifted(const node_t *c, double dx, double dy)
{
    node_t s = *c;
    s.p.x -= dx;
    s.p.y -= dy;
    return s;
}

/* A cylinder node test (Sec. 3.2): the overlap decision with the inherited
 * interval [tmin, tmax], moved by how far the node's own cropping planes move,
 * and, for an inner node that is hit, the partition decisions (near child,
 * both children). */
static void probe_node(const node_t *c, double tmin, double tmax, double ray_tmax, int over, int leaf)
{
    if (!g_probe || g_probe->amb) return;
    double dl = g_probe->delta, r = cons_radius(c), lo0, hi0, c0 = 0, c1 = 0, tp0 = 0;
    slab(c, ray_tmax, &lo0, &hi0);
    int gr0 = 0, both0 = 0;
    v4 dp, tc;
    split_terms(c, &dp, &tc);
    if (over && !leaf) {
        cylinder(c->p, c->d, r, &c0, &c1);
        if (plane_t(add4(c->p, dp), tc, &tp0)) {
            gr0 = (tp0 > c0) != (tc.z > 0.0);
            both0 = (c0 < tp0) && (c1 > tp0);
        } else {
            gr0 = -dot3(add4(c->p, dp), tc) >= 0.0;
        }
    }
    for (int k = 0; k < 8; ++k) {
        double a = k * (3.14159265358979323846 / 4.0);
        node_t s = shifted(c, dl * cos(a), dl * sin(a));
        double lo, hi, s0, s1;
        slab(&s, ray_tmax, &lo, &hi);
        double ilo = tmin + ((isfinite(lo) && isfinite(lo0)) ? lo - lo0 : 0.0);
        double ihi = tmax + ((isfinite(hi) && isfinite(hi0)) ? hi - hi0 : 0.0);
        int ov = cylinder(s.p, s.d, r, &s0, &s1) && dmax(s0, ilo) <= dmin(s1, ihi);
        if (ov != over) { g_probe->amb = 1; return; }
        /* the interval's far end is the closest hit so far (the t_max of the
           search), itself a result of earlier tests: the overlap is in the
           band when its margin against that bound is within delta */
        if (ov && ihi >= ray_tmax && isfinite(ray_tmax) && dmin(s1, ihi) - dmax(s0, ilo) <= dl) {
            g_probe->amb = 1;
            return;
        }
        if (over && !leaf) {
            double tp;
            int gr, both = 0;
            if (plane_t(add4(s.p, dp), tc, &tp)) {
                gr = (tp > s0) != (tc.z > 0.0);
                both = (s0 < tp) && (s1 > tp);
            } else {
                gr = -dot3(add4(s.p, dp), tc) >= 0.0;
            }
            if (gr != gr0 || both != both0) { g_probe->amb = 1; return; }
        }
    }
}

/* A comparison of two distances along the ray (a hit against the closest so
 * far, two boxes' near ends): in the band when they are within delta. */
static void probe_order(double a, double b)
{
    if (!g_probe || g_probe->amb || !isfinite(a) || !isfinite(b)) return;
    if (fabs(a - b) <= g_probe->delta) g_probe->amb = 1;
}

/* ----------------------------------------------------------- traversal */

/*
 * Closest hit of a unit ray with one curve (Sec. 3, Sec. 3.2-3.3, the
 * iterative routine of App. C), curve already in the ray frame.
 *
 * State: the current node, its t-interval [tmin, tmax], the bit string (one
 * bit per level, set iff both children must be visited), and the integer
 * interval (start, size).  Each step tests the node's bounding cylinder
 * against the interval:
 *   - overlap and size <= min_size: leaf; the hit is the entry into the
 *     capped leaf cylinder, max(c0, tmin); stop (immediate
 *     termination, Sec. 3.2);
 *   - overlap otherwise: partition by the plane through the split point with
 *     normal tc, continue with the child the ray reaches first, tighten one
 *     bound of the interval, set the bit if the ray crosses the plane inside
 *     the cylinder (Sec. 3.2, Fig. 5);
 *   - no overlap: if no bit is set, stop; otherwise jump to the sibling at the
 *     deepest set bit and recompute its node and interval.
 * Overlap means the cylinder is hit and max(c0, tmin) <= min(c1, tmax): the
 * listing's comparisons plus non-emptiness of both intervals.
 */
static void traverse(const v4 Q[4], int depth, double ray_tmax, orc_hit *h)
{
    node_t c;
    node_of_points(Q, &c);
    uint32_t bits = 0, size = ROOT_SIZE, start = 0;
    uint32_t min_size = ROOT_SIZE >> depth;
    double tmin, tmax, t = INFINITY;
    int hit = 0;
    slab(&c, ray_tmax, &tmin, &tmax);
    h->nodes = h->descents = h->backtracks = 0;
    for (;;) {
        double r = cons_radius(&c), c0 = 0.0, c1 = 0.0;
        h->nodes++;
        int over = cylinder(c.p, c.d, r, &c0, &c1) && dmax(c0, tmin) <= dmin(c1, tmax);
        probe_node(&c, tmin, tmax, ray_tmax, over, size <= min_size);
        if (over) {
            if (size <= min_size) {
                t = dmax(c0, tmin);
                hit = 1;
                break;
            }
            v4 dp, tc;
            split_terms(&c, &dp, &tc);
            v4 s = add4(c.p, dp);
            double tp;
            int go_right, both;
            if (plane_t(s, tc, &tp)) {
                go_right = (tp > c0) != (tc.z > 0.0);
                both = (c0 < tp) && (c1 > tp);
                if (tp > c0) tmax = dmin(tmax, tp);
                else tmin = dmax(tmin, tp);
            } else {
                /* plane parallel to the ray: the ray stays on the origin's side */
                go_right = -dot3(s, tc) >= 0.0;
                both = 0;
            }
            subdivide(&c, go_right, dp, tc);
            size >>= 1;
            if (both) bits ^= size;
            if (go_right) start ^= size;
            h->descents++;
        } else {
            if (!bits) break;
            size = bits & (~bits + 1u); /* lowest set bit: deepest pending level */
            start ^= size;
            bits ^= size;
            start &= ~(size - 1u);
            node_at(Q, start, size, &c);
            slab(&c, ray_tmax, &tmin, &tmax);
            h->backtracks++;
        }
    }
    h->hit = 0;
    h->t = INFINITY;
    h->u = -1.0;
    h->leaf = -1;
    if (hit && t < ray_tmax) {
        /* u: projection of the hit point onto the leaf axis (App. C) */
        double dd = dot3(c.d, c.d);
        double ul = 0.0;
        if (dd > 0.0) {
            v4 hb = V(-c.p.x, -c.p.y, t - c.p.z, 0.0);
            ul = dot3(hb, c.d) / dd;
            ul = dmax(0.0, dmin(1.0, ul));
        }
        double u0 = start * U_UNIT, u1 = (double)(start + size) * U_UNIT;
        h->hit = 1;
        h->t = t;
        h->u = u0 + ul * (u1 - u0);
        h->leaf = (int32_t)start;
    }
}

/* ------------------------------------------------- curve constraints */

/* The five inequalities of Sec. 3.4 / App. B.2 on the positions. */
int orc_valid_cubic(const double *cp)
{
    v4 P[4];
    for (int k = 0; k < 4; ++k) P[k] = load_cp(cp, k);
    v4 p20 = sub4(P[2], P[0]), p10 = sub4(P[1], P[0]), p31 = sub4(P[3], P[1]), p32 = sub4(P[3], P[2]);
    return dot3(p20, p10) >= 0.0 && dot3(p31, p10) >= 0.0 && dot3(p31, p32) >= 0.0 &&
           dot3(p20, p32) >= 0.0 && dot3(p20, p31) >= 0.0;
}

static double norm3(v4 a) { return sqrt(dot3(a, a)); }

/* ------------------------------------------- polynomials on [0, 1] */

#define PMAX 11 /* degree <= 10 */
typedef struct { double a[PMAX]; int n; } poly_t; /* power basis, a[k] u^k */

static poly_t pz(int n) { poly_t p; memset(&p, 0, sizeof p); p.n = n; return p; }

static poly_t padd(poly_t x, poly_t y, double sy)
{
    poly_t r = pz(x.n > y.n ? x.n : y.n);
    for (int k = 0; k <= x.n; ++k) r.a[k] += x.a[k];
    for (int k = 0; k <= y.n; ++k) r.a[k] += sy * y.a[k];
    return r;
}

static poly_t pmul(poly_t x, poly_t y)
{
    poly_t r = pz(x.n + y.n);
    for (int i = 0; i <= x.n; ++i)
        for (int j = 0; j <= y.n; ++j) r.a[i + j] += x.a[i] * y.a[j];
    return r;
}

/* x / (u - root), x having that root (the remainder is dropped) */
static poly_t pdiv_root(poly_t x, double root)
{
    poly_t q = pz(x.n - 1);
    double c = x.a[x.n];
    for (int k = x.n - 1; k >= 0; --k) {
        q.a[k] = c;
        c = x.a[k] + root * c;
    }
    return q;
}

/*
 * x >= 0 on [0, 1].  In the Bernstein basis of degree n on an interval,
 * b_k = sum_{i <= k} C(k, i) / C(n, i) a_i on [0, 1]; the polynomial lies
 * between the smallest and largest b_k, and b_0, b_n are its end values.  So
 * all b_k >= 0 proves x >= 0, a negative end value disproves it, and
 * otherwise the interval is halved (de Casteljau) and both halves checked.
 * Values within 1e-12 of the largest coefficient count as zero (FP64
 * rounding of the coefficients); 40 halvings without a decision count as a
 * violation.
 */
static int bern_nonneg(const double *b, int n, double tol, int depth)
{
    if (b[0] < -tol || b[n] < -tol) return 0;
    int all = 1;
    for (int k = 0; k <= n; ++k) all &= b[k] >= -tol;
    if (all) return 1;
    if (depth >= 40) return 0;
    double w[PMAX], L[PMAX], R[PMAX];
    for (int k = 0; k <= n; ++k) w[k] = b[k];
    for (int lvl = 0; lvl <= n; ++lvl) {
        L[lvl] = w[0];
        R[n - lvl] = w[n - lvl];
        for (int k = 0; k < n - lvl; ++k) w[k] = 0.5 * (w[k] + w[k + 1]);
    }
    return bern_nonneg(L, n, tol, depth + 1) && bern_nonneg(R, n, tol, depth + 1);
}

static double binom(int n, int k)
{
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (n - k + i) / i;
    return r;
}

static int nonneg01(poly_t x)
{
    double b[PMAX], m = 0.0;
    for (int k = 0; k <= x.n; ++k) {
        b[k] = 0.0;
        for (int i = 0; i <= k; ++i) b[k] += binom(k, i) / binom(x.n, i) * x.a[i];
        m = dmax(m, fabs(b[k]));
    }
    return bern_nonneg(b, x.n, 1e-12 * m, 0);
}

/*
 * The end-plane condition for thick fibers (Sec. 3.4, Fig. 7): the surface
 * point of the cross-section at u that comes closest to the end plane
 * through p3 with normal n1 = p3 - p2 lies r sin(theta(u)) beyond c(u)
 * towards it, theta(u) the angle between c'(u) and n1 (the Gram-Schmidt
 * displacement of the paper); with rbar the largest control radius the
 * fiber is not cropped when <p3 - c(u), n1> / |n1| >= rbar sin(theta(u))
 * for all u in [0, 1].  With t = c' / 3 and D1 = <p3 - c, n1> this is
 * D1 >= 0 and D1^2 |t|^2 - rbar^2 |n1 x t|^2 >= 0 (both sides multiplied by
 * |n1| |t|), polynomials of degree 3 and 10 in u with a simple and a double
 * root at u = 1, where the fiber meets its own end plane; divided by them,
 * both must be non-negative on [0, 1] (at u = 1 the second reduces to
 * rbar * curvature <= 1).  The start plane through p0 with normal p1 - p0
 * likewise, roots at u = 0.  The paper speaks of a quartic; these are the
 * same conditions, checked exactly on the polynomials.
 * Returns 1 if neither end plane crops the fiber.
 */
int orc_thick_ok(const double *cp)
{
    v4 P[4];
    double rbar = 0.0;
    for (int k = 0; k < 4; ++k) {
        P[k] = load_cp(cp, k);
        rbar = dmax(rbar, P[k].w);
    }
    double pc[3][4];
    for (int j = 0; j < 3; ++j) {
        double p0 = (&P[0].x)[j], p1 = (&P[1].x)[j], p2 = (&P[2].x)[j], p3 = (&P[3].x)[j];
        pc[j][0] = p0;
        pc[j][1] = 3.0 * (p1 - p0);
        pc[j][2] = 3.0 * (p0 - 2.0 * p1 + p2);
        pc[j][3] = p3 - 3.0 * p2 + 3.0 * p1 - p0;
    }
    poly_t c[3], t[3];
    for (int j = 0; j < 3; ++j) {
        c[j] = pz(3);
        for (int k = 0; k < 4; ++k) c[j].a[k] = pc[j][k];
        t[j] = pz(2);
        for (int k = 0; k < 3; ++k) t[j].a[k] = (k + 1) * pc[j][k + 1] / 3.0;
    }
    poly_t T = pz(0);
    for (int j = 0; j < 3; ++j) T = padd(T, pmul(t[j], t[j]), 1.0);
    v4 nrm[2] = {sub4(P[1], P[0]), sub4(P[3], P[2])};
    for (int e = 0; e < 2; ++e) {
        v4 n = nrm[e];
        double nn = dot3(n, n);
        if (!(nn > 0.0)) return 0;
        poly_t D = pz(0), G = pz(0);
        for (int j = 0; j < 3; ++j) {
            double nj = (&n.x)[j];
            poly_t cj = c[j];
            if (e == 1) { /* <p3 - c, n1> */
                for (int k = 0; k <= 3; ++k) cj.a[k] = -cj.a[k];
                cj.a[0] += (&P[3].x)[j];
            } else {      /* <c - p0, n0> */
                cj.a[0] -= (&P[0].x)[j];
            }
            poly_t sj = pz(0); sj.a[0] = nj;
            D = padd(D, pmul(sj, cj), 1.0);
            G = padd(G, pmul(sj, t[j]), 1.0);
        }
        poly_t X = padd(T, pmul(G, G), -1.0 / nn);
        for (int k = 0; k <= X.n; ++k) X.a[k] *= nn; /* |n|^2 T - <n, t>^2 = |n x t|^2 */
        poly_t Pq = padd(pmul(pmul(D, D), T), X, -rbar * rbar);
        double root = e == 1 ? 1.0 : 0.0;
        poly_t E = pdiv_root(D, root);
        if (e == 1) for (int k = 0; k <= E.n; ++k) E.a[k] = -E.a[k]; /* D1 = (1 - u) E */
        poly_t Q = pdiv_root(pdiv_root(Pq, root), root);
        if (!nonneg01(E) || !nonneg01(Q)) return 0;
    }
    return 1;
}

/* De Casteljau halving at u = 1/2, all four components (App. B.2). */
void orc_split_half(const double *cp, double *L, double *R)
{
    for (int a = 0; a < 4; ++a) {
        double p0 = cp[a], p1 = cp[4 + a], p2 = cp[8 + a], p3 = cp[12 + a];
        double p01 = 0.5 * (p0 + p1), p12 = 0.5 * (p1 + p2), p23 = 0.5 * (p2 + p3);
        double p012 = 0.5 * (p01 + p12), p123 = 0.5 * (p12 + p23);
        double s = 0.5 * (p012 + p123);
        L[a] = p0; L[4 + a] = p01; L[8 + a] = p012; L[12 + a] = s;
        R[a] = s; R[4 + a] = p123; R[8 + a] = p23; R[12 + a] = p3;
    }
}

/*
 * Pre-split (Sec. 3.4: a curve violating the constraints has to be split before it
 * is traversed): a curve failing the constraints or the
 * thick-fiber check is halved at u = 1/2, recursively, left before right, up
 * to max_level levels.  A piece still failing at max_level is kept and
 * flagged unsupported (flag bit 0).
 */
typedef struct {
    double *cp;
    int32_t *seg, *level, *off, *flags;
    int64_t n, cap;
} piece_out;

static void presplit_rec(const double *cp, int32_t seg, int level, int32_t off, int max_level,
                         int thick, piece_out *o)
{
    int ok = orc_valid_cubic(cp) && (!thick || orc_thick_ok(cp));
    if (ok || level >= max_level) {
        if (o->n < o->cap) {
            memcpy(o->cp + 16 * o->n, cp, 16 * sizeof(double));
            o->seg[o->n] = seg;
            o->level[o->n] = level;
            o->off[o->n] = off;
            o->flags[o->n] = ok ? 0 : 1;
        }
        o->n++;
        return;
    }
    double L[16], R[16];
    orc_split_half(cp, L, R);
    presplit_rec(L, seg, level + 1, 2 * off, max_level, thick, o);
    presplit_rec(R, seg, level + 1, 2 * off + 1, max_level, thick, o);
}

/* cps: n_seg x 16 floats.  Returns the number of pieces (written if <= cap). */
int64_t orc_presplit(const float *cps, int64_t n_seg, int max_level, int thick, double *piece_cp,
                     int32_t *piece_seg, int32_t *piece_level, int32_t *piece_off,
                     int32_t *piece_flags, int64_t cap)
{
    piece_out o = {piece_cp, piece_seg, piece_level, piece_off, piece_flags, 0, cap};
    for (int64_t s = 0; s < n_seg; ++s) {
        double cp[16];
        for (int i = 0; i < 16; ++i) cp[i] = cps[16 * s + i];
        presplit_rec(cp, (int32_t)s, 0, 0, max_level, thick, &o);
    }
    return o.n;
}

/* The same for control points given in double precision. */
int64_t orc_presplit_d(const double *cps, int64_t n_seg, int max_level, int thick, double *piece_cp,
                       int32_t *piece_seg, int32_t *piece_level, int32_t *piece_off,
                       int32_t *piece_flags, int64_t cap)
{
    piece_out o = {piece_cp, piece_seg, piece_level, piece_off, piece_flags, 0, cap};
    for (int64_t s = 0; s < n_seg; ++s)
        presplit_rec(cps + 16 * s, (int32_t)s, 0, 0, max_level, thick, &o);
    return o.n;
}

/* ---------------------------------------------- pruning-test statistics */

/*
 * Fig. 8 compares the number of pruning tests of the oriented bounding
 * cylinders with axis-aligned boxes in the ray's frame (the
 * boxes in Duff et al.'s frame, below).  Per
 * ray, each candidate is searched in row order with the closest hit so far
 * as t_max, with no test before the root's, so that only the bounding volume
 * differs:
 *   - cylinders: the traversal of Sec. 3.3 (one test per node visited);
 *   - boxes: the same subdivision without partition planes.  A node's box is
 *     [min_k (q_k - r_k), max_k (q_k + r_k)] over its four control points q_k
 *     and radii r_k (the tube lies in the hull of the control spheres); it is
 *     hit if it contains the ray's axis (x = y = 0) and meets [0, t_max] in
 *     z.  At a hit inner node both children's boxes are tested, the one with
 *     the smaller z_min (the left one on a tie) is searched first, and the
 *     other is tested again when taken up; without disjoint volumes the
 *     search does not end at the first leaf hit.  A leaf whose box is hit
 *     takes the leaf test of Sec. 3.3 (capped cylinder), which finds the
 *     hits.
 * Returns the number of bounding-volume tests (boxes) in *count.
 */
static int piece_depth(int depth, int level);

/*
 * A box aligned to the ray's frame depends on the frame's rotation about the
 * ray (the cylinder test does not).  The boxes use the frame Sec. 3.3 cites,
 * Duff et al.'s orthonormal basis ("Building an orthonormal basis,
 * revisited", 2017): with s = sign(w_z), a = -1 / (s + w_z), b = w_x w_y a,
 * e1 = (1 + s w_x^2 a, s b, -s w_x), e2 = (b, s + w_y^2 a, -w_y).
 */
static void duff_frame(const double w[3], double e1[3], double e2[3])
{
    double s = copysign(1.0, w[2]);
    double a = -1.0 / (s + w[2]);
    double b = w[0] * w[1] * a;
    e1[0] = 1.0 + s * w[0] * w[0] * a; e1[1] = s * b; e1[2] = -s * w[0];
    e2[0] = b; e2[1] = s + w[1] * w[1] * a; e2[2] = -w[1];
}

static void node_points(const node_t *c, v4 q[4])
{
    q[0] = c->p;
    q[1] = add4(c->p, c->t0);
    q[2] = sub4(add4(c->p, c->d), c->t1);
    q[3] = add4(c->p, c->d);
}

static int box_hit(const node_t *c, double tmax)
{
    v4 q[4];
    node_points(c, q);
    double lo[3], hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int k = 0; k < 4; ++k) {
        double v[3] = {q[k].x, q[k].y, q[k].z};
        for (int a = 0; a < 3; ++a) {
            lo[a] = dmin(lo[a], v[a] - q[k].w);
            hi[a] = dmax(hi[a], v[a] + q[k].w);
        }
    }
    if (g_probe && !g_probe->amb) {  /* a face of the box within delta of the ray */
        double dl = g_probe->delta;
        if (fabs(lo[0]) <= dl || fabs(hi[0]) <= dl || fabs(lo[1]) <= dl || fabs(hi[1]) <= dl ||
            fabs(hi[2]) <= dl)
            g_probe->amb = 1;
        probe_order(lo[2], tmax);
    }
    return lo[0] <= 0.0 && hi[0] >= 0.0 && lo[1] <= 0.0 && hi[1] >= 0.0 && hi[2] >= 0.0 && lo[2] <= tmax;
}

static double box_zmin(const node_t *c)
{
    v4 q[4];
    node_points(c, q);
    double z = INFINITY;
    for (int k = 0; k < 4; ++k) z = dmin(z, q[k].z - q[k].w);
    return z;
}

/* The leaf test of the traversal: capped leaf cylinder, entry max(c0, tmin). */
static int leaf_test(const node_t *c, double tmax, double *t)
{
    double tmin, tm, c0, c1;
    slab(c, tmax, &tmin, &tm);
    double r = cons_radius(c);
    int over = cylinder(c->p, c->d, r, &c0, &c1) && dmax(c0, tmin) <= dmin(c1, tm);
    probe_node(c, tmin, tm, tmax, over, 1);
    if (!over) return 0;
    *t = dmax(c0, tmin);
    return *t < tmax;
}

static void box_visit(const node_t *c, uint32_t size, uint32_t min_size, double *best, int64_t *count)
{
    if (size <= min_size) {
        double t;
        if (leaf_test(c, *best, &t)) *best = t;
        return;
    }
    v4 dp, tc;
    split_terms(c, &dp, &tc);
    node_t L = *c, R = *c;
    subdivide(&L, 0, dp, tc);
    subdivide(&R, 1, dp, tc);
    *count += 2;
    int hl = box_hit(&L, *best), hr = box_hit(&R, *best);
    if (hl && hr) {
        int right_first = box_zmin(&R) < box_zmin(&L);
        probe_order(box_zmin(&R), box_zmin(&L));
        const node_t *a = right_first ? &R : &L, *b = right_first ? &L : &R;
        box_visit(a, size >> 1, min_size, best, count);
        *count += 1;
        if (box_hit(b, *best)) box_visit(b, size >> 1, min_size, best, count);
    } else if (hl) {
        box_visit(&L, size >> 1, min_size, best, count);
    } else if (hr) {
        box_visit(&R, size >> 1, min_size, best, count);
    }
}

/* One curve (ray frame) with t_max: box-pruned search, tests and closest t. */
static double box_search(const v4 Q[4], int depth, double tmax, int64_t *count)
{
    node_t c;
    node_of_points(Q, &c);
    double best = tmax;
    *count += 1;
    if (box_hit(&c, best)) box_visit(&c, ROOT_SIZE, ROOT_SIZE >> depth, &best, count);
    return best;
}

/*
 * Per ray: pruning tests of its candidates searched in row order with the
 * closest hit so far as t_max; mode 0 cylinders (node tests of the
 * traversal), mode 1 boxes.  counts: n_ray int64; t_out (nullable): the
 * closest hit found (inf on a miss).
 */
static void ray_counts_impl(const float *rays_f, const double *rays_d, int64_t n_ray, const int32_t *row_ptr,
                            const int32_t *seg_idx, const double *piece_cp, const int32_t *piece_begin,
                            const int32_t *piece_level, int depth, int mode, int nthreads, int64_t *counts,
                            double *t_out, const double *delta, int32_t *amb)
{
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t i = 0; i < n_ray; ++i) {
        ray_t r = rays_f ? make_ray_f(rays_f + 8 * i) : make_ray_d(rays_d + 7 * i);
        if (mode == 1) duff_frame(r.w, r.e1, r.e2);
        double best = r.tmax;
        int64_t n = 0;
        probe_t pr = {delta ? delta[i] : 0.0, 0};
        g_probe = delta ? &pr : NULL;
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
            int32_t s = seg_idx[j];
            for (int32_t k = piece_begin[s]; k < piece_begin[s + 1]; ++k) {
                v4 Q[4];
                to_ray_frame(&r, piece_cp + 16 * k, Q);
                int d = piece_depth(depth, piece_level[k]);
                if (mode == 0) {
                    orc_hit h;
                    traverse(Q, d, best, &h);
                    n += h.nodes;
                    if (h.hit && h.t < best) best = h.t;
                } else {
                    best = box_search(Q, d, best, &n);
                }
            }
        }
        counts[i] = n;
        if (t_out) t_out[i] = best < r.tmax ? best : INFINITY;
        if (amb) amb[i] = pr.amb;
        g_probe = NULL;
    }
}

void orc_ray_counts(const float *rays, int64_t n_ray, const int32_t *row_ptr, const int32_t *seg_idx,
                    const double *piece_cp, const int32_t *piece_begin, const int32_t *piece_level,
                    int depth, int mode, int nthreads, int64_t *counts, double *t_out)
{
    ray_counts_impl(rays, NULL, n_ray, row_ptr, seg_idx, piece_cp, piece_begin, piece_level, depth, mode,
                    nthreads, counts, t_out, NULL, NULL);
}

/* The same with rays given in double precision (7 doubles: o, w, t_max). */
void orc_ray_counts_d(const double *rays7, int64_t n_ray, const int32_t *row_ptr, const int32_t *seg_idx,
                      const double *piece_cp, const int32_t *piece_begin, const int32_t *piece_level,
                      int depth, int mode, int nthreads, int64_t *counts, double *t_out)
{
    ray_counts_impl(NULL, rays7, n_ray, row_ptr, seg_idx, piece_cp, piece_begin, piece_level, depth, mode,
                    nthreads, counts, t_out, NULL, NULL);
}

/*
 * orc_ray_counts with, per ray, a flag: 1 if any decision of its search lies
 * within delta[i] of flipping under a sideways move of the ray (the probes
 * above).  A count on such a ray may legitimately come out differently in
 * lower precision; on any other ray every decision has a margin of at least
 * delta[i].  Rays as 8 floats (the workload's FP32 rays).
 */
void orc_ray_counts_amb(const float *rays, int64_t n_ray, const int32_t *row_ptr, const int32_t *seg_idx,
                        const double *piece_cp, const int32_t *piece_begin, const int32_t *piece_level,
                        int depth, int mode, int nthreads, const double *delta, int64_t *counts,
                        int32_t *amb)
{
    ray_counts_impl(rays, NULL, n_ray, row_ptr, seg_idx, piece_cp, piece_begin, piece_level, depth, mode,
                    nthreads, counts, NULL, delta, amb);
}

/* ------------------------------------------------------ quadratic curves */

/*
 * App. B.1: a quadratic curve (p0, p1, p2) can be split recursively at the
 * domain centre into subcurves with disjoint bounding volumes when
 * <p1 - p0, p1 - p2> <= 0 (positions).  (The lemma claims an equivalence,
 * but its two one-sided conditions <p1 - p0, p2 - p0> >= 0 and
 * <p1 - p2, p0 - p2> >= 0 do not imply the combined one; the combined one is
 * the one its second lemma carries to every subcurve.)
 */
int orc_valid_quadratic(const double *cp12)
{
    v4 a = sub4(load_cp(cp12, 1), load_cp(cp12, 0)), b = sub4(load_cp(cp12, 1), load_cp(cp12, 2));
    return dot3(a, b) <= 0.0;
}

/*
 * Degree elevation of a quadratic Bezier curve to the cubic with the same
 * curve and parametrisation (all four components, radius included):
 * q0 = p0, q1 = (p0 + 2 p1) / 3, q2 = (2 p1 + p2) / 3, q3 = p2.  The method's
 * representation and subdivision rules (Sec. 3.1) are stated for cubics; a
 * quadratic fiber is intersected as its raised cubic.
 */
void orc_elevate_quadratic(const double *cp12, double *cp16)
{
    for (int a = 0; a < 4; ++a) {
        double p0 = cp12[a], p1 = cp12[4 + a], p2 = cp12[8 + a];
        cp16[a] = p0;
        cp16[4 + a] = (p0 + 2.0 * p1) / 3.0;
        cp16[8 + a] = (2.0 * p1 + p2) / 3.0;
        cp16[12 + a] = p2;
    }
}

/* ------------------------------------------------------ exported entries */

/* One ray (7 doubles: o, w, t_max) against one curve at the given depth. */
void orc_intersect(const double *ray7, const double *cp, int depth, orc_hit *h)
{
    ray_t r = make_ray_d(ray7);
    v4 Q[4];
    to_ray_frame(&r, cp, Q);
    traverse(Q, depth, r.tmax, h);
}

static int piece_depth(int depth, int level) { return depth > level ? depth - level : 0; }

/*
 * One candidate segment against a ray: its pieces in order, each traversed to
 * depth - level; the pieces' best hit (ties keep the earlier
 * piece, so a piece is tested with the best t of the earlier pieces as t_max).
 * Returns 1 on a hit closer than tmax; u and leaf refer to the segment.
 */
static int candidate_hit(const ray_t *r, int32_t s, const double *piece_cp,
                         const int32_t *piece_begin, const int32_t *piece_level,
                         const int32_t *piece_off, int depth, double tmax, double *t_out,
                         double *u_out, int32_t *leaf_out, int64_t *cn, int64_t *cd, int64_t *cb,
                         int64_t *ch, int64_t *ct)
{
    double best = tmax, bu = -1.0;
    int32_t bl = -1;
    int got = 0;
    for (int32_t k = piece_begin[s]; k < piece_begin[s + 1]; ++k) {
        v4 Q[4];
        orc_hit h;
        to_ray_frame(r, piece_cp + 16 * k, Q);
        int lv = piece_level[k];
        traverse(Q, piece_depth(depth, lv), best, &h);
        *cn += h.nodes; *cd += h.descents; *cb += h.backtracks; *ct += 1;
        if (h.hit && h.t < best) {
            *ch += 1;
            best = h.t;
            bu = (piece_off[k] + h.u) * ldexp(1.0, -lv);
            bl = (int32_t)(((int64_t)piece_off[k] << (23 - lv)) + (h.leaf >> lv));
            got = 1;
        }
    }
    *t_out = got ? best : INFINITY;
    *u_out = bu;
    *leaf_out = bl;
    return got;
}

/*
 * Closest hit per ray over its CSR candidates: the smallest t among the
 * candidates' own hits, each candidate tested with the ray's t_max; ties keep
 * the earlier candidate (row order).  The top-level structure that supplies
 * candidates is orthogonal to the intersector (Sec. 2, Sec. 4), so the ray's
 * result is the plain minimum over independent candidate tests.  Outputs t
 * (inf on miss), u in the segment's parameter (-1), segment (-1), leaf start
 * in units of 2^-23 of the segment (-1).  counters (nullable): [nodes,
 * descents, backtracks, accepted leaf hits, piece tests].
 */
static void closest_impl(const float *rays_f, const double *rays_d, int64_t n_ray,
                         const int32_t *row_ptr, const int32_t *seg_idx, const double *piece_cp,
                         const int32_t *piece_begin, const int32_t *piece_level,
                         const int32_t *piece_off, int depth, int nthreads, double *t_out,
                         double *u_out, int32_t *seg_out, int32_t *leaf_out, int64_t *counters)
{
    int64_t cn = 0, cd = 0, cb = 0, ch = 0, ct = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : cn, cd, cb, ch, ct)
    for (int64_t i = 0; i < n_ray; ++i) {
        ray_t r = rays_f ? make_ray_f(rays_f + 8 * i) : make_ray_d(rays_d + 7 * i);
        double best = INFINITY, bu = -1.0;
        int32_t bs = -1, bl = -1;
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
            double t, u;
            int32_t leaf;
            if (candidate_hit(&r, seg_idx[j], piece_cp, piece_begin, piece_level, piece_off, depth,
                              r.tmax, &t, &u, &leaf, &cn, &cd, &cb, &ch, &ct) && t < best) {
                best = t;
                bu = u;
                bs = seg_idx[j];
                bl = leaf;
            }
        }
        t_out[i] = best;
        u_out[i] = bu;
        seg_out[i] = bs;
        if (leaf_out) leaf_out[i] = bl;
    }
    if (counters) {
        counters[0] = cn; counters[1] = cd; counters[2] = cb; counters[3] = ch; counters[4] = ct;
    }
}

void orc_closest(const float *rays, int64_t n_ray, const int32_t *row_ptr, const int32_t *seg_idx,
                 const double *piece_cp, const int32_t *piece_begin, const int32_t *piece_level,
                 const int32_t *piece_off, int depth, int nthreads, double *t_out, double *u_out,
                 int32_t *seg_out, int32_t *leaf_out, int64_t *counters)
{
    closest_impl(rays, NULL, n_ray, row_ptr, seg_idx, piece_cp, piece_begin, piece_level, piece_off,
                 depth, nthreads, t_out, u_out, seg_out, leaf_out, counters);
}

/* The same with rays given in double precision (7 doubles: o, w, t_max). */
void orc_closest_d(const double *rays7, int64_t n_ray, const int32_t *row_ptr,
                   const int32_t *seg_idx, const double *piece_cp, const int32_t *piece_begin,
                   const int32_t *piece_level, const int32_t *piece_off, int depth, int nthreads,
                   double *t_out, double *u_out, int32_t *seg_out, int32_t *leaf_out,
                   int64_t *counters)
{
    closest_impl(NULL, rays7, n_ray, row_ptr, seg_idx, piece_cp, piece_begin, piece_level, piece_off,
                 depth, nthreads, t_out, u_out, seg_out, leaf_out, counters);
}

/* Per-pair hits: each candidate tested with the ray's own t_max (see
 * candidate_hit).  Outputs indexed by pair. */
void orc_pairs(const float *rays, int64_t n_ray, const int32_t *row_ptr, const int32_t *seg_idx,
               const double *piece_cp, const int32_t *piece_begin, const int32_t *piece_level,
               const int32_t *piece_off, int depth, int nthreads, double *t_out, double *u_out,
               int32_t *leaf_out, int64_t *counters)
{
    int64_t cn = 0, cd = 0, cb = 0, ch = 0, ct = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : cn, cd, cb, ch, ct)
    for (int64_t i = 0; i < n_ray; ++i) {
        ray_t r = make_ray_f(rays + 8 * i);
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; ++j) {
            int32_t leaf;
            candidate_hit(&r, seg_idx[j], piece_cp, piece_begin, piece_level, piece_off, depth, r.tmax,
                          &t_out[j], &u_out[j], &leaf, &cn, &cd, &cb, &ch, &ct);
            if (leaf_out) leaf_out[j] = leaf;
        }
    }
    if (counters) {
        counters[0] = cn; counters[1] = cd; counters[2] = cb; counters[3] = ch; counters[4] = ct;
    }
}

/* ---------------------------------------------------- internals for pins */

void orc_to_ray_frame(const double *ray7, const double *cp, double *out16)
{
    ray_t r = make_ray_d(ray7);
    v4 Q[4];
    to_ray_frame(&r, cp, Q);
    for (int k = 0; k < 4; ++k) {
        out16[4 * k] = Q[k].x; out16[4 * k + 1] = Q[k].y; out16[4 * k + 2] = Q[k].z; out16[4 * k + 3] = Q[k].w;
    }
}

static void node_store(const node_t *c, double *o)
{
    const v4 *v[4] = {&c->p, &c->d, &c->t0, &c->t1};
    for (int k = 0; k < 4; ++k) { o[4 * k] = v[k]->x; o[4 * k + 1] = v[k]->y; o[4 * k + 2] = v[k]->z; o[4 * k + 3] = v[k]->w; }
}

static void node_load(const double *o, node_t *c)
{
    v4 *v[4] = {&c->p, &c->d, &c->t0, &c->t1};
    for (int k = 0; k < 4; ++k) *v[k] = V(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
}

/* Node (p, d, t0, t1) of the sub-interval (start, size) of the curve cp. */
void orc_node_at(const double *cp, uint32_t start, uint32_t size, double *out16)
{
    v4 P[4];
    node_t c;
    for (int k = 0; k < 4; ++k) P[k] = load_cp(cp, k);
    if (start == 0 && size == ROOT_SIZE) node_of_points(P, &c);
    else node_at(P, start, size, &c);
    node_store(&c, out16);
}

/* One subdivision step applied to a node (left or right child). */
void orc_subdivide(const double *node16, int go_right, double *out16)
{
    node_t c;
    v4 dp, tc;
    node_load(node16, &c);
    split_terms(&c, &dp, &tc);
    subdivide(&c, go_right, dp, tc);
    node_store(&c, out16);
}

double orc_cons_radius(const double *node16)
{
    node_t c;
    node_load(node16, &c);
    return cons_radius(&c);
}

int orc_cylinder(const double *p3, const double *a3, double r, double *out2)
{
    return cylinder(V(p3[0], p3[1], p3[2], 0.0), V(a3[0], a3[1], a3[2], 0.0), r, &out2[0], &out2[1]);
}

int orc_slab(const double *node16, double ray_tmax, double *out2)
{
    node_t c;
    node_load(node16, &c);
    return slab(&c, ray_tmax, &out2[0], &out2[1]);
}

/*
 * The capped cylinder of one leaf, tested on its own: the leaf's node from
 * node_at, its conservative radius and its own end-plane interval.  This is
 * the plain definition of a leaf bounding volume (Sec. 3.3); the brute-force
 * pin enumerates it over all 2^depth leaves.  Returns 1 and the entry t and u
 * (projection onto the leaf axis) if the ray meets it.
 */
int orc_leaf_hit(const double *ray7, const double *cp, int depth, uint32_t leaf, double *t_out,
                 double *u_out)
{
    ray_t r = make_ray_d(ray7);
    v4 Q[4];
    node_t c;
    to_ray_frame(&r, cp, Q);
    uint32_t size = ROOT_SIZE >> depth, start = leaf * size;
    if (start == 0 && size == ROOT_SIZE) node_of_points(Q, &c);
    else node_at(Q, start, size, &c);
    double tmin, tmax, c0, c1;
    slab(&c, r.tmax, &tmin, &tmax);
    double rad = cons_radius(&c);
    if (!(cylinder(c.p, c.d, rad, &c0, &c1) && dmax(c0, tmin) <= dmin(c1, tmax))) return 0;
    double t = dmax(c0, tmin);
    double dd = dot3(c.d, c.d), ul = 0.0;
    if (dd > 0.0) ul = dmax(0.0, dmin(1.0, (-c.p.x * c.d.x - c.p.y * c.d.y + (t - c.p.z) * c.d.z) / dd));
    *t_out = t;
    *u_out = (start + ul * size) * U_UNIT;
    return 1;
}

/* ---------------------------------------------------------- hit normal */

/*
 * Normal at a hit (App. C, the routine that computes the intersection's u
 * and normal).  The hit leaf [start, start + size) of the curve cp is
 * rebuilt in the ray frame; the hit point (0, 0, t) is projected onto the
 * leaf axis, u_local clamped to [0, 1], and u = u0 + u_local (u1 - u0).
 *   - an end cap: the normal is p0 - p1, resp. p3 - p2, normalised (the
 *     outward end-disk normal);
 *   - otherwise the axis point a = p + u_local d and the normal is the hit
 *     point minus a, taken back to world space (x e1 + y e2 + z w) and
 *     normalised.
 * (The listing's cur_c.axis and ray_direction are the leaf's d and the ray
 * direction w.)  The listing takes u == 0 or u == 1 for an end
 * cap; a hit on an end disk projects onto the leaf axis a rounding away from
 * either side of u_local = 0, so that test classifies end-disk hits by their
 * rounding.  Here the hit is on the cap at u = 0 (u = 1) if its leaf
 * is the first (last) one and the hit point lies on or beyond the segment's
 * end plane through p0 with normal p1 - p0 (through p3, normal p3 - p2), to
 * within 1e-12 (t + |p0|) here in FP64.  Writes n3 and returns 1 for a
 * lateral normal, 2 for the cap at u = 0, 3 for the cap at u = 1; *u_out is
 * the u above and *len_out (if not null) the length of the vector before it
 * was normalised (for a lateral hit, the hit point's distance from the axis
 * point).
 */
int orc_normal(const double *ray7, const double *cp, uint32_t start, uint32_t size, double t,
               double *n3, double *u_out, double *len_out)
{
    ray_t r = make_ray_d(ray7);
    v4 Q[4];
    node_t c;
    to_ray_frame(&r, cp, Q);
    if (start == 0 && size == ROOT_SIZE) node_of_points(Q, &c);
    else node_at(Q, start, size, &c);
    double dd = dot3(c.d, c.d), ul = 0.0;
    if (dd > 0.0) {
        v4 hb = V(-c.p.x, -c.p.y, t - c.p.z, 0.0);
        ul = dmax(0.0, dmin(1.0, dot3(hb, c.d) / dd));
    }
    double u = (start + ul * size) * U_UNIT;
    *u_out = u;
    /* signed distances of the hit point beyond the two end planes */
    v4 x = V(0.0, 0.0, t, 0.0);
    v4 a0 = sub4(Q[0], Q[1]), a1 = sub4(Q[3], Q[2]);
    double tol = 1e-12 * (t + sqrt(dot3(Q[0], Q[0])));
    int cap0 = 0, cap1 = 0;
    if (start == 0 && dot3(a0, a0) > 0.0) cap0 = dot3(sub4(x, Q[0]), a0) / sqrt(dot3(a0, a0)) >= -tol;
    if (start + size == ROOT_SIZE && dot3(a1, a1) > 0.0)
        cap1 = dot3(sub4(x, Q[3]), a1) / sqrt(dot3(a1, a1)) >= -tol;
    double n[3];
    int kind;
    if (cap0 || cap1) {
        int a = cap0 ? 0 : 3, b = cap0 ? 1 : 2;
        for (int i = 0; i < 3; ++i) n[i] = cp[4 * a + i] - cp[4 * b + i];
        kind = cap0 ? 2 : 3;
    } else {
        v4 ap = add4(c.p, mul4(ul, c.d));
        double xx = -ap.x, yy = -ap.y, zz = t - ap.z;
        for (int i = 0; i < 3; ++i) n[i] = xx * r.e1[i] + yy * r.e2[i] + zz * r.w[i];
        kind = 1;
    }
    double len = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
    for (int i = 0; i < 3; ++i) n3[i] = len > 0.0 ? n[i] / len : 0.0;
    if (len_out) *len_out = len;
    return kind;
}

/* ---------------------------------------------------------- limit surface */

/*
 * The surface the leaf cylinders converge to as the depth grows (Sec. 3.2:
 * the cylinders' limit surface): circles of radius r(u) in the
 * plane through c(u) normal to c'(u), closed by the flat end disks at u = 0
 * and u = 1.  With x = o + t w:
 *   G1(t, u) = <x - c(u), c'(u)> = 0,   G2(t, u) = |x - c(u)|^2 - r(u)^2 = 0.
 * G1 is linear in t; h(u) = G2(t(u), u) is sampled on n_grid + 1 points, every
 * sign change is bisected to 1e-15 in u and polished by two-dimensional
 * Newton steps.  Returns 1 (lateral), 2 (end disk at u = 0), 3 (u = 1) or 0.
 */
static void cps_world(const double *cp, v4 P[4])
{
    for (int k = 0; k < 4; ++k) P[k] = load_cp(cp, k);
}

static int t_of_u(const ray_t *r, const v4 P[4], double u, double *t, double *h)
{
    v4 c = bez_eval(P, u), d1 = mul4(3.0, bez_deriv3(P, u));
    v4 o = V(r->o[0], r->o[1], r->o[2], 0.0), w = V(r->w[0], r->w[1], r->w[2], 0.0);
    double den = dot3(w, d1);
    if (den == 0.0) return 0;
    *t = dot3(sub4(c, o), d1) / den;
    v4 x = add4(o, mul4(*t, w));
    v4 e = sub4(x, c);
    *h = dot3(e, e) - c.w * c.w;
    return 1;
}

static void newton_tu(const ray_t *r, const v4 P[4], double *t, double *u, int iters)
{
    v4 o = V(r->o[0], r->o[1], r->o[2], 0.0), w = V(r->w[0], r->w[1], r->w[2], 0.0);
    for (int it = 0; it < iters; ++it) {
        v4 c = bez_eval(P, *u), d1 = mul4(3.0, bez_deriv3(P, *u)), d2 = bez_deriv2(P, *u);
        v4 e = sub4(add4(o, mul4(*t, w)), c);
        double G1 = dot3(e, d1), G2 = dot3(e, e) - c.w * c.w;
        double J00 = dot3(w, d1), J01 = dot3(e, d2) - dot3(d1, d1);
        double J10 = 2.0 * dot3(e, w), J11 = -2.0 * dot3(e, d1) - 2.0 * c.w * d1.w;
        double det = J00 * J11 - J01 * J10;
        if (det == 0.0 || !isfinite(det)) return;
        double dt = (J11 * G1 - J01 * G2) / det, du = (-J10 * G1 + J00 * G2) / det;
        *t -= dt;
        *u -= du;
    }
}

int orc_limit_hit(const double *ray7, const double *cp, int n_grid, double *t_out, double *u_out)
{
    ray_t r = make_ray_d(ray7);
    v4 P[4];
    cps_world(cp, P);
    double best = INFINITY, bu = -1.0;
    int kind = 0;
    double tp = 0.0, hp = 0.0;
    int okp = t_of_u(&r, P, 0.0, &tp, &hp);
    for (int i = 1; i <= n_grid; ++i) {
        double u = (double)i / n_grid, t = 0.0, h = 0.0;
        int ok = t_of_u(&r, P, u, &t, &h);
        if (ok && okp && ((hp <= 0.0) != (h <= 0.0))) {
            double a = (double)(i - 1) / n_grid, b = u, ha = hp;
            /* no pole of t(u) inside: the denominators keep their sign */
            v4 wv = V(r.w[0], r.w[1], r.w[2], 0.0);
            double da = dot3(wv, bez_deriv3(P, a)), db = dot3(wv, bez_deriv3(P, b));
            if ((da > 0.0) == (db > 0.0)) {
                for (int it = 0; it < 200 && b - a > 1e-15; ++it) {
                    double m = 0.5 * (a + b), tm, hm;
                    if (!t_of_u(&r, P, m, &tm, &hm)) break;
                    if ((hm <= 0.0) == (ha <= 0.0)) { a = m; ha = hm; }
                    else b = m;
                }
                double uu = 0.5 * (a + b), tt, hh;
                if (t_of_u(&r, P, uu, &tt, &hh)) {
                    newton_tu(&r, P, &tt, &uu, 3);
                    if (tt >= 0.0 && tt < r.tmax && tt < best && uu >= 0.0 && uu <= 1.0) {
                        best = tt; bu = uu; kind = 1;
                    }
                }
            }
        }
        okp = ok; tp = t; hp = h;
    }
    for (int e = 0; e < 2; ++e) {
        double u = (double)e, t, h;
        if (t_of_u(&r, P, u, &t, &h) && h <= 0.0 && t >= 0.0 && t < r.tmax && t < best) {
            best = t; bu = u; kind = 2 + e;
        }
    }
    *t_out = best;
    *u_out = bu;
    return kind;
}

/*
 * dt / d(p_k, r_k) at a hit of the limit surface, by the
 * implicit function theorem on G(t, u; theta) = 0:
 *   [dt, du]^T = -J^{-1} dG/dtheta,  J = dG/d(t, u),
 *   dG1/dp_k = -B_k c' + B_k' (x - c),  dG2/dp_k = -2 B_k (x - c),
 *   dG2/dr_k = -2 r B_k,  dG1/dr_k = 0.
 * End-disk hits (u exactly 0 or 1) use G1 alone with u fixed.  (t, u) are
 * first refined by Newton steps.  grad: 16 doubles (p_k.xyz, r_k per k).
 * Returns 1 on success, 0 for a singular system.
 */
int orc_grad_t(const double *ray7, const double *cp, double t, double u, double *grad)
{
    ray_t r = make_ray_d(ray7);
    v4 P[4];
    cps_world(cp, P);
    v4 o = V(r.o[0], r.o[1], r.o[2], 0.0), w = V(r.w[0], r.w[1], r.w[2], 0.0);
    int cap = (u == 0.0 || u == 1.0);
    if (!cap) newton_tu(&r, P, &t, &u, 4);
    v4 c = bez_eval(P, u), d1 = mul4(3.0, bez_deriv3(P, u)), d2 = bez_deriv2(P, u);
    v4 e = sub4(add4(o, mul4(t, w)), c);
    double v = 1.0 - u;
    double B[4] = {v * v * v, 3.0 * u * v * v, 3.0 * u * u * v, u * u * u};
    double dB[4] = {-3.0 * v * v, 3.0 * v * v - 6.0 * u * v, 6.0 * u * v - 3.0 * u * u, 3.0 * u * u};
    double a1, a2; /* dt/dtheta = -(a1 dG1/dtheta + a2 dG2/dtheta) */
    if (cap) {
        double J00 = dot3(w, d1);
        if (J00 == 0.0) return 0;
        a1 = 1.0 / J00;
        a2 = 0.0;
    } else {
        double J00 = dot3(w, d1), J01 = dot3(e, d2) - dot3(d1, d1);
        double J10 = 2.0 * dot3(e, w), J11 = -2.0 * dot3(e, d1) - 2.0 * c.w * d1.w;
        double det = J00 * J11 - J01 * J10;
        if (det == 0.0 || !isfinite(det)) return 0;
        a1 = J11 / det;
        a2 = -J01 / det;
    }
    for (int k = 0; k < 4; ++k) {
        v4 g1 = sub4(mul4(dB[k], e), mul4(B[k], d1));
        v4 g2 = mul4(-2.0 * B[k], e);
        grad[4 * k + 0] = -(a1 * g1.x + a2 * g2.x);
        grad[4 * k + 1] = -(a1 * g1.y + a2 * g2.y);
        grad[4 * k + 2] = -(a1 * g1.z + a2 * g2.z);
        grad[4 * k + 3] = -(a2 * (-2.0 * c.w * B[k]));
    }
    return 1;
}

/* Refined (t, u) of a lateral limit-surface hit near the given estimate. */
void orc_refine_hit(const double *ray7, const double *cp, double *t, double *u)
{
    ray_t r = make_ray_d(ray7);
    v4 P[4];
    cps_world(cp, P);
    newton_tu(&r, P, t, u, 6);
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
