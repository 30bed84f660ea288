/*
 * fiberx.h -- C ABI of the GB300 (sm_103a) ray / cubic-fiber intersector.
 *
 * Method: Binder & Keller, "Fast, High Precision Ray/Fiber Intersection using
 * Tight, Disjoint Bounding Volumes" (arXiv 1811.03374).  A fiber segment is a
 * cubic Bezier curve with a radius per control point (Sec. 3.3).  A ray is
 * intersected with a segment by stackless recursive subdivision (Sec. 3, the
 * iterative routine of App. C): each region is bounded by a cylinder along its
 * chord with a conservative radius (Sec. 3.3), partitioned by the plane through
 * the split point orthogonal to the split tangent (Sec. 3.2, Fig. 5); the child
 * the ray reaches first is visited first, one bit per level records whether
 * the sibling must be visited too, and the first leaf hit ends the search.
 * The hit is the entry into the leaf's capped cylinder; u is the projection of
 * the hit point onto the leaf axis (App. C).
 *
 * Conventions for every entry point:
 *  - Array arguments are DEVICE pointers unless the call says otherwise; the
 *    caller owns them.  No entry point keeps a pointer to caller memory after
 *    it returns.
 *  - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls are
 *    asynchronous and stream-ordered; only fiber_upload, fx_stream_status and
 *    intersect_closest_host synchronise.
 *  - Argument errors are reported synchronously, before any launch, and leave
 *    outputs untouched.  CUDA errors are returned as FX_ECUDA; the message is
 *    available from fx_last_error().
 *  - Device-side conditions never trap: they set bits of the handle's sticky
 *    status word (FX_DEV_*), read and cleared by fx_stream_status.
 *  - A handle's arrays live on the device that was current at its upload;
 *    every intersect_* call must be made with that device current
 *    (FX_EDEVICE otherwise, before any launch).
 *  - Calls on one handle may run concurrently on unordered streams: each
 *    call's work-queue counter and scratch come from the handle's
 *    stream-ordered memory pool.  They share the sticky status word and the
 *    counters (bits and sums of all of them).  Exceptions:
 *    intersect_closest_host (the handle's staging) and
 *    intersect_closest_noalloc (one key array per device) must not overlap
 *    another call of their own kind.
 */
#ifndef FIBERX_H
#define FIBERX_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FX_OK = 0,
    FX_EINVAL = -1,       /* bad argument (null pointer, negative size, bad CSR, ...) */
    FX_ECUDA = -2,        /* a CUDA runtime call failed */
    FX_ENOMEM = -3,       /* device or host allocation failed */
    FX_EUNSUPPORTED = -4, /* option not supported */
    FX_ETIMEOUT = -5,     /* reserved: a bounded device wait ran out */
    FX_EDEPTH = -6,       /* subdivision depth outside [0, 23] */
    FX_EDEVICE = -7       /* no usable sm_103 device, or the current device is not the handle's */
} fx_status;

/* Sticky device status bits (fx_stream_status). */
#define FX_DEV_ITER_LIMIT 0x1u  /* a (ray, segment) test hit the per-pair iteration cap */
#define FX_DEV_UNSUPPORTED 0x2u /* a hit was reported on a piece flagged unsupported */
#define FX_DEV_BAD_INDEX 0x4u   /* a segment id was out of range (skipped), or with FX_CHECK_INDEX a CSR row (clamped) */
#define FX_DEV_BAD_DEPTH 0x8u   /* a per-ray depth was outside [0, 23] (clamped to it) */

/* intersect_* flags */
#define FX_KERNEL_PERSISTENT 0x0u /* default: persistent work-queue kernel */
#define FX_KERNEL_NAIVE 0x1u      /* one thread per (ray, segment) pair (baseline) */
#define FX_FAST_MATH 0x2u         /* approximate reciprocal / square root in the traversal */
#define FX_POLISH_FP64 0x4u       /* re-evaluate each hit's leaf and its neighbours in FP64, keep the nearest (intersect_closest) */
#define FX_COUNT 0x8u             /* accumulate node / descent / backtrack counters */
#define FX_CHECK_INDEX 0x10u      /* range-check candidate segment ids and rows on the device */
#define FX_COUNT_BOXES 0x20u      /* intersect_counts: ray-frame axis-aligned boxes instead of cylinders */

typedef struct fx_fibers fx_fibers; /* opaque; owns the device copy of the fibers */

typedef struct {
    int32_t max_presplit; /* levels of dyadic pre-split for invalid curves, 0..8 (default 8) */
    int32_t thick_check;  /* 1 (default): exact end-plane check for thick fibers (Sec. 3.4) */
} fx_upload_opts;

typedef struct {
    int64_t n_seg;         /* segments uploaded */
    int64_t n_piece;       /* pieces after pre-split (>= n_seg) */
    int64_t n_presplit;    /* segments split into more than one piece */
    int64_t n_unsupported; /* pieces still failing the checks at the maximum level */
    int32_t max_level;     /* deepest pre-split level used */
    int32_t sm_count;      /* SMs of the device the handle lives on */
} fx_fibers_info;

/* Persistent kernel variants (fx_launch.variant). */
#define FX_VARIANT_AUTO 0   /* the library's choice: RAY for rows of at most two candidates on
                               average (n_pair <= 2 n_ray) on handles without pre-split
                               segments, LANE otherwise */
#define FX_VARIANT_LANE 1   /* each lane owns a ray and walks its candidates front to back */
#define FX_VARIANT_WARP 2   /* a warp owns a ray; its candidates are staged in shared memory */
#define FX_VARIANT_FILTER 3 /* two phases: the root test of every pair, one lane per pair, then
                               LANE's traversal of the passing candidates of the rays that have
                               any.  Same results and counters as LANE.  intersect_closest on
                               handles whose segments are single level-0 pieces (none pre-split
                               or unsupported) only; elsewhere LANE runs.  Its work lists
                               (8 B per pair, 8 B per ray) come from the handle's memory pool. */
#define FX_VARIANT_SCAN 4   /* each lane owns a ray as in LANE; the warp tests 32 candidates of a
                               lane's row at once (bound and root cylinder, one lane per
                               candidate) and the owner traverses the root hits in row order.
                               Same results as LANE.  Handles whose segments are single level-0
                               pieces only; elsewhere LANE runs. */
#define FX_VARIANT_RAY 5    /* one thread per ray walking its candidates in row order with LANE's
                               arithmetic, no work queue: for rows of one or a few candidates
                               (many rays against one fiber).  Closest hits take two passes: rays
                               needing more than 4 node tests save their walk (128 bytes, pool
                               memory for one per ray) and a second pass continues it.  Same
                               results as LANE, pre-split segments included. */

/* Launch configuration of the persistent kernels (fx_set_launch). */
typedef struct {
    int32_t block;         /* reserved: 64, 128 or 256 (the variants fix their own block sizes) */
    int32_t blocks_per_sm; /* blocks per SM the grid is sized for (1..16; 0 = as many as fit) */
    int32_t chunk;         /* lane-per-ray: rays a warp takes from the queue at a time (1..1024) */
    int32_t variant;       /* FX_VARIANT_* */
} fx_launch;

/*
 * fiber_upload -- validate, pre-split and copy fiber segments to the device.
 *
 * cps: n_seg x 4 control points x (x, y, z, r) floats, r >= 0 (Sec. 3.3:
 * four-dimensional control points, radius interpolated by the Bezier basis).
 * cps_on_device: 0 = host pointer, 1 = device pointer.  The data is copied;
 * the caller keeps ownership.  opts may be NULL (defaults).
 *
 * Each segment is checked in FP64 against the five inequalities of Sec. 3.4
 * (App. B.2) and an exact end-plane check for thick fibers (Sec. 3.4,
 * Fig. 7: no end plane cuts the tube swept by the largest control radius,
 * decided on polynomials in u by Bernstein subdivision); failing curves are
 * halved at u = 1/2 recursively (Sec. 3.4 requires such curves to be split
 * first) up to max_presplit levels.  A piece at level k is
 * later traversed to depth d - k, so its leaves coincide with the unsplit
 * curve's.  Pieces still failing at the last level are kept and counted as
 * unsupported (not an error).
 *
 * Errors: FX_EINVAL (n_seg < 0, null pointers, non-finite values, r < 0),
 * FX_ENOMEM, FX_ECUDA, FX_EDEVICE.  Synchronises `stream`.
 */
fx_status fiber_upload(const float *cps, int64_t n_seg, int32_t cps_on_device,
                       const fx_upload_opts *opts, void *stream, fx_fibers **out);

/*
 * fiber_upload_quadratic -- fiber_upload for quadratic Bezier segments (the
 * paper evaluates quadratic and cubic fibers, Sec. 4; their constraint is
 * App. B.1's <p1 - p0, p1 - p2> <= 0).
 *
 * cps: n_seg x 3 control points x (x, y, z, r) floats, r >= 0; host or device
 * memory as cps_on_device says; copied.  Each segment is raised to the cubic
 * with the same curve and parametrisation (degree elevation, in FP64, all
 * four components: q0 = p0, q1 = (p0 + 2 p1) / 3, q2 = (2 p1 + p2) / 3,
 * q3 = p2) and then uploaded as fiber_upload does, so every intersect_* call
 * and its u, leaf and segment ids refer to the quadratic segment.  A
 * quadratic that meets App. B.1's constraint raises to a cubic that meets the
 * five cubic constraints of Sec. 3.4, so it is not pre-split.
 * intersect_backward on such a handle returns the gradient with respect to
 * the quadratic control points p0..p2 (n_seg x 3 x 4; the kernel applies the
 * chain rule through the elevation).  Errors as fiber_upload.
 */
fx_status fiber_upload_quadratic(const float *cps, int64_t n_seg, int32_t cps_on_device,
                                 const fx_upload_opts *opts, void *stream, fx_fibers **out);

/* Releases the handle and its device memory (NULL is a no-op). */
void fiber_free(fx_fibers *f);

/* Counts describing the uploaded fibers. */
fx_status fiber_info(const fx_fibers *f, fx_fibers_info *out);

/*
 * intersect_closest -- closest hit of every ray over its candidate segments.
 *
 * rays: n_ray x 8 floats {o.x, o.y, o.z, t_max, w.x, w.y, w.z, 0}; w is
 * normalised on the device (unit ray, Sec. 3.3); hits need 0 <= t < t_max.
 * row_ptr: n_ray + 1 int32 (row_ptr[0] = 0, non-decreasing, row_ptr[n_ray] =
 * n_pair); seg_idx: n_pair int32 segment ids.  The CSR is validated on the
 * host only for its sizes; set FX_CHECK_INDEX to range-check ids on the
 * device and to clamp each row to [0, n_pair], non-decreasing (both flagged
 * FX_DEV_BAD_INDEX), so that a malformed CSR reads nothing out of range; the
 * filter and warp variants then run as the lane kernel.
 * depth: subdivision depth d in [0, 23]; leaves have size 2^-d (Sec. 3.3:
 * termination after a fixed number of subdivisions).
 * ray_depth: nullable; n_ray int8 per-ray depths (device pointer) that
 * replace `depth` ray by ray, e.g. chosen from each ray's footprint (the
 * paper's routine takes its termination size per call).  Entries outside
 * [0, 23] are clamped to it and set FX_DEV_BAD_DEPTH.
 *
 * Candidates are visited in row order, pieces in order; the closest hit so
 * far is the t_max of the next test and only a strictly closer hit replaces
 * it (Sec. 3.2: instant termination; ties keep the earlier candidate).
 * Outputs per ray: tu (2 floats: t, u in the segment's parameter; miss:
 * t = +inf, u = -1), seg (int32, -1 on miss), leaf (nullable; int32 start of
 * the hit leaf in units of 2^-23 of the segment; -1 on miss).
 * flags: FX_KERNEL_*, FX_FAST_MATH, FX_POLISH_FP64, FX_COUNT, FX_CHECK_INDEX.
 * Scratch (FX_VARIANT_FILTER's work lists, the naive kernel's per-ray keys,
 * a leaf buffer for the polish) is allocated stream-ordered from a memory
 * pool owned by the handle, which keeps freed memory for the next call.
 * Errors: FX_EINVAL, FX_EDEPTH, FX_ECUDA.
 */
fx_status intersect_closest(const fx_fibers *f, const float *rays, int64_t n_ray,
                            const int32_t *row_ptr, const int32_t *seg_idx, int64_t n_pair,
                            int32_t depth, const int8_t *ray_depth, uint32_t flags, float *tu,
                            int32_t *seg, int32_t *leaf, void *stream);

/*
 * intersect_pairs -- one result per (ray, candidate) pair, each tested with
 * the ray's own t_max (no pruning across candidates).  Same inputs as
 * intersect_closest (ray_depth included); outputs per pair: tu (2 floats),
 * leaf (nullable) and pair_flags (nullable, one byte per pair: the FX_DEV_*
 * bits -- iteration cap, unsupported piece hit, bad segment id -- that this
 * pair's test raised, a hit on an unsupported piece counting even when a
 * later piece of the segment replaced it; the sticky status word gets them
 * too).  flags:
 * FX_KERNEL_*, FX_FAST_MATH, FX_COUNT, FX_CHECK_INDEX.
 */
fx_status intersect_pairs(const fx_fibers *f, const float *rays, int64_t n_ray,
                          const int32_t *row_ptr, const int32_t *seg_idx, int64_t n_pair,
                          int32_t depth, const int8_t *ray_depth, uint32_t flags, float *tu,
                          int32_t *leaf, uint8_t *pair_flags, void *stream);

/*
 * intersect_backward -- adjoint of the closest hit's t with respect to the
 * segments' control points and radii.
 *
 * The surface the leaf cylinders converge to (Sec. 3.2) is the sweep of
 * circles of radius r(u) in the planes normal to c'(u), closed by flat end
 * disks.  With x = o + t w, a hit satisfies G1 = <x - c(u), c'(u)> = 0 and
 * G2 = |x - c(u)|^2 - r(u)^2 = 0; (t, u) from the forward pass are refined by
 * Newton steps on G and dt/dtheta = -[J^-1 dG/dtheta]_t (implicit function
 * theorem).  End-disk hits (u = 0 or 1) use G1 with u fixed.
 *
 * Inputs: rays (as above), tu and seg from intersect_closest, grad_t (n_ray
 * floats, dL/dt_i).  Output: grad_cps, same layout as the cps the handle was
 * uploaded from -- n_seg x 16 floats for fiber_upload, n_seg x 12 for
 * fiber_upload_quadratic (with respect to p0..p2: the adjoint of the raised
 * cubic q0..q3 carried back through q0 = p0, q1 = (p0 + 2 p1) / 3,
 * q2 = (2 p1 + p2) / 3, q3 = p2) -- ACCUMULATED (+=) with atomics; zero it
 * first for a fresh gradient.
 * Misses and rays with grad_t == 0 contribute nothing; hits whose system
 * is singular (|det J| tiny: grazing) are skipped and counted in
 * *n_skipped_dev (device int64, nullable).
 */
fx_status intersect_backward(const fx_fibers *f, const float *rays, int64_t n_ray,
                             const float *tu, const int32_t *seg, const float *grad_t,
                             float *grad_cps, unsigned long long *n_skipped_dev, void *stream);

/*
 * intersect_normals -- surface normals at the closest hits (App. C, the
 * routine that computes the intersection's u and normal).
 *
 * Inputs: rays (as above), and tu, seg, leaf from intersect_closest on the
 * same handle with the same depth and ray_depth (leaf is required).  Output: normal, n_ray x
 * 3 floats, world space, unit length; (0, 0, 0) for misses.  The hit leaf is
 * rebuilt in the ray frame and the hit point projected onto its axis; a
 * lateral hit's normal is the hit point minus that axis point.  A hit on an
 * end disk -- the first (last) leaf, hit point on or beyond the segment's end
 * plane through p0 with normal p1 - p0 (through p3 with normal p3 - p2) to
 * within 8 ulp of (t + |p0 - o|) -- gets the outward disk normal p0 - p1
 * (p3 - p2).  flags: FX_FAST_MATH (approximate square root).
 * Errors: FX_EINVAL (null pointers, negative size), FX_EDEPTH, FX_ECUDA.
 */
fx_status intersect_normals(const fx_fibers *f, const float *rays, int64_t n_ray, const float *tu,
                            const int32_t *seg, const int32_t *leaf, int32_t depth,
                            const int8_t *ray_depth, uint32_t flags, float *normal, void *stream);

/*
 * intersect_counts -- per-ray pruning-test counts, the statistic of Fig. 8
 * (oriented bounding cylinders against axis-aligned boxes).
 *
 * Same inputs as intersect_closest (uniform depth only).  Each ray's
 * candidates are searched in row order with the closest hit so far as
 * t_max, with no test before the root's, so only the bounding volume
 * differs:
 *   - default: the traversal of Sec. 3.3; one count per node tested;
 *   - FX_COUNT_BOXES: the same subdivision without partition planes, each
 *     node bounded by the box [min_k (q_k - r_k), max_k (q_k + r_k)] of its
 *     control points q_k and radii r_k in the ray's frame.  Both children of
 *     a hit node are tested (two counts), the one with the smaller z_min is
 *     searched first and the other tested again (one count) when taken up;
 *     the search does not end at the first leaf hit.
 * A pre-split segment's pieces are searched in order, each to depth - level
 * (the unsplit curve's leaves), with the closest hit so far as t_max.
 * Output: counts, n_ray uint32 (saturating).  flags: FX_FAST_MATH,
 * FX_CHECK_INDEX, FX_COUNT_BOXES.  Errors: FX_EINVAL, FX_EDEPTH, FX_EDEVICE,
 * FX_ECUDA.
 */
fx_status intersect_counts(const fx_fibers *f, const float *rays, int64_t n_ray, const int32_t *row_ptr,
                           const int32_t *seg_idx, int64_t n_pair, int32_t depth, uint32_t flags,
                           uint32_t *counts, void *stream);

/*
 * intersect_closest_host -- intersect_closest on HOST buffers: copies rays,
 * row_ptr and seg_idx to device staging owned by the handle, runs, copies
 * tu / seg / leaf back and synchronises (ray_depth, when given, is a host
 * array too).  Large calls are cut into up to 4
 * chunks of rows with about equal input bytes; each chunk's copy in, kernels
 * and copy out run on copy and compute streams owned by the handle (after
 * the work already queued on `stream`), so copies overlap the other chunks'
 * kernels and a chunk's kernels overlap the tail of the chunk before (the
 * naive kernel takes one chunk).  Rays in pinned host memory that the
 * runtime maps into the device's address space (cudaHostAlloc, or
 * cudaHostRegister with the mapped flag) are read by the kernels in place,
 * 32 bytes per ray that has a candidate; other rays are copied, in blocks of
 * 8192 rows that hold a candidate (the ray of an empty row is never read;
 * its result is a miss).  The chunk with the fewest rays is copied last.
 * Both rely on the CSR contract above (row_ptr[0] = 0, non-decreasing,
 * row_ptr[n_ray] = n_pair).  Host buffers should be pinned
 * for full copy bandwidth and asynchronous copies.  Calls on one handle must
 * not overlap (they share its staging).  Same flags and errors as
 * intersect_closest, plus FX_ENOMEM if the staging cannot grow.
 */
fx_status intersect_closest_host(fx_fibers *f, const float *rays, int64_t n_ray,
                                 const int32_t *row_ptr, const int32_t *seg_idx, int64_t n_pair,
                                 int32_t depth, const int8_t *ray_depth, uint32_t flags, float *tu,
                                 int32_t *seg, int32_t *leaf, void *stream);

/*
 * fx_host_bytes -- bytes the last intersect_closest_host call on this handle
 * moved host to device (*h2d: copies, with rays read in place counted as the
 * rays of the blocks of 8192 rows that hold a candidate) and device to host
 * (*d2h); 0 before the first call.  Errors: FX_EINVAL (null pointers).
 */
fx_status fx_host_bytes(const fx_fibers *f, int64_t *h2d, int64_t *d2h);

/*
 * fx_set_launch / fx_get_launch -- launch shape of the persistent kernels of
 * this handle (the autotuner's knobs).  Invalid values give FX_EINVAL.
 */
fx_status fx_set_launch(fx_fibers *f, const fx_launch *cfg);
fx_status fx_get_launch(const fx_fibers *f, fx_launch *cfg);

/*
 * fx_counters -- node tests, descents, backtracks, pair tests and hits
 * accumulated by launches with FX_COUNT since the last reset (host array of
 * 5 uint64; synchronises `stream`).  reset != 0 clears them afterwards.
 */
fx_status fx_counters(fx_fibers *f, void *stream, uint64_t *out5, int32_t reset);

/*
 * fx_stream_status -- synchronises `stream`, returns the handle's sticky
 * device status bits (FX_DEV_*) in *device_flags and clears them.
 */
fx_status fx_stream_status(fx_fibers *f, void *stream, uint32_t *device_flags);

/*
 * intersect_closest_noalloc -- intersect_closest, with the one-thread-per-pair
 * kernel, for callers that must not allocate device memory while they run:
 * a renderer whose device memory is handed out up front by another
 * allocator, or a real-time loop that cannot afford the implicit
 * synchronisation of cudaMalloc / cudaFree.  (The paper has no counterpart;
 * this is a property of the library, not of the method.)
 *
 * intersect_closest allocates the naive kernel's scratch, one 64-bit key per
 * ray, on each call.  This entry point allocates nothing: the keys live in a
 * fixed device array of FX_NOALLOC_MAX_RAYS entries (8 MiB) that every GPU
 * loading the library holds until the process exits.  The caller passes the
 * handle, inputs and outputs as for intersect_closest (uniform depth only, no
 * ray_depth); n_ray above
 * FX_NOALLOC_MAX_RAYS is refused with FX_EINVAL.  Results equal
 * intersect_closest with FX_KERNEL_NAIVE and the same flags (FX_FAST_MATH,
 * FX_COUNT, FX_CHECK_INDEX; FX_POLISH_FP64 needs a non-null leaf).
 *
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current and keeps it for the
 * process; make that first call before any stream capture.  A
 * cudaDeviceReset destroys the array with every other allocation of the
 * device (and every handle): the kept address is then stale, so do not use
 * the library on a device after resetting it.  The handle's device must be
 * current (FX_EDEVICE otherwise).  Every call shares the array: each clears
 * the keys it uses before its kernels run, and calls that overlap on the GPU
 * (unordered streams) race on it.
 */
#define FX_NOALLOC_MAX_RAYS (1 << 20)
fx_status intersect_closest_noalloc(const fx_fibers *f, const float *rays, int64_t n_ray,
                                    const int32_t *row_ptr, const int32_t *seg_idx, int64_t n_pair,
                                    int32_t depth, uint32_t flags, float *tu, int32_t *seg,
                                    int32_t *leaf, void *stream);

/*
 * fx_fma_peak -- measures the FP32 FMA throughput of the current device: one
 * launch of blocks_per_sm x 256-thread blocks per SM, each thread running
 * eight independent FMA chains of 16 * iters steps, timed with CUDA events on
 * `stream` (synchronises it).  *ms: the launch's time; *tflops: FMA flops
 * (2 per FMA) per second / 1e12.  A measurement helper for the FP32 FMA
 * roofline the traversal is reported against (the paper has no counterpart).
 * Errors: FX_EINVAL (null outputs, blocks_per_sm outside 1..8, iters < 1),
 * FX_ECUDA.
 */
fx_status fx_fma_peak(int32_t blocks_per_sm, int32_t iters, float *ms, double *tflops, void *stream);

/* Text of the last error on this thread ("" if none). */
const char *fx_last_error(void);

/* Library version, major * 10000 + minor * 100 + patch. */
int32_t fx_version(void);

#ifdef __cplusplus
}
#endif

#endif /* FIBERX_H */
