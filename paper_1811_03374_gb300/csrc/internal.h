// internal.h -- host/device shared declarations of the fiberx library (not
// part of the public C ABI).
#pragma once
#include <cstdint>
#include <string>

#include <cuda_runtime.h>

#include "../../include/fiberx.h"

// Workspace words of a handle (device, zeroed at upload).
enum {
  FX_WS_QUEUE = 0,    // persistent-kernel ray queue counter (reset before each launch)
  FX_WS_STATUS = 1,   // sticky FX_DEV_* bits
  FX_WS_WORDS = 32,   // 128 bytes of uint32 words, then the counters
};

// chunks of the host-buffer entry's copy / compute pipeline (at most)
#ifndef FX_HOST_CHUNKS
#define FX_HOST_CHUNKS 4
#endif
constexpr int kFxHostChunks = FX_HOST_CHUNKS;
// streams the host-buffer entry runs its chunks' kernels on (round robin), so
// that a chunk's kernels start once its own copy has landed, alongside the
// tail of the chunk before
#ifndef FX_HOST_STREAMS
#define FX_HOST_STREAMS 3
#endif
constexpr int kFxHostStreams = FX_HOST_STREAMS;

struct fx_fibers {
  int device = 0;
  int sm_count = 0;
  int64_t n_seg = 0, n_piece = 0, n_presplit = 0, n_unsupported = 0;
  int32_t max_level = 0;
  bool identity = true;                 // one level-0 piece per segment, none unsupported
  bool quadratic = false;               // uploaded as quadratics (stored raised to cubics)
  float4 *piece = nullptr;              // n_piece x {p, d, t0, t1} world space
  int32_t *piece_begin = nullptr;       // n_seg + 1
  int32_t *piece_info = nullptr;        // n_piece: level | off << 4 | unsupported << 31
  float *piece_rad = nullptr;           // n_piece: root conservative radius
  float4 *piece_root = nullptr;         // n_piece x {p.xyz, root radius}, {d.xyz, 0}
  float4 *seg_cp = nullptr;             // n_seg x 4 control points (backward, polish)
  uint32_t *ws = nullptr;               // FX_WS_WORDS words + 8 uint64 counters
  fx_launch launch{128, 0, 32, FX_VARIANT_LANE};  // blocks_per_sm 0: as many as fit
  // stream-ordered scratch of the intersect calls; keeps its memory between
  // calls (release threshold: never), so repeated calls do not remap it
  cudaMemPool_t pool = nullptr;
  // host-buffer entry staging (grow-only), its copy streams and the events
  // that order its chunks (created on first use)
  void *stage = nullptr;
  size_t stage_bytes = 0;
  cudaStream_t copy_in = nullptr, copy_out = nullptr;
  cudaStream_t compute[kFxHostStreams] = {};
  cudaEvent_t host_ev[1 + 2 * kFxHostChunks] = {};
  int64_t host_h2d = 0, host_d2h = 0;  // bytes the last host-buffer call copied
};

namespace fx {

constexpr int kMaxDepth = 23;

// Whether the calling thread's current device is the one the handle's arrays
// live on (its kernels must run there).
inline bool on_handle_device(const fx_fibers *f) {
  int d = -1;
  return cudaGetDevice(&d) == cudaSuccess && d == f->device;
}

struct TraceArgs {
  const float4 *piece;
  const int32_t *piece_begin;
  const int32_t *piece_info;
  const float *piece_rad;
  const float4 *piece_root;
  const float4 *rays;
  const int32_t *row_ptr;
  const int32_t *seg_idx;
  int64_t n_ray;
  int64_t n_pair;
  int32_t n_seg;
  int32_t depth;             // uniform subdivision depth
  const int8_t *ray_depth;   // nullable: each ray's own depth
  int32_t chunk;
  int32_t identity;
  float2 *tu;       // per ray (closest) or per pair (pairs)
  int32_t *seg;     // per ray (closest only)
  int32_t *leaf;    // nullable
  uint8_t *pair_flags;  // pairs only, nullable: FX_DEV_* bits of each pair's test
  uint32_t *queue;
  uint32_t *status;
  unsigned long long *counters;  // 5: nodes, descents, backtracks, tests, hits
  unsigned long long *scratch;   // naive kernel: per-ray packed (t, pair) keys
};

#ifdef __CUDACC__
// Subdivision depth of ray r: the call's uniform depth, or the ray's own
// entry of ray_depth, clamped to [0, 23] (FX_DEV_BAD_DEPTH when it was not).
__device__ __forceinline__ int depth_of(const TraceArgs &a, int64_t r) {
  if (!a.ray_depth) return a.depth;
  int d = __ldg(a.ray_depth + r);
  if (d < 0 || d > kMaxDepth) {
    atomicOr(a.status, FX_DEV_BAD_DEPTH);
    d = d < 0 ? 0 : kMaxDepth;
  }
  return d;
}
// With FX_CHECK_INDEX, a row of the CSR is clamped to [0, n_pair] and made
// non-decreasing (FX_DEV_BAD_INDEX when it had to be), so that a malformed
// row_ptr makes no kernel read or write out of range.
__device__ __forceinline__ void clamp_row(const TraceArgs &a, int32_t &crow, int32_t &cend) {
  const int32_t n = (int32_t)a.n_pair;
  const int32_t c0 = min(max(crow, 0), n), c1 = min(max(cend, c0), n);
  if (c0 != crow || c1 != cend) atomicOr(a.status, FX_DEV_BAD_INDEX);
  crow = c0;
  cend = c1;
}
// Iteration cap of one (ray, piece) test at a depth: a guard against runaway
// loops, far above any depth's node count.  (Compile-time settings, so that
// a test build can make the guard trip.)
#ifndef FX_ITER_CAP_BASE
#define FX_ITER_CAP_BASE 1024
#endif
#ifndef FX_ITER_CAP_PER_LEVEL
#define FX_ITER_CAP_PER_LEVEL 64
#endif
__device__ __forceinline__ int iter_cap(int depth) { return FX_ITER_CAP_BASE + FX_ITER_CAP_PER_LEVEL * depth; }
// The cap of a call: its depth's, or with per-ray depths that of depth 23,
// so that no register holds a ray's depth for it.
__device__ __forceinline__ int iter_cap_of(const TraceArgs &a) {
  return iter_cap(a.ray_depth ? kMaxDepth : a.depth);
}
#endif

// Work lists of the two-phase path (filter_kernels.cu), allocated per call.
struct FilterArgs {
  int2 *pass;          // n_pair, CSR aligned: {segment, entry bound as float bits} of passing pairs
  int32_t *pass_cnt;   // n_ray: passing pairs per ray
  int32_t *active;     // n_ray: rays with at least one passing pair (first *n_active entries)
  uint32_t *n_active;  // 1, zeroed before the filter runs
  uint32_t *group_queue;  // 1, zeroed before the filter runs: next group of 32 rays
};

// Launchers (trace_kernels.cu).  flags: FX_* bits of the public header.
cudaError_t launch_naive(const TraceArgs &a, bool pairs, uint32_t flags, cudaStream_t s);
cudaError_t launch_polish(const TraceArgs &a, const float4 *seg_cp, cudaStream_t s);

// lane_kernels.cu
cudaError_t launch_lane_ray(const TraceArgs &a, bool pairs, uint32_t flags, int blocks_per_sm_cap,
                            int sm_count, cudaStream_t s);

// filter_kernels.cu: root filter, then traversal of the active rays (closest
// hit, handles with single level-0 pieces only)
cudaError_t launch_filter(const TraceArgs &a, const FilterArgs &o, uint32_t flags, int blocks_per_sm_cap,
                          int sm_count, cudaStream_t s);

// Work list of the scan path (scan_kernels.cu), allocated per call: the rays
// that have candidates, as {ray, row begin, row end, 0}.
struct ScanArgs {
  int4 *act;        // n_ray entries (the first *n_act used)
  uint32_t *n_act;  // 1, zeroed before the rows pass runs
};

// scan_kernels.cu: rows pass (misses of rays without candidates, list of the
// others), then lane-per-ray traversal with candidates scanned 32 at a time
// by the warp (handles with single level-0 pieces only)
cudaError_t launch_scan_ray(const TraceArgs &a, const ScanArgs &o, bool pairs, uint32_t flags,
                            int blocks_per_sm_cap, int sm_count, cudaStream_t s);

// ray_kernels.cu: one thread per ray (handles with single level-0 pieces only)
// Walks the per-ray variant's first pass leaves to its second (closest
// hits; null walks: one pass).  A walk is ray_walk_bytes() (128) bytes.
struct RayDefer {
  void *walks;        // capacity saved walks, 16-byte aligned
  uint32_t *count;    // zeroed before the first pass
  uint32_t capacity;  // walks the list holds: one per ray
};
size_t ray_walk_bytes();
cudaError_t launch_ray(const TraceArgs &a, bool pairs, uint32_t flags, const RayDefer &d, int sm_count,
                       cudaStream_t s);

// warp_kernels.cu
cudaError_t launch_warp_ray(const TraceArgs &a, bool pairs, uint32_t flags, int blocks_per_sm_cap,
                            int sm_count, cudaStream_t s);

// normal_kernels.cu: hit normals from closest-hit results (App. C)
cudaError_t launch_normals(const TraceArgs &a, const float4 *seg_cp, float *normal, uint32_t flags,
                           cudaStream_t s);

// count_kernels.cu: per-ray pruning-test counts, cylinders or boxes (Fig. 8)
cudaError_t launch_counts(const TraceArgs &a, uint32_t *counts, bool box, uint32_t flags, cudaStream_t s);

// peak.cu: FP32 FMA microbenchmark (synchronises s); flops = FMA flops of the
// timed launch
cudaError_t fma_peak(int sm_count, int blocks_per_sm, int iters, float *ms, double *flops, cudaStream_t s);

// fiberx_api.cu: text returned by fx_last_error() on this thread
void set_last_error(const std::string &msg);

// backward.cu
// quadratic: the handle holds raised quadratics; grad_cps is n_seg x 12
// (p0..p2), else n_seg x 16
cudaError_t launch_backward(const float4 *seg_cp, int64_t n_seg, bool quadratic, const float4 *rays,
                            int64_t n_ray, const float2 *tu, const int32_t *seg, const float *grad_t,
                            float *grad_cps, unsigned long long *n_skipped, cudaStream_t s);

}  // namespace fx
