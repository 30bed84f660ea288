// ray_kernels.cu -- one thread per ray (FX_VARIANT_RAY), for rows of one or
// a few candidates, such as many rays against a single fiber (the shape of
// the paper's own benchmark, Fig. 1).
//
// Each thread loads its ray, builds the ray frame (Sec. 3.3) and walks its
// candidates in row order with the closest hit so far as t_max (Sec. 3.2:
// instant termination, carried across candidates).  Per candidate it runs
// the lane kernel's arithmetic step for step -- the bound test on the root
// record, the root cylinder with the precomputed radius, the slab once a
// cylinder is hit, the bit-string traversal of Sec. 3.3 -- so the results are
// the lane kernel's bit for bit.  There is no work queue and no staging:
// with one candidate per ray the persistent kernels' machinery costs more
// than the traversal.  On handles with pre-split segments (IDENTITY false) a
// candidate's pieces are traversed in order, each to depth d - level, as the
// lane kernel does there; each piece first takes the bound test on its own
// root record (the lane kernel tests every piece's root instead: the bound
// only drops roots that cannot pass, so the results are the same).
//
// Closest hits take two passes.  The first gives each ray a budget of node
// tests.  A ray done within it (most rays against a single fiber miss at the
// root) is finished there; a ray that needs more saves its walk -- the node
// about to be tested, the bit string, the slab, the closest hit so far, the
// candidate -- to a list, and the second pass continues it from there.  The
// few rays with long traversals thus no longer hold warps of rays with short
// ones, and no node test is done twice.
#include <algorithm>
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kRayBlock = 128;
// relative slack of the bound test against FP32 rounding (the lane kernel's)
constexpr float kBoundSlack = 1.0f / 262144.0f;
// node tests a ray may take in the first pass of closest hits
#ifndef FX_RAY_BUDGET
#define FX_RAY_BUDGET 4
#endif
constexpr int kBudget = FX_RAY_BUDGET;
static_assert(kBudget >= 1, "the first pass takes at least the root test");

// Walk modes: the whole walk in one pass (closest hits or per pair); the
// first pass of closest hits (at most kBudget node tests, then the walk is
// saved); the second pass (continues a saved walk).
enum WalkMode { kWalkAll = 0, kWalkFirst = 1, kWalkResume = 2 };

// A closest-hit walk saved between the passes (128 bytes).
struct alignas(16) RayWalk {
  Node c;                     // the node about to be tested, ray frame
  float tmin, tmax, root_r, best_t;
  float best_u;
  int32_t ray, j, best_seg;   // ray, current candidate, closest hit's segment
  int32_t best_leaf, iters;
  uint32_t bits, start;
  uint32_t size, slab_ok;
  int32_t piece, pad0;        // the piece of the candidate (pre-split segments)
};
static_assert(sizeof(RayWalk) == 128, "two cache sectors per saved walk");

__device__ __forceinline__ void rotate_piece(const float4* __restrict__ piece, int32_t k, const RayFrame& r,
                                             Node& n) {
  const float4 p = __ldg(piece + 4 * (int64_t)k), d = __ldg(piece + 4 * (int64_t)k + 1);
  const float4 t0 = __ldg(piece + 4 * (int64_t)k + 2), t1 = __ldg(piece + 4 * (int64_t)k + 3);
  n.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
  n.d = rotate(r, d.x, d.y, d.z, d.w);
  n.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
  n.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
}

// Ray r against its candidates.  kWalkFirst returns true when the ray needs
// more than kBudget node tests: `w` then holds its walk, nothing is written,
// and the events so far are counted.  kWalkResume continues the walk in `w`.
// Otherwise the ray's result is written and it returns false.
template <bool FAST, bool PAIRS, bool COUNT, bool IDENTITY, int MODE>
__device__ __forceinline__ bool ray_walk(const TraceArgs& a, int64_t r, RayWalk& w, int check,
                                         uint32_t (&cnt)[5]) {
  static_assert(MODE == kWalkAll || !PAIRS, "the two passes serve closest hits");
  uint32_t n_nodes = 0, n_desc = 0, n_back = 0, n_tests = 0, n_hits = 0;
  auto flush = [&]() {
    if (COUNT) {
      cnt[0] += n_nodes;
      cnt[1] += n_desc;
      cnt[2] += n_back;
      cnt[3] += n_tests;
      cnt[4] += n_hits;
    }
  };
  int32_t crow = __ldg(a.row_ptr + r), cend = __ldg(a.row_ptr + r + 1);
  if (check) clamp_row(a, crow, cend);
  float ray_tmax = 0.0f, best_t = 0.0f, best_u = -1.0f;
  int32_t best_seg = -1, best_leaf = -1;
  RayFrame rf{};
  if (crow < cend) {
    rf = load_ray<FAST>(a.rays, r, ray_tmax);
    best_t = ray_tmax;
  }
  const int rdepth = depth_of(a, r);
  int32_t j = crow;
  bool resume = false;
  if (MODE == kWalkResume) {
    best_t = w.best_t;
    best_u = w.best_u;
    best_seg = w.best_seg;
    best_leaf = w.best_leaf;
    j = w.j;
    resume = true;
  }
  int used = 0;  // node tests of this pass (kWalkFirst's budget)
  for (; j < cend; ++j) {
    const int32_t s = __ldg(a.seg_idx + j);
    float cand_t = ray_tmax, cand_u = -1.0f;
    int32_t cand_leaf = -1;
    uint32_t cand_flags = 0;  // FX_DEV_* bits of this pair (per-pair mode)
    const bool resumed = MODE == kWalkResume && resume;
    if (!resumed && !(s >= 0 && (!check || s < a.n_seg))) {
      atomicOr(a.status, FX_DEV_BAD_INDEX);
      if (PAIRS) {
        a.tu[j] = make_float2(kInf, -1.0f);
        if (a.leaf) a.leaf[j] = -1;
        if (a.pair_flags) a.pair_flags[j] = FX_DEV_BAD_INDEX;
      }
      continue;
    }
    // the candidate's pieces: the segment itself, or its pre-split pieces
    int32_t k = IDENTITY ? s : __ldg(a.piece_begin + s);
    const int32_t kend = IDENTITY ? s + 1 : __ldg(a.piece_begin + s + 1);
    if (resumed) k = w.piece;
    for (; k < kend; ++k) {
      const int32_t info = IDENTITY ? 0 : __ldg(a.piece_info + k);
      const uint32_t min_size = 1u << piece_min_size_shift(rdepth, info & 15);
      Node R, c;
      float tmin = 0.0f, tmax = PAIRS ? cand_t : best_t, root_r = 0.0f;
      uint32_t bits = 0, start = 0, size = kRootSize;
      bool slab_ok = false;
      int iters = 0;
      bool test = true;
      if (MODE == kWalkResume && resume) {
        // the saved walk of this piece; its root is rebuilt by the same
        // arithmetic as when the first pass began it
        resume = false;
        rotate_piece(a.piece, k, rf, R);
        c = w.c;
        tmin = w.tmin;
        tmax = w.tmax;
        root_r = w.root_r;
        bits = w.bits;
        start = w.start;
        size = w.size;
        slab_ok = w.slab_ok != 0u;
        iters = w.iters;
      } else {
        // bound test on the piece's root record: the sphere that holds the
        // root node's capped cylinder lies beyond t_max
        const float4 P = __ldg(a.piece_root + 2 * (int64_t)k), D = __ldg(a.piece_root + 2 * (int64_t)k + 1);
        const float px = P.x - rf.o.x, py = P.y - rf.o.y, pz = P.z - rf.o.z;
        const float zp = fmaf(px, rf.w.x, fmaf(py, rf.w.y, pz * rf.w.z));
        const float zd = fmaf(D.x, rf.w.x, fmaf(D.y, rf.w.y, D.z * rf.w.z));
        const float near = fmaf(0.5f, zd, zp) - D.w;
        if (COUNT) ++n_tests;
        if (near - kBoundSlack * (fabsf(zp) + fabsf(zd) + D.w) > tmax) test = false;
        root_r = P.w;
        if (test) {
          rotate_piece(a.piece, k, rf, R);
          c = R;
        }
      }
      if (!test) continue;
      for (;;) {
        if (MODE == kWalkFirst) {
          if (used == kBudget) {  // save the walk for the second pass
            w.c = c;
            w.tmin = tmin;
            w.tmax = tmax;
            w.root_r = root_r;
            w.best_t = best_t;
            w.best_u = best_u;
            w.ray = (int32_t)r;
            w.j = j;
            w.best_seg = best_seg;
            w.best_leaf = best_leaf;
            w.iters = iters;
            w.bits = bits;
            w.start = start;
            w.size = size;
            w.slab_ok = slab_ok ? 1u : 0u;
            w.piece = k;
            flush();
            return true;
          }
          ++used;
        }
        const float pair_tmax = PAIRS ? cand_t : best_t;
        const float rad = (iters == 0) ? root_r : cons_radius<FAST>(c);
        float c0 = 0.0f, c1 = 0.0f;
        bool over = cylinder<FAST>(c.p, c.d, rad, c0, c1);
        if (over && !slab_ok) {
          const float l = tmax;
          slab<FAST>(c, l, tmin, tmax);
          slab_ok = true;
        }
        over = over && fmaxf(c0, tmin) <= fminf(c1, tmax);
        ++iters;
        if (COUNT) ++n_nodes;
        if (over && size <= min_size) {
          const float t = fmaxf(c0, tmin);
          if (t < pair_tmax) {
            float u;
            int32_t lf;
            to_segment(info, leaf_u<FAST>(c, t, start, size), start, u, lf);
            if (!IDENTITY && info < 0) {
              atomicOr(a.status, FX_DEV_UNSUPPORTED);
              cand_flags |= FX_DEV_UNSUPPORTED;
            }
            if (PAIRS) {
              cand_t = t;
              cand_u = u;
              cand_leaf = lf;
            } else {
              best_t = t;
              best_u = u;
              best_seg = s;
              best_leaf = lf;
            }
            if (COUNT) ++n_hits;
          }
          break;
        } else if (over) {
          descend<FAST>(c, c0, c1, tmin, tmax, bits, start, size);
          if (COUNT) ++n_desc;
        } else if (bits == 0u) {
          break;
        } else {
          take_pending(bits, start, size);
          recompute(R, start, size, c);
          tmax = pair_tmax;
          slab_ok = false;
          if (COUNT) ++n_back;
        }
        if (iters >= iter_cap(rdepth)) {
          atomicOr(a.status, FX_DEV_ITER_LIMIT);
          cand_flags |= FX_DEV_ITER_LIMIT;
          break;
        }
      }
    }
    if (PAIRS) {
      a.tu[j] = make_float2(cand_t < ray_tmax ? cand_t : kInf, cand_u);
      if (a.leaf) a.leaf[j] = cand_leaf;
      if (a.pair_flags) a.pair_flags[j] = (uint8_t)cand_flags;
    }
  }
  if (!PAIRS) {
    const bool hit = best_seg >= 0;
    a.tu[r] = make_float2(hit ? best_t : kInf, hit ? best_u : -1.0f);
    a.seg[r] = best_seg;
    if (a.leaf) a.leaf[r] = best_leaf;
  }
  flush();
  return false;
}

template <bool COUNT>
__device__ __forceinline__ void add_counts(const TraceArgs& a, const uint32_t (&cnt)[5]) {
  if (!COUNT) return;
  unsigned long long v[5] = {cnt[0], cnt[1], cnt[2], cnt[3], cnt[4]};
  for (int k = 0; k < 5; ++k) {
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
    if ((threadIdx.x & 31) == 0 && v[k]) atomicAdd(a.counters + k, v[k]);
  }
}

__device__ __forceinline__ void store_walk(RayWalk* dst, const RayWalk& w) {
  const float4* src = reinterpret_cast<const float4*>(&w);
  float4* out = reinterpret_cast<float4*>(dst);
#pragma unroll
  for (int k = 0; k < 8; ++k) out[k] = src[k];
}

__device__ __forceinline__ void load_walk(const RayWalk* src, RayWalk& w) {
  const float4* in = reinterpret_cast<const float4*>(src);
  float4* dst = reinterpret_cast<float4*>(&w);
#pragma unroll
  for (int k = 0; k < 8; ++k) dst[k] = __ldg(in + k);
}

// One thread per ray, the whole walk (per-pair results, or closest hits in
// one pass).
template <bool FAST, bool PAIRS, bool COUNT, bool IDENTITY>
__global__ void __launch_bounds__(kRayBlock) k_ray(const TraceArgs a, int check) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t cnt[5] = {0, 0, 0, 0, 0};
  RayWalk w;
  if (r < a.n_ray) ray_walk<FAST, PAIRS, COUNT, IDENTITY, kWalkAll>(a, r, w, check, cnt);
  add_counts<COUNT>(a, cnt);
}

// First pass of closest hits.  A ray that runs out of budget takes a slot of
// the list (one atomic per warp; the list has a slot for every ray).
template <bool FAST, bool COUNT, bool IDENTITY>
__global__ void __launch_bounds__(kRayBlock) k_ray_first(const TraceArgs a, int check, RayDefer d) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t cnt[5] = {0, 0, 0, 0, 0};
  RayWalk w;
  bool defer = false;
  if (r < a.n_ray) defer = ray_walk<FAST, false, COUNT, IDENTITY, kWalkFirst>(a, r, w, check, cnt);
  const unsigned m = __ballot_sync(kFull, defer);
  if (m) {
    const int lane = threadIdx.x & 31, lead = __ffs(m) - 1;
    uint32_t off = 0;
    if (lane == lead) off = atomicAdd(d.count, (uint32_t)__popc(m));
    off = __shfl_sync(kFull, off, lead);
    const uint32_t slot = off + __popc(m & ((1u << lane) - 1u));
    if (defer && slot < d.capacity) store_walk(reinterpret_cast<RayWalk*>(d.walks) + slot, w);
  }
  add_counts<COUNT>(a, cnt);
}

// Second pass: the saved walks, one thread each, grid-stride over the list.
template <bool FAST, bool COUNT, bool IDENTITY>
__global__ void __launch_bounds__(kRayBlock) k_ray_resume(const TraceArgs a, int check, RayDefer d) {
  const uint32_t n = min(*d.count, d.capacity);
  uint32_t cnt[5] = {0, 0, 0, 0, 0};
  const uint32_t stride = gridDim.x * blockDim.x;
  // a warp-uniform trip count, so that the counters' shuffles see full warps
  const uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u);
  for (uint32_t i0 = base; i0 < n; i0 += stride) {
    const uint32_t i = i0 + (threadIdx.x & 31);
    if (i < n) {
      RayWalk w;
      load_walk(reinterpret_cast<const RayWalk*>(d.walks) + i, w);
      ray_walk<FAST, false, COUNT, IDENTITY, kWalkResume>(a, w.ray, w, check, cnt);
    }
  }
  add_counts<COUNT>(a, cnt);
}

template <bool FAST, bool PAIRS, bool COUNT, bool IDENTITY>
cudaError_t launch_r(const TraceArgs& a, int check, const RayDefer& d, int sms, cudaStream_t s) {
  const int64_t grid = (a.n_ray + kRayBlock - 1) / kRayBlock;
  if (PAIRS || !d.walks) {
    k_ray<FAST, PAIRS, COUNT, IDENTITY><<<(unsigned)grid, kRayBlock, 0, s>>>(a, check);
    return cudaGetLastError();
  }
  k_ray_first<FAST, COUNT, IDENTITY><<<(unsigned)grid, kRayBlock, 0, s>>>(a, check, d);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  // the saved walks are a small share of the rays: 8 blocks per SM at most
  const int64_t grid2 = std::min<int64_t>(grid, (int64_t)sms * 8);
  k_ray_resume<FAST, COUNT, IDENTITY><<<(unsigned)grid2, kRayBlock, 0, s>>>(a, check, d);
  return cudaGetLastError();
}

template <bool FAST, bool PAIRS, bool COUNT>
cudaError_t launch_r1(const TraceArgs& a, int check, const RayDefer& d, int sms, cudaStream_t s) {
  return a.identity ? launch_r<FAST, PAIRS, COUNT, true>(a, check, d, sms, s)
                    : launch_r<FAST, PAIRS, COUNT, false>(a, check, d, sms, s);
}

template <bool FAST, bool PAIRS>
cudaError_t launch_r2(const TraceArgs& a, uint32_t flags, const RayDefer& d, int sms, cudaStream_t s) {
  const int chk = (flags & FX_CHECK_INDEX) ? 1 : 0;
  return (flags & FX_COUNT) ? launch_r1<FAST, PAIRS, true>(a, chk, d, sms, s)
                            : launch_r1<FAST, PAIRS, false>(a, chk, d, sms, s);
}

}  // namespace

size_t ray_walk_bytes() { return sizeof(RayWalk); }

cudaError_t launch_ray(const TraceArgs& a, bool pairs, uint32_t flags, const RayDefer& d, int sm_count,
                       cudaStream_t s) {
  if (a.n_ray == 0) return cudaSuccess;
  const bool fast = flags & FX_FAST_MATH;
  if (pairs)
    return fast ? launch_r2<true, true>(a, flags, d, sm_count, s) : launch_r2<false, true>(a, flags, d, sm_count, s);
  return fast ? launch_r2<true, false>(a, flags, d, sm_count, s) : launch_r2<false, false>(a, flags, d, sm_count, s);
}

}  // namespace fx
