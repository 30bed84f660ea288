// count_kernels.cu -- per-ray pruning-test counts (Fig. 8: oriented bounding
// cylinders against axis-aligned boxes in the ray's frame), one thread per
// ray.
//
// Each ray's candidates are searched in row order with the closest hit so
// far as t_max and no test before the root's, so only the bounding volume
// differs between the two modes:
//   - cylinders: the traversal of Sec. 3.3; one count per node tested;
//   - boxes: the same subdivision without partition planes.  A node's box is
//     [min_k (q_k - r_k), max_k (q_k + r_k)] over its four control points
//     q_k and radii r_k; it is hit if it contains the ray's axis and meets
//     [0, t_max] in z.  At a hit inner node both children's boxes are tested
//     (two counts) and the one with the smaller z_min is searched first (the
//     left one on a tie); the other is recorded in the bit string and tested
//     again (one count) when taken up after the first one's subtree.  The
//     search does not end at the first leaf hit; a leaf whose box is hit
//     takes the capped-cylinder leaf test of Sec. 3.3.
// A pre-split segment's pieces are searched in order, each to depth - level
// (its leaves are the unsplit curve's), with the closest hit so far as t_max.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr int kCountBlock = 128;

// Ray-frame box of a node's control points dilated by their radii.
__device__ __forceinline__ void node_box(const Node& c, float lo[3], float hi[3]) {
  const float4 q0 = c.p;
  const float4 q1 = make_float4(c.p.x + c.t0.x, c.p.y + c.t0.y, c.p.z + c.t0.z, c.p.w + c.t0.w);
  const float4 q3 = make_float4(c.p.x + c.d.x, c.p.y + c.d.y, c.p.z + c.d.z, c.p.w + c.d.w);
  const float4 q2 = make_float4(q3.x - c.t1.x, q3.y - c.t1.y, q3.z - c.t1.z, q3.w - c.t1.w);
  lo[0] = fminf(fminf(q0.x - q0.w, q1.x - q1.w), fminf(q2.x - q2.w, q3.x - q3.w));
  hi[0] = fmaxf(fmaxf(q0.x + q0.w, q1.x + q1.w), fmaxf(q2.x + q2.w, q3.x + q3.w));
  lo[1] = fminf(fminf(q0.y - q0.w, q1.y - q1.w), fminf(q2.y - q2.w, q3.y - q3.w));
  hi[1] = fmaxf(fmaxf(q0.y + q0.w, q1.y + q1.w), fmaxf(q2.y + q2.w, q3.y + q3.w));
  lo[2] = fminf(fminf(q0.z - q0.w, q1.z - q1.w), fminf(q2.z - q2.w, q3.z - q3.w));
  hi[2] = fmaxf(fmaxf(q0.z + q0.w, q1.z + q1.w), fmaxf(q2.z + q2.w, q3.z + q3.w));
}

__device__ __forceinline__ bool box_hit(const Node& c, float tmax, float& zmin) {
  float lo[3], hi[3];
  node_box(c, lo, hi);
  zmin = lo[2];
  return lo[0] <= 0.0f && hi[0] >= 0.0f && lo[1] <= 0.0f && hi[1] >= 0.0f && hi[2] >= 0.0f && lo[2] <= tmax;
}

// The two children of c (Sec. 3.1 subdivision rules).
__device__ __forceinline__ void children(const Node& c, Node& L, Node& R) {
  float4 dp, tc;
  dp.x = fmaf(0.375f, c.t0.x - c.t1.x, 0.5f * c.d.x);
  dp.y = fmaf(0.375f, c.t0.y - c.t1.y, 0.5f * c.d.y);
  dp.z = fmaf(0.375f, c.t0.z - c.t1.z, 0.5f * c.d.z);
  dp.w = fmaf(0.375f, c.t0.w - c.t1.w, 0.5f * c.d.w);
  tc.x = fmaf(-0.125f, c.t0.x + c.t1.x, 0.25f * c.d.x);
  tc.y = fmaf(-0.125f, c.t0.y + c.t1.y, 0.25f * c.d.y);
  tc.z = fmaf(-0.125f, c.t0.z + c.t1.z, 0.25f * c.d.z);
  tc.w = fmaf(-0.125f, c.t0.w + c.t1.w, 0.25f * c.d.w);
  L.p = c.p;
  L.d = dp;
  L.t0 = make_float4(0.5f * c.t0.x, 0.5f * c.t0.y, 0.5f * c.t0.z, 0.5f * c.t0.w);
  L.t1 = tc;
  R.p = make_float4(c.p.x + dp.x, c.p.y + dp.y, c.p.z + dp.z, c.p.w + dp.w);
  R.d = make_float4(c.d.x - dp.x, c.d.y - dp.y, c.d.z - dp.z, c.d.w - dp.w);
  R.t0 = tc;
  R.t1 = make_float4(0.5f * c.t1.x, 0.5f * c.t1.y, 0.5f * c.t1.z, 0.5f * c.t1.w);
}

// The capped-cylinder leaf test of the traversal.
template <bool FAST>
__device__ __forceinline__ bool leaf_test(const Node& c, float tmax, float& t) {
  float tmin, tm;
  slab<FAST>(c, tmax, tmin, tm);
  float c0 = 0.0f, c1 = 0.0f;
  if (!(cylinder<FAST>(c.p, c.d, cons_radius<FAST>(c), c0, c1) && fmaxf(c0, tmin) <= fminf(c1, tm))) return false;
  t = fmaxf(c0, tmin);
  return t < tmax;
}

// Box-pruned search of one piece (root node R in the ray frame) with t_max
// best; adds its box tests to n and returns the closest t (best if none).
// A leaf counts only its box test; the cap keeps a runaway ray finite.
template <bool FAST>
__device__ float box_search(const Node& R, uint32_t min_size, float best, uint64_t& n, uint32_t* status) {
  float zmin;
  ++n;
  if (!box_hit(R, best, zmin)) return best;
  Node c = R;
  uint32_t bits = 0, start = 0, size = kRootSize;
  uint64_t steps = 0;
  for (;;) {
    bool next = false;  // c is a node whose box is hit, to be expanded
    if (size <= min_size) {
      float t;
      if (leaf_test<FAST>(c, best, t)) best = t;
    } else {
      Node L, Rc;
      children(c, L, Rc);
      float zl, zr;
      n += 2;
      const bool hl = box_hit(L, best, zl), hr = box_hit(Rc, best, zr);
      if (hl || hr) {
        const bool right = hl && hr ? zr < zl : hr;
        size >>= 1;
        if (hl && hr) bits |= size;
        if (right) start |= size;
        c = right ? Rc : L;
        next = true;
      }
    }
    // take up the deepest deferred sibling, tested again against t_max
    while (!next && bits != 0u) {
      take_pending(bits, start, size);
      recompute(R, start, size, c);
      ++n;
      next = box_hit(c, best, zmin);
    }
    if (!next) break;
    if (++steps > (1ull << 26)) {  // far beyond any depth <= 23 search of one piece
      atomicOr(status, FX_DEV_ITER_LIMIT);
      break;
    }
  }
  return best;
}

template <bool FAST, bool BOX>
__global__ void __launch_bounds__(kCountBlock) k_counts(const TraceArgs a, uint32_t* __restrict__ counts,
                                                        int check) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n_ray) return;
  int32_t crow = __ldg(a.row_ptr + r), cend = __ldg(a.row_ptr + r + 1);
  if (check) clamp_row(a, crow, cend);
  uint64_t n = 0;
  if (crow < cend) {
    float ray_tmax;
    const RayFrame rf = load_ray<FAST>(a.rays, r, ray_tmax);
    float best = ray_tmax;
    for (int32_t j = crow; j < cend; ++j) {
      const int32_t s = __ldg(a.seg_idx + j);
      if (s < 0 || (check && s >= a.n_seg)) {
        atomicOr(a.status, FX_DEV_BAD_INDEX);
        continue;
      }
      const int32_t pb = a.identity ? s : __ldg(a.piece_begin + s);
      const int32_t pe = a.identity ? s + 1 : __ldg(a.piece_begin + s + 1);
      for (int32_t k = pb; k < pe; ++k) {
        const int32_t info = a.identity ? 0 : __ldg(a.piece_info + k);
        PairState st;
        begin_piece<FAST>(st, a.piece, k, rf, info, a.depth, best);
        if (BOX) {
          best = box_search<FAST>(st.R, st.min_size, best, n, a.status);
        } else {
          unsigned long long nd = 0, nb = 0;
          for (;;) {
            float t;
            const StepResult res = node_step<FAST, false>(st, best, t, nd, nb);
            ++n;
            if (res == kStepLeaf) {
              if (t < best) best = t;
              break;
            }
            if (res == kStepDone) break;
            if (st.iters >= iter_cap(a.depth)) {
              atomicOr(a.status, FX_DEV_ITER_LIMIT);
              break;
            }
          }
        }
      }
    }
  }
  counts[r] = n > 0xffffffffull ? 0xffffffffu : (uint32_t)n;
}

}  // namespace

cudaError_t launch_counts(const TraceArgs& a, uint32_t* counts, bool box, uint32_t flags, cudaStream_t s) {
  if (a.n_ray == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.n_ray + kCountBlock - 1) / kCountBlock);
  const int chk = (flags & FX_CHECK_INDEX) ? 1 : 0;
  const bool fast = flags & FX_FAST_MATH;
  if (box) {
    if (fast) k_counts<true, true><<<grid, kCountBlock, 0, s>>>(a, counts, chk);
    else k_counts<false, true><<<grid, kCountBlock, 0, s>>>(a, counts, chk);
  } else {
    if (fast) k_counts<true, false><<<grid, kCountBlock, 0, s>>>(a, counts, chk);
    else k_counts<false, false><<<grid, kCountBlock, 0, s>>>(a, counts, chk);
  }
  return cudaGetLastError();
}

}  // namespace fx
