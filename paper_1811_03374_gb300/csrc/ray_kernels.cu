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
// than the traversal.  Handles whose segments are single level-0 pieces
// only; others run the lane kernel.
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

__device__ __forceinline__ void rotate_piece(const float4* __restrict__ piece, int32_t k, const RayFrame& r,
                                             Node& n) {
  const float4 p = __ldg(piece + 4 * (int64_t)k), d = __ldg(piece + 4 * (int64_t)k + 1);
  const float4 t0 = __ldg(piece + 4 * (int64_t)k + 2), t1 = __ldg(piece + 4 * (int64_t)k + 3);
  n.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
  n.d = rotate(r, d.x, d.y, d.z, d.w);
  n.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
  n.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
}

template <bool FAST, bool PAIRS, bool COUNT>
__global__ void __launch_bounds__(kRayBlock) k_ray(const TraceArgs a, int check) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  uint32_t n_nodes = 0, n_desc = 0, n_back = 0, n_tests = 0, n_hits = 0;
  if (r < a.n_ray) {
    const int32_t crow = __ldg(a.row_ptr + r), cend = __ldg(a.row_ptr + r + 1);
    float ray_tmax = 0.0f, best_t = 0.0f, best_u = -1.0f;
    int32_t best_seg = -1, best_leaf = -1;
    RayFrame rf{};
    if (crow < cend) {
      rf = load_ray<FAST>(a.rays, r, ray_tmax);
      best_t = ray_tmax;
    }
    const int min_size = 1 << piece_min_size_shift(a.depth, 0);
    for (int32_t j = crow; j < cend; ++j) {
      const int32_t s = __ldg(a.seg_idx + j);
      float cand_t = ray_tmax, cand_u = -1.0f;
      int32_t cand_leaf = -1;
      const float lim = PAIRS ? ray_tmax : best_t;
      bool test = s >= 0 && (!check || s < a.n_seg);
      if (!test) atomicOr(a.status, FX_DEV_BAD_INDEX);
      float root_r = 0.0f;
      if (test) {
        // bound test on the root record: the sphere that holds the root
        // node's capped cylinder lies beyond t_max
        const float4 P = __ldg(a.piece_root + 2 * (int64_t)s), D = __ldg(a.piece_root + 2 * (int64_t)s + 1);
        const float px = P.x - rf.o.x, py = P.y - rf.o.y, pz = P.z - rf.o.z;
        const float zp = fmaf(px, rf.w.x, fmaf(py, rf.w.y, pz * rf.w.z));
        const float zd = fmaf(D.x, rf.w.x, fmaf(D.y, rf.w.y, D.z * rf.w.z));
        const float near = fmaf(0.5f, zd, zp) - D.w;
        if (COUNT) ++n_tests;
        if (near - kBoundSlack * (fabsf(zp) + fabsf(zd) + D.w) > lim) test = false;
        root_r = P.w;
      }
      if (test) {
        Node R, c;
        rotate_piece(a.piece, s, rf, R);
        c = R;
        float tmin = 0.0f, tmax = lim;
        uint32_t bits = 0, start = 0, size = kRootSize;
        bool slab_ok = false;
        for (int iters = 0;;) {
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
          if (over && size <= (uint32_t)min_size) {
            const float t = fmaxf(c0, tmin);
            if (t < pair_tmax) {
              float u;
              int32_t lf;
              to_segment(0, leaf_u<FAST>(c, t, start, size), start, u, lf);
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
            jump_up(bits, start, size);
            recompute(R, start, size, c);
            tmax = pair_tmax;
            slab_ok = false;
            if (COUNT) ++n_back;
          }
          if (iters >= iter_cap(a.depth)) {
            atomicOr(a.status, FX_DEV_ITER_LIMIT);
            break;
          }
        }
      }
      if (PAIRS) {
        a.tu[j] = make_float2(cand_t < ray_tmax ? cand_t : kInf, cand_u);
        if (a.leaf) a.leaf[j] = cand_leaf;
      }
    }
    if (!PAIRS) {
      const bool hit = best_seg >= 0;
      a.tu[r] = make_float2(hit ? best_t : kInf, hit ? best_u : -1.0f);
      a.seg[r] = best_seg;
      if (a.leaf) a.leaf[r] = best_leaf;
    }
  }
  if (COUNT) {
    unsigned long long v[5] = {n_nodes, n_desc, n_back, n_tests, n_hits};
    for (int k = 0; k < 5; ++k) {
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
      if ((threadIdx.x & 31) == 0 && v[k]) atomicAdd(a.counters + k, v[k]);
    }
  }
}

template <bool FAST, bool PAIRS, bool COUNT>
cudaError_t launch_r(const TraceArgs& a, int check, cudaStream_t s) {
  const int64_t grid = (a.n_ray + kRayBlock - 1) / kRayBlock;
  k_ray<FAST, PAIRS, COUNT><<<(unsigned)grid, kRayBlock, 0, s>>>(a, check);
  return cudaGetLastError();
}

template <bool FAST, bool PAIRS>
cudaError_t launch_r2(const TraceArgs& a, uint32_t flags, cudaStream_t s) {
  const int chk = (flags & FX_CHECK_INDEX) ? 1 : 0;
  return (flags & FX_COUNT) ? launch_r<FAST, PAIRS, true>(a, chk, s) : launch_r<FAST, PAIRS, false>(a, chk, s);
}

}  // namespace

cudaError_t launch_ray(const TraceArgs& a, bool pairs, uint32_t flags, cudaStream_t s) {
  if (a.n_ray == 0) return cudaSuccess;
  const bool fast = flags & FX_FAST_MATH;
  if (pairs) return fast ? launch_r2<true, true>(a, flags, s) : launch_r2<false, true>(a, flags, s);
  return fast ? launch_r2<true, false>(a, flags, s) : launch_r2<false, false>(a, flags, s);
}

}  // namespace fx
