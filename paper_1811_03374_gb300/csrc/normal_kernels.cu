// normal_kernels.cu -- hit normals (App. C, the routine that computes the
// intersection's u and normal), as a pass over the closest-hit results of
// any traversal kernel: one thread per ray.
//
// The hit leaf is rebuilt in the ray frame from the root node of the piece
// that holds it (the power-form recomputation of Sec. 3.3, as after a
// backtrack); the hit point (0, 0, t) is projected onto the leaf axis and
// u_local clamped to [0, 1].  A lateral hit's normal is the hit point minus
// the axis point p + u_local d, taken back to world space and normalised.
// An end-cap hit -- the first (last) leaf, with the hit point on or beyond
// the segment's end plane through p0 with normal p1 - p0 (through p3, normal
// p3 - p2), to within the FP32 spacing of ray-frame coordinates, 8 ulp of
// (t + |p0|) -- gets the outward disk normal p0 - p1 (p3 - p2), normalised.
// (The paper's listing takes u == 0 or u == 1 for a cap, which decides a hit
// on the disk by the rounding of its projection.)  Misses get (0, 0, 0), and
// so do entries whose segment or leaf is out of range (flagged as a bad
// index).
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr int kNormalBlock = 256;

__device__ __forceinline__ float3 sub3(const float3& a, const float3& b) {
  return make_float3(a.x - b.x, a.y - b.y, a.z - b.z);
}
__device__ __forceinline__ float dot3f(const float3& a, const float3& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

template <bool FAST>
__device__ __forceinline__ float3 unit(const float3& v) {
  const float l2 = dot3f(v, v);
  if (!(l2 > 0.0f)) return make_float3(0.0f, 0.0f, 0.0f);
  const float inv = FAST ? rsqrtf(l2) : __frcp_rn(__fsqrt_rn(l2));
  return make_float3(v.x * inv, v.y * inv, v.z * inv);
}

template <bool FAST>
__global__ void __launch_bounds__(kNormalBlock) k_normals(const TraceArgs a, const float4* __restrict__ seg_cp,
                                                          float* __restrict__ normal) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n_ray) return;
  int32_t s = a.seg[r];
  const int32_t leaf = s >= 0 ? a.leaf[r] : -1;
  if (s >= a.n_seg || (s >= 0 && (leaf < 0 || leaf >= (int32_t)kRootSize))) {
    atomicOr(a.status, FX_DEV_BAD_INDEX);  // not a result of intersect_closest
    s = -1;
  }
  float3 n = make_float3(0.0f, 0.0f, 0.0f);
  if (s >= 0) {
    const float t = a.tu[r].x;
    // the piece holding the leaf: its level, its first leaf (segment units)
    int32_t k = s, lvl = 0, off = 0;
    if (!a.identity) {
      const int pb = __ldg(a.piece_begin + s), pe = __ldg(a.piece_begin + s + 1);
      k = pb;
      for (int q = pb; q < pe; ++q) {
        const int32_t info = __ldg(a.piece_info + q);
        const int ql = info & 15, qo = (info >> 4) & 0x7ffff;
        if (leaf >= (qo << (23 - ql)) && leaf < ((qo + 1) << (23 - ql))) {
          k = q;
          lvl = ql;
          off = qo;
          break;
        }
      }
    }
    const uint32_t start = (uint32_t)(leaf - (off << (23 - lvl))) << lvl;
    const uint32_t size = 1u << piece_min_size_shift(depth_of(a, r), lvl);
    const uint32_t seg_size = size >> lvl;  // the leaf's size in segment units
    float tmax_unused;
    const RayFrame rf = load_ray<FAST>(a.rays, r, tmax_unused);
    Node R;
    {
      const float4 p = __ldg(a.piece + 4 * (int64_t)k), d = __ldg(a.piece + 4 * (int64_t)k + 1);
      const float4 t0 = __ldg(a.piece + 4 * (int64_t)k + 2), t1 = __ldg(a.piece + 4 * (int64_t)k + 3);
      R.p = rotate(rf, p.x - rf.o.x, p.y - rf.o.y, p.z - rf.o.z, p.w);
      R.d = rotate(rf, d.x, d.y, d.z, d.w);
      R.t0 = rotate(rf, t0.x, t0.y, t0.z, t0.w);
      R.t1 = rotate(rf, t1.x, t1.y, t1.z, t1.w);
    }
    Node c = R;
    if (size < kRootSize) recompute(R, start, size, c);
    // projection of the hit point onto the leaf axis
    const float dd = dot3(c.d, c.d);
    float ul = 0.0f;
    if (dd > 0.0f) {
      const float num = fmaf(-c.p.x, c.d.x, fmaf(-c.p.y, c.d.y, (t - c.p.z) * c.d.z));
      ul = fminf(1.0f, fmaxf(0.0f, fdiv<FAST>(num, dd)));
    }
    // end caps of the segment (its control points in world space)
    bool cap0 = false, cap1 = false;
    float3 P0, P1, P2, P3;
    if (leaf == 0 || leaf + (int32_t)seg_size == (int32_t)kRootSize) {
      const float4 q0 = __ldg(seg_cp + 4 * (int64_t)s), q1 = __ldg(seg_cp + 4 * (int64_t)s + 1);
      const float4 q2 = __ldg(seg_cp + 4 * (int64_t)s + 2), q3 = __ldg(seg_cp + 4 * (int64_t)s + 3);
      P0 = make_float3(q0.x, q0.y, q0.z);
      P1 = make_float3(q1.x, q1.y, q1.z);
      P2 = make_float3(q2.x, q2.y, q2.z);
      P3 = make_float3(q3.x, q3.y, q3.z);
      // the hit point relative to p0 (p3) as t w - (p0 - o): differences
      // from the ray origin, at the scale of t as in the ray frame
      const float3 d0 = sub3(P0, rf.o), d3 = sub3(P3, rf.o);
      const float tol = 8.0f * 0x1p-24f * (t + sqrtf(dot3f(d0, d0)));
      if (leaf == 0) {
        const float3 a0 = sub3(P0, P1);
        const float3 x0 = make_float3(fmaf(t, rf.w.x, -d0.x), fmaf(t, rf.w.y, -d0.y), fmaf(t, rf.w.z, -d0.z));
        const float l = sqrtf(dot3f(a0, a0));
        cap0 = l > 0.0f && dot3f(x0, a0) >= -tol * l;
      }
      if (!cap0 && leaf + (int32_t)seg_size == (int32_t)kRootSize) {
        const float3 a1 = sub3(P3, P2);
        const float3 x3 = make_float3(fmaf(t, rf.w.x, -d3.x), fmaf(t, rf.w.y, -d3.y), fmaf(t, rf.w.z, -d3.z));
        const float l = sqrtf(dot3f(a1, a1));
        cap1 = l > 0.0f && dot3f(x3, a1) >= -tol * l;
      }
    }
    if (cap0) {
      n = unit<FAST>(sub3(P0, P1));
    } else if (cap1) {
      n = unit<FAST>(sub3(P3, P2));
    } else {
      const float ax = fmaf(ul, c.d.x, c.p.x), ay = fmaf(ul, c.d.y, c.p.y), az = fmaf(ul, c.d.z, c.p.z);
      const float vx = -ax, vy = -ay, vz = t - az;
      n = unit<FAST>(make_float3(fmaf(vx, rf.e1.x, fmaf(vy, rf.e2.x, vz * rf.w.x)),
                                 fmaf(vx, rf.e1.y, fmaf(vy, rf.e2.y, vz * rf.w.y)),
                                 fmaf(vx, rf.e1.z, fmaf(vy, rf.e2.z, vz * rf.w.z))));
    }
  }
  normal[3 * r] = n.x;
  normal[3 * r + 1] = n.y;
  normal[3 * r + 2] = n.z;
}

}  // namespace

cudaError_t launch_normals(const TraceArgs& a, const float4* seg_cp, float* normal, uint32_t flags,
                           cudaStream_t s) {
  if (a.n_ray == 0) return cudaSuccess;
  const unsigned grid = (unsigned)((a.n_ray + kNormalBlock - 1) / kNormalBlock);
  if (flags & FX_FAST_MATH) k_normals<true><<<grid, kNormalBlock, 0, s>>>(a, seg_cp, normal);
  else k_normals<false><<<grid, kNormalBlock, 0, s>>>(a, seg_cp, normal);
  return cudaGetLastError();
}

}  // namespace fx
