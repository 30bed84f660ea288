// backward.cu -- adjoint of the closest hit's distance t with respect to the
// segments' control points and radii (hand-written, FP32).
//
// The leaf cylinders converge, as the depth grows, to the sweep of circles of
// radius r(u) in the planes normal to c'(u) (Sec. 3.2: the cylinders' limit
// surface), closed by flat end disks.  A hit x = o + t w satisfies
//   G1(t, u) = <x - c(u), c'(u)> = 0,   G2(t, u) = |x - c(u)|^2 - r(u)^2 = 0.
// The forward (t, u) is refined by Newton steps on G; then the implicit
// function theorem gives dt/dtheta = -[J^-1 dG/dtheta]_t with
//   J = [[<w, c'>, <x - c, c''> - |c'|^2], [2 <x - c, w>, -2 <x - c, c'> - 2 r r']],
//   dG1/dp_k = -B_k c' + B_k' (x - c),  dG2/dp_k = -2 B_k (x - c),
//   dG2/dr_k = -2 r B_k.
// Two candidates are formed from the forward (t, u): a lateral hit, refined
// by Newton steps, valid if u stays in [0, 1]; and a hit of the end disk at
// the nearer end (u fixed at 0 or 1, t from the disk's plane, G1 alone),
// valid if the point lies in the disk.  Each must stay close to the forward
// t; of the valid ones, the one nearer along the ray is the hit.  The forward u cannot tell a lateral
// hit near an end from the disk in FP32 (u = 1 - 5e-8 rounds to 1), so the
// classification is geometric.
// One thread per ray; contributions are added to grad_cps with atomics.
//
// Quadratic segments (App. B.1) are stored as their degree elevation,
// q0 = p0, q1 = (p0 + 2 p1) / 3, q2 = (2 p1 + p2) / 3, q3 = p2 (the same
// curve), so the adjoint is first formed with respect to q0..q3 and then
// carried to p0..p2 by the chain rule through that linear map:
// dL/dp0 = g0 + g1 / 3, dL/dp1 = 2 (g1 + g2) / 3, dL/dp2 = g2 / 3 + g3.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace fx {
namespace {

struct V4 {
  float x, y, z, w;
};

__device__ __forceinline__ V4 ld(const float4* p) {
  const float4 v = __ldg(p);
  return V4{v.x, v.y, v.z, v.w};
}
__device__ __forceinline__ float d3(const V4& a, const V4& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

// Exact difference a - b as hi + lo (Knuth's TwoSum).
__device__ __forceinline__ void two_diff(float a, float b, float& hi, float& lo) {
  hi = a - b;
  const float bb = hi - a;
  lo = (a - (hi - bb)) - (b + bb);
}

template <bool QUAD>
__global__ void __launch_bounds__(256)
    k_backward(const float4* __restrict__ cp, const float4* __restrict__ rays, int64_t n_ray,
               const float2* __restrict__ tu, const int32_t* __restrict__ seg,
               const float* __restrict__ grad_t, float* __restrict__ grad_cps,
               unsigned long long* n_skipped) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_ray) return;
  const int32_t s = seg[r];
  if (s < 0) return;
  const float gw = grad_t[r];
  if (gw == 0.0f) return;  // contributes nothing
  const float4 ra = __ldg(rays + 2 * r), rb = __ldg(rays + 2 * r + 1);
  const float inv = __frcp_rn(__fsqrt_rn(fmaf(rb.x, rb.x, fmaf(rb.y, rb.y, rb.z * rb.z))));
  const V4 w{rb.x * inv, rb.y * inv, rb.z * inv, 0.0f};
  const V4 P0 = ld(cp + 4 * s), P1 = ld(cp + 4 * s + 1), P2 = ld(cp + 4 * s + 2), P3 = ld(cp + 4 * s + 3);
  // everything relative to p0; o - p0 kept as an exact hi + lo pair
  V4 oh, ol;
  two_diff(ra.x, P0.x, oh.x, ol.x);
  two_diff(ra.y, P0.y, oh.y, ol.y);
  two_diff(ra.z, P0.z, oh.z, ol.z);
  // power form around p0: c(u) - p0 = A1 u + A2 u^2 + A3 u^3 (all four components)
  const V4 D0{P1.x - P0.x, P1.y - P0.y, P1.z - P0.z, P1.w - P0.w};
  const V4 D1{P2.x - P1.x, P2.y - P1.y, P2.z - P1.z, P2.w - P1.w};
  const V4 D2{P3.x - P2.x, P3.y - P2.y, P3.z - P2.z, P3.w - P2.w};
  const V4 A1{3.f * D0.x, 3.f * D0.y, 3.f * D0.z, 3.f * D0.w};
  const V4 A2{3.f * (D1.x - D0.x), 3.f * (D1.y - D0.y), 3.f * (D1.z - D0.z), 3.f * (D1.w - D0.w)};
  const V4 A3{D2.x - 2.f * D1.x + D0.x, D2.y - 2.f * D1.y + D0.y, D2.z - 2.f * D1.z + D0.z,
              D2.w - 2.f * D1.w + D0.w};
  const float t_fwd = tu[r].x, u_fwd = tu[r].y;
  // Newton may leave the forward hit for another root of G (the exit through
  // the lateral surface of a ray that entered through an end disk): a
  // candidate counts only within tol of the forward t, a tenth of the largest
  // control radius, far below the distance between entry and exit except for
  // grazing rays, whose system is singular anyway.
  const float tol = 0.1f * fmaxf(fmaxf(P0.w, P1.w), fmaxf(P2.w, P3.w));

  V4 c, c1, c2, e;
  float J00 = 0.f, J01 = 0.f, J10 = 0.f, J11 = 0.f;
  auto evaluate = [&](float uu, float tt) {
    c.x = uu * fmaf(uu, fmaf(uu, A3.x, A2.x), A1.x);
    c.y = uu * fmaf(uu, fmaf(uu, A3.y, A2.y), A1.y);
    c.z = uu * fmaf(uu, fmaf(uu, A3.z, A2.z), A1.z);
    c.w = fmaf(uu, fmaf(uu, fmaf(uu, A3.w, A2.w), A1.w), P0.w);  // r(u)
    c1.x = fmaf(uu, fmaf(3.f * uu, A3.x, 2.f * A2.x), A1.x);
    c1.y = fmaf(uu, fmaf(3.f * uu, A3.y, 2.f * A2.y), A1.y);
    c1.z = fmaf(uu, fmaf(3.f * uu, A3.z, 2.f * A2.z), A1.z);
    c1.w = fmaf(uu, fmaf(3.f * uu, A3.w, 2.f * A2.w), A1.w);
    c2.x = fmaf(6.f * uu, A3.x, 2.f * A2.x);
    c2.y = fmaf(6.f * uu, A3.y, 2.f * A2.y);
    c2.z = fmaf(6.f * uu, A3.z, 2.f * A2.z);
    e.x = (fmaf(tt, w.x, oh.x) - c.x) + ol.x;
    e.y = (fmaf(tt, w.y, oh.y) - c.y) + ol.y;
    e.z = (fmaf(tt, w.z, oh.z) - c.z) + ol.z;
    J00 = d3(w, c1);
    J01 = d3(e, c2) - d3(c1, c1);
    J10 = 2.f * d3(e, w);
    J11 = -2.f * d3(e, c1) - 2.f * c.w * c1.w;
  };
  // candidate 1: the lateral surface, Newton steps from the forward hit
  float tl = t_fwd, ul = fminf(fmaxf(u_fwd, 1e-6f), 1.0f - 1e-6f);
  bool lateral = true;
  for (int it = 0; it < 5; ++it) {
    evaluate(ul, tl);
    const float G1 = d3(e, c1), G2 = d3(e, e) - c.w * c.w;
    const float det = J00 * J11 - J01 * J10;
    if (!(fabsf(det) > 0.0f)) {
      lateral = false;
      break;
    }
    const float id = __frcp_rn(det);
    tl -= (J11 * G1 - J01 * G2) * id;
    ul -= (J00 * G2 - J10 * G1) * id;
  }
  lateral = lateral && ul >= 0.0f && ul <= 1.0f && fabsf(tl - t_fwd) <= tol;
  // candidate 2: the end disk at the end nearer to the forward u (u fixed,
  // t where the ray meets the disk's plane, inside the disk)
  const float ue = u_fwd >= 0.5f ? 1.0f : 0.0f;
  evaluate(ue, t_fwd);
  bool disk = fabsf(J00) > 1e-7f * sqrtf(d3(c1, c1));
  float td = t_fwd;
  if (disk) {
    td = t_fwd - d3(e, c1) / J00;  // G1 is linear in t
    evaluate(ue, td);
    disk = d3(e, e) <= c.w * c.w * 1.0001f && fabsf(td - t_fwd) <= tol;
  }
  // of the valid candidates, the one nearer along the ray is the hit
  float t, u, a1 = 0.f, a2 = 0.f;  // dt/dtheta = -(a1 dG1/dtheta + a2 dG2/dtheta)
  bool ok;
  if (lateral && (!disk || tl <= td)) {
    t = tl;
    u = ul;
    evaluate(u, t);
    const float det = J00 * J11 - J01 * J10;
    ok = fabsf(det) > 1e-5f * (fabsf(J00 * J11) + fabsf(J01 * J10));
    if (ok) {
      const float id = __frcp_rn(det);
      a1 = J11 * id;
      a2 = -J01 * id;
    }
  } else {
    t = td;
    u = ue;
    ok = disk;
    if (ok) {
      evaluate(u, t);
      a1 = __frcp_rn(J00);
    }
  }
  if (!ok) {
    if (n_skipped) atomicAdd(n_skipped, 1ull);
    return;
  }
  const float v = 1.0f - u;
  const float B[4] = {v * v * v, 3.f * u * v * v, 3.f * u * u * v, u * u * u};
  const float dB[4] = {-3.f * v * v, 3.f * v * v - 6.f * u * v, 6.f * u * v - 3.f * u * u, 3.f * u * u};
  // dL/dq_k of the (stored) cubic control points
  float gq[4][4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float gx = dB[k] * e.x - B[k] * c1.x, gy = dB[k] * e.y - B[k] * c1.y,
                gz = dB[k] * e.z - B[k] * c1.z;
    const float hb = -2.f * B[k];
    gq[k][0] = -gw * (a1 * gx + a2 * hb * e.x);
    gq[k][1] = -gw * (a1 * gy + a2 * hb * e.y);
    gq[k][2] = -gw * (a1 * gz + a2 * hb * e.z);
    gq[k][3] = -gw * (a2 * hb * c.w);
  }
  if (QUAD) {
    float* g = grad_cps + 12 * (int64_t)s;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      atomicAdd(g + a, fmaf(gq[1][a], 1.f / 3.f, gq[0][a]));
      atomicAdd(g + 4 + a, (2.f / 3.f) * (gq[1][a] + gq[2][a]));
      atomicAdd(g + 8 + a, fmaf(gq[2][a], 1.f / 3.f, gq[3][a]));
    }
  } else {
    float* g = grad_cps + 16 * (int64_t)s;
#pragma unroll
    for (int k = 0; k < 4; ++k)
#pragma unroll
      for (int a = 0; a < 4; ++a) atomicAdd(g + 4 * k + a, gq[k][a]);
  }
}

}  // namespace

cudaError_t launch_backward(const float4* seg_cp, int64_t n_seg, bool quadratic, const float4* rays,
                            int64_t n_ray, const float2* tu, const int32_t* seg, const float* grad_t,
                            float* grad_cps, unsigned long long* n_skipped, cudaStream_t s) {
  (void)n_seg;
  if (n_ray <= 0) return cudaSuccess;
  const int block = 256;
  const unsigned grid = (unsigned)((n_ray + block - 1) / block);
  if (quadratic)
    k_backward<true><<<grid, block, 0, s>>>(seg_cp, rays, n_ray, tu, seg, grad_t, grad_cps, n_skipped);
  else
    k_backward<false><<<grid, block, 0, s>>>(seg_cp, rays, n_ray, tu, seg, grad_t, grad_cps, n_skipped);
  return cudaGetLastError();
}

}  // namespace fx
