// trace.cuh -- FP32 device core of the ray / cubic-fiber traversal
// (Binder & Keller, arXiv 1811.03374), sm_103a.
//
// Everything here runs in the ray-centric frame of Sec. 3.3: the ray starts at
// the origin and runs along +z, so a plane or cylinder test needs only the
// z components and the xy cross terms.  A node is the paper's
// (p, d, t0, t1) tuple (Sec. 3.1), four float4 whose w lanes carry the radius
// (Sec. 3.3: four-dimensional control points).
//
// FAST selects the approximate reciprocal / square root instructions of the
// PTX ISA (rcp.approx, sqrt.approx); otherwise IEEE round-to-nearest
// division and square root are used.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace fx {

constexpr uint32_t kRootSize = 1u << 23;  // [0, 1] in units of 2^-23
constexpr float kUnit = 1.0f / 8388608.0f;
constexpr float kInf = __builtin_huge_valf();

struct Node {
  float4 p, d, t0, t1;
};

struct RayFrame {
  float3 o, e1, e2, w;  // origin and orthonormal frame, w = unit direction
};

__device__ __forceinline__ float rcp_approx(float x) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float sqrt_approx(float x) {
  float y;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
template <bool FAST>
__device__ __forceinline__ float frcp(float x) {
  return FAST ? rcp_approx(x) : __frcp_rn(x);
}
template <bool FAST>
__device__ __forceinline__ float fsqrt(float x) {
  return FAST ? sqrt_approx(x) : __fsqrt_rn(x);
}
template <bool FAST>
__device__ __forceinline__ float fdiv(float a, float b) {
  return FAST ? a * rcp_approx(b) : __fdiv_rn(a, b);
}

__device__ __forceinline__ float dot3(const float4& a, const float4& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, a.z * b.z));
}

// Orthonormal basis around the unit vector w: Duff et al. 2017 ("Building an
// orthonormal basis, revisited"), the construction Sec. 3.3 cites.
__device__ __forceinline__ void make_onb(const float3& w, float3& e1, float3& e2) {
  const float sign = copysignf(1.0f, w.z);
  const float a = -1.0f / (sign + w.z);
  const float b = w.x * w.y * a;
  e1 = make_float3(1.0f + sign * w.x * w.x * a, sign * b, -sign * w.x);
  e2 = make_float3(b, sign + w.y * w.y * a, -w.y);
}

// Ray record {o.xyz, t_max}, {w.xyz, 0}; the direction is normalised here.
template <bool FAST>
__device__ __forceinline__ RayFrame load_ray(const float4* __restrict__ rays, int64_t i,
                                             float& tmax) {
  const float4 a = __ldg(rays + 2 * i), b = __ldg(rays + 2 * i + 1);
  RayFrame r;
  r.o = make_float3(a.x, a.y, a.z);
  tmax = a.w;
  const float n2 = fmaf(b.x, b.x, fmaf(b.y, b.y, b.z * b.z));
  const float inv = FAST ? rsqrtf(n2) : __frcp_rn(__fsqrt_rn(n2));
  r.w = make_float3(b.x * inv, b.y * inv, b.z * inv);
  make_onb(r.w, r.e1, r.e2);
  return r;
}

__device__ __forceinline__ float4 rotate(const RayFrame& r, float x, float y, float z, float wcomp) {
  return make_float4(fmaf(x, r.e1.x, fmaf(y, r.e1.y, z * r.e1.z)),
                     fmaf(x, r.e2.x, fmaf(y, r.e2.y, z * r.e2.z)),
                     fmaf(x, r.w.x, fmaf(y, r.w.y, z * r.w.z)), wcomp);
}

// A piece is stored as its world-space (p, d, t0, t1): p = p0 (with r0),
// d = p3 - p0, t0 = p1 - p0, t1 = p3 - p2 (radius differences in w).  Only
// p is offset by the ray origin; the difference vectors are rotated as they
// are, so no cancellation p3 - p0 happens in FP32 (Sec. 3.1's point).
__device__ __forceinline__ Node load_local(const float4* __restrict__ piece, int64_t k,
                                           const RayFrame& r) {
  const float4 p = __ldg(piece + 4 * k), d = __ldg(piece + 4 * k + 1);
  const float4 t0 = __ldg(piece + 4 * k + 2), t1 = __ldg(piece + 4 * k + 3);
  Node n;
  n.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
  n.d = rotate(r, d.x, d.y, d.z, d.w);
  n.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
  n.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
  return n;
}

// Conservative radius (Sec. 3.3): farthest inner control point from the axis
// (p, p + d) -- relative to p they are t0 and d - t1, at the distances of t0
// and t1 -- plus the largest control radius (convex hull).  Zero-length axis:
// distance from p.
template <bool FAST>
__device__ __forceinline__ float cons_radius(const Node& c) {
  const float dd = dot3(c.d, c.d);
  float m;
  if (dd > 0.0f) {
    const float inv = frcp<FAST>(dd);
    const float b0 = dot3(c.t0, c.d) * inv, b1 = dot3(c.t1, c.d) * inv;
    const float qx = fmaf(-b0, c.d.x, c.t0.x), qy = fmaf(-b0, c.d.y, c.t0.y),
                qz = fmaf(-b0, c.d.z, c.t0.z);
    const float sx = fmaf(-b1, c.d.x, c.t1.x), sy = fmaf(-b1, c.d.y, c.t1.y),
                sz = fmaf(-b1, c.d.z, c.t1.z);
    m = fmaxf(fmaf(qx, qx, fmaf(qy, qy, qz * qz)), fmaf(sx, sx, fmaf(sy, sy, sz * sz)));
  } else {
    m = fmaxf(dot3(c.t0, c.t0), dot3(c.t1, c.t1));
  }
  const float rmax = c.p.w + fmaxf(fmaxf(0.0f, c.t0.w), fmaxf(c.d.w, c.d.w - c.t1.w));
  return fsqrt<FAST>(m) + rmax;
}

// Unit ray vs the infinite cylinder of radius r through p along a (App. A):
// g = a_x^2 + a_y^2, e = r^2 - (a_x p_y - a_y p_x)^2 / g,
// t_cpa = p_z - a_z (a_x p_x + a_y p_y) / g, s = sqrt(e (a_z^2 + g) / g).
// g == 0: inside -> (-inf, inf), outside -> miss.  Returns false on a miss.
template <bool FAST>
__device__ __forceinline__ bool cylinder(const float4& p, const float4& a, float r, float& c0,
                                         float& c1) {
  const float g = fmaf(a.x, a.x, a.y * a.y);
  if (g == 0.0f) {
    c0 = -kInf;
    c1 = kInf;
    return fmaf(p.x, p.x, p.y * p.y) < r * r;
  }
  const float h = frcp<FAST>(g);
  const float cr = fmaf(a.x, p.y, -a.y * p.x);
  const float e = fmaf(-cr * cr, h, r * r);
  if (e < 0.0f) return false;
  const float tcpa = fmaf(-a.z * h, fmaf(a.x, p.x, a.y * p.y), p.z);
  const float s = fsqrt<FAST>(e * fmaf(a.z, a.z, g) * h);
  c0 = tcpa - s;
  c1 = tcpa + s;
  return true;
}

// t-interval between the start plane (through p, normal t0, kept side
// <x - p, t0> >= 0) and the end plane (through p + d, normal t1, kept side
// <x - p - d, t1> <= 0), clipped to [0, ray_tmax] (Sec. 3.3).  A plane
// parallel to the ray leaves the interval alone unless the ray is on its
// excluded side, which empties it.
template <bool FAST>
__device__ __forceinline__ void slab(const Node& c, float ray_tmax, float& tmin, float& tmax) {
  float lo = 0.0f, hi = ray_tmax;
  const float n0 = dot3(c.t0, c.p);
  if (c.t0.z != 0.0f) {
    const float t = fdiv<FAST>(n0, c.t0.z);
    if (c.t0.z > 0.0f) lo = fmaxf(lo, t);
    else hi = fminf(hi, t);
  } else if (n0 > 0.0f) {
    lo = kInf;
  }
  const float4 q = make_float4(c.p.x + c.d.x, c.p.y + c.d.y, c.p.z + c.d.z, 0.0f);
  const float n1 = dot3(c.t1, q);
  if (c.t1.z != 0.0f) {
    const float t = fdiv<FAST>(n1, c.t1.z);
    if (c.t1.z < 0.0f) lo = fmaxf(lo, t);
    else hi = fminf(hi, t);
  } else if (n1 < 0.0f) {
    lo = kInf;
  }
  tmin = lo;
  tmax = hi;
}

// One subdivision step (Sec. 3.1 rules, Sec. 3.2 partition):
// dp = 3/8 t0 + 1/2 d - 3/8 t1, tc = -1/8 t0 + 1/4 d - 1/8 t1; the plane
// through p + dp with normal tc meets the ray at tp; the ray reaches the
// right child first iff (tp > c0) xor (tc_z > 0); both children need a visit
// iff c0 < tp < c1; the bound on the near side of the plane is tightened.
// A plane parallel to the ray keeps the ray on the origin's side.
template <bool FAST>
__device__ __forceinline__ void descend(Node& c, float c0, float c1, float& tmin, float& tmax,
                                        uint32_t& bits, uint32_t& start, uint32_t& size) {
  float4 dp, tc;
  dp.x = fmaf(0.375f, c.t0.x - c.t1.x, 0.5f * c.d.x);
  dp.y = fmaf(0.375f, c.t0.y - c.t1.y, 0.5f * c.d.y);
  dp.z = fmaf(0.375f, c.t0.z - c.t1.z, 0.5f * c.d.z);
  dp.w = fmaf(0.375f, c.t0.w - c.t1.w, 0.5f * c.d.w);
  tc.x = fmaf(-0.125f, c.t0.x + c.t1.x, 0.25f * c.d.x);
  tc.y = fmaf(-0.125f, c.t0.y + c.t1.y, 0.25f * c.d.y);
  tc.z = fmaf(-0.125f, c.t0.z + c.t1.z, 0.25f * c.d.z);
  tc.w = fmaf(-0.125f, c.t0.w + c.t1.w, 0.25f * c.d.w);
  const float sx = c.p.x + dp.x, sy = c.p.y + dp.y, sz = c.p.z + dp.z;
  const float num = fmaf(tc.x, sx, fmaf(tc.y, sy, tc.z * sz));
  bool go_right, both;
  if (tc.z != 0.0f) {
    const float tp = fdiv<FAST>(num, tc.z);
    const bool before = tp > c0;
    go_right = before != (tc.z > 0.0f);
    both = (c0 < tp) && (c1 > tp);
    if (before) tmax = fminf(tmax, tp);
    else tmin = fmaxf(tmin, tp);
  } else {
    go_right = num <= 0.0f;
    both = false;
  }
  if (go_right) {
    c.p = make_float4(sx, sy, sz, c.p.w + dp.w);
    c.d = make_float4(c.d.x - dp.x, c.d.y - dp.y, c.d.z - dp.z, c.d.w - dp.w);
    c.t0 = tc;
    c.t1 = make_float4(0.5f * c.t1.x, 0.5f * c.t1.y, 0.5f * c.t1.z, 0.5f * c.t1.w);
  } else {
    c.d = dp;
    c.t0 = make_float4(0.5f * c.t0.x, 0.5f * c.t0.y, 0.5f * c.t0.z, 0.5f * c.t0.w);
    c.t1 = tc;
  }
  size >>= 1;
  if (both) bits |= size;
  if (go_right) start |= size;
}

// Backtracking without a stack (Sec. 3.3).  The search is a depth-first
// descent whose stack would only ever hold "the other child" of some
// ancestors; one bit per level (set at the level's node size) records which
// ancestors still owe that visit.  The node to resume is the other child at
// the deepest such level: with h its size (the lowest pending bit), its
// interval begins at the start of the current node's ancestor of size 2h,
// plus h if the current path took that ancestor's left child.  The bit is
// consumed; the node's geometry is recomputed by the caller.
__device__ __forceinline__ void take_pending(uint32_t& pending, uint32_t& start, uint32_t& size) {
  const uint32_t h = pending & (0u - pending);
  start = (start & (0u - (h << 1))) | (~start & h);
  pending &= pending - 1u;
  size = h;
}

// Node of the interval [u0, u0 + h] recomputed from the local root node R
// after backtracking (Sec. 3.3).  The curve is written in power form around
// p: c(u) = p + 3 t0 u + 3/2 E1 u^2 + E2 u^3 with E1 = 2 (d - t1) - 4 t0,
// E2 = 3 (t0 + t1) - 2 d, so c'(u)/3 = t0 + E1 u + E2 u^2 and the chord
// c(u0 + h) - c(u0) = h (c'(u0) + h (3/2 E1 + 3 E2 u0 + h E2)) is formed from
// small differences only (no subtraction of two points near the camera
// distance).  Same mathematics as the paper's eval / eval_derivative.
__device__ __forceinline__ void recompute1(float p, float d, float t0, float t1, float u0, float h,
                                           float& pn, float& dn, float& a0, float& a1) {
  const float E1 = fmaf(-4.0f, t0, 2.0f * (d - t1));
  const float E2 = fmaf(3.0f, t0 + t1, -2.0f * d);
  const float tau0 = fmaf(u0, fmaf(u0, E2, E1), t0);
  const float u1 = u0 + h;
  const float tau1 = fmaf(u1, fmaf(u1, E2, E1), t0);
  pn = fmaf(u0, fmaf(u0, fmaf(u0, E2, 1.5f * E1), 3.0f * t0), p);
  dn = h * fmaf(h, fmaf(h, E2, fmaf(3.0f * u0, E2, 1.5f * E1)), 3.0f * tau0);
  a0 = h * tau0;
  a1 = h * tau1;
}

__device__ __forceinline__ void recompute(const Node& R, uint32_t start, uint32_t size, Node& c) {
  const float u0 = __uint2float_rn(start) * kUnit, h = __uint2float_rn(size) * kUnit;
  recompute1(R.p.x, R.d.x, R.t0.x, R.t1.x, u0, h, c.p.x, c.d.x, c.t0.x, c.t1.x);
  recompute1(R.p.y, R.d.y, R.t0.y, R.t1.y, u0, h, c.p.y, c.d.y, c.t0.y, c.t1.y);
  recompute1(R.p.z, R.d.z, R.t0.z, R.t1.z, u0, h, c.p.z, c.d.z, c.t0.z, c.t1.z);
  recompute1(R.p.w, R.d.w, R.t0.w, R.t1.w, u0, h, c.p.w, c.d.w, c.t0.w, c.t1.w);
}

// u of a leaf hit: projection of (0, 0, t) onto the leaf axis, clamped
// (App. C), mapped to the interval [start, start + size) of the piece.
template <bool FAST>
__device__ __forceinline__ float leaf_u(const Node& c, float t, uint32_t start, uint32_t size) {
  const float dd = dot3(c.d, c.d);
  float ul = 0.0f;
  if (dd > 0.0f) {
    const float num = fmaf(-c.p.x, c.d.x, fmaf(-c.p.y, c.d.y, (t - c.p.z) * c.d.z));
    ul = fminf(1.0f, fmaxf(0.0f, fdiv<FAST>(num, dd)));
  }
  return fmaf(ul, __uint2float_rn(size), __uint2float_rn(start)) * kUnit;
}

// ---------------------------------------------------------------------------
// per-(ray, piece) traversal state shared by the kernels
// ---------------------------------------------------------------------------


__device__ __forceinline__ int piece_min_size_shift(int depth, int level) {
  const int d = depth > level ? depth - level : 0;
  return 23 - d;
}

// State of one lane's current (ray, piece) test.
struct PairState {
  Node R;  // root node of the piece in the ray frame (for backtracking)
  Node c;  // current node
  float tmin, tmax;
  uint32_t bits, start, size, min_size;
  int32_t info;  // level | off << 4 | unsupported << 31
  int32_t iters;
};

// Starts a test of piece data (p, d, t0, t1), world space, against the ray.
template <bool FAST>
__device__ __forceinline__ void begin_local(PairState& st, const float4& p, const float4& d,
                                            const float4& t0, const float4& t1, const RayFrame& r,
                                            int32_t info, int depth, float pair_tmax) {
  st.R.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
  st.R.d = rotate(r, d.x, d.y, d.z, d.w);
  st.R.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
  st.R.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
  st.c = st.R;
  st.bits = 0;
  st.start = 0;
  st.size = kRootSize;
  st.info = info;
  st.min_size = 1u << piece_min_size_shift(depth, info & 15);
  st.iters = 0;
  slab<FAST>(st.c, pair_tmax, st.tmin, st.tmax);
}

template <bool FAST>
__device__ __forceinline__ void begin_piece(PairState& st, const float4* __restrict__ piece, int k,
                                            const RayFrame& r, int32_t info, int depth,
                                            float pair_tmax) {
  begin_local<FAST>(st, __ldg(piece + 4 * k), __ldg(piece + 4 * k + 1), __ldg(piece + 4 * k + 2),
                    __ldg(piece + 4 * k + 3), r, info, depth, pair_tmax);
}

// Segment-parameter u and leaf start of a piece-local hit.
__device__ __forceinline__ void to_segment(int32_t info, float u_piece, uint32_t start, float& u,
                                           int32_t& leaf) {
  const int lvl = info & 15;
  const int off = (info >> 4) & 0x7ffff;
  u = lvl ? ldexpf(__int2float_rn(off) + u_piece, -lvl) : u_piece;
  leaf = (int32_t)(((uint32_t)off << (23 - lvl)) + (start >> lvl));
}

// Outcome of one node step.
enum StepResult { kStepContinue = 0, kStepLeaf = 1, kStepDone = 2 };

// One node test (Sec. 3.2 / 3.3) and the move it implies: leaf, descent or
// backtrack.  On kStepLeaf, t is the entry into the capped leaf cylinder,
// max(c0, t_min), and the test of this piece ends (instant termination); on
// kStepDone the piece is exhausted without a hit.
template <bool FAST, bool COUNT>
__device__ __forceinline__ StepResult node_step(PairState& st, float pair_tmax, float& t,
                                                unsigned long long& nd, unsigned long long& nb) {
  const float r = cons_radius<FAST>(st.c);
  float c0 = 0.0f, c1 = 0.0f;
  const bool over = cylinder<FAST>(st.c.p, st.c.d, r, c0, c1) &&
                    fmaxf(c0, st.tmin) <= fminf(c1, st.tmax);
  ++st.iters;
  if (!over) {
    // pruned: resume at the deepest pending sibling, or the piece is done
    if (st.bits == 0u) return kStepDone;
    take_pending(st.bits, st.start, st.size);
    recompute(st.R, st.start, st.size, st.c);
    slab<FAST>(st.c, pair_tmax, st.tmin, st.tmax);
    if (COUNT) ++nb;
    return kStepContinue;
  }
  if (st.size > st.min_size) {
    descend<FAST>(st.c, c0, c1, st.tmin, st.tmax, st.bits, st.start, st.size);
    if (COUNT) ++nd;
    return kStepContinue;
  }
  // a leaf whose capped cylinder the ray enters: the hit (instant termination)
  t = fmaxf(c0, st.tmin);
  return kStepLeaf;
}

}  // namespace fx
