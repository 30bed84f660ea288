// trace_kernels.cu -- forward kernels of the ray / cubic-fiber intersector.
//
// (the persistent kernels live in lane_kernels.cu and warp_kernels.cu)
// k_naive       one thread per (ray, candidate) pair, same arithmetic; the
//               closest hit per ray is an atomicMin over packed (t, pair)
//               keys followed by a resolve pass.  The baseline K1 must beat.
// k_polish      re-evaluates each hit's leaf cylinder in FP64.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {

constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// naive kernel: one thread per pair
// ---------------------------------------------------------------------------

// Full traversal of one piece (Sec. 3 / App. C iterative routine).
template <bool FAST>
__device__ __forceinline__ bool trace_piece(const TraceArgs& a, int piece, const RayFrame& rf, int depth,
                                            float pair_tmax, float& t_out, float& u_out,
                                            int32_t& leaf_out, unsigned long long* cnt, uint32_t& flags) {
  PairState st;
  begin_piece<FAST>(st, a.piece, piece, rf, a.identity ? 0 : __ldg(a.piece_info + piece), depth, pair_tmax);
  for (;;) {
    const float r = cons_radius<FAST>(st.c);
    float c0 = 0.0f, c1 = 0.0f;
    const bool over = cylinder<FAST>(st.c.p, st.c.d, r, c0, c1) &&
                      fmaxf(c0, st.tmin) <= fminf(c1, st.tmax);
    ++st.iters;
    if (cnt) ++cnt[0];
    if (over && st.size <= st.min_size) {
      const float t = fmaxf(c0, st.tmin);
      if (!(t < pair_tmax)) return false;
      const float up = leaf_u<FAST>(st.c, t, st.start, st.size);
      to_segment(st.info, up, st.start, u_out, leaf_out);
      if (st.info < 0) {
        atomicOr(a.status, FX_DEV_UNSUPPORTED);
        flags |= FX_DEV_UNSUPPORTED;
      }
      t_out = t;
      return true;
    } else if (over) {
      descend<FAST>(st.c, c0, c1, st.tmin, st.tmax, st.bits, st.start, st.size);
      if (cnt) ++cnt[1];
    } else if (st.bits == 0u) {
      return false;
    } else {
      take_pending(st.bits, st.start, st.size);
      recompute(st.R, st.start, st.size, st.c);
      slab<FAST>(st.c, pair_tmax, st.tmin, st.tmax);
      if (cnt) ++cnt[2];
    }
    if (st.iters >= iter_cap(depth)) {
      atomicOr(a.status, FX_DEV_ITER_LIMIT);
      flags |= FX_DEV_ITER_LIMIT;
      return false;
    }
  }
}

__device__ __forceinline__ int64_t ray_of_pair(const int32_t* __restrict__ row_ptr, int64_t n_ray,
                                               int64_t j) {
  // last row r with row_ptr[r] <= j (rows may be empty)
  int64_t lo = 0, hi = n_ray;  // invariant: row_ptr[lo] <= j < row_ptr[hi]
  while (hi - lo > 1) {
    const int64_t mid = (lo + hi) >> 1;
    if (__ldg(row_ptr + mid) <= j) lo = mid;
    else hi = mid;
  }
  return lo;
}

// Closest over the pieces of one candidate, tested with t_max.
template <bool FAST>
__device__ __forceinline__ bool trace_candidate(const TraceArgs& a, int32_t s, const RayFrame& rf, int depth,
                                                float tmax, float& t, float& u, int32_t& leaf,
                                                unsigned long long* cnt, uint32_t& flags) {
  int pb = s, pe = s + 1;
  if (!a.identity) {
    pb = __ldg(a.piece_begin + s);
    pe = __ldg(a.piece_begin + s + 1);
  }
  bool got = false;
  float lim = tmax;
  for (int k = pb; k < pe; ++k) {
    float tk, uk;
    int32_t lk;
    if (cnt) ++cnt[3];
    if (trace_piece<FAST>(a, k, rf, depth, lim, tk, uk, lk, cnt, flags)) {
      lim = tk;
      t = tk;
      u = uk;
      leaf = lk;
      got = true;
    }
  }
  return got;
}

template <bool FAST, bool PAIRS, bool COUNT, bool CHECK>
__global__ void __launch_bounds__(256) k_naive(const TraceArgs a) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long cnt[5] = {0, 0, 0, 0, 0};
  if (j < a.n_pair) {
    const int64_t r = ray_of_pair(a.row_ptr, a.n_ray, j);
    float ray_tmax;
    const RayFrame rf = load_ray<FAST>(a.rays, r, ray_tmax);
    const int32_t s = __ldg(a.seg_idx + j);
    float t = kInf, u = -1.0f;
    int32_t leaf = -1;
    bool got = false;
    uint32_t flags = 0;  // FX_DEV_* bits of this pair
    if (s < 0 || (CHECK && s >= a.n_seg)) {
      atomicOr(a.status, FX_DEV_BAD_INDEX);
      flags = FX_DEV_BAD_INDEX;
    } else {
      got = trace_candidate<FAST>(a, s, rf, depth_of(a, r), ray_tmax, t, u, leaf, COUNT ? cnt : nullptr, flags);
    }
    if (COUNT && got) cnt[4] = 1;
    if (PAIRS) {
      a.tu[j] = make_float2(got ? t : kInf, got ? u : -1.0f);
      if (a.leaf) a.leaf[j] = got ? leaf : -1;
      if (a.pair_flags) a.pair_flags[j] = (uint8_t)flags;
    } else if (got) {
      // t >= 0, so its bit pattern orders like the value once a -0 (fmaxf
      // may return either zero) has lost its sign; ties keep the smaller
      // pair index (the earlier candidate)
      const unsigned long long key = ((unsigned long long)(__float_as_uint(t) & 0x7fffffffu) << 32) | (uint32_t)j;
      atomicMin(a.scratch + r, key);
    }
  }
  if (COUNT) {
    for (int k = 0; k < 5; ++k) {
      unsigned long long v = cnt[k];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(kFull, v, o);
      if ((threadIdx.x & 31) == 0 && v) atomicAdd(a.counters + k, v);
    }
  }
}

// Per ray: decode the winning (t, pair) key and recompute that pair's u/leaf.
template <bool FAST>
__global__ void __launch_bounds__(256) k_naive_resolve(const TraceArgs a) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n_ray) return;
  const unsigned long long key = a.scratch[r];
  if (key == ~0ull) {
    a.tu[r] = make_float2(kInf, -1.0f);
    a.seg[r] = -1;
    if (a.leaf) a.leaf[r] = -1;
    return;
  }
  const int64_t j = (int64_t)(key & 0xffffffffull);
  float ray_tmax;
  const RayFrame rf = load_ray<FAST>(a.rays, r, ray_tmax);
  const int32_t s = __ldg(a.seg_idx + j);
  float t = kInf, u = -1.0f;
  int32_t leaf = -1;
  uint32_t flags = 0;
  trace_candidate<FAST>(a, s, rf, depth_of(a, r), ray_tmax, t, u, leaf, nullptr, flags);
  a.tu[r] = make_float2(__uint_as_float((uint32_t)(key >> 32)), u);
  a.seg[r] = s;
  if (a.leaf) a.leaf[r] = leaf;
}

// ---------------------------------------------------------------------------
// FP64 leaf re-evaluation
// ---------------------------------------------------------------------------
struct D4 {
  double x, y, z, w;
};
__device__ __forceinline__ double ddot3(const D4& a, const D4& b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}

// Node of the leaf [u0, u0 + size] recomputed in FP64 from the segment's
// control points Q in the ray frame (Sec. 3.3 recomputation), its slab,
// conservative radius and cylinder (App. A): the entry t = max(c0, t_min)
// into the capped leaf cylinder and u by projection; false if the ray misses
// it within [0, tmax].
__device__ bool polish_leaf(const D4 (&Q)[4], double u0, double size, double tmax, double& t_out,
                            double& u_out) {
  const double u1 = u0 + size;
  auto eval = [&](double u) {
    const double v = 1.0 - u, b0 = v * v * v, b1 = 3 * u * v * v, b2 = 3 * u * u * v, b3 = u * u * u;
    return D4{b0 * Q[0].x + b1 * Q[1].x + b2 * Q[2].x + b3 * Q[3].x,
              b0 * Q[0].y + b1 * Q[1].y + b2 * Q[2].y + b3 * Q[3].y,
              b0 * Q[0].z + b1 * Q[1].z + b2 * Q[2].z + b3 * Q[3].z,
              b0 * Q[0].w + b1 * Q[1].w + b2 * Q[2].w + b3 * Q[3].w};
  };
  auto deriv3 = [&](double u) {
    const double v = 1.0 - u, b0 = v * v, b1 = 2 * u * v, b2 = u * u;
    return D4{b0 * (Q[1].x - Q[0].x) + b1 * (Q[2].x - Q[1].x) + b2 * (Q[3].x - Q[2].x),
              b0 * (Q[1].y - Q[0].y) + b1 * (Q[2].y - Q[1].y) + b2 * (Q[3].y - Q[2].y),
              b0 * (Q[1].z - Q[0].z) + b1 * (Q[2].z - Q[1].z) + b2 * (Q[3].z - Q[2].z),
              b0 * (Q[1].w - Q[0].w) + b1 * (Q[2].w - Q[1].w) + b2 * (Q[3].w - Q[2].w)};
  };
  const D4 cp0 = eval(u0), cp1 = eval(u1), g0 = deriv3(u0), g1 = deriv3(u1);
  const D4 p = cp0;
  const D4 d{cp1.x - cp0.x, cp1.y - cp0.y, cp1.z - cp0.z, cp1.w - cp0.w};
  const D4 t0{size * g0.x, size * g0.y, size * g0.z, size * g0.w};
  const D4 t1{size * g1.x, size * g1.y, size * g1.z, size * g1.w};
  // slab
  double lo = 0.0, hi = tmax;
  if (t0.z != 0.0) {
    const double t = ddot3(t0, p) / t0.z;
    if (t0.z > 0.0) lo = fmax(lo, t); else hi = fmin(hi, t);
  } else if (ddot3(t0, p) > 0.0) {
    return false;
  }
  const D4 q{p.x + d.x, p.y + d.y, p.z + d.z, 0.0};
  if (t1.z != 0.0) {
    const double t = ddot3(t1, q) / t1.z;
    if (t1.z < 0.0) lo = fmax(lo, t); else hi = fmin(hi, t);
  } else if (ddot3(t1, q) < 0.0) {
    return false;
  }
  // conservative radius
  const double dd = ddot3(d, d);
  double m;
  if (dd > 0.0) {
    const double b0 = ddot3(t0, d) / dd, b1 = ddot3(t1, d) / dd;
    const double qx = t0.x - b0 * d.x, qy = t0.y - b0 * d.y, qz = t0.z - b0 * d.z;
    const double sx = t1.x - b1 * d.x, sy = t1.y - b1 * d.y, sz = t1.z - b1 * d.z;
    m = fmax(qx * qx + qy * qy + qz * qz, sx * sx + sy * sy + sz * sz);
  } else {
    m = fmax(ddot3(t0, t0), ddot3(t1, t1));
  }
  const double rad = sqrt(m) + p.w + fmax(fmax(0.0, t0.w), fmax(d.w, d.w - t1.w));
  // cylinder
  const double g = d.x * d.x + d.y * d.y;
  double c0, c1;
  if (g == 0.0) {
    if (!(p.x * p.x + p.y * p.y < rad * rad)) return false;
    c0 = -1e300;
    c1 = 1e300;
  } else {
    const double cr = d.x * p.y - d.y * p.x;
    const double e = rad * rad - cr * cr / g;
    if (e < 0.0) return false;
    const double tcpa = p.z - d.z * (d.x * p.x + d.y * p.y) / g;
    const double sq = sqrt(e * (d.z * d.z + g) / g);
    c0 = tcpa - sq;
    c1 = tcpa + sq;
  }
  if (!(fmax(c0, lo) <= fmin(c1, hi))) return false;
  t_out = fmax(c0, lo);
  double ul = 0.0;
  if (dd > 0.0) ul = fmin(1.0, fmax(0.0, (-p.x * d.x - p.y * d.y + (t_out - p.z) * d.z) / dd));
  u_out = u0 + ul * size;
  return true;
}

// FP64 re-evaluation of a hit: the FP32 traversal's leaf and its K
// neighbours on either side (within the same piece) are recomputed in FP64
// and the nearest entry is kept.  The FP32 traversal places a split plane
// along the fiber only to within the FP32 spacing of ray-frame coordinates,
// about 8 ulp(t) (they are differences from the ray origin, at the scale of
// t); where leaves are shorter than that, or a split plane is nearly
// parallel to the ray, the first leaf hit is a neighbour of the leaf it chose.
// K = 2 + that spacing in leaf lengths, at most kPolishMaxK.  If FP64 hits
// none of them, the FP32 result stays.
constexpr int kPolishMaxK = 32;

__global__ void __launch_bounds__(256) k_polish(const TraceArgs a, const float4* __restrict__ cp) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= a.n_ray) return;
  const int32_t s = a.seg[r];
  if (s < 0) return;
  const int32_t leaf = a.leaf[r];
  // leaf size 2^-max(depth, level of the piece holding the leaf); the
  // neighbours stay inside that piece's range of the segment
  int lvl = 0;
  int64_t plo = 0, phi = kRootSize;
  if (!a.identity) {
    const int pb = __ldg(a.piece_begin + s), pe = __ldg(a.piece_begin + s + 1);
    for (int k = pb; k < pe; ++k) {
      const int32_t info = __ldg(a.piece_info + k);
      const int kl = info & 15, off = (info >> 4) & 0x7ffff;
      const int64_t lo = (int64_t)off << (23 - kl), hi = (int64_t)(off + 1) << (23 - kl);
      if (leaf >= lo && leaf < hi) {
        lvl = kl;
        plo = lo;
        phi = hi;
        break;
      }
    }
  }
  const int rd = depth_of(a, r);
  const int dl = rd > lvl ? rd : lvl;
  const int64_t isize = (int64_t)1 << (23 - dl);
  const double size = (double)isize * (1.0 / 8388608.0);
  // ray frame in FP64 (Duff et al.; any orthonormal frame gives the same result)
  const float4 ra = a.rays[2 * r], rb = a.rays[2 * r + 1];
  double w[3] = {rb.x, rb.y, rb.z};
  const double wn = sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
  w[0] /= wn; w[1] /= wn; w[2] /= wn;
  double e1[3], e2[3];
  {
    const double s0 = copysign(1.0, w[2]);
    const double aa = -1.0 / (s0 + w[2]);
    const double bb = w[0] * w[1] * aa;
    e1[0] = 1.0 + s0 * w[0] * w[0] * aa; e1[1] = s0 * bb; e1[2] = -s0 * w[0];
    e2[0] = bb; e2[1] = s0 + w[1] * w[1] * aa; e2[2] = -w[1];
  }
  D4 Q[4];
  for (int k = 0; k < 4; ++k) {
    const float4 P = cp[4 * s + k];
    const double q0 = (double)P.x - ra.x, q1 = (double)P.y - ra.y, q2 = (double)P.z - ra.z;
    Q[k].x = q0 * e1[0] + q1 * e1[1] + q2 * e1[2];
    Q[k].y = q0 * e2[0] + q1 * e2[1] + q2 * e2[2];
    Q[k].z = q0 * w[0] + q1 * w[1] + q2 * w[2];
    Q[k].w = P.w;
  }
  // leaf length in world units at the chosen leaf (|c'| = 3 |deriv3|)
  double leaf_len;
  {
    const double um = ((double)leaf + 0.5 * (double)isize) * (1.0 / 8388608.0), v = 1.0 - um;
    const double b0 = v * v, b1 = 2 * um * v, b2 = um * um;
    const double dx = b0 * (Q[1].x - Q[0].x) + b1 * (Q[2].x - Q[1].x) + b2 * (Q[3].x - Q[2].x);
    const double dy = b0 * (Q[1].y - Q[0].y) + b1 * (Q[2].y - Q[1].y) + b2 * (Q[3].y - Q[2].y);
    const double dz = b0 * (Q[1].z - Q[0].z) + b1 * (Q[2].z - Q[1].z) + b2 * (Q[3].z - Q[2].z);
    leaf_len = 3.0 * sqrt(dx * dx + dy * dy + dz * dz) * size;
  }
  const double spacing = 8.0 * 0x1p-24 * fmax((double)a.tu[r].x, 1e-30);
  int K = kPolishMaxK;
  if (leaf_len > 0.0 && spacing / leaf_len < (double)kPolishMaxK) K = min(kPolishMaxK, 2 + (int)ceil(spacing / leaf_len));
  double best_t = 1e300, best_u = 0.0;
  int64_t best_leaf = -1;
  for (int k = -K; k <= K; ++k) {
    const int64_t start = (int64_t)leaf + k * isize;
    if (start < plo || start + isize > phi) continue;
    double t, u;
    if (polish_leaf(Q, (double)start * (1.0 / 8388608.0), size, ra.w, t, u) && t < best_t) {
      best_t = t;
      best_u = u;
      best_leaf = start;
    }
  }
  if (best_leaf < 0) return;
  a.tu[r] = make_float2((float)best_t, (float)best_u);
  a.leaf[r] = (int32_t)best_leaf;
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
template <bool FAST, bool PAIRS, bool COUNT, bool CHECK>
static cudaError_t launch_n(const TraceArgs& a, cudaStream_t s) {
  const int block = 256;
  if (a.n_pair > 0) {
    const int64_t grid = (a.n_pair + block - 1) / block;
    k_naive<FAST, PAIRS, COUNT, CHECK><<<(unsigned)grid, block, 0, s>>>(a);
  }
  if (!PAIRS && a.n_ray > 0) {
    k_naive_resolve<FAST><<<(unsigned)((a.n_ray + block - 1) / block), block, 0, s>>>(a);
  }
  return cudaGetLastError();
}

template <bool FAST, bool PAIRS>
static cudaError_t launch_n2(const TraceArgs& a, uint32_t flags, cudaStream_t s) {
  const bool cnt = flags & FX_COUNT, chk = flags & FX_CHECK_INDEX;
  if (cnt) return chk ? launch_n<FAST, PAIRS, true, true>(a, s) : launch_n<FAST, PAIRS, true, false>(a, s);
  return chk ? launch_n<FAST, PAIRS, false, true>(a, s) : launch_n<FAST, PAIRS, false, false>(a, s);
}

cudaError_t launch_naive(const TraceArgs& a, bool pairs, uint32_t flags, cudaStream_t s) {
  const bool fast = flags & FX_FAST_MATH;
  if (pairs) return fast ? launch_n2<true, true>(a, flags, s) : launch_n2<false, true>(a, flags, s);
  return fast ? launch_n2<true, false>(a, flags, s) : launch_n2<false, false>(a, flags, s);
}

cudaError_t launch_polish(const TraceArgs& a, const float4* seg_cp, cudaStream_t s) {
  if (a.n_ray > 0) {
    const int block = 256;
    k_polish<<<(unsigned)((a.n_ray + block - 1) / block), block, 0, s>>>(a, seg_cp);
  }
  return cudaGetLastError();
}

}  // namespace fx
