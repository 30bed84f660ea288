// filter_kernels.cu -- two-phase closest-hit path (FX_VARIANT_FILTER).
//
// Most candidate pairs of a frame fail at their root node; those that pass
// belong to the few rays that actually meet the fibers.  A lane that owns a
// ray and walks its candidates therefore spends most of its time on root
// tests, and whenever one lane of its warp descends, the others wait.  Here
// the two kinds of work are separated:
//
//   k_filter   one lane per pair, all lanes in step: the root test of
//              Sec. 3.2 / App. A (conservative cylinder of the piece, the
//              slab between its end planes, their overlap) against the ray's
//              own t_max.  Passing candidates are appended, in row order, to
//              a CSR-aligned list with their entry bound max(c0, t_min); rays
//              with no passing candidate are misses and are written here; the
//              others are compacted into a list of active rays.
//   k_active   one lane per active ray, persistent: the ray's passing
//              candidates in row order, each traversed exactly as the lane
//              kernel does (bit-string traversal, Sec. 3.3) with the closest
//              hit so far as t_max.  A candidate whose entry bound lies
//              beyond that hit cannot pass its root test and is skipped
//              without being read.
//
// The filter is conservative: it tests a cylinder whose radius is larger by
// a relative 2^-20 than the one the traversal tests, so it passes every
// candidate whose root test can pass, and its entry bound is never larger
// than the traversal's.  The traversal itself repeats the exact root test.
// Results and counters are the lane kernel's.  Handles whose segments are
// all single level-0 pieces only (no pre-split, no unsupported piece).
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kFilterWarps = 8;
constexpr int kActiveBlock = 128;
constexpr float kGrow = 1.0f + 1.0f / 1048576.0f;

// ---------------------------------------------------------------------------
// phase 1: root filter, one lane per pair
// ---------------------------------------------------------------------------

template <bool FAST, bool COUNT>
__global__ void __launch_bounds__(32 * kFilterWarps, 3)
    k_filter(const TraceArgs a, const FilterArgs o, int check) {
  // ray frames of the warp's 32 rays: [warp][o + t_max | e1 | e2 | w][lane]
  __shared__ float4 s_fr[kFilterWarps][4][32];
  __shared__ int32_t s_rp[kFilterWarps][33];
  __shared__ int32_t s_cnt[kFilterWarps][32];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t n_groups = (a.n_ray + 31) / 32;
  uint32_t n_tests = 0;

  // groups of 32 consecutive rays, handed out one at a time: their pair
  // counts range from 0 to thousands, so a static split leaves long tails
  for (;;) {
    uint32_t gq = 0;
    if (lane == 0) gq = atomicAdd(o.group_queue, 1u);
    const int64_t g = __shfl_sync(kFull, gq, 0);
    if (g >= n_groups) break;
    const int64_t r = g * 32 + lane;
    const bool rv = r < a.n_ray;
    const int64_t left = a.n_ray - g * 32;
    const int nv = left < 32 ? (int)left : 32;
    int32_t rp0 = 0, rp1 = 0;
    if (rv) {
      rp0 = __ldg(a.row_ptr + r);
      rp1 = __ldg(a.row_ptr + r + 1);
    }
    const int32_t end = __shfl_sync(kFull, rp1, nv - 1);
    if (!rv) rp0 = rp1 = end;  // lanes past the last ray: empty rows
    s_rp[wib][lane] = rp0;
    if (lane == 31) s_rp[wib][32] = end;
    s_cnt[wib][lane] = 0;
    if (rv && rp1 > rp0) {
      float tmax = 0.0f;
      const RayFrame f = load_ray<FAST>(a.rays, r, tmax);
      s_fr[wib][0][lane] = make_float4(f.o.x, f.o.y, f.o.z, tmax);
      s_fr[wib][1][lane] = make_float4(f.e1.x, f.e1.y, f.e1.z, 0.0f);
      s_fr[wib][2][lane] = make_float4(f.e2.x, f.e2.y, f.e2.z, 0.0f);
      s_fr[wib][3][lane] = make_float4(f.w.x, f.w.y, f.w.z, 0.0f);
    }
    __syncwarp();
    const int32_t P0 = s_rp[wib][0], P1 = end;

    // Software pipeline: segment ids are read two batches of 32 pairs ahead,
    // their root records one batch ahead of the batch being tested.
    auto seg_of = [&](int32_t j) -> int32_t { return j < P1 ? __ldg(a.seg_idx + j) : -1; };
    auto usable = [&](int32_t s) -> bool { return s >= 0 && (!check || s < a.n_seg); };
    int32_t sA = seg_of(P0 + lane), sB = seg_of(P0 + 32 + lane);
    float4 g0 = make_float4(0.f, 0.f, 0.f, 0.f), g1 = g0, g2 = g0, g3 = g0;
    if (usable(sA)) {
      g0 = __ldg(a.piece_root + 2 * (int64_t)sA);
      g1 = __ldg(a.piece_root + 2 * (int64_t)sA + 1);
      g2 = __ldg(a.piece + 4 * (int64_t)sA + 2);
      g3 = __ldg(a.piece + 4 * (int64_t)sA + 3);
    }

    for (int32_t j0 = P0; j0 < P1; j0 += 32) {
      const int32_t sC = seg_of(j0 + 64 + lane);
      float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), h1 = h0, h2 = h0, h3 = h0;
      if (usable(sB)) {
        h0 = __ldg(a.piece_root + 2 * (int64_t)sB);
        h1 = __ldg(a.piece_root + 2 * (int64_t)sB + 1);
        h2 = __ldg(a.piece + 4 * (int64_t)sB + 2);
        h3 = __ldg(a.piece + 4 * (int64_t)sB + 3);
      }

      const int32_t j = j0 + lane;
      const bool in = j < P1;
      // the row holding pair j: the last of the 32 rows starting at or before j
      int slot = 32;
      if (in) {
        slot = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (s_rp[wib][slot + step] <= j) slot += step;
      }
      const int32_t s = sA;
      bool pass = false;
      float entry = 0.0f;
      if (in && !usable(s)) atomicOr(a.status, FX_DEV_BAD_INDEX);
      if (in && usable(s)) {
        if (COUNT) ++n_tests;
        const float4 fo = s_fr[wib][0][slot], f1 = s_fr[wib][1][slot], f2 = s_fr[wib][2][slot],
                     fw = s_fr[wib][3][slot];
        RayFrame rf;
        rf.o = make_float3(fo.x, fo.y, fo.z);
        rf.e1 = make_float3(f1.x, f1.y, f1.z);
        rf.e2 = make_float3(f2.x, f2.y, f2.z);
        rf.w = make_float3(fw.x, fw.y, fw.z);
        Node n;
        n.p = rotate(rf, g0.x - rf.o.x, g0.y - rf.o.y, g0.z - rf.o.z, 0.0f);
        n.d = rotate(rf, g1.x, g1.y, g1.z, 0.0f);
        float c0 = 0.0f, c1 = 0.0f;
        if (cylinder<FAST>(n.p, n.d, g0.w * kGrow, c0, c1)) {
          n.t0 = rotate(rf, g2.x, g2.y, g2.z, 0.0f);
          n.t1 = rotate(rf, g3.x, g3.y, g3.z, 0.0f);
          float tmin = 0.0f, tmax = 0.0f;
          slab<FAST>(n, fo.w, tmin, tmax);
          entry = fmaxf(c0, tmin);
          pass = entry <= fminf(c1, tmax);
        }
      }
      sA = sB;
      sB = sC;
      g0 = h0;
      g1 = h1;
      g2 = h2;
      g3 = h3;

      // append the passing pairs to their rows' lists, in row order; the
      // lanes of one row are contiguous
      const int prev = __shfl_up_sync(kFull, slot, 1);
      const unsigned heads = __ballot_sync(kFull, lane == 0 || prev != slot);
      const unsigned passes = __ballot_sync(kFull, pass);
      const int first = 31 - __clz(heads & (kFull >> (31 - lane)));
      const unsigned below = lt & ~((1u << first) - 1u);
      const int done = slot < 32 ? s_cnt[wib][slot] : 0;
      if (pass) {
        const int32_t pos = s_rp[wib][slot] + done + __popc(passes & below);
        if (pos >= 0 && pos < a.n_pair) o.pass[pos] = make_int2(s, __float_as_int(entry));
        else atomicOr(a.status, FX_DEV_BAD_INDEX);  // row_ptr not a valid CSR
      }
      __syncwarp();
      const bool tail = lane == 31 || ((heads >> (lane + 1)) & 1u);
      if (tail && slot < 32) s_cnt[wib][slot] = done + __popc(passes & (below | (1u << lane)));
      __syncwarp();
    }

    const int32_t c = s_cnt[wib][lane];
    if (rv) {
      o.pass_cnt[r] = c;
      if (c == 0) {
        a.tu[r] = make_float2(kInf, -1.0f);
        a.seg[r] = -1;
        if (a.leaf) a.leaf[r] = -1;
      }
    }
    const unsigned act = __ballot_sync(kFull, rv && c > 0);
    if (act) {
      uint32_t base = 0;
      if (lane == 0) base = atomicAdd(o.n_active, (uint32_t)__popc(act));
      base = __shfl_sync(kFull, base, 0);
      if (rv && c > 0) o.active[base + __popc(act & lt)] = (int32_t)r;
    }
    __syncwarp();
  }

  if (COUNT) {
    unsigned long long v = n_tests;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_down_sync(kFull, v, off);
    if (lane == 0 && v) {
      atomicAdd(a.counters + 0, v);  // a root node test per pair
      atomicAdd(a.counters + 3, v);  // and a candidate test
    }
  }
}

// ---------------------------------------------------------------------------
// phase 2: traversal of the active rays' passing candidates, lane per ray
// ---------------------------------------------------------------------------

__device__ __forceinline__ void rotate_piece(const float4* __restrict__ piece, int32_t k,
                                             const RayFrame& r, Node& n) {
  const float4 p = __ldg(piece + 4 * (int64_t)k), d = __ldg(piece + 4 * (int64_t)k + 1);
  const float4 t0 = __ldg(piece + 4 * (int64_t)k + 2), t1 = __ldg(piece + 4 * (int64_t)k + 3);
  n.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
  n.d = rotate(r, d.x, d.y, d.z, d.w);
  n.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
  n.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
}

template <bool FAST, bool COUNT>
__global__ void __launch_bounds__(kActiveBlock, 6) k_active(const TraceArgs a, const FilterArgs o) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  const int64_t n_act = *o.n_active;

  int64_t pool_next = 0, pool_end = 0;  // warp-uniform chunk of the active list
  bool exhausted = false, done = false;

  int64_t ray = -1;
  RayFrame rf;
  float best_t = 0.0f, best_u = -1.0f;
  int32_t best_seg = -1, best_leaf = -1;
  int32_t kw = 0, kend = 0, base = 0;  // the window holds list entries kw .. kw + 3
  int2 w0, w1, w2, w3;
  // an entry past the list's end: no segment, and a NaN bound, which no
  // comparison accepts (the ray's t_max may itself be +inf)
  constexpr int kNone = 0x7fc00000;
  w0 = w1 = w2 = w3 = make_int2(-1, kNone);

  bool trav = false;  // a candidate is being traversed
  Node c;
  float tmin = 0.0f, tmax = 0.0f, root_r = 0.0f;
  uint32_t bits = 0, start = 0, size = 0;
  uint32_t min_size = 1u << piece_min_size_shift(a.depth, 0);
  int32_t piece = -1, iters = 0;
  bool slab_ok = false;
  uint32_t n_nodes = 0, n_desc = 0, n_back = 0, n_hits = 0;

  auto entry_at = [&](int32_t i) -> int2 { return i < kend ? __ldg(o.pass + base + i) : make_int2(-1, kNone); };
  auto refill = [&](int32_t from) {
    kw = from;
    w0 = entry_at(from);
    w1 = entry_at(from + 1);
    w2 = entry_at(from + 2);
    w3 = entry_at(from + 3);
  };

  for (;;) {
    // ---- 1. rays for idle lanes ------------------------------------------------
    for (;;) {
      const bool want = ray < 0 && !done;
      const unsigned m = __ballot_sync(kFull, want);
      if (m == 0u) break;
      if (pool_next >= pool_end) {
        if (exhausted) {
          if (want) done = true;
          continue;
        }
        uint32_t b = 0;
        if (lane == 0) b = atomicAdd(a.queue, (uint32_t)a.chunk);
        b = __shfl_sync(kFull, b, 0);
        if ((int64_t)b >= n_act) {
          exhausted = true;
          continue;
        }
        pool_next = b;
        pool_end = min((int64_t)b + a.chunk, n_act);
      }
      const int rank = __popc(m & lt);
      const int64_t avail = pool_end - pool_next;
      if (want && rank < avail) {
        ray = __ldg(o.active + pool_next + rank);
        float rt = 0.0f;
        rf = load_ray<FAST>(a.rays, ray, rt);
        min_size = 1u << piece_min_size_shift(depth_of(a, ray), 0);
        best_t = rt;
        best_u = -1.0f;
        best_seg = -1;
        best_leaf = -1;
        base = __ldg(a.row_ptr + ray);
        kend = __ldg(o.pass_cnt + ray);
        refill(0);
      }
      pool_next += min((int64_t)__popc(m), avail);
    }
    if (__all_sync(kFull, ray < 0)) break;

    // ---- 2. next candidate whose root test can pass --------------------------
    // At most the four entries of the window are examined per step, so a long
    // run of skipped entries does not hold up the warp's other lanes.
    if (ray >= 0 && !trav) {
      const float bt = best_t;
      int pick = -1;
      int2 e = w3;
      const int32_t left = kend - kw;  // entries of the window inside the list
      if (left > 0 && __int_as_float(w0.y) <= bt) {
        pick = 0;
        e = w0;
      } else if (left > 1 && __int_as_float(w1.y) <= bt) {
        pick = 1;
        e = w1;
      } else if (left > 2 && __int_as_float(w2.y) <= bt) {
        pick = 2;
        e = w2;
      } else if (left > 3 && __int_as_float(w3.y) <= bt) {
        pick = 3;
      }
      if (pick >= 0) {
        piece = e.x;
        refill(kw + pick + 1);
        rotate_piece(a.piece, piece, rf, c);
        root_r = __ldg(a.piece_rad + piece);
        bits = 0;
        start = 0;
        size = kRootSize;
        iters = 0;
        tmax = best_t;
        slab_ok = false;
        trav = true;
      } else if (kw + 4 < kend) {
        refill(kw + 4);
      } else {  // the ray's list is exhausted
        const bool hit = best_seg >= 0;
        a.tu[ray] = make_float2(hit ? best_t : kInf, hit ? best_u : -1.0f);
        a.seg[ray] = best_seg;
        if (a.leaf) a.leaf[ray] = best_leaf;
        ray = -1;
      }
    }

    // ---- 3. one node step ---------------------------------------------------
    if (trav) {
      const float r = iters == 0 ? root_r : cons_radius<FAST>(c);
      float c0 = 0.0f, c1 = 0.0f;
      bool over = cylinder<FAST>(c.p, c.d, r, c0, c1);
      if (over && !slab_ok) {
        const float lim = tmax;
        slab<FAST>(c, lim, tmin, tmax);
        slab_ok = true;
      }
      over = over && fmaxf(c0, tmin) <= fminf(c1, tmax);
      // the root test repeats the filter's; only deeper nodes are counted
      if (COUNT && iters > 0) ++n_nodes;
      ++iters;
      bool piece_done = false;
      if (over && size <= min_size) {
        const float t = fmaxf(c0, tmin);
        if (t < best_t) {
          best_t = t;
          best_u = leaf_u<FAST>(c, t, start, size);
          best_seg = piece;
          best_leaf = (int32_t)start;
          if (COUNT) ++n_hits;
        }
        piece_done = true;
      } else if (over) {
        descend<FAST>(c, c0, c1, tmin, tmax, bits, start, size);
        if (COUNT) ++n_desc;
      } else if (bits == 0u) {
        piece_done = true;
      } else {
        take_pending(bits, start, size);
        Node R;
        rotate_piece(a.piece, piece, rf, R);  // the root node, rebuilt
        recompute(R, start, size, c);
        tmax = best_t;
        slab_ok = false;
        if (COUNT) ++n_back;
      }
      if (!piece_done && iters >= iter_cap_of(a)) {
        atomicOr(a.status, FX_DEV_ITER_LIMIT);
        piece_done = true;
      }
      if (piece_done) trav = false;
    }
  }

  if (COUNT) {
    unsigned long long v[4] = {n_nodes, n_desc, n_back, n_hits};
    const int slot[4] = {0, 1, 2, 4};
    for (int q = 0; q < 4; ++q) {
      for (int off = 16; off > 0; off >>= 1) v[q] += __shfl_down_sync(kFull, v[q], off);
      if (lane == 0 && v[q]) atomicAdd(a.counters + slot[q], v[q]);
    }
  }
}

template <bool FAST, bool COUNT>
cudaError_t launch_f(const TraceArgs& a, const FilterArgs& o, int check, int bps_cap, int sms,
                     cudaStream_t s) {
  const int64_t groups = (a.n_ray + 31) / 32;
  int fo = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fo, k_filter<FAST, COUNT>, 32 * kFilterWarps, 0);
  if (fo < 1) fo = 1;
  int64_t blocks = (int64_t)sms * fo;  // persistent: one resident wave
  const int64_t need = (groups + kFilterWarps - 1) / kFilterWarps;
  if (blocks > need) blocks = need;
  if (blocks < 1) blocks = 1;
  k_filter<FAST, COUNT><<<(unsigned)blocks, 32 * kFilterWarps, 0, s>>>(a, o, check);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_active<FAST, COUNT>, kActiveBlock, 0);
  if (occ < 1) occ = 1;
  if (bps_cap > 0 && bps_cap < occ) occ = bps_cap;
  k_active<FAST, COUNT><<<sms * occ, kActiveBlock, 0, s>>>(a, o);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_filter(const TraceArgs& a, const FilterArgs& o, uint32_t flags, int blocks_per_sm_cap,
                          int sm_count, cudaStream_t s) {
  const bool fast = flags & FX_FAST_MATH, cnt = flags & FX_COUNT;
  const int chk = (flags & FX_CHECK_INDEX) ? 1 : 0;
  if (fast) return cnt ? launch_f<true, true>(a, o, chk, blocks_per_sm_cap, sm_count, s)
                       : launch_f<true, false>(a, o, chk, blocks_per_sm_cap, sm_count, s);
  return cnt ? launch_f<false, true>(a, o, chk, blocks_per_sm_cap, sm_count, s)
             : launch_f<false, false>(a, o, chk, blocks_per_sm_cap, sm_count, s);
}

}  // namespace fx
