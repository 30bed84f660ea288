// lane_kernels.cu -- lane-per-ray persistent kernel (the default forward
// kernel).
//
// Each lane owns one ray and tests its candidate segments in row order with
// the closest hit so far as t_max (instant termination, Sec. 3.2, applied
// across candidates: rows listed front to back make later candidates fail at
// their root).  Warps take chunks of rays from an atomic queue and refill a
// lane from the warp's chunk (ballot + popc ranking) the moment its ray is
// finished.  Every loop iteration performs one node test per active lane; the
// traversal state is the paper's bit string, start and size in registers
// (Sec. 3.3).
//
// Most candidates miss their root cylinder.  The root test needs only p and d
// of the piece and its conservative radius, which a rigid motion leaves
// unchanged and the upload precomputes; these 32-byte root records stream
// through a 4-slot ring per lane in shared memory, copied with cp.async three
// candidates ahead of use (segment ids five ahead), so the gathers overlap the
// tests of the preceding candidates.  Only when a root cylinder is hit is the
// full 64-byte piece read and rotated into the ray frame; after a backtrack
// the root node is rebuilt from it the same way.  The slab of a node (two
// plane divisions) is formed only once its cylinder is hit.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLaneBlock = 128;
#ifndef FX_LANE_RING
#define FX_LANE_RING 4
#endif
#ifndef FX_LANE_SKIP
#define FX_LANE_SKIP 1
#endif
constexpr int kRing = FX_LANE_RING;  // slots per lane (4 or 8)
// root records are copied this many candidates ahead of use; the ids of the
// next five (ring of 4) or seven (ring of 8) candidates are held in registers
constexpr int kAhead = kRing == 8 ? 6 : 3;
static_assert(kRing == 4 || kRing == 8, "ring of 4 or 8 slots");
constexpr int kSkipCap = FX_LANE_SKIP;  // candidates a lane may reject by their bound in one step
// relative slack of the bound test against FP32 rounding of the rotation
constexpr float kBoundSlack = 1.0f / 262144.0f;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void wait_ring() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(kAhead) : "memory");
}
__device__ __forceinline__ void wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct Lite {  // traversal state kept in registers
  Node c;
  float tmin, tmax;
  uint32_t bits, start, size, min_size;
  int32_t info, iters, piece;
  float root_r;  // precomputed radius of the root cylinder
  bool slab_ok;  // tmin / tmax hold the current node's slab
  bool at_root;  // only p, d of the root are in the ray frame so far
};

__device__ __forceinline__ void to_local(const float4* __restrict__ piece, int32_t k, const RayFrame& r,
                                         Node& n) {
  const float4 p = __ldg(piece + 4 * (int64_t)k), d = __ldg(piece + 4 * (int64_t)k + 1);
  const float4 t0 = __ldg(piece + 4 * (int64_t)k + 2), t1 = __ldg(piece + 4 * (int64_t)k + 3);
  n.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
  n.d = rotate(r, d.x, d.y, d.z, d.w);
  n.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
  n.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
}

template <bool FAST, bool PAIRS, bool COUNT, bool IDENTITY>
__global__ void __launch_bounds__(kLaneBlock, 6) k_lane(const TraceArgs a, int check) {
  __shared__ __align__(16) float4 s_rec[kRing][2][kLaneBlock];  // [slot][p|d][lane]
  const int tid = threadIdx.x, lane = tid & 31;
  const unsigned lt_mask = (1u << lane) - 1u;

  int64_t pool_next = 0, pool_end = 0;  // warp-uniform ray pool
  bool exhausted = false;

  int64_t ray = -1;
  int32_t cand = 0, cend = 0, crow = 0;
  int32_t s_cur = -1, q1 = -1, q2 = -1, q3 = -1, q4 = -1, q5 = -1, q6 = -1, q7 = -1;  // cand, cand + 1..7
  int32_t pc = 0, pend = 0;  // remaining pieces of a pre-split segment
  RayFrame rf;
  float ray_tmax = 0.0f, best_t = 0.0f, best_u = -1.0f;
  int32_t best_seg = -1, best_leaf = -1;
  float cand_t = 0.0f, cand_u = -1.0f;
  int32_t cand_leaf = -1;
  uint32_t cand_flags = 0;  // FX_DEV_* bits of the current pair (per-pair mode)
  bool active = false, done = false;
  Lite st;
  uint32_t n_nodes = 0, n_desc = 0, n_back = 0, n_tests = 0, n_hits = 0;

  // Ids are checked where they are used, so their loads stay off the
  // critical path.
  auto seg_at = [&](int32_t j) -> int32_t { return j < cend ? __ldg(a.seg_idx + j) : -1; };
  auto valid = [&](int32_t s) -> bool { return s >= 0 && (!check || s < a.n_seg); };
  auto prefetch = [&](int32_t s, int32_t pos) {
    if (IDENTITY && valid(s)) {
      const int slot = pos & (kRing - 1);
      cp16(&s_rec[slot][0][tid], a.piece_root + 2 * (int64_t)s);
      cp16(&s_rec[slot][1][tid], a.piece_root + 2 * (int64_t)s + 1);
    }
    commit();  // one group per candidate, empty or not
  };
  auto init_state = [&](int32_t info) {
    st.bits = 0;
    st.start = 0;
    st.size = kRootSize;
    st.info = info;
    st.min_size = 1u << piece_min_size_shift(depth_of(a, ray), info & 15);
    st.iters = 0;
    st.tmax = PAIRS ? cand_t : best_t;
    st.slab_ok = false;
    active = true;
    if (COUNT) ++n_tests;
  };
  // Piece k read from global memory and rotated in full (pre-split segments).
  auto begin_piece_k = [&](int32_t k) {
    to_local(a.piece, k, rf, st.c);
    st.piece = k;
    st.root_r = __ldg(a.piece_rad + k);
    st.at_root = false;
    init_state(__ldg(a.piece_info + k));
  };
  // The current candidate's root record from its slot.  The record's d.w is
  // the radius of a sphere around the chord's midpoint that holds the root
  // node's capped cylinder (the region its test can accept); if the whole
  // sphere lies beyond the closest hit so far, the root test cannot pass and
  // the candidate is rejected from the ray-frame z components alone.
  // Otherwise p and d are rotated.  Returns false on a rejection.
  auto begin_slot = [&](int32_t pos) -> bool {
    const int slot = pos & (kRing - 1);
    const float4 p = s_rec[slot][0][tid], d = s_rec[slot][1][tid];
    const float px = p.x - rf.o.x, py = p.y - rf.o.y, pz = p.z - rf.o.z;
    const float zp = fmaf(px, rf.w.x, fmaf(py, rf.w.y, pz * rf.w.z));
    const float zd = fmaf(d.x, rf.w.x, fmaf(d.y, rf.w.y, d.z * rf.w.z));
    const float near = fmaf(0.5f, zd, zp) - d.w;
    const float lim = PAIRS ? cand_t : best_t;
    if (near - kBoundSlack * (fabsf(zp) + fabsf(zd) + d.w) > lim) return false;
    st.c.p = rotate(rf, px, py, pz, 0.0f);
    st.c.d = rotate(rf, d.x, d.y, d.z, 0.0f);
    st.root_r = p.w;
    st.piece = s_cur;
    st.at_root = true;
    init_state(0);
    return true;
  };
  auto finish_candidate = [&]() {
    if (PAIRS) {
      a.tu[cand] = make_float2(cand_t < ray_tmax ? cand_t : kInf, cand_u);
      if (a.leaf) a.leaf[cand] = cand_leaf;
      if (a.pair_flags) a.pair_flags[cand] = (uint8_t)cand_flags;
    }
  };
  // Moves to the next candidate of the ray (or finishes the ray).  A lane
  // rejects at most kSkipCap candidates by their bound per step, so that one
  // lane's long run of rejections does not hold up the rest of its warp.
  auto next_candidate = [&]() {
    int rejected = 0;
    while (ray >= 0) {
      if (!IDENTITY && pc < pend) {
        begin_piece_k(pc++);
        return;
      }
      if (cand >= crow) finish_candidate();
      if (++cand >= cend) {
        if (!PAIRS) {
          const bool hit = best_seg >= 0;
          a.tu[ray] = make_float2(hit ? best_t : kInf, hit ? best_u : -1.0f);
          a.seg[ray] = best_seg;
          if (a.leaf) a.leaf[ray] = best_leaf;
        }
        ray = -1;
        return;
      }
      s_cur = q1;
      q1 = q2;
      q2 = q3;
      q3 = q4;
      q4 = q5;
      if (kRing == 8) {  // ids seven ahead
        q5 = q6;
        q6 = q7;
        q7 = seg_at(cand + 7);
      } else {  // ids five ahead
        q5 = seg_at(cand + 5);
      }
      const int32_t q_ahead = kAhead == 6 ? q6 : q3;
      if (PAIRS) {
        cand_t = ray_tmax;
        cand_u = -1.0f;
        cand_leaf = -1;
        cand_flags = 0;
      }
      if (!valid(s_cur)) {
        atomicOr(a.status, FX_DEV_BAD_INDEX);
        if (PAIRS) cand_flags |= FX_DEV_BAD_INDEX;
        s_cur = -1;
      }
      if (IDENTITY) {
        prefetch(q_ahead, cand + kAhead);
        wait_ring();  // this candidate's group has landed
        if (s_cur < 0) continue;
        if (begin_slot(cand)) return;
        if (COUNT) ++n_tests;
        if (++rejected >= kSkipCap) return;  // the lane idles this step
        continue;
      } else {
        if (s_cur < 0) continue;
        pc = __ldg(a.piece_begin + s_cur);
        pend = __ldg(a.piece_begin + s_cur + 1);
        begin_piece_k(pc++);
        return;
      }
    }
  };

  for (;;) {
    // ---- 1. acquire work for idle lanes ------------------------------------
    if (!active && !done && ray >= 0) next_candidate();
    for (;;) {
      const bool want = !active && !done && ray < 0;
      const unsigned m = __ballot_sync(kFull, want);
      if (m == 0u) break;
      if (pool_next >= pool_end) {
        if (exhausted) {
          if (want) done = true;
          continue;
        }
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(a.queue, (unsigned)a.chunk);
        base = __shfl_sync(kFull, base, 0);
        if ((int64_t)base >= a.n_ray) {
          exhausted = true;
          continue;
        }
        pool_next = base;
        pool_end = min((int64_t)base + a.chunk, a.n_ray);
      }
      const int rank = __popc(m & lt_mask);
      const int64_t avail = pool_end - pool_next;
      if (want && rank < avail) {
        const int64_t r = pool_next + rank;
        crow = __ldg(a.row_ptr + r);
        cend = __ldg(a.row_ptr + r + 1);
        if (check) clamp_row(a, crow, cend);
        if (crow >= cend) {
          if (!PAIRS) {  // no candidates: a miss, without loading the ray
            a.tu[r] = make_float2(kInf, -1.0f);
            a.seg[r] = -1;
            if (a.leaf) a.leaf[r] = -1;
          }
        } else {
          ray = r;
          rf = load_ray<FAST>(a.rays, ray, ray_tmax);
          best_t = ray_tmax;
          best_u = -1.0f;
          best_seg = -1;
          best_leaf = -1;
          cand = crow - 1;
          pc = pend = 0;
          q1 = seg_at(crow);
          q2 = seg_at(crow + 1);
          q3 = seg_at(crow + 2);
          q4 = seg_at(crow + 3);
          q5 = seg_at(crow + 4);
          if (kRing == 8) {
            q6 = seg_at(crow + 5);
            q7 = seg_at(crow + 6);
          }
          if (IDENTITY) {
            prefetch(q1, crow);
            prefetch(q2, crow + 1);
            prefetch(q3, crow + 2);  // kAhead >= 3
            if (kAhead > 3) prefetch(q4, crow + 3);
            if (kAhead > 4) prefetch(q5, crow + 4);
            if (kAhead > 5) prefetch(q6, crow + 5);
          }
          next_candidate();
        }
      }
      pool_next += min((int64_t)__popc(m), avail);
    }
    if (__all_sync(kFull, !active && ray < 0)) break;

    // ---- 2. one node step per active lane ----------------------------------
    if (active) {
      const float pair_tmax = PAIRS ? cand_t : best_t;
      const float r = (st.iters == 0) ? st.root_r : cons_radius<FAST>(st.c);
      float c0 = 0.0f, c1 = 0.0f;
      bool over = cylinder<FAST>(st.c.p, st.c.d, r, c0, c1);
      if (over && st.at_root) {
        // the root cylinder is hit: the whole piece in the ray frame
        to_local(a.piece, st.piece, rf, st.c);
        st.at_root = false;
      }
      if (over && !st.slab_ok) {
        const float lim = st.tmax;
        slab<FAST>(st.c, lim, st.tmin, st.tmax);
        st.slab_ok = true;
      }
      over = over && fmaxf(c0, st.tmin) <= fminf(c1, st.tmax);
      ++st.iters;
      if (COUNT) ++n_nodes;
      bool piece_done = false;
      if (over && st.size <= st.min_size) {
        // leaf: entry into the capped leaf cylinder; the piece's test ends
        const float t = fmaxf(c0, st.tmin);
        if (t < pair_tmax) {
          float u;
          int32_t lf;
          to_segment(st.info, leaf_u<FAST>(st.c, t, st.start, st.size), st.start, u, lf);
          if (st.info < 0) {
            atomicOr(a.status, FX_DEV_UNSUPPORTED);
            if (PAIRS) cand_flags |= FX_DEV_UNSUPPORTED;
          }
          if (PAIRS) {
            cand_t = t;
            cand_u = u;
            cand_leaf = lf;
          } else {
            best_t = t;
            best_u = u;
            best_seg = s_cur;
            best_leaf = lf;
          }
          if (COUNT) ++n_hits;
        }
        piece_done = true;
      } else if (over) {
        descend<FAST>(st.c, c0, c1, st.tmin, st.tmax, st.bits, st.start, st.size);
        if (COUNT) ++n_desc;
      } else if (st.bits == 0u) {
        piece_done = true;
      } else {
        take_pending(st.bits, st.start, st.size);
        Node R;
        to_local(a.piece, st.piece, rf, R);  // the root node, rebuilt
        recompute(R, st.start, st.size, st.c);
        st.tmax = pair_tmax;
        st.slab_ok = false;
        if (COUNT) ++n_back;
      }
      if (!piece_done && st.iters >= iter_cap_of(a)) {
        atomicOr(a.status, FX_DEV_ITER_LIMIT);
        if (PAIRS) cand_flags |= FX_DEV_ITER_LIMIT;
        piece_done = true;
      }
      if (piece_done) active = false;
    }
  }
  wait_all();

  if (COUNT) {
    unsigned long long v[5] = {n_nodes, n_desc, n_back, n_tests, n_hits};
    for (int k = 0; k < 5; ++k) {
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
      if (lane == 0) atomicAdd(a.counters + k, v[k]);
    }
  }
}

template <bool FAST, bool PAIRS, bool COUNT, bool IDENTITY>
cudaError_t launch_l(const TraceArgs& a, int check, int bps_cap, int sms, cudaStream_t s) {
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_lane<FAST, PAIRS, COUNT, IDENTITY>, kLaneBlock, 0);
  if (occ < 1) occ = 1;
  if (bps_cap > 0 && bps_cap < occ) occ = bps_cap;
  k_lane<FAST, PAIRS, COUNT, IDENTITY><<<sms * occ, kLaneBlock, 0, s>>>(a, check);
  return cudaGetLastError();
}

template <bool FAST, bool PAIRS>
cudaError_t launch_l2(const TraceArgs& a, uint32_t flags, int bps, int sms, cudaStream_t s) {
  const int chk = (flags & FX_CHECK_INDEX) ? 1 : 0;
  const bool cnt = flags & FX_COUNT;
  if (a.identity) return cnt ? launch_l<FAST, PAIRS, true, true>(a, chk, bps, sms, s)
                             : launch_l<FAST, PAIRS, false, true>(a, chk, bps, sms, s);
  return cnt ? launch_l<FAST, PAIRS, true, false>(a, chk, bps, sms, s)
             : launch_l<FAST, PAIRS, false, false>(a, chk, bps, sms, s);
}

}  // namespace

cudaError_t launch_lane_ray(const TraceArgs& a, bool pairs, uint32_t flags, int blocks_per_sm_cap,
                            int sm_count, cudaStream_t s) {
  const bool fast = flags & FX_FAST_MATH;
  if (pairs) return fast ? launch_l2<true, true>(a, flags, blocks_per_sm_cap, sm_count, s)
                         : launch_l2<false, true>(a, flags, blocks_per_sm_cap, sm_count, s);
  return fast ? launch_l2<true, false>(a, flags, blocks_per_sm_cap, sm_count, s)
              : launch_l2<false, false>(a, flags, blocks_per_sm_cap, sm_count, s);
}

}  // namespace fx
