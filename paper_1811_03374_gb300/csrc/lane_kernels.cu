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
// Latency of the per-candidate gathers is taken off the critical path by a
// per-lane software pipeline: the piece (64 B) and its root radius of the next
// candidate are copied into the lane's shared-memory slot with cp.async while
// the current one is traversed, and segment ids are loaded two candidates
// ahead.  Most candidates miss their root cylinder, so the root test needs
// only p and d in the ray frame and the piece's precomputed root radius (a
// rigid motion does not change it); t0, t1 are rotated, the root node saved
// for backtracking (in shared memory) and the slab (two plane divisions)
// formed only once that cylinder is hit.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kLaneBlock = 128;

__device__ __forceinline__ uint32_t saddr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(saddr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void wait_all_but_one() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
__device__ __forceinline__ void wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

struct Lite {  // traversal state kept in registers (the root node is in shared memory)
  Node c;
  float tmin, tmax;
  uint32_t bits, start, size, min_size;
  int32_t info, iters;
  float root_r;   // precomputed radius of the root cylinder
  bool slab_ok;   // tmin / tmax hold the current node's slab
  bool at_root;   // t0, t1 not yet rotated (still in the lane's slot)
};

template <bool FAST>
__device__ __forceinline__ void to_local(const float4& p, const float4& d, const float4& t0,
                                         const float4& t1, const RayFrame& r, Node& n) {
  n.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
  n.d = rotate(r, d.x, d.y, d.z, d.w);
  n.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
  n.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
}

template <bool FAST, bool PAIRS, bool COUNT, bool IDENTITY>
__global__ void __launch_bounds__(kLaneBlock, 7) k_lane(const TraceArgs a, int check) {
  __shared__ __align__(16) float4 s_slot[2][4][kLaneBlock];  // [parity][component][lane]
  __shared__ float s_rad[2][kLaneBlock];
  __shared__ __align__(16) float4 s_root[4][kLaneBlock];
  const int tid = threadIdx.x, lane = tid & 31;
  const unsigned lt_mask = (1u << lane) - 1u;

  int64_t pool_next = 0, pool_end = 0;  // warp-uniform ray pool
  bool exhausted = false;

  int64_t ray = -1;
  int32_t cand = 0, cend = 0, crow = 0;
  int32_t s_cur = -1, s_n1 = -1, s_n2 = -1;  // segment ids of cand, cand + 1, cand + 2
  int32_t pc = 0, pend = 0;                   // remaining pieces of a pre-split segment
  RayFrame rf;
  float ray_tmax = 0.0f, best_t = 0.0f, best_u = -1.0f;
  int32_t best_seg = -1, best_leaf = -1;
  float cand_t = 0.0f, cand_u = -1.0f;
  int32_t cand_leaf = -1;
  bool active = false, done = false;
  Lite st;
  uint32_t n_nodes = 0, n_desc = 0, n_back = 0, n_tests = 0, n_hits = 0;

  // Loaded ids are checked only where they are used (one and two candidates
  // later), so the loads stay off the critical path.
  auto seg_at = [&](int32_t j) -> int32_t { return j < cend ? __ldg(a.seg_idx + j) : -1; };
  auto valid = [&](int32_t s) -> bool {
    if (s < 0) return false;
    if (check && s >= a.n_seg) return false;
    return true;
  };
  auto prefetch = [&](int32_t s, int parity) {
    if (IDENTITY && valid(s)) {
      const float4* src = a.piece + 4 * (int64_t)s;
      cp16(&s_slot[parity][0][tid], src);
      cp16(&s_slot[parity][1][tid], src + 1);
      cp16(&s_slot[parity][2][tid], src + 2);
      cp16(&s_slot[parity][3][tid], src + 3);
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(saddr(&s_rad[parity][tid])),
                   "l"(a.piece_rad + s)
                   : "memory");
    }
    commit();
  };
  auto init_state = [&](int32_t info) {
    st.bits = 0;
    st.start = 0;
    st.size = kRootSize;
    st.info = info;
    st.min_size = 1u << piece_min_size_shift(a.depth, info & 15);
    st.iters = 0;
    st.tmax = PAIRS ? cand_t : best_t;
    st.slab_ok = false;
    active = true;
    if (COUNT) ++n_tests;
  };
  // Piece k from global memory, fully rotated (pre-split segments).
  auto begin_piece_k = [&](int32_t k) {
    to_local<FAST>(__ldg(a.piece + 4 * (int64_t)k), __ldg(a.piece + 4 * (int64_t)k + 1),
                   __ldg(a.piece + 4 * (int64_t)k + 2), __ldg(a.piece + 4 * (int64_t)k + 3), rf, st.c);
    s_root[0][tid] = st.c.p;
    s_root[1][tid] = st.c.d;
    s_root[2][tid] = st.c.t0;
    s_root[3][tid] = st.c.t1;
    st.root_r = __ldg(a.piece_rad + k);
    st.at_root = false;
    init_state(__ldg(a.piece_info + k));
  };
  // Piece of the current candidate from the lane's slot: only p and d rotated.
  auto begin_slot = [&](int par) {
    const float4 p = s_slot[par][0][tid], d = s_slot[par][1][tid];
    st.c.p = rotate(rf, p.x - rf.o.x, p.y - rf.o.y, p.z - rf.o.z, p.w);
    st.c.d = rotate(rf, d.x, d.y, d.z, d.w);
    st.root_r = s_rad[par][tid];
    st.at_root = true;
    init_state(0);
  };
  auto finish_candidate = [&]() {
    if (PAIRS) {
      a.tu[cand] = make_float2(cand_t < ray_tmax ? cand_t : kInf, cand_u);
      if (a.leaf) a.leaf[cand] = cand_leaf;
    }
  };
  // Moves to the next candidate of the ray (or finishes the ray).
  auto next_candidate = [&]() {
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
      s_cur = s_n1;
      s_n1 = s_n2;
      s_n2 = seg_at(cand + 2);
      if (PAIRS) {
        cand_t = ray_tmax;
        cand_u = -1.0f;
        cand_leaf = -1;
      }
      if (!valid(s_cur)) {
        atomicOr(a.status, FX_DEV_BAD_INDEX);
        s_cur = -1;
      }
      if (IDENTITY) {
        prefetch(s_n1, (cand + 1) & 1);  // one group per candidate
        wait_all_but_one();              // this candidate's group has landed
        if (s_cur < 0) continue;
        begin_slot(cand & 1);
        return;
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
          s_n1 = seg_at(crow);
          s_n2 = seg_at(crow + 1);
          if (IDENTITY) prefetch(s_n1, crow & 1);
          next_candidate();
        }
      }
      pool_next += min((int64_t)__popc(m), avail);
    }
    if (__all_sync(kFull, !active)) break;

    // ---- 2. one node step per active lane ----------------------------------
    if (active) {
      const float pair_tmax = PAIRS ? cand_t : best_t;
      const float r = (st.iters == 0) ? st.root_r : cons_radius<FAST>(st.c);
      float c0 = 0.0f, c1 = 0.0f;
      bool over = cylinder<FAST>(st.c.p, st.c.d, r, c0, c1);
      if (over && st.at_root) {
        // the root cylinder is hit: rotate the tangents and keep the root node
        const int par = cand & 1;
        const float4 t0 = s_slot[par][2][tid], t1 = s_slot[par][3][tid];
        st.c.t0 = rotate(rf, t0.x, t0.y, t0.z, t0.w);
        st.c.t1 = rotate(rf, t1.x, t1.y, t1.z, t1.w);
        s_root[0][tid] = st.c.p;
        s_root[1][tid] = st.c.d;
        s_root[2][tid] = st.c.t0;
        s_root[3][tid] = st.c.t1;
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
          if (st.info < 0) atomicOr(a.status, FX_DEV_UNSUPPORTED);
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
        jump_up(st.bits, st.start, st.size);
        Node R;
        R.p = s_root[0][tid];
        R.d = s_root[1][tid];
        R.t0 = s_root[2][tid];
        R.t1 = s_root[3][tid];
        recompute(R, st.start, st.size, st.c);
        st.tmax = pair_tmax;
        st.slab_ok = false;
        if (COUNT) ++n_back;
      }
      if (!piece_done && st.iters >= iter_cap(a.depth)) {
        atomicOr(a.status, FX_DEV_ITER_LIMIT);
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
