// warp_kernels.cu -- warp-per-ray persistent kernel for rays with many
// candidates.
//
// A warp takes 32 consecutive rays from the atomic queue.  Their candidate
// lists are one contiguous range of seg_idx (CSR rows are consecutive), which
// the warp streams through a ring of staging slots in shared memory with
// cp.async: each slot holds one candidate's piece (64 B, world-space
// (p, d, t0, t1)), filled up to kRing - 1 batches of 32 ahead of use, so the
// gathers of upcoming candidates -- across ray boundaries too -- overlap the
// traversal of the current ones.
//
// The rays of the chunk are processed one after another by the whole warp:
// idle lanes take the ray's next staged candidates (ballot + popc ranking),
// every lane advances its own bit-string traversal by one node per loop
// iteration (Sec. 3.3), and leaf hits are reduced across the warp at once,
// so the closest hit so far (the t_max of every later node test) is shared by
// all lanes.  Ties in t keep the earlier candidate.  Rays without candidates
// are answered from the row pointers alone.
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kWarpsPerBlock = 4;
constexpr int kRing = 4;              // batches of 32 slots per warp
constexpr int kSlots = kRing * 32;    // power of two

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(smem_addr(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all_but_one() {
  asm volatile("cp.async.wait_group 1;\n" ::: "memory");
}
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

template <bool FAST, bool PAIRS, bool COUNT, bool CHECK>
__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    k_warp_ray(const TraceArgs a) {
  __shared__ __align__(16) float4 s_piece[kWarpsPerBlock][kSlots][4];
  __shared__ int32_t s_seg[kWarpsPerBlock][kSlots];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float4(*ring)[4] = s_piece[wid];
  int32_t* rseg = s_seg[wid];
  const unsigned lt_mask = (1u << lane) - 1u;
  unsigned long long n_nodes = 0, n_desc = 0, n_back = 0, n_tests = 0, n_hits = 0;

  for (;;) {
    // ---- a chunk of 32 rays -----------------------------------------------
    unsigned base = 0;
    if (lane == 0) base = atomicAdd(a.queue, 32u);
    base = __shfl_sync(kFull, base, 0);
    if ((int64_t)base >= a.n_ray) break;
    const int64_t rl = (int64_t)base + lane;
    const bool in = rl < a.n_ray;
    const int32_t rp0 = in ? __ldg(a.row_ptr + rl) : 0;
    const int32_t rp1 = in ? __ldg(a.row_ptr + rl + 1) : 0;
    const bool nonempty = in && rp1 > rp0;
    if (!PAIRS && in && !nonempty) {
      a.tu[rl] = make_float2(kInf, -1.0f);
      a.seg[rl] = -1;
      if (a.leaf) a.leaf[rl] = -1;
    }
    unsigned todo = __ballot_sync(kFull, nonempty);
    if (todo == 0u) continue;
    // candidate stream of the chunk: seg_idx[s0, s0 + n_stream)
    const int32_t s0 = __shfl_sync(kFull, rp0, __ffs(todo) - 1);
    const int32_t n_stream = __shfl_sync(kFull, rp1, 31 - __clz(todo)) - s0;
    int32_t fetched = 0;       // stream positions requested
    int32_t prev_fetched = 0;  // positions requested before the latest commit
    int32_t ready = 0;         // positions complete and visible to the warp
    int32_t consumed = 0;      // positions taken by lanes
    int32_t pre = lane < n_stream ? __ldg(a.seg_idx + s0 + lane) : 0;

    // Requests the next batch of 32 positions into the ring if it has room;
    // always commits one group (possibly empty) so group counts stay uniform.
    auto issue = [&]() {
      prev_fetched = fetched;
      if (fetched < n_stream && fetched - consumed <= (kRing - 1) * 32) {
        const int32_t pos = fetched + lane;
        if (pos < n_stream) {
          const int slot = pos & (kSlots - 1);
          int32_t s = pre;
          if (s < 0 || (CHECK && s >= a.n_seg)) {
            atomicOr(a.status, FX_DEV_BAD_INDEX);
            s = -1;
          }
          rseg[slot] = s;
          if (s >= 0) {
            const int32_t k = a.identity ? s : __ldg(a.piece_begin + s);
            const float4* src = a.piece + 4 * (int64_t)k;
            cp_async16(&ring[slot][0], src);
            cp_async16(&ring[slot][1], src + 1);
            cp_async16(&ring[slot][2], src + 2);
            cp_async16(&ring[slot][3], src + 3);
          }
        }
        fetched = min(fetched + 32, n_stream);
        const int32_t nxt = fetched + lane;
        pre = nxt < n_stream ? __ldg(a.seg_idx + s0 + nxt) : 0;
      }
      cp_commit();
    };
    issue();
    issue();

    while (todo) {
      // ---- one ray of the chunk, processed by the whole warp --------------
      const int rr = __ffs(todo) - 1;
      todo &= todo - 1;
      const int64_t ray = (int64_t)base + rr;
      const int32_t cend = __shfl_sync(kFull, rp1, rr) - s0;
      float ray_tmax;
      const RayFrame rf = load_ray<FAST>(a.rays, ray, ray_tmax);
      const int rdepth = depth_of(a, ray);  // warp-uniform: one ray per warp
      float best_t = ray_tmax, best_u = -1.0f;
      int32_t best_pos = INT_MAX, best_seg = -1, best_leaf = -1;
      bool active = false;
      PairState st;
      int32_t my_pos = -1, my_seg = -1, pc = 0, pend = 0;
      float cand_t = 0.0f, cand_u = -1.0f;  // pairs mode: best over the candidate's pieces
      int32_t cand_leaf = -1;
      uint32_t cand_flags = 0;  // FX_DEV_* bits of the lane's pair (pairs mode)

      for (;;) {
        // everything but the latest request is complete; publish warp-wide
        cp_wait_all_but_one();
        __syncwarp();
        ready = prev_fetched;
        issue();
        // refill idle lanes with the ray's staged candidates
        const int32_t navail = max(0, min(ready, cend) - consumed);
        const unsigned idle = __ballot_sync(kFull, !active);
        const int rank = __popc(idle & lt_mask);
        const int take = min(__popc(idle), navail);
        if (!active && rank < take) {
          my_pos = consumed + rank;
          const int slot = my_pos & (kSlots - 1);
          my_seg = rseg[slot];
          if (my_seg >= 0) {
            int32_t info = 0;
            pc = pend = 0;
            if (!a.identity) {
              const int32_t k0 = __ldg(a.piece_begin + my_seg);
              pc = k0 + 1;
              pend = __ldg(a.piece_begin + my_seg + 1);
              info = __ldg(a.piece_info + k0);
            }
            cand_t = ray_tmax;
            cand_u = -1.0f;
            cand_leaf = -1;
            cand_flags = 0;
            begin_local<FAST>(st, ring[slot][0], ring[slot][1], ring[slot][2], ring[slot][3], rf, info,
                              rdepth, PAIRS ? ray_tmax : best_t);
            active = true;
            if (COUNT) ++n_tests;
          } else if (PAIRS) {
            a.tu[s0 + my_pos] = make_float2(kInf, -1.0f);
            if (a.leaf) a.leaf[s0 + my_pos] = -1;
            if (a.pair_flags) a.pair_flags[s0 + my_pos] = FX_DEV_BAD_INDEX;
          }
        }
        consumed += take;
        if (__all_sync(kFull, !active) && consumed >= cend) break;

        // ---- one node step per active lane --------------------------------
        bool leaf_hit = false;
        float hit_t = 0.0f, hit_u = -1.0f;
        int32_t hit_leaf = -1;
        if (active) {
          float t;
          const StepResult r = node_step<FAST, COUNT>(st, PAIRS ? cand_t : best_t, t, n_desc, n_back);
          if (COUNT) ++n_nodes;
          bool piece_done = r != kStepContinue;
          if (r == kStepLeaf) {
            const float lim = PAIRS ? cand_t : best_t;
            if (t < lim || (!PAIRS && t == lim && my_pos < best_pos)) {
              float u;
              int32_t lf;
              to_segment(st.info, leaf_u<FAST>(st.c, t, st.start, st.size), st.start, u, lf);
              if (st.info < 0) {
                atomicOr(a.status, FX_DEV_UNSUPPORTED);
                cand_flags |= FX_DEV_UNSUPPORTED;
              }
              if (PAIRS) {
                cand_t = t;
                cand_u = u;
                cand_leaf = lf;
              } else {
                leaf_hit = true;
                hit_t = t;
                hit_u = u;
                hit_leaf = lf;
              }
              if (COUNT) ++n_hits;
            }
          }
          if (!piece_done && st.iters >= iter_cap(rdepth)) {
            atomicOr(a.status, FX_DEV_ITER_LIMIT);
            cand_flags |= FX_DEV_ITER_LIMIT;
            piece_done = true;
          }
          if (piece_done) {
            if (pc < pend) {
              // next piece of a pre-split segment
              begin_piece<FAST>(st, a.piece, pc, rf, __ldg(a.piece_info + pc), rdepth,
                                PAIRS ? cand_t : best_t);
              ++pc;
              if (COUNT) ++n_tests;
            } else {
              active = false;
              if (PAIRS) {
                a.tu[s0 + my_pos] = make_float2(cand_t < ray_tmax ? cand_t : kInf, cand_u);
                if (a.leaf) a.leaf[s0 + my_pos] = cand_leaf;
                if (a.pair_flags) a.pair_flags[s0 + my_pos] = (uint8_t)cand_flags;
              }
            }
          }
        }
        // ---- share the closest hit of this step across the warp -----------
        if (!PAIRS && __any_sync(kFull, leaf_hit)) {
          // hit_t >= 0 (a -0 loses its sign), so the bit patterns order like the values
          const unsigned tb = leaf_hit ? (__float_as_uint(hit_t) & 0x7fffffffu) : 0xffffffffu;
          const unsigned tmin = __reduce_min_sync(kFull, tb);
          const unsigned pb = (leaf_hit && tb == tmin) ? (unsigned)my_pos : 0xffffffffu;
          const unsigned pmin = __reduce_min_sync(kFull, pb);
          const int win = __ffs(__ballot_sync(kFull, leaf_hit && tb == tmin && (unsigned)my_pos == pmin)) - 1;
          const float wt = __uint_as_float(tmin);
          const float wu = __shfl_sync(kFull, hit_u, win);
          const int32_t wl = __shfl_sync(kFull, hit_leaf, win);
          const int32_t ws = __shfl_sync(kFull, my_seg, win);
          if (wt < best_t || (wt == best_t && (int32_t)pmin < best_pos)) {
            best_t = wt;
            best_pos = (int32_t)pmin;
            best_u = wu;
            best_leaf = wl;
            best_seg = ws;
          }
        }
      }
      if (!PAIRS && lane == 0) {
        const bool hit = best_seg >= 0;
        a.tu[ray] = make_float2(hit ? best_t : kInf, hit ? best_u : -1.0f);
        a.seg[ray] = best_seg;
        if (a.leaf) a.leaf[ray] = best_leaf;
      }
    }
    cp_wait_all();
    __syncwarp();
  }

  if (COUNT) {
    for (int o = 16; o > 0; o >>= 1) {
      n_nodes += __shfl_down_sync(kFull, n_nodes, o);
      n_desc += __shfl_down_sync(kFull, n_desc, o);
      n_back += __shfl_down_sync(kFull, n_back, o);
      n_tests += __shfl_down_sync(kFull, n_tests, o);
      n_hits += __shfl_down_sync(kFull, n_hits, o);
    }
    if (lane == 0) {
      atomicAdd(a.counters + 0, n_nodes);
      atomicAdd(a.counters + 1, n_desc);
      atomicAdd(a.counters + 2, n_back);
      atomicAdd(a.counters + 3, n_tests);
      atomicAdd(a.counters + 4, n_hits);
    }
  }
}

template <bool FAST, bool PAIRS, bool COUNT, bool CHECK>
cudaError_t launch_w(const TraceArgs& a, int grid, cudaStream_t s) {
  k_warp_ray<FAST, PAIRS, COUNT, CHECK><<<grid, kWarpsPerBlock * 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <bool FAST, bool PAIRS, bool COUNT, bool CHECK>
int occ_w() {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_warp_ray<FAST, PAIRS, COUNT, CHECK>,
                                                    kWarpsPerBlock * 32, 0) != cudaSuccess)
    return 0;
  return n;
}

}  // namespace

cudaError_t launch_warp_ray(const TraceArgs& a, bool pairs, uint32_t flags, int blocks_per_sm_cap,
                            int sm_count, cudaStream_t s) {
  const bool fast = flags & FX_FAST_MATH, cnt = flags & FX_COUNT, chk = flags & FX_CHECK_INDEX;
  int occ;
#define FX_W(F, P, C, K) (occ = occ_w<F, P, C, K>(), launch_w<F, P, C, K>(a, sm_count * (blocks_per_sm_cap > 0 ? min(occ, blocks_per_sm_cap) : max(occ, 1)), s))
  if (pairs) {
    if (fast) return cnt ? (chk ? FX_W(true, true, true, true) : FX_W(true, true, true, false))
                         : (chk ? FX_W(true, true, false, true) : FX_W(true, true, false, false));
    return cnt ? (chk ? FX_W(false, true, true, true) : FX_W(false, true, true, false))
               : (chk ? FX_W(false, true, false, true) : FX_W(false, true, false, false));
  }
  if (fast) return cnt ? (chk ? FX_W(true, false, true, true) : FX_W(true, false, true, false))
                       : (chk ? FX_W(true, false, false, true) : FX_W(true, false, false, false));
  return cnt ? (chk ? FX_W(false, false, true, true) : FX_W(false, false, true, false))
             : (chk ? FX_W(false, false, false, true) : FX_W(false, false, false, false));
#undef FX_W
}

}  // namespace fx
