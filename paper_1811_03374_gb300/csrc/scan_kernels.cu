// scan_kernels.cu -- lane-per-ray traversal with warp-wide candidate scans
// (FX_VARIANT_SCAN).
//
// Each lane owns one ray and traverses its candidates in row order with the
// closest hit so far as t_max (instant termination, Sec. 3.2, carried across
// candidates), as in the lane kernel.  What differs is how a lane finds its
// next candidate worth traversing: the whole warp tests a window of 32
// consecutive candidates of that lane's row at once, one candidate per lane
// -- a coalesced load of 32 segment ids, their 32-byte root records copied
// to shared memory, the bound of the root node's capped cylinder against the
// ray's t_max, then the root cylinder test itself (Sec. 3.3, unit ray against
// the cylinder of the precomputed conservative radius).  A ballot ranks the
// candidates whose root cylinder is hit; the first kPL of them go, in row
// order, to a short list of the owner's in shared memory (segment, the bound
// test's left-hand side, root radius, and for per-pair results the candidate
// index), and if there are more, the owner's row resumes at the next one.  Candidates rejected in the
// scan cost a thirty-second of a warp step each instead of a full lane step.
//
// A rows pass runs first: it writes the misses of the rays without
// candidates and lists the others (ray, row begin, row end), prefetching
// those rays into L2, so that the persistent kernel's queue holds only rays
// with work.
//
// Scans are software-pipelined across the iterations of the warp's loop, so
// that their memory latency overlaps the node steps of the other lanes:
// iteration i loads the segment ids of up to kS new windows (one per hungry
// lane), iteration i + 1 copies their root records into shared memory
// (cp.async), iteration i + 2 tests them and hands out the lists.  When a
// ray is taken, its whole row of segment ids is prefetched into L2 with one
// bulk prefetch.
//
// The scan tests a window against the ray's t_max at the time of the scan,
// which is never smaller than at the time the owner traverses a candidate
// of the window; before a traversal the owner repeats the bound test with
// the current t_max (from the kept left-hand side: the same float), and the
// traversal starts with the full root test (cylinder and end-plane slab).
// So exactly the candidates that the lane kernel traverses are traversed
// here, with the same t_max: the results are the same bit for bit.
//
// Handles whose segments are single level-0 pieces only (segment id = piece
// id); others run the lane kernel.
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"
#include "trace.cuh"

namespace fx {
namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr int kScanBlock = 128;
#ifndef FX_SCAN_S
#define FX_SCAN_S 4
#endif
// windows entering the scan pipeline per iteration (at most one per lane)
constexpr int kS = FX_SCAN_S;
static_assert(kS >= 1 && kS <= 8, "1 to 8 windows per iteration");
// CTAs per SM the register budget is sized for (5: up to 102 registers)
#ifndef FX_SCAN_MINB
#define FX_SCAN_MINB 5
#endif
// root hits of a window handed to its owner at once; a window with more
// resumes at the next one
#ifndef FX_SCAN_PL
#define FX_SCAN_PL 5
#endif
constexpr int kPL = FX_SCAN_PL;
// relative slack of the bound test against FP32 rounding of the rotation
// (the lane kernel uses the same)
constexpr float kBoundSlack = 1.0f / 262144.0f;

__device__ __forceinline__ void prefetch_l1(const void* p) {
  asm volatile("prefetch.global.L1 [%0];\n" ::"l"(p));
}
__device__ __forceinline__ void cp16(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;\n" ::"r"(
                   static_cast<uint32_t>(__cvta_generic_to_shared(dst))),
               "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }
// Prefetch of ids [first, last) into L2, trimmed inward to 16-byte
// boundaries (the bulk prefetch's alignment); nothing outside the range is
// touched.
__device__ __forceinline__ void prefetch_ids_l2(const int32_t* first, const int32_t* last) {
  const uintptr_t lo = (reinterpret_cast<uintptr_t>(first) + 15u) & ~uintptr_t(15);
  const uintptr_t hi = reinterpret_cast<uintptr_t>(last) & ~uintptr_t(15);
  if (hi > lo)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(lo), "r"((uint32_t)(hi - lo))
                 : "memory");
}

// Nearest point along the ray of the sphere that holds the root node's
// capped cylinder, less a slack for FP32 rounding: if it lies beyond the
// ray's t_max, the root test cannot pass.  zp, zd: ray-frame z of p
// (relative to the origin) and d; rb: the sphere's radius about the chord
// midpoint p + d / 2.  (The lane kernel's bound test, the same arithmetic.)
__device__ __forceinline__ float bound_lhs(float zp, float zd, float rb) {
  const float near = fmaf(0.5f, zd, zp) - rb;
  return near - kBoundSlack * (fabsf(zp) + fabsf(zd) + rb);
}

// Rows pass: one lane per ray.  Rays without candidates are misses (closest
// hit) and are written here; the others are appended to o.act, 32
// consecutive rays of a warp as one group (one atomic per warp).
template <bool PAIRS>
__global__ void __launch_bounds__(256) k_rows(const TraceArgs a, const ScanArgs o, int check) {
  const int lane = threadIdx.x & 31;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31); r0 < a.n_ray; r0 += stride) {
    const int64_t r = r0 + lane;
    int32_t crow = 0, cend = 0;
    if (r < a.n_ray) {
      crow = __ldg(a.row_ptr + r);
      cend = __ldg(a.row_ptr + r + 1);
      if (check) clamp_row(a, crow, cend);
    }
    const bool has = crow < cend;
    if (r < a.n_ray && !has && !PAIRS) {
      a.tu[r] = make_float2(kInf, -1.0f);
      a.seg[r] = -1;
      if (a.leaf) a.leaf[r] = -1;
    }
    if (has) asm volatile("prefetch.global.L2 [%0];\n" ::"l"(a.rays + 2 * r));
    const unsigned m = __ballot_sync(kFull, has);
    if (m == 0u) continue;
    uint32_t off = 0;
    if (lane == 0) off = atomicAdd(o.n_act, (uint32_t)__popc(m));
    off = __shfl_sync(kFull, off, 0);
    if (has) o.act[off + __popc(m & ((1u << lane) - 1u))] = make_int4((int32_t)r, crow, cend, 0);
  }
}

// Shared memory is 31.5 KB per CTA, so that five CTAs, with the 1 KB each
// reserves, fit the SM's 168 KB shared-memory configuration rather than the
// 196 KB one (the former 34.8 KB layout, with the ids in shared memory and
// the candidate index in every list entry, measured 2 % slower on the hair
// frame at the same list length).
template <bool FAST, bool PAIRS, bool COUNT, bool CHECK>
__global__ void __launch_bounds__(kScanBlock, FX_SCAN_MINB) k_scan(const TraceArgs a, const ScanArgs o) {
  constexpr int check = CHECK ? 1 : 0;
  // per lane's ray: {o.xyz, closest hit so far t}, {w.xyz, ray t_max (pairs) or
  // hit leaf}, {e1.xyz, hit u}, {e2.xyz, hit segment}; the hit's u, leaf and
  // segment stay here rather than in registers until the ray is finished
  __shared__ __align__(16) float4 s_fr[4][kScanBlock];
  // root records of the windows at the test stage: [window][p | d][lane]
  // (their segment ids stay in registers)
  __shared__ __align__(16) float4 s_rec[kS][2][kScanBlock];
  // per lane: its window's root hits, in row order: segment, left-hand side
  // of the bound test, root radius and (per-pair results) candidate index
  __shared__ int32_t s_pls[kPL][kScanBlock];
  __shared__ float s_pll[kPL][kScanBlock];
  __shared__ float s_plr[kPL][kScanBlock];
  __shared__ int32_t s_plj[PAIRS ? kPL : 1][kScanBlock];
  const int tid = threadIdx.x, lane = tid & 31, warp0 = tid & ~31;
  const unsigned lt_mask = (1u << lane) - 1u;

  const uint32_t n_act = *o.n_act;      // rays with candidates (rows pass)
  int32_t pool_next = 0, pool_end = 0;  // warp-uniform pool of o.act entries
  bool exhausted = false, done = false;

  int32_t ray = -1, cend = 0;
  int32_t wpos = 0;    // first candidate of the row not scanned yet
  int32_t pl_next = 0, pl_end = 0;  // root hits of the window not traversed yet: entries [pl_next, pl_end)
  bool scanning = false;  // this lane's next window is in the scan pipeline
  // scan pipeline (warp-uniform lane sets; a window's slot is its owner's
  // rank in the set): hA -- ids loaded into idA, hB -- records in flight
  unsigned hA = 0u, hB = 0u;
  int32_t idA[kS], idB[kS];  // ids of the windows in hA, in hB
  float ray_tmax = 0.0f, best_t = 0.0f;
  bool active = false;

  // traversal state of the current candidate (the paper's bit string, start
  // and size; Sec. 3.3)
  Node c;
  float tmin = 0.0f, tmax = 0.0f, root_r = 0.0f;
  uint32_t bits = 0, start = 0, size = 0, min_size = 1u << piece_min_size_shift(a.depth, 0);
  int32_t iters = 0, s_cur = -1, cand_j = 0;
  bool slab_ok = false;
  float cand_t = 0.0f, cand_u = -1.0f;
  int32_t cand_leaf = -1;
  uint32_t n_nodes = 0, n_desc = 0, n_back = 0, n_tests = 0, n_hits = 0;

  auto frame = [&]() {
    RayFrame r;
    const float4 A = s_fr[0][tid], B = s_fr[1][tid], C = s_fr[2][tid], D = s_fr[3][tid];
    r.o = make_float3(A.x, A.y, A.z);
    r.w = make_float3(B.x, B.y, B.z);
    r.e1 = make_float3(C.x, C.y, C.z);
    r.e2 = make_float3(D.x, D.y, D.z);
    return r;
  };
  auto to_local = [&](int32_t k, Node& n) {
    const RayFrame r = frame();
    const float4 p = __ldg(a.piece + 4 * (int64_t)k), d = __ldg(a.piece + 4 * (int64_t)k + 1);
    const float4 t0 = __ldg(a.piece + 4 * (int64_t)k + 2), t1 = __ldg(a.piece + 4 * (int64_t)k + 3);
    n.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
    n.d = rotate(r, d.x, d.y, d.z, d.w);
    n.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
    n.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
  };
  // Starts the traversal of the lane's next root hit whose bound still
  // admits it (the bound's left-hand side was kept by the scan, so the
  // re-test against the current t_max reads no memory); false when there is
  // none.  The piece is the only load.
  auto begin_next = [&]() -> bool {
    const float lim = PAIRS ? ray_tmax : best_t;
    while (pl_next < pl_end) {
      const int32_t s = s_pls[pl_next][tid];
      const float lhs = s_pll[pl_next][tid], rr = s_plr[pl_next][tid];
      const int32_t j = PAIRS ? s_plj[pl_next][tid] : 0;
      ++pl_next;
      if (!PAIRS && lhs > lim) continue;
      const float4* pc = a.piece + 4 * (int64_t)s;
      const float4 p = __ldg(pc), d = __ldg(pc + 1), t0 = __ldg(pc + 2), t1 = __ldg(pc + 3);
      const RayFrame r = frame();
      c.p = rotate(r, p.x - r.o.x, p.y - r.o.y, p.z - r.o.z, p.w);
      c.d = rotate(r, d.x, d.y, d.z, d.w);
      c.t0 = rotate(r, t0.x, t0.y, t0.z, t0.w);
      c.t1 = rotate(r, t1.x, t1.y, t1.z, t1.w);
      s_cur = s;
      cand_j = j;
      root_r = rr;
      bits = 0;
      start = 0;
      size = kRootSize;
      iters = 0;
      slab_ok = false;
      tmax = lim;
      if (PAIRS) {
        cand_t = ray_tmax;
        cand_u = -1.0f;
        cand_leaf = -1;
      }
      active = true;
      return true;
    }
    return false;
  };
  // Test stage: the windows of the lanes in hB, whose root records have
  // landed in shared memory; lane i takes candidate wpos + i of each.  The
  // first kPL root hits go to the owner's list; if there are more, the
  // owner's row resumes at the next one (its later candidates are tested
  // again, against the t_max of then).
  auto scan_test = [&]() {
    unsigned h = hB;
#pragma unroll
    for (int q = 0; q < kS; ++q) {
      if (h == 0u) break;  // warp-uniform
      const int L = __ffs(h) - 1;
      h &= h - 1u;
      const int32_t base = __shfl_sync(kFull, wpos, L);
      const int32_t end = __shfl_sync(kFull, cend, L);
      const int slot = warp0 + L;
      const int32_t j = base + lane;
      const int32_t s = idB[q];
      const bool valid = j < end && s >= 0 && (!check || s < a.n_seg);
      bool pass = false;
      float lhs = 0.0f, rr = 0.0f;
      if (valid) {
        const float4 O = s_fr[0][slot], W = s_fr[1][slot];
        const float lim = PAIRS ? W.w : O.w;
        const float4 Pk = s_rec[q][0][tid], Dk = s_rec[q][1][tid];
        const float px = Pk.x - O.x, py = Pk.y - O.y, pz = Pk.z - O.z;
        const float zp = fmaf(px, W.x, fmaf(py, W.y, pz * W.z));
        const float zd = fmaf(Dk.x, W.x, fmaf(Dk.y, W.y, Dk.z * W.z));
        lhs = bound_lhs(zp, zd, Dk.w);
        rr = Pk.w;
        if (!(lhs > lim)) {
          const float4 E1 = s_fr[2][slot], E2 = s_fr[3][slot];
          const float4 pp = make_float4(fmaf(px, E1.x, fmaf(py, E1.y, pz * E1.z)),
                                        fmaf(px, E2.x, fmaf(py, E2.y, pz * E2.z)), zp, 0.0f);
          const float4 dd = make_float4(fmaf(Dk.x, E1.x, fmaf(Dk.y, E1.y, Dk.z * E1.z)),
                                        fmaf(Dk.x, E2.x, fmaf(Dk.y, E2.y, Dk.z * E2.z)), zd, 0.0f);
          float c0 = 0.0f, c1 = 0.0f;
          // the traversal's root test intersects [c0, c1] with the slab,
          // which lies inside [0, lim]
          pass = cylinder<FAST>(pp, dd, rr, c0, c1) && c0 <= lim && c1 >= 0.0f;
        }
      }
      const unsigned m = __ballot_sync(kFull, pass);
      const int rank = __popc(m & lt_mask);
      // candidates from `resume` on are tested again later
      int32_t resume = base + 32;
      if (__popc(m) > kPL) {
        unsigned mm = m;
#pragma unroll
        for (int i = 0; i < kPL; ++i) mm &= mm - 1u;
        resume = base + __ffs(mm) - 1;
      }
      if (pass && rank < kPL) {
        s_pls[rank][slot] = s;
        s_pll[rank][slot] = lhs;
        s_plr[rank][slot] = rr;
        if (PAIRS) s_plj[rank][slot] = j;
        prefetch_l1(a.piece + 4 * (int64_t)s);
      }
      if (j < end && j < resume) {
        if (valid) {
          if (COUNT) ++n_tests;
        } else {
          atomicOr(a.status, FX_DEV_BAD_INDEX);
        }
        if (PAIRS && !pass) {
          a.tu[j] = make_float2(kInf, -1.0f);
          if (a.leaf) a.leaf[j] = -1;
          if (a.pair_flags) a.pair_flags[j] = valid ? 0 : FX_DEV_BAD_INDEX;
        }
      }
      if (lane == L) {
        pl_next = 0;
        pl_end = min(__popc(m), kPL);
        wpos = resume;
        scanning = false;
      }
    }
    hB = 0u;
  };
  // Copy stage: root records of the windows in hA (ids in idA) to shared
  // memory; they move to hB (ids to idB).
  auto scan_copy = [&]() {
    const int n = __popc(hA);
#pragma unroll
    for (int q = 0; q < kS; ++q) {
      if (q >= n) break;  // warp-uniform
      const int32_t s = idA[q];
      idB[q] = s;
      if (s >= 0 && (!check || s < a.n_seg)) {
        cp16(&s_rec[q][0][tid], a.piece_root + 2 * (int64_t)s);
        cp16(&s_rec[q][1][tid], a.piece_root + 2 * (int64_t)s + 1);
      }
    }
    cp_commit();
    hB = hA;
    hA = 0u;
  };
  // Load stage: up to kS hungry lanes (in h) put their next window in the
  // pipeline; lane i loads id wpos + i of each.
  auto scan_load = [&](unsigned h) {
#pragma unroll
    for (int q = 0; q < kS; ++q) {
      if (h == 0u) break;  // warp-uniform
      const int L = __ffs(h) - 1;
      h &= h - 1u;
      hA |= 1u << L;
      const int32_t j = __shfl_sync(kFull, wpos, L) + lane;
      const int32_t end = __shfl_sync(kFull, cend, L);
      idA[q] = j < end ? __ldg(a.seg_idx + j) : -1;
    }
    if ((hA >> lane) & 1u) scanning = true;
  };

  for (;;) {
    // ---- 1. idle lanes take rays from the warp's pool ------------------------
    for (;;) {
      const bool want = !active && !done && ray < 0;
      const unsigned m = __ballot_sync(kFull, want);
      if (m == 0u) break;
      if (pool_next >= pool_end) {
        if (exhausted) {
          if (want) done = true;
          continue;
        }
        unsigned b = 0;
        if (lane == 0) b = atomicAdd(a.queue, (unsigned)a.chunk);
        b = __shfl_sync(kFull, b, 0);
        if (b >= n_act) {
          exhausted = true;
          continue;
        }
        pool_next = (int32_t)b;
        pool_end = (int32_t)min(b + (unsigned)a.chunk, n_act);
      }
      const int rank = __popc(m & lt_mask);
      const int32_t avail = pool_end - pool_next;
      if (want && rank < avail) {
        const int4 e = __ldg(o.act + pool_next + rank);  // a ray with candidates
        ray = e.x;
        cend = e.z;
        const RayFrame rf = load_ray<FAST>(a.rays, ray, ray_tmax);
        min_size = 1u << piece_min_size_shift(depth_of(a, ray), 0);
        s_fr[0][tid] = make_float4(rf.o.x, rf.o.y, rf.o.z, ray_tmax);
        s_fr[1][tid] = make_float4(rf.w.x, rf.w.y, rf.w.z, PAIRS ? ray_tmax : __int_as_float(-1));
        s_fr[2][tid] = make_float4(rf.e1.x, rf.e1.y, rf.e1.z, -1.0f);
        s_fr[3][tid] = make_float4(rf.e2.x, rf.e2.y, rf.e2.z, __int_as_float(-1));
        best_t = ray_tmax;
        wpos = e.y;
        pl_next = pl_end = 0;
        if (cend - e.y > 32) prefetch_ids_l2(a.seg_idx + e.y + 32, a.seg_idx + cend);
      }
      pool_next += min(__popc(m), avail);
    }
    if (__all_sync(kFull, !active && ray < 0)) break;

    // ---- 2. the scan pipeline; lanes without a candidate get one, put their
    //         next window in the pipeline or end their ray -------------------
    __syncwarp();  // frames and t_max written by the lanes are visible
    if (hB) {
      cp_wait_all();  // the records copied in the previous iteration
      scan_test();
    }
    if (hA) scan_copy();
    bool hungry = false;
    if (!active && ray >= 0 && !scanning && !begin_next()) {
      if (wpos < cend) {
        hungry = true;
      } else {  // row exhausted: the ray's closest hit is final
        if (!PAIRS) {
          const int32_t best_seg = __float_as_int(s_fr[3][tid].w);
          const bool hit = best_seg >= 0;
          a.tu[ray] = make_float2(hit ? best_t : kInf, hit ? s_fr[2][tid].w : -1.0f);
          a.seg[ray] = best_seg;
          if (a.leaf) a.leaf[ray] = __float_as_int(s_fr[1][tid].w);
        }
        ray = -1;
      }
    }
    scan_load(__ballot_sync(kFull, hungry));

    // ---- 3. one node step per active lane ------------------------------------
    if (active) {
      const float pair_tmax = PAIRS ? cand_t : best_t;
      const float r = (iters == 0) ? root_r : cons_radius<FAST>(c);
      float c0 = 0.0f, c1 = 0.0f;
      bool over = cylinder<FAST>(c.p, c.d, r, c0, c1);
      if (over && !slab_ok) {
        const float lim = tmax;
        slab<FAST>(c, lim, tmin, tmax);
        slab_ok = true;
      }
      over = over && fmaxf(c0, tmin) <= fminf(c1, tmax);
      ++iters;
      if (COUNT) ++n_nodes;
      bool piece_done = false;
      if (over && size <= min_size) {
        // leaf: entry into the capped leaf cylinder; the candidate's test ends
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
            s_fr[0][tid].w = t;
            s_fr[1][tid].w = __int_as_float(lf);
            s_fr[2][tid].w = u;
            s_fr[3][tid].w = __int_as_float(s_cur);
          }
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
        to_local(s_cur, R);  // the root node, rebuilt
        recompute(R, start, size, c);
        tmax = pair_tmax;
        slab_ok = false;
        if (COUNT) ++n_back;
      }
      bool capped = false;
      if (!piece_done && iters >= iter_cap_of(a)) {
        atomicOr(a.status, FX_DEV_ITER_LIMIT);
        piece_done = capped = true;
      }
      if (piece_done) {
        active = false;
        if (PAIRS) {
          a.tu[cand_j] = make_float2(cand_t < ray_tmax ? cand_t : kInf, cand_u);
          if (a.leaf) a.leaf[cand_j] = cand_leaf;
          if (a.pair_flags) a.pair_flags[cand_j] = capped ? FX_DEV_ITER_LIMIT : 0;
        }
      }
    }
  }

  if (COUNT) {
    unsigned long long v[5] = {n_nodes, n_desc, n_back, n_tests, n_hits};
    for (int k = 0; k < 5; ++k) {
      for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(kFull, v[k], o);
      if (lane == 0) atomicAdd(a.counters + k, v[k]);
    }
  }
}

template <bool FAST, bool PAIRS, bool COUNT, bool CHECK>
cudaError_t launch_s(const TraceArgs& a, const ScanArgs& o, int bps_cap, int sms, cudaStream_t s) {
  k_rows<PAIRS><<<sms * 8, 256, 0, s>>>(a, o, CHECK ? 1 : 0);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int occ = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_scan<FAST, PAIRS, COUNT, CHECK>, kScanBlock, 0);
  if (occ < 1) occ = 1;
  if (bps_cap > 0 && bps_cap < occ) occ = bps_cap;
  k_scan<FAST, PAIRS, COUNT, CHECK><<<sms * occ, kScanBlock, 0, s>>>(a, o);
  return cudaGetLastError();
}

template <bool FAST, bool PAIRS, bool COUNT>
cudaError_t launch_s1(const TraceArgs& a, const ScanArgs& o, uint32_t flags, int bps, int sms, cudaStream_t s) {
  return (flags & FX_CHECK_INDEX) ? launch_s<FAST, PAIRS, COUNT, true>(a, o, bps, sms, s)
                                  : launch_s<FAST, PAIRS, COUNT, false>(a, o, bps, sms, s);
}

template <bool FAST, bool PAIRS>
cudaError_t launch_s2(const TraceArgs& a, const ScanArgs& o, uint32_t flags, int bps, int sms, cudaStream_t s) {
  return (flags & FX_COUNT) ? launch_s1<FAST, PAIRS, true>(a, o, flags, bps, sms, s)
                            : launch_s1<FAST, PAIRS, false>(a, o, flags, bps, sms, s);
}

}  // namespace

cudaError_t launch_scan_ray(const TraceArgs& a, const ScanArgs& o, bool pairs, uint32_t flags,
                            int blocks_per_sm_cap, int sm_count, cudaStream_t s) {
  const bool fast = flags & FX_FAST_MATH;
  if (pairs) return fast ? launch_s2<true, true>(a, o, flags, blocks_per_sm_cap, sm_count, s)
                         : launch_s2<false, true>(a, o, flags, blocks_per_sm_cap, sm_count, s);
  return fast ? launch_s2<true, false>(a, o, flags, blocks_per_sm_cap, sm_count, s)
              : launch_s2<false, false>(a, o, flags, blocks_per_sm_cap, sm_count, s);
}

}  // namespace fx
