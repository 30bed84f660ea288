// fiberx_api.cu -- the C ABI of include/fiberx.h: argument checks, upload,
// launches and status.  All compute runs in the kernels of trace_kernels.cu
// and backward.cu; there is no host fallback.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "presplit.h"

namespace {

thread_local std::string g_err;

fx_status fail(fx_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

fx_status cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return FX_ECUDA;
}

#define FX_CUDA(call)                                   \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call); \
  } while (0)

unsigned long long* counters_of(const fx_fibers* f) {
  return reinterpret_cast<unsigned long long*>(f->ws + FX_WS_WORDS);
}

// Host-side checks shared by the intersect entries; no device access.
fx_status check_common(const fx_fibers* f, const float* rays, int64_t n_ray, const int32_t* row_ptr,
                       const int32_t* seg_idx, int64_t n_pair, int32_t depth) {
  if (!f) return fail(FX_EINVAL, "null fiber handle");
  if (!fx::on_handle_device(f)) return fail(FX_EDEVICE, "the current device is not the handle's device");
  if (n_ray < 0 || n_pair < 0) return fail(FX_EINVAL, "negative size");
  if (n_ray > 0x7fffffffLL || n_pair > 0x7fffffffLL)
    return fail(FX_EINVAL, "more than 2^31 - 1 rays or pairs");
  if (depth < 0 || depth > fx::kMaxDepth) return fail(FX_EDEPTH, "depth outside [0, 23]");
  if (n_ray > 0 && (!rays || !row_ptr)) return fail(FX_EINVAL, "null rays / row_ptr");
  if (n_pair > 0 && !seg_idx) return fail(FX_EINVAL, "null seg_idx");
  if (n_ray == 0 && n_pair != 0) return fail(FX_EINVAL, "pairs without rays");
  return FX_OK;
}

fx::TraceArgs make_args(const fx_fibers* f, const float* rays, int64_t n_ray, const int32_t* row_ptr,
                        const int32_t* seg_idx, int64_t n_pair, int32_t depth) {
  fx::TraceArgs a{};
  a.piece = f->piece;
  a.piece_begin = f->piece_begin;
  a.piece_info = f->piece_info;
  a.piece_rad = f->piece_rad;
  a.piece_root = f->piece_root;
  a.rays = reinterpret_cast<const float4*>(rays);
  a.row_ptr = row_ptr;
  a.seg_idx = seg_idx;
  a.n_ray = n_ray;
  a.n_pair = n_pair;
  a.n_seg = (int32_t)f->n_seg;
  a.depth = depth;
  a.chunk = f->launch.chunk;
  a.identity = f->identity ? 1 : 0;
  a.queue = f->ws + FX_WS_QUEUE;
  a.status = f->ws + FX_WS_STATUS;
  a.counters = counters_of(f);
  return a;
}

// The persistent variants; a.queue is this call's work-queue counter.
fx_status run_variant(const fx_fibers* f, fx::TraceArgs& a, bool pairs, uint32_t flags,
                      cudaStream_t s) {
  FX_CUDA(cudaMemsetAsync(a.queue, 0, sizeof(uint32_t), s));
  int variant = f->launch.variant;
  // rows of one or two candidates on average, segments not pre-split: the
  // per-ray kernel without a queue measured up to 2.6x the lane kernel on
  // such rows (single fibers, one ray per segment) and at worst 7 % behind
  // it; on pre-split segments (0.7x) and longer rows: the lane kernel
  if (variant == FX_VARIANT_AUTO)
    variant = (a.n_pair <= 2 * a.n_ray && f->identity) ? FX_VARIANT_RAY : FX_VARIANT_LANE;
  // the two-phase path covers closest hits on handles of single level-0 pieces
  if (variant == FX_VARIANT_FILTER && (pairs || !f->identity)) variant = FX_VARIANT_LANE;
  // FX_CHECK_INDEX also guards against a malformed row_ptr (rows clamped to
  // [0, n_pair]); the filter and warp variants stream several rows as one
  // range and rely on a well-formed CSR, so the lane kernel runs instead
  if ((flags & FX_CHECK_INDEX) && (variant == FX_VARIANT_FILTER || variant == FX_VARIANT_WARP))
    variant = FX_VARIANT_LANE;
  // the scan path covers handles of single level-0 pieces
  if (variant == FX_VARIANT_SCAN && !f->identity) variant = FX_VARIANT_LANE;
  if (variant == FX_VARIANT_FILTER) {
    int2* pass = nullptr;
    int32_t* ibuf = nullptr;
    FX_CUDA(cudaMallocFromPoolAsync((void**)&pass, sizeof(int2) * (size_t)std::max<int64_t>(1, a.n_pair),
                                    f->pool, s));
    cudaError_t e = cudaMallocFromPoolAsync((void**)&ibuf, sizeof(int32_t) * (size_t)(2 * a.n_ray + 4), f->pool, s);
    if (e != cudaSuccess) {
      cudaFreeAsync(pass, s);
      return cuda_fail(e, "cudaMallocFromPoolAsync filter lists");
    }
    fx::FilterArgs o{pass, ibuf, ibuf + a.n_ray, reinterpret_cast<uint32_t*>(ibuf + 2 * a.n_ray),
                     reinterpret_cast<uint32_t*>(ibuf + 2 * a.n_ray + 1)};
    e = cudaMemsetAsync(o.n_active, 0, 2 * sizeof(uint32_t), s);  // n_active, group_queue
    if (e == cudaSuccess) e = fx::launch_filter(a, o, flags, f->launch.blocks_per_sm, f->sm_count, s);
    cudaFreeAsync(ibuf, s);
    cudaFreeAsync(pass, s);
    if (e != cudaSuccess) return cuda_fail(e, "filter kernels");
    return FX_OK;
  }
  if (variant == FX_VARIANT_WARP) {
    FX_CUDA(fx::launch_warp_ray(a, pairs, flags, f->launch.blocks_per_sm, f->sm_count, s));
  } else if (variant == FX_VARIANT_RAY) {
    // closest hits: room for a walk per ray that the first pass may leave to
    // the second (128 bytes each, from the pool; only the saved ones are
    // written), the count in the first 256 bytes
    fx::RayDefer d{nullptr, nullptr, 0};
    char* buf = nullptr;
    if (!pairs) {
      const uint32_t cap = (uint32_t)a.n_ray;
      FX_CUDA(cudaMallocFromPoolAsync((void**)&buf, 256 + fx::ray_walk_bytes() * cap, f->pool, s));
      d = fx::RayDefer{buf + 256, reinterpret_cast<uint32_t*>(buf), cap};
    }
    cudaError_t e = buf ? cudaMemsetAsync(buf, 0, sizeof(uint32_t), s) : cudaSuccess;
    if (e == cudaSuccess) e = fx::launch_ray(a, pairs, flags, d, f->sm_count, s);
    if (buf) cudaFreeAsync(buf, s);
    if (e != cudaSuccess) return cuda_fail(e, "per-ray kernels");
  } else if (variant == FX_VARIANT_SCAN) {
    int4* act = nullptr;
    FX_CUDA(cudaMallocFromPoolAsync((void**)&act, sizeof(int4) * (size_t)(a.n_ray + 1), f->pool, s));
    fx::ScanArgs o{act + 1, reinterpret_cast<uint32_t*>(act)};
    cudaError_t e = cudaMemsetAsync(o.n_act, 0, sizeof(uint32_t), s);
    if (e == cudaSuccess) e = fx::launch_scan_ray(a, o, pairs, flags, f->launch.blocks_per_sm, f->sm_count, s);
    cudaFreeAsync(act, s);
    if (e != cudaSuccess) return cuda_fail(e, "scan kernels");
  } else {
    FX_CUDA(fx::launch_lane_ray(a, pairs, flags, f->launch.blocks_per_sm, f->sm_count, s));
  }
  return FX_OK;
}

fx_status run_forward(const fx_fibers* f, fx::TraceArgs& a, bool pairs, uint32_t flags,
                      cudaStream_t s) {
  if (a.n_ray == 0) return FX_OK;
  if (flags & FX_KERNEL_NAIVE) {
    unsigned long long* scratch = nullptr;
    if (!pairs) {
      FX_CUDA(cudaMallocFromPoolAsync((void**)&scratch, sizeof(unsigned long long) * a.n_ray, f->pool, s));
      const cudaError_t e0 = cudaMemsetAsync(scratch, 0xff, sizeof(unsigned long long) * a.n_ray, s);
      if (e0 != cudaSuccess) {
        cudaFreeAsync(scratch, s);
        return cuda_fail(e0, "naive kernel keys");
      }
    }
    a.scratch = scratch;
    cudaError_t e = fx::launch_naive(a, pairs, flags, s);
    if (scratch) cudaFreeAsync(scratch, s);
    if (e != cudaSuccess) return cuda_fail(e, "naive kernel launch");
    return FX_OK;
  }
  // each call's work-queue counter comes from the handle's pool on the
  // call's stream, so that calls on one handle in unordered streams do not
  // share one
  uint32_t* queue = nullptr;
  FX_CUDA(cudaMallocFromPoolAsync((void**)&queue, sizeof(uint32_t), f->pool, s));
  a.queue = queue;
  const fx_status st = run_variant(f, a, pairs, flags, s);
  cudaFreeAsync(queue, s);
  return st;
}

bool device_is_sm103(int dev, int* sm_count) {
  cudaDeviceProp p{};
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return false;
  *sm_count = p.multiProcessorCount;
  return p.major == 10 && p.minor == 3;
}

// Reads n_seg x n_cp x 4 floats from host or device memory and checks them:
// finite, radius >= 0.
fx_status read_cps(const float* cps, int64_t n_seg, int n_cp, int32_t on_device, cudaStream_t s,
                   std::vector<float>& host) {
  host.resize((size_t)n_seg * n_cp * 4);
  if (n_seg > 0) {
    if (on_device) {
      FX_CUDA(cudaMemcpyAsync(host.data(), cps, host.size() * sizeof(float), cudaMemcpyDeviceToHost, s));
      FX_CUDA(cudaStreamSynchronize(s));
    } else {
      std::memcpy(host.data(), cps, host.size() * sizeof(float));
    }
  }
  for (size_t i = 0; i < host.size(); ++i) {
    if (!std::isfinite(host[i])) return fail(FX_EINVAL, "non-finite control point");
    if (i % 4 == 3 && host[i] < 0.0f) return fail(FX_EINVAL, "negative radius");
  }
  return FX_OK;
}

// Upload of cubic segments given in double precision (n_seg x 16); `host` is
// the FP32 copy kept on the device for the polish, adjoint and normals.
fx_status upload_cubics(const std::vector<double>& cps64, const std::vector<float>& host, int64_t n_seg,
                        const fx_upload_opts* opts, cudaStream_t s, fx_fibers** out) {
  const int max_presplit = opts ? opts->max_presplit : 8;
  const bool thick = opts ? opts->thick_check != 0 : true;
  if (max_presplit < 0 || max_presplit > 8) return fail(FX_EINVAL, "max_presplit outside [0, 8]");
  int dev = 0, sms = 0;
  FX_CUDA(cudaGetDevice(&dev));
  if (!device_is_sm103(dev, &sms)) return fail(FX_EDEVICE, "current device is not sm_103");

  std::vector<fx::PieceRec> pieces;
  std::vector<int32_t> begin;
  const int nt = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  fx::presplit_all(cps64.data(), n_seg, max_presplit, thick, n_seg > 4096 ? nt : 1, pieces, begin);

  fx_fibers* f = new (std::nothrow) fx_fibers();
  if (!f) return fail(FX_ENOMEM, "handle allocation");
  f->device = dev;
  f->sm_count = sms;
  f->n_seg = n_seg;
  f->n_piece = (int64_t)pieces.size();
  std::vector<float> packed(pieces.size() * 16);
  std::vector<int32_t> info(pieces.size());
  std::vector<float> rad(pieces.size());
  std::vector<float> rootrec(pieces.size() * 8);
  for (size_t k = 0; k < pieces.size(); ++k) {
    std::memcpy(&packed[16 * k], pieces[k].pdt, sizeof(pieces[k].pdt));
    rad[k] = pieces[k].root_radius;
    for (int a = 0; a < 3; ++a) {
      rootrec[8 * k + a] = pieces[k].pdt[a];          // p
      rootrec[8 * k + 4 + a] = pieces[k].pdt[4 + a];  // d
    }
    rootrec[8 * k + 3] = pieces[k].root_radius;
    rootrec[8 * k + 7] = pieces[k].bound_radius;
    info[k] = pieces[k].level | (pieces[k].off << 4) | (pieces[k].unsupported ? (int32_t)0x80000000 : 0);
    f->max_level = std::max(f->max_level, pieces[k].level);
    if (pieces[k].unsupported) f->n_unsupported++;
    if (pieces[k].level != 0 || pieces[k].unsupported) f->identity = false;
  }
  for (int64_t i = 0; i < n_seg; ++i)
    if (begin[i + 1] - begin[i] > 1) f->n_presplit++;

  auto cleanup = [&](fx_status st, cudaError_t e, const char* where) {
    fiber_free(f);
    return e != cudaSuccess ? cuda_fail(e, where) : st;
  };
  cudaError_t e;
  const size_t np = std::max<size_t>(1, pieces.size()), ns = (size_t)std::max<int64_t>(1, n_seg);
  if ((e = cudaMalloc((void**)&f->piece, np * 64)) != cudaSuccess) return cleanup(FX_ENOMEM, e, "cudaMalloc pieces");
  if ((e = cudaMalloc((void**)&f->piece_begin, (ns + 1) * 4)) != cudaSuccess) return cleanup(FX_ENOMEM, e, "cudaMalloc begin");
  if ((e = cudaMalloc((void**)&f->piece_info, np * 4)) != cudaSuccess) return cleanup(FX_ENOMEM, e, "cudaMalloc info");
  if ((e = cudaMalloc((void**)&f->seg_cp, ns * 64)) != cudaSuccess) return cleanup(FX_ENOMEM, e, "cudaMalloc seg_cp");
  if ((e = cudaMalloc((void**)&f->piece_rad, np * 4)) != cudaSuccess) return cleanup(FX_ENOMEM, e, "cudaMalloc rad");
  if ((e = cudaMalloc((void**)&f->piece_root, np * 32)) != cudaSuccess) return cleanup(FX_ENOMEM, e, "cudaMalloc root");
  {
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    if ((e = cudaMemPoolCreate(&f->pool, &props)) != cudaSuccess) return cleanup(FX_ECUDA, e, "cudaMemPoolCreate");
    uint64_t keep = UINT64_MAX;
    if ((e = cudaMemPoolSetAttribute(f->pool, cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
      return cleanup(FX_ECUDA, e, "cudaMemPoolSetAttribute");
  }
  const size_t ws_bytes = FX_WS_WORDS * 4 + 8 * 8;
  if ((e = cudaMalloc((void**)&f->ws, ws_bytes)) != cudaSuccess) return cleanup(FX_ENOMEM, e, "cudaMalloc ws");
  if ((e = cudaMemsetAsync(f->ws, 0, ws_bytes, s)) != cudaSuccess) return cleanup(FX_ECUDA, e, "memset ws");
  if (!pieces.empty() &&
      (e = cudaMemcpyAsync(f->piece, packed.data(), packed.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cleanup(FX_ECUDA, e, "copy pieces");
  if ((e = cudaMemcpyAsync(f->piece_begin, begin.data(), begin.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cleanup(FX_ECUDA, e, "copy begin");
  if (!info.empty() &&
      (e = cudaMemcpyAsync(f->piece_info, info.data(), info.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cleanup(FX_ECUDA, e, "copy info");
  if (!rootrec.empty() &&
      (e = cudaMemcpyAsync(f->piece_root, rootrec.data(), rootrec.size() * 4, cudaMemcpyHostToDevice, s)) !=
          cudaSuccess)
    return cleanup(FX_ECUDA, e, "copy root records");
  if (!rad.empty() &&
      (e = cudaMemcpyAsync(f->piece_rad, rad.data(), rad.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cleanup(FX_ECUDA, e, "copy rad");
  if (n_seg > 0 &&
      (e = cudaMemcpyAsync(f->seg_cp, host.data(), host.size() * 4, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cleanup(FX_ECUDA, e, "copy cps");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cleanup(FX_ECUDA, e, "upload sync");
  *out = f;
  return FX_OK;
}

}  // namespace

namespace fx {
void set_last_error(const std::string& msg) { g_err = msg; }
}  // namespace fx

extern "C" {

const char* fx_last_error(void) { return g_err.c_str(); }

fx_status fx_fma_peak(int32_t blocks_per_sm, int32_t iters, float* ms, double* tflops, void* stream) {
  if (!ms || !tflops) return fail(FX_EINVAL, "null output");
  if (blocks_per_sm < 1 || blocks_per_sm > 8 || iters < 1) return fail(FX_EINVAL, "blocks_per_sm or iters out of range");
  int dev = 0, sms = 0;
  FX_CUDA(cudaGetDevice(&dev));
  FX_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  double flops = 0.0;
  FX_CUDA(fx::fma_peak(sms, blocks_per_sm, iters, ms, &flops, (cudaStream_t)stream));
  *tflops = flops / (*ms * 1e-3) / 1e12;
  return FX_OK;
}

int32_t fx_version(void) { return 10000; }

fx_status fiber_upload(const float* cps, int64_t n_seg, int32_t cps_on_device, const fx_upload_opts* opts,
                       void* stream, fx_fibers** out) {
  if (!out) return fail(FX_EINVAL, "null output handle");
  *out = nullptr;
  if (n_seg < 0 || n_seg > 0x7ffffffeLL) return fail(FX_EINVAL, "n_seg out of range");
  if (n_seg > 0 && !cps) return fail(FX_EINVAL, "null control points");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> host;
  fx_status st = read_cps(cps, n_seg, 4, cps_on_device, s, host);
  if (st != FX_OK) return st;
  std::vector<double> cps64(host.begin(), host.end());
  return upload_cubics(cps64, host, n_seg, opts, s, out);
}

fx_status fiber_upload_quadratic(const float* cps, int64_t n_seg, int32_t cps_on_device,
                                 const fx_upload_opts* opts, void* stream, fx_fibers** out) {
  if (!out) return fail(FX_EINVAL, "null output handle");
  *out = nullptr;
  if (n_seg < 0 || n_seg > 0x7ffffffeLL) return fail(FX_EINVAL, "n_seg out of range");
  if (n_seg > 0 && !cps) return fail(FX_EINVAL, "null control points");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<float> host;
  fx_status st = read_cps(cps, n_seg, 3, cps_on_device, s, host);
  if (st != FX_OK) return st;
  // exact degree elevation (all four components): q0 = p0, q1 = (p0 + 2 p1) / 3,
  // q2 = (2 p1 + p2) / 3, q3 = p2 -- the same curve and parametrisation
  std::vector<double> cps64((size_t)n_seg * 16);
  std::vector<float> cps32((size_t)n_seg * 16);
  for (int64_t i = 0; i < n_seg; ++i) {
    const float* q = &host[12 * i];
    double* c = &cps64[16 * i];
    for (int a = 0; a < 4; ++a) {
      const double p0 = q[a], p1 = q[4 + a], p2 = q[8 + a];
      c[a] = p0;
      c[4 + a] = (p0 + 2.0 * p1) / 3.0;
      c[8 + a] = (2.0 * p1 + p2) / 3.0;
      c[12 + a] = p2;
    }
    for (int k = 0; k < 16; ++k) cps32[16 * i + k] = (float)c[k];
  }
  st = upload_cubics(cps64, cps32, n_seg, opts, s, out);
  if (st == FX_OK) (*out)->quadratic = true;
  return st;
}


void fiber_free(fx_fibers* f) {
  if (!f) return;
  cudaFree(f->piece);
  cudaFree(f->piece_begin);
  cudaFree(f->piece_info);
  cudaFree(f->seg_cp);
  cudaFree(f->piece_rad);
  cudaFree(f->piece_root);
  cudaFree(f->ws);
  cudaFree(f->stage);
  for (cudaEvent_t e : f->host_ev)
    if (e) cudaEventDestroy(e);
  if (f->copy_in) cudaStreamDestroy(f->copy_in);
  if (f->copy_out) cudaStreamDestroy(f->copy_out);
  for (cudaStream_t c : f->compute)
    if (c) cudaStreamDestroy(c);
  if (f->pool) cudaMemPoolDestroy(f->pool);  // released once its last allocation is freed
  delete f;
}

fx_status fiber_info(const fx_fibers* f, fx_fibers_info* out) {
  if (!f || !out) return fail(FX_EINVAL, "null argument");
  out->n_seg = f->n_seg;
  out->n_piece = f->n_piece;
  out->n_presplit = f->n_presplit;
  out->n_unsupported = f->n_unsupported;
  out->max_level = f->max_level;
  out->sm_count = f->sm_count;
  return FX_OK;
}

fx_status fx_set_launch(fx_fibers* f, const fx_launch* cfg) {
  if (!f || !cfg) return fail(FX_EINVAL, "null argument");
  const int b = cfg->block;
  if (!(b == 64 || b == 128 || b == 256)) return fail(FX_EINVAL, "block must be 64, 128 or 256");
  if (cfg->blocks_per_sm < 0 || cfg->blocks_per_sm > 16) return fail(FX_EINVAL, "blocks_per_sm outside [0, 16]");
  if (cfg->chunk < 1 || cfg->chunk > 1024) return fail(FX_EINVAL, "chunk outside [1, 1024]");
  if (cfg->variant < FX_VARIANT_AUTO || cfg->variant > FX_VARIANT_RAY) return fail(FX_EINVAL, "unknown variant");
  f->launch = *cfg;
  return FX_OK;
}

fx_status fx_get_launch(const fx_fibers* f, fx_launch* cfg) {
  if (!f || !cfg) return fail(FX_EINVAL, "null argument");
  *cfg = f->launch;
  return FX_OK;
}

fx_status intersect_closest(const fx_fibers* f, const float* rays, int64_t n_ray, const int32_t* row_ptr,
                            const int32_t* seg_idx, int64_t n_pair, int32_t depth, const int8_t* ray_depth,
                            uint32_t flags, float* tu, int32_t* seg, int32_t* leaf, void* stream) {
  fx_status st = check_common(f, rays, n_ray, row_ptr, seg_idx, n_pair, depth);
  if (st != FX_OK) return st;
  if (n_ray > 0 && (!tu || !seg)) return fail(FX_EINVAL, "null tu / seg output");
  cudaStream_t s = (cudaStream_t)stream;
  fx::TraceArgs a = make_args(f, rays, n_ray, row_ptr, seg_idx, n_pair, depth);
  a.ray_depth = ray_depth;
  a.tu = reinterpret_cast<float2*>(tu);
  a.seg = seg;
  a.leaf = leaf;
  int32_t* tmp_leaf = nullptr;
  if ((flags & FX_POLISH_FP64) && !leaf && n_ray > 0) {
    FX_CUDA(cudaMallocFromPoolAsync((void**)&tmp_leaf, sizeof(int32_t) * n_ray, f->pool, s));
    a.leaf = tmp_leaf;
  }
  st = run_forward(f, a, false, flags, s);
  if (st == FX_OK && (flags & FX_POLISH_FP64)) {
    cudaError_t e = fx::launch_polish(a, f->seg_cp, s);
    if (e != cudaSuccess) st = cuda_fail(e, "polish launch");
  }
  if (tmp_leaf) cudaFreeAsync(tmp_leaf, s);
  return st;
}

fx_status intersect_pairs(const fx_fibers* f, const float* rays, int64_t n_ray, const int32_t* row_ptr,
                          const int32_t* seg_idx, int64_t n_pair, int32_t depth, const int8_t* ray_depth,
                          uint32_t flags, float* tu, int32_t* leaf, uint8_t* pair_flags, void* stream) {
  fx_status st = check_common(f, rays, n_ray, row_ptr, seg_idx, n_pair, depth);
  if (st != FX_OK) return st;
  if (n_pair > 0 && !tu) return fail(FX_EINVAL, "null tu output");
  if (flags & FX_POLISH_FP64) return fail(FX_EUNSUPPORTED, "FP64 polish applies to intersect_closest only");
  fx::TraceArgs a = make_args(f, rays, n_ray, row_ptr, seg_idx, n_pair, depth);
  a.ray_depth = ray_depth;
  a.tu = reinterpret_cast<float2*>(tu);
  a.leaf = leaf;
  a.pair_flags = pair_flags;
  return run_forward(f, a, true, flags, (cudaStream_t)stream);
}

fx_status intersect_backward(const fx_fibers* f, const float* rays, int64_t n_ray, const float* tu,
                             const int32_t* seg, const float* grad_t, float* grad_cps,
                             unsigned long long* n_skipped_dev, void* stream) {
  if (!f) return fail(FX_EINVAL, "null fiber handle");
  if (!fx::on_handle_device(f)) return fail(FX_EDEVICE, "the current device is not the handle's device");
  if (n_ray < 0 || n_ray > 0x7fffffffLL) return fail(FX_EINVAL, "n_ray out of range");
  if (n_ray == 0) return FX_OK;
  if (!rays || !tu || !seg || !grad_t || !grad_cps) return fail(FX_EINVAL, "null argument");
  FX_CUDA(fx::launch_backward(f->seg_cp, f->n_seg, f->quadratic, reinterpret_cast<const float4*>(rays), n_ray,
                              reinterpret_cast<const float2*>(tu), seg, grad_t, grad_cps, n_skipped_dev,
                              (cudaStream_t)stream));
  return FX_OK;
}

fx_status intersect_counts(const fx_fibers* f, const float* rays, int64_t n_ray, const int32_t* row_ptr,
                           const int32_t* seg_idx, int64_t n_pair, int32_t depth, uint32_t flags,
                           uint32_t* counts, void* stream) {
  fx_status st = check_common(f, rays, n_ray, row_ptr, seg_idx, n_pair, depth);
  if (st != FX_OK) return st;
  if (n_ray > 0 && !counts) return fail(FX_EINVAL, "null counts output");
  fx::TraceArgs a = make_args(f, rays, n_ray, row_ptr, seg_idx, n_pair, depth);
  FX_CUDA(fx::launch_counts(a, counts, (flags & FX_COUNT_BOXES) != 0, flags, (cudaStream_t)stream));
  return FX_OK;
}

fx_status intersect_normals(const fx_fibers* f, const float* rays, int64_t n_ray, const float* tu,
                            const int32_t* seg, const int32_t* leaf, int32_t depth, const int8_t* ray_depth,
                            uint32_t flags, float* normal, void* stream) {
  if (!f) return fail(FX_EINVAL, "null fiber handle");
  if (!fx::on_handle_device(f)) return fail(FX_EDEVICE, "the current device is not the handle's device");
  if (n_ray < 0 || n_ray > 0x7fffffffLL) return fail(FX_EINVAL, "n_ray out of range");
  if (depth < 0 || depth > fx::kMaxDepth) return fail(FX_EDEPTH, "depth outside [0, 23]");
  if (n_ray == 0) return FX_OK;
  if (!rays || !tu || !seg || !leaf || !normal) return fail(FX_EINVAL, "null argument");
  fx::TraceArgs a = make_args(f, rays, n_ray, nullptr, nullptr, 0, depth);
  a.ray_depth = ray_depth;
  a.tu = reinterpret_cast<float2*>(const_cast<float*>(tu));
  a.seg = const_cast<int32_t*>(seg);
  a.leaf = const_cast<int32_t*>(leaf);
  FX_CUDA(fx::launch_normals(a, f->seg_cp, normal, flags, (cudaStream_t)stream));
  return FX_OK;
}

fx_status intersect_closest_host(fx_fibers* f, const float* rays, int64_t n_ray, const int32_t* row_ptr,
                                 const int32_t* seg_idx, int64_t n_pair, int32_t depth, const int8_t* ray_depth,
                                 uint32_t flags, float* tu, int32_t* seg, int32_t* leaf, void* stream) {
  fx_status st = check_common(f, rays, n_ray, row_ptr, seg_idx, n_pair, depth);
  if (st != FX_OK) return st;
  if (n_ray > 0 && (!tu || !seg)) return fail(FX_EINVAL, "null tu / seg output");
  if (n_ray == 0) return FX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  const size_t b_rays = al((size_t)n_ray * 32), b_rp = al((size_t)(n_ray + 1) * 4),
               b_si = al((size_t)std::max<int64_t>(n_pair, 1) * 4), b_tu = al((size_t)n_ray * 8),
               b_seg = al((size_t)n_ray * 4), b_leaf = al((size_t)n_ray * 4), b_dep = al((size_t)n_ray);
  const size_t need = b_rays + b_rp + b_si + b_tu + b_seg + b_leaf + b_dep;
  if (need > f->stage_bytes) {
    FX_CUDA(cudaStreamSynchronize(s));
    cudaFree(f->stage);
    f->stage = nullptr;
    f->stage_bytes = 0;
    if (cudaMalloc(&f->stage, need) != cudaSuccess) return fail(FX_ENOMEM, "staging allocation");
    f->stage_bytes = need;
  }
  if (!f->copy_in) {
    FX_CUDA(cudaStreamCreateWithFlags(&f->copy_in, cudaStreamNonBlocking));
    FX_CUDA(cudaStreamCreateWithFlags(&f->copy_out, cudaStreamNonBlocking));
    for (cudaStream_t& c : f->compute) FX_CUDA(cudaStreamCreateWithFlags(&c, cudaStreamNonBlocking));
    for (cudaEvent_t& e : f->host_ev) FX_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  char* base = (char*)f->stage;
  float* d_rays = (float*)base;
  int32_t* d_rp = (int32_t*)(base + b_rays);
  int32_t* d_si = (int32_t*)(base + b_rays + b_rp);
  float* d_tu = (float*)(base + b_rays + b_rp + b_si);
  int32_t* d_seg = (int32_t*)(base + b_rays + b_rp + b_si + b_tu);
  int32_t* d_leaf = (leaf || (flags & FX_POLISH_FP64)) ? (int32_t*)(base + b_rays + b_rp + b_si + b_tu + b_seg)
                                                       : nullptr;
  int8_t* d_dep = ray_depth ? (int8_t*)(base + b_rays + b_rp + b_si + b_tu + b_seg + b_leaf) : nullptr;

  // Rows are cut into up to kFxHostChunks chunks of about equal input bytes
  // (32 per ray, 4 per row_ptr entry, 4 per pair), found by bisection on the
  // host row_ptr.  Chunk c is copied in on copy_in, intersected on compute
  // stream c mod kFxHostStreams once its copy is done, and its results copied
  // out on copy_out, so copies overlap the other chunks' kernels, and a
  // chunk's kernels overlap the tail of the chunk before (a kernel lasts at
  // least as long as its longest rows' chains of scans and node steps).  Each chunk's
  // kernels read the CSR in place (row_ptr values index the whole seg_idx
  // staging), and the copies run in row order, so a chunk's pairs have
  // arrived with it.  No kernel reads the ray of an empty row, so rays are
  // copied only in blocks of kRayBlock rows that hold a candidate, one copy
  // per run of such blocks.  The pair-parallel naive kernel indexes pairs of
  // the whole CSR: one chunk.
#ifndef FX_HOST_CHUNK_MB
#define FX_HOST_CHUNK_MB 32
#endif
#ifndef FX_HOST_RAY_BLOCK
#define FX_HOST_RAY_BLOCK 8192
#endif
#ifndef FX_HOST_LAST_SHARE
#define FX_HOST_LAST_SHARE 25
#endif
  constexpr int64_t kChunkBytes = (int64_t)FX_HOST_CHUNK_MB << 20;
  constexpr int64_t kRayBlock = FX_HOST_RAY_BLOCK;
  const int64_t in_bytes = 36 * n_ray + 4 * n_pair;
  int n_chunk = (int)std::min<int64_t>(kFxHostChunks, std::max<int64_t>(1, in_bytes / kChunkBytes));
  if (flags & FX_KERNEL_NAIVE) n_chunk = 1;
  auto pairs_at = [&](int64_t r) { return std::min<int64_t>(std::max<int32_t>(row_ptr[r], 0), n_pair); };
  int64_t cut[kFxHostChunks + 1];
  cut[0] = 0;
  cut[n_chunk] = n_ray;
  // the last chunk takes FX_HOST_LAST_SHARE percent of the bytes (its
  // kernels and copy out are the part of the step no copy in overlaps), the
  // others share the rest evenly
  const int64_t last_share = n_chunk > 1 ? std::min<int64_t>(FX_HOST_LAST_SHARE, 100 / n_chunk) : 100;
  for (int c = 1; c < n_chunk; ++c) {
    const int64_t target = in_bytes * (100 - last_share) / 100 * c / (n_chunk - 1);
    int64_t lo = cut[c - 1], hi = n_ray;  // smallest r in [lo, hi] with bytes(r) >= target
    while (lo < hi) {
      const int64_t mid = lo + (hi - lo) / 2;
      if (36 * mid + 4 * pairs_at(mid) >= target) hi = mid;
      else lo = mid + 1;
    }
    cut[c] = lo;
  }

  cudaEvent_t* ev_in = f->host_ev + 1;
  cudaEvent_t* ev_done = f->host_ev + 1 + kFxHostChunks;
  cudaError_t e = cudaEventRecord(f->host_ev[0], s);  // work queued on the caller's stream comes first
  if (e == cudaSuccess) e = cudaStreamWaitEvent(f->copy_in, f->host_ev[0], 0);
  for (int k = 0; k < kFxHostStreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(f->compute[k], f->host_ev[0], 0);
  f->host_h2d = f->host_d2h = 0;
  auto empty_block = [&](int64_t b, int64_t b_end) { return pairs_at(b) == pairs_at(b_end); };
  // Rays in pinned host memory that the runtime maps into the device's
  // address space are read by the kernels in place, over the host link, 32
  // bytes per ray that has a candidate; other rays are copied.  The bytes are
  // counted the same way either way (the rays of blocks of rows that hold a
  // candidate).
  auto mapped = [](const void* p) -> void* {
    cudaPointerAttributes pa{};
    if (cudaPointerGetAttributes(&pa, p) != cudaSuccess) {
      cudaGetLastError();  // a failed query leaves no sticky error behind: copy instead
      return nullptr;
    }
    return pa.type == cudaMemoryTypeHost ? pa.devicePointer : nullptr;
  };
  // (Results are still written to device staging and copied out: written in
  // place over the host link they lengthen every lane's chain, measured
  // 0.98 ms per hair frame against 0.88.)
  const float* rays_in_place = static_cast<const float*>(mapped(rays));
  // each chunk's range of pairs, in row order (together they cover all pairs)
  int64_t plo[kFxHostChunks], phi[kFxHostChunks];
  {
    int64_t p_done = 0;
    for (int c = 0; c < n_chunk; ++c) {
      plo[c] = p_done;
      phi[c] = c + 1 == n_chunk ? n_pair : std::max(p_done, pairs_at(cut[c + 1]));
      p_done = phi[c];
    }
  }
  // Copy order: row order, except that the chunk with the fewest rays goes
  // last.  What no copy in overlaps is the last chunk's kernels and its copy
  // out; the copy out is 12 to 16 bytes per ray, and the chunk with the
  // fewest rays has the smallest (the candidate-free rows of an image lie in
  // wide chunks of few pairs).
  int order[kFxHostChunks];
  int last = 0;
  for (int c = 0; c < n_chunk; ++c)
    if (cut[c + 1] - cut[c] < cut[last + 1] - cut[last]) last = c;
  for (int c = 0, k = 0; c < n_chunk; ++c)
    if (c != last) order[k++] = c;
  order[n_chunk - 1] = last;
  for (int k = 0; k < n_chunk && e == cudaSuccess && st == FX_OK; ++k) {
    const int c = order[k];
    const int64_t r0 = cut[c], r1 = cut[c + 1], n = r1 - r0;
    const int64_t p_done = plo[c], p1 = phi[c];
    for (int64_t b = r0; b < r1 && e == cudaSuccess;) {
      int64_t run_end = std::min(b + kRayBlock, r1);
      if (empty_block(b, run_end)) {
        b = run_end;
        continue;
      }
      while (run_end < r1 && !empty_block(run_end, std::min(run_end + kRayBlock, r1)))
        run_end = std::min(run_end + kRayBlock, r1);
      if (!rays_in_place)
        e = cudaMemcpyAsync(d_rays + 8 * b, rays + 8 * b, (size_t)(run_end - b) * 32, cudaMemcpyHostToDevice,
                            f->copy_in);
      f->host_h2d += (run_end - b) * 32;
      b = run_end;
    }
    f->host_h2d += (n + 1) * 4 + std::max<int64_t>(0, p1 - p_done) * 4;
    if (e == cudaSuccess && d_dep && n > 0) {
      e = cudaMemcpyAsync(d_dep + r0, ray_depth + r0, (size_t)n, cudaMemcpyHostToDevice, f->copy_in);
      f->host_h2d += n;
    }
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_rp + r0, row_ptr + r0, (size_t)(n + 1) * 4, cudaMemcpyHostToDevice, f->copy_in);
    if (e == cudaSuccess && p1 > p_done)
      e = cudaMemcpyAsync(d_si + p_done, seg_idx + p_done, (size_t)(p1 - p_done) * 4, cudaMemcpyHostToDevice,
                          f->copy_in);
    cudaStream_t cs = f->compute[k % kFxHostStreams];
    if (e == cudaSuccess) e = cudaEventRecord(ev_in[c], f->copy_in);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev_in[c], 0);
    if (e != cudaSuccess || n == 0) continue;
    st = intersect_closest(f, (rays_in_place ? rays_in_place : d_rays) + 8 * r0, n, d_rp + r0, d_si, n_pair, depth,
                           d_dep ? d_dep + r0 : nullptr, flags, d_tu + 2 * r0, d_seg + r0,
                           d_leaf ? d_leaf + r0 : nullptr, cs);
    if (st != FX_OK) break;
    f->host_d2h += n * (leaf ? 16 : 12);
    e = cudaEventRecord(ev_done[c], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(f->copy_out, ev_done[c], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(tu + 2 * r0, d_tu + 2 * r0, (size_t)n * 8, cudaMemcpyDeviceToHost, f->copy_out);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(seg + r0, d_seg + r0, (size_t)n * 4, cudaMemcpyDeviceToHost, f->copy_out);
    if (e == cudaSuccess && leaf)
      e = cudaMemcpyAsync(leaf + r0, d_leaf + r0, (size_t)n * 4, cudaMemcpyDeviceToHost, f->copy_out);
  }
  // nothing of this call may still touch the caller's buffers on return
  const cudaError_t e_in = cudaStreamSynchronize(f->copy_in);
  cudaError_t e_s = cudaStreamSynchronize(s);
  for (int k = 0; k < kFxHostStreams; ++k) {
    const cudaError_t e_k = cudaStreamSynchronize(f->compute[k]);
    if (e_s == cudaSuccess) e_s = e_k;
  }
  const cudaError_t e_out = cudaStreamSynchronize(f->copy_out);
  if (st != FX_OK) return st;
  if (e != cudaSuccess) return cuda_fail(e, "host-buffer pipeline");
  if (e_in != cudaSuccess) return cuda_fail(e_in, "copy-in stream");
  if (e_s != cudaSuccess) return cuda_fail(e_s, "intersect stream");
  if (e_out != cudaSuccess) return cuda_fail(e_out, "copy-out stream");
  return FX_OK;
}

fx_status fx_host_bytes(const fx_fibers* f, int64_t* h2d, int64_t* d2h) {
  if (!f || !h2d || !d2h) return fail(FX_EINVAL, "null argument");
  *h2d = f->host_h2d;
  *d2h = f->host_d2h;
  return FX_OK;
}

fx_status fx_counters(fx_fibers* f, void* stream, uint64_t* out5, int32_t reset) {
  if (!f || !out5) return fail(FX_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  FX_CUDA(cudaMemcpyAsync(out5, counters_of(f), 5 * 8, cudaMemcpyDeviceToHost, s));
  if (reset) FX_CUDA(cudaMemsetAsync(counters_of(f), 0, 8 * 8, s));
  FX_CUDA(cudaStreamSynchronize(s));
  return FX_OK;
}

fx_status fx_stream_status(fx_fibers* f, void* stream, uint32_t* device_flags) {
  if (!f || !device_flags) return fail(FX_EINVAL, "null argument");
  cudaStream_t s = (cudaStream_t)stream;
  FX_CUDA(cudaStreamSynchronize(s));
  FX_CUDA(cudaMemcpy(device_flags, f->ws + FX_WS_STATUS, 4, cudaMemcpyDeviceToHost));
  FX_CUDA(cudaMemset(f->ws + FX_WS_STATUS, 0, 4));
  return FX_OK;
}

}  // extern "C"
