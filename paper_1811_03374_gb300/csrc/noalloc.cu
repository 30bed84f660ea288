// noalloc.cu -- intersect_closest_noalloc: the one-thread-per-pair closest-hit
// kernel with its per-ray scratch in a fixed device array instead of memory
// allocated per call.
//
// Who needs it: callers that must not allocate device memory while they run,
// for instance a renderer whose device memory is handed out up front by
// another allocator, or a real-time loop that cannot afford the implicit
// synchronisation of cudaMalloc / cudaFree.  intersect_closest allocates the
// naive kernel's scratch (one 64-bit key per ray) on every call; this entry
// point uses the static array below and allocates nothing.
//
// The array (FX_NOALLOC_MAX_RAYS keys, 8 MiB) lives in every GPU that loads
// the library until the process exits.  All calls share it: each call clears
// the keys it uses before the kernels run, and calls that overlap on the GPU
// (different streams, no ordering between them) race on it.
#include <cstdint>
#include <mutex>
#include <string>

#include "internal.h"

namespace {

__device__ __align__(256) unsigned long long g_noalloc_keys[FX_NOALLOC_MAX_RAYS];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned long long* g_keys_dev[kMaxDevices] = {};

// Device address of the array on the current device.  The name of a
// __device__ variable is only a host-side stand-in, so the address is looked
// up once per device (with that device current) and cached.
cudaError_t keys_address(unsigned long long** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_keys_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_keys);
    if (e != cudaSuccess) return e;
    g_keys_dev[dev] = static_cast<unsigned long long*>(p);
  }
  *out = g_keys_dev[dev];
  return cudaSuccess;
}

fx_status fail(fx_status s, const std::string& m) {
  fx::set_last_error(m);
  return s;
}

}  // namespace

extern "C" fx_status intersect_closest_noalloc(const fx_fibers* f, const float* rays, int64_t n_ray,
                                               const int32_t* row_ptr, const int32_t* seg_idx,
                                               int64_t n_pair, int32_t depth, uint32_t flags, float* tu,
                                               int32_t* seg, int32_t* leaf, void* stream) {
  if (!f) return fail(FX_EINVAL, "null fiber handle");
  // the key array looked up below is the current device's; the handle's
  // arrays must live on that device too
  if (!fx::on_handle_device(f)) return fail(FX_EDEVICE, "the current device is not the handle's device");
  if (n_ray < 0 || n_pair < 0) return fail(FX_EINVAL, "negative size");
  if (n_ray > FX_NOALLOC_MAX_RAYS)
    return fail(FX_EINVAL, "intersect_closest_noalloc: n_ray exceeds FX_NOALLOC_MAX_RAYS (1048576)");
  if (n_pair > 0x7fffffffLL) return fail(FX_EINVAL, "more than 2^31 - 1 pairs");
  if (depth < 0 || depth > fx::kMaxDepth) return fail(FX_EDEPTH, "depth outside [0, 23]");
  if (n_ray > 0 && (!rays || !row_ptr || !tu || !seg)) return fail(FX_EINVAL, "null argument");
  if (n_pair > 0 && !seg_idx) return fail(FX_EINVAL, "null seg_idx");
  if (n_ray == 0 && n_pair != 0) return fail(FX_EINVAL, "pairs without rays");
  if ((flags & FX_POLISH_FP64) && !leaf) return fail(FX_EINVAL, "FP64 polish needs the leaf output");
  if (n_ray == 0) return FX_OK;
  cudaStream_t s = (cudaStream_t)stream;
  unsigned long long* keys = nullptr;
  cudaError_t e = keys_address(&keys);
  if (e != cudaSuccess) return fail(FX_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
  // keys start at "no hit" (all ones), for the rays of this call only
  e = cudaMemsetAsync(keys, 0xff, sizeof(unsigned long long) * (size_t)n_ray, s);
  if (e != cudaSuccess) return fail(FX_ECUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
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
  a.tu = reinterpret_cast<float2*>(tu);
  a.seg = seg;
  a.leaf = leaf;
  a.queue = f->ws + FX_WS_QUEUE;
  a.status = f->ws + FX_WS_STATUS;
  a.counters = reinterpret_cast<unsigned long long*>(f->ws + FX_WS_WORDS);
  a.scratch = keys;
  e = fx::launch_naive(a, false, flags, s);
  if (e == cudaSuccess && (flags & FX_POLISH_FP64)) e = fx::launch_polish(a, f->seg_cp, s);
  if (e != cudaSuccess) return fail(FX_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
  return FX_OK;
}
