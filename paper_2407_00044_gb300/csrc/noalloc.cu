// sk_gemm_static_ws: sk_gemm with the workspace in a fixed, library-owned
// device array instead of caller-provided memory.
//
// Some callers cannot allocate device memory: code whose device memory is
// owned entirely by another allocator (a framework's caching allocator or a
// pre-reserved memory pool) must not call cudaMalloc -- it may synchronise
// the device and can fail once the pool has claimed the memory -- and some
// plug-in style callers have nowhere to keep a workspace pointer between
// calls.  This entry point serves them: the Stream-K partial slots, flags
// and status word live in `g_static_ws` below, a file-scope __device__ array
// that every GPU which loads this library holds until the process exits.
//
// It allocates nothing: no cudaMalloc/cudaFree and no allocating library
// routine.  It runs the same kernels as sk_gemm by passing the array's
// device address as the workspace.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/skgemm.h"
#include "common.cuh"

namespace {

// 12 MiB: room for 128x128 tiles on up to 191 CTAs, or 128x256 tiles on up
// to 95 CTAs (each CTA needs one FP32 tile of partials, plus 1 KB of
// status word and flags).
constexpr size_t kStaticWsBytes = (size_t)12 << 20;

static __device__ __align__(256) unsigned char g_static_ws[kStaticWsBytes];

std::mutex g_mu;
void *g_ptr[64] = {};

// Device address of g_static_ws on the current device, looked up once per
// device.  Host code cannot use `g_static_ws` itself as a device address.
sk_status static_ws_address(void **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return SK_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_static_ws) != cudaSuccess || !p) return SK_ERR_CUDA;
    g_ptr[dev] = p;
  }
  *out = g_ptr[dev];
  return SK_OK;
}

}  // namespace

extern "C" SK_API sk_status sk_gemm_static_ws(const sk_problem *problem, const sk_config *cfg,
                                              sk_stream_t stream) {
  if (!problem) return SK_ERR_INVALID_ARG;
  sk_config c;
  std::memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  if (c.tile_n == 0) c.tile_n = 128;   // the tile that fits all SMs in the fixed array
  sk_plan_info plan;
  sk_status rc = sk_plan_query(problem, 1, &c, 0, &plan);
  if (rc != SK_OK) return rc;
  if (plan.workspace_bytes > kStaticWsBytes) return SK_ERR_WORKSPACE_TOO_SMALL;
  void *ws = nullptr;
  rc = static_ws_address(&ws);
  if (rc != SK_OK) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // The array keeps whatever the previous call left.  The flag region must
  // start at zero (a call that timed out can leave flags raised); the
  // partial slots are always written before being read.  The status word
  // is left alone: a timeout stays recorded until sk_static_ws_status
  // clears it, like the status word of a caller's workspace.
  if (cudaMemsetAsync(static_cast<unsigned char *>(ws) + sk::WS_FLAG_OFFSET, 0, sk::WS_FLAG_BYTES, st) !=
      cudaSuccess)
    return SK_ERR_CUDA;
  return sk_gemm(problem, &c, ws, kStaticWsBytes, stream);
}

extern "C" SK_API sk_status sk_static_ws_status(sk_stream_t stream, int clear, sk_status *device_status) {
  if (!device_status) return SK_ERR_INVALID_ARG;
  void *ws = nullptr;
  sk_status rc = static_ws_address(&ws);
  if (rc != SK_OK) return rc;
  // The status word is the first word of the array (the workspace layout
  // every kernel uses); reading it through sk_get_status keeps one
  // definition of how a status word is read and cleared.
  return sk_get_status(ws, kStaticWsBytes, stream, clear, device_status);
}
