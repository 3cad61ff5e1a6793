// btmv_apply_host_noalloc: y = T x for host-resident x and y, staged through a
// fixed, file-scope device array instead of device memory allocated on demand.
//
// btmv_apply with host pointers allocates its two staging buffers with
// cudaMalloc the first time it sees host pointers.  Some callers cannot allow
// an allocation at that moment: a process whose device memory is fully
// reserved by another allocator (a framework's caching pool, a serving
// budget), or code that must not take the driver's allocation path in the
// middle of a latency-critical solver loop.  This entry point calls no
// cudaMalloc, cudaFree or allocating library routine: the staging space is
// the static array below, which every GPU that loads the library holds for
// the life of the process.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/btmv.h"

btmv_status btmv_check_apply_args(btmv_plan p, const void* x, void* y, int nrhs);
size_t btmv_apply_vector_bytes(btmv_plan p, int nrhs);
btmv_status btmv_apply_on_device(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st);
btmv_status btmv_set_error(btmv_status st, const char* msg);
void btmv_clear_error();
int btmv_plan_device(btmv_plan p);

namespace {

// Two halves: staged x, then staged y (BTMV_NOALLOC_MAX_BYTES each).
static __device__ __align__(256) unsigned char g_stage[2 * BTMV_NOALLOC_MAX_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_stage_ptr[kMaxDevices] = {nullptr};

// Device address of g_stage on the plan's device, which must be the current
// one (looked up once per device, with that device current).  In host code
// the name g_stage is only a host stand-in, so the address must come from
// cudaGetSymbolAddress.
btmv_status stage_address(int plan_dev, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return btmv_set_error(BTMV_E_CUDA, "apply_host_noalloc: cudaGetDevice failed");
  // the staging array of another device would be read by kernels that run on
  // the plan's device, next to the plan's symbol, tables and workspace
  if (dev != plan_dev)
    return btmv_set_error(BTMV_E_ARG, "apply_host_noalloc: the current device is not the plan's device");
  if (dev < 0 || dev >= kMaxDevices) return btmv_set_error(BTMV_E_UNSUPPORTED, "apply_host_noalloc: device index too large");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_stage_ptr[dev]) {
    void* ptr = nullptr;
    e = cudaGetSymbolAddress(&ptr, g_stage);
    if (e != cudaSuccess || !ptr)
      return btmv_set_error(BTMV_E_CUDA, "apply_host_noalloc: cudaGetSymbolAddress of the staging array failed");
    g_stage_ptr[dev] = ptr;
  }
  *out = g_stage_ptr[dev];
  return BTMV_OK;
}

}  // namespace

extern "C" BTMV_API btmv_status btmv_apply_host_noalloc(btmv_plan p, const void* x, void* y, int nrhs,
                                                        void* stream) {
  btmv_clear_error();
  btmv_status st = btmv_check_apply_args(p, x, y, nrhs);
  if (st != BTMV_OK) return st;
  if (nrhs == 0) return BTMV_OK;
  const size_t V = btmv_apply_vector_bytes(p, nrhs);
  if (V > (size_t)BTMV_NOALLOC_MAX_BYTES)
    return btmv_set_error(BTMV_E_UNSUPPORTED,
                          "apply_host_noalloc: nrhs * c * prod(n) * element size exceeds "
                          "BTMV_NOALLOC_MAX_BYTES (16 MiB); use btmv_apply");
  void* base = nullptr;
  st = stage_address(btmv_plan_device(p), &base);
  if (st != BTMV_OK) return st;
  unsigned char* xs = (unsigned char*)base;
  unsigned char* ys = xs + BTMV_NOALLOC_MAX_BYTES;
  cudaStream_t s = (cudaStream_t)stream;
  // x is copied in whole and y is written in whole by the apply, so nothing
  // left in the array by an earlier call is read.
  cudaError_t e = cudaMemcpyAsync(xs, x, V, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return btmv_set_error(BTMV_E_CUDA, "apply_host_noalloc: copy of x to the device failed");
  st = btmv_apply_on_device(p, xs, ys, nrhs, s);
  if (st != BTMV_OK) return st;
  e = cudaMemcpyAsync(y, ys, V, cudaMemcpyDefault, s);
  if (e != cudaSuccess) return btmv_set_error(BTMV_E_CUDA, "apply_host_noalloc: copy of y to the host failed");
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return btmv_set_error(BTMV_E_CUDA, "apply_host_noalloc: stream synchronisation failed");
  return BTMV_OK;
}
