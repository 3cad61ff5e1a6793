// btmv_apply_host_async / btmv_host_wait: applies on pinned host buffers,
// pipelined across calls.  Each call copies x into one of two plan-owned
// staging slots on a copy-in stream, applies on the caller's stream and
// copies y back on a copy-out stream; the slots are used in turn, so the
// copies of one call overlap the apply of the next (the host link carries
// one direction per engine; a GB300's C2C link moves about 180 GB/s each
// way from pinned memory, a 128^3 c = 3 complex64 vector in 0.28 ms).
#include <cuda_runtime.h>

#include "../../include/btmv.h"
#include "plan.h"

btmv_status btmv_check_apply_args(btmv_plan p, const void* x, void* y, int nrhs);
size_t btmv_apply_vector_bytes(btmv_plan p, int nrhs);
btmv_status btmv_apply_on_device(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st);
btmv_status btmv_set_error(btmv_status st, const char* msg);

namespace {

// Staging slots, copy streams and events, made on the first call.
btmv_status ensure_pipe(btmv_plan p) {
  if (p->cp_out) return BTMV_OK;
  const size_t Vmax = btmv_apply_vector_bytes(p, p->max_rhs);
  for (int s = 0; s < 2; ++s) {
    if (cudaMalloc(&p->ring_x[s], Vmax) != cudaSuccess || cudaMalloc(&p->ring_y[s], Vmax) != cudaSuccess)
      return btmv_set_error(BTMV_E_NOMEM, "apply_host_async: staging slots");
    if (cudaEventCreateWithFlags(&p->ev_in[s], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_comp[s], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&p->ev_out[s], cudaEventDisableTiming) != cudaSuccess)
      return btmv_set_error(BTMV_E_CUDA, "apply_host_async: events");
  }
  if (cudaStreamCreateWithFlags(&p->cp_in, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&p->cp_out, cudaStreamNonBlocking) != cudaSuccess)
    return btmv_set_error(BTMV_E_CUDA, "apply_host_async: copy streams");
  return BTMV_OK;
}

}  // namespace

extern "C" BTMV_API btmv_status btmv_apply_host_async(btmv_plan p, const void* x, void* y, int nrhs,
                                                      void* stream) {
  btmv_status st = btmv_check_apply_args(p, x, y, nrhs);
  if (st != BTMV_OK) return st;
  if (nrhs == 0) return BTMV_OK;
  st = ensure_pipe(p);
  if (st != BTMV_OK) return st;
  const int s = (int)(p->pipe_k & 1);
  const bool reuse = p->pipe_k >= 2;       // the slot served call k-2
  const size_t V = btmv_apply_vector_bytes(p, nrhs);
  cudaStream_t cs = (cudaStream_t)stream;
  bool ok = true;
  // copy in, once the apply of call k-2 has read this slot's x
  if (reuse) ok = ok && cudaStreamWaitEvent(p->cp_in, p->ev_comp[s], 0) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(p->ring_x[s], x, V, cudaMemcpyHostToDevice, p->cp_in) == cudaSuccess;
  ok = ok && cudaEventRecord(p->ev_in[s], p->cp_in) == cudaSuccess;
  // apply, once x is in and the copy out of call k-2 has read this slot's y
  ok = ok && cudaStreamWaitEvent(cs, p->ev_in[s], 0) == cudaSuccess;
  if (reuse) ok = ok && cudaStreamWaitEvent(cs, p->ev_out[s], 0) == cudaSuccess;
  if (!ok) return btmv_set_error(BTMV_E_CUDA, "apply_host_async: copy in");
  st = btmv_apply_on_device(p, p->ring_x[s], p->ring_y[s], nrhs, cs);
  if (st != BTMV_OK) return st;
  ok = cudaEventRecord(p->ev_comp[s], cs) == cudaSuccess;
  // copy out
  ok = ok && cudaStreamWaitEvent(p->cp_out, p->ev_comp[s], 0) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(y, p->ring_y[s], V, cudaMemcpyDeviceToHost, p->cp_out) == cudaSuccess;
  ok = ok && cudaEventRecord(p->ev_out[s], p->cp_out) == cudaSuccess;
  if (!ok) return btmv_set_error(BTMV_E_CUDA, "apply_host_async: copy out");
  ++p->pipe_k;
  return BTMV_OK;
}

extern "C" BTMV_API btmv_status btmv_host_wait(btmv_plan p) {
  if (!p) return btmv_set_error(BTMV_E_ARG, "host_wait: plan is NULL");
  if (!p->cp_out) return BTMV_OK;
  // every copy out follows its apply, which follows its copy in
  if (cudaStreamSynchronize(p->cp_out) != cudaSuccess || cudaStreamSynchronize(p->cp_in) != cudaSuccess)
    return btmv_set_error(BTMV_E_CUDA, "host_wait: stream synchronisation failed");
  return BTMV_OK;
}
