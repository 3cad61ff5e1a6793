// Persistent batched kernel: the line passes of many independent problems in
// one launch (see btmv_apply_batched).
#include "generic.cuh"

namespace btmv {

// ------------------------------------------------------------- persistent
// One launch runs the line passes of many independent problems.  Items
// (stage, tile) are handed out in increasing order by one atomic counter;
// an item first waits until the stage it depends on has finished all its
// tiles, so every wait is for items already taken by running blocks and the
// launch cannot deadlock whatever the grid size.  Waits are bounded: past
// the time or iteration limit the block records BTMV_E_TIMEOUT in the
// control word, skips the tile, and later waits give up at once.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <class T>
__global__ void __launch_bounds__(256) k_persistent(const BatchStage* __restrict__ stages, int nstages,
                                                    long long nitems, BatchCtl* ctl, unsigned* done,
                                                    long long timeout_ns) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_item;
  __shared__ int s_stage, s_skip;
  BatchStage* sst = (BatchStage*)smem;
  unsigned char* work = smem + align_up(sizeof(BatchStage), 16);
  for (;;) {
    if (threadIdx.x == 0) {
      const long long it = (long long)atomicAdd(&ctl->next, 1ULL);
      s_item = it;
      s_skip = 0;
      if (it < nitems) {
        int lo = 0, hi = nstages - 1;
        while (lo < hi) {
          const int mid = (lo + hi + 1) >> 1;
          if (stages[mid].item0 <= it) lo = mid; else hi = mid - 1;
        }
        s_stage = lo;
        const int dep = stages[lo].dep;
        if (dep >= 0) {
          const unsigned need = (unsigned)stages[dep].tiles + (unsigned)ctl->withhold;
          const unsigned long long t0 = global_ns();
          long long iter = 0;
          while (*(volatile unsigned*)&done[dep] < need) {
            if (*(volatile int*)&ctl->error) { s_skip = 1; break; }
            if (++iter > 200000000LL || (long long)(global_ns() - t0) > timeout_ns) {
              atomicCAS(&ctl->error, 0, (int)BTMV_E_TIMEOUT);
              ctl->err_stage = lo;
              s_skip = 1;
              break;
            }
            __nanosleep(256);
          }
        }
        __threadfence();
      }
    }
    __syncthreads();
    const long long it = s_item;
    if (it >= nitems) break;
    const int si = s_stage;
    if (!s_skip) {
      const int* src = (const int*)&stages[si];
      int* dst = (int*)sst;
      for (int i = threadIdx.x; i < (int)(sizeof(BatchStage) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      const long long tile = it - sst->item0;
      if (sst->kind == 2) {
        leaf_body<T>(sst->la, work, tile % sst->la.tiles_per_node, (int)(tile / sst->la.tiles_per_node));
      } else if (sst->kind == 0) {
        if (sst->pa.g.contig) pass_body<T, 0, false>(sst->pa, work, tile);
        else                  pass_body<T, 0, true>(sst->pa, work, tile);
      } else if (sst->kind == 1) {
        if (sst->pa.g.contig) pass_body<T, 1, false>(sst->pa, work, tile);
        else                  pass_body<T, 1, true>(sst->pa, work, tile);
      }                        // kind 3: no work (self test)
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[si], 1u);
    }
  }
}

template <class T>
cudaError_t launch_persistent(const BatchStage* stages, int nstages, long long nitems, BatchCtl* ctl,
                              unsigned* done, long long timeout_ns, int grid, size_t smem, cudaStream_t st) {
  // the kernel also holds a few bytes of static shared memory
  const size_t dyn_max = kMaxSmem - 1024;
  const cudaError_t e = set_smem_attr<k_persistent<T>>((int)dyn_max);
  if (e != cudaSuccess) return e;
  if (smem + align_up(sizeof(BatchStage), 16) > dyn_max) return cudaErrorInvalidValue;
  k_persistent<T><<<grid, 256, smem + align_up(sizeof(BatchStage), 16), st>>>(stages, nstages, nitems, ctl, done,
                                                                            timeout_ns);
  return cudaGetLastError();
}

template <class T>
int persistent_blocks_per_sm(size_t smem) {
  int nb = 0;
  set_smem_attr<k_persistent<T>>((int)(kMaxSmem - 1024));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_persistent<T>, 256, smem + align_up(sizeof(BatchStage), 16));
  return nb;
}

template cudaError_t launch_persistent<float2>(const BatchStage*, int, long long, BatchCtl*, unsigned*, long long, int,
                                               size_t, cudaStream_t);
template cudaError_t launch_persistent<double2>(const BatchStage*, int, long long, BatchCtl*, unsigned*, long long,
                                                int, size_t, cudaStream_t);
template int persistent_blocks_per_sm<float2>(size_t);
template int persistent_blocks_per_sm<double2>(size_t);

}  // namespace btmv
