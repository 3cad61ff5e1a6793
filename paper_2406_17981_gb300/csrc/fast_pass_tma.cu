// Strided line passes (forward split, merge) with TMA-staged input tiles.
//
// Same arithmetic as k_pass_reg (fast_pass.cu): a tile is 16 adjacent lines
// (columns) of N points, one line per T = N / R1 threads, first radix stage
// in registers, shared-memory transposes for the later stages.  Here the
// blocks are persistent: each walks the tiles with a grid stride, and its
// input tiles arrive by TMA -- one cp.async.bulk.tensor.2d of a 16 x N box per
// input array, completing on an mbarrier -- into a shared staging area, the
// next tile's copy issued as soon as the current tile has been read into
// registers.  Loads in flight then cost no registers, so the next tile's HBM
// latency hides behind the current tile's transforms.
//
// Views: an array of the pass (x or a tree node) is [outer][N][inner]
// complex64; the tensor map sees it as a 2-D array of 8-byte elements,
// inner columns by outer * N rows.  Tiles never straddle two outer indices
// (inner % 16 == 0), so a tile is the box at (column ii0, row o * N).
//
// Every wait on an mbarrier is bounded; on expiry the block records it in a
// host-mapped error word of the plan (reported by the next pass launch on the
// host), drains its other copies in flight (again bounded) and returns.
#include <cuda.h>

#include <algorithm>
#include <atomic>
#include <cstring>
#include <mutex>

#include "../../include/btmv.h"
#include "fast.cuh"

namespace btmv {

namespace {

constexpr int TPW = 16;                       // lines (columns) per tile
constexpr unsigned kWaitLimit = 1u << 22;     // try_wait rounds before a wait is abandoned

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (TMA) writes to it
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// true once the phase with the given parity has completed; false if the
// wait was abandoned after kWaitLimit rounds or limit_ns nanoseconds
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity, unsigned long long limit_ns) {
  const unsigned a = smem_u32(bar);
  const unsigned long long t0 = global_ns();
  for (unsigned i = 0; i < kWaitLimit; ++i) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    if ((i & 63) == 63 && global_ns() - t0 > limit_ns) return false;
  }
  return false;
}

// 2-D tiled TMA load of the box at (x = column, y = row) into shared memory
__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];"
      ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

template <class P, int MODE, int NSTAGE> struct TmaCfg {
  static constexpr int NIN = MODE == 0 ? 1 : 2;           // input arrays
  static constexpr int NS = NSTAGE;                       // staging buffers
  static constexpr int THREADS = TPW * P::T;
  static constexpr unsigned TILE_BYTES = (unsigned)P::N * TPW * sizeof(float2);
  // mbarriers at the start; the staging tiles from the next 1024-byte
  // boundary of the shared window (the slack covers any base alignment)
  static constexpr size_t HDR = 2048;
  static constexpr size_t smem() { return HDR + (size_t)(NS * NIN + 1) * TILE_BYTES; }
};

template <class P, int MODE, int NSTAGE>
__global__ void __launch_bounds__(TmaCfg<P, MODE, NSTAGE>::THREADS)
    k_pass_tma(const PassArgs a, const __grid_constant__ CUtensorMap tm0, const __grid_constant__ CUtensorMap tm1,
               unsigned ntiles, int* err, unsigned long long limit_ns, unsigned withhold) {
  typedef TmaCfg<P, MODE, NSTAGE> CF;
  constexpr int R1 = P::R1, TT = P::T, N = P::N, NIN = CF::NIN, NS = CF::NS;
  extern __shared__ __align__(1024) unsigned char smem_tma[];
  uint64_t* bar = (uint64_t*)smem_tma;
  const unsigned sbase = smem_u32(smem_tma);
  const unsigned pad = ((sbase + 64u + 1023u) & ~1023u) - sbase;   // >= 64: room for the barriers
  float2* stage = (float2*)(smem_tma + pad);              // [NS][NIN][N][TPW], 1024-byte aligned
  float2* tsm = stage + (size_t)NS * NIN * N * TPW;        // transpose buffer [N][TPW]
  const int col = threadIdx.x % TPW;
  const int t = threadIdx.x / TPW;
  const unsigned inner = (unsigned)a.g.Itot;
  const SmCol<TPW, TT> smc{tsm + col};
  const float2* __restrict__ tw = (const float2*)a.fft.tw;
  const float2* __restrict__ ph = (const float2*)a.fft.ph;

  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) mbar_init(&bar[s], 1);
    fence_mbar_init();
  }
  __syncthreads();
  grid_dep_wait();                                         // the node written by the previous kernel

  // tile it covers lines it * 16 .. it * 16 + 15: outer o, first column ii0
  auto issue = [&](unsigned it, int s) {
    const unsigned gl0 = it * (unsigned)TPW;
    const unsigned o = gl0 / inner;
    const int x = (int)(gl0 - o * inner);
    const int y = (int)(o * (unsigned)N);
    float2* dst = stage + (size_t)s * NIN * N * TPW;
    mbar_expect_tx(&bar[s], CF::TILE_BYTES * NIN + withhold);   // withhold > 0: self test only
    tma_load_2d(dst, &tm0, x, y, &bar[s]);
    if constexpr (NIN == 2) tma_load_2d(dst + N * TPW, &tm1, x, y, &bar[s]);
  };
  if (threadIdx.x == 0)
    for (int s = 0; s < NS; ++s) {
      const unsigned it = blockIdx.x + (unsigned)s * gridDim.x;
      if (it < ntiles) issue(it, s);
    }

  unsigned k = 0;
  for (unsigned it = blockIdx.x; it < ntiles; it += gridDim.x, ++k) {
    const int s = (int)(k % NS);
    const bool got = mbar_wait(&bar[s], (k / NS) & 1u, limit_ns);
    if (__syncthreads_or(!got)) {
      // a copy did not arrive in time: record it, let the other copies in
      // flight land (bounded), and stop
      if (threadIdx.x == 0) {
        atomicExch(err, 1);
        for (unsigned j = 1; j < (unsigned)NS; ++j) {
          const unsigned nx = it + j * gridDim.x;
          if (nx < ntiles) mbar_wait(&bar[(s + j) % NS], ((k + j) / NS) & 1u, limit_ns);
        }
      }
      return;
    }
    const float2* tl = stage + (size_t)s * NIN * N * TPW;
    float2 e[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) e[m] = tl[(t + TT * m) * TPW + col];
    float2 od[MODE == 1 ? R1 : 1];
    if constexpr (MODE == 1) {
#pragma unroll
      for (int m = 0; m < R1; ++m) od[m] = tl[N * TPW + (t + TT * m) * TPW + col];
    }
    __syncthreads();                                       // stage s has been read by every thread
    if (threadIdx.x == 0) {
      const unsigned nx = it + (unsigned)NS * gridDim.x;
      if (nx < ntiles) {
        fence_proxy_async();
        issue(nx, s);
      }
    }
    const unsigned gl0 = it * (unsigned)TPW;
    const unsigned o = gl0 / inner;
    const unsigned ii = gl0 - o * inner + (unsigned)col;
    const long long base = ((long long)o * N + t) * inner + ii;
    const long long step = (long long)TT * inner;
    if constexpr (MODE == 0) {
      if (a.out0) {
        float2 w[R1];
#pragma unroll
        for (int m = 0; m < R1; ++m) w[m] = e[m];
        fft_reg<P, false>(w, t, smc, tw);
        float2* __restrict__ out = (float2*)a.out0;
#pragma unroll
        for (int m = 0; m < R1; ++m) out[base + m * step] = w[m];
      }
      if (a.out1) {
#pragma unroll
        for (int m = 0; m < R1; ++m) e[m] = cmul(e[m], __ldg(&ph[t + TT * m]));
        fft_reg<P, false>(e, t, smc, tw);
        float2* __restrict__ out = (float2*)a.out1;
#pragma unroll
        for (int m = 0; m < R1; ++m) out[base + m * step] = e[m];
      }
    } else {
      fft_reg<P, true>(e, t, smc, tw);
      fft_reg<P, true>(od, t, smc, tw);
#pragma unroll
      for (int m = 0; m < R1; ++m) e[m] = cadd(e[m], cmulc(od[m], __ldg(&ph[t + TT * m])));
      float2* __restrict__ out = (float2*)a.out0;
#pragma unroll
      for (int m = 0; m < R1; ++m) out[base + m * step] = e[m];
    }
  }
}

}  // namespace

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  });
  return fn;
}

// Tensor map of one pass array: inner columns x (outer * N) rows of 8-byte
// elements, box of 16 columns x N rows, no swizzle.
bool encode_array(CUtensorMap* map, const void* base, unsigned inner, unsigned rows, int N) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t gdim[2] = {inner, rows};
  const cuuint64_t gstride[1] = {(cuuint64_t)inner * sizeof(float2)};
  const cuuint32_t box[2] = {(cuuint32_t)TPW, (cuuint32_t)N};
  const cuuint32_t estride[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 2, const_cast<void*>(base), gdim, gstride, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// time limit of a wait for a tile in normal operation (a tile lands in
// microseconds)
constexpr unsigned long long kWaitNs = 2000000000ull;

template <class P, int MODE, int NSTAGE>
cudaError_t pass_tma_p(const PassArgs& a, int* err, cudaStream_t st, unsigned long long limit_ns = kWaitNs,
                       unsigned withhold = 0) {
  typedef TmaCfg<P, MODE, NSTAGE> CF;
  const unsigned inner = (unsigned)a.g.Itot;
  const unsigned rows = (unsigned)(a.g.lines / a.g.Itot) * (unsigned)P::N;
  const unsigned ntiles = (unsigned)(a.g.lines / TPW);
  if (ntiles == 0) return cudaSuccess;
  CUtensorMap m0, m1;
  memset(&m0, 0, sizeof m0);
  if (!encode_array(&m0, a.in0, inner, rows, P::N)) return cudaErrorInvalidValue;
  m1 = m0;
  if (MODE == 1 && !encode_array(&m1, a.in1, inner, rows, P::N)) return cudaErrorInvalidValue;
  const size_t sm = CF::smem();
  cudaError_t e = set_smem_attr<k_pass_tma<P, MODE, NSTAGE>>((int)sm);
  if (e != cudaSuccess) return e;
  // persistent grid: the resident blocks of all SMs
  static std::atomic<int> per_sm{0};
  int bps = per_sm.load(std::memory_order_relaxed);
  if (bps == 0) {
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bps, k_pass_tma<P, MODE, NSTAGE>, CF::THREADS, sm);
    if (e != cudaSuccess) return e;
    if (bps < 1) bps = 1;
    per_sm.store(bps, std::memory_order_relaxed);
  }
  int dev = 0, nsm = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const unsigned grid = std::min<unsigned>(ntiles, (unsigned)(nsm * bps));
#ifndef BTMV_NO_PDL
  return launch_pdl(k_pass_tma<P, MODE, NSTAGE>, dim3(grid), dim3(CF::THREADS), sm, st, a, m0, m1, ntiles, err,
                    limit_ns, withhold);
#else
  k_pass_tma<P, MODE, NSTAGE><<<grid, CF::THREADS, sm, st>>>(a, m0, m1, ntiles, err, limit_ns, withhold);
  return cudaGetLastError();
#endif
}

// One staging buffer: each thread moves its points to registers at once, so
// the next tile's copy (issued right after) already overlaps the current
// tile's transforms, and the smaller footprint keeps more blocks resident
// (two buffers measured slower: 128^3 merge 34.1 against 32.5 us, 256^3
// merge 210.4 against 201.0 us).
template <class P>
cudaError_t pass_tma_n(int mode, const PassArgs& a, int* err, cudaStream_t st) {
  return mode == 0 ? pass_tma_p<P, 0, 1>(a, err, st) : pass_tma_p<P, 1, 1>(a, err, st);
}

}  // namespace

// The TMA pass applies where k_pass_reg does (plain node geometry, register
// plan) and additionally: N <= 256 (one box spans a line), 16 | inner (tiles
// within one outer index), 16-byte aligned arrays, a 32-bit row count, and
// for a merge both inputs present.
bool pass_tma_supported(int mode, const PassArgs& a, size_t esz) {
  if (!pass_reg_supported(a, esz)) return false;
  const int N = a.g.N;
  if (!(N == 32 || N == 64 || N == 128 || N == 256)) return false;
  if (a.g.Itot % TPW != 0) return false;
  if (a.g.lines / a.g.Itot * (long long)N >= (1ll << 31)) return false;
  if (mode == 1 && !a.in1) return false;
  const void* ptrs[4] = {a.in0, a.in1, a.out0, a.out1};
  for (const void* p : ptrs)
    if (((uintptr_t)p) & 15) return false;
  return encode_fn() != nullptr;
}

// Self test of the bounded waits: one forward-split tile of 32-point lines
// (16 lines) whose mbarrier is told to expect 16 bytes more than the copy
// delivers, so that its phase never completes and the wait expires after
// timeout_ms.  The copy itself lands; nothing faults.  Returns 1 if the
// kernel reported the expired wait, 0 if not, -1 on a CUDA error.
static int pass_tma_selftest(int timeout_ms, cudaStream_t st) {
  if (!encode_fn()) return -1;
  const int N = 32, inner = TPW;
  const size_t bytes = (size_t)N * inner * sizeof(float2);
  void *in = nullptr, *out = nullptr, *tabs = nullptr;
  int* err_h = nullptr;
  int* err_d = nullptr;
  int result = -1;
  do {
    if (cudaMalloc(&in, bytes) != cudaSuccess || cudaMalloc(&out, bytes) != cudaSuccess) break;
    if (cudaMalloc(&tabs, 2 * N * sizeof(float2)) != cudaSuccess) break;
    if (cudaMemsetAsync(in, 0, bytes, st) != cudaSuccess) break;
    if (cudaMemsetAsync(tabs, 0, 2 * N * sizeof(float2), st) != cudaSuccess) break;
    if (cudaHostAlloc((void**)&err_h, sizeof(int), cudaHostAllocMapped) != cudaSuccess) break;
    *err_h = 0;
    if (cudaHostGetDevicePointer((void**)&err_d, err_h, 0) != cudaSuccess) break;
    PassArgs a;
    memset(&a, 0, sizeof a);
    a.g.N = N; a.g.ni = 1; a.g.I[0] = inner; a.g.Itot = inner; a.g.lines = inner; a.g.TL = TPW; a.g.halves = 1;
    ArrMap m;
    memset(&m, 0, sizeof m);
    m.os = (long long)N * inner; m.is[0] = 1; m.es = inner; m.len = N;
    m.vI[0] = m.vI[1] = m.vI[2] = 1 << 30;
    a.a_in0 = a.a_in1 = a.a_out0 = a.a_out1 = m;
    a.in0 = in; a.out0 = out;
    a.fft.N = N;
    a.fft.tw = (const unsigned char*)tabs;
    a.fft.ph = (const unsigned char*)tabs + N * sizeof(float2);
    if (pass_tma_p<RP32, 0, 1>(a, err_d, st, (unsigned long long)timeout_ms * 1000000ull, 16) != cudaSuccess) break;
    if (cudaStreamSynchronize(st) != cudaSuccess) break;
    result = *(volatile int*)err_h ? 1 : 0;
  } while (false);
  cudaStreamSynchronize(st);
  if (in) cudaFree(in);
  if (out) cudaFree(out);
  if (tabs) cudaFree(tabs);
  if (err_h) cudaFreeHost(err_h);
  return result;
}

cudaError_t launch_pass_tma(int mode, const PassArgs& a, int* err, cudaStream_t st) {
  if (mode == 1 && !a.in1) return cudaErrorInvalidValue;
  switch (a.g.N) {
    case 32: return pass_tma_n<RP32>(mode, a, err, st);
    case 64: return pass_tma_n<RP64>(mode, a, err, st);
    case 128: return pass_tma_n<RP128>(mode, a, err, st);
    case 256: return pass_tma_n<RP256>(mode, a, err, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace btmv

void btmv_clear_error();
btmv_status btmv_set_error(btmv_status st, const char* msg);

extern "C" BTMV_API btmv_status btmv_selftest_tma_timeout(int timeout_ms, void* stream) {
  btmv_clear_error();
  if (timeout_ms < 1 || timeout_ms > 10000)
    return btmv_set_error(BTMV_E_ARG, "selftest_tma_timeout: timeout_ms outside [1, 10000]");
  const int r = btmv::pass_tma_selftest(timeout_ms, (cudaStream_t)stream);
  if (r < 0) return btmv_set_error(BTMV_E_CUDA, "selftest_tma_timeout: CUDA error or no tensor-map encoder");
  if (r == 0) return btmv_set_error(BTMV_E_STATE, "selftest_tma_timeout: the withheld wait was not reported");
  return btmv_set_error(BTMV_E_TIMEOUT, "selftest_tma_timeout: expired wait reported (expected)");
}
