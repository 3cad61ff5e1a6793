// The whole split apply of a small two-level problem in one launch: d = 2,
// c = 1, n = 64 x 64 (either precision), one thread-block cluster per
// right-hand side.
//
// For d = 2 the last two levels of Algorithm 1 are the whole tree: the
// dim-0 split of x into its even and odd children (Sec. II.A), the leaf
// along dim 1 on every row of both children (both halves, the symbol
// multiply, the merge; Sec. II.B), and the dim-0 merge into y.  Run as three
// kernels, each is a few microseconds of work behind a launch and a round
// trip through global memory; here the K CTAs of one cluster share the grid
// through distributed shared memory:
//
//   1  CTA k takes columns [R k, R k + R) of x (R = 64 / K), transforms each
//      along dim 0 for both children (P0^b0 x), and stores every spectrum
//      value straight into the shared memory of the CTA that owns its row;
//   2  CTA k runs the leaf on rows [R k, R k + R) of both children and stores
//      each result value into the CTA that owns its column;
//   3  CTA k inverse-transforms its columns of both children along dim 0 and
//      writes y = IDFT(z_0) + conj(P0) IDFT(z_1).
//
// Cluster barriers separate the phases (the first one also guarantees that
// every CTA of the cluster runs before any remote store); no CTA touches
// another's shared memory after the last one.  A line of 64 points is held
// by 8 threads, 8 points each, and transformed in two radix-8 stages that
// exchange through a per-group buffer, as in the fused d = 3 kernel; the
// leaf runs the two halves b1 of a row in two groups (twice the threads of
// the column phases, where half of the warps idle).
#include <cooperative_groups.h>

#include <atomic>
#include <cstdint>
#include <cstdlib>
#include <cstring>

#include "../../include/btmv.h"
#include "fast.cuh"

namespace cgx = cooperative_groups;

namespace btmv {

namespace s2 {
constexpr int N = 64;
__device__ __forceinline__ int rho(int p) { return (p & ~7) | ((p + (p >> 3)) & 7); }

// a group's exchange buffer: point p at base[rho(p) ^ flip]
template <class T>
struct Xb {
  T* base;
  int flip;
  __device__ __forceinline__ T ld(int p) const { return base[rho(p) ^ flip]; }
  __device__ __forceinline__ void st(int p, T v) const { base[rho(p) ^ flip] = v; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// In: a[m] = v[t + 8 m].  Out: a[m] = DFT(v)[t + 8 m] (unnormalised);
// tw = this thread's twiddle row, tw[r] = exp(-2 pi i r t / 64).
template <bool INV, class T, class V>
__device__ __forceinline__ void fft64(T (&a)[8], int t, const V& v, const T* tw) {
  dft<8, INV>(a);
  v.sync();
#pragma unroll
  for (int f = 0; f < 8; ++f) v.st(t + 8 * f, a[f]);
  v.sync();
#pragma unroll
  for (int r = 0; r < 8; ++r) a[r] = v.ld(8 * t + r);
#pragma unroll
  for (int r = 1; r < 8; ++r) a[r] = twm<INV>(a[r], tw[r]);
  dft<8, INV>(a);
}
}  // namespace s2

struct Small2dArgs {
  const void* x;
  void* y;
  const void* tw;            // exp(-2 pi i k / 64), k < 64 (plan precision)
  const void* ph;            // exp(-i pi k / 64)
  SymDev sym;
};

template <class T, int K>
struct Small2dCfg {
  static constexpr int R = s2::N / K;          // columns (rows) per CTA
  static constexpr int L = 2 * R;              // lines per phase: R columns (rows) x 2 children
  static constexpr int G = 2 * L;              // 8-thread groups: the leaf runs its two halves b1 apart
  static constexpr int THREADS = 8 * G;
  // rows[L][N] | cols[L][N] | odd[L][N] | exchange[G][N] | twiddles[8][9] | phase[N]
  static constexpr size_t SMEM = (size_t)(3 * L * s2::N + G * s2::N + 72 + s2::N) * sizeof(T);
};

template <class T, int K>
__global__ void __launch_bounds__(Small2dCfg<T, K>::THREADS) k_small2d(const Small2dArgs a) {
  using namespace s2;
  typedef Small2dCfg<T, K> CF;
  constexpr int R = CF::R;
  extern __shared__ __align__(16) unsigned char s2mem[];
  constexpr int L = CF::L;
  T* const rows = (T*)s2mem;                       // [2][R][N]: rows of both children owned here
  T* const cols = rows + L * N;                    // [2][R][N]: columns of both children owned here
  T* const odd = cols + L * N;                     // [2][R][N]: the leaf's odd halves
  T* const xbuf = odd + L * N;                     // [G][N]
  T* const twt = xbuf + CF::G * N;                 // [8][9]
  T* const phs = twt + 72;                         // [N]
  cgx::cluster_group cluster = cgx::this_cluster();
  const int k = (int)cluster.block_rank();
  const int g = threadIdx.x >> 3, t = threadIdx.x & 7;
  const long long q = blockIdx.y;                  // right-hand side
  const T* __restrict__ x = (const T*)a.x + q * N * N;
  T* __restrict__ y = (T*)a.y + q * N * N;
  for (int e = threadIdx.x; e < N; e += CF::THREADS) {
    twt[(e >> 3) * 9 + (e & 7)] = ((const T*)a.tw)[(e & 7) * (e >> 3)];
    phs[e] = ((const T*)a.ph)[e];
  }
  const T* const tw = twt + t * 9;
  const Xb<T> xv{xbuf + g * N, (g & 1) << 3};
  __syncthreads();
  cluster.sync();                                  // every CTA of the cluster is running
  grid_dep_wait();                                 // x and y of the previous kernel on the stream

  // 1: column i1 of child b0, forward along dim 0, each value sent to the owner
  // of its row (groups g < L; the others idle as whole warps)
  if (g < L) {
    const int j = g % R, b0 = g / R, i1 = R * k + j;
    T v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const T e = x[(long long)(t + 8 * m) * N + i1];
      v[m] = b0 ? cmul(e, phs[t + 8 * m]) : e;
    }
    fft64<false>(v, t, xv, tw);
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int f0 = t + 8 * m;
      *cluster.map_shared_rank(rows + (b0 * R + f0 % R) * N + i1, f0 / R) = v[m];
    }
  }
  cluster.sync();

  // 2: the leaf on row f0 of child b0 (dim-0 frequency 2 f0 + b0), half b1
  // in group b1 L + line; the even half adds the odd half's conj(P1) term and
  // sends each result value to the owner of its column
  {
    const int b1 = g / L, line = g % L, r = line % R, b0 = line / R, f0 = R * k + r;
    const T* const row = rows + line * N;
    const SymDev& S = a.sym;
    int fp0 = 2 * f0 + b0, foldp = 0;
    if (S.compressed && fp0 > S.n[0]) { fp0 = 2 * S.n[0] - fp0; foldp = 1; }
    const int c = (b0 << 1) | b1;
    const T* __restrict__ rw = (const T*)S.data + S.cls_off[c] + (long long)(fp0 >> 1) * S.J[c][1];
    T v[8];
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const T e = row[t + 8 * m];
      v[m] = b1 ? cmul(e, phs[t + 8 * m]) : e;
    }
    fft64<false>(v, t, xv, tw);
    // frequency f = 2 l + b1, l = t + 8 m: full store at l; compressed
    // store at l for l < N/2, else at N - b1 - l with the fold's sign
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int l = t + 8 * m;
      const bool hi = S.compressed && l >= N / 2;
      T s = __ldg(rw + (hi ? N - b1 - l : l));
      if (__popc(S.oddmask[0] & (hi ? (foldp | 2) : foldp)) & 1) { s.x = -s.x; s.y = -s.y; }
      v[m] = cmul(s, v[m]);
    }
    fft64<true>(v, t, xv, tw);
    if (b1 == 1) {
#pragma unroll
      for (int m = 0; m < 8; ++m) odd[line * N + t + 8 * m] = cmulc(v[m], phs[t + 8 * m]);
    }
    __syncthreads();
    if (b1 == 0) {
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int i1 = t + 8 * m;
        *cluster.map_shared_rank(cols + (b0 * R + i1 % R) * N + f0, i1 / R) = cadd(v[m], odd[line * N + i1]);
      }
    }
  }
  cluster.sync();                                  // no remote access after this

  // 3: column i1 of both children inverse along dim 0, y = z_0 + conj(P0) z_1
  // (groups g < L)
  {
    const int j = g % R, b0 = g / R, i1 = R * k + j;
    T* const col = cols + (b0 * R + j) * N;
    T v[8];
    if (g < L) {
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = col[t + 8 * m];
      fft64<true>(v, t, xv, tw);
      if (b0 == 1) {
#pragma unroll
        for (int m = 0; m < 8; ++m) col[t + 8 * m] = cmulc(v[m], phs[t + 8 * m]);
      }
    }
    __syncthreads();
    if (g < L && b0 == 0) {
      const T* const z1 = cols + (R + j) * N;
#pragma unroll
      for (int m = 0; m < 8; ++m) y[(long long)(t + 8 * m) * N + i1] = cadd(v[m], z1[t + 8 * m]);
    }
  }
}

// d = 2, c = 1, n = 64 x 64 split plans (full or compressed store).
bool small2d_supported(int d, int c, const int* n, const SymDev& S) {
  return d == 2 && c == 1 && n[0] == s2::N && n[1] == s2::N && S.nsym == 1 && S.comp[0][0] == 0;
}

// Set a function attribute once per device (devices 0..63), as
// set_smem_attr does for the shared-memory size.
template <auto K>
static cudaError_t func_attr_once(cudaFuncAttribute attr, int value) {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(K, attr, value);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

template <class T, int K>
static cudaError_t small2d_k(const Small2dArgs& a, int nrhs, cudaStream_t st) {
  typedef Small2dCfg<T, K> CF;
  cudaError_t e = cudaSuccess;
  if (K > 8) e = func_attr_once<k_small2d<T, K>>(cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  if (CF::SMEM > 48 * 1024) e = set_smem_attr<k_small2d<T, K>>((int)CF::SMEM);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(K, (unsigned)nrhs);
  cfg.blockDim = dim3(CF::THREADS);
  cfg.dynamicSmemBytes = CF::SMEM;
  cfg.stream = st;
  // programmatic dependent launch: the prologue (tables, the first cluster
  // barrier) runs while the previous kernel of the stream retires
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = K;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_small2d<T, K>, a);
}

// Clusters of 16 CTAs where the device schedules them (a non-portable
// size), else of 8 (BTMV_SMALL2D_CLUSTER=8 in the environment forces 8, to
// exercise that form); right-hand sides on the grid's y dimension, at most
// 65535 per launch (more are launched in chunks).
template <class T>
static cudaError_t small2d_t(const Small2dArgs& a, int nrhs, cudaStream_t st) {
  if (nrhs < 1) return cudaErrorInvalidValue;
  static std::atomic<int> k16[64];                 // per device: 0 unknown, 1 yes, 2 no
  int dev = 0;
  cudaGetDevice(&dev);
  const char* force = getenv("BTMV_SMALL2D_CLUSTER");
  int ok = (force && force[0] == '8') ? 2 : k16[dev & 63].load(std::memory_order_relaxed);
  if (ok == 0) {
    typedef Small2dCfg<T, 16> CF;
    int maxc = 0;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(16, 1);
    cfg.blockDim = dim3(CF::THREADS);
    cfg.dynamicSmemBytes = CF::SMEM;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = 16;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    const bool attr = cudaFuncSetAttribute(k_small2d<T, 16>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) ==
                      cudaSuccess;
    ok = (attr && cudaOccupancyMaxActiveClusters(&maxc, k_small2d<T, 16>, &cfg) == cudaSuccess && maxc > 0) ? 1 : 2;
    cudaGetLastError();
    k16[dev & 63].store(ok, std::memory_order_relaxed);
  }
  constexpr int YMAX = 65535;
  for (int q0 = 0; q0 < nrhs; q0 += YMAX) {
    Small2dArgs c = a;
    c.x = (const T*)a.x + (size_t)q0 * s2::N * s2::N;
    c.y = (T*)a.y + (size_t)q0 * s2::N * s2::N;
    const int nq = nrhs - q0 < YMAX ? nrhs - q0 : YMAX;
    const cudaError_t e = ok == 1 ? small2d_k<T, 16>(c, nq, st) : small2d_k<T, 8>(c, nq, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_small2d(const void* x, void* y, int nrhs, bool dbl, const FftDev& f, const SymDev& sym,
                           cudaStream_t st) {
  if (f.N != s2::N) return cudaErrorInvalidValue;
  Small2dArgs a;
  memset(&a, 0, sizeof a);
  a.x = x; a.y = y; a.tw = f.tw; a.ph = f.ph; a.sym = sym;
  return dbl ? small2d_t<double2>(a, nrhs, st) : small2d_t<float2>(a, nrhs, st);
}

}  // namespace btmv
