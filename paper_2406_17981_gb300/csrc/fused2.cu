// Two-level fusion: the last two levels of Algorithm 1 for one node in one
// kernel, with the node's slab held on chip.
//
// A level-(d-2) node v (transformed along the prefix dims 0..d-3, parity
// bits b_0..b_{d-3}) is, in the unfused schedule, split along dim d-2 into
// two children (two more vectors of HBM traffic each way), each child's leaf
// runs along dim d-1, and the children are merged back along dim d-2
// (Sec. II.B, Algorithm 1).  The subtree below v acts on every prefix index
// of v independently, so one block takes the slab of one prefix index (3
// components x N1 x N2 points, N1 along dim d-2 = the columns, N2 along dim
// d-1 = the rows) into shared memory and runs, for both halves b1 of the
// column dim:
//
//   B  column transforms of P1^b1 v (the split, Sec. II.A),
//   C  the leaf on each row: for both halves b2 of the row dim the forward
//      transform of P2^b2 row, the 3 x 3 symbol multiply of class
//      (b_0..b_{d-3}, b1, b2), the inverse transform, merged as
//      y_e + conj(P2) y_o,
//   D  inverse column transforms,
//   E  b1 = 0: the result (the even half of the merge along the column dim)
//      is parked in a scratch vector; b1 = 1: v = parked + conj(P1) result
//      (the merge).
//
// The slab stays on chip between the two levels: at d = 3 an apply moves
// about 16 V (5 V per fused node: the node read twice, the scratch written
// and read, the node written) instead of 26 V.
//
// Thread layout: 256 threads, 32 groups of 8, two blocks per SM (so that
// one block's slab copies overlap the other's transforms); a 64-point line is
// held 8 points per thread (point t + 8 m in thread t of its group) and
// transformed in two radix-8 stages that exchange through shared memory.  A
// column transform exchanges through the column's own storage (its values
// are in registers meanwhile); a row transform through a 64-point buffer of
// its group, because the row's values are needed again for the second half
// b2.  Both exchanges use the rotation rho(8a + b) = 8a + ((a + b) mod 8),
// which puts the stage-1 writes (points t + 8 f) and stage-2 reads (points
// 8 t + r) of the 8 threads in distinct banks.  The slab is stored dense,
// element (i1, i2) at i1 N + (i2 xor 2 (i1 mod 8)): columns and rows are read
// without bank conflicts and 16-byte pairs stay contiguous for the copies.
//
// Layout: c = 3 on the mirror-compressed block-symmetric store (stored
// blocks 00 11 22 01 02 12), complex64, N1 = N2 = 64, d >= 3.
#include <atomic>
#include <cstdint>
#include <cstring>

#include "../../include/btmv.h"
#include "fast.cuh"

namespace btmv {

namespace fz {
constexpr int N = 64;                   // N1 = N2
constexpr int T = 8;                    // threads per line
constexpr int THREADS = 256;
constexpr int GROUPS = THREADS / T;
constexpr int SLAB = 3 * N * N;         // float2
constexpr int CHUNKS = SLAB / 2;        // 16-byte chunks of a slab
constexpr int CPT = CHUNKS / THREADS;   // chunks per thread (CPT / 3 per component)
static_assert(CHUNKS % (3 * THREADS) == 0, "whole chunks per thread and component");
// slab | row exchange buffers | twiddles by thread: 115264 bytes, two blocks per SM
constexpr int TWS = 9;                  // twiddle row stride (distinct banks for t = 0..7)
constexpr size_t SMEM = (size_t)(SLAB + GROUPS * N + T * TWS) * sizeof(float2);

// slab element (i1, i2) of a component
__device__ __forceinline__ int sidx(int i1, int i2) { return i1 * N + (i2 ^ ((i1 & 7) << 1)); }
__device__ __forceinline__ int rho(int p) { return (p & ~7) | ((p + (p >> 3)) & 7); }

// a row exchange buffer: point p at base[rho(p) ^ flip]; flip = 8 swaps rows
// of 8 in pairs so that the two groups of a half-warp use distinct banks
struct RowX {
  float2* base;
  int flip;
  __device__ __forceinline__ float2 ld(int p) const { return base[rho(p) ^ flip]; }
  __device__ __forceinline__ void st(int p, float2 v) const { base[rho(p) ^ flip] = v; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};
// column j of a component's slab as its own exchange buffer: point p in row rho(p)
struct ColX {
  float2* comp;
  int j;
  __device__ __forceinline__ float2* at(int p) const { return comp + sidx(rho(p), j); }
  __device__ __forceinline__ float2 ld(int p) const { return *at(p); }
  __device__ __forceinline__ void st(int p, float2 v) const { *at(p) = v; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

// In: a[m] = v[t + 8 m].  Out: a[m] = DFT(v)[t + 8 m] (unnormalised), two
// radix-8 stages; tw[r] = exp(-2 pi i r t / 64) (this thread's twiddle row).
template <bool INV, class V>
__device__ __forceinline__ void fft64(float2 (&a)[8], int t, const V& v, const float2* tw) {
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

__device__ __forceinline__ void cp16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_wait_all() {
  asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}
// 16-byte chunk k of this thread: component, row, first column of the pair
__device__ __forceinline__ void chunk(int k, int& c, int& i1, int& i2) {
  c = k / (CPT / 3);
  const int r2 = (int)threadIdx.x + THREADS * (k % (CPT / 3));
  i1 = r2 >> 5;
  i2 = (r2 & 31) * 2;
}
}  // namespace fz

struct FuseArgs {
  float2* node;              // the level-(d-2) node, updated in place
  float2* scratch;           // a vector the fused levels no longer need
  int pd;                    // prefix dims 0..d-3 (d - 2 >= 1)
  int ext[MAX_D];            // their extents
  int prefix;                // the node's parity bits (bit m for prefix dim m)
  int nrhs;
  unsigned nslab;            // slabs per right-hand side: prod of the prefix extents
  long long comp_stride;     // nslab * N1 * N2
  const float2* tw;          // exp(-2 pi i k / 64), k < 64
  const float2* ph;          // exp(-i pi k / 64), k < 64 (the split phase)
  SymDev sym;
};

__global__ void __launch_bounds__(fz::THREADS, 2) k_fuse2(const FuseArgs a) {
  using namespace fz;
  extern __shared__ __align__(16) float2 fsm[];
  float2* const slab = fsm;                        // [3][N][N], swizzled rows
  float2* const xb = fsm + SLAB;                   // [GROUPS][N] row exchange buffers
  float2* const twt = xb + GROUPS * N;             // [T][TWS] twiddles by thread
  const int g = threadIdx.x >> 3, t = threadIdx.x & 7;
  // blocks ordered right-hand side fastest: concurrent blocks share symbol rows
  const unsigned sl = blockIdx.x / (unsigned)a.nrhs;   // slab (prefix index)
  const unsigned q = blockIdx.x - sl * (unsigned)a.nrhs;
  const long long cs = a.comp_stride;
  const long long slab_off = (long long)q * 3 * cs + (long long)sl * N * N;
  const SymDev& S = a.sym;
  // the slab's prefix frequencies 2 i_m + b_m (dims 0..pd-1, row-major
  // slab index): their parity class bits, mirror folds and the prefix part
  // of the symbol row index
  int clspp = 0, foldpp = 0;
  unsigned linp = 0;
  {
    int fpre[MAX_D - 2];
    unsigned r = sl;
#pragma unroll
    for (int m = MAX_D - 3; m >= 0; --m)
      if (m < a.pd) {
        const unsigned e = (unsigned)a.ext[m], r2 = r / e;
        fpre[m] = 2 * (int)(r - r2 * e) + ((a.prefix >> m) & 1);
        r = r2;
      }
#pragma unroll
    for (int m = 0; m < MAX_D - 2; ++m)
      if (m < a.pd) {
        clspp = (clspp << 1) | (fpre[m] & 1);
        int fm = fpre[m];
        if (fm > S.n[m]) { fm = 2 * S.n[m] - fm; foldpp |= 1 << m; }
        fpre[m] = fm;
      }
    // strides of the prefix dims depend only on their own parity bits
#pragma unroll
    for (int m = 0; m < MAX_D - 2; ++m)
      if (m < a.pd) linp = linp * (unsigned)S.J[clspp << 2][m] + (unsigned)(fpre[m] >> 1);
  }
  if (threadIdx.x < N) {
    const int tt = threadIdx.x >> 3, r = threadIdx.x & 7;
    twt[tt * TWS + r] = __ldg(a.tw + r * tt);
  }
  const float2* const tw = twt + t * TWS;
  const float2* __restrict__ phs = a.ph;           // split phase (read through L1)
  // leaf rows rbase and rbase + 32: the two groups of a half-warp take rows 4
  // apart, whose swizzles put them in distinct banks
  const int rbase = (g & ~7) | ((g >> 1) & 3) | ((g & 1) << 2);
  const float2* __restrict__ Sd = (const float2*)S.data;
  float2* const node = a.node + slab_off;
  float2* const scr = a.scratch + slab_off;
  const RowX xv{xb + g * N, (g & 1) << 3};
  __syncthreads();
  grid_dep_wait();                                 // the node written by the previous kernel

#pragma unroll 1
  for (int b1 = 0; b1 < 2; ++b1) {
    // A: the slab into shared memory, all copies in flight at once
#pragma unroll
    for (int k = 0; k < CPT; ++k) {
      int c, i1, i2;
      chunk(k, c, i1, i2);
      cp16(slab + c * N * N + sidx(i1, i2), node + c * cs + i1 * N + i2);
    }
    cp_wait_all();
    __syncthreads();
    // B: column transforms along dim 1 (of P1 v for b1 = 1); columns g, g + 32 of each component
#pragma unroll 1
    for (int col = g; col < 3 * N; col += GROUPS) {
      const ColX cx{slab + (col / N) * N * N, col % N};
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float2 x = cx.comp[sidx(t + 8 * m, cx.j)];
        v[m] = b1 ? cmul(x, __ldg(phs + t + 8 * m)) : x;
      }
      fft64<false>(v, t, cx, tw);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) cx.comp[sidx(t + 8 * m, cx.j)] = v[m];
    }
    __syncthreads();
    // C: the leaf on rows f1 (frequency 2 f1 + b1 of dim 1) of the three components
#pragma unroll 1
    for (int kr = 0; kr < 2; ++kr) {
      const int f1 = rbase + (N / 2) * kr;
      // the column dim pd: frequency 2 f1 + b1
      const int pd = a.pd, fp1 = 2 * f1 + b1;
      const int clsp = (clspp << 1) | (fp1 & 1);
      int foldp = foldpp, fm = fp1;
      if (fm > S.n[pd]) { fm = 2 * S.n[pd] - fm; foldp |= 1 << pd; }
      const unsigned lin = linp * (unsigned)S.J[clsp << 1][pd] + (unsigned)(fm >> 1);
      // sign bit k: stored block k read negated (low / folded high frequencies
      // of the row dim pd + 1)
      unsigned sgl = 0, sgh = 0;
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        sgl |= (unsigned)(__popc(S.oddmask[k] & foldp) & 1) << k;
        sgh |= (unsigned)(__popc(S.oddmask[k] & (foldp | (2 << pd))) & 1) << k;
      }
      // point t + 8 m of row f1 sits at (t + 8 m) xor swz = tt + 8 (m xor s3):
      // one base for even m, one for odd m (+ c N N for component c)
      const int swz = (f1 & 7) << 1, tt = (t ^ swz) & 7, s3 = swz >> 3;
      float2* const rev = slab + f1 * N + tt + 8 * s3;
      float2* const rod = slab + f1 * N + tt - 8 * s3;
#define ROWP(c, m) (((m) & 1 ? rod : rev) + (c) * N * N + 8 * (m))
      float2 w[3][8];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 8; ++m) w[c][m] = *ROWP(c, m);
#pragma unroll 1
      for (int b2 = 0; b2 < 2; ++b2) {
        const int cl = (clsp << 1) | b2;
        const float2* __restrict__ rw = Sd + S.cls_off[cl] + (long long)lin * S.J[cl][pd + 1];
        const long long bk = S.blk[cl];
#pragma unroll
        for (int c = 0; c < 3; ++c) fft64<false>(w[c], t, xv, tw);
        // frequencies l = t + 8 m, f = 2 l + b2: stored at l for l < 32, else
        // folded to 64 - l - b2 with the last dim's fold signs; low and folded
        // high frequencies in pairs (their symbol entries share cache lines)
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int m = (i & 1) ? 7 - (i >> 1) : (i >> 1);
          const bool hi = m >= 4;
          const int idx = hi ? (N - b2 - t - 8 * m) : (t + 8 * m);
          const unsigned sg = hi ? sgh : sgl;
          float2 s[6];
#pragma unroll
          for (int k = 0; k < 6; ++k) {
            float2 v = __ldg(rw + (long long)k * bk + idx);
            if ((sg >> k) & 1) { v.x = -v.x; v.y = -v.y; }
            s[k] = v;
          }
          const float2 x0 = w[0][m], x1 = w[1][m], x2 = w[2][m];
          w[0][m] = cadd(cadd(cmul(s[0], x0), cmul(s[3], x1)), cmul(s[4], x2));
          w[1][m] = cadd(cadd(cmul(s[3], x0), cmul(s[1], x1)), cmul(s[5], x2));
          w[2][m] = cadd(cadd(cmul(s[4], x0), cmul(s[5], x1)), cmul(s[2], x2));
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) fft64<true>(w[c], t, xv, tw);
        if (b2 == 0) {
          // park the even half in the row while taking the row for the odd half
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              float2* const p = ROWP(c, m);
              const float2 x = *p;
              *p = w[c][m];
              w[c][m] = cmul(x, __ldg(phs + t + 8 * m));
            }
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int m = 0; m < 8; ++m) {
              float2* const p = ROWP(c, m);
              *p = cadd(*p, cmulc(w[c][m], __ldg(phs + t + 8 * m)));
            }
        }
      }
    }
#undef ROWP
    __syncthreads();
    // D: inverse column transforms along dim 1
#pragma unroll 1
    for (int col = g; col < 3 * N; col += GROUPS) {
      const ColX cx{slab + (col / N) * N * N, col % N};
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = cx.comp[sidx(t + 8 * m, cx.j)];
      fft64<true>(v, t, cx, tw);
      __syncwarp();
#pragma unroll
      for (int m = 0; m < 8; ++m) cx.comp[sidx(t + 8 * m, cx.j)] = v[m];
    }
    __syncthreads();
    // E: park the even half of dim 1 (b1 = 0) or merge into the node (b1 = 1)
    if (b1 == 0) {
#pragma unroll
      for (int k = 0; k < CPT; ++k) {
        int c, i1, i2;
        chunk(k, c, i1, i2);
        *(float4*)(scr + c * cs + i1 * N + i2) = *(const float4*)(slab + c * N * N + sidx(i1, i2));
      }
    } else {
      // scratch loads in batches of EB (all of them at once spill)
      constexpr int EB = CPT / 4;
#pragma unroll 1
      for (int kb = 0; kb < CPT; kb += EB) {
        float4 e[EB];
#pragma unroll
        for (int k = 0; k < EB; ++k) {
          int c, i1, i2;
          chunk(kb + k, c, i1, i2);
          e[k] = __ldcs((const float4*)(scr + c * cs + i1 * N + i2));
        }
#pragma unroll
        for (int k = 0; k < EB; ++k) {
          int c, i1, i2;
          chunk(kb + k, c, i1, i2);
          const float4 o = *(const float4*)(slab + c * N * N + sidx(i1, i2));
          const float2 p = __ldg(phs + i1);
          const float2 lo = cadd(make_float2(e[k].x, e[k].y), cmulc(make_float2(o.x, o.y), p));
          const float2 hi = cadd(make_float2(e[k].z, e[k].w), cmulc(make_float2(o.z, o.w), p));
          *(float4*)(node + c * cs + i1 * N + i2) = make_float4(lo.x, lo.y, hi.x, hi.y);
        }
      }
    }
    __syncthreads();                               // the slab is reloaded by the next half
  }
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

// c = 3 split plan, d >= 3, with n_{d-2} = n_{d-1} = 64, on the compressed
// block-symmetric store, complex64.
bool fuse2_supported(int d, int c, const int* n, size_t esz, const SymDev& S) {
  if (d < 3 || d > MAX_D || c != 3 || esz != sizeof(float2)) return false;
  if (n[d - 2] != fz::N || n[d - 1] != fz::N) return false;
  if (!S.compressed || S.nsym != 6) return false;
  if (S.comp[0][0] != 0 || S.comp[1][1] != 1 || S.comp[2][2] != 2 || S.comp[0][1] != 3 || S.comp[0][2] != 4 ||
      S.comp[1][2] != 5)
    return false;
  return true;
}

// node: a level-(d-2) node with parity bits `prefix` (bit m for dim m),
// scratch: a vector of the same size.  Errors: cudaErrorInvalidValue for a
// shape the kernel does not take, cudaErrorMisalignedAddress unless node and
// scratch are 16-byte aligned.
cudaError_t launch_fuse2(float2* node, float2* scratch, int prefix, int d, const int* n, int nrhs,
                         const FftDev& f1, const FftDev& f2, const SymDev& sym, cudaStream_t st) {
  if (d < 3 || d > MAX_D || f1.N != fz::N || f2.N != fz::N || nrhs < 0) return cudaErrorInvalidValue;
  if (((uintptr_t)node | (uintptr_t)scratch) & 15) return cudaErrorMisalignedAddress;
  FuseArgs a;
  memset(&a, 0, sizeof a);
  long long nslab = 1;
  a.pd = d - 2;
  for (int m = 0; m < a.pd; ++m) {
    if (n[m] < 1) return cudaErrorInvalidValue;
    a.ext[m] = n[m];
    nslab *= n[m];
  }
  const long long blocks = (long long)nrhs * nslab;
  if (blocks == 0) return cudaSuccess;
  if (blocks >= (1ll << 31)) return cudaErrorInvalidValue;
  a.node = node; a.scratch = scratch; a.prefix = prefix; a.nrhs = nrhs; a.nslab = (unsigned)nslab;
  a.comp_stride = nslab * fz::N * fz::N;
  a.tw = (const float2*)f2.tw; a.ph = (const float2*)f2.ph;
  a.sym = sym;
  cudaError_t e = set_smem_attr<k_fuse2>((int)fz::SMEM);
  if (e != cudaSuccess) return e;
  // all of the unified L1 as shared memory: two blocks of 113 KB per SM
  e = func_attr_once<k_fuse2>(cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  return launch_pdl(k_fuse2, dim3((unsigned)blocks), dim3(fz::THREADS), fz::SMEM, st, a);
}

}  // namespace btmv
