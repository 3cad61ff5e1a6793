// Two-level fusion for 128 x 128 slabs: the last two levels of Algorithm 1
// for one level-(d-2) node, with the node's slab spread over the shared
// memory of a 16-CTA thread-block cluster.
//
// The work per slab is that of the single-CTA fused kernel (fused2.cu): for
// both halves b1 of the column dim d-2, the column transforms of P1^b1 v (the
// split, Sec. II.A), the leaf on each row of the row dim d-1 (both halves b2,
// the 3 x 3 symbol multiply, the merge; Sec. II.B), the inverse column
// transforms, and the merge along the column dim through a parked even half.
// A 128 x 128 x 3 slab (393 KB) does not fit one CTA, so CTA k of the cluster
// owns columns [8k, 8k + 8) for the column phases and rows [8k, 8k + 8) for
// the leaf, and every transformed value goes straight into the shared memory
// of the CTA that needs it next (column -> row owner after the forward
// column transforms, row -> column owner after the leaf):
//
//   B  columns of the node (from global memory), forward along dim d-2,
//      values to the row owners;
//   C  the leaf on the CTA's rows, values to the column owners;
//   D  inverse column transforms;
//   E  b1 = 0: park the result in the scratch vector; b1 = 1: node = parked +
//      conj(P1) result.
//
// Cluster barriers order the phases (the first one also makes sure that
// every CTA of the cluster runs before any remote store); no CTA touches
// another's shared memory after the last one.  A 128-point line is held by
// 16 threads, 8 points each, and transformed in three stages (8 x 4 x 4).
//
// Layout: c = 3 on the mirror-compressed block-symmetric store (stored
// blocks 00 11 22 01 02 12), complex64, n_{d-2} = n_{d-1} = 128, d >= 3.
#include <cooperative_groups.h>

#include <atomic>
#include <cstdint>
#include <cstring>

#include "../../include/btmv.h"
#include "fast.cuh"

namespace cgf = cooperative_groups;

namespace btmv {

namespace fc {
constexpr int N = 128;                     // N1 = N2
constexpr int K = 16;                      // CTAs per cluster
constexpr int R = N / K;                   // columns (rows) per CTA
typedef RP<128, 8, 4, 4> P;                // 16 threads x 8 points per line
constexpr int T = P::T;
constexpr int LINES = 3 * R;               // column lines per CTA (3 components)
constexpr int THREADS = LINES * T;         // 384
constexpr int LEAF_GROUPS = 2 * R;         // leaf: a row's two halves b2 in two groups
constexpr int PD = pad_div<P>();
constexpr int GS = padded_len<P>() + ((0 - padded_len<P>() % 16) + 16) % 16;   // group stride, = 0 (mod 16)
// rows[3][R][N] | cols[3][R][N] | odd[3][R][N] | exchange[LINES][GS] | twiddles[N] | phase[N]
constexpr size_t SMEM = (size_t)(9 * R * N + LINES * GS + 2 * N) * sizeof(float2);
}  // namespace fc

struct FuseCArgs {
  float2* node;              // the level-(d-2) node, updated in place
  float2* scratch;           // a vector the fused levels no longer need
  int pd;                    // prefix dims 0..d-3
  int ext[MAX_D];            // their extents
  int prefix;                // the node's parity bits (bit m for prefix dim m)
  int nrhs;
  long long comp_stride;     // nslab * N * N
  const float2* tw;          // exp(-2 pi i k / 128), k < 128
  const float2* ph;          // exp(-i pi k / 128), k < 128
  SymDev sym;
};

__global__ void __launch_bounds__(fc::THREADS, 1) k_fuse2c(const FuseCArgs a) {
  using namespace fc;
  extern __shared__ __align__(16) float2 fcm[];
  float2* const rows = fcm;                        // [3][R][N]: rows owned here (column spectra)
  float2* const cols = rows + 3 * R * N;           // [3][R][N]: columns owned here (leaf results)
  float2* const odd = cols + 3 * R * N;            // [3][R][N]: the leaf's odd halves
  float2* const xb = odd + 3 * R * N;              // [LINES][GS]: transpose buffers
  float2* const tws = xb + LINES * GS;             // [N]
  float2* const phs = tws + N;                     // [N]
  cgf::cluster_group cluster = cgf::this_cluster();
  const int k = (int)cluster.block_rank();
  const int g = threadIdx.x / T, t = threadIdx.x % T;
  const SmLine<PD, T> sm{xb + g * GS};
  // blocks ordered right-hand side fastest: concurrent clusters share symbol rows
  const unsigned sl = blockIdx.y / (unsigned)a.nrhs;   // slab (prefix index)
  const unsigned q = blockIdx.y - sl * (unsigned)a.nrhs;
  const long long cs = a.comp_stride;
  const long long slab_off = (long long)q * 3 * cs + (long long)sl * N * N;
  const SymDev& S = a.sym;
  // prefix frequencies 2 i_m + b_m of the slab: class bits, folds, the
  // prefix part of the symbol row index
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
#pragma unroll
    for (int m = 0; m < MAX_D - 2; ++m)
      if (m < a.pd) linp = linp * (unsigned)S.J[clspp << 2][m] + (unsigned)(fpre[m] >> 1);
  }
  for (int e = threadIdx.x; e < N; e += THREADS) {
    tws[e] = __ldg(a.tw + e);
    phs[e] = __ldg(a.ph + e);
  }
  const float2* __restrict__ Sd = (const float2*)S.data;
  float2* const node = a.node + slab_off;
  float2* const scr = a.scratch + slab_off;
  // column phases: group g takes component c of column j
  const int cc = g / R, jj = g % R, j = R * k + jj;
  __syncthreads();
  cluster.sync();                                  // every CTA of the cluster is running
  grid_dep_wait();                                 // the node written by the previous kernel

#pragma unroll 1
  for (int b1 = 0; b1 < 2; ++b1) {
    // B: column j of component cc of P1^b1 v, forward along the column dim;
    // each spectrum value to the owner of its row
    {
      const float2* const col = node + cc * cs + j;
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const float2 x = col[(long long)(t + T * m) * N];
        v[m] = b1 ? cmul(x, phs[t + T * m]) : x;
      }
      fft_reg<P, false, SmLine<PD, T>, true>(v, t, sm, tws);
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const int f1 = t + T * m;
        *cluster.map_shared_rank(rows + (cc * R + f1 % R) * N + j, f1 / R) = v[m];
      }
    }
    cluster.sync();

    // C: the leaf on row f1 = R k + r (frequency 2 f1 + b1 of the column
    // dim), half b2 in group b2 R + r; the even half adds the odd half's
    // conj(P2) term and sends each value to the owner of its column
    float2 w[3][8];
    const int b2 = g / R, r = g % R, f1 = R * k + r;
    if (g < LEAF_GROUPS) {
      const int pd = a.pd, fp1 = 2 * f1 + b1;
      const int clsp = (clspp << 1) | (fp1 & 1);
      int foldp = foldpp, fm = fp1;
      if (fm > S.n[pd]) { fm = 2 * S.n[pd] - fm; foldp |= 1 << pd; }
      const unsigned lin = linp * (unsigned)S.J[clsp << 1][pd] + (unsigned)(fm >> 1);
      // sign bit kk: stored block kk read negated (low / folded high frequencies
      // of the row dim pd + 1)
      unsigned sgl = 0, sgh = 0;
#pragma unroll
      for (int kk = 0; kk < 6; ++kk) {
        sgl |= (unsigned)(__popc(S.oddmask[kk] & foldp) & 1) << kk;
        sgh |= (unsigned)(__popc(S.oddmask[kk] & (foldp | (2 << pd))) & 1) << kk;
      }
      const int cl = (clsp << 1) | b2;
      const float2* __restrict__ rw = Sd + S.cls_off[cl] + (long long)lin * S.J[cl][pd + 1];
      const long long bk = S.blk[cl];
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const float2 x = rows[(c * R + r) * N + t + T * m];
          w[c][m] = b2 ? cmul(x, phs[t + T * m]) : x;
        }
#pragma unroll
      for (int c = 0; c < 3; ++c) fft_reg<P, false, SmLine<PD, T>, true>(w[c], t, sm, tws);
      // frequencies l = t + 16 m, f = 2 l + b2: stored at l for l < 64, else
      // folded to 128 - l - b2 with the row dim's fold signs; low and folded
      // high frequencies in pairs
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int m = (i & 1) ? 7 - (i >> 1) : (i >> 1);
        const bool hi = m >= 4;
        const int idx = hi ? (N - b2 - t - T * m) : (t + T * m);
        const unsigned sg = hi ? sgh : sgl;
        float2 s[6];
#pragma unroll
        for (int kk = 0; kk < 6; ++kk) {
          float2 v = __ldg(rw + (long long)kk * bk + idx);
          if ((sg >> kk) & 1) { v.x = -v.x; v.y = -v.y; }
          s[kk] = v;
        }
        const float2 x0 = w[0][m], x1 = w[1][m], x2 = w[2][m];
        w[0][m] = cadd(cadd(cmul(s[0], x0), cmul(s[3], x1)), cmul(s[4], x2));
        w[1][m] = cadd(cadd(cmul(s[3], x0), cmul(s[1], x1)), cmul(s[5], x2));
        w[2][m] = cadd(cadd(cmul(s[4], x0), cmul(s[5], x1)), cmul(s[2], x2));
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) fft_reg<P, true, SmLine<PD, T>, true>(w[c], t, sm, tws);
      if (b2 == 1) {
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
          for (int m = 0; m < 8; ++m) odd[(c * R + r) * N + t + T * m] = cmulc(w[c][m], phs[t + T * m]);
      }
    }
    __syncthreads();
    if (g < R) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < 8; ++m) {
          const int i2 = t + T * m;
          *cluster.map_shared_rank(cols + (c * R + i2 % R) * N + f1, i2 / R) =
              cadd(w[c][m], odd[(c * R + r) * N + i2]);
        }
    }
    cluster.sync();

    // D: column j of component cc inverse along the column dim; E: park it
    // (b1 = 0) or merge it into the node (b1 = 1)
    {
      const float2* const colb = cols + (cc * R + jj) * N;
      float2 v[8];
#pragma unroll
      for (int m = 0; m < 8; ++m) v[m] = colb[t + T * m];
      fft_reg<P, true, SmLine<PD, T>, true>(v, t, sm, tws);
#pragma unroll
      for (int m = 0; m < 8; ++m) {
        const long long o = cc * cs + (long long)(t + T * m) * N + j;
        if (b1 == 0) scr[o] = v[m];
        else node[o] = cadd(scr[o], cmulc(v[m], phs[t + T * m]));
      }
    }
  }
}

// c = 3 split plan, d >= 3, with n_{d-2} = n_{d-1} = 128, on the compressed
// block-symmetric store, complex64.
bool fuse2c_supported(int d, int c, const int* n, size_t esz, const SymDev& S) {
  if (d < 3 || d > MAX_D || c != 3 || esz != sizeof(float2)) return false;
  if (n[d - 2] != fc::N || n[d - 1] != fc::N) return false;
  if (!S.compressed || S.nsym != 6) return false;
  if (S.comp[0][0] != 0 || S.comp[1][1] != 1 || S.comp[2][2] != 2 || S.comp[0][1] != 3 || S.comp[0][2] != 4 ||
      S.comp[1][2] != 5)
    return false;
  return true;
}

// The current device schedules a cluster of 16 CTAs of this kernel (a
// non-portable size); set up once per device (devices 0..63).
bool fuse2c_available() {
  static std::atomic<int> state[64];               // 0 unknown, 1 yes, 2 no
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  int s = state[dev & 63].load(std::memory_order_relaxed);
  if (s == 0) {
    bool ok = cudaFuncSetAttribute(k_fuse2c, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fc::SMEM) ==
                  cudaSuccess &&
              cudaFuncSetAttribute(k_fuse2c, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess;
    int maxc = 0;
    if (ok) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(fc::K, 1);
      cfg.blockDim = dim3(fc::THREADS);
      cfg.dynamicSmemBytes = fc::SMEM;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = fc::K;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      ok = cudaOccupancyMaxActiveClusters(&maxc, k_fuse2c, &cfg) == cudaSuccess && maxc > 0;
    }
    cudaGetLastError();
    s = ok ? 1 : 2;
    state[dev & 63].store(s, std::memory_order_relaxed);
  }
  return s == 1;
}

// Clusters (16 CTAs each) of one fused launch: one per prefix index and
// right-hand side, at most 65535 (the grid's y dimension).
long long fuse2c_clusters(int d, const int* n, int nrhs) {
  long long b = nrhs;
  for (int m = 0; m + 2 < d; ++m) b *= n[m];
  return b;
}

// node: a level-(d-2) node with parity bits `prefix`, scratch: a vector of
// the same size.  Errors: cudaErrorInvalidValue for a shape the kernel does
// not take (or more than 65535 clusters), cudaErrorNotSupported where the
// device does not schedule the cluster, cudaErrorMisalignedAddress unless
// node and scratch are 16-byte aligned.
cudaError_t launch_fuse2c(float2* node, float2* scratch, int prefix, int d, const int* n, int nrhs,
                          const FftDev& f1, const FftDev& f2, const SymDev& sym, cudaStream_t st) {
  if (d < 3 || d > MAX_D || f1.N != fc::N || f2.N != fc::N || nrhs < 0) return cudaErrorInvalidValue;
  if (((uintptr_t)node | (uintptr_t)scratch) & 15) return cudaErrorMisalignedAddress;
  const long long clusters = fuse2c_clusters(d, n, nrhs);
  if (clusters == 0) return cudaSuccess;
  if (clusters > 65535) return cudaErrorInvalidValue;
  if (!fuse2c_available()) return cudaErrorNotSupported;
  FuseCArgs a;
  memset(&a, 0, sizeof a);
  long long nslab = 1;
  a.pd = d - 2;
  for (int m = 0; m < a.pd; ++m) {
    a.ext[m] = n[m];
    nslab *= n[m];
  }
  a.node = node; a.scratch = scratch; a.prefix = prefix; a.nrhs = nrhs;
  a.comp_stride = nslab * fc::N * fc::N;
  a.tw = (const float2*)f2.tw; a.ph = (const float2*)f2.ph;
  a.sym = sym;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(fc::K, (unsigned)clusters);
  cfg.blockDim = dim3(fc::THREADS);
  cfg.dynamicSmemBytes = fc::SMEM;
  cfg.stream = st;
  cudaLaunchAttribute at[2];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = fc::K;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  at[1].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[1].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 2;
  return cudaLaunchKernelEx(&cfg, k_fuse2c, a);
}

}  // namespace btmv
