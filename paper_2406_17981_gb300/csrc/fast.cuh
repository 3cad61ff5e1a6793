// Register-resident line FFT building blocks (shared by fast_pass.cu and
// fast_leaf.cu).  Register-resident line FFT kernels for power-of-two line lengths
// 32..512 (complex64).  A line of N points is held by T = N / R1 threads,
// thread t owning the points t + T m (m < R1); the first radix-R1 stage runs
// in registers, the remaining one or two stages read a shared-memory copy
// written by stage 1, and the result comes back in the same cyclic
// distribution (thread t owns frequencies t + T m).  Because the forward
// output and the inverse input share that distribution, the leaf pass does
// forward FFT -> c x c symbol multiply -> inverse FFT without touching
// shared memory between the two transforms.
//
//   k_pass_reg<P, 0>  forward split pass (even and odd children of a node)
//   k_pass_reg<P, 1>  merge pass (IFFT(even) + conj(P) IFFT(odd))
//   k_leaf_cg<P, C>   leaf pass: both halves of the last level, symbol
//                     multiply, merge; one thread group per (line,
//                     component), spectra exchanged through shared memory.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "kernels.cuh"

namespace btmv {

template <int N_, int R1_, int R2_, int R3_>
struct RP {
  static constexpr int N = N_, R1 = R1_, R2 = R2_, R3 = R3_, T = N_ / R1_;
};
typedef RP<32, 16, 2, 1> RP32;
typedef RP<64, 16, 4, 1> RP64;
typedef RP<128, 16, 8, 1> RP128;
typedef RP<256, 16, 16, 1> RP256;
typedef RP<512, 16, 8, 4> RP512;
// non-power-of-two lines: composite first-stage radix R1 with R2 = T | R1
typedef RP<24, 12, 2, 1> RP24;
typedef RP<48, 12, 4, 1> RP48;
typedef RP<60, 30, 2, 1> RP60;
typedef RP<96, 24, 4, 1> RP96;
typedef RP<192, 24, 8, 1> RP192;
typedef RP<84, 42, 2, 1> RP84;
// three-stage plans: T | N/R2, T | N/R3 and R3 | R1
typedef RP<160, 20, 4, 2> RP160;
typedef RP<320, 20, 4, 4> RP320;
typedef RP<384, 24, 8, 2> RP384;
typedef RP<768, 24, 4, 8> RP768;
typedef RP<640, 40, 4, 4> RP640;
typedef RP<1024, 16, 8, 8> RP1024;

// shared-memory views of one line
// Shared-memory views of one line.  ld/st take a point index p; cyc(t, m)
// is the address of point t + T m and ld2(t, q, r) the address of point
// (t + T q) T + r (the stage-2 input of a two-stage plan, where R2 = T), both
// written so that only the t-dependent part is computed at run time.
template <int W, int TT>
struct SmCol {            // [p][col] with W columns, col fastest
  float2* base;
  __device__ __forceinline__ float2 ld(int p) const { return base[p * W]; }
  __device__ __forceinline__ void st(int p, float2 v) const { base[p * W] = v; }
  __device__ __forceinline__ float2* cyc(int t, int m) const { return base + (t * W + m * TT * W); }
  __device__ __forceinline__ float2* ld2(int t, int q, int r) const { return base + (t * TT * W + (q * TT * TT + r) * W); }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
// One line owned by one thread group (warp-resident for T <= 32), one pad
// slot every PD points (PD = min(T, 16)).  With groups spaced by a stride that is T modulo
// 16 (in 8-byte words), the stage-1 writes and stage-2 reads of all groups
// sharing a half-warp fall into distinct banks.
template <int PD, int TT>
struct SmLine {
  float2* base;
  __device__ __forceinline__ float2 ld(int p) const { return base[p + p / PD]; }
  __device__ __forceinline__ void st(int p, float2 v) const { base[p + p / PD] = v; }
  // valid when PD == TT: point t + T m sits at t + m (T + 1)
  __device__ __forceinline__ float2* cyc(int t, int m) const { return base + (t + m * (TT + 1)); }
  __device__ __forceinline__ float2* ld2(int t, int q, int r) const {
    return base + (t * (TT + 1) + q * TT * (TT + 1) + r);
  }
  // a group of up to 32 threads lies in one warp; longer lines (T = 64)
  // span several warps and synchronise the whole block (every group of the
  // block reaches the same barriers)
  __device__ __forceinline__ void sync() const {
    if constexpr (TT > 32) __syncthreads();
    else __syncwarp();
  }
};

// Programmatic dependent launch.  The register kernels are launched with
// cudaLaunchAttributeProgrammaticStreamSerialization: the next kernel of the
// stream is launched once every block of the running one has exited (the
// implicit trigger), before that grid's completion and memory flush, so its
// blocks are scheduled and run their prologue (index arithmetic, constant
// tables, the symbol rows written at set-kernel time) while the previous
// grid retires.  Data written by the previous kernel is read only after
// grid_dep_wait(), which returns when that grid has completed and its
// writes are visible.  (An explicit early trigger measured slower: waiting
// blocks then shared the SMs with the previous kernel's last wave.)
// Without the attribute the wait is a no-op.
__device__ __forceinline__ void grid_dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <class... KArgs, class... Args>
static cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <class P> __host__ __device__ constexpr int pad_div() { return P::T < 16 ? P::T : 16; }
template <class P> __host__ __device__ constexpr int padded_len() { return P::N + P::N / pad_div<P>(); }

// Stage twiddle load: from the read-only global table (TWSM = false) or from
// a copy in shared memory (TWSM = true; a plain load, re-read at every use
// rather than held in registers across transforms).
template <bool TWSM>
__device__ __forceinline__ float2 twld(const float2* __restrict__ tw, int i) {
  if constexpr (TWSM) return tw[i];
  else return __ldg(&tw[i]);
}

// In: a[m] = v[t + T m].  Out: a[m] = DFT(v)[t + T m] (forward or inverse, unnormalised).
template <class P, bool INV, class SM, bool TWSM = false>
__device__ __forceinline__ void fft_reg(float2 (&a)[P::R1], int t, const SM& sm, const float2* __restrict__ tw) {
  constexpr int R1 = P::R1, R2 = P::R2, R3 = P::R3, TT = P::T;
  dft<R1, INV>(a);
  sm.sync();
#pragma unroll
  for (int f2 = 0; f2 < R1; ++f2) sm.st(t + TT * f2, a[f2]);
  sm.sync();
  if constexpr (R3 == 1) {
    constexpr int NQ = R1 / TT;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int f1 = t + TT * q;
      float2 b[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) b[r] = sm.ld(f1 * R2 + r);
#pragma unroll
      for (int r = 1; r < R2; ++r) b[r] = twm<INV>(b[r], twld<TWSM>(tw, r * f1));
      dft<R2, INV>(b);
#pragma unroll
      for (int f2 = 0; f2 < R2; ++f2) a[q + NQ * f2] = b[f2];
    }
  } else {
    constexpr int MP = R3;
    constexpr int NQ2 = P::N / (R2 * TT);
    float2 c2[NQ2][R2];
#pragma unroll
    for (int q = 0; q < NQ2; ++q) {
      const int j = t + TT * q;
      const int f1 = j / MP, kp = j % MP;
#pragma unroll
      for (int r = 0; r < R2; ++r) c2[q][r] = sm.ld(kp + MP * (R2 * f1 + r));
#pragma unroll
      for (int r = 1; r < R2; ++r) c2[q][r] = twm<INV>(c2[q][r], twld<TWSM>(tw, r * f1 * MP));
      dft<R2, INV>(c2[q]);
    }
    sm.sync();
#pragma unroll
    for (int q = 0; q < NQ2; ++q) {
      const int j = t + TT * q;
#pragma unroll
      for (int f2 = 0; f2 < R2; ++f2) sm.st(j + MP * R1 * f2, c2[q][f2]);
    }
    sm.sync();
    constexpr int L3 = R1 * R2, NQ3 = L3 / TT;
#pragma unroll
    for (int q = 0; q < NQ3; ++q) {
      const int f1 = t + TT * q;
      float2 b[R3];
#pragma unroll
      for (int r = 0; r < R3; ++r) b[r] = sm.ld(f1 * R3 + r);
#pragma unroll
      for (int r = 1; r < R3; ++r) b[r] = twm<INV>(b[r], twld<TWSM>(tw, r * f1));
      dft<R3, INV>(b);
#pragma unroll
      for (int f2 = 0; f2 < R3; ++f2) a[q + NQ3 * f2] = b[f2];
    }
  }
}

// Stage-2 twiddles of a two-stage plan held in registers: w[q][r] =
// exp(-2 pi i r f1 / N) for the thread's butterflies f1 = t + T q.
template <class P>
struct TwReg {
  static constexpr int NQ = P::R1 / P::T > 0 ? P::R1 / P::T : 1;   // (unused by three-stage plans)
  float2 w[NQ][P::R2];
  __device__ __forceinline__ void load(int t, const float2* __restrict__ tw) {
#pragma unroll
    for (int q = 0; q < NQ; ++q)
#pragma unroll
      for (int r = 0; r < P::R2; ++r) w[q][r] = __ldg(&tw[r * (t + P::T * q)]);
  }
};

// fft_reg for two-stage plans with the stage-2 twiddles already in registers.
template <class P, bool INV, class SM>
__device__ __forceinline__ void fft_reg2(float2 (&a)[P::R1], int t, const SM& sm, const TwReg<P>& tw) {
  constexpr int R1 = P::R1, R2 = P::R2, TT = P::T;
  static_assert(P::R3 == 1, "two-stage plans only");
  static_assert(R2 == TT, "two-stage plans have R2 == T");
  dft<R1, INV>(a);
  sm.sync();
#pragma unroll
  for (int f2 = 0; f2 < R1; ++f2) *sm.cyc(t, f2) = a[f2];
  sm.sync();
  constexpr int NQ = R1 / TT;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    float2 b[R2];
#pragma unroll
    for (int r = 0; r < R2; ++r) b[r] = *sm.ld2(t, q, r);
#pragma unroll
    for (int r = 1; r < R2; ++r) b[r] = twm<INV>(b[r], tw.w[q][r]);
    dft<R2, INV>(b);
#pragma unroll
    for (int f2 = 0; f2 < R2; ++f2) a[q + NQ * f2] = b[f2];
  }
}

template <class P, bool INV, class SM>
__device__ __forceinline__ void fft_any(float2 (&a)[P::R1], int t, const SM& sm, const TwReg<P>& twr,
                                        const float2* __restrict__ tw) {
  if constexpr (P::R3 == 1) fft_reg2<P, INV>(a, t, sm, twr);
  else fft_reg<P, INV>(a, t, sm, tw);
}

static inline bool reg_length(int N) {
  switch (N) {
    case 24: case 32: case 48: case 60: case 64: case 84: case 96: case 128: case 160: case 192: case 256: case 320:
    case 384: case 512: case 640: case 768: case 1024: return true;
  }
  return false;
}

}  // namespace btmv
