// Register-resident strided line passes (forward split and merge) for the
// line lengths fast.cuh provides plans for.
#include "fast.cuh"

namespace btmv {

// ------------------------------------------------------------- strided pass
// columns per tile: 16 x 8 B = 128 B rows; fewer for long lines so that the
// tile stays within the 48 KB of static shared memory
template <class P> __host__ __device__ constexpr int pass_cols() { return P::N <= 256 ? 16 : P::N <= 768 ? 8 : 4; }

// minimum resident blocks per SM for the radix-16 plans of 128..512 points,
// scaled to 128-thread blocks: 6 for the forward split (80 registers), 4 for
// the merge (two transforms in flight).  Both passes read the stage twiddles
// from the L1-resident table (measured faster than register twiddles at
// these occupancies).  The composite-radix plans hold more values per thread
// and run unbounded, except the forward split of 160 and 192 points, which
// fits 4 blocks in 128 registers without spills (2.4% faster at 160^3 and
// 192^3).
template <class P, int MODE> __host__ __device__ constexpr int pass_minb() {
  constexpr int b = (MODE == 0 ? 6 : 4) * 128 / (pass_cols<P>() * P::T);
  if (MODE == 0 && (P::N == 160 || P::N == 192)) return 4 * 128 / (pass_cols<P>() * P::T);  // 128 registers
  return (P::R1 == 16 && P::N >= 128 && P::N <= 512 && b > 0) ? b : 1;
}
template <class P, int MODE>
__global__ void __launch_bounds__(pass_cols<P>() * P::T, pass_minb<P, MODE>()) k_pass_reg(const PassArgs a) {
  constexpr int R1 = P::R1, TT = P::T, N = P::N, PW = pass_cols<P>();
  __shared__ float2 sm[N * PW];
  const int col = threadIdx.x % PW;
  const int t = threadIdx.x / PW;
  // 32-bit line arithmetic (the launcher guarantees lines < 2^31)
  const unsigned gl = blockIdx.x * (unsigned)PW + (unsigned)col;
  const bool ok = gl < (unsigned)a.g.lines;
  const unsigned inner = (unsigned)a.g.Itot;
  const unsigned o = ok ? gl / inner : 0u;
  const unsigned ii = ok ? gl - o * inner : 0u;
  // point t + T m of this line, the same geometry for every array
  const long long base = ((long long)o * N + t) * inner + ii;
  const long long step = (long long)TT * inner;
  const float2* __restrict__ tw = (const float2*)a.fft.tw;
  const float2* __restrict__ ph = (const float2*)a.fft.ph;
  const SmCol<PW, TT> smc{sm + col};
  grid_dep_wait();                                // the node written by the previous kernel

  if (MODE == 0) {
    const float2* __restrict__ in = (const float2*)a.in0;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = ok ? in[base + m * step] : make_float2(0.f, 0.f);
    if (a.out0) {
      float2 w[R1];
#pragma unroll
      for (int m = 0; m < R1; ++m) w[m] = v[m];
      fft_reg<P, false>(w, t, smc, tw);
      float2* __restrict__ out = (float2*)a.out0;
      if (ok)
#pragma unroll
        for (int m = 0; m < R1; ++m) out[base + m * step] = w[m];
    }
    if (a.out1) {
#pragma unroll
      for (int m = 0; m < R1; ++m) v[m] = cmul(v[m], __ldg(&ph[t + TT * m]));
      fft_reg<P, false>(v, t, smc, tw);
      float2* __restrict__ out = (float2*)a.out1;
      if (ok)
#pragma unroll
        for (int m = 0; m < R1; ++m) out[base + m * step] = v[m];
    }
  } else {
    const float2* __restrict__ ine = (const float2*)a.in0;
    const float2* __restrict__ ino = (const float2*)a.in1;
    float2 e[R1], od[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) e[m] = ok ? ine[base + m * step] : make_float2(0.f, 0.f);
    if (ino) {
#pragma unroll
      for (int m = 0; m < R1; ++m) od[m] = ok ? ino[base + m * step] : make_float2(0.f, 0.f);
    }
    fft_reg<P, true>(e, t, smc, tw);
    if (ino) {
      fft_reg<P, true>(od, t, smc, tw);
#pragma unroll
      for (int m = 0; m < R1; ++m) e[m] = cadd(e[m], cmulc(od[m], __ldg(&ph[t + TT * m])));
    }
    float2* __restrict__ out = (float2*)a.out0;
    if (ok)
#pragma unroll
      for (int m = 0; m < R1; ++m) out[base + m * step] = e[m];
  }
}

template <class P>
static cudaError_t pass_reg_p(int mode, const PassArgs& a, cudaStream_t st) {
  constexpr int PW = pass_cols<P>();
  const long long nt = (a.g.lines + PW - 1) / PW;
  if (nt <= 0) return cudaSuccess;
#ifndef BTMV_NO_PDL
  if (mode == 0) return launch_pdl(k_pass_reg<P, 0>, dim3((unsigned)nt), dim3(PW * P::T), 0, st, a);
  return launch_pdl(k_pass_reg<P, 1>, dim3((unsigned)nt), dim3(PW * P::T), 0, st, a);
#else
  if (mode == 0) k_pass_reg<P, 0><<<(unsigned)nt, PW * P::T, 0, st>>>(a);
  else           k_pass_reg<P, 1><<<(unsigned)nt, PW * P::T, 0, st>>>(a);
  return cudaGetLastError();
#endif
}

bool pass_reg_supported(const PassArgs& a, size_t esz) {
  if (esz != sizeof(float2)) return false;
  if (a.g.contig || a.g.ni != 1) return false;
  const int N = a.g.N;
  if (!reg_length(N)) return false;
  if (a.g.lines >= (1ll << 31)) return false;                     // 32-bit line indices
  // plain contiguous node geometry: every array [outer][N][inner], full lines
  const ArrMap* ms[4] = {&a.a_in0, &a.a_in1, &a.a_out0, &a.a_out1};
  for (auto m : ms)
    if (m->os != (long long)N * a.g.Itot || m->es != a.g.Itot || m->is[0] != 1 || m->len != N) return false;
  return true;
}

cudaError_t launch_pass_reg(int mode, const PassArgs& a, cudaStream_t st) {
  switch (a.g.N) {
    case 24: return pass_reg_p<RP24>(mode, a, st);
    case 48: return pass_reg_p<RP48>(mode, a, st);
    case 60: return pass_reg_p<RP60>(mode, a, st);
    case 84: return pass_reg_p<RP84>(mode, a, st);
    case 96: return pass_reg_p<RP96>(mode, a, st);
    case 192: return pass_reg_p<RP192>(mode, a, st);
    case 160: return pass_reg_p<RP160>(mode, a, st);
    case 320: return pass_reg_p<RP320>(mode, a, st);
    case 384: return pass_reg_p<RP384>(mode, a, st);
    case 768: return pass_reg_p<RP768>(mode, a, st);
    case 640: return pass_reg_p<RP640>(mode, a, st);
    case 1024: return pass_reg_p<RP1024>(mode, a, st);
    case 32: return pass_reg_p<RP32>(mode, a, st);
    case 64: return pass_reg_p<RP64>(mode, a, st);
    case 128: return pass_reg_p<RP128>(mode, a, st);
    case 256: return pass_reg_p<RP256>(mode, a, st);
    case 512: return pass_reg_p<RP512>(mode, a, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace btmv
