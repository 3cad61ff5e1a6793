// Register-resident line FFT kernels for power-of-two line lengths
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
//   k_leaf_reg<P, C>  leaf pass: both halves of the last level, symbol
//                     multiply, merge; the two halves run in two thread
//                     groups and are summed through shared memory.
#include <cuda_runtime.h>
#include <stdint.h>

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

// shared-memory views of one line
struct SmCol {            // [p][col] with W columns, col fastest
  float2* base;
  int W;
  __device__ __forceinline__ float2 ld(int p) const { return base[p * W]; }
  __device__ __forceinline__ void st(int p, float2 v) const { base[p * W] = v; }
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};
struct SmLine {           // one line, one pad slot every 16 points
  float2* base;
  __device__ __forceinline__ float2 ld(int p) const { return base[p + (p >> 4)]; }
  __device__ __forceinline__ void st(int p, float2 v) const { base[p + (p >> 4)] = v; }
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};

template <class P> __host__ __device__ constexpr int padded_len() { return P::N + P::N / 16; }

// In: a[m] = v[t + T m].  Out: a[m] = DFT(v)[t + T m] (forward or inverse, unnormalised).
template <class P, bool INV, class SM>
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
      for (int r = 1; r < R2; ++r) b[r] = twm<INV>(b[r], __ldg(&tw[r * f1]));
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
      for (int r = 1; r < R2; ++r) c2[q][r] = twm<INV>(c2[q][r], __ldg(&tw[r * f1 * MP]));
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
      for (int r = 1; r < R3; ++r) b[r] = twm<INV>(b[r], __ldg(&tw[r * f1]));
      dft<R3, INV>(b);
#pragma unroll
      for (int f2 = 0; f2 < R3; ++f2) a[q + NQ3 * f2] = b[f2];
    }
  }
}

// ------------------------------------------------------------- strided pass
// columns per tile: 16 x 8 B = 128 B rows (8 for N = 512 to stay in 32 KB)
template <class P> __host__ __device__ constexpr int pass_cols() { return P::N <= 256 ? 16 : 8; }

template <class P, int MODE>
__global__ void __launch_bounds__(pass_cols<P>() * P::T) k_pass_reg(const PassArgs a) {
  constexpr int R1 = P::R1, TT = P::T, N = P::N, PW = pass_cols<P>();
  __shared__ float2 sm[N * PW];
  const int col = threadIdx.x % PW;
  const int t = threadIdx.x / PW;
  const long long gl = (long long)blockIdx.x * PW + col;
  const bool ok = gl < a.g.lines;
  const long long inner = a.g.Itot;
  const long long o = ok ? gl / inner : 0;
  const long long ii = ok ? gl - o * inner : 0;
  const long long base = o * (long long)N * inner + ii;   // same geometry for every array
  const float2* __restrict__ tw = (const float2*)a.fft.tw;
  const float2* __restrict__ ph = (const float2*)a.fft.ph;
  const SmCol smc{sm + col, PW};

  if (MODE == 0) {
    const float2* __restrict__ in = (const float2*)a.in0;
    float2 v[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) v[m] = ok ? in[base + (long long)(t + TT * m) * inner] : make_float2(0.f, 0.f);
    if (a.out0) {
      float2 w[R1];
#pragma unroll
      for (int m = 0; m < R1; ++m) w[m] = v[m];
      fft_reg<P, false>(w, t, smc, tw);
      float2* __restrict__ out = (float2*)a.out0;
      if (ok)
#pragma unroll
        for (int m = 0; m < R1; ++m) out[base + (long long)(t + TT * m) * inner] = w[m];
    }
    if (a.out1) {
#pragma unroll
      for (int m = 0; m < R1; ++m) v[m] = cmul(v[m], __ldg(&ph[t + TT * m]));
      fft_reg<P, false>(v, t, smc, tw);
      float2* __restrict__ out = (float2*)a.out1;
      if (ok)
#pragma unroll
        for (int m = 0; m < R1; ++m) out[base + (long long)(t + TT * m) * inner] = v[m];
    }
  } else {
    const float2* __restrict__ ine = (const float2*)a.in0;
    const float2* __restrict__ ino = (const float2*)a.in1;
    float2 e[R1], od[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) e[m] = ok ? ine[base + (long long)(t + TT * m) * inner] : make_float2(0.f, 0.f);
    if (ino) {
#pragma unroll
      for (int m = 0; m < R1; ++m) od[m] = ok ? ino[base + (long long)(t + TT * m) * inner] : make_float2(0.f, 0.f);
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
      for (int m = 0; m < R1; ++m) out[base + (long long)(t + TT * m) * inner] = e[m];
  }
}

// ------------------------------------------------------------------- leaf
constexpr int LEAF_THREADS = 256;

// Split leaf: thread groups 2g and 2g+1 take the even and odd half of one
// line.  Plain embedding (a.split == 0): every group takes its own 2n line.
template <class P, int C>
__global__ void __launch_bounds__(LEAF_THREADS) k_leaf_reg(const LeafArgs a) {
  constexpr int R1 = P::R1, TT = P::T, N = P::N, PN = padded_len<P>();
  constexpr int GROUPS = LEAF_THREADS / TT;
  __shared__ float2 sm[GROUPS * PN];
  const int gid = threadIdx.x / TT;
  const int t = threadIdx.x % TT;
  const int LPC = a.split ? GROUPS / 2 : GROUPS;   // lines per CTA
  const int b = a.split ? (gid & 1) : 0;
  const int li = a.split ? (gid >> 1) : gid;
  const SmLine sml{sm + gid * PN};
  const SmLine partner{sm + (gid ^ 1) * PN};
  const LeafNode nd = a.nodes[blockIdx.y];
  const long long gline = (long long)blockIdx.x * LPC + li;  // over (rhs, line)
  const bool ok = gline < (long long)a.nrhs * a.lines;
  const long long q = ok ? gline / a.lines : 0;
  const long long line = ok ? gline - q * a.lines : 0;
  const long long base = q * a.rhs_stride + line * N;
  const float2* __restrict__ tw = (const float2*)a.fft.tw;
  const float2* __restrict__ ph = (const float2*)a.fft.ph;
  const float2* __restrict__ in = (const float2*)nd.in;

  float2 v[C][R1];
#pragma unroll
  for (int c = 0; c < C; ++c)
#pragma unroll
    for (int m = 0; m < R1; ++m)
      v[c][m] = ok ? in[base + c * a.comp_stride + t + TT * m] : make_float2(0.f, 0.f);
  if (b) {
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const float2 p = __ldg(&ph[t + TT * m]);
#pragma unroll
      for (int c = 0; c < C; ++c) v[c][m] = cmul(v[c][m], p);
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) fft_reg<P, false>(v[c], t, sml, tw);

  // symbol rows of this line for both parities of the last dim: class,
  // fold mask and linear prefix of dims 0..d-2
  const SymDev& S = a.sym;
  const int dl = a.dl;
  int clsp = 0, foldp = 0;
  int fpre[MAX_D];
  {
    long long r = line;
    for (int m = dl - 1; m >= 0; --m) {
      const int im = (int)(r % a.ext[m]);
      r /= a.ext[m];
      fpre[m] = a.split ? 2 * im + ((nd.prefix >> m) & 1) : im;
    }
    for (int m = 0; m < dl; ++m) clsp = (clsp << 1) | (fpre[m] & 1);
  }
  long long lin = 0;
  for (int m = 0; m < dl; ++m) {
    int fm = fpre[m];
    if (S.compressed && fm > S.n[m]) { fm = 2 * S.n[m] - fm; foldp |= 1 << m; }
    lin = lin * S.J[clsp << 1][m] + (fm >> 1);    // J of dims < dl does not depend on the last bit
  }
  const int nl = S.n[dl];
  long long rowc[2], blkc[2];
#pragma unroll
  for (int bb = 0; bb < 2; ++bb) {
    const int cl = (clsp << 1) | bb;
    rowc[bb] = S.cls_off[cl] + lin * S.J[cl][dl];
    blkc[bb] = S.blk[cl];
  }
  const float2* __restrict__ Sd = (const float2*)S.data;
  int kk[3][3];
#pragma unroll
  for (int i = 0; i < C; ++i)
#pragma unroll
    for (int j = 0; j < C; ++j) kk[i][j] = S.comp[i][j];

#pragma unroll
  for (int m = 0; m < R1; ++m) {
    const int l = t + TT * m;
    int f = a.split ? 2 * l + b : l;
    int fold = foldp;
    if (S.compressed && f > nl) { f = 2 * nl - f; fold |= 1 << dl; }
    const int pb = f & 1;                 // parity class bit of the last dim
    const long long idx = rowc[pb] + (f >> 1);
    const long long blk = blkc[pb];
    if (C == 1) {
      float2 s = __ldg(&Sd[idx]);
      if (__popc(S.oddmask[0] & fold) & 1) { s.x = -s.x; s.y = -s.y; }
      v[0][m] = cmul(s, v[0][m]);
    } else {
      float2 x[C];
#pragma unroll
      for (int c = 0; c < C; ++c) x[c] = v[c][m];
#pragma unroll
      for (int i = 0; i < C; ++i) {
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const int k = kk[i][j];
          float2 s = __ldg(&Sd[idx + k * blk]);
          if (__popc(S.oddmask[k] & fold) & 1) { s.x = -s.x; s.y = -s.y; }
          acc = cadd(acc, cmul(s, x[j]));
        }
        v[i][m] = acc;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < C; ++c) fft_reg<P, true>(v[c], t, sml, tw);

  // merge the halves: the odd group hands conj(P) y_odd to the even group
  float2* __restrict__ out = (float2*)nd.out;
#pragma unroll
  for (int c = 0; c < C; ++c) {
    __syncthreads();
    if (a.split && b) {
#pragma unroll
      for (int m = 0; m < R1; ++m) sml.st(t + TT * m, cmulc(v[c][m], __ldg(&ph[t + TT * m])));
    }
    __syncthreads();
    if (!b && ok) {
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        float2 y = v[c][m];
        if (a.split) y = cadd(y, partner.ld(t + TT * m));
        out[base + c * a.comp_stride + t + TT * m] = y;
      }
    }
  }
}

// ------------------------------------------------------------- dispatch
template <class P>
static cudaError_t pass_reg_p(int mode, const PassArgs& a, cudaStream_t st) {
  constexpr int PW = pass_cols<P>();
  const long long nt = (a.g.lines + PW - 1) / PW;
  if (nt <= 0) return cudaSuccess;
  if (mode == 0) k_pass_reg<P, 0><<<(unsigned)nt, PW * P::T, 0, st>>>(a);
  else           k_pass_reg<P, 1><<<(unsigned)nt, PW * P::T, 0, st>>>(a);
  return cudaGetLastError();
}

bool pass_reg_supported(const PassArgs& a, size_t esz) {
  if (esz != sizeof(float2)) return false;
  if (a.g.contig || a.g.ni != 1) return false;
  const int N = a.g.N;
  if (!(N == 32 || N == 64 || N == 128 || N == 256 || N == 512)) return false;
  // plain contiguous node geometry: every array [outer][N][inner], full lines
  const ArrMap* ms[4] = {&a.a_in0, &a.a_in1, &a.a_out0, &a.a_out1};
  for (auto m : ms)
    if (m->os != (long long)N * a.g.Itot || m->es != a.g.Itot || m->is[0] != 1 || m->len != N) return false;
  return true;
}

cudaError_t launch_pass_reg(int mode, const PassArgs& a, cudaStream_t st) {
  switch (a.g.N) {
    case 32: return pass_reg_p<RP32>(mode, a, st);
    case 64: return pass_reg_p<RP64>(mode, a, st);
    case 128: return pass_reg_p<RP128>(mode, a, st);
    case 256: return pass_reg_p<RP256>(mode, a, st);
    case 512: return pass_reg_p<RP512>(mode, a, st);
  }
  return cudaErrorNotSupported;
}

template <class P, int C>
static cudaError_t leaf_reg_p(const LeafArgs& a, cudaStream_t st) {
  const int LPC = a.split ? LEAF_THREADS / P::T / 2 : LEAF_THREADS / P::T;
  const long long total = (long long)a.nrhs * a.lines;
  const long long nt = (total + LPC - 1) / LPC;
  if (nt <= 0 || a.nnodes <= 0) return cudaSuccess;
  dim3 grid((unsigned)nt, (unsigned)a.nnodes);
  k_leaf_reg<P, C><<<grid, LEAF_THREADS, 0, st>>>(a);
  return cudaGetLastError();
}

bool leaf_reg_supported(const LeafArgs& a, size_t esz) {
  if (esz != sizeof(float2)) return false;
  if (!(a.c == 1 || a.c == 3)) return false;
  const int N = a.N;
  return N == 32 || N == 64 || N == 128 || N == 256 || N == 512;
}

template <int C>
static cudaError_t leaf_reg_c(const LeafArgs& a, cudaStream_t st) {
  switch (a.N) {
    case 32: return leaf_reg_p<RP32, C>(a, st);
    case 64: return leaf_reg_p<RP64, C>(a, st);
    case 128: return leaf_reg_p<RP128, C>(a, st);
    case 256: return leaf_reg_p<RP256, C>(a, st);
    case 512: return leaf_reg_p<RP512, C>(a, st);
  }
  return cudaErrorNotSupported;
}

cudaError_t launch_leaf_reg(const LeafArgs& a, cudaStream_t st) {
  return a.c == 1 ? leaf_reg_c<1>(a, st) : leaf_reg_c<3>(a, st);
}

}  // namespace btmv
