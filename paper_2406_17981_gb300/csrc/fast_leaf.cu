// Register-resident fused leaf pass for the line lengths fast.cuh provides
// plans for.
#include <cstdlib>

#include "fast.cuh"

namespace btmv {

// ------------------------------------------------------------------- leaf
// One thread group of T threads per (line, component); a line's C groups
// sit next to each other in the block.  Each group runs the even half, then
// the odd half of the last level: forward FFT, spectrum to shared memory, the
// row cc of the c x c symbol multiply (reading the other components'
// spectra), inverse FFT.  The even result waits in a per-group stash until
// the odd one is added with conj(P).  The plain embedding (a.split == 0)
// runs a single 2n-point pass per line.
template <class P, int C> struct LeafCfg {
  // lines per block: 96 threads for c = 3, 128 for c = 1 (whole warps);
  // one line when its groups alone fill more (T = 64)
  static constexpr int LPC = (C == 1 ? 128 / P::T : 32 / P::T) > 0 ? (C == 1 ? 128 / P::T : 32 / P::T) : 1;
  static constexpr int THREADS = LPC * C * P::T;
  static constexpr int SPN = padded_len<P>();
  static constexpr int BASE = SPN + P::N;                        // spectrum + stash
  static constexpr int TGT = P::T < 16 ? P::T : 0;
  static constexpr int GS = BASE + ((TGT - BASE % 16) + 16) % 16;  // group stride, = T mod 16
  // staged symbol rows: stored block k of a line's row starts at
  // k * JP + 8 * s(k) and lines are LS apart, chosen so that the rows two
  // thread groups of a half-warp read together sit in opposite bank halves
  static constexpr int JP = ((P::N / 2 + 1 + 8) + 15) / 16 * 16;
  static __host__ __device__ constexpr int line_stride(int nsym) { return nsym * JP + 8; }
  // blocks per SM to aim for; the c = 3 160- and 192-point plans run four with
  // their stage twiddles read from the table (measured faster than two or
  // three with register twiddles; the other composite plans spill at four)
  static constexpr bool OCC4 = C == 3 && (P::N == 160 || P::N == 192);
  static constexpr int MINB = OCC4 ? 4 : P::R3 == 1 ? (C == 1 ? 2 : (P::R1 <= 16 ? 5 : 2)) : 1;
  // dynamic smem: groups | phase table | staged symbol rows (nsym per line)
  static size_t smem(int nsym) {
    return ((size_t)LPC * C * GS + P::N + (size_t)LPC * line_stride(nsym)) * sizeof(float2);
  }
};

__device__ __forceinline__ void cp_async8(void* sdst, const void* gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <class P, int C, bool FF>
__global__ void __launch_bounds__(LeafCfg<P, C>::THREADS, LeafCfg<P, C>::MINB) k_leaf_cg(const LeafArgs a) {
  typedef LeafCfg<P, C> CF;
  constexpr int R1 = P::R1, TT = P::T, N = P::N, PD = pad_div<P>(), JP = CF::JP;
  extern __shared__ __align__(16) float2 smem_cg[];
  const int gid = threadIdx.x / TT;           // group in block
  const int t = threadIdx.x % TT;
  const int li = gid / C;                     // line in block
  const int cc = gid - li * C;                // component of this group
  const int lt = threadIdx.x - li * C * TT;   // thread index within the line
  float2* const gbuf = smem_cg + gid * CF::GS;
  const SmLine<PD, TT> spec{gbuf};
  float2* const stash = gbuf + CF::SPN;
  float2* const phs = smem_cg + CF::LPC * C * CF::GS;           // phase table P (N values)
  const SymDev& S = a.sym;
  constexpr int NS = C == 3 ? 6 : 1;                            // stored blocks staged by FF kernels
  const LeafNode nd = a.nodes[blockIdx.y];
  // 32-bit line arithmetic: the launcher guarantees nrhs * lines < 2^31.
  // Lines are ordered right-hand side fastest: the lines of one spatial line
  // for several right-hand sides sit in one block and share one staged
  // symbol row (slot li0, the block's first line of that spatial line), so
  // the row is read once for all of them.
  const unsigned lines = (unsigned)a.lines;
  const unsigned nr = (unsigned)a.nrhs;
  const unsigned gline = blockIdx.x * (unsigned)CF::LPC + (unsigned)li;   // over (line, rhs)
  const bool ok = gline < nr * lines;
  const unsigned line = ok ? gline / nr : 0u;
  const unsigned q = ok ? gline - line * nr : 0u;
  const int li0 = li - (int)(q < (unsigned)li ? q : (unsigned)li);
  float2* const rowb = phs + N + li0 * CF::line_stride(FF ? NS : 0);  // staged symbol row of this line
  const long long base = (long long)q * a.rhs_stride + cc * a.comp_stride + (long long)line * N + t;
  const float2* __restrict__ tw = (const float2*)a.fft.tw;
  const float2* __restrict__ ph = (const float2*)a.fft.ph;

  // symbol addressing for this line: split-grid frequency of each line dim,
  // its parity class and (compressed store) the fold to 2n - f
  const int dl = a.dl;
  int clsp = 0, foldp = 0;
  unsigned lin = 0;
  {
    int fpre[MAX_D - 1];
    unsigned r = line;
#pragma unroll
    for (int m = MAX_D - 2; m >= 1; --m) {
      if (m < dl) {
        const unsigned e = (unsigned)a.ext[m];
        const unsigned r2 = r / e;
        fpre[m] = (int)(r - r2 * e);
        r = r2;
      }
    }
    fpre[0] = (int)r;
#pragma unroll
    for (int m = 0; m < MAX_D - 1; ++m)
      if (m < dl) {
        fpre[m] = a.split ? 2 * fpre[m] + ((nd.prefix >> m) & 1) : fpre[m];
        clsp = (clsp << 1) | (fpre[m] & 1);
      }
#pragma unroll
    for (int m = 0; m < MAX_D - 1; ++m)
      if (m < dl) {
        int fm = fpre[m];
        if (S.compressed && fm > S.n[m]) { fm = 2 * S.n[m] - fm; foldp |= 1 << m; }
        lin = lin * (unsigned)S.J[clsp << 1][m] + (unsigned)(fm >> 1);
      }
  }
  const int nl = S.n[dl];
  const float2* __restrict__ Sd = (const float2*)S.data;
  // FF: split leaf on the mirror-compressed store with n_d == N and NS
  // stored blocks (block-symmetric c = 3, or c = 1); the line's row of each
  // parity class is staged in shared memory while the transforms run
  const int nsym = FF ? NS : S.nsym;
  // bank-half shift of each stored block of the c = 3 block-symmetric row:
  // blocks 00 11 22 01 02 12 -> 0 0 0 1 0 1
  auto row_pos = [&](int k) { return k * JP + ((C == 3 && nsym == 6 && (k == 3 || k == 5)) ? 8 : 0); };
  auto stage_row = [&](int bb) {
    if constexpr (FF) {
      if (!ok || li0 != li) return;    // staged by the first line of the block with this spatial line
      const int cl = (clsp << 1) | bb;
      const int J = S.J[cl][dl];
      const float2* src = Sd + S.cls_off[cl] + (long long)lin * J;
      const long long blk = S.blk[cl];
      constexpr int IT = (N / 2 + 1 + C * TT - 1) / (C * TT);
#pragma unroll
      for (int k = 0; k < NS; ++k)
#pragma unroll
        for (int i = 0; i < IT; ++i) {
          const int j = lt + i * C * TT;
          if (j < J) cp_async8(rowb + row_pos(k) + j, src + k * blk + j);
        }
    }
  };
  for (int e = threadIdx.x; e < N; e += CF::THREADS) cp_async8(phs + e, ph + e);
  stage_row(0);

  constexpr bool REGTW = P::R3 == 1 && !CF::OCC4;   // stage-2 twiddles held in registers
  TwReg<P> twr;
  if constexpr (REGTW) twr.load(t, tw);

  // the input line is read once per half (the odd half's read hits in cache)
  // rather than held in registers across both halves
  const float2* __restrict__ xin = (const float2*)nd.in + base;

  // OWN: the group's own spectrum is taken from registers.  Row cc is then
  // walked in the order cc, cc+1, ... (mod C).  With T < 16 two groups of
  // different components share a half-warp and the walk in the plain order
  // 0..C-1 keeps their shared-memory reads conflict-free (the same
  // spectrum, or buffers in opposite bank halves) and as few wavefronts, so
  // OWN is used by the split leaf when a group fills its half-warps
  // (T >= 16) or c = 1.
  constexpr bool OWN = FF && (TT >= 16 || C == 1);   // (measured slower in the plain-embedding leaf)
  int jo[C];
#pragma unroll
  for (int jj = 0; jj < C; ++jj) jo[jj] = !OWN ? jj : cc + jj < C ? cc + jj : cc + jj - C;
  long long off[2][C];
  int kr[C];
  unsigned sg0 = 0, sg1 = 0;      // sign bits of row cc without / with a fold of the last dim
#pragma unroll
  for (int jj = 0; jj < C; ++jj) {
    const int k = S.comp[cc][jo[jj]];
    kr[jj] = row_pos(k);
#pragma unroll
    for (int bb = 0; bb < 2; ++bb) {
      const int cl = (clsp << 1) | bb;
      off[bb][jj] = S.cls_off[cl] + (long long)lin * S.J[cl][dl] + (long long)k * S.blk[cl];
    }
    sg0 |= (unsigned)(__popc(S.oddmask[k] & foldp) & 1) << jj;
    sg1 |= (unsigned)(__popc(S.oddmask[k] & (foldp | (1 << dl))) & 1) << jj;
  }
  float sgf0[C], sgf1[C];
#pragma unroll
  for (int jj = 0; jj < C; ++jj) {
    sgf0[jj] = ((sg0 >> jj) & 1) ? -1.f : 1.f;
    sgf1[jj] = ((sg1 >> jj) & 1) ? -1.f : 1.f;
  }
  float2* const lbase = smem_cg + (li * C) * CF::GS;   // spectra of this line's groups
  float2* sp[C];
#pragma unroll
  for (int jj = 0; jj < C; ++jj) sp[jj] = lbase + jo[jj] * CF::GS;

  grid_dep_wait();                    // the nodes written by the previous kernel

  // split leaves run both halves; the loop stays rolled (half the code of
  // the unrolled form, which measured slower)
  const int nbr = FF ? 2 : (a.split ? 2 : 1);
#pragma unroll 1
  for (int b = 0; b < nbr; ++b) {
    if (b) cp_async_wait_all();       // phase table staged
    __syncthreads();
    float2 w[R1];
#pragma unroll
    for (int m = 0; m < R1; ++m) {
      const float2 xv0 = ok ? xin[TT * m] : make_float2(0.f, 0.f);
      w[m] = b ? cmul(xv0, phs[t + TT * m]) : xv0;
    }
    if constexpr (REGTW) fft_reg2<P, false>(w, t, spec, twr);
    else fft_reg<P, false>(w, t, spec, tw);
    spec.sync();                      // the transform's last reads of the line buffer are done
    if constexpr (!(FF && C == 1)) {   // the other groups' operand (c = 1 fast-fold needs none)
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        if constexpr (PD == TT) *spec.cyc(t, m) = w[m];
        else spec.st(t + TT * m, w[m]);
      }
    }
    cp_async_wait_all();              // this branch's symbol row
    __syncthreads();
    // row cc of the symbol multiply at the thread's frequencies
    if constexpr (FF) {
      // frequency f = 2l + b is stored directly for l < N/2 (m < R1/2) and
      // folded to 2N - f, index N - l - b, with the fold signs for l >= N/2
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        const bool hi = m >= R1 / 2;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          const float2 sv = hi ? rowb[kr[j] + (N - b - t - TT * m)] : rowb[kr[j] + (t + TT * m)];
          const float sgn = hi ? sgf1[j] : sgf0[j];
          const SmLine<PD, TT> sj{sp[j]};
          const float2 xv = (OWN && j == 0) ? w[m] : (PD == TT) ? *sj.cyc(t, m) : sj.ld(t + TT * m);
          // acc += sgn * (sv * xv): the parity sign rides on the accumulating FMA
          const float px = fmaf(sv.x, xv.x, -sv.y * xv.y);
          const float py = fmaf(sv.x, xv.y, sv.y * xv.x);
          acc.x = fmaf(sgn, px, acc.x);
          acc.y = fmaf(sgn, py, acc.y);
        }
        w[m] = acc;
      }
    } else {
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        const int l = t + TT * m;
        int f = a.split ? 2 * l + b : l;
        unsigned sg = sg0;
        if (S.compressed && f > nl) { f = 2 * nl - f; sg = sg1; }
        const int pb = f & 1;
        const int fi = f >> 1;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int j = 0; j < C; ++j) {
          float2 sv = __ldg(&Sd[off[pb][j] + fi]);
          if ((sg >> j) & 1) { sv.x = -sv.x; sv.y = -sv.y; }
          const SmLine<PD, TT> sj{sp[j]};
          acc = cadd(acc, cmul(sv, (OWN && j == 0) ? w[m] : sj.ld(l)));
        }
        w[m] = acc;
      }
    }
    __syncthreads();
    if (b == 0 && a.split) stage_row(1);   // overlaps the inverse and the odd forward transform
    if constexpr (REGTW) fft_reg2<P, true>(w, t, spec, twr);
    else fft_reg<P, true>(w, t, spec, tw);
    if (a.split && b == 0) {
#pragma unroll
      for (int m = 0; m < R1; ++m) stash[t + TT * m] = w[m];
    } else {
      float2* __restrict__ out = (float2*)nd.out + base;
      if (ok) {
#pragma unroll
        for (int m = 0; m < R1; ++m) {
          float2 y = w[m];
          if (a.split) y = cadd(stash[t + TT * m], cmulc(y, phs[t + TT * m]));
          out[TT * m] = y;
        }
      }
    }
  }
  cp_async_wait_all();
}

template <class P, int C, bool FF>
static cudaError_t leaf_reg_pf(const LeafArgs& a, cudaStream_t st) {
  typedef LeafCfg<P, C> CF;
  const long long total = (long long)a.nrhs * a.lines;
  const long long nt = (total + CF::LPC - 1) / CF::LPC;
  if (nt <= 0 || a.nnodes <= 0) return cudaSuccess;
  const size_t sm = CF::smem(FF ? a.sym.nsym : 0);
  if (sm > 227 * 1024) return cudaErrorInvalidValue;
  const cudaError_t ae = set_smem_attr<k_leaf_cg<P, C, FF>>(227 * 1024);
  if (ae != cudaSuccess) return ae;
  dim3 grid((unsigned)nt, (unsigned)a.nnodes);
#ifndef BTMV_NO_PDL
  return launch_pdl(k_leaf_cg<P, C, FF>, grid, dim3(CF::THREADS), sm, st, a);
#else
  k_leaf_cg<P, C, FF><<<grid, CF::THREADS, sm, st>>>(a);
  return cudaGetLastError();
#endif
}

template <class P, int C>
static cudaError_t leaf_reg_p(const LeafArgs& a, cudaStream_t st) {
  const bool ff = a.split && a.sym.compressed && a.sym.n[a.dl] == a.N && a.sym.nsym == (C == 3 ? 6 : 1);
  return ff ? leaf_reg_pf<P, C, true>(a, st) : leaf_reg_pf<P, C, false>(a, st);
}

bool leaf_reg_supported(const LeafArgs& a, size_t esz) {
  if (esz != sizeof(float2)) return false;
  if (!(a.c == 1 || a.c == 3)) return false;
  if ((long long)a.nrhs * a.lines >= (1ll << 31)) return false;   // 32-bit line indices
  return reg_length(a.N);
}

template <int C>
static cudaError_t leaf_reg_c(const LeafArgs& a, cudaStream_t st) {
  switch (a.N) {
    case 24: return leaf_reg_p<RP24, C>(a, st);
    case 48: return leaf_reg_p<RP48, C>(a, st);
    case 60: return leaf_reg_p<RP60, C>(a, st);
    case 84: return leaf_reg_p<RP84, C>(a, st);
    case 96: return leaf_reg_p<RP96, C>(a, st);
    case 192: return leaf_reg_p<RP192, C>(a, st);
    case 160: return leaf_reg_p<RP160, C>(a, st);
    case 320: return leaf_reg_p<RP320, C>(a, st);
    case 384: return leaf_reg_p<RP384, C>(a, st);
    case 768: return leaf_reg_p<RP768, C>(a, st);
    case 640: return leaf_reg_p<RP640, C>(a, st);
    case 1024: return leaf_reg_p<RP1024, C>(a, st);
    case 32: return leaf_reg_p<RP32, C>(a, st);
    case 64: return leaf_reg_p<RP64, C>(a, st);
    case 128: return leaf_reg_p<RP128, C>(a, st);
    case 256: return leaf_reg_p<RP256, C>(a, st);
    case 512: return leaf_reg_p<RP512, C>(a, st);
  }
  return cudaErrorNotSupported;
}

// The c = 3 split leaf on the compressed block-symmetric store takes the
// component-in-thread kernel (fast_leaf3.cu) for 64- and 128-point lines,
// where it measured faster (128^3: 115 against 124 us per launch), and the
// component-group kernel above for longer lines (256^3: 891 against 901 us).
// BTMV_LEAF3=0 / 1 in the environment forces one or the other (comparisons).
static bool use_leaf3(const LeafArgs& a) {
  if (a.c != 3 || !leaf3_supported(a, sizeof(float2))) return false;
  const char* v = getenv("BTMV_LEAF3");
  if (v && v[0] == '0') return false;
  if (v && v[0] == '1') return true;
  return a.N <= 128;
}

cudaError_t launch_leaf_reg(const LeafArgs& a, cudaStream_t st) {
  if (use_leaf3(a)) return launch_leaf3(a, st);
  return a.c == 1 ? leaf_reg_c<1>(a, st) : leaf_reg_c<3>(a, st);
}

}  // namespace btmv
