// Register-resident fused leaf pass, c = 3, one thread group per line
// holding all three components.
//
// The leaf (Algorithm 1, the last level; Sec. II.B) runs, per contiguous
// line and for both halves b of the last level: forward FFT of x_a (b = 1:
// of P_d x_a), the c x c symbol multiply Y_a(f) = sum_b' S_ab'(f) X_b'(f) at
// f = 2l + b, inverse FFT, and the merge y = y_even + conj(P_d) y_odd.
//
// Here a line's T threads own the points t + T m of every component, so the
// three spectra a frequency needs are in one thread's registers: the c x c
// multiply reads no other thread's data and the six stored symbol blocks are
// loaded straight from global memory (the mirror-compressed, block-symmetric
// store: f <= n read at f, f > n at 2n - f with the block's parity sign).
// Shared memory holds only the line's transpose buffer (one component at a
// time) and the even half's result until the odd half is added.  Lines are
// ordered right-hand side fastest, so with several right-hand sides the
// lines of one warp share symbol addresses (the symbol row is fetched once
// for all of them).
#include "fast.cuh"

namespace btmv {

template <class P, int MB> struct Leaf3Cfg {
  static constexpr int THREADS = 128;
  static constexpr int LPB = THREADS / P::T;                     // lines per block
  static constexpr int SPN = padded_len<P>();                    // transpose buffer
  static constexpr int BASE = SPN + 3 * P::N;                    // + stash of the three components
  static constexpr int TGT = P::T < 16 ? P::T : 0;
  static constexpr int LS = BASE + ((TGT - BASE % 16) + 16) % 16;  // line stride = T (mod 16) words
  static constexpr int MINB = MB;
  // lines | stage twiddle table (N) | phase table (N)
  static size_t smem() { return ((size_t)LPB * LS + 2 * P::N) * sizeof(float2); }
};

// IL: the multiply walks the low and folded high frequencies in pairs
// (m, R1 - 1 - m), whose symbol entries a warp fetches from the same lines,
// so the second read of an entry hits in L1.
template <class P, int MB, bool IL>
__global__ void __launch_bounds__(Leaf3Cfg<P, MB>::THREADS, MB) k_leaf3(const LeafArgs a) {
  typedef Leaf3Cfg<P, MB> CF;
  constexpr int R1 = P::R1, TT = P::T, N = P::N, PD = pad_div<P>();
  extern __shared__ __align__(16) float2 smem3[];
  const int li = threadIdx.x / TT;            // line in block
  const int t = threadIdx.x - li * TT;
  float2* const lbuf = smem3 + li * CF::LS;
  const SmLine<PD, TT> sm{lbuf};
  float2* const stash = lbuf + CF::SPN;
  const SymDev& S = a.sym;
  const LeafNode nd = a.nodes[blockIdx.y];
  // 32-bit line arithmetic: the launcher guarantees nrhs * lines < 2^31
  const unsigned lines = (unsigned)a.lines;
  const unsigned nr = (unsigned)a.nrhs;
  const unsigned gline = blockIdx.x * (unsigned)CF::LPB + (unsigned)li;   // over (line, rhs), rhs fastest
  const bool ok = gline < nr * lines;
  const unsigned line = ok ? gline / nr : 0u;
  const unsigned q = ok ? gline - line * nr : 0u;
  const long long base = (long long)q * a.rhs_stride + (long long)line * N + t;
  const long long cs = a.comp_stride;
  // the twiddle and phase tables are copied to shared memory, where every
  // use re-reads them (held in registers across the three components they
  // would cost about 60 registers)
  float2* const tws = smem3 + CF::LPB * CF::LS;
  float2* const phs = tws + N;
  {
    const float2* __restrict__ tw = (const float2*)a.fft.tw;
    const float2* __restrict__ ph = (const float2*)a.fft.ph;
    for (int e = threadIdx.x; e < N; e += CF::THREADS) {
      tws[e] = __ldg(&tw[e]);
      phs[e] = __ldg(&ph[e]);
    }
  }

  // symbol addressing of this line: split-grid frequency of each line dim,
  // its parity class and the fold to 2n - f of the compressed store
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
        fpre[m] = 2 * fpre[m] + ((nd.prefix >> m) & 1);
        clsp = (clsp << 1) | (fpre[m] & 1);
      }
#pragma unroll
    for (int m = 0; m < MAX_D - 1; ++m)
      if (m < dl) {
        int fm = fpre[m];
        if (fm > S.n[m]) { fm = 2 * S.n[m] - fm; foldp |= 1 << m; }
        lin = lin * (unsigned)S.J[clsp << 1][m] + (unsigned)(fm >> 1);
      }
  }
  const float2* __restrict__ Sd = (const float2*)S.data;
  const int cl0 = clsp << 1, cl1 = cl0 | 1;
  const float2* __restrict__ row0 = Sd + S.cls_off[cl0] + (long long)lin * S.J[cl0][dl];
  const float2* __restrict__ row1 = Sd + S.cls_off[cl1] + (long long)lin * S.J[cl1][dl];
  const unsigned blk0 = (unsigned)S.blk[cl0], blk1 = (unsigned)S.blk[cl1];
  // sign bit k: stored block k is read negated (without / with the fold of the last dim)
  unsigned sg0 = 0, sg1 = 0;
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    sg0 |= (unsigned)(__popc(S.oddmask[k] & foldp) & 1) << k;
    sg1 |= (unsigned)(__popc(S.oddmask[k] & (foldp | (1 << dl))) & 1) << k;
  }

  __syncthreads();                    // tables staged
  grid_dep_wait();                    // the nodes written by the previous kernel

  const float2* __restrict__ xin = (const float2*)nd.in + base;
  float2* __restrict__ yout = (float2*)nd.out + base;
#pragma unroll 1
  for (int b = 0; b < 2; ++b) {
    float2 w[3][R1];
#pragma unroll
    for (int c = 0; c < 3; ++c)
#pragma unroll
      for (int m = 0; m < R1; ++m) {
        const float2 v = ok ? xin[c * cs + TT * m] : make_float2(0.f, 0.f);
        w[c][m] = b ? cmul(v, phs[t + TT * m]) : v;
      }
#pragma unroll
    for (int c = 0; c < 3; ++c) fft_reg<P, false, SmLine<PD, TT>, true>(w[c], t, sm, tws);
    // c x c multiply at the thread's frequencies l = t + T m, f = 2l + b:
    // stored at l for l < N/2, else folded to index N - l - b with the signs
    // of the last dim's fold.  Stored blocks: 00 11 22 01 02 12.
    const float2* __restrict__ rw = b ? row1 : row0;
    const unsigned bk = b ? blk1 : blk0;
#pragma unroll
    for (int i = 0; i < R1; ++i) {
      const int m = !IL ? i : (i & 1) ? R1 - 1 - (i >> 1) : (i >> 1);
      const bool hi = m >= R1 / 2;
      const int idx = hi ? (N - b - t - TT * m) : (t + TT * m);
      const unsigned sg = hi ? sg1 : sg0;
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
    for (int c = 0; c < 3; ++c) fft_reg<P, true, SmLine<PD, TT>, true>(w[c], t, sm, tws);
    if (b == 0) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < R1; ++m) stash[c * N + t + TT * m] = w[c][m];
    } else if (ok) {
#pragma unroll
      for (int c = 0; c < 3; ++c)
#pragma unroll
        for (int m = 0; m < R1; ++m)
          yout[c * cs + TT * m] = cadd(stash[c * N + t + TT * m], cmulc(w[c][m], phs[t + TT * m]));
    }
  }
}

template <class P, int MB, bool IL>
static cudaError_t leaf3_p(const LeafArgs& a, cudaStream_t st) {
  typedef Leaf3Cfg<P, MB> CF;
  const long long total = (long long)a.nrhs * a.lines;
  const long long nt = (total + CF::LPB - 1) / CF::LPB;
  if (nt <= 0 || a.nnodes <= 0) return cudaSuccess;
  const size_t sm = CF::smem();
  const cudaError_t ae = set_smem_attr<k_leaf3<P, MB, IL>>((int)sm);
  if (ae != cudaSuccess) return ae;
  dim3 grid((unsigned)nt, (unsigned)a.nnodes);
#ifndef BTMV_NO_PDL
  return launch_pdl(k_leaf3<P, MB, IL>, grid, dim3(CF::THREADS), sm, st, a);
#else
  k_leaf3<P, MB, IL><<<grid, CF::THREADS, sm, st>>>(a);
  return cudaGetLastError();
#endif
}

// The split leaf of a c = 3 plan on the mirror-compressed, block-symmetric
// store (stored blocks 00 11 22 01 02 12), complex64, radix-16 line plans.
bool leaf3_supported(const LeafArgs& a, size_t esz) {
  if (esz != sizeof(float2) || a.c != 3 || !a.split) return false;
  const SymDev& S = a.sym;
  if (!S.compressed || S.nsym != 6 || S.n[a.dl] != a.N) return false;
  if (S.comp[0][0] != 0 || S.comp[1][1] != 1 || S.comp[2][2] != 2 || S.comp[0][1] != 3 || S.comp[0][2] != 4 ||
      S.comp[1][2] != 5 || S.comp[1][0] != 3 || S.comp[2][0] != 4 || S.comp[2][1] != 5)
    return false;
  if ((long long)a.nrhs * a.lines >= (1ll << 31)) return false;
  for (int c = 0; c < MAX_CLS; ++c)
    if (S.blk[c] >= (1ll << 31)) return false;                      // 32-bit block strides
  switch (a.N) {
    case 64: case 128: case 256: case 512: case 1024: return true;
  }
  return false;
}

// Two blocks of 128 threads per SM (255 registers, no spills): measured
// faster than three blocks with 168 registers and spills (115 against 159 us
// per launch at 128^3), low / folded-high symbol reads paired.
cudaError_t launch_leaf3(const LeafArgs& a, cudaStream_t st) {
  switch (a.N) {
    case 64: return leaf3_p<RP64, 2, true>(a, st);
    case 128: return leaf3_p<RP128, 2, true>(a, st);
    case 256: return leaf3_p<RP256, 2, true>(a, st);
    case 512: return leaf3_p<RP512, 2, true>(a, st);
    case 1024: return leaf3_p<RP1024, 2, true>(a, st);
  }
  return cudaErrorNotSupported;
}

}  // namespace btmv
