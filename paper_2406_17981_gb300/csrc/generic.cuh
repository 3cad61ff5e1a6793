// Generic line-pass device bodies (any 7-smooth length, complex64 and
// complex128), shared by the per-launch kernels (kernels.cu) and the
// persistent batched kernel (persistent.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "kernels.cuh"

namespace btmv {

static const size_t kMaxSmem = 227 * 1024;

static __host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

static __host__ __device__ inline size_t pass_hdr_bytes(int TL) {
  return align_up((size_t)TL * (4 * sizeof(long long) + sizeof(int)), 16);
}


// per line of a leaf tile: the split-grid frequencies of its d-1 line dims
// and a valid flag (last slot)
constexpr int FPS = MAX_D;

static __host__ __device__ inline size_t leaf_hdr_bytes(int Lt) {
  return align_up((size_t)Lt * FPS * sizeof(int), 16);
}


template <class T> __device__ __forceinline__ T czero() { T z; z.x = 0; z.y = 0; return z; }

// ----------------------------------------------------------------- k_pass
template <class T>
__device__ __forceinline__ void pass_load(T* __restrict__ d0, T* __restrict__ d1, const T* __restrict__ src,
                                          const ArrMap& m, const long long* __restrict__ off,
                                          const int* __restrict__ okl, const PassGeom& g, int ls, int es,
                                          const T* __restrict__ ph, bool tw0) {
  // d0 receives the line (times P when tw0), d1 (if non-null) receives P * line
  const int TL = g.TL, N = g.N;
  const int total = TL * N;
  const FDiv dN(N), dTL(TL);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int line, k;
    if (g.contig) { line = dN.div(e); k = e - line * N; }
    else          { k = dTL.div(e); line = e - k * TL; }
    T v = czero<T>();
    if ((okl[line] & 2) && k < m.len) v = src[off[line] + (long long)k * m.es];
    const int si = line * ls + k * es;
    if (d1) {
      d0[si] = v;
      d1[si] = cmul(v, __ldg(&ph[k]));
    } else {
      d0[si] = tw0 ? cmul(v, __ldg(&ph[k])) : v;
    }
  }
}

template <class T>
__device__ __forceinline__ void pass_store(T* __restrict__ dst, const T* __restrict__ r0,
                                           const T* __restrict__ r1, const ArrMap& m,
                                           const long long* __restrict__ off, const int* __restrict__ okl,
                                           const PassGeom& g, int ls, int es, const T* __restrict__ ph) {
  const int TL = g.TL, N = g.N;
  const int total = TL * N;
  const FDiv dN(N), dTL(TL);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    int line, k;
    if (g.contig) { line = dN.div(e); k = e - line * N; }
    else          { k = dTL.div(e); line = e - k * TL; }
    if (!(okl[line] & 1) || k >= m.len) continue;
    const int si = line * ls + k * es;
    T v = r0[si];
    if (r1) v = cadd(v, cmulc(r1[si], __ldg(&ph[k])));
    dst[off[line] + (long long)k * m.es] = v;
  }
}

template <class T, int MODE, bool LF>
__device__ __forceinline__ void pass_body(const PassArgs& a, unsigned char* smem, long long tile) {
  const PassGeom& g = a.g;
  const int TL = g.TL, N = g.N;
  const int ls = g.contig ? (N | 1) : 1;
  const int es = g.contig ? 1 : TL;
  const int bufsz = g.contig ? TL * ls : TL * N;
  long long* offs = (long long*)smem;         // [4][TL]
  int* okl = (int*)(offs + 4 * TL);           // [TL]
  T* B0 = (T*)(smem + pass_hdr_bytes(TL));
  T* B1 = B0 + bufsz;
  T* B2 = B1 + bufsz;                         // B2, B3: scratch of a two-half transform
  const T* ph = (const T*)a.fft.ph;
  // two halves (both children of a split, both inputs of a merge) are
  // transformed together as one tile of 2 TL lines in B0..B1: the second
  // half's lines follow the first's (line-major tiles) or interleave with
  // element stride 2 TL (line-fast tiles), so each Stockham stage serves
  // both halves and the number of dependent stages per tile is halved
  const int es2 = g.contig ? 1 : 2 * TL;
  const int h2 = g.contig ? TL * ls : TL;     // offset of the second half's line 0

  const long long tile0 = tile * TL;
  for (int l = threadIdx.x; l < TL; l += blockDim.x) {
    const long long gl = tile0 + l;
    int ok = gl < g.lines;
    long long o = 0;
    int ii[3] = {0, 0, 0};
    if (ok) {
      o = gl / g.Itot;
      long long r = gl - o * g.Itot;
      for (int j = g.ni - 1; j >= 0; --j) { ii[j] = (int)(r % g.I[j]); r /= g.I[j]; }
    }
    const ArrMap* ms[4] = {&a.a_in0, &a.a_in1, &a.a_out0, &a.a_out1};
    for (int q = 0; q < 4; ++q) {
      long long v = o * ms[q]->os;
      for (int j = 0; j < g.ni; ++j) v += (long long)ii[j] * ms[q]->is[j];
      offs[q * TL + l] = v;
    }
    int valid = ok;
    for (int j = 0; j < g.ni; ++j)
      if (ii[j] >= a.a_in0.vI[j]) valid = 0;
    okl[l] = ok | (valid << 1);
  }
  __syncthreads();

  if (MODE == 0) {
    const bool both = a.out0 && a.out1;
    if (both && g.halves == 2) {
      pass_load<T>(B0, B0 + h2, (const T*)a.in0, a.a_in0, offs, okl, g, ls, es2, ph, false);
      __syncthreads();
      T* r = fft_lines<false, LF>(B0, B2, 2 * TL, ls, es2, a.fft);
      pass_store<T>((T*)a.out0, r, nullptr, a.a_out0, offs + 2 * TL, okl, g, ls, es2, ph);
      pass_store<T>((T*)a.out1, r + h2, nullptr, a.a_out1, offs + 3 * TL, okl, g, ls, es2, ph);
    } else if (both) {
      // both children, one after the other (three tile buffers)
      pass_load<T>(B0, B1, (const T*)a.in0, a.a_in0, offs, okl, g, ls, es, ph, false);
      __syncthreads();
      T* r0 = fft_lines<false, LF>(B0, B2, TL, ls, es, a.fft);
      pass_store<T>((T*)a.out0, r0, nullptr, a.a_out0, offs + 2 * TL, okl, g, ls, es, ph);
      __syncthreads();
      T* r1 = fft_lines<false, LF>(B1, (r0 == B0) ? B2 : B0, TL, ls, es, a.fft);
      pass_store<T>((T*)a.out1, r1, nullptr, a.a_out1, offs + 3 * TL, okl, g, ls, es, ph);
    } else {
      const bool odd = a.out1 != nullptr;
      pass_load<T>(B0, nullptr, (const T*)a.in0, a.a_in0, offs, okl, g, ls, es, ph, odd);
      __syncthreads();
      T* r = fft_lines<false, LF>(B0, B1, TL, ls, es, a.fft);
      if (odd) pass_store<T>((T*)a.out1, r, nullptr, a.a_out1, offs + 3 * TL, okl, g, ls, es, ph);
      else     pass_store<T>((T*)a.out0, r, nullptr, a.a_out0, offs + 2 * TL, okl, g, ls, es, ph);
    }
  } else {
    const bool two = a.in1 != nullptr;
    if (two && g.halves == 2) {
      pass_load<T>(B0, nullptr, (const T*)a.in0, a.a_in0, offs, okl, g, ls, es2, ph, false);
      pass_load<T>(B0 + h2, nullptr, (const T*)a.in1, a.a_in1, offs + TL, okl, g, ls, es2, ph, false);
      __syncthreads();
      T* r = fft_lines<true, LF>(B0, B2, 2 * TL, ls, es2, a.fft);
      pass_store<T>((T*)a.out0, r, r + h2, a.a_out0, offs + 2 * TL, okl, g, ls, es2, ph);
    } else if (two) {
      // both inputs, one after the other (three tile buffers)
      pass_load<T>(B0, nullptr, (const T*)a.in0, a.a_in0, offs, okl, g, ls, es, ph, false);
      pass_load<T>(B1, nullptr, (const T*)a.in1, a.a_in1, offs + TL, okl, g, ls, es, ph, false);
      __syncthreads();
      T* r0 = fft_lines<true, LF>(B0, B2, TL, ls, es, a.fft);
      T* r1 = fft_lines<true, LF>(B1, (r0 == B0) ? B2 : B0, TL, ls, es, a.fft);
      pass_store<T>((T*)a.out0, r0, r1, a.a_out0, offs + 2 * TL, okl, g, ls, es, ph);
    } else {
      pass_load<T>(B0, nullptr, (const T*)a.in0, a.a_in0, offs, okl, g, ls, es, ph, false);
      __syncthreads();
      T* r0 = fft_lines<true, LF>(B0, B2, TL, ls, es, a.fft);
      pass_store<T>((T*)a.out0, r0, nullptr, a.a_out0, offs + 2 * TL, okl, g, ls, es, ph);
    }
  }
}

// ----------------------------------------------------------------- k_leaf
// Stored-symbol lookup: f = full-grid frequency per dim (f_m in [0, 2 n_m)).
__device__ __forceinline__ long long sym_index(const SymDev& S, const int* f, int& fold, int& cls) {
  cls = 0;
  fold = 0;
  for (int m = 0; m < S.d; ++m) cls = (cls << 1) | (f[m] & 1);
  long long lin = 0;
  for (int m = 0; m < S.d; ++m) {
    int fm = f[m];
    if (S.compressed && fm > S.n[m]) { fm = 2 * S.n[m] - fm; fold |= 1 << m; }
    lin = lin * S.J[cls][m] + (fm >> 1);
  }
  return S.cls_off[cls] + lin;
}

// c x c symbol multiply at every frequency of the tile, CUDA cores: each
// frequency's block is loaded once and applied to all rq right-hand sides.
template <class T>
__device__ __forceinline__ void leaf_multiply(T* __restrict__ R, const LeafArgs& a, int b,
                                              const int* __restrict__ fpre, int ls) {
  const int N = a.N, Lt = a.Lt, c = a.c, rq = a.rq;
  const int total = Lt * N;
  const T* __restrict__ S = (const T*)a.sym.data;
  const FDiv dN(N);
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int li = dN.div(e);
    const int l = e - li * N;
    if (fpre[li * FPS + FPS - 1] == 0) continue;   // line beyond the node
    int f[MAX_D];
    for (int m = 0; m < a.dl; ++m) f[m] = fpre[li * FPS + m];
    f[a.dl] = a.split ? 2 * l + b : l;
    int fold, cls;
    const long long base = sym_index(a.sym, f, fold, cls);
    const long long blk = a.sym.blk[cls];
    T sv[3][3];
    for (int ai = 0; ai < c; ++ai)
      for (int bi = 0; bi < c; ++bi) {
        const int kk = a.sym.comp[ai][bi];
        T s = __ldg(&S[base + kk * blk]);
        if (__popc(a.sym.oddmask[kk] & fold) & 1) { s.x = -s.x; s.y = -s.y; }
        sv[ai][bi] = s;
      }
    for (int q = 0; q < rq; ++q) {
      T x[3], y[3];
      for (int ai = 0; ai < c; ++ai) x[ai] = R[((q * c + ai) * Lt + li) * ls + l];
      for (int ai = 0; ai < c; ++ai) {
        T acc = czero<T>();
        for (int bi = 0; bi < c; ++bi) acc = cadd(acc, cmul(sv[ai][bi], x[bi]));
        y[ai] = acc;
      }
      for (int ai = 0; ai < c; ++ai) R[((q * c + ai) * Lt + li) * ls + l] = y[ai];
    }
  }
}

// The same multiply on tensor cores for c = 3 and complex64 (mma.sync
// m16n8k8, TF32 inputs, FP32 accumulation).  A warp takes two frequencies:
// their 3x3 complex blocks, written as real 6x6 blocks [[Re, -Im], [Im, Re]],
// sit block-diagonally in a 16x16 A tile; the columns of B are eight
// right-hand sides, rows the real and imaginary parts of the three
// components of both frequencies.  Each operand is split into a TF32 high
// part and a TF32 remainder and the product is formed as
// hi*hi + hi*lo + lo*hi, which keeps FP32-level accuracy.
__device__ __forceinline__ unsigned f2tf32(float x) {
  unsigned r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const unsigned (&a)[4], const unsigned (&b)[2]) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// element (row i, col j) of the real 6x6 block of a complex 3x3 matrix
__device__ __forceinline__ float real_block(const float2 (&s)[3][3], int i, int j) {
  const float2 v = s[i % 3][j % 3];
  if ((i < 3) == (j < 3)) return v.x;     // Re on the diagonal blocks
  return i < 3 ? -v.y : v.y;              // -Im upper right, Im lower left
}

__device__ __forceinline__ void leaf_multiply_tc(float2* __restrict__ R, const LeafArgs& a, int b,
                                                 const int* __restrict__ fpre, int ls) {
  const int N = a.N, Lt = a.Lt, rq = a.rq;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int g = lane >> 2, tq = lane & 3;
  const int nfreq = Lt * N;
  const int npair = (nfreq + 1) / 2;
  const float2* __restrict__ S = (const float2*)a.sym.data;
  for (int pr = warp; pr < npair; pr += nwarp) {
    // the two frequencies of this pair (the second may not exist)
    int fl[2], fli[2];
    bool fok[2];
    float2 sv[2][3][3];
    for (int h = 0; h < 2; ++h) {
      const int e = 2 * pr + h;
      fok[h] = e < nfreq;
      fl[h] = fok[h] ? e % N : 0;
      fli[h] = fok[h] ? e / N : 0;
      if (fok[h] && fpre[fli[h] * FPS + FPS - 1] == 0) fok[h] = false;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) sv[h][i][j] = make_float2(0.f, 0.f);
      if (!fok[h]) continue;
      int f[MAX_D];
      for (int m = 0; m < a.dl; ++m) f[m] = fpre[fli[h] * FPS + m];
      f[a.dl] = a.split ? 2 * fl[h] + b : fl[h];
      int fold, cls;
      const long long base = sym_index(a.sym, f, fold, cls);
      const long long blk = a.sym.blk[cls];
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
          const int kk = a.sym.comp[i][j];
          float2 v = __ldg(&S[base + kk * blk]);
          if (__popc(a.sym.oddmask[kk] & fold) & 1) { v.x = -v.x; v.y = -v.y; }
          sv[h][i][j] = v;
        }
    }
    // A fragments (two k-steps), split into TF32 high and low parts
    unsigned ahi[2][4], alo[2][4];
    for (int ks = 0; ks < 2; ++ks) {
      const int rows[4] = {g, g + 8, g, g + 8};
      const int cols[4] = {tq + 8 * ks, tq + 8 * ks, tq + 4 + 8 * ks, tq + 4 + 8 * ks};
      for (int u = 0; u < 4; ++u) {
        const int r = rows[u], k = cols[u];
        float v = 0.f;
        if (r < 12 && k < 12 && r / 6 == k / 6) v = real_block(sv[r / 6], r % 6, k % 6);
        ahi[ks][u] = f2tf32(v);
        alo[ks][u] = f2tf32(v - __uint_as_float(ahi[ks][u]));
      }
    }
    // element of B / D: row k -> frequency k / 6, component (k % 6) % 3, part (k % 6) / 3
    auto addr = [&](int k, int q) -> float* {
      const int h = k / 6, comp = (k % 6) % 3, part = (k % 6) / 3;
      float2* p = R + ((q * 3 + comp) * Lt + fli[h]) * ls + fl[h];
      return part ? &p->y : &p->x;
    };
    for (int q0 = 0; q0 < rq; q0 += 8) {
      const int qn = q0 + g;                       // this lane's B column / D column source
      unsigned bhi[2][2], blo[2][2];
      for (int ks = 0; ks < 2; ++ks)
        for (int u = 0; u < 2; ++u) {
          const int k = tq + 4 * u + 8 * ks;
          float v = 0.f;
          if (k < 12 && qn < rq && fok[k / 6]) v = *addr(k, qn);
          bhi[ks][u] = f2tf32(v);
          blo[ks][u] = f2tf32(v - __uint_as_float(bhi[ks][u]));
        }
      float d[4] = {0.f, 0.f, 0.f, 0.f};
      for (int ks = 0; ks < 2; ++ks) {
        mma_tf32(d, ahi[ks], bhi[ks]);
        mma_tf32(d, ahi[ks], blo[ks]);
        mma_tf32(d, alo[ks], bhi[ks]);
      }
      __syncwarp();                               // every lane has read its B values
      const int rows[4] = {g, g, g + 8, g + 8};
      const int colq[4] = {q0 + 2 * tq, q0 + 2 * tq + 1, q0 + 2 * tq, q0 + 2 * tq + 1};
      for (int u = 0; u < 4; ++u) {
        const int r = rows[u], q = colq[u];
        if (r < 12 && q < rq && fok[r / 6]) *addr(r, q) = d[u];
      }
      __syncwarp();
    }
  }
}

template <class T>
__device__ __forceinline__ void leaf_multiply_any(T* __restrict__ R, const LeafArgs& a, int b,
                                                  const int* __restrict__ fpre, int ls) {
  if constexpr (sizeof(T) == sizeof(float2)) {
    if (a.tensor && a.c == 3) { leaf_multiply_tc((float2*)R, a, b, fpre, ls); return; }
  }
  leaf_multiply<T>(R, a, b, fpre, ls);
}

template <class T>
__device__ __forceinline__ void leaf_body(const LeafArgs& a, unsigned char* smem, long long tile, int node) {
  const int N = a.N, c = a.c, rq = a.rq, Lt = a.Lt;
  const int NV = rq * c * Lt;
  const int ls = N | 1;
  const int bufsz = NV * ls;
  int* fpre = (int*)smem;                    // [Lt][FPS]: f of line dims, valid flag
  // X | B0: the odd half's lines (twiddled input), then the even half's; the
  // split leaf transforms both halves as one tile of 2 NV lines (each
  // Stockham stage serves both), with B1..B2 as scratch
  T* X = (T*)(smem + leaf_hdr_bytes(Lt));
  T* B0 = X + bufsz;
  T* B1 = B0 + bufsz;
  const T* ph = (const T*)a.fft.ph;

  const LeafNode nd = a.nodes[node];
  const long long nlt = (a.lines + Lt - 1) / Lt;
  const long long lt = tile % nlt;
  const int q0 = (int)(tile / nlt) * rq;
  const long long l0 = lt * Lt;

  for (int li = threadIdx.x; li < Lt; li += blockDim.x) {
    const long long gl = l0 + li;
    int ok = gl < a.lines;
    long long r = ok ? gl : 0;
    for (int m = a.dl - 1; m >= 0; --m) {
      const int im = (int)(r % a.ext[m]);
      r /= a.ext[m];
      fpre[li * FPS + m] = a.split ? 2 * im + ((nd.prefix >> m) & 1) : im;
    }
    fpre[li * FPS + FPS - 1] = ok;
  }
  __syncthreads();

  const T* __restrict__ in = (const T*)nd.in;
  const int totalv = NV * N;
  const FDiv dN(N), dLt(Lt), dc(c);
  for (int e = threadIdx.x; e < totalv; e += blockDim.x) {
    const int vl = dN.div(e);
    const int k = e - vl * N;
    const int qa = dLt.div(vl);
    const int li = vl - qa * Lt;
    const int qq = dc.div(qa);
    const int ai = qa - qq * c;
    const int q = q0 + qq;
    T v = czero<T>();
    if (fpre[li * FPS + FPS - 1] && q < a.nrhs)
      v = in[(long long)q * a.rhs_stride + (long long)ai * a.comp_stride + (l0 + li) * N + k];
    B0[vl * ls + k] = v;
    if (a.split) X[vl * ls + k] = cmul(v, __ldg(&ph[k]));
  }
  __syncthreads();

  T* A0;
  T* A1 = nullptr;
  if (a.split) {
    T* r = fft_lines<false, false>(X, B1, 2 * NV, ls, 1, a.fft);
    leaf_multiply_any<T>(r + bufsz, a, 0, fpre, ls);   // even half
    leaf_multiply_any<T>(r, a, 1, fpre, ls);           // odd half
    __syncthreads();
    A1 = fft_lines<true, false>(r, (r == X) ? B1 : X, 2 * NV, ls, 1, a.fft);
    A0 = A1 + bufsz;
  } else {
    // the whole 2n line (plain embedding)
    T* r = fft_lines<false, false>(B0, B1, NV, ls, 1, a.fft);
    leaf_multiply_any<T>(r, a, 0, fpre, ls);
    __syncthreads();
    A0 = fft_lines<true, false>(r, (r == B0) ? B1 : B0, NV, ls, 1, a.fft);
  }

  T* __restrict__ out = (T*)nd.out;
  for (int e = threadIdx.x; e < totalv; e += blockDim.x) {
    const int vl = dN.div(e);
    const int k = e - vl * N;
    const int qa = dLt.div(vl);
    const int li = vl - qa * Lt;
    const int qq = dc.div(qa);
    const int ai = qa - qq * c;
    const int q = q0 + qq;
    if (!fpre[li * FPS + FPS - 1] || q >= a.nrhs) continue;
    T v = A0[vl * ls + k];
    if (A1) v = cadd(v, cmulc(A1[vl * ls + k], __ldg(&ph[k])));
    out[(long long)q * a.rhs_stride + (long long)ai * a.comp_stride + (l0 + li) * N + k] = v;
  }
}

}  // namespace btmv
