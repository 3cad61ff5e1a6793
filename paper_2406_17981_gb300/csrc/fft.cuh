// Device FFT building blocks: complex helpers, radix 2/3/4/5/7/8/16
// butterflies and a self-sorting (Stockham) decimation-in-time stage loop
// over lines held in shared memory.
//
// Convention: forward DFT X[f] = sum_k x[k] exp(-2 pi i f k / N), inverse with
// the + sign, both unnormalised.  Butterfly constants are cos/sin of rational
// multiples of 2 pi, written out as decimal literals; stage twiddles come
// from per-size tables built on the host in double precision.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace btmv {

template <class R> struct cx;
template <> struct cx<float> { typedef float2 t; };
template <> struct cx<double> { typedef double2 t; };

__device__ __forceinline__ float2 mkc(float a, float b) { return make_float2(a, b); }
__device__ __forceinline__ double2 mkc(double a, double b) { return make_double2(a, b); }

template <class T> __device__ __forceinline__ T cadd(T a, T b) { T r; r.x = a.x + b.x; r.y = a.y + b.y; return r; }
template <class T> __device__ __forceinline__ T csub(T a, T b) { T r; r.x = a.x - b.x; r.y = a.y - b.y; return r; }
template <class T> __device__ __forceinline__ T cmul(T a, T b) {
  T r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
// a * conj(b)
template <class T> __device__ __forceinline__ T cmulc(T a, T b) {
  T r; r.x = a.x * b.x + a.y * b.y; r.y = a.y * b.x - a.x * b.y; return r;
}
template <class T, class S> __device__ __forceinline__ T cscale(T a, S s) { T r; r.x = a.x * s; r.y = a.y * s; return r; }
// multiply by -i (forward quarter turn) or +i (inverse)
template <bool INV, class T> __device__ __forceinline__ T rot90(T a) {
  T r;
  if (INV) { r.x = -a.y; r.y = a.x; } else { r.x = a.y; r.y = -a.x; }
  return r;
}
// twiddle multiply: a * w (forward) or a * conj(w) (inverse)
template <bool INV, class T> __device__ __forceinline__ T twm(T a, T w) { return INV ? cmulc(a, w) : cmul(a, w); }

template <class T> struct K {  // real scalar type of a complex type
  typedef float r;
};
template <> struct K<double2> { typedef double r; };

// ------------------------------------------------------------ radix kernels
template <bool INV, class T> __device__ __forceinline__ void dft2(T* a) {
  T t = a[0]; a[0] = cadd(t, a[1]); a[1] = csub(t, a[1]);
}

template <bool INV, class T> __device__ __forceinline__ void dft4(T& a0, T& a1, T& a2, T& a3) {
  T s0 = cadd(a0, a2), d0 = csub(a0, a2);
  T s1 = cadd(a1, a3), d1 = rot90<INV>(csub(a1, a3));
  a0 = cadd(s0, s1); a2 = csub(s0, s1);
  a1 = cadd(d0, d1); a3 = csub(d0, d1);
}
template <bool INV, class T> __device__ __forceinline__ void dft4(T* a) { dft4<INV>(a[0], a[1], a[2], a[3]); }

// exp(-+ i pi/4) * a
template <bool INV, class T> __device__ __forceinline__ T w8_1(T a) {
  typedef typename K<T>::r R;
  const R h = (R)0.7071067811865475244008;
  T r;
  if (INV) { r.x = (a.x - a.y) * h; r.y = (a.x + a.y) * h; }
  else     { r.x = (a.x + a.y) * h; r.y = (a.y - a.x) * h; }
  return r;
}
// exp(-+ 3 i pi/4) * a
template <bool INV, class T> __device__ __forceinline__ T w8_3(T a) {
  typedef typename K<T>::r R;
  const R h = (R)0.7071067811865475244008;
  T r;
  if (INV) { r.x = (-a.x - a.y) * h; r.y = (a.x - a.y) * h; }
  else     { r.x = (a.y - a.x) * h; r.y = (-a.x - a.y) * h; }
  return r;
}

template <bool INV, class T> __device__ __forceinline__ void dft8(T* a) {
  // X[k] = E[k] + w8^k O[k], X[k+4] = E[k] - w8^k O[k]
  T e0 = a[0], e1 = a[2], e2 = a[4], e3 = a[6];
  T o0 = a[1], o1 = a[3], o2 = a[5], o3 = a[7];
  dft4<INV>(e0, e1, e2, e3);
  dft4<INV>(o0, o1, o2, o3);
  o1 = w8_1<INV>(o1); o2 = rot90<INV>(o2); o3 = w8_3<INV>(o3);
  a[0] = cadd(e0, o0); a[4] = csub(e0, o0);
  a[1] = cadd(e1, o1); a[5] = csub(e1, o1);
  a[2] = cadd(e2, o2); a[6] = csub(e2, o2);
  a[3] = cadd(e3, o3); a[7] = csub(e3, o3);
}

template <bool INV, class T> __device__ __forceinline__ void dft16(T* a) {
  typedef typename K<T>::r R;
  const R c1 = (R)0.9238795325112867561282, s1 = (R)0.3826834323650897717285;
  // n = 4 n1 + n2, k = k1 + 4 k2:  inner DFT4 over n1, twiddle w16^{n2 k1}, outer DFT4 over n2
  T b[16];
#pragma unroll
  for (int n2 = 0; n2 < 4; ++n2) {
    T x0 = a[n2], x1 = a[4 + n2], x2 = a[8 + n2], x3 = a[12 + n2];
    dft4<INV>(x0, x1, x2, x3);
    b[n2 * 4 + 0] = x0; b[n2 * 4 + 1] = x1; b[n2 * 4 + 2] = x2; b[n2 * 4 + 3] = x3;
  }
  // twiddles w16^e for e = n2 * k1
  const T w1 = mkc(c1, INV ? s1 : -s1);       // e = 1
  const T w3 = mkc(s1, INV ? c1 : -c1);       // e = 3: cos(3pi/8) = sin(pi/8)
  const T w9 = mkc(-c1, INV ? -s1 : s1);      // e = 9 = 8 + 1: -w1
  b[1 * 4 + 1] = cmul(b[1 * 4 + 1], w1);
  b[1 * 4 + 2] = w8_1<INV>(b[1 * 4 + 2]);
  b[1 * 4 + 3] = cmul(b[1 * 4 + 3], w3);
  b[2 * 4 + 1] = w8_1<INV>(b[2 * 4 + 1]);
  b[2 * 4 + 2] = rot90<INV>(b[2 * 4 + 2]);
  b[2 * 4 + 3] = w8_3<INV>(b[2 * 4 + 3]);
  b[3 * 4 + 1] = cmul(b[3 * 4 + 1], w3);
  b[3 * 4 + 2] = w8_3<INV>(b[3 * 4 + 2]);
  b[3 * 4 + 3] = cmul(b[3 * 4 + 3], w9);
#pragma unroll
  for (int k1 = 0; k1 < 4; ++k1) {
    T x0 = b[k1], x1 = b[4 + k1], x2 = b[8 + k1], x3 = b[12 + k1];
    dft4<INV>(x0, x1, x2, x3);
    a[k1] = x0; a[k1 + 4] = x1; a[k1 + 8] = x2; a[k1 + 12] = x3;
  }
}

template <bool INV, class T> __device__ __forceinline__ void dft3(T* a) {
  typedef typename K<T>::r R;
  const R s = (R)0.8660254037844386467637;
  T t = cadd(a[1], a[2]);
  T u = csub(a[1], a[2]);
  T m; m.x = a[0].x - (R)0.5 * t.x; m.y = a[0].y - (R)0.5 * t.y;
  a[0] = cadd(a[0], t);
  // X1 = m -+ i s u, X2 = m +- i s u
  T v = rot90<INV>(cscale(u, s));
  a[1] = cadd(m, v);
  a[2] = csub(m, v);
}

// odd prime radix by pairing r and R - r: X_k = a0 + sum cos(th)(a_r + a_{R-r})
//   -+ i sum sin(th)(a_r - a_{R-r}),  th = 2 pi r k / R
template <int RAD> struct OddC;
template <> struct OddC<5> {
  __device__ static __forceinline__ double c(int m) {
    const double v[5] = {1.0, 0.3090169943749474241023, -0.8090169943749474241023,
                         -0.8090169943749474241023, 0.3090169943749474241023};
    return v[m];
  }
  __device__ static __forceinline__ double s(int m) {
    const double v[5] = {0.0, 0.9510565162951535721164, 0.5877852522924731291687,
                         -0.5877852522924731291687, -0.9510565162951535721164};
    return v[m];
  }
};
template <> struct OddC<7> {
  __device__ static __forceinline__ double c(int m) {
    const double v[7] = {1.0, 0.623489801858733530525, -0.2225209339563144042889,
                         -0.9009688679024191262361, -0.9009688679024191262361,
                         -0.2225209339563144042889, 0.623489801858733530525};
    return v[m];
  }
  __device__ static __forceinline__ double s(int m) {
    const double v[7] = {0.0, 0.7818314824680298087084, 0.9749279121818236070181,
                         0.4338837391175581204758, -0.4338837391175581204758,
                         -0.9749279121818236070181, -0.7818314824680298087084};
    return v[m];
  }
};

template <int RAD, bool INV, class T> __device__ __forceinline__ void dft_odd(T* a) {
  typedef typename K<T>::r R;
  constexpr int H = (RAD - 1) / 2;
  T sp[H], sm[H];
#pragma unroll
  for (int r = 1; r <= H; ++r) { sp[r - 1] = cadd(a[r], a[RAD - r]); sm[r - 1] = csub(a[r], a[RAD - r]); }
  T out[RAD];
  T x0 = a[0];
#pragma unroll
  for (int r = 0; r < H; ++r) x0 = cadd(x0, sp[r]);
  out[0] = x0;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    T re = a[0];
    T im; im.x = 0; im.y = 0;
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const int m = (r * k) % RAD;
      const R cc = (R)OddC<RAD>::c(m), ss = (R)OddC<RAD>::s(m);
      re.x += cc * sp[r - 1].x; re.y += cc * sp[r - 1].y;
      im.x += ss * sm[r - 1].x; im.y += ss * sm[r - 1].y;
    }
    T v = rot90<INV>(im);   // -i*im (forward) / +i*im (inverse)
    out[k] = cadd(re, v);
    out[RAD - k] = csub(re, v);
  }
#pragma unroll
  for (int r = 0; r < RAD; ++r) a[r] = out[r];
}

// cos and sin of 2 pi e / R evaluated at compile time: the angle is reduced
// to [-pi, pi] on the integer e, then summed by the Taylor series (20 terms,
// truncation below 1e-20 on that interval).
constexpr double kPiD = 3.141592653589793238462643383279502884;
constexpr double ct_angle(int e, int R) {
  e %= R;
  if (2 * e > R) e -= R;
  return 2.0 * kPiD * (double)e / (double)R;
}
constexpr double ct_sin2pi(int e, int R) {
  const double x = ct_angle(e, R), x2 = x * x;
  double term = x, sum = x;
  for (int k = 1; k <= 20; ++k) { term = -term * x2 / ((2.0 * k) * (2.0 * k + 1.0)); sum += term; }
  return sum;
}
constexpr double ct_cos2pi(int e, int R) {
  const double x = ct_angle(e, R), x2 = x * x;
  double term = 1.0, sum = 1.0;
  for (int k = 1; k <= 20; ++k) { term = -term * x2 / ((2.0 * k - 1.0) * (2.0 * k)); sum += term; }
  return sum;
}

template <int RAD, bool INV, class T> __device__ __forceinline__ void dft(T* a);

// DFT of size P*Q from P-point and Q-point DFTs (Cooley-Tukey): with
// n = Q n1 + n2 and k = k1 + P k2, inner DFT_P over n1, twiddle
// w_{PQ}^{n2 k1} (compile-time constants), outer DFT_Q over n2.
template <int P, int Q, bool INV, class T> __device__ __forceinline__ void dft_pq(T* a) {
  typedef typename K<T>::r R;
  constexpr int RR = P * Q;
  T b[RR];
#pragma unroll
  for (int n2 = 0; n2 < Q; ++n2) {
    T v[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) v[n1] = a[Q * n1 + n2];
    dft<P, INV>(v);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) {
      const int e = n2 * k1;
      if (e == 0) {
        b[n2 * P + k1] = v[k1];
      } else {
        const R c = (R)ct_cos2pi(e, RR), sn = (R)ct_sin2pi(e, RR);
        b[n2 * P + k1] = twm<INV>(v[k1], mkc(c, -sn));
      }
    }
  }
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) {
    T u[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) u[n2] = b[n2 * P + k1];
    dft<Q, INV>(u);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) a[k1 + P * k2] = u[k2];
  }
}

template <int RAD, bool INV, class T> __device__ __forceinline__ void dft(T* a) {
  if constexpr (RAD == 2) dft2<INV>(a);
  else if constexpr (RAD == 3) dft3<INV>(a);
  else if constexpr (RAD == 4) dft4<INV>(a);
  else if constexpr (RAD == 5) dft_odd<5, INV>(a);
  else if constexpr (RAD == 7) dft_odd<7, INV>(a);
  else if constexpr (RAD == 8) dft8<INV>(a);
  else if constexpr (RAD == 16) dft16<INV>(a);
  else if constexpr (RAD == 6) dft_pq<2, 3, INV>(a);
  else if constexpr (RAD == 12) dft_pq<4, 3, INV>(a);
  else if constexpr (RAD == 20) dft_pq<4, 5, INV>(a);
  else if constexpr (RAD == 24) dft_pq<8, 3, INV>(a);
  else if constexpr (RAD == 30) dft_pq<6, 5, INV>(a);
  else if constexpr (RAD == 42) dft_pq<6, 7, INV>(a);
  else if constexpr (RAD == 40) dft_pq<8, 5, INV>(a);
  else static_assert(RAD == 2, "radix not provided");
}

// Quotient x / d for 0 <= x < 2^22 through a float reciprocal: with inv the
// rounded 1/d, (x + 0.5) * inv lies within 2^-23 relative of x/d + 0.5/d,
// which is at least 0.5/d from the next integer, so truncation is exact.
struct FDiv {
  int d;
  float inv;
  __device__ __forceinline__ explicit FDiv(int d_) : d(d_), inv(1.0f / (float)d_) {}
  __device__ __forceinline__ int div(int x) const { return (int)(((float)x + 0.5f) * inv); }
};

// ------------------------------------------------------------ FFT plan
constexpr int MAX_STAGES = 12;

struct FftDev {
  int N;                 // transform length
  int nst;               // number of stages (0 when N == 1)
  int rad[MAX_STAGES];   // radix of each stage
  const void* tw;        // N entries: exp(-2 pi i k / N)
  const void* ph;        // N entries: exp(-i pi k / N)  (the split phase P)
};

// Smem line geometry: element k of line l is at base[l * ls + k * es].
//   LF == true : consecutive threads take consecutive lines (es = #lines, ls = 1)
//   LF == false: consecutive threads take consecutive butterflies of one line (es = 1)
template <int RAD, bool INV, bool LF, class T>
__device__ __forceinline__ void stage_smem(const T* __restrict__ src, T* __restrict__ dst, int nl, int ls,
                                           int es, int N, int L, const T* __restrict__ tw) {
  const int nb = N / RAD;      // butterflies per line
  const int mp = nb / L;       // N / (L * RAD)
  const int total = nl * nb;
  const FDiv dnl(nl), dnb(nb), dmp(mp);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    int line, j;
    if (LF) { j = dnl.div(idx); line = idx - j * nl; }
    else    { line = dnb.div(idx); j = idx - line * nb; }
    const int f1 = dmp.div(j);
    const T* s = src + line * ls;
    T* o = dst + line * ls;
    const int base = j + (RAD - 1) * mp * f1;
    T a[RAD];
#pragma unroll
    for (int r = 0; r < RAD; ++r) a[r] = s[(base + r * mp) * es];
    if (f1 > 0) {
#pragma unroll
      for (int r = 1; r < RAD; ++r) a[r] = twm<INV>(a[r], __ldg(&tw[r * f1 * mp]));
    }
    dft<RAD, INV>(a);
    const int ostep = mp * L;
#pragma unroll
    for (int f2 = 0; f2 < RAD; ++f2) o[(j + ostep * f2) * es] = a[f2];
  }
}

// Runs all stages on nl lines; data starts in buf0; returns the buffer that
// holds the result (buf0 or buf1).  Must be called by every thread of the block.
template <bool INV, bool LF, class T>
__device__ T* fft_lines(T* buf0, T* buf1, int nl, int ls, int es, const FftDev& P) {
  const T* tw = (const T*)P.tw;
  T* s = buf0;
  T* d = buf1;
  int L = 1;
  for (int st = 0; st < P.nst; ++st) {
    const int R = P.rad[st];
    switch (R) {
      case 2: stage_smem<2, INV, LF>(s, d, nl, ls, es, P.N, L, tw); break;
      case 3: stage_smem<3, INV, LF>(s, d, nl, ls, es, P.N, L, tw); break;
      case 4: stage_smem<4, INV, LF>(s, d, nl, ls, es, P.N, L, tw); break;
      case 5: stage_smem<5, INV, LF>(s, d, nl, ls, es, P.N, L, tw); break;
      case 7: stage_smem<7, INV, LF>(s, d, nl, ls, es, P.N, L, tw); break;
      case 8: stage_smem<8, INV, LF>(s, d, nl, ls, es, P.N, L, tw); break;
      default: stage_smem<16, INV, LF>(s, d, nl, ls, es, P.N, L, tw); break;
    }
    __syncthreads();
    T* t = s; s = d; d = t;
    L *= R;
  }
  return s;
}

}  // namespace btmv
