// C ABI of libbtmv: plans, the one-time FP64 symbol build, and the
// depth-first schedule of Algorithm 1 (split) or the plain full embedding.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "../../include/btmv.h"
#include "kernels.cuh"
#include "plan.h"

using namespace btmv;

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

btmv_status btmv::fail(btmv_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define CUDA_TRY(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(e_ == cudaErrorMemoryAllocation ? BTMV_E_NOMEM : BTMV_E_CUDA,          \
                  "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
  } while (0)

static bool factor_radices(int N, FftDev& f) { return factor_radices_mode(N, f, 0); }

bool btmv::factor_radices_mode(int N, FftDev& f, int mode) {
  f.N = N;
  f.nst = 0;
  int a = 0, m = N;
  while (m % 2 == 0) { m /= 2; ++a; }
  int c3 = 0, c5 = 0, c7 = 0;
  while (m % 3 == 0) { m /= 3; ++c3; }
  while (m % 5 == 0) { m /= 5; ++c5; }
  while (m % 7 == 0) { m /= 7; ++c7; }
  if (m != 1) return false;
  std::vector<int> r;
  if (mode == 1)
    while (a >= 3) { r.push_back(8); a -= 3; }
  while (a >= 4) {
    if (a == 5) { r.push_back(8); r.push_back(4); a = 0; break; }
    r.push_back(16);
    a -= 4;
  }
  if (a == 3) r.push_back(8);
  if (a == 2) r.push_back(4);
  if (a == 1) r.push_back(2);
  for (int i = 0; i < c7; ++i) r.push_back(7);
  for (int i = 0; i < c5; ++i) r.push_back(5);
  for (int i = 0; i < c3; ++i) r.push_back(3);
  if ((int)r.size() > MAX_STAGES) return false;
  for (size_t i = 0; i < r.size(); ++i) f.rad[i] = r[i];
  f.nst = (int)r.size();
  return true;
}

// exp(-2 pi i k / N) and exp(-i pi k / N) in extended precision, rounded once.
static void fill_tables(int N, std::vector<long double>& twc, std::vector<long double>& tws,
                        std::vector<long double>& phc, std::vector<long double>& phs) {
  const long double PI = 3.141592653589793238462643383279502884L;
  twc.resize(N); tws.resize(N); phc.resize(N); phs.resize(N);
  for (int k = 0; k < N; ++k) {
    const long double t = 2.0L * PI * (long double)k / (long double)N;
    twc[k] = cosl(t); tws[k] = -sinl(t);
    const long double p = PI * (long double)k / (long double)N;
    phc[k] = cosl(p); phs[k] = -sinl(p);
  }
}

static btmv_status build_tables(btmv_plan p, const std::vector<int>& Nf, const std::vector<int>& Nd) {
  std::map<int, int> uf, ud;
  for (int N : Nf) uf[N] = 1;
  for (int N : Nd) ud[N] = 1;
  size_t off = 0;
  for (auto& kv : uf) { p->tab.off_f[kv.first] = off; off += (size_t)2 * kv.first * sizeof(float2); off = (off + 255) / 256 * 256; }
  for (auto& kv : ud) { p->tab.off_d[kv.first] = off; off += (size_t)2 * kv.first * sizeof(double2); off = (off + 255) / 256 * 256; }
  p->tab.bytes = off;
  std::vector<unsigned char> host(off, 0);
  std::vector<long double> a, b, c, d;
  for (auto& kv : p->tab.off_f) {
    const int N = kv.first;
    fill_tables(N, a, b, c, d);
    float2* t = (float2*)(host.data() + kv.second);
    for (int k = 0; k < N; ++k) { t[k] = make_float2((float)a[k], (float)b[k]); t[N + k] = make_float2((float)c[k], (float)d[k]); }
  }
  for (auto& kv : p->tab.off_d) {
    const int N = kv.first;
    fill_tables(N, a, b, c, d);
    double2* t = (double2*)(host.data() + kv.second);
    for (int k = 0; k < N; ++k) { t[k] = make_double2((double)a[k], (double)b[k]); t[N + k] = make_double2((double)c[k], (double)d[k]); }
  }
  CUDA_TRY(cudaMalloc(&p->tab.mem, off));
  p->tab.owner = std::make_shared<DevBuf>(p->tab.mem);
  CUDA_TRY(cudaMemcpy(p->tab.mem, host.data(), off, cudaMemcpyHostToDevice));
  return BTMV_OK;
}

// complex128 transforms take radix-8-first plans: a radix-16 butterfly on
// double2 holds 32 registers of values plus as many temporaries per thread
static void set_fft(btmv_plan p, FftDev& f, int N, bool dbl) {
  factor_radices_mode(N, f, dbl ? 1 : 0);
  const size_t off = dbl ? p->tab.off_d[N] : p->tab.off_f[N];
  const size_t esz = dbl ? sizeof(double2) : sizeof(float2);
  f.tw = (const unsigned char*)p->tab.mem + off;
  f.ph = (const unsigned char*)p->tab.mem + off + (size_t)N * esz;
}

static void free_plan(btmv_plan p) {
  if (!p) return;
  cufft_plan_destroy(p);
  if (p->tma_err_host) cudaFreeHost(p->tma_err_host);
  for (auto& r : p->pending) { p->pool.push_back(r.a); p->pool.push_back(r.b); }
  for (auto e : p->pool) cudaEventDestroy(e);
  p->tab.owner.reset();       // freed with the last plan sharing them
  p->sym_owner.reset();
  if (p->ws) cudaFree(p->ws);
  if (p->ws2) cudaFree(p->ws2);
  if (p->side) cudaStreamDestroy(p->side);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->stage_x) cudaFree(p->stage_x);
  if (p->stage_y) cudaFree(p->stage_y);
  if (p->xpad) cudaFree(p->xpad);
  if (p->ypad) cudaFree(p->ypad);
  for (int s = 0; s < 2; ++s) {
    if (p->ring_x[s]) cudaFree(p->ring_x[s]);
    if (p->ring_y[s]) cudaFree(p->ring_y[s]);
    if (p->ev_in[s]) cudaEventDestroy(p->ev_in[s]);
    if (p->ev_comp[s]) cudaEventDestroy(p->ev_comp[s]);
    if (p->ev_out[s]) cudaEventDestroy(p->ev_out[s]);
  }
  if (p->cp_in) cudaStreamDestroy(p->cp_in);
  if (p->cp_out) cudaStreamDestroy(p->cp_out);
  delete p;
}

// BTMV_FLAG_TWO_STREAMS with d >= 3: a second set of d-2 workspace vectors
// for the second top-level subtree, a plan stream and fork / join events.
static btmv_status setup_two_streams(btmv_plan p, size_t V) {
  if (!(p->flags & BTMV_FLAG_TWO_STREAMS) || p->algo != BTMV_ALGO_SPLIT || p->d < 3) return BTMV_OK;
  const size_t n2 = (size_t)(p->d - 2);
  cudaError_t e = cudaMalloc(&p->ws2, n2 * V);
  if (e != cudaSuccess) return fail(BTMV_E_NOMEM, "plan: second-subtree workspace: %s", cudaGetErrorString(e));
  p->ws_bytes += n2 * V;
  p->W2.push_back(nullptr);                       // index m = 1..d-2 as in W
  for (size_t i = 0; i < n2; ++i) p->W2.push_back((unsigned char*)p->ws2 + i * V);
  if (cudaStreamCreateWithFlags(&p->side, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming) != cudaSuccess)
    return fail(BTMV_E_CUDA, "plan: side stream");
  return BTMV_OK;
}

// Smallest 7-smooth size >= n that the FFT plans take (<= 1024), or -1.
static int next_smooth(int n) {
  for (int m = n; m <= 1024; ++m) {
    FftDev f;
    if (factor_radices(m, f)) return m;
  }
  return -1;
}

// Padded plans: device copies of x and y at the padded sizes (V bytes each).
static btmv_status setup_padding(btmv_plan p, size_t V) {
  if (!p->padded) return BTMV_OK;
  if (cudaMalloc(&p->xpad, V) != cudaSuccess || cudaMalloc(&p->ypad, V) != cudaSuccess)
    return fail(BTMV_E_NOMEM, "plan: padded x and y of %zu bytes", V);
  p->ws_bytes += 2 * V;
  return BTMV_OK;
}

// The host-mapped error word of the TMA-staged passes.
static btmv_status setup_tma_error_word(btmv_plan p) {
  if (cudaHostAlloc((void**)&p->tma_err_host, sizeof(int), cudaHostAllocMapped) != cudaSuccess)
    return fail(BTMV_E_NOMEM, "plan: host-mapped error word");
  *p->tma_err_host = 0;
  if (cudaHostGetDevicePointer((void**)&p->tma_err_dev, p->tma_err_host, 0) != cudaSuccess)
    return fail(BTMV_E_CUDA, "plan: device address of the host-mapped error word");
  return BTMV_OK;
}

static void read_profile_every(btmv_plan p) {
  const char* v = getenv("BTMV_PROFILE_EVERY");
  p->prof_every = v && atoi(v) > 1 ? atoi(v) : 1;
}

extern "C" btmv_status btmv_plan_create(btmv_plan* out, int d, const int32_t* n, int c, int precision,
                                        int algo, int max_rhs, uint32_t flags) {
  g_err.clear();
  if (!out) return fail(BTMV_E_ARG, "plan_create: out is NULL");
  *out = nullptr;
  if (d < 1 || d > MAX_D) return fail(BTMV_E_ARG, "plan_create: d=%d outside [1,%d]", d, MAX_D);
  if (!n) return fail(BTMV_E_ARG, "plan_create: n is NULL");
  if (c < 1 || c > 3) return fail(BTMV_E_ARG, "plan_create: c=%d outside [1,3]", c);
  if (precision != BTMV_C64 && precision != BTMV_C128) return fail(BTMV_E_ARG, "plan_create: bad precision %d", precision);
  if (algo != BTMV_ALGO_SPLIT && algo != BTMV_ALGO_FULL && algo != BTMV_ALGO_FULL_CUFFT)
    return fail(BTMV_E_ARG, "plan_create: bad algo %d", algo);
  if (max_rhs < 1) return fail(BTMV_E_ARG, "plan_create: max_rhs=%d < 1", max_rhs);
  if (flags & ~(uint32_t)(BTMV_FLAG_PROFILE | BTMV_FLAG_GENERIC | BTMV_FLAG_SHARED_RHS | BTMV_FLAG_TENSOR_CORE |
                          BTMV_FLAG_TWO_STREAMS | BTMV_FLAG_FUSED_LEVELS))
    return fail(BTMV_E_ARG, "plan_create: unknown flags 0x%x", flags);
  if (algo == BTMV_ALGO_FULL && d > 4)
    return fail(BTMV_E_UNSUPPORTED, "plan_create: the plain embedding takes d <= 4 (d=%d)", d);
  if (algo == BTMV_ALGO_FULL_CUFFT && d > 3)
    return fail(BTMV_E_UNSUPPORTED, "plan_create: the cuFFT embedding takes d <= 3 (d=%d)", d);
  int np[MAX_D];
  for (int m = 0; m < d; ++m) {
    if (n[m] < 1) return fail(BTMV_E_ARG, "plan_create: n[%d]=%d < 1", m, n[m]);
    if (n[m] > 1024) return fail(BTMV_E_UNSUPPORTED, "plan_create: n[%d]=%d > 1024", m, n[m]);
    FftDev f;
    if (algo != BTMV_ALGO_SPLIT) {
      if (!factor_radices(2 * n[m], f))
        return fail(BTMV_E_UNSUPPORTED, "plan_create: the plain embedding needs 7-smooth sizes (n[%d]=%d)", m, n[m]);
      np[m] = n[m];
    } else {
      np[m] = next_smooth(n[m]);
      if (np[m] < 0)
        return fail(BTMV_E_UNSUPPORTED, "plan_create: no 7-smooth size <= 1024 at or above n[%d]=%d", m, n[m]);
    }
  }
  bool padded = false;
  for (int m = 0; m < d; ++m) padded = padded || np[m] != n[m];
  if (padded && d > 4) return fail(BTMV_E_UNSUPPORTED, "plan_create: sizes that are not 7-smooth need d <= 4");
  btmv_plan p = new btmv_plan_s();
  p->d = d; p->c = c; p->prec = precision; p->algo = algo; p->max_rhs = max_rhs; p->flags = flags;
  p->esz = precision == BTMV_C64 ? sizeof(float2) : sizeof(double2);
  p->padded = padded;
  for (int m = 0; m < d; ++m) {
    p->nu[m] = n[m]; p->su *= n[m];
    p->n[m] = np[m]; p->s *= np[m]; p->s2 *= 2 * np[m];
  }
  n = p->n;                        // the padded sizes from here on
  if (cudaGetDevice(&p->dev) != cudaSuccess) { free_plan(p); return fail(BTMV_E_CUDA, "plan_create: no CUDA device"); }
  cudaDeviceGetAttribute(&p->nsm, cudaDevAttrMultiProcessorCount, p->dev);

  std::vector<int> Nf, Nd;
  for (int m = 0; m < d; ++m) {
    const int N = algo != BTMV_ALGO_SPLIT ? 2 * n[m] : n[m];
    if (precision == BTMV_C64) Nf.push_back(N); else Nd.push_back(N);
    Nd.push_back(n[m]);  // FP64 symbol build
  }
  btmv_status st = build_tables(p, Nf, Nd);
  if (st != BTMV_OK) { free_plan(p); return st; }
  for (int m = 0; m < d; ++m) {
    const int N = algo != BTMV_ALGO_SPLIT ? 2 * n[m] : n[m];
    set_fft(p, p->fft_apply[m], N, precision == BTMV_C128);
    set_fft(p, p->fft_sym[m], n[m], true);
  }
  const size_t V = (size_t)max_rhs * c * p->s * p->esz;
  size_t nvec = 0;
  if (algo == BTMV_ALGO_SPLIT) nvec = (size_t)(d - 1);
  p->ws_bytes = algo == BTMV_ALGO_SPLIT ? nvec * V : (size_t)max_rhs * c * p->s2 * p->esz;
  if (p->ws_bytes) {
    cudaError_t e = cudaMalloc(&p->ws, p->ws_bytes);
    if (e != cudaSuccess) { free_plan(p); return fail(BTMV_E_NOMEM, "plan_create: workspace of %zu bytes: %s", p->ws_bytes, cudaGetErrorString(e)); }
    if (algo == BTMV_ALGO_SPLIT)
      for (size_t i = 0; i < nvec; ++i) p->W.push_back((unsigned char*)p->ws + i * V);
    else
      p->W.push_back(p->ws);
  }
  st = setup_two_streams(p, V);
  if (st != BTMV_OK) { free_plan(p); return st; }
  st = setup_padding(p, V);
  if (st != BTMV_OK) { free_plan(p); return st; }
  if (algo == BTMV_ALGO_FULL_CUFFT) {
    st = cufft_plan_setup(p);
    if (st != BTMV_OK) { free_plan(p); return st; }
  }
  st = setup_tma_error_word(p);
  if (st != BTMV_OK) { free_plan(p); return st; }
  read_profile_every(p);
  *out = p;
  return BTMV_OK;
}

extern "C" btmv_status btmv_plan_clone(btmv_plan src, int max_rhs, uint32_t flags, btmv_plan* out) {
  g_err.clear();
  if (!src || !out) return fail(BTMV_E_ARG, "plan_clone: NULL argument");
  *out = nullptr;
  if (max_rhs < 1) return fail(BTMV_E_ARG, "plan_clone: max_rhs=%d < 1", max_rhs);
  if (flags & ~(uint32_t)(BTMV_FLAG_PROFILE | BTMV_FLAG_GENERIC | BTMV_FLAG_SHARED_RHS | BTMV_FLAG_TENSOR_CORE |
                          BTMV_FLAG_TWO_STREAMS | BTMV_FLAG_FUSED_LEVELS))
    return fail(BTMV_E_ARG, "plan_clone: unknown flags 0x%x", flags);
  btmv_plan p = new btmv_plan_s();
  p->d = src->d; p->c = src->c; p->prec = src->prec; p->algo = src->algo; p->max_rhs = max_rhs; p->flags = flags;
  for (int m = 0; m < MAX_D; ++m) { p->n[m] = src->n[m]; p->fft_apply[m] = src->fft_apply[m]; p->fft_sym[m] = src->fft_sym[m]; }
  p->s = src->s; p->s2 = src->s2; p->esz = src->esz; p->dev = src->dev; p->nsm = src->nsm;
  for (int m = 0; m < MAX_D; ++m) p->nu[m] = src->nu[m];
  p->su = src->su; p->padded = src->padded;
  p->tab = src->tab;                                  // shared twiddle tables
  p->sym = src->sym; p->sym_owner = src->sym_owner;   // shared symbol store
  p->sym_bytes = src->sym_bytes; p->symdev = src->symdev; p->has_sym = src->has_sym;
  p->nsym = src->nsym; p->compressed = src->compressed;
  const size_t V = (size_t)max_rhs * p->c * p->s * p->esz;
  const size_t nvec = p->algo == BTMV_ALGO_SPLIT ? (size_t)(p->d - 1) : 0;
  p->ws_bytes = p->algo == BTMV_ALGO_SPLIT ? nvec * V : (size_t)max_rhs * p->c * p->s2 * p->esz;
  if (p->ws_bytes) {
    cudaError_t e = cudaMalloc(&p->ws, p->ws_bytes);
    if (e != cudaSuccess) { free_plan(p); return fail(BTMV_E_NOMEM, "plan_clone: workspace of %zu bytes: %s", p->ws_bytes, cudaGetErrorString(e)); }
    if (p->algo == BTMV_ALGO_SPLIT)
      for (size_t i = 0; i < nvec; ++i) p->W.push_back((unsigned char*)p->ws + i * V);
    else
      p->W.push_back(p->ws);
  }
  {
    btmv_status st = setup_padding(p, V);
    if (st != BTMV_OK) { free_plan(p); return st; }
    if (p->algo == BTMV_ALGO_FULL_CUFFT) {
      st = cufft_plan_setup(p);
      if (st != BTMV_OK) { free_plan(p); return st; }
    }
    st = setup_tma_error_word(p);
    if (st != BTMV_OK) { free_plan(p); return st; }
  }
  read_profile_every(p);
  *out = p;
  return BTMV_OK;
}

// --------------------------------------------------------- symbol build
static int block_index(int c, bool bsym, int a, int b) {
  if (!bsym) return a * c + b;
  if (a == b) return a;
  if (a > b) { int t = a; a = b; b = t; }
  // upper triangle after the c diagonal blocks, row-major
  int k = c;
  for (int i = 0; i < c; ++i)
    for (int j = i + 1; j < c; ++j) {
      if (i == a && j == b) return k;
      ++k;
    }
  return -1;
}

// Generator of the conjugate transpose: T^H has blocks (T^H)_ab[i - j] =
// conj(T_ba[j - i]), i.e. t^H_ab[p] = conj(t_ba[-p]).  Full layout: the
// offset index p_m + n_m - 1 becomes (n_m - 1) - p_m (reversed along every
// dim).  Orthant layout with parity: t_ba[-p] = (prod_m parity_ba[m]) t_ba[p]
// for p >= 0, and t^H_ab has the parity of t_ba.  With block symmetry only
// blocks a <= b of t are read, t_ba = t_ab.
static void adjoint_generator(btmv_plan p, const double* t, const int8_t* parity, bool bsym,
                              std::vector<double>& out, std::vector<int8_t>& par_out) {
  const int d = p->d, c = p->c;
  long long tb = 1;
  int ext[MAX_D];
  for (int m = 0; m < d; ++m) { ext[m] = parity ? p->nu[m] : 2 * p->nu[m] - 1; tb *= ext[m]; }
  out.assign((size_t)c * c * tb * 2, 0.0);
  if (parity) par_out.assign((size_t)c * c * d, 1);
  for (int a = 0; a < c; ++a)
    for (int b = 0; b < c; ++b) {
      const int sa = bsym ? std::min(a, b) : b, sb = bsym ? std::max(a, b) : a;   // source block (b, a)
      const double* src = t + ((size_t)sa * c + sb) * tb * 2;
      double* dst = out.data() + ((size_t)a * c + b) * tb * 2;
      double sign = 1.0;
      if (parity)
        for (int m = 0; m < d; ++m) {
          const int8_t v = parity[((size_t)b * c + a) * d + m];
          par_out[((size_t)a * c + b) * d + m] = v;
          sign *= v;
        }
      for (long long i = 0; i < tb; ++i) {
        long long j = i;
        if (!parity) {           // reversed multi-index
          long long r = i, acc = 0, stride = 1;
          for (int m = d - 1; m >= 0; --m) {
            const long long im = r % ext[m];
            r /= ext[m];
            acc += (ext[m] - 1 - im) * stride;
            stride *= ext[m];
          }
          j = acc;
        }
        dst[2 * i] = sign * src[2 * j];
        dst[2 * i + 1] = -sign * src[2 * j + 1];
      }
    }
}

// Padded plans: the generator given at the caller's sizes nu, zero outside
// them, laid out at the padded sizes n (full layout: offset p_m at
// p_m + n_m - 1; orthant layout: p_m >= 0).  The padded operator restricted
// to the first nu_m points of every level is the caller's operator.
static void pad_generator(btmv_plan p, const double* t, bool orthant, std::vector<double>& out) {
  const int d = p->d, c = p->c;
  int eu[MAX_D], ep[MAX_D], sh[MAX_D];
  long long tu = 1, tp = 1;
  for (int m = 0; m < d; ++m) {
    eu[m] = orthant ? p->nu[m] : 2 * p->nu[m] - 1;
    ep[m] = orthant ? p->n[m] : 2 * p->n[m] - 1;
    sh[m] = orthant ? 0 : p->n[m] - p->nu[m];      // offset index shift
    tu *= eu[m];
    tp *= ep[m];
  }
  out.assign((size_t)c * c * tp * 2, 0.0);
  for (int blk = 0; blk < c * c; ++blk)
    for (long long i = 0; i < tu; ++i) {
      long long r = i, j = 0, stride = 1;
      for (int m = d - 1; m >= 0; --m) {
        const long long im = r % eu[m];
        r /= eu[m];
        j += (im + sh[m]) * stride;
        stride *= ep[m];
      }
      out[((size_t)blk * tp + j) * 2] = t[((size_t)blk * tu + i) * 2];
      out[((size_t)blk * tp + j) * 2 + 1] = t[((size_t)blk * tu + i) * 2 + 1];
    }
}

extern "C" btmv_status btmv_set_kernel(btmv_plan p, const double* t, uint32_t sym_flags, const int8_t* parity,
                                       void* stream) {
  g_err.clear();
  if (!p) return fail(BTMV_E_ARG, "set_kernel: plan is NULL");
  if (!t) return fail(BTMV_E_ARG, "set_kernel: t is NULL");
  if (sym_flags & ~(uint32_t)(BTMV_SYM_BLOCK | BTMV_SYM_PARITY | BTMV_SYM_ADJOINT))
    return fail(BTMV_E_ARG, "set_kernel: unknown sym flags 0x%x", sym_flags);
  const bool bsym = (sym_flags & BTMV_SYM_BLOCK) != 0;
  const bool par = (sym_flags & BTMV_SYM_PARITY) != 0;
  const int d = p->d, c = p->c;
  if (par && !parity) return fail(BTMV_E_ARG, "set_kernel: BTMV_SYM_PARITY needs a parity array");
  // BTMV_SYM_ADJOINT: replace (t, parity) by the generator of T^H on the host
  std::vector<double> t_adj;
  std::vector<int8_t> par_adj;
  if (sym_flags & BTMV_SYM_ADJOINT) {
    adjoint_generator(p, t, par ? parity : nullptr, bsym, t_adj, par_adj);
    t = t_adj.data();
    if (par) parity = par_adj.data();
  }
  std::vector<double> t_pad;
  if (p->padded) {
    pad_generator(p, t, par, t_pad);
    t = t_pad.data();
  }
  if (par) {
    for (int a = 0; a < c; ++a)
      for (int b = 0; b < c; ++b)
        for (int m = 0; m < d; ++m) {
          const int8_t v = parity[(a * c + b) * d + m];
          if (v != 1 && v != -1) return fail(BTMV_E_ARG, "set_kernel: parity[%d][%d][%d]=%d not +-1", a, b, m, v);
          if (bsym && v != parity[(b * c + a) * d + m]) return fail(BTMV_E_ARG, "set_kernel: BTMV_SYM_BLOCK with asymmetric parity");
        }
  }
  cudaStream_t st = (cudaStream_t)stream;
  const int nsym = bsym ? c * (c + 1) / 2 : c * c;
  // the mirror-compressed store serves both algorithms: the plain embedding's
  // leaf reads its full-grid frequencies f_m in [0, 2 n_m) folded to 2 n_m - f_m
  const int compressed = par ? 1 : 0;

  // class geometry
  SymDev sd;
  memset(&sd, 0, sizeof sd);
  sd.d = d; sd.nsym = nsym; sd.compressed = compressed;
  for (int m = 0; m < d; ++m) sd.n[m] = p->n[m];
  long long off = 0;
  const int ncls = 1 << d;
  for (int cls = 0; cls < ncls; ++cls) {
    long long blk = 1;
    for (int m = 0; m < d; ++m) {
      const int bm = (cls >> (d - 1 - m)) & 1;
      const int J = compressed ? (p->n[m] - bm) / 2 + 1 : p->n[m];
      sd.J[cls][m] = J;
      blk *= J;
    }
    sd.cls_off[cls] = off;
    sd.blk[cls] = blk;
    off += blk * nsym;
  }
  const size_t store_bytes = (size_t)off * p->esz;
  int pairs[9][2];
  for (int a = 0; a < c; ++a)
    for (int b = 0; b < c; ++b) {
      const int k = block_index(c, bsym, a, b);
      sd.comp[a][b] = k;
      if (!bsym || a <= b) { pairs[k][0] = a; pairs[k][1] = b; }
    }
  for (int k = 0; k < nsym; ++k) {
    int mask = 0;
    if (par)
      for (int m = 0; m < d; ++m)
        if (parity[(pairs[k][0] * c + pairs[k][1]) * d + m] < 0) mask |= 1 << m;
    sd.oddmask[k] = mask;
  }

  // device copy of t (only the needed blocks are used)
  long long tb = 1;
  for (int m = 0; m < d; ++m) tb *= par ? p->n[m] : (2 * p->n[m] - 1);
  const size_t t_bytes = (size_t)c * c * tb * sizeof(double2);
  void* t_dev = nullptr;
  void* F = nullptr;
  // reuse this plan's own store when it has the right size; a store shared
  // with clones is left to them and a new one is built
  void* store = (p->sym && p->sym_bytes == store_bytes && p->sym_owner.use_count() == 1) ? p->sym : nullptr;
  cudaError_t e = cudaMalloc(&t_dev, t_bytes);
  if (e != cudaSuccess) return fail(BTMV_E_NOMEM, "set_kernel: %zu bytes for t: %s", t_bytes, cudaGetErrorString(e));
  e = cudaMalloc(&F, (size_t)nsym * p->s * sizeof(double2));
  if (e != cudaSuccess) { cudaFree(t_dev); return fail(BTMV_E_NOMEM, "set_kernel: FP64 work buffer: %s", cudaGetErrorString(e)); }
  if (!store) {
    e = cudaMalloc(&store, store_bytes);
    if (e != cudaSuccess) { cudaFree(t_dev); cudaFree(F); return fail(BTMV_E_NOMEM, "set_kernel: symbol store of %zu bytes: %s", store_bytes, cudaGetErrorString(e)); }
  }
  btmv_status ret = BTMV_OK;
  auto bail = [&](btmv_status s2, const char* what, cudaError_t ce) {
    ret = fail(s2, "set_kernel: %s: %s", what, cudaGetErrorString(ce));
  };
  e = cudaMemcpyAsync(t_dev, t, t_bytes, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) bail(BTMV_E_CUDA, "copy of t", e);

  FoldArgs fa;
  memset(&fa, 0, sizeof fa);
  fa.F = (double2*)F; fa.t = (const double2*)t_dev; fa.d = d; fa.c = c; fa.nsym = nsym;
  fa.parity_layout = par ? 1 : 0; fa.s = p->s;
  double scale = 1.0;
  for (int m = 0; m < d; ++m) { fa.n[m] = p->n[m]; scale /= (2.0 * p->n[m]); }
  fa.scale = scale;
  for (int k = 0; k < nsym; ++k) { fa.pairs[k][0] = pairs[k][0]; fa.pairs[k][1] = pairs[k][1]; }
  if (par)
    for (int a = 0; a < c; ++a)
      for (int b = 0; b < c; ++b)
        for (int m = 0; m < d; ++m) fa.par[a][b][m] = parity[(a * c + b) * d + m];

  for (int cls = 0; cls < ncls && ret == BTMV_OK; ++cls) {
    for (int m = 0; m < d; ++m) fa.cls_bits[m] = (cls >> (d - 1 - m)) & 1;
    if ((e = launch_fold(fa, st)) != cudaSuccess) { bail(BTMV_E_CUDA, "fold kernel", e); break; }
    // FP64 forward transforms along every dim, P_{b_m}-twiddled, in place
    for (int m = 0; m < d && ret == BTMV_OK; ++m) {
      long long outer = nsym, inner = 1;
      for (int q = 0; q < m; ++q) outer *= p->n[q];
      for (int q = m + 1; q < d; ++q) inner *= p->n[q];
      PassArgs pa;
      memset(&pa, 0, sizeof pa);
      const int N = p->n[m];
      pa.g.N = N; pa.g.ni = inner > 1 ? 1 : 0; pa.g.I[0] = (int)inner; pa.g.Itot = inner;
      pa.g.lines = outer * inner; pa.g.contig = inner == 1;
      int TL = pa.g.contig ? std::max(1, std::min(64, 2048 / N)) : 16;
      pa.g.TL = TL;
      while (TL > 1 && pass_smem_bytes(pa.g, sizeof(double2)) > 96 * 1024) { TL /= 2; pa.g.TL = TL; }
      ArrMap am;
      memset(&am, 0, sizeof am);
      am.os = (long long)N * inner; am.is[0] = 1; am.es = inner; am.vI[0] = am.vI[1] = am.vI[2] = 1 << 30; am.len = N;
      pa.a_in0 = pa.a_in1 = pa.a_out0 = pa.a_out1 = am;
      pa.in0 = F;
      if (fa.cls_bits[m]) pa.out1 = F; else pa.out0 = F;
      pa.fft = p->fft_sym[m];
      if ((e = launch_pass<double2>(0, pa, st)) != cudaSuccess) bail(BTMV_E_CUDA, "FP64 symbol pass", e);
    }
    if (ret != BTMV_OK) break;
    StoreArgs sa;
    memset(&sa, 0, sizeof sa);
    sa.store = store; sa.F = (const double2*)F; sa.d = d; sa.nsym = nsym; sa.prec = p->prec == BTMV_C128 ? 1 : 0;
    for (int m = 0; m < d; ++m) { sa.n[m] = p->n[m]; sa.J[m] = sd.J[cls][m]; }
    sa.s = p->s; sa.cls_off = sd.cls_off[cls]; sa.blk = sd.blk[cls];
    if ((e = launch_store(sa, st)) != cudaSuccess) bail(BTMV_E_CUDA, "store kernel", e);
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess && ret == BTMV_OK) bail(BTMV_E_CUDA, "symbol build", e);
  cudaFree(t_dev);
  cudaFree(F);
  if (ret != BTMV_OK) {
    if (store != p->sym) cudaFree(store);
    return ret;
  }
  if (store != p->sym) {
    p->sym_owner = std::make_shared<DevBuf>(store);
    p->sym = store;
  }
  p->sym_bytes = store_bytes;
  sd.data = store;
  p->symdev = sd;
  p->nsym = nsym;
  p->compressed = compressed;
  p->has_sym = true;
  return BTMV_OK;
}

// ------------------------------------------------------------ profiling
static cudaEvent_t get_event(btmv_plan p) {
  if (!p->pool.empty()) { cudaEvent_t e = p->pool.back(); p->pool.pop_back(); return e; }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

static void drain_profile(btmv_plan p) {
  for (auto& r : p->pending) {
    cudaEventSynchronize(r.b);
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, r.a, r.b) == cudaSuccess) { p->acc_ms[r.kind] += ms; p->acc_n[r.kind] += 1; }
    p->pool.push_back(r.a);
    p->pool.push_back(r.b);
  }
  p->pending.clear();
}

struct ProfScope {
  btmv_plan p;
  int kind;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  ProfScope(btmv_plan p_, int k, cudaStream_t s) : p(p_), kind(k), st(s) {
    if (p->prof_on) { a = get_event(p); cudaEventRecord(a, st); }
    p->launches++;
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = get_event(p);
      cudaEventRecord(b, st);
      p->pending.push_back({kind, a, b});
      if (p->pending.size() > 65536) drain_profile(p);
    }
  }
};

// ------------------------------------------------------------ schedule
static ArrMap contig_map(long long N, long long inner) {
  ArrMap am;
  memset(&am, 0, sizeof am);
  am.os = N * inner; am.is[0] = 1; am.es = inner;
  am.vI[0] = am.vI[1] = am.vI[2] = 1 << 30;
  am.len = (int)N;
  return am;
}

// Tile of lines for the generic pass: as many lines as fit 64 KB of shared
// memory (at most 16 strided / 2048 points contiguous), then fewer while the
// launch would have fewer than two blocks per SM.
static void choose_tile(PassGeom& g, size_t esz) {
  int TL = g.contig ? std::max(1, std::min(64, 2048 / g.N)) : 16;
  g.TL = TL;
  while (TL > 1 && pass_smem_bytes(g, esz) > 64 * 1024) { TL /= 2; g.TL = TL; }
  while (TL > 1 && (g.lines + TL - 1) / TL < 2 * 152) { TL /= 2; g.TL = TL; }
}

// Register-resident kernels where the geometry allows, else the generic
// shared-memory kernels (or always the generic ones with BTMV_FLAG_GENERIC).
// The TMA-staged passes (fast_pass_tma.cu) take the merge of 256-point lines,
// where they measured faster than the register passes (256^3: 201 against
// 216 us).  The 128-point forward split was faster with one right-hand side
// (28.7 against 29.8 us) but slower with sixteen (128^3 r16: 2822 against
// 2953 rhs-matvecs/s over the apply), and the other cases slower, so the
// register passes keep them.  BTMV_PASS_TMA=0 / 1 in the environment turns
// the TMA passes off / on for every pass they can take (comparisons).
static bool use_pass_tma(int mode, const PassArgs& pa) {
  const char* v = getenv("BTMV_PASS_TMA");
  if (v && v[0] == '0') return false;
  if (v && v[0] == '1') return true;
  return mode == 1 && pa.g.N == 256;
}

template <class T>
static cudaError_t run_pass(btmv_plan p, int mode, const PassArgs& pa, cudaStream_t st) {
  if (!(p->flags & BTMV_FLAG_GENERIC) && pass_reg_supported(pa, sizeof(T))) {
    if (p->tma_err_dev && use_pass_tma(mode, pa) && pass_tma_supported(mode, pa, sizeof(T)))
      return launch_pass_tma(mode, pa, p->tma_err_dev, st);
    return launch_pass_reg(mode, pa, st);
  }
  return launch_pass<T>(mode, pa, st);
}

PassArgs btmv::split_pass_args(btmv_plan p, const Step& stp, int nrhs, size_t esz, int TL) {
  const int m = stp.dim;
  long long outer = (long long)nrhs * p->c, inner = 1;
  for (int q = 0; q < m; ++q) outer *= p->n[q];
  for (int q = m + 1; q < p->d; ++q) inner *= p->n[q];
  PassArgs pa;
  memset(&pa, 0, sizeof pa);
  const int N = p->n[m];
  pa.g.N = N; pa.g.ni = inner > 1 ? 1 : 0; pa.g.I[0] = (int)inner; pa.g.Itot = inner;
  pa.g.lines = outer * inner; pa.g.contig = inner == 1;
  pa.g.halves = ((stp.kind == 0 && stp.out0 && stp.out1) || (stp.kind == 1 && stp.in1)) ? 2 : 1;
  choose_tile(pa.g, esz);
  if (TL > 0) {
    pa.g.TL = TL;
    while (pa.g.TL > 1 && pass_smem_bytes(pa.g, esz) > 96 * 1024) pa.g.TL /= 2;
  }
  pa.a_in0 = pa.a_in1 = pa.a_out0 = pa.a_out1 = contig_map(N, inner);
  pa.in0 = stp.in0; pa.in1 = stp.in1; pa.out0 = stp.out0; pa.out1 = stp.out1;
  pa.fft = p->fft_apply[m];
  return pa;
}

template <class T>
static btmv_status split_pass(btmv_plan p, const Step& stp, int nrhs, cudaStream_t st) {
  const int mode = stp.kind;
  if (p->tma_err_host && *(volatile int*)p->tma_err_host) {
    *(volatile int*)p->tma_err_host = 0;
    return fail(BTMV_E_TIMEOUT, "split pass: a bounded wait for a TMA tile expired in an earlier launch");
  }
  PassArgs pa = split_pass_args(p, stp, nrhs, sizeof(T), 0);
  ProfScope ps(p, mode == 0 ? BTMV_K_FWD_SPLIT : BTMV_K_MERGE, st);
  cudaError_t e = run_pass<T>(p, mode, pa, st);
  if (e != cudaSuccess) return fail(BTMV_E_CUDA, "split pass (dim %d, mode %d): %s", stp.dim, mode, cudaGetErrorString(e));
  return BTMV_OK;
}

static void leaf_tiling(int N, int c, int nrhs, size_t esz, int& rq, int& Lt) {
  rq = 1;
  const size_t per = 3 * (size_t)c * (size_t)(N | 1) * esz;  // smem per (rhs, line)
  Lt = (int)std::max<size_t>(1, (48 * 1024) / per);
  if (Lt > 16) Lt = 16;
  (void)nrhs;
}

LeafArgs btmv::leaf_step_args(btmv_plan p, int nrhs, int nn, const LeafNode* nodes, bool full, size_t esz, int Lt,
                              int rq) {
  LeafArgs la;
  memset(&la, 0, sizeof la);
  const int d = p->d;
  la.N = full ? 2 * p->n[d - 1] : p->n[d - 1];
  la.c = p->c;
  la.nrhs = nrhs;
  la.dl = d - 1;
  la.lines = 1;
  for (int m = 0; m < d - 1; ++m) { la.ext[m] = full ? 2 * p->n[m] : p->n[m]; la.lines *= la.ext[m]; }
  la.comp_stride = full ? p->s2 : p->s;
  la.rhs_stride = la.comp_stride * p->c;
  la.split = full ? 0 : 1;
  leaf_tiling(la.N, la.c, nrhs, esz, la.rq, la.Lt);
  // enough blocks for small problems: at least two per SM over the nodes
  while (la.Lt > 1 && ((la.lines + la.Lt - 1) / la.Lt) * nrhs * nn < 2 * 152) la.Lt /= 2;
  if (rq > 0) la.rq = std::min(rq, std::max(1, nrhs));
  if (Lt > 0) la.Lt = Lt;
  while ((la.Lt > 1 || la.rq > 1) && leaf_smem_bytes(la.N, la.c, la.rq, la.Lt, esz) > 96 * 1024) {
    if (la.Lt > 1) la.Lt /= 2; else la.rq = (la.rq + 1) / 2;
  }
  const long long nlt = (la.lines + la.Lt - 1) / la.Lt;
  const long long nrc = (nrhs + la.rq - 1) / la.rq;
  la.tiles_per_node = nlt * nrc;
  la.nnodes = nn;
  for (int i = 0; i < nn; ++i) la.nodes[i] = nodes[i];
  la.fft = p->fft_apply[d - 1];
  la.sym = p->symdev;
  return la;
}

template <class T>
static btmv_status leaf_launch(btmv_plan p, int nrhs, int nn, const LeafNode* nodes, bool full,
                               cudaStream_t st) {
  const bool shared = (p->flags & (BTMV_FLAG_SHARED_RHS | BTMV_FLAG_TENSOR_CORE)) && nrhs > 1;
  LeafArgs la = leaf_step_args(p, nrhs, nn, nodes, full, sizeof(T), 0, shared ? std::min(nrhs, 16) : 0);
  la.tensor = (shared && (p->flags & BTMV_FLAG_TENSOR_CORE) && p->c == 3 && sizeof(T) == sizeof(float2)) ? 1 : 0;
  ProfScope ps(p, full ? BTMV_K_FULL_LEAF : BTMV_K_LEAF, st);
  const bool reg = !(p->flags & BTMV_FLAG_GENERIC) && !shared && leaf_reg_supported(la, sizeof(T));
  cudaError_t e = reg ? launch_leaf_reg(la, st) : launch_leaf<T>(la, st);
  if (e != cudaSuccess) return fail(BTMV_E_CUDA, "leaf pass: %s", cudaGetErrorString(e));
  return BTMV_OK;
}

#define TRY(x) do { btmv_status s_ = (x); if (s_ != BTMV_OK) return s_; } while (0)

// Depth-first traversal of Algorithm 1 (see btmv_apply in btmv.h): a node at
// level m (transformed along dims 0..m-1) is split along dim m into itself
// (even half) and W[m] (odd half); at the last split level both children go
// to one leaf launch; merges run on the way back up.  With fuse, a node at
// level d-2 is one kind-3 step instead (its split, leaf and merge in one
// kernel, W[d-2] as scratch).
static void split_children(btmv_plan p, int m, void* e, void* o, int pe, int po, std::vector<Step>& out,
                           const std::vector<void*>& W, bool fuse);

static void split_descend(btmv_plan p, int m, void* buf, int prefix, std::vector<Step>& out,
                          const std::vector<void*>& W, bool fuse) {
  void* Wm = W[m];
  if (fuse && m == p->d - 2) {
    Step z = {3, m, buf, nullptr, buf, Wm, 1, {{buf, buf, prefix}}};
    out.push_back(z);
    return;
  }
  Step f = {0, m, buf, nullptr, buf, Wm, 0, {}};
  out.push_back(f);
  split_children(p, m, buf, Wm, prefix, prefix | (1 << m), out, W, fuse);
  Step g = {1, m, buf, Wm, buf, nullptr, 0, {}};
  out.push_back(g);
}

static void split_children(btmv_plan p, int m, void* e, void* o, int pe, int po, std::vector<Step>& out,
                           const std::vector<void*>& W, bool fuse) {
  if (m + 1 == p->d - 1) {
    Step l = {2, p->d - 1, nullptr, nullptr, nullptr, nullptr, 2, {{e, e, pe}, {o, o, po}}};
    out.push_back(l);
    return;
  }
  split_descend(p, m + 1, e, pe, out, W, fuse);
  split_descend(p, m + 1, o, po, out, W, fuse);
}

bool btmv::two_level_fusable(btmv_plan p) {
  if (!(p->flags & BTMV_FLAG_FUSED_LEVELS) || p->algo != BTMV_ALGO_SPLIT || p->prec != BTMV_C64) return false;
  if (fuse2_supported(p->d, p->c, p->n, sizeof(float2), p->symdev)) return true;
  // 128 x 128 slabs (one 16-CTA cluster per slab) measured 4x slower than the
  // unfused schedule at 128^3 (1468 against 373 us per apply), so that form
  // is taken only with BTMV_FUSE_CLUSTER=1 in the environment
  const char* v = getenv("BTMV_FUSE_CLUSTER");
  if (!v || v[0] != '1') return false;
  return fuse2c_supported(p->d, p->c, p->n, sizeof(float2), p->symdev) && fuse2c_available();
}

// 128 x 128 slabs take the cluster kernel (16 CTAs per slab)
static bool fuse_cluster_form(btmv_plan p) { return p->n[p->d - 1] == 128; }

// The fused kernel runs one block per (prefix index, right-hand side) and
// measured slower than the unfused schedule on small grids (64^3 with one
// right-hand side, 64 blocks: 0.116 against 0.071 ms), level at 512 blocks
// and 9-13% faster from 1024 blocks (two blocks per SM), so an apply fuses
// from 4 blocks per SM; with the two-stream traversal the two subtrees'
// fused launches run side by side, and 512 blocks each measured faster
// (64^3, 8 right-hand sides: 0.338 against 0.362 ms), so from 2 blocks per
// SM there.  BTMV_FUSE_MIN_BLOCKS=k in the environment sets another
// threshold (0: always).  The kernel copies the node it updates in
// 16-byte pieces; btmv_apply already requires 16-byte aligned x and y, and
// the test below keeps any other caller unfused.
static long long fuse_min_blocks(btmv_plan p) {
  const char* v = getenv("BTMV_FUSE_MIN_BLOCKS");
  if (v && *v) return atoll(v);
  return (p->side ? 2ll : 4ll) * std::max(1, p->nsm);
}

// CTAs of one fused launch: one per prefix index and right-hand side (16
// per slab for the cluster form, whose grid takes at most 65535 slabs)
static long long fuse_blocks(btmv_plan p, int nrhs) {
  long long b = nrhs;
  for (int m = 0; m + 2 < p->d; ++m) b *= p->n[m];
  if (fuse_cluster_form(p)) return b > 65535 ? 0 : 16 * b;
  return b;
}

bool btmv::fuse_this_apply(btmv_plan p, int nrhs, const void* y) {
  if (!two_level_fusable(p) || ((uintptr_t)y & 15)) return false;
  const long long b = fuse_blocks(p, nrhs);
  return b > 0 && b >= fuse_min_blocks(p);
}

void btmv::split_steps(btmv_plan p, const void* x, void* y, std::vector<Step>& out, bool fuse) {
  out.clear();
  if (p->d == 1) {
    Step l = {2, 0, nullptr, nullptr, nullptr, nullptr, 1, {{x, y, 0}, {}}};
    out.push_back(l);
    return;
  }
  Step f = {0, 0, x, nullptr, y, p->W[0], 0, {}};
  out.push_back(f);
  split_children(p, 0, y, p->W[0], 0, 1, out, p->W, fuse);
  Step g = {1, 0, y, p->W[0], y, nullptr, 0, {}};
  out.push_back(g);
}

// The kind-3 step: one fused kernel for the node's last two levels.
static btmv_status fused_levels(btmv_plan p, const Step& s, int nrhs, cudaStream_t st) {
  ProfScope ps(p, BTMV_K_FUSED_LEVELS, st);
  const int m = s.dim;
  cudaError_t e = fuse_cluster_form(p)
      ? launch_fuse2c((float2*)s.out0, (float2*)s.out1, s.nodes[0].prefix, p->d, p->n, nrhs, p->fft_apply[m],
                      p->fft_apply[m + 1], p->symdev, st)
      : launch_fuse2((float2*)s.out0, (float2*)s.out1, s.nodes[0].prefix, p->d, p->n, nrhs, p->fft_apply[m],
                     p->fft_apply[m + 1], p->symdev, st);
  if (e != cudaSuccess) return fail(BTMV_E_CUDA, "fused levels: %s", cudaGetErrorString(e));
  return BTMV_OK;
}

template <class T>
static btmv_status run_steps(btmv_plan p, const std::vector<Step>& steps, int nrhs, cudaStream_t st) {
  for (const Step& s : steps) {
    if (s.kind == 2)      TRY(leaf_launch<T>(p, nrhs, s.nn, s.nodes, false, st));
    else if (s.kind == 3) TRY(fused_levels(p, s, nrhs, st));
    else                  TRY(split_pass<T>(p, s, nrhs, st));
  }
  return BTMV_OK;
}

// d = 2, c = 1, 64 x 64: the three kernels of the split apply (dim-0 split,
// leaf, dim-0 merge) as one launch of a thread-block cluster per right-hand
// side (small2d.cu).  BTMV_SMALL2D=0 in the environment, or
// BTMV_FLAG_GENERIC, keeps the three kernels (comparisons).
bool btmv::use_small2d(btmv_plan p) {
  if (p->algo != BTMV_ALGO_SPLIT || (p->flags & BTMV_FLAG_GENERIC)) return false;
  const char* v = getenv("BTMV_SMALL2D");
  if (v && v[0] == '0') return false;
  return small2d_supported(p->d, p->c, p->n, p->symdev) && p->fft_apply[0].N == 64 && p->fft_apply[1].N == 64;
}

template <class T>
static btmv_status split_apply(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st) {
  if (use_small2d(p)) {
    ProfScope ps(p, BTMV_K_FUSED_LEVELS, st);
    const cudaError_t e = launch_small2d(x, y, nrhs, sizeof(T) == sizeof(double2), p->fft_apply[0], p->symdev, st);
    if (e != cudaSuccess) return fail(BTMV_E_CUDA, "small two-level apply: %s", cudaGetErrorString(e));
    return BTMV_OK;
  }
  std::vector<Step> steps;
  const bool fuse = fuse_this_apply(p, nrhs, y);
  if (!p->side) {
    split_steps(p, x, y, steps, fuse);
    return run_steps<T>(p, steps, nrhs, st);
  }
  // two top-level subtrees on two streams: the even one on st with W, the
  // odd one on the plan's side stream with its own workspace W2, so that the
  // memory-bound passes of one overlap the compute-bound leaves of the other
  Step f = {0, 0, x, nullptr, y, p->W[0], 0, {}};
  TRY(split_pass<T>(p, f, nrhs, st));
  CUDA_TRY(cudaEventRecord(p->ev_fork, st));
  CUDA_TRY(cudaStreamWaitEvent(p->side, p->ev_fork, 0));
  std::vector<Step> a, b;
  if (p->d - 1 == 1) {
    Step l = {2, 1, nullptr, nullptr, nullptr, nullptr, 2, {{y, y, 0}, {p->W[0], p->W[0], 1}}};
    a.push_back(l);
  } else {
    split_descend(p, 1, y, 0, a, p->W, fuse);
    split_descend(p, 1, p->W[0], 1, b, p->W2, fuse);
  }
  TRY(run_steps<T>(p, a, nrhs, st));
  TRY(run_steps<T>(p, b, nrhs, p->side));
  CUDA_TRY(cudaEventRecord(p->ev_join, p->side));
  CUDA_TRY(cudaStreamWaitEvent(st, p->ev_join, 0));
  Step g = {1, 0, y, p->W[0], y, nullptr, 0, {}};
  return split_pass<T>(p, g, nrhs, st);
}

// Plain full embedding with own kernels: pad fused into the first forward
// pass, multiply into the last-dim pass, projection into the last inverse pass.
template <class T>
static btmv_status full_apply(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st) {
  const int d = p->d;
  void* Z = p->W[0];
  const size_t esz = sizeof(T);
  if (d == 1) {
    const size_t rows = (size_t)nrhs * p->c;
    const size_t nb = (size_t)p->n[0] * esz;
    {
      ProfScope ps(p, BTMV_K_FULL_FWD, st);
      CUDA_TRY(cudaMemsetAsync(Z, 0, rows * 2 * nb, st));
      CUDA_TRY(cudaMemcpy2DAsync(Z, 2 * nb, x, nb, nb, rows, cudaMemcpyDeviceToDevice, st));
    }
    LeafNode nd = {Z, Z, 0};
    TRY(leaf_launch<T>(p, nrhs, 1, &nd, true, st));
    ProfScope ps(p, BTMV_K_FULL_INV, st);
    CUDA_TRY(cudaMemcpy2DAsync(y, nb, Z, 2 * nb, nb, rows, cudaMemcpyDeviceToDevice, st));
    return BTMV_OK;
  }
  // strides of x/y (n grid) and Z (2n grid)
  long long sx[MAX_D], sz[MAX_D];
  sx[d - 1] = 1; sz[d - 1] = 1;
  for (int m = d - 2; m >= 0; --m) { sx[m] = sx[m + 1] * p->n[m + 1]; sz[m] = sz[m + 1] * 2 * p->n[m + 1]; }
  // first pass: dim 0, x (n grid, zero padded) -> Z (2n grid), every Z line written
  {
    PassArgs pa;
    memset(&pa, 0, sizeof pa);
    pa.g.N = 2 * p->n[0];
    pa.g.ni = d - 1;
    pa.g.Itot = 1;
    for (int j = 0; j < d - 1; ++j) { pa.g.I[j] = 2 * p->n[j + 1]; pa.g.Itot *= pa.g.I[j]; }
    pa.g.lines = (long long)nrhs * p->c * pa.g.Itot;
    pa.g.contig = 0;
    choose_tile(pa.g, esz);
    ArrMap ai, ao;
    memset(&ai, 0, sizeof ai);
    memset(&ao, 0, sizeof ao);
    ai.os = p->s; ai.es = sx[0]; ai.len = p->n[0];
    ao.os = p->s2; ao.es = sz[0]; ao.len = 2 * p->n[0];
    for (int j = 0; j < 3; ++j) { ai.vI[j] = 1 << 30; ao.vI[j] = 1 << 30; }
    for (int j = 0; j < d - 1; ++j) { ai.is[j] = sx[j + 1]; ai.vI[j] = p->n[j + 1]; ao.is[j] = sz[j + 1]; }
    pa.a_in0 = pa.a_in1 = ai;
    pa.a_out0 = pa.a_out1 = ao;
    pa.in0 = x; pa.out0 = Z;
    pa.fft = p->fft_apply[0];
    ProfScope ps(p, BTMV_K_FULL_FWD, st);
    cudaError_t e = launch_pass<T>(0, pa, st);
    if (e != cudaSuccess) return fail(BTMV_E_CUDA, "full first pass: %s", cudaGetErrorString(e));
  }
  auto big_pass = [&](int mode, int m) -> btmv_status {
    long long outer = (long long)nrhs * p->c, inner = 1;
    for (int q = 0; q < m; ++q) outer *= 2 * p->n[q];
    for (int q = m + 1; q < d; ++q) inner *= 2 * p->n[q];
    PassArgs pa;
    memset(&pa, 0, sizeof pa);
    const int N = 2 * p->n[m];
    pa.g.N = N; pa.g.ni = inner > 1 ? 1 : 0; pa.g.I[0] = (int)inner; pa.g.Itot = inner;
    pa.g.lines = outer * inner; pa.g.contig = inner == 1;
    choose_tile(pa.g, esz);
    pa.a_in0 = pa.a_in1 = pa.a_out0 = pa.a_out1 = contig_map(N, inner);
    pa.in0 = Z; pa.out0 = Z;
    pa.fft = p->fft_apply[m];
    ProfScope ps(p, mode == 0 ? BTMV_K_FULL_FWD : BTMV_K_FULL_INV, st);
    cudaError_t e = run_pass<T>(p, mode, pa, st);
    if (e != cudaSuccess) return fail(BTMV_E_CUDA, "full pass dim %d: %s", m, cudaGetErrorString(e));
    return BTMV_OK;
  };
  for (int m = 1; m < d - 1; ++m) TRY(big_pass(0, m));
  {
    LeafNode nd = {Z, Z, 0};
    TRY(leaf_launch<T>(p, nrhs, 1, &nd, true, st));
  }
  for (int m = d - 2; m >= 1; --m) TRY(big_pass(1, m));
  // last pass: dim 0 inverse on the surviving lines, projected into y
  {
    PassArgs pa;
    memset(&pa, 0, sizeof pa);
    pa.g.N = 2 * p->n[0];
    pa.g.ni = d - 1;
    pa.g.Itot = 1;
    for (int j = 0; j < d - 1; ++j) { pa.g.I[j] = p->n[j + 1]; pa.g.Itot *= pa.g.I[j]; }
    pa.g.lines = (long long)nrhs * p->c * pa.g.Itot;
    pa.g.contig = 0;
    choose_tile(pa.g, esz);
    ArrMap ai, ao;
    memset(&ai, 0, sizeof ai);
    memset(&ao, 0, sizeof ao);
    ai.os = p->s2; ai.es = sz[0]; ai.len = 2 * p->n[0];
    ao.os = p->s; ao.es = sx[0]; ao.len = p->n[0];
    for (int j = 0; j < 3; ++j) { ai.vI[j] = 1 << 30; ao.vI[j] = 1 << 30; }
    for (int j = 0; j < d - 1; ++j) { ai.is[j] = sz[j + 1]; ao.is[j] = sx[j + 1]; }
    pa.a_in0 = pa.a_in1 = ai;
    pa.a_out0 = pa.a_out1 = ao;
    pa.in0 = Z; pa.out0 = y;
    pa.fft = p->fft_apply[0];
    ProfScope ps(p, BTMV_K_FULL_INV, st);
    cudaError_t e = launch_pass<T>(1, pa, st);
    if (e != cudaSuccess) return fail(BTMV_E_CUDA, "full last pass: %s", cudaGetErrorString(e));
  }
  return BTMV_OK;
}

static int is_device_ptr(const void* ptr) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) { cudaGetLastError(); return 0; }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Padded plans: x is copied into the padded buffer (zeros outside the
// caller's sizes), the apply runs at the padded sizes, and the caller's part
// of the padded result is copied to y.
template <class T>
static btmv_status pad_copy(btmv_plan p, const void* src, void* dst, int nrhs, bool to_pad, cudaStream_t st) {
  PadArgs a;
  memset(&a, 0, sizeof a);
  a.src = src; a.dst = dst; a.d = p->d; a.to_pad = to_pad ? 1 : 0;
  for (int m = 0; m < p->d; ++m) { a.nu[m] = p->nu[m]; a.np[m] = p->n[m]; }
  a.total = (long long)nrhs * p->c * (to_pad ? p->s : p->su);
  ProfScope ps(p, BTMV_K_COPY, st);
  const cudaError_t e = launch_pad<T>(a, st);
  if (e != cudaSuccess) return fail(BTMV_E_CUDA, "padding copy: %s", cudaGetErrorString(e));
  return BTMV_OK;
}

static btmv_status apply_device(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st) {
  p->prof_on = (p->flags & BTMV_FLAG_PROFILE) && (p->prof_count++ % p->prof_every) == 0;
  const bool c64 = p->prec == BTMV_C64;
  if (p->padded) {
    TRY(c64 ? pad_copy<float2>(p, x, p->xpad, nrhs, true, st) : pad_copy<double2>(p, x, p->xpad, nrhs, true, st));
    TRY(c64 ? split_apply<float2>(p, p->xpad, p->ypad, nrhs, st) : split_apply<double2>(p, p->xpad, p->ypad, nrhs, st));
    return c64 ? pad_copy<float2>(p, p->ypad, y, nrhs, false, st) : pad_copy<double2>(p, p->ypad, y, nrhs, false, st);
  }
  if (p->algo == BTMV_ALGO_SPLIT)
    return c64 ? split_apply<float2>(p, x, y, nrhs, st) : split_apply<double2>(p, x, y, nrhs, st);
  if (p->algo == BTMV_ALGO_FULL_CUFFT) {
    ProfScope ps(p, BTMV_K_FULL_LEAF, st);
    return cufft_full_apply(p, x, y, nrhs, st);
  }
  return c64 ? full_apply<float2>(p, x, y, nrhs, st) : full_apply<double2>(p, x, y, nrhs, st);
}

static btmv_status check_apply(btmv_plan p, const void* x, void* y, int nrhs) {
  if (!p) return fail(BTMV_E_ARG, "apply: plan is NULL");
  if (nrhs < 0 || nrhs > p->max_rhs) return fail(BTMV_E_ARG, "apply: nrhs=%d outside [0,%d]", nrhs, p->max_rhs);
  if (!p->has_sym) return fail(BTMV_E_STATE, "apply: btmv_set_kernel has not been called");
  if (nrhs == 0) return BTMV_OK;
  if (!x || !y) return fail(BTMV_E_ARG, "apply: x or y is NULL");
  if (((uintptr_t)x | (uintptr_t)y) & 15) return fail(BTMV_E_ARG, "apply: x and y must be 16-byte aligned");
  const size_t V = (size_t)nrhs * p->c * p->su * p->esz;
  const char* xa = (const char*)x;
  const char* ya = (const char*)y;
  if (xa < ya + V && ya < xa + V) return fail(BTMV_E_ARG, "apply: x and y overlap");
  return BTMV_OK;
}

// Hooks for entry points defined in other translation units of the library
// (not exported): argument checks, vector size, and the device-pointer apply.
btmv_status btmv_check_apply_args(btmv_plan p, const void* x, void* y, int nrhs) {
  return check_apply(p, x, y, nrhs);
}
size_t btmv_apply_vector_bytes(btmv_plan p, int nrhs) { return (size_t)nrhs * p->c * p->su * p->esz; }
btmv_status btmv_apply_on_device(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st) {
  p->launches = 0;
  return apply_device(p, x, y, nrhs, st);
}
btmv_status btmv_set_error(btmv_status st, const char* msg) { return fail(st, "%s", msg); }
void btmv_clear_error() { g_err.clear(); }
int btmv_plan_device(btmv_plan p) { return p->dev; }
int btmv_is_device_ptr(const void* ptr) { return is_device_ptr(ptr); }

extern "C" btmv_status btmv_apply(btmv_plan p, const void* x, void* y, int nrhs, void* stream) {
  g_err.clear();
  TRY(check_apply(p, x, y, nrhs));
  if (nrhs == 0) return BTMV_OK;
  cudaStream_t st = (cudaStream_t)stream;
  const int dx = is_device_ptr(x), dy = is_device_ptr(y);
  p->launches = 0;
  if (dx && dy) return apply_device(p, x, y, nrhs, st);
  // host staging
  const size_t V = (size_t)nrhs * p->c * p->su * p->esz;
  const size_t Vmax = (size_t)p->max_rhs * p->c * p->su * p->esz;
  if (!dx && !p->stage_x) CUDA_TRY(cudaMalloc(&p->stage_x, Vmax));
  if (!dy && !p->stage_y) CUDA_TRY(cudaMalloc(&p->stage_y, Vmax));
  const void* xd = x;
  void* yd = y;
  if (!dx) {
    ProfScope ps(p, BTMV_K_COPY, st);
    CUDA_TRY(cudaMemcpyAsync(p->stage_x, x, V, cudaMemcpyHostToDevice, st));
    xd = p->stage_x;
  }
  if (!dy) yd = p->stage_y;
  TRY(apply_device(p, xd, yd, nrhs, st));
  if (!dy) {
    ProfScope ps(p, BTMV_K_COPY, st);
    CUDA_TRY(cudaMemcpyAsync(y, yd, V, cudaMemcpyDeviceToHost, st));
  }
  CUDA_TRY(cudaStreamSynchronize(st));
  return BTMV_OK;
}

extern "C" btmv_status btmv_destroy(btmv_plan p) {
  g_err.clear();
  if (!p) return BTMV_OK;
  cudaDeviceSynchronize();
  batch_forget_plan(p);
  free_plan(p);
  return BTMV_OK;
}

extern "C" const char* btmv_last_error(void) { return g_err.c_str(); }

static int launches_per_apply(btmv_plan p) {
  const int d = p->d;
  if (p->algo == BTMV_ALGO_SPLIT) {
    if (d == 1 || use_small2d(p)) return 1;
    int n = 0;
    if (two_level_fusable(p) && fuse_blocks(p, p->max_rhs) > 0 && fuse_blocks(p, p->max_rhs) >= fuse_min_blocks(p)) {
      // forward + merge per node of levels 0..d-3, one fused launch per level-(d-2) node
      for (int m = 0; m < d - 2; ++m) n += 2 * (1 << m);
      return n + (1 << (d - 2));
    }
    // forward + merge per internal node of levels 0..d-2, one leaf launch per level-(d-2) node
    for (int m = 0; m < d - 1; ++m) n += 2 * (1 << m);
    n += 1 << (d - 2);
    return n;
  }
  if (p->algo == BTMV_ALGO_FULL_CUFFT) return 3;   // pad, multiply, projection (+ cuFFT's own kernels)
  if (d == 1) return 3;
  return 2 * (d - 2) + 3;
}

extern "C" btmv_status btmv_plan_get_info(btmv_plan p, btmv_plan_info_t* info) {
  g_err.clear();
  if (!p || !info) return fail(BTMV_E_ARG, "plan_get_info: NULL argument");
  memset(info, 0, sizeof *info);
  info->d = p->d; info->c = p->c; info->precision = p->prec; info->algo = p->algo; info->max_rhs = p->max_rhs;
  for (int m = 0; m < MAX_D; ++m) info->n[m] = m < p->d ? p->nu[m] : 0;
  info->nsym = p->nsym;
  info->compressed = p->compressed;
  info->has_symbol = p->has_sym ? 1 : 0;
  info->launches_per_apply = launches_per_apply(p);
  info->symbol_bytes = p->sym_bytes;
  info->workspace_bytes = p->ws_bytes;
  info->table_bytes = p->tab.bytes;
  info->vector_bytes = (size_t)p->c * p->su * p->esz;
  return BTMV_OK;
}

extern "C" btmv_status btmv_get_symbol(btmv_plan p, void* out, size_t bytes) {
  g_err.clear();
  if (!p || !out) return fail(BTMV_E_ARG, "get_symbol: NULL argument");
  if (!p->has_sym) return fail(BTMV_E_STATE, "get_symbol: no symbol");
  if (bytes < p->sym_bytes) return fail(BTMV_E_ARG, "get_symbol: need %zu bytes", p->sym_bytes);
  CUDA_TRY(cudaDeviceSynchronize());
  CUDA_TRY(cudaMemcpy(out, p->sym, p->sym_bytes, cudaMemcpyDeviceToHost));
  return BTMV_OK;
}

extern "C" btmv_status btmv_profile_read(btmv_plan p, double* ms_total, int64_t* launches) {
  g_err.clear();
  if (!p || !ms_total || !launches) return fail(BTMV_E_ARG, "profile_read: NULL argument");
  if (!(p->flags & BTMV_FLAG_PROFILE)) return fail(BTMV_E_STATE, "profile_read: plan created without BTMV_FLAG_PROFILE");
  drain_profile(p);
  for (int k = 0; k < BTMV_K_NKINDS; ++k) {
    ms_total[k] = p->acc_ms[k];
    launches[k] = p->acc_n[k];
    p->acc_ms[k] = 0;
    p->acc_n[k] = 0;
  }
  p->prof_count = 0;                  // the next apply is a sampled one
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(BTMV_E_CUDA, "profile_read: %s", cudaGetErrorString(e));
  return BTMV_OK;
}
