// BTMV_ALGO_FULL_CUFFT: the plain full circulant embedding (Sec. I) with
// cuFFT doing the 2n-point transforms -- the library-FFT comparator of the
// split algorithm.  Nothing on the split path uses it.
//
//   x --pad (own kernel)--> Z (2^d-sized, zero outside the n grid)
//     --cuFFT forward (all dims)--> Z
//     --c x c symbol multiply per frequency (own kernel, full or
//       mirror-compressed store)--> Z
//     --cuFFT inverse--> Z --project the n grid (own kernel)--> y
//
// cuFFT is opened with dlopen when the first such plan is created, so the
// library itself does not depend on it.
#include <cuda_runtime.h>
#include <cufft.h>
#include <dlfcn.h>

#include <algorithm>
#include <cstring>
#include <mutex>

#include "generic.cuh"
#include "plan.h"

namespace btmv {

namespace {

struct CufftApi {
  bool ok = false;
  cufftResult (*plan_many)(cufftHandle*, int, int*, int*, int, int, int*, int, int, cufftType, int) = nullptr;
  cufftResult (*exec_c2c)(cufftHandle, cufftComplex*, cufftComplex*, int) = nullptr;
  cufftResult (*exec_z2z)(cufftHandle, cufftDoubleComplex*, cufftDoubleComplex*, int) = nullptr;
  cufftResult (*set_stream)(cufftHandle, cudaStream_t) = nullptr;
  cufftResult (*destroy)(cufftHandle) = nullptr;
};

CufftApi g_api;
std::once_flag g_api_once;

void load_api() {
  void* h = nullptr;
  for (const char* name : {"libcufft.so.12", "libcufft.so", "/usr/local/cuda/lib64/libcufft.so.12"}) {
    h = dlopen(name, RTLD_NOW | RTLD_LOCAL);
    if (h) break;
  }
  if (!h) return;
  g_api.plan_many = (decltype(g_api.plan_many))dlsym(h, "cufftPlanMany");
  g_api.exec_c2c = (decltype(g_api.exec_c2c))dlsym(h, "cufftExecC2C");
  g_api.exec_z2z = (decltype(g_api.exec_z2z))dlsym(h, "cufftExecZ2Z");
  g_api.set_stream = (decltype(g_api.set_stream))dlsym(h, "cufftSetStream");
  g_api.destroy = (decltype(g_api.destroy))dlsym(h, "cufftDestroy");
  g_api.ok = g_api.plan_many && g_api.exec_c2c && g_api.exec_z2z && g_api.set_stream && g_api.destroy;
}

// Per-frequency c x c multiply on the 2n grid, in place: Z[r][a][f] <-
// sum_b S_ab(f) Z[r][b][f], S read from the class-major store at class f & 1,
// index f >> 1 (folded to 2n - f with the parity sign on the compressed store).
template <class T>
__global__ void k_full_multiply(T* __restrict__ Z, const SymDev S, int c, int d, long long s2, long long total,
                                int n2_0, int n2_1, int n2_2) {
  const int n2[3] = {n2_0, n2_1, n2_2};
  const T* __restrict__ Sd = (const T*)S.data;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long r = e / s2;
    const long long k = e - r * s2;
    int f[MAX_D];
    long long rem = k;
    for (int m = d - 1; m >= 0; --m) {
      f[m] = (int)(rem % n2[m]);
      rem /= n2[m];
    }
    int fold, cls;
    const long long base = sym_index(S, f, fold, cls);
    const long long blk = S.blk[cls];
    T* z = Z + r * c * s2 + k;
    T xv[3], yv[3];
    for (int b = 0; b < c; ++b) xv[b] = z[b * s2];
    for (int a = 0; a < c; ++a) {
      T acc = czero<T>();
      for (int b = 0; b < c; ++b) {
        const int kk = S.comp[a][b];
        T sv = __ldg(&Sd[base + kk * blk]);
        if (__popc(S.oddmask[kk] & fold) & 1) { sv.x = -sv.x; sv.y = -sv.y; }
        acc = cadd(acc, cmul(sv, xv[b]));
      }
      yv[a] = acc;
    }
    for (int a = 0; a < c; ++a) z[a * s2] = yv[a];
  }
}

}  // namespace

btmv_status cufft_plan_setup(btmv_plan p) {
  std::call_once(g_api_once, load_api);
  if (!g_api.ok) return fail(BTMV_E_UNSUPPORTED, "plan_create: BTMV_ALGO_FULL_CUFFT needs libcufft (not found)");
  if (p->d > 3) return fail(BTMV_E_UNSUPPORTED, "plan_create: BTMV_ALGO_FULL_CUFFT takes d <= 3");
  int dims[3];
  for (int m = 0; m < p->d; ++m) dims[m] = 2 * p->n[m];
  cufftHandle h = 0;
  // one plan transforms the c components of one right-hand side
  const cufftType ty = p->prec == BTMV_C64 ? CUFFT_C2C : CUFFT_Z2Z;
  const cufftResult r = g_api.plan_many(&h, p->d, dims, nullptr, 1, (int)p->s2, nullptr, 1, (int)p->s2, ty, p->c);
  if (r != CUFFT_SUCCESS) return fail(BTMV_E_NOMEM, "plan_create: cufftPlanMany failed (%d)", (int)r);
  p->cufft = (int)h;
  p->has_cufft = true;
  return BTMV_OK;
}

void cufft_plan_destroy(btmv_plan p) {
  if (p->has_cufft && g_api.ok) g_api.destroy((cufftHandle)p->cufft);
  p->has_cufft = false;
}

template <class T>
static btmv_status cufft_apply_t(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st) {
  T* Z = (T*)p->W[0];
  const int d = p->d;
  PadArgs pa;
  memset(&pa, 0, sizeof pa);
  pa.d = d;
  for (int m = 0; m < d; ++m) { pa.nu[m] = p->n[m]; pa.np[m] = 2 * p->n[m]; }
  {
    pa.src = x; pa.dst = Z; pa.to_pad = 1; pa.total = (long long)nrhs * p->c * p->s2;
    cudaError_t e = launch_pad<T>(pa, st);
    if (e != cudaSuccess) return fail(BTMV_E_CUDA, "cufft pad: %s", cudaGetErrorString(e));
    if (g_api.set_stream((cufftHandle)p->cufft, st) != CUFFT_SUCCESS) return fail(BTMV_E_CUDA, "cufftSetStream failed");
    for (int r = 0; r < nrhs; ++r) {
      T* zr = Z + (size_t)r * p->c * p->s2;
      const cufftResult fr = sizeof(T) == sizeof(float2)
          ? g_api.exec_c2c((cufftHandle)p->cufft, (cufftComplex*)zr, (cufftComplex*)zr, CUFFT_FORWARD)
          : g_api.exec_z2z((cufftHandle)p->cufft, (cufftDoubleComplex*)zr, (cufftDoubleComplex*)zr, CUFFT_FORWARD);
      if (fr != CUFFT_SUCCESS) return fail(BTMV_E_CUDA, "cuFFT forward failed (%d)", (int)fr);
    }
  }
  {
    const long long total = (long long)nrhs * p->s2;
    const int threads = 256;
    const long long want = (total + threads - 1) / threads;
    const int grid = (int)std::min<long long>(want, 152LL * 16);
    k_full_multiply<T><<<grid, threads, 0, st>>>(Z, p->symdev, p->c, d, p->s2, total, 2 * p->n[0],
                                                 d > 1 ? 2 * p->n[1] : 1, d > 2 ? 2 * p->n[2] : 1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(BTMV_E_CUDA, "cufft multiply: %s", cudaGetErrorString(e));
  }
  {
    for (int r = 0; r < nrhs; ++r) {
      T* zr = Z + (size_t)r * p->c * p->s2;
      const cufftResult fr = sizeof(T) == sizeof(float2)
          ? g_api.exec_c2c((cufftHandle)p->cufft, (cufftComplex*)zr, (cufftComplex*)zr, CUFFT_INVERSE)
          : g_api.exec_z2z((cufftHandle)p->cufft, (cufftDoubleComplex*)zr, (cufftDoubleComplex*)zr, CUFFT_INVERSE);
      if (fr != CUFFT_SUCCESS) return fail(BTMV_E_CUDA, "cuFFT inverse failed (%d)", (int)fr);
    }
    pa.src = Z; pa.dst = y; pa.to_pad = 0; pa.total = (long long)nrhs * p->c * p->s;
    cudaError_t e = launch_pad<T>(pa, st);
    if (e != cudaSuccess) return fail(BTMV_E_CUDA, "cufft projection: %s", cudaGetErrorString(e));
  }
  return BTMV_OK;
}

btmv_status cufft_full_apply(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st) {
  return p->prec == BTMV_C64 ? cufft_apply_t<float2>(p, x, y, nrhs, st) : cufft_apply_t<double2>(p, x, y, nrhs, st);
}

}  // namespace btmv
