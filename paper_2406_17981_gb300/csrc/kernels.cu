// Line-pass kernels of the split-FFT block Toeplitz product.
//
//   k_pass<T, 0>  forward split pass along one level (Sec. II.A splitting
//                 property): one read of the parent node, both children
//                 written -- even = FFT_n(v), odd = FFT_n(P v).
//   k_pass<T, 1>  backward merge pass (Sec. II.A merge, Algorithm 1 mrgBrn
//                 + iFFT): out = IFFT_n(v_even) + conj(P) IFFT_n(v_odd).
//   k_leaf<T>     leaf pass along the last level: both halves, the c x c
//                 symbol multiply (Algorithm 1 mulBrn with T[bId]) and the
//                 merge, fused per contiguous line.
//   k_fold / k_store  FP64 symbol build (see btmv_set_kernel).
//
// Every pass stages a tile of lines through shared memory: coalesced global
// loads, Stockham stages ping-ponging between smem buffers, coalesced stores.
#include <cuda_runtime.h>
#include <stdint.h>

#include <algorithm>

#include "generic.cuh"

namespace btmv {

size_t pass_smem_bytes(const PassGeom& g, size_t esz) {
  const size_t ls = g.contig ? (size_t)(g.N | 1) : 1;
  const size_t buf = g.contig ? (size_t)g.TL * ls : (size_t)g.TL * g.N;
  return pass_hdr_bytes(g.TL) + (g.halves == 2 ? 4 : 3) * buf * esz;   // (two-half) tile + scratch
}

size_t leaf_smem_bytes(int N, int c, int rq, int Lt, size_t esz) {
  const size_t ls = (size_t)(N | 1);
  return leaf_hdr_bytes(Lt) + 4 * (size_t)rq * c * Lt * ls * esz;   // two-half tile + its scratch
}

template <class T, int MODE>
__global__ void __launch_bounds__(256) k_pass(const PassArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  if (a.g.contig) pass_body<T, MODE, false>(a, smem, blockIdx.x);
  else            pass_body<T, MODE, true>(a, smem, blockIdx.x);
}


template <class T>
cudaError_t launch_pass(int mode, const PassArgs& a, cudaStream_t st) {
  const size_t sm = pass_smem_bytes(a.g, sizeof(T));
  if (sm > kMaxSmem) return cudaErrorInvalidValue;
  const long long nt = (a.g.lines + a.g.TL - 1) / a.g.TL;
  if (nt <= 0) return cudaSuccess;
  if (nt > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (mode == 0) {
    const cudaError_t ae = set_smem_attr<k_pass<T, 0>>((int)kMaxSmem);
    if (ae != cudaSuccess) return ae;
    k_pass<T, 0><<<(unsigned)nt, 256, sm, st>>>(a);
  } else {
    const cudaError_t ae = set_smem_attr<k_pass<T, 1>>((int)kMaxSmem);
    if (ae != cudaSuccess) return ae;
    k_pass<T, 1><<<(unsigned)nt, 256, sm, st>>>(a);
  }
  return cudaGetLastError();
}

template <class T>
__global__ void __launch_bounds__(256) k_leaf(const LeafArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  leaf_body<T>(a, smem, blockIdx.x, blockIdx.y);
}

template <class T>
cudaError_t launch_leaf(const LeafArgs& a, cudaStream_t st) {
  const size_t sm = leaf_smem_bytes(a.N, a.c, a.rq, a.Lt, sizeof(T));
  if (sm > kMaxSmem) return cudaErrorInvalidValue;
  if (a.tiles_per_node <= 0 || a.nnodes <= 0) return cudaSuccess;
  if (a.tiles_per_node > 0x7fffffffLL || a.nnodes > MAX_LEAF_NODES) return cudaErrorInvalidValue;
  const cudaError_t ae = set_smem_attr<k_leaf<T>>((int)kMaxSmem);
  if (ae != cudaSuccess) return ae;
  dim3 grid((unsigned)a.tiles_per_node, (unsigned)a.nnodes);
  k_leaf<T><<<grid, 256, sm, st>>>(a);
  return cudaGetLastError();
}

// ------------------------------------------------------------------- pad
template <class T>
__global__ void __launch_bounds__(256) k_pad(const PadArgs a) {
  const int* wn = a.to_pad ? a.np : a.nu;     // shape of the written vector
  const int* on = a.to_pad ? a.nu : a.np;     // shape of the other one
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < a.total;
       e += (long long)gridDim.x * blockDim.x) {
    long long r = e, src = 0, stride = 1;
    bool inside = true;
    for (int m = a.d - 1; m >= 0; --m) {
      const int im = (int)(r % wn[m]);
      r /= wn[m];
      inside = inside && im < on[m] && im < wn[m];
      src += (long long)im * stride;
      stride *= on[m];
    }
    src += r * stride;                        // (rhs, component) index
    T v;
    v.x = 0; v.y = 0;
    if (inside) v = ((const T*)a.src)[src];
    ((T*)a.dst)[e] = v;
  }
}

template <class T>
cudaError_t launch_pad(const PadArgs& a, cudaStream_t st) {
  if (a.total <= 0) return cudaSuccess;
  const long long blocks = std::min<long long>((a.total + 255) / 256, 152LL * 16);
  k_pad<T><<<(unsigned)blocks, 256, 0, st>>>(a);
  return cudaGetLastError();
}
template cudaError_t launch_pad<float2>(const PadArgs&, cudaStream_t);
template cudaError_t launch_pad<double2>(const PadArgs&, cudaStream_t);

// ----------------------------------------------------------------- symbol
// F[kk][k] = scale * sum_{h in {0,1}^d} (-1)^{<h, b>} c~_kk[k + h n]  with
// c~[k + n] = t[k - n] for k > 0 and the free entry s0 = 0 for k = 0: the
// 2n-point embedded generator folded onto n points for parity class b, so
// that DFT_n(P_b F) is the leaf part S_b.
__global__ void k_fold(const FoldArgs a) {
  const long long total = (long long)a.nsym * a.s;
  long long tb = 1;
  if (!a.parity_layout)
    for (int m = 0; m < a.d; ++m) tb *= (2 * a.n[m] - 1);
  else
    tb = a.s;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(idx / a.s);
    long long r = idx - (long long)kk * a.s;
    int k[MAX_D];
    for (int m = a.d - 1; m >= 0; --m) { k[m] = (int)(r % a.n[m]); r /= a.n[m]; }
    const int A = a.pairs[kk][0], B = a.pairs[kk][1];
    const double2* tb0 = a.t + (long long)(A * a.c + B) * tb;
    double ax = 0.0, ay = 0.0;
    for (int h = 0; h < (1 << a.d); ++h) {
      double sg = 1.0;
      bool ok = true;
      long long toff = 0;
      for (int m = 0; m < a.d; ++m) {
        int p;
        if ((h >> m) & 1) {
          if (k[m] == 0) { ok = false; break; }
          p = k[m] - a.n[m];
          if (a.cls_bits[m]) sg = -sg;
        } else {
          p = k[m];
        }
        if (a.parity_layout) {
          if (p < 0) { sg *= (double)a.par[A][B][m]; p = -p; }
          toff = toff * a.n[m] + p;
        } else {
          toff = toff * (2 * a.n[m] - 1) + (p + a.n[m] - 1);
        }
      }
      if (!ok) continue;
      const double2 v = tb0[toff];
      ax += sg * v.x;
      ay += sg * v.y;
    }
    a.F[idx] = make_double2(ax * a.scale, ay * a.scale);
  }
}

__global__ void k_store(const StoreArgs a) {
  const long long total = (long long)a.nsym * a.blk;
  for (long long idx = (long long)blockIdx.x * blockDim.x + threadIdx.x; idx < total;
       idx += (long long)gridDim.x * blockDim.x) {
    const int kk = (int)(idx / a.blk);
    long long r = idx - (long long)kk * a.blk;
    long long lin = 0, mul = 1;
    for (int m = a.d - 1; m >= 0; --m) {
      const int j = (int)(r % a.J[m]);
      r /= a.J[m];
      lin += (long long)j * mul;
      mul *= a.n[m];
    }
    const double2 v = a.F[(long long)kk * a.s + lin];
    if (a.prec == 0) ((float2*)a.store)[a.cls_off + idx] = make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
    else             ((double2*)a.store)[a.cls_off + idx] = v;
  }
}

cudaError_t launch_fold(const FoldArgs& a, cudaStream_t st) {
  k_fold<<<152 * 8, 256, 0, st>>>(a);
  return cudaGetLastError();
}
cudaError_t launch_store(const StoreArgs& a, cudaStream_t st) {
  k_store<<<152 * 8, 256, 0, st>>>(a);
  return cudaGetLastError();
}

template cudaError_t launch_pass<float2>(int, const PassArgs&, cudaStream_t);
template cudaError_t launch_pass<double2>(int, const PassArgs&, cudaStream_t);
template cudaError_t launch_leaf<float2>(const LeafArgs&, cudaStream_t);
template cudaError_t launch_leaf<double2>(const LeafArgs&, cudaStream_t);


}  // namespace btmv
