// Internal kernel interfaces of libbtmv (not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>

#include "../../include/btmv.h"
#include "fft.cuh"

namespace btmv {

// Addressing of one global array in a line pass.  A line is identified by
// (outer o, inner multi-index (i_0, .., i_{ni-1})); its element k lives at
//   o * os + sum_j i_j * is[j] + k * es.
struct ArrMap {
  long long os;
  long long is[3];
  long long es;
  int vI[3];   // input: lines with i_j >= vI[j] read as zero
  int len;     // input: elements k >= len read as zero; output: only k < len written
};

struct PassGeom {
  int N;             // transform length
  int ni;            // number of inner dims (0..3)
  int I[3];          // inner extents (iteration)
  long long Itot;    // product of inner extents (1 when ni == 0)
  long long lines;   // outer count * Itot
  int TL;            // lines per tile
  int contig;        // 1: element stride 1 (line-major smem), 0: line-fast smem
  int halves;        // 2: a tile transforms two halves at once (both children
                     // of a forward split, both inputs of a merge): four tile
                     // buffers of shared memory instead of three
};

// Forward split pass (MODE 0): out0 = FFT(in0), out1 = FFT(P in0); either
// output may be null.  Inverse merge pass (MODE 1): out0 = IFFT(in0) +
// conj(P) IFFT(in1); in1 may be null (then out0 = IFFT(in0)).
struct PassArgs {
  PassGeom g;
  ArrMap a_in0, a_in1, a_out0, a_out1;
  const void* in0;
  const void* in1;
  void* out0;
  void* out1;
  FftDev fft;
};

constexpr int MAX_D = 6;               // split algorithm; the plain embedding takes d <= 4
constexpr int MAX_CLS = 1 << MAX_D;

struct SymDev {
  const void* data;          // store (float2 or double2)
  int d;
  int nsym;
  int compressed;            // 1: mirror-compressed parity store
  int n[MAX_D];              // level sizes of the split grid
  long long cls_off[MAX_CLS];
  long long blk[MAX_CLS];    // values per stored block in each class
  int J[MAX_CLS][MAX_D];     // box extents per class
  int comp[3][3];            // (a, b) -> stored block
  int oddmask[9];            // stored block -> dims with parity -1
};

constexpr int MAX_LEAF_NODES = 8;
struct LeafNode {
  const void* in;
  void* out;
  int prefix;                // parity bits of dims 0..d-2 (bit m for dim m)
};

struct LeafArgs {
  int N;                     // line length (n_d split, 2 n_d full)
  int c;
  int rq;                    // rhs per tile
  int Lt;                    // lines per tile
  int nrhs;
  long long lines;           // lines per (rhs, component)
  long long comp_stride;     // elements between components
  long long rhs_stride;      // elements between rhs
  int dl;                    // number of line dims (d - 1)
  int ext[MAX_D - 1];        // extents of the line dims
  int split;                 // 1: split halves f = 2 l + b; 0: full grid f = l
  int tensor;                // 1: c x c x rq contraction on tensor cores (c = 3, complex64)
  long long tiles_per_node;
  int nnodes;
  LeafNode nodes[MAX_LEAF_NODES];
  FftDev fft;
  SymDev sym;
};

// Symbol build (FP64): fold of the embedded generator for one parity class.
struct FoldArgs {
  double2* F;                // [nsym][n_1..n_d]
  const double2* t;          // device copy of the generator
  int d, c, nsym, parity_layout;
  int n[MAX_D];
  long long s;
  int pairs[9][2];           // stored block -> (a, b)
  int8_t par[3][3][MAX_D];   // parity signs (parity layout)
  int cls_bits[MAX_D];       // b_m of the class
  double scale;
};

struct StoreArgs {
  void* store;
  const double2* F;
  int d, nsym, prec;         // prec: 0 float2, 1 double2
  int n[MAX_D];
  long long s;
  long long cls_off;
  int J[MAX_D];
  long long blk;
};

// A stage of the batched persistent launch: one line pass or leaf launch of
// one problem, with the stage it waits for.
struct BatchStage {
  int kind;            // 0 forward split pass, 1 merge pass, 2 leaf, 3 no work
  int dep;             // stage index this one waits for, -1 for none
  long long item0;     // first work item of this stage
  long long tiles;     // work items (tiles) of this stage
  PassArgs pa;
  LeafArgs la;
};
struct BatchCtl {
  unsigned long long next;   // work-item dispenser
  int error;                 // 0, or BTMV_E_TIMEOUT when a wait expired
  int err_stage;             // stage whose wait expired
  int withhold;              // self test: completion count a wait never reaches
  int pad;
};

// Opt a kernel in to more than 48 KB of dynamic shared memory on the
// current device.  The attribute is per device, so the first launch on each
// device sets it (devices 0..63).
template <auto K>
inline cudaError_t set_smem_attr(int bytes) {
  static std::atomic<unsigned long long> done{0};
  int dev = 0;
  cudaGetDevice(&dev);
  const unsigned long long bit = 1ull << (dev & 63);
  if (done.load(std::memory_order_relaxed) & bit) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e == cudaSuccess) done.fetch_or(bit);
  return e;
}

// Copy between a vector of the caller's sizes nu and one of the padded sizes
// np (same [r][c][..] layout): to_pad = 1 writes every padded element (zero
// outside nu), 0 writes the nu-part back.
struct PadArgs {
  const void* src;
  void* dst;
  int d, to_pad;
  int nu[MAX_D], np[MAX_D];
  long long total;           // elements of the written vector
};
template <class T> cudaError_t launch_pad(const PadArgs& a, cudaStream_t st);

// launchers (return cudaGetLastError())
template <class T> cudaError_t launch_pass(int mode, const PassArgs& a, cudaStream_t st);
template <class T> cudaError_t launch_leaf(const LeafArgs& a, cudaStream_t st);
cudaError_t launch_fold(const FoldArgs& a, cudaStream_t st);
template <class T>
cudaError_t launch_persistent(const BatchStage* stages, int nstages, long long nitems, BatchCtl* ctl, unsigned* done,
                              long long timeout_ns, int grid, size_t smem, cudaStream_t st);
template <class T> int persistent_blocks_per_sm(size_t smem);
cudaError_t launch_store(const StoreArgs& a, cudaStream_t st);

// register-resident kernels for power-of-two lines (complex64); the
// *_supported checks say whether a launch can take them.
bool pass_reg_supported(const PassArgs& a, size_t esz);
cudaError_t launch_pass_reg(int mode, const PassArgs& a, cudaStream_t st);
// the same passes with TMA-staged input tiles and persistent blocks
// (fast_pass_tma.cu); err: device address of a word set to 1 when a bounded
// wait expired
bool pass_tma_supported(int mode, const PassArgs& a, size_t esz);
cudaError_t launch_pass_tma(int mode, const PassArgs& a, int* err, cudaStream_t st);
bool leaf_reg_supported(const LeafArgs& a, size_t esz);
cudaError_t launch_leaf_reg(const LeafArgs& a, cudaStream_t st);
// c = 3 split leaf with all components of a line in one thread group
// (fast_leaf3.cu); launch_leaf_reg takes it where supported and faster.
bool leaf3_supported(const LeafArgs& a, size_t esz);
cudaError_t launch_leaf3(const LeafArgs& a, cudaStream_t st);

size_t pass_smem_bytes(const PassGeom& g, size_t esz);
size_t leaf_smem_bytes(int N, int c, int rq, int Lt, size_t esz);

}  // namespace btmv
