// Internal plan representation and schedule helpers of libbtmv (shared by
// the per-call launcher, btmv.cu, and the batched persistent launcher,
// batch.cu).  Not part of the C ABI.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <memory>
#include <vector>

#include "../../include/btmv.h"
#include "kernels.cuh"

namespace btmv {

// Device allocation shared by reference count (twiddle tables and symbol
// stores are shared between a plan and its clones).
struct DevBuf {
  void* ptr = nullptr;
  explicit DevBuf(void* p) : ptr(p) {}
  ~DevBuf() { if (ptr) cudaFree(ptr); }
};

struct TableSet {
  void* mem = nullptr;                 // device
  std::shared_ptr<DevBuf> owner;
  std::map<int, size_t> off_f, off_d;  // N -> byte offset of [tw N][ph N]
  size_t bytes = 0;
};

}  // namespace btmv

// The opaque plan of the C ABI (global namespace, as declared in btmv.h).
struct btmv_plan_s {
  int d = 0, c = 0, prec = 0, algo = 0, max_rhs = 0;
  uint32_t flags = 0;
  int n[btmv::MAX_D] = {1, 1, 1, 1, 1, 1};
  long long s = 1;          // prod n
  // sizes the caller uses.  A split plan whose sizes are not all 7-smooth
  // runs on the operator zero-padded to the next 7-smooth sizes (n above);
  // x and y are copied into and out of the padded buffers around the apply
  int nu[btmv::MAX_D] = {1, 1, 1, 1, 1, 1};
  long long su = 1;         // prod nu
  bool padded = false;
  void* xpad = nullptr;
  void* ypad = nullptr;
  long long s2 = 1;         // prod 2n
  size_t esz = 8;           // bytes per complex
  int dev = 0;
  int nsm = 0;              // SMs of dev
  btmv::TableSet tab;
  btmv::FftDev fft_apply[btmv::MAX_D];  // per dim, plan precision (N = n_m split, 2 n_m full)
  btmv::FftDev fft_sym[btmv::MAX_D];    // per dim, FP64, N = n_m
  // symbol
  void* sym = nullptr;
  std::shared_ptr<btmv::DevBuf> sym_owner;
  size_t sym_bytes = 0;
  btmv::SymDev symdev;
  bool has_sym = false;
  int nsym = 0;
  int compressed = 0;
  // workspace
  void* ws = nullptr;
  size_t ws_bytes = 0;
  std::vector<void*> W;     // split: d-1 vectors; full: Z
  // two-stream schedule (BTMV_FLAG_TWO_STREAMS): workspace of the second
  // top-level subtree, its stream and the fork / join events
  void* ws2 = nullptr;
  std::vector<void*> W2;
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  // BTMV_ALGO_FULL_CUFFT: the cuFFT plan (cufftHandle) of one right-hand side
  int cufft = 0;
  bool has_cufft = false;
  // TMA-staged passes: host-mapped word the kernels set when a bounded wait
  // expired (read and cleared by the next pass launch on the host)
  int* tma_err_host = nullptr;
  int* tma_err_dev = nullptr;
  // host staging
  void* stage_x = nullptr;
  void* stage_y = nullptr;
  // btmv_apply_host_async: two staging slots used in turn, the copy streams
  // and per-slot events (copy in done, apply done, copy out done)
  void* ring_x[2] = {nullptr, nullptr};
  void* ring_y[2] = {nullptr, nullptr};
  cudaStream_t cp_in = nullptr, cp_out = nullptr;
  cudaEvent_t ev_in[2] = {nullptr, nullptr}, ev_comp[2] = {nullptr, nullptr}, ev_out[2] = {nullptr, nullptr};
  long long pipe_k = 0;
  // profiling
  struct Rec { int kind; cudaEvent_t a, b; };
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> pool;
  double acc_ms[BTMV_K_NKINDS] = {0};
  int64_t acc_n[BTMV_K_NKINDS] = {0};
  int launches = 0;
  // BTMV_FLAG_PROFILE: events around the launches of one apply in every
  // prof_every (environment BTMV_PROFILE_EVERY, default 1)
  int prof_every = 1;
  long long prof_count = 0;
  bool prof_on = false;
};

namespace btmv {

// One launch of the depth-first schedule of Algorithm 1.
struct Step {
  int kind;            // 0 forward split pass, 1 merge pass, 2 leaf,
                       // 3 the last two levels fused (node in0/out0, scratch out1,
                       // parity prefix nodes[0].prefix; per-call launcher only)
  int dim;             // level (dimension) of a pass
  const void* in0;
  const void* in1;
  void* out0;
  void* out1;
  int nn;              // leaf: number of nodes
  LeafNode nodes[2];
};

btmv_status fail(btmv_status st, const char* fmt, ...);
// Radix factorisation of N into stages: mode 0 prefers radix 16, mode 1 radix 8.
bool factor_radices_mode(int N, FftDev& f, int mode);
// Steps of one split apply on device pointers (d >= 1); fuse: the last two
// levels as kind-3 steps where two_level_fusable(p).
void split_steps(btmv_plan p, const void* x, void* y, std::vector<Step>& out, bool fuse = false);
// BTMV_FLAG_FUSED_LEVELS is set and the plan's shape has a fused kernel.
bool two_level_fusable(btmv_plan p);
// ... and an apply with nrhs right-hand sides into y takes it (grid size and
// alignment rules of btmv.h).
bool fuse_this_apply(btmv_plan p, int nrhs, const void* y);
// The fused last two levels (fused2.cu): d >= 3, c = 3, complex64, block-
// symmetric compressed store, n_{d-2} = n_{d-1} = 64.
bool fuse2_supported(int d, int c, const int* n, size_t esz, const SymDev& S);
cudaError_t launch_fuse2(float2* node, float2* scratch, int prefix, int d, const int* n, int nrhs,
                         const FftDev& f1, const FftDev& f2, const SymDev& sym, cudaStream_t st);
// The same for n_{d-2} = n_{d-1} = 128 on a 16-CTA cluster per slab
// (fused2c.cu); available: the current device schedules that cluster.
bool fuse2c_supported(int d, int c, const int* n, size_t esz, const SymDev& S);
bool fuse2c_available();
long long fuse2c_clusters(int d, const int* n, int nrhs);
cudaError_t launch_fuse2c(float2* node, float2* scratch, int prefix, int d, const int* n, int nrhs,
                          const FftDev& f1, const FftDev& f2, const SymDev& sym, cudaStream_t st);
// The whole apply of a d = 2, c = 1, 64 x 64 split plan as one cluster
// kernel (small2d.cu); dbl: complex128.
bool small2d_supported(int d, int c, const int* n, const SymDev& S);
cudaError_t launch_small2d(const void* x, void* y, int nrhs, bool dbl, const FftDev& f, const SymDev& sym,
                           cudaStream_t st);
// The plan's applies take launch_small2d.
bool use_small2d(btmv_plan p);
// Arguments of a split pass step; TL = 0 picks the default tile.
PassArgs split_pass_args(btmv_plan p, const Step& s, int nrhs, size_t esz, int TL);
// Arguments of a leaf step; Lt, rq = 0 pick the defaults.
LeafArgs leaf_step_args(btmv_plan p, int nrhs, int nn, const LeafNode* nodes, bool full, size_t esz, int Lt, int rq);
// Drop every cached batch that refers to plan p (called by btmv_destroy).
void batch_forget_plan(btmv_plan p);
// BTMV_ALGO_FULL_CUFFT (cufft_full.cu): cuFFT plan set-up / release, apply.
btmv_status cufft_plan_setup(btmv_plan p);
void cufft_plan_destroy(btmv_plan p);
btmv_status cufft_full_apply(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st);

}  // namespace btmv
