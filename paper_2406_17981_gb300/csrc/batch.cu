// btmv_apply_batched: many independent split applies per call, replayed from
// a CUDA graph captured once per argument set, in one of two execution modes
// chosen per problem mix by an autotuner:
//
//   mode 0  ONE persistent kernel launch (k_persistent).  Each problem
//           contributes the steps of its depth-first schedule (the same steps
//           btmv_apply launches one by one) as a chain of stages, each
//           waiting for the previous one of the same problem.  Stages are
//           ordered step-slot by step-slot across problems, so different
//           problems' passes run side by side on the GPU while each problem
//           keeps the (d+1)-vector peak of its plan.  It runs the generic
//           shared-memory line bodies.
//   mode 1  one graph whose parallel branches (16, 4 or 1) run the problems'
//           own register-kernel launches, largest problems first.
//
// The autotuner times both: for mode 0 a small coordinate descent over the
// tile sizes and radix order of the line bodies, for mode 1 each branch
// count, with CUDA events on the caller's data; it keeps the winner for the
// process and, when the environment variable BTMV_TUNE_CACHE names a file, in
// that file.  On mixes of large problems mode 1 wins (the register kernels
// are specialised per line length); BTMV_NO_AUTOTUNE with BTMV_BATCH_MODE=0|1
// fixes the mode.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/btmv.h"
#include "kernels.cuh"
#include "plan.h"

btmv_status btmv_check_apply_args(btmv_plan p, const void* x, void* y, int nrhs);
btmv_status btmv_apply_on_device(btmv_plan p, const void* x, void* y, int nrhs, cudaStream_t st);
int btmv_is_device_ptr(const void* ptr);

using namespace btmv;

namespace {

constexpr int kBranchStreams = 16;

struct TuneCfg {
  int mode = 0;    // 0: one persistent kernel; 1: graph with one branch per problem
  int TL = 0;      // strided-pass tile lines (0 = default)
  int Lt = 0;      // leaf lines per tile (0 = default)
  int rq = 0;      // leaf right-hand sides per tile (0 = default)
  int radix = 0;   // 0: radix-16 first, 1: radix-8 first
  int nbr = 16;    // mode 1: parallel branches (problems placed largest first)
  std::string str() const {
    char b[80];
    snprintf(b, sizeof b, "%d %d %d %d %d %d", mode, TL, Lt, rq, radix, nbr);
    return b;
  }
};

struct Entry {
  std::vector<btmv_plan> plans;
  std::vector<const void*> x;
  std::vector<void*> y;
  std::vector<int> nrhs;
  int prec = 0;
  TuneCfg cfg;
  BatchStage* d_stages = nullptr;
  unsigned char* d_ctl = nullptr;     // BatchCtl, then done[nstages]
  int nstages = 0;
  long long nitems = 0;
  size_t smem = 0;
  int grid = 0;
  int* h_err = nullptr;               // pinned copy of ctl->error after each launch
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t ev = nullptr;
  // mode 1: branch streams and fork / join events
  cudaStream_t bst[kBranchStreams] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kBranchStreams] = {};
  bool launched = false;
  unsigned long long lru = 0;
  int cfg_mode = 0;                   // mode of the stage table / graph in place
  int cfg_nbr = 1;                    // mode 1: branches in use
  std::vector<int> branch;            // mode 1: branch of each problem
  int kernels = 0;                    // kernel nodes of the captured graph
  void* h_err_dev() const { return &((BatchCtl*)d_ctl)->error; }
};

std::mutex g_mu;
std::vector<Entry*> g_cache;
std::map<std::string, TuneCfg> g_tuned;
unsigned long long g_clock = 0;
bool g_tune_loaded = false;

void free_entry(Entry* e) {
  if (e->ev) { cudaEventSynchronize(e->ev); cudaEventDestroy(e->ev); }
  for (int i = 0; i < kBranchStreams; ++i) {
    if (e->bst[i]) cudaStreamDestroy(e->bst[i]);
    if (e->join[i]) cudaEventDestroy(e->join[i]);
  }
  if (e->fork) cudaEventDestroy(e->fork);
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->d_stages) cudaFree(e->d_stages);
  if (e->d_ctl) cudaFree(e->d_ctl);
  if (e->h_err) cudaFreeHost(e->h_err);
  delete e;
}

long long timeout_ns() {
  const char* v = getenv("BTMV_WAIT_TIMEOUT_MS");
  long long ms = v ? atoll(v) : 5000;
  if (ms <= 0) ms = 5000;
  return ms * 1000000LL;
}

std::string signature(const Entry& e) {
  std::string s;
  char b[96];
  for (size_t i = 0; i < e.plans.size(); ++i) {
    const btmv_plan p = e.plans[i];
    snprintf(b, sizeof b, "%d:%d,%d,%d,%d:%d:%d:%d|", p->d, p->n[0], p->n[1], p->n[2], p->n[3], p->c, p->prec, e.nrhs[i]);
    s += b;
  }
  return s;
}

void load_tune_file() {
  if (g_tune_loaded) return;
  g_tune_loaded = true;
  const char* path = getenv("BTMV_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "r");
  if (!f) return;
  char line[1 << 16];
  while (fgets(line, sizeof line, f)) {
    char* tab = strchr(line, '\t');
    if (!tab) continue;
    *tab = 0;
    TuneCfg c;
    if (sscanf(tab + 1, "%d %d %d %d %d %d", &c.mode, &c.TL, &c.Lt, &c.rq, &c.radix, &c.nbr) == 6 && c.nbr >= 1 &&
        c.nbr <= kBranchStreams)
      g_tuned[line] = c;
  }
  fclose(f);
}

void save_tune(const std::string& sig, const TuneCfg& c) {
  const char* path = getenv("BTMV_TUNE_CACHE");
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s\t%s\n", sig.c_str(), c.str().c_str());
  fclose(f);
}

void apply_radix(FftDev& f, int mode) {
  FftDev g = f;
  if (factor_radices_mode(f.N, g, mode)) {
    f.nst = g.nst;
    for (int i = 0; i < MAX_STAGES; ++i) f.rad[i] = g.rad[i];
  }
}

// Stage table of the batch for one tuning choice (host side).
btmv_status build_stages(const Entry& e, const TuneCfg& cfg, std::vector<BatchStage>& out, size_t& smem) {
  out.clear();
  smem = 0;
  const size_t esz = e.prec == BTMV_C64 ? sizeof(float2) : sizeof(double2);
  std::vector<std::vector<Step>> steps(e.plans.size());
  size_t slots = 0;
  for (size_t i = 0; i < e.plans.size(); ++i) {
    if (e.nrhs[i] == 0) continue;
    split_steps(e.plans[i], e.x[i], e.y[i], steps[i]);
    slots = std::max(slots, steps[i].size());
  }
  std::vector<int> last(e.plans.size(), -1);
  long long item = 0;
  for (size_t sl = 0; sl < slots; ++sl) {
    for (size_t i = 0; i < e.plans.size(); ++i) {
      if (sl >= steps[i].size()) continue;
      const Step& s = steps[i][sl];
      const btmv_plan p = e.plans[i];
      if (s.kind > 2) return fail(BTMV_E_STATE, "batch: step kind %d has no batched form", s.kind);
      BatchStage bs;
      memset(&bs, 0, sizeof bs);
      bs.kind = s.kind;
      bs.dep = last[i];
      if (s.kind == 2) {
        bs.la = leaf_step_args(p, e.nrhs[i], s.nn, s.nodes, false, esz, cfg.Lt, cfg.rq);
        apply_radix(bs.la.fft, cfg.radix);
        bs.tiles = bs.la.tiles_per_node * bs.la.nnodes;
        smem = std::max(smem, leaf_smem_bytes(bs.la.N, bs.la.c, bs.la.rq, bs.la.Lt, esz));
      } else {
        bs.pa = split_pass_args(p, s, e.nrhs[i], esz, cfg.TL);
        apply_radix(bs.pa.fft, cfg.radix);
        bs.tiles = (bs.pa.g.lines + bs.pa.g.TL - 1) / bs.pa.g.TL;
        smem = std::max(smem, pass_smem_bytes(bs.pa.g, esz));
      }
      bs.item0 = item;
      item += bs.tiles;
      last[i] = (int)out.size();
      out.push_back(bs);
    }
  }
  return BTMV_OK;
}

// Mode 1 placement: problems in decreasing order of vector bytes, each to
// the branch with the least bytes so far (longest-processing-time first).
void place_branches(Entry& e, int nbr) {
  const int n = (int)e.plans.size();
  nbr = std::max(1, std::min(nbr, std::min(kBranchStreams, std::max(1, n))));
  e.cfg_nbr = nbr;
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  auto bytes = [&](int i) {
    double v = (double)e.nrhs[i] * e.plans[i]->c * (e.prec ? 16.0 : 8.0);
    for (int m = 0; m < e.plans[i]->d; ++m) v *= e.plans[i]->n[m];
    return v;
  };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return bytes(a) > bytes(b); });
  std::vector<double> load(nbr, 0.0);
  e.branch.assign(n, 0);
  for (int i : order) {
    const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    e.branch[i] = k;
    load[k] += bytes(i);
  }
}

btmv_status upload(Entry& e, const TuneCfg& cfg) {
  e.cfg_mode = cfg.mode;
  if (cfg.mode == 1) place_branches(e, cfg.nbr);
  std::vector<BatchStage> st;
  size_t smem = 0;
  if (cfg.mode == 0) build_stages(e, cfg, st, smem);
  if (e.d_stages) { cudaFree(e.d_stages); e.d_stages = nullptr; }
  if (e.d_ctl) { cudaFree(e.d_ctl); e.d_ctl = nullptr; }
  e.nstages = (int)st.size();
  e.nitems = st.empty() ? 0 : st.back().item0 + st.back().tiles;
  e.smem = smem;
  cudaError_t ce = cudaMalloc(&e.d_stages, std::max<size_t>(1, st.size()) * sizeof(BatchStage));
  if (ce != cudaSuccess) return fail(BTMV_E_NOMEM, "apply_batched: stage table: %s", cudaGetErrorString(ce));
  ce = cudaMalloc(&e.d_ctl, sizeof(BatchCtl) + std::max<size_t>(1, st.size()) * sizeof(unsigned));
  if (ce != cudaSuccess) return fail(BTMV_E_NOMEM, "apply_batched: control words: %s", cudaGetErrorString(ce));
  if (!st.empty()) {
    ce = cudaMemcpy(e.d_stages, st.data(), st.size() * sizeof(BatchStage), cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: stage upload: %s", cudaGetErrorString(ce));
  }
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int per = e.prec == BTMV_C64 ? persistent_blocks_per_sm<float2>(smem) : persistent_blocks_per_sm<double2>(smem);
  e.grid = (int)std::max<long long>(1, std::min<long long>(e.nitems, (long long)std::max(1, per) * sms));
  return BTMV_OK;
}

// Mode 1: every problem's own schedule (register-resident kernels where they
// apply) on one of kBranchStreams streams forked from st and joined back.
btmv_status enqueue_branches(Entry& e, cudaStream_t st) {
  if (!e.fork) {
    if (cudaEventCreateWithFlags(&e.fork, cudaEventDisableTiming) != cudaSuccess)
      return fail(BTMV_E_CUDA, "apply_batched: fork event");
    for (int i = 0; i < kBranchStreams; ++i)
      if (cudaStreamCreateWithFlags(&e.bst[i], cudaStreamNonBlocking) != cudaSuccess ||
          cudaEventCreateWithFlags(&e.join[i], cudaEventDisableTiming) != cudaSuccess)
        return fail(BTMV_E_CUDA, "apply_batched: branch streams");
  }
  cudaEventRecord(e.fork, st);
  const int nb = e.cfg_nbr;
  for (int i = 0; i < nb; ++i) cudaStreamWaitEvent(e.bst[i], e.fork, 0);
  for (size_t i = 0; i < e.plans.size(); ++i) {
    if (!e.nrhs[i]) continue;
    btmv_status s = btmv_apply_on_device(e.plans[i], e.x[i], e.y[i], e.nrhs[i], e.bst[e.branch[i]]);
    if (s != BTMV_OK) return s;
  }
  for (int i = 0; i < nb; ++i) {
    cudaEventRecord(e.join[i], e.bst[i]);
    cudaStreamWaitEvent(st, e.join[i], 0);
  }
  cudaError_t ce = cudaMemsetAsync(e.h_err_dev(), 0, sizeof(int), st);
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: status reset: %s", cudaGetErrorString(ce));
  ce = cudaMemcpyAsync(e.h_err, e.h_err_dev(), sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: status copy: %s", cudaGetErrorString(ce));
  return BTMV_OK;
}

// Enqueue one run: reset the control words, launch, copy the error word back.
btmv_status enqueue(Entry& e, cudaStream_t st) {
  if (e.cfg_mode == 1) return enqueue_branches(e, st);
  const size_t ctl_bytes = sizeof(BatchCtl) + std::max(1, e.nstages) * sizeof(unsigned);
  cudaError_t ce = cudaMemsetAsync(e.d_ctl, 0, ctl_bytes, st);
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: reset: %s", cudaGetErrorString(ce));
  if (e.nitems > 0) {
    BatchCtl* ctl = (BatchCtl*)e.d_ctl;
    unsigned* done = (unsigned*)(e.d_ctl + sizeof(BatchCtl));
    ce = e.prec == BTMV_C64
             ? launch_persistent<float2>(e.d_stages, e.nstages, e.nitems, ctl, done, timeout_ns(), e.grid, e.smem, st)
             : launch_persistent<double2>(e.d_stages, e.nstages, e.nitems, ctl, done, timeout_ns(), e.grid, e.smem, st);
    if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: persistent launch: %s", cudaGetErrorString(ce));
  }
  ce = cudaMemcpyAsync(e.h_err, &((BatchCtl*)e.d_ctl)->error, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: status copy: %s", cudaGetErrorString(ce));
  return BTMV_OK;
}

float time_cfg(Entry& e, const TuneCfg& cfg, cudaStream_t st) {
  if (upload(e, cfg) != BTMV_OK) return 1e30f;
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  float best = 1e30f;
  if (enqueue(e, st) == BTMV_OK) {
    for (int r = 0; r < 2; ++r) {
      cudaEventRecord(a, st);
      if (enqueue(e, st) != BTMV_OK) break;
      cudaEventRecord(b, st);
      cudaEventSynchronize(b);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, a, b);
      if (*e.h_err) { ms = 1e30f; }
      best = std::min(best, ms);
    }
  }
  cudaStreamSynchronize(st);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return best;
}

// Execution mode first (persistent kernel or graph branches), then
// coordinate descent over tile lines, leaf lines, leaf rhs and radix order
// for the persistent kernel.
TuneCfg autotune(Entry& e, cudaStream_t st) {
  TuneCfg best;
  float bt = time_cfg(e, best, st);
  // graph of branches: 16, 4 or 1 parallel branches
  TuneCfg br;
  br.mode = 1;
  float tb = 1e30f;
  for (int nb : {16, 4, 1}) {
    TuneCfg c = br;
    c.nbr = nb;
    const float t = time_cfg(e, c, st);
    if (t < tb) { tb = t; br = c; }
  }
  if (tb < bt) return br;
  int maxr = 1;
  for (int r : e.nrhs) maxr = std::max(maxr, r);
  const std::vector<std::vector<int>> cand = {{8, 16, 32}, {1, 2, 4, 8}, {1, 2, 4, 8, 16}, {0, 1}};
  for (int axis = 0; axis < 4; ++axis) {
    for (int v : cand[axis]) {
      TuneCfg c = best;
      if (axis == 0) c.TL = v;
      if (axis == 1) c.Lt = v;
      if (axis == 2) { if (v > maxr) continue; c.rq = v; }
      if (axis == 3) c.radix = v;
      if (c.str() == best.str()) continue;
      const float t = time_cfg(e, c, st);
      if (t < bt) { bt = t; best = c; }
    }
  }
  return best;
}

btmv_status capture(Entry& e, cudaStream_t user) {
  cudaStream_t cs = nullptr;
  cudaError_t ce = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: capture stream: %s", cudaGetErrorString(ce));
  cudaGraph_t g = nullptr;
  ce = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  btmv_status s = ce == cudaSuccess ? enqueue(e, cs) : fail(BTMV_E_CUDA, "apply_batched: begin capture: %s",
                                                           cudaGetErrorString(ce));
  ce = cudaStreamEndCapture(cs, &g);
  cudaStreamDestroy(cs);
  if (s != BTMV_OK) { if (g) cudaGraphDestroy(g); return s; }
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: end capture: %s", cudaGetErrorString(ce));
  size_t nn = 0;
  e.kernels = 0;
  if (cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
    std::vector<cudaGraphNode_t> nodes(nn);
    if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess)
      for (size_t i = 0; i < nn; ++i) {
        cudaGraphNodeType ty;
        if (cudaGraphNodeGetType(nodes[i], &ty) == cudaSuccess && ty == cudaGraphNodeTypeKernel) ++e.kernels;
      }
  }
  ce = cudaGraphInstantiate(&e.exec, g, 0);
  cudaGraphDestroy(g);
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: instantiate: %s", cudaGetErrorString(ce));
  (void)user;
  return BTMV_OK;
}

Entry* find_entry(int count, const btmv_plan* plans, const void* const* x, void* const* y, const int* nrhs) {
  for (Entry* e : g_cache) {
    if ((int)e->plans.size() != count) continue;
    bool same = true;
    for (int i = 0; i < count && same; ++i)
      same = e->plans[i] == plans[i] && e->x[i] == x[i] && e->y[i] == y[i] && e->nrhs[i] == nrhs[i];
    if (same) return e;
  }
  return nullptr;
}

}  // namespace

void btmv::batch_forget_plan(btmv_plan p) {
  std::lock_guard<std::mutex> lk(g_mu);
  for (size_t i = 0; i < g_cache.size();) {
    Entry* e = g_cache[i];
    if (std::find(e->plans.begin(), e->plans.end(), p) != e->plans.end()) {
      free_entry(e);
      g_cache.erase(g_cache.begin() + i);
    } else {
      ++i;
    }
  }
}

extern "C" BTMV_API btmv_status btmv_apply_batched(int count, const btmv_plan* plans, const void* const* x,
                                                   void* const* y, const int* nrhs, void* stream) {
  if (count < 0) return fail(BTMV_E_ARG, "apply_batched: count < 0");
  if (count == 0) return BTMV_OK;
  if (!plans || !x || !y || !nrhs) return fail(BTMV_E_ARG, "apply_batched: NULL array");
  bool persistent = true;
  for (int i = 0; i < count; ++i) {
    btmv_status s = btmv_check_apply_args(plans[i], x[i], y[i], nrhs[i]);
    if (s != BTMV_OK) return s;
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(BTMV_E_ARG, "apply_batched: plan %d repeated at %d", j, i);
    if (nrhs[i] && (!btmv_is_device_ptr(x[i]) || !btmv_is_device_ptr(y[i])))
      return fail(BTMV_E_ARG, "apply_batched: entry %d is not a device pointer", i);
    if (plans[i]->algo != BTMV_ALGO_SPLIT || plans[i]->prec != plans[0]->prec || plans[i]->padded) persistent = false;
  }
  cudaStream_t st = (cudaStream_t)stream;
  if (getenv("BTMV_BATCH_DIRECT")) {
    // argument sets that change every call (serving ticks): fork every
    // problem's schedule onto a pool of streams and join, without a graph
    // (streams and events belong to a device: one pool per device)
    constexpr int kMaxDev = 64;
    static std::mutex mu;
    static cudaStream_t pools[kMaxDev][kBranchStreams] = {};
    static cudaEvent_t forks[kMaxDev] = {}, joins[kMaxDev][kBranchStreams] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev)
      return fail(BTMV_E_CUDA, "apply_batched: current device");
    std::lock_guard<std::mutex> lk(mu);
    cudaStream_t* pool = pools[dev];
    cudaEvent_t* join = joins[dev];
    cudaEvent_t& fork = forks[dev];
    if (!fork) {
      if (cudaEventCreateWithFlags(&fork, cudaEventDisableTiming) != cudaSuccess)
        return fail(BTMV_E_CUDA, "apply_batched: fork event");
      for (int i = 0; i < kBranchStreams; ++i)
        if (cudaStreamCreateWithFlags(&pool[i], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming) != cudaSuccess)
          return fail(BTMV_E_CUDA, "apply_batched: branch streams");
    }
    const int nb = std::min(kBranchStreams, count);
    cudaEventRecord(fork, st);
    for (int i = 0; i < nb; ++i) cudaStreamWaitEvent(pool[i], fork, 0);
    for (int i = 0; i < count; ++i)
      if (nrhs[i]) {
        btmv_status s = btmv_apply_on_device(plans[i], x[i], y[i], nrhs[i], pool[i % nb]);
        if (s != BTMV_OK) return s;
      }
    for (int i = 0; i < nb; ++i) {
      cudaEventRecord(join[i], pool[i]);
      cudaStreamWaitEvent(st, join[i], 0);
    }
    return BTMV_OK;
  }
  if (!persistent || getenv("BTMV_BATCH_SEQUENTIAL")) {
    // mixed precisions or plain-embedding plans: one apply after the other
    for (int i = 0; i < count; ++i)
      if (nrhs[i]) {
        btmv_status s = btmv_apply_on_device(plans[i], x[i], y[i], nrhs[i], st);
        if (s != BTMV_OK) return s;
      }
    return BTMV_OK;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  load_tune_file();
  Entry* e = find_entry(count, plans, x, y, nrhs);
  if (e) {
    // a finished previous launch of this batch reports a wait that expired
    // there; an unfinished one is ordered before this launch on the stream
    if (cudaEventQuery(e->ev) == cudaSuccess) {
      if (*e->h_err) {
        const int err = *e->h_err;
        *e->h_err = 0;
        return fail((btmv_status)err, "apply_batched: a previous launch of this batch hit its wait limit");
      }
    } else {
      cudaGetLastError();
      cudaStreamWaitEvent(st, e->ev, 0);
    }
  } else {
    e = new Entry();
    e->plans.assign(plans, plans + count);
    e->x.assign(x, x + count);
    e->y.assign(y, y + count);
    e->nrhs.assign(nrhs, nrhs + count);
    e->prec = plans[0]->prec;
    if (cudaHostAlloc((void**)&e->h_err, sizeof(int), cudaHostAllocDefault) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->ev, cudaEventDisableTiming) != cudaSuccess) {
      free_entry(e);
      return fail(BTMV_E_NOMEM, "apply_batched: pinned status word");
    }
    *e->h_err = 0;
    const std::string sig = signature(*e);
    auto it = g_tuned.find(sig);
    if (getenv("BTMV_NO_AUTOTUNE")) {
      e->cfg = TuneCfg();
      const char* m = getenv("BTMV_BATCH_MODE");
      e->cfg.mode = (m && atoi(m) == 1) ? 1 : 0;
    } else if (it != g_tuned.end()) {
      e->cfg = it->second;
    } else {
      e->cfg = autotune(*e, st);
      g_tuned[sig] = e->cfg;
      save_tune(sig, e->cfg);
    }
    btmv_status s = upload(*e, e->cfg);
    if (s == BTMV_OK) s = capture(*e, st);
    if (s != BTMV_OK) { free_entry(e); return s; }
    if (g_cache.size() >= 32) {
      auto old = std::min_element(g_cache.begin(), g_cache.end(),
                                  [](const Entry* a, const Entry* b) { return a->lru < b->lru; });
      free_entry(*old);
      g_cache.erase(old);
    }
    g_cache.push_back(e);
  }
  e->lru = ++g_clock;
  cudaError_t ce = cudaGraphLaunch(e->exec, st);
  if (ce != cudaSuccess) return fail(BTMV_E_CUDA, "apply_batched: graph launch: %s", cudaGetErrorString(ce));
  cudaEventRecord(e->ev, st);
  e->launched = true;
  return BTMV_OK;
}

extern "C" BTMV_API btmv_status btmv_batch_tuning(int count, const btmv_plan* plans, const void* const* x,
                                                  void* const* y, const int* nrhs, int* cfg_out) {
  if (!plans || !x || !y || !nrhs || !cfg_out) return fail(BTMV_E_ARG, "batch_tuning: NULL argument");
  std::lock_guard<std::mutex> lk(g_mu);
  Entry* e = find_entry(count, plans, x, y, nrhs);
  if (!e) return fail(BTMV_E_STATE, "batch_tuning: no batch with these arguments has run");
  cfg_out[7] = e->cfg.mode;
  cfg_out[0] = e->cfg.TL; cfg_out[1] = e->cfg.Lt; cfg_out[2] = e->cfg.rq; cfg_out[3] = e->cfg.radix;
  cfg_out[4] = e->cfg.mode == 1 ? e->kernels : e->nstages; cfg_out[5] = (int)std::min<long long>(e->nitems, 0x7fffffff);
  cfg_out[6] = e->cfg.mode == 1 ? e->cfg_nbr : e->grid;
  return BTMV_OK;
}

extern "C" BTMV_API btmv_status btmv_selftest_wait_timeout(int timeout_ms, void* stream) {
  // stage 0 has no items and a withheld completion count, so the single item
  // of stage 1 (a no-op) waits on a count nothing ever reaches
  cudaStream_t st = (cudaStream_t)stream;
  std::vector<BatchStage> s(2);
  memset(s.data(), 0, 2 * sizeof(BatchStage));
  s[0].kind = 3; s[0].dep = -1; s[0].item0 = 0; s[0].tiles = 0;
  s[1].kind = 3; s[1].dep = 0; s[1].item0 = 0; s[1].tiles = 1;
  BatchStage* d = nullptr;
  unsigned char* ctl = nullptr;
  int* h = nullptr;
  btmv_status ret = BTMV_OK;
  if (cudaMalloc(&d, 2 * sizeof(BatchStage)) != cudaSuccess ||
      cudaMalloc(&ctl, sizeof(BatchCtl) + 2 * sizeof(unsigned)) != cudaSuccess ||
      cudaHostAlloc((void**)&h, sizeof(int), cudaHostAllocDefault) != cudaSuccess) {
    ret = fail(BTMV_E_NOMEM, "selftest_wait_timeout: allocation");
  } else {
    BatchCtl c0;
    memset(&c0, 0, sizeof c0);
    c0.withhold = 1;
    cudaMemcpy(d, s.data(), 2 * sizeof(BatchStage), cudaMemcpyHostToDevice);
    cudaMemset(ctl, 0, sizeof(BatchCtl) + 2 * sizeof(unsigned));
    cudaMemcpy(ctl, &c0, sizeof c0, cudaMemcpyHostToDevice);
    cudaError_t ce = launch_persistent<float2>(d, 2, 1, (BatchCtl*)ctl, (unsigned*)(ctl + sizeof(BatchCtl)),
                                               (long long)std::max(1, timeout_ms) * 1000000LL, 1, 0, st);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h, &((BatchCtl*)ctl)->error, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(st);
    if (ce != cudaSuccess) ret = fail(BTMV_E_CUDA, "selftest_wait_timeout: %s", cudaGetErrorString(ce));
    else if (*h == BTMV_E_TIMEOUT) ret = fail(BTMV_E_TIMEOUT, "selftest_wait_timeout: the bounded wait expired as intended");
    else ret = fail(BTMV_E_STATE, "selftest_wait_timeout: the wait did not report a timeout");
  }
  if (d) cudaFree(d);
  if (ctl) cudaFree(ctl);
  if (h) cudaFreeHost(h);
  return ret;
}
