/*
 * btmv.h -- d-level block Toeplitz matrix-vector product y = T x on one GPU,
 *           by the lazy-embedding / eager-projection split FFT of
 *           Siron & Molesky, "A Split Fast Fourier Transform Algorithm for
 *           Block Toeplitz Matrix-Vector Multiplication" (arXiv 2406.17981).
 *
 * The operation (Sec. I, "extending the diagonal bands"): T has d levels of
 * Toeplitz structure with c x c blocks generated by t_ab[p],
 * p_m in [-(n_m - 1), n_m - 1]; block (i, j) holds t[i - j], so
 *
 *     y_a[i] = sum_b sum_j t_ab[i - j] x_b[j],   i, j in [0,n_1) x ... x [0,n_d).
 *
 * The split method (Sec. II.A-B, Algorithm 1) never forms the 2^d-times larger
 * circulant embedding: along each level the doubled transform is computed as
 * its even half FFT_n(v) and its odd half FFT_n(P v), P[k] = exp(-i pi k/n),
 * recursively; each leaf multiplies by its 2^-d part S_b[l] = S[2l + b] of
 * the transformed embedded generator, and the halves are
 * merged back as v_even + conj(P) v_odd right after each inverse transform.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Complex numbers are interleaved (re, im): float2 for BTMV_C64, double2
 *   for BTMV_C128.  Generators are always given in double precision.
 * - Vectors x and y are laid out [nrhs][c][n_1]...[n_d], last index fastest,
 *   contiguous, 16-byte aligned.  They may be device pointers (cudaMalloc,
 *   torch tensors) or host pointers (pinned or pageable); host pointers are
 *   staged through device buffers owned by the plan.
 * - Streams are passed as void* (a cudaStream_t; NULL is the legacy default
 *   stream).  Work on device pointers is enqueued asynchronously.
 * - Every call returns a btmv_status.  On failure, btmv_last_error() gives
 *   a message for the calling thread.  Asynchronous device errors surface on
 *   the next call that synchronises or checks the stream.
 * - A plan may be used by one stream at a time.
 */
#ifndef BTMV_H
#define BTMV_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define BTMV_API __attribute__((visibility("default")))
#else
#define BTMV_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct btmv_plan_s* btmv_plan;

typedef enum {
  BTMV_OK = 0,
  BTMV_E_ARG = 1,          /* invalid argument (null, size, alias, layout) */
  BTMV_E_NOMEM = 2,        /* device or host allocation failed             */
  BTMV_E_CUDA = 3,         /* a CUDA runtime call or kernel launch failed  */
  BTMV_E_STATE = 4,        /* call out of order (apply before set_kernel)  */
  BTMV_E_UNSUPPORTED = 5,  /* size / combination not supported             */
  BTMV_E_TIMEOUT = 6       /* a bounded device-side wait expired           */
} btmv_status;

/* precision of vectors, symbol and arithmetic */
enum { BTMV_C64 = 0, BTMV_C128 = 1 };

/* algorithm */
enum {
  BTMV_ALGO_SPLIT = 0,     /* Algorithm 1: lazy embedding, eager projection      */
  BTMV_ALGO_FULL = 1,      /* plain full 2^d circulant embedding (Sec. I), own
                              kernels; for comparison                          */
  BTMV_ALGO_FULL_CUFFT = 2 /* the same embedding with cuFFT transforms (own pad,
                              multiply and projection kernels); d <= 3; cuFFT
                              is loaded at run time (dlopen) by the first such
                              plan; for comparison only                       */
};

/* symmetry flags for btmv_set_kernel (may be OR-ed) */
enum {
  BTMV_SYM_NONE = 0,
  BTMV_SYM_BLOCK = 1,      /* t_ab = t_ba: only blocks a <= b are read/stored   */
  BTMV_SYM_PARITY = 2,     /* per-(block, dim) parity t(-p_m) = +-t(p_m): the
                              generator is given on the non-negative orthant and
                              the symbol is stored mirror-compressed (Sec. II.C) */
  BTMV_SYM_ADJOINT = 4     /* build the symbol of the conjugate transpose T^H
                              (generator t^H_ab[p] = conj(t_ba[-p]); the other
                              flags and parity describe the t passed in), for
                              BiCG-type solvers.  The paper has no adjoint; the
                              split algorithm is unchanged                     */
};

/* plan flags for btmv_plan_create (may be OR-ed) */
enum {
  BTMV_FLAG_NONE = 0,
  BTMV_FLAG_PROFILE = 1u << 0, /* record a CUDA event pair around every kernel
                                  launch of btmv_apply (see btmv_profile_read);
                                  with BTMV_PROFILE_EVERY=k in the environment
                                  at plan creation, of one apply in every k */
  BTMV_FLAG_GENERIC = 1u << 1, /* use only the generic shared-memory line kernels
                                  (any 7-smooth size, both precisions) instead of
                                  the register-resident power-of-two kernels   */
  BTMV_FLAG_SHARED_RHS = 1u << 2,  /* multi-rhs leaf: all right-hand sides of a
                                      line in one tile, each frequency's c x c
                                      symbol block read once for all of them
                                      (CUDA-core contraction)                  */
  BTMV_FLAG_TENSOR_CORE = 1u << 3, /* as BTMV_FLAG_SHARED_RHS, with the c x c x
                                      nrhs contraction on tensor cores (c = 3,
                                      complex64, nrhs >= 2): TF32 mma with a
                                      high/low split, FP32 accumulation        */
  BTMV_FLAG_TWO_STREAMS = 1u << 4, /* split, d >= 3: run the two top-level
                                      subtrees of Algorithm 1 on two streams
                                      (the caller's and a plan stream) so the
                                      passes of one overlap the leaves of the
                                      other; costs d-2 more workspace vectors
                                      (peak d+1 -> 2d-1 vectors)              */
  BTMV_FLAG_FUSED_LEVELS = 1u << 5 /* split, d >= 3, c = 3, complex64,
                                      block-symmetric compressed store,
                                      n_{d-1} = n_d = 64 (1-based levels): the
                                      last two levels of Algorithm 1 (the
                                      level d-1 split, the leaf, the level
                                      d-1 merge) run as one kernel per level
                                      d-2 node, its n_{d-1} x n_d slabs held
                                      in shared memory (Sec. II.B); other
                                      plans ignore the flag.  An apply fuses
                                      when its grid has at least 4 blocks per
                                      SM (nrhs n_1 .. n_{d-2} >= 4 x SMs, 2 x
                                      SMs with BTMV_FLAG_TWO_STREAMS, whose
                                      two subtrees' launches run side by
                                      side; BTMV_FUSE_MIN_BLOCKS=k in the
                                      environment sets k), else it runs
                                      unfused; plan info counts launches for
                                      max_rhs.  Trailing sizes 128 x 128 take
                                      a 16-CTA cluster per slab only with
                                      BTMV_FUSE_CLUSTER=1 in the environment
                                      (measured slower than unfused)          */
};

/*
 * btmv_plan_create -- allocate a plan for one problem geometry.
 *   out       [out] receives the plan handle (host pointer).
 *   d         number of Toeplitz levels, 1 <= d <= 6 (BTMV_ALGO_FULL: d <= 4).
 *   n         host array of d level sizes, 1 <= n[m] <= 1024.  BTMV_ALGO_FULL
 *             needs every n[m] to factor into 2, 3, 5 and 7.  A split plan
 *             with other sizes (primes, ...; d <= 4) runs on the operator
 *             zero-padded to the next 7-smooth size of each level -- exact,
 *             since that operator restricted to the first n[m] points is T --
 *             with x and y copied into and out of two padded device vectors
 *             around each apply (btmv_get_symbol then returns the padded
 *             operator's symbol).
 *   c         block size (components), 1 <= c <= 3.
 *   precision BTMV_C64 or BTMV_C128.
 *   algo      BTMV_ALGO_SPLIT, BTMV_ALGO_FULL or BTMV_ALGO_FULL_CUFFT (as FULL,
 *             d <= 3; BTMV_E_UNSUPPORTED when libcufft cannot be loaded).
 *   max_rhs   largest nrhs later passed to btmv_apply (>= 1).
 *   flags     BTMV_FLAG_*.
 * Allocates the twiddle tables and the workspace: (d - 1) vectors of
 * max_rhs * c * prod(n) complex for SPLIT (the paper's (d+1)-vector peak with
 * x and y, Sec. II.C), 2^d such vectors for FULL and FULL_CUFFT (plus
 * cuFFT's own work area for FULL_CUFFT), and one word of pinned, device-mapped
 * host memory in which the TMA-staged passes report an expired wait.  The
 * device is the current CUDA device.
 * Errors: BTMV_E_ARG, BTMV_E_UNSUPPORTED, BTMV_E_NOMEM, BTMV_E_CUDA.
 */
BTMV_API btmv_status btmv_plan_create(btmv_plan* out, int d, const int32_t* n, int c,
                             int precision, int algo, int max_rhs, uint32_t flags);

/*
 * btmv_plan_clone -- a new plan for the same operator: same geometry,
 * precision and algorithm, sharing src's symbol store and twiddle tables
 * (reference counted: they live until the last plan using them is
 * destroyed) with its own workspace for up to max_rhs right-hand sides.
 * Lets many concurrent solves of one operator keep a single resident symbol
 * while each runs its own applies (one stream per plan).  A later
 * btmv_set_kernel on any of them builds a private symbol for that plan only.
 *   src      plan to clone (its symbol may or may not be set yet).
 *   max_rhs  >= 1.   flags  BTMV_FLAG_*.   out  receives the new plan.
 * Errors: BTMV_E_ARG, BTMV_E_NOMEM.
 */
BTMV_API btmv_status btmv_plan_clone(btmv_plan src, int max_rhs, uint32_t flags, btmv_plan* out);

/*
 * btmv_set_kernel -- set the generating coefficients (one-time symbol build).
 *   t         host, complex128 interleaved (2 doubles per value):
 *             without BTMV_SYM_PARITY: [c][c][2n_1 - 1]...[2n_d - 1], offset p_m
 *               stored at index p_m + n_m - 1;
 *             with BTMV_SYM_PARITY: [c][c][n_1]...[n_d], offsets p_m >= 0 only.
 *             With BTMV_SYM_BLOCK only blocks a <= b are read.
 *   sym_flags BTMV_SYM_*.
 *   parity    host int8 [c][c][d] of +1 / -1 (t(.., -p_m, ..) = parity * t(.., p_m, ..)),
 *             required with BTMV_SYM_PARITY, else ignored (may be NULL).  A -1
 *             entry requires t = 0 on the plane p_m = 0 of that block.
 *   stream    stream for the build; the call synchronises it before returning.
 * Computes, in FP64 on the device, every leaf part S_b = DFT_n(P_b (c~_lo +
 * (-1)^b c~_hi)) / prod(2 n_m) of the transformed embedded generator
 * (Sec. I embedding with free entry s0 = 0; Sec. II.C split into 2^d parts)
 * and rounds it once to the plan precision.  Storage: full, 2^d prod(n) values
 * per stored block; or with BTMV_SYM_PARITY the mirror-compressed
 * prod(n_m + 1) values per stored block (Sec. II.C symmetric /
 * skew-symmetric storage; both algorithms read it, the plain embedding at
 * its full-grid frequencies folded by f -> 2n - f).  May be called again to replace the generator.
 * Errors: BTMV_E_ARG, BTMV_E_NOMEM, BTMV_E_CUDA.
 */
BTMV_API btmv_status btmv_set_kernel(btmv_plan p, const double* t, uint32_t sym_flags,
                            const int8_t* parity, void* stream);

/*
 * btmv_apply -- y = T x for nrhs right-hand sides.
 *   x, y      [nrhs][c][n_1]..[n_d] complex (plan precision); device or host
 *             pointers, 16-byte aligned; must not overlap.  x is read only,
 *             y is overwritten.
 *   nrhs      0 <= nrhs <= max_rhs (0 is a no-op).
 *   stream    work is enqueued on it; with host pointers the call copies
 *             through plan-owned device buffers and synchronises the stream.
 * SPLIT: depth-first traversal of Algorithm 1 -- forward split passes along
 * levels 1..d-1, a fused leaf pass along level d (both halves, symbol
 * multiply, merge), merge passes back up; peak (d+1) vectors.  d = 2, c = 1,
 * 64 x 64 plans run the whole traversal as one launch of a 16-CTA cluster
 * per right-hand side (BTMV_SMALL2D=0 in the environment, or
 * BTMV_FLAG_GENERIC, keeps the three kernels); BTMV_FLAG_FUSED_LEVELS fuses
 * the last two levels of d = 3 plans it supports.
 * Errors: BTMV_E_ARG, BTMV_E_STATE (no generator set), BTMV_E_CUDA,
 * BTMV_E_TIMEOUT (a bounded wait of a TMA-staged pass expired in an earlier
 * apply on this plan; reported once, by the next apply).
 */
BTMV_API btmv_status btmv_apply(btmv_plan p, const void* x, void* y, int nrhs, void* stream);

/*
 * btmv_apply_batched -- y_k = T_k x_k for count independent plans, enqueued
 * on stream as one replay of a captured CUDA graph.
 *   plans, x, y, nrhs  host arrays of length count; entry k as in btmv_apply
 *                      (device pointers only).  Plans must be distinct.
 * SPLIT plans of one precision run together.  The graph holds one of two
 * execution modes:
 *   0  one persistent kernel: every plan's depth-first schedule (the
 *      launches btmv_apply would make) becomes a chain of stages, stages of
 *      different plans run side by side, and each wait for a previous stage
 *      is bounded (BTMV_WAIT_TIMEOUT_MS, default 5000 ms);
 *   1  parallel branches (16, 4 or 1), each running its problems' own
 *      btmv_apply launches; problems are placed largest first on the branch
 *      with the least work.
 * The graph is captured once per argument set (plans, x, y, nrhs) and
 * replayed on later calls with the same arguments; the first call for a new
 * set of problem shapes times the modes (and, for mode 0, a few tile / radix
 * choices) on the caller's data and keeps the fastest (process wide, and in
 * the file named by BTMV_TUNE_CACHE if set).  BTMV_NO_AUTOTUNE with
 * BTMV_BATCH_MODE=0|1 fixes the mode instead; BTMV_BATCH_DIRECT runs the
 * problems on forked streams without a graph (for mixes that change every
 * call).  Other mixes (BTMV_ALGO_FULL plans, mixed precisions) run one
 * apply after the other.  The first call for an argument set allocates its
 * stage table; a wait that expired in a launch is reported (BTMV_E_TIMEOUT)
 * by the next call with the same arguments.
 * Errors: as btmv_apply; on an argument error nothing is enqueued.
 */
BTMV_API btmv_status btmv_apply_batched(int count, const btmv_plan* plans, const void* const* x,
                               void* const* y, const int* nrhs, void* stream);

/*
 * btmv_apply_host_async -- y = T x with x and y in pinned HOST memory,
 * pipelined across calls.  The call enqueues the copy of x into one of two
 * plan-owned device staging slots (used in turn) on a plan copy stream, the
 * apply on `stream`, and the copy of y back to the host on a second plan
 * copy stream, and returns without waiting: consecutive calls on one plan
 * overlap the copies of one call with the apply of the next.
 *   p, nrhs   as btmv_apply.
 *   x, y      host pointers (page-locked memory for the copies to overlap);
 *             x must stay unchanged and y untouched until btmv_host_wait.
 *   stream    the apply runs on it; a later btmv_apply on the same stream
 *             follows the apply but not the copy of y.
 * y is valid after btmv_host_wait(p).  The first call allocates the two
 * slots (2 x 2 vectors of max_rhs right-hand sides) and the copy streams.
 * Errors: as btmv_apply; BTMV_E_NOMEM on the first call.
 */
BTMV_API btmv_status btmv_apply_host_async(btmv_plan p, const void* x, void* y, int nrhs, void* stream);

/* btmv_host_wait -- wait until every btmv_apply_host_async call made on p so
 * far has its y on the host.  Errors: BTMV_E_ARG, BTMV_E_CUDA. */
BTMV_API btmv_status btmv_host_wait(btmv_plan p);

/*
 * btmv_apply_host_noalloc -- y = T x with x and y in HOST memory, like
 * btmv_apply with host pointers, but without allocating anything.
 *
 * The paper has no counterpart to this call; it exists for callers that
 * cannot let the library allocate device memory when they call it.
 * btmv_apply with host pointers allocates two staging buffers (cudaMalloc) on
 * its first such call; a process whose device memory is reserved by another
 * allocator, or a solver loop that must not enter the driver's allocation
 * path, cannot accept that.  This call stages x and y through a fixed array
 * compiled into the library instead (2 x BTMV_NOALLOC_MAX_BYTES of device
 * memory that every GPU loading the library holds until the process exits)
 * and calls no cudaMalloc, cudaFree or allocating library routine.
 *   p, nrhs   as btmv_apply; the plan (symbol, tables, workspace) is created
 *             beforehand and is only read here.
 *   x, y      host pointers to [nrhs][c][n_1]..[n_d] complex; x is read, y is
 *             overwritten.
 *   stream    the copies and kernels are enqueued on it and the call
 *             synchronises it before returning.
 * Limit: nrhs * c * prod(n) * element size <= BTMV_NOALLOC_MAX_BYTES, else
 * BTMV_E_UNSUPPORTED with a message (use btmv_apply then).
 * The first call on each device looks up the array's device address
 * (cudaGetSymbolAddress, with that device current); make that first call
 * before any stream capture.  Every call on a device shares the one array,
 * whose contents persist between calls (no call reads what an earlier one
 * left there); calls whose work overlaps on the same GPU (other host threads
 * or streams) race on it and must be serialised by the caller.
 * The plan's device must be the current device (BTMV_E_ARG otherwise): the
 * array staged on is the current device's copy.
 * Errors: as btmv_apply, plus BTMV_E_UNSUPPORTED for the size limit.
 */
#define BTMV_NOALLOC_MAX_BYTES (16u << 20)
BTMV_API btmv_status btmv_apply_host_noalloc(btmv_plan p, const void* x, void* y, int nrhs, void* stream);

/*
 * btmv_batch_tuning -- report the tuning chosen for a batch that has run:
 * cfg_out[0..7] = strided-pass tile lines, leaf lines per tile, leaf
 * right-hand sides per tile, radix order (0: 16 first, 1: 8 first), stages
 * of the persistent launch (mode 1: kernel launches per graph replay), work
 * items, blocks of the persistent launch (mode 1: parallel branches),
 * execution mode (0: one persistent kernel, 1: one graph whose parallel
 * branches run the problems' own launches, largest problems placed first).  Arguments as for the
 * btmv_apply_batched call.  Errors: BTMV_E_ARG, BTMV_E_STATE (no such batch).
 */
BTMV_API btmv_status btmv_batch_tuning(int count, const btmv_plan* plans, const void* const* x,
                                       void* const* y, const int* nrhs, int* cfg_out /* [8] */);

/*
 * btmv_selftest_wait_timeout -- failure-detection self test of the bounded
 * waits of the persistent kernel: launches it with one work item whose
 * dependency count is withheld, so that its wait expires after timeout_ms.
 * Returns BTMV_E_TIMEOUT when the kernel detected the expired wait and
 * returned normally (the expected outcome; the CUDA context stays usable),
 * BTMV_E_STATE if no timeout was reported, BTMV_E_CUDA / BTMV_E_NOMEM on
 * other failures.  Synchronises stream.
 */
BTMV_API btmv_status btmv_selftest_wait_timeout(int timeout_ms, void* stream);

/*
 * btmv_selftest_tma_timeout -- failure-detection self test of the bounded
 * waits of the TMA-staged strided passes: launches one such pass on a small
 * scratch tile whose mbarrier is told to expect 16 bytes more than the copy
 * delivers, so that its wait expires after timeout_ms (1..10000).  Returns
 * BTMV_E_TIMEOUT when the kernel reported the expired wait and returned
 * normally (the expected outcome; the CUDA context stays usable),
 * BTMV_E_STATE if no expiry was reported, BTMV_E_CUDA on other failures.
 * Allocates and frees its scratch; synchronises stream.
 */
BTMV_API btmv_status btmv_selftest_tma_timeout(int timeout_ms, void* stream);

/* btmv_destroy -- free every device and host resource of the plan (NULL ok).
 * Synchronises the device work of the plan first. */
BTMV_API btmv_status btmv_destroy(btmv_plan p);

/* btmv_last_error -- message of the last failure on this thread ("" if none).
 * The pointer stays valid until the next btmv call on this thread. */
BTMV_API const char* btmv_last_error(void);

/* ------------------------------------------------------------------------
 * Introspection (tests, benchmarks, serving admission)
 * ---------------------------------------------------------------------- */
typedef struct {
  int d, c, precision, algo, max_rhs;
  int n[6];
  int nsym;                 /* stored symbol blocks: c*c, or c(c+1)/2 with BTMV_SYM_BLOCK */
  int compressed;           /* 1 if the mirror-compressed parity store is in use */
  int has_symbol;
  int launches_per_apply;   /* kernel launches of one btmv_apply (device pointers) */
  size_t symbol_bytes;      /* device bytes of the symbol store */
  size_t workspace_bytes;   /* device bytes of the workspace vectors */
  size_t table_bytes;       /* device bytes of twiddle tables */
  size_t vector_bytes;      /* bytes of one vector at nrhs = 1 */
} btmv_plan_info_t;

/* btmv_plan_get_info -- fill *info (host pointer).  Errors: BTMV_E_ARG. */
BTMV_API btmv_status btmv_plan_get_info(btmv_plan p, btmv_plan_info_t* info);

/*
 * btmv_get_symbol -- copy the device symbol store to host memory `out`
 * (bytes >= info.symbol_bytes), synchronously.  Layout: 2^d parity classes
 * b = (b_1..b_d) in order sum_m b_m 2^(d-m) (b_1 most significant); class b
 * holds nsym blocks, each a row-major box of J_1(b_1) x .. x J_d(b_d) values
 * S[2 j + b] (j_m < J_m).  Full store: J_m = n_m.  Compressed store:
 * J_m(b_m) = floor((n_m - b_m)/2) + 1 (the frequencies f <= n_m; the others
 * follow from S[2n - f] = +-S[f]).  Stored block order: c = 1: (0,0); c = 3
 * with BTMV_SYM_BLOCK: (0,0),(1,1),(2,2),(0,1),(0,2),(1,2); otherwise
 * row-major (a, b).  Errors: BTMV_E_ARG, BTMV_E_STATE, BTMV_E_CUDA.
 */
BTMV_API btmv_status btmv_get_symbol(btmv_plan p, void* out, size_t bytes);

/* kernel kinds reported by btmv_profile_read */
enum {
  BTMV_K_FWD_SPLIT = 0,    /* forward split pass (levels 1..d-1)              */
  BTMV_K_LEAF = 1,         /* fused leaf pass (level d)                        */
  BTMV_K_MERGE = 2,        /* backward merge pass (levels d-1..1)              */
  BTMV_K_FULL_FWD = 3,     /* full embedding: forward passes on the 2n grid    */
  BTMV_K_FULL_LEAF = 4,    /* full embedding: last-dim forward+multiply+inverse */
  BTMV_K_FULL_INV = 5,     /* full embedding: inverse passes (+ projection)    */
  BTMV_K_COPY = 6,         /* host staging copies                              */
  BTMV_K_FUSED_LEVELS = 7, /* last two levels in one kernel: BTMV_FLAG_FUSED_LEVELS
                              launches, and the one-launch d = 2 apply         */
  BTMV_K_NKINDS = 8
};

/*
 * btmv_profile_read -- with BTMV_FLAG_PROFILE, synchronise the events
 * recorded since the last read and return per-kernel-kind totals (over the
 * sampled applies when BTMV_PROFILE_EVERY is set; sampling restarts with the
 * next apply, which is recorded).  The events separate the
 * launches they bracket, which then lose the programmatic-dependent-launch
 * overlap of the register kernels.
 *   ms_total  host double[BTMV_K_NKINDS]: summed event-measured milliseconds.
 *   launches  host int64[BTMV_K_NKINDS]: launch counts.
 * Resets the accumulators.  Errors: BTMV_E_ARG, BTMV_E_STATE (flag not set),
 * BTMV_E_CUDA.
 */
BTMV_API btmv_status btmv_profile_read(btmv_plan p, double* ms_total, int64_t* launches);

#ifdef __cplusplus
}
#endif
#endif /* BTMV_H */
