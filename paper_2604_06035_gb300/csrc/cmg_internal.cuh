// cmg_internal.cuh -- internal types and device helpers of libcmg.so.
//
// Data layout (GB300-first):
//  * every MG level keeps its cell fields in a colour-planar oct layout:
//      field[plane][oct][slot],  plane = parity(c) (0 = red, 1 = black),
//      slot = c >> 1,  c = bx + 2 by + 4 bz.
//    A red (black) sweep then reads the whole black (red) plane and writes the
//    red (black) plane: 12 B/cell per colour pass in FP64, the algorithmic
//    minimum, with 32-byte (FP64) / 16-byte (FP32) vector loads per oct.
//  * the source is stored pre-scaled, g = -h^2 f / 6, so the Gauss-Seidel
//    update of App. D.2 Eq. (gs_update) is one FMA after the neighbour sum.
//  * oct arrays hold n real octs, then the Dirichlet ghost octs of a refined
//    level (missing neighbours whose cells are interpolated from the parent),
//    then one oct of zeros that stands for "no neighbour" on coarse MG levels.
//    Kernels therefore never branch on missing neighbours.
//  * neighbour and interpolation-block tables are structure-of-arrays
//    ([6][n], [8][n]) so that a warp's index loads are coalesced.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <stdexcept>
#include <string>
#include <vector>

#include "cmg.h"

namespace cmg {

constexpr uint64_t kEmptyKey = ~0ull;
constexpr int kMortonBits = 21;

// A 128-bit Morton key (B = 42 bits per coordinate, Sec. 4.2): key bits 0..63
// in lo, 64..127 in hi (keys.cuh).
struct alignas(16) Key128 {
  uint64_t lo, hi;
};

// ------------------------------------------------------------------ errors

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string &m) : std::runtime_error(m), code(c) {}
};

void cuda_check(cudaError_t e, const char *what);
// tests: the after'th next library allocation fails with CMG_ERR_OOM (0: off)
void inject_alloc_failure(int64_t after);
#define CMG_CUDA(x) ::cmg::cuda_check((x), #x)

// ------------------------------------------------------- Morton keys (A1)
// Sec. 4.2 Eq. (morton_encode): bit b of i, j, k goes to key bits 3b, 3b+1,
// 3b+2.  Written with the usual bit-spreading masks (21 bits per axis).

__host__ __device__ inline uint64_t spread3(uint32_t v) {
  uint64_t x = v & 0x1fffffu;
  x = (x | (x << 32)) & 0x001f00000000ffffull;
  x = (x | (x << 16)) & 0x001f0000ff0000ffull;
  x = (x | (x << 8)) & 0x100f00f00f00f00full;
  x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
  x = (x | (x << 2)) & 0x1249249249249249ull;
  return x;
}

__host__ __device__ inline uint32_t compact3(uint64_t x) {
  x &= 0x1249249249249249ull;
  x = (x ^ (x >> 2)) & 0x10c30c30c30c30c3ull;
  x = (x ^ (x >> 4)) & 0x100f00f00f00f00full;
  x = (x ^ (x >> 8)) & 0x001f0000ff0000ffull;
  x = (x ^ (x >> 16)) & 0x001f00000000ffffull;
  x = (x ^ (x >> 32)) & 0x00000000001fffffull;
  return (uint32_t)x;
}

__host__ __device__ inline uint64_t morton_encode(uint32_t i, uint32_t j, uint32_t k) {
  return spread3(i) | (spread3(j) << 1) | (spread3(k) << 2);
}

__host__ __device__ inline void morton_decode(uint64_t m, uint32_t &i, uint32_t &j, uint32_t &k) {
  i = compact3(m);
  j = compact3(m >> 1);
  k = compact3(m >> 2);
}

// App. A Alg. 2: neighbour key in direction d (0..5 = -x,+x,-y,+y,-z,+z) on a
// grid of npd octs per axis; periodic wrap on the axes of pmask, else the
// all-ones key meaning "outside the box".
__host__ __device__ inline uint64_t neighbor_key(uint64_t m, int d, uint32_t npd, int pmask) {
  uint32_t c[3];
  morton_decode(m, c[0], c[1], c[2]);
  const int a = d >> 1;
  int64_t v = (int64_t)c[a] + ((d & 1) ? 1 : -1);
  if ((pmask >> a) & 1) {
    if (v < 0) v += npd;
    if (v >= (int64_t)npd) v -= npd;
  } else if (v < 0 || v >= (int64_t)npd) {
    return kEmptyKey;
  }
  c[a] = (uint32_t)v;
  return morton_encode(c[0], c[1], c[2]);
}

// ------------------------------------------------------------ hash (A5/A6)
// App. B Eq. (hash_func): multiplicative hash with a mixing step, modulo 2^64.

__host__ __device__ inline uint64_t hash_mix(uint64_t h) {
  uint64_t t = ((h * 2654435761ull) ^ (h >> 16)) * 0x9E3779B97F4A7C15ull;
  return t ^ (t >> 13);
}

inline int64_t hash_capacity(int64_t n) {
  int64_t cap = 1;
  while (10 * n > 7 * cap) cap <<= 1;
  return cap;
}

// Linear probing (App. B), at most cap probes.
__device__ inline int32_t ht_find(const uint64_t *__restrict__ keys, const int32_t *__restrict__ vals,
                                  uint64_t mask, uint64_t k) {
  uint64_t s = hash_mix(k) & mask;
  for (uint64_t p = 0; p <= mask; ++p) {
    const uint64_t kk = keys[s];
    if (kk == k) return vals[s];
    if (kk == kEmptyKey) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}

// Returns the slot of k, inserting it if absent; *inserted tells which.
// -1 if the table is full (cannot happen at fill <= 0.7).
__device__ inline int64_t ht_insert_slot(uint64_t *keys, uint64_t mask, uint64_t k, bool *inserted) {
  uint64_t s = hash_mix(k) & mask;
  for (uint64_t p = 0; p <= mask; ++p) {
    const unsigned long long prev =
        atomicCAS(reinterpret_cast<unsigned long long *>(keys + s), (unsigned long long)kEmptyKey,
                  (unsigned long long)k);
    if (prev == kEmptyKey) {
      *inserted = true;
      return (int64_t)s;
    }
    if (prev == k) {
      *inserted = false;
      return (int64_t)s;
    }
    s = (s + 1) & mask;
  }
  return -1;
}

__device__ inline int64_t ht_slot(const uint64_t *__restrict__ keys, uint64_t mask, uint64_t k) {
  uint64_t s = hash_mix(k) & mask;
  for (uint64_t p = 0; p <= mask; ++p) {
    const uint64_t kk = keys[s];
    if (kk == k) return (int64_t)s;
    if (kk == kEmptyKey) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}

__device__ inline void set_error(int *err, int code) { atomicCAS(err, 0, code); }
// message returned by cmg_last_error() on this thread
void record_error(const char *msg);

// -------------------------------------------------------------- cell maps

__host__ __device__ constexpr int cell_parity(int c) { return ((c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1)) & 1; }
// child index of (plane, slot)
__host__ __device__ constexpr int plane_cell(int p, int q) {
  return p == 0 ? (q == 0 ? 0 : q == 1 ? 3 : q == 2 ? 5 : 6) : (q == 0 ? 1 : q == 1 ? 2 : q == 2 ? 4 : 7);
}

// ------------------------------------------------------------------ types

struct MgLev {
  int lev = 0;
  int64_t n = 0;        // real octs
  int64_t n_ghost = 0;  // Dirichlet ghost octs (level 0 of a refined AMR level)
  int64_t n_alloc = 0;  // n + n_ghost + 1 (zero oct last)
  double h = 0.0;
  bool all_active = true;
  uint64_t *keys = nullptr;      // [n] (128-bit levels: the keys' low words)
  uint64_t *ht_keys = nullptr;   // [cap] (64-bit levels)
  Key128 *keys128 = nullptr;     // [n] (128-bit levels)
  Key128 *ht_keys128 = nullptr;  // [cap] (128-bit levels)
  int32_t *ht_vals = nullptr;    // [cap]
  int64_t cap = 0;
  int32_t *nbr = nullptr;        // [6][n] internal neighbour index (>= n: ghost / zero oct)
  uint8_t *active = nullptr;     // [n] 8-bit cell mask
  int32_t *father = nullptr;     // [n] coarse cell (p*8 + cc) of fully active octs, else -1
  int32_t *blk = nullptr;        // [8][n] 2x2x2 coarse octs around the father cell
  double *phi = nullptr;         // [2][n_alloc][4]
  double *g = nullptr;           // [2][n][4], g = -h^2 f / 6
  float *phi32 = nullptr;        // [2][n_alloc][4]
  float *g32 = nullptr;          // [2][n][4]
  // log2 of the octs per axis when the level is a full periodic grid stored
  // in lexicographic order (x fastest): its neighbours are implicit and the
  // colour passes may run the shared-memory brick kernel; else -1
  int lex_log2 = -1;
};

struct DeviceBuffers {
  std::vector<void *> ptrs;
  template <class T>
  T *alloc(int64_t count, bool zero = false, cudaStream_t s = nullptr);
  void release();
};

}  // namespace cmg

namespace cmg {
enum KernelClass {
  K_SWEEP64 = 0, K_SWEEP32, K_RESID64, K_RESID32, K_PROLONG64, K_PROLONG32, K_GHOST, K_COARSE, K_REDUCE,
  K_CONVERT, K_CONV_FWD, K_CONV_DGRAD, K_CONV_WGRAD, K_FFT, K_NCLASS
};
struct ProfClass {
  int64_t launches = 0;
  double ms = 0.0, bytes = 0.0, flops = 0.0;
};
struct PendingEvent {
  int cls;
  int slot;
};
}  // namespace cmg

struct cmg_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  int num_sms = 0;
  int *d_err = nullptr;       // device error flag
  int *h_pinned = nullptr;    // pinned staging (ints)
  double *h_dpinned = nullptr;  // pinned staging (doubles)
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // device staging of host-memory arguments (grow-only; [0] inputs, [1] outputs)
  void *stage[2] = {nullptr, nullptr};
  size_t stage_bytes[2] = {0, 0};
  // host<->device copies of host-memory arguments run on streams of their own
  // (created on first use), so that they overlap work queued on `stream`
  cudaStream_t h2d_stream = nullptr, d2h_stream = nullptr;
  cudaEvent_t h2d_done = nullptr;      // the last upload into stage[0] has finished
  cudaEvent_t stage0_free = nullptr;   // `stream` has finished reading stage[0]
  cudaEvent_t stage1_ready = nullptr;  // `stream` has finished writing stage[1]
  cudaEvent_t d2h_done = nullptr;      // the last download from stage[1] has finished
  bool stage0_used = false;            // stage0_free has been recorded
  bool d2h_pending = false;            // a queued download may still read stage[1]
  // graph capture (private streams; the caller's stream may be the legacy one)
  cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
  bool capturing = false;
  int64_t captured = 0;  // kernels recorded into the graph being built
  // instrumentation
  int64_t launches = 0;
  bool profiling = false;
  cmg::ProfClass prof[cmg::K_NCLASS];
  std::vector<cudaEvent_t> ev_pool;  // pairs (2k, 2k+1)
  std::vector<cmg::PendingEvent> pending;
};

namespace cmg {
// Counts a launch of family cls and, when profiling, brackets it with events.
struct LaunchScope {
  cmg_ctx *ctx;
  int slot = -1;
  LaunchScope(cmg_ctx *c, int cls, double bytes, double flops);
  ~LaunchScope();
};
void harvest_profile(cmg_ctx *ctx);
const char *kernel_class_name(int cls);
}  // namespace cmg

struct cmg_level {
  cmg_ctx *ctx = nullptr;
  int device = 0;                // copies of the context's device and stream, so
  cudaStream_t stream = nullptr; // that destroying a level never reads its context
  int lev = 0, nx = 1, pmask = 7;
  int64_t n = 0;
  cmg_level *parent = nullptr;
  bool periodic_full = false;
  bool exact_coarse = false;
  std::vector<cmg::MgLev> mg;
  // ghosts of level 0
  uint64_t *ghost_keys = nullptr;  // [n_ghost] (128-bit levels: the low words)
  cmg::Key128 *ghost_keys128 = nullptr;  // [n_ghost] (128-bit levels)
  int key_bits = 64;               // Morton key width of the level (and of its parent)
  int32_t *ghost_blk = nullptr;    // [8][n_ghost] parent octs around the ghost's father cell
  uint32_t *ghost_mask = nullptr;  // [n_ghost] cells some real oct reads
  // reductions
  double *partials = nullptr;  // [blocks of the largest MG level]
  double *scal = nullptr;      // device scalars (norms, scales)
  double *rbuf = nullptr;      // [n][8] residual for the API (lazy)
  uint8_t *ctrl = nullptr;     // device solve control block (cycles, status, history)
  void *h_ctrl = nullptr;      // pinned host copy
  // a queued solve (solve_launch) until solve_wait reports it
  struct Pending {
    bool empty = false;
    int64_t launches_fixed = 0, launches_body = 0, updates_per_cycle = 0;
  } pend;
  bool solve_pending = false;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;  // around the queued solve
  std::vector<void *> graphs;  // instantiated solve graphs, keyed by parameters
  bool has32 = false;
  // schedule: MG levels with at most this many octs (and all coarser ones) run
  // in one "tail" launch (tail.cu); 0 = one launch per operation everywhere
  int64_t tail_octs_fp64 = 32768;
  int64_t tail_octs_fp32 = 2048;
  // colour passes of lexicographic full periodic levels in the shared-memory
  // brick kernel (brick.cu): 0 = never, 1 = FP32 passes (default; the FP64
  // pass measured faster with the neighbour table), 2 = FP32 and FP64 passes
  int staged = 1;
  int64_t tail_spin_budget = 1ll << 30;  // SM clock cycles a grid-tail barrier wait may last
  // FFT solve of a full periodic level (fft.cu): dense complex work array,
  // oct-coordinate -> oct-index map, twiddles (lazy)
  float2 *fft_buf = nullptr;
  int32_t *fft_map = nullptr;
  float2 *fft_tw = nullptr;
  double *pcg = nullptr;  // CG vectors, partial sums and scalars (pcg.cu, lazy)
  cmg::DeviceBuffers mem;
};

struct cmg_batch {
  cmg_level *lvl = nullptr;
  int n_patches = 0;
  cmg_batch_schedule sched = {256, 2, 2, 2, 1};
  long long spin_budget = 2000000000ll;
  std::vector<int32_t *> pid;  // patch of each oct, per MG level
  double *pstate = nullptr;    // n0, norm, s_emit, s_acc, rel: 5 x n_patches
  int32_t *conv_at = nullptr;
  int *ctrl = nullptr;         // 8 ints
  unsigned *bar = nullptr;     // grid barrier words
  int *h_ctrl = nullptr;       // pinned copy of ctrl
  double *cg = nullptr;        // CG vectors and per-patch scalars (krylov = 1, lazy)
  int32_t *cg_done = nullptr;  // per-patch "reached tol" flags of the CG iteration
  cmg::DeviceBuffers mem;
  // the recorded solve graph and what it was recorded for
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  cmg_batch_schedule g_sched = {};
  cmg_solve_params g_params = {};
  int g_grid = 0;
  long long g_budget = 0;
};

namespace cmg {

constexpr int kThreads = 256;

inline unsigned blocks_for(int64_t n, int t = kThreads) { return (unsigned)((n + t - 1) / t); }

// Launch with programmatic dependent launch allowed: the next kernel on the
// stream (or in the captured graph) may be scheduled while this one drains.
// Every kernel launched this way calls pdl_enter(), which waits for the
// preceding grid to complete, before it touches memory that any kernel
// writes after the level build; only reads of the build's index arrays
// (neighbours, masks, father cells, interpolation blocks, keys), which the
// build finishes with a stream synchronisation and nothing writes again,
// may come before it.
template <typename... KArgs, typename... Args>
inline void launch_k(void (*kernel)(KArgs...), unsigned grid, unsigned block, cudaStream_t s, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(block);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cuda_check(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(args)...), "cudaLaunchKernelEx");
}

__device__ __forceinline__ void pdl_enter() {
#if defined(__CUDA_ARCH__) && __CUDA_ARCH__ >= 900
  cudaTriggerProgrammaticLaunchCompletion();
  cudaGridDependencySynchronize();
#endif
}

// scan.cu
void scan_exclusive(const int32_t *in, int32_t *out, int64_t n, int32_t *d_total, int32_t *scratch,
                    int64_t scratch_n, cudaStream_t s);
int64_t scan_scratch_size(int64_t n);

// build.cu
// keys: [n] uint64 (L->key_bits == 64) or [n] Key128 (128), host or device
void build_level(cmg_level *L, const void *keys, cmg_mem mem);
void hash_lookup(const MgLev &g, const uint64_t *q, int64_t n, int32_t *out, cudaStream_t s);
void hash_lookup128(const MgLev &g, const Key128 *q, int64_t n, int32_t *out, cudaStream_t s);
void encode_keys(const uint32_t *ijk, int64_t n, uint64_t *keys, int *err, cudaStream_t s);
void decode_keys(const uint64_t *keys, int64_t n, uint32_t *ijk, cudaStream_t s);
void encode_keys128(const uint64_t *ijk, int64_t n, Key128 *keys, int *err, cudaStream_t s);
void decode_keys128(const Key128 *keys, int64_t n, uint64_t *ijk, cudaStream_t s);
void ext_neighbors(const cmg_level *L, int32_t *out, cudaStream_t s);
void father_cells(const cmg_level *L, int32_t *out, cudaStream_t s);
void mg_active_bytes(const MgLev &g, uint8_t *out, cudaStream_t s);

// ops.cu
void set_density(cmg_level *L, const double *rho, double rho_bar, double four_pi_g);
// rows [n][6] -> out [n], device memory (the FP64 stencil's neighbour sums;
// which: 0 = colour passes and colour-1 residuals, 1 = colour-0 residuals)
void neighbour_sum(const double *rows, int64_t n, int which, double *out, cudaStream_t s);
void pack_field(cmg_level *L, int m, int field, int prec, const void *in);
void unpack_field(cmg_level *L, int m, int field, int prec, void *out);
void fill_ghosts(cmg_level *L);
void get_ghosts(cmg_level *L, double *out);
void ensure_fp32(cmg_level *L);
// pcg.cu (and the V-cycle it preconditions with, solve.cu)
void vcycle64_from_zero(cmg_level *L, const cmg_solve_params *p, int64_t *updates);
void vcycle32_from_zero(cmg_level *L, const cmg_solve_params *p, int64_t *updates);
void pcg_prepare(cmg_level *L);
void pcg_pre(cmg_level *L);
void pcg_body(cmg_level *L, const cmg_solve_params *p, int64_t *updates);
void pcg_post(cmg_level *L);
// fft.cu
bool fft_supported(const cmg_level *L);
void fft_prepare(cmg_level *L);
void fft_solve32(cmg_level *L);
template <typename T>
void sweep(cmg_level *L, int m, bool zero_init);
// c1_swept: the last operation on MG level m was a colour-1 pass over all of
// it (the colour-1 residuals are exactly zero and are not evaluated).
// finalize = false: a norm's per-block partial sums are left in L->partials
// for the caller's reduction (norm_out is not written).
template <typename T>
void resid_restrict(cmg_level *L, int m, bool restrict_to_coarse, bool norm, bool zero_coarse_phi,
                    double *norm_out, const double *emit_scale = nullptr, bool c1_swept = false,
                    bool finalize = true);
void residual_out(cmg_level *L, int m, int prec, double *out);
double residual_norm2_host(cmg_level *L, int m, int prec);
template <typename T>
void prolong(cmg_level *L, int m, bool c0_dead = false);  // c0_dead: a colour-0 pass follows
void coarse_solve(cmg_level *L, int prec, int coarse_sweeps);
void zero_phi_norm(cmg_level *L, double *out);
void subtract_mean(cmg_level *L);
// brick.cu: one colour pass of a lexicographic full periodic MG level (lex_log2 >= 4)
// through shared memory; mark_lexicographic sets lex_log2 on every MG level
template <typename T>
void brick_pass(cmg_level *L, int m, int colour);
void mark_lexicographic(cmg_level *L);
// sharded level solve (shard.cu): operations on the octs [lo, hi) of MG level
// m, FP64, and cell-granular gather / scatter (field 0 = phi, 1 = stored g;
// cell = oct * 8 + child; an index outside the level sets *bad)
void range_sweep_pass(cmg_level *L, int m, int colour, bool zero_other, int64_t lo, int64_t hi);
void range_residual(cmg_level *L, int m, bool restrict_to_coarse, bool c1_swept, int64_t lo, int64_t hi,
                    double *norm_out);
void range_prolong(cmg_level *L, int m, bool c0_dead, int64_t lo, int64_t hi);
void range_sum_phi(cmg_level *L, int m, int64_t lo, int64_t hi, double *out);
void range_shift_phi(cmg_level *L, int m, int64_t lo, int64_t hi, double v);
void gather_cells(cmg_level *L, int m, int field, const int32_t *idx, int64_t cnt, double *out, int *bad);
void scatter_cells(cmg_level *L, int m, int field, const int32_t *idx, int64_t cnt, const double *in, int *bad);
void accumulate(cmg_level *L, const double *scale);
void finalize_norm(cmg_level *L, int n_partials, double scale, double *out);

// tail.cu
template <typename T>
void tail_vcycle(cmg_level *L, int m0, const cmg_solve_params *p, const bool *zero_coarse);
// the solve's sticky device error word and the tail kernel's grid-barrier
// words (control block of the level's solve)
int *solve_err_word(cmg_level *L);
unsigned *solve_bar_words(cmg_level *L);

// batch.cu
void batch_create(cmg_level *L, const int64_t *offsets, int n_patches, cmg_batch **out);
void batch_destroy(cmg_batch *b);
int batch_solve(cmg_batch *b, const cmg_solve_params *p, cmg_batch_stats *st);
void batch_patch_stats(cmg_batch *b, double *rel, int32_t *conv, double *norm0);
void batch_set_schedule(cmg_batch *b, const cmg_batch_schedule *s);
void batch_autotune(cmg_batch *b, const cmg_solve_params *p, cmg_batch_schedule *best, double *best_ms);

// solve.cu
int solve(cmg_level *L, const cmg_solve_params *p, cmg_solve_stats *st);
void solve_launch(cmg_level *L, const cmg_solve_params *p);
int solve_wait(cmg_level *L, cmg_solve_stats *st);
void destroy_graphs(cmg_level *L);

}  // namespace cmg
