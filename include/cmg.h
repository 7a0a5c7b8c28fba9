/*
 * cmg.h -- C ABI of libcmg.so: a GB300 (sm_103a) level-by-level multigrid
 * Poisson solver on RAMSES oct grids, after cuRAMSES (arXiv 2604.06035).
 *
 * Problem (Sec. 5, Sec. 5.1.1): on one AMR level l, solve the 7-point
 * cell-centred discretisation of  lap(phi) = f,  f = 4 pi G (rho - rho_bar),
 * with cell size h = 2^-l / n_x in a unit box.  A level without a parent must
 * be complete and periodic (the base level); a level with a parent takes
 * Dirichlet values at its coarse-fine faces, interpolated from the parent's phi.
 *
 * Conventions shared by every call:
 *  - Return value: CMG_OK (0) or a negative cmg_status.  cmg_last_error()
 *    gives a message for the calling thread.  No C++ exception crosses the ABI.
 *  - Octs are numbered by their position in the key array given to
 *    cmg_level_build.  Oct-major arrays are [n_octs][8] with child index
 *    c = bx + 2 by + 4 bz (bit b of the cell offset inside its oct).
 *  - A pointer argument is host or device memory as its cmg_mem tag says.  The
 *    caller owns every buffer it passes; the library reads or writes it on the
 *    context's stream and keeps no reference after the call returns.  Calls
 *    that return data to host memory synchronise the stream first.
 *  - All computation runs in the library's CUDA kernels on the context's GPU;
 *    there is no CPU fallback.  A missing or failing GPU gives CMG_ERR_CUDA.
 *  - Objects are not thread-safe; use one context per host thread.
 */
#ifndef CMG_H
#define CMG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CMG_OK = 0,
  CMG_ERR_INVALID_ARG = -1,      /* bad pointer, size, level, parameter */
  CMG_ERR_DUPLICATE_KEY = -2,    /* the same Morton key given twice */
  CMG_ERR_KEY_OUT_OF_RANGE = -3, /* coordinate >= 2^(l-1) n_x or key >= 2^63 */
  CMG_ERR_MISSING_PARENT = -4,   /* a coarse-fine ghost value has no parent cells */
  CMG_ERR_OOM = -5,              /* device allocation failed */
  CMG_ERR_CUDA = -6,             /* any other CUDA error */
  CMG_ERR_NOT_CONVERGED = -7,    /* max_cycles reached above tol */
  CMG_ERR_DIVERGED = -8,         /* residual NaN or grew 1000-fold */
  CMG_ERR_TIMEOUT = -9           /* a bounded device-side wait gave up */
} cmg_status;

typedef enum { CMG_MEM_HOST = 0, CMG_MEM_DEVICE = 1 } cmg_mem;

typedef enum {
  CMG_PREC_FP64 = 0,  /* every step in FP64 */
  CMG_PREC_MIXED = 1, /* FP32 V-cycle inside FP64 iterative refinement */
  CMG_PREC_FFT = 2    /* FP32 FFT direct solve inside FP64 iterative refinement:
                         full periodic levels of 4^3 .. 512^3 cells only (the
                         paper's FFT base-level solve, Sec. 5.2); n_pre, n_post,
                         coarse_sweeps and inner_cycles are ignored */
} cmg_precision;

typedef struct cmg_ctx cmg_ctx;
typedef struct cmg_level cmg_level;

typedef struct {
  double tol;        /* stop when ||f - L phi|| <= tol ||f - L 0|| (2-norms) */
  int max_cycles;    /* <= 256 */
  int n_pre, n_post; /* red-black Gauss-Seidel sweeps before / after the coarse correction */
  int coarse_sweeps; /* sweeps on a non-periodic coarsest level */
  int fixed_cycles;  /* > 0: run exactly this many cycles and ignore tol */
  int precision;     /* cmg_precision */
  int inner_cycles;  /* MIXED: FP32 V-cycles per FP64 refinement step (>= 1; 2 is
                        the fastest to 1e-10 on the two-level 128^3 workload) */
  int krylov;        /* 0: stationary V-cycle iteration; 1: conjugate gradients
                        preconditioned by one V-cycle per iteration (App. D.2
                        names multigrid as the CG preconditioner); cycles then
                        counts CG iterations.  The preconditioner is an FP64
                        V-cycle (FP64) or inner_cycles FP32 V-cycles on
                        r / ||r|| (MIXED); FFT is rejected.  Batches: per-patch
                        CG with the same preconditioners. */
} cmg_solve_params;

typedef struct {
  int cycles;            /* V-cycles (FP64) or refinement steps (MIXED) run */
  int status;            /* same value as the call's return */
  double rel_initial;    /* relative residual of the initial guess */
  double rel_final;      /* relative residual at return */
  double norm0;          /* ||f - L 0||_2 */
  double ms;             /* device time of the call (CUDA events) */
  int64_t cell_updates;  /* cells visited by full red-black sweeps, all MG levels */
  double rel_history[256];
} cmg_solve_stats;

/* Library version string, e.g. "cmg 0.1.0 sm_103a". */
const char *cmg_version(void);
/* Message of the last failing call on this host thread ("" if none). */
const char *cmg_last_error(void);

/* Context: a device and a stream.  stream is a cudaStream_t (NULL = the
 * legacy default stream); the caller keeps it alive while the context lives. */
int cmg_ctx_create(int device, void *stream, cmg_ctx **out);
int cmg_ctx_destroy(cmg_ctx *ctx);
/* Waits for all work queued by the context: on its stream and on the copy
 * streams of host-memory arguments (cmg_level_get_phi_async downloads). */
int cmg_ctx_synchronize(cmg_ctx *ctx);

/* ---- instrumentation (no counterpart in the paper; used by the benchmark) ----
 * With profiling on, every solver kernel launch on the context's stream is
 * bracketed by CUDA events; cmg_ctx_get_profile synchronises the stream and
 * returns, per kernel family, the launches, the summed event time and the
 * algorithmic bytes / flops of those launches (the minimum traffic and
 * arithmetic of the operation, not hardware counters). */
typedef struct {
  char name[32];
  int64_t launches;
  double ms;
  double bytes;
  double flops;
} cmg_kernel_profile;
int cmg_ctx_set_profiling(cmg_ctx *ctx, int enable);
int cmg_ctx_get_profile(cmg_ctx *ctx, cmg_kernel_profile *out, int max_entries, int *n_entries);
int cmg_ctx_reset_profile(cmg_ctx *ctx);
/* Kernels this context has launched since creation or the last reset. */
int cmg_ctx_launch_count(cmg_ctx *ctx, int64_t *launches);

/* Host-side fault injection for tests (no GPU involvement): the after'th next
 * device allocation made by the library, on any context, fails as if the
 * device were out of memory, so the call in progress returns CMG_ERR_OOM and
 * releases what it allocated; 0 switches it off (the default).
 * INVALID_ARG if negative. */
int cmg_debug_inject_alloc_failure(int64_t after);

/* The FP64 stencil's neighbour sums on their own, for testing that
 * arithmetic (Sec. 5.1.1: the 7-point update sums the six face neighbours).
 * rows is [n][6] FP64, the neighbours of one cell in the order -x, +x, -y,
 * +y, -z, +z; out[i] receives exactly the value the library's FP64 kernels
 * form as that cell's neighbour sum:
 *   which = 0 (colour passes and colour-1 residuals): the first five in one
 *     exact integer-scaled sum rounded once to nearest, ties to even, then one
 *     FP64 addition of the sixth;
 *   which = 1 (colour-0 residuals): all six in the integer-scaled sum.
 * In the integer-scaled sum each operand more than seven binades below the
 * largest is truncated at 2^-59 of the largest's binade; FP64 additions in
 * order take its place when an operand is infinite, NaN or at least 2^1021,
 * or all are below 2^-960.  rows and out are both host or both device memory
 * (mem), owned by the caller; the call returns when out is written.
 * INVALID_ARG on a NULL context or pointer, negative n, which not 0 or 1, or
 * an unknown mem. */
int cmg_debug_neighbour_sum(cmg_ctx *ctx, const double *rows, int64_t n, int which, double *out, cmg_mem mem);

/* Morton keys (Sec. 4.2 Eq. (morton_encode), App. A Alg. 1; B = 21 bits per
 * coordinate): ijk is [n][3] uint32 (i, j, k), keys is [n] uint64.  Both in
 * the same memory space.  Coordinates >= 2^21 give CMG_ERR_KEY_OUT_OF_RANGE. */
int cmg_morton_encode(cmg_ctx *ctx, const uint32_t *ijk, int64_t n, uint64_t *keys, cmg_mem mem);
int cmg_morton_decode(cmg_ctx *ctx, const uint64_t *keys, int64_t n, uint32_t *ijk, cmg_mem mem);

/* 128-bit Morton keys (Sec. 4.2: B = 42 bits per coordinate, levels up to 43
 * with n_x = 1): ijk is [n][3] uint64, keys is [n][2] uint64 = (bits 0..63,
 * bits 64..127) of each key; bit b of i, j, k goes to key bit 3b, 3b+1, 3b+2
 * as in the 64-bit key, which a 128-bit key of coordinates below 2^21 equals
 * in its low word.  Coordinates >= 2^42 give CMG_ERR_KEY_OUT_OF_RANGE. */
int cmg_morton_encode128(cmg_ctx *ctx, const uint64_t *ijk, int64_t n, uint64_t *keys, cmg_mem mem);
int cmg_morton_decode128(cmg_ctx *ctx, const uint64_t *keys, int64_t n, uint64_t *ijk, cmg_mem mem);

/* Build level `level` (>= 1) from n_octs Morton keys (Sec. 4.2; App. B):
 * per-level open-addressing hash table (hash of App. B Eq. (hash_func),
 * linear probing, power-of-two capacity with fill <= 0.7), the neighbour
 * cache of App. D.1 Eq. (nbor_precompute) (directions -x,+x,-y,+y,-z,+z, with
 * periodic wrap on the axes set in periodic_mask), the coarse-fine ghost
 * stencils (morton_nbor_cell, App. B) and the multigrid hierarchy.
 * parent: NULL for a base level (which must then hold all (2^(l-1) n_x)^3
 * octs with periodic_mask = 7 to be solvable), else the level l-1 whose phi
 * gives the Dirichlet values; it must outlive this level.
 * Errors: DUPLICATE_KEY, KEY_OUT_OF_RANGE, MISSING_PARENT, INVALID_ARG, OOM. */
int cmg_level_build(cmg_ctx *ctx, int level, int nx, int periodic_mask, const uint64_t *keys,
                    int64_t n_octs, cmg_mem mem, cmg_level *parent, cmg_level **out);
/* The same with 128-bit keys ([n_octs][2] uint64, see cmg_morton_encode128)
 * for levels up to 43: the hash reduces a key to 64 bits by the XOR of its
 * halves before Eq. (hash_func) (App. B).  The parent must be a 128-bit level
 * too (INVALID_ARG otherwise; likewise for the 64-bit call); everything else
 * (solve, fields, batches) is the same for both widths. */
int cmg_level_build128(cmg_ctx *ctx, int level, int nx, int periodic_mask, const uint64_t *keys,
                       int64_t n_octs, cmg_mem mem, cmg_level *parent, cmg_level **out);
/* 64 or 128. */
int cmg_level_key_bits(const cmg_level *lvl, int *bits);
int cmg_level_destroy(cmg_level *lvl);
int cmg_level_n_octs(const cmg_level *lvl, int64_t *n_octs);
/* Hash capacity (power of two) of the level's table. */
int cmg_level_hash_capacity(const cmg_level *lvl, int64_t *capacity);

/* Hash lookup (App. B): idx[t] = oct index of key q[t], or -1. */
int cmg_level_lookup(cmg_level *lvl, const uint64_t *q, int64_t n, int32_t *idx, cmg_mem mem);
/* The same for a 128-bit level; q is [n][2] uint64.  Each call rejects a
 * level of the other width with INVALID_ARG. */
int cmg_level_lookup128(cmg_level *lvl, const uint64_t *q, int64_t n, int32_t *idx, cmg_mem mem);
/* Neighbour cache, [n][7] int32: column 0 = the oct itself, 1..6 = the
 * same-level neighbour in -x,+x,-y,+y,-z,+z or -1 (App. D.1). */
int cmg_level_get_neighbors(cmg_level *lvl, int32_t *out, cmg_mem mem);
/* morton_nbor_cell (App. B): for each missing neighbour, the father cell in
 * the parent level as (parent oct, octant); (-1,-1) elsewhere.  [n][6][2]. */
int cmg_level_get_father_cells(cmg_level *lvl, int32_t *out, cmg_mem mem);

/* f = four_pi_g * (rho - rho_bar) (Sec. 5.1.1 item (iii)); rho [n][8] FP64. */
int cmg_level_set_density(cmg_level *lvl, const double *rho, cmg_mem mem, double rho_bar, double four_pi_g);
/* phi [n][8] FP64: the initial guess (warm start) of the next solve. */
int cmg_level_set_phi(cmg_level *lvl, const double *phi, cmg_mem mem);
int cmg_level_get_phi(cmg_level *lvl, double *out, cmg_mem mem);
/* cmg_level_get_phi without waiting: the read-back is queued behind the work
 * already queued on the context's stream (e.g. a cmg_level_solve_async), and
 * a host-memory `out` is written by a download on a copy stream of its own,
 * so that work queued afterwards (the next level's solve) overlaps it.
 * `out` must stay valid, and holds phi, once cmg_ctx_synchronize returns.
 * A host-memory argument of any call (cmg_level_set_density, ...) is
 * likewise uploaded on a copy stream, overlapping queued work; those calls
 * return once their upload has finished. */
int cmg_level_get_phi_async(cmg_level *lvl, double *out, cmg_mem mem);
/* r = f - lap_h(phi) of the current phi, [n][8] FP64. */
int cmg_level_get_residual(cmg_level *lvl, double *out, cmg_mem mem);
/* Dirichlet ghost values last interpolated from the parent (by a solve or by
 * CMG_OP_GHOSTS): [n][6][4], face cells of direction d in increasing child
 * index; NaN where the neighbour oct exists. */
int cmg_level_get_ghosts(cmg_level *lvl, double *out, cmg_mem mem);

/* Solve the level (App. G Alg. (vcycle) run as a stationary iteration, red
 * black Gauss-Seidel smoothing of App. D.2 Eq. (gs_update)).  Periodic base
 * levels return zero-mean phi.  stats may be NULL. */
int cmg_level_solve(cmg_level *lvl, const cmg_solve_params *params, cmg_solve_stats *stats);
/* The same solve split in two: cmg_level_solve_async validates the
 * parameters, queues the solve on the context's stream and returns without
 * waiting (errors: INVALID_ARG, including a solve of this level still
 * pending; CUDA); cmg_level_solve_wait waits for it and returns its status
 * and statistics (INVALID_ARG when none is pending).  Queueing the solves of
 * several levels before waiting keeps the GPU busy between them: later calls
 * on the same stream (a finer level's coarse-fine values reading this
 * level's phi, a read-back) are ordered after the queued solve.  With
 * profiling on, the solve runs when queued (its host-driven loop waits every
 * cycle). */
int cmg_level_solve_async(cmg_level *lvl, const cmg_solve_params *params);
int cmg_level_solve_wait(cmg_level *lvl, cmg_solve_stats *stats);

/* Execution schedule of the V-cycle (no effect on the arithmetic): MG levels
 * with at most tail_octs_fp64 (FP64 cycles) / tail_octs_fp32 (FP32 inner
 * cycles) octs, together with every coarser level, run in one launch instead
 * of one launch per operation -- in a single CTA when they all fit one SM (at
 * most 64 octs in FP64, 512 in FP32, and a coarsest level swept in FP64 of at
 * most 64), else in one cooperative launch of one CTA per SM with grid
 * barriers, whose first CTA alone takes the levels that fit one SM.  Defaults
 * 32768 / 2048 (measured on GB300, two-level 128^3 workload: FP64 levels from
 * 32^3 octs down are cheaper under grid barriers than as separate launches;
 * FP32 levels above 512 octs are not, but a refined level's coarsest MG level
 * of a few thousand octs, swept in FP64, is); 0 disables.  Negative values
 * leave the current setting. */
int cmg_level_set_schedule(cmg_level *lvl, int64_t tail_octs_fp64, int64_t tail_octs_fp32);

/* Colour passes of full periodic levels stored in lexicographic oct order (x
 * fastest; every MG level of such a base level, when at least 16 octs per
 * axis): the shared-memory brick kernel stages each CTA's 16 x 4 x 4 octs and
 * their face halo in shared memory and finds neighbours by index arithmetic
 * (App. D.1 and Sec. 9.4 describe the neighbour access it replaces), the
 * neighbour-table kernel reads the level's neighbour cache.  Both give the
 * same bits.  staged = 0: table kernel everywhere; 1 (default): brick kernel
 * for FP32 passes (faster on GB300), table kernel for FP64 passes (faster
 * there); 2: brick kernel for both.  Other levels always use the table
 * kernel.  CMG_ERR_INVALID_ARG for another value. */
int cmg_level_set_stencil(cmg_level *lvl, int staged);

/* SM clock cycles one wait at a grid barrier of the tail kernel may last
 * (default 2^30, about half a second).  A wait that runs out records
 * CMG_ERR_TIMEOUT, every later barrier of that launch stops waiting, and the
 * solve returns CMG_ERR_TIMEOUT with the context still usable (0 makes
 * every wait give up at once: for tests).  CMG_ERR_INVALID_ARG if negative. */
int cmg_level_set_spin_budget(cmg_level *lvl, int64_t cycles);

/* ---- multigrid hierarchy introspection and single steps (for tests) ----
 * m = 0 is the level itself; m + 1 is the coarsening of m (octs = the parents
 * of m's fully active octs, in order of first appearance; a cell is active iff
 * a fully active oct of m refines it). */
int cmg_level_mg_depth(const cmg_level *lvl, int *depth);
int cmg_level_mg_info(const cmg_level *lvl, int m, int64_t *n_octs, int *amr_level);
int cmg_level_mg_keys(cmg_level *lvl, int m, uint64_t *out, cmg_mem mem);
/* Keys of MG level m of a 128-bit level, [n][2] uint64. */
int cmg_level_mg_keys128(cmg_level *lvl, int m, uint64_t *out, cmg_mem mem);
int cmg_level_mg_active(cmg_level *lvl, int m, uint8_t *out /* [n][8] 0/1 */, cmg_mem mem);

typedef enum { CMG_FIELD_PHI = 0, CMG_FIELD_F = 1 } cmg_field;
/* Read / write a field of MG level m as [n][8] FP64 (precision FP64) or FP32
 * (precision MIXED selects the FP32 copy). */
int cmg_level_mg_get(cmg_level *lvl, int m, int field, int precision, void *out, cmg_mem mem);
int cmg_level_mg_set(cmg_level *lvl, int m, int field, int precision, const void *in, cmg_mem mem);

typedef enum {
  CMG_OP_SWEEP = 0,    /* n red-black sweeps on MG level m (ghosts at m = 0) */
  CMG_OP_RESIDUAL = 1, /* *norm2 = sum of r^2 on MG level m */
  CMG_OP_RESTRICT = 2, /* f[m+1] = mean of the children's residual; phi[m+1] = 0 */
  CMG_OP_PROLONG = 3,  /* phi[m] += trilinear interpolation of phi[m+1] */
  CMG_OP_COARSE = 4,   /* the coarsest-level solve (m must be depth - 1) */
  CMG_OP_GHOSTS = 5    /* interpolate the Dirichlet ghosts from the parent's phi */
} cmg_op;
int cmg_level_mg_step(cmg_level *lvl, int m, int op, int precision, int n, double *norm2);

/* ---- batched solve of many independent patches (no counterpart in the paper;
 * its nearest idea is the batched grid buffering of the GPU offload section,
 * "Batched Grid Buffering") ----
 * A batch is a built level whose octs form n_patches independent patches:
 * patch k is octs [offsets[k], offsets[k+1]) of the level (host array,
 * offsets[0] = 0, offsets[n_patches] = n_octs), and no same-level neighbour
 * link, at any multigrid level, joins two patches (else CMG_ERR_INVALID_ARG).
 * cmg_batch_solve runs the whole solve of all patches -- every cycle, every
 * multigrid level, the per-patch residual norms and the stopping test -- in
 * ONE persistent cooperative kernel launch, recorded in a CUDA graph.  Grid
 * barriers inside the kernel spin with a bounded budget; if a barrier gives
 * up the solve returns CMG_ERR_TIMEOUT and the context stays usable.
 * Each patch stops counting when its own relative residual reaches tol;
 * all patches iterate until the slowest one has.  With MIXED precision the
 * cycles are FP32 V-cycles inside FP64 refinement, scaled per patch.
 * The coarsest solve of every patch is n_pre + n_post red-black sweeps (the
 * schedule's), so a patch's result equals the solve of that patch alone.
 * With krylov = 1 every patch runs its own flexible conjugate-gradient
 * iteration (its own alpha and beta; a patch that reached tol stops
 * updating) with the batch's V-cycle from zero as the preconditioner
 * (MIXED: FP32 V-cycles on the residual scaled by its previous norm; needs at
 * least two multigrid levels). */
typedef struct cmg_batch cmg_batch;
typedef struct {
  int threads;        /* threads per block of the persistent kernel (multiple of 32, <= 1024) */
  int blocks_per_sm;  /* resident blocks per SM: grid = SMs x this (capped by occupancy) */
  int n_pre, n_post;  /* red-black sweeps before / after the coarse correction */
  int inner_cycles;   /* MIXED: FP32 V-cycles per FP64 refinement step */
} cmg_batch_schedule;
typedef struct {
  int cycles;          /* V-cycles (FP64) or refinement steps (MIXED) run */
  int status;
  int n_patches;
  int n_converged;     /* patches at or below tol */
  double rel_max;      /* largest per-patch relative residual at return */
  double ms;           /* device time of the solve */
  int64_t cell_updates;
  int64_t grid_barriers;
} cmg_batch_stats;
int cmg_batch_create(cmg_level *lvl, const int64_t *offsets, int n_patches, cmg_batch **out);
int cmg_batch_destroy(cmg_batch *batch);
int cmg_batch_set_schedule(cmg_batch *batch, const cmg_batch_schedule *schedule);
int cmg_batch_get_schedule(cmg_batch *batch, cmg_batch_schedule *schedule);
/* Spin budget of the grid barriers in SM clock cycles (default 2e9, ~1 s). */
int cmg_batch_set_spin_budget(cmg_batch *batch, int64_t cycles);
/* params: tol, max_cycles, fixed_cycles, precision and krylov are used; the
 * sweep counts come from the batch schedule. */
int cmg_batch_solve(cmg_batch *batch, const cmg_solve_params *params, cmg_batch_stats *stats);
/* Per-patch results of the last solve (host arrays of n_patches; any may be
 * NULL): relative residual, cycle at which the patch reached tol (-1 if it
 * did not), and ||f - L 0|| of the patch. */
int cmg_batch_patch_stats(cmg_batch *batch, double *rel, int32_t *converged_at, double *norm0);
/* Times candidate schedules with full solves (with params' precision and
 * krylov) on the batch's current data, keeps the fastest and sets it; phi of
 * the level is restored afterwards.  Two stages: block shapes {256, 512
 * threads} x {1, 2, 4 blocks per SM} (x {1, 2} inner cycles in MIXED) with
 * V(2,2), then V(1,1), V(2,3), V(3,2), V(3,3) with the best shape.
 * best / best_ms may be NULL. */
int cmg_batch_autotune(cmg_batch *batch, const cmg_solve_params *params, cmg_batch_schedule *best,
                       double *best_ms);

/* ---- learned warm start (no counterpart in the paper) ----
 * A 3-level 3-D U-Net (16/32/64 channels) on periodic D^3 blocks predicts
 * phi from (rho, phi_prev); its prediction is the initial guess of a level
 * solve.  Layers (3x3x3 convs with circular padding, bias and ReLU):
 *   enc0a 16->16, enc0b 16->16 (D) | pool | enc1a 16->32, enc1b 32->32 (D/2) |
 *   pool | bota 32->64, botb 64->64 (D/4) | up x2, concat with enc1b |
 *   dec1a 96->32, dec1b 32->32 | up x2, concat with enc0b | dec0a 48->16,
 *   dec0b 16->16 | head 1x1x1 16->1 (linear) = delta.
 * Input channels: (rho - mean)/std, field/rms(field), 14 zeros; the
 * prediction is base + c * rms(field) * delta (base defaults to field; c is
 * the output scale, 1 unless set).  For the
 * warm start, field = the FP64 residual f - L phi_prev of the previous
 * potential for the new density and base = phi_prev, so the network learns
 * the correction of phi_prev.  Parameters: FP32 master
 * vector (per layer [Cout][27][Cin] weights then biases; head 16 + 1);
 * convolutions run on BF16 weights and BF16 activations with FP32
 * accumulation (tensor cores), the head and the optimiser in FP32.
 * Fields are dense [batch][D][D][D] (z, y, x) FP32 arrays in `mem`. */
typedef struct cmg_unet cmg_unet;
/* grid_dim: multiple of 16; max_batch: samples per call. */
int cmg_unet_create(cmg_ctx *ctx, int grid_dim, int max_batch, cmg_unet **out);
int cmg_unet_destroy(cmg_unet *net);
int cmg_unet_n_params(const cmg_unet *net, int64_t *n);
/* Replace the master parameters (resets the Adam moments). */
int cmg_unet_set_params(cmg_unet *net, const float *params, cmg_mem mem);
int cmg_unet_get_params(cmg_unet *net, float *out, cmg_mem mem);
/* Convolution kernels: 1 (default) = tcgen05 tensor-core kernels with TMEM
 * accumulators on every grid whose size is a multiple of 16 (the warp-level
 * mma.sync kernels below that); 0 = the warp-level mma.sync kernels
 * everywhere.  Both compute the same convolutions in BF16 x BF16 -> FP32. */
int cmg_unet_set_kernels(cmg_unet *net, int tensor_path);
/* Output scale c > 0 (finite), kept with the network: the trainer sets it to
 * the typical size of (target - base)/rms(field) so that delta is O(1).
 * CMG_ERR_INVALID_ARG otherwise. */
int cmg_unet_set_output_scale(cmg_unet *net, float scale);
int cmg_unet_get_output_scale(const cmg_unet *net, float *scale);
/* Inference: prediction and/or delta (either may be NULL); base may be NULL.
 * Every wait inside the tensor-core kernels is bounded; an expired wait is
 * reported as CMG_ERR_TIMEOUT by the next call that synchronises (host
 * buffers, or cmg_unet_gradients with a loss). */
int cmg_unet_forward(cmg_unet *net, const float *rho, const float *field, const float *base, int batch,
                     float *pred, float *delta, cmg_mem mem);
/* Loss = mean over all voxels of (delta - (target - base)/(c rms(field)))^2 and its
 * gradient (kept inside for cmg_unet_adam_step; copied to grads if not NULL;
 * loss is written as a host double when mem is HOST, else it is the device
 * sum of squared errors). */
int cmg_unet_gradients(cmg_unet *net, const float *rho, const float *field, const float *base, const float *target,
                       int batch, float *grads, double *loss, cmg_mem mem);
/* One Adam step on the master parameters with the last gradients. */
int cmg_unet_adam_step(cmg_unet *net, float lr, float beta1, float beta2, float eps);
/* Gradient-norm clipping of the Adam steps (training robustness; no
 * counterpart in the paper): with k >= 1 each step's gradient 2-norm is
 * capped at k times the running mean (weight 0.05 per step) of the earlier
 * steps' capped norms, once 20 steps have formed that mean; computed on the
 * device inside cmg_unet_adam_step, without a host synchronisation.  k = 0
 * switches it off (the default).  INVALID_ARG for 0 < k < 1.
 * cmg_unet_set_params resets the running mean and the counters. */
int cmg_unet_set_grad_clip(cmg_unet *net, float k);
/* The clipping record (synchronises the stream): last step's gradient norm
 * (before capping), the running mean, steps seen and steps capped; any
 * pointer may be NULL. */
int cmg_unet_grad_clip_stats(cmg_unet *net, double *last_norm, double *mean_norm, int64_t *steps, int64_t *clipped);
/* Device copy between a dense [D][D][D] (z, y, x) FP64 field and the oct-major
 * [n][8] field of the full periodic level whose octs are listed x fastest
 * (to_octs = 1: dense -> octs; 0: octs -> dense).  Both device pointers. */
int cmg_dense_octs(cmg_ctx *ctx, const double *src, int grid_dim, double *dst, int to_octs);

/* ---- sharded level solve (App. G, GPU V-cycle algorithm; Sec. 9.5, halo
 * exchange between GPUs) ----
 * Building blocks of a V-cycle split over ranks by owner-computes: each rank
 * holds a replica of the level (built from the same keys, sorted so that each
 * rank's octs, and the octs of every coarser MG level, form one contiguous
 * range), runs every operation on its own range [lo, hi) only, and exchanges
 * the cells other ranks read between operations (cmg_level_mg_gather /
 * cmg_level_mg_scatter).  The range kernels are the whole-level kernels'
 * per-oct bodies, so a sharded V-cycle computes the single-rank result cell
 * for cell; only the order of the norm sums differs.  The driver that orders
 * the calls and the exchanges is paper_2604_06035_gb300/shard.py.  FP64 only.
 *
 * cmg_level_mg_step_range(lvl, m, op, arg, lo, hi, value): octs [lo, hi) of
 * MG level m (0 <= lo <= hi <= octs of the level, else CMG_ERR_INVALID_ARG),
 * on the context's stream, synchronised before return.
 *   CMG_OPR_SWEEP     one red-black colour pass; arg = colour (0 red, 1
 *                     black) | 2 when the other colour is known to be zero
 *                     (the first pass after a restriction, phi = g)
 *   CMG_OPR_RESIDUAL  *value = sum of r^2 over the range; arg = 1 when the
 *                     last operation on the level was a colour-1 pass (the
 *                     colour-1 residuals are then exactly zero and skipped)
 *   CMG_OPR_RESTRICT  the range's fully active octs write their father
 *                     cell's source (mean of the 8 residuals) and zero its
 *                     phi on MG level m + 1; arg as for CMG_OPR_RESIDUAL
 *   CMG_OPR_PROLONG   phi += trilinear interpolation of phi at m + 1; arg =
 *                     1 when a colour-0 pass follows (only colour-1 cells are
 *                     corrected, the colour-0 corrections being dead)
 *   CMG_OPR_SUM_PHI   *value = sum of phi over the range's cells
 *   CMG_OPR_SHIFT_PHI phi -= *value on the range's cells
 * cmg_level_mg_gather / _scatter(lvl, m, field, cells, n, buf): copy n cells
 * of MG level m between the level and buf.  field 0 = phi, 1 = the stored
 * source (the solver's internal scaling g = -h^2 f / 6, moved unchanged so
 * that replicas stay bit-identical).  cells[k] = oct * 8 + child (child =
 * bx + 2 by + 4 bz), DEVICE int32; buf DEVICE double[n]; both owned by the
 * caller.  An index outside the level is CMG_ERR_INVALID_ARG (the other cells
 * are still copied). */
enum {
  CMG_OPR_SWEEP = 0,
  CMG_OPR_RESIDUAL = 1,
  CMG_OPR_RESTRICT = 2,
  CMG_OPR_PROLONG = 3,
  CMG_OPR_SUM_PHI = 4,
  CMG_OPR_SHIFT_PHI = 5
};
int cmg_level_mg_step_range(cmg_level *lvl, int m, int op, int arg, int64_t lo, int64_t hi, double *value);
int cmg_level_mg_gather(cmg_level *lvl, int m, int field, const int32_t *cells, int64_t n, double *out);
int cmg_level_mg_scatter(cmg_level *lvl, int m, int field, const int32_t *cells, int64_t n, const double *in);

/* ---- residual norm without allocation (the paper has no counterpart) ----
 * The level objects above allocate device memory when they are built, and
 * their residual norm reduces through scratch the level owns.  Callers that
 * cannot allocate when they need a residual check -- real-time loops that
 * forbid allocation after start-up (cudaMalloc can block and synchronise the
 * device), hosts whose device memory is a fixed arena handed out by their own
 * allocator -- can use this entry point: it allocates nothing and reduces
 * through a fixed scratch array compiled into the library (512 KiB, held by
 * every GPU that loads the library until the process exits).
 *
 * Computes *norm2 = sum over cells of r^2, r = f - (sum_6 phi_nb - 6 phi) / h^2
 * (the residual of Sec. 5.1.1 item (iii)), on the current device, on `stream`
 * (a cudaStream_t, NULL = legacy default stream).  All pointers are DEVICE
 * memory owned by the caller, in the public layouts: neighbors [n][7] as
 * cmg_level_get_neighbors returns it (-1 = no same-level neighbour), ghosts
 * [n][6][4] as cmg_level_get_ghosts returns it or NULL (missing neighbours
 * then count as 0), phi and f [n][8] FP64, norm2 one double.  The result is
 * written asynchronously; synchronise the stream before reading it.
 * Limits and behaviour: n_octs <= 2^24 (16 777 216), else CMG_ERR_INVALID_ARG;
 * the first call on a device looks up the scratch array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture;
 * all calls share the scratch array, so calls that overlap on the GPU race
 * and the caller must serialise them.  The looked-up address is kept for the
 * life of the process: after a cudaDeviceReset (or any other teardown of the
 * device's primary context) the entry point must not be called again in that
 * process.  Returns CMG_OK, CMG_ERR_INVALID_ARG or CMG_ERR_CUDA; it does not
 * set cmg_last_error(). */
int cmg_residual_norm2_noalloc(const int32_t *neighbors, const double *ghosts, const double *phi, const double *f,
                               int64_t n_octs, double h, double *norm2, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* CMG_H */
