/*
 * oracle.h -- plain, slow, FP64 CPU oracle for the level-by-level multigrid
 * Poisson solve on oct grids (cuRAMSES, arXiv 2604.06035).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may include, link or
 * call this code: only tests/, __graft_entry__.smoke() and bench.py's
 * cpu_baseline / reference legs use it.  It shares no code with the CUDA
 * library (no headers, helpers, tables or constants).
 *
 * Every function restates the paper's definition in the most direct form:
 *   Morton keys           Sec. 4.2 Eq. (morton_encode), App. A Alg. 1
 *   neighbour keys        Sec. 4.2, App. A Alg. 2
 *   parent/child keys     Sec. 4.2 (M>>3, (M<<3)|i_child)
 *   hash table            App. B Eq. (hash_func), linear probing, pow2 capacity, fill <= 0.7
 *   neighbour cache       App. D.1 Eq. (nbor_precompute), morton_nbor_grid / morton_nbor_cell (App. B)
 *   RBGS update           App. D.2 Eq. (gs_update)
 *   residual + norm       Sec. 5.1.1 item (iii), App. D.2
 *   restriction           Sec. 5.1.1 (mean of the eight children)
 *   prolongation          Sec. 5.1.1 (trilinear interpolation of the correction)
 *   V-cycle               App. G Alg. (vcycle), without halo exchanges
 * Readings where the paper is silent are listed in the repository design notes
 * (ghost interpolation, masked coarse levels, coarsest solve, stop test).
 *
 * Status codes match the values of the product library so that tests can
 * compare error behaviour, but the constants are defined here independently.
 */
#ifndef CMG_ORACLE_H
#define CMG_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  OR_OK = 0,
  OR_ERR_INVALID_ARG = -1,
  OR_ERR_DUPLICATE_KEY = -2,
  OR_ERR_KEY_OUT_OF_RANGE = -3,
  OR_ERR_MISSING_PARENT = -4,
  OR_ERR_OOM = -5,
  OR_ERR_NOT_CONVERGED = -7,
  OR_ERR_DIVERGED = -8
};

/* ---- threads ----
 * Threads of the oracle's per-oct loops (default 1; needs an OpenMP build,
 * else stays 1).  Returns the count now in force.  Results are bit-identical
 * for every thread count: only loops whose iterations write disjoint cells
 * and read nothing another iteration writes run in parallel, and every sum
 * over cells stays serial. */
int or_set_threads(int n);
int or_get_threads(void);

/* ---- keys ---- */
uint64_t or_morton_encode(uint32_t i, uint32_t j, uint32_t k);
void or_morton_decode(uint64_t m, uint32_t *i, uint32_t *j, uint32_t *k);
void or_encode_many(const uint32_t *ijk, int64_t n, uint64_t *out);
void or_decode_many(const uint64_t *keys, int64_t n, uint32_t *ijk);
/* 128-bit keys (Sec. 4.2, B = 42): ijk [n][3] uint64 <-> keys [n][2] uint64
 * (bits 0..63, bits 64..127). */
void or_encode128_many(const uint64_t *ijk, int64_t n, uint64_t *out);
void or_decode128_many(const uint64_t *keys, int64_t n, uint64_t *ijk);
/* Neighbour key of m in direction d (0..5 = -x,+x,-y,+y,-z,+z) on a grid of
 * n_per_dim octs per axis; periodic wrap on axes whose bit is set in
 * periodic_mask, else -1 when the step leaves [0, n_per_dim). */
int64_t or_neighbor_key(uint64_t m, int d, uint32_t n_per_dim, int periodic_mask);
uint64_t or_hash_fn(uint64_t h);
int64_t or_hash_capacity_for(int64_t n);

/* ---- levels ---- */
typedef struct or_level or_level;

int or_level_build(int level, int nx, int periodic_mask, const uint64_t *keys,
                   int64_t n, or_level *parent, or_level **out);
/* The same with 128-bit keys [n][2] (Sec. 4.2, B = 42, levels up to 43); the
 * hash reduces a key by the XOR of its halves (App. B). */
int or_level_build128(int level, int nx, int periodic_mask, const uint64_t *keys, int64_t n, or_level *parent,
                      or_level **out);
void or_level_free(or_level *L);
int64_t or_level_n_octs(const or_level *L);
int64_t or_level_hash_capacity(const or_level *L);
/* Hash-table contents: slot keys (UINT64_MAX = empty) and values. */
void or_level_hash_dump(const or_level *L, uint64_t *keys, int32_t *vals);
void or_level_lookup(const or_level *L, const uint64_t *q, int64_t n, int32_t *out);
void or_level_lookup128(const or_level *L, const uint64_t *q, int64_t n, int32_t *out);
void or_level_neighbors(const or_level *L, int32_t *out /* [n][7] */);
/* Father cell of each missing same-level neighbour: [n][6][2] = (parent oct,
 * octant), (-1,-1) where the neighbour exists or no parent is given. */
void or_level_father_cells(const or_level *L, int32_t *out);

void or_level_set_density(or_level *L, const double *rho, double rho_bar, double four_pi_g);
void or_level_set_f(or_level *L, const double *f);
void or_level_set_phi(or_level *L, const double *phi);
void or_level_get_phi(const or_level *L, double *out);
void or_level_get_f(const or_level *L, double *out);
/* Dirichlet ghost values from the parent's current phi: [n][6][4]; face cells
 * of direction d ordered by increasing child index; NaN where the neighbour
 * oct exists. */
void or_level_compute_ghosts(or_level *L);
void or_level_get_ghosts(const or_level *L, double *out);

/* ---- multigrid hierarchy introspection (m = 0 is the level itself) ---- */
int or_level_mg_depth(const or_level *L);
int64_t or_level_mg_n_octs(const or_level *L, int m);
int or_level_mg_lev(const or_level *L, int m);
void or_level_mg_keys(const or_level *L, int m, uint64_t *out);
void or_level_mg_keys128(const or_level *L, int m, uint64_t *out);
void or_level_mg_active(const or_level *L, int m, uint8_t *out /* [n][8] */);
/* field: 0 = phi, 1 = f, 2 = r */
void or_level_mg_get(const or_level *L, int m, int field, double *out);
void or_level_mg_set(or_level *L, int m, int field, const double *in);

/* ---- single steps (use_ghost = 1: Dirichlet ghosts at m = 0) ---- */
void or_rb_sweeps(or_level *L, int m, int n_sweeps, int use_ghost);
void or_rb_colour_pass(or_level *L, int m, int color, int use_ghost); /* one colour of a sweep */
double or_residual(or_level *L, int m, int use_ghost); /* writes r, returns sum r^2 */
void or_restrict(or_level *L, int m);    /* f[m+1] from r[m]; phi[m+1] = 0 */
void or_prolong(or_level *L, int m);     /* phi[m] += P phi[m+1] */
void or_coarse_solve(or_level *L, int coarse_sweeps);

typedef struct {
  double tol;
  int max_cycles;
  int n_pre, n_post;
  int coarse_sweeps;
  int fixed_cycles; /* > 0: run exactly this many cycles, ignore tol */
} or_params;

typedef struct {
  int cycles;
  double rel_initial;
  double rel_final;
  double norm0;
  double rel_history[256];
} or_stats;

int or_level_solve(or_level *L, const or_params *p, or_stats *st);
/* Mixed precision reference: FP64 residual and accumulation, FP32 inner V-cycle
 * on r/||r|| (FP64 coarsest solve).  inner_cycles V-cycles per outer step. */
int or_level_solve_mixed(or_level *L, const or_params *p, int inner_cycles, or_stats *st);
/* Multigrid-preconditioned conjugate gradients (App. D.2: MG as the CG
 * preconditioner).  Flexible (Polak-Ribiere) beta, since a V-cycle with red
 * first in both smoothing legs is not exactly symmetric; preconditioner = one
 * V-cycle from zero on the residual with homogeneous coarse-fine values;
 * operator applied with homogeneous values after the initial (true)
 * residual; zero-mean preconditioned vectors on a periodic level.  cycles =
 * CG iterations (one V-cycle and one operator application each); the
 * relative residual is the CG recurrence's. */
int or_level_solve_pcg(or_level *L, const or_params *p, or_stats *st);

#ifdef __cplusplus
}
#endif
#endif
