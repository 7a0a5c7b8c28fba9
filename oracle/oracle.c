/*
 * oracle.c -- plain FP64 CPU oracle for the level-by-level multigrid Poisson
 * solve on oct grids (cuRAMSES, arXiv 2604.06035).  TEST INFRASTRUCTURE ONLY:
 * see oracle.h for who may use it and which passage each step follows.
 *
 * Deliberately simple: every neighbour, parent and interpolation cell is found
 * from integer coordinates and a hash lookup, exactly as the paper describes
 * (Sec. 4.2, App. A, App. B), with no blocking, fusion or reordering.
 * Compiled with -O2 -ffp-contract=off so that the arithmetic is the one written.
 */
#include "oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the per-oct loops (1 unless or_set_threads asks for more).  A
 * loop runs in parallel only where every iteration writes its own cells and
 * reads nothing another iteration writes: the cells of one colour in a
 * red-black pass (their neighbours are all of the other colour), the residual
 * of each cell, restriction, prolongation, ghost values, element-wise vector
 * updates.  Sums over cells (norms, dot products, the mean) stay serial in
 * the same order, so results are bit-identical for any thread count. */
static int or_threads = 1;
#ifdef _OPENMP
#define OR_PRAGMA(x) _Pragma(#x)
#define OR_PAR_FOR OR_PRAGMA(omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1))
/* the same, OR-reducing an int flag set by any iteration */
#define OR_PAR_FOR_OR(v) \
  OR_PRAGMA(omp parallel for schedule(static) num_threads(or_threads) if (or_threads > 1) reduction(| : v))
#else
#define OR_PAR_FOR
#define OR_PAR_FOR_OR(v)
#endif

int or_set_threads(int n) {
#ifdef _OPENMP
  or_threads = n < 1 ? 1 : n;
#else
  (void)n;
  or_threads = 1;
#endif
  return or_threads;
}
int or_get_threads(void) { return or_threads; }

#define MORTON_BITS 21      /* 64-bit keys (Sec. 4.2) */
#define MORTON_BITS_WIDE 42 /* 128-bit keys (Sec. 4.2) */

/* Every level keeps its keys as 128-bit integers: a 64-bit key (B = 21) is the
 * same integer with its upper half zero, and its hash (the XOR fold of the two
 * halves, App. B) is the key itself. */
typedef unsigned __int128 okey;
#define EMPTY_KEY (~(okey)0)

/* ------------------------------------------------------------------ keys */

/* Sec. 4.2 Eq. (morton_encode), App. A Alg. 1: bit b of i goes to bit 3b,
 * of j to 3b+1, of k to 3b+2, for b = 0..B-1 with B = 21. */
uint64_t or_morton_encode(uint32_t i, uint32_t j, uint32_t k) {
  uint64_t m = 0;
  for (int b = 0; b < MORTON_BITS; b++) {
    m |= (uint64_t)((i >> b) & 1u) << (3 * b);
    m |= (uint64_t)((j >> b) & 1u) << (3 * b + 1);
    m |= (uint64_t)((k >> b) & 1u) << (3 * b + 2);
  }
  return m;
}

/* Inverse of Alg. 1. */
void or_morton_decode(uint64_t m, uint32_t *i, uint32_t *j, uint32_t *k) {
  uint32_t a = 0, b2 = 0, c = 0;
  for (int b = 0; b < MORTON_BITS; b++) {
    a |= (uint32_t)((m >> (3 * b)) & 1u) << b;
    b2 |= (uint32_t)((m >> (3 * b + 1)) & 1u) << b;
    c |= (uint32_t)((m >> (3 * b + 2)) & 1u) << b;
  }
  *i = a;
  *j = b2;
  *k = c;
}

void or_encode_many(const uint32_t *ijk, int64_t n, uint64_t *out) {
  for (int64_t t = 0; t < n; t++) out[t] = or_morton_encode(ijk[3 * t], ijk[3 * t + 1], ijk[3 * t + 2]);
}

void or_decode_many(const uint64_t *keys, int64_t n, uint32_t *ijk) {
  for (int64_t t = 0; t < n; t++) or_morton_decode(keys[t], &ijk[3 * t], &ijk[3 * t + 1], &ijk[3 * t + 2]);
}

/* App. A Alg. 1 with B = 42 on 128-bit keys. */
static okey key_encode(uint64_t i, uint64_t j, uint64_t k) {
  okey m = 0;
  /* bits above the highest set coordinate bit contribute nothing */
  for (int b = 0; b < MORTON_BITS_WIDE && ((i | j | k) >> b) != 0; b++) {
    m |= (okey)((i >> b) & 1u) << (3 * b);
    m |= (okey)((j >> b) & 1u) << (3 * b + 1);
    m |= (okey)((k >> b) & 1u) << (3 * b + 2);
  }
  return m;
}

static void key_decode(okey m, uint64_t c[3]) {
  c[0] = c[1] = c[2] = 0;
  for (int b = 0; b < MORTON_BITS_WIDE && (m >> (3 * b)) != 0; b++) {
    c[0] |= (uint64_t)((m >> (3 * b)) & 1u) << b;
    c[1] |= (uint64_t)((m >> (3 * b + 1)) & 1u) << b;
    c[2] |= (uint64_t)((m >> (3 * b + 2)) & 1u) << b;
  }
}

static okey key_from_words(const uint64_t *w) { return ((okey)w[1] << 64) | (okey)w[0]; }
static void key_to_words(okey k, uint64_t *w) {
  w[0] = (uint64_t)k;
  w[1] = (uint64_t)(k >> 64);
}

void or_encode128_many(const uint64_t *ijk, int64_t n, uint64_t *out) {
  for (int64_t t = 0; t < n; t++) key_to_words(key_encode(ijk[3 * t], ijk[3 * t + 1], ijk[3 * t + 2]), out + 2 * t);
}

void or_decode128_many(const uint64_t *keys, int64_t n, uint64_t *ijk) {
  for (int64_t t = 0; t < n; t++) key_decode(key_from_words(keys + 2 * t), ijk + 3 * t);
}

/* App. A Alg. 2 on keys of either width: returns 0 for "no neighbour". */
static int key_neighbor(okey m, int d, uint64_t n_per_dim, int periodic_mask, okey *out) {
  uint64_t c[3];
  key_decode(m, c);
  int axis = d / 2;
  int64_t v = (int64_t)c[axis] + ((d & 1) ? 1 : -1);
  if ((periodic_mask >> axis) & 1) {
    v = ((v % (int64_t)n_per_dim) + (int64_t)n_per_dim) % (int64_t)n_per_dim;
  } else if (v < 0 || v >= (int64_t)n_per_dim) {
    return 0;
  }
  c[axis] = (uint64_t)v;
  *out = key_encode(c[0], c[1], c[2]);
  return 1;
}

/* App. A Alg. 2: decode, step one cell along the axis of direction d, wrap
 * periodically (mod n_d) or report "no neighbour" (-1), re-encode. */
int64_t or_neighbor_key(uint64_t m, int d, uint32_t n_per_dim, int periodic_mask) {
  uint32_t c[3];
  or_morton_decode(m, &c[0], &c[1], &c[2]);
  int axis = d / 2;
  int64_t v = (int64_t)c[axis] + ((d & 1) ? 1 : -1);
  if ((periodic_mask >> axis) & 1) {
    v = ((v % (int64_t)n_per_dim) + (int64_t)n_per_dim) % (int64_t)n_per_dim;
  } else if (v < 0 || v >= (int64_t)n_per_dim) {
    return -1;
  }
  c[axis] = (uint32_t)v;
  return (int64_t)or_morton_encode(c[0], c[1], c[2]);
}

/* App. B Eq. (hash_func), all arithmetic modulo 2^64 with logical shifts. */
uint64_t or_hash_fn(uint64_t h) {
  const uint64_t phi1 = 2654435761ULL;
  const uint64_t phi2 = 0x9E3779B97F4A7C15ULL;
  uint64_t t = ((h * phi1) ^ (h >> 16)) * phi2;
  return t ^ (t >> 13);
}

/* App. B: a key is reduced to 64 bits before Eq. (hash_func) -- the XOR of its
 * upper and lower halves (128-bit keys), the key itself (64-bit keys). */
static uint64_t key_hash(okey k) { return or_hash_fn((uint64_t)k ^ (uint64_t)(k >> 64)); }

/* Smallest power of two with fill n/cap <= 0.7 (App. B). */
int64_t or_hash_capacity_for(int64_t n) {
  int64_t cap = 1;
  while (10 * n > 7 * cap) cap *= 2;
  return cap;
}

/* ------------------------------------------------------------- hash table */

typedef struct {
  int64_t cap;
  okey *key;
  int32_t *val;
} hashtab;

static int ht_init(hashtab *h, int64_t n) {
  h->cap = or_hash_capacity_for(n);
  h->key = (okey *)malloc(sizeof(okey) * h->cap);
  h->val = (int32_t *)malloc(sizeof(int32_t) * h->cap);
  if (!h->key || !h->val) return OR_ERR_OOM;
  for (int64_t s = 0; s < h->cap; s++) {
    h->key[s] = EMPTY_KEY;
    h->val[s] = -1;
  }
  return OR_OK;
}

static void ht_free(hashtab *h) {
  free(h->key);
  free(h->val);
  h->key = NULL;
  h->val = NULL;
}

/* Linear probing from slot h(M) & (cap-1) (App. B). */
static int ht_insert(hashtab *h, okey k, int32_t v) {
  uint64_t mask = (uint64_t)h->cap - 1;
  uint64_t s = key_hash(k) & mask;
  for (;;) {
    if (h->key[s] == EMPTY_KEY) {
      h->key[s] = k;
      h->val[s] = v;
      return OR_OK;
    }
    if (h->key[s] == k) return OR_ERR_DUPLICATE_KEY;
    s = (s + 1) & mask;
  }
}

static int32_t ht_find(const hashtab *h, okey k) {
  uint64_t mask = (uint64_t)h->cap - 1;
  uint64_t s = key_hash(k) & mask;
  for (;;) {
    if (h->key[s] == EMPTY_KEY) return -1;
    if (h->key[s] == k) return h->val[s];
    s = (s + 1) & mask;
  }
}

/* ----------------------------------------------------------------- levels */

typedef struct {
  int lev;
  int64_t n;
  okey *key;
  hashtab ht;
  int32_t *nbr;    /* [n][7]: j = 0 self, 1..6 = -x,+x,-y,+y,-z,+z */
  uint8_t *active; /* [n][8] */
  int32_t *child;  /* [n][8]: oct at the next finer MG level refining this cell */
  double *phi, *f, *r;
  float *phi32, *f32, *r32;
} mglev;

struct or_level {
  int lev, nx, pmask;
  int64_t n;
  or_level *parent;
  int depth;
  mglev *mg;       /* mg[0] = the level itself, mg[m+1] = one coarsening of mg[m] */
  int32_t *father; /* [n][6][2] */
  double *ghost;   /* [n][6][4] */
  int periodic_full;
};

static uint64_t octs_per_dim(int lev, int nx) { return (uint64_t)nx << (lev - 1); }
static uint64_t cells_per_dim(int lev, int nx) { return (uint64_t)nx << lev; }
static double cell_h(int lev, int nx) { return ldexp(1.0, -lev) / (double)nx; }

static int parity(int c) { return ((c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1)) & 1; }

static int build_nbr(mglev *g, uint64_t npd, int pmask) {
  g->nbr = (int32_t *)malloc(sizeof(int32_t) * 7 * (g->n ? g->n : 1));
  if (!g->nbr) return OR_ERR_OOM;
  OR_PAR_FOR
  for (int64_t i = 0; i < g->n; i++) {
    g->nbr[7 * i] = (int32_t)i;
    for (int d = 0; d < 6; d++) {
      okey nk;
      g->nbr[7 * i + 1 + d] = key_neighbor(g->key[i], d, npd, pmask, &nk) ? ht_find(&g->ht, nk) : -1;
    }
  }
  return OR_OK;
}

static int alloc_fields(mglev *g) {
  int64_t m = 8 * (g->n ? g->n : 1);
  g->phi = (double *)calloc(m, sizeof(double));
  g->f = (double *)calloc(m, sizeof(double));
  g->r = (double *)calloc(m, sizeof(double));
  g->active = (uint8_t *)calloc(m, 1);
  g->child = (int32_t *)malloc(sizeof(int32_t) * m);
  if (!g->phi || !g->f || !g->r || !g->active || !g->child) return OR_ERR_OOM;
  for (int64_t t = 0; t < m; t++) g->child[t] = -1;
  g->phi32 = g->f32 = g->r32 = NULL;
  return OR_OK;
}

static void free_mg(mglev *g) {
  free(g->key);
  ht_free(&g->ht);
  free(g->nbr);
  free(g->active);
  free(g->child);
  free(g->phi);
  free(g->f);
  free(g->r);
  free(g->phi32);
  free(g->f32);
  free(g->r32);
}

/* Global cell coordinates at level lev of child c of the oct with key k. */
static void cell_coords(okey k, int c, uint64_t X[3]) {
  uint64_t o[3];
  key_decode(k, o);
  for (int a = 0; a < 3; a++) X[a] = 2 * o[a] + ((c >> a) & 1);
}

/* Look up the cell at global coordinates Y (level lev, possibly outside the
 * box) in MG level g: returns 1 and (oct, child) if its oct exists. */
static int find_cell(const hashtab *ht, int64_t Y[3], int lev, int nx, int pmask, int32_t *oct, int *child) {
  int64_t ncell = (int64_t)cells_per_dim(lev, nx);
  uint64_t o[3];
  int ch = 0;
  for (int a = 0; a < 3; a++) {
    int64_t v = Y[a];
    if ((pmask >> a) & 1) {
      v = ((v % ncell) + ncell) % ncell;
    } else if (v < 0 || v >= ncell) {
      return 0;
    }
    o[a] = (uint64_t)(v >> 1);
    ch |= (int)(v & 1) << a;
  }
  int32_t idx = ht_find(ht, key_encode(o[0], o[1], o[2]));
  if (idx < 0) return 0;
  *oct = idx;
  *child = ch;
  return 1;
}

/* Trilinear cell-centred interpolation of a coarse field (level lev-1) at the
 * centre of the fine cell X (level lev): the coarse cell containing X and its
 * neighbours toward X's octant, 1-D weights 3/4 (own) and 1/4 (neighbour).
 * Sec. 5.1.1 (trilinear prolongation); also the coarse-fine ghost value.
 * Absent coarse cells: *missing is set and they contribute 0. */
static double interp_coarse(const hashtab *ht, const double *field, int clev, int nx, int pmask,
                            const uint64_t X[3], int *missing) {
  int64_t Xc[3], o[3];
  for (int a = 0; a < 3; a++) {
    Xc[a] = (int64_t)(X[a] >> 1);
    o[a] = (X[a] & 1) ? 1 : -1;
  }
  double sum = 0.0;
  for (int cz = 0; cz < 2; cz++)
    for (int cy = 0; cy < 2; cy++)
      for (int cx = 0; cx < 2; cx++) {
        double w = (cx ? 0.25 : 0.75) * (cy ? 0.25 : 0.75) * (cz ? 0.25 : 0.75);
        int64_t Y[3] = {Xc[0] + cx * o[0], Xc[1] + cy * o[1], Xc[2] + cz * o[2]};
        int32_t oct;
        int ch;
        if (find_cell(ht, Y, clev, nx, pmask, &oct, &ch)) {
          sum += w * field[8 * (int64_t)oct + ch];
        } else {
          *missing = 1;
        }
      }
  return sum;
}

/* Remove bit a from a 3-bit child index: rank of a face cell on its face. */
static int face_rank(int c, int a) {
  if (a == 0) return c >> 1;
  if (a == 1) return (c & 1) | ((c >> 2) << 1);
  return c & 3;
}

/* Position of the ghost cell across face d of cell (k, c) at level lev. */
static int ghost_position(okey k, int c, int d, int lev, int nx, int pmask, uint64_t G[3]) {
  cell_coords(k, c, G);
  int a = d / 2;
  int64_t v = (int64_t)G[a] + ((d & 1) ? 1 : -1);
  int64_t ncell = (int64_t)cells_per_dim(lev, nx);
  if ((pmask >> a) & 1) {
    v = ((v % ncell) + ncell) % ncell;
  } else if (v < 0 || v >= ncell) {
    return 0;
  }
  G[a] = (uint64_t)v;
  return 1;
}

/* Level build on 128-bit keys; bits = 21 or 42 sets the coordinate range. */
static int level_build(int level, int nx, int pmask, const okey *keys, int64_t n, or_level *parent,
                       or_level **out, int bits) {
  *out = NULL;
  if (level < 1 || nx < 1 || nx > (1 << 20) || n < 0 || pmask < 0 || pmask > 7) return OR_ERR_INVALID_ARG;
  if (level > bits + 1 || (uint64_t)nx << (level - 1) > (1ull << bits)) return OR_ERR_INVALID_ARG;
  if (parent && (parent->lev != level - 1 || parent->nx != nx || parent->pmask != pmask))
    return OR_ERR_INVALID_ARG;
  uint64_t npd = octs_per_dim(level, nx);
  for (int64_t t = 0; t < n; t++) {
    if (bits == MORTON_BITS ? (keys[t] >> 63) != 0 : (keys[t] >> 126) != 0) return OR_ERR_KEY_OUT_OF_RANGE;
    uint64_t c[3];
    key_decode(keys[t], c);
    if (key_encode(c[0], c[1], c[2]) != keys[t]) return OR_ERR_KEY_OUT_OF_RANGE;
    if (c[0] >= npd || c[1] >= npd || c[2] >= npd) return OR_ERR_KEY_OUT_OF_RANGE;
  }
  or_level *L = (or_level *)calloc(1, sizeof(or_level));
  if (!L) return OR_ERR_OOM;
  L->lev = level;
  L->nx = nx;
  L->pmask = pmask;
  L->n = n;
  L->parent = parent;
  L->mg = (mglev *)calloc((size_t)level + 1, sizeof(mglev));
  mglev *g = &L->mg[0];
  g->lev = level;
  g->n = n;
  g->key = (okey *)malloc(sizeof(okey) * (n ? n : 1));
  memcpy(g->key, keys, sizeof(okey) * n);
  int st = ht_init(&g->ht, n);
  for (int64_t t = 0; t < n && st == OR_OK; t++) st = ht_insert(&g->ht, keys[t], (int32_t)t);
  if (st == OR_OK) st = build_nbr(g, npd, pmask);
  if (st == OR_OK) st = alloc_fields(g);
  if (st != OR_OK) {
    L->depth = 1;
    or_level_free(L);
    return st;
  }
  for (int64_t t = 0; t < 8 * n; t++) g->active[t] = 1;
  L->depth = 1;
  L->periodic_full = (parent == NULL && pmask == 7 && npd <= 2048 && (uint64_t)n == npd * npd * npd);

  /* morton_nbor_cell (App. B): father cell of every missing neighbour, and a
   * check that every Dirichlet ghost value can be interpolated. */
  L->father = (int32_t *)malloc(sizeof(int32_t) * 12 * (n ? n : 1));
  L->ghost = (double *)malloc(sizeof(double) * 24 * (n ? n : 1));
  for (int64_t t = 0; t < 12 * n; t++) L->father[t] = -1;
  for (int64_t t = 0; t < 24 * n; t++) L->ghost[t] = NAN;
  if (parent) {
    int bad = 0;
    OR_PAR_FOR_OR(bad)
    for (int64_t i = 0; i < n; i++)
      for (int d = 0; d < 6; d++) {
        if (g->nbr[7 * i + 1 + d] >= 0) continue;
        okey nk;
        if (!key_neighbor(keys[i], d, npd, pmask, &nk)) {
          bad |= 1;
          continue;
        }
        int32_t p = ht_find(&parent->mg[0].ht, nk >> 3);
        if (p < 0) {
          bad |= 1;
          continue;
        }
        L->father[12 * i + 2 * d] = p;
        L->father[12 * i + 2 * d + 1] = (int32_t)(nk & 7);
        int a = d / 2, side = d & 1;
        for (int c = 0; c < 8; c++) {
          if (((c >> a) & 1) != side) continue;
          uint64_t G[3];
          ghost_position(keys[i], c, d, level, nx, pmask, G);
          int missing = 0;
          interp_coarse(&parent->mg[0].ht, parent->mg[0].phi, level - 1, nx, pmask, G, &missing);
          if (missing) bad |= 1;
        }
      }
    if (bad) st = OR_ERR_MISSING_PARENT;
  }
  if (st != OR_OK) {
    or_level_free(L);
    return st;
  }

  /* Multigrid hierarchy: MG level m+1 is made of the parents of the octs of
   * level m whose eight cells are all active, in order of first appearance; a
   * coarse cell is active iff such a child oct refines it. */
  for (;;) {
    mglev *cur = &L->mg[L->depth - 1];
    if (cur->lev == 1) break;
    hashtab tmp;
    ht_init(&tmp, cur->n);
    okey *pk = (okey *)malloc(sizeof(okey) * (cur->n ? cur->n : 1));
    int64_t np = 0;
    for (int64_t i = 0; i < cur->n; i++) {
      int full = 1;
      for (int c = 0; c < 8; c++) full &= cur->active[8 * i + c];
      if (!full) continue;
      okey k = cur->key[i] >> 3;
      if (ht_find(&tmp, k) < 0) {
        ht_insert(&tmp, k, (int32_t)np);
        pk[np++] = k;
      }
    }
    ht_free(&tmp);
    if (np == 0) {
      free(pk);
      break;
    }
    mglev *cg = &L->mg[L->depth];
    cg->lev = cur->lev - 1;
    cg->n = np;
    cg->key = pk;
    ht_init(&cg->ht, np);
    for (int64_t t = 0; t < np; t++) ht_insert(&cg->ht, pk[t], (int32_t)t);
    build_nbr(cg, octs_per_dim(cg->lev, nx), pmask);
    alloc_fields(cg);
    for (int64_t i = 0; i < cur->n; i++) {
      int full = 1;
      for (int c = 0; c < 8; c++) full &= cur->active[8 * i + c];
      if (!full) continue;
      int32_t p = ht_find(&cg->ht, cur->key[i] >> 3);
      int cc = (int)(cur->key[i] & 7);
      cg->active[8 * (int64_t)p + cc] = 1;
      cg->child[8 * (int64_t)p + cc] = (int32_t)i;
    }
    L->depth++;
  }
  *out = L;
  return OR_OK;
}

int or_level_build(int level, int nx, int pmask, const uint64_t *keys, int64_t n, or_level *parent,
                   or_level **out) {
  okey *k = (okey *)malloc(sizeof(okey) * (n > 0 ? n : 1));
  if (!k) return OR_ERR_OOM;
  for (int64_t t = 0; t < n; t++) k[t] = (okey)keys[t];
  int st = level_build(level, nx, pmask, k, n, parent, out, MORTON_BITS);
  free(k);
  return st;
}

int or_level_build128(int level, int nx, int pmask, const uint64_t *keys, int64_t n, or_level *parent,
                      or_level **out) {
  okey *k = (okey *)malloc(sizeof(okey) * (n > 0 ? n : 1));
  if (!k) return OR_ERR_OOM;
  for (int64_t t = 0; t < n; t++) k[t] = key_from_words(keys + 2 * t);
  int st = level_build(level, nx, pmask, k, n, parent, out, MORTON_BITS_WIDE);
  free(k);
  return st;
}

void or_level_free(or_level *L) {
  if (!L) return;
  for (int m = 0; m < L->depth; m++) free_mg(&L->mg[m]);
  free(L->mg);
  free(L->father);
  free(L->ghost);
  free(L);
}

int64_t or_level_n_octs(const or_level *L) { return L->n; }
int64_t or_level_hash_capacity(const or_level *L) { return L->mg[0].ht.cap; }

/* slot keys as their low 64 bits (a 64-bit level's keys; empty slots all ones) */
void or_level_hash_dump(const or_level *L, uint64_t *keys, int32_t *vals) {
  for (int64_t t = 0; t < L->mg[0].ht.cap; t++) keys[t] = (uint64_t)L->mg[0].ht.key[t];
  memcpy(vals, L->mg[0].ht.val, sizeof(int32_t) * L->mg[0].ht.cap);
}

void or_level_lookup(const or_level *L, const uint64_t *q, int64_t n, int32_t *out) {
  for (int64_t t = 0; t < n; t++) out[t] = ht_find(&L->mg[0].ht, (okey)q[t]);
}

void or_level_lookup128(const or_level *L, const uint64_t *q, int64_t n, int32_t *out) {
  for (int64_t t = 0; t < n; t++) out[t] = ht_find(&L->mg[0].ht, key_from_words(q + 2 * t));
}

void or_level_neighbors(const or_level *L, int32_t *out) {
  memcpy(out, L->mg[0].nbr, sizeof(int32_t) * 7 * L->n);
}

void or_level_father_cells(const or_level *L, int32_t *out) {
  memcpy(out, L->father, sizeof(int32_t) * 12 * L->n);
}

/* Source term f = 4 pi G (rho - rho_bar) (Sec. 5.1.1 item (iii)). */
void or_level_set_density(or_level *L, const double *rho, double rho_bar, double four_pi_g) {
  OR_PAR_FOR
  for (int64_t t = 0; t < 8 * L->n; t++) L->mg[0].f[t] = four_pi_g * (rho[t] - rho_bar);
}

void or_level_set_f(or_level *L, const double *f) { memcpy(L->mg[0].f, f, sizeof(double) * 8 * L->n); }
void or_level_set_phi(or_level *L, const double *phi) {
  memcpy(L->mg[0].phi, phi, sizeof(double) * 8 * L->n);
}
void or_level_get_phi(const or_level *L, double *out) {
  memcpy(out, L->mg[0].phi, sizeof(double) * 8 * L->n);
}
void or_level_get_f(const or_level *L, double *out) { memcpy(out, L->mg[0].f, sizeof(double) * 8 * L->n); }

/* Dirichlet ghost values interpolated from the parent level's phi. */
void or_level_compute_ghosts(or_level *L) {
  if (!L->parent) return;
  const mglev *g = &L->mg[0];
  const mglev *pg = &L->parent->mg[0];
  OR_PAR_FOR
  for (int64_t i = 0; i < L->n; i++)
    for (int d = 0; d < 6; d++) {
      if (g->nbr[7 * i + 1 + d] >= 0) continue;
      int a = d / 2, side = d & 1;
      for (int c = 0; c < 8; c++) {
        if (((c >> a) & 1) != side) continue;
        uint64_t G[3];
        ghost_position(g->key[i], c, d, L->lev, L->nx, L->pmask, G);
        int missing = 0;
        L->ghost[24 * i + 4 * d + face_rank(c, a)] =
            interp_coarse(&pg->ht, pg->phi, L->lev - 1, L->nx, L->pmask, G, &missing);
      }
    }
}

void or_level_get_ghosts(const or_level *L, double *out) {
  memcpy(out, L->ghost, sizeof(double) * 24 * L->n);
}

int or_level_mg_depth(const or_level *L) { return L->depth; }
int64_t or_level_mg_n_octs(const or_level *L, int m) { return L->mg[m].n; }
int or_level_mg_lev(const or_level *L, int m) { return L->mg[m].lev; }
void or_level_mg_keys(const or_level *L, int m, uint64_t *out) {
  for (int64_t t = 0; t < L->mg[m].n; t++) out[t] = (uint64_t)L->mg[m].key[t];
}
void or_level_mg_keys128(const or_level *L, int m, uint64_t *out) {
  for (int64_t t = 0; t < L->mg[m].n; t++) key_to_words(L->mg[m].key[t], out + 2 * t);
}
void or_level_mg_active(const or_level *L, int m, uint8_t *out) {
  memcpy(out, L->mg[m].active, 8 * L->mg[m].n);
}

static double *field_ptr(const or_level *L, int m, int field) {
  const mglev *g = &L->mg[m];
  return field == 0 ? g->phi : field == 1 ? g->f : g->r;
}
void or_level_mg_get(const or_level *L, int m, int field, double *out) {
  memcpy(out, field_ptr(L, m, field), sizeof(double) * 8 * L->mg[m].n);
}
void or_level_mg_set(or_level *L, int m, int field, const double *in) {
  memcpy(field_ptr(L, m, field), in, sizeof(double) * 8 * L->mg[m].n);
}

/* --------------------------------------------------- FP64 level operators */

/* Value seen across face d of cell (i, c) at MG level m: the same-level cell,
 * else the Dirichlet ghost (m = 0 with ghosts), else 0 (the correction
 * vanishes outside the covered region). */
static double nb_value(const or_level *L, int m, int64_t i, int c, int d, int use_ghost) {
  const mglev *g = &L->mg[m];
  int a = d / 2, side = d & 1;
  int c2 = c ^ (1 << a);
  if (((c >> a) & 1) != side) return g->phi[8 * i + c2];
  int32_t nb = g->nbr[7 * i + 1 + d];
  if (nb >= 0) return g->phi[8 * (int64_t)nb + c2];
  if (m == 0 && use_ghost && L->parent) return L->ghost[24 * i + 4 * d + face_rank(c, a)];
  return 0.0;
}

static double nb_sum(const or_level *L, int m, int64_t i, int c, int use_ghost) {
  double s = nb_value(L, m, i, c, 0, use_ghost);
  for (int d = 1; d < 6; d++) s = s + nb_value(L, m, i, c, d, use_ghost);
  return s;
}

/* App. D.2 Eq. (gs_update): phi = (sum_j phi_j - h^2 f) * (1/6) on the
 * active cells of one colour (0 = red, (i+j+k) even; 1 = black). */
void or_rb_colour_pass(or_level *L, int m, int color, int use_ghost) {
  mglev *g = &L->mg[m];
  double h = cell_h(g->lev, L->nx), h2 = h * h, inv6 = 1.0 / 6.0;
  OR_PAR_FOR
  for (int64_t i = 0; i < g->n; i++)
    for (int c = 0; c < 8; c++) {
      if (parity(c) != color || !g->active[8 * i + c]) continue;
      double sum = nb_sum(L, m, i, c, use_ghost);
      g->phi[8 * i + c] = (sum - h2 * g->f[8 * i + c]) * inv6;
    }
}

/* n_sweeps red-black sweeps: red cells first, then black. */
void or_rb_sweeps(or_level *L, int m, int n_sweeps, int use_ghost) {
  for (int s = 0; s < n_sweeps; s++)
    for (int color = 0; color < 2; color++) or_rb_colour_pass(L, m, color, use_ghost);
}

/* r = f - lap_h(phi), lap_h = (sum_j phi_j - 6 phi) / h^2; returns sum r^2
 * (Sec. 5.1.1 item (iii): residual and squared norm in one loop). */
double or_residual(or_level *L, int m, int use_ghost) {
  mglev *g = &L->mg[m];
  double h = cell_h(g->lev, L->nx), h2 = h * h, norm2 = 0.0;
  OR_PAR_FOR
  for (int64_t i = 0; i < g->n; i++)
    for (int c = 0; c < 8; c++) {
      double r = 0.0;
      if (g->active[8 * i + c]) {
        double sum = nb_sum(L, m, i, c, use_ghost);
        r = g->f[8 * i + c] - (sum - 6.0 * g->phi[8 * i + c]) / h2;
      }
      g->r[8 * i + c] = r;
    }
  for (int64_t t = 0; t < 8 * g->n; t++) norm2 += g->r[t] * g->r[t];
  return norm2;
}

/* Coarse value = mean of the eight fine children (Sec. 5.1.1). */
void or_restrict(or_level *L, int m) {
  mglev *g = &L->mg[m], *cg = &L->mg[m + 1];
  OR_PAR_FOR
  for (int64_t p = 0; p < cg->n; p++)
    for (int cc = 0; cc < 8; cc++) {
      double v = 0.0;
      if (cg->active[8 * p + cc]) {
        int64_t k = cg->child[8 * p + cc];
        double sum = 0.0;
        for (int c = 0; c < 8; c++) sum += g->r[8 * k + c];
        v = sum / 8.0;
      }
      cg->f[8 * p + cc] = v;
      cg->phi[8 * p + cc] = 0.0;
    }
}

/* phi[m] += trilinear interpolation of phi[m+1] (Sec. 5.1.1). */
void or_prolong(or_level *L, int m) {
  mglev *g = &L->mg[m], *cg = &L->mg[m + 1];
  OR_PAR_FOR
  for (int64_t i = 0; i < g->n; i++)
    for (int c = 0; c < 8; c++) {
      if (!g->active[8 * i + c]) continue;
      uint64_t X[3];
      cell_coords(g->key[i], c, X);
      int missing = 0;
      g->phi[8 * i + c] += interp_coarse(&cg->ht, cg->phi, cg->lev, L->nx, L->pmask, X, &missing);
    }
}

/* Exact solve of the periodic 2^3 problem by an 8-point Walsh-Hadamard
 * transform: eigenvector (-1)^{k.b}, eigenvalue -4 |k|_1 / h^2, the k = 0
 * (mean) mode dropped. */
static void wht_solve(const double *f, double *phi, double h) {
  double fh[8];
  for (int k = 0; k < 8; k++) {
    double s = 0.0;
    for (int b = 0; b < 8; b++) s += (parity(k & b) ? -1.0 : 1.0) * f[b];
    fh[k] = s / 8.0;
  }
  for (int b = 0; b < 8; b++) {
    double s = 0.0;
    for (int k = 1; k < 8; k++) {
      int odd = (k & 1) + ((k >> 1) & 1) + ((k >> 2) & 1);
      double lam = -4.0 * odd / (h * h);
      s += (parity(k & b) ? -1.0 : 1.0) * fh[k] / lam;
    }
    phi[b] = s;
  }
}

static int coarse_is_exact(const or_level *L, int m) {
  return L->periodic_full && L->mg[m].lev == 1 && L->nx == 1 && L->mg[m].n == 1;
}

void or_coarse_solve(or_level *L, int coarse_sweeps) {
  int m = L->depth - 1;
  mglev *g = &L->mg[m];
  if (coarse_is_exact(L, m)) {
    wht_solve(g->f, g->phi, cell_h(1, 1));
  } else {
    or_rb_sweeps(L, m, coarse_sweeps, m == 0);
  }
}

/* App. G Alg. (vcycle) on one GPU: no halo exchanges. */
static void vcycle(or_level *L, int m, const or_params *p, int use_ghost) {
  if (m == L->depth - 1) {
    or_coarse_solve(L, p->coarse_sweeps);
    return;
  }
  or_rb_sweeps(L, m, p->n_pre, use_ghost && m == 0);
  or_residual(L, m, use_ghost && m == 0);
  or_restrict(L, m);
  vcycle(L, m + 1, p, use_ghost);
  or_prolong(L, m);
  or_rb_sweeps(L, m, p->n_post, use_ghost && m == 0);
}

static void subtract_mean(double *phi, int64_t n) {
  double s = 0.0;
  for (int64_t t = 0; t < n; t++) s += phi[t];
  s /= (double)n;
  OR_PAR_FOR
  for (int64_t t = 0; t < n; t++) phi[t] -= s;
}

/* ||f - L_h 0||^2: the residual of a zero guess (includes ghost forcing). */
static double zero_guess_norm2(or_level *L) {
  mglev *g = &L->mg[0];
  double *save = (double *)malloc(sizeof(double) * 8 * (g->n ? g->n : 1));
  memcpy(save, g->phi, sizeof(double) * 8 * g->n);
  memset(g->phi, 0, sizeof(double) * 8 * g->n);
  double n0 = or_residual(L, 0, 1);
  memcpy(g->phi, save, sizeof(double) * 8 * g->n);
  free(save);
  return n0;
}

static int check_solvable(const or_level *L, const or_params *p) {
  if (!p || p->n_pre < 0 || p->n_post < 0 || p->coarse_sweeps < 0 || p->max_cycles < 0 ||
      p->fixed_cycles < 0 || p->fixed_cycles > 256 || p->max_cycles > 256)
    return OR_ERR_INVALID_ARG;
  if (L->periodic_full && L->nx != 1) return OR_ERR_INVALID_ARG;
  return OR_OK;
}

int or_level_solve(or_level *L, const or_params *p, or_stats *st) {
  int rc = check_solvable(L, p);
  if (rc != OR_OK) return rc;
  memset(st, 0, sizeof(*st));
  or_level_compute_ghosts(L);
  double n0 = zero_guess_norm2(L);
  st->norm0 = sqrt(n0);
  if (n0 == 0.0) {
    memset(L->mg[0].phi, 0, sizeof(double) * 8 * L->n);
    return OR_OK;
  }
  double rel = sqrt(or_residual(L, 0, 1) / n0);
  st->rel_initial = rel;
  st->rel_final = rel;
  int target = p->fixed_cycles > 0 ? p->fixed_cycles : p->max_cycles;
  if (p->fixed_cycles == 0 && rel <= p->tol) return OR_OK;
  for (int cyc = 1; cyc <= target; cyc++) {
    vcycle(L, 0, p, 1);
    if (L->periodic_full) subtract_mean(L->mg[0].phi, 8 * L->n);
    rel = sqrt(or_residual(L, 0, 1) / n0);
    st->cycles = cyc;
    st->rel_history[cyc - 1] = rel;
    st->rel_final = rel;
    if (!isfinite(rel) || rel > 1e3 * (st->rel_initial > 1.0 ? st->rel_initial : 1.0))
      return OR_ERR_DIVERGED;
    if (p->fixed_cycles == 0 && rel <= p->tol) return OR_OK;
  }
  return p->fixed_cycles > 0 ? OR_OK : OR_ERR_NOT_CONVERGED;
}

/* ------------------------------------------- FP32 inner cycle (mixed) */

static void ensure32(mglev *g) {
  if (g->phi32) return;
  int64_t m = 8 * (g->n ? g->n : 1);
  g->phi32 = (float *)calloc(m, sizeof(float));
  g->f32 = (float *)calloc(m, sizeof(float));
  g->r32 = (float *)calloc(m, sizeof(float));
}

static float nb_value32(const mglev *g, int64_t i, int c, int d) {
  int a = d / 2, side = d & 1;
  int c2 = c ^ (1 << a);
  if (((c >> a) & 1) != side) return g->phi32[8 * i + c2];
  int32_t nb = g->nbr[7 * i + 1 + d];
  return nb >= 0 ? g->phi32[8 * (int64_t)nb + c2] : 0.0f;
}

static float nb_sum32(const mglev *g, int64_t i, int c) {
  float s = nb_value32(g, i, c, 0);
  for (int d = 1; d < 6; d++) s = s + nb_value32(g, i, c, d);
  return s;
}

static void sweeps32(or_level *L, int m, int n_sweeps) {
  mglev *g = &L->mg[m];
  float h = (float)cell_h(g->lev, L->nx), h2 = h * h, inv6 = 1.0f / 6.0f;
  for (int s = 0; s < n_sweeps; s++)
    for (int color = 0; color < 2; color++)
      OR_PAR_FOR
      for (int64_t i = 0; i < g->n; i++)
        for (int c = 0; c < 8; c++) {
          if (parity(c) != color || !g->active[8 * i + c]) continue;
          float sum = nb_sum32(g, i, c);
          g->phi32[8 * i + c] = (sum - h2 * g->f32[8 * i + c]) * inv6;
        }
}

static void residual32(or_level *L, int m) {
  mglev *g = &L->mg[m];
  float h = (float)cell_h(g->lev, L->nx), h2 = h * h;
  OR_PAR_FOR
  for (int64_t i = 0; i < g->n; i++)
    for (int c = 0; c < 8; c++) {
      float r = 0.0f;
      if (g->active[8 * i + c]) r = g->f32[8 * i + c] - (nb_sum32(g, i, c) - 6.0f * g->phi32[8 * i + c]) / h2;
      g->r32[8 * i + c] = r;
    }
}

static void restrict32(or_level *L, int m) {
  mglev *g = &L->mg[m], *cg = &L->mg[m + 1];
  OR_PAR_FOR
  for (int64_t p = 0; p < cg->n; p++)
    for (int cc = 0; cc < 8; cc++) {
      float v = 0.0f;
      if (cg->active[8 * p + cc]) {
        int64_t k = cg->child[8 * p + cc];
        float sum = 0.0f;
        for (int c = 0; c < 8; c++) sum += g->r32[8 * k + c];
        v = sum / 8.0f;
      }
      cg->f32[8 * p + cc] = v;
      cg->phi32[8 * p + cc] = 0.0f;
    }
}

static void prolong32(or_level *L, int m) {
  mglev *g = &L->mg[m], *cg = &L->mg[m + 1];
  OR_PAR_FOR
  for (int64_t i = 0; i < g->n; i++)
    for (int c = 0; c < 8; c++) {
      if (!g->active[8 * i + c]) continue;
      uint64_t X[3];
      cell_coords(g->key[i], c, X);
      int64_t Xc[3], o[3];
      for (int a = 0; a < 3; a++) {
        Xc[a] = (int64_t)(X[a] >> 1);
        o[a] = (X[a] & 1) ? 1 : -1;
      }
      float sum = 0.0f;
      for (int cz = 0; cz < 2; cz++)
        for (int cy = 0; cy < 2; cy++)
          for (int cx = 0; cx < 2; cx++) {
            float w = (cx ? 0.25f : 0.75f) * (cy ? 0.25f : 0.75f) * (cz ? 0.25f : 0.75f);
            int64_t Y[3] = {Xc[0] + cx * o[0], Xc[1] + cy * o[1], Xc[2] + cz * o[2]};
            int32_t oct;
            int ch;
            if (find_cell(&cg->ht, Y, cg->lev, L->nx, L->pmask, &oct, &ch)) sum += w * cg->phi32[8 * (int64_t)oct + ch];
          }
      g->phi32[8 * i + c] += sum;
    }
}

/* Inner FP32 V-cycle for the correction (homogeneous Dirichlet ghosts); the
 * coarsest level is solved in FP64. */
static void vcycle32(or_level *L, int m, const or_params *p) {
  mglev *g = &L->mg[m];
  if (m == L->depth - 1) {
    for (int64_t t = 0; t < 8 * g->n; t++) {
      g->f[t] = (double)g->f32[t];
      g->phi[t] = (double)g->phi32[t];
    }
    if (coarse_is_exact(L, m)) {
      wht_solve(g->f, g->phi, cell_h(1, 1));
    } else {
      or_rb_sweeps(L, m, p->coarse_sweeps, 0);
    }
    for (int64_t t = 0; t < 8 * g->n; t++) g->phi32[t] = (float)g->phi[t];
    return;
  }
  sweeps32(L, m, p->n_pre);
  residual32(L, m);
  restrict32(L, m);
  vcycle32(L, m + 1, p);
  prolong32(L, m);
  sweeps32(L, m, p->n_post);
}

int or_level_solve_mixed(or_level *L, const or_params *p, int inner_cycles, or_stats *st) {
  int rc = check_solvable(L, p);
  if (rc != OR_OK || inner_cycles < 1) return rc != OR_OK ? rc : OR_ERR_INVALID_ARG;
  if (L->depth < 2) return OR_ERR_INVALID_ARG;
  memset(st, 0, sizeof(*st));
  for (int m = 0; m < L->depth; m++) ensure32(&L->mg[m]);
  or_level_compute_ghosts(L);
  mglev *g = &L->mg[0];
  double n0 = zero_guess_norm2(L);
  st->norm0 = sqrt(n0);
  if (n0 == 0.0) {
    memset(g->phi, 0, sizeof(double) * 8 * L->n);
    return OR_OK;
  }
  double nr = or_residual(L, 0, 1);
  double rel = sqrt(nr / n0);
  st->rel_initial = rel;
  st->rel_final = rel;
  int target = p->fixed_cycles > 0 ? p->fixed_cycles : p->max_cycles;
  if (p->fixed_cycles == 0 && rel <= p->tol) return OR_OK;
  for (int cyc = 1; cyc <= target; cyc++) {
    double nrm = sqrt(nr);
    OR_PAR_FOR
    for (int64_t t = 0; t < 8 * L->n; t++) {
      g->f32[t] = (float)(g->r[t] / nrm);
      g->phi32[t] = 0.0f;
    }
    for (int k = 0; k < inner_cycles; k++) vcycle32(L, 0, p);
    OR_PAR_FOR
    for (int64_t t = 0; t < 8 * L->n; t++) g->phi[t] += nrm * (double)g->phi32[t];
    if (L->periodic_full) subtract_mean(g->phi, 8 * L->n);
    nr = or_residual(L, 0, 1);
    rel = sqrt(nr / n0);
    st->cycles = cyc;
    st->rel_history[cyc - 1] = rel;
    st->rel_final = rel;
    if (!isfinite(rel) || rel > 1e3 * (st->rel_initial > 1.0 ? st->rel_initial : 1.0))
      return OR_ERR_DIVERGED;
    if (p->fixed_cycles == 0 && rel <= p->tol) return OR_OK;
  }
  return p->fixed_cycles > 0 ? OR_OK : OR_ERR_NOT_CONVERGED;
}

/* ------------------------------- MG-preconditioned CG (App. D.2 reading) */

static double dot8(const double *a, const double *b, int64_t n) {
  double s = 0.0;
  for (int64_t t = 0; t < n; t++) s += a[t] * b[t];
  return s;
}

/* q = L_h v with zero values across the coarse-fine boundary (the operator
 * acting on corrections): the residual of v for a zero source, negated. */
static void apply_L0(or_level *L, const double *v, double *q, const double *zero) {
  mglev *g = &L->mg[0];
  double *f_save = g->f;
  memcpy(g->phi, v, sizeof(double) * 8 * g->n);
  g->f = (double *)zero;
  or_residual(L, 0, 0);
  g->f = f_save;
  for (int64_t t = 0; t < 8 * g->n; t++) q[t] = -g->r[t];
}

/* z = one V-cycle from zero on L z = r, homogeneous coarse-fine boundary
 * values; zero mean on a periodic level (the operator's null space). */
static void precondition(or_level *L, const or_params *p, const double *r, double *z) {
  mglev *g = &L->mg[0];
  double *f_save = g->f;
  g->f = (double *)r;
  memset(g->phi, 0, sizeof(double) * 8 * g->n);
  vcycle(L, 0, p, 0);
  g->f = f_save;
  memcpy(z, g->phi, sizeof(double) * 8 * g->n);
  if (L->periodic_full) subtract_mean(z, 8 * g->n);
}

int or_level_solve_pcg(or_level *L, const or_params *p, or_stats *st) {
  int rc = check_solvable(L, p);
  if (rc != OR_OK) return rc;
  memset(st, 0, sizeof(*st));
  or_level_compute_ghosts(L);
  mglev *g = &L->mg[0];
  const int64_t N = 8 * g->n;
  double n0 = zero_guess_norm2(L);
  st->norm0 = sqrt(n0);
  if (n0 == 0.0) {
    memset(g->phi, 0, sizeof(double) * N);
    return OR_OK;
  }
  const int64_t m = N ? N : 1;
  double *x = (double *)malloc(sizeof(double) * m), *r = (double *)malloc(sizeof(double) * m);
  double *rn = (double *)malloc(sizeof(double) * m), *z = (double *)malloc(sizeof(double) * m);
  double *d = (double *)malloc(sizeof(double) * m), *q = (double *)malloc(sizeof(double) * m);
  double *zero = (double *)calloc(m, sizeof(double));
  memcpy(x, g->phi, sizeof(double) * N);
  double nr = or_residual(L, 0, 1); /* true residual of the initial guess */
  memcpy(r, g->r, sizeof(double) * N);
  double rel = sqrt(nr / n0);
  st->rel_initial = rel;
  st->rel_final = rel;
  int target = p->fixed_cycles > 0 ? p->fixed_cycles : p->max_cycles;
  rc = p->fixed_cycles > 0 ? OR_OK : OR_ERR_NOT_CONVERGED;
  if (p->fixed_cycles == 0 && rel <= p->tol) {
    rc = OR_OK;
    target = 0;
  }
  if (target > 0) {
    precondition(L, p, r, z);
    memcpy(d, z, sizeof(double) * N);
    double rz = dot8(r, z, N);
    for (int it = 1; it <= target; it++) {
      apply_L0(L, d, q, zero);
      double alpha = rz / dot8(d, q, N);
      for (int64_t t = 0; t < N; t++) {
        x[t] += alpha * d[t];
        rn[t] = r[t] - alpha * q[t];
      }
      rel = sqrt(dot8(rn, rn, N) / n0);
      st->cycles = it;
      st->rel_history[it - 1] = rel;
      st->rel_final = rel;
      if (!isfinite(rel) || rel > 1e3 * (st->rel_initial > 1.0 ? st->rel_initial : 1.0)) {
        rc = OR_ERR_DIVERGED;
        break;
      }
      if (p->fixed_cycles == 0 && rel <= p->tol) {
        rc = OR_OK;
        break;
      }
      precondition(L, p, rn, z);
      /* flexible (Polak-Ribiere) beta: (z_new, r_new - r_old) / (z_old, r_old) */
      double rz_new = dot8(rn, z, N);
      double beta = (rz_new - dot8(r, z, N)) / rz;
      for (int64_t t = 0; t < N; t++) d[t] = z[t] + beta * d[t];
      rz = rz_new;
      memcpy(r, rn, sizeof(double) * N);
    }
  }
  memcpy(g->phi, x, sizeof(double) * N);
  if (L->periodic_full) subtract_mean(g->phi, N);
  free(x);
  free(r);
  free(rn);
  free(z);
  free(d);
  free(q);
  free(zero);
  return rc;
}
