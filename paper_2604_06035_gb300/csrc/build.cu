// build.cu -- level construction on the device: Morton keys (Sec. 4.2),
// the per-level hash table (App. B), the neighbour cache (App. D.1), the
// coarse-fine ghost octs and their parent stencils (morton_nbor_cell, App. B),
// and the multigrid hierarchy of a level.
#include <atomic>
#include <climits>
#include <cmath>

#include "cmg_internal.cuh"
#include "keys.cuh"

namespace cmg {

void cuda_check(cudaError_t e, const char *what) {
  if (e == cudaSuccess) return;
  if (e == cudaErrorMemoryAllocation) throw Error(CMG_ERR_OOM, std::string("out of device memory: ") + what);
  throw Error(CMG_ERR_CUDA, std::string(cudaGetErrorString(e)) + " in " + what);
}

// Host-side fault injection for tests: when positive, the countdown'th
// next library allocation fails as if the device were out of memory.
static std::atomic<int64_t> g_alloc_countdown{0};

void inject_alloc_failure(int64_t after) { g_alloc_countdown.store(after > 0 ? after : 0); }

template <class T>
T *DeviceBuffers::alloc(int64_t count, bool zero, cudaStream_t s) {
  void *p = nullptr;
  const size_t bytes = sizeof(T) * (size_t)(count > 0 ? count : 1);
  if (g_alloc_countdown.load() > 0 && g_alloc_countdown.fetch_sub(1) == 1)
    throw Error(CMG_ERR_OOM, "injected allocation failure (" + std::to_string(bytes) + " bytes)");
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    throw Error(CMG_ERR_OOM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  ptrs.push_back(p);
  if (zero) CMG_CUDA(cudaMemsetAsync(p, 0, bytes, s));
  return static_cast<T *>(p);
}

void DeviceBuffers::release() {
  for (void *p : ptrs) cudaFree(p);
  ptrs.clear();
}

template uint64_t *DeviceBuffers::alloc<uint64_t>(int64_t, bool, cudaStream_t);
template int64_t *DeviceBuffers::alloc<int64_t>(int64_t, bool, cudaStream_t);
template uint16_t *DeviceBuffers::alloc<uint16_t>(int64_t, bool, cudaStream_t);
template int32_t *DeviceBuffers::alloc<int32_t>(int64_t, bool, cudaStream_t);
template uint32_t *DeviceBuffers::alloc<uint32_t>(int64_t, bool, cudaStream_t);
template uint8_t *DeviceBuffers::alloc<uint8_t>(int64_t, bool, cudaStream_t);
template double *DeviceBuffers::alloc<double>(int64_t, bool, cudaStream_t);
template float *DeviceBuffers::alloc<float>(int64_t, bool, cudaStream_t);
template Key128 *DeviceBuffers::alloc<Key128>(int64_t, bool, cudaStream_t);

namespace {

// --------------------------------------------------------------- kernels

__global__ void k_encode(const uint32_t *__restrict__ ijk, int64_t n, uint64_t *__restrict__ keys, int *err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint32_t i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  if ((i | j | k) >> kMortonBits) set_error(err, CMG_ERR_KEY_OUT_OF_RANGE);
  keys[t] = morton_encode(i, j, k);
}

__global__ void k_decode(const uint64_t *__restrict__ keys, int64_t n, uint32_t *__restrict__ ijk) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint32_t i, j, k;
  morton_decode(keys[t], i, j, k);
  ijk[3 * t] = i;
  ijk[3 * t + 1] = j;
  ijk[3 * t + 2] = k;
}

__global__ void k_encode128(const uint64_t *__restrict__ ijk, int64_t n, Key128 *__restrict__ keys, int *err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const uint64_t i = ijk[3 * t], j = ijk[3 * t + 1], k = ijk[3 * t + 2];
  if ((i | j | k) >> KeyOps<Key128>::kBits) set_error(err, CMG_ERR_KEY_OUT_OF_RANGE);
  keys[t] = KeyOps<Key128>::encode(i, j, k);
}

__global__ void k_decode128(const Key128 *__restrict__ keys, int64_t n, uint64_t *__restrict__ ijk) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  uint64_t c[3];
  KeyOps<Key128>::decode(keys[t], c);
  ijk[3 * t] = c[0];
  ijk[3 * t + 1] = c[1];
  ijk[3 * t + 2] = c[2];
}

// low words of 128-bit keys (the octant bits the solver kernels read)
__global__ void k_low_words(const Key128 *__restrict__ keys, int64_t n, uint64_t *__restrict__ lo) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) lo[t] = keys[t].lo;
}

// Range check (valid key, coordinates < npd) and hash insert (A2).
template <class K>
__global__ void k_insert_keys(const K *__restrict__ keys, int64_t n, uint64_t npd, K *ht_keys, int32_t *ht_vals,
                              uint64_t mask, int *err) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  const K k = keys[t];
  uint64_t c[3];
  KeyOps<K>::decode(k, c);
  if (!KeyOps<K>::in_range(k) || c[0] >= npd || c[1] >= npd || c[2] >= npd) {
    set_error(err, CMG_ERR_KEY_OUT_OF_RANGE);
    return;
  }
  bool inserted = false;
  const int64_t s = ht_insert_slot_k(ht_keys, mask, k, &inserted);
  if (s < 0) {
    set_error(err, CMG_ERR_INVALID_ARG);
    return;
  }
  if (!inserted) {
    set_error(err, CMG_ERR_DUPLICATE_KEY);
    return;
  }
  ht_vals[s] = (int32_t)t;
}

template <class K>
__global__ void k_lookup(const K *__restrict__ ht_keys, const int32_t *__restrict__ ht_vals, uint64_t mask,
                         const K *__restrict__ q, int64_t n, int32_t *__restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= n) return;
  out[t] = ht_find_k(ht_keys, ht_vals, mask, q[t]);
}

// Neighbour cache (App. D.1 Eq. (nbor_precompute)), SoA [6][n]; missing
// neighbours get `missing` (patched later for ghosts).
template <class K>
__global__ void k_neighbors(const K *__restrict__ keys, int64_t n, uint64_t npd, int pmask,
                            const K *__restrict__ ht_keys, const int32_t *__restrict__ ht_vals, uint64_t mask,
                            int32_t missing, int32_t *__restrict__ nbr, int32_t *__restrict__ n_missing) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const K k = keys[i];
  const K e = KeyOps<K>::empty();
  int miss = 0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const K nk = neighbor_key_k(k, d, npd, pmask);
    int32_t v = nk == e ? -1 : ht_find_k(ht_keys, ht_vals, mask, nk);
    if (v < 0) {
      v = missing;
      ++miss;
    }
    nbr[d * n + i] = v;
  }
  if (n_missing && miss) atomicAdd(n_missing, miss);
}

// Ghost octs: one per distinct missing-neighbour position.
template <class K>
__global__ void k_ghost_insert(const K *__restrict__ keys, int64_t n, uint64_t npd, int pmask,
                               const int32_t *__restrict__ nbr, int32_t missing, K *g_ht_keys, int32_t *g_ht_vals,
                               uint64_t g_mask, int32_t *counter, K *__restrict__ ghost_keys, int *err) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const K e = KeyOps<K>::empty();
#pragma unroll 1
  for (int d = 0; d < 6; ++d) {
    if (nbr[d * n + i] != missing) continue;
    const K nk = neighbor_key_k(keys[i], d, npd, pmask);
    if (nk == e) {  // outside a non-periodic box: no parent cell to interpolate from
      set_error(err, CMG_ERR_MISSING_PARENT);
      continue;
    }
    bool inserted = false;
    const int64_t s = ht_insert_slot_k(g_ht_keys, g_mask, nk, &inserted);
    if (s < 0) {
      set_error(err, CMG_ERR_INVALID_ARG);
      continue;
    }
    if (inserted) {
      const int32_t gi = atomicAdd(counter, 1);
      g_ht_vals[s] = gi;
      ghost_keys[gi] = nk;
    }
  }
}

// Patch missing neighbours to ghost octs (index n + g) and record which ghost
// cells are read: the face of the ghost oct that touches oct i.
template <class K>
__global__ void k_ghost_resolve(const K *__restrict__ keys, int64_t n, uint64_t npd, int pmask,
                                int32_t *__restrict__ nbr, int32_t missing, const K *__restrict__ g_ht_keys,
                                const int32_t *__restrict__ g_ht_vals, uint64_t g_mask,
                                uint32_t *__restrict__ ghost_mask) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const K e = KeyOps<K>::empty();
#pragma unroll 1
  for (int d = 0; d < 6; ++d) {
    if (nbr[d * n + i] != missing) continue;
    const K nk = neighbor_key_k(keys[i], d, npd, pmask);
    if (nk == e) continue;
    const int32_t gi = ht_find_k(g_ht_keys, g_ht_vals, g_mask, nk);
    nbr[d * n + i] = (int32_t)n + gi;
    // cells of the ghost oct on its face opposite to direction d
    const int a = d >> 1, side_in_ghost = (d & 1) ? 0 : 1;
    uint32_t m = 0;
    for (int c = 0; c < 8; ++c)
      if (((c >> a) & 1) == side_in_ghost) m |= 1u << c;
    atomicOr(ghost_mask + gi, m);
  }
}

// 2x2x2 block of octs (in the coarse table) around the father cell (parent
// key, octant) of an oct with key `k` one level finer: block entry
// bx + 2 by + 4 bz is the oct displaced by b toward the octant.
template <class K>
__device__ inline void father_block(const K &k, uint64_t cnpd, int pmask, const K *__restrict__ ht_keys,
                                    const int32_t *__restrict__ ht_vals, uint64_t mask, int32_t zero_oct,
                                    int32_t out[8]) {
  const int cc = KeyOps<K>::octant(k);
  uint64_t c[3];
  KeyOps<K>::decode(KeyOps<K>::parent(k), c);
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    bool ok = true;
    uint64_t q[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      uint64_t v = c[a];
      if ((b >> a) & 1) {
        if ((cc >> a) & 1) {
          if (v + 1 < cnpd) v += 1;
          else if ((pmask >> a) & 1) v = 0;
          else ok = false;
        } else {
          if (v > 0) v -= 1;
          else if ((pmask >> a) & 1) v = cnpd - 1;
          else ok = false;
        }
      }
      q[a] = v;
    }
    int32_t idx = ok ? ht_find_k(ht_keys, ht_vals, mask, KeyOps<K>::encode(q[0], q[1], q[2])) : -1;
    out[b] = idx < 0 ? zero_oct : idx;
  }
}

// Block (which of the 8 octs) and child of the coarse cell at offset e-1
// (e = 0, 1, 2) along one axis from a father cell with octant bit cx.
__device__ inline void axis_cell(int cx, int e, int &a, int &bit) {
  if (cx == 0) {
    a = (e == 0);
    bit = (e != 1);
  } else {
    a = (e == 2);
    bit = (e == 1);
  }
}

template <class K>
__global__ void k_ghost_blocks(const K *__restrict__ ghost_keys, int64_t n_ghost,
                               const uint32_t *__restrict__ ghost_mask, uint64_t pnpd, int pmask,
                               const K *__restrict__ p_ht_keys, const int32_t *__restrict__ p_ht_vals,
                               uint64_t p_mask, int32_t p_zero, int32_t *__restrict__ blk, int *err) {
  const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (g >= n_ghost) return;
  const K k = ghost_keys[g];
  int32_t b[8];
  father_block(k, pnpd, pmask, p_ht_keys, p_ht_vals, p_mask, p_zero, b);
#pragma unroll
  for (int t = 0; t < 8; ++t) blk[t * n_ghost + g] = b[t];
  // every needed ghost cell must find its 8 interpolation cells in the parent
  const uint32_t need = ghost_mask[g];
  const int cc = KeyOps<K>::octant(k);
  for (int c = 0; c < 8; ++c) {
    if (!((need >> c) & 1)) continue;
    for (int t = 0; t < 8; ++t) {
      // interpolation cell t: offsets {0, toward c's octant} per axis
      int blk_idx = 0;
      for (int a = 0; a < 3; ++a) {
        const int fx = (c >> a) & 1;
        const int e = ((t >> a) & 1) ? (fx ? 2 : 0) : 1;
        int aa, bit;
        axis_cell((cc >> a) & 1, e, aa, bit);
        blk_idx |= aa << a;
      }
      if (b[blk_idx] == p_zero) set_error(err, CMG_ERR_MISSING_PARENT);
    }
  }
}

// ---- hierarchy

template <class K>
__global__ void k_parent_first(const K *__restrict__ keys, const uint8_t *__restrict__ active, bool all_active,
                               int64_t n, K *t_keys, int32_t *t_min, uint64_t t_mask) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (!all_active && active[i] != 0xFF) return;
  bool inserted;
  const int64_t s = ht_insert_slot_k(t_keys, t_mask, KeyOps<K>::parent(keys[i]), &inserted);
  if (s >= 0) atomicMin(t_min + s, (int32_t)i);
}

template <class K>
__global__ void k_parent_flag(const K *__restrict__ keys, const uint8_t *__restrict__ active, bool all_active,
                              int64_t n, const K *__restrict__ t_keys, const int32_t *__restrict__ t_min,
                              uint64_t t_mask, int32_t *__restrict__ flag) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t f = 0;
  if (all_active || active[i] == 0xFF) {
    const int64_t s = ht_slot_k(t_keys, t_mask, KeyOps<K>::parent(keys[i]));
    f = (s >= 0 && t_min[s] == (int32_t)i);
  }
  flag[i] = f;
}

template <class K>
__global__ void k_parent_emit(const K *__restrict__ keys, int64_t n, const int32_t *__restrict__ flag,
                              const int32_t *__restrict__ pos, K *__restrict__ ckeys) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  if (flag[i]) ckeys[pos[i]] = KeyOps<K>::parent(keys[i]);
}

// Coarse cell active iff a fully active fine oct refines it (pull).
template <class K>
__global__ void k_coarse_active(const K *__restrict__ ckeys, int64_t cn, const K *__restrict__ f_ht_keys,
                                const int32_t *__restrict__ f_ht_vals, uint64_t f_mask,
                                const uint8_t *__restrict__ f_active, bool f_all_active,
                                uint8_t *__restrict__ cactive) {
  const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (p >= cn) return;
  const K k = ckeys[p];
  uint8_t m = 0;
  for (int c = 0; c < 8; ++c) {
    const int32_t i = ht_find_k(f_ht_keys, f_ht_vals, f_mask, KeyOps<K>::child(k, c));
    if (i >= 0 && (f_all_active || f_active[i] == 0xFF)) m |= (uint8_t)(1u << c);
  }
  cactive[p] = m;
}

template <class K>
__global__ void k_father_and_block(const K *__restrict__ keys, const uint8_t *__restrict__ active, bool all_active,
                                   int64_t n, uint64_t cnpd, int pmask, const K *__restrict__ c_ht_keys,
                                   const int32_t *__restrict__ c_ht_vals, uint64_t c_mask, int32_t c_zero,
                                   int32_t *__restrict__ father, int32_t *__restrict__ blk) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const K k = keys[i];
  int32_t fa = -1;
  if (all_active || active[i] == 0xFF) {
    const int32_t p = ht_find_k(c_ht_keys, c_ht_vals, c_mask, KeyOps<K>::parent(k));
    if (p >= 0) fa = p * 8 + (int32_t)KeyOps<K>::octant(k);
  }
  father[i] = fa;
  int32_t b[8];
  father_block(k, cnpd, pmask, c_ht_keys, c_ht_vals, c_mask, c_zero, b);
#pragma unroll
  for (int t = 0; t < 8; ++t) blk[t * n + i] = b[t];
}

__global__ void k_fill_u8(uint8_t *p, int64_t n, uint8_t v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_replace_i32(int32_t *p, int64_t n, int32_t from, int32_t to) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n && p[i] == from) p[i] = to;
}

__global__ void k_fill_i32(int32_t *p, int64_t n, int32_t v) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) p[i] = v;
}

__global__ void k_ext_neighbors(const int32_t *__restrict__ nbr, int64_t n, int32_t *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[7 * i] = (int32_t)i;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int32_t v = nbr[d * n + i];
    out[7 * i + 1 + d] = v < n ? v : -1;
  }
}

template <class K>
__global__ void k_father_cells(const K *__restrict__ keys, const int32_t *__restrict__ nbr, int64_t n, uint64_t npd,
                               int pmask, bool has_parent, const K *__restrict__ p_ht_keys,
                               const int32_t *__restrict__ p_ht_vals, uint64_t p_mask, int32_t *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  const K e = KeyOps<K>::empty();
#pragma unroll 1
  for (int d = 0; d < 6; ++d) {
    int32_t p = -1, oc = -1;
    if (has_parent && nbr[d * n + i] >= n) {
      const K nk = neighbor_key_k(keys[i], d, npd, pmask);
      if (nk != e) {
        p = ht_find_k(p_ht_keys, p_ht_vals, p_mask, KeyOps<K>::parent(nk));
        oc = p >= 0 ? (int32_t)KeyOps<K>::octant(nk) : -1;
      }
    }
    out[12 * i + 2 * d] = p;
    out[12 * i + 2 * d + 1] = oc;
  }
}

__global__ void k_active_bytes(const uint8_t *__restrict__ active, bool all_active, int64_t n,
                               uint8_t *__restrict__ out) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  out[t] = all_active ? 1 : ((active[t >> 3] >> (t & 7)) & 1);
}

// ------------------------------------------------------------ host helpers

int read_error(cmg_ctx *ctx) {
  CMG_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CMG_CUDA(cudaStreamSynchronize(ctx->stream));
  const int e = ctx->h_pinned[0];
  if (e != 0) CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
  return e;
}

int32_t read_i32(cmg_ctx *ctx, const int32_t *d) {
  CMG_CUDA(cudaMemcpyAsync(ctx->h_pinned + 1, d, sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
  CMG_CUDA(cudaStreamSynchronize(ctx->stream));
  return ctx->h_pinned[1];
}

const char *status_text(int e) {
  switch (e) {
    case CMG_ERR_DUPLICATE_KEY: return "duplicate Morton key";
    case CMG_ERR_KEY_OUT_OF_RANGE: return "Morton key outside the level's coordinate range";
    case CMG_ERR_MISSING_PARENT: return "a coarse-fine ghost value has no parent cells to interpolate from";
    default: return "level build failed";
  }
}

template <class K>
void build_hash(cmg_level *L, cmg::MgLev &g, uint64_t npd) {
  cudaStream_t s = L->ctx->stream;
  g.cap = hash_capacity(g.n);
  K *&tab = LevelKeys<K>::table(g);
  tab = L->mem.alloc<K>(g.cap);
  g.ht_vals = L->mem.alloc<int32_t>(g.cap);
  CMG_CUDA(cudaMemsetAsync(tab, 0xFF, sizeof(K) * g.cap, s));
  if (g.n > 0)
    k_insert_keys<K><<<blocks_for(g.n), kThreads, 0, s>>>(LevelKeys<K>::keys(g), g.n, npd, tab, g.ht_vals,
                                                            (uint64_t)g.cap - 1, L->ctx->d_err);
  CMG_CUDA(cudaGetLastError());
}

// 128-bit levels keep their keys' low words for the solver kernels
template <class K>
void low_words(cmg_level *L, cmg::MgLev &g) {
  if constexpr (sizeof(K) == 16) {
    g.keys = L->mem.alloc<uint64_t>(g.n > 0 ? g.n : 1);
    if (g.n > 0) k_low_words<<<blocks_for(g.n), kThreads, 0, L->ctx->stream>>>(g.keys128, g.n, g.keys);
    CMG_CUDA(cudaGetLastError());
  }
}

uint64_t octs_per_dim(const cmg_level *L, int lev) { return (uint64_t)L->nx << (lev - 1); }

// Build L->mg[0] from keys, then the ghosts and the MG hierarchy.
template <class K>
void build_level_t(cmg_level *L, const K *keys, cmg_mem mem) {
  cmg_ctx *ctx = L->ctx;
  cudaStream_t s = ctx->stream;
  const uint64_t npd = octs_per_dim(L, L->lev);
  L->mg.clear();
  L->mg.emplace_back();
  MgLev &top = L->mg[0];
  top.lev = L->lev;
  top.n = L->n;
  top.h = std::ldexp(1.0, -L->lev) / L->nx;
  top.all_active = true;
  K *&tkeys = LevelKeys<K>::keys(top);
  tkeys = L->mem.alloc<K>(top.n);
  if (top.n > 0)
    CMG_CUDA(cudaMemcpyAsync(tkeys, keys, sizeof(K) * top.n,
                             mem == CMG_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), s));
  build_hash<K>(L, top, npd);
  low_words<K>(L, top);
  int e = read_error(ctx);
  if (e) throw Error(e, status_text(e));
  const K *ttab = LevelKeys<K>::table(top);

  // neighbour cache; INT_MIN marks "missing" until ghosts are assigned
  int32_t *d_cnt = L->mem.alloc<int32_t>(4, true, s);
  top.nbr = L->mem.alloc<int32_t>(6 * top.n);
  if (top.n > 0)
    k_neighbors<K><<<blocks_for(top.n), kThreads, 0, s>>>(tkeys, top.n, npd, L->pmask, ttab, top.ht_vals,
                                                           (uint64_t)top.cap - 1, INT_MIN, top.nbr, d_cnt);
  CMG_CUDA(cudaGetLastError());
  const int32_t n_missing = read_i32(ctx, d_cnt);

  top.n_ghost = 0;
  if (L->parent && n_missing > 0) {
    const int64_t gcap = hash_capacity(n_missing);
    K *g_keys = L->mem.alloc<K>(gcap);
    int32_t *g_vals = L->mem.alloc<int32_t>(gcap);
    CMG_CUDA(cudaMemsetAsync(g_keys, 0xFF, sizeof(K) * gcap, s));
    K *gk = L->mem.alloc<K>(n_missing);
    k_ghost_insert<K><<<blocks_for(top.n), kThreads, 0, s>>>(tkeys, top.n, npd, L->pmask, top.nbr, INT_MIN, g_keys,
                                                              g_vals, (uint64_t)gcap - 1, d_cnt + 1, gk, ctx->d_err);
    CMG_CUDA(cudaGetLastError());
    e = read_error(ctx);
    if (e) throw Error(e, status_text(e));
    top.n_ghost = read_i32(ctx, d_cnt + 1);
    if constexpr (sizeof(K) == 16) {
      L->ghost_keys128 = gk;
      L->ghost_keys = L->mem.alloc<uint64_t>(top.n_ghost > 0 ? top.n_ghost : 1);
      if (top.n_ghost > 0)
        k_low_words<<<blocks_for(top.n_ghost), kThreads, 0, s>>>(gk, top.n_ghost, L->ghost_keys);
    } else {
      L->ghost_keys = gk;
    }
    L->ghost_mask = L->mem.alloc<uint32_t>(top.n_ghost, true, s);
    k_ghost_resolve<K><<<blocks_for(top.n), kThreads, 0, s>>>(tkeys, top.n, npd, L->pmask, top.nbr, INT_MIN, g_keys,
                                                               g_vals, (uint64_t)gcap - 1, L->ghost_mask);
    CMG_CUDA(cudaGetLastError());
    const MgLev &pg = L->parent->mg[0];
    L->ghost_blk = L->mem.alloc<int32_t>(8 * top.n_ghost);
    k_ghost_blocks<K><<<blocks_for(top.n_ghost), kThreads, 0, s>>>(
        gk, top.n_ghost, L->ghost_mask, octs_per_dim(L, L->lev - 1), L->pmask, LevelKeys<K>::table(pg), pg.ht_vals,
        (uint64_t)pg.cap - 1, (int32_t)(pg.n_alloc - 1), L->ghost_blk, ctx->d_err);
    CMG_CUDA(cudaGetLastError());
    e = read_error(ctx);
    if (e) throw Error(e, status_text(e));
  }
  top.n_alloc = top.n + top.n_ghost + 1;
  // remaining missing neighbours (no parent): the zero oct
  if (top.n > 0)
    k_replace_i32<<<blocks_for(6 * top.n), kThreads, 0, s>>>(top.nbr, 6 * top.n, INT_MIN, (int32_t)(top.n_alloc - 1));
  CMG_CUDA(cudaGetLastError());
  top.active = L->mem.alloc<uint8_t>(top.n);
  if (top.n > 0) k_fill_u8<<<blocks_for(top.n), kThreads, 0, s>>>(top.active, top.n, 0xFF);
  top.phi = L->mem.alloc<double>(8 * top.n_alloc, true, s);
  top.g = L->mem.alloc<double>(8 * top.n, true, s);

  // multigrid hierarchy
  const int64_t scratch_n = scan_scratch_size(top.n > 0 ? top.n : 1);
  int32_t *scratch = L->mem.alloc<int32_t>(scratch_n);
  int32_t *flag = L->mem.alloc<int32_t>(top.n > 0 ? top.n : 1);
  int32_t *pos = L->mem.alloc<int32_t>(top.n > 0 ? top.n : 1);
  for (;;) {
    const size_t m = L->mg.size() - 1;
    if (L->mg[m].lev == 1 || L->mg[m].n == 0) break;
    const int64_t n = L->mg[m].n;
    const int64_t tcap = hash_capacity(n);
    K *t_keys = L->mem.alloc<K>(tcap);
    int32_t *t_min = L->mem.alloc<int32_t>(tcap);
    CMG_CUDA(cudaMemsetAsync(t_keys, 0xFF, sizeof(K) * tcap, s));
    k_fill_i32<<<blocks_for(tcap), kThreads, 0, s>>>(t_min, tcap, INT_MAX);
    {
      MgLev &f = L->mg[m];
      k_parent_first<K><<<blocks_for(n), kThreads, 0, s>>>(LevelKeys<K>::keys(f), f.active, f.all_active, n, t_keys,
                                                             t_min, (uint64_t)tcap - 1);
      k_parent_flag<K><<<blocks_for(n), kThreads, 0, s>>>(LevelKeys<K>::keys(f), f.active, f.all_active, n, t_keys,
                                                            t_min, (uint64_t)tcap - 1, flag);
    }
    CMG_CUDA(cudaGetLastError());
    scan_exclusive(flag, pos, n, d_cnt + 2, scratch, scratch_n, s);
    const int32_t np = read_i32(ctx, d_cnt + 2);
    if (np == 0) break;
    L->mg.emplace_back();
    MgLev &c = L->mg.back();
    MgLev &f = L->mg[m];
    c.lev = f.lev - 1;
    c.n = np;
    c.n_ghost = 0;
    c.n_alloc = np + 1;
    c.h = 2.0 * f.h;
    c.all_active = L->periodic_full;
    K *&ckeys = LevelKeys<K>::keys(c);
    ckeys = L->mem.alloc<K>(np);
    k_parent_emit<K><<<blocks_for(n), kThreads, 0, s>>>(LevelKeys<K>::keys(f), n, flag, pos, ckeys);
    CMG_CUDA(cudaGetLastError());
    const uint64_t cnpd = octs_per_dim(L, c.lev);
    build_hash<K>(L, c, cnpd);
    low_words<K>(L, c);
    const K *ctab = LevelKeys<K>::table(c);
    c.nbr = L->mem.alloc<int32_t>(6 * np);
    k_neighbors<K><<<blocks_for(np), kThreads, 0, s>>>(ckeys, np, cnpd, L->pmask, ctab, c.ht_vals,
                                                        (uint64_t)c.cap - 1, (int32_t)np, c.nbr, nullptr);
    c.active = L->mem.alloc<uint8_t>(np);
    k_coarse_active<K><<<blocks_for(np), kThreads, 0, s>>>(ckeys, np, LevelKeys<K>::table(f), f.ht_vals,
                                                            (uint64_t)f.cap - 1, f.active, f.all_active, c.active);
    f.father = L->mem.alloc<int32_t>(n);
    f.blk = L->mem.alloc<int32_t>(8 * n);
    k_father_and_block<K><<<blocks_for(n), kThreads, 0, s>>>(LevelKeys<K>::keys(f), f.active, f.all_active, n, cnpd,
                                                              L->pmask, ctab, c.ht_vals, (uint64_t)c.cap - 1,
                                                              (int32_t)np, f.father, f.blk);
    CMG_CUDA(cudaGetLastError());
    c.phi = L->mem.alloc<double>(8 * c.n_alloc, true, s);
    c.g = L->mem.alloc<double>(8 * c.n, true, s);
    e = read_error(ctx);
    if (e) throw Error(e, status_text(e));
  }
  const MgLev &last = L->mg.back();
  L->exact_coarse = L->periodic_full && last.lev == 1 && L->nx == 1 && last.n == 1;
  CMG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace

void encode_keys(const uint32_t *ijk, int64_t n, uint64_t *keys, int *err, cudaStream_t s) {
  if (n > 0) k_encode<<<blocks_for(n), kThreads, 0, s>>>(ijk, n, keys, err);
  CMG_CUDA(cudaGetLastError());
}

void decode_keys(const uint64_t *keys, int64_t n, uint32_t *ijk, cudaStream_t s) {
  if (n > 0) k_decode<<<blocks_for(n), kThreads, 0, s>>>(keys, n, ijk);
  CMG_CUDA(cudaGetLastError());
}

void encode_keys128(const uint64_t *ijk, int64_t n, Key128 *keys, int *err, cudaStream_t s) {
  if (n > 0) k_encode128<<<blocks_for(n), kThreads, 0, s>>>(ijk, n, keys, err);
  CMG_CUDA(cudaGetLastError());
}

void decode_keys128(const Key128 *keys, int64_t n, uint64_t *ijk, cudaStream_t s) {
  if (n > 0) k_decode128<<<blocks_for(n), kThreads, 0, s>>>(keys, n, ijk);
  CMG_CUDA(cudaGetLastError());
}

void hash_lookup(const MgLev &g, const uint64_t *q, int64_t n, int32_t *out, cudaStream_t s) {
  if (n > 0) k_lookup<uint64_t><<<blocks_for(n), kThreads, 0, s>>>(g.ht_keys, g.ht_vals, (uint64_t)g.cap - 1, q, n, out);
  CMG_CUDA(cudaGetLastError());
}

void hash_lookup128(const MgLev &g, const Key128 *q, int64_t n, int32_t *out, cudaStream_t s) {
  if (n > 0)
    k_lookup<Key128><<<blocks_for(n), kThreads, 0, s>>>(g.ht_keys128, g.ht_vals, (uint64_t)g.cap - 1, q, n, out);
  CMG_CUDA(cudaGetLastError());
}

void ext_neighbors(const cmg_level *L, int32_t *out, cudaStream_t s) {
  const MgLev &g = L->mg[0];
  if (g.n > 0) k_ext_neighbors<<<blocks_for(g.n), kThreads, 0, s>>>(g.nbr, g.n, out);
  CMG_CUDA(cudaGetLastError());
}

void father_cells(const cmg_level *L, int32_t *out, cudaStream_t s) {
  const MgLev &g = L->mg[0];
  const bool hp = L->parent != nullptr;
  const MgLev *pg = hp ? &L->parent->mg[0] : nullptr;
  if (g.n == 0) return;
  const uint64_t npd = (uint64_t)L->nx << (L->lev - 1);
  if (L->key_bits == 128)
    k_father_cells<Key128><<<blocks_for(g.n), kThreads, 0, s>>>(
        g.keys128, g.nbr, g.n, npd, L->pmask, hp, hp ? pg->ht_keys128 : nullptr, hp ? pg->ht_vals : nullptr,
        hp ? (uint64_t)pg->cap - 1 : 0, out);
  else
    k_father_cells<uint64_t><<<blocks_for(g.n), kThreads, 0, s>>>(
        g.keys, g.nbr, g.n, npd, L->pmask, hp, hp ? pg->ht_keys : nullptr, hp ? pg->ht_vals : nullptr,
        hp ? (uint64_t)pg->cap - 1 : 0, out);
  CMG_CUDA(cudaGetLastError());
}

void mg_active_bytes(const MgLev &g, uint8_t *out, cudaStream_t s) {
  if (g.n > 0) k_active_bytes<<<blocks_for(8 * g.n), kThreads, 0, s>>>(g.active, g.all_active, g.n, out);
  CMG_CUDA(cudaGetLastError());
}

void build_level(cmg_level *L, const void *keys, cmg_mem mem) {
  if (L->key_bits == 128)
    build_level_t<Key128>(L, static_cast<const Key128 *>(keys), mem);
  else
    build_level_t<uint64_t>(L, static_cast<const uint64_t *>(keys), mem);
  mark_lexicographic(L);
}

}  // namespace cmg
