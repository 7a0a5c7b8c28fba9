// keys.cuh -- Morton keys of either width (Sec. 4.2: a 64-bit key with B = 21
// bits per coordinate, a 128-bit key with B = 42) behind one interface, and
// the per-level hash table (App. B) over them, for the level build.
//
//   KeyOps<uint64_t>  levels up to 22 (n_x = 1): the default
//   KeyOps<Key128>    levels up to 43: key bits 0..125, stored as (lo, hi)
//
// Both interleave bit b of (i, j, k) into key bits (3b, 3b+1, 3b+2) (Sec. 4.2
// Eq. (morton_encode)).  A 128-bit key is the 64-bit interleave of the low 21
// bits of each coordinate (key bits 0..62) plus that of the high 21 bits
// shifted up by 63.  The hash reduces a key to 64 bits first -- the key itself,
// or the XOR of its two halves for 128-bit keys (App. B) -- then mixes it with
// Eq. (hash_func).  Insertion claims a slot with a compare-and-swap of the
// whole key (16-byte CAS on sm_90 and later for 128-bit keys).
//
// The solver kernels never see the key width: they read only a key's lowest
// three bits (the oct's octant in its father), which a 128-bit level keeps in
// an array of its keys' low words.
#pragma once

#include "cmg_internal.cuh"

namespace cmg {

__host__ __device__ inline bool operator==(const Key128 &a, const Key128 &b) { return a.lo == b.lo && a.hi == b.hi; }
__host__ __device__ inline bool operator!=(const Key128 &a, const Key128 &b) { return !(a == b); }

template <class K>
struct KeyOps;

template <>
struct KeyOps<uint64_t> {
  static constexpr int kBits = 21;
  __host__ __device__ static uint64_t empty() { return kEmptyKey; }
  __host__ __device__ static uint64_t encode(uint64_t i, uint64_t j, uint64_t k) {
    return morton_encode((uint32_t)i, (uint32_t)j, (uint32_t)k);
  }
  __host__ __device__ static void decode(uint64_t m, uint64_t c[3]) {
    uint32_t i, j, k;
    morton_decode(m, i, j, k);
    c[0] = i;
    c[1] = j;
    c[2] = k;
  }
  __host__ __device__ static uint64_t parent(uint64_t m) { return m >> 3; }
  __host__ __device__ static uint64_t child(uint64_t m, int c) { return (m << 3) | (uint64_t)c; }
  __host__ __device__ static int octant(uint64_t m) { return (int)(m & 7); }
  __host__ __device__ static uint64_t fold(uint64_t m) { return m; }
  __host__ __device__ static uint64_t low(uint64_t m) { return m; }
  // valid keys leave the top bit clear (the all-ones key marks empty slots)
  __host__ __device__ static bool in_range(uint64_t m) { return (m >> 63) == 0; }
};

template <>
struct KeyOps<Key128> {
  static constexpr int kBits = 42;
  __host__ __device__ static Key128 empty() { return Key128{~0ull, ~0ull}; }
  __host__ __device__ static Key128 encode(uint64_t i, uint64_t j, uint64_t k) {
    const uint64_t m21 = (1ull << 21) - 1;
    const uint64_t a = morton_encode((uint32_t)(i & m21), (uint32_t)(j & m21), (uint32_t)(k & m21));
    const uint64_t b = morton_encode((uint32_t)(i >> 21), (uint32_t)(j >> 21), (uint32_t)(k >> 21));
    return Key128{a | (b << 63), b >> 1};
  }
  __host__ __device__ static void decode(const Key128 &m, uint64_t c[3]) {
    const uint64_t a = m.lo & ~(1ull << 63);
    const uint64_t b = (m.hi << 1) | (m.lo >> 63);
    uint32_t al[3], bh[3];
    morton_decode(a, al[0], al[1], al[2]);
    morton_decode(b, bh[0], bh[1], bh[2]);
    for (int t = 0; t < 3; ++t) c[t] = (uint64_t)al[t] | ((uint64_t)bh[t] << 21);
  }
  __host__ __device__ static Key128 parent(const Key128 &m) { return Key128{(m.lo >> 3) | (m.hi << 61), m.hi >> 3}; }
  __host__ __device__ static Key128 child(const Key128 &m, int c) {
    return Key128{(m.lo << 3) | (uint64_t)c, (m.hi << 3) | (m.lo >> 61)};
  }
  __host__ __device__ static int octant(const Key128 &m) { return (int)(m.lo & 7); }
  __host__ __device__ static uint64_t fold(const Key128 &m) { return m.lo ^ m.hi; }
  __host__ __device__ static uint64_t low(const Key128 &m) { return m.lo; }
  // 3 B = 126 key bits
  __host__ __device__ static bool in_range(const Key128 &m) { return (m.hi >> 62) == 0; }
};

// App. A Alg. 2 for either width: neighbour key in direction d (0..5 =
// -x,+x,-y,+y,-z,+z) on a grid of npd octs per axis, periodic on the axes of
// pmask, else the empty key ("outside the box").
template <class K>
__host__ __device__ inline K neighbor_key_k(const K &m, int d, uint64_t npd, int pmask) {
  uint64_t c[3];
  KeyOps<K>::decode(m, c);
  const int a = d >> 1;
  if (d & 1) {
    if (c[a] + 1 < npd) c[a] += 1;
    else if ((pmask >> a) & 1) c[a] = 0;
    else return KeyOps<K>::empty();
  } else {
    if (c[a] > 0) c[a] -= 1;
    else if ((pmask >> a) & 1) c[a] = npd - 1;
    else return KeyOps<K>::empty();
  }
  return KeyOps<K>::encode(c[0], c[1], c[2]);
}

// ------------------------------------------------------------------ hash

__device__ inline bool cas_key(uint64_t *slot, uint64_t expect, uint64_t k, uint64_t *prev) {
  *prev = atomicCAS(reinterpret_cast<unsigned long long *>(slot), (unsigned long long)expect, (unsigned long long)k);
  return *prev == expect;
}
__device__ inline bool cas_key(Key128 *slot, Key128 expect, Key128 k, Key128 *prev) {
  *prev = atomicCAS(slot, expect, k);
  return *prev == expect;
}

template <class K>
__device__ inline int32_t ht_find_k(const K *__restrict__ keys, const int32_t *__restrict__ vals, uint64_t mask,
                                    const K &k) {
  uint64_t s = hash_mix(KeyOps<K>::fold(k)) & mask;
  const K e = KeyOps<K>::empty();
  for (uint64_t p = 0; p <= mask; ++p) {
    const K kk = keys[s];
    if (kk == k) return vals[s];
    if (kk == e) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}

// Slot of k, inserting it if absent (*inserted says which); -1 if the table is
// full (cannot happen at fill <= 0.7).
template <class K>
__device__ inline int64_t ht_insert_slot_k(K *keys, uint64_t mask, const K &k, bool *inserted) {
  uint64_t s = hash_mix(KeyOps<K>::fold(k)) & mask;
  const K e = KeyOps<K>::empty();
  for (uint64_t p = 0; p <= mask; ++p) {
    K prev;
    if (cas_key(keys + s, e, k, &prev)) {
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

template <class K>
__device__ inline int64_t ht_slot_k(const K *__restrict__ keys, uint64_t mask, const K &k) {
  uint64_t s = hash_mix(KeyOps<K>::fold(k)) & mask;
  const K e = KeyOps<K>::empty();
  for (uint64_t p = 0; p <= mask; ++p) {
    const K kk = keys[s];
    if (kk == k) return (int64_t)s;
    if (kk == e) return -1;
    s = (s + 1) & mask;
  }
  return -1;
}

// Key arrays of a multigrid level by width: the keys and the hash table's key
// slots (a 128-bit level also keeps its keys' low words in MgLev::keys).
template <class K>
struct LevelKeys;
template <>
struct LevelKeys<uint64_t> {
  static uint64_t *&keys(MgLev &g) { return g.keys; }
  static uint64_t *&table(MgLev &g) { return g.ht_keys; }
  static const uint64_t *table(const MgLev &g) { return g.ht_keys; }
};
template <>
struct LevelKeys<Key128> {
  static Key128 *&keys(MgLev &g) { return g.keys128; }
  static Key128 *&table(MgLev &g) { return g.ht_keys128; }
  static const Key128 *table(const MgLev &g) { return g.ht_keys128; }
};

}  // namespace cmg
