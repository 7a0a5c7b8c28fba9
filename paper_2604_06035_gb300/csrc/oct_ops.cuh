// oct_ops.cuh -- per-oct bodies of the multigrid operators, shared by the
// one-kernel-per-operation path (launch.cu, kernels.cuh) and the tail kernels
// (tail.cu).  Layout: see cmg_internal.cuh.  CG = true routes every load of
// data that another thread block of the same launch may have written through
// L2 (ld.global.cg), as the grid tail's blocks exchange data via global
// memory between grid barriers.
#pragma once

#include "cmg_internal.cuh"

namespace cmg {
namespace dev {

template <bool CG>
__device__ __forceinline__ double2 ldv(const double2 *p) {
  if constexpr (CG) return __ldcg(p); else return *p;
}
template <bool CG>
__device__ __forceinline__ float4 ldv(const float4 *p) {
  if constexpr (CG) return __ldcg(p); else return *p;
}
template <bool CG, typename T>
__device__ __forceinline__ T ld1(const T *p) {
  if constexpr (CG) return __ldcg(p); else return *p;
}

template <bool CG>
__device__ __forceinline__ void load4(const double *p, double v[4]) {
  const double2 a = ldv<CG>(reinterpret_cast<const double2 *>(p));
  const double2 b = ldv<CG>(reinterpret_cast<const double2 *>(p + 2));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = b.x;
  v[3] = b.y;
}
template <bool CG>
__device__ __forceinline__ void load4(const float *p, float v[4]) {
  const float4 a = ldv<CG>(reinterpret_cast<const float4 *>(p));
  v[0] = a.x;
  v[1] = a.y;
  v[2] = a.z;
  v[3] = a.w;
}
__device__ __forceinline__ void store4(double *p, const double v[4]) {
  *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
  *reinterpret_cast<double2 *>(p + 2) = make_double2(v[2], v[3]);
}
__device__ __forceinline__ void store4(float *p, const float v[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// ---------------------------------------------------------------------------
// The six-neighbour sum of the 7-point stencil.
//
// GB300 issues FP64 at about 2 lanes per SM per clock, 1/64 of its FP32 rate,
// while its integer pipes sit idle in these kernels.  An FP64 sum can instead
// be formed exactly in integers: with E the largest biased exponent of the
// operands, each operand's 53-bit significand is shifted to the common scale
// 2^(E - 1082) (operands more than 7 binades below the largest lose the bits
// under that scale: at most 2^-59 of the largest operand each), the signed
// 64-bit integers are added (|sum| < 6 * 2^60, no overflow), and the integer
// sum is rounded once to the nearest FP64 value, ties to even.  The result is
// within half an ulp of the exact sum plus those truncations, more accurate
// than five sequential FP64 additions, and does not depend on the order of
// the operands.  Zero and subnormal operands contribute nothing (a subnormal
// is below 2^-1022, far under the scale).  The rounding is written out in
// integer operations: one biased truncation (CMG_FXNORM = 2, the default) or
// the dropped part compared with half (0); or it is the int64 -> FP64
// conversion (1).  The alignment below costs ~15 integer instructions per
// operand; an earlier form (significand assembled with its leading bit,
// shifted left 7 and right by E - e, negated as (m ^ s) - s) gave the same
// bits on 10^6 probe sums and ran 15 % slower on GB300.
// Measured on GB300 (512^3 FP64 colour pass): CMG_FXNORM = 2 0.407 ms
// against 0.422 ms for 0 (same bits); 1 was slower in the 4 + 2 split
// (0.486 -> 0.603 ms): the conversion issues on the FP64 pipe.
#ifndef CMG_FXNORM
#define CMG_FXNORM 2
#endif
// CMG_FXALIGN: 1 = the alignment below; 0 = the earlier form (same bits
// whenever some operand is 2^-960 or larger).
#ifndef CMG_FXALIGN
#define CMG_FXALIGN 1
#endif
// x >> s with PTX semantics: a shift of 64 or more gives 0.
__device__ __forceinline__ unsigned long long shr_clamped(unsigned long long x, unsigned s) {
  unsigned long long r;
  asm("shr.b64 %0, %1, %2;" : "=l"(r) : "l"(x), "r"(s));
  return r;
}

template <int N>
__device__ __forceinline__ double fixed_sum(const double *v) {
  uint32_t hi[N], lo[N];
  int e[N];
  int E = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    hi[k] = (uint32_t)__double2hiint(v[k]);
    lo[k] = (uint32_t)__double2loint(v[k]);
    e[k] = (int)((hi[k] >> 20) & 0x7FFu);
    E = max(E, e[k]);
  }
  // an infinity or NaN, an operand of 2^1021 or more (whose sum could
  // overflow the exponent field below), or every operand below 2^-960 (zeros
  // included): FP64 additions
  if (E >= 0x7FC || E < 64) {
    if (E == 0) {
      // all operands +-0 (a solve's first passes and residuals see whole
      // neighbourhoods of zeros): the FP64 additions' result without them,
      // -0 only when every operand is -0
      uint32_t nz = 0, neg = 0xFFFFFFFFu;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        nz |= (hi[k] & 0x7FFFFFFFu) | lo[k];
        neg &= hi[k];
      }
      if (nz == 0) return __longlong_as_double((long long)((unsigned long long)(neg & 0x80000000u) << 32));
    }
    double s = v[0];
#pragma unroll
    for (int k = 1; k < N; ++k) s += v[k];
    return s;
  }
  // each significand with its leading bit at bit 63 (one funnel shift and
  // the bit), then one right shift by E - e + 4 to the scale 2^(E - 1082);
  // zero and subnormal operands (e = 0) shift by E + 4 >= 68 and vanish.
  // Negative operands enter as ones' complements; the count of them, added
  // once, completes the two's complements.
  long long S = 0;
#if CMG_FXALIGN == 0
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const int ek = max(e[k], 1);
    const uint32_t lead = (hi[k] & 0x7FF00000u) ? 0x100000u : 0u;
    unsigned long long m = ((unsigned long long)((hi[k] & 0xFFFFFu) | lead) << 32) | lo[k];
    m = (m << 7) >> min(E - ek, 63);
    const long long sg = (long long)((int)hi[k] >> 31);
    S += ((long long)m ^ sg) - sg;
  }
#else
  int negs = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    const uint32_t top = __funnelshift_l(lo[k], hi[k], 11) | 0x80000000u;
    const unsigned long long m = ((unsigned long long)top << 32) | (lo[k] << 11);
    const unsigned long long a = shr_clamped(m, (unsigned)(E - e[k] + 4));
    const long long sg = (long long)((int)hi[k] >> 31);  // 0 or -1
    S += (long long)a ^ sg;
    negs -= (int)sg;
  }
  S += negs;
#endif
#if CMG_FXNORM == 1
  // rounding by the int64 -> FP64 conversion (round to nearest even), then
  // the exact scaling by 2^(E - 1082) through the exponent field
  const double d = __ll2double_rn(S);
  return d == 0.0 ? 0.0 : __hiloint2double(__double2hiint(d) + ((E - 1082) << 20), __double2loint(d));
#else
  if (S == 0) return 0.0;
  const unsigned long long neg = S < 0 ? 1ull : 0ull;
  const unsigned long long a = neg ? 0ull - (unsigned long long)S : (unsigned long long)S;
  const int p = 63 - __clzll((long long)a);  // leading bit of |S|, <= 62
  const int eb = E + p - 59;                 // biased exponent of the sum
  if (eb <= 0) return ldexp((double)S, E - 1082);  // subnormal sum (never in practice)
  unsigned long long mant;
  if (p > 52) {
    const int r = p - 52;  // 1 .. 10
#if CMG_FXNORM == 2
    // round half to even by one biased truncation: adding 2^(r-1) - 1 plus
    // the last kept bit carries into the kept bits exactly when the dropped
    // part is above half, or equal to it with the kept part odd
    const uint32_t lo = (uint32_t)a, hi = (uint32_t)(a >> 32);
    const unsigned long long b = a + (((1u << (r - 1)) - 1u) + ((__funnelshift_r(lo, hi, r)) & 1u));
    mant = ((unsigned long long)((uint32_t)(b >> 32) >> r) << 32) |
           __funnelshift_r((uint32_t)b, (uint32_t)(b >> 32), r);
#else
    const unsigned long long q = a >> r, rem = a & ((1ull << r) - 1ull), half = 1ull << (r - 1);
    mant = q + (unsigned long long)((rem > half) | ((rem == half) & (q & 1ull)));
#endif
  } else {
    mant = a << (52 - p);
  }
  // mant carries the leading bit at 2^52 (2^53 after a rounding carry), which
  // adds the last 1 (or 2) to the exponent field
  return __longlong_as_double((long long)(((unsigned long long)(eb - 1) << 52) + mant + (neg << 63)));
#endif
}

// Neighbour sum in the order (-x, +x, -y, +y, -z, +z).  FP32: sequential
// additions.  FP64 (CMG_NBSUM): 0 = five sequential FP64 additions; 1 = all
// six in the integer sum; 2 = the x and y neighbours in the integer sum, the
// two z neighbours by FP64 additions; 3 = five in the integer sum, the last
// by one FP64 addition (the FP64 and integer pipes share the work).
// Measured on GB300 (512^3 FP64 colour pass; 256^3 + 3-level FP64 chain on
// one box): 0 = 0.771 ms; 1 = 0.471 ms; 2 = 0.483 ms, 54.8 ms; 3 = 0.424 ms,
// 51.6 ms.  Every kernel forms every neighbour sum through this
// function, so a residual formed right after a colour pass repeats that
// pass's sums bit for bit.
#ifndef CMG_NBSUM
#define CMG_NBSUM 3
#endif
__device__ __forceinline__ float nbsum6(const float v[6]) {
  return ((((v[0] + v[1]) + v[2]) + v[3]) + v[4]) + v[5];
}
__device__ __forceinline__ double nbsum6(const double v[6]) {
#if CMG_NBSUM == 1
  return fixed_sum<6>(v);
#elif CMG_NBSUM == 2
  return (fixed_sum<4>(v) + v[4]) + v[5];
#elif CMG_NBSUM == 3
  return fixed_sum<5>(v) + v[5];
#else
  return ((((v[0] + v[1]) + v[2]) + v[3]) + v[4]) + v[5];
#endif
}

// The neighbour sum of a colour-0 residual cell (CMG_RESID_NB): 0 = nbsum6;
// 1 = all six in the integer sum.  No colour-0 residual has to repeat a
// colour pass's sum (only the colour-1 residuals after a colour-1 pass do,
// and they keep nbsum6), and the residual spends twice the sweep's FP64
// instructions per cell (the subtraction of phi and the norm or restriction
// sum), so its best split differs: measured on GB300 (256^3 + 3-level FP64
// chain, one box), the residual family 11.6 -> 10.9 ms per step with all six
// in integers.
#ifndef CMG_RESID_NB
#define CMG_RESID_NB 1
#endif
__device__ __forceinline__ float nbsum6_r0(const float v[6]) { return nbsum6(v); }
__device__ __forceinline__ double nbsum6_r0(const double v[6]) {
#if CMG_RESID_NB == 1
  return fixed_sum<6>(v);
#else
  return nbsum6(v);
#endif
}

template <typename T>
__device__ __forceinline__ T fma_t(T a, T b, T c);
template <>
__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
template <>
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }

// One colour pass of red-black Gauss-Seidel (App. D.2 Eq. (gs_update)) on
// oct i: plane P from the other plane of the oct and of its six face
// neighbours.  ZERO: the other plane is known to be zero, so phi = g.
//
// The *_idx loaders read an oct's index data (neighbours, active mask,
// father, interpolation block, octant), which only the level build writes;
// a one-launch-per-operation kernel reads it before its grid-dependency wait,
// overlapping the preceding kernel, and passes it to the *_oct_idx body.
struct SweepIdx {
  int32_t nb[6];
  unsigned m;
};
template <bool ZERO, bool MASK>
__device__ __forceinline__ SweepIdx sweep_idx(int64_t i, const int32_t *__restrict__ nbr,
                                              const uint8_t *__restrict__ active, int64_t n) {
  SweepIdx x;
#pragma unroll
  for (int d = 0; d < 6; ++d) x.nb[d] = ZERO ? 0 : __ldg(nbr + d * n + i);
  x.m = MASK ? __ldg(active + i) : 0xFFu;
  return x;
}

template <typename T, int P, bool ZERO, bool MASK, bool CG>
__device__ __forceinline__ void sweep_oct_idx(int64_t i, const SweepIdx &x, const T *src, T *dst, const T *g) {
  T gv[4], out[4];
  load4<CG>(g + i * 4, gv);
  if (ZERO) {
#pragma unroll
    for (int q = 0; q < 4; ++q) out[q] = gv[q];
  } else {
    T own[4];
    load4<CG>(src + i * 4, own);
    const int32_t *nb = x.nb;
    const T inv6 = T(1) / T(6);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = plane_cell(P, q);
      T v[6];
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
        v[d] = (((c >> a) & 1) != side) ? own[c2 >> 1] : ld1<CG>(src + (int64_t)nb[d] * 4 + (c2 >> 1));
      }
      out[q] = fma_t(nbsum6(v), inv6, gv[q]);
    }
  }
  if (MASK) {
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (!((x.m >> plane_cell(P, q)) & 1)) out[q] = T(0);
  }
  store4(dst + i * 4, out);
}

template <typename T, int P, bool ZERO, bool MASK, bool CG>
__device__ __forceinline__ void sweep_oct(int64_t i, const int32_t *__restrict__ nbr, const T *src, T *dst,
                                          const T *g, const uint8_t *__restrict__ active, int64_t n) {
  sweep_oct_idx<T, P, ZERO, MASK, CG>(i, sweep_idx<ZERO, MASK>(i, nbr, active, n), src, dst, g);
}

// sweep_oct for one cell (cell plane_cell(P, q) of oct i), one thread per
// cell: the same loads, sums in the same order and the same FMA, so the
// result is bit-identical to sweep_oct's.
template <typename T, int P, bool ZERO, bool MASK, bool CG>
__device__ __forceinline__ void sweep_cell(int64_t i, int q, const int32_t *__restrict__ nbr, const T *src, T *dst,
                                           const T *g, const uint8_t *__restrict__ active, int64_t n) {
  T out = ld1<CG>(g + i * 4 + q);
  if (!ZERO) {
    const int c = plane_cell(P, q);
    const T inv6 = T(1) / T(6);
    T v[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
      const int64_t o = (((c >> a) & 1) != side) ? i : (int64_t)__ldg(nbr + d * n + i);
      v[d] = ld1<CG>(src + o * 4 + (c2 >> 1));
    }
    out = fma_t(nbsum6(v), inv6, out);
  }
  if (MASK && !((__ldg(active + i) >> plane_cell(P, q)) & 1)) out = T(0);
  dst[i * 4 + q] = out;
}

// Residual of oct i: d = fma(s, 1/6, g) - phi per cell, r = (-6 / h^2) d.
// Returns the sum of d^2 over the oct (NORM; accumulated in FP64 for FP64
// data, in FP32 within the oct for FP32 data, whose FP64 conversions would
// otherwise bind the kernel to GB300's FP64 pipe).  RESTRICT: a fully active oct
// writes its father cell g_c = 0.5 * sum_8 d (= -h_c^2/6 * mean_8 r) and, if
// zero_cphi, zeroes the father's phi.  EMIT: g32 = (float)(d * inv_s).
// ROUT: r oct-major.  ZPHI: phi taken as zero on real octs.
// The FP32 right-hand side of a mixed-precision solve's correction problem,
// (float)(x * s) with s a power of two: the scaling and the rounding to FP32
// (to nearest, ties to even) formed in integer operations, since GB300
// issues FP64 multiplications and conversions at its low FP64 rate (the
// residual kernel that emits it went 11 % faster).  Zero, a scale that is
// not a normal power of two, and results outside FP32's normal range take
// the FP64 operations instead (same results).
__device__ __forceinline__ float f32_scaled(double x, double s) {
  const unsigned long long sb = (unsigned long long)__double_as_longlong(s);
  const unsigned long long xb = (unsigned long long)__double_as_longlong(x);
  const int es = (int)((sb >> 52) & 0x7FF), ex = (int)((xb >> 52) & 0x7FF);
  const int fe = ex + es - 2046 + 127;  // FP32 biased exponent of x * s
  if ((sb & 0x800FFFFFFFFFFFFFull) != 0 || es == 0 || es == 0x7FF || ex == 0 || fe <= 0 || fe >= 255)
    return (float)(x * s);
  const unsigned long long mant = xb & 0x000FFFFFFFFFFFFFull;
  // round the 52-bit fraction to 23 bits: a carry runs into the exponent
  // field (and from the largest binade to infinity, as the conversion does)
  const uint32_t m = (uint32_t)((mant + 0x0FFFFFFFull + ((mant >> 29) & 1ull)) >> 29);
  return __uint_as_float((((uint32_t)fe << 23) + m) | ((uint32_t)(xb >> 32) & 0x80000000u));
}
struct ResidIdx {
  int32_t nb[6];
  unsigned m;
  int32_t fa;
};
template <bool RESTRICT>
__device__ __forceinline__ ResidIdx resid_idx(int64_t i, const int32_t *__restrict__ nbr,
                                              const uint8_t *__restrict__ active, int64_t n,
                                              const int32_t *__restrict__ father) {
  ResidIdx x;
#pragma unroll
  for (int d = 0; d < 6; ++d) x.nb[d] = __ldg(nbr + d * n + i);
  x.m = active ? __ldg(active + i) : 0xFFu;
  x.fa = RESTRICT ? __ldg(father + i) : -1;
  return x;
}

//
// C1Z: the last operation on this level was a colour-1 pass over every oct
// with the colour-0 values, g and ghost values the residual now reads.  That
// pass wrote fma(s, 1/6, g) at each active colour-1 cell, and this function
// forms the same s from the same values in the same order, so each
// colour-1 residual is exactly +0 (inactive cells are +0 anyway): their
// stencils are skipped.  Skipping changes no result bit: the norm gains
// +0 terms (acc >= +0 throughout), the restriction sum would gain +0 four
// times, which leaves it unchanged (it is never -0), and EMIT / ROUT write
// what dv = +0 gives.
template <typename T, bool NORM, bool RESTRICT, bool EMIT, bool ROUT, bool ZPHI, bool CG, bool C1Z = false>
__device__ __forceinline__ double resid_oct_idx(int64_t i, const ResidIdx &x, const T *phi, const T *g, int64_t n,
                                                int64_t n_alloc, T *cg, T *cphi, int64_t cn, int64_t cn_alloc,
                                                int zero_cphi, float *g32, double inv_s, double *rout,
                                                double rscale) {
  T pl[2][4], gv[2][4];
  if (ZPHI) {
#pragma unroll
    for (int q = 0; q < 4; ++q) pl[0][q] = pl[1][q] = T(0);
  } else {
    load4<CG>(phi + i * 4, pl[0]);
    load4<CG>(phi + (n_alloc + i) * 4, pl[1]);
  }
  load4<CG>(g + i * 4, gv[0]);
  if (!C1Z) load4<CG>(g + (n + i) * 4, gv[1]);
  const int32_t *nb = x.nb;
  const T inv6 = T(1) / T(6);
  const unsigned m = x.m;
  T rsum = T(0);
  double acc = 0.0;
  T tacc = T(0);  // FP32 data: the oct's squares summed in FP32, one conversion
#pragma unroll
  for (int p = 0; p < 2; ++p) {
    if (C1Z && p == 1) {
      // rsum needs no + 0 for the four zeros: it starts at +0 and a sum that
      // cancels rounds to +0, so it is never -0
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (EMIT) g32[(p * n + i) * 4 + q] = f32_scaled((double)T(0), inv_s);
        if (ROUT) rout[i * 8 + plane_cell(p, q)] = rscale * 0.0;
      }
      continue;
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = plane_cell(p, q);
      T v[6];
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
        if (((c >> a) & 1) != side) {
          v[d] = pl[1 - p][c2 >> 1];
        } else {
          const int64_t o = nb[d];
          v[d] = (ZPHI && o < n) ? T(0) : ld1<CG>(phi + ((1 - p) * n_alloc + o) * 4 + (c2 >> 1));
        }
      }
      T dv = fma_t(p == 0 ? nbsum6_r0(v) : nbsum6(v), inv6, gv[p][q]) - pl[p][q];
      if (!((m >> c) & 1)) dv = T(0);
      if (NORM) {
        if constexpr (sizeof(T) == 8)
          acc = fma((double)dv, (double)dv, acc);
        else
          tacc = fma_t(dv, dv, tacc);
      }
      if (RESTRICT) rsum += dv;
      if (EMIT) g32[(p * n + i) * 4 + q] = f32_scaled((double)dv, inv_s);
      if (ROUT) rout[i * 8 + c] = rscale * (double)dv;
    }
  }
  if (NORM && sizeof(T) == 4) acc = (double)tacc;
  if (RESTRICT) {
    const int32_t fa = x.fa;
    if (fa >= 0) {
      const int64_t pc = fa >> 3;
      const int cc = fa & 7;
      cg[((int64_t)cell_parity(cc) * cn + pc) * 4 + (cc >> 1)] = T(0.5) * rsum;
      if (zero_cphi) cphi[((int64_t)cell_parity(cc) * cn_alloc + pc) * 4 + (cc >> 1)] = T(0);
    }
  }
  return acc;
}

template <typename T, bool NORM, bool RESTRICT, bool EMIT, bool ROUT, bool ZPHI, bool CG, bool C1Z = false>
__device__ __forceinline__ double resid_oct(int64_t i, const int32_t *__restrict__ nbr, const T *phi, const T *g,
                                            const uint8_t *__restrict__ active, int64_t n, int64_t n_alloc,
                                            const int32_t *__restrict__ father, T *cg, T *cphi, int64_t cn,
                                            int64_t cn_alloc, int zero_cphi, float *g32, double inv_s,
                                            double *rout, double rscale) {
  return resid_oct_idx<T, NORM, RESTRICT, EMIT, ROUT, ZPHI, CG, C1Z>(i, resid_idx<RESTRICT>(i, nbr, active, n, father),
                                                                phi, g, n, n_alloc, cg, cphi, cn, cn_alloc,
                                                                zero_cphi, g32, inv_s, rout, rscale);
}

// resid_oct<NORM = false, RESTRICT = true> with one thread per cell: lane k
// of an aligned group of 8 lanes takes cell plane_cell(k >> 2, k & 3) of oct
// i (plane k >> 2, slot k & 3).  Every lane of the warp calls it (the father
// value is summed across the group by shuffles, in resid_oct's order);
// `valid` is false for a group past the end of the range.
template <typename T, bool CG>
__device__ __forceinline__ void resid_restrict_cell(bool valid, int64_t i, const int32_t *__restrict__ nbr, const T *phi,
                                                    const T *g, const uint8_t *__restrict__ active, int64_t n,
                                                    int64_t n_alloc, const int32_t *__restrict__ father, T *cg, T *cphi,
                                                    int64_t cn, int64_t cn_alloc, int zero_cphi) {
  const int k = (int)(threadIdx.x & 7), p = k >> 2, q = k & 3, c = plane_cell(p, q);
  T dv = T(0);
  if (valid) {
    const T pv = ld1<CG>(phi + (p * n_alloc + i) * 4 + q);
    const T gv = ld1<CG>(g + (p * n + i) * 4 + q);
    const T inv6 = T(1) / T(6);
    T v[6];
#pragma unroll
    for (int d = 0; d < 6; ++d) {
      const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
      const int64_t o = (((c >> a) & 1) != side) ? i : (int64_t)__ldg(nbr + d * n + i);
      v[d] = ld1<CG>(phi + ((1 - p) * n_alloc + o) * 4 + (c2 >> 1));
    }
    if (p == 0)
      dv = fma_t(nbsum6_r0(v), inv6, gv) - pv;
    else
      dv = fma_t(nbsum6(v), inv6, gv) - pv;
    const unsigned m = active ? __ldg(active + i) : 0xFFu;
    if (!((m >> c) & 1)) dv = T(0);
  }
  const int base = (int)(threadIdx.x & 31) & ~7;
  T rsum = T(0);
#pragma unroll
  for (int j = 0; j < 8; ++j) rsum += __shfl_sync(0xFFFFFFFFu, dv, base + j);
  if (valid && k == 0) {
    const int32_t fa = __ldg(father + i);
    if (fa >= 0) {
      const int64_t pc = fa >> 3;
      const int cc = fa & 7;
      cg[((int64_t)cell_parity(cc) * cn + pc) * 4 + (cc >> 1)] = T(0.5) * rsum;
      if (zero_cphi) cphi[((int64_t)cell_parity(cc) * cn_alloc + pc) * 4 + (cc >> 1)] = T(0);
    }
  }
}

// Block index and child bit of the coarse cell at offset e - 1 (e = 0, 1, 2)
// along one axis from a father cell whose octant bit is cx; the block of 8
// coarse octs is displaced toward the father's octant.
__device__ __forceinline__ void axis_cell(int cx, int e, int &a, int &bit) {
  if (cx == 0) {
    a = (e == 0);
    bit = (e != 1);
  } else {
    a = (e == 2);
    bit = (e == 1);
  }
}

// Trilinear cell-centred interpolation of a coarse field onto the 8 children
// of the coarse cell (block octs b, octant cc): per axis weight 3/4 for the
// father, 1/4 for its neighbour toward the child (Sec. 5.1.1).
//
// CMG_PROLONG_SEP = 1: separably, in units of 1/4 per axis: along x each pair
// (father, neighbour) becomes 3 a + b in one FMA, then the same along y and
// along z, giving 64 x the value (weights 27, 9, 3, 1).  A child costs 7 FMAs
// and the children of an oct share their x and y stages (the 4 colour-1
// children of an oct 26 FMAs, all 8 of them 38, against 32 and 64 for the
// weighted eight-term sum); the 64 is divided out exactly (a power of two)
// in the FMA that adds the correction to phi, or by a multiplication for a
// plain value.  CMG_PROLONG_SEP = 0: the eight weighted terms in one FMA
// chain.
#ifndef CMG_PROLONG_SEP
#define CMG_PROLONG_SEP 1
#endif
// 3 a + b with one rounding
template <typename T>
__device__ __forceinline__ T tri3(T father, T side) {
  return fma_t(T(3), father, side);
}
// 64 x the interpolated value of one child from the coarse values around
// it: vXYZ with 1 = the father's coordinate on that axis, s = its neighbour
// toward the child.
template <typename T>
__device__ __forceinline__ T interp64(T v111, T vs11, T v1s1, T vss1, T v11s, T vs1s, T v1ss, T vsss) {
  return tri3(tri3(tri3(v111, vs11), tri3(v1s1, vss1)), tri3(tri3(v11s, vs1s), tri3(v1ss, vsss)));
}
constexpr double kInv64 = 0.015625;

// The 8 children's values (X64 = false) or, with CMG_PROLONG_SEP = 1 and
// X64 = true, 64 x them.
template <typename T, bool CG, bool X64 = false>
__device__ __forceinline__ void interp8(const T *cphi, int64_t cn_alloc, const int32_t b[8], int cc, T out[8]) {
  T v[27];
#pragma unroll
  for (int ez = 0; ez < 3; ++ez)
#pragma unroll
    for (int ey = 0; ey < 3; ++ey)
#pragma unroll
      for (int ex = 0; ex < 3; ++ex) {
        int ax, bx, ay, by, az, bz;
        axis_cell(cc & 1, ex, ax, bx);
        axis_cell((cc >> 1) & 1, ey, ay, by);
        axis_cell((cc >> 2) & 1, ez, az, bz);
        const int ch = bx | (by << 1) | (bz << 2);
        const int64_t oct = b[ax | (ay << 1) | (az << 2)];
        v[ex + 3 * ey + 9 * ez] = ld1<CG>(cphi + ((int64_t)cell_parity(ch) * cn_alloc + oct) * 4 + (ch >> 1));
      }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int fx = c & 1, fy = (c >> 1) & 1, fz = (c >> 2) & 1;
    const int ex1 = fx ? 2 : 0, ey1 = fy ? 2 : 0, ez1 = fz ? 2 : 0;
#if CMG_PROLONG_SEP
    const T z = interp64(v[1 + 3 * 1 + 9 * 1], v[ex1 + 3 * 1 + 9 * 1], v[1 + 3 * ey1 + 9 * 1],
                         v[ex1 + 3 * ey1 + 9 * 1], v[1 + 3 * 1 + 9 * ez1], v[ex1 + 3 * 1 + 9 * ez1],
                         v[1 + 3 * ey1 + 9 * ez1], v[ex1 + 3 * ey1 + 9 * ez1]);
    out[c] = X64 ? z : z * T(kInv64);
#else
    const T w0 = T(0.75), w1 = T(0.25);
    T acc = w0 * w0 * w0 * v[1 + 3 * 1 + 9 * 1];
    acc = fma_t(w1 * w0 * w0, v[ex1 + 3 * 1 + 9 * 1], acc);
    acc = fma_t(w0 * w1 * w0, v[1 + 3 * ey1 + 9 * 1], acc);
    acc = fma_t(w1 * w1 * w0, v[ex1 + 3 * ey1 + 9 * 1], acc);
    acc = fma_t(w0 * w0 * w1, v[1 + 3 * 1 + 9 * ez1], acc);
    acc = fma_t(w1 * w0 * w1, v[ex1 + 3 * 1 + 9 * ez1], acc);
    acc = fma_t(w0 * w1 * w1, v[1 + 3 * ey1 + 9 * ez1], acc);
    acc = fma_t(w1 * w1 * w1, v[ex1 + 3 * ey1 + 9 * ez1], acc);
    out[c] = acc;
#endif
  }
}

// phi + the child's correction as interp8<..., true> gives it
template <typename T>
__device__ __forceinline__ T add_corr(T phi, T corr) {
#if CMG_PROLONG_SEP
  return fma_t(corr, T(kInv64), phi);
#else
  return phi + corr;
#endif
}

// phi[i] += trilinear interpolation of the coarse correction (active cells).
struct ProlongIdx {
  int32_t b[8];
  int cc;
  unsigned m;
};
template <bool MASK>
__device__ __forceinline__ ProlongIdx prolong_idx(int64_t i, const uint64_t *__restrict__ keys,
                                                  const int32_t *__restrict__ blk, int64_t n,
                                                  const uint8_t *__restrict__ active) {
  ProlongIdx x;
  x.cc = (int)(__ldg(keys + i) & 7);
#pragma unroll
  for (int t = 0; t < 8; ++t) x.b[t] = __ldg(blk + t * n + i);
  x.m = MASK ? __ldg(active + i) : 0xFFu;
  return x;
}

// C0D: a colour-0 pass over every oct comes next; it overwrites each
// colour-0 value without reading it (the update uses only the colour-1
// neighbours and g), so the colour-0 corrections are dead and only colour-1
// cells are corrected (the unused interpolation terms and loads drop out).
template <typename T, bool MASK, bool CG, bool C0D = false>
__device__ __forceinline__ void prolong_oct_idx(int64_t i, const ProlongIdx &x, int64_t n_alloc, T *phi,
                                                const T *cphi, int64_t cn_alloc) {
  T corr[8];
  interp8<T, CG, true>(cphi, cn_alloc, x.b, x.cc, corr);
  const unsigned m = x.m;
#pragma unroll
  for (int p = C0D ? 1 : 0; p < 2; ++p) {
    T v[4];
    load4<CG>(phi + (p * n_alloc + i) * 4, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int c = plane_cell(p, q);
      if ((m >> c) & 1) v[q] = add_corr(v[q], corr[c]);
    }
    store4(phi + (p * n_alloc + i) * 4, v);
  }
}

template <typename T, bool MASK, bool CG, bool C0D = false>
__device__ __forceinline__ void prolong_oct(int64_t i, const uint64_t *__restrict__ keys,
                                            const int32_t *__restrict__ blk, int64_t n, int64_t n_alloc, T *phi,
                                            const uint8_t *__restrict__ active, const T *cphi, int64_t cn_alloc) {
  prolong_oct_idx<T, MASK, CG, C0D>(i, prolong_idx<MASK>(i, keys, blk, n, active), n_alloc, phi, cphi, cn_alloc);
}

// prolong_oct for one cell c of oct i, one thread per cell: the 8 coarse
// values interp8 combines for this cell, in its order and with its weights
// (bit-identical); inactive cells are left untouched.
template <typename T, bool MASK, bool CG>
__device__ __forceinline__ void prolong_cell(int64_t i, int c, const uint64_t *__restrict__ keys,
                                             const int32_t *__restrict__ blk, int64_t n, int64_t n_alloc, T *phi,
                                             const uint8_t *__restrict__ active, const T *cphi, int64_t cn_alloc) {
  if (MASK && !((__ldg(active + i) >> c) & 1)) return;
  const int cc = (int)(__ldg(keys + i) & 7);
  auto val = [&](int ex, int ey, int ez) -> T {
    int ax, bx, ay, by, az, bz;
    axis_cell(cc & 1, ex, ax, bx);
    axis_cell((cc >> 1) & 1, ey, ay, by);
    axis_cell((cc >> 2) & 1, ez, az, bz);
    const int ch = bx | (by << 1) | (bz << 2);
    const int64_t oct = __ldg(blk + (int64_t)(ax | (ay << 1) | (az << 2)) * n + i);
    return ld1<CG>(cphi + ((int64_t)cell_parity(ch) * cn_alloc + oct) * 4 + (ch >> 1));
  };
  const int ex1 = (c & 1) ? 2 : 0, ey1 = ((c >> 1) & 1) ? 2 : 0, ez1 = ((c >> 2) & 1) ? 2 : 0;
#if CMG_PROLONG_SEP
  const T acc = interp64(val(1, 1, 1), val(ex1, 1, 1), val(1, ey1, 1), val(ex1, ey1, 1), val(1, 1, ez1),
                         val(ex1, 1, ez1), val(1, ey1, ez1), val(ex1, ey1, ez1));
#else
  const T w0 = T(0.75), w1 = T(0.25);
  T acc = w0 * w0 * w0 * val(1, 1, 1);
  acc = fma_t(w1 * w0 * w0, val(ex1, 1, 1), acc);
  acc = fma_t(w0 * w1 * w0, val(1, ey1, 1), acc);
  acc = fma_t(w1 * w1 * w0, val(ex1, ey1, 1), acc);
  acc = fma_t(w0 * w0 * w1, val(1, 1, ez1), acc);
  acc = fma_t(w1 * w0 * w1, val(ex1, 1, ez1), acc);
  acc = fma_t(w0 * w1 * w1, val(1, ey1, ez1), acc);
  acc = fma_t(w1 * w1 * w1, val(ex1, ey1, ez1), acc);
#endif
  T *dst = phi + ((int64_t)cell_parity(c) * n_alloc + i) * 4 + (c >> 1);
  *dst = add_corr(ld1<CG>(dst), acc);
}

// Exact solve of the periodic 2^3 oct by one warp (all 32 lanes call it;
// lanes 0..7 own cell c = lane): eigenvectors (-1)^{k.b}, eigenvalues
// -4 |k|_1 / h^2, mean mode dropped; FP64 inside.  Each lane forms one
// transform coefficient and one output from the others' values (shuffles),
// in the same order of operations as a serial evaluation.
template <typename S, typename T, bool CG>
__device__ void wht_solve_warp(const S *g, T *phi, int64_t n_alloc, double h) {
  const unsigned all = 0xFFFFFFFFu;
  const int c = (int)(threadIdx.x & 7);
  const double f = (double)ld1<CG>(g + cell_parity(c) * 4 + (c >> 1)) * (-6.0 / (h * h));
  double s = 0.0;
#pragma unroll
  for (int b = 0; b < 8; ++b) {
    const double fb = __shfl_sync(all, f, b);
    s += cell_parity(c & b) ? -fb : fb;
  }
  const double fh = s * 0.125;
  const int odd = (c & 1) + ((c >> 1) & 1) + ((c >> 2) & 1);
  const double x = c ? fh / (-4.0 * odd / (h * h)) : 0.0;
  double t = 0.0;
#pragma unroll
  for (int k = 1; k < 8; ++k) {
    const double xk = __shfl_sync(all, x, k);
    t += cell_parity(k & c) ? -xk : xk;
  }
  if ((threadIdx.x & 31) < 8) phi[(int64_t)cell_parity(c) * n_alloc * 4 + (c >> 1)] = (T)t;
}

}  // namespace dev
}  // namespace cmg
