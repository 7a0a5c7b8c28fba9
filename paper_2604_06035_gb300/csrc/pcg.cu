// pcg.cu -- multigrid-preconditioned conjugate gradients on one level (the
// paper names multigrid as the preconditioner of a CG solve, App. D.2).
//
// Flexible (Polak-Ribiere) CG, because a V-cycle that smooths red first in
// both legs is not exactly symmetric:
//   r0 = f - L phi0 (true residual, Dirichlet ghosts); z = M r; p = z (first)
//   loop: q = L0 p; alpha = (r, z) / (p, q); phi += alpha p; r' = r - alpha q;
//         stop on ||r'||; z' = M r'; beta = (z', r' - r) / (z, r); p = z' + beta p
// (r' - r = -alpha q, so the numerator is formed as -alpha (z', q) and the old
// residual is never stored)
// M = one V-cycle from zero with homogeneous coarse-fine values (the level's
// own V-cycle, reading its right-hand side array, which holds r during the
// iteration), or in mixed precision inner_cycles FP32 V-cycles on r / ||r||
// scaled back by ||r|| (flexible CG tolerates the inexact FP32 solve);
// L0 = the operator with homogeneous coarse-fine values.  On a
// periodic level z is projected to zero mean (the operator's null space).
// Everything is FP64 and in the solver's pre-scaled units (d = -h^2 r / 6;
// the iteration is invariant to that scale); r lives in the level's
// right-hand side array, saved at set-up and restored at wrap-up.  Dot products are per-block
// partial sums reduced in a fixed order (deterministic), alpha and beta are
// formed on the device, and the iteration runs as the set-up / body /
// wrap-up segments of the level solve's CUDA graph (solve.cu): the residual
// norm goes to the same control block as the stationary iteration's.
#include <cmath>

#include "cmg_internal.cuh"

namespace cmg {
namespace {

constexpr int kPcgThreads = 256;

__device__ __forceinline__ int64_t at(int64_t o, int c, int64_t ps) {
  return (int64_t)cell_parity(c) * ps + o * 4 + (c >> 1);
}

// sum of the six face neighbours of cell c of oct i; missing neighbours are
// ghost octs or the zero oct of V (colour-planar, plane stride ps)
__device__ __forceinline__ double nbsum(const double *__restrict__ V, const int32_t *__restrict__ nbr, int64_t n,
                                        int64_t i, int c, int64_t ps) {
  double s = 0.0;
#pragma unroll
  for (int d = 0; d < 6; ++d) {
    const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
    const int64_t o = (((c >> a) & 1) != side) ? i : (int64_t)nbr[(int64_t)d * n + i];
    s += V[at(o, c2, ps)];
  }
  return s;
}

__device__ __forceinline__ void block_partial(double v, double *part) {
  __shared__ double ws[kPcgThreads / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kPcgThreads / 32; ++w) s += ws[w];
    part[blockIdx.x] = s;
  }
}

// r = g + nbsum(phi) / 6 - phi (phi's ghost octs hold the Dirichlet values),
// in place in the right-hand side array g (plane stride 4 n), which holds r
// for the rest of the iteration; partial sums of r^2
__global__ void k_pcg_resid(const int32_t *__restrict__ nbr, const double *__restrict__ phi, double *__restrict__ g,
                            int64_t n, int64_t ps, double *__restrict__ part) {
  double acc = 0.0;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t gi = (int64_t)cell_parity(c) * (n * 4) + i * 4 + (c >> 1);
      const double v = fma(nbsum(phi, nbr, n, i, c, ps), 1.0 / 6.0, g[gi]) - phi[at(i, c, ps)];
      g[gi] = v;
      acc += v * v;
    }
  }
  block_partial(acc, part);
}

// The two direction buffers alternate: sc[8] names the one written this
// iteration.
__device__ __forceinline__ int cur_dir(const double *sc) { return sc[8] != 0.0 ? 1 : 0; }

// p = z + beta p_old (into the other direction buffer) and q = p - nbsum(p) / 6,
// the neighbours' p formed on the fly from z and p_old exactly as their owners
// form it (z and p_old are zero on the ghost and zero octs); partial (p, q)
__global__ void k_pcg_dir_apply(const int32_t *__restrict__ nbr, const double *__restrict__ z, double *P0,
                                double *P1, int64_t n, int64_t ps, const double *__restrict__ sc,
                                double *__restrict__ q, double *__restrict__ part) {
  double acc = 0.0;
  const double b = sc[3];
  const int cur = cur_dir(sc);
  double *__restrict__ pn = cur ? P1 : P0;
  const double *__restrict__ po = cur ? P0 : P1;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t k = at(i, c, ps);
      const double pv = fma(b, po[k], z[k]);
      double s = 0.0;
#pragma unroll
      for (int d = 0; d < 6; ++d) {
        const int a = d >> 1, side = d & 1, c2 = c ^ (1 << a);
        const int64_t o = (((c >> a) & 1) != side) ? i : (int64_t)nbr[(int64_t)d * n + i];
        const int64_t k2 = at(o, c2, ps);
        s += fma(b, po[k2], z[k2]);
      }
      const double v = pv - s * (1.0 / 6.0);
      pn[k] = pv;
      q[k] = v;
      acc += pv * v;
    }
  }
  block_partial(acc, part);
}

// x += alpha p; r -= alpha q (r in the right-hand side array); partial (r, r)
__global__ void k_pcg_step(double *__restrict__ x, const double *P0, const double *P1, double *__restrict__ r,
                           const double *__restrict__ q, int64_t n, int64_t ps, const double *__restrict__ sc,
                           double *__restrict__ part) {
  double acc = 0.0;
  const double a = sc[5];
  const double *__restrict__ p = cur_dir(sc) ? P1 : P0;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t k = at(i, c, ps);
      const int64_t gi = (int64_t)cell_parity(c) * (n * 4) + i * 4 + (c >> 1);
      x[k] += a * p[k];
      const double nv = r[gi] - a * q[k];
      r[gi] = nv;
      acc += nv * nv;
    }
  }
  block_partial(acc, part);
}

// partial (z, r) into part[b], (z, q) into part[nb + b]; q is the previous
// iteration's L0 p, so that r' - r = -alpha q
__global__ void k_pcg_dots(const double *__restrict__ z, const double *__restrict__ r, const double *__restrict__ q,
                           int64_t n, int64_t ps, double *__restrict__ part) {
  double a = 0.0, b = 0.0;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t k = at(i, c, ps);
      const double zv = z[k];
      a += zv * r[(int64_t)cell_parity(c) * (n * 4) + i * 4 + (c >> 1)];
      b += zv * q[k];
    }
  }
  block_partial(a, part);
  __syncthreads();
  block_partial(b, part + gridDim.x);
}

// sum of part[0..np) in a fixed order, on all threads of a one-block launch
__device__ double block_sum(const double *__restrict__ part, int np) {
  __shared__ double ws[32];
  __shared__ double total;
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) v += part[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    total = s;
  }
  __syncthreads();
  const double r = total;
  __syncthreads();
  return r;
}

// Scalars: sc[0] (z, r), sc[1] (z, q), sc[2] (z, r) of the last beta, sc[3]
// beta, sc[4] (p, q), sc[5] alpha, sc[6] (r, r), sc[7] first-iteration flag,
// sc[8] current direction buffer.  The reductions finish into them:
enum { FIN_BETA, FIN_ALPHA, FIN_NORM, FIN_NORM_FIRST };

// beta = (z', r' - r) / (z, r) = -alpha (z', q) / (z, r) (Polak-Ribiere; 0 on
// the first iteration); alpha = (z, r) / (p, q); ||r||^2 to the solve control
// in source units (and, at set-up, the first-iteration flag)
template <int MODE>
__global__ void k_pcg_fin(const double *__restrict__ part, int np, double *sc, double d2f, double *scal2) {
  const double a = block_sum(part, np);
  if (MODE == FIN_BETA) {
    const double b = block_sum(part + np, np);
    if (threadIdx.x == 0) {
      sc[0] = a;
      sc[1] = b;
      sc[3] = sc[7] != 0.0 ? 0.0 : -sc[5] * b / sc[2];
      sc[2] = a;
      sc[7] = 0.0;
      sc[8] = sc[8] != 0.0 ? 0.0 : 1.0;
    }
  } else if (threadIdx.x == 0) {
    if (MODE == FIN_ALPHA) {
      sc[4] = a;
      sc[5] = sc[2] / a;
    } else {
      sc[6] = a;
      *scal2 = a * d2f;
      if (MODE == FIN_NORM_FIRST) {
        sc[7] = 1.0;
        sc[8] = 0.0;
      }
    }
  }
}

// FP32 right-hand side of the mixed-precision preconditioner: r / ||r||
// (||r||^2 in sc[6]), g layout [2][n][4]
__global__ void k_pcg_emit32(const double *__restrict__ r, int64_t n, const double *__restrict__ sc,
                             float *__restrict__ g32) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const double s = sqrt(sc[6]);
  g32[t] = (float)(r[t] * (s > 0.0 ? 1.0 / s : 1.0));
}

// z = ||r|| e in phi (real octs; FP64) from the FP32 correction e
__global__ void k_pcg_z64(const float *__restrict__ e, int64_t n, int64_t ps, const double *__restrict__ sc,
                          double *__restrict__ z) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t >= 8 * n) return;
  const int pl = (int)(t / (4 * n));
  const int64_t k = pl * ps + (t - pl * 4 * n);
  const double s = sqrt(sc[6]);
  z[k] = (s > 0.0 ? s : 1.0) * (double)e[k];
}

struct PcgView {
  double *x, *p0, *p1, *q, *gsave, *part, *sc;
  int64_t n, ps, nv;
  unsigned nb;
};

PcgView view(cmg_level *L) {
  MgLev &g = L->mg[0];
  PcgView v;
  v.n = g.n;
  v.ps = g.n_alloc * 4;
  v.nv = 8 * g.n_alloc;
  v.nb = blocks_for(g.n, kPcgThreads);
  v.x = L->pcg;
  v.p0 = v.x + v.nv;
  v.p1 = v.p0 + v.nv;
  v.q = v.p1 + v.nv;
  v.gsave = v.q + v.nv;
  v.part = v.gsave + v.nv;
  v.sc = v.part + 2 * v.nb;
  return v;
}

double d2f_of(const cmg_level *L) {
  const double h = L->mg[0].h;
  return 36.0 / (h * h * h * h);  // squared pre-scaled norms -> source units
}

constexpr int kFinThreads = 1024;

}  // namespace

void pcg_prepare(cmg_level *L) {
  if (L->pcg) return;
  MgLev &g = L->mg[0];
  const int64_t nv = 8 * g.n_alloc;
  const unsigned nb = blocks_for(g.n, kPcgThreads);
  // x, two direction buffers, q, saved right-hand side; partials; scalars
  // (zeroed, so that q and both directions start finite)
  L->pcg = L->mem.alloc<double>(5 * nv + 2 * (int64_t)nb + 16, true, L->ctx->stream);
  CMG_CUDA(cudaStreamSynchronize(L->ctx->stream));
}

// Set-up (inside the solve graph): ghosts, ||f - L 0||^2 into scal[0], the
// true residual r0 in place of the right-hand side (the first right-hand side
// of the preconditioner) with ||r0||^2 into scal[2], x = phi, p = 0, ghost
// octs of phi cleared.
void pcg_pre(cmg_level *L) {
  MgLev &g = L->mg[0];
  cudaStream_t s = L->ctx->stream;
  const PcgView v = view(L);
  fill_ghosts(L);
  zero_phi_norm(L, L->scal + 0);
  CMG_CUDA(cudaMemcpyAsync(v.gsave, g.g, sizeof(double) * 8 * v.n, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemcpyAsync(v.x, g.phi, sizeof(double) * v.nv, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemsetAsync(v.p0, 0, sizeof(double) * 2 * v.nv, s));
  {
    LaunchScope ls(L->ctx, K_RESID64, 8.0 * v.n * 24.0, 8.0 * v.n * 9.0);
    k_pcg_resid<<<v.nb, kPcgThreads, 0, s>>>(g.nbr, g.phi, g.g, v.n, v.ps, v.part);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, 8.0 * v.nb, v.nb);
    k_pcg_fin<FIN_NORM_FIRST><<<1, kFinThreads, 0, s>>>(v.part, (int)v.nb, v.sc, d2f_of(L), L->scal + 2);
  }
  // corrections see zero coarse-fine values: clear the ghost octs of phi
  if (g.n_alloc > v.n) {
    CMG_CUDA(cudaMemsetAsync(g.phi + 4 * v.n, 0, sizeof(double) * 4 * (g.n_alloc - v.n), s));
    CMG_CUDA(cudaMemsetAsync(g.phi + v.ps + 4 * v.n, 0, sizeof(double) * 4 * (g.n_alloc - v.n), s));
  }
  CMG_CUDA(cudaGetLastError());
}

// One CG iteration: z = M r (V-cycle), beta, p and q = L0 p, alpha, x and r
// updates; ||r||^2 into scal[2] for the control's check.
void pcg_body(cmg_level *L, const cmg_solve_params *p, int64_t *updates) {
  MgLev &g = L->mg[0];
  cudaStream_t s = L->ctx->stream;
  const PcgView v = view(L);
  int64_t upc = 0;
  if (p->precision == CMG_PREC_MIXED) {
    // z = ||r|| e, e = FP32 V-cycles on r / ||r|| (FP32 right-hand side)
    {
      LaunchScope ls(L->ctx, K_CONVERT, 8.0 * v.n * 12.0, 8.0 * v.n);
      k_pcg_emit32<<<blocks_for(8 * v.n), kThreads, 0, s>>>(g.g, v.n, v.sc, g.g32);
    }
    vcycle32_from_zero(L, p, &upc);
    {
      LaunchScope ls(L->ctx, K_CONVERT, 8.0 * v.n * 12.0, 8.0 * v.n);
      k_pcg_z64<<<blocks_for(8 * v.n), kThreads, 0, s>>>(g.phi32, v.n, v.ps, v.sc, g.phi);
    }
  } else {
    vcycle64_from_zero(L, p, &upc);  // z = M r in phi
  }
  *updates += upc;
  if (L->periodic_full) subtract_mean(L);
  {
    LaunchScope ls(L->ctx, K_REDUCE, 8.0 * v.n * 24.0, 8.0 * v.n * 4.0);
    k_pcg_dots<<<v.nb, kPcgThreads, 0, s>>>(g.phi, g.g, v.q, v.n, v.ps, v.part);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, 16.0 * v.nb, 2.0 * v.nb);
    k_pcg_fin<FIN_BETA><<<1, kFinThreads, 0, s>>>(v.part, (int)v.nb, v.sc, 0.0, nullptr);
  }
  {
    LaunchScope ls(L->ctx, K_RESID64, 8.0 * v.n * 32.0 + 24.0 * v.n, 8.0 * v.n * 11.0);
    k_pcg_dir_apply<<<v.nb, kPcgThreads, 0, s>>>(g.nbr, g.phi, v.p0, v.p1, v.n, v.ps, v.sc, v.q, v.part);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, 8.0 * v.nb, v.nb);
    k_pcg_fin<FIN_ALPHA><<<1, kFinThreads, 0, s>>>(v.part, (int)v.nb, v.sc, 0.0, nullptr);
  }
  {
    LaunchScope ls(L->ctx, K_CONVERT, 8.0 * v.n * 48.0, 8.0 * v.n * 6.0);
    k_pcg_step<<<v.nb, kPcgThreads, 0, s>>>(v.x, v.p0, v.p1, g.g, v.q, v.n, v.ps, v.sc, v.part);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, 8.0 * v.nb, v.nb);
    k_pcg_fin<FIN_NORM><<<1, kFinThreads, 0, s>>>(v.part, (int)v.nb, v.sc, d2f_of(L), L->scal + 2);
  }
  CMG_CUDA(cudaGetLastError());
}

// Wrap-up: phi = x, the source restored, the ghosts refilled.
void pcg_post(cmg_level *L) {
  MgLev &g = L->mg[0];
  cudaStream_t s = L->ctx->stream;
  const PcgView v = view(L);
  CMG_CUDA(cudaMemcpyAsync(g.phi, v.x, sizeof(double) * v.nv, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemcpyAsync(g.g, v.gsave, sizeof(double) * 8 * v.n, cudaMemcpyDeviceToDevice, s));
}

}  // namespace cmg
