// pcg.cu -- multigrid-preconditioned conjugate gradients on one level (the
// paper names multigrid as the preconditioner of a CG solve, App. D.2).
//
// Flexible (Polak-Ribiere) CG, because a V-cycle that smooths red first in
// both legs is not exactly symmetric:
//   r0 = f - L phi0 (true residual, Dirichlet ghosts); z = M r; p = z (first)
//   loop: q = L0 p; alpha = (r, z) / (p, q); phi += alpha p; r' = r - alpha q;
//         stop on ||r'||; z' = M r'; beta = (z', r' - r) / (z, r); p = z' + beta p
// M = one V-cycle from zero with homogeneous coarse-fine values (the level's
// own V-cycle, reading its right-hand side array, which holds r during the
// iteration); L0 = the operator with homogeneous coarse-fine values.  On a
// periodic level z is projected to zero mean (the operator's null space).
// Everything is FP64 and in the solver's pre-scaled units (d = -h^2 r / 6;
// the iteration is invariant to that scale).  Dot products are per-block
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
// written to r (plane stride ps) and to the right-hand side gtop (plane
// stride 4 n); partial sums of r^2
__global__ void k_pcg_resid(const int32_t *__restrict__ nbr, const double *__restrict__ phi,
                            const double *__restrict__ g, int64_t n, int64_t ps, double *__restrict__ r,
                            double *__restrict__ gtop, double *__restrict__ part) {
  double acc = 0.0;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t gi = (int64_t)cell_parity(c) * (n * 4) + i * 4 + (c >> 1);
      const double v = fma(nbsum(phi, nbr, n, i, c, ps), 1.0 / 6.0, g[gi]) - phi[at(i, c, ps)];
      r[at(i, c, ps)] = v;
      gtop[gi] = v;
      acc += v * v;
    }
  }
  block_partial(acc, part);
}

// q = p - nbsum(p) / 6 (p is zero on the ghost and zero octs); partial (p, q)
__global__ void k_pcg_apply(const int32_t *__restrict__ nbr, const double *__restrict__ p, int64_t n, int64_t ps,
                            double *__restrict__ q, double *__restrict__ part) {
  double acc = 0.0;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const double pv = p[at(i, c, ps)];
      const double v = pv - nbsum(p, nbr, n, i, c, ps) * (1.0 / 6.0);
      q[at(i, c, ps)] = v;
      acc += pv * v;
    }
  }
  block_partial(acc, part);
}

// x += alpha p; ro = r; r -= alpha q; gtop = r; partial (r, r)
__global__ void k_pcg_step(double *__restrict__ x, const double *__restrict__ p, double *__restrict__ r,
                           double *__restrict__ ro, const double *__restrict__ q, double *__restrict__ gtop, int64_t n,
                           int64_t ps, const double *__restrict__ alpha, double *__restrict__ part) {
  double acc = 0.0;
  const double a = *alpha;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t k = at(i, c, ps);
      x[k] += a * p[k];
      const double rv = r[k];
      ro[k] = rv;
      const double nv = rv - a * q[k];
      r[k] = nv;
      gtop[(int64_t)cell_parity(c) * (n * 4) + i * 4 + (c >> 1)] = nv;
      acc += nv * nv;
    }
  }
  block_partial(acc, part);
}

// partial (z, r) into part[b], (z, ro) into part[nb + b]
__global__ void k_pcg_dots(const double *__restrict__ z, const double *__restrict__ r, const double *__restrict__ ro,
                           int64_t n, int64_t ps, double *__restrict__ part) {
  double a = 0.0, b = 0.0;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t k = at(i, c, ps);
      a += z[k] * r[k];
      b += z[k] * ro[k];
    }
  }
  block_partial(a, part);
  __syncthreads();
  block_partial(b, part + gridDim.x);
}

// p = z + beta p
__global__ void k_pcg_dir(const double *__restrict__ z, double *__restrict__ p, int64_t n, int64_t ps,
                          const double *__restrict__ beta) {
  const double b = *beta;
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i < n) {
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int64_t k = at(i, c, ps);
      p[k] = z[k] + b * p[k];
    }
  }
}

// out = sum of part[0..np) in a fixed order (one block)
__global__ void k_pcg_reduce(const double *__restrict__ part, int np, double *__restrict__ out) {
  __shared__ double ws[32];
  double v = 0.0;
  for (int t = threadIdx.x; t < np; t += blockDim.x) v += part[t];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += ws[w];
    *out = s;
  }
}

// scalars: sc[0] (z, r), sc[1] (z, ro), sc[2] previous (z, r), sc[3] beta,
// sc[4] (p, q), sc[5] alpha, sc[6] (r, r), sc[7] first-iteration flag
__global__ void k_pcg_beta(double *sc) {
  sc[3] = sc[7] != 0.0 ? 0.0 : (sc[0] - sc[1]) / sc[2];
  sc[2] = sc[0];
  sc[7] = 0.0;
}
__global__ void k_pcg_alpha(double *sc) { sc[5] = sc[2] / sc[4]; }
// the solve control reads ||r||^2 in source units from scal[2]
__global__ void k_pcg_norm_out(double *sc, double d2f, double *scal2) {
  *scal2 = sc[6] * d2f;
}
__global__ void k_pcg_first(double *sc) { sc[7] = 1.0; }

struct PcgView {
  double *x, *r, *ro, *pd, *q, *gsave, *part, *sc;
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
  v.r = v.x + v.nv;
  v.ro = v.r + v.nv;
  v.pd = v.ro + v.nv;
  v.q = v.pd + v.nv;
  v.gsave = v.q + v.nv;
  v.part = v.gsave + v.nv;
  v.sc = v.part + 2 * v.nb;
  return v;
}

double d2f_of(const cmg_level *L) {
  const double h = L->mg[0].h;
  return 36.0 / (h * h * h * h);  // squared pre-scaled norms -> source units
}

}  // namespace

void pcg_prepare(cmg_level *L) {
  if (L->pcg) return;
  MgLev &g = L->mg[0];
  const int64_t nv = 8 * g.n_alloc;
  const unsigned nb = blocks_for(g.n, kPcgThreads);
  // x, r, ro, p, q, saved right-hand side; partials; scalars
  L->pcg = L->mem.alloc<double>(6 * nv + 2 * (int64_t)nb + 16, true, L->ctx->stream);
  CMG_CUDA(cudaStreamSynchronize(L->ctx->stream));
}

// Set-up (inside the solve graph): ghosts, ||f - L 0||^2 into scal[0], the
// true residual r0 (also the first right-hand side of the preconditioner)
// with ||r0||^2 into scal[2], x = phi, p = 0, ghost octs of phi cleared.
void pcg_pre(cmg_level *L) {
  MgLev &g = L->mg[0];
  cudaStream_t s = L->ctx->stream;
  const PcgView v = view(L);
  fill_ghosts(L);
  zero_phi_norm(L, L->scal + 0);
  CMG_CUDA(cudaMemcpyAsync(v.gsave, g.g, sizeof(double) * 8 * v.n, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemcpyAsync(v.x, g.phi, sizeof(double) * v.nv, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemsetAsync(v.pd, 0, sizeof(double) * v.nv, s));
  {
    LaunchScope ls(L->ctx, K_RESID64, 8.0 * v.n * 24.0, 8.0 * v.n * 9.0);
    k_pcg_resid<<<v.nb, kPcgThreads, 0, s>>>(g.nbr, g.phi, g.g, v.n, v.ps, v.r, g.g, v.part);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, 8.0 * v.nb, v.nb);
    k_pcg_reduce<<<1, 1024, 0, s>>>(v.part, (int)v.nb, v.sc + 6);
  }
  k_pcg_norm_out<<<1, 1, 0, s>>>(v.sc, d2f_of(L), L->scal + 2);
  k_pcg_first<<<1, 1, 0, s>>>(v.sc);
  // corrections see zero coarse-fine values: clear the ghost octs of phi
  if (g.n_alloc > v.n) {
    CMG_CUDA(cudaMemsetAsync(g.phi + 4 * v.n, 0, sizeof(double) * 4 * (g.n_alloc - v.n), s));
    CMG_CUDA(cudaMemsetAsync(g.phi + v.ps + 4 * v.n, 0, sizeof(double) * 4 * (g.n_alloc - v.n), s));
  }
  CMG_CUDA(cudaGetLastError());
}

// One CG iteration: z = M r (V-cycle), beta, p, q = L0 p, alpha, x and r
// updates; ||r||^2 into scal[2] for the control's check.
void pcg_body(cmg_level *L, const cmg_solve_params *p, int64_t *updates) {
  MgLev &g = L->mg[0];
  cudaStream_t s = L->ctx->stream;
  const PcgView v = view(L);
  int64_t upc = 0;
  vcycle64_from_zero(L, p, &upc);  // z = M r in phi
  *updates += upc;
  if (L->periodic_full) subtract_mean(L);
  {
    LaunchScope ls(L->ctx, K_REDUCE, 8.0 * v.n * 24.0, 8.0 * v.n * 4.0);
    k_pcg_dots<<<v.nb, kPcgThreads, 0, s>>>(g.phi, v.r, v.ro, v.n, v.ps, v.part);
  }
  k_pcg_reduce<<<1, 1024, 0, s>>>(v.part, (int)v.nb, v.sc + 0);
  k_pcg_reduce<<<1, 1024, 0, s>>>(v.part + v.nb, (int)v.nb, v.sc + 1);
  k_pcg_beta<<<1, 1, 0, s>>>(v.sc);
  {
    LaunchScope ls(L->ctx, K_CONVERT, 8.0 * v.n * 24.0, 8.0 * v.n * 2.0);
    k_pcg_dir<<<v.nb, kPcgThreads, 0, s>>>(g.phi, v.pd, v.n, v.ps, v.sc + 3);
  }
  {
    LaunchScope ls(L->ctx, K_RESID64, 8.0 * v.n * 16.0, 8.0 * v.n * 9.0);
    k_pcg_apply<<<v.nb, kPcgThreads, 0, s>>>(g.nbr, v.pd, v.n, v.ps, v.q, v.part);
  }
  k_pcg_reduce<<<1, 1024, 0, s>>>(v.part, (int)v.nb, v.sc + 4);
  k_pcg_alpha<<<1, 1, 0, s>>>(v.sc);
  {
    LaunchScope ls(L->ctx, K_CONVERT, 8.0 * v.n * 56.0, 8.0 * v.n * 6.0);
    k_pcg_step<<<v.nb, kPcgThreads, 0, s>>>(v.x, v.pd, v.r, v.ro, v.q, g.g, v.n, v.ps, v.sc + 5, v.part);
  }
  k_pcg_reduce<<<1, 1024, 0, s>>>(v.part, (int)v.nb, v.sc + 6);
  k_pcg_norm_out<<<1, 1, 0, s>>>(v.sc, d2f_of(L), L->scal + 2);
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
