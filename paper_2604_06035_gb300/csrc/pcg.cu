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
// partial sums reduced in a fixed order (deterministic).  One host
// synchronisation per iteration reads the residual norm for the stop test.
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
// sc[4] (p, q), sc[5] alpha, sc[6] (r, r)
__global__ void k_pcg_beta(double *sc, int first) {
  sc[3] = first ? 0.0 : (sc[0] - sc[1]) / sc[2];
  sc[2] = sc[0];
}
__global__ void k_pcg_alpha(double *sc) { sc[5] = sc[2] / sc[4]; }

}  // namespace

void pcg_solve(cmg_level *L, const cmg_solve_params *p, cmg_solve_stats &S) {
  MgLev &g = L->mg[0];
  cmg_ctx *ctx = L->ctx;
  cudaStream_t s = ctx->stream;
  const int64_t n = g.n, ps = g.n_alloc * 4, nv = 8 * g.n_alloc;
  const unsigned nb = blocks_for(n, kPcgThreads);
  if (!L->pcg) {
    // x, r, ro, p, q, saved right-hand side; partials; scalars
    L->pcg = L->mem.alloc<double>(6 * nv + 2 * (int64_t)nb + 16, true, s);
  }
  double *x = L->pcg, *r = x + nv, *ro = r + nv, *pd = ro + nv, *q = pd + nv, *gsave = q + nv;
  double *part = gsave + nv, *sc = part + 2 * nb;
  const double h = g.h, d2f = 36.0 / (h * h * h * h);  // squared d-unit norms -> source units
  CMG_CUDA(cudaEventRecord(ctx->ev0, s));
  fill_ghosts(L);
  zero_phi_norm(L, L->scal + 0);  // ||f - L 0||^2 (source units) and its root
  CMG_CUDA(cudaMemcpyAsync(gsave, g.g, sizeof(double) * 8 * n, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemcpyAsync(x, g.phi, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
  CMG_CUDA(cudaMemsetAsync(pd, 0, sizeof(double) * nv, s));
  {
    LaunchScope ls(ctx, K_RESID64, 8.0 * n * 24.0, 8.0 * n * 9.0);
    k_pcg_resid<<<nb, kPcgThreads, 0, s>>>(g.nbr, g.phi, g.g, n, ps, r, g.g, part);
  }
  k_pcg_reduce<<<1, 1024, 0, s>>>(part, (int)nb, sc + 6);
  // corrections see zero coarse-fine values: clear the ghost octs of phi
  if (g.n_alloc > n) {
    CMG_CUDA(cudaMemsetAsync(g.phi + 4 * n, 0, sizeof(double) * 4 * (g.n_alloc - n), s));
    CMG_CUDA(cudaMemsetAsync(g.phi + ps + 4 * n, 0, sizeof(double) * 4 * (g.n_alloc - n), s));
  }
  CMG_CUDA(cudaGetLastError());
  double *h_pin = ctx->h_dpinned;
  CMG_CUDA(cudaMemcpyAsync(h_pin, L->scal, sizeof(double), cudaMemcpyDeviceToHost, s));
  CMG_CUDA(cudaMemcpyAsync(h_pin + 1, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
  CMG_CUDA(cudaStreamSynchronize(s));
  const double n0 = h_pin[0];
  S.norm0 = std::sqrt(n0);
  S.status = CMG_OK;
  int cycles = 0;
  int64_t updates = 0, upc = 0;
  if (n0 > 0.0) {
    double rel = std::sqrt(h_pin[1] * d2f / n0);
    S.rel_initial = rel;
    S.rel_final = rel;
    const int target = p->fixed_cycles > 0 ? p->fixed_cycles : p->max_cycles;
    if (!(p->fixed_cycles == 0 && rel <= p->tol)) {
      S.status = p->fixed_cycles > 0 ? CMG_OK : CMG_ERR_NOT_CONVERGED;
      for (int it = 1; it <= target; ++it) {
        upc = 0;
        vcycle64_from_zero(L, p, &upc);  // z = M r in phi
        updates += upc;
        if (L->periodic_full) subtract_mean(L);
        k_pcg_dots<<<nb, kPcgThreads, 0, s>>>(g.phi, r, ro, n, ps, part);
        k_pcg_reduce<<<1, 1024, 0, s>>>(part, (int)nb, sc + 0);
        k_pcg_reduce<<<1, 1024, 0, s>>>(part + nb, (int)nb, sc + 1);
        k_pcg_beta<<<1, 1, 0, s>>>(sc, it == 1);
        k_pcg_dir<<<nb, kPcgThreads, 0, s>>>(g.phi, pd, n, ps, sc + 3);
        {
          LaunchScope ls(ctx, K_RESID64, 8.0 * n * 16.0, 8.0 * n * 9.0);
          k_pcg_apply<<<nb, kPcgThreads, 0, s>>>(g.nbr, pd, n, ps, q, part);
        }
        k_pcg_reduce<<<1, 1024, 0, s>>>(part, (int)nb, sc + 4);
        k_pcg_alpha<<<1, 1, 0, s>>>(sc);
        k_pcg_step<<<nb, kPcgThreads, 0, s>>>(x, pd, r, ro, q, g.g, n, ps, sc + 5, part);
        k_pcg_reduce<<<1, 1024, 0, s>>>(part, (int)nb, sc + 6);
        CMG_CUDA(cudaGetLastError());
        CMG_CUDA(cudaMemcpyAsync(h_pin, sc + 6, sizeof(double), cudaMemcpyDeviceToHost, s));
        CMG_CUDA(cudaStreamSynchronize(s));
        rel = std::sqrt(h_pin[0] * d2f / n0);
        cycles = it;
        if (it <= 256) S.rel_history[it - 1] = rel;
        S.rel_final = rel;
        if (!std::isfinite(rel) || rel > 1e3 * std::max(S.rel_initial, 1.0)) {
          S.status = CMG_ERR_DIVERGED;
          break;
        }
        if (p->fixed_cycles == 0 && rel <= p->tol) {
          S.status = CMG_OK;
          break;
        }
      }
    }
    CMG_CUDA(cudaMemcpyAsync(g.phi, x, sizeof(double) * nv, cudaMemcpyDeviceToDevice, s));
    if (L->periodic_full) subtract_mean(L);
  } else {
    CMG_CUDA(cudaMemsetAsync(g.phi, 0, sizeof(double) * 4 * n, s));
    CMG_CUDA(cudaMemsetAsync(g.phi + ps, 0, sizeof(double) * 4 * n, s));
    S.rel_initial = S.rel_final = 0.0;
  }
  CMG_CUDA(cudaMemcpyAsync(g.g, gsave, sizeof(double) * 8 * n, cudaMemcpyDeviceToDevice, s));
  fill_ghosts(L);
  CMG_CUDA(cudaEventRecord(ctx->ev1, s));
  CMG_CUDA(cudaEventSynchronize(ctx->ev1));
  float ms = 0.f;
  CMG_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  S.ms = ms;
  S.cycles = cycles;
  S.cell_updates = updates;
}

}  // namespace cmg
