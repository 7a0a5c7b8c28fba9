// solve.cu -- the level solve: V-cycles (App. G Alg. (vcycle), one GPU, no
// halo exchanges) iterated to a relative residual, in FP64 or as FP32
// V-cycles inside FP64 iterative refinement.
#include <cmath>

#include "cmg_internal.cuh"

namespace cmg {
namespace {

// Coarse phi must start at zero unless the next operation on it overwrites
// it without reading it (first sweep in zero-init mode, or the exact solve).
bool coarse_needs_zero(const cmg_level *L, int m, const cmg_solve_params *p) {
  const int last = (int)L->mg.size() - 1;
  if (m + 1 < last) return p->n_pre == 0;
  return !L->exact_coarse && p->coarse_sweeps == 0;
}

template <typename T>
void vcycle(cmg_level *L, int m, const cmg_solve_params *p, bool zero_top, int64_t *updates) {
  const int last = (int)L->mg.size() - 1;
  const int prec = sizeof(T) == 8 ? CMG_PREC_FP64 : CMG_PREC_MIXED;
  if (m == last) {
    coarse_solve(L, prec, p->coarse_sweeps);
    if (!L->exact_coarse) *updates += (int64_t)p->coarse_sweeps * 8 * L->mg[m].n;
    return;
  }
  for (int k = 0; k < p->n_pre; ++k) sweep<T>(L, m, k == 0 && (m > 0 || zero_top));
  resid_restrict<T>(L, m, true, false, coarse_needs_zero(L, m, p), nullptr);
  vcycle<T>(L, m + 1, p, false, updates);
  prolong<T>(L, m);
  for (int k = 0; k < p->n_post; ++k) sweep<T>(L, m, false);
  *updates += (int64_t)(p->n_pre + p->n_post) * 8 * L->mg[m].n;
}

double read_scalar(cmg_level *L, const double *d) {
  CMG_CUDA(cudaMemcpyAsync(L->ctx->h_dpinned, d, sizeof(double), cudaMemcpyDeviceToHost, L->ctx->stream));
  CMG_CUDA(cudaStreamSynchronize(L->ctx->stream));
  return L->ctx->h_dpinned[0];
}

}  // namespace

int solve(cmg_level *L, const cmg_solve_params *p, cmg_solve_stats *st) {
  if (!p || p->n_pre < 0 || p->n_post < 0 || p->coarse_sweeps < 0 || p->max_cycles < 0 || p->max_cycles > 256 ||
      p->fixed_cycles < 0 || p->fixed_cycles > 256 || !(p->tol >= 0.0) ||
      (p->precision != CMG_PREC_FP64 && p->precision != CMG_PREC_MIXED) ||
      (p->precision == CMG_PREC_MIXED && p->inner_cycles < 1))
    throw Error(CMG_ERR_INVALID_ARG, "invalid solve parameters");
  if (L->periodic_full && L->nx != 1)
    throw Error(CMG_ERR_INVALID_ARG, "periodic base levels need n_x = 1 (exact 2^3 coarsest solve)");
  if (p->precision == CMG_PREC_MIXED && L->mg.size() < 2)
    throw Error(CMG_ERR_INVALID_ARG, "mixed precision needs at least two multigrid levels");
  cmg_solve_stats local;
  cmg_solve_stats &S = st ? *st : local;
  S = cmg_solve_stats{};
  cmg_ctx *ctx = L->ctx;
  cudaStream_t s = ctx->stream;
  double *scal = L->scal;  // [0,1] norm0^2, norm0; [2,3] norm^2, norm; [4] emit scale; [6] mean
  CMG_CUDA(cudaEventRecord(ctx->ev0, s));

  fill_ghosts(L);
  zero_phi_norm(L, scal + 0);
  const double n0sq = read_scalar(L, scal + 0);
  S.norm0 = std::sqrt(n0sq);
  int status = CMG_OK;
  if (n0sq == 0.0) {
    MgLev &g = L->mg[0];
    CMG_CUDA(cudaMemsetAsync(g.phi, 0, sizeof(double) * 4 * g.n, s));
    CMG_CUDA(cudaMemsetAsync(g.phi + 4 * g.n_alloc, 0, sizeof(double) * 4 * g.n, s));
  } else {
    const bool mixed = p->precision == CMG_PREC_MIXED;
    if (mixed) {
      ensure_fp32(L);
      CMG_CUDA(cudaMemcpyAsync(scal + 4, scal + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
      resid_restrict<double>(L, 0, false, true, false, scal + 2, scal + 4);
    } else {
      resid_restrict<double>(L, 0, false, true, false, scal + 2);
    }
    double rel = std::sqrt(read_scalar(L, scal + 2) / n0sq);
    S.rel_initial = rel;
    S.rel_final = rel;
    const int target = p->fixed_cycles > 0 ? p->fixed_cycles : p->max_cycles;
    const double blowup = 1e3 * (S.rel_initial > 1.0 ? S.rel_initial : 1.0);
    bool done = p->fixed_cycles == 0 && rel <= p->tol;
    status = done ? CMG_OK : CMG_ERR_NOT_CONVERGED;
    for (int cyc = 1; cyc <= target && !done; ++cyc) {
      if (!mixed) {
        vcycle<double>(L, 0, p, false, &S.cell_updates);
        resid_restrict<double>(L, 0, false, true, false, scal + 2);
      } else {
        MgLev &g = L->mg[0];
        if (p->n_pre == 0) {
          CMG_CUDA(cudaMemsetAsync(g.phi32, 0, sizeof(float) * 4 * g.n, s));
          CMG_CUDA(cudaMemsetAsync(g.phi32 + 4 * g.n_alloc, 0, sizeof(float) * 4 * g.n, s));
        }
        for (int k = 0; k < p->inner_cycles; ++k) vcycle<float>(L, 0, p, k == 0, &S.cell_updates);
        accumulate(L, scal + 4);
        CMG_CUDA(cudaMemcpyAsync(scal + 4, scal + 3, sizeof(double), cudaMemcpyDeviceToDevice, s));
        resid_restrict<double>(L, 0, false, true, false, scal + 2, scal + 4);
      }
      rel = std::sqrt(read_scalar(L, scal + 2) / n0sq);
      S.cycles = cyc;
      S.rel_history[cyc - 1] = rel;
      S.rel_final = rel;
      if (!std::isfinite(rel) || rel > blowup) {
        status = CMG_ERR_DIVERGED;
        break;
      }
      if (p->fixed_cycles > 0) {
        status = CMG_OK;
      } else if (rel <= p->tol) {
        status = CMG_OK;
        done = true;
      }
    }
    if (L->periodic_full) subtract_mean(L);
  }
  CMG_CUDA(cudaEventRecord(ctx->ev1, s));
  CMG_CUDA(cudaEventSynchronize(ctx->ev1));
  float ms = 0.f;
  CMG_CUDA(cudaEventElapsedTime(&ms, ctx->ev0, ctx->ev1));
  S.ms = ms;
  S.status = status;
  return status;
}

}  // namespace cmg
