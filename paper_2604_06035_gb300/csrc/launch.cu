// launch.cu -- host launchers of the one-operation-per-launch kernels
// (kernels.cuh), with the algorithmic work each launch reports to the
// profiler.
#include <cmath>

#include "cmg_internal.cuh"
#include "kernels.cuh"

namespace cmg {

// ------------------------------------------------------------ launchers
// Algorithmic work per launch (for the profile): bytes are the minimum
// traffic of the operation with perfect reuse, flops its floating-point
// operations (FMA = 2).  The neighbour cache counts 24 B per oct per full
// red-black sweep (6 int32; 12 B per colour pass) and 24 B per oct per
// residual evaluation.

template <typename T>
void sweep(cmg_level *L, int m, bool zero_init) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  T *phi = phi_of<T>(g);
  T *gg = g_of<T>(g);
  const int64_t st = g.n_alloc * 4;
  const unsigned nb = blocks_for(g.n);
  const bool mask = !g.all_active;
  const int cls = sizeof(T) == 8 ? K_SWEEP64 : K_SWEEP32;
  const double u = 4.0 * (double)g.n;  // cells updated per colour pass
  const double nbr_bytes = 12.0 * (double)g.n;
  const double full_bytes = 3.0 * u * sizeof(T) + nbr_bytes, full_flops = 7.0 * u;
  const bool pre = kPreloadIdx<T> && g.n <= kPreloadSweepOcts;
#define CMG_SWEEP(P, Z, M)                                                                                  \
  do {                                                                                                      \
    LaunchScope ls(L->ctx, cls, (Z) ? 2.0 * u * sizeof(T) + nbr_bytes : full_bytes, (Z) ? 0.0 : full_flops); \
    if (pre)                                                                                                \
      launch_k(k_sweep<T, P, Z, M, kPreloadIdx<T>>, nb, kThreads, s, g.nbr, phi + (1 - P) * st, phi + P * st, \
               gg + P * g.n * 4, g.active, g.n);                                                            \
    else                                                                                                    \
      launch_k(k_sweep<T, P, Z, M, false>, nb, kThreads, s, g.nbr, phi + (1 - P) * st, phi + P * st,        \
               gg + P * g.n * 4, g.active, g.n);                                                            \
  } while (0)
  // full periodic levels in lexicographic order: the shared-memory brick
  // kernel (brick.cu), same results bit for bit; by default for FP32 passes
  // only (512^3: FP32 0.185 -> 0.158 ms, FP64 0.422 -> 0.439 ms)
  const bool brick = L->staged >= (sizeof(T) == 4 ? 1 : 2) && g.lex_log2 >= 4 && !mask;
  if (mask) {
    if (zero_init) CMG_SWEEP(0, true, true); else CMG_SWEEP(0, false, true);
    CMG_SWEEP(1, false, true);
  } else {
    if (zero_init) CMG_SWEEP(0, true, false);
    else if (brick) brick_pass<T>(L, m, 0);
    else CMG_SWEEP(0, false, false);
    if (brick) brick_pass<T>(L, m, 1); else CMG_SWEEP(1, false, false);
  }
#undef CMG_SWEEP
  CMG_CUDA(cudaGetLastError());
}
template void sweep<double>(cmg_level *, int, bool);
template void sweep<float>(cmg_level *, int, bool);

template <typename T>
void resid_restrict(cmg_level *L, int m, bool restrict_to_coarse, bool norm, bool zero_coarse_phi, double *norm_out,
                    const double *emit_scale, bool c1_swept, bool finalize) {
  MgLev &g = L->mg[m];
  cudaStream_t s = L->ctx->stream;
  const unsigned nb = blocks_for(g.n);
  MgLev *c = restrict_to_coarse ? &L->mg[m + 1] : nullptr;
  T *cg = c ? g_of<T>(*c) : nullptr;
  T *cphi = c ? phi_of<T>(*c) : nullptr;
  const int64_t cn = c ? c->n : 0, cna = c ? c->n_alloc : 0;
  const uint8_t *act = g.all_active ? nullptr : g.active;
  const double cells = 8.0 * (double)g.n;
  const double bytes = cells * 2.0 * sizeof(T) + 24.0 * g.n + (restrict_to_coarse ? g.n * sizeof(T) : 0.0) +
                       (emit_scale ? cells * 4.0 : 0.0);
  const double flops = cells * (c1_swept ? 0.5 : 1.0) * (8.0 + (norm ? 2.0 : 0.0)) + (restrict_to_coarse ? cells : 0.0);
  const int cls = sizeof(T) == 8 ? K_RESID64 : K_RESID32;
  if (g.n > 0) {
    LaunchScope ls(L->ctx, cls, bytes, flops);
    if (restrict_to_coarse && !norm && !emit_scale && c1_swept)
      launch_k(k_resid<T, false, true, false, false, false, true>, nb, kThreads, s,
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, g.father, cg, cphi, cn, cna, zero_coarse_phi,
          nullptr, nullptr, nullptr, nullptr, 0.0);
    else if (!restrict_to_coarse && norm && !emit_scale && c1_swept)
      launch_k(k_resid<T, true, false, false, false, false, true>, nb, kThreads, s,
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L->partials,
          nullptr, nullptr, nullptr, 0.0);
    else if (c1_swept)
      throw Error(CMG_ERR_INVALID_ARG, "unsupported residual variant");
    else if (restrict_to_coarse && !norm && !emit_scale)
      launch_k(k_resid<T, false, true, false, false, false>, nb, kThreads, s,
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, g.father, cg, cphi, cn, cna, zero_coarse_phi,
          nullptr, nullptr, nullptr, nullptr, 0.0);
    else if (restrict_to_coarse && norm && !emit_scale)
      launch_k(k_resid<T, true, true, false, false, false>, nb, kThreads, s, 
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, g.father, cg, cphi, cn, cna, zero_coarse_phi,
          L->partials, nullptr, nullptr, nullptr, 0.0);
    else if (!restrict_to_coarse && norm && !emit_scale)
      launch_k(k_resid<T, true, false, false, false, false>, nb, kThreads, s, 
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L->partials,
          nullptr, nullptr, nullptr, 0.0);
    else if (!restrict_to_coarse && norm && emit_scale)
      launch_k(k_resid<T, true, false, true, false, false>, nb, kThreads, s, 
          g.nbr, phi_of<T>(g), g_of<T>(g), act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L->partials,
          g.g32, emit_scale, nullptr, 0.0);
    else
      throw Error(CMG_ERR_INVALID_ARG, "unsupported residual variant");
    CMG_CUDA(cudaGetLastError());
  }
  if (norm && finalize) {
    const double scale = 36.0 / (g.h * g.h * g.h * g.h);
    if (g.n == 0) {
      CMG_CUDA(cudaMemsetAsync(norm_out, 0, 2 * sizeof(double), s));
    } else {
      LaunchScope ls(L->ctx, K_REDUCE, nb * 8.0, nb);
      launch_k(k_finalize, 1, 1024, s, L->partials, (int)nb, scale, norm_out, 1);
      CMG_CUDA(cudaGetLastError());
    }
  }
}
template void resid_restrict<double>(cmg_level *, int, bool, bool, bool, double *, const double *, bool, bool);
template void resid_restrict<float>(cmg_level *, int, bool, bool, bool, double *, const double *, bool, bool);

void residual_out(cmg_level *L, int m, int prec, double *out) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const uint8_t *act = g.all_active ? nullptr : g.active;
  const double rscale = -6.0 / (g.h * g.h);
  LaunchScope ls(L->ctx, prec == CMG_PREC_FP64 ? K_RESID64 : K_RESID32, 8.0 * g.n * 24.0, 8.0 * g.n * 9.0);
  if (prec == CMG_PREC_FP64)
    launch_k(k_resid<double, false, false, false, true, false>, blocks_for(g.n), kThreads, s, 
        g.nbr, g.phi, g.g, act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr, out,
        rscale);
  else
    launch_k(k_resid<float, false, false, false, true, false>, blocks_for(g.n), kThreads, s, 
        g.nbr, g.phi32, g.g32, act, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, nullptr, nullptr, nullptr,
        out, rscale);
  CMG_CUDA(cudaGetLastError());
}

// ||f - L 0||^2 at level 0 (ghost forcing included) -> out[0], sqrt -> out[1]
void zero_phi_norm(cmg_level *L, double *out) {
  MgLev &g = L->mg[0];
  cudaStream_t s = L->ctx->stream;
  const unsigned nb = blocks_for(g.n);
  if (g.n == 0) {
    CMG_CUDA(cudaMemsetAsync(out, 0, 2 * sizeof(double), s));
    return;
  }
  {
    LaunchScope ls(L->ctx, K_RESID64, 8.0 * g.n * 8.0, 8.0 * g.n * 9.0);
    launch_k(k_resid<double, true, false, false, false, true>, nb, kThreads, s, 
        g.nbr, g.phi, g.g, nullptr, g.n, g.n_alloc, nullptr, nullptr, nullptr, 0, 0, 0, L->partials, nullptr,
        nullptr, nullptr, 0.0);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, nb * 8.0, nb);
    launch_k(k_finalize, 1, 1024, s, L->partials, (int)nb, 36.0 / (g.h * g.h * g.h * g.h), out, 1);
  }
  CMG_CUDA(cudaGetLastError());
}

template <typename T>
void prolong(cmg_level *L, int m, bool c0_dead) {
  MgLev &g = L->mg[m];
  MgLev &c = L->mg[m + 1];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  LaunchScope ls(L->ctx, sizeof(T) == 8 ? K_PROLONG64 : K_PROLONG32,
                 g.n * (c0_dead ? 9.0 : 17.0) * sizeof(T), g.n * (c0_dead ? 64.0 : 128.0));
  const unsigned nb = blocks_for(g.n);
  if (g.all_active && c0_dead)
    launch_k(k_prolong<T, false, true>, nb, kThreads, s, g.keys, g.blk, g.n, g.n_alloc, phi_of<T>(g), g.active,
             phi_of<T>(c), c.n_alloc);
  else if (g.all_active)
    launch_k(k_prolong<T, false, false>, nb, kThreads, s, g.keys, g.blk, g.n, g.n_alloc, phi_of<T>(g), g.active,
             phi_of<T>(c), c.n_alloc);
  else if (c0_dead)
    launch_k(k_prolong<T, true, true>, nb, kThreads, s, g.keys, g.blk, g.n, g.n_alloc, phi_of<T>(g), g.active,
             phi_of<T>(c), c.n_alloc);
  else
    launch_k(k_prolong<T, true, false>, nb, kThreads, s, g.keys, g.blk, g.n, g.n_alloc, phi_of<T>(g), g.active,
             phi_of<T>(c), c.n_alloc);
  CMG_CUDA(cudaGetLastError());
}
template void prolong<double>(cmg_level *, int, bool);
template void prolong<float>(cmg_level *, int, bool);

void fill_ghosts(cmg_level *L) {
  MgLev &g = L->mg[0];
  if (!L->parent || g.n_ghost == 0) return;
  MgLev &pg = L->parent->mg[0];
  LaunchScope ls(L->ctx, K_GHOST, g.n_ghost * (64.0 + 8.0 + 32.0 + 4.0), g.n_ghost * 120.0);
  k_ghost_fill<<<blocks_for(g.n_ghost), kThreads, 0, L->ctx->stream>>>(
      L->ghost_keys, L->ghost_blk, L->ghost_mask, g.n_ghost, g.n, g.n_alloc, g.phi, pg.phi, pg.n_alloc);
  CMG_CUDA(cudaGetLastError());
}

void get_ghosts(cmg_level *L, double *out) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 24.0 * 8.0, 0.0);
  k_get_ghosts<<<blocks_for(g.n), kThreads, 0, L->ctx->stream>>>(g.nbr, g.n, g.n_ghost, g.n_alloc, g.phi, out);
  CMG_CUDA(cudaGetLastError());
}

void coarse_solve(cmg_level *L, int prec, int coarse_sweeps) {
  const int m = (int)L->mg.size() - 1;
  MgLev &g = L->mg[m];
  cudaStream_t s = L->ctx->stream;
  if (L->exact_coarse) {
    LaunchScope ls(L->ctx, K_COARSE, 128.0, 256.0);
    if (prec == CMG_PREC_FP64)
      launch_k(k_wht<double>, 1, 32, s, g.g, g.phi, g.n_alloc, g.h);
    else
      launch_k(k_wht<float>, 1, 32, s, g.g32, g.phi32, g.n_alloc, g.h);
    CMG_CUDA(cudaGetLastError());
    return;
  }
  if (prec == CMG_PREC_FP64) {
    for (int k = 0; k < coarse_sweeps; ++k) sweep<double>(L, m, k == 0 && m > 0);
    return;
  }
  // mixed: the coarsest level is solved in FP64 on FP64 copies
  const int64_t mg = 8 * g.n, ma = 8 * g.n_alloc;
  {
    LaunchScope ls(L->ctx, K_CONVERT, 12.0 * (mg + ma), 0.0);
    launch_k(k_copy_convert_f2d, blocks_for(mg), kThreads, s, g.g32, g.g, mg);
  }
  {
    LaunchScope ls(L->ctx, K_CONVERT, 12.0 * ma, 0.0);
    launch_k(k_copy_convert_f2d, blocks_for(ma), kThreads, s, g.phi32, g.phi, ma);
  }
  CMG_CUDA(cudaGetLastError());
  for (int k = 0; k < coarse_sweeps; ++k) sweep<double>(L, m, k == 0 && m > 0);
  {
    LaunchScope ls(L->ctx, K_CONVERT, 12.0 * ma, 0.0);
    launch_k(k_copy_convert_d2f, blocks_for(ma), kThreads, s, g.phi, g.phi32, ma);
  }
  CMG_CUDA(cudaGetLastError());
}

void subtract_mean(cmg_level *L) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const unsigned nb = blocks_for(g.n);
  {
    LaunchScope ls(L->ctx, K_REDUCE, 64.0 * g.n, 8.0 * g.n);
    launch_k(k_sum_phi, nb, kThreads, s, g.phi, g.n, g.n_alloc, L->partials);
  }
  {
    LaunchScope ls(L->ctx, K_REDUCE, nb * 8.0, nb);
    launch_k(k_finalize, 1, 1024, s, L->partials, (int)nb, 1.0 / (8.0 * (double)g.n), L->scal + 6, 0);
  }
  {
    LaunchScope ls(L->ctx, K_CONVERT, 128.0 * g.n, 8.0 * g.n);
    launch_k(k_sub_scalar, blocks_for(8 * g.n), kThreads, s, g.phi, g.n, g.n_alloc, L->scal + 6);
  }
  CMG_CUDA(cudaGetLastError());
}

void accumulate(cmg_level *L, const double *scale) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * (16.0 + 4.0), g.n * 16.0);
  launch_k(k_accumulate, blocks_for(2 * g.n), kThreads, L->ctx->stream, g.phi, g.phi32, g.n, g.n_alloc, scale);
  CMG_CUDA(cudaGetLastError());
}

void set_density(cmg_level *L, const double *rho, double rho_bar, double four_pi_g) {
  MgLev &g = L->mg[0];
  if (g.n == 0) return;
  const double scale = -g.h * g.h / 6.0 * four_pi_g;
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * 16.0, g.n * 16.0);
  k_set_density<<<blocks_for(8 * g.n), kThreads, 0, L->ctx->stream>>>(rho, g.n, rho_bar, scale, g.g);
  CMG_CUDA(cudaGetLastError());
}

void ensure_fp32(cmg_level *L) {
  if (L->has32) return;
  for (auto &g : L->mg) {
    g.phi32 = L->mem.alloc<float>(8 * g.n_alloc, true, L->ctx->stream);
    g.g32 = L->mem.alloc<float>(8 * g.n, true, L->ctx->stream);
  }
  L->has32 = true;
}

// field 0 = phi, 1 = f (stored as g = -h^2 f / 6)
void pack_field(cmg_level *L, int m, int field, int prec, const void *in) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const double scale = field == 0 ? 1.0 : -g.h * g.h / 6.0;
  const int64_t stride = field == 0 ? g.n_alloc : g.n;
  const unsigned nb = blocks_for(8 * g.n);
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * 2.0 * (prec == CMG_PREC_FP64 ? 8.0 : 4.0), 0.0);
  if (prec == CMG_PREC_FP64)
    launch_k(k_pack<double, double>, nb, kThreads, s, (const double *)in, g.n, stride, scale, field == 0 ? g.phi : g.g);
  else
    launch_k(k_pack<float, float>, nb, kThreads, s, (const float *)in, g.n, stride, scale, field == 0 ? g.phi32 : g.g32);
  CMG_CUDA(cudaGetLastError());
}

void unpack_field(cmg_level *L, int m, int field, int prec, void *out) {
  MgLev &g = L->mg[m];
  if (g.n == 0) return;
  cudaStream_t s = L->ctx->stream;
  const double scale = field == 0 ? 1.0 : -6.0 / (g.h * g.h);
  const int64_t stride = field == 0 ? g.n_alloc : g.n;
  const unsigned nb = blocks_for(8 * g.n);
  LaunchScope ls(L->ctx, K_CONVERT, g.n * 8.0 * 2.0 * (prec == CMG_PREC_FP64 ? 8.0 : 4.0), 0.0);
  if (prec == CMG_PREC_FP64)
    launch_k(k_unpack<double, double>, nb, kThreads, s, field == 0 ? g.phi : g.g, g.n, stride, scale, (double *)out);
  else
    launch_k(k_unpack<float, float>, nb, kThreads, s, field == 0 ? g.phi32 : g.g32, g.n, stride, scale, (float *)out);
  CMG_CUDA(cudaGetLastError());
}

// The stencil's neighbour sums applied to given rows of six values: out[i] =
// the sum the kernels form for a cell whose neighbours (-x, +x, -y, +y, -z,
// +z) hold rows[i][0..5] -- in colour passes and colour-1 residuals (which =
// 0) or in colour-0 residuals (which = 1) -- for checking that arithmetic on
// its own.
template <int WHICH>
__global__ void k_neighbour_sum(const double *__restrict__ rows, int64_t n, double *__restrict__ out) {
  const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v[6];
#pragma unroll
  for (int d = 0; d < 6; ++d) v[d] = rows[i * 6 + d];
  out[i] = WHICH == 0 ? dev::nbsum6(v) : dev::nbsum6_r0(v);
}

void neighbour_sum(const double *rows, int64_t n, int which, double *out, cudaStream_t s) {
  if (n == 0) return;
  if (which == 0)
    k_neighbour_sum<0><<<blocks_for(n), kThreads, 0, s>>>(rows, n, out);
  else
    k_neighbour_sum<1><<<blocks_for(n), kThreads, 0, s>>>(rows, n, out);
  CMG_CUDA(cudaGetLastError());
}

}  // namespace cmg
