// profile.cu -- launch counting and per-kernel-family CUDA-event timing on
// the context's stream (the benchmark's roofline numbers come from here).
#include <cstdio>

#include "cmg_internal.cuh"

namespace cmg {

namespace {
constexpr int kPoolPairs = 4096;
const char *kNames[K_NCLASS] = {"rbgs_fp64",    "rbgs_fp32",    "residual_fp64", "residual_fp32",
                                "prolong_fp64", "prolong_fp32", "ghost_fill",    "coarse_solve",
                                "reduce",       "convert",      "conv_fwd",      "conv_dgrad",
                                "conv_wgrad",   "fft_fp32"};
}  // namespace

const char *kernel_class_name(int cls) { return cls >= 0 && cls < K_NCLASS ? kNames[cls] : "?"; }

void harvest_profile(cmg_ctx *ctx) {
  if (ctx->pending.empty()) return;
  CMG_CUDA(cudaEventSynchronize(ctx->ev_pool[2 * ctx->pending.back().slot + 1]));
  for (const PendingEvent &p : ctx->pending) {
    float ms = 0.f;
    CMG_CUDA(cudaEventElapsedTime(&ms, ctx->ev_pool[2 * p.slot], ctx->ev_pool[2 * p.slot + 1]));
    ctx->prof[p.cls].ms += ms;
  }
  ctx->pending.clear();
}

LaunchScope::LaunchScope(cmg_ctx *c, int cls, double bytes, double flops) : ctx(c) {
  if (ctx->capturing) {  // counted per replay by the solver
    ctx->captured += 1;
    return;
  }
  ctx->launches += 1;
  if (!ctx->profiling) return;
  if (ctx->ev_pool.empty()) {
    ctx->ev_pool.resize(2 * kPoolPairs);
    for (auto &e : ctx->ev_pool) CMG_CUDA(cudaEventCreate(&e));
  }
  if ((int)ctx->pending.size() == kPoolPairs) harvest_profile(ctx);
  slot = (int)ctx->pending.size();
  ctx->pending.push_back({cls, slot});
  ctx->prof[cls].launches += 1;
  ctx->prof[cls].bytes += bytes;
  ctx->prof[cls].flops += flops;
  CMG_CUDA(cudaEventRecord(ctx->ev_pool[2 * slot], ctx->stream));
}

LaunchScope::~LaunchScope() {
  if (slot >= 0) cudaEventRecord(ctx->ev_pool[2 * slot + 1], ctx->stream);
}

}  // namespace cmg

extern "C" {

int cmg_ctx_set_profiling(cmg_ctx *ctx, int enable) {
  if (!ctx) return CMG_ERR_INVALID_ARG;
  ctx->profiling = enable != 0;
  return CMG_OK;
}

int cmg_ctx_get_profile(cmg_ctx *ctx, cmg_kernel_profile *out, int max_entries, int *n_entries) {
  if (!ctx || (max_entries > 0 && !out) || max_entries < 0) return CMG_ERR_INVALID_ARG;
  try {
    cudaSetDevice(ctx->device);
    cmg::harvest_profile(ctx);
  } catch (const cmg::Error &e) {
    return e.code;
  }
  int k = 0;
  for (int c = 0; c < cmg::K_NCLASS && k < max_entries; ++c) {
    if (ctx->prof[c].launches == 0) continue;
    cmg_kernel_profile &o = out[k++];
    std::snprintf(o.name, sizeof(o.name), "%s", cmg::kernel_class_name(c));
    o.launches = ctx->prof[c].launches;
    o.ms = ctx->prof[c].ms;
    o.bytes = ctx->prof[c].bytes;
    o.flops = ctx->prof[c].flops;
  }
  if (n_entries) *n_entries = k;
  return CMG_OK;
}

int cmg_ctx_reset_profile(cmg_ctx *ctx) {
  if (!ctx) return CMG_ERR_INVALID_ARG;
  try {
    cudaSetDevice(ctx->device);
    cmg::harvest_profile(ctx);
  } catch (const cmg::Error &e) {
    return e.code;
  }
  for (auto &p : ctx->prof) p = cmg::ProfClass{};
  ctx->launches = 0;
  return CMG_OK;
}

int cmg_ctx_launch_count(cmg_ctx *ctx, int64_t *launches) {
  if (!ctx || !launches) return CMG_ERR_INVALID_ARG;
  *launches = ctx->launches;
  return CMG_OK;
}

}  // extern "C"
