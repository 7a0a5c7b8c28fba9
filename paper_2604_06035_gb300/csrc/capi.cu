// capi.cu -- the extern "C" boundary of libcmg.so (declared in include/cmg.h).
// Every entry point converts C++ exceptions into a status code and a
// thread-local message; nothing here computes on the host.
#include <cstring>
#include <new>
#include <string>

#include "cmg_internal.cuh"

namespace {

thread_local std::string g_last_error;

int fail(int code, const std::string &msg) {
  g_last_error = msg;
  return code;
}

}  // namespace

namespace cmg {
void record_error(const char *msg) { g_last_error = msg; }
}  // namespace cmg

namespace {

template <class F>
int guard(F &&f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const cmg::Error &e) {
    return fail(e.code, e.what());
  } catch (const std::bad_alloc &) {
    return fail(CMG_ERR_OOM, "host allocation failed");
  } catch (const std::exception &e) {
    return fail(CMG_ERR_CUDA, e.what());
  } catch (...) {
    return fail(CMG_ERR_CUDA, "unknown error");
  }
}

struct DeviceScope {
  int prev = -1;
  explicit DeviceScope(int d) {
    cudaGetDevice(&prev);
    CMG_CUDA(cudaSetDevice(d));
  }
  ~DeviceScope() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

void check_mem(int mem) {
  if (mem != CMG_MEM_HOST && mem != CMG_MEM_DEVICE) throw cmg::Error(CMG_ERR_INVALID_ARG, "bad cmg_mem tag");
}

void need(bool ok, const char *what) {
  if (!ok) throw cmg::Error(CMG_ERR_INVALID_ARG, what);
}

// Run `produce(device_out)` and deliver `bytes` to `out` in memory space mem.
// The context's staging buffer `which` with at least `bytes` (grow-only: a
// cudaMalloc / cudaFree per call would synchronise the device every time).
// Every user synchronises the stream before returning, so the next call may
// reuse it.
void *staging(cmg_ctx *ctx, int which, size_t bytes) {
  if (bytes == 0) bytes = 1;
  if (ctx->stage_bytes[which] < bytes) {
    if (ctx->stage[which]) {
      CMG_CUDA(cudaStreamSynchronize(ctx->stream));
      if (ctx->h2d_stream) CMG_CUDA(cudaStreamSynchronize(ctx->h2d_stream));
      if (ctx->d2h_stream) CMG_CUDA(cudaStreamSynchronize(ctx->d2h_stream));
      ctx->d2h_pending = false;
      cudaFree(ctx->stage[which]);
      ctx->stage[which] = nullptr;
      ctx->stage_bytes[which] = 0;
    }
    if (cudaMalloc(&ctx->stage[which], bytes) != cudaSuccess) {
      cudaGetLastError();
      ctx->stage[which] = nullptr;
      throw cmg::Error(CMG_ERR_OOM, "device staging buffer");
    }
    ctx->stage_bytes[which] = bytes;
  }
  return ctx->stage[which];
}

// The copy streams and their events, on first use.
void copy_streams(cmg_ctx *ctx) {
  if (ctx->d2h_done) return;
  if (!ctx->h2d_stream) CMG_CUDA(cudaStreamCreateWithFlags(&ctx->h2d_stream, cudaStreamNonBlocking));
  if (!ctx->d2h_stream) CMG_CUDA(cudaStreamCreateWithFlags(&ctx->d2h_stream, cudaStreamNonBlocking));
  for (cudaEvent_t *e : {&ctx->h2d_done, &ctx->stage0_free, &ctx->stage1_ready})
    if (!*e) CMG_CUDA(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
  cudaEvent_t e = nullptr;  // set last: marks the whole set ready
  CMG_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  ctx->d2h_done = e;
}

// A queued download may still read stage[1]: later writes to it wait.
void wait_stage1(cmg_ctx *ctx) {
  if (ctx->d2h_pending) CMG_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->d2h_done, 0));
}

template <class F>
void deliver(cmg_ctx *ctx, void *out, size_t bytes, int mem, F &&produce) {
  if (mem == CMG_MEM_DEVICE) {
    produce(out);
    CMG_CUDA(cudaGetLastError());
    return;
  }
  void *t = staging(ctx, 1, bytes);
  wait_stage1(ctx);
  produce(t);
  if (bytes) CMG_CUDA(cudaMemcpyAsync(out, t, bytes, cudaMemcpyDeviceToHost, ctx->stream));
  CMG_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->d2h_pending = false;
}

// deliver() without waiting: produce() is queued on the context's stream and
// the download on the download stream, behind it; `out` is written once
// cmg_ctx_synchronize() returns.  Work queued afterwards on the context's
// stream overlaps the download.
template <class F>
void deliver_async(cmg_ctx *ctx, void *out, size_t bytes, int mem, F &&produce) {
  if (mem == CMG_MEM_DEVICE) {
    produce(out);
    CMG_CUDA(cudaGetLastError());
    return;
  }
  void *t = staging(ctx, 1, bytes);
  copy_streams(ctx);
  wait_stage1(ctx);
  produce(t);
  CMG_CUDA(cudaGetLastError());
  CMG_CUDA(cudaEventRecord(ctx->stage1_ready, ctx->stream));
  CMG_CUDA(cudaStreamWaitEvent(ctx->d2h_stream, ctx->stage1_ready, 0));
  if (bytes) CMG_CUDA(cudaMemcpyAsync(out, t, bytes, cudaMemcpyDeviceToHost, ctx->d2h_stream));
  CMG_CUDA(cudaEventRecord(ctx->d2h_done, ctx->d2h_stream));
  ctx->d2h_pending = true;
}

// Make `in` device-resident for the duration of `use(device_in)`.  A host
// buffer is uploaded on the upload stream (overlapping work already queued
// on the context's stream) and `use` is queued behind the upload; the call
// returns once the upload has finished, so the caller may reuse its buffer.
template <class F>
void accept(cmg_ctx *ctx, const void *in, size_t bytes, int mem, F &&use) {
  if (mem == CMG_MEM_DEVICE) {
    use(in);
    return;
  }
  void *t = staging(ctx, 0, bytes);
  copy_streams(ctx);
  if (ctx->stage0_used) CMG_CUDA(cudaStreamWaitEvent(ctx->h2d_stream, ctx->stage0_free, 0));
  if (bytes) CMG_CUDA(cudaMemcpyAsync(t, in, bytes, cudaMemcpyHostToDevice, ctx->h2d_stream));
  CMG_CUDA(cudaEventRecord(ctx->h2d_done, ctx->h2d_stream));
  CMG_CUDA(cudaStreamWaitEvent(ctx->stream, ctx->h2d_done, 0));
  use(static_cast<const void *>(t));
  CMG_CUDA(cudaGetLastError());
  CMG_CUDA(cudaEventRecord(ctx->stage0_free, ctx->stream));
  ctx->stage0_used = true;
  CMG_CUDA(cudaEventSynchronize(ctx->h2d_done));
}

}  // namespace

extern "C" {

const char *cmg_version(void) { return "cmg 0.1.0 sm_103a"; }

int cmg_debug_inject_alloc_failure(int64_t after) {
  return guard([&] {
    need(after >= 0, "negative count");
    cmg::inject_alloc_failure(after);
    return CMG_OK;
  });
}

int cmg_debug_neighbour_sum(cmg_ctx *ctx, const double *rows, int64_t n, int which, double *out, cmg_mem mem) {
  return guard([&] {
    need(ctx && n >= 0 && (n == 0 || (rows && out)), "bad arguments");
    need(which == 0 || which == 1, "which must be 0 or 1");
    check_mem(mem);
    DeviceScope ds(ctx->device);
    accept(ctx, rows, sizeof(double) * 6 * n, mem, [&](const void *din) {
      deliver(ctx, out, sizeof(double) * n, mem, [&](void *dout) {
        cmg::neighbour_sum(static_cast<const double *>(din), n, which, static_cast<double *>(dout), ctx->stream);
      });
    });
    CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    return CMG_OK;
  });
}

const char *cmg_last_error(void) { return g_last_error.c_str(); }

int cmg_ctx_create(int device, void *stream, cmg_ctx **out) {
  return guard([&] {
    need(out != nullptr, "out is NULL");
    *out = nullptr;
    int count = 0;
    CMG_CUDA(cudaGetDeviceCount(&count));
    need(device >= 0 && device < count, "no such CUDA device");
    DeviceScope ds(device);
    cmg_ctx *c = new cmg_ctx();
    c->device = device;
    c->stream = static_cast<cudaStream_t>(stream);
    try {
      CMG_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
      CMG_CUDA(cudaMalloc(&c->d_err, 64));
      CMG_CUDA(cudaMemsetAsync(c->d_err, 0, 64, c->stream));
      CMG_CUDA(cudaMallocHost(&c->h_pinned, 64));
      CMG_CUDA(cudaMallocHost(&c->h_dpinned, 64));
      CMG_CUDA(cudaEventCreate(&c->ev0));
      CMG_CUDA(cudaEventCreate(&c->ev1));
      CMG_CUDA(cudaStreamSynchronize(c->stream));
    } catch (...) {
      cmg_ctx_destroy(c);
      throw;
    }
    *out = c;
    return CMG_OK;
  });
}

int cmg_ctx_destroy(cmg_ctx *ctx) {
  if (!ctx) return CMG_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(ctx->device);
  cudaStreamSynchronize(ctx->stream);
  if (ctx->h2d_stream) cudaStreamSynchronize(ctx->h2d_stream);
  if (ctx->d2h_stream) cudaStreamSynchronize(ctx->d2h_stream);
  for (cudaEvent_t e : {ctx->h2d_done, ctx->stage0_free, ctx->stage1_ready, ctx->d2h_done})
    if (e) cudaEventDestroy(e);
  if (ctx->h2d_stream) cudaStreamDestroy(ctx->h2d_stream);
  if (ctx->d2h_stream) cudaStreamDestroy(ctx->d2h_stream);
  if (ctx->d_err) cudaFree(ctx->d_err);
  if (ctx->h_pinned) cudaFreeHost(ctx->h_pinned);
  if (ctx->h_dpinned) cudaFreeHost(ctx->h_dpinned);
  if (ctx->ev0) cudaEventDestroy(ctx->ev0);
  if (ctx->ev1) cudaEventDestroy(ctx->ev1);
  for (void *p : ctx->stage)
    if (p) cudaFree(p);
  for (cudaEvent_t e : ctx->ev_pool) cudaEventDestroy(e);
  if (ctx->cap_stream) cudaStreamDestroy(ctx->cap_stream);
  if (ctx->cap_stream2) cudaStreamDestroy(ctx->cap_stream2);
  delete ctx;
  if (prev >= 0) cudaSetDevice(prev);
  return CMG_OK;
}

int cmg_ctx_synchronize(cmg_ctx *ctx) {
  return guard([&] {
    need(ctx != nullptr, "ctx is NULL");
    DeviceScope ds(ctx->device);
    CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->h2d_stream) CMG_CUDA(cudaStreamSynchronize(ctx->h2d_stream));
    if (ctx->d2h_stream) CMG_CUDA(cudaStreamSynchronize(ctx->d2h_stream));
    ctx->d2h_pending = false;
    return CMG_OK;
  });
}

int cmg_morton_encode(cmg_ctx *ctx, const uint32_t *ijk, int64_t n, uint64_t *keys, cmg_mem mem) {
  return guard([&] {
    need(ctx && n >= 0 && (n == 0 || (ijk && keys)), "bad arguments");
    check_mem(mem);
    DeviceScope ds(ctx->device);
    CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    accept(ctx, ijk, sizeof(uint32_t) * 3 * n, mem, [&](const void *din) {
      deliver(ctx, keys, sizeof(uint64_t) * n, mem, [&](void *dout) {
        cmg::encode_keys(static_cast<const uint32_t *>(din), n, static_cast<uint64_t *>(dout), ctx->d_err,
                         ctx->stream);
      });
    });
    CMG_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->h_pinned[0]) {
      CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
      throw cmg::Error(ctx->h_pinned[0], "coordinate outside [0, 2^21)");
    }
    return CMG_OK;
  });
}

int cmg_morton_decode(cmg_ctx *ctx, const uint64_t *keys, int64_t n, uint32_t *ijk, cmg_mem mem) {
  return guard([&] {
    need(ctx && n >= 0 && (n == 0 || (ijk && keys)), "bad arguments");
    check_mem(mem);
    DeviceScope ds(ctx->device);
    accept(ctx, keys, sizeof(uint64_t) * n, mem, [&](const void *din) {
      deliver(ctx, ijk, sizeof(uint32_t) * 3 * n, mem, [&](void *dout) {
        cmg::decode_keys(static_cast<const uint64_t *>(din), n, static_cast<uint32_t *>(dout), ctx->stream);
      });
    });
    return CMG_OK;
  });
}

int cmg_morton_encode128(cmg_ctx *ctx, const uint64_t *ijk, int64_t n, uint64_t *keys, cmg_mem mem) {
  return guard([&] {
    need(ctx && n >= 0 && (n == 0 || (ijk && keys)), "bad arguments");
    check_mem(mem);
    DeviceScope ds(ctx->device);
    CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    accept(ctx, ijk, sizeof(uint64_t) * 3 * n, mem, [&](const void *din) {
      deliver(ctx, keys, sizeof(cmg::Key128) * n, mem, [&](void *dout) {
        cmg::encode_keys128(static_cast<const uint64_t *>(din), n, static_cast<cmg::Key128 *>(dout), ctx->d_err,
                            ctx->stream);
      });
    });
    CMG_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
    CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    if (ctx->h_pinned[0]) {
      CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
      throw cmg::Error(ctx->h_pinned[0], "coordinate outside [0, 2^42)");
    }
    return CMG_OK;
  });
}

int cmg_morton_decode128(cmg_ctx *ctx, const uint64_t *keys, int64_t n, uint64_t *ijk, cmg_mem mem) {
  return guard([&] {
    need(ctx && n >= 0 && (n == 0 || (ijk && keys)), "bad arguments");
    check_mem(mem);
    DeviceScope ds(ctx->device);
    accept(ctx, keys, sizeof(cmg::Key128) * n, mem, [&](const void *din) {
      deliver(ctx, ijk, sizeof(uint64_t) * 3 * n, mem, [&](void *dout) {
        cmg::decode_keys128(static_cast<const cmg::Key128 *>(din), n, static_cast<uint64_t *>(dout), ctx->stream);
      });
    });
    return CMG_OK;
  });
}

namespace {

int level_build(cmg_ctx *ctx, int level, int nx, int periodic_mask, const void *keys, int64_t n_octs, cmg_mem mem,
                cmg_level *parent, cmg_level **out, int key_bits) {
  return guard([&] {
    need(out != nullptr, "out is NULL");
    *out = nullptr;
    need(ctx != nullptr, "ctx is NULL");
    const int bits = key_bits == 128 ? 42 : cmg::kMortonBits;
    const int max_level = bits + 1;
    need(level >= 1 && level <= max_level && nx >= 1,
         key_bits == 128 ? "level must be in [1, 43] and nx >= 1" : "level must be in [1, 22] and nx >= 1");
    need(nx <= (1 << 20) && ((uint64_t)nx << (level - 1)) <= (1ull << bits),
         key_bits == 128 ? "2^(level-1) nx exceeds 2^42" : "2^(level-1) nx exceeds 2^21");
    need(periodic_mask >= 0 && periodic_mask <= 7, "periodic_mask must be in [0, 7]");
    need(n_octs >= 0 && n_octs < (1ll << 31) - 1 && (n_octs == 0 || keys), "bad keys / n_octs");
    check_mem(mem);
    if (parent) {
      need(parent->ctx == ctx && parent->lev == level - 1 && parent->nx == nx && parent->pmask == periodic_mask,
           "parent must be level-1 of the same context, nx and periodic_mask");
      need(parent->key_bits == key_bits, "parent must use the same Morton key width");
    }
    DeviceScope ds(ctx->device);
    cmg_level *L = new cmg_level();
    L->ctx = ctx;
    L->device = ctx->device;
    L->stream = ctx->stream;
    L->lev = level;
    L->nx = nx;
    L->pmask = periodic_mask;
    L->n = n_octs;
    L->parent = parent;
    L->key_bits = key_bits;
    const uint64_t npd = (uint64_t)nx << (level - 1);
    L->periodic_full = parent == nullptr && periodic_mask == 7 && npd <= 2048 && (uint64_t)n_octs == npd * npd * npd;
    try {
      cmg::build_level(L, keys, mem);
      L->partials = L->mem.alloc<double>(cmg::blocks_for(n_octs > 0 ? n_octs : 1));
      L->scal = L->mem.alloc<double>(16, true, ctx->stream);
      CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    } catch (...) {
      cudaStreamSynchronize(ctx->stream);
      L->mem.release();
      delete L;
      throw;
    }
    *out = L;
    return CMG_OK;
  });
}

}  // namespace

int cmg_level_build(cmg_ctx *ctx, int level, int nx, int periodic_mask, const uint64_t *keys, int64_t n_octs,
                    cmg_mem mem, cmg_level *parent, cmg_level **out) {
  return level_build(ctx, level, nx, periodic_mask, keys, n_octs, mem, parent, out, 64);
}

int cmg_level_build128(cmg_ctx *ctx, int level, int nx, int periodic_mask, const uint64_t *keys, int64_t n_octs,
                       cmg_mem mem, cmg_level *parent, cmg_level **out) {
  return level_build(ctx, level, nx, periodic_mask, keys, n_octs, mem, parent, out, 128);
}

int cmg_level_key_bits(const cmg_level *lvl, int *bits) {
  return guard([&] {
    need(lvl && bits, "bad arguments");
    *bits = lvl->key_bits;
    return CMG_OK;
  });
}

int cmg_level_destroy(cmg_level *lvl) {
  if (!lvl) return CMG_OK;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(lvl->device);  // the level's own copies: no use of its context
  cudaStreamSynchronize(lvl->stream);
  cmg::destroy_graphs(lvl);
  if (lvl->h_ctrl) cudaFreeHost(lvl->h_ctrl);
  if (lvl->ev_start) cudaEventDestroy(lvl->ev_start);
  if (lvl->ev_end) cudaEventDestroy(lvl->ev_end);
  lvl->mem.release();
  delete lvl;
  if (prev >= 0) cudaSetDevice(prev);
  return CMG_OK;
}

int cmg_level_n_octs(const cmg_level *lvl, int64_t *n) {
  return guard([&] {
    need(lvl && n, "NULL argument");
    *n = lvl->n;
    return CMG_OK;
  });
}

int cmg_level_hash_capacity(const cmg_level *lvl, int64_t *cap) {
  return guard([&] {
    need(lvl && cap, "NULL argument");
    *cap = lvl->mg[0].cap;
    return CMG_OK;
  });
}

int cmg_level_lookup(cmg_level *lvl, const uint64_t *q, int64_t n, int32_t *idx, cmg_mem mem) {
  return guard([&] {
    need(lvl && n >= 0 && (n == 0 || (q && idx)), "bad arguments");
    need(lvl->key_bits == 64, "the level has 128-bit keys: use cmg_level_lookup128");
    check_mem(mem);
    cmg_ctx *ctx = lvl->ctx;
    DeviceScope ds(ctx->device);
    accept(ctx, q, sizeof(uint64_t) * n, mem, [&](const void *din) {
      deliver(ctx, idx, sizeof(int32_t) * n, mem, [&](void *dout) {
        cmg::hash_lookup(lvl->mg[0], static_cast<const uint64_t *>(din), n, static_cast<int32_t *>(dout),
                         ctx->stream);
      });
    });
    return CMG_OK;
  });
}

int cmg_level_lookup128(cmg_level *lvl, const uint64_t *q, int64_t n, int32_t *idx, cmg_mem mem) {
  return guard([&] {
    need(lvl && n >= 0 && (n == 0 || (q && idx)), "bad arguments");
    need(lvl->key_bits == 128, "the level has 64-bit keys: use cmg_level_lookup");
    check_mem(mem);
    cmg_ctx *ctx = lvl->ctx;
    DeviceScope ds(ctx->device);
    accept(ctx, q, sizeof(cmg::Key128) * n, mem, [&](const void *din) {
      deliver(ctx, idx, sizeof(int32_t) * n, mem, [&](void *dout) {
        cmg::hash_lookup128(lvl->mg[0], static_cast<const cmg::Key128 *>(din), n, static_cast<int32_t *>(dout),
                            ctx->stream);
      });
    });
    return CMG_OK;
  });
}

int cmg_level_get_neighbors(cmg_level *lvl, int32_t *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || out), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, sizeof(int32_t) * 7 * lvl->n, mem,
            [&](void *d) { cmg::ext_neighbors(lvl, static_cast<int32_t *>(d), lvl->ctx->stream); });
    return CMG_OK;
  });
}

int cmg_level_get_father_cells(cmg_level *lvl, int32_t *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || out), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, sizeof(int32_t) * 12 * lvl->n, mem,
            [&](void *d) { cmg::father_cells(lvl, static_cast<int32_t *>(d), lvl->ctx->stream); });
    return CMG_OK;
  });
}

int cmg_level_set_density(cmg_level *lvl, const double *rho, cmg_mem mem, double rho_bar, double four_pi_g) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || rho), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    accept(lvl->ctx, rho, sizeof(double) * 8 * lvl->n, mem,
           [&](const void *d) { cmg::set_density(lvl, static_cast<const double *>(d), rho_bar, four_pi_g); });
    return CMG_OK;
  });
}

int cmg_level_set_phi(cmg_level *lvl, const double *phi, cmg_mem mem) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || phi), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    accept(lvl->ctx, phi, sizeof(double) * 8 * lvl->n, mem,
           [&](const void *d) { cmg::pack_field(lvl, 0, CMG_FIELD_PHI, CMG_PREC_FP64, d); });
    return CMG_OK;
  });
}

int cmg_level_get_phi_async(cmg_level *lvl, double *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || out), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    deliver_async(lvl->ctx, out, sizeof(double) * 8 * lvl->n, mem,
                  [&](void *d) { cmg::unpack_field(lvl, 0, CMG_FIELD_PHI, CMG_PREC_FP64, d); });
    return CMG_OK;
  });
}

int cmg_level_get_phi(cmg_level *lvl, double *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || out), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, sizeof(double) * 8 * lvl->n, mem,
            [&](void *d) { cmg::unpack_field(lvl, 0, CMG_FIELD_PHI, CMG_PREC_FP64, d); });
    return CMG_OK;
  });
}

int cmg_level_get_residual(cmg_level *lvl, double *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || out), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, sizeof(double) * 8 * lvl->n, mem,
            [&](void *d) { cmg::residual_out(lvl, 0, CMG_PREC_FP64, static_cast<double *>(d)); });
    return CMG_OK;
  });
}

int cmg_level_get_ghosts(cmg_level *lvl, double *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && (lvl->n == 0 || out), "bad arguments");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, sizeof(double) * 24 * lvl->n, mem,
            [&](void *d) { cmg::get_ghosts(lvl, static_cast<double *>(d)); });
    return CMG_OK;
  });
}

int cmg_level_solve(cmg_level *lvl, const cmg_solve_params *params, cmg_solve_stats *stats) {
  return guard([&] {
    need(lvl && params, "NULL argument");
    DeviceScope ds(lvl->ctx->device);
    const int st = cmg::solve(lvl, params, stats);
    if (st == CMG_ERR_NOT_CONVERGED) g_last_error = "max_cycles reached above tol";
    if (st == CMG_ERR_DIVERGED) g_last_error = "residual diverged";
    return st;
  });
}

int cmg_level_solve_async(cmg_level *lvl, const cmg_solve_params *params) {
  return guard([&] {
    need(lvl && params, "NULL argument");
    DeviceScope ds(lvl->ctx->device);
    cmg::solve_launch(lvl, params);
    return CMG_OK;
  });
}

int cmg_level_solve_wait(cmg_level *lvl, cmg_solve_stats *stats) {
  return guard([&] {
    need(lvl != nullptr, "NULL level");
    DeviceScope ds(lvl->ctx->device);
    const int st = cmg::solve_wait(lvl, stats);
    if (st == CMG_ERR_NOT_CONVERGED) g_last_error = "max_cycles reached above tol";
    if (st == CMG_ERR_DIVERGED) g_last_error = "residual diverged";
    return st;
  });
}

int cmg_level_set_schedule(cmg_level *lvl, int64_t tail_octs_fp64, int64_t tail_octs_fp32) {
  return guard([&] {
    need(lvl != nullptr, "NULL level");
    DeviceScope ds(lvl->device);
    CMG_CUDA(cudaStreamSynchronize(lvl->stream));
    if (tail_octs_fp64 >= 0) lvl->tail_octs_fp64 = tail_octs_fp64;
    if (tail_octs_fp32 >= 0) lvl->tail_octs_fp32 = tail_octs_fp32;
    cmg::destroy_graphs(lvl);  // recorded graphs follow the old schedule
    return CMG_OK;
  });
}

int cmg_level_set_stencil(cmg_level *lvl, int staged) {
  return guard([&] {
    need(lvl != nullptr && staged >= 0 && staged <= 2, "bad arguments");
    DeviceScope ds(lvl->device);
    CMG_CUDA(cudaStreamSynchronize(lvl->stream));
    lvl->staged = staged;
    cmg::destroy_graphs(lvl);  // recorded graphs hold the old kernels
    return CMG_OK;
  });
}

int cmg_level_set_spin_budget(cmg_level *lvl, int64_t cycles) {
  return guard([&] {
    need(lvl != nullptr, "NULL level");
    need(cycles >= 0, "negative spin budget");
    DeviceScope ds(lvl->device);
    CMG_CUDA(cudaStreamSynchronize(lvl->stream));
    lvl->tail_spin_budget = cycles;
    cmg::destroy_graphs(lvl);  // recorded graphs hold the old budget
    return CMG_OK;
  });
}

int cmg_batch_create(cmg_level *lvl, const int64_t *offsets, int n_patches, cmg_batch **out) {
  return guard([&] {
    need(out != nullptr, "out is NULL");
    *out = nullptr;
    need(lvl && offsets && n_patches >= 1, "bad batch arguments");
    DeviceScope ds(lvl->device);
    cmg::batch_create(lvl, offsets, n_patches, out);
    return CMG_OK;
  });
}

int cmg_batch_destroy(cmg_batch *batch) {
  if (!batch) return CMG_OK;
  return guard([&] {
    cmg::batch_destroy(batch);
    return CMG_OK;
  });
}

int cmg_batch_set_schedule(cmg_batch *batch, const cmg_batch_schedule *schedule) {
  return guard([&] {
    need(batch && schedule, "NULL argument");
    need(schedule->threads <= 512, "batch kernels use at most 512 threads per block");
    need(schedule->n_pre >= 1, "the batch schedule needs n_pre >= 1");
    cmg::batch_set_schedule(batch, schedule);
    return CMG_OK;
  });
}

int cmg_batch_get_schedule(cmg_batch *batch, cmg_batch_schedule *schedule) {
  return guard([&] {
    need(batch && schedule, "NULL argument");
    *schedule = batch->sched;
    return CMG_OK;
  });
}

int cmg_batch_set_spin_budget(cmg_batch *batch, int64_t cycles) {
  return guard([&] {
    need(batch && cycles >= 0, "bad spin budget");
    batch->spin_budget = cycles;
    return CMG_OK;
  });
}

int cmg_batch_solve(cmg_batch *batch, const cmg_solve_params *params, cmg_batch_stats *stats) {
  return guard([&] {
    need(batch && params, "NULL argument");
    DeviceScope ds(batch->lvl->device);
    const int st = cmg::batch_solve(batch, params, stats);
    if (st == CMG_ERR_TIMEOUT) g_last_error = "a grid barrier of the persistent kernel gave up (spin budget)";
    if (st == CMG_ERR_NOT_CONVERGED) g_last_error = "max_cycles reached above tol";
    if (st == CMG_ERR_DIVERGED) g_last_error = "residual diverged";
    return st;
  });
}

int cmg_batch_patch_stats(cmg_batch *batch, double *rel, int32_t *converged_at, double *norm0) {
  return guard([&] {
    need(batch != nullptr, "NULL batch");
    DeviceScope ds(batch->lvl->device);
    cmg::batch_patch_stats(batch, rel, converged_at, norm0);
    return CMG_OK;
  });
}

int cmg_batch_autotune(cmg_batch *batch, const cmg_solve_params *params, cmg_batch_schedule *best,
                       double *best_ms) {
  return guard([&] {
    need(batch && params, "NULL argument");
    DeviceScope ds(batch->lvl->device);
    cmg::batch_autotune(batch, params, best, best_ms);
    return CMG_OK;
  });
}

int cmg_level_mg_depth(const cmg_level *lvl, int *depth) {
  return guard([&] {
    need(lvl && depth, "NULL argument");
    *depth = (int)lvl->mg.size();
    return CMG_OK;
  });
}

int cmg_level_mg_info(const cmg_level *lvl, int m, int64_t *n_octs, int *amr_level) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    if (n_octs) *n_octs = lvl->mg[m].n;
    if (amr_level) *amr_level = lvl->mg[m].lev;
    return CMG_OK;
  });
}

int cmg_level_mg_keys(cmg_level *lvl, int m, uint64_t *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    need(lvl->key_bits == 64, "the level has 128-bit keys: use cmg_level_mg_keys128");
    check_mem(mem);
    const cmg::MgLev &g = lvl->mg[m];
    need(g.n == 0 || out, "out is NULL");
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, sizeof(uint64_t) * g.n, mem, [&](void *d) {
      if (g.n) CMG_CUDA(cudaMemcpyAsync(d, g.keys, sizeof(uint64_t) * g.n, cudaMemcpyDeviceToDevice, lvl->ctx->stream));
    });
    return CMG_OK;
  });
}

int cmg_level_mg_keys128(cmg_level *lvl, int m, uint64_t *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    need(lvl->key_bits == 128, "the level has 64-bit keys: use cmg_level_mg_keys");
    check_mem(mem);
    const cmg::MgLev &g = lvl->mg[m];
    need(g.n == 0 || out, "out is NULL");
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, sizeof(cmg::Key128) * g.n, mem, [&](void *d) {
      if (g.n)
        CMG_CUDA(cudaMemcpyAsync(d, g.keys128, sizeof(cmg::Key128) * g.n, cudaMemcpyDeviceToDevice, lvl->ctx->stream));
    });
    return CMG_OK;
  });
}

int cmg_level_mg_active(cmg_level *lvl, int m, uint8_t *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    check_mem(mem);
    const cmg::MgLev &g = lvl->mg[m];
    need(g.n == 0 || out, "out is NULL");
    DeviceScope ds(lvl->ctx->device);
    deliver(lvl->ctx, out, 8 * g.n, mem,
            [&](void *d) { cmg::mg_active_bytes(g, static_cast<uint8_t *>(d), lvl->ctx->stream); });
    return CMG_OK;
  });
}

int cmg_level_mg_get(cmg_level *lvl, int m, int field, int precision, void *out, cmg_mem mem) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    need(field == CMG_FIELD_PHI || field == CMG_FIELD_F, "bad field");
    need(precision == CMG_PREC_FP64 || precision == CMG_PREC_MIXED, "bad precision");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    if (precision == CMG_PREC_MIXED) cmg::ensure_fp32(lvl);
    const size_t es = precision == CMG_PREC_FP64 ? 8 : 4;
    need(lvl->mg[m].n == 0 || out, "out is NULL");
    deliver(lvl->ctx, out, es * 8 * lvl->mg[m].n, mem,
            [&](void *d) { cmg::unpack_field(lvl, m, field, precision, d); });
    return CMG_OK;
  });
}

int cmg_level_mg_set(cmg_level *lvl, int m, int field, int precision, const void *in, cmg_mem mem) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    need(field == CMG_FIELD_PHI || field == CMG_FIELD_F, "bad field");
    need(precision == CMG_PREC_FP64 || precision == CMG_PREC_MIXED, "bad precision");
    check_mem(mem);
    DeviceScope ds(lvl->ctx->device);
    if (precision == CMG_PREC_MIXED) cmg::ensure_fp32(lvl);
    const size_t es = precision == CMG_PREC_FP64 ? 8 : 4;
    need(lvl->mg[m].n == 0 || in, "in is NULL");
    accept(lvl->ctx, in, es * 8 * lvl->mg[m].n, mem,
           [&](const void *d) { cmg::pack_field(lvl, m, field, precision, d); });
    return CMG_OK;
  });
}

int cmg_level_mg_step(cmg_level *lvl, int m, int op, int precision, int n, double *norm2) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    need(precision == CMG_PREC_FP64 || precision == CMG_PREC_MIXED, "bad precision");
    const int depth = (int)lvl->mg.size();
    DeviceScope ds(lvl->ctx->device);
    const bool f64 = precision == CMG_PREC_FP64;
    if (!f64) cmg::ensure_fp32(lvl);
    switch (op) {
      case CMG_OP_SWEEP:
        need(n >= 0, "n < 0");
        for (int k = 0; k < n; ++k) f64 ? cmg::sweep<double>(lvl, m, false) : cmg::sweep<float>(lvl, m, false);
        break;
      case CMG_OP_RESIDUAL:
        need(norm2 != nullptr, "norm2 is NULL");
        f64 ? cmg::resid_restrict<double>(lvl, m, false, true, false, lvl->scal + 2)
            : cmg::resid_restrict<float>(lvl, m, false, true, false, lvl->scal + 2);
        CMG_CUDA(cudaMemcpyAsync(lvl->ctx->h_dpinned, lvl->scal + 2, sizeof(double), cudaMemcpyDeviceToHost,
                                 lvl->ctx->stream));
        CMG_CUDA(cudaStreamSynchronize(lvl->ctx->stream));
        *norm2 = lvl->ctx->h_dpinned[0];
        break;
      case CMG_OP_RESTRICT:
        need(m + 1 < depth, "no coarser MG level");
        f64 ? cmg::resid_restrict<double>(lvl, m, true, false, true, nullptr)
            : cmg::resid_restrict<float>(lvl, m, true, false, true, nullptr);
        break;
      case CMG_OP_PROLONG:
        need(m + 1 < depth, "no coarser MG level");
        f64 ? cmg::prolong<double>(lvl, m) : cmg::prolong<float>(lvl, m);
        break;
      case CMG_OP_COARSE:
        need(m == depth - 1 && n >= 0, "CMG_OP_COARSE needs m = depth - 1");
        cmg::coarse_solve(lvl, precision, n);
        break;
      case CMG_OP_GHOSTS:
        cmg::fill_ghosts(lvl);
        break;
      default:
        throw cmg::Error(CMG_ERR_INVALID_ARG, "unknown op");
    }
    CMG_CUDA(cudaStreamSynchronize(lvl->ctx->stream));
    return CMG_OK;
  });
}

// ---- sharded level solve (App. G V-cycle per rank, Sec. 9.5 halo exchange)

int cmg_level_mg_step_range(cmg_level *lvl, int m, int op, int arg, int64_t lo, int64_t hi, double *value) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    const int64_t n = lvl->mg[m].n;
    need(lo >= 0 && lo <= hi && hi <= n, "range outside the MG level");
    const int depth = (int)lvl->mg.size();
    DeviceScope ds(lvl->ctx->device);
    cmg_ctx *ctx = lvl->ctx;
    switch (op) {
      case CMG_OPR_SWEEP:
        need(arg >= 0 && arg <= 3, "sweep arg: colour | 2 * zero_other");
        cmg::range_sweep_pass(lvl, m, arg & 1, (arg & 2) != 0, lo, hi);
        break;
      case CMG_OPR_RESIDUAL:
        need(value != nullptr, "value is NULL");
        need(arg == 0 || arg == 1, "residual arg: c1_swept 0 or 1");
        cmg::range_residual(lvl, m, false, arg == 1, lo, hi, lvl->scal + 2);
        CMG_CUDA(cudaMemcpyAsync(ctx->h_dpinned, lvl->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CMG_CUDA(cudaStreamSynchronize(ctx->stream));
        *value = ctx->h_dpinned[0];
        break;
      case CMG_OPR_RESTRICT:
        need(m + 1 < depth, "no coarser MG level");
        need(arg == 0 || arg == 1, "restrict arg: c1_swept 0 or 1");
        cmg::range_residual(lvl, m, true, arg == 1, lo, hi, nullptr);
        break;
      case CMG_OPR_PROLONG:
        need(m + 1 < depth, "no coarser MG level");
        need(arg == 0 || arg == 1, "prolong arg: c0_dead 0 or 1");
        cmg::range_prolong(lvl, m, arg == 1, lo, hi);
        break;
      case CMG_OPR_SUM_PHI:
        need(value != nullptr, "value is NULL");
        cmg::range_sum_phi(lvl, m, lo, hi, lvl->scal + 2);
        CMG_CUDA(cudaMemcpyAsync(ctx->h_dpinned, lvl->scal + 2, sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
        CMG_CUDA(cudaStreamSynchronize(ctx->stream));
        *value = ctx->h_dpinned[0];
        break;
      case CMG_OPR_SHIFT_PHI:
        need(value != nullptr, "value is NULL");
        cmg::range_shift_phi(lvl, m, lo, hi, *value);
        break;
      default:
        throw cmg::Error(CMG_ERR_INVALID_ARG, "unknown range op");
    }
    CMG_CUDA(cudaStreamSynchronize(ctx->stream));
    return CMG_OK;
  });
}

namespace {
// Reads and clears the context's device error word (an index outside the
// level in a gather or scatter).
int take_device_error(cmg_ctx *ctx) {
  CMG_CUDA(cudaMemcpyAsync(ctx->h_pinned, ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CMG_CUDA(cudaStreamSynchronize(ctx->stream));
  const int e = ctx->h_pinned[0];
  if (e != 0) {
    CMG_CUDA(cudaMemsetAsync(ctx->d_err, 0, sizeof(int), ctx->stream));
    CMG_CUDA(cudaStreamSynchronize(ctx->stream));
  }
  return e;
}
}  // namespace

int cmg_level_mg_gather(cmg_level *lvl, int m, int field, const int32_t *cells, int64_t n, double *out) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    need(field == 0 || field == 1, "field must be 0 (phi) or 1 (stored source)");
    need(n >= 0 && (n == 0 || (cells && out)), "bad arguments");
    DeviceScope ds(lvl->ctx->device);
    cmg::gather_cells(lvl, m, field, cells, n, out, lvl->ctx->d_err);
    if (take_device_error(lvl->ctx)) throw cmg::Error(CMG_ERR_INVALID_ARG, "cell index outside the MG level");
    return CMG_OK;
  });
}

int cmg_level_mg_scatter(cmg_level *lvl, int m, int field, const int32_t *cells, int64_t n, const double *in) {
  return guard([&] {
    need(lvl && m >= 0 && m < (int)lvl->mg.size(), "bad MG level");
    need(field == 0 || field == 1, "field must be 0 (phi) or 1 (stored source)");
    need(n >= 0 && (n == 0 || (cells && in)), "bad arguments");
    DeviceScope ds(lvl->ctx->device);
    cmg::scatter_cells(lvl, m, field, cells, n, in, lvl->ctx->d_err);
    if (take_device_error(lvl->ctx)) throw cmg::Error(CMG_ERR_INVALID_ARG, "cell index outside the MG level");
    return CMG_OK;
  });
}

}  // extern "C"
