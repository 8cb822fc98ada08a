// The C ABI of libharu (declared in include/haru.h): contexts, the reference
// store, and the batch entry point of the sDTW hot path.

#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "engine.h"

using haru::Group;
using haru::Item;
using haru::grow;

namespace {

int cuda_fail(haru_ctx *c, cudaError_t e) {
  if (e == cudaSuccess) return HARU_OK;
  if (c->sticky == HARU_OK) c->sticky = HARU_ECUDA;
  return HARU_ECUDA;
}

#define HARU_CUDA(call)                                \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(ctx, e_);  \
  } while (0)

// Free a reference image allocated with its kRefFront front pad, given the
// pointer to its column 0 (nullptr: nothing).
template <class T>
void free_ref_image(T *col0) {
  if (col0) cudaFree(col0 - haru::kRefFront);
}

int pick_warps(const haru_config &cfg) {
  int w = cfg.warps_per_cta;
  if (w != 2 && w != 4 && w != 8 && w != 12) w = 8;
  return w;
}

int pick_tile(const haru_config &cfg) {
  int t = cfg.tile_cols;
  if (t < 2048 || t > haru::kMaxTile) t = 4096;
  return t;
}

// At least 1 ms: a CTA whose wait ran out drains its reference copies still
// in flight within the same limit before it exits, and a tile copy (at most
// 67 KB) lands in microseconds, so the drain always outlasts it.
unsigned long long wait_ns(const haru_config &cfg) {
  if (!cfg.wait_limit) return 2000000000ull;
  return std::max<unsigned long long>(cfg.wait_limit, 1000ull) * 1000ull;
}

}  // namespace

haru::LaunchCfg haru_ctx::launch_cfg() const {
  haru::LaunchCfg lc;
  lc.warps = pick_warps(cfg);
  lc.tile = pick_tile(cfg);
  lc.ctas_per_sm = cfg.ctas_per_sm;
  lc.sms = sms;
  lc.units_target = cfg.units_target;
  lc.stack_short = cfg.stack_short > 0 ? 1 : (cfg.stack_short < 0 ? -1 : 0);
  lc.wait_ns = wait_ns(cfg);
  return lc;
}

haru::RefView haru_ctx::ref_view() const {
  haru::RefView r;
  r.img16 = img16;
  r.img32 = img32;
  r.N = static_cast<long>(N);
  r.scale_log2 = scale_log2;
  return r;
}

namespace haru {

// Reference and launch settings of a context, for haru_sdtw_batch_noalloc
// (noalloc.cu). Reads state only; allocates nothing.
int ctx_reference(haru_ctx *ctx, int precision, const void **img, long *N, int *scale_log2, int *device,
                  cudaStream_t *stream, int *warps, int *tile, unsigned long long *wait, int *per_sm, int *sms) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (ctx->N == 0) return HARU_ENOREF;
  *img = precision != HARU_FP32 ? static_cast<const void *>(ctx->img16) : static_cast<const void *>(ctx->img32);
  *N = static_cast<long>(ctx->N);
  *scale_log2 = ctx->scale_log2;
  *device = ctx->device;
  *stream = ctx->stream;
  *warps = pick_warps(ctx->cfg);
  *tile = pick_tile(ctx->cfg);
  *wait = wait_ns(ctx->cfg);
  *sms = ctx->sms;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return HARU_ECUDA;
  *per_sm = ctx->cfg.ctas_per_sm;
  return HARU_OK;
}

// Record a CUDA failure of a call that does not hold the context lock (the
// no-allocation path): the first CUDA error of a context is sticky.
int ctx_cuda_fail(haru_ctx *ctx, cudaError_t e) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  return cuda_fail(ctx, e);
}

}  // namespace haru

extern "C" {

int haru_config_default(haru_config *cfg) {
  if (!cfg) return HARU_EINVAL;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->warps_per_cta = 8;
  cfg->tile_cols = 4096;
  cfg->ctas_per_sm = 0;
  cfg->wait_limit = 0;
  cfg->threshold = 0.0f;
  cfg->serve_precision = HARU_INT16;
  cfg->serve_budget_bytes = 64u << 20;
  cfg->serve_max_batch = 1024;
  cfg->serve_prefix = 250;
  haru::event_params_default(&cfg->serve_events);
  return HARU_OK;
}

const char *haru_strerror(int code) {
  switch (code) {
    case HARU_OK: return "ok";
    case HARU_EINVAL: return "invalid argument";
    case HARU_ENOREF: return "no reference loaded";
    case HARU_ENOMEM: return "out of memory or admission budget";
    case HARU_EBUSY: return "busy (serving queue full, or the reference of a serving context)";
    case HARU_ETIMEDOUT: return "bounded wait timed out";
    case HARU_ECUDA: return "CUDA error";
    default: return "unknown error";
  }
}

int haru_create(haru_ctx **out, int device, const haru_config *cfg) {
  if (!out) return HARU_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HARU_EINVAL;
  haru_ctx *ctx = new (std::nothrow) haru_ctx();
  if (!ctx) return HARU_ENOMEM;
  ctx->device = device;
  if (cfg)
    ctx->cfg = *cfg;
  else
    haru_config_default(&ctx->cfg);
  int rc = HARU_OK;
  do {
    if (cudaSetDevice(device) != cudaSuccess) { rc = HARU_ECUDA; break; }
    if (cudaDeviceGetAttribute(&ctx->sms, cudaDevAttrMultiProcessorCount, device) != cudaSuccess) {
      rc = HARU_ECUDA;
      break;
    }
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) { rc = HARU_ECUDA; break; }
    size_t ci = 0;
    if (grow(&ctx->ws.ints, &ci, (size_t)haru::kIntWords) != cudaSuccess) { rc = HARU_ENOMEM; break; }
    if (cudaMalloc(&ctx->stats, 2 * sizeof(double)) != cudaSuccess) { rc = HARU_ENOMEM; break; }
    bool ev_ok = true;
    for (auto &e : ctx->ev) ev_ok = ev_ok && cudaEventCreate(&e) == cudaSuccess;
    if (!ev_ok) { rc = HARU_ECUDA; break; }
  } while (0);
  if (rc != HARU_OK) {
    haru_destroy(ctx);
    return rc;
  }
  *out = ctx;
  return HARU_OK;
}

int haru_configure(haru_ctx *ctx, const haru_config *cfg) {
  if (!ctx || !cfg) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  ctx->cfg = *cfg;
  return HARU_OK;
}

int haru_get_config(haru_ctx *ctx, haru_config *cfg) {
  if (!ctx || !cfg) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  *cfg = ctx->cfg;
  return HARU_OK;
}

void haru_destroy(haru_ctx *ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->server) {
    haru::server_destroy(ctx->server);
    ctx->server = nullptr;
  }
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  void *ptrs[] = {ctx->ref_z,     ctx->stats,       ctx->partials,    ctx->d_events,   ctx->d_offsets,
                  ctx->d_cost,    ctx->d_col,       ctx->d_start,     ctx->d_samples,  ctx->d_soff,
                  ctx->sig_strided, ctx->sig_events, ctx->sig_counts, ctx->sig_off};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  free_ref_image(ctx->img16);
  free_ref_image(ctx->img32);
  haru::ws_free(ctx->ws);
  for (auto e : ctx->ev)
    if (e) cudaEventDestroy(e);
  if (ctx->stream) cudaStreamDestroy(ctx->stream);
  delete ctx;
}

size_t haru_ref_length(const haru_ctx *ctx) { return ctx ? ctx->N : 0; }

// Normalise/quantise `x_dev` (n floats on the device) into the reference store.
// Each image is kRefFront zero words, then columns 0 .. N - 1, then kRefPad
// zero words; the context keeps the pointer to column 0.
static int ref_install(haru_ctx *ctx, const float *x_dev, size_t n, int normalize, int scale_log2) {
  cudaStream_t s = ctx->stream;
  const size_t img_len = n + haru::kRefPad;
  const size_t all = static_cast<size_t>(haru::kRefFront) + img_len;
  float *z = nullptr, *i32b = nullptr;
  uint32_t *i16b = nullptr;
  cudaError_t e = cudaMalloc(&z, n * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&i16b, all * sizeof(uint32_t));
  if (e == cudaSuccess) e = cudaMalloc(&i32b, all * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(z); cudaFree(i16b); cudaFree(i32b);
    cudaGetLastError();
    return HARU_ENOMEM;
  }
  uint32_t *i16 = i16b + haru::kRefFront;
  float *i32 = i32b + haru::kRefFront;
  const size_t nb = (n + 4095) / 4096;
  int st = 0;
  e = grow(&ctx->partials, &ctx->partials_cap, nb);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws.ints, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(i16b, 0, all * sizeof(uint32_t), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(i32b, 0, all * sizeof(float), s);
  if (e == cudaSuccess && normalize)
    e = haru::launch_zscore_stats(x_dev, n, ctx->partials, ctx->stats, ctx->ws.ints, s);
  if (e == cudaSuccess)
    e = haru::launch_ref_finish(x_dev, n, ctx->stats, normalize, scale_log2, z, i16, i32, img_len, ctx->ws.ints, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, ctx->ws.ints, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess || st != HARU_OK) {  // the previous reference stays in place
    const int rc = e != cudaSuccess ? cuda_fail(ctx, e) : st;
    cudaStreamSynchronize(s);
    cudaFree(z); cudaFree(i16b); cudaFree(i32b);
    return rc;
  }
  cudaFree(ctx->ref_z);
  free_ref_image(ctx->img16);
  free_ref_image(ctx->img32);
  ctx->ref_z = z;
  ctx->img16 = i16;
  ctx->img32 = i32;
  ctx->N = n;
  ctx->scale_log2 = scale_log2;
  return HARU_OK;
}

int haru_ref_load(haru_ctx *ctx, const float *levels, size_t n, int normalize, int scale_log2) {
  if (!ctx) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (ctx->server) return HARU_EBUSY;  // the serving loop holds the reference it started with
  if (!levels || n == 0 || scale_log2 < 1 || scale_log2 > 7) return HARU_EINVAL;
  if (n > (size_t)1 << 31) return HARU_EINVAL;
  HARU_CUDA(cudaSetDevice(ctx->device));
  float *x = nullptr;
  if (cudaMalloc(&x, n * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return HARU_ENOMEM;
  }
  cudaError_t e = cudaMemcpyAsync(x, levels, n * sizeof(float), cudaMemcpyHostToDevice, ctx->stream);
  int rc = e == cudaSuccess ? ref_install(ctx, x, n, normalize, scale_log2) : cuda_fail(ctx, e);
  cudaStreamSynchronize(ctx->stream);
  cudaFree(x);
  return rc;
}

int haru_ref_build(haru_ctx *ctx, const uint8_t *bases, size_t n_bases, const float *kmer_levels, int k,
                   int scale_log2) {
  if (!ctx) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (ctx->server) return HARU_EBUSY;  // as haru_ref_load
  if (!bases || !kmer_levels || k < 1 || k > 12 || n_bases < (size_t)k || scale_log2 < 1 || scale_log2 > 7)
    return HARU_EINVAL;
  const size_t per = n_bases - k + 1;
  const size_t n = 2 * per;
  if (n > (size_t)1 << 31) return HARU_EINVAL;
  HARU_CUDA(cudaSetDevice(ctx->device));
  const size_t nmodel = (size_t)1 << (2 * k);
  uint8_t *db = nullptr;
  float *dm = nullptr, *x = nullptr;
  cudaError_t e = cudaMalloc(&db, n_bases);
  if (e == cudaSuccess) e = cudaMalloc(&dm, nmodel * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&x, n * sizeof(float));
  if (e != cudaSuccess) {
    cudaFree(db); cudaFree(dm); cudaFree(x);
    cudaGetLastError();
    return HARU_ENOMEM;
  }
  int rc = HARU_OK;
  cudaStream_t s = ctx->stream;
  e = cudaMemcpyAsync(db, bases, n_bases, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dm, kmer_levels, nmodel * sizeof(float), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(ctx->ws.ints, 0, sizeof(int), s);
  if (e == cudaSuccess) e = haru::launch_ref_levels(db, n_bases, dm, k, x, ctx->ws.ints, s);
  int st = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&st, ctx->ws.ints, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess)
    rc = cuda_fail(ctx, e);
  else if (st != HARU_OK)
    rc = st;
  else
    rc = ref_install(ctx, x, n, 1, scale_log2);
  cudaStreamSynchronize(s);
  cudaFree(db); cudaFree(dm); cudaFree(x);
  return rc;
}

int haru_ref_read(haru_ctx *ctx, float *z, int16_t *q, size_t n) {
  if (!ctx) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (ctx->N == 0) return HARU_ENOREF;
  if (n != ctx->N) return HARU_EINVAL;
  HARU_CUDA(cudaSetDevice(ctx->device));
  if (z) HARU_CUDA(cudaMemcpyAsync(z, ctx->ref_z, n * sizeof(float), cudaMemcpyDeviceToHost, ctx->stream));
  if (q) {
    std::vector<uint32_t> w(n);
    HARU_CUDA(cudaMemcpyAsync(w.data(), ctx->img16, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, ctx->stream));
    HARU_CUDA(cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < n; ++i) q[i] = static_cast<int16_t>(w[i] & 0xffffu);
  }
  HARU_CUDA(cudaStreamSynchronize(ctx->stream));
  return HARU_OK;
}

namespace {

// The batch path shared by haru_sdtw_batch and haru_sdtw_batch_span;
// `precision` is the kernels' (kPrecF32Span / kPrecWideSpan when out_start
// is wanted).
int batch_call(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets, uint32_t nq,
               float *out_cost, int64_t *out_col, int64_t *out_start, uintptr_t stream, uint32_t flags) {
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (ctx->N == 0) return HARU_ENOREF;
  if (nq == 0) return HARU_OK;
  const bool span = haru::prec_span(precision);
  if (!events || !offsets || !out_cost || !out_col || (span && !out_start)) return HARU_EINVAL;
  const bool on_dev = flags & HARU_ON_DEVICE;
  const bool async = (flags & HARU_ASYNC) && on_dev;
  const int raw = (flags & HARU_RAW) ? 1 : 0;
  HARU_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : ctx->stream;

  const uint32_t *d_off = offsets;
  const float *d_ev = events;
  float *d_cost = out_cost;
  int64_t *d_col = out_col;
  int64_t *d_start = out_start;
  if (!on_dev) {
    // Host inputs: validate on the host, then stage on the device.
    const long lim = std::min<long>((long)ctx->N, HARU_MAX_QUERY);
    if (offsets[0] != 0) return HARU_EINVAL;
    for (uint32_t q = 0; q < nq; ++q) {
      if (offsets[q + 1] < offsets[q]) return HARU_EINVAL;
      long m = (long)offsets[q + 1] - (long)offsets[q];
      if (m < 1 || m > lim) return HARU_EINVAL;
    }
    const size_t ne = offsets[nq];
    HARU_CUDA(grow(&ctx->d_events, &ctx->cap_events, ne));
    if (ctx->cap_q < (size_t)nq + 1) {
      size_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
      cudaFree(ctx->d_offsets); cudaFree(ctx->d_cost); cudaFree(ctx->d_col); cudaFree(ctx->d_start);
      ctx->d_offsets = nullptr; ctx->d_cost = nullptr; ctx->d_col = nullptr; ctx->d_start = nullptr;
      ctx->cap_q = 0;
      HARU_CUDA(grow(&ctx->d_offsets, &c0, (size_t)nq + 1));
      HARU_CUDA(grow(&ctx->d_cost, &c1, (size_t)nq + 1));
      HARU_CUDA(grow(&ctx->d_col, &c2, (size_t)nq + 1));
      HARU_CUDA(grow(&ctx->d_start, &c3, (size_t)nq + 1));
      ctx->cap_q = (size_t)nq + 1;
    }
    HARU_CUDA(cudaMemcpyAsync(ctx->d_events, events, ne * sizeof(float), cudaMemcpyHostToDevice, s));
    HARU_CUDA(cudaMemcpyAsync(ctx->d_offsets, offsets, ((size_t)nq + 1) * sizeof(uint32_t),
                              cudaMemcpyHostToDevice, s));
    d_off = ctx->d_offsets;
    d_ev = ctx->d_events;
    d_cost = ctx->d_cost;
    d_col = ctx->d_col;
    d_start = span ? ctx->d_start : nullptr;
  }
  const haru::LaunchCfg lc = ctx->launch_cfg();
  HARU_CUDA(haru::ws_reserve(ctx->ws, precision, nq, lc));
  const bool prof = flags & HARU_PROFILE;
  HARU_CUDA(haru::ws_enqueue(ctx->ws, precision, ctx->ref_view(), d_ev, d_off, nq, raw, d_cost, d_col, lc, s,
                             prof ? ctx->ev[0] : nullptr, prof ? ctx->ev[1] : nullptr, d_start, true,
                             prof ? ctx->ev[3] : nullptr));
  if (prof) {
    HARU_CUDA(haru::record_event(ctx->ev[2], s));
    ctx->profiled = true;
  }

  if (async) {
    ctx->last_status = HARU_OK;
    return HARU_OK;
  }
  if (!on_dev) {
    HARU_CUDA(cudaMemcpyAsync(out_cost, d_cost, (size_t)nq * sizeof(float), cudaMemcpyDeviceToHost, s));
    HARU_CUDA(cudaMemcpyAsync(out_col, d_col, (size_t)nq * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (span)
      HARU_CUDA(cudaMemcpyAsync(out_start, d_start, (size_t)nq * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  }
  int st = 0;
  HARU_CUDA(cudaMemcpyAsync(&st, ctx->ws.ints, sizeof(int), cudaMemcpyDeviceToHost, s));
  HARU_CUDA(cudaStreamSynchronize(s));
  ctx->last_status = st;
  return st;
}

}  // namespace

int haru_sdtw_batch(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets, uint32_t nq,
                    float *out_cost, int64_t *out_col, uintptr_t stream, uint32_t flags) {
  if (!ctx) return HARU_EINVAL;
  if (precision != HARU_FP32 && precision != HARU_INT16 && precision != HARU_INT16_ACC32) return HARU_EINVAL;
  return batch_call(ctx, precision, events, offsets, nq, out_cost, out_col, nullptr, stream, flags);
}

int haru_sdtw_batch_span(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets, uint32_t nq,
                         float *out_cost, int64_t *out_col, int64_t *out_start, uintptr_t stream, uint32_t flags) {
  if (!ctx) return HARU_EINVAL;
  if (precision != HARU_FP32 && precision != HARU_INT16_ACC32) return HARU_EINVAL;
  return batch_call(ctx, precision == HARU_FP32 ? haru::kPrecF32Span : haru::kPrecWideSpan, events, offsets, nq,
                    out_cost, out_col, out_start, stream, flags);
}

int haru_last_timing(haru_ctx *ctx, float *ms_prep, float *ms_sweep) {
  if (!ctx) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (!ctx->profiled) return HARU_EINVAL;
  HARU_CUDA(cudaSetDevice(ctx->device));
  HARU_CUDA(cudaEventSynchronize(ctx->ev[2]));
  float a = 0.0f, b = 0.0f;
  HARU_CUDA(cudaEventElapsedTime(&a, ctx->ev[0], ctx->ev[1]));
  HARU_CUDA(cudaEventElapsedTime(&b, ctx->ev[1], ctx->ev[3]));
  if (ms_prep) *ms_prep = a;
  if (ms_sweep) *ms_sweep = b;
  return HARU_OK;
}

int haru_last_stats(haru_ctx *ctx, haru_batch_stats *out) {
  if (!ctx || !out) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  HARU_CUDA(cudaSetDevice(ctx->device));
  int w[haru::kIntWords];
  HARU_CUDA(cudaMemcpy(w, ctx->ws.ints, sizeof(w), cudaMemcpyDeviceToHost));
  out->items = (uint32_t)w[haru::kIntItems];
  out->groups = (uint32_t)w[haru::kIntGroups];
  out->fixups = (uint32_t)w[haru::kIntFixups];
  out->max_segments = (uint32_t)w[haru::kIntMaxSeg];
  return HARU_OK;
}

int haru_last_status(haru_ctx *ctx) {
  if (!ctx) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  int st = 0;
  HARU_CUDA(cudaSetDevice(ctx->device));
  HARU_CUDA(cudaMemcpy(&st, ctx->ws.ints, sizeof(int), cudaMemcpyDeviceToHost));
  ctx->last_status = st;
  return st;
}

}  // extern "C"
