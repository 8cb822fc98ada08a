// The raw-signal entry points of the C ABI (include/haru.h): event
// detection on the device (kernels in events.cu), alone or followed by the
// sDTW batch path on each read's query.

#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "engine.h"

namespace {

int sig_fail(haru_ctx *c, cudaError_t e) {  // the context lock is held
  if (e == cudaSuccess) return HARU_OK;
  if (c->sticky == HARU_OK) c->sticky = HARU_ECUDA;
  return HARU_ECUDA;
}

#define SIG_CUDA(call)                                \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return sig_fail(ctx, e_);  \
  } while (0)

// Host-side checks of a sample CSR: offsets[0] = 0, non-decreasing, every
// read at most HARU_MAX_READ_SAMPLES long.
bool samples_valid(const uint32_t *off, uint32_t nreads) {
  if (off[0] != 0) return false;
  for (uint32_t r = 0; r < nreads; ++r) {
    if (off[r + 1] < off[r]) return false;
    if (off[r + 1] - off[r] > static_cast<uint32_t>(HARU_MAX_READ_SAMPLES)) return false;
  }
  return true;
}

// Device copies of the inputs (host mode) and the detection buffers; sets
// *d_smp and *d_soff to the device samples and offsets. Lock held.
int stage_signal(haru_ctx *ctx, const int16_t *samples, const uint32_t *offsets, uint32_t nreads, bool on_dev,
                 uint32_t max_events, cudaStream_t s, const int16_t **d_smp, const uint32_t **d_soff) {
  using haru::grow;
  *d_smp = samples;
  *d_soff = offsets;
  if (!on_dev) {
    if (!samples_valid(offsets, nreads)) return HARU_EINVAL;
    const size_t ns = offsets[nreads];
    SIG_CUDA(grow(&ctx->d_samples, &ctx->cap_samples, ns));
    SIG_CUDA(grow(&ctx->d_soff, &ctx->cap_soff, static_cast<size_t>(nreads) + 1));
    if (ns) SIG_CUDA(cudaMemcpyAsync(ctx->d_samples, samples, ns * sizeof(int16_t), cudaMemcpyHostToDevice, s));
    SIG_CUDA(cudaMemcpyAsync(ctx->d_soff, offsets, (static_cast<size_t>(nreads) + 1) * sizeof(uint32_t),
                             cudaMemcpyHostToDevice, s));
    *d_smp = ctx->d_samples;
    *d_soff = ctx->d_soff;
  }
  const size_t cap = static_cast<size_t>(nreads) * max_events;
  SIG_CUDA(grow(&ctx->sig_strided, &ctx->cap_strided, cap));
  SIG_CUDA(grow(&ctx->sig_counts, &ctx->cap_sig_counts, nreads));
  return HARU_OK;
}

}  // namespace

extern "C" {

int haru_event_params_default(haru_event_params *p) {
  if (!p) return HARU_EINVAL;
  haru::event_params_default(p);
  return HARU_OK;
}

int haru_detect_events(haru_ctx *ctx, const int16_t *samples, const uint32_t *sample_offsets, uint32_t nreads,
                       const haru_event_params *params, float *events, uint32_t *event_offsets, uintptr_t stream,
                       uint32_t flags) {
  using haru::grow;
  if (!ctx) return HARU_EINVAL;
  haru_event_params p;
  haru::event_params_default(&p);
  if (params) p = *params;
  if (!haru::event_params_valid(p)) return HARU_EINVAL;
  if (flags & ~static_cast<uint32_t>(HARU_ON_DEVICE | HARU_ASYNC)) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (nreads == 0) return HARU_OK;
  if (!samples || !sample_offsets || !events || !event_offsets) return HARU_EINVAL;
  const bool on_dev = flags & HARU_ON_DEVICE;
  const bool async = on_dev && (flags & HARU_ASYNC);
  SIG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : ctx->stream;
  const int16_t *d_smp = nullptr;
  const uint32_t *d_soff = nullptr;
  int rc = stage_signal(ctx, samples, sample_offsets, nreads, on_dev, p.max_events, s, &d_smp, &d_soff);
  if (rc != HARU_OK) return rc;
  float *d_ev = events;
  uint32_t *d_eoff = event_offsets;
  if (!on_dev) {
    SIG_CUDA(grow(&ctx->sig_events, &ctx->cap_sig_events, static_cast<size_t>(nreads) * p.max_events));
    SIG_CUDA(grow(&ctx->sig_off, &ctx->cap_sig_off, static_cast<size_t>(nreads) + 1));
    d_ev = ctx->sig_events;
    d_eoff = ctx->sig_off;
  }
  SIG_CUDA(cudaMemsetAsync(ctx->ws.ints, 0, sizeof(int), s));
  SIG_CUDA(haru::enqueue_events(d_smp, d_soff, nreads, p, ctx->sig_strided, ctx->sig_counts, d_eoff, d_ev,
                                ctx->ws.ints + haru::kIntStatus, s));
  if (async) {
    ctx->last_status = HARU_OK;
    return HARU_OK;
  }
  int st = 0;
  SIG_CUDA(cudaMemcpyAsync(&st, ctx->ws.ints + haru::kIntStatus, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (!on_dev) {
    SIG_CUDA(cudaMemcpyAsync(event_offsets, d_eoff, (static_cast<size_t>(nreads) + 1) * sizeof(uint32_t),
                             cudaMemcpyDeviceToHost, s));
    SIG_CUDA(cudaStreamSynchronize(s));
    if (event_offsets[nreads])
      SIG_CUDA(cudaMemcpyAsync(events, d_ev, static_cast<size_t>(event_offsets[nreads]) * sizeof(float),
                               cudaMemcpyDeviceToHost, s));
  }
  SIG_CUDA(cudaStreamSynchronize(s));
  ctx->last_status = st;
  return st;
}

int haru_sdtw_batch_signal(haru_ctx *ctx, int precision, const int16_t *samples, const uint32_t *sample_offsets,
                           uint32_t nreads, const haru_event_params *params, float *out_cost, int64_t *out_col,
                           uint32_t *out_events, uintptr_t stream, uint32_t flags) {
  using haru::grow;
  if (!ctx) return HARU_EINVAL;
  if (precision != HARU_FP32 && precision != HARU_INT16 && precision != HARU_INT16_ACC32) return HARU_EINVAL;
  haru_event_params p;
  haru::event_params_default(&p);
  if (params) p = *params;
  if (!haru::event_params_valid(p)) return HARU_EINVAL;
  if (flags & ~static_cast<uint32_t>(HARU_ON_DEVICE | HARU_ASYNC | HARU_PROFILE)) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (ctx->N == 0) return HARU_ENOREF;
  if (nreads == 0) return HARU_OK;
  if (!samples || !sample_offsets || !out_cost || !out_col) return HARU_EINVAL;
  const bool on_dev = flags & HARU_ON_DEVICE;
  const bool async = on_dev && (flags & HARU_ASYNC);
  const bool prof = flags & HARU_PROFILE;
  SIG_CUDA(cudaSetDevice(ctx->device));
  cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : ctx->stream;
  const int16_t *d_smp = nullptr;
  const uint32_t *d_soff = nullptr;
  int rc = stage_signal(ctx, samples, sample_offsets, nreads, on_dev, p.max_events, s, &d_smp, &d_soff);
  if (rc != HARU_OK) return rc;
  SIG_CUDA(grow(&ctx->sig_events, &ctx->cap_sig_events, static_cast<size_t>(nreads) * p.max_events));
  SIG_CUDA(grow(&ctx->sig_off, &ctx->cap_sig_off, static_cast<size_t>(nreads) + 1));
  float *d_cost = out_cost;
  int64_t *d_col = out_col;
  if (!on_dev) {
    if (ctx->cap_q < static_cast<size_t>(nreads) + 1) {
      size_t c0 = 0, c1 = 0, c2 = 0, c3 = 0;
      cudaFree(ctx->d_offsets); cudaFree(ctx->d_cost); cudaFree(ctx->d_col); cudaFree(ctx->d_start);
      ctx->d_offsets = nullptr; ctx->d_cost = nullptr; ctx->d_col = nullptr; ctx->d_start = nullptr;
      ctx->cap_q = 0;
      SIG_CUDA(grow(&ctx->d_offsets, &c0, static_cast<size_t>(nreads) + 1));
      SIG_CUDA(grow(&ctx->d_cost, &c1, static_cast<size_t>(nreads) + 1));
      SIG_CUDA(grow(&ctx->d_col, &c2, static_cast<size_t>(nreads) + 1));
      SIG_CUDA(grow(&ctx->d_start, &c3, static_cast<size_t>(nreads) + 1));
      ctx->cap_q = static_cast<size_t>(nreads) + 1;
    }
    d_cost = ctx->d_cost;
    d_col = ctx->d_col;
  }
  const haru::LaunchCfg lc = ctx->launch_cfg();
  SIG_CUDA(haru::ws_reserve(ctx->ws, precision, nreads, lc));
  // counters zeroed once: the detection reports into the same status word
  SIG_CUDA(cudaMemsetAsync(ctx->ws.ints, 0, haru::kIntWords * sizeof(int), s));
  if (prof) SIG_CUDA(haru::record_event(ctx->ev[0], s));
  SIG_CUDA(haru::enqueue_events(d_smp, d_soff, nreads, p, ctx->sig_strided, ctx->sig_counts, ctx->sig_off,
                                ctx->sig_events, ctx->ws.ints + haru::kIntStatus, s));
  SIG_CUDA(haru::ws_enqueue(ctx->ws, precision, ctx->ref_view(), ctx->sig_events, ctx->sig_off, nreads, 1, d_cost,
                            d_col, lc, s, nullptr, prof ? ctx->ev[1] : nullptr, nullptr, false,
                            prof ? ctx->ev[3] : nullptr));
  if (prof) {
    SIG_CUDA(haru::record_event(ctx->ev[2], s));
    ctx->profiled = true;
  }
  if (out_events)
    SIG_CUDA(cudaMemcpyAsync(out_events, ctx->sig_counts, static_cast<size_t>(nreads) * sizeof(uint32_t),
                             on_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
  if (async) {
    ctx->last_status = HARU_OK;
    return HARU_OK;
  }
  if (!on_dev) {
    SIG_CUDA(cudaMemcpyAsync(out_cost, d_cost, static_cast<size_t>(nreads) * sizeof(float), cudaMemcpyDeviceToHost,
                             s));
    SIG_CUDA(cudaMemcpyAsync(out_col, d_col, static_cast<size_t>(nreads) * sizeof(int64_t), cudaMemcpyDeviceToHost,
                             s));
  }
  int st = 0;
  SIG_CUDA(cudaMemcpyAsync(&st, ctx->ws.ints + haru::kIntStatus, sizeof(int), cudaMemcpyDeviceToHost, s));
  SIG_CUDA(cudaStreamSynchronize(s));
  ctx->last_status = st;
  return st;
}

}  // extern "C"
