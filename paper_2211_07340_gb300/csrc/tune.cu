// Autotuner: times the batch path on the caller's own batch over a grid of
// launch shapes and keeps the fastest in the context's configuration.
//
// Tuned: warps per CTA (queries or pairs sharing one reference tile stream),
// reference tile width and the work-unit target (how finely sweeps are cut
// into verified reference segments; 1 = never cut), then at the best of
// those the strip geometry of queries of <= 256 events (32-lane strips or
// stacked 16-lane strips with twice the rows per lane). Beyond that the
// strip height is not a free choice: S = floor(M / 32) + 1 rows per
// lane (at most 16) is the smallest strip that holds a query with a pad row
// on top, and a taller one only adds padding.

#include <cuda_runtime.h>

#include <cstring>
#include <vector>

#include "engine.h"

extern "C" int haru_autotune(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets,
                             uint32_t nq, uint32_t flags, haru_config *chosen) {
  using namespace haru;
  if (!ctx || (precision != HARU_FP32 && precision != HARU_INT16 && precision != HARU_INT16_ACC32) || nq == 0 ||
      !events || !offsets)
    return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (ctx->N == 0) return HARU_ENOREF;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return HARU_ECUDA;
  cudaStream_t s = ctx->stream;
  const bool on_dev = flags & HARU_ON_DEVICE;
  const int raw = (flags & HARU_RAW) ? 1 : 0;
  const uint32_t *d_off = offsets;
  const float *d_ev = events;
  std::vector<uint32_t> h_off(nq + 1);
  if (on_dev) {
    if (cudaMemcpy(h_off.data(), offsets, (nq + 1) * sizeof(uint32_t), cudaMemcpyDeviceToHost) != cudaSuccess)
      return HARU_ECUDA;
  } else {
    std::memcpy(h_off.data(), offsets, (nq + 1) * sizeof(uint32_t));
  }
  const long lim = std::min<long>(static_cast<long>(ctx->N), HARU_MAX_QUERY);
  if (h_off[0] != 0) return HARU_EINVAL;
  for (uint32_t q = 0; q < nq; ++q) {
    const long m = static_cast<long>(h_off[q + 1]) - static_cast<long>(h_off[q]);
    if (m < 1 || m > lim) return HARU_EINVAL;
  }
  float *t_ev = nullptr, *t_cost = nullptr;
  uint32_t *t_off = nullptr;
  int64_t *t_col = nullptr;
  cudaError_t e = cudaSuccess;
  if (!on_dev) {
    e = cudaMalloc(&t_ev, static_cast<size_t>(h_off[nq]) * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&t_off, (nq + 1) * sizeof(uint32_t));
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(t_ev, events, static_cast<size_t>(h_off[nq]) * sizeof(float), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(t_off, offsets, (nq + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    d_ev = t_ev;
    d_off = t_off;
  }
  if (e == cudaSuccess) e = cudaMalloc(&t_cost, nq * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&t_col, nq * sizeof(int64_t));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const LaunchCfg base = ctx->launch_cfg();
  const int auto_units = 4 * ctx->sms * 8;
  const int warps_c[] = {4, 8, 12};
  const int tiles_c[] = {2048, 4096, 8192, 16384};
  const int units_c[] = {1, auto_units / 2, auto_units, 2 * auto_units};
  float best_ms = -1.0f;
  LaunchCfg best = base;
  // One trial: the minimum of two timed runs after one warm-up; kept if fastest.
  auto trial = [&](const LaunchCfg &lc) {
    if (e != cudaSuccess) return;
    e = ws_reserve(ctx->ws, precision, nq, lc);
    float ms_min = -1.0f;
    for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
      e = cudaEventRecord(e0, s);
      if (e == cudaSuccess)
        e = ws_enqueue(ctx->ws, precision, ctx->ref_view(), d_ev, d_off, nq, raw, t_cost, t_col, lc, s, nullptr,
                       nullptr);
      if (e == cudaSuccess) e = cudaEventRecord(e1, s);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.0f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e == cudaSuccess && rep > 0 && (ms_min < 0.0f || ms < ms_min)) ms_min = ms;
    }
    int st = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&st, ctx->ws.ints + kIntStatus, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && st == HARU_OK && ms_min > 0.0f && (best_ms < 0.0f || ms_min < best_ms)) {
      best_ms = ms_min;
      best = lc;
    }
  };
  // Launch shape first, at the context's stacking rule ...
  for (int w : warps_c)
    for (int t : tiles_c)
      for (int u : units_c) {
        LaunchCfg lc = base;
        lc.warps = w;
        lc.tile = t;
        lc.units_target = u;
        trial(lc);
      }
  // ... then the strip geometry of short queries at that shape: 32-lane
  // strips of S = floor(M / 32) + 1 rows per lane, or stacked 16-lane strips
  // of floor(M / 16) + 1 rows (stack_short: auto, always, never).
  const LaunchCfg shape = best;
  for (int st : {0, 1, -1}) {
    if (st == shape.stack_short) continue;
    LaunchCfg lc = shape;
    lc.stack_short = st;
    trial(lc);
  }
  cudaFree(t_ev);
  cudaFree(t_off);
  cudaFree(t_cost);
  cudaFree(t_col);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess) {
    if (ctx->sticky == HARU_OK) ctx->sticky = HARU_ECUDA;
    return HARU_ECUDA;
  }
  if (best_ms < 0.0f) return HARU_EINVAL;
  ctx->cfg.warps_per_cta = best.warps;
  ctx->cfg.tile_cols = best.tile;
  ctx->cfg.units_target = best.units_target;
  ctx->cfg.stack_short = best.stack_short;
  if (chosen) *chosen = ctx->cfg;
  return HARU_OK;
}
