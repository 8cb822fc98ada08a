// The batch engine: workspace sizing and the stream-ordered sequence of
// kernels of one batch (planner, pack, sweep, segment fix-up).

#include <cuda_runtime.h>

#include <algorithm>

#include "engine.h"

namespace haru {

cudaError_t record_event(cudaEvent_t e, cudaStream_t s) {
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  cudaError_t r = cudaStreamIsCapturing(s, &cs);
  if (r != cudaSuccess) return r;
  if (cs == cudaStreamCaptureStatusActive) return cudaEventRecordWithFlags(e, s, cudaEventRecordExternal);
  return cudaEventRecord(e, s);
}

void ws_free(Workspace &ws) {
  void *p[] = {ws.ints, ws.items, ws.groups, ws.img, ws.states, ws.bests, ws.qstats};
  for (void *q : p)
    if (q) cudaFree(q);
  ws = Workspace();
}

namespace {

// Buffer sizes one batch of nq queries needs.
struct WsNeeds {
  size_t max_items, units, qstats, states;
  int nseg_cap, units_target;
};

WsNeeds ws_needs(int precision, uint32_t nq, const LaunchCfg &lc) {
  WsNeeds w;
  const int mode = plan_mode(precision);
  w.max_items = items_bound(mode, nq);
  // Work units: enough (query x reference segment) units to keep every SM
  // busy to the end; nseg_cap bounds the segments per item for storage.
  w.units_target = lc.units_target > 0 ? lc.units_target : 4 * lc.sms * kernel_warps(precision, lc);
  // Fewest items the batch can make (stacked: four int16 or two other
  // queries per item); the segment cap is sized for that case.
  const size_t items_min = (mode == 0 || mode == 3) ? (static_cast<size_t>(nq) + 1) / 2
                                                   : (static_cast<size_t>(nq) + 3) / 4;
  // (twice that: the planner doubles the segments of the queue's tail)
  w.nseg_cap = static_cast<int>(std::min<size_t>(
      kMaxSeg, 2 * ((static_cast<size_t>(w.units_target) + items_min - 1) / std::max<size_t>(items_min, 1))));
  if (w.nseg_cap < 1) w.nseg_cap = 1;
  w.units = w.max_items * static_cast<size_t>(w.nseg_cap);
  w.qstats = 2 * static_cast<size_t>(nq);
  w.states = w.nseg_cap > 1 ? w.units * 2 * state_words(precision) : 0;
  return w;
}

cudaError_t ws_alloc(Workspace &ws, size_t max_items, size_t units, size_t qstats, size_t states) {
  cudaError_t e = cudaSuccess;
  size_t c = ws.ints ? static_cast<size_t>(kIntWords) : 0;
  if ((e = grow(&ws.ints, &c, kIntWords)) != cudaSuccess) return e;
  if (ws.cap_items < max_items) {
    cudaFree(ws.items);
    cudaFree(ws.groups);
    cudaFree(ws.img);
    ws.items = nullptr;
    ws.groups = nullptr;
    ws.img = nullptr;
    ws.cap_items = 0;
    size_t c0 = 0, c1 = 0, c2 = 0;
    if ((e = grow(&ws.items, &c0, max_items)) != cudaSuccess) return e;
    if ((e = grow(&ws.groups, &c1, (max_items + kMaxS) * kMaxSeg)) != cudaSuccess) return e;
    if ((e = grow(&ws.img, &c2, max_items * kImgStride)) != cudaSuccess) return e;
    ws.cap_items = max_items;
  }
  if ((e = grow(&ws.bests, &ws.cap_bests, 2 * units)) != cudaSuccess) return e;
  if ((e = grow(&ws.qstats, &ws.cap_qstats, qstats)) != cudaSuccess) return e;
  if (states > 0 && (e = grow(&ws.states, &ws.cap_states, states)) != cudaSuccess) return e;
  return cudaSuccess;
}

}  // namespace

cudaError_t ws_reserve(Workspace &ws, int precision, uint32_t nq, const LaunchCfg &lc) {
  const WsNeeds w = ws_needs(precision, nq, lc);
  cudaError_t e = ws_alloc(ws, w.max_items, w.units, w.qstats, w.states);
  if (e != cudaSuccess) return e;
  ws.max_items = w.max_items;
  ws.nseg_cap = w.nseg_cap;
  ws.units_target = w.units_target;
  return cudaSuccess;
}

cudaError_t ws_reserve_upto(Workspace &ws, int precision, uint32_t max_nq, const LaunchCfg &lc) {
  size_t items = 0, units = 0, qstats = 0, states = 0;
  for (uint32_t n = 1; n <= max_nq; ++n) {  // sizing arithmetic only; one allocation per buffer
    const WsNeeds w = ws_needs(precision, n, lc);
    items = std::max(items, w.max_items);
    units = std::max(units, w.units);
    qstats = std::max(qstats, w.qstats);
    states = std::max(states, w.states);
  }
  return ws_alloc(ws, items, units, qstats, states);
}

cudaError_t ws_enqueue(Workspace &ws, int precision, const RefView &ref, const float *d_events,
                       const uint32_t *d_offsets, uint32_t nq, int raw, float *d_cost, int64_t *d_col,
                       const LaunchCfg &lc, cudaStream_t s, cudaEvent_t ev_prep, cudaEvent_t ev_sweep,
                       int64_t *d_start, bool zero_counters, cudaEvent_t ev_fix) {
  cudaError_t e;
  // (a caller that ran kernels reporting into the status word first has zeroed the counters itself)
  if (zero_counters && (e = cudaMemsetAsync(ws.ints, 0, kIntWords * sizeof(int), s)) != cudaSuccess) return e;
  if (ev_prep && (e = record_event(ev_prep, s)) != cudaSuccess) return e;
  PlanArgs pa;
  pa.offsets = d_offsets;
  pa.nq = nq;
  pa.N = ref.N;
  pa.pair = plan_mode(precision);
  const int warps = kernel_warps(precision, lc);
  pa.warps = warps;
  pa.units_target = ws.units_target;
  // Auto stacking: when the batch alone fills the unit target, or when its
  // stacked items (up to four queries each) cut into reference segments
  // (at most 64, each counted as 8,192 steps: about four warm-ups of a 16-row strip)
  // still do; small batches on short references stay unstacked for latency.
  const long seg_room = std::min<long>(kMaxSeg, ref.N / 8192);
  const bool fills = nq >= static_cast<uint32_t>(ws.units_target) ||
                     static_cast<long>(nq) * seg_room >= 4L * ws.units_target;
  pa.stack = lc.stack_short > 0 || (lc.stack_short == 0 && fills) ? 1 : 0;
  pa.nseg_cap = ws.nseg_cap;
  pa.items = ws.items;
  pa.groups = ws.groups;
  pa.ints = ws.ints;
  if ((e = launch_plan(pa, s)) != cudaSuccess) return e;
  if (raw && (e = launch_qstats(d_events, d_offsets, nq, ws.qstats, ws.ints + kIntStatus, s)) != cudaSuccess)
    return e;

  PackArgs ka;
  ka.events = d_events;
  ka.offsets = d_offsets;
  ka.items = ws.items;
  ka.n_items = ws.ints + kIntItems;
  ka.img = ws.img;
  ka.raw = raw;
  ka.qstats = ws.qstats;
  ka.pair = pa.pair;
  ka.scale_log2 = ref.scale_log2;
  ka.status = ws.ints + kIntStatus;
  if ((e = launch_pack(ka, static_cast<uint32_t>(ws.max_items), s)) != cudaSuccess) return e;

  SdtwArgs sa;
  const bool fp_ref = precision == HARU_FP32 || precision == kPrecF32Span;
  sa.ref_img = fp_ref ? static_cast<const void *>(ref.img32) : static_cast<const void *>(ref.img16);
  sa.N = ref.N;
  sa.img = ws.img;
  sa.items = ws.items;
  sa.groups = ws.groups;
  sa.ints = ws.ints;
  sa.states = ws.states;
  sa.bests = ws.bests;
  sa.bests2 = ws.bests + ws.max_items * static_cast<size_t>(ws.nseg_cap);
  sa.out_start = d_start;
  sa.nseg_cap = ws.nseg_cap;
  sa.out_cost = d_cost;
  sa.out_col = d_col;
  sa.inv_scale = 1.0f / static_cast<float>(1 << ref.scale_log2);
  sa.tile_cols = lc.tile;
  sa.warps = warps;
  sa.wait_ns = lc.wait_ns;
  const size_t groups_max = ((ws.max_items + warps - 1) / warps + kMaxS) * static_cast<size_t>(ws.nseg_cap);
  if (ev_sweep && (e = record_event(ev_sweep, s)) != cudaSuccess) return e;
  // One persistent sweep kernel over the whole group list (tallest strips
  // first), then the fix-up kernel, which verifies segments and writes every
  // query's result.
  int per_sm = lc.ctas_per_sm > 0 ? lc.ctas_per_sm : sdtw_max_ctas_per_sm(precision, lc.tile, warps);
  if (per_sm < 1) per_sm = 1;
  const int grid = static_cast<int>(std::min<size_t>(static_cast<size_t>(lc.sms) * per_sm, groups_max));
  return launch_sdtw(precision, sa, grid, static_cast<int>(ws.max_items), s, ev_fix);
}

}  // namespace haru
