// Host-side structures shared by the C ABI (api.cu), the batch engine
// (batch.cu) and the serving loop (serve.cu).
#pragma once

#include <cuda_runtime.h>

#include <atomic>
#include <condition_variable>
#include <cstdint>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "haru_internal.h"

namespace haru {

template <class T>
cudaError_t grow(T **p, size_t *cap, size_t need) {
  if (*cap >= need && *p) return cudaSuccess;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  const size_t n = need > 1 ? need : 1;
  cudaError_t e = cudaMalloc(reinterpret_cast<void **>(p), n * sizeof(T));
  if (e == cudaSuccess) *cap = n;
  return e;
}

// Launch settings derived from a context's configuration.
struct LaunchCfg {
  int warps = 8;
  int tile = 4096;
  int ctas_per_sm = 0;
  int sms = 1;
  int units_target = 0;  // 0: 4 x sms x warps
  int stack_short = 0;   // stack short queries: 0 auto (batch >= units target), 1 always, -1 never
  unsigned long long wait_ns = 2000000000ull;
};

// Warps per CTA that the kernels of `precision` run: the start-column forms
// hold over 200 registers a thread and launch at most 8 warps; the others fit
// 12 warps (3 per scheduler) in an SM's register file.
inline int kernel_warps(int precision, const LaunchCfg &lc) {
  return prec_span(precision) && lc.warps > 8 ? 8 : lc.warps;
}

// Planner mode of a batch: 0 FP32, 1 int16 pairs, 3 int16 inputs with wide
// accumulation (one exact strip per query).
inline int plan_mode(int precision) {
  if (precision == HARU_INT16_ACC32 || precision == kPrecWideSpan) return 3;
  return precision == HARU_INT16 ? 1 : 0;
}

// Most items a batch of nq queries can make in `mode` (per-bucket rounding
// included: each strip height has a plain and a stacked bucket).
inline size_t items_bound(int mode, size_t nq) {
  if (mode == 0 || mode == 3) return nq + kMaxS;
  return (nq + 1) / 2 + 2 * kMaxS;
}

// The reference as the kernels read it.
struct RefView {
  const uint32_t *img16 = nullptr;
  const float *img32 = nullptr;
  long N = 0;
  int scale_log2 = 6;
};

// Device scratch of one batch in flight: status/counter words, planner
// output, packed query images, segment states and per-unit minima.
struct Workspace {
  int *ints = nullptr;
  Item *items = nullptr;
  Group *groups = nullptr;
  uint32_t *img = nullptr;
  size_t cap_items = 0;
  uint32_t *states = nullptr;
  size_t cap_states = 0;
  Best *bests = nullptr;  // 2 x units: upper stacks, then lower stacks
  size_t cap_bests = 0;
  double *qstats = nullptr;  // per query (mean, sigma) of raw batches
  size_t cap_qstats = 0;
  // plan of the last reservation
  size_t max_items = 0;
  int nseg_cap = 1;
  int units_target = 0;
};

// Size `ws` for a batch of nq queries (allocates only when it must grow).
cudaError_t ws_reserve(Workspace &ws, int precision, uint32_t nq, const LaunchCfg &lc);
// Size `ws` for every batch of 1..max_nq queries at once, so that later
// ws_reserve calls for such batches never allocate.
cudaError_t ws_reserve_upto(Workspace &ws, int precision, uint32_t max_nq, const LaunchCfg &lc);
void ws_free(Workspace &ws);

// Enqueue the whole batch path on stream s: zero the counters, plan, pack
// (z-score and quantise when raw), sweep, verify segments and write (cost,
// column) per query. ev_prep/ev_sweep (optional) are recorded after the
// counters are zeroed and after packing.
cudaError_t ws_enqueue(Workspace &ws, int precision, const RefView &ref, const float *d_events,
                       const uint32_t *d_offsets, uint32_t nq, int raw, float *d_cost, int64_t *d_col,
                       const LaunchCfg &lc, cudaStream_t s, cudaEvent_t ev_prep, cudaEvent_t ev_sweep,
                       int64_t *d_start = nullptr, bool zero_counters = true, cudaEvent_t ev_fix = nullptr);

// Event detection (events.cu): parameter defaults and checks, and the
// stream-ordered detection of nreads raw-signal reads: strided events and
// per-read counts, then CSR offsets (nreads + 1) and CSR events.
void event_params_default(haru_event_params *p);
bool event_params_valid(const haru_event_params &p);
cudaError_t enqueue_events(const int16_t *d_samples, const uint32_t *d_soff, uint32_t nreads,
                           const haru_event_params &p, float *strided, uint32_t *counts, uint32_t *ev_off,
                           float *ev_csr, int *status, cudaStream_t s);
// Detection over serving slots: read r's len[r] samples in slot slot[r]
// (sample_stride per slot), its query events to event slot slot[r]
// (event_stride floats per slot), counts[r] = events whose closing boundary
// is at or before final_limit[r].
cudaError_t enqueue_events_slots(const int16_t *samples, int sample_stride, const uint32_t *slot, const uint32_t *len,
                                 const int *final_limit, uint32_t nreads, const haru_event_params &p, float *events,
                                 int event_stride, uint32_t *counts, int *status, cudaStream_t s);
// Load the detection kernels into the current context now (see load_sdtw).
cudaError_t load_event_kernels();

// Record `e` on `s`; inside a stream capture, as an external event node so
// its time can be read after every replay.
cudaError_t record_event(cudaEvent_t e, cudaStream_t s);

class Server;  // serve.cu
void server_destroy(Server *s);

}  // namespace haru

struct haru_ctx {
  int device = 0;
  haru_config cfg{};
  cudaStream_t stream = nullptr;
  int sms = 0;
  int sticky = HARU_OK;
  int last_status = HARU_OK;
  std::mutex mu;

  // reference store
  size_t N = 0;
  int scale_log2 = 6;
  float *ref_z = nullptr;       // N
  uint32_t *img16 = nullptr;    // N + kRefPad, packed (q, q)
  float *img32 = nullptr;       // N + kRefPad
  double *stats = nullptr;      // mean, sigma
  double *partials = nullptr;
  size_t partials_cap = 0;

  // batch path
  haru::Workspace ws;
  float *d_events = nullptr;
  size_t cap_events = 0;
  uint32_t *d_offsets = nullptr;
  float *d_cost = nullptr;
  int64_t *d_col = nullptr;
  int64_t *d_start = nullptr;
  size_t cap_q = 0;

  // raw-signal path (signal.cu): staged samples and offsets, detected events
  int16_t *d_samples = nullptr;
  size_t cap_samples = 0;
  uint32_t *d_soff = nullptr;
  size_t cap_soff = 0;
  float *sig_strided = nullptr;
  size_t cap_strided = 0;
  float *sig_events = nullptr;
  size_t cap_sig_events = 0;
  uint32_t *sig_counts = nullptr;
  size_t cap_sig_counts = 0;
  uint32_t *sig_off = nullptr;
  size_t cap_sig_off = 0;
  cudaEvent_t ev[4] = {nullptr, nullptr, nullptr, nullptr};  // HARU_PROFILE: prep, sweep, end, fix-up
  bool profiled = false;

  // serving (serve.cu): created by the first haru_stream_submit
  haru::Server *server = nullptr;

  haru::LaunchCfg launch_cfg() const;
  haru::RefView ref_view() const;
};
