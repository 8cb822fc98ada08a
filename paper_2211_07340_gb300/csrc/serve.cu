// Serving: a continuous-batching request loop for Read Until decisions.
//
// The paper's software layer (Section 4.1) collects reads from the
// sequencer, waits until a read has its 250-event prefix, normalises it and
// hands it to the sDTW accelerator, then takes the accept/eject decision
// from the alignment. Here one worker thread per context does that for
// many reads at once:
//   * submitted chunks are staged in pinned memory and, every loop turn,
//     copied to the device with one transfer and scattered by a kernel into
//     per-read device slots (a read is admitted to a slot on its first
//     chunk while the memory budget has room, otherwise it waits on the
//     host in arrival order);
//   * reads whose prefix is complete are gathered into the next batch,
//     which runs the whole device path (z-score, quantise, plan, sweep,
//     verify) on one of several batch contexts; a batch launches as soon as
//     a context is free, while earlier batches are still on the GPU;
//   * finished batches are detected by event query, decided on the host
//     (cost <= threshold) and handed to haru_stream_poll.
// A context serves either event chunks (haru_stream_submit) or raw ADC
// samples (haru_stream_submit_signal), fixed by its first submit. Samples go
// to per-read device sample slots the same way; after each upload one
// launch of the event detector covers every read with new samples and
// writes its query events into the read's event slot, counting only the
// events whose closing boundary is final (w_short + 2 w_long samples before
// the newest sample, or anywhere once the read has ended). A read is
// complete once serve_prefix final events exist, or when it ends, and then
// goes through the same batches as an event read.
// Every wait here is bounded: the loop sleeps at most 200 us between turns
// and polls events without blocking.

#include <cuda_runtime.h>
#include <pthread.h>
#include <sys/resource.h>
#include <unistd.h>
#ifdef __linux__
#include <link.h>
#endif

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdlib>
#include <cstring>
#include <list>
#include <unordered_set>

#include "engine.h"

namespace haru {
namespace {

// Voluntary and involuntary context switches and minor and major page
// faults of the calling thread so far (Linux; zeros elsewhere).
void thread_usage(long u[4]) {
#ifdef RUSAGE_THREAD
  struct rusage ru;
  if (getrusage(RUSAGE_THREAD, &ru) == 0) {
    u[0] = ru.ru_nvcsw;
    u[1] = ru.ru_nivcsw;
    u[2] = ru.ru_minflt;
    u[3] = ru.ru_majflt;
    return;
  }
#endif
  u[0] = u[1] = u[2] = u[3] = 0;
}

#ifdef __linux__
// Read one byte of every page of the executable segments of this library
// and of the runtime libraries the worker runs (CUDA driver, C and C++
// runtimes): code that a serving loop reaches for the first time mid-run
// must not wait for its pages to come from disk (a worker thread sampled
// there sat ~44 ms in the kernel's file-fault path).
int touch_code_pages(struct dl_phdr_info *info, size_t, void *arg) {
  static const char *kLibs[] = {"libharu", "libcuda.so", "libstdc++", "libc.so", "libm.so", "libgcc_s", "ld-linux"};
  const char *name = info->dlpi_name ? info->dlpi_name : "";
  bool wanted = false;
  for (const char *l : kLibs) wanted = wanted || std::strstr(name, l) != nullptr;
  if (!wanted) return 0;
  const size_t page = *static_cast<const size_t *>(arg);
  volatile unsigned char sink = 0;
  for (int i = 0; i < info->dlpi_phnum; ++i) {
    const ElfW(Phdr) &ph = info->dlpi_phdr[i];
    if (ph.p_type != PT_LOAD || !(ph.p_flags & PF_X) || !(ph.p_flags & PF_R)) continue;  // readable code only
    const unsigned char *p = reinterpret_cast<const unsigned char *>(info->dlpi_addr + ph.p_vaddr);
    for (size_t o = 0; o < ph.p_memsz; o += page) sink = static_cast<unsigned char>(sink ^ p[o]);
  }
  return 0;
}
void prefault_code() {
  const long pg = sysconf(_SC_PAGESIZE);
  size_t page = pg > 0 ? static_cast<size_t>(pg) : 4096;
  dl_iterate_phdr(touch_code_pages, &page);
}
#else
void prefault_code() {}
#endif

uint64_t now_ns() {
  return static_cast<uint64_t>(
      std::chrono::duration_cast<std::chrono::nanoseconds>(std::chrono::steady_clock::now().time_since_epoch())
          .count());
}

// Staged chunk copy: `count` events at staging[src] go to slot `slot` at `dst`.
struct CopyOp {
  uint32_t slot;
  uint32_t dst;
  uint32_t src;
  uint32_t count;
};

template <class T>
__global__ void scatter_kernel(const T *staging, const CopyOp *ops, int nops, T *slots, int slot_len) {
  const int op = blockIdx.x;
  if (op >= nops) return;
  const CopyOp o = ops[op];
  for (uint32_t i = threadIdx.x; i < o.count; i += blockDim.x)
    slots[static_cast<size_t>(o.slot) * slot_len + o.dst + i] = staging[o.src + i];
}

// Batch events from slots: request r's first len[r] events of slot[r].
__global__ void gather_kernel(const float *slots, int slot_len, const uint32_t *slot_of, const uint32_t *off,
                              int nreq, float *events) {
  const int r = blockIdx.x;
  if (r >= nreq) return;
  const uint32_t b = off[r], e = off[r + 1];
  for (uint32_t i = threadIdx.x; i < e - b; i += blockDim.x)
    events[b + i] = slots[static_cast<size_t>(slot_of[r]) * slot_len + i];
}

}  // namespace

class Server {
 public:
  explicit Server(haru_ctx *ctx) : ctx_(ctx) {}
  ~Server() { stop(); }

  int start(int mode);
  void stop();
  int mode() const { return mode_; }
  // ev: n floats (event mode) or n int16 samples (signal mode)
  int submit(uint64_t read_id, uint32_t channel, const void *ev, uint32_t n, uint64_t t_arrival, int last);
  int poll(haru_result *out, uint32_t max, uint32_t *n_out, uint32_t timeout_us);
  void stats(haru_stream_stats *out);

 private:
  struct Read {
    uint64_t id = 0;
    uint32_t channel = 0;
    std::vector<float> host;     // events not yet on the device
    uint32_t on_device = 0;      // events already in its slot
    uint32_t total = 0;          // events accepted (<= prefix)
    int slot = -1;
    bool complete = false;       // prefix complete (or read ended)
    bool queued = false;         // handed to a batch
    bool bad = false;            // non-finite event seen
    float lo = 0.0f, hi = 0.0f;  // range of the accepted events (a flat prefix has no z-score)
    uint64_t t_arrival = 0;
    uint64_t t_received = 0;
    uint64_t t_queued = 0;
    uint64_t t_launched = 0;
    // signal mode
    std::vector<int16_t> host_smp;  // samples not yet on the device
    uint32_t smp_dev = 0;           // samples in its sample slot
    uint32_t smp_total = 0;         // samples accepted (<= HARU_MAX_READ_SAMPLES)
    uint32_t smp_detected = 0;      // samples the latest finished detection covered
    bool ended = false;             // last chunk seen (or the slot is full)
    bool seen_last = false;         // the read's last chunk arrived
    bool det_pending = false;       // a detection covering it is in flight
    uint64_t t_arrival_last = 0, t_received_last = 0;  // the newest chunk's
  };
  // What a detection launch saw of a read (its result applies to that).
  struct DetSnap {
    uint64_t id;
    uint32_t len;
    bool ended;
    uint64_t t_arrival, t_received;
  };
  struct BatchCtx {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t start = nullptr;  // device time of the batch: start -> done
    cudaEvent_t done = nullptr;
    float *d_events = nullptr;
    uint32_t *d_off = nullptr;
    uint32_t *d_slot = nullptr;
    float *d_cost = nullptr;
    int64_t *d_col = nullptr;
    uint32_t *h_off = nullptr;   // pinned
    uint32_t *h_slot = nullptr;  // pinned
    float *h_cost = nullptr;     // pinned
    int64_t *h_col = nullptr;    // pinned
    int *h_status = nullptr;     // pinned
    std::vector<uint64_t> reads;
    bool busy = false;
  };

  // A chunk handed over by submit (events copied), on the intake list.
  struct Chunk {
    Chunk *next;
    uint64_t read_id;
    uint64_t t_arrival;
    uint64_t t_received;
    uint32_t channel;
    uint32_t n;
    int last;
    float ev[1];  // n events, or n int16 samples in signal mode (allocated past the struct)
  };

  void worker();
  int turn_detect();
  void reject(std::unordered_map<uint64_t, Read>::iterator it);
  void drain_intake();
  void take_chunk(const Chunk *c);
  int turn_upload();
  int turn_launch();
  int turn_complete();
  void fail(int code);

  haru_ctx *ctx_;
  std::thread thread_;
  std::atomic<bool> run_{false};
  std::mutex mu_;                       // reads_ and the queues (the worker; stats() reads them)
  std::condition_variable cv_work_;
  // submit pushes chunks here without a lock (newest first); the worker
  // takes the whole list each turn, so neither side ever waits for the other
  std::atomic<Chunk *> intake_{nullptr};
  // chunks the worker has consumed, handed back to the submitting side to be
  // freed there: the worker never frees memory the submitter allocated (a
  // free into another thread's malloc arena takes that arena's lock, and a
  // submitter descheduled inside malloc then stalls the worker)
  std::atomic<Chunk *> garbage_{nullptr};
  static void free_list(Chunk *c) {
    while (c) {
      Chunk *nx = c->next;
      std::free(c);
      c = nx;
    }
  }
  std::atomic<size_t> intake_events_{0};
  std::unordered_map<uint64_t, Read> reads_;
  // reads decided before their last chunk: later chunks are dropped, and the
  // entry goes when the last chunk arrives (a flow cell keeps delivering a
  // read's signal after the decision prefix)
  std::unordered_set<uint64_t> decided_;
  void forget(const Read &r) {  // worker, under mu_: the read leaves reads_ decided
    if (!r.seen_last) decided_.insert(r.id);
  }
  // Host buffers of finished reads, reused by new reads at full capacity:
  // in steady state the worker allocates no buffer memory and touches no
  // new pages.
  std::vector<std::vector<float>> spare_host_;
  std::vector<std::vector<int16_t>> spare_smp_;
  void retire(std::unordered_map<uint64_t, Read>::iterator it) {  // worker, under mu_
    Read &r = it->second;
    if (r.host.capacity()) {
      r.host.clear();
      spare_host_.push_back(std::move(r.host));
    }
    if (r.host_smp.capacity()) {
      r.host_smp.clear();
      spare_smp_.push_back(std::move(r.host_smp));
    }
    reads_.erase(it);
  }
  template <class T>
  static void take_buffer(std::vector<std::vector<T>> &spare, std::vector<T> &v, size_t cap) {
    if (!spare.empty()) {
      v = std::move(spare.back());
      spare.pop_back();
      return;
    }
    v.resize(cap);  // touch every page now, once
    v.clear();
  }
  std::deque<uint64_t> admit_q_;        // reads waiting for a slot
  std::deque<uint64_t> ready_q_;        // admitted reads with complete prefix, uploaded
  std::vector<int> free_slots_;
  std::atomic<size_t> host_events_{0};  // events held on the host (taken from the intake)
  std::mutex out_mu_;
  std::condition_variable cv_out_;
  // finished results, a ring under out_mu_: the worker appends (and alone
  // grows the storage), poll copies out and advances the head; no thread
  // frees memory another thread allocated
  std::vector<haru_result> out_buf_;
  size_t out_head_ = 0, out_n_ = 0;
  void push_out(const haru_result &o) {  // worker, out_mu_ held
    if (out_n_ == out_buf_.size()) {
      std::vector<haru_result> grown(std::max<size_t>(4096, 2 * out_buf_.size()));
      for (size_t i = 0; i < out_n_; ++i) grown[i] = out_buf_[(out_head_ + i) % out_buf_.size()];
      out_buf_.swap(grown);
      out_head_ = 0;
    }
    out_buf_[(out_head_ + out_n_) % out_buf_.size()] = o;
    ++out_n_;
  }
  int error_ = HARU_OK;

  // device resources
  int prefix_ = 250;
  int slot_len_ = 256;
  int nslots_ = 0;
  int max_batch_ = 1024;
  int precision_ = HARU_INT16;
  float threshold_ = 0.0f;
  float *d_slots_ = nullptr;
  float *h_stage_ = nullptr;   // pinned staging for chunk uploads
  float *d_stage_ = nullptr;
  CopyOp *h_ops_ = nullptr;    // pinned
  CopyOp *d_ops_ = nullptr;
  size_t stage_cap_ = 0;       // events per upload turn
  size_t ops_cap_ = 0;
  cudaStream_t up_stream_ = nullptr;
  cudaEvent_t up_done_ = nullptr;
  cudaStream_t det_stream_ = nullptr;  // signal mode: detection launches (not behind uploads)
  std::vector<BatchCtx> batches_;
  // per-turn scratch of the worker, kept between turns so that a turn does
  // not allocate once the vectors have grown
  std::vector<CopyOp> ops_;
  std::vector<uint64_t> finished_;
  std::vector<haru_result> res_;
  std::vector<CopyOp> ops16_;
  // signal mode: sample slots, staging, and one detection launch in flight
  int mode_ = 0;  // 0 events, 1 raw samples
  haru_event_params evp_{};
  int margin_ = 0;               // samples past a boundary before it is final: w_short + 2 w_long
  int16_t *d_smp_ = nullptr;     // [nslots][HARU_MAX_READ_SAMPLES]
  int16_t *h_stage16_ = nullptr, *d_stage16_ = nullptr;
  CopyOp *h_ops16_ = nullptr, *d_ops16_ = nullptr;
  size_t stage16_cap_ = 0;
  uint32_t *h_det_slot_ = nullptr, *h_det_len_ = nullptr, *h_det_cnt_ = nullptr;  // pinned
  int *h_det_lim_ = nullptr;
  uint32_t *d_det_slot_ = nullptr, *d_det_len_ = nullptr, *d_det_cnt_ = nullptr;
  int *d_det_lim_ = nullptr, *d_det_status_ = nullptr;
  cudaEvent_t det_done_ = nullptr;
  bool det_busy_ = false;
  std::vector<DetSnap> det_snap_;
  LaunchCfg lc_;
  RefView ref_;

  // stats
  std::atomic<uint64_t> n_submitted_{0}, n_decided_{0}, n_batches_{0}, max_batch_seen_{0}, max_conc_{0};
  // per-stage latency diagnosis (worker thread writes, stats() reads)
  std::atomic<uint64_t> max_stage_[3] = {{0}, {0}, {0}}, slow_stage_[3] = {{0}, {0}, {0}};
  std::atomic<uint64_t> max_sync_{0}, max_gap_{0};
  // device execution of the slowest batch, and the longest host-side share of
  // a batch's GPU stage (launch -> completion seen, minus device execution)
  std::atomic<uint64_t> max_exec_{0}, max_notice_{0};
  std::atomic<uint64_t> max_drain_{0};  // longest intake drain (part of the upload stage)
  // longest time in each group of CUDA calls of a turn: upload = the staged
  // copy, the scatter launch and the event record; launch = the batch's input
  // copies and gather, the device path's launches, the result copies and
  // the completion event
  std::atomic<uint64_t> max_part_[5] = {{0}, {0}, {0}, {0}, {0}};
  void note_part(int k, uint64_t dt) {
    if (dt > max_part_[k]) max_part_[k] = dt;
  }
  uint64_t spin_ns_ = 0;  // keep polling this long after the last piece of work
  std::atomic<uint64_t> worst_[9] = {};  // parts, switches and faults of the slowest turn
  std::atomic<uint64_t> worst_at_{0}, slow_turns_{0};  // its start after the loop's; turns over 5 ms
  std::atomic<uint64_t> run_faults_{0}, run_switches_{0};  // the worker's, since the loop started
  // The worker's lock acquisitions, timed: the longest wait for a lock that
  // another thread held, and the longest locked host pass of an upload turn.
  std::atomic<uint64_t> max_lock_wait_{0}, max_upload_host_{0};
  struct TimedLock {
    std::mutex &m;
    TimedLock(std::mutex &mu, std::atomic<uint64_t> &longest) : m(mu) {
      if (m.try_lock()) return;
      const uint64_t t0 = now_ns();
      m.lock();
      const uint64_t dt = now_ns() - t0;
      if (dt > longest) longest = dt;
    }
    ~TimedLock() { m.unlock(); }
    TimedLock(const TimedLock &) = delete;
    TimedLock &operator=(const TimedLock &) = delete;
  };
  void note_stage(int k, uint64_t dt) {
    if (dt > max_stage_[k]) max_stage_[k] = dt;
    if (dt > 10000000ull) slow_stage_[k]++;
  }
};

int Server::start(int mode) {
  const haru_config &c = ctx_->cfg;
  mode_ = mode;
  prefix_ = c.serve_prefix ? static_cast<int>(c.serve_prefix) : 250;
  if (prefix_ < 1 || prefix_ > HARU_MAX_QUERY) return HARU_EINVAL;
  slot_len_ = (prefix_ + 31) / 32 * 32;
  spin_ns_ = c.serve_spin_us < 0 ? 0 : 1000ull * static_cast<uint64_t>(c.serve_spin_us ? c.serve_spin_us : 2000);
  precision_ = c.serve_precision == HARU_FP32 ? HARU_FP32 : HARU_INT16;
  threshold_ = c.threshold;
  if (mode_ == 1) {
    evp_ = c.serve_events;
    if (evp_.window_short == 0 && evp_.window_long == 0) event_params_default(&evp_);
    evp_.max_events = static_cast<uint32_t>(prefix_);  // the query is the decision prefix
    if (!event_params_valid(evp_)) return HARU_EINVAL;
    margin_ = evp_.window_short + 2 * evp_.window_long;
  }
  const size_t budget = c.serve_budget_bytes ? c.serve_budget_bytes : (64u << 20);
  // an admitted read holds an event slot, and in signal mode a sample slot too
  const size_t per_slot = static_cast<size_t>(slot_len_) * sizeof(float) +
                          (mode_ == 1 ? static_cast<size_t>(HARU_MAX_READ_SAMPLES) * sizeof(int16_t) : 0);
  nslots_ = static_cast<int>(std::min<size_t>(budget / per_slot, 1u << 22));
  if (nslots_ < 1) return HARU_ENOMEM;
  // a batch holds admitted reads, one per slot: never more than the slots
  max_batch_ = static_cast<int>(
      std::min<uint64_t>(c.serve_max_batch ? c.serve_max_batch : 1024u, static_cast<uint64_t>(nslots_)));
  lc_ = ctx_->launch_cfg();
  ref_ = ctx_->ref_view();
  stage_cap_ = static_cast<size_t>(std::max(nslots_, 64)) * slot_len_;
  if (stage_cap_ > (8u << 20) / sizeof(float)) stage_cap_ = (8u << 20) / sizeof(float);
  ops_cap_ = 65536;
  cudaError_t e = cudaSetDevice(ctx_->device);
  if (e == cudaSuccess) e = cudaMalloc(&d_slots_, static_cast<size_t>(nslots_) * slot_len_ * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_stage_, stage_cap_ * sizeof(float));
  if (e == cudaSuccess) e = cudaMallocHost(&h_stage_, stage_cap_ * sizeof(float));
  if (e == cudaSuccess) e = cudaMalloc(&d_ops_, ops_cap_ * sizeof(CopyOp));
  if (e == cudaSuccess) e = cudaMallocHost(&h_ops_, ops_cap_ * sizeof(CopyOp));
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&up_stream_, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&up_done_, cudaEventDisableTiming);
  if (mode_ == 1) {
    stage16_cap_ = std::min<size_t>(static_cast<size_t>(std::max(nslots_, 64)) * 1024, (16u << 20) / sizeof(int16_t));
    const size_t nd = static_cast<size_t>(nslots_);
    if (e == cudaSuccess) e = cudaMalloc(&d_smp_, nd * HARU_MAX_READ_SAMPLES * sizeof(int16_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_stage16_, stage16_cap_ * sizeof(int16_t));
    if (e == cudaSuccess) e = cudaMallocHost(&h_stage16_, stage16_cap_ * sizeof(int16_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_ops16_, ops_cap_ * sizeof(CopyOp));
    if (e == cudaSuccess) e = cudaMallocHost(&h_ops16_, ops_cap_ * sizeof(CopyOp));
    if (e == cudaSuccess) e = cudaMallocHost(&h_det_slot_, nd * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&h_det_len_, nd * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&h_det_lim_, nd * sizeof(int));
    if (e == cudaSuccess) e = cudaMallocHost(&h_det_cnt_, nd * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_det_slot_, nd * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_det_len_, nd * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_det_lim_, nd * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&d_det_cnt_, nd * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&d_det_status_, sizeof(int));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&det_done_, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&det_stream_, cudaStreamNonBlocking);
    det_snap_.reserve(nd);
  }
  const int nb = 3;
  batches_.resize(nb);
  for (auto &b : batches_) {
    if (e != cudaSuccess) break;
    e = cudaStreamCreateWithFlags(&b.stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&b.start);
    if (e == cudaSuccess) e = cudaEventCreate(&b.done);
    if (e == cudaSuccess) e = cudaMalloc(&b.d_events, static_cast<size_t>(max_batch_) * slot_len_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_off, (max_batch_ + 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_slot, max_batch_ * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_cost, max_batch_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b.d_col, max_batch_ * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_off, (max_batch_ + 1) * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_slot, max_batch_ * sizeof(uint32_t));
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_cost, max_batch_ * sizeof(float));
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_col, max_batch_ * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMallocHost(&b.h_status, sizeof(int));
    // size the workspace for every batch size up to max_batch (segments per
    // item grow as batches shrink) so the loop never allocates
    if (e == cudaSuccess) e = ws_reserve_upto(b.ws, precision_, static_cast<uint32_t>(max_batch_), lc_);
  }
  // every kernel the loop launches, loaded now rather than inside the first requests
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, scatter_kernel<float>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, scatter_kernel<int16_t>);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, gather_kernel);
  if (e == cudaSuccess) e = load_prep_kernels();
  if (e == cudaSuccess) e = load_sdtw(precision_);
  if (e == cudaSuccess && mode_ == 1) e = load_event_kernels();
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e == cudaErrorMemoryAllocation ? HARU_ENOMEM : HARU_ECUDA;
  }
  reads_.reserve(static_cast<size_t>(std::min(2 * nslots_, 1 << 16)));
  decided_.reserve(1024);
  free_slots_.resize(nslots_);
  for (int i = 0; i < nslots_; ++i) free_slots_[i] = nslots_ - 1 - i;
  prefault_code();
  run_ = true;
  thread_ = std::thread([this] { worker(); });
  return HARU_OK;
}

void Server::stop() {
  if (run_.exchange(false)) {
    cv_work_.notify_all();
    if (thread_.joinable()) thread_.join();
  }
  free_list(intake_.exchange(nullptr));  // chunks never taken
  free_list(garbage_.exchange(nullptr));
  cudaSetDevice(ctx_->device);
  for (auto &b : batches_) {
    if (b.stream) cudaStreamSynchronize(b.stream);
    ws_free(b.ws);
    void *d[] = {b.d_events, b.d_off, b.d_slot, b.d_cost, b.d_col};
    for (void *p : d)
      if (p) cudaFree(p);
    void *h[] = {b.h_off, b.h_slot, b.h_cost, b.h_col, b.h_status};
    for (void *p : h)
      if (p) cudaFreeHost(p);
    if (b.start) cudaEventDestroy(b.start);
    if (b.done) cudaEventDestroy(b.done);
    if (b.stream) cudaStreamDestroy(b.stream);
  }
  batches_.clear();
  if (up_stream_) cudaStreamSynchronize(up_stream_);
  if (det_stream_) cudaStreamSynchronize(det_stream_);
  if (d_slots_) cudaFree(d_slots_);
  if (d_stage_) cudaFree(d_stage_);
  if (h_stage_) cudaFreeHost(h_stage_);
  if (d_ops_) cudaFree(d_ops_);
  if (h_ops_) cudaFreeHost(h_ops_);
  if (up_done_) cudaEventDestroy(up_done_);
  if (up_stream_) cudaStreamDestroy(up_stream_);
  void *dsig[] = {d_smp_, d_stage16_, d_ops16_, d_det_slot_, d_det_len_, d_det_lim_, d_det_cnt_, d_det_status_};
  for (void *q : dsig)
    if (q) cudaFree(q);
  void *hsig[] = {h_stage16_, h_ops16_, h_det_slot_, h_det_len_, h_det_lim_, h_det_cnt_};
  for (void *q : hsig)
    if (q) cudaFreeHost(q);
  if (det_done_) cudaEventDestroy(det_done_);
  if (det_stream_) cudaStreamDestroy(det_stream_);
  det_stream_ = nullptr;
  d_smp_ = d_stage16_ = h_stage16_ = nullptr;
  d_ops16_ = h_ops16_ = nullptr;
  d_det_slot_ = d_det_len_ = d_det_cnt_ = h_det_slot_ = h_det_len_ = h_det_cnt_ = nullptr;
  d_det_lim_ = d_det_status_ = h_det_lim_ = nullptr;
  det_done_ = nullptr;
  d_slots_ = d_stage_ = h_stage_ = nullptr;
  d_ops_ = h_ops_ = nullptr;
  up_done_ = nullptr;
  up_stream_ = nullptr;
}

void Server::fail(int code) {
  std::lock_guard<std::mutex> lk(out_mu_);
  if (error_ == HARU_OK) error_ = code;
  cv_out_.notify_all();
}

int Server::submit(uint64_t read_id, uint32_t channel, const void *ev, uint32_t n, uint64_t t_arrival, int last) {
  {
    std::lock_guard<std::mutex> lk(out_mu_);
    if (error_ != HARU_OK) return error_;
  }
  if (n > 0 && !ev) return HARU_EINVAL;
  // a read uses at most its first serve_prefix events (HARU_MAX_READ_SAMPLES
  // samples), so no chunk can contribute more: the rest is dropped here
  // rather than copied, and a chunk larger than the staging budget is not
  // refused as busy on every retry
  n = std::min<uint32_t>(n, mode_ == 1 ? static_cast<uint32_t>(HARU_MAX_READ_SAMPLES) : static_cast<uint32_t>(prefix_));
  free_list(garbage_.exchange(nullptr, std::memory_order_acquire));
  const size_t cap = mode_ == 1 ? stage16_cap_ : stage_cap_;
  if (intake_events_.load() + host_events_.load() + n > cap * 4) return HARU_EBUSY;
  const size_t elem = mode_ == 1 ? sizeof(int16_t) : sizeof(float);
  Chunk *c = static_cast<Chunk *>(std::malloc(offsetof(Chunk, ev) + std::max<size_t>(elem * n, sizeof(float))));
  if (!c) return HARU_ENOMEM;
  c->read_id = read_id;
  c->t_arrival = t_arrival;
  c->channel = channel;
  c->n = n;
  c->last = last;
  if (n) std::memcpy(c->ev, ev, elem * n);
  intake_events_ += n;
  c->t_received = now_ns();
  Chunk *head = intake_.load(std::memory_order_relaxed);
  do {
    c->next = head;
  } while (!intake_.compare_exchange_weak(head, c, std::memory_order_release, std::memory_order_relaxed));
  cv_work_.notify_one();
  return HARU_OK;
}

// Worker: take every chunk submitted so far, in submission order, then hand
// the chunks back to the submitting side for freeing.
void Server::drain_intake() {
  const uint64_t t0 = now_ns();
  Chunk *list = intake_.exchange(nullptr, std::memory_order_acquire);
  if (!list) return;
  Chunk *ord = nullptr, *last = list;
  while (list) {
    Chunk *nx = list->next;
    list->next = ord;
    ord = list;
    list = nx;
  }
  {
    TimedLock lk(mu_, max_lock_wait_);
    for (Chunk *c = ord; c; c = c->next) {
      take_chunk(c);
      intake_events_ -= c->n;
    }
  }
  // ord .. last is one list: push it onto the garbage list as a whole
  Chunk *head = garbage_.load(std::memory_order_relaxed);
  do {
    last->next = head;
  } while (!garbage_.compare_exchange_weak(head, ord, std::memory_order_release, std::memory_order_relaxed));
  const uint64_t dt = now_ns() - t0;
  if (dt > max_drain_) max_drain_ = dt;
}

// Worker, under mu_: decide a read without the GPU (its prefix has no
// z-score or no alignment) and drop it.
void Server::reject(std::unordered_map<uint64_t, Read>::iterator it) {
  Read &r = it->second;
  haru_result o;
  std::memset(&o, 0, sizeof(o));
  o.read_id = r.id;
  o.channel = r.channel;
  o.status = HARU_EINVAL;
  o.events = r.total;
  o.end_col = -1;
  o.t_arrival_ns = r.t_arrival;
  o.t_done_ns = now_ns();
  o.t_received_ns = r.t_received;
  host_events_ -= r.host.size() + r.host_smp.size();
  if (r.slot >= 0) free_slots_.push_back(r.slot);
  auto qi = std::find(admit_q_.begin(), admit_q_.end(), r.id);
  if (qi != admit_q_.end()) admit_q_.erase(qi);
  forget(r);
  retire(it);
  {
    TimedLock lo(out_mu_, max_lock_wait_);
    push_out(o);
  }
  n_decided_++;
  cv_out_.notify_all();
}

// Worker, under mu_: append a chunk to its read: events up to the prefix, or
// samples up to a sample slot.
void Server::take_chunk(const Chunk *c) {
  if (!decided_.empty()) {
    auto d = decided_.find(c->read_id);
    if (d != decided_.end()) {
      if (c->last) decided_.erase(d);
      return;
    }
  }
  auto it = reads_.find(c->read_id);
  if (it == reads_.end()) {
    Read r;
    r.id = c->read_id;
    r.channel = c->channel;
    if (mode_ == 1)
      take_buffer(spare_smp_, r.host_smp, HARU_MAX_READ_SAMPLES);
    else
      take_buffer(spare_host_, r.host, static_cast<size_t>(prefix_));
    it = reads_.emplace(c->read_id, std::move(r)).first;
    admit_q_.push_back(c->read_id);
    n_submitted_++;
  }
  Read &r = it->second;
  if (c->last) r.seen_last = true;
  if (r.complete) return;  // later chunks of a decided prefix are not needed
  if (mode_ == 1) {
    if (r.ended) return;
    const int16_t *smp = reinterpret_cast<const int16_t *>(c->ev);
    const uint32_t take = std::min<uint32_t>(c->n, static_cast<uint32_t>(HARU_MAX_READ_SAMPLES) - r.smp_total);
    r.host_smp.insert(r.host_smp.end(), smp, smp + take);
    host_events_ += take;
    r.smp_total += take;
    r.t_arrival_last = c->t_arrival;
    r.t_received_last = c->t_received;
    if (c->last || r.smp_total >= static_cast<uint32_t>(HARU_MAX_READ_SAMPLES)) r.ended = true;
    return;
  }
  const float *ev = c->ev;
  const uint32_t take = std::min<uint32_t>(c->n, static_cast<uint32_t>(prefix_) - r.total);
  for (uint32_t i = 0; i < take; ++i) {
    const float x = ev[i];
    if (!std::isfinite(x)) r.bad = true;
    if (r.total == 0 && i == 0) r.lo = r.hi = x;
    r.lo = std::min(r.lo, x);
    r.hi = std::max(r.hi, x);
  }
  r.host.insert(r.host.end(), ev, ev + take);
  host_events_ += take;
  r.total += take;
  if (r.total >= static_cast<uint32_t>(prefix_) || c->last) {
    r.complete = true;
    r.t_arrival = c->t_arrival;
    r.t_received = c->t_received;
    // no z-score or no alignment for this prefix: decided (eject) without the GPU
    if (r.bad || r.total < 2 || !(r.hi > r.lo) || r.total > static_cast<uint32_t>(ref_.N)) reject(it);
  }
}

int Server::poll(haru_result *out, uint32_t max, uint32_t *n_out, uint32_t timeout_us) {
  *n_out = 0;
  std::unique_lock<std::mutex> lk(out_mu_);
  if (out_n_ == 0 && error_ == HARU_OK && timeout_us > 0)
    cv_out_.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return out_n_ > 0 || error_ != HARU_OK; });
  uint32_t k = 0;
  while (k < max && out_n_ > 0) {
    out[k++] = out_buf_[out_head_];
    out_head_ = (out_head_ + 1) % out_buf_.size();
    --out_n_;
  }
  *n_out = k;
  if (k == 0 && error_ != HARU_OK) return error_;
  return HARU_OK;
}

void Server::stats(haru_stream_stats *out) {
  std::memset(out, 0, sizeof(*out));
  out->reads_submitted = n_submitted_;
  out->reads_decided = n_decided_;
  out->batches = n_batches_;
  out->max_batch = max_batch_seen_;
  out->max_concurrent = max_conc_;
  out->max_upload_ns = max_stage_[0];
  out->max_queue_ns = max_stage_[1];
  out->max_gpu_ns = max_stage_[2];
  out->slow_upload = slow_stage_[0];
  out->slow_queue = slow_stage_[1];
  out->slow_gpu = slow_stage_[2];
  out->max_upload_sync_ns = max_sync_;
  out->max_turn_gap_ns = max_gap_;
  out->max_gpu_exec_ns = max_exec_;
  out->max_notice_ns = max_notice_;
  out->max_drain_ns = max_drain_;
  out->max_upload_calls_ns = max_part_[0];
  out->max_launch_inputs_ns = max_part_[1];
  out->max_launch_path_ns = max_part_[2];
  out->max_launch_results_ns = max_part_[3];
  out->max_detect_calls_ns = max_part_[4];
  out->worst_turn_complete_ns = worst_[0];
  out->worst_turn_upload_ns = worst_[1];
  out->worst_turn_launch_ns = worst_[2];
  out->worst_turn_wait_ns = worst_[3];
  out->worst_turn_voluntary_switches = worst_[4];
  out->worst_turn_involuntary_switches = worst_[5];
  out->worst_turn_detect_ns = worst_[6];
  out->worst_turn_minor_faults = worst_[7];
  out->worst_turn_major_faults = worst_[8];
  out->worst_turn_at_ns = worst_at_;
  out->turns_over_5ms = slow_turns_;
  out->worker_minor_faults = run_faults_;
  out->worker_voluntary_switches = run_switches_;
  out->max_lock_wait_ns = max_lock_wait_;
  out->max_upload_host_ns = max_upload_host_;
  out->slots = static_cast<uint64_t>(nslots_);
  std::lock_guard<std::mutex> lk(mu_);
  out->reads_waiting = admit_q_.size();
  uint64_t inflight = 0;
  for (auto &kv : reads_)
    if (kv.second.slot >= 0) ++inflight;
  out->reads_in_flight = inflight;
}

// Admit waiting reads to free slots and copy every host-held event of an
// admitted read to its slot (one staged transfer and one scatter kernel).
int Server::turn_upload() {
  drain_intake();
  std::vector<CopyOp> &ops = ops_;
  ops.clear();
  size_t staged = 0;
  std::vector<uint64_t> &finished = finished_;
  finished.clear();
  ops16_.clear();
  const uint64_t th = now_ns();
  {
    TimedLock lk(mu_, max_lock_wait_);
    while (!admit_q_.empty() && !free_slots_.empty()) {
      Read &r = reads_[admit_q_.front()];
      admit_q_.pop_front();
      r.slot = free_slots_.back();
      free_slots_.pop_back();
    }
    for (auto &kv : reads_) {
      Read &r = kv.second;
      if (mode_ == 1) {  // raw samples to the read's sample slot
        if (r.slot < 0 || r.host_smp.empty()) continue;
        const size_t cnt = r.host_smp.size();
        if (staged + cnt > stage16_cap_ || ops16_.size() >= ops_cap_) break;
        std::memcpy(h_stage16_ + staged, r.host_smp.data(), cnt * sizeof(int16_t));
        ops16_.push_back(CopyOp{static_cast<uint32_t>(r.slot), r.smp_dev, static_cast<uint32_t>(staged),
                                static_cast<uint32_t>(cnt)});
        staged += cnt;
        r.smp_dev += static_cast<uint32_t>(cnt);
        host_events_ -= cnt;
        r.host_smp.clear();
        continue;
      }
      if (r.slot < 0 || r.host.empty()) continue;
      const size_t cnt = r.host.size();
      if (staged + cnt > stage_cap_ || ops.size() >= ops_cap_) break;
      std::memcpy(h_stage_ + staged, r.host.data(), cnt * sizeof(float));
      ops.push_back(CopyOp{static_cast<uint32_t>(r.slot), r.on_device, static_cast<uint32_t>(staged),
                           static_cast<uint32_t>(cnt)});
      staged += cnt;
      r.on_device += static_cast<uint32_t>(cnt);
      host_events_ -= cnt;
      r.host.clear();
      if (r.complete && !r.queued && r.on_device == r.total) finished.push_back(r.id);
    }
    // reads completed earlier whose events were already on the device
    for (auto &kv : reads_) {
      Read &r = kv.second;
      if (mode_ == 0 && r.slot >= 0 && r.complete && !r.queued && r.host.empty() && r.on_device == r.total &&
          std::find(finished.begin(), finished.end(), r.id) == finished.end())
        finished.push_back(r.id);
    }
  }
  {
    const uint64_t dh = now_ns() - th;
    if (dh > max_upload_host_) max_upload_host_ = dh;
  }
  if (!ops16_.empty()) {
    std::memcpy(h_ops16_, ops16_.data(), ops16_.size() * sizeof(CopyOp));
    const uint64_t tc = now_ns();
    cudaError_t e = cudaMemcpyAsync(d_stage16_, h_stage16_, staged * sizeof(int16_t), cudaMemcpyHostToDevice,
                                    up_stream_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_ops16_, h_ops16_, ops16_.size() * sizeof(CopyOp), cudaMemcpyHostToDevice, up_stream_);
    if (e == cudaSuccess) {
      scatter_kernel<int16_t><<<static_cast<unsigned>(ops16_.size()), 128, 0, up_stream_>>>(
          d_stage16_, d_ops16_, static_cast<int>(ops16_.size()), d_smp_, HARU_MAX_READ_SAMPLES);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(up_done_, up_stream_);
    note_part(0, now_ns() - tc);
    const uint64_t ts = now_ns();
    if (e == cudaSuccess) {
      while ((e = cudaEventQuery(up_done_)) == cudaErrorNotReady) {
        if (now_ns() - ts > lc_.wait_ns) return HARU_ETIMEDOUT;
      }
    }
    const uint64_t dts = now_ns() - ts;
    if (dts > max_sync_) max_sync_ = dts;
    if (e != cudaSuccess) return HARU_ECUDA;
  }
  if (!ops.empty()) {
    std::memcpy(h_ops_, ops.data(), ops.size() * sizeof(CopyOp));
    const uint64_t tc = now_ns();
    cudaError_t e = cudaMemcpyAsync(d_stage_, h_stage_, staged * sizeof(float), cudaMemcpyHostToDevice, up_stream_);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_ops_, h_ops_, ops.size() * sizeof(CopyOp), cudaMemcpyHostToDevice, up_stream_);
    if (e == cudaSuccess) {
      scatter_kernel<float><<<static_cast<unsigned>(ops.size()), 64, 0, up_stream_>>>(
          d_stage_, d_ops_, static_cast<int>(ops.size()), d_slots_, slot_len_);
      e = cudaGetLastError();
    }
    // the staging buffers are reused next turn: wait for this transfer
    if (e == cudaSuccess) e = cudaEventRecord(up_done_, up_stream_);
    note_part(0, now_ns() - tc);
    // Poll for the transfer (a few tens of microseconds) rather than block
    // in the CUDA driver; bounded by the context's wait limit.
    const uint64_t ts = now_ns();
    if (e == cudaSuccess) {
      while ((e = cudaEventQuery(up_done_)) == cudaErrorNotReady) {
        if (now_ns() - ts > lc_.wait_ns) return HARU_ETIMEDOUT;
      }
    }
    const uint64_t dts = now_ns() - ts;
    if (dts > max_sync_) max_sync_ = dts;
    if (e != cudaSuccess) return HARU_ECUDA;
  }
  if (!finished.empty()) {
    TimedLock lk(mu_, max_lock_wait_);
    const uint64_t tq = now_ns();
    for (uint64_t id : finished) {
      Read &r = reads_[id];
      if (!r.queued) {
        r.queued = true;
        r.t_queued = tq;
        ready_q_.push_back(id);
      }
    }
  }
  return HARU_OK;
}

// Signal mode: take the counts of a finished detection launch (reads with
// serve_prefix final events, or ended reads, are complete and queued), then
// launch the detector over every admitted read with samples it has not
// covered. One launch is in flight at a time; the samples it reads were
// uploaded (and waited for) before it, and later uploads write past them.
int Server::turn_detect() {
  if (mode_ != 1) return HARU_OK;
  if (det_busy_) {
    const cudaError_t q = cudaEventQuery(det_done_);
    if (q == cudaErrorNotReady) return HARU_OK;
    if (q != cudaSuccess) return HARU_ECUDA;
    det_busy_ = false;
    TimedLock lk(mu_, max_lock_wait_);
    const uint64_t tq = now_ns();
    for (size_t i = 0; i < det_snap_.size(); ++i) {
      const DetSnap &d = det_snap_[i];
      auto it = reads_.find(d.id);
      if (it == reads_.end()) continue;
      Read &r = it->second;
      r.det_pending = false;
      r.smp_detected = d.len;
      const uint32_t cnt = h_det_cnt_[i];
      if (cnt < static_cast<uint32_t>(prefix_) && !d.ended) continue;
      r.complete = true;
      r.t_arrival = d.t_arrival;
      r.t_received = d.t_received;
      r.total = cnt;
      r.on_device = cnt;
      if (cnt < 2) {
        reject(it);
        continue;
      }
      r.queued = true;
      r.t_queued = tq;
      ready_q_.push_back(r.id);
    }
  }
  uint32_t n = 0;
  {
    TimedLock lk(mu_, max_lock_wait_);
    det_snap_.clear();
    // a live read can only complete once it has (trim + prefix) events of at
    // least w_short + 1 samples each, plus the finality margin
    const uint32_t least = (evp_.trim_events + static_cast<uint32_t>(prefix_)) *
                               static_cast<uint32_t>(evp_.window_short + 1) + static_cast<uint32_t>(margin_);
    for (auto &kv : reads_) {
      Read &r = kv.second;
      if (r.slot < 0 || r.complete || r.det_pending || !r.host_smp.empty()) continue;
      const bool ended = r.ended && r.smp_dev == r.smp_total;
      if (!ended && (r.smp_dev <= r.smp_detected || r.smp_dev < least)) continue;
      h_det_slot_[n] = static_cast<uint32_t>(r.slot);
      h_det_len_[n] = r.smp_dev;
      h_det_lim_[n] = ended ? static_cast<int>(r.smp_dev) : static_cast<int>(r.smp_dev) - margin_;
      det_snap_.push_back(DetSnap{r.id, r.smp_dev, ended, r.t_arrival_last, r.t_received_last});
      r.det_pending = true;
      ++n;
    }
  }
  if (n == 0) return HARU_OK;
  // Its own stream: the next upload's wait covers that upload alone. The
  // samples read here were uploaded and waited for before this launch, and
  // the reads it completes are queued only once the host has seen det_done_.
  cudaStream_t s = det_stream_;
  const uint64_t tc = now_ns();
  cudaError_t e = cudaMemcpyAsync(d_det_slot_, h_det_slot_, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_det_len_, h_det_len_, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d_det_lim_, h_det_lim_, n * sizeof(int), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_det_status_, 0, sizeof(int), s);
  if (e == cudaSuccess)
    e = enqueue_events_slots(d_smp_, HARU_MAX_READ_SAMPLES, d_det_slot_, d_det_len_, d_det_lim_, n, evp_, d_slots_,
                             slot_len_, d_det_cnt_, d_det_status_, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_det_cnt_, d_det_cnt_, n * sizeof(uint32_t), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaEventRecord(det_done_, s);
  note_part(4, now_ns() - tc);
  if (e != cudaSuccess) return HARU_ECUDA;
  det_busy_ = true;
  return HARU_OK;
}

// Launch a batch of ready reads on a free batch context.
int Server::turn_launch() {
  for (auto &b : batches_) {
    if (b.busy) continue;
    uint32_t n = 0;
    {
      TimedLock lk(mu_, max_lock_wait_);
      if (ready_q_.empty()) return HARU_OK;
      b.reads.clear();
      b.h_off[0] = 0;
      const uint64_t tl = now_ns();
      while (!ready_q_.empty() && n < static_cast<uint32_t>(max_batch_)) {
        Read &r = reads_[ready_q_.front()];
        ready_q_.pop_front();
        r.t_launched = tl;
        b.reads.push_back(r.id);
        b.h_slot[n] = static_cast<uint32_t>(r.slot);
        b.h_off[n + 1] = b.h_off[n] + r.total;
        ++n;
      }
    }
    cudaStream_t s = b.stream;
    const uint64_t t0 = now_ns();
    cudaError_t e = cudaStreamWaitEvent(s, up_done_, 0);
    if (e == cudaSuccess) e = cudaEventRecord(b.start, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.d_off, b.h_off, (n + 1) * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.d_slot, b.h_slot, n * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
      gather_kernel<<<n, 128, 0, s>>>(d_slots_, slot_len_, b.d_slot, b.d_off, static_cast<int>(n), b.d_events);
      e = cudaGetLastError();
    }
    const uint64_t t1 = now_ns();
    if (e == cudaSuccess) e = ws_reserve(b.ws, precision_, n, lc_);
    if (e == cudaSuccess)
      e = ws_enqueue(b.ws, precision_, ref_, b.d_events, b.d_off, n, 1, b.d_cost, b.d_col, lc_, s, nullptr,
                     nullptr, nullptr);
    const uint64_t t2 = now_ns();
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.h_cost, b.d_cost, n * sizeof(float), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b.h_col, b.d_col, n * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(b.h_status, b.ws.ints + kIntStatus, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaEventRecord(b.done, s);
    const uint64_t t3 = now_ns();
    note_part(1, t1 - t0);
    note_part(2, t2 - t1);
    note_part(3, t3 - t2);
    if (e != cudaSuccess) return HARU_ECUDA;
    b.busy = true;
    n_batches_++;
    if (n > max_batch_seen_) max_batch_seen_ = n;
    uint64_t conc = 0;
    for (auto &x : batches_) conc += x.busy ? 1 : 0;
    if (conc > max_conc_) max_conc_ = conc;
  }
  return HARU_OK;
}

// Collect finished batches: decisions, latency stamps, slots freed.
int Server::turn_complete() {
  for (auto &b : batches_) {
    if (!b.busy) continue;
    cudaError_t q = cudaEventQuery(b.done);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return HARU_ECUDA;
    const uint64_t t = now_ns();
    float exec_ms = 0.0f;
    if (cudaEventElapsedTime(&exec_ms, b.start, b.done) != cudaSuccess) return HARU_ECUDA;
    const uint64_t exec_ns = static_cast<uint64_t>(static_cast<double>(exec_ms) * 1e6);
    if (exec_ns > max_exec_) max_exec_ = exec_ns;
    const int st = *b.h_status;
    const float s = static_cast<float>(1 << ref_.scale_log2);
    const float thr = precision_ == HARU_INT16 ? std::floor(threshold_ * s) / s : threshold_;
    std::vector<haru_result> &res = res_;
    res.resize(b.reads.size());
    {
      TimedLock lk(mu_, max_lock_wait_);
      for (size_t i = 0; i < b.reads.size(); ++i) {
        auto it = reads_.find(b.reads[i]);
        Read &r = it->second;
        haru_result &o = res[i];
        std::memset(&o, 0, sizeof(o));
        o.read_id = r.id;
        o.channel = r.channel;
        o.cost = b.h_cost[i];
        o.end_col = b.h_col[i];
        o.events = r.total;
        o.status = st;
        o.decision = (st == HARU_OK && o.cost <= thr) ? 1 : 0;
        o.t_arrival_ns = r.t_arrival;
        o.t_done_ns = t;
        o.t_received_ns = r.t_received;
        note_stage(0, r.t_queued - r.t_received);
        note_stage(1, r.t_launched - r.t_queued);
        note_stage(2, t - r.t_launched);
        const uint64_t stage = t - r.t_launched;
        const uint64_t host_share = stage > exec_ns ? stage - exec_ns : 0;
        if (host_share > max_notice_) max_notice_ = host_share;
        free_slots_.push_back(r.slot);
        forget(r);
        retire(it);
      }
    }
    b.busy = false;
    {
      TimedLock lk(out_mu_, max_lock_wait_);
      for (auto &o : res) push_out(o);
    }
    n_decided_ += res.size();
    cv_out_.notify_all();
  }
  return HARU_OK;
}

void Server::worker() {
#ifdef __linux__
  pthread_setname_np(pthread_self(), "haru-serve");  // findable in /proc and by debuggers
#endif
  if (cudaSetDevice(ctx_->device) != cudaSuccess) {
    fail(HARU_ECUDA);
    return;
  }
  {
    TimedLock lk(out_mu_, max_lock_wait_);  // the result ring, allocated by this thread
    if (out_buf_.empty()) out_buf_.resize(4096);
  }
  uint64_t t_prev = now_ns();
  const uint64_t t_loop = t_prev;
  long use0[4];
  thread_usage(use0);
  const long base_faults = use0[2], base_switches = use0[0];
  uint64_t part[5] = {0, 0, 0, 0, 0};
  uint64_t t_work = now_ns();  // last turn that had work
  while (run_) {
    const uint64_t t_turn = now_ns();
    long use[4];
    thread_usage(use);
    if (t_turn - t_prev > 5000000ull) slow_turns_++;
    if (t_turn - t_prev > max_gap_) {  // the previous turn was the slowest so far
      max_gap_ = t_turn - t_prev;
      worst_at_ = t_prev - t_loop;
      for (int k = 0; k < 4; ++k) worst_[k] = part[k];
      worst_[6] = part[4];
      worst_[4] = static_cast<uint64_t>(use[0] - use0[0]);
      worst_[5] = static_cast<uint64_t>(use[1] - use0[1]);
      worst_[7] = static_cast<uint64_t>(use[2] - use0[2]);
      worst_[8] = static_cast<uint64_t>(use[3] - use0[3]);
    }
    t_prev = t_turn;
    for (int k = 0; k < 4; ++k) use0[k] = use[k];
    run_faults_ = static_cast<uint64_t>(use[2] - base_faults);
    run_switches_ = static_cast<uint64_t>(use[0] - base_switches);
    int rc = turn_complete();
    const uint64_t t1 = now_ns();
    if (rc == HARU_OK) rc = turn_upload();
    const uint64_t tu = now_ns();
    if (rc == HARU_OK) rc = turn_detect();
    const uint64_t t2 = now_ns();
    if (rc == HARU_OK) rc = turn_launch();
    const uint64_t t3 = now_ns();
    if (rc != HARU_OK) {
      fail(rc);
      return;
    }
    {
      std::unique_lock<std::mutex> lk(mu_);
      bool busy = false;
      for (auto &b : batches_) busy = busy || b.busy;
      const bool work = !ready_q_.empty() || host_events_ > 0 || intake_.load() != nullptr || det_busy_;
      if (work || busy || !reads_.empty()) t_work = t3;
      // poll (no sleep) while reads are in progress or within the spin window
      if (!work && t3 - t_work >= spin_ns_)
        cv_work_.wait_for(lk, std::chrono::microseconds(busy ? 50 : 200));
    }
    part[0] = t1 - t_turn;
    part[1] = tu - t1;
    part[4] = t2 - tu;
    part[2] = t3 - t2;
    part[3] = now_ns() - t3;
  }
}

void server_destroy(Server *s) { delete s; }

}  // namespace haru

namespace {

// The context's serving loop, started in `mode` (0 events, 1 raw samples) by
// the first submit; a submit of the other kind is HARU_EINVAL.
int serve_submit(haru_ctx *ctx, int mode, uint64_t read_id, uint32_t channel, const void *data, uint32_t n,
                 uint64_t t_arrival_ns, int last_chunk) {
  if (!ctx) return HARU_EINVAL;
  haru::Server *srv = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    if (ctx->sticky) return ctx->sticky;
    if (ctx->N == 0) return HARU_ENOREF;
    if (!ctx->server) {
      auto *s = new (std::nothrow) haru::Server(ctx);
      if (!s) return HARU_ENOMEM;
      const int rc = s->start(mode);
      if (rc != HARU_OK) {
        delete s;
        return rc;
      }
      ctx->server = s;
    }
    srv = ctx->server;
  }
  if (srv->mode() != mode) return HARU_EINVAL;
  return srv->submit(read_id, channel, data, n, t_arrival_ns, last_chunk);
}

}  // namespace

extern "C" {

int haru_stream_submit(haru_ctx *ctx, uint64_t read_id, uint32_t channel, const float *events, uint32_t n,
                       uint64_t t_arrival_ns, int last_chunk) {
  return serve_submit(ctx, 0, read_id, channel, events, n, t_arrival_ns, last_chunk);
}

int haru_stream_submit_signal(haru_ctx *ctx, uint64_t read_id, uint32_t channel, const int16_t *samples, uint32_t n,
                              uint64_t t_arrival_ns, int last_chunk) {
  return serve_submit(ctx, 1, read_id, channel, samples, n, t_arrival_ns, last_chunk);
}

int haru_stream_poll(haru_ctx *ctx, haru_result *out, uint32_t max, uint32_t *n_out, uint32_t timeout_us) {
  if (!ctx || !n_out || (max > 0 && !out)) return HARU_EINVAL;
  *n_out = 0;
  haru::Server *srv = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    srv = ctx->server;
  }
  if (!srv) return HARU_OK;
  return srv->poll(out, max, n_out, timeout_us);
}

int haru_stream_get_stats(haru_ctx *ctx, haru_stream_stats *out) {
  if (!ctx || !out) return HARU_EINVAL;
  std::memset(out, 0, sizeof(*out));
  haru::Server *srv = nullptr;
  {
    std::lock_guard<std::mutex> lk(ctx->mu);
    srv = ctx->server;
  }
  if (srv) srv->stats(out);
  return HARU_OK;
}

}  // extern "C"
