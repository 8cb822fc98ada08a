// Event detection on the device: the pre-processing of HARU's software layer
// (Section 4.1; Section 5.1 lists event detection, prefix trimming and
// normalisation) turned into kernels, so that raw samples go in and the
// existing z-score / quantise / sDTW path runs on their events.
//
// The detector is the two-window t-test of the Nanopolish/f5c tool chain
// that Section 5.2 names (R9.4 defaults: windows 3 and 6 samples,
// thresholds 1.40 and 9.00). At sample position i the w samples before i and
// the w samples from i on give
//   t^2 = w (B - A)^2 / max(1, w (QA + QB) - A^2 - B^2)
// for their sums A, B and sums of squares QA, QB (the squared difference of
// the window means over (v1 + v2) / w with population variances), defined
// for w <= i <= n - w. Statistics are compared as exact rationals (128-bit
// cross products), never rounded: a peak of a window is a position above the
// window's threshold, strictly above the w statistics before it and at least
// the w after it; boundaries are the long window's peaks and the short
// window's peaks with no long-window peak within w_short. Event e spans
// [b_e, b_{e+1}) (b_0 = 0, last b = n) and its value is the mean
// (float)((double) sum / length). A read's query is events
// [trim, trim + max_events).
//
// Kernels: detect_kernel (one CTA per read: the read's samples in shared
// memory, statistics over tiles of kEvTile positions with halos, each thread
// sliding its window sums along a run of positions; peaks compared on float
// t^2 values with a margin that covers their rounding, falling back to the
// exact integers when it cannot decide; an ordered block-wide compaction of
// boundaries that stops once the query's boundaries are known; then the
// event means), scan_kernel (CSR offsets of the per-read event counts) and
// compact_kernel (strided -> CSR).

#include <cuda_runtime.h>

#include <cstring>

#include "engine.h"

namespace haru {
namespace {

constexpr int kEvThreads = 256;
constexpr int kEvTile = 1024;                      // boundary positions per tile
constexpr int kEvPer = kEvTile / kEvThreads;       // consecutive positions per thread
constexpr int kEvMaxW = 16;                        // longest window
constexpr int kEvTpos = kEvTile + 4 * kEvMaxW;     // statistics per tile (halo w1 + w2 on each side)
constexpr int kEvRun = (kEvTpos + kEvThreads - 1) / kEvThreads;  // statistics per thread (a contiguous run)
constexpr int kEvLp = kEvTile + 2 * kEvMaxW;       // long-peak flags per tile (halo w1 on each side)
static_assert(kEvTile % kEvThreads == 0 && kEvPer <= 32, "tile split");

// Shared-memory layout of detect_kernel (bytes); the boundary list follows,
// as many ints as the query needs (trim + max_events).
constexpr size_t kSmX = 0;                                                  // int16 samples
constexpr size_t kSmT = kSmX + HARU_MAX_READ_SAMPLES * sizeof(int16_t);     // 2 x kEvTpos float t^2
constexpr size_t kSmLp = kSmT + 2 * kEvTpos * sizeof(float);
constexpr size_t kSmBounds = kSmLp + (kEvLp + 15) / 16 * 16;
size_t detect_smem_bytes(int need) { return kSmBounds + static_cast<size_t>(need) * sizeof(int); }

struct EvArgs {
  const int16_t *samples;
  const uint32_t *offsets;  // nreads + 1
  uint32_t nreads;
  int w1, w2;
  unsigned long long tau1sq, tau2sq;  // (100 tau)^2
  float tau1f, tau2f;                 // tau^2 as floats (for the fast path)
  int trim, maxev;
  float *out;        // [nreads][maxev] (CSR mode) or the event slots (slot mode)
  uint32_t *counts;  // nreads
  int *status;
  // Slot mode (serving; slot != nullptr): read r's samples are
  // samples[slot[r] * sample_stride ...] (len[r] of them), its events go to
  // out[slot[r] * out_stride ...], and only events whose closing boundary
  // lies at or before final_limit[r] are counted (a live read's later
  // boundaries can still move as samples arrive).
  const uint32_t *slot;
  const uint32_t *len;
  const int *final_limit;
  int sample_stride, out_stride;
};

// a * b > c * d for 64-bit factors (128-bit products): every product of a
// statistic's numerator (< 2^45) or denominator (< 2^40) with another, or
// with a squared threshold.
__device__ __forceinline__ bool mul_gt(unsigned long long a, unsigned long long b, unsigned long long c,
                                       unsigned long long d) {
  const unsigned long long h1 = __umul64hi(a, b), h2 = __umul64hi(c, d);
  return h1 > h2 || (h1 == h2 && a * b > c * d);
}

// Window sums at position i: A, QA over [i - w, i), B, QB over [i, i + w).
struct Win {
  long long A, B, QA, QB;
  __device__ __forceinline__ void direct(const int16_t *x, int w, int i) {
    A = B = QA = QB = 0;
    for (int k = i - w; k < i; ++k) {
      const int v = x[k];
      A += v;
      QA += v * v;
    }
    for (int k = i; k < i + w; ++k) {
      const int v = x[k];
      B += v;
      QB += v * v;
    }
  }
  // from position i - 1 to i
  __device__ __forceinline__ void slide(const int16_t *x, int w, int i) {
    const int in_l = x[i - 1], out_l = x[i - 1 - w], in_r = x[i + w - 1];
    A += in_l - out_l;
    QA += in_l * in_l - out_l * out_l;
    B += in_r - in_l;
    QB += in_r * in_r - in_l * in_l;
  }
  // t^2 = num / den (exact integers)
  __device__ __forceinline__ void stat(int w, unsigned long long *num, unsigned long long *den) const {
    const long long d = B - A;
    long long D = static_cast<long long>(w) * (QA + QB) - A * A - B * B;
    if (D < 1) D = 1;
    *num = static_cast<unsigned long long>(static_cast<long long>(w) * d * d);
    *den = static_cast<unsigned long long>(D);
  }
};

// t^2 of window w at position i, exactly (for the rare comparisons the
// float values cannot decide).
__device__ __noinline__ void exact_stat(const int16_t *x, int w, int i, unsigned long long *num,
                                        unsigned long long *den) {
  Win s;
  s.direct(x, w, i);
  s.stat(w, num, den);
}

// The float t^2 of a statistic carries a relative error below 2^-21 (the
// numerator and denominator each rounded once to float, one correctly
// rounded division), so two of them decide a comparison of the exact values
// whenever they differ by more than the margin; otherwise the comparison is
// redone on the exact integers.
constexpr float kMarginUp = 1.0f + 1.0f / 262144.0f, kMarginDown = 1.0f - 1.0f / 262144.0f;  // 2^-18

// t_i > t_j for positions qi, qj of window w (tf_* their float t^2, >= 0).
__device__ __forceinline__ bool t_greater(const int16_t *x, int w, int qi, float ti, int qj, float tj) {
  if (ti > tj * kMarginUp) return true;
  if (ti < tj * kMarginDown) return false;
  unsigned long long ni, di, nj, dj;
  exact_stat(x, w, qi, &ni, &di);
  exact_stat(x, w, qj, &nj, &dj);
  return mul_gt(ni, dj, nj, di);
}

// t_i > tau, i.e. 10000 num > (100 tau)^2 den.
__device__ __forceinline__ bool t_above(const int16_t *x, int w, int qi, float ti, float tauf,
                                        unsigned long long tausq) {
  if (ti > tauf * kMarginUp) return true;
  if (ti < tauf * kMarginDown) return false;
  unsigned long long ni, di;
  exact_stat(x, w, qi, &ni, &di);
  return mul_gt(ni, 10000ull, di, tausq);
}

// Peak test of statistic index j (position q) of a tile: above the threshold,
// strictly above the w defined statistics before it, at least the w after
// it. Undefined statistics hold -1. The caller keeps j - w >= 0 and
// j + w < kEvTpos.
__device__ __forceinline__ bool peak(const int16_t *x, const float *tf, int j, int q, int w, float tauf,
                                     unsigned long long tausq) {
  const float tj = tf[j];
  if (tj < 0.0f || !t_above(x, w, q, tj, tauf, tausq)) return false;
  for (int k = 1; k <= w; ++k) {
    const float tl = tf[j - k];
    if (tl >= 0.0f && !t_greater(x, w, q, tj, q - k, tl)) return false;  // need t_q > t_{q-k}
    const float tr = tf[j + k];
    if (tr >= 0.0f && t_greater(x, w, q + k, tr, q, tj)) return false;   // need t_{q+k} <= t_q
  }
  return true;
}

// Statistics of window w at positions q = p0 - H + j for this thread's run
// of j, sliding the window sums along the run.
__device__ __forceinline__ void tile_stats(const int16_t *x, int n, int w, int p0, int H, int jmax, float *tf) {
  Win s;
  bool have = false;
#pragma unroll
  for (int r = 0; r < kEvRun; ++r) {
    const int j = threadIdx.x * kEvRun + r;
    if (j >= jmax) break;
    const int q = p0 - H + j;
    if (q < w || q > n - w) {
      tf[j] = -1.0f;
      have = false;
      continue;
    }
    if (have)
      s.slide(x, w, q);
    else
      s.direct(x, w, q);
    have = true;
    unsigned long long num, den;
    s.stat(w, &num, &den);
    tf[j] = __fdiv_rn(__ull2float_rn(num), __ull2float_rn(den));
  }
}

// Four CTAs per SM (shared memory ~44 KB each with the default parameters).
__global__ void __launch_bounds__(kEvThreads, 4) detect_kernel(EvArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  int16_t *x = reinterpret_cast<int16_t *>(sm + kSmX);
  float *t1 = reinterpret_cast<float *>(sm + kSmT), *t2 = t1 + kEvTpos;
  unsigned char *lp = sm + kSmLp;
  int *bounds = reinterpret_cast<int *>(sm + kSmBounds);
  __shared__ int warp_tot[kEvThreads / 32];
  __shared__ int s_nb;
  const uint32_t r = blockIdx.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  size_t base;
  long len;
  float *out_row;
  if (a.slot) {
    base = static_cast<size_t>(a.slot[r]) * a.sample_stride;
    len = a.len[r];
    out_row = a.out + static_cast<size_t>(a.slot[r]) * a.out_stride;
  } else {
    base = a.offsets[r];
    len = static_cast<long>(a.offsets[r + 1]) - static_cast<long>(base);
    out_row = a.out + static_cast<size_t>(r) * a.maxev;
  }
  if (len < 0 || len > HARU_MAX_READ_SAMPLES) {
    if (tid == 0) {
      report(a.status, HARU_EINVAL);
      a.counts[r] = 0;
    }
    return;
  }
  const int n = static_cast<int>(len);
  for (int i = tid; i < n; i += kEvThreads) x[i] = a.samples[base + i];
  if (tid == 0) s_nb = 0;
  __syncthreads();
  const int w1 = a.w1, w2 = a.w2, H = w1 + w2;
  const int need = a.trim + a.maxev;  // boundaries b_1 .. b_need close the query's last event
  for (int p0 = 0; p0 < n; p0 += kEvTile) {
    // statistics at positions q = p0 - H + j, j in [0, kEvTile + 2H)
    tile_stats(x, n, w1, p0, H, kEvTile + 2 * H, t1);
    tile_stats(x, n, w2, p0, H, kEvTile + 2 * H, t2);
    __syncthreads();
    // long-window peaks at q = p0 - w1 + j, j in [0, kEvTile + 2 w1) (statistic index j + w2)
    for (int j = tid; j < kEvTile + 2 * w1; j += kEvThreads)
      lp[j] = peak(x, t2, j + w2, p0 - w1 + j, w2, a.tau2f, a.tau2sq) ? 1 : 0;
    __syncthreads();
    // boundaries among this thread's positions p0 + tid * kEvPer + u
    unsigned flags = 0;
    int cnt = 0;
#pragma unroll
    for (int u = 0; u < kEvPer; ++u) {
      const int p = p0 + tid * kEvPer + u;
      if (p < 1 || p > n - 1) continue;
      const int jl = p - p0 + w1;  // its long-peak flag
      bool b = lp[jl] != 0;
      if (!b && peak(x, t1, p - p0 + H, p, w1, a.tau1f, a.tau1sq)) {
        bool near = false;
        for (int k = -w1; k <= w1; ++k) near = near || lp[jl + k] != 0;
        b = !near;
      }
      if (b) {
        flags |= 1u << u;
        ++cnt;
      }
    }
    // ordered compaction: exclusive prefix of cnt over the block; only the
    // first `need` boundaries are kept (the query uses b_1 .. b_need)
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int before = 0, total = 0;
#pragma unroll
    for (int w = 0; w < kEvThreads / 32; ++w) {
      const int t = warp_tot[w];
      before += w < warp ? t : 0;
      total += t;
    }
    int pos = s_nb + before + incl - cnt;
#pragma unroll
    for (int u = 0; u < kEvPer; ++u)
      if (flags & (1u << u)) {
        if (pos < need) bounds[pos] = p0 + tid * kEvPer + u;
        ++pos;
      }
    __syncthreads();
    if (tid == 0) s_nb += total;
    __syncthreads();
    if (s_nb >= need) break;  // uniform: every thread reads the same s_nb
  }
  const int nb = s_nb;
  int K = n > 0 ? nb + 1 - a.trim : 0;  // events after the trim (an empty read has none)
  K = K < 0 ? 0 : (K > a.maxev ? a.maxev : K);
  if (a.final_limit) {  // slot mode: keep the events whose closing boundary is final
    const int lim = a.final_limit[r];
    while (K > 0) {
      const int e = a.trim + K - 1;
      if ((e + 1 <= nb ? bounds[e] : n) <= lim) break;
      --K;
    }
  }
  for (int k = tid; k < K; k += kEvThreads) {
    const int e = a.trim + k;  // e + 1 <= need: both ends are stored boundaries (or 0, n)
    const int lo = e == 0 ? 0 : bounds[e - 1];
    const int hi = e + 1 <= nb ? bounds[e] : n;
    long long s = 0;
    for (int i = lo; i < hi; ++i) s += x[i];
    out_row[k] = __double2float_rn(__ddiv_rn(static_cast<double>(s), static_cast<double>(hi - lo)));
  }
  if (tid == 0) a.counts[r] = static_cast<uint32_t>(K);
}

// CSR offsets of the per-read event counts (one CTA).
__global__ void __launch_bounds__(1024) scan_kernel(const uint32_t *counts, uint32_t nreads, uint32_t *offsets) {
  __shared__ uint32_t warp_tot[32];
  __shared__ uint32_t carry;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  if (tid == 0) {
    carry = 0;
    offsets[0] = 0;
  }
  __syncthreads();
  for (uint32_t b = 0; b < nreads; b += 1024) {
    const uint32_t r = b + tid;
    const uint32_t c = r < nreads ? counts[r] : 0u;
    uint32_t incl = c;
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t before = 0, total = 0;
    for (int w = 0; w < 32; ++w) {
      before += w < warp ? warp_tot[w] : 0u;
      total += warp_tot[w];
    }
    if (r < nreads) offsets[r + 1] = carry + before + incl;
    __syncthreads();
    if (tid == 0) carry += total;
    __syncthreads();
  }
}

// Strided per-read events -> CSR (one warp per read).
__global__ void compact_kernel(const float *strided, int maxev, const uint32_t *counts, const uint32_t *offsets,
                               uint32_t nreads, float *csr) {
  const uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (r >= nreads) return;
  const int lane = threadIdx.x & 31;
  const uint32_t c = counts[r], o = offsets[r];
  for (uint32_t i = lane; i < c; i += 32) csr[o + i] = strided[static_cast<size_t>(r) * maxev + i];
}

}  // namespace

// Fill defaults (R9.4 readings).
void event_params_default(haru_event_params *p) {
  std::memset(p, 0, sizeof(*p));
  p->window_short = 3;
  p->window_long = 6;
  p->threshold_short_centi = 140;
  p->threshold_long_centi = 900;
  p->trim_events = 50;
  p->max_events = 250;
}

bool event_params_valid(const haru_event_params &p) {
  return p.window_short >= 2 && p.window_long >= p.window_short && p.window_long <= kEvMaxW &&
         p.threshold_short_centi >= 1 && p.threshold_short_centi <= 10000 && p.threshold_long_centi >= 1 &&
         p.threshold_long_centi <= 10000 && p.trim_events <= HARU_MAX_READ_SAMPLES && p.max_events >= 1 &&
         p.max_events <= HARU_MAX_QUERY;
}

static SmemOptIn detect_opt_in;  // the detection kernel's dynamic shared memory, per device

cudaError_t load_event_kernels() {
  cudaFuncAttributes f;
  cudaError_t e = cudaFuncGetAttributes(&f, detect_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&f, scan_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&f, compact_kernel);
  return e;
}

// Enqueue detection of nreads reads on s: strided events and counts, then
// CSR offsets and events (ev_csr holds up to nreads * max_events floats).
cudaError_t enqueue_events(const int16_t *d_samples, const uint32_t *d_soff, uint32_t nreads,
                           const haru_event_params &p, float *strided, uint32_t *counts, uint32_t *ev_off,
                           float *ev_csr, int *status, cudaStream_t s) {
  if (nreads == 0) return cudaSuccess;
  const int need = static_cast<int>(p.trim_events + p.max_events);
  const size_t smem = detect_smem_bytes(need);
  cudaError_t e = opt_in_smem(detect_kernel, detect_opt_in, smem);
  if (e != cudaSuccess) return e;
  EvArgs a;
  a.samples = d_samples;
  a.offsets = d_soff;
  a.nreads = nreads;
  a.w1 = p.window_short;
  a.w2 = p.window_long;
  a.tau1sq = static_cast<unsigned long long>(p.threshold_short_centi) * p.threshold_short_centi;
  a.tau2sq = static_cast<unsigned long long>(p.threshold_long_centi) * p.threshold_long_centi;
  a.tau1f = static_cast<float>(a.tau1sq) / 10000.0f;
  a.tau2f = static_cast<float>(a.tau2sq) / 10000.0f;
  a.trim = static_cast<int>(p.trim_events);
  a.maxev = static_cast<int>(p.max_events);
  a.out = strided;
  a.counts = counts;
  a.status = status;
  a.slot = nullptr;
  a.len = nullptr;
  a.final_limit = nullptr;
  a.sample_stride = a.out_stride = 0;
  detect_kernel<<<nreads, kEvThreads, smem, s>>>(a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  scan_kernel<<<1, 1024, 0, s>>>(counts, nreads, ev_off);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  compact_kernel<<<(nreads + 7) / 8, 256, 0, s>>>(strided, a.maxev, counts, ev_off, nreads, ev_csr);
  return cudaGetLastError();
}

// Detection over serving slots (one launch for every read with new samples):
// read r = 0..nreads-1 has len[r] samples in slot slot[r] of `samples`
// (sample_stride per slot); its query events go to slot slot[r] of `events`
// (event_stride floats per slot) and counts[r] is how many of them are
// final (closing boundary at or before final_limit[r]).
cudaError_t enqueue_events_slots(const int16_t *samples, int sample_stride, const uint32_t *slot, const uint32_t *len,
                                 const int *final_limit, uint32_t nreads, const haru_event_params &p, float *events,
                                 int event_stride, uint32_t *counts, int *status, cudaStream_t s) {
  if (nreads == 0) return cudaSuccess;
  const int need = static_cast<int>(p.trim_events + p.max_events);
  const size_t smem = detect_smem_bytes(need);
  cudaError_t e = opt_in_smem(detect_kernel, detect_opt_in, smem);
  if (e != cudaSuccess) return e;
  EvArgs a;
  a.samples = samples;
  a.offsets = nullptr;
  a.nreads = nreads;
  a.w1 = p.window_short;
  a.w2 = p.window_long;
  a.tau1sq = static_cast<unsigned long long>(p.threshold_short_centi) * p.threshold_short_centi;
  a.tau2sq = static_cast<unsigned long long>(p.threshold_long_centi) * p.threshold_long_centi;
  a.tau1f = static_cast<float>(a.tau1sq) / 10000.0f;
  a.tau2f = static_cast<float>(a.tau2sq) / 10000.0f;
  a.trim = static_cast<int>(p.trim_events);
  a.maxev = static_cast<int>(p.max_events);
  a.out = events;
  a.counts = counts;
  a.status = status;
  a.slot = slot;
  a.len = len;
  a.final_limit = final_limit;
  a.sample_stride = sample_stride;
  a.out_stride = event_stride;
  detect_kernel<<<nreads, kEvThreads, smem, s>>>(a);
  return cudaGetLastError();
}

}  // namespace haru
