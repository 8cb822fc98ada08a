// Oracle for the event detection and prefix trimming that precede the sDTW
// in HARU's software processing layer (Section 4.1: each thread detects
// events in a read's raw signal until enough are collected, drops the events
// of the read adaptor, and normalises the rest; Section 5.1 lists event
// detection, prefix trimming and normalisation as the pre-processing steps;
// Section 5.2 takes the R9.4 event detection parameters from the
// Nanopolish/f5c tool chain).
//
// TEST INFRASTRUCTURE ONLY. Plain, slow, single-threaded-per-read C++ written
// from the published method; only the test suite, the smoke check and the
// benchmark's CPU legs may load it. It shares no code, header, constant or
// helper with the CUDA library.
//
// The published detector is a two-window t-test: at every sample position i
// the w samples before i and the w samples from i on are compared by a t
// statistic, once with a short and once with a long window, and a new event
// starts where a statistic peaks above its threshold. The paper gives no
// formula or parameters; the readings used here are:
//   * samples are the raw integer ADC values of the read;
//   * t^2 = w (B - A)^2 / D for the window sums A (before i) and B (from i
//     on), with D = w (QA + QB) - A^2 - B^2 from the sums of squares QA, QB:
//     the squared difference of the window means over (v1 + v2) / w, with
//     population variances v1, v2. D is floored at 1 (a variance floor for
//     two flat windows). Defined for w <= i <= n - w;
//   * every comparison of statistics is exact: t_i > t_j is
//     num_i * den_j > num_j * den_i and t > tau is
//     10000 * num > (100 tau)^2 * den, with tau given in hundredths;
//   * a peak of a detector is a position whose statistic is above the
//     threshold, strictly above every defined statistic of the w positions
//     before it and at least every one of the w positions after it (the
//     first of equal maxima); this local-maximum test stands in for the
//     published peak-height hysteresis;
//   * boundaries are the peaks of the long window, and the peaks of the short
//     window with no long-window peak within w_short of them;
//   * event e spans samples [b_e, b_{e+1}) with b_0 = 0 and a last boundary
//     n; its value is the mean (float)((double) sum / (double) length);
//   * the query is events [trim, trim + max) (fewer if the read has fewer).
// R9.4 parameters (read from the Nanopolish/f5c defaults the paper cites):
// windows 3 and 6 samples, thresholds 1.40 and 9.00; trim 50 (Section 4.1's
// ~50 adaptor events); 250 query events.

#include <atomic>
#include <cstdint>
#include <thread>
#include <vector>

namespace {

typedef __int128 i128;

// The statistic of window w at position i as the rational num / den.
void tstat_at(const int16_t *x, long n, int w, long i, int64_t *num, int64_t *den) {
  if (i < w || i > n - w) {
    *num = 0;
    *den = 0;
    return;
  }
  int64_t A = 0, B = 0, QA = 0, QB = 0;
  for (long k = i - w; k < i; ++k) {
    A += x[k];
    QA += (int64_t)x[k] * x[k];
  }
  for (long k = i; k < i + w; ++k) {
    B += x[k];
    QB += (int64_t)x[k] * x[k];
  }
  const int64_t d = B - A;
  int64_t D = (int64_t)w * (QA + QB) - A * A - B * B;
  if (D < 1) D = 1;
  *num = (int64_t)w * d * d;
  *den = D;
}

bool greater(int64_t na, int64_t da, int64_t nb, int64_t db) { return (i128)na * db > (i128)nb * da; }

// Peaks of one detector: statistics num/den over positions 0..n.
std::vector<char> peaks(long n, int w, int tau_centi, const std::vector<int64_t> &num,
                        const std::vector<int64_t> &den) {
  std::vector<char> pk((size_t)n + 1, 0);
  const i128 tau2 = (i128)tau_centi * tau_centi;
  for (long i = 0; i <= n; ++i) {
    if (den[(size_t)i] == 0) continue;  // undefined here
    if (!((i128)10000 * num[(size_t)i] > tau2 * den[(size_t)i])) continue;
    bool ok = true;
    for (long j = i - w; j <= i + w && ok; ++j) {
      if (j < 0 || j > n || j == i || den[(size_t)j] == 0) continue;
      if (j < i) ok = greater(num[(size_t)i], den[(size_t)i], num[(size_t)j], den[(size_t)j]);
      else ok = !greater(num[(size_t)j], den[(size_t)j], num[(size_t)i], den[(size_t)i]);
    }
    pk[(size_t)i] = ok ? 1 : 0;
  }
  return pk;
}

}  // namespace

extern "C" {

// t statistics of window w at every position 0..n (num/den, 0/0 where undefined).
void oracle_event_tstat(const int16_t *x, long n, int w, int64_t *num, int64_t *den) {
  for (long i = 0; i <= n; ++i) tstat_at(x, n, w, i, &num[i], &den[i]);
}

// Event boundaries of one read (the sample positions where an event starts,
// excluding 0), ascending; returns how many (at most cap are written).
long oracle_event_boundaries(const int16_t *x, long n, int w1, int w2, int tau1_centi, int tau2_centi, long *out,
                             long cap) {
  std::vector<int64_t> n1((size_t)n + 1), d1((size_t)n + 1), n2((size_t)n + 1), d2((size_t)n + 1);
  oracle_event_tstat(x, n, w1, n1.data(), d1.data());
  oracle_event_tstat(x, n, w2, n2.data(), d2.data());
  const std::vector<char> p1 = peaks(n, w1, tau1_centi, n1, d1);
  const std::vector<char> p2 = peaks(n, w2, tau2_centi, n2, d2);
  long nb = 0;
  for (long i = 1; i < n; ++i) {
    bool b = p2[(size_t)i] != 0;
    if (!b && p1[(size_t)i]) {
      bool near_long = false;
      for (long j = i - w1; j <= i + w1; ++j)
        if (j >= 0 && j <= n && p2[(size_t)j]) near_long = true;
      b = !near_long;
    }
    if (b) {
      if (nb < cap) out[nb] = i;
      ++nb;
    }
  }
  return nb;
}

// The query of one read: events [trim, trim + max_events) as float means.
// Returns how many were written.
long oracle_read_events(const int16_t *x, long n, int w1, int w2, int tau1_centi, int tau2_centi, long trim,
                        long max_events, float *out) {
  if (n < 1) return 0;
  std::vector<long> b((size_t)n + 1);
  const long nb = oracle_event_boundaries(x, n, w1, w2, tau1_centi, tau2_centi, b.data(), n + 1);
  // event e spans [start(e), start(e + 1)), start(0) = 0, start(nb + 1) = n
  auto start = [&](long e) -> long { return e == 0 ? 0 : (e <= nb ? b[(size_t)e - 1] : n); };
  const long nev = nb + 1;
  long k = 0;
  for (long e = trim; e < nev && k < max_events; ++e, ++k) {
    const long lo = start(e), hi = start(e + 1);
    int64_t s = 0;
    for (long i = lo; i < hi; ++i) s += x[i];
    out[k] = (float)((double)s / (double)(hi - lo));
  }
  return k;
}

// Every read of a batch (samples in CSR form): out[r * max_events + e] and
// counts[r], reads spread over `threads` workers (0 = hardware count).
void oracle_signal_batch(const int16_t *samples, const uint32_t *offsets, uint32_t nreads, int w1, int w2,
                         int tau1_centi, int tau2_centi, long trim, long max_events, int threads, float *out,
                         uint32_t *counts) {
  std::atomic<uint32_t> next(0);
  auto worker = [&]() {
    for (;;) {
      const uint32_t r = next.fetch_add(1);
      if (r >= nreads) break;
      const long n = (long)offsets[r + 1] - (long)offsets[r];
      counts[r] = (uint32_t)oracle_read_events(samples + offsets[r], n, w1, w2, tau1_centi, tau2_centi, trim,
                                               max_events, out + (size_t)r * (size_t)max_events);
    }
  };
  int nt = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if ((uint32_t)nt > nreads) nt = (int)(nreads > 0 ? nreads : 1);
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto &t : pool) t.join();
}

}  // extern "C"
