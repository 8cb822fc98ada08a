// Oracle for subsequence DTW (sDTW) as used by HARU's Read Until.
//
// TEST INFRASTRUCTURE ONLY. This file is a plain, slow, single-threaded-per-
// query CPU restatement of the method, written from the paper. Only the test
// suite, the smoke check and the benchmark's CPU-baseline leg may load it. It
// shares no code, header, constant or helper with the CUDA library.
//
// What it computes (paper sections):
//   * Eq. 1 (Section 2.3): gamma(i,j) = delta(i,j) + min(gamma(i-1,j),
//     gamma(i-1,j-1), gamma(i,j-1)), boundaries gamma(i,0) = inf for i >= 1 and
//     gamma(0,j) = 0 for j >= 0 (free start), delta = |x_i - y_j| (Manhattan,
//     the distance of the HARU processing elements, Section 4.3).
//   * Algorithm 1 (Section 2.3): the full M x N cost matrix, then the minimum
//     of the last row; the scan keeps the first column on ties (strict "<").
//   * Algorithm 2 (Section 4.3): the same result with one cost array of M+1
//     entries swept column by column.
//   * Section 4.1: reference = k-mer model levels of the forward strand
//     followed by those of the reverse complement; z-score normalisation of
//     the reference and of every query; fixed-point scaling by a power of two.
//
// Readings where the paper is silent:
//   * z-score: population standard deviation; mean and variance accumulated in
//     double, in blocks of 4096 consecutive samples summed in index order, the
//     block sums added in index order; z = (float)((x - mean) / sigma);
//     sigma == 0 is an error.
//   * quantiser: q = clamp(round_half_even(z * 2^k), -2047, 2047) with the
//     product formed in float (exact for a power of two).
//   * int16 form: costs saturate at CAP = 32767 - 2*2047 = 28673, which also
//     stands for infinity: gamma = min(CAP, delta + min3(...)).
//   * end column: 0-based index into the concatenated reference; ties go to
//     the smallest column.
//   * wide accumulation (the PE of Section 4.3: 16-bit samples, 32-bit cost
//     registers): the exact integer DP of the quantised samples, unsaturated.
//   * start column (the paper drops backtracking): carried forward; among
//     minimum-cost predecessors a cell keeps the up one's start, else the
//     diagonal one's, else the left one's; a path entering row 1 at column j
//     starts at j.
//
// Parity pins live in tests/ (brute-force path enumeration, exact copies,
// closed-form special cases, bounds, algorithm equivalences).

#include <atomic>
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <limits>
#include <thread>
#include <type_traits>
#include <vector>

namespace {

const int kQmax = 2047;
const int kCap = 32767 - 2 * kQmax;  // 28673
const size_t kZBlock = 4096;

inline double dmin3(double a, double b, double c) {
  double m = a < b ? a : b;
  return m < c ? m : c;
}
inline float fmin3_(float a, float b, float c) {
  float m = a < b ? a : b;
  return m < c ? m : c;
}
inline int32_t imin3(int32_t a, int32_t b, int32_t c) {
  int32_t m = a < b ? a : b;
  return m < c ? m : c;
}

}  // namespace

extern "C" {

int oracle_cap(void) { return kCap; }
int oracle_qmax(void) { return kQmax; }

// ---------------------------------------------------------------- z-score --
// Section 4.1: (x - mean) / sigma over the whole sequence.
int oracle_zscore(const float *x, size_t n, float *z) {
  if (n == 0) return -1;
  double sum = 0.0;
  for (size_t b = 0; b < n; b += kZBlock) {
    size_t e = b + kZBlock < n ? b + kZBlock : n;
    double bs = 0.0;
    for (size_t i = b; i < e; ++i) bs += (double)x[i];
    sum += bs;
  }
  double mean = sum / (double)n;
  double ss = 0.0;
  for (size_t b = 0; b < n; b += kZBlock) {
    size_t e = b + kZBlock < n ? b + kZBlock : n;
    double bs = 0.0;
    for (size_t i = b; i < e; ++i) {
      double d = (double)x[i] - mean;
      double d2 = d * d;
      bs += d2;
    }
    ss += bs;
  }
  double var = ss / (double)n;
  double sigma = std::sqrt(var);
  if (!(sigma > 0.0)) return -1;
  for (size_t i = 0; i < n; ++i) z[i] = (float)(((double)x[i] - mean) / sigma);
  return 0;
}

// -------------------------------------------------------------- quantiser --
// Sections 4.1 and 4.3: scale the normalised values by 2^k and keep 16 bits.
void oracle_quantise(const float *z, size_t n, int scale_log2, int16_t *q) {
  const float s = (float)(1 << scale_log2);
  for (size_t i = 0; i < n; ++i) {
    float p = z[i] * s;
    float r = std::nearbyint(p);  // default rounding: half to even
    long v = (long)r;
    if (v > kQmax) v = kQmax;
    if (v < -kQmax) v = -kQmax;
    q[i] = (int16_t)v;
  }
}

// ------------------------------------------------------- reference levels --
// Section 2.2 (k-mer model) and Section 4.1 (forward and reverse strands):
// out[0 .. n-k] = model[kmer(bases, j)], out[n-k+1 .. 2(n-k+1)-1] = the same
// over the reverse complement. Bases are 0..3 = A, C, G, T; a k-mer's code
// reads its first base as the most significant base-4 digit.
long oracle_ref_levels(const uint8_t *bases, size_t n, const float *model, int k, float *out) {
  if (k < 1 || n < (size_t)k) return -1;
  size_t per = n - (size_t)k + 1;
  for (size_t j = 0; j < per; ++j) {
    long code = 0;
    for (int u = 0; u < k; ++u) code = code * 4 + bases[j + u];
    out[j] = model[code];
  }
  // reverse complement: rc[u] = 3 - bases[n - 1 - u]
  for (size_t j = 0; j < per; ++j) {
    long code = 0;
    for (int u = 0; u < k; ++u) code = code * 4 + (3 - bases[n - 1 - (j + u)]);
    out[per + j] = model[code];
  }
  return (long)(2 * per);
}

// ------------------------------------------------ Algorithm 1: full matrix --
// C is (M+1) x (N+1) with row 0 = 0 and column 0 = +inf (rows >= 1).
void oracle_sdtw_full_f64(const double *x, int M, const double *y, long N, double *cost, long *col) {
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> C((size_t)(M + 1) * (size_t)(N + 1));
  auto at = [&](long i, long j) -> double & { return C[(size_t)i * (size_t)(N + 1) + (size_t)j]; };
  for (long j = 0; j <= N; ++j) at(0, j) = 0.0;
  for (long i = 1; i <= M; ++i) at(i, 0) = inf;
  for (long i = 1; i <= M; ++i)
    for (long j = 1; j <= N; ++j)
      at(i, j) = std::fabs(x[i - 1] - y[j - 1]) + dmin3(at(i - 1, j), at(i - 1, j - 1), at(i, j - 1));
  double score = inf;
  long pos = -1;
  for (long j = 1; j <= N; ++j)
    if (at(M, j) < score) {
      score = at(M, j);
      pos = j - 1;
    }
  *cost = score;
  *col = pos;
}

void oracle_sdtw_full_i16(const int16_t *x, int M, const int16_t *y, long N, int32_t *cost, long *col) {
  std::vector<int32_t> C((size_t)(M + 1) * (size_t)(N + 1));
  auto at = [&](long i, long j) -> int32_t & { return C[(size_t)i * (size_t)(N + 1) + (size_t)j]; };
  for (long j = 0; j <= N; ++j) at(0, j) = 0;
  for (long i = 1; i <= M; ++i) at(i, 0) = kCap;
  for (long i = 1; i <= M; ++i)
    for (long j = 1; j <= N; ++j) {
      int32_t d = std::abs((int32_t)x[i - 1] - (int32_t)y[j - 1]);
      int32_t v = d + imin3(at(i - 1, j), at(i - 1, j - 1), at(i, j - 1));
      at(i, j) = v < kCap ? v : kCap;
    }
  int32_t score = std::numeric_limits<int32_t>::max();
  long pos = -1;
  for (long j = 1; j <= N; ++j)
    if (at(M, j) < score) {
      score = at(M, j);
      pos = j - 1;
    }
  *cost = score;
  *col = pos;
}

// The last row of the full matrix (used by tests for bounds and runner-ups).
void oracle_sdtw_lastrow_f64(const double *x, int M, const double *y, long N, double *last) {
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> prev((size_t)N + 1, 0.0), cur((size_t)N + 1);
  for (int i = 1; i <= M; ++i) {
    cur[0] = inf;
    for (long j = 1; j <= N; ++j)
      cur[j] = std::fabs(x[i - 1] - y[j - 1]) + dmin3(prev[j], prev[j - 1], cur[j - 1]);
    prev.swap(cur);
  }
  for (long j = 0; j < N; ++j) last[j] = prev[(size_t)j + 1];
}

// ---------------------------------------------- Algorithm 2: rolling array --
// C[0..M], C[0] is the free-start row (0); C[1..M] start at +inf (column 0).
// For each reference sample j: walk i = 1..M keeping the north-west value of
// the previous column, then compare C[M] against the best so far (strict <).
void oracle_sdtw_roll_f64(const double *x, int M, const double *y, long N, double *cost, long *col,
                          double *runner_up) {
  const double inf = std::numeric_limits<double>::infinity();
  std::vector<double> C((size_t)M + 1, inf);
  C[0] = 0.0;
  double score = inf, second = inf;
  long pos = -1;
  for (long j = 0; j < N; ++j) {
    double nw = C[0];  // gamma(0, j-1) = 0
    for (int i = 1; i <= M; ++i) {
      double w = C[i];  // gamma(i, j-1)
      double v = std::fabs(x[i - 1] - y[j]) + dmin3(C[i - 1], nw, w);
      nw = w;
      C[i] = v;
    }
    double last = C[M];
    if (last < score) {
      second = score;
      score = last;
      pos = j;
    } else if (last < second) {
      second = last;
    }
  }
  *cost = score;
  *col = pos;
  if (runner_up) *runner_up = second;
}

// ------------------------------------- Section 4.3: the pipelined PE chain --
// The same recurrence evaluated in the oblique order of the processing-element
// chain (Section 4.3, Fig. 5): PE i holds query sample x_i and at step t
// computes gamma(i, t - i), while the reference streams past one PE per step.
// Within a step every PE updates at once from values of the two previous
// steps: up = gamma(i-1, j) is PE i-1's value of step t-1, diagonal =
// gamma(i-1, j-1) is PE i-1's value of step t-2, left = gamma(i, j-1) is PE
// i's own value of step t-1. Row 0 (above PE 1) is the free-start 0 and
// column 0 is +inf. The chain needs N + M - 1 steps for all cells; *steps
// reports how many it ran. The last PE's values, in column order, give the
// cost and the first column reaching it (strict <).
void oracle_sdtw_wavefront_f64(const double *x, int M, const double *y, long N, double *cost, long *col,
                               long *steps) {
  const double inf = std::numeric_limits<double>::infinity();
  // val1[i]: PE i's value after the previous step; val2[i]: the step before.
  // Index 0 is the free-start row, always 0.
  std::vector<double> val1((size_t)M + 1, inf), val2((size_t)M + 1, inf), next((size_t)M + 1, inf);
  val1[0] = val2[0] = next[0] = 0.0;
  double score = inf;
  long pos = -1, t = 0;
  for (; t < N + M - 1; ++t) {
    for (int i = 1; i <= M; ++i) {
      const long j = t - (i - 1);  // 0-based column of PE i at step t
      if (j < 0 || j >= N) {
        next[(size_t)i] = (j < 0) ? inf : val1[(size_t)i];  // not started: column 0's +inf; done: hold
        continue;
      }
      const double up = val1[(size_t)i - 1];
      const double diag = (j == 0) ? (i == 1 ? 0.0 : inf) : val2[(size_t)i - 1];
      const double left = (j == 0) ? inf : val1[(size_t)i];
      next[(size_t)i] = std::fabs(x[i - 1] - y[j]) + dmin3(up, diag, left);
    }
    val2.swap(val1);
    val1.swap(next);
    const long jl = t - (M - 1);  // the last PE's column at this step
    if (jl >= 0 && jl < N && val1[(size_t)M] < score) {
      score = val1[(size_t)M];
      pos = jl;
    }
  }
  *cost = score;
  *col = pos;
  *steps = t;
}

void oracle_sdtw_roll_f32(const float *x, int M, const float *y, long N, float *cost, long *col) {
  const float inf = std::numeric_limits<float>::infinity();
  std::vector<float> C((size_t)M + 1, inf);
  C[0] = 0.0f;
  float score = inf;
  long pos = -1;
  for (long j = 0; j < N; ++j) {
    float nw = C[0];
    for (int i = 1; i <= M; ++i) {
      float w = C[i];
      float d = std::fabs(x[i - 1] - y[j]);
      float v = d + fmin3_(C[i - 1], nw, w);
      nw = w;
      C[i] = v;
    }
    if (C[M] < score) {
      score = C[M];
      pos = j;
    }
  }
  *cost = score;
  *col = pos;
}

void oracle_sdtw_roll_i16(const int16_t *x, int M, const int16_t *y, long N, int32_t *cost, long *col) {
  std::vector<int32_t> C((size_t)M + 1, kCap);
  C[0] = 0;
  int32_t score = std::numeric_limits<int32_t>::max();
  long pos = -1;
  for (long j = 0; j < N; ++j) {
    int32_t nw = C[0];
    for (int i = 1; i <= M; ++i) {
      int32_t w = C[i];
      int32_t d = std::abs((int32_t)x[i - 1] - (int32_t)y[j]);
      int32_t v = d + imin3(C[i - 1], nw, w);
      nw = w;
      C[i] = v < kCap ? v : kCap;
    }
    if (C[M] < score) {
      score = C[M];
      pos = j;
    }
  }
  *cost = score;
  *col = pos;
}

// int16 inputs with wide accumulation (the PE of Section 4.3: 16-bit
// fixed-point samples, 32-bit cost registers): the exact integer DP, no
// saturation. Accumulated in 64 bits here; for M <= 512 every value is below
// 512 * 4094 < 2^31, so a 32-bit accumulator gives the same numbers.
void oracle_sdtw_roll_i32(const int16_t *x, int M, const int16_t *y, long N, int64_t *cost, long *col) {
  const int64_t kInf = (int64_t)1 << 60;
  std::vector<int64_t> C((size_t)M + 1, kInf);
  C[0] = 0;
  int64_t score = kInf;
  long pos = -1;
  for (long j = 0; j < N; ++j) {
    int64_t nw = C[0];
    for (int i = 1; i <= M; ++i) {
      int64_t w = C[i];
      int64_t d = std::abs((int64_t)x[i - 1] - (int64_t)y[j]);
      int64_t m = C[i - 1] < nw ? C[i - 1] : nw;
      m = m < w ? m : w;
      nw = w;
      C[i] = m >= kInf ? kInf : d + m;
    }
    if (C[M] < score) {
      score = C[M];
      pos = j;
    }
  }
  *cost = score;
  *col = pos;
}

// Start column of the alignment (the paper drops backtracking; this carries
// the start forward instead). Every cell keeps the start of the predecessor
// that gives its minimum: the up neighbour if it is a minimum, else the
// diagonal one if it is, else the left one (a fixed preference on equal
// costs); a path that enters row 1 at column j starts at j. The cost and the
// end column are those of the plain DP. T: float (FP32 form) or int64_t
// (int16 inputs, wide accumulation).
}  // extern "C"

template <class T, class D>
static void roll_span(const D *x, int M, const D *y, long N, T inf, T *cost, long *col, long *start) {
  std::vector<T> C((size_t)M + 1, inf);
  std::vector<long> P((size_t)M + 1, -1);
  C[0] = 0;
  T score = inf;
  long pos = -1, spos = -1;
  for (long j = 0; j < N; ++j) {
    T nw = C[0];
    long nws = j;
    for (int i = 1; i <= M; ++i) {
      const T w = C[i];
      const long ws = P[i];
      // up: row i-1 of this column; diagonal: row i-1 of the previous one
      // (row 0 on both: cost 0, and the path starts here, at column j)
      T mc = i == 1 ? T(0) : C[i - 1];
      long ms = i == 1 ? j : P[i - 1];
      const T dc = i == 1 ? T(0) : nw;
      const long ds = i == 1 ? j : nws;
      if (dc < mc) { mc = dc; ms = ds; }
      if (w < mc) { mc = w; ms = ws; }
      T d;
      if constexpr (std::is_same<T, float>::value) d = std::fabs(x[i - 1] - y[j]);
      else d = std::abs((T)x[i - 1] - (T)y[j]);
      nw = w;
      nws = ws;
      C[i] = mc >= inf ? inf : d + mc;
      P[i] = ms;
    }
    if (C[M] < score) {
      score = C[M];
      pos = j;
      spos = P[M];
    }
  }
  *cost = score;
  *col = pos;
  *start = spos;
}

extern "C" {

void oracle_sdtw_span_f32(const float *x, int M, const float *y, long N, float *cost, long *col, long *start) {
  roll_span<float, float>(x, M, y, N, std::numeric_limits<float>::infinity(), cost, col, start);
}

void oracle_sdtw_span_i32(const int16_t *x, int M, const int16_t *y, long N, int64_t *cost, long *col,
                          long *start) {
  roll_span<int64_t, int16_t>(x, M, y, N, (int64_t)1 << 60, cost, col, start);
}

// ------------------------------------------------------------------ batch --
// The whole path as the library exposes it: z-score the reference and each
// query (when asked), quantise for the int16 form, run Algorithm 2 per query.
// prec: 0 = FP32, 1 = int16 (saturating), 2 = FP64 (inputs are the FP32
// z-values widened), 3 = int16 inputs with 32-bit accumulation (no
// saturation). cost is reported in z units (integer forms: integer / 2^k).
// start (optional, FP32 and the wide form): the alignment's start column
// (roll_span); the cost and column are the same as without it.
// Queries are spread over `threads` worker threads (0 = hardware count).
// Returns 0, or -1 on invalid input (first offending query in *bad).
int oracle_batch(int prec, const float *ref, size_t N, int normalize_ref, const float *events,
                 const uint32_t *offsets, uint32_t nq, int normalize_q, int scale_log2, int threads,
                 double *cost, int64_t *col, double *runner_up, int32_t *icost, int64_t *start, long *bad) {
  if (N == 0) return -1;
  std::vector<float> rz(N);
  if (normalize_ref) {
    if (oracle_zscore(ref, N, rz.data()) != 0) return -1;
  } else {
    std::memcpy(rz.data(), ref, N * sizeof(float));
  }
  std::vector<int16_t> rq;
  std::vector<double> rd;
  if (prec == 1 || prec == 3) {
    rq.resize(N);
    oracle_quantise(rz.data(), N, scale_log2, rq.data());
  }
  if (prec == 2) {
    rd.resize(N);
    for (size_t j = 0; j < N; ++j) rd[j] = (double)rz[j];
  }
  for (uint32_t q = 0; q < nq; ++q) {
    long m = (long)offsets[q + 1] - (long)offsets[q];
    if (m < 1 || (size_t)m > N) {
      if (bad) *bad = q;
      return -1;
    }
  }
  std::atomic<uint32_t> next(0);
  std::atomic<int> err(0);
  const double s = (double)(1 << scale_log2);
  auto worker = [&]() {
    std::vector<float> qz;
    std::vector<int16_t> qq;
    std::vector<double> qd;
    for (;;) {
      uint32_t q = next.fetch_add(1);
      if (q >= nq) break;
      int M = (int)(offsets[q + 1] - offsets[q]);
      const float *ev = events + offsets[q];
      qz.resize((size_t)M);
      if (normalize_q) {
        if (oracle_zscore(ev, (size_t)M, qz.data()) != 0) {
          err.store(1);
          if (bad) *bad = q;
          continue;
        }
      } else {
        std::memcpy(qz.data(), ev, (size_t)M * sizeof(float));
      }
      long c = -1;
      if (prec == 0 && start) {
        float f;
        long st;
        oracle_sdtw_span_f32(qz.data(), M, rz.data(), (long)N, &f, &c, &st);
        cost[q] = (double)f;
        start[q] = (int64_t)st;
      } else if (prec == 0) {
        float f;
        oracle_sdtw_roll_f32(qz.data(), M, rz.data(), (long)N, &f, &c);
        cost[q] = (double)f;
      } else if (prec == 1) {
        qq.resize((size_t)M);
        oracle_quantise(qz.data(), (size_t)M, scale_log2, qq.data());
        int32_t v;
        oracle_sdtw_roll_i16(qq.data(), M, rq.data(), (long)N, &v, &c);
        cost[q] = (double)v / s;
        if (icost) icost[q] = v;
      } else if (prec == 3) {
        qq.resize((size_t)M);
        oracle_quantise(qz.data(), (size_t)M, scale_log2, qq.data());
        int64_t v;
        if (start) {
          long st;
          oracle_sdtw_span_i32(qq.data(), M, rq.data(), (long)N, &v, &c, &st);
          start[q] = (int64_t)st;
        } else {
          oracle_sdtw_roll_i32(qq.data(), M, rq.data(), (long)N, &v, &c);
        }
        cost[q] = (double)v / s;
        if (icost) icost[q] = (int32_t)v;
      } else {
        qd.resize((size_t)M);
        for (int i = 0; i < M; ++i) qd[(size_t)i] = (double)qz[(size_t)i];
        double v, r;
        oracle_sdtw_roll_f64(qd.data(), M, rd.data(), (long)N, &v, &c, &r);
        cost[q] = v;
        if (runner_up) runner_up[q] = r;
      }
      col[q] = (int64_t)c;
    }
  };
  int nt = threads > 0 ? threads : (int)std::thread::hardware_concurrency();
  if (nt < 1) nt = 1;
  if ((uint32_t)nt > nq) nt = (int)(nq > 0 ? nq : 1);
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto &t : pool) t.join();
  return err.load() ? -1 : 0;
}

}  // extern "C"
