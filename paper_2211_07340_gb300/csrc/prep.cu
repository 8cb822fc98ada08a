// Device-side preparation: reference synthesis and normalisation (Section
// 4.1), the batch planner, and per-query normalisation, quantisation and
// packing into the warp-strip register images the sweep kernels load.
//
// z-score reading (the paper does not say how mean and sigma are formed):
// population sigma; sums in double, in blocks of 4096 consecutive samples
// added in index order, block sums added in index order; every double
// operation is an explicitly rounded intrinsic so no contraction occurs;
// z = (float)((x - mean) / sigma). Quantiser: clamp(rint(z * 2^k), +-2047).

#include <cuda_runtime.h>

#include "haru_internal.h"

namespace haru {
namespace {

constexpr int kZBlock = 4096;

__device__ __forceinline__ bool finite_d(double v) { return isfinite(v); }

__device__ __forceinline__ int quantise(float z, float s) {
  int v = __float2int_rn(__fmul_rn(z, s));
  return v > kQmax ? kQmax : (v < -kQmax ? -kQmax : v);
}

// ------------------------------------------------------------ reference --
__global__ void ref_levels_kernel(const uint8_t *bases, size_t n, const float *model, int k, float *out,
                                  int *status) {
  const size_t per = n - static_cast<size_t>(k) + 1;
  for (size_t j = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; j < 2 * per;
       j += static_cast<size_t>(gridDim.x) * blockDim.x) {
    long code = 0;
    bool bad = false;
    if (j < per) {
      for (int u = 0; u < k; ++u) {
        uint8_t b = bases[j + u];
        bad |= b > 3;
        code = code * 4 + (b & 3);
      }
    } else {
      const size_t jj = j - per;  // k-mer jj of the reverse complement
      for (int u = 0; u < k; ++u) {
        uint8_t b = bases[n - 1 - (jj + u)];
        bad |= b > 3;
        code = code * 4 + (3 - (b & 3));
      }
    }
    if (bad) report(status, HARU_EINVAL);
    out[j] = model[code];
  }
}

// One thread per block of kZBlock samples: the block's sum (pass 0) or sum
// of squared deviations from stats[0] (pass 1), in index order.
__global__ void block_sums_kernel(const float *x, size_t n, const double *stats, int pass, double *partials) {
  const size_t b = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x;
  const size_t lo = b * kZBlock;
  if (lo >= n) return;
  const size_t hi = lo + kZBlock < n ? lo + kZBlock : n;
  double acc = 0.0;
  if (pass == 0) {
    for (size_t i = lo; i < hi; ++i) acc = __dadd_rn(acc, static_cast<double>(x[i]));
  } else {
    const double mean = stats[0];
    for (size_t i = lo; i < hi; ++i) {
      const double d = __dsub_rn(static_cast<double>(x[i]), mean);
      acc = __dadd_rn(acc, __dmul_rn(d, d));
    }
  }
  partials[b] = acc;
}

// Single thread: add the block sums in order; pass 0 -> mean, pass 1 -> sigma.
__global__ void finish_sums_kernel(const double *partials, size_t nblocks, size_t n, int pass, double *stats,
                                   int *status) {
  double acc = 0.0;
  for (size_t b = 0; b < nblocks; ++b) acc = __dadd_rn(acc, partials[b]);
  if (pass == 0) {
    stats[0] = __ddiv_rn(acc, static_cast<double>(n));
    if (!finite_d(stats[0])) report(status, HARU_EINVAL);
  } else {
    const double sigma = __dsqrt_rn(__ddiv_rn(acc, static_cast<double>(n)));
    stats[1] = sigma;
    if (!(sigma > 0.0) || !finite_d(sigma)) report(status, HARU_EINVAL);
  }
}

__global__ void ref_finish_kernel(const float *x, size_t n, const double *stats, int normalize, float s,
                                  float *z, uint32_t *img16, float *img32, int *status) {
  for (size_t i = blockIdx.x * static_cast<size_t>(blockDim.x) + threadIdx.x; i < n;
       i += static_cast<size_t>(gridDim.x) * blockDim.x) {
    float v = x[i];
    if (normalize) {
      const double mean = stats[0], sigma = stats[1];
      v = __double2float_rn(__ddiv_rn(__dsub_rn(static_cast<double>(v), mean), sigma));
    }
    if (!isfinite(v)) report(status, HARU_EINVAL);
    const int q = quantise(v, s);
    z[i] = v;
    img16[i] = (static_cast<uint32_t>(q) & 0xffffu) | (static_cast<uint32_t>(q) << 16);
    img32[i] = v;
  }
}

// --------------------------------------------------------------- planner --
// Bucket key of query q: its strip height S (rows per lane), plus kMaxS + 1
// if it is stacked (16 lanes); 0 for an invalid length. S is the least
// height that leaves a pad row on top of the query (S = floor(M / 32) + 1,
// or floor(M / 16) + 1 stacked), at most kMaxS: the sweep relies on that
// row to hold the free-start zero in strips lower than kMaxS.
__device__ __forceinline__ int bucket_key(const uint32_t *off, uint32_t q, long N, int mode, int stack, int *status) {
  const uint32_t m = off[q + 1] - off[q];
  const long lim = N < HARU_MAX_QUERY ? N : HARU_MAX_QUERY;
  if (m < 1 || static_cast<long>(m) > lim) {
    if (status) report(status, HARU_EINVAL);
    return 0;
  }
  if (stack && m <= static_cast<uint32_t>(kStackMax))
    return min(static_cast<int>(m / 16) + 1, kMaxS) + kMaxS + 1;
  return min(static_cast<int>(m / 32) + 1, kMaxS);
}

// Items of a bucket of n queries. Modes 0 (FP32) and 3 (int16 inputs, wide
// accumulation) make one item per query (two per stacked item); mode 1
// pairs int16 queries (four per stacked item).
__device__ __forceinline__ bool singles(int mode) { return mode == 0 || mode == 3; }
__device__ __forceinline__ int stacked_items(int mode, int n) { return singles(mode) ? (n + 1) / 2 : (n + 3) / 4; }
__device__ __forceinline__ int bucket_items(int mode, int n) { return singles(mode) ? n : (n + 1) / 2; }

// One CTA of 1024 threads. Buckets queries by strip height S (descending,
// the longest-processing-time-first order of the work queue), keeps the
// input order inside a bucket, pairs neighbours for the int16 form, and cuts
// each bucket into groups of `warps` items.
__global__ void __launch_bounds__(1024) plan_kernel(PlanArgs a) {
  constexpr int kKeys = 2 * (kMaxS + 1);  // plain and stacked buckets of each S
  __shared__ int cnt[kKeys], ibase[kMaxS + 1], sbase[kMaxS + 1], icount[kMaxS + 1], nseg_of[kMaxS + 1];
  __shared__ int gbase[kMaxS + 1], gcount[kMaxS + 1];
  __shared__ int wrun[32][kKeys];  // per warp and bucket: count, then next position
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nw = blockDim.x >> 5;
  int *status = a.ints + kIntStatus;
  // Each warp owns a contiguous range of queries, so bucket positions
  // (earlier warps first, then the order inside the warp) keep input order.
  const uint32_t per_warp = (a.nq + nw - 1) / nw;
  const uint32_t q_lo = min(a.nq, static_cast<uint32_t>(warp) * per_warp);
  const uint32_t q_hi = min(a.nq, q_lo + per_warp);
  for (int b = lane; b < kKeys; b += 32) wrun[warp][b] = 0;
  __syncwarp();
  for (uint32_t q0 = q_lo; q0 < q_hi; q0 += 32) {
    const uint32_t q = q0 + lane;
    const int key = q < q_hi ? bucket_key(a.offsets, q, a.N, a.pair, a.stack, status) : 0;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key && lane == __ffs(peers) - 1) wrun[warp][key] += __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  if (tid >= 1 && tid < kKeys) {
    int c = 0;
    for (int w = 0; w < nw; ++w) {
      const int t = wrun[w][tid];
      wrun[w][tid] = c;
      c += t;
    }
    cnt[tid] = c;
  }
  __syncthreads();
  if (tid == 0) {
    int base = 0;
    for (int S = kMaxS; S >= 1; --S) {  // plain items of height S, then stacked ones
      const int plain = bucket_items(a.pair, cnt[S]);
      icount[S] = plain + stacked_items(a.pair, cnt[S + kMaxS + 1]);
      ibase[S] = base;
      sbase[S] = base + plain;
      base += icount[S];
    }
    a.ints[kIntItems] = base;
    // Segments per item: enough work units for the machine, each segment
    // at least four warm-ups (and 2048 steps) long.
    int want = base > 0 ? (a.units_target + base - 1) / base : 1;
    if (want < 1) want = 1;
    if (want > a.nseg_cap) want = a.nseg_cap;
    // The buckets at the end of the longest-first queue (the cheapest strips,
    // up to a fifth of the work) get twice the segments: shorter final work
    // units leave less of the machine idle while the last ones finish.
    long total = 0, acc = 0;
    for (int S = 1; S <= kMaxS; ++S) total += static_cast<long>(icount[S]) * S;
    int tail_to = 0;  // buckets S <= tail_to form the tail
    if (a.units_target > 1) {
      for (int S = 1; S <= kMaxS; ++S) {
        const long w = static_cast<long>(icount[S]) * S;
        if ((acc + w) * 5 > total) break;
        acc += w;
        tail_to = S;
      }
    }
    // Groups, tallest strips first: one longest-first queue for the sweep kernel.
    int g = 0;
    a.ints[kIntQueue] = 0;
    for (int S = kMaxS; S >= 1; --S) {
      const long minlen = 4 * warmup_steps(S) > 2048 ? 4 * warmup_steps(S) : 2048;
      long lim = sweep_steps(S, a.N) / minlen;
      if (lim < 1) lim = 1;
      int ws = S <= tail_to ? 2 * want : want;
      if (ws > a.nseg_cap) ws = a.nseg_cap;
      nseg_of[S] = ws < lim ? ws : static_cast<int>(lim);
      gbase[S] = g;
      gcount[S] = nseg_of[S] * ((icount[S] + a.warps - 1) / a.warps);
      g += gcount[S];
    }
    a.ints[kIntGroups] = g;
    int most = 0;
    for (int S = 1; S <= kMaxS; ++S)
      if (icount[S] > 0 && nseg_of[S] > most) most = nseg_of[S];
    a.ints[kIntMaxSeg] = most;
  }
  __syncthreads();
  // Groups of each bucket, segment-major: (seg, first item), in parallel.
  for (int S = kMaxS; S >= 1; --S) {
    const int per_seg = (icount[S] + a.warps - 1) / a.warps;
    for (int j = tid; j < gcount[S]; j += blockDim.x) {
      const int seg = j / per_seg, f = (j % per_seg) * a.warps;
      Group gr;
      gr.S = S;
      gr.first = ibase[S] + f;
      gr.count = icount[S] - f < a.warps ? icount[S] - f : a.warps;
      gr.seg = seg;
      gr.nseg = nseg_of[S];
      gr.pad[0] = gr.pad[1] = gr.pad[2] = 0;
      a.groups[gbase[S] + j] = gr;
    }
  }
  __syncthreads();
  const int n_items = a.ints[kIntItems];
  for (int i = tid; i < n_items; i += blockDim.x) {
    Item it;
    it.qa = -1; it.qb = -1; it.S = 0; it.nseg = 1;
    it.kind = a.pair == 0 ? kItemF32 : (a.pair == 3 ? kItemExact : kItemPair);
    it.qc = -1; it.qd = -1; it.stacked = 0;
    a.items[i] = it;
  }
  __syncthreads();
  const unsigned lt = (1u << lane) - 1u;
  for (uint32_t q0 = q_lo; q0 < q_hi; q0 += 32) {
    const uint32_t q = q0 + lane;
    const int key = q < q_hi ? bucket_key(a.offsets, q, a.N, a.pair, a.stack, nullptr) : 0;
    const unsigned peers = __match_any_sync(0xffffffffu, key);
    if (key > kMaxS) {  // stacked: slots qa, qb | qc, qd (INT16) or qa | qc (FP32)
      const int b = key - kMaxS - 1;
      const int pos = wrun[warp][key] + __popc(peers & lt);
      const int per = singles(a.pair) ? 2 : 4;
      const int slot = singles(a.pair) ? 2 * (pos % 2) : pos % 4;
      Item *it = &a.items[sbase[b] + pos / per];
      if (slot == 0) { it->qa = static_cast<int>(q); it->S = b; it->nseg = nseg_of[b]; it->stacked = 1; }
      else if (slot == 1) it->qb = static_cast<int>(q);
      else if (slot == 2) it->qc = static_cast<int>(q);
      else it->qd = static_cast<int>(q);
    } else if (key) {
      const int b = key;
      const int pos = wrun[warp][b] + __popc(peers & lt);  // position in bucket b
      if (a.pair == 1) {
        Item *it = &a.items[ibase[b] + pos / 2];
        if (pos % 2 == 0) { it->qa = static_cast<int>(q); it->S = b; it->nseg = nseg_of[b]; }
        else it->qb = static_cast<int>(q);
      } else {
        Item it;
        it.qa = static_cast<int>(q); it.qb = -1; it.S = b; it.nseg = nseg_of[b];
        it.kind = a.pair == 3 ? kItemExact : kItemF32;
        it.qc = -1; it.qd = -1; it.stacked = 0;
        a.items[ibase[b] + pos] = it;
      }
    }
    __syncwarp();
    if (key && lane == __ffs(peers) - 1) wrun[warp][key] += __popc(peers);
    __syncwarp();
  }
}

// ----------------------------------------------------------------- pack --
// Mean and sigma of one query, sequentially (a query is shorter than one
// z-score block, so this is the blocked rule's order).
// Loads are issued eight at a time ahead of the (sequential) additions.
__device__ void query_stats(const float *x, int m, double &mean, double &sigma) {
  constexpr int B = 8;
  float v[B];
  double acc = 0.0;
  int i = 0;
  for (; i + B <= m; i += B) {
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = __ldg(x + i + j);
#pragma unroll
    for (int j = 0; j < B; ++j) acc = __dadd_rn(acc, static_cast<double>(v[j]));
  }
  for (; i < m; ++i) acc = __dadd_rn(acc, static_cast<double>(__ldg(x + i)));
  mean = __ddiv_rn(acc, static_cast<double>(m));
  double ss = 0.0;
  i = 0;
  for (; i + B <= m; i += B) {
#pragma unroll
    for (int j = 0; j < B; ++j) v[j] = __ldg(x + i + j);
#pragma unroll
    for (int j = 0; j < B; ++j) {
      const double d = __dsub_rn(static_cast<double>(v[j]), mean);
      ss = __dadd_rn(ss, __dmul_rn(d, d));
    }
  }
  for (; i < m; ++i) {
    const double d = __dsub_rn(static_cast<double>(__ldg(x + i)), mean);
    ss = __dadd_rn(ss, __dmul_rn(d, d));
  }
  sigma = __dsqrt_rn(__ddiv_rn(ss, static_cast<double>(m)));
}

// One thread per query: its mean and sigma (the sums are sequential chains,
// so a query gets a thread of its own rather than a lane of a packing warp).
__global__ void qstats_kernel(const float *events, const uint32_t *offsets, uint32_t nq, double *qstats,
                              int *status) {
  const uint32_t q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= nq) return;
  const uint32_t b = offsets[q];
  const uint32_t m = offsets[q + 1] - b;
  double mu = 0.0, sg = 1.0;
  if (m >= 1 && m <= HARU_MAX_QUERY) {  // other lengths are rejected by the planner
    query_stats(events + b, static_cast<int>(m), mu, sg);
    if (!(sg > 0.0) || !isfinite(sg) || !isfinite(mu)) report(status, HARU_EINVAL);
  }
  qstats[2 * static_cast<size_t>(q)] = mu;
  qstats[2 * static_cast<size_t>(q) + 1] = sg;
}

// One warp per item: lane l writes rows l*S .. l*S+S-1 of both halves (of
// its own stack, for stacked items).
__global__ void pack_kernel(PackArgs a) {
  const int item = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (item >= *a.n_items) return;
  const Item it = a.items[item];
  const int S = it.S;
  // Stacked items: lanes 16..31 hold the lower stack (qc, qd).
  const bool low = it.stacked && lane >= 16;
  const int qs[2] = {low ? it.qc : it.qa, low ? it.qd : it.qb};
  const int H = it.stacked ? 16 * S : 32 * S;             // rows of this lane's stack
  const int lane_in = it.stacked ? (lane & 15) : lane;   // lane within the stack
  int m[2] = {0, 0};
  uint32_t base[2] = {0, 0};
  double mean[2] = {0.0, 0.0}, sigma[2] = {1.0, 1.0};
  const bool packed = it.kind == kItemPair;   // two int16 queries per word
  const bool codes = it.kind != kItemF32;     // int16 codes (packed, or as floats)
  const int halves = packed ? 2 : 1;
  for (int h = 0; h < halves; ++h) {
    if (qs[h] >= 0) {
      base[h] = a.offsets[qs[h]];
      m[h] = static_cast<int>(a.offsets[qs[h] + 1] - base[h]);
    }
  }
  if (a.raw) {
    for (int h = 0; h < halves; ++h) {
      if (qs[h] >= 0) {
        mean[h] = a.qstats[2 * static_cast<size_t>(qs[h])];
        sigma[h] = a.qstats[2 * static_cast<size_t>(qs[h]) + 1];
      }
    }
  }
  const float s = static_cast<float>(1 << a.scale_log2);
  uint32_t *img = a.img + static_cast<size_t>(item) * kImgStride;
  for (int k = 0; k < S; ++k) {
    const int row = lane_in * S + k;
    uint32_t w0 = 0, w1 = 0;
    for (int h = 0; h < halves; ++h) {
      const int P = H - m[h];
      const bool real = m[h] > 0 && row >= P;
      float z = 0.0f;
      if (real) {
        const float x = a.events[base[h] + (row - P)];
        if (a.raw)
          z = __double2float_rn(__ddiv_rn(__dsub_rn(static_cast<double>(x), mean[h]), sigma[h]));
        else
          z = x;
        if (!isfinite(z) || fabsf(z) > 1.0e20f) report(a.status, HARU_EINVAL);
      }
      if (packed) {
        // real row: (q, -q); pad row: (-4095, -4095), read by the sweep as distance 0
        const int qv = real ? quantise(z, s) : -4095;
        const int nv = real ? -qv : -4095;
        w0 |= (static_cast<uint32_t>(qv) & 0xffffu) << (16 * h);
        w1 |= (static_cast<uint32_t>(nv) & 0xffffu) << (16 * h);
      } else {
        // FP32: the z-value; exact form: the int16 code as a float; the row
        // weight the sweep multiplies the reference sample by: -1 on real
        // rows (fma(r, -1, q) = q - r, rounded once), 0 on pad rows (which
        // hold q = 0, so their distance is 0)
        w0 = __float_as_uint(codes ? (real ? static_cast<float>(quantise(z, s)) : 0.0f) : z);
        w1 = __float_as_uint(real ? -1.0f : 0.0f);
      }
    }
    img[k * 32 + lane] = w0;
    img[(S + k) * 32 + lane] = w1;
  }
}

}  // namespace

cudaError_t launch_plan(const PlanArgs &a, cudaStream_t s) {
  plan_kernel<<<1, 1024, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t load_prep_kernels() {
  cudaFuncAttributes f;
  cudaError_t e = cudaFuncGetAttributes(&f, plan_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&f, qstats_kernel);
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&f, pack_kernel);
  return e;
}

cudaError_t launch_pack(const PackArgs &a, uint32_t max_items, cudaStream_t s) {
  if (max_items == 0) return cudaSuccess;
  const int warps = 8;
  pack_kernel<<<(max_items + warps - 1) / warps, warps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_qstats(const float *events, const uint32_t *offsets, uint32_t nq, double *qstats, int *status,
                          cudaStream_t s) {
  if (nq == 0) return cudaSuccess;
  const int th = 32;  // one warp per block: the sequential chains spread over every SM
  qstats_kernel<<<(nq + th - 1) / th, th, 0, s>>>(events, offsets, nq, qstats, status);
  return cudaGetLastError();
}

cudaError_t launch_ref_levels(const uint8_t *bases, size_t n, const float *model, int k, float *out, int *status,
                              cudaStream_t s) {
  const size_t total = 2 * (n - k + 1);
  const int th = 256;
  size_t blocks = (total + th - 1) / th;
  if (blocks > 65535) blocks = 65535;
  ref_levels_kernel<<<static_cast<unsigned>(blocks), th, 0, s>>>(bases, n, model, k, out, status);
  return cudaGetLastError();
}

cudaError_t launch_zscore_stats(const float *x, size_t n, double *partials, double *stats, int *status,
                                cudaStream_t s) {
  const size_t nb = (n + kZBlock - 1) / kZBlock;
  const int th = 128;
  const unsigned blocks = static_cast<unsigned>((nb + th - 1) / th);
  block_sums_kernel<<<blocks, th, 0, s>>>(x, n, stats, 0, partials);
  finish_sums_kernel<<<1, 1, 0, s>>>(partials, nb, n, 0, stats, status);
  block_sums_kernel<<<blocks, th, 0, s>>>(x, n, stats, 1, partials);
  finish_sums_kernel<<<1, 1, 0, s>>>(partials, nb, n, 1, stats, status);
  return cudaGetLastError();
}

cudaError_t launch_ref_finish(const float *x, size_t n, const double *stats, int normalize, int scale_log2,
                              float *z, uint32_t *img16, float *img32, size_t img_len, int *status,
                              cudaStream_t s) {
  (void)img_len;
  const int th = 256;
  size_t blocks = (n + th - 1) / th;
  if (blocks > 65535) blocks = 65535;
  ref_finish_kernel<<<static_cast<unsigned>(blocks), th, 0, s>>>(x, n, stats, normalize,
                                                                 static_cast<float>(1 << scale_log2), z, img16,
                                                                 img32, status);
  return cudaGetLastError();
}

}  // namespace haru
