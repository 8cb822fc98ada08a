// The sDTW wavefront kernels (Eq. 1, Section 2.3; the pipelined oblique column
// of Section 4.3 / Fig. 5, mapped onto warps).
//
// Layout of one warp's work. A query of M events is padded at the top to
// 32 * S rows (S = floor(M / 32) + 1, at most 16, so that a strip lower than
// 16 rows per lane has at least one pad row); lane l holds rows l*S .. l*S + S - 1 in
// registers. Row i processes reference column t - i at step t, so every row
// is one processing element of the paper's PE chain and the whole strip is
// one oblique column: the S cells of a lane in one step are independent
// (instruction-level parallelism S), a cell reads
//   up   = row i-1 at step t-1,  diag = row i-1 at step t-2,  left = row i at step t-1,
// and each step one value (the bottom row's cost) crosses from lane l-1 to
// lane l by __shfl_up_sync; lane 0 takes the free-start row gamma(0, .) = 0.
// Each lane reads its row 0's reference sample, column t - l*S, from the
// shared tile itself, and the sample moves down the lane's rows by register
// renaming (the oblique column's reference stream, Fig. 5). A sweep is
// N + 32*S - 1 steps, the paper's N + M - 1 (Section 4.3) for the padded
// height. Pad rows sit above the query and hold exactly 0, the free-start
// boundary row, so the last query row is always lane 31's last register.
// A pad row's minimum includes its own 0, so whatever lane 0 receives from
// above is absorbed there, and only full-height strips (16 rows per lane,
// no pad row) have lane 0 replace that value by the zero.
//
// INT16 form: two queries share a warp, one per 16-bit half (DPX
// __viaddmax_s16x2_relu for |q - r|, __vimin3_u16x2, and __viaddmin_u16x2 on
// the rows that saturate at CAP); pad rows hold 0. FP32 form: one query per warp, 3-input min.f32,
// gamma = |d| + min3 with d = fma(r, w, q): w = -1 on real rows, 0 on pad rows (and q = 0 there).
//
// Segments. The steps of one query are cut into segments that run as
// independent work units. Segment s > 0 starts V steps early from a fresh
// state (as if the reference began there) and records its state (the last
// two oblique columns) when it reaches its own first step B_s; segment s-1
// records its exact state at the same step. The fix-up kernel compares the
// two: equal states give identical computations from B_s on (the DP is a
// deterministic function of that state and the reference), so the segment's
// results stand; otherwise it recomputes the segment from the exact state.
// The result is always the plain DP's.
//
// The reference streams through shared memory: every CTA sweeps a group of
// warps (same S, same segment) over the same columns; tiles of T_S columns,
// each with the kRefFront columns before it (the lanes lag the warp's step by
// up to 31 * S columns), are fetched by cp.async.bulk (TMA) into a two-slot
// ring guarded by mbarriers. The warp that releases a slot last issues the
// copy of the tile two ahead.
//
// The last-row minimum and its first column (Algorithm 1's final scan,
// Algorithm 2's per-column compare) are tracked through a small per-warp
// shared ring: lane 31 stores its bottom-row cost every step, and every
// <= 32 steps each lane scans one stored value; a warp reduction keeps the
// smallest cost, then the smallest column.
//
// Every wait is bounded by a global-timer deadline; on expiry the kernel
// records HARU_ETIMEDOUT, waits (bounded) for its own copies in flight and
// returns.

#pragma once

#include <cuda_runtime.h>

#include "haru_internal.h"

namespace haru {
namespace {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned smem_u32(const void *p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of `bar` to complete, giving up at `deadline`.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, unsigned long long deadline) {
  while (!mbar_try_wait(bar, parity)) {
    if (now_ns() > deadline) return false;
  }
  return true;
}
__device__ __forceinline__ void tma_load_1d(void *dst, const void *src, unsigned bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ float fmin3f(float a, float b, float c) {
  float d;
  asm("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// x == m ? a : b as a compare and a select (never a branch).
__device__ __forceinline__ int sel_eq(float x, float m, int a, int b) {
  int d;
  asm("{\n\t.reg .pred p;\n\tsetp.eq.f32 p, %1, %2;\n\tselp.b32 %0, %3, %4, p;\n\t}"
      : "=r"(d) : "f"(x), "f"(m), "r"(a), "r"(b));
  return d;
}

// d = a * b + c on the integer multiply-add unit (keeps lane-0 fix-ups off
// the half-rate pipe that the DPX min/max instructions use).
__device__ __forceinline__ uint32_t imad(uint32_t a, uint32_t b, uint32_t c) {
  uint32_t d;
  asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// This lane's reference sample of step u of a chunk, read A at a time. The
// lane's window starts at column t0 - lane * S, a multiple of A (4 when the
// strip height S is a multiple of 4, 2 when it is even, else 1; the chunk's
// first step t0 is a multiple of U, which A divides), so every vector load is
// aligned.
template <int S>
struct LaneWindow {
  static constexpr int A = S % 4 == 0 ? 4 : (S % 2 == 0 ? 2 : 1);
  uint4 v4;
  uint2 v2;
  __device__ __forceinline__ uint32_t get(const uint32_t *ref, int u) {
    if constexpr (A == 4) {
      if (u % 4 == 0) v4 = reinterpret_cast<const uint4 *>(ref)[u / 4];
      const int c = u % 4;
      return c == 0 ? v4.x : (c == 1 ? v4.y : (c == 2 ? v4.z : v4.w));
    } else if constexpr (A == 2) {
      if (u % 2 == 0) v2 = reinterpret_cast<const uint2 *>(ref)[u / 2];
      return (u % 2 == 0) ? v2.x : v2.y;
    } else {
      return ref[u];
    }
  }
};

// The tracked lane's last-row value of step u goes to ring[e0 + u]. Values
// are held for four steps (two when U is not a multiple of four; U is always
// even) and written by one vector store: e0 is a multiple of U and the ring
// is 16-byte aligned, so every store is aligned. The FP32 strips use it; the
// int16 strip stores every step, which measured faster there (the held
// values must be moved into consecutive registers).
template <int U>
struct RingStore {
  static constexpr int W = U % 4 == 0 ? 4 : 2;
  uint32_t v[W];
  __device__ __forceinline__ void put(uint32_t *ring, int e0, int u, bool tracked, uint32_t x) {
    v[u % W] = x;
    if (u % W == W - 1 && tracked) {
      if constexpr (W == 4)
        *reinterpret_cast<uint4 *>(ring + e0 + u - 3) = make_uint4(v[0], v[1], v[2], v[3]);
      else
        *reinterpret_cast<uint2 *>(ring + e0 + u - 1) = make_uint2(v[0], v[1]);
    }
  }
};

template <int S>
struct Geo {
  static constexpr int U = (S % 2 == 0) ? S : 2 * S;  // steps per unrolled chunk (register renaming period)
};

// ---------------------------------------------------------------- INT16 --
// Pad rows carry the code -4095 in both Q and NQ: |q - r| is then taken as
// relu(max(r + NQ, Q - r)) = relu(negative) = 0, so a pad row stays 0 (the
// free-start row) without a per-row cap, and real rows (|q|, |r| <= 2047)
// get max(r - q, q - r) unchanged.
constexpr uint32_t kPadQ2 = 0xf001f001u;  // -4095 in both halves
constexpr uint32_t kCap2 = (static_cast<uint32_t>(kCap) << 16) | static_cast<uint32_t>(kCap);

// Sparse saturation. Costs are held as unsigned 16-bit halves and only rows
// k = S-1, S-1-kCapRun, ... of each lane take min(CAP, .); the rows between
// add without a cap: a plain 32-bit add of the two packed words, which is the
// per-half add exactly because no half's sum reaches 2^16 (see below), and
// keeps those rows off the DPX min/max pipe. Every cell lies between min(CAP, exact)
// and the exact cost, and a min3 is at most its `up` input, so the j-th
// uncapped row after a capped one holds at most CAP + j * 4094. Runs are at
// most kCapRun - 1 = 8 rows (also across lanes: row S-1 is capped), so every
// value and every sum before a cap stays below 2^16 (28673 + 9 * 4094 =
// 65519), and each capped row -- the query's last row among them -- equals
// min(CAP, exact), the value of the all-saturating recurrence.
constexpr int kCapRun = 9;

template <int S>
struct StripI16 {
  uint32_t Q[S], NQ[S], G[2][S], Rr[S];
  uint32_t gprev;

  __device__ __forceinline__ void load(const uint32_t *img, int lane) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      Q[k] = img[k * 32 + lane];
      NQ[k] = img[(S + k) * 32 + lane];
    }
  }
  // As if the reference began at the current step: every row, pad rows
  // included, holds CAP (infinity), and the row above a stack's top row held
  // the free-start 0 one step back (gprev). The top row then turns 0 at
  // step 0 (min(up, 0, CAP) + 0; a pad row's distance is 0), each pad row
  // below turns 0 exactly at its own first column, and a real row stays at
  // or above CAP until its first column: infinity under min(CAP, .). No
  // cell is masked; every value is the plain DP's modulo min(CAP, .), which
  // is all the tracked (capped) last row and the segment check look at.
  __device__ __forceinline__ void fresh(long, int, uint32_t ng) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      G[0][k] = kCap2;
      G[1][k] = kCap2;
      Rr[k] = 0u;
    }
    gprev = ng ? kCap2 : 0u;
  }
  // Exact state before step t: G[1] = step t-1, G[0] = step t-2, and the
  // reference samples the cells used at step t-1 (from the global image).
  __device__ __forceinline__ void restore(const uint32_t *st, const uint32_t *gref, long t, int lane, uint32_t ng) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      G[1][k] = st[k * 32 + lane];
      G[0][k] = st[(S + k) * 32 + lane];
      Rr[(1 + k) % S] = gref[t - 1 - static_cast<long>(lane) * S - k];
    }
    const uint32_t g = __shfl_up_sync(kFull, G[0][S - 1], 1);
    gprev = ng ? g : 0u;
  }
  __device__ __forceinline__ void save(uint32_t *st, int lane) const {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      st[k * 32 + lane] = G[1][k];
      st[(S + k) * 32 + lane] = G[0][k];
    }
  }

  __device__ __forceinline__ void chunk(const uint32_t *ref, int lane, uint32_t *ring, int e0, uint32_t ng,
                                        bool tracked, int, int) {
    constexpr int U = Geo<S>::U;
    LaneWindow<S> win;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = (S - (u % S)) % S;
      const int a = (u + 1) & 1;
      const int b = u & 1;
      uint32_t gup = __shfl_up_sync(kFull, G[a][S - 1], 1);
      // A stack's first lane needs the free-start row, 0, above it. Strips
      // of fewer than kMaxS rows per lane are planned with a pad row on top
      // of every stack, which stays 0 whatever comes from above (its own
      // previous value, 0, is in the minimum), so only full-height strips
      // put the zero in.
      if constexpr (S == kMaxS) gup = imad(gup, ng, 0u);
      Rr[p] = win.get(ref, u);  // row 0's reference: column t - lane * S
#pragma unroll
      for (int k = S - 1; k >= 0; --k) {
        const uint32_t r = Rr[(p + k) % S];
        const uint32_t d = __viaddmax_s16x2_relu(r, NQ[k], __vsub2(Q[k], r));  // |q - r| per half
        const uint32_t up = k ? G[a][k - 1] : gup;
        const uint32_t dg = k ? G[b][k - 1] : gprev;
        const uint32_t m = __vimin3_u16x2(up, dg, G[a][k]);
        // rows between caps: one 32-bit add, exact per half (no carry leaves a half: every sum is below 2^16)
        G[b][k] = (S - 1 - k) % kCapRun == 0 ? __viaddmin_u16x2(d, m, kCap2) : m + d;
      }
      gprev = gup;
      // The last row's values of steps u - 1 and u sit in G[0] and G[1]: one
      // 8-byte store every two steps (U is even, the ring 16-byte aligned).
      if ((u & 1) && tracked)
        *reinterpret_cast<uint2 *>(ring + e0 + u - 1) = make_uint2(G[0][S - 1], G[1][S - 1]);
    }
  }
};

struct TrackI16 {
  int ba = 0x7fffffff, bb = 0x7fffffff;
  long ca = -1, cb = -1;
  __device__ __forceinline__ void add(const uint32_t *rg, int j, long c) {
    const uint32_t v = rg[j];
    const int va = static_cast<int>(v & 0xffffu);
    const int vb = static_cast<int>(v >> 16);
    if (va < ba) { ba = va; ca = c; }
    if (vb < bb) { bb = vb; cb = c; }
  }
  __device__ __forceinline__ void reduce(int width) {  // over aligned groups of `width` lanes
    for (int o = width >> 1; o > 0; o >>= 1) {
      int oa = __shfl_xor_sync(kFull, ba, o), ob = __shfl_xor_sync(kFull, bb, o);
      long pa = __shfl_xor_sync(kFull, ca, o), pb = __shfl_xor_sync(kFull, cb, o);
      if (oa < ba || (oa == ba && static_cast<unsigned long>(pa) < static_cast<unsigned long>(ca))) { ba = oa; ca = pa; }
      if (ob < bb || (ob == bb && static_cast<unsigned long>(pb) < static_cast<unsigned long>(cb))) { bb = ob; cb = pb; }
    }
  }
  __device__ __forceinline__ void store(Best *b) const {
    b->ia = ba; b->ib = bb; b->f = 0.0f; b->pad = 0; b->ca = ca; b->cb = cb;
  }
};

// ----------------------------------------------------------------- FP32 --
// CODES: the reference words are int16 codes (q | q << 16) and the query
// samples are int16 codes held as floats: the exact-integer form of the
// int16 arithmetic, run through the FP32 units (see FormOf below).
template <int S, bool CODES>
struct StripF32 {
  float Q[S], W[S], G[2][S], Rr[S];
  float gprev;

  __device__ __forceinline__ static float ref_value(uint32_t w) {
    if constexpr (CODES)
      return __int2float_rn(static_cast<int>(static_cast<short>(w & 0xffffu)));
    else
      return __uint_as_float(w);
  }

  __device__ __forceinline__ void load(const uint32_t *img, int lane) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      Q[k] = __uint_as_float(img[k * 32 + lane]);
      W[k] = __uint_as_float(img[(S + k) * 32 + lane]);
    }
  }
  // As if the reference began at the current step, as in the int16 strip:
  // every row, pad rows included, holds kBig (+inf; sums of these stay
  // finite), and the row above a stack's top row held the free-start 0 one
  // step back. The top row turns 0 at step 0, each pad row below at its own
  // first column, and a real row stays at kBig or above until its first
  // column whatever reference samples its lane reads before the start.
  __device__ __forceinline__ void fresh(long, int, uint32_t ng) {
    const float kBig = 1.0e30f;
#pragma unroll
    for (int k = 0; k < S; ++k) {
      G[0][k] = kBig;
      G[1][k] = kBig;
      Rr[k] = 0.0f;
    }
    gprev = ng ? kBig : 0.0f;
  }
  __device__ __forceinline__ void restore(const uint32_t *st, const uint32_t *gref, long t, int lane, uint32_t ng) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      G[1][k] = __uint_as_float(st[k * 32 + lane]);
      G[0][k] = __uint_as_float(st[(S + k) * 32 + lane]);
      Rr[(1 + k) % S] = ref_value(gref[t - 1 - static_cast<long>(lane) * S - k]);
    }
    const float g = __shfl_up_sync(kFull, G[0][S - 1], 1);
    gprev = ng ? g : 0.0f;
  }
  __device__ __forceinline__ void save(uint32_t *st, int lane) const {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      st[k * 32 + lane] = __float_as_uint(G[1][k]);
      st[(S + k) * 32 + lane] = __float_as_uint(G[0][k]);
    }
  }

  __device__ __forceinline__ void chunk(const uint32_t *ref, int lane, uint32_t *ring, int e0, uint32_t ng,
                                        bool tracked, int, int) {
    constexpr int U = Geo<S>::U;
    LaneWindow<S> win;
    RingStore<U> out;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = (S - (u % S)) % S;
      const int a = (u + 1) & 1;
      const int b = u & 1;
      float gup = __shfl_up_sync(kFull, G[a][S - 1], 1);
      // The free-start row above a stack's first lane: a pad row on top of
      // the stack (weight 0, value 0) keeps it for strips of fewer than
      // kMaxS rows per lane, as in the int16 strip.
      if constexpr (S == kMaxS) gup = ng ? gup : 0.0f;
      Rr[p] = ref_value(win.get(ref, u));  // row 0's reference: column t - lane * S
#pragma unroll
      for (int k = S - 1; k >= 0; --k) {
        const float r = Rr[(p + k) % S];
        // q - r rounded once on real rows (weight -1), exactly 0 on pad rows
        // (weight 0, q = 0); off the critical path, so the cost update that
        // depends on the minimum is a plain add
        const float d = __fmaf_rn(r, W[k], Q[k]);
        const float up = k ? G[a][k - 1] : gup;
        const float dg = k ? G[b][k - 1] : gprev;
        const float m = fmin3f(up, dg, G[a][k]);
        G[b][k] = __fadd_rn(fabsf(d), m);
      }
      gprev = gup;
      out.put(ring, e0, u, tracked, __float_as_uint(G[b][S - 1]));
    }
  }
};

struct TrackF32 {
  float best;
  long col;
  __device__ TrackF32() : best(__builtin_huge_valf()), col(-1) {}
  __device__ __forceinline__ void add(const uint32_t *rg, int j, long c) {
    const float f = __uint_as_float(rg[j]);
    if (f < best) { best = f; col = c; }
  }
  __device__ __forceinline__ void reduce(int width) {  // over aligned groups of `width` lanes
    for (int o = width >> 1; o > 0; o >>= 1) {
      float ob = __shfl_xor_sync(kFull, best, o);
      long oc = __shfl_xor_sync(kFull, col, o);
      if (ob < best || (ob == best && static_cast<unsigned long>(oc) < static_cast<unsigned long>(col))) {
        best = ob;
        col = oc;
      }
    }
  }
  __device__ __forceinline__ void store(Best *b) const {
    b->ia = 0; b->ib = 0; b->f = best; b->pad = 0; b->ca = col; b->cb = -1;
  }
};

// ------------------------------------------------------ start columns --
// The FP32 strip that also carries each cell's alignment start column: a
// cell takes the start of its up neighbour if that is a minimum
// predecessor, else of its diagonal one if that is, else of its left one.
// Pad rows (weight 0, cost 0) take their up neighbour's start on the cost
// tie, so they pass down "my own column" from the row injected above the
// first lane of a stack (the row above row i processed column t - i at
// step t - 1); the first real row therefore starts its paths at its own
// column, like the free-start row of Eq. 1. CODES as for StripF32.
template <int S, bool CODES>
struct StripF32Span {
  float Q[S], W[S], G[2][S], Rr[S];
  int P[2][S];
  float gprev;
  int pprev;

  __device__ __forceinline__ static float ref_value(uint32_t w) {
    if constexpr (CODES)
      return __int2float_rn(static_cast<int>(static_cast<short>(w & 0xffffu)));
    else
      return __uint_as_float(w);
  }
  __device__ __forceinline__ void load(const uint32_t *img, int lane) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      Q[k] = __uint_as_float(img[k * 32 + lane]);
      W[k] = __uint_as_float(img[(S + k) * 32 + lane]);
    }
  }
  // As in StripF32: every row starts at kBig and the free-start zero reaches
  // each row at its first column (a stack's top row takes the injected row
  // above it, 0 with the current column, every step), so each pad row passes
  // down its own column from then on. Before step t_start row i = lane * S +
  // k held column t_start - 1 - i (t_start - 2 - i one step earlier); those
  // starts belong to values at kBig, which no finite cost takes.
  __device__ __forceinline__ void fresh(long t_start, int lane, uint32_t ng) {
    const float kBig = 1.0e30f;
#pragma unroll
    for (int k = 0; k < S; ++k) {
      G[0][k] = kBig;
      G[1][k] = kBig;
      Rr[k] = 0.0f;
      const int i = lane * S + k;
      P[1][k] = static_cast<int>(t_start) - 1 - i;
      P[0][k] = static_cast<int>(t_start) - 2 - i;
    }
    gprev = ng ? kBig : 0.0f;
    pprev = static_cast<int>(t_start) - 1 - lane * S;  // the row above row 0 at step t_start - 2
  }
  // States hold G (2S rows of 32 words) then P (2S rows).
  __device__ __forceinline__ void restore(const uint32_t *st, const uint32_t *gref, long t, int lane, uint32_t ng) {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      G[1][k] = __uint_as_float(st[k * 32 + lane]);
      G[0][k] = __uint_as_float(st[(S + k) * 32 + lane]);
      P[1][k] = static_cast<int>(st[(2 * S + k) * 32 + lane]);
      P[0][k] = static_cast<int>(st[(3 * S + k) * 32 + lane]);
      Rr[(1 + k) % S] = ref_value(gref[t - 1 - static_cast<long>(lane) * S - k]);
    }
    const float g = __shfl_up_sync(kFull, G[0][S - 1], 1);
    const int pg = __shfl_up_sync(kFull, P[0][S - 1], 1);
    gprev = ng ? g : 0.0f;
    pprev = ng ? pg : static_cast<int>(t) - 1 - lane * S;
  }
  __device__ __forceinline__ void save(uint32_t *st, int lane) const {
#pragma unroll
    for (int k = 0; k < S; ++k) {
      st[k * 32 + lane] = __float_as_uint(G[1][k]);
      st[(S + k) * 32 + lane] = __float_as_uint(G[0][k]);
      st[(2 * S + k) * 32 + lane] = static_cast<uint32_t>(P[1][k]);
      st[(3 * S + k) * 32 + lane] = static_cast<uint32_t>(P[0][k]);
    }
  }

  // t0: the absolute step of the chunk's first step; top: the first row of
  // this lane's stack (0, or 16 * S in the lower stack). The ring's start
  // columns sit 128 words after the costs.
  __device__ __forceinline__ void chunk(const uint32_t *ref, int lane, uint32_t *ring, int e0, uint32_t ng,
                                        bool tracked, int t0, int top) {
    constexpr int U = Geo<S>::U;
    LaneWindow<S> win;
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int p = (S - (u % S)) % S;
      const int a = (u + 1) & 1;
      const int b = u & 1;
      float gup = __shfl_up_sync(kFull, G[a][S - 1], 1);
      int pup = __shfl_up_sync(kFull, P[a][S - 1], 1);
      gup = ng ? gup : 0.0f;             // a stack's first lane: the free-start row, 0 ...
      pup = ng ? pup : t0 + u - top;      // ... whose row processed column t - top at step t - 1
      Rr[p] = ref_value(win.get(ref, u));  // row 0's reference: column t - lane * S
#pragma unroll
      for (int k = S - 1; k >= 0; --k) {
        const float r = Rr[(p + k) % S];
        const float d = __fmaf_rn(r, W[k], Q[k]);  // q - r on real rows, 0 on pad rows
        const float up = k ? G[a][k - 1] : gup;
        const int pu = k ? P[a][k - 1] : pup;
        const float dg = k ? G[b][k - 1] : gprev;
        const int pd = k ? P[b][k - 1] : pprev;
        const float m = fmin3f(up, dg, G[a][k]);
        // The start of the preferred minimum predecessor: up, else diagonal, else left.
        G[b][k] = __fadd_rn(fabsf(d), m);
        P[b][k] = sel_eq(up, m, pu, sel_eq(dg, m, pd, P[a][k]));
      }
      gprev = gup;
      pprev = pup;
      if (tracked) {
        ring[e0 + u] = __float_as_uint(G[b][S - 1]);
        ring[2 * flush_words(kPrecF32Span) + e0 + u] = static_cast<uint32_t>(P[b][S - 1]);
      }
    }
  }
};

struct TrackF32Span {
  float best;
  long col;
  int start;
  __device__ TrackF32Span() : best(__builtin_huge_valf()), col(-1), start(-1) {}
  __device__ __forceinline__ void add(const uint32_t *rg, int j, long c) {
    const float f = __uint_as_float(rg[j]);
    if (f < best) { best = f; col = c; start = static_cast<int>(rg[2 * flush_words(kPrecF32Span) + j]); }
  }
  __device__ __forceinline__ void reduce(int width) {  // over aligned groups of `width` lanes
    for (int o = width >> 1; o > 0; o >>= 1) {
      float ob = __shfl_xor_sync(kFull, best, o);
      long oc = __shfl_xor_sync(kFull, col, o);
      int os = __shfl_xor_sync(kFull, start, o);
      if (ob < best || (ob == best && static_cast<unsigned long>(oc) < static_cast<unsigned long>(col))) {
        best = ob;
        col = oc;
        start = os;
      }
    }
  }
  __device__ __forceinline__ void store(Best *b) const {
    b->ia = 0; b->ib = 0; b->f = best; b->pad = 0; b->ca = col; b->cb = start;
  }
};

// Arithmetic forms of a strip: FP32 queries, int16 pairs (DPX), and int16
// codes computed exactly without saturation: wide accumulation (every cost
// of a query of <= 512 events is an integer below 512 * 4094 < 2^24, so FP32
// holds it exactly).
constexpr int kFormF32 = 0, kFormI16 = 1, kFormExactWide = 3;
// and the FP32 and wide forms carrying the start column
constexpr int kFormF32Span = 4, kFormWideSpan = 5;
// Rows of 32 words in a saved strip state, per strip row: two oblique
// columns of costs, and of start columns in the span forms.
template <int FORM>
constexpr int state_rows_per_s() { return (FORM == kFormF32Span || FORM == kFormWideSpan) ? 4 : 2; }

template <int FORM, int S>
struct FormOf;
template <int S>
struct FormOf<kFormI16, S> {
  using Strip = StripI16<S>;
  using Track = TrackI16;
};
template <int S>
struct FormOf<kFormF32, S> {
  using Strip = StripF32<S, false>;
  using Track = TrackF32;
};
template <int S>
struct FormOf<kFormExactWide, S> {
  using Strip = StripF32<S, true>;
  using Track = TrackF32;
};
template <int S>
struct FormOf<kFormF32Span, S> {
  using Strip = StripF32Span<S, false>;
  using Track = TrackF32Span;
};
template <int S>
struct FormOf<kFormWideSpan, S> {
  using Strip = StripF32Span<S, true>;
  using Track = TrackF32Span;
};

// ----------------------------------------------------------- tile sources --
// Shared state of one CTA.
struct Shared {
  uint64_t full[2];
  int cnt[2];
  int uses[2];
  int group;
  int tile_base;
  int abort;
  int pad;
};

// Reference tiles streamed into shared memory by TMA (the sweep kernel).
// Slot of tile k: the kRefFront columns before the tile, then its
// tile_cols columns, so a lane that reads up to 31 * S columns behind the
// warp's step finds its samples in the current slot.
struct TileStream {
  Shared *sh;
  char *slots;                 // two slots of tile_cols + kRefFront words
  const char *src;             // reference image (column 0; kRefFront zero words before it)
  int tile_cols;               // T_S
  int k_first;                 // first global tile of this group's steps
  int K;                       // tiles in this group's sweep
  int n_active;                // warps consuming this stream
  unsigned long long wait_ns;  // longest single wait
  int *status;

  __device__ void issue(int k) {  // one thread
    const int gk = sh->tile_base + k;
    const int slot = gk & 1;
    const unsigned words = static_cast<unsigned>(tile_cols + kRefFront);
    const unsigned bytes = words * 4u;
    // from column (k_first + k) * tile_cols - kRefFront >= -kRefFront: the
    // image's front pad; 16-byte aligned (tile_cols and kRefFront are
    // multiples of 4 words)
    const long first = static_cast<long>(k_first + k) * tile_cols - kRefFront;
    fence_proxy_async();
    mbar_expect_tx(&sh->full[slot], bytes);
    tma_load_1d(slots + static_cast<size_t>(slot) * words * 4, src + first * 4, bytes, &sh->full[slot]);
    sh->uses[slot] += 1;
  }
  __device__ const uint32_t *acquire(int k) {  // whole warp
    const int gk = sh->tile_base + k;
    const int slot = gk & 1;
    if (!mbar_wait_bounded(&sh->full[slot], (gk >> 1) & 1, now_ns() + wait_ns)) {
      report(status, HARU_ETIMEDOUT);
      sh->abort = 1;
      return nullptr;
    }
    return reinterpret_cast<const uint32_t *>(slots + static_cast<size_t>(slot) * (tile_cols + kRefFront) * 4);
  }
  __device__ void release(int k) {  // lane 0 of a warp
    const int gk = sh->tile_base + k;
    const int slot = gk & 1;
    __threadfence_block();
    const int old = atomicAdd(&sh->cnt[slot], 1);
    if (old == n_active - 1) {
      sh->cnt[slot] = 0;
      __threadfence_block();
      if (k + 2 < K) issue(k + 2);
    }
  }
};

// The reference read straight from global memory (the fix-up kernel), in
// the same layout as a tile slot: the pointer of tile k is at the column
// kRefFront before the tile (inside the image's front pad for tile 0).
struct GlobalTiles {
  const uint32_t *img;
  int tile_cols;
  long k_first;
  __device__ __forceinline__ const uint32_t *acquire(int k) {
    return img + ((k_first + k) * tile_cols - kRefFront);
  }
  __device__ __forceinline__ void release(int) {}
};

// ------------------------------------------------------------ one unit --
// Runs steps [t_start, t_end) of one strip (a query or a pair) and tracks
// the last row over own steps [t_own, t_end). fresh: the strip starts from
// the fresh state at t_start.
// save_start / save_final: where to store the state before step t_own and
// before step t_end (nullptr: not stored). stk: a stacked item (lanes 0..15
// and 16..31 are two strips; each lane tracks its own stack's last row).
// `ring` holds ring_words() words per warp: two flush buffers of W =
// flush_words() words, each filled by the strip's tracked lane between two
// scans (or half by each stack's, the lower stack's at +W/2); forms that
// carry start columns keep them 2W further on. Each flush scans W/32
// entries per lane.
// Returns false on abort.
template <int FORM, int S, class Src>
__device__ bool run_steps(typename FormOf<FORM, S>::Strip &st, typename FormOf<FORM, S>::Track &tr, Src &src,
                          int TS, long t_start, long t_own, long t_end, bool fresh, long N, uint32_t *save_start,
                          uint32_t *save_final, uint32_t *ring, int lane, bool stk) {
  constexpr int U = Geo<S>::U;
  constexpr int W = flush_words(FORM == kFormI16 ? HARU_INT16 : HARU_FP32);
  // chunks between two flushes: a stack's entries fill its share of a buffer
  constexpr int kWhole = W / U > 0 ? W / U : 1;
  constexpr int kHalf = W / 2 / U > 0 ? W / 2 / U : 1;
  constexpr int nscan = W / 32;
  const int F = stk ? kHalf : kWhole;
  // ng: 0 on a lane that starts a stack from the free-start row
  const uint32_t ng = (stk ? (lane & 15) : lane) != 0 ? 1u : 0u;
  const bool tracked = lane == 31 || (stk && lane == 15);
  const int soff = stk && lane >= 16 ? W / 2 : 0;
  const int top = stk && lane >= 16 ? 16 * S : 0;  // first row of this lane's stack
  const long last_row = (stk && lane < 16 ? 16L : 32L) * S - 1;
  const long k_first = t_start / TS;
  const int K = static_cast<int>((t_end + TS - 1) / TS - k_first);
  int fl = 0, buf = 0;
  long tflush = t_start;
  for (int k = 0; k < K; ++k) {
    const uint32_t *tile = src.acquire(k);
    if (!tile) return false;
    // This tile's steps [lo, hi), walked in 32-bit offsets from lo.
    const long tk0 = (k_first + k) * TS;
    const long lo = tk0 > t_start ? tk0 : t_start;
    const long hi = tk0 + TS < t_end ? tk0 + TS : t_end;
    const int n = static_cast<int>(hi - lo);
    const int own_at = (save_start && t_own >= lo && t_own < hi) ? static_cast<int>(t_own - lo) : -1;
    const bool last_tile = t_end <= tk0 + TS;
    // this lane's reference window of the chunk at o: columns from
    // lo + o - lane * S, found at (column - tk0 + kRefFront) in the slot;
    // lane * S <= 31 * kMaxS <= kRefFront keeps it inside the slot
    const uint32_t *tref = tile + (kRefFront + (lo - tk0) - static_cast<long>(lane) * S);
    for (int o = 0; o < n; o += U) {
      if (o == own_at) st.save(save_start, lane);
      uint32_t *rg = ring + buf * W + soff;
      const int tabs = static_cast<int>(lo) + o;
      st.chunk(tref + o, lane, rg, fl * U, ng, tracked, tabs, top);
      if (++fl == F || (last_tile && o + U >= n)) {
        __syncwarp();
        for (int r = 0; r < nscan; ++r) {  // entry j = step tflush + j of this lane's stack
          const int j = stk ? (lane & 15) + 16 * r : lane + 32 * r;
          if (j < fl * U) {
            const long t = tflush + j;
            const long c = t - last_row;
            if (t >= t_own && c >= 0 && c < N) tr.add(rg, j, c);
          }
        }
        tflush += static_cast<long>(fl) * U;
        fl = 0;
        buf ^= 1;
      }
    }
    __syncwarp();
    if (lane == 0) src.release(k);
  }
  if (save_final) st.save(save_final, lane);
  return true;
}

// Speculative sweep of one unit (item, segment) in the sweep kernel.
template <int FORM, int S>
__device__ void sweep_unit(const SdtwArgs &A, TileStream &ts, const Group &g, int item, uint32_t *ring,
                           int lane) {
  typename FormOf<FORM, S>::Strip st;
  typename FormOf<FORM, S>::Track tr;
  st.load(A.img + static_cast<size_t>(item) * kImgStride, lane);
  long t_start, t_own, t_end;
  seg_bounds(S, g.nseg, g.seg, A.N, &t_start, &t_own, &t_end);
  const bool stk0 = A.items[item].stacked != 0;
  st.fresh(t_start, lane, (stk0 ? (lane & 15) : lane) != 0 ? 1u : 0u);
  uint32_t *ss = nullptr, *sf = nullptr;
  const size_t unit = static_cast<size_t>(item) * A.nseg_cap + g.seg;
  constexpr size_t kWords = state_rows_per_s<FORM>() * 16 * 32;
  if (g.seg > 0) ss = A.states + (unit * 2 + 0) * kWords;
  if (g.seg + 1 < g.nseg) sf = A.states + (unit * 2 + 1) * kWords;
  const bool stk = A.items[item].stacked != 0;
  const bool ok =
      run_steps<FORM, S>(st, tr, ts, ts.tile_cols, t_start, t_own, t_end, true, A.N, ss, sf, ring, lane, stk);
  tr.reduce(stk ? 16 : 32);
  if (ok && lane == 0) tr.store(A.bests + unit);
  if (ok && stk && lane == 16) tr.store(A.bests2 + unit);
}

template <int PREC, int S>
__device__ __forceinline__ void sweep_any(const SdtwArgs &A, TileStream &ts, const Group &g, int item,
                                          uint32_t *ring, int lane) {
  if constexpr (PREC == HARU_FP32) {
    sweep_unit<kFormF32, S>(A, ts, g, item, ring, lane);
  } else if constexpr (PREC == HARU_INT16_ACC32) {
    sweep_unit<kFormExactWide, S>(A, ts, g, item, ring, lane);
  } else if constexpr (PREC == kPrecF32Span) {
    sweep_unit<kFormF32Span, S>(A, ts, g, item, ring, lane);
  } else if constexpr (PREC == kPrecWideSpan) {
    sweep_unit<kFormWideSpan, S>(A, ts, g, item, ring, lane);
  } else {
    sweep_unit<kFormI16, S>(A, ts, g, item, ring, lane);
  }
}

// One kernel covers every strip height S = 1..16 (registers are allocated
// for the tallest), fed by one longest-first queue of groups.
template <int PREC, int S = 1>
__device__ __forceinline__ void dispatch_sweep(int s, const SdtwArgs &A, TileStream &ts, const Group &g, int item,
                                               uint32_t *ring, int lane) {
  if constexpr (S <= kMaxS) {
    if (s == S)
      sweep_any<PREC, S>(A, ts, g, item, ring, lane);
    else
      dispatch_sweep<PREC, S + 1>(s, A, ts, g, item, ring, lane);
  }
}

// Up to 12 warps per CTA (3 per scheduler): the int16, FP32 and wide strips
// fit in 168 registers a thread; the start-column strips (~240) up to 8.
template <int PREC>
__global__ void __launch_bounds__(prec_span(PREC) ? 256 : 384, 1) sdtw_kernel(SdtwArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  Shared *sh = reinterpret_cast<Shared *>(smem);
  // layout: Shared (128 B) | per-warp tracking rings | two tile slots
  uint32_t *rings = reinterpret_cast<uint32_t *>(smem + 128);
  constexpr int kRing = ring_words(PREC);
  char *slots = reinterpret_cast<char *>(smem + 128 + A.warps * kRing * 4);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    mbar_init(&sh->full[0], 1);
    mbar_init(&sh->full[1], 1);
    sh->cnt[0] = sh->cnt[1] = 0;
    sh->uses[0] = sh->uses[1] = 0;
    sh->tile_base = 0;
    sh->abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  const int count = A.ints[kIntGroups];
  int *queue = A.ints + kIntQueue;
  for (;;) {
    if (threadIdx.x == 0) sh->group = atomicAdd(queue, 1);
    __syncthreads();
    const int gi = sh->group;
    if (gi >= count || sh->abort) break;
    const Group grp = A.groups[gi];
    const int S = grp.S;
    const int TS = tile_width(S, A.tile_cols);
    long t_start, t_own, t_end;
    seg_bounds(S, grp.nseg, grp.seg, A.N, &t_start, &t_own, &t_end);
    TileStream ts;
    ts.sh = sh;
    ts.slots = slots;
    ts.src = reinterpret_cast<const char *>(A.ref_img);
    ts.tile_cols = TS;
    ts.k_first = static_cast<int>(t_start / TS);
    ts.K = static_cast<int>((t_end + TS - 1) / TS - t_start / TS);
    ts.n_active = grp.count;
    ts.wait_ns = A.wait_ns;
    ts.status = A.ints + kIntStatus;
    if (threadIdx.x == 0) {
      ts.issue(0);
      if (ts.K > 1) ts.issue(1);
    }
    __syncthreads();
    if (warp < grp.count) dispatch_sweep<PREC>(S, A, ts, grp, grp.first + warp, rings + warp * kRing, lane);
    __syncthreads();
    if (threadIdx.x == 0) sh->tile_base += ts.K;
  }
  // On abort, wait (bounded) for this CTA's copies still in flight before exit.
  __syncthreads();
  if (threadIdx.x == 0 && sh->abort) {
    const unsigned long long dl = now_ns() + A.wait_ns;
    for (int s = 0; s < 2; ++s)
      if (sh->uses[s] > 0) mbar_wait_bounded(&sh->full[s], (sh->uses[s] - 1) & 1, dl);
  }
}

// --------------------------------------------------------------- fix-up --
// One warp per item: verify every segment boundary, recompute segments whose
// speculative start state differs from the exact one, combine the segments'
// last-row minima (smallest cost, then smallest column) and write the
// outputs.
// Segment minima combine in segment order: the smaller cost wins, and on a
// tie the earlier segment's (smaller) column stays.
template <int FORM>
__device__ __forceinline__ void combine(Best &b, const Best &o) {
  if (FORM == kFormI16) {
    if (o.ia < b.ia) { b.ia = o.ia; b.ca = o.ca; }
    if (o.ib < b.ib) { b.ib = o.ib; b.cb = o.cb; }
  } else {
    if (o.f < b.f) { b.f = o.f; b.ca = o.ca; b.cb = o.cb; }  // cb: the start column of the span forms
  }
}

template <int FORM>
__device__ __forceinline__ void write_out(const SdtwArgs &A, const Best &b, int qa, int qb) {
  if (qa < 0) return;
  if (FORM == kFormI16) {
    A.out_cost[qa] = static_cast<float>(b.ia) * A.inv_scale;
    A.out_col[qa] = b.ca;
    if (qb >= 0) {
      A.out_cost[qb] = static_cast<float>(b.ib) * A.inv_scale;
      A.out_col[qb] = b.cb;
    }
  } else if (FORM == kFormExactWide || FORM == kFormWideSpan) {
    A.out_cost[qa] = b.f * A.inv_scale;
    A.out_col[qa] = b.ca;
  } else {
    A.out_cost[qa] = b.f;
    A.out_col[qa] = b.ca;
  }
  if (FORM == kFormF32Span || FORM == kFormWideSpan) A.out_start[qa] = b.cb;
}

template <int FORM, int S>
__device__ void fixup_item(const SdtwArgs &A, int item, uint32_t *ring, int lane) {
  const Item it = A.items[item];
  const int nseg = it.nseg;
  const bool stk = it.stacked != 0;
  const size_t base = static_cast<size_t>(item) * A.nseg_cap;
  Best b = A.bests[base];
  Best b2 = stk ? A.bests2[base] : b;
  if (nseg > 1) {
    typename FormOf<FORM, S>::Strip st;
    st.load(A.img + static_cast<size_t>(item) * kImgStride, lane);
    const int TS = tile_width(S, A.tile_cols);
    const uint32_t ng = (stk ? (lane & 15) : lane) != 0 ? 1u : 0u;
    constexpr int kRows = state_rows_per_s<FORM>();
    constexpr size_t kWords = kRows * 16 * 32;
    for (int s = 1; s < nseg; ++s) {
      // The segment is exact iff its speculative start state (costs, and
      // start columns in the span forms) equals the previous segment's final one.
      const uint32_t *exact = A.states + ((base + s - 1) * 2 + 1) * kWords;
      const uint32_t *spec = A.states + ((base + s) * 2 + 0) * kWords;
      // (int16: equal modulo min(CAP, .), which fixes every later capped value)
      bool eq = true;
      for (int k = 0; k < kRows * S; ++k) {
        const uint32_t x = exact[k * 32 + lane], y = spec[k * 32 + lane];
        eq = eq && (FORM == kFormI16 ? __vminu2(x, kCap2) == __vminu2(y, kCap2) : x == y);
      }
      if (!__all_sync(kFull, eq)) {
        long t_start, t_own, t_end;
        seg_bounds(S, nseg, s, A.N, &t_start, &t_own, &t_end);
        st.restore(exact, reinterpret_cast<const uint32_t *>(A.ref_img), t_own, lane, ng);
        typename FormOf<FORM, S>::Track tr;
        GlobalTiles src{reinterpret_cast<const uint32_t *>(A.ref_img), TS, t_own / TS};
        uint32_t *sf = s + 1 < nseg ? A.states + ((base + s) * 2 + 1) * kWords : nullptr;
        run_steps<FORM, S>(st, tr, src, TS, t_own, t_own, t_end, false, A.N, nullptr, sf, ring, lane, stk);
        tr.reduce(stk ? 16 : 32);
        if (lane == 0) {
          tr.store(A.bests + base + s);
          atomicAdd(A.ints + kIntFixups, 1);
        }
        if (stk && lane == 16) tr.store(A.bests2 + base + s);
        __syncwarp();
      }
      combine<FORM>(b, A.bests[base + s]);
      if (stk) combine<FORM>(b2, A.bests2[base + s]);
    }
  }
  if (lane == 0) {
    write_out<FORM>(A, b, it.qa, it.qb);
    if (stk) write_out<FORM>(A, b2, it.qc, it.qd);
  }
}

template <int PREC, int S>
__device__ __forceinline__ void fixup_any(const SdtwArgs &A, int item, uint32_t *ring, int lane) {
  if constexpr (PREC == HARU_FP32) {
    fixup_item<kFormF32, S>(A, item, ring, lane);
  } else if constexpr (PREC == HARU_INT16_ACC32) {
    fixup_item<kFormExactWide, S>(A, item, ring, lane);
  } else if constexpr (PREC == kPrecF32Span) {
    fixup_item<kFormF32Span, S>(A, item, ring, lane);
  } else if constexpr (PREC == kPrecWideSpan) {
    fixup_item<kFormWideSpan, S>(A, item, ring, lane);
  } else {
    fixup_item<kFormI16, S>(A, item, ring, lane);
  }
}

template <int PREC, int S = 1>
__device__ __forceinline__ void dispatch_fixup(int s, const SdtwArgs &A, int item, uint32_t *ring, int lane) {
  if constexpr (S <= kMaxS) {
    if (s == S)
      fixup_any<PREC, S>(A, item, ring, lane);
    else
      dispatch_fixup<PREC, S + 1>(s, A, item, ring, lane);
  }
}

constexpr int kFixWarps = 4;

template <int PREC>
__global__ void __launch_bounds__(kFixWarps * 32) fixup_kernel(SdtwArgs A) {
  __shared__ __align__(16) uint32_t rings[kFixWarps * ring_words(PREC)];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int count = A.ints[kIntItems];
  const int item = blockIdx.x * kFixWarps + warp;
  if (item >= count) return;
  dispatch_fixup<PREC>(A.items[item].S, A, item, rings + warp * ring_words(PREC), lane);
}

template <int PREC>
cudaError_t launch_sweep_prec(const SdtwArgs &a, int grid, cudaStream_t s) {
  static SmemOptIn opt;
  const size_t sm = sdtw_smem_bytes(PREC, a.tile_cols, a.warps);
  cudaError_t e = opt_in_smem(sdtw_kernel<PREC>, opt, sm);
  if (e != cudaSuccess) return e;
  sdtw_kernel<PREC><<<grid, a.warps * 32, sm, s>>>(a);
  return cudaGetLastError();
}

template <int PREC>
cudaError_t launch_fixup_prec(const SdtwArgs &a, int fix_items, cudaStream_t s) {
  if (fix_items <= 0) return cudaSuccess;
  fixup_kernel<PREC><<<(fix_items + kFixWarps - 1) / kFixWarps, kFixWarps * 32, 0, s>>>(a);
  return cudaGetLastError();
}

template <int PREC>
int occupancy_prec(int tile_cols, int warps) {
  int n = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sdtw_kernel<PREC>, warps * 32,
                                                sdtw_smem_bytes(PREC, tile_cols, warps));
  return n;
}

}  // namespace
}  // namespace haru

// Define the entry points of the sweep kernel (launch, occupancy) or of the
// segment fix-up kernel for kernel precision P (0 FP32, 1 INT16, 2 int16
// inputs with wide accumulation, 3 FP32 with start columns, 4 wide with start
// columns); one per translation unit, so the kernels compile in parallel.
#define HARU_SDTW_SWEEP_INSTANCE(P)                                                            \
  namespace haru {                                                                             \
  cudaError_t sdtw_sweep_##P(const SdtwArgs &a, int grid, cudaStream_t s) {                   \
    return launch_sweep_prec<P>(a, grid, s);                                                   \
  }                                                                                            \
  int sdtw_occupancy_##P(int tile_cols, int warps) { return occupancy_prec<P>(tile_cols, warps); } \
  cudaError_t sdtw_sweep_load_##P() {                                                          \
    cudaFuncAttributes f;                                                                      \
    return cudaFuncGetAttributes(&f, sdtw_kernel<P>);                                          \
  }                                                                                            \
  }
#define HARU_SDTW_FIXUP_INSTANCE(P)                                                            \
  namespace haru {                                                                             \
  cudaError_t sdtw_fixup_##P(const SdtwArgs &a, int fix_items, cudaStream_t s) {              \
    return launch_fixup_prec<P>(a, fix_items, s);                                              \
  }                                                                                            \
  cudaError_t sdtw_fixup_load_##P() {                                                          \
    cudaFuncAttributes f;                                                                      \
    return cudaFuncGetAttributes(&f, fixup_kernel<P>);                                         \
  }                                                                                            \
  }
