// The sDTW wavefront kernels (Eq. 1, Section 2.3; the pipelined oblique column
// of Section 4.3 / Fig. 5, mapped onto warps).
//
// Layout of one warp's work. A query of M events is padded at the top to
// 32 * S rows (S = ceil(M / 32)); lane l holds rows l*S .. l*S + S - 1 in
// registers. Row i processes reference column t - i at step t, so every row
// is one processing element of the paper's PE chain and the whole strip is
// one oblique column: the S cells of a lane in one step are independent
// (instruction-level parallelism S), a cell reads
//   up   = row i-1 at step t-1,  diag = row i-1 at step t-2,  left = row i at step t-1,
// and each step one value (the bottom row's cost) and the reference sample
// it used cross from lane l-1 to lane l by __shfl_up_sync. Lane 0 injects
// reference sample t and the free-start row gamma(0, .) = 0. A sweep is
// N + 32*S - 1 steps, the paper's N + M - 1 (Section 4.3) for the padded
// height. Pad rows sit above the query and hold exactly 0, the free-start
// boundary row, so the last query row is always lane 31's last register.
//
// INT16 form: two queries share a warp, one per 16-bit half (DPX
// __vimin3_s16x2 / __viaddmin_s16x2 / __viaddmax_s16x2); costs saturate at
// CAP, pad rows have cap 0. FP32 form: one query per warp, 3-input min.f32,
// pad rows have weight 0 in gamma = fma(|q - r|, w, min3).
//
// The reference streams through shared memory: every CTA sweeps a group of
// warps (same S) over the same columns; tiles of T_S columns are fetched by
// cp.async.bulk (TMA) into a two-slot ring guarded by mbarriers. The warp
// that releases a slot last issues the copy of the tile two ahead.
//
// The last-row minimum and its first column (Algorithm 1's final scan,
// Algorithm 2's per-column compare) are tracked through a small per-warp
// shared ring: lane 31 stores its bottom-row cost every step, and every
// <= 32 steps each lane scans one stored value; a warp reduction at the end
// keeps the smallest cost, then the smallest column.
//
// Every wait is bounded by a global-timer deadline; on expiry the kernel
// records HARU_ETIMEDOUT, waits (bounded) for its own copies in flight and
// returns.

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

constexpr int cx_gcd(int a, int b) { return b == 0 ? a : cx_gcd(b, a % b); }
constexpr int cx_lcm(int a, int b) { return a / cx_gcd(a, b) * b; }

template <int S>
struct Geo {
  static constexpr int U = (S % 2 == 0) ? S : 2 * S;  // steps per unrolled chunk (register renaming period)
  static constexpr int F = (32 / U) > 0 ? (32 / U) : 1; // chunks per tracking flush
  static constexpr int E = F * U;                      // tracked steps per flush (<= 32)
  static constexpr int L = cx_lcm(U, 4);               // tile widths are multiples of L
};

__host__ __device__ inline int tile_width(int S, int T) {
  int U = (S % 2 == 0) ? S : 2 * S;
  int g = U % 4 == 0 ? 4 : (U % 2 == 0 ? 2 : 1);
  int L = U / g * 4;  // lcm(U, 4)
  int w = (T / L) * L;
  return w > 0 ? w : L;
}

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

struct TileStream {
  Shared *sh;
  char *slots;                 // 2 slots of slot_bytes
  const char *src;             // reference image
  int tile_cols;               // T_S
  int K;                       // tiles in this group's sweep
  int n_active;                // warps consuming this stream
  unsigned long long wait_ns;  // longest single wait

  __device__ void issue(int k) {  // one thread
    int gk = sh->tile_base + k;
    int slot = gk & 1;
    unsigned bytes = static_cast<unsigned>(tile_cols) * 4u;
    fence_proxy_async();
    mbar_expect_tx(&sh->full[slot], bytes);
    tma_load_1d(slots + static_cast<size_t>(slot) * tile_cols * 4, src + static_cast<size_t>(k) * tile_cols * 4,
                bytes, &sh->full[slot]);
    sh->uses[slot] += 1;
  }
  __device__ const char *acquire(int k, int *status) {  // whole warp
    int gk = sh->tile_base + k;
    int slot = gk & 1;
    if (!mbar_wait_bounded(&sh->full[slot], (gk >> 1) & 1, now_ns() + wait_ns)) {
      report(status, HARU_ETIMEDOUT);
      sh->abort = 1;
      return nullptr;
    }
    return slots + static_cast<size_t>(slot) * tile_cols * 4;
  }
  __device__ void release(int k) {  // lane 0 of a warp
    int gk = sh->tile_base + k;
    int slot = gk & 1;
    __threadfence_block();
    int old = atomicAdd(&sh->cnt[slot], 1);
    if (old == n_active - 1) {
      sh->cnt[slot] = 0;
      __threadfence_block();
      if (k + 2 < K) issue(k + 2);
    }
  }
};

// ---------------------------------------------------------------- INT16 --
template <int S, bool MASK>
__device__ __forceinline__ void chunk_i16(const uint32_t (&Q)[S], const uint32_t (&NQ)[S], const uint32_t (&C)[S],
                                          uint32_t (&G)[2][S], uint32_t (&Rr)[S], uint32_t &gprev,
                                          const uint32_t *ref, int t0, int lane, uint32_t *ring, int e0) {
  constexpr int U = Geo<S>::U;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int p = (S - (u % S)) % S;
    const int a = (u + 1) & 1;
    const int b = u & 1;
    uint32_t gup = __shfl_up_sync(kFull, G[a][S - 1], 1);
    uint32_t rin = __shfl_up_sync(kFull, Rr[p], 1);
    const uint32_t rv = ref[u];
    gup = lane ? gup : 0u;
    rin = lane ? rin : rv;
    Rr[p] = rin;
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
      const uint32_t r = Rr[(p + k) % S];
      const uint32_t d = __viaddmax_s16x2(r, NQ[k], __vsub2(Q[k], r));  // |q - r| per half
      const uint32_t up = k ? G[a][k - 1] : gup;
      const uint32_t dg = k ? G[b][k - 1] : gprev;
      const uint32_t m = __vimin3_s16x2(up, dg, G[a][k]);
      uint32_t v = __viaddmin_s16x2(d, m, C[k]);
      if (MASK) v = (t0 + u - lane * S >= k) ? v : C[k];
      G[b][k] = v;
    }
    gprev = gup;
    if (lane == 31) ring[e0 + u] = G[b][S - 1];
  }
}

__device__ __forceinline__ void track_i16(uint32_t v, long c, long N, int &ba, int &bb, long &ca, long &cb) {
  if (c >= 0 && c < N) {
    const int va = static_cast<int>(v & 0xffffu);
    const int vb = static_cast<int>(v >> 16);
    if (va < ba) { ba = va; ca = c; }
    if (vb < bb) { bb = vb; cb = c; }
  }
}

template <int S>
__device__ void sweep_i16(const SdtwArgs &A, TileStream &ts, int item, uint32_t *ring, int lane) {
  constexpr int U = Geo<S>::U, F = Geo<S>::F, E = Geo<S>::E;
  const Item it = A.items[item];
  const uint32_t *img = A.img + static_cast<size_t>(item) * kImgStride;
  uint32_t Q[S], NQ[S], C[S], G[2][S], Rr[S];
#pragma unroll
  for (int k = 0; k < S; ++k) {
    Q[k] = img[k * 32 + lane];
    C[k] = img[(S + k) * 32 + lane];
    NQ[k] = __vsub2(0u, Q[k]);
    G[0][k] = C[k];
    G[1][k] = C[k];
    Rr[k] = 0u;
  }
  uint32_t gprev = 0u;
  int ba = 0x7fffffff, bb = 0x7fffffff;
  long ca = -1, cb = -1;
  const long N = A.N;
  const long total = N + 32L * S - 1;           // steps of the sweep
  const long tstop = (total + U - 1) / U * U;   // whole chunks
  const int TS = ts.tile_cols;                  // multiple of U
  const int K = ts.K;
  const int prologue = 32 * S;                  // masked steps (multiple of U)
  int fl = 0, buf = 0;
  long tflush = 0;
  bool ok = true;
  for (int k = 0; k < K && ok; ++k) {
    const char *tile = ts.acquire(k, A.status);
    if (!tile) { ok = false; break; }
    const uint32_t *tref = reinterpret_cast<const uint32_t *>(tile);
    const long tk0 = static_cast<long>(k) * TS;
    const long tend = tk0 + TS < tstop ? tk0 + TS : tstop;
    for (long t0 = tk0; t0 < tend; t0 += U) {
      const uint32_t *ref = tref + (t0 - tk0);
      uint32_t *rg = ring + buf * 32;
      if (t0 < prologue)
        chunk_i16<S, true>(Q, NQ, C, G, Rr, gprev, ref, static_cast<int>(t0), lane, rg, fl * U);
      else
        chunk_i16<S, false>(Q, NQ, C, G, Rr, gprev, ref, 0, lane, rg, fl * U);
      if (++fl == F || t0 + U >= total) {
        __syncwarp();
        if (lane < fl * U) track_i16(rg[lane], tflush + lane - (32L * S - 1), N, ba, bb, ca, cb);
        tflush += static_cast<long>(fl) * U;
        fl = 0;
        buf ^= 1;
      }
    }
    __syncwarp();
    if (lane == 0) ts.release(k);
  }
  (void)E;
  // warp reduction: smallest cost, then smallest column
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    int oa = __shfl_xor_sync(kFull, ba, o), ob = __shfl_xor_sync(kFull, bb, o);
    long pa = __shfl_xor_sync(kFull, ca, o), pb = __shfl_xor_sync(kFull, cb, o);
    if (oa < ba || (oa == ba && static_cast<unsigned long>(pa) < static_cast<unsigned long>(ca))) { ba = oa; ca = pa; }
    if (ob < bb || (ob == bb && static_cast<unsigned long>(pb) < static_cast<unsigned long>(cb))) { bb = ob; cb = pb; }
  }
  if (lane == 0 && ok) {
    A.out_cost[it.qa] = static_cast<float>(ba) * A.inv_scale;
    A.out_col[it.qa] = ca;
    if (it.qb >= 0) {
      A.out_cost[it.qb] = static_cast<float>(bb) * A.inv_scale;
      A.out_col[it.qb] = cb;
    }
  }
}

// ----------------------------------------------------------------- FP32 --
template <int S>
__device__ __forceinline__ void chunk_f32(const float (&Q)[S], const float (&W)[S], float (&G)[2][S], float (&Rr)[S],
                                          float &gprev, const float *ref, int lane, float *ring, int e0) {
  constexpr int U = Geo<S>::U;
#pragma unroll
  for (int u = 0; u < U; ++u) {
    const int p = (S - (u % S)) % S;
    const int a = (u + 1) & 1;
    const int b = u & 1;
    float gup = __shfl_up_sync(kFull, G[a][S - 1], 1);
    float rin = __shfl_up_sync(kFull, Rr[p], 1);
    const float rv = ref[u];
    gup = lane ? gup : 0.0f;
    rin = lane ? rin : rv;
    Rr[p] = rin;
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
      const float r = Rr[(p + k) % S];
      const float d = __fsub_rn(Q[k], r);
      const float up = k ? G[a][k - 1] : gup;
      const float dg = k ? G[b][k - 1] : gprev;
      const float m = fmin3f(up, dg, G[a][k]);
      G[b][k] = __fmaf_rn(fabsf(d), W[k], m);
    }
    gprev = gup;
    if (lane == 31) ring[e0 + u] = G[b][S - 1];
  }
}

template <int S>
__device__ void sweep_f32(const SdtwArgs &A, TileStream &ts, int item, float *ring, int lane) {
  constexpr int U = Geo<S>::U, F = Geo<S>::F;
  const Item it = A.items[item];
  const uint32_t *img = A.img + static_cast<size_t>(item) * kImgStride;
  float Q[S], W[S], G[2][S], Rr[S];
  const float kBig = 1.0e30f;  // stands for +inf; sums of these stay finite
#pragma unroll
  for (int k = 0; k < S; ++k) {
    Q[k] = __uint_as_float(img[k * 32 + lane]);
    W[k] = __uint_as_float(img[(S + k) * 32 + lane]);
    G[0][k] = W[k] != 0.0f ? kBig : 0.0f;
    G[1][k] = G[0][k];
    Rr[k] = kBig;  // columns before the reference start: distance ~1e30 for real rows
  }
  float gprev = 0.0f;
  float best = __int_as_float(0x7f800000);
  long col = -1;
  const long N = A.N;
  const long total = N + 32L * S - 1;
  const long tstop = (total + U - 1) / U * U;
  const int TS = ts.tile_cols;
  const int K = ts.K;
  int fl = 0, buf = 0;
  long tflush = 0;
  bool ok = true;
  for (int k = 0; k < K && ok; ++k) {
    const char *tile = ts.acquire(k, A.status);
    if (!tile) { ok = false; break; }
    const float *tref = reinterpret_cast<const float *>(tile);
    const long tk0 = static_cast<long>(k) * TS;
    const long tend = tk0 + TS < tstop ? tk0 + TS : tstop;
    for (long t0 = tk0; t0 < tend; t0 += U) {
      float *rg = ring + buf * 32;
      chunk_f32<S>(Q, W, G, Rr, gprev, tref + (t0 - tk0), lane, rg, fl * U);
      if (++fl == F || t0 + U >= total) {
        __syncwarp();
        if (lane < fl * U) {
          const long c = tflush + lane - (32L * S - 1);
          const float v = rg[lane];
          if (c >= 0 && c < N && v < best) { best = v; col = c; }
        }
        tflush += static_cast<long>(fl) * U;
        fl = 0;
        buf ^= 1;
      }
    }
    __syncwarp();
    if (lane == 0) ts.release(k);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    float ob = __shfl_xor_sync(kFull, best, o);
    long oc = __shfl_xor_sync(kFull, col, o);
    if (ob < best || (ob == best && static_cast<unsigned long>(oc) < static_cast<unsigned long>(col))) {
      best = ob;
      col = oc;
    }
  }
  if (lane == 0 && ok) {
    A.out_cost[it.qa] = best;
    A.out_col[it.qa] = col;
  }
}

template <int PREC>
__device__ void dispatch(int S, const SdtwArgs &A, TileStream &ts, int item, uint32_t *ring, int lane) {
#define HARU_CASE(s)                                                             \
  case s:                                                                        \
    if (PREC == HARU_INT16)                                                      \
      sweep_i16<s>(A, ts, item, ring, lane);                                     \
    else                                                                         \
      sweep_f32<s>(A, ts, item, reinterpret_cast<float *>(ring), lane);          \
    break;
  switch (S) {
    HARU_CASE(1) HARU_CASE(2) HARU_CASE(3) HARU_CASE(4) HARU_CASE(5) HARU_CASE(6) HARU_CASE(7) HARU_CASE(8)
    HARU_CASE(9) HARU_CASE(10) HARU_CASE(11) HARU_CASE(12) HARU_CASE(13) HARU_CASE(14) HARU_CASE(15)
    HARU_CASE(16)
    default: break;
  }
#undef HARU_CASE
}

template <int PREC>
__global__ void __launch_bounds__(256, 1) sdtw_kernel(SdtwArgs A) {
  extern __shared__ __align__(128) unsigned char smem[];
  Shared *sh = reinterpret_cast<Shared *>(smem);
  uint32_t *rings = reinterpret_cast<uint32_t *>(smem + 128);
  char *slots = reinterpret_cast<char *>(smem + 128 + A.warps * 64 * 4);
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
  const int n_groups = *A.n_groups;
  for (;;) {
    if (threadIdx.x == 0) sh->group = atomicAdd(A.queue, 1);
    __syncthreads();
    const int g = sh->group;
    if (g >= n_groups || sh->abort) break;
    const Group grp = A.groups[g];
    const int S = grp.S;
    const int TS = tile_width(S, A.tile_cols);
    const long total = A.N + 32L * S - 1;
    TileStream ts;
    ts.sh = sh;
    ts.slots = slots;
    ts.src = reinterpret_cast<const char *>(A.ref_img);
    ts.tile_cols = TS;
    ts.K = static_cast<int>((total + TS - 1) / TS);
    ts.n_active = grp.count;
    ts.wait_ns = A.wait_ns;
    if (threadIdx.x == 0) {
      ts.issue(0);
      if (ts.K > 1) ts.issue(1);
    }
    __syncthreads();
    if (warp < grp.count) dispatch<PREC>(S, A, ts, grp.first + warp, rings + warp * 64, lane);
    __syncthreads();
    if (threadIdx.x == 0) sh->tile_base += ts.K;
  }
  // On abort, wait (bounded) for this CTA's copies still in flight before exit.
  __syncthreads();
  if (threadIdx.x == 0 && sh->abort) {
    unsigned long long dl = now_ns() + A.wait_ns;
    for (int s = 0; s < 2; ++s)
      if (sh->uses[s] > 0) mbar_wait_bounded(&sh->full[s], (sh->uses[s] - 1) & 1, dl);
  }
}

}  // namespace

size_t sdtw_smem_bytes(int tile_cols, int warps) {
  return 128 + static_cast<size_t>(warps) * 64 * 4 + 2 * static_cast<size_t>(tile_cols) * 4;
}

int sdtw_max_ctas_per_sm(int precision, int tile_cols, int warps) {
  int n = 0;
  size_t sm = sdtw_smem_bytes(tile_cols, warps);
  if (precision == HARU_INT16)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sdtw_kernel<HARU_INT16>, warps * 32, sm);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sdtw_kernel<HARU_FP32>, warps * 32, sm);
  return n;
}

cudaError_t launch_sdtw(int precision, const SdtwArgs &a, int grid, cudaStream_t s) {
  size_t sm = sdtw_smem_bytes(a.tile_cols, a.warps);
  cudaError_t e;
  if (precision == HARU_INT16) {
    e = cudaFuncSetAttribute(sdtw_kernel<HARU_INT16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    sdtw_kernel<HARU_INT16><<<grid, a.warps * 32, sm, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(sdtw_kernel<HARU_FP32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             static_cast<int>(sm));
    if (e != cudaSuccess) return e;
    sdtw_kernel<HARU_FP32><<<grid, a.warps * 32, sm, s>>>(a);
  }
  return cudaGetLastError();
}

}  // namespace haru
