// haru_sdtw_batch_noalloc: the batch path with its scratch memory in a
// fixed, file-scope device array instead of buffers the library allocates.
//
// Who needs this: callers that cannot let the library call cudaMalloc. A
// service that reserves its whole device-memory budget at start-up and must
// not grow afterwards; a host that forbids run-time device allocation; a
// latency-critical caller that cannot accept cudaMalloc's implicit
// synchronisation, which can stall work queued on its other streams. Such a
// caller owns every input and output buffer (device pointers) and this entry
// point allocates nothing: the planner's items and groups, the packed query
// images and the status and work-queue counters all live in `scratch` below,
// which every GPU that loads the library holds until the process exits.
//
// The paper has no counterpart; it is an interface option of this library.

#include <cuda_runtime.h>

#include <mutex>

#include "engine.h"

namespace haru {
namespace {

// Layout of the scratch array (bytes): the status and counter words, then
// items, groups, per-item last-row minima (upper and lower stacks), the per-item register images
// for up to HARU_NOALLOC_MAX_QUERIES queries (the FP32 form needs one item
// per query, the int16 form one per pair) and each query's mean and sigma
// (raw events). This path never splits the reference into segments, so it
// needs no saved states.
constexpr size_t kNaItems = HARU_NOALLOC_MAX_QUERIES + kMaxS;  // items_bound(0, max), >= items_bound(1, max)
constexpr size_t kNaHead = 256;  // kIntWords status and counter words
constexpr size_t kNaItemsOff = kNaHead;
constexpr size_t kNaGroupsOff = kNaItemsOff + ((kNaItems * sizeof(Item) + 255) / 256) * 256;
constexpr size_t kNaBestsOff = kNaGroupsOff + ((kNaItems * sizeof(Group) + 255) / 256) * 256;
constexpr size_t kNaImgOff = kNaBestsOff + ((2 * kNaItems * sizeof(Best) + 255) / 256) * 256;
constexpr size_t kNaStatsOff = kNaImgOff + ((kNaItems * kImgStride * sizeof(uint32_t) + 255) / 256) * 256;
constexpr size_t kNaBytes = kNaStatsOff + 2 * HARU_NOALLOC_MAX_QUERIES * sizeof(double);
// The size include/haru.h states for this array.
static_assert(kNaBytes == 4409600, "the documented scratch size (4,409,600 bytes) is out of date");

static __device__ __align__(256) unsigned char scratch[kNaBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_ptr[kMaxDevices] = {nullptr};

// Device address of `scratch` on `device` (current). Looked up once per
// device; the first lookup may load the module.
cudaError_t scratch_on(int device, unsigned char **out) {
  if (device < 0 || device >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_ptr[device]) {
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, scratch);
    if (e != cudaSuccess) return e;
    if (!p) return cudaErrorInvalidSymbol;
    g_ptr[device] = p;
  }
  *out = static_cast<unsigned char *>(g_ptr[device]);
  return cudaSuccess;
}

}  // namespace

// Reference access and sticky CUDA errors for the no-allocation path (defined in api.cu).
int ctx_reference(haru_ctx *ctx, int precision, const void **img, long *N, int *scale_log2, int *device,
                  cudaStream_t *stream, int *warps, int *tile, unsigned long long *wait, int *per_sm, int *sms);
int ctx_cuda_fail(haru_ctx *ctx, cudaError_t e);

}  // namespace haru

extern "C" int haru_sdtw_batch_noalloc(haru_ctx *ctx, int precision, const float *events, const uint32_t *offsets,
                                       uint32_t nq, float *out_cost, int64_t *out_col, uintptr_t stream,
                                       uint32_t flags) {
  using namespace haru;
  if (!ctx) return HARU_EINVAL;
  if (precision != HARU_FP32 && precision != HARU_INT16) return HARU_EINVAL;
  if (nq > HARU_NOALLOC_MAX_QUERIES) return HARU_EINVAL;
  if (flags & ~static_cast<uint32_t>(HARU_RAW)) return HARU_EINVAL;
  if (nq == 0) return HARU_OK;
  if (!events || !offsets || !out_cost || !out_col) return HARU_EINVAL;
  const void *img = nullptr;
  long N = 0;
  int scale = 0, device = 0, warps = 0, tile = 0, per_sm = 0, sms = 0;
  unsigned long long wait = 0;
  cudaStream_t own = nullptr;
  int rc = ctx_reference(ctx, precision, &img, &N, &scale, &device, &own, &warps, &tile, &wait, &per_sm, &sms);
  if (rc != HARU_OK) return rc;
  cudaError_t e = cudaSetDevice(device);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e);
  unsigned char *base = nullptr;
  e = scratch_on(device, &base);
  if (e != cudaSuccess) return ctx_cuda_fail(ctx, e);
  cudaStream_t s = stream ? reinterpret_cast<cudaStream_t>(stream) : own;
  int *status = reinterpret_cast<int *>(base);
  Item *items = reinterpret_cast<Item *>(base + kNaItemsOff);
  Group *groups = reinterpret_cast<Group *>(base + kNaGroupsOff);
  Best *bests = reinterpret_cast<Best *>(base + kNaBestsOff);
  uint32_t *imgs = reinterpret_cast<uint32_t *>(base + kNaImgOff);
  double *qstats = reinterpret_cast<double *>(base + kNaStatsOff);
  const size_t max_items = items_bound(precision == HARU_INT16 ? 1 : 0, nq);

  // The array keeps the previous call's contents: the status word and the
  // counters must start at zero; items, groups and images are rewritten.
  if ((e = cudaMemsetAsync(status, 0, kIntWords * sizeof(int), s)) != cudaSuccess) return ctx_cuda_fail(ctx, e);
  PlanArgs pa;
  pa.offsets = offsets;
  pa.nq = nq;
  pa.N = N;
  pa.pair = precision == HARU_INT16;
  pa.warps = warps;
  pa.units_target = 1;
  pa.stack = 0;  // at most HARU_NOALLOC_MAX_QUERIES queries: latency over throughput
  pa.nseg_cap = 1;
  pa.items = items;
  pa.groups = groups;
  pa.ints = status;
  if ((e = launch_plan(pa, s)) != cudaSuccess) return ctx_cuda_fail(ctx, e);
  if ((flags & HARU_RAW) &&
      (e = launch_qstats(events, offsets, nq, qstats, status + kIntStatus, s)) != cudaSuccess)
    return ctx_cuda_fail(ctx, e);
  PackArgs ka;
  ka.events = events;
  ka.offsets = offsets;
  ka.items = items;
  ka.n_items = status + kIntItems;
  ka.img = imgs;
  ka.raw = (flags & HARU_RAW) ? 1 : 0;
  ka.qstats = qstats;
  ka.pair = pa.pair;
  ka.scale_log2 = scale;
  ka.status = status + kIntStatus;
  if ((e = launch_pack(ka, static_cast<uint32_t>(max_items), s)) != cudaSuccess) return ctx_cuda_fail(ctx, e);
  SdtwArgs sa;
  sa.ref_img = img;
  sa.N = N;
  sa.img = imgs;
  sa.items = items;
  sa.groups = groups;
  sa.ints = status;
  sa.states = nullptr;
  sa.bests = bests;
  sa.bests2 = bests + kNaItems;
  sa.nseg_cap = 1;
  sa.out_cost = out_cost;
  sa.out_col = out_col;
  sa.inv_scale = 1.0f / static_cast<float>(1 << scale);
  sa.tile_cols = tile;
  sa.warps = warps;
  sa.wait_ns = wait;
  const size_t groups_max = (max_items + warps - 1) / warps + kMaxS;
  const int cps = per_sm > 0 ? per_sm : sdtw_max_ctas_per_sm(precision, tile, warps);
  size_t grid = static_cast<size_t>(sms) * (cps > 0 ? cps : 1);
  if (grid > groups_max) grid = groups_max;
  if ((e = launch_sdtw(precision, sa, static_cast<int>(grid), static_cast<int>(max_items), s)) != cudaSuccess)
    return ctx_cuda_fail(ctx, e);
  int st = 0;
  if ((e = cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return ctx_cuda_fail(ctx, e);
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return ctx_cuda_fail(ctx, e);
  return st;
}
