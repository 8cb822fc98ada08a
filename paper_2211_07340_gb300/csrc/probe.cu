// The roofline denominator, measured: the cell update of each arithmetic form
// run on independent chains with no wavefront data movement (no shuffles,
// no reference stream, no tracking), as fast as the SM can issue it.

#include <cuda_runtime.h>

#include "engine.h"

namespace haru {
namespace {

constexpr int kChains = 8;
constexpr int kLevels = 4;

__device__ __forceinline__ float fmin3p(float a, float b, float c) {
  float d;
  asm volatile("min.f32 %0, %1, %2, %3;" : "=f"(d) : "f"(a), "f"(b), "f"(c));
  return d;
}

// Each level updates kChains cells (int16: cell pairs) from the previous
// level's values, like one oblique step: d = |q - r|, m = min3, new = d + m
// (int16: saturated at CAP in one chain of eight, as the sweep's rows are).
template <int PREC>
__global__ void probe_kernel(uint32_t *out, int iters) {
  uint32_t a[kChains], x[kChains];
  float f[kChains], g[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    a[i] = threadIdx.x * 977u + i * 0x10001u;
    x[i] = blockIdx.x * 31u + i;
    f[i] = 1.0f + i * 0.001f * threadIdx.x;
    g[i] = 0.5f - i;
  }
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int l = 0; l < kLevels; ++l) {
      uint32_t an[kChains], xn[kChains];
      float fn[kChains], gn[kChains];
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        const int j = (i + 1) % kChains, k = (i + 3) % kChains;
        if (PREC == HARU_INT16) {
          const uint32_t d = __viaddmax_s16x2_relu(x[i], a[k], __vsub2(x[j], x[i]));
          const uint32_t m = __vimin3_u16x2(a[i], a[j], a[k]);
          an[i] = i == 0 ? __viaddmin_u16x2(d, m, x[k]) : __vadd2(m, d);  // one row in eight saturates
          xn[i] = d;
        } else {
          const float t = __fsub_rn(g[i], g[j]);
          const float m = fmin3p(f[i], f[j], f[k]);
          fn[i] = __fmaf_rn(fabsf(t), g[k], m);
          gn[i] = t;
        }
      }
#pragma unroll
      for (int i = 0; i < kChains; ++i) {
        if (PREC == HARU_INT16) {
          a[i] = an[i];
          x[i] = xn[i];
        } else {
          f[i] = fn[i];
          g[i] = gn[i];
        }
      }
    }
  }
  uint32_t r = 0;
#pragma unroll
  for (int i = 0; i < kChains; ++i) r ^= a[i] ^ x[i] ^ __float_as_uint(f[i]) ^ __float_as_uint(g[i]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

}  // namespace
}  // namespace haru

extern "C" int haru_probe_peak(haru_ctx *ctx, int precision, double *cells_per_s) {
  using namespace haru;
  if (!ctx || !cells_per_s || (precision != HARU_FP32 && precision != HARU_INT16)) return HARU_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->mu);
  if (ctx->sticky) return ctx->sticky;
  if (cudaSetDevice(ctx->device) != cudaSuccess) return HARU_ECUDA;
  const int threads = 256, blocks = ctx->sms * 4, iters = 4000;
  uint32_t *out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaMalloc(&out, sizeof(uint32_t) * threads * blocks);
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.0f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {
    if (e == cudaSuccess) e = cudaEventRecord(e0, ctx->stream);
    if (precision == HARU_INT16)
      probe_kernel<HARU_INT16><<<blocks, threads, 0, ctx->stream>>>(out, iters);
    else
      probe_kernel<HARU_FP32><<<blocks, threads, 0, ctx->stream>>>(out, iters);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventRecord(e1, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (rep == 0 || ms < best_ms)) best_ms = ms;
  }
  if (out) cudaFree(out);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess || best_ms <= 0.0f) return HARU_ECUDA;
  const double cells_per_thread_pass = precision == HARU_INT16 ? 2.0 : 1.0;
  const double cells = static_cast<double>(blocks) * threads * iters * kLevels * kChains * cells_per_thread_pass;
  *cells_per_s = cells / (best_ms * 1e-3);
  return HARU_OK;
}
