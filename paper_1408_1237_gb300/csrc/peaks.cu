// Issue-rate microbenchmarks for the ALU roofline of the kernel product:
// MUFU.EX2 (ex2.approx.ftz.f32), scalar FFMA and packed FFMA2 (f32x2)
// results per second on this GPU, measured at its current clocks; the
// reciprocal square root (rsqrtf) the Matern kernel takes per pair; and the
// rates that decide the reduced-precision design: packed half-precision
// exponentials (ex2.approx.f16x2, ex2.approx.ftz.bf16x2: two values per
// instruction) and the warp-level tensor-core MMA (mma.sync m16n8k16, f16 in,
// f32 accumulate) the multi-column product issues.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "api_util.h"
#include "common.cuh"
#include "internal.h"

namespace krr {
namespace {

constexpr int CHAINS = 8;
constexpr int ITERS = 4096;

__global__ void __launch_bounds__(256) ex2_rate_kernel(float* out, float seed) {
  float x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = seed + 0.01f * c + 1e-6f * threadIdx.x;
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = ex2(-x[c]);  // converges to x = 2^-x
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma_rate_kernel(float* out, float seed) {
  float x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = seed + 0.01f * c;
  const float a = 0.999f, b = 1e-3f * seed;
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = fmaf(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) ffma2_rate_kernel(float* out, float seed) {
  float2 x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = make_float2(seed + 0.01f * c, seed - 0.01f * c);
  const float2 a = make_float2(0.999f, 0.998f), b = make_float2(1e-3f * seed, 2e-3f * seed);
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = ffma2(x[c], a, b);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c].x + x[c].y;
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(256) rsqrt_rate_kernel(float* out, float seed) {
  float x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) x[c] = seed + 0.01f * c + 1e-6f * threadIdx.x;
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) x[c] = rsqrtf(x[c]);  // oscillates towards x = 1
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// Two exponentials per instruction: a chain of ex2.approx.f16x2 on packed
// halves (2^-x converges to a fixed point, so the values stay finite).
__global__ void __launch_bounds__(256) ex2_f16x2_rate_kernel(float* out, float seed) {
  uint32_t x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    __half2 h = __floats2half2_rn(-(seed + 0.01f * c), -(seed + 0.02f * c));
    x[c] = *reinterpret_cast<uint32_t*>(&h);
  }
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      uint32_t y;
      asm volatile("ex2.approx.f16x2 %0, %1;" : "=r"(y) : "r"(x[c] ^ 0x80008000u));
      x[c] = y;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s ^= x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

__global__ void __launch_bounds__(256) ex2_bf16x2_rate_kernel(float* out, float seed) {
  uint32_t x[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) {
    __nv_bfloat162 h = __floats2bfloat162_rn(seed + 0.01f * c, seed + 0.02f * c);
    x[c] = *reinterpret_cast<uint32_t*>(&h);
  }
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) {
      uint32_t y;
      asm volatile("ex2.approx.ftz.bf16x2 %0, %1;" : "=r"(y) : "r"(x[c] ^ 0x80008000u));
      x[c] = y;
    }
  }
  uint32_t s = 0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s ^= x[c];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (float)s;
}

// Four independent accumulator chains per warp, each m16n8k16 (f16 in, f32
// out).  Every chain starts from its own accumulator and multiplies its own
// B operand, so no two MMAs are the same computation (identical chains could
// be merged by the compiler and would overstate the rate).
constexpr int MMA_CHAINS = 4;
__global__ void __launch_bounds__(256) mma_sync_rate_kernel(float* out, float seed) {
  float d[MMA_CHAINS][4];
  uint32_t b[MMA_CHAINS];
#pragma unroll
  for (int a = 0; a < MMA_CHAINS; ++a) {
#pragma unroll
    for (int e = 0; e < 4; ++e) d[a][e] = seed * (float)(a + 1) + 1e-3f * (float)(e + threadIdx.x);
    __half2 hb = __floats2half2_rn(0.25f * (a + 1), -0.125f * (a + 1));
    b[a] = *reinterpret_cast<uint32_t*>(&hb);
  }
  __half2 h = __floats2half2_rn(seed, 0.5f * seed);
  const uint32_t v = *reinterpret_cast<uint32_t*>(&h);
  for (int it = 0; it < ITERS; ++it) {
#pragma unroll
    for (int a = 0; a < MMA_CHAINS; ++a)
      asm volatile(
          "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
          "{%8,%9}, {%0,%1,%2,%3};"
          : "+f"(d[a][0]), "+f"(d[a][1]), "+f"(d[a][2]), "+f"(d[a][3])
          : "r"(v), "r"(v), "r"(v), "r"(v), "r"(b[a]), "r"(b[a]));
  }
  float s = 0.f;
#pragma unroll
  for (int a = 0; a < MMA_CHAINS; ++a)
#pragma unroll
    for (int e = 0; e < 4; ++e) s += d[a][e];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace krr

using namespace krr;

extern "C" krr_status krr_measure_alu_peaks(krr_handle h, double* ex2_per_s, double* ffma_per_s,
                                            double* ffma2_lanes_per_s, void* stream) {
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = c.num_sms * 8, threads = 256;
  void* out;
  cudaError_t e = c.ws.get("peaks.out", sizeof(float) * blocks * threads, &out);
  if (e) return cuda_error(c, e, "krr_measure_alu_peaks");
  const double ops = (double)blocks * threads * CHAINS * ITERS;
  double res[3];
  for (int k = 0; k < 3; ++k) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(c.ev0, st);
      if (k == 0) ex2_rate_kernel<<<blocks, threads, 0, st>>>((float*)out, 0.5f); count_launch();
      if (k == 1) ffma_rate_kernel<<<blocks, threads, 0, st>>>((float*)out, 0.5f); count_launch();
      if (k == 2) ffma2_rate_kernel<<<blocks, threads, 0, st>>>((float*)out, 0.5f); count_launch();
      cudaEventRecord(c.ev1, st);
      if ((e = cudaEventSynchronize(c.ev1))) return cuda_error(c, e, "krr_measure_alu_peaks");
      float ms;
      cudaEventElapsedTime(&ms, c.ev0, c.ev1);
      if (rep > 0 && ms < best) best = ms;
    }
    res[k] = ops / (best * 1e-3);
  }
  if (ex2_per_s) *ex2_per_s = res[0];
  if (ffma_per_s) *ffma_per_s = res[1];
  if (ffma2_lanes_per_s) *ffma2_lanes_per_s = 2.0 * res[2];
  return KRR_OK;
}

extern "C" krr_status krr_measure_rsqrt_rate(krr_handle h, double* rsqrt_per_s, void* stream) {
  if (!h || !rsqrt_per_s) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = c.num_sms * 8, threads = 256;
  void* out;
  cudaError_t e = c.ws.get("peaks.out", sizeof(float) * blocks * threads, &out);
  if (e) return cuda_error(c, e, "krr_measure_rsqrt_rate");
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(c.ev0, st);
    rsqrt_rate_kernel<<<blocks, threads, 0, st>>>((float*)out, 0.5f); count_launch();
    cudaEventRecord(c.ev1, st);
    if ((e = cudaEventSynchronize(c.ev1))) return cuda_error(c, e, "krr_measure_rsqrt_rate");
    float ms;
    cudaEventElapsedTime(&ms, c.ev0, c.ev1);
    if (rep > 0 && ms < best) best = ms;
  }
  *rsqrt_per_s = (double)blocks * threads * CHAINS * ITERS / (best * 1e-3);
  return KRR_OK;
}

extern "C" krr_status krr_measure_half_rates(krr_handle h, double* ex2_f16x2_values_per_s,
                                             double* ex2_bf16x2_values_per_s,
                                             double* mma_sync_f16_flops_per_s, void* stream) {
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  cudaStream_t st = (cudaStream_t)stream;
  const int blocks = c.num_sms * 8, threads = 256;
  void* out;
  cudaError_t e = c.ws.get("peaks.out", sizeof(float) * blocks * threads, &out);
  if (e) return cuda_error(c, e, "krr_measure_half_rates");
  double res[3];
  for (int k = 0; k < 3; ++k) {
    float best = 1e30f;
    for (int rep = 0; rep < 4; ++rep) {
      cudaEventRecord(c.ev0, st);
      if (k == 0) ex2_f16x2_rate_kernel<<<blocks, threads, 0, st>>>((float*)out, 0.5f);
      if (k == 1) ex2_bf16x2_rate_kernel<<<blocks, threads, 0, st>>>((float*)out, 0.5f);
      if (k == 2) mma_sync_rate_kernel<<<blocks, threads, 0, st>>>((float*)out, 0.5f);
      count_launch();
      cudaEventRecord(c.ev1, st);
      if ((e = cudaEventSynchronize(c.ev1))) return cuda_error(c, e, "krr_measure_half_rates");
      float ms;
      cudaEventElapsedTime(&ms, c.ev0, c.ev1);
      if (rep > 0 && ms < best) best = ms;
    }
    const double threads_it = (double)blocks * threads * ITERS;
    // values: 2 per ex2 instruction and chain; MMA: one per warp and chain,
    // 2 * 16 * 8 * 16 flops
    const double work = k < 2 ? threads_it * CHAINS * 2.0 : threads_it / 32.0 * MMA_CHAINS * 4096.0;
    res[k] = work / (best * 1e-3);
  }
  if (ex2_f16x2_values_per_s) *ex2_f16x2_values_per_s = res[0];
  if (ex2_bf16x2_values_per_s) *ex2_bf16x2_values_per_s = res[1];
  if (mma_sync_f16_flops_per_s) *mma_sync_f16_flops_per_s = res[2];
  return KRR_OK;
}
