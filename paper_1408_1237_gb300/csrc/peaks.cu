// Issue-rate microbenchmarks for the ALU roofline of the kernel product:
// MUFU.EX2 (ex2.approx.ftz.f32), scalar FFMA and packed FFMA2 (f32x2)
// results per second on this GPU, measured at its current clocks; and the
// reciprocal square root (rsqrtf) the Matern kernel takes per pair.
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
