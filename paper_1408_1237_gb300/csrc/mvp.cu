// On-the-fly Gaussian kernel product (hot-path steps A2/A4/A6):
//
//   y_i = sum_j q_j exp(-|x_i - x_j|^2 / (2 sigma^2)) + shift q_i
//
// (Eqs. 1-3; the weighted kernel sum of Sec. 3.1, computed on the fly in O(N)
// memory).  Points arrive prepared by prep.cu: Morton-sorted, unscaled; with
// s = sqrt(log2(e) / (2 sigma^2)) a kernel value is 2^(-s^2 |x_i - x_j|^2).
//
// Kernel design:
//  * Targets are processed in warp blocks of WB = 32*T consecutive sorted
//    points (T per thread, held in registers); a CTA has 8 warps, each on its
//    own warp block, and a grid row y covers one contiguous range of source
//    tiles (source splitting balances the grid over the 152 SMs).
//  * Expanded form, for warp blocks within squared radius EXPANDED_R2 of
//    their centre c in scaled units x^ = s (x - c):
//      -|x^_i - x^_j|^2 = -|x^_i|^2 + (b_j + sum_k x^_ik (2 x^_jk)),
//    b_j = -|x^_j|^2, and 2^(-|x^_i|^2) is factored out of the sum, so a pair
//    costs d FMAs for the exponent, one MUFU.EX2 and one FMA.  The factored
//    exponent never exceeds |x^_i|^2 <= EXPANDED_R2, so nothing overflows; its
//    rounding error is a few ulps of EXPANDED_R2.  x - c is formed from the raw
//    float32 coordinates, so recentring loses no digits.
//  * Direct form (warp blocks that are not compact): d subtractions of the raw
//    coordinates (exact for near pairs), d multiply-adds, one multiply by
//    -s^2, one MUFU.EX2, one FMA.
//  * prep.cu orders the warp blocks expanded-first, so every CTA but one runs a
//    single form and its warps stay in step.
//  * Source tiles (TS points: d coordinates + weights, contiguous in the
//    tile-blocked layout) arrive by 1-D TMA bulk copies in a RS-stage
//    shared-memory ring (mbarrier completion, bounded waits); each warp then
//    transforms the tile for its own centre into a private shared buffer.
//  * Two sources share each packed f32x2 FMA (FFMA2/FADD2/FMUL2).
//  * Per-tile float32 partial sums are folded with Kahan compensation; each
//    source split writes one FP64 partial per target, and a finalize kernel
//    adds the splits in fixed order (deterministic), applies 2^(-|x^_i|^2), the
//    shift term and the fused epilogue (axpy, dot, scatter).
//  * Other kernel functions (the Matern kernel of Sec. 6.1) take the direct
//    form in the multi-column CUDA-core kernel, templated on the pair
//    function (KF): a = s |x_i - x_j| with s = sqrt(3) / h by one reciprocal
//    square root and one multiply, then (1 + a) 2^(-a log2(e)) by one
//    MUFU.EX2 and one FMA.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace krr {

namespace {

constexpr int NT = 256;   // threads per CTA: 8 warps
constexpr int NW = NT / 32;

template <int D>
constexpr int raw_stages() { return D >= 8 ? 3 : 4; }

struct MvpParams {
  const float* xt;      // targets, tile-blocked SoA (raw coordinates)
  int64_t Nt, Nt_pad;
  const float* tctr;    // target warp-block centres [nblk][D]
  const int* torder;    // warp blocks, expanded-form first
  const int* tn_exp;    // number of expanded-form warp blocks
  int64_t nblk;
  const float* xs;      // sources, tile-blocked SoA (raw coordinates)
  const float* q;       // source weights, sorted order, zero padded
  int ntiles;           // source tiles
  int tiles_per_split;
  double* part;         // [splits][Nt_pad]
  float* fac;           // [Nt_pad] factored scale 2^(-|x^_i|^2) (1 for the direct form)
  int* err;
  float s;              // sqrt(log2(e) / (2 sigma^2))
  const int* active;    // predication flag (null: always run)
  int64_t part_stride;  // distance between splits in part (Nt_pad for one column)
  int64_t slot0;        // first block slot of the grid (blocks before it are not processed)
  // sorted target rows computed (shard emulation): blocks outside are skipped
  int64_t row_lo = 0, row_hi = INT64_MAX;
};

// Warp-cooperative transform of one raw source tile for this warp's centre:
// expanded form -> (2 x^_j, b_j = -|x^_j|^2, q_j); direct form -> (-x_j, q_j).
template <int D>
__device__ __forceinline__ void transform_tile(const float* __restrict__ rs, float* __restrict__ wb,
                                               const float (&ctr)[D], float s, bool expanded) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int v = 0; v < TS / 32; ++v) {
    const int j = lane + 32 * v;
    if (expanded) {
      float xh[D];
#pragma unroll
      for (int k = 0; k < D; ++k) xh[k] = s * (rs[k * TS + j] - ctr[k]);
      float b = -(xh[0] * xh[0]);
#pragma unroll
      for (int k = 1; k < D; ++k) b = fmaf(-xh[k], xh[k], b);
#pragma unroll
      for (int k = 0; k < D; ++k) wb[k * TS + j] = 2.f * xh[k];
      wb[D * TS + j] = b;
    } else {
#pragma unroll
      for (int k = 0; k < D; ++k) wb[k * TS + j] = -rs[k * TS + j];
    }
    wb[(D + 1) * TS + j] = rs[D * TS + j];
  }
}

template <int D, int T>
__device__ __forceinline__ void compute_expanded(const float* __restrict__ cb,
                                                 const float2 (&tx)[T][D], float2 (&acc)[T]) {
  const float* cX = cb;
  const float* cB = cb + D * TS;
  const float* cQ = cb + (D + 1) * TS;
#pragma unroll 2
  for (int j = 0; j < TS; j += 4) {
    float4 xk[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xk[k] = *reinterpret_cast<const float4*>(cX + k * TS + j);
    const float4 bb = *reinterpret_cast<const float4*>(cB + j);
    const float4 qq = *reinterpret_cast<const float4*>(cQ + j);
#pragma unroll
    for (int u = 0; u < T; ++u) {
      float2 e0 = make_float2(bb.x, bb.y), e1 = make_float2(bb.z, bb.w);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        e0 = ffma2(tx[u][k], make_float2(xk[k].x, xk[k].y), e0);
        e1 = ffma2(tx[u][k], make_float2(xk[k].z, xk[k].w), e1);
      }
      e0.x = ex2(e0.x);
      e0.y = ex2(e0.y);
      e1.x = ex2(e1.x);
      e1.y = ex2(e1.y);
      acc[u] = ffma2(make_float2(qq.x, qq.y), e0, acc[u]);
      acc[u] = ffma2(make_float2(qq.z, qq.w), e1, acc[u]);
    }
  }
}

constexpr float kLog2e = 1.4426950408889634f;  // log2(e) = 1 / ln 2

// Matern 3/2 value from the squared raw distance: a = s r, (1 + a) 2^(-a log2 e).
// r = r2 / sqrt(r2) through the reciprocal square root (a 2-ulp routine); the
// clamp keeps r2 = 0 (a point against itself) at a = 0 instead of 0 * inf.
__device__ __forceinline__ float matern32_value(float r2, float s) {
  const float a = s * (r2 * rsqrtf(fmaxf(r2, 1e-30f)));
  const float e = ex2(a * -kLog2e);
  return fmaf(a, e, e);
}

// KF: pair function, 0 = Gaussian 2^(-s^2 r^2), 1 = Matern 3/2 (s = sqrt(3)/h).
template <int D, int T, int KF>
__device__ __forceinline__ void compute_direct(const float* __restrict__ cb,
                                               const float2 (&tx)[T][D], float2 (&acc)[T],
                                               float s2, float s) {
  const float* cX = cb;  // holds -x_j (raw)
  const float* cQ = cb + (D + 1) * TS;
  const float2 ns2 = make_float2(-s2, -s2);
  const float2 sv = make_float2(s, s), nl2e = make_float2(-kLog2e, -kLog2e);
#pragma unroll 2
  for (int j = 0; j < TS; j += 4) {
    float4 xk[D];
#pragma unroll
    for (int k = 0; k < D; ++k) xk[k] = *reinterpret_cast<const float4*>(cX + k * TS + j);
    const float4 qq = *reinterpret_cast<const float4*>(cQ + j);
#pragma unroll
    for (int u = 0; u < T; ++u) {
      float2 d0 = fadd2(tx[u][0], make_float2(xk[0].x, xk[0].y));
      float2 d1 = fadd2(tx[u][0], make_float2(xk[0].z, xk[0].w));
      float2 r0 = fmul2(d0, d0), r1 = fmul2(d1, d1);
#pragma unroll
      for (int k = 1; k < D; ++k) {
        d0 = fadd2(tx[u][k], make_float2(xk[k].x, xk[k].y));
        d1 = fadd2(tx[u][k], make_float2(xk[k].z, xk[k].w));
        r0 = ffma2(d0, d0, r0);
        r1 = ffma2(d1, d1, r1);
      }
      float2 e0, e1;
      if constexpr (KF == 0) {
        r0 = fmul2(r0, ns2);
        r1 = fmul2(r1, ns2);
        e0.x = ex2(r0.x);
        e0.y = ex2(r0.y);
        e1.x = ex2(r1.x);
        e1.y = ex2(r1.y);
      } else {
        // a = s r (r = r^2 rsqrt(r^2), clamped at r^2 = 0), then (1 + a) 2^(-a log2 e)
        const float2 a0 = fmul2(sv, fmul2(r0, make_float2(rsqrtf(fmaxf(r0.x, 1e-30f)),
                                                          rsqrtf(fmaxf(r0.y, 1e-30f)))));
        const float2 a1 = fmul2(sv, fmul2(r1, make_float2(rsqrtf(fmaxf(r1.x, 1e-30f)),
                                                          rsqrtf(fmaxf(r1.y, 1e-30f)))));
        const float2 t0 = fmul2(a0, nl2e), t1 = fmul2(a1, nl2e);
        e0 = make_float2(ex2(t0.x), ex2(t0.y));
        e1 = make_float2(ex2(t1.x), ex2(t1.y));
        e0 = ffma2(a0, e0, e0);
        e1 = ffma2(a1, e1, e1);
      }
      acc[u] = ffma2(make_float2(qq.x, qq.y), e0, acc[u]);
      acc[u] = ffma2(make_float2(qq.z, qq.w), e1, acc[u]);
    }
  }
}

template <int D, int T, int KF>
__global__ void __launch_bounds__(NT, 2) mvp_f32_kernel(const MvpParams p) {
  constexpr int RS = raw_stages<D>();
  constexpr uint32_t kRawFloats = (D + 1) * TS;
  constexpr uint32_t kWbFloats = (D + 2) * TS;
  extern __shared__ __align__(128) float smem[];
  float* raw = smem;                                   // RS * (D+1) * TS
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  float* wbuf = smem + RS * kRawFloats + warp * kWbFloats;  // this warp's (D+2) * TS
  __shared__ __align__(8) uint64_t bars[RS];
  __shared__ volatile int abort_flag;
  if (p.active && *p.active == 0) return;

  // ---- this warp's target block
  const int64_t slot = p.slot0 + (int64_t)blockIdx.x * NW + warp;
  const int64_t nexp = *p.tn_exp;
  const bool live = slot < p.nblk;
  int64_t blk = live ? p.torder[slot] : 0;
  // a warp whose block lies outside the shard computes nothing; a CTA with
  // no such warp leaves at once
  const bool work = live && blk * 32 * T >= p.row_lo && blk * 32 * T < p.row_hi;
  if (!__syncthreads_or(work)) return;
  const int64_t last = min(p.slot0 + ((int64_t)blockIdx.x + 1) * NW, p.nblk);  // CTA's block slots end
  const bool expanded = last <= nexp;  // uniform over the CTA
  float ctr[D];
#pragma unroll
  for (int k = 0; k < D; ++k) ctr[k] = p.tctr[blk * D + k];

  float2 tx[T][D];
  float r2[T];
#pragma unroll
  for (int u = 0; u < T; ++u) {
    const int64_t i = blk * 32 * T + lane + 32 * u;
    const bool inmem = live && i < p.Nt_pad;
    const int64_t base = (i / TS) * (int64_t)D * TS + (i % TS);
    float a = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float x = inmem ? p.xt[base + (int64_t)k * TS] : ctr[k];
      const float xh = p.s * (x - ctr[k]);
      a = fmaf(xh, xh, a);
      const float v = expanded ? xh : x;
      tx[u][k] = make_float2(v, v);
    }
    r2[u] = a;
  }
  if (blockIdx.y == 0 && work) {
#pragma unroll
    for (int u = 0; u < T; ++u) {
      const int64_t i = blk * 32 * T + lane + 32 * u;
      if (i < p.Nt_pad) p.fac[i] = expanded ? exp2f(-r2[u]) : 1.f;
    }
  }
  const float s2 = p.s * p.s;

  // ---- source range of this split
  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;

  float sum[T], comp[T];
  float2 acc[T];
#pragma unroll
  for (int u = 0; u < T; ++u) {
    sum[u] = comp[u] = 0.f;
    acc[u] = make_float2(0.f, 0.f);
  }

  auto issue = [&](int r) {
    const int stage = r % RS;
    const int64_t tile = t_begin + r;
    float* dst = raw + stage * kRawFloats;
    mbar_arrive_expect_tx(&bars[stage], kRawFloats * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    bulk_g2s(dst + D * TS, p.q + tile * (int64_t)TS, TS * 4, &bars[stage]);
  };

  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < RS; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0)
    for (; issued < min(RS, nt); ++issued) issue(issued);

  for (int r = 0; r < nt; ++r) {
    // stage (r-1) % RS was released by the barrier that ended iteration r-1
    if (tid == 0 && r >= 1 && r - 1 + RS < nt) {
      fence_proxy_async_smem();
      issue(r - 1 + RS);
      ++issued;
    }
    // warp-uniform outcome: a lane that gave up takes its whole warp with it
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[r % RS], (r / RS) & 1));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    } else if (work) {
      transform_tile<D>(raw + (r % RS) * kRawFloats, wbuf, ctr, p.s, expanded);
      __syncwarp();
      if (expanded)
        compute_expanded<D, T>(wbuf, tx, acc);
      else
        compute_direct<D, T, KF>(wbuf, tx, acc, s2, p.s);
#pragma unroll
      for (int u = 0; u < T; ++u) {
        kahan_add(sum[u], comp[u], acc[u].x + acc[u].y);
        acc[u] = make_float2(0.f, 0.f);
      }
    }
    __syncthreads();
    if (abort_flag) break;
  }
  if (abort_flag) {
    // drain copies still in flight before the CTA's shared memory is released
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % RS], (r / RS) & 1);
    __syncthreads();
    return;
  }

  if (work) {
    double* part = p.part + (int64_t)blockIdx.y * p.part_stride;
#pragma unroll
    for (int u = 0; u < T; ++u) {
      const int64_t i = blk * 32 * T + lane + 32 * u;
      if (i < p.Nt_pad) part[i] = (double)sum[u] - (double)comp[u];
    }
  }
}

// Direct-form warp blocks for several columns at once: one exponential per
// pair, shared by the m <= MC weight columns (a pair costs d subtractions, d
// multiply-adds, a multiply by -s^2, one MUFU.EX2 and m FMAs).  One target
// per thread; the eight warps of a CTA cover 256 consecutive targets, that is
// 8 / T target blocks of 32 T points (T = 8: one super-block).  Coordinates and the m weight columns of
// a source tile arrive by 1-D TMA bulk copies (RS-stage ring); weight rows
// m..MC-1 of every stage are zero.  Per-tile float32 sums fold with Kahan
// compensation into one FP64 partial per (split, column, target).
template <int D, int MC>
constexpr int dirm_stages() {
  return sizeof(float) * 3 * (D + MC) * TS <= 160 * 1024 ? 3 : 2;
}

template <int D, int MC>
constexpr size_t dirm_smem_bytes() {
  return sizeof(float) * dirm_stages<D, MC>() * (D + MC) * TS;
}

// (high-dimensional instances hold D coordinates per thread: one CTA per SM)
// KF: pair function, 0 = Gaussian 2^(-s^2 r^2), 1 = Matern 3/2.
template <int D, int MC, int KF>
__global__ void __launch_bounds__(NT, (D > 8 ? 1 : 2)) mvp_dirm_kernel(const MvpParams p, const float* __restrict__ Q,
                                                                      int64_t q_stride, int m, int T, int64_t slot0) {
  constexpr int RS = dirm_stages<D, MC>();
  constexpr uint32_t kStage = (D + MC) * TS;
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t bars[RS];
  __shared__ volatile int abort_flag;
  if (p.active && *p.active == 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bpc = NW / T;  // warp blocks per CTA
  const int64_t nexp = *p.tn_exp;
  const int64_t cta_end = min(slot0 + ((int64_t)blockIdx.x + 1) * bpc, p.nblk);
  if (cta_end <= nexp) return;  // every block of this CTA is expanded-form
  const int64_t slot = slot0 + (int64_t)blockIdx.x * bpc + warp / T;
  const bool in_range = slot < p.nblk && slot >= nexp;
  const int64_t blk = in_range ? p.torder[slot] : 0;
  const bool live = in_range && blk * 32 * T >= p.row_lo && blk * 32 * T < p.row_hi;  // shard
  if (!__syncthreads_or(live)) return;  // no block of this CTA to compute
  const int64_t i = blk * 32 * T + 32 * (warp % T) + lane;
  const bool valid = live && i < p.Nt_pad;
  float xi[D];
  {
    const int64_t base = (i / TS) * (int64_t)D * TS + (i % TS);
#pragma unroll
    for (int k = 0; k < D; ++k) xi[k] = valid ? p.xt[base + (int64_t)k * TS] : 0.f;
  }
  if (blockIdx.y == 0 && valid) p.fac[i] = 1.f;
  const float ns2 = -(p.s * p.s);
  const float s = p.s;

  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;

  float sum[MC], comp[MC];
#pragma unroll
  for (int c = 0; c < MC; ++c) sum[c] = comp[c] = 0.f;

  auto issue = [&](int r) {
    const int stage = r % RS;
    const int64_t tile = t_begin + r;
    float* dst = smem + stage * kStage;
    mbar_arrive_expect_tx(&bars[stage], (uint32_t)(D + m) * TS * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    for (int c = 0; c < m; ++c)
      bulk_g2s(dst + (D + c) * TS, Q + c * q_stride + tile * (int64_t)TS, TS * 4, &bars[stage]);
  };

  // weight rows of absent columns stay zero in every stage
  for (int idx = tid; idx < RS * (MC - m) * TS; idx += NT) {
    const int stage = idx / ((MC - m) * TS), rem = idx % ((MC - m) * TS);
    smem[stage * kStage + (D + m) * TS + rem] = 0.f;
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < RS; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0)
    for (; issued < min(RS, nt); ++issued) issue(issued);

  for (int r = 0; r < nt; ++r) {
    if (tid == 0 && r >= 1 && r - 1 + RS < nt) {
      fence_proxy_async_smem();
      issue(r - 1 + RS);
      ++issued;
    }
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[r % RS], (r / RS) & 1));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    } else if (live) {
      const float* cx = smem + (r % RS) * kStage;
      const float* cq = cx + D * TS;
      float acc[MC];
#pragma unroll
      for (int c = 0; c < MC; ++c) acc[c] = 0.f;
#pragma unroll 1
      for (int j = 0; j < TS; j += 4) {
        float e[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) e[v] = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float4 xk = *reinterpret_cast<const float4*>(cx + k * TS + j);
          const float d0 = xi[k] - xk.x, d1 = xi[k] - xk.y, d2 = xi[k] - xk.z, d3 = xi[k] - xk.w;
          e[0] = fmaf(d0, d0, e[0]);
          e[1] = fmaf(d1, d1, e[1]);
          e[2] = fmaf(d2, d2, e[2]);
          e[3] = fmaf(d3, d3, e[3]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          if constexpr (KF == 0)
            e[v] = ex2(e[v] * ns2);
          else
            e[v] = matern32_value(e[v], s);
        }
#pragma unroll
        for (int c = 0; c < MC; ++c) {
          const float4 qq = *reinterpret_cast<const float4*>(cq + c * TS + j);
          acc[c] = fmaf(qq.x, e[0], acc[c]);
          acc[c] = fmaf(qq.y, e[1], acc[c]);
          acc[c] = fmaf(qq.z, e[2], acc[c]);
          acc[c] = fmaf(qq.w, e[3], acc[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < MC; ++c) kahan_add(sum[c], comp[c], acc[c]);
    }
    __syncthreads();
    if (abort_flag) break;
  }
  if (abort_flag) {
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % RS], (r / RS) & 1);
    __syncthreads();
    return;
  }
  if (valid) {
    double* part = p.part + (int64_t)blockIdx.y * p.part_stride + i;
#pragma unroll
    for (int c = 0; c < MC; ++c)
      if (c < m) part[(int64_t)c * p.Nt_pad] = (double)sum[c] - (double)comp[c];
  }
}

struct FinParams {
  const double* part;
  int splits;
  // multi-column products: targets of direct-form super-blocks (sb_flag 0)
  // take their sums from part2 (splits2 splits) instead
  const double* part2;
  int splits2;
  const int* sb_flag;
  int64_t part_stride;
  int64_t N, Npad;
  const float* fac;
  const float* qdiag;
  float shift;
  MvpOut o;
  double* dot_part;        // [columns][gridDim.x] per-block dot partials
  unsigned int* dot_count; // [columns] arrival counters (reset by the last block)
  int64_t row_lo = 0, row_hi = INT64_MAX;  // sorted rows written (shard emulation)
};

__global__ void __launch_bounds__(256) mvp_finalize_kernel(const FinParams f) {
  __shared__ double red[8];
  __shared__ bool is_last;
  if (f.o.active && *f.o.active == 0) return;
  // column blockIdx.y: its vectors are Npad (original order: N) apart, its
  // scalars state_stride bytes apart
  const int col = blockIdx.y;
  const size_t so = (size_t)col * f.o.state_stride;
  auto at = [so](auto* ptr) { return (decltype(ptr))((const char*)ptr + so); };
  if (f.o.col_active && *at(f.o.col_active) == 0) return;
  const int64_t cv = (int64_t)col * f.Npad;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double out = 0.0, dotv = 0.0;
  const bool mine = i >= f.row_lo && i < f.row_hi;
  if (i < f.N && mine) {
    const bool second = f.sb_flag && f.sb_flag[i / SB] == 0;
    const double* part = (second ? f.part2 : f.part) + cv;
    const int splits = second ? f.splits2 : f.splits;
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += part[(int64_t)sp * f.part_stride + i];
    double y = (double)f.fac[i] * s;
    if (f.qdiag) y += (double)f.shift * (double)f.qdiag[cv + i];
    out = (double)f.o.alpha * y;
    if (f.o.u) out += (double)f.o.beta * (double)f.o.u[cv + i];
    if (f.o.out_orig) f.o.out_orig[(int64_t)col * f.N + f.o.perm[i]] = (float)out;
    if (f.o.dotw) dotv = out * (double)f.o.dotw[cv + i];
  }
  if (i < f.Npad && mine) {
    if (f.o.out_f) f.o.out_f[cv + i] = (float)out;
    if (f.o.out_d) f.o.out_d[cv + i] = out;
  }
  if (f.o.dot) {
    double* dot_part = f.dot_part + (int64_t)col * gridDim.x;
    unsigned* dot_count = f.dot_count + col;
    const double bs = block_sum(dotv, red);
    if (threadIdx.x == 0) {
      dot_part[blockIdx.x] = bs;
      __threadfence();
      is_last = atomicAdd(dot_count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      double t = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += dot_part[b];
      t = block_sum(t, red);
      if (threadIdx.x == 0) {
        *at(f.o.dot) = t;
        if (f.o.ratio_out) {
          const bool good = t > 0.0 && isfinite(t);
          *at(f.o.ratio_out) = good ? *at(f.o.ratio_num) / t : 0.0;
          if (!good) *at(f.o.brk_flag) = 1;
        }
        *dot_count = 0u;
      }
    }
  }
}

template <int D>
constexpr size_t smem_bytes() {
  return sizeof(float) * (raw_stages<D>() * (D + 1) * TS + NW * (D + 2) * TS);
}

// Dynamic shared-memory opt-in, once per kernel instance and device.
template <int D, int T, int KF>
cudaError_t set_attr() {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mvp_f32_kernel<D, T, KF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem_bytes<D>());
  if (!e && dev < 128) done[dev] = true;
  return e;
}

template <int D, int T, int KF>
cudaError_t launch_typed(const MvpParams& p, int splits, cudaStream_t st) {
  cudaError_t e = set_attr<D, T, KF>();
  if (e) return e;
  dim3 grid((unsigned)std::max<int64_t>(1, (p.nblk - p.slot0 + NW - 1) / NW), (unsigned)splits);
  mvp_f32_kernel<D, T, KF><<<grid, NT, smem_bytes<D>(), st>>>(p); count_launch();
  return cudaGetLastError();
}

// Split count minimising the makespan ceil(blocks*S/slots) * (ceil(tiles/S) +
// setup), setup = a CTA's fixed cost in units of one source tile.
int choose_splits(int64_t blocks, int tiles, int slots, double setup = 0.0) {
  int best = 1;
  double best_cost = 1e300;
  for (int s = 1; s <= std::min(tiles, 64); ++s) {
    const double waves = std::ceil((double)blocks * s / slots);
    const double cost = waves * (std::ceil((double)tiles / s) + setup);
    if (cost < best_cost - 1e-9) {
      best_cost = cost;
      best = s;
    }
  }
  return best;
}

template <int D>
constexpr int large_T() {
  // targets per thread of the large variant (register budget of 128)
  return (D <= 3) ? 8 : (D <= 5 ? 4 : 2);
}

int large_T_of(int d) {
  switch (d) {
    case 1: return large_T<1>();
    case 2: return large_T<2>();
    case 3: return large_T<3>();
    case 4: return large_T<4>();
    case 5: return large_T<5>();
    case 6: return large_T<6>();
    case 7: return large_T<7>();
    default: return large_T<8>();
  }
}

struct Plan {
  int splits = 1;
  int tiles_per_split = 1;
};

// scale: the autotuner's factor on the modelled split count (1: the model);
// setup: a CTA's fixed cost in source tiles.
Plan make_plan(int64_t nblk, int ntiles, int num_sms, int plan_slots, double scale, double setup = 0.0) {
  const int slots = plan_slots > 0 ? plan_slots : num_sms * 2;
  const int64_t ctas = (nblk + NW - 1) / NW;
  Plan pl;
  int splits = choose_splits(ctas, ntiles, slots, setup);
  if (scale != 1.0)
    splits = std::max(1, std::min({(int)std::lround(splits * scale), ntiles, 256}));
  pl.tiles_per_split = (ntiles + splits - 1) / splits;
  pl.splits = (ntiles + pl.tiles_per_split - 1) / pl.tiles_per_split;
  return pl;
}

template <int D, int KF = 0>
cudaError_t attrs_T(int T) {
  constexpr int TL = large_T<D>();
  if (T == TL) return set_attr<D, TL, KF>();
  if (T == 1) return set_attr<D, 1, KF>();
  return cudaErrorNotSupported;
}

template <int D, int KF = 0>
cudaError_t dispatch_T(MvpParams p, int T, const Plan& pl, cudaStream_t st) {
  constexpr int TL = large_T<D>();
  p.tiles_per_split = pl.tiles_per_split;
  if (T == TL) return launch_typed<D, TL, KF>(p, pl.splits, st);
  if (T == 1) return launch_typed<D, 1, KF>(p, pl.splits, st);
  return cudaErrorNotSupported;
}

// The packed CUDA-core kernel for d <= 8 and kernel family kf (KRR_KERNEL_*):
// launch (launch = true) or only its shared-memory attribute.
template <int KF>
cudaError_t f32_any_k(const MvpParams& p, int d, int T, const Plan& pl, cudaStream_t st, bool launch) {
  switch (d) {
#define KRR_F32_CASE(DV) \
    case DV: return launch ? dispatch_T<DV, KF>(p, T, pl, st) : attrs_T<DV, KF>(T);
    KRR_F32_CASE(1) KRR_F32_CASE(2) KRR_F32_CASE(3) KRR_F32_CASE(4)
    KRR_F32_CASE(5) KRR_F32_CASE(6) KRR_F32_CASE(7) KRR_F32_CASE(8)
#undef KRR_F32_CASE
    default: return cudaErrorNotSupported;
  }
}
cudaError_t f32_any(const MvpParams& p, int d, int kf, int T, const Plan& pl, cudaStream_t st, bool launch) {
  if (kf == KRR_KERNEL_MATERN32) return f32_any_k<1>(p, d, T, pl, st, launch);
  if (kf != KRR_KERNEL_GAUSSIAN) return cudaErrorNotSupported;
  return f32_any_k<0>(p, d, T, pl, st, launch);
}

template <int D, int MC, int KF>
cudaError_t set_dirm_attr() {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mvp_dirm_kernel<D, MC, KF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)dirm_smem_bytes<D, MC>());
  if (!e && dev < 128) done[dev] = true;
  return e;
}

// Multi-column direct-form launch (or, with launch = false, only its
// attribute), MC the smallest of 4, 8, 16 that holds m columns.
template <int D, int KF>
cudaError_t dirm_typed(const MvpParams& p, const float* Q, int64_t q_stride, int m, int T,
                       int64_t slot0, const Plan& pl, cudaStream_t st, bool launch) {
  const int bpc = NW / T;
  dim3 grid((unsigned)std::max<int64_t>(1, (p.nblk - slot0 + bpc - 1) / bpc), (unsigned)pl.splits);
  MvpParams pp = p;
  pp.tiles_per_split = pl.tiles_per_split;
  cudaError_t e;
#define KRR_DIRM(MCV)                                                                       \
  if ((e = set_dirm_attr<D, MCV, KF>())) return e;                                         \
  if (launch) {                                                                            \
    mvp_dirm_kernel<D, MCV, KF><<<grid, NT, dirm_smem_bytes<D, MCV>(), st>>>(pp, Q, q_stride, m, T, slot0); \
    count_launch();                                                                        \
  }                                                                                        \
  return cudaGetLastError();
  if (m <= 1) { KRR_DIRM(1) }
  if (m <= 4) { KRR_DIRM(4) }
  if (m <= 8) { KRR_DIRM(8) }
  KRR_DIRM(16)
#undef KRR_DIRM
}

template <int KF>
cudaError_t dirm_dispatch_k(const MvpParams& p, int d, const float* Q, int64_t q_stride, int m, int T,
                            int64_t slot0, const Plan& pl, cudaStream_t st, bool launch) {
  switch (d) {
    case 1: return dirm_typed<1, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 2: return dirm_typed<2, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 3: return dirm_typed<3, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 4: return dirm_typed<4, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 5: return dirm_typed<5, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 6: return dirm_typed<6, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 7: return dirm_typed<7, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 8: return dirm_typed<8, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 16: return dirm_typed<16, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 32: return dirm_typed<32, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 48: return dirm_typed<48, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    case 64: return dirm_typed<64, KF>(p, Q, q_stride, m, T, slot0, pl, st, launch);
    default: return cudaErrorNotSupported;
  }
}

// kf: the kernel family of the points (KRR_KERNEL_*)
cudaError_t dirm_dispatch(const MvpParams& p, int d, int kf, const float* Q, int64_t q_stride, int m,
                          int T, int64_t slot0, const Plan& pl, cudaStream_t st, bool launch) {
  if (T < 1 || T > NW || NW % T) return cudaErrorNotSupported;
  if (kf == KRR_KERNEL_MATERN32) return dirm_dispatch_k<1>(p, d, Q, q_stride, m, T, slot0, pl, st, launch);
  if (kf != KRR_KERNEL_GAUSSIAN) return cudaErrorNotSupported;
  return dirm_dispatch_k<0>(p, d, Q, q_stride, m, T, slot0, pl, st, launch);
}

// Source splits of the multi-column kernels (one CTA per super-block): the
// tensor-core kernel over the expanded-form super-blocks, the CUDA-core
// kernel over the direct-form ones, each planned for its own grid.
Plan multi_plan_tc(const Ctx& c, const PointsDev& Tp, const PointsDev& Sp, krr_precision prec, int m) {
  // two CTAs (of 128 targets) per super-block, at most two per SM (tensor memory)
  // one CTA per super-block (mma.sync kernel), or two of 128 targets with at
  // most two per SM (tcgen05 kernel: tensor memory)
  return make_plan((tc5_on(c, prec, m, Tp) ? 2 : 1) * Tp.h_sb_nexp * NW, (int)(Sp.Npad / TS), c.num_sms,
                   c.plan_slots, c.split_scale);
}
// Multi-column products keep the tensor cores to d <= 8 (Gaussian); elsewhere
// every super-block takes the direct form, whatever its compactness flag.
bool multi_direct_only(const PointsDev& Tp) { return Tp.d > 8 || Tp.kfam != KRR_KERNEL_GAUSSIAN; }
int64_t multi_nexp(const PointsDev& Tp) { return multi_direct_only(Tp) ? 0 : Tp.h_sb_nexp; }
// Direct-form super-blocks of a multi-column product up to 8 dimensions take
// the kernel with the weighted sum on the tensor cores (mvp_dirtc.cu: one CTA
// of 16 warps per super-block, one resident per SM) unless the handle asks
// for the CUDA-core kernel (KRR_OPT_DIRECT_TENSOR = 0).
bool use_dirtc(const Ctx& c, const PointsDev& Tp) {
  return c.direct_tensor && Tp.d <= 8 &&
         (Tp.kfam == KRR_KERNEL_GAUSSIAN || Tp.kfam == KRR_KERNEL_MATERN32);
}
Plan multi_plan_dir(const Ctx& c, const PointsDev& Tp, const PointsDev& Sp) {
  if (use_dirtc(c, Tp))
    return make_plan((Tp.nsb - multi_nexp(Tp)) * NW, (int)(Sp.Npad / TS), c.num_sms,
                     c.plan_slots > 0 ? c.plan_slots : c.num_sms, c.split_scale);
  return make_plan((Tp.nsb - multi_nexp(Tp)) * NW, (int)(Sp.Npad / TS), c.num_sms, c.plan_slots,
                   c.split_scale);
}

// The single-column float32 product takes the tensor-core exponent path when
// there are enough target super-blocks to fill the GPU (one CTA of 4 warps
// each, several per SM) and at least half of them are compact; otherwise the
// CUDA-core kernel with its finer per-warp blocks.
// Above 8 dimensions the direct form costs 2d + 2 FP32 operations per pair,
// so any compact super-block is worth the tensor-core kernel (mvp_tch_kernel).
bool use_tcx(const Ctx& c, const PointsDev& Tp) {
  if (Tp.d > 8) return c.allow_tcx && Tp.kfam == KRR_KERNEL_GAUSSIAN && Tp.h_sb_nexp > 0;
  return c.allow_tcx && Tp.nsb >= c.num_sms && 2 * Tp.h_sb_nexp >= Tp.nsb;
}

// Direct-form super-blocks of the single-column tensor-core path: through the
// packed CUDA-core kernel (8 super-blocks per CTA) when its warp blocks are
// the super-blocks, else the multi-column direct kernel with one column.
bool tcx_dir_f32(const PointsDev& Tp) { return Tp.T * 32 == SB; }
Plan tcx_dir_plan(const Ctx& c, const PointsDev& Tp, const PointsDev& Sp) {
  if (tcx_dir_f32(Tp))
    return make_plan(Tp.nsb - Tp.h_sb_nexp, (int)(Sp.Npad / TS), c.num_sms, c.plan_slots,
                     c.split_scale);
  return make_plan((Tp.nsb - Tp.h_sb_nexp) * NW, (int)(Sp.Npad / TS), c.num_sms, c.plan_slots,
                   c.split_scale);
}

Plan tcx_plan(const Ctx& c, const PointsDev& Tp, const PointsDev& Sp) {
  if (Tp.d > 8) {
    if (c.highd_tcgen05) {
      // tcgen05 kernel: two CTAs of 128 targets per super-block, one
      // resident per SM (two at d = 16: shared and tensor memory); a CTA
      // first builds its 128 target K-vectors (about half a source tile)
      const int occ = Tp.d <= 16 ? 2 : 1;
      return make_plan(2 * Tp.h_sb_nexp * NW, (int)(Sp.Npad / TS), c.num_sms,
                       c.plan_slots > 0 ? c.plan_slots : occ * c.num_sms, c.split_scale, 0.5);
    }
    // high-dimensional kernel: one CTA per SM (two at d = 16), and a CTA
    // first builds its 256 target K-vectors (about one source tile of work)
    const int occ = Tp.d <= 16 ? 2 : 1;
    return make_plan(Tp.h_sb_nexp * NW, (int)(Sp.Npad / TS), c.num_sms,
                     c.plan_slots > 0 ? c.plan_slots : occ * c.num_sms, c.split_scale, 1.0);
  }
  return make_plan(Tp.h_sb_nexp * NW, (int)(Sp.Npad / TS), c.num_sms,
                   c.plan_slots > 0 ? c.plan_slots : 4 * c.num_sms, c.split_scale);
}

// Buffers every product path uses: the factored scale and the dot scratch.
cudaError_t common_reserve(Ctx& c, const PointsDev& Tp, cudaStream_t st) {
  void* v;
  cudaError_t e;
  const unsigned fin_blocks = (unsigned)((Tp.Npad + 255) / 256);
  if ((e = c.ws.get("mvp.fac", sizeof(float) * (size_t)Tp.Npad, &v))) return e;
  if ((e = c.ws.get("mvp.dotpart", sizeof(double) * MAX_COLS * fin_blocks, &v))) return e;
  const bool fresh = c.ws.slots.find("mvp.dotcnt") == c.ws.slots.end();
  if ((e = c.ws.get("mvp.dotcnt", sizeof(unsigned) * MAX_COLS, &v))) return e;
  if (fresh && (e = cudaMemsetAsync(v, 0, sizeof(unsigned) * MAX_COLS, st))) return e;
  // a device zero: the expanded-form block count of products that take the
  // direct form everywhere
  const bool fresh0 = c.ws.slots.find("mvp.zero") == c.ws.slots.end();
  if ((e = c.ws.get("mvp.zero", sizeof(int), &v))) return e;
  if (fresh0 && (e = cudaMemsetAsync(v, 0, sizeof(int), st))) return e;
  return cudaSuccess;
}

// Largest source-split count among the kernels of a product route at the
// split scale in force (sizes the partial-sum buffers of a tuning candidate).
int route_splits(const Ctx& c, const PointsDev& Tp, const PointsDev& Sp, int m, krr_precision prec) {
  if (m == 1 && prec == KRR_FP32) {
    if (use_tcx(c, Tp)) return std::max(tcx_plan(c, Tp, Sp).splits, tcx_dir_plan(c, Tp, Sp).splits);
    if (Tp.d <= 8) return make_plan(Tp.nblk, (int)(Sp.Npad / TS), c.num_sms, c.plan_slots, c.split_scale).splits;
  }
  int s = multi_plan_dir(c, Tp, Sp).splits;
  if (!multi_direct_only(Tp)) s = std::max(s, multi_plan_tc(c, Tp, Sp, prec, m).splits);
  return s;
}

// The autotuner of the fast products: times the real launch of this route
// (scratch zero weights; the instruction stream does not depend on them),
// best of two after a warm-up, first for each kernel variant of the shape
// (kept in c.tune_variant), then for that variant at each split scale of
// TUNE_SCALES (kept in c.tune_cache; the modelled split unless another is 2%
// faster).  Split candidates whose partial sums would exceed TUNE_MAX_BYTES
// are skipped.
cudaError_t autotune_mvp(Ctx& c, const PointsDev& Tp, const PointsDev& Sp, int m, krr_precision prec,
                         cudaStream_t st, const std::string& key, bool tcgen05_only = false) {
  struct Restore {
    Ctx& c;
    bool prof;
    ~Restore() {
      c.tuning = false;
      c.profiling = prof;
    }
  } restore{c, c.profiling};
  c.tuning = true;
  c.profiling = false;
  void *qv, *yv;
  cudaError_t e;
  if ((e = c.ws.get("tune.q", sizeof(float) * (size_t)m * Sp.Npad, &qv))) return e;
  if ((e = c.ws.get("tune.y", sizeof(float) * (size_t)m * Tp.Npad, &yv))) return e;
  if ((e = cudaMemsetAsync(qv, 0, sizeof(float) * (size_t)m * Sp.Npad, st))) return e;
  cudaEvent_t ev[2];
  if ((e = cudaEventCreate(&ev[0]))) return e;
  if ((e = cudaEventCreate(&ev[1]))) {
    cudaEventDestroy(ev[0]);
    return e;
  }
  MvpOut o;
  o.out_f = (float*)yv;
  const bool single = m == 1 && prec == KRR_FP32;
  auto run = [&]() {
    return single ? mvp_launch(c, Tp, Sp, (const float*)qv, nullptr, 0.f, prec, o, st)
                  : mvp_multi_launch(c, Tp, Sp, (const float*)qv, m, nullptr, 0.f, prec, o, st);
  };
  // one candidate: warm-up (workspace and attributes), then the best of two
  auto time_it = [&](float& ms) -> cudaError_t {
    cudaError_t ee = run();
    ms = 1e30f;
    for (int rep = 0; rep < 2 && !ee; ++rep) {
      cudaEventRecord(ev[0], st);
      ee = run();
      cudaEventRecord(ev[1], st);
      if (!ee) ee = cudaEventSynchronize(ev[1]);
      float t = 0.f;
      if (!ee) cudaEventElapsedTime(&t, ev[0], ev[1]);
      ms = std::min(ms, t);
    }
    return ee;
  };
  // 1. the kernel variant at the modelled split: single-column float32
  // products up to 8 dimensions that would take the tensor-core exponent
  // path also try the packed CUDA-core kernel; multi-column Gaussian products
  // up to 8 dimensions try both kernels for compact blocks and both for
  // direct-form blocks.  The handle's own variant is kept unless another is
  // 2% faster.
  const int cur = current_variant(c, prec, m, Tp);
  std::vector<int> variants{cur};
  if (tcgen05_only) {
    variants.push_back(cur ^ TV_TCGEN05);
  } else if (single && Tp.d <= 8 && use_tcx(c, Tp)) {
    variants.push_back(cur & ~TV_TENSOR_EXP);
  } else if (!single && Tp.d <= 8 && Tp.kfam == KRR_KERNEL_GAUSSIAN) {
    for (int v : {0, (int)TV_TCGEN05, (int)TV_DIRECT_TENSOR, TV_TCGEN05 | TV_DIRECT_TENSOR}) {
      const int vv = (cur & TV_TENSOR_EXP) | v;
      if (vv != cur) variants.push_back(vv);
    }
  }
  c.tune_cache[key] = 1.0;
  int best_v = cur;
  float best_v_ms = -1.f;
  for (int v : variants) {
    c.tune_variant[key] = v;
    float ms;
    if ((e = time_it(ms))) break;
    if (best_v_ms < 0.f || ms < 0.98f * best_v_ms) {
      best_v_ms = ms;
      best_v = v;
    }
  }
  c.tune_variant[key] = best_v;
  // 2. the source split of that variant (not for the solvers' kernel-only
  // choice, which keeps the modelled split)
  double best = 1.0;
  float best_ms = -1.f;
  for (double s : TUNE_SCALES) {
    if (e || tcgen05_only) break;
    c.tune_cache[key] = s;
    {
      TuneScope ts(c, s);
      VariantScope vs(c, key);
      if (s > 1.0 && 8.0 * route_splits(c, Tp, Sp, m, prec) * m * (double)Tp.Npad > TUNE_MAX_BYTES)
        continue;
    }
    float ms;
    if ((e = time_it(ms))) break;
    if (best_ms < 0.f || ms < 0.98f * best_ms) {
      best_ms = ms;
      best = s;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  c.tune_cache[key] = e ? 1.0 : best;
  if (e) c.tune_variant.erase(key);
  return e;
}

// Whether a solver's reserve of this multi-column shape times the two
// kernels of its compact blocks (automatic kernel choice, float32, more than
// TC5_AUTO_MIN_COLS columns, compact blocks present, not nested in another
// product or tuning, stream not capturing).
bool solver_kernel_choice(const Ctx& c, const PointsDev& Tp, int m, krr_precision prec, cudaStream_t st) {
  if (!c.tcgen05_auto || c.tuning || c.prod_depth > 0) return false;
  if (prec != KRR_FP32 || m <= TC5_AUTO_MIN_COLS || multi_direct_only(Tp) || Tp.h_sb_nexp == 0) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs == cudaStreamCaptureStatusNone;
}

}  // namespace

int mvp_targets_per_thread(int d, int64_t N) {
  // the large-T variant amortises shared-memory loads over more pairs; T = 1
  // gives small problems enough CTAs
  const int TL = large_T_of(d);
  return (N / (256LL * TL) >= 32) ? TL : 1;
}

cudaError_t mvp_reserve(Ctx& c, const PointsDev& Tp, const PointsDev& Sp, cudaStream_t st) {
  if (Tp.N == 0) return cudaSuccess;
  const std::string key = tune_key(c, "mvp", Tp, Sp, 1, KRR_FP32);
  if (can_tune(c, st) && !c.tune_cache.count(key)) {
    cudaError_t te = autotune_mvp(c, Tp, Sp, 1, KRR_FP32, st, key);
    if (te) return te;
  }
  TuneScope scope(c, tuned_scale(c, key));
  VariantScope vscope(c, key);
  // above 8 dimensions: the high-dimensional tensor-core kernel on compact
  // super-blocks with the multi-column direct-form kernel on the rest, or
  // that direct-form kernel alone
  if (Tp.d > 8) {
    if (!use_tcx(c, Tp)) return mvp_multi_reserve(c, Tp, Sp, 1, KRR_FP32, st);
    cudaError_t e = common_reserve(c, Tp, st);
    if (e) return e;
    const Plan pt = tcx_plan(c, Tp, Sp), pd = tcx_dir_plan(c, Tp, Sp);
    void* v;
    if ((e = c.ws.get("mvp.partt", sizeof(double) * pt.splits * (size_t)Tp.Npad, &v))) return e;
    if ((e = c.ws.get("mvp.partd", sizeof(double) * pd.splits * (size_t)Tp.Npad, &v))) return e;
    if ((e = mvp_tcx_partials(c, Tp, Sp, nullptr, pt.splits, pt.tiles_per_split, nullptr, nullptr,
                              nullptr, st, true)))
      return e;
    MvpParams p{};
    p.nblk = Tp.nsb;
    return dirm_dispatch(p, Tp.d, Tp.kfam, nullptr, 0, 1, SB / 32, Tp.h_sb_nexp, pd, st, false);
  }
  if (Tp.d < 1) return cudaErrorNotSupported;
  const Plan pl = make_plan(Tp.nblk, (int)(Sp.Npad / TS), c.num_sms, c.plan_slots, c.split_scale);
  void* v;
  cudaError_t e;
  const unsigned fin_blocks = (unsigned)((Tp.Npad + 255) / 256);
  if ((e = c.ws.get("mvp.part", sizeof(double) * pl.splits * (size_t)Tp.Npad, &v))) return e;
  if ((e = c.ws.get("mvp.fac", sizeof(float) * (size_t)Tp.Npad, &v))) return e;
  if ((e = c.ws.get("mvp.dotpart", sizeof(double) * MAX_COLS * fin_blocks, &v))) return e;
  const bool fresh = c.ws.slots.find("mvp.dotcnt") == c.ws.slots.end();
  if ((e = c.ws.get("mvp.dotcnt", sizeof(unsigned) * MAX_COLS, &v))) return e;
  if (fresh && (e = cudaMemsetAsync(v, 0, sizeof(unsigned) * MAX_COLS, st))) return e;
  if (use_tcx(c, Tp)) {
    const Plan pt = tcx_plan(c, Tp, Sp), pd = tcx_dir_plan(c, Tp, Sp);
    if ((e = c.ws.get("mvp.partt", sizeof(double) * pt.splits * (size_t)Tp.Npad, &v))) return e;
    if ((e = c.ws.get("mvp.partd", sizeof(double) * pd.splits * (size_t)Tp.Npad, &v))) return e;
    if ((e = mvp_tcx_partials(c, Tp, Sp, nullptr, pt.splits, pt.tiles_per_split, nullptr, nullptr,
                              nullptr, st, true)))
      return e;
    MvpParams p{};
    p.nblk = Tp.nsb;
    if ((e = dirm_dispatch(p, Tp.d, Tp.kfam, nullptr, 0, 1, SB / 32, Tp.h_sb_nexp, pd, st, false))) return e;
  }
  MvpParams p0{};
  return f32_any(p0, Tp.d, Tp.kfam, Tp.T, pl, st, false);
}

namespace {

// Profiling events around the product kernels (krr_profile_*): returns the
// stop event to record after them, or null.
cudaEvent_t prof_begin(Ctx& c, const PointsDev& Tp, const PointsDev& Sp, cudaStream_t st) {
  if (!c.profiling) return nullptr;
  if (c.prof_used + 2 > c.prof_ev.size() && c.prof_ev.size() < 8192) {
    for (int k = 0; k < 2; ++k) {
      cudaEvent_t ev;
      if (cudaEventCreate(&ev)) return nullptr;
      c.prof_ev.push_back(ev);
    }
  }
  if (c.prof_used + 2 > c.prof_ev.size()) return nullptr;
  cudaEventRecord(c.prof_ev[c.prof_used], st);
  cudaEvent_t stop = c.prof_ev[c.prof_used + 1];
  c.prof_used += 2;
  c.prof_pairs += (double)Tp.N * (double)Sp.N;
  return stop;
}

// Single-column float32 product with the exponent on the tensor cores:
// expanded-form super-blocks in mvp_tcx_kernel, direct-form ones in the
// CUDA-core kernel, then the finalize.
cudaError_t tcx_path(Ctx& c, const PointsDev& Tp, const PointsDev& Sp, const float* q,
                     const float* qdiag, float shift, const MvpOut& o, cudaStream_t st) {
  cudaError_t e = mvp_reserve(c, Tp, Sp, st);
  if (e) return e;
  const Plan pt = tcx_plan(c, Tp, Sp), pd = tcx_dir_plan(c, Tp, Sp);
  void *partt, *partd, *fac, *dpart, *dcnt;
  const unsigned fin_blocks = (unsigned)((Tp.Npad + 255) / 256);
  if ((e = c.ws.get("mvp.partt", sizeof(double) * pt.splits * (size_t)Tp.Npad, &partt))) return e;
  if ((e = c.ws.get("mvp.partd", sizeof(double) * pd.splits * (size_t)Tp.Npad, &partd))) return e;
  if ((e = c.ws.get("mvp.fac", sizeof(float) * (size_t)Tp.Npad, &fac))) return e;
  if ((e = c.ws.get("mvp.dotpart", sizeof(double) * MAX_COLS * fin_blocks, &dpart))) return e;
  if ((e = c.ws.get("mvp.dotcnt", sizeof(unsigned) * MAX_COLS, &dcnt))) return e;
  cudaEvent_t pev1 = prof_begin(c, Tp, Sp, st);
  if (pev1) c.prof_tensor_exp += 1;
  if ((e = mvp_tcx_partials(c, Tp, Sp, q, pt.splits, pt.tiles_per_split, (double*)partt, (float*)fac,
                            o.active, st)))
    return e;
  if (Tp.nsb > Tp.h_sb_nexp) {
    MvpParams p{};
    p.xt = Tp.xs;
    p.Nt = Tp.N;
    p.Nt_pad = Tp.Npad;
    p.tctr = Tp.sb_ctr;
    p.torder = Tp.sb_order;
    p.tn_exp = Tp.sb_nexp;
    p.nblk = Tp.nsb;
    p.xs = Sp.xs;
    p.q = q;
    p.ntiles = (int)(Sp.Npad / TS);
    p.err = c.d_err;
  p.row_lo = c.row_lo;
  p.row_hi = c.row_hi;
    p.s = Sp.scale;
    p.active = o.active;
    p.part_stride = Tp.Npad;
    p.part = (double*)partd;
    p.fac = (float*)fac;
    p.slot0 = Tp.h_sb_nexp;
    if (tcx_dir_f32(Tp)) {
      // the warp blocks are the super-blocks: the packed CUDA-core kernel's
      // direct form, over the direct-form slots only
      switch (Tp.d) {
        case 1: e = dispatch_T<1>(p, Tp.T, pd, st); break;
        case 2: e = dispatch_T<2>(p, Tp.T, pd, st); break;
        case 3: e = dispatch_T<3>(p, Tp.T, pd, st); break;
        case 4: e = dispatch_T<4>(p, Tp.T, pd, st); break;
        case 5: e = dispatch_T<5>(p, Tp.T, pd, st); break;
        case 6: e = dispatch_T<6>(p, Tp.T, pd, st); break;
        case 7: e = dispatch_T<7>(p, Tp.T, pd, st); break;
        default: e = dispatch_T<8>(p, Tp.T, pd, st); break;
      }
      if (e) return e;
    } else if ((e = dirm_dispatch(p, Tp.d, Tp.kfam, q, Sp.Npad, 1, SB / 32, Tp.h_sb_nexp, pd, st, true))) {
      return e;
    }
  }
  if (pev1) cudaEventRecord(pev1, st);
  FinParams f{};
  f.part = (const double*)partt;
  f.splits = pt.splits;
  f.part2 = (const double*)partd;
  f.splits2 = pd.splits;
  f.sb_flag = Tp.sb_flag;
  f.part_stride = Tp.Npad;
  f.N = Tp.N;
  f.Npad = Tp.Npad;
  f.fac = (const float*)fac;
  f.qdiag = qdiag;
  f.shift = shift;
  f.o = o;
  f.dot_part = (double*)dpart;
  f.dot_count = (unsigned*)dcnt;
  f.row_lo = c.row_lo;
  f.row_hi = c.row_hi;
  mvp_finalize_kernel<<<fin_blocks, 256, 0, st>>>(f); count_launch();
  return cudaGetLastError();
}

}  // namespace

cudaError_t mvp_launch(Ctx& c, const PointsDev& Tp, const PointsDev& Sp, const float* q,
                       const float* qdiag, float shift, krr_precision prec, const MvpOut& o,
                       cudaStream_t st) {
  if (prec != KRR_FP32) return mvp_multi_launch(c, Tp, Sp, q, 1, qdiag, shift, prec, o, st);
  if (Tp.N == 0) return cudaSuccess;
  if (Tp.d > 8 && !use_tcx(c, Tp)) return mvp_multi_launch(c, Tp, Sp, q, 1, qdiag, shift, prec, o, st);
  const std::string key = tune_key(c, "mvp", Tp, Sp, 1, KRR_FP32);
  if (can_tune(c, st) && !c.tune_cache.count(key)) {
    cudaError_t te = autotune_mvp(c, Tp, Sp, 1, KRR_FP32, st, key);
    if (te) return te;
  }
  TuneScope scope(c, tuned_scale(c, key));
  VariantScope vscope(c, key);
  if (use_tcx(c, Tp)) return tcx_path(c, Tp, Sp, q, qdiag, shift, o, st);
  MvpParams p{};
  p.xt = Tp.xs;
  p.Nt = Tp.N;
  p.Nt_pad = Tp.Npad;
  p.tctr = Tp.ctr;
  p.torder = Tp.order;
  p.tn_exp = Tp.n_exp;
  p.nblk = Tp.nblk;
  p.xs = Sp.xs;
  p.q = q;
  p.ntiles = (int)(Sp.Npad / TS);
  p.s = Sp.scale;
  p.active = o.active;
  p.part_stride = Tp.Npad;
  p.err = c.d_err;
  p.row_lo = c.row_lo;
  p.row_hi = c.row_hi;
  if (Tp.d < 1 || Tp.d > 8) return cudaErrorNotSupported;
  const Plan pl = make_plan(Tp.nblk, p.ntiles, c.num_sms, c.plan_slots, c.split_scale);
  cudaError_t e = mvp_reserve(c, Tp, Sp, st);
  if (e) return e;
  void *part, *fac, *dpart, *dcnt;
  const unsigned fin_blocks = (unsigned)((Tp.Npad + 255) / 256);
  if ((e = c.ws.get("mvp.part", sizeof(double) * pl.splits * (size_t)Tp.Npad, &part))) return e;
  if ((e = c.ws.get("mvp.fac", sizeof(float) * (size_t)Tp.Npad, &fac))) return e;
  if ((e = c.ws.get("mvp.dotpart", sizeof(double) * MAX_COLS * fin_blocks, &dpart))) return e;
  if ((e = c.ws.get("mvp.dotcnt", sizeof(unsigned) * MAX_COLS, &dcnt))) return e;
  p.part = (double*)part;
  p.fac = (float*)fac;
  cudaEvent_t pev1 = nullptr;
  if (c.profiling) {
    if (c.prof_used + 2 > c.prof_ev.size() && c.prof_ev.size() < 8192) {
      for (int k = 0; k < 2; ++k) {
        cudaEvent_t ev;
        if ((e = cudaEventCreate(&ev))) return e;
        c.prof_ev.push_back(ev);
      }
    }
    if (c.prof_used + 2 <= c.prof_ev.size()) {
      cudaEventRecord(c.prof_ev[c.prof_used], st);
      pev1 = c.prof_ev[c.prof_used + 1];
      c.prof_used += 2;
      c.prof_pairs += (double)Tp.N * (double)Sp.N;
    }
  }
  e = f32_any(p, Tp.d, Tp.kfam, Tp.T, pl, st, true);
  if (e) return e;
  if (pev1) cudaEventRecord(pev1, st);
  FinParams f{};
  f.part = p.part;
  f.splits = pl.splits;
  f.part_stride = Tp.Npad;
  f.N = Tp.N;
  f.Npad = Tp.Npad;
  f.fac = p.fac;
  f.qdiag = qdiag;
  f.shift = shift;
  f.o = o;
  f.dot_part = (double*)dpart;
  f.dot_count = (unsigned*)dcnt;
  f.row_lo = c.row_lo;
  f.row_hi = c.row_hi;
  mvp_finalize_kernel<<<fin_blocks, 256, 0, st>>>(f); count_launch();
  return cudaGetLastError();
}

cudaError_t mvp_multi_reserve(Ctx& c, const PointsDev& Tp, const PointsDev& Sp, int m,
                              krr_precision prec, cudaStream_t st) {
  if (Tp.N == 0) return cudaSuccess;
  if (m < 1 || m > MAX_COLS) return cudaErrorNotSupported;
  const std::string key = tune_key(c, "mvp", Tp, Sp, m, prec);
  if (can_tune(c, st) && !c.tune_cache.count(key)) {
    cudaError_t te = autotune_mvp(c, Tp, Sp, m, prec, st, key);
    if (te) return te;
  } else if (solver_kernel_choice(c, Tp, m, prec, st) && !c.tune_variant.count(key)) {
    // a solver reserving a float32 multi-column shape under the automatic
    // kernel choice: time mvp_umx_kernel against the mma.sync kernel once
    // (a few products, before any graph capture) and keep the faster
    cudaError_t te = autotune_mvp(c, Tp, Sp, m, prec, st, key, true);
    if (te) return te;
  }
  TuneScope scope(c, tuned_scale(c, key));
  VariantScope vscope(c, key);
  const bool direct_only = multi_direct_only(Tp);
  cudaError_t e = direct_only ? common_reserve(c, Tp, st) : mvp_reserve(c, Tp, Sp, st);
  if (e) return e;
  const Plan pt = multi_plan_tc(c, Tp, Sp, prec, m), pd = multi_plan_dir(c, Tp, Sp);
  void* v;
  if ((e = c.ws.get("mvp.partm", sizeof(double) * pt.splits * (size_t)m * Tp.Npad, &v))) return e;
  if ((e = c.ws.get("mvp.partd", sizeof(double) * pd.splits * (size_t)m * Tp.Npad, &v))) return e;
  MvpParams p{};
  p.nblk = Tp.nsb;
  if (use_dirtc(c, Tp)) {
    if ((e = mvp_dirtc_partials(c, Tp, Sp, nullptr, m, prec, pd.splits, pd.tiles_per_split, multi_nexp(Tp),
                                nullptr, nullptr, nullptr, nullptr, st, true)))
      return e;
  } else if ((e = dirm_dispatch(p, Tp.d, Tp.kfam, nullptr, 0, m, SB / 32, multi_nexp(Tp), pd, st, false))) {
    return e;
  }
  if (direct_only) return cudaSuccess;  // no expanded-form blocks: no tensor-core kernel
  if (tc5_on(c, prec, m, Tp))
    return mvp_umma_partials(c, Tp, Sp, nullptr, m, prec == KRR_FP32, prec == KRR_BF16, pt.splits,
                             pt.tiles_per_split, nullptr, nullptr, nullptr, st, true);
  return mvp_tc_partials(c, Tp, Sp, nullptr, m, prec == KRR_FP32, prec == KRR_BF16, pt.splits,
                         pt.tiles_per_split, nullptr, nullptr, nullptr, st, true);
}

cudaError_t mvp_multi_launch(Ctx& c, const PointsDev& Tp, const PointsDev& Sp, const float* Q, int m,
                             const float* qdiag, float shift, krr_precision prec, const MvpOut& o,
                             cudaStream_t st) {
  if (Tp.N == 0) return cudaSuccess;
  if (Tp.d < 1 || (Tp.d > 8 && Tp.d % 16) || Tp.d > 64 || m < 1 || m > MAX_COLS) return cudaErrorNotSupported;
  const std::string key = tune_key(c, "mvp", Tp, Sp, m, prec);
  if (can_tune(c, st) && !c.tune_cache.count(key)) {
    cudaError_t te = autotune_mvp(c, Tp, Sp, m, prec, st, key);
    if (te) return te;
  }
  TuneScope scope(c, tuned_scale(c, key));
  VariantScope vscope(c, key);
  MvpParams p{};
  p.xt = Tp.xs;
  p.Nt = Tp.N;
  p.Nt_pad = Tp.Npad;
  // super-blocks of SB targets, expanded-form first
  p.tctr = Tp.sb_ctr;
  p.torder = Tp.sb_order;
  p.tn_exp = Tp.sb_nexp;
  p.nblk = Tp.nsb;
  p.xs = Sp.xs;
  p.ntiles = (int)(Sp.Npad / TS);
  p.err = c.d_err;
  p.row_lo = c.row_lo;
  p.row_hi = c.row_hi;
  p.s = Sp.scale;
  p.active = o.active;
  p.part_stride = (int64_t)m * Tp.Npad;
  const Plan pt = multi_plan_tc(c, Tp, Sp, prec, m), pd = multi_plan_dir(c, Tp, Sp);
  const bool direct_only = multi_direct_only(Tp);
  const int64_t nexp = multi_nexp(Tp);
  cudaError_t e = direct_only ? common_reserve(c, Tp, st) : mvp_reserve(c, Tp, Sp, st);
  if (e) return e;
  void *part, *partd, *fac, *dpart, *dcnt;
  const unsigned fin_blocks = (unsigned)((Tp.Npad + 255) / 256);
  if ((e = c.ws.get("mvp.partm", sizeof(double) * pt.splits * (size_t)m * Tp.Npad, &part))) return e;
  if ((e = c.ws.get("mvp.partd", sizeof(double) * pd.splits * (size_t)m * Tp.Npad, &partd))) return e;
  if ((e = c.ws.get("mvp.fac", sizeof(float) * (size_t)Tp.Npad, &fac))) return e;
  if ((e = c.ws.get("mvp.dotpart", sizeof(double) * MAX_COLS * fin_blocks, &dpart))) return e;
  if ((e = c.ws.get("mvp.dotcnt", sizeof(unsigned) * MAX_COLS, &dcnt))) return e;
  p.fac = (float*)fac;
  cudaEvent_t pev1 = prof_begin(c, Tp, Sp, st);
  // expanded-form super-blocks: all columns on the tensor cores (float32
  // products of more than 8 columns: P Q by tcgen05 in mvp_umx_kernel; the
  // others: mma.sync; KRR_OPT_TCGEN05 overrides)
  if (nexp > 0) {
    e = tc5_on(c, prec, m, Tp)
            ? mvp_umma_partials(c, Tp, Sp, Q, m, prec == KRR_FP32, prec == KRR_BF16, pt.splits,
                                pt.tiles_per_split, (double*)part, p.fac, o.active, st)
            : mvp_tc_partials(c, Tp, Sp, Q, m, prec == KRR_FP32, prec == KRR_BF16, pt.splits,
                              pt.tiles_per_split, (double*)part, p.fac, o.active, st);
    if (e) return e;
  }
  // direct-form super-blocks: all columns in one launch (the weighted sum
  // on the tensor cores, or the CUDA-core kernel by option)
  if (Tp.nsb > nexp) {
    p.part = (double*)partd;
    if (direct_only) {
      // every super-block direct: the kernel reads an expanded-form count of 0
      void* zero;
      if ((e = c.ws.get("mvp.zero", sizeof(int), &zero))) return e;
      p.tn_exp = (const int*)zero;
    }
    if (use_dirtc(c, Tp)) {
      if ((e = mvp_dirtc_partials(c, Tp, Sp, Q, m, prec, pd.splits, pd.tiles_per_split, nexp, p.tn_exp,
                                  (double*)partd, p.fac, o.active, st, false)))
        return e;
    } else if ((e = dirm_dispatch(p, Tp.d, Tp.kfam, Q, Sp.Npad, m, SB / 32, nexp, pd, st, true))) {
      return e;
    }
  }
  if (pev1) cudaEventRecord(pev1, st);
  FinParams f{};
  f.part = (const double*)(direct_only ? partd : part);
  f.splits = direct_only ? pd.splits : pt.splits;
  f.part2 = (const double*)partd;
  f.splits2 = pd.splits;
  f.sb_flag = direct_only ? nullptr : Tp.sb_flag;
  f.part_stride = (int64_t)m * Tp.Npad;
  f.N = Tp.N;
  f.Npad = Tp.Npad;
  f.fac = p.fac;
  f.qdiag = qdiag;
  f.shift = shift;
  f.o = o;
  f.dot_part = (double*)dpart;
  f.dot_count = (unsigned*)dcnt;
  f.row_lo = c.row_lo;
  f.row_hi = c.row_hi;
  mvp_finalize_kernel<<<dim3(fin_blocks, (unsigned)m), 256, 0, st>>>(f); count_launch();
  return cudaGetLastError();
}

}  // namespace krr
