// Multi-column product over the direct-form super-blocks with the weighted
// sum on the tensor cores (hot-path steps A3/A4 where target blocks are not
// compact):
//
//   Y[i, c] = sum_j P_ij Q[j, c],   P_ij = k(x_i, x_j)        (Eqs. 1-3)
//
// Super-blocks that are too wide for the expanded exponent form (prep.cu) need
// the exact differences x_i - x_j of the raw float32 coordinates, so the
// kernel value stays on the CUDA cores: d packed f32x2 subtractions and
// multiply-adds per pair of sources, one multiply(-add) and one MUFU.EX2
// (Gaussian, 2^(-s^2 r^2)), or the Matern 3/2 value of Sec. 6.1.  What the
// CUDA-core kernel (mvp_dirm_kernel) spent on the m columns, m FMAs per pair,
// becomes a dense contraction on the tensor cores (mma.sync, 8 columns per
// MMA), each thread computing the kernel values of the A fragment it owns:
//   * float32-grade products use tf32 operands split into hi + lo, with
//     P = Ph + Pl, Ph = P with its low 13 mantissa bits cleared (one logical
//     operation) and Pl = P - Ph exact (one subtraction): Ph Qh + Pl Qh +
//     Ph Ql (m16n8k8), relative error per term below 3 * 2^-20.  No format
//     conversion is needed (tf32 is float32's layout), and tf32 has float32's
//     exponent range, so small kernel values and large weights keep their
//     precision;
//   * reduced-precision products (the inner M p of Sec. 5.1) issue P Q with
//     single f16 or bf16 operands (m16n8k16); f16 kernel values are formed as
//     2^15 P (the offset enters the exponent) so that small values stay out
//     of the f16 subnormal range, and the sums are scaled back by 2^-15.
// Accumulators fold into float32 Kahan sums once per source tile; each source
// split writes one FP64 partial per (column, target), summed in fixed order by
// the finalize kernel (deterministic).
//
// One CTA of 16 warps per direct-form super-block (256 targets, one m-tile of
// 16 per warp).  Source tiles (raw coordinates and the m weight columns) arrive
// by 1-D TMA bulk copies into an RS-stage ring (mbarrier completion, bounded
// waits); the CTA then rewrites each tile into a work buffer: the coordinates
// negated and permuted so that one 16-byte load gives a thread its four
// sources of a 16-source step, and the weights in the B-fragment order (tf32
// hi and lo, or one f16 / bf16 row).  Work buffers are double-buffered so
// tile r + 1 is rewritten before tile r is consumed.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace krr {
namespace {

constexpr int DT_THREADS = 512;            // 16 warps: one m-tile of 16 targets each
constexpr int DT_RS = 2;                   // raw stages
constexpr int QS = 264;                    // halves per f16 weight row of a work buffer (256 + pad)
constexpr int QSW = 260;                   // words per tf32 weight row (256 + pad: conflict-free)
constexpr uint32_t TF32_MASK = 0xFFFFE000u;  // clears the 13 mantissa bits tf32 drops
constexpr float F16_OFFSET = 15.f;         // f16 kernel values are 2^15 P
constexpr float kLog2eDt = 1.4426950408889634f;

struct DtParams {
  const float* xt;      // targets, tile-blocked SoA (raw coordinates)
  int64_t Nt, Nt_pad;
  const int* torder;    // super-blocks, expanded-form first
  const int* tn_exp;    // device count of expanded-form super-blocks
  int64_t nsb;          // super-blocks
  int64_t slot0;        // first super-block slot of the grid (the host's count)
  const float* xs;      // sources, tile-blocked SoA (raw coordinates)
  const float* Q;       // sorted source weights, m columns of stride q_stride
  int64_t q_stride;
  int m;
  int ntiles, tiles_per_split;
  double* part;         // [split][column][Nt_pad]
  float* fac;           // [Nt_pad]: 1 for direct-form targets
  int* err;
  float s;              // Gaussian: sqrt(log2(e) / (2 sigma^2)); Matern: sqrt(3) / h
  const int* active;
  int64_t row_lo, row_hi;
};

template <bool BF>
struct HalfOps;
template <>
struct HalfOps<false> {
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    __half2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ uint16_t bits(float v) {
    __half h = __float2half_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
  }
};
template <>
struct HalfOps<true> {
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    __nv_bfloat162 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ uint16_t bits(float v) {
    __nv_bfloat16 h = __float2bfloat16_rn(v);
    return *reinterpret_cast<uint16_t*>(&h);
  }
};

template <bool BF>
__device__ __forceinline__ void mma_16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  if constexpr (BF) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  } else {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
        "{%8,%9}, {%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
  }
}

__device__ __forceinline__ void mma_1688_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Kernel values of two pairs from their squared raw distances, times 2^off.
template <int KF>
__device__ __forceinline__ float2 pair_values(float2 r2, float s, float off) {
  if constexpr (KF == 0) {
    const float2 e = ffma2(r2, make_float2(-s * s, -s * s), make_float2(off, off));
    return make_float2(ex2(e.x), ex2(e.y));
  } else {
    // Matern 3/2: a = s r, (1 + a) 2^(off - a log2 e); r through the
    // reciprocal square root, the clamp keeping r2 = 0 at a = 0
    float2 v;
    float a = s * (r2.x * rsqrtf(fmaxf(r2.x, 1e-30f)));
    float e = ex2(fmaf(a, -kLog2eDt, off));
    v.x = fmaf(a, e, e);
    a = s * (r2.y * rsqrtf(fmaxf(r2.y, 1e-30f)));
    e = ex2(fmaf(a, -kLog2eDt, off));
    v.y = fmaf(a, e, e);
    return v;
  }
}

template <int D, int NRT, bool SPLIT>
constexpr uint32_t dt_raw_floats() {
  return (uint32_t)(D + 8 * NRT) * TS;
}
// work buffer: D x 256 permuted negated coordinates, then the weight rows of
// 8 NRT columns: tf32 hi and lo at QSW words each (split), else QS halves
template <int D, int NRT, bool SPLIT>
constexpr uint32_t dt_work_bytes() {
  return (uint32_t)(sizeof(float) * D * TS +
                    (SPLIT ? 4 * 2 * 8 * NRT * QSW : 2 * 8 * NRT * QS));
}
template <int D, int NRT, bool SPLIT>
constexpr size_t dt_smem_bytes() {
  return sizeof(float) * DT_RS * dt_raw_floats<D, NRT, SPLIT>() + 2 * (size_t)dt_work_bytes<D, NRT, SPLIT>();
}

template <int D, int NRT, bool SPLIT, bool BF, int KF>
__global__ void __launch_bounds__(DT_THREADS, 1) mvp_dirtc_kernel(const DtParams p) {
  using H = HalfOps<BF>;
  constexpr int MC = 8 * NRT;
  constexpr uint32_t RAW = dt_raw_floats<D, NRT, SPLIT>();
  constexpr uint32_t WORK = dt_work_bytes<D, NRT, SPLIT>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[DT_RS];
  __shared__ volatile int abort_flag;
  if (p.active && *p.active == 0) return;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int64_t slot = p.slot0 + blockIdx.x;
  if (slot >= p.nsb || slot < *p.tn_exp) return;  // not a direct-form super-block
  const int64_t blk = p.torder[slot];
  if (blk * SB < p.row_lo || blk * SB >= p.row_hi) return;  // outside the shard
  float* raw = reinterpret_cast<float*>(smem_raw);
  unsigned char* work = smem_raw + sizeof(float) * DT_RS * RAW;

  // this thread's targets: rows g and g + 8 of the warp's m-tile, each
  // coordinate held twice (both halves of a packed f32x2 operand)
  const int64_t row0 = blk * SB + 16 * warp;
  float2 xd[2][D];
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t i = row0 + g + 8 * h;  // < Nt_pad: padding repeats the last point
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float x = p.xt[(i / TS) * (int64_t)D * TS + (int64_t)k * TS + i % TS];
      xd[h][k] = make_float2(x, x);
    }
    if (blockIdx.y == 0 && t == 0) p.fac[i] = 1.f;
  }

  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;

  float acc[NRT][4], S[NRT][4], C[NRT][4];
#pragma unroll
  for (int rt = 0; rt < NRT; ++rt)
#pragma unroll
    for (int e = 0; e < 4; ++e) acc[rt][e] = S[rt][e] = C[rt][e] = 0.f;

  auto issue = [&](int r) {
    const int stage = r % DT_RS;
    const int64_t tile = t_begin + r;
    float* dst = raw + stage * RAW;
    mbar_arrive_expect_tx(&bars[stage], (uint32_t)(D + p.m) * TS * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    for (int c = 0; c < p.m; ++c)
      bulk_g2s(dst + (D + c) * TS, p.Q + (int64_t)c * p.q_stride + tile * (int64_t)TS, TS * 4, &bars[stage]);
  };

  // raw tile r -> work buffer b.  Coordinate k of source j = 16 kk + jj,
  // negated, at float (kk D + k) 16 + pos(jj), so that thread t's four
  // sources of the step are one float4 at 4 t: tf32 fragments (k = 8) take
  // sources t, t + 4, t + 8, t + 12 (pos = 4 (jj mod 4) + jj / 4); f16
  // fragments (k = 16) take 2t, 2t + 1, 2t + 8, 2t + 9
  // (pos = 4 ((jj mod 8) / 2) + 2 (jj / 8) + jj mod 2).  Weight column c of
  // source j: split, tf32 hi at word c QSW + j and lo MC QSW words later;
  // else one f16 / bf16 value at half c QS + j.
  auto rewrite = [&](int r, int b) {
    const float* rs = raw + (r % DT_RS) * RAW;
    float* xw = reinterpret_cast<float*>(work + b * WORK);
    for (int e = tid; e < D * TS; e += DT_THREADS) {
      const int k = e / TS, j = e % TS, kk = j >> 4, jj = j & 15;
      const int pos = SPLIT ? 4 * (jj & 3) + (jj >> 2) : 4 * ((jj & 7) >> 1) + 2 * (jj >> 3) + (jj & 1);
      xw[(kk * D + k) * 16 + pos] = -rs[k * TS + j];
    }
    if constexpr (SPLIT) {
      uint32_t* qw = reinterpret_cast<uint32_t*>(xw + D * TS);
      for (int e = tid; e < MC * TS; e += DT_THREADS) {
        const int c = e / TS, j = e % TS;
        const float v = c < p.m ? rs[(D + c) * TS + j] : 0.f;
        const uint32_t hi = __float_as_uint(v) & TF32_MASK;
        qw[c * QSW + j] = hi;
        qw[(MC + c) * QSW + j] = __float_as_uint(v - __uint_as_float(hi));
      }
    } else {
      uint16_t* qh = reinterpret_cast<uint16_t*>(xw + D * TS);
      for (int e = tid; e < MC * TS; e += DT_THREADS) {
        const int c = e / TS, j = e % TS;
        qh[c * QS + j] = H::bits(c < p.m ? rs[(D + c) * TS + j] : 0.f);
      }
    }
  };

  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < DT_RS; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0)
    for (; issued < min(DT_RS, nt); ++issued) issue(issued);
  if (nt > 0) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[0], 0));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    }
    __syncthreads();
    if (!abort_flag) rewrite(0, 0);
    __syncthreads();
  }

  for (int r = 0; r < nt && !abort_flag; ++r) {
    // raw stage r % RS was consumed by rewrite(r); refill it with tile r + RS
    if (tid == 0 && r + DT_RS < nt) {
      fence_proxy_async_smem();
      issue(r + DT_RS);
      ++issued;
    }
    if (r + 1 < nt) {
      const bool ok =
          __all_sync(0xffffffffu, mbar_wait_bounded(&bars[(r + 1) % DT_RS], ((r + 1) / DT_RS) & 1));
      if (!ok) {
        abort_flag = 1;
        if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
      } else {
        rewrite(r + 1, (r + 1) & 1);
      }
    }
    const float* xw = reinterpret_cast<const float*>(work + (r & 1) * WORK);
    const uint32_t* qw = reinterpret_cast<const uint32_t*>(xw + D * TS);
#pragma unroll 1
    for (int kk = 0; kk < TS / 16; ++kk) {
      // squared distances of rows g, g + 8 to this thread's four sources of
      // the step, as two packed pairs (f32x2)
      float2 r2[2][2];
#pragma unroll
      for (int h = 0; h < 2; ++h) r2[h][0] = r2[h][1] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float4 nx = *reinterpret_cast<const float4*>(xw + (kk * D + k) * 16 + 4 * t);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float2 d0 = fadd2(xd[h][k], make_float2(nx.x, nx.y));
          const float2 d1 = fadd2(xd[h][k], make_float2(nx.z, nx.w));
          r2[h][0] = ffma2(d0, d0, r2[h][0]);
          r2[h][1] = ffma2(d1, d1, r2[h][1]);
        }
      }
      const float off = (SPLIT || BF) ? 0.f : F16_OFFSET;
      const float2 v0 = pair_values<KF>(r2[0][0], p.s, off), v1 = pair_values<KF>(r2[1][0], p.s, off);
      const float2 v2 = pair_values<KF>(r2[0][1], p.s, off), v3 = pair_values<KF>(r2[1][1], p.s, off);
      if constexpr (SPLIT) {
        // tf32 A fragments of the two k = 8 halves of the step: a0 (g; t),
        // a1 (g+8; t), a2 (g; t+4), a3 (g+8; t+4); v0 = row g at sources
        // (t, t + 4), v2 = row g at (t + 8, t + 12), v1 / v3 the same for g + 8
        uint32_t ah[2][4], al[2][4];
        const float vv[2][4] = {{v0.x, v1.x, v0.y, v1.y}, {v2.x, v3.x, v2.y, v3.y}};
#pragma unroll
        for (int hf = 0; hf < 2; ++hf)
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            ah[hf][w] = __float_as_uint(vv[hf][w]) & TF32_MASK;
            al[hf][w] = __float_as_uint(vv[hf][w] - __uint_as_float(ah[hf][w]));
          }
#pragma unroll
        for (int rt = 0; rt < NRT; ++rt) {
          const int c = rt * 8 + g;
#pragma unroll
          for (int hf = 0; hf < 2; ++hf) {
            const int j0 = kk * 16 + hf * 8 + t;
            const uint32_t b0 = qw[c * QSW + j0], b1 = qw[c * QSW + j0 + 4];
            const uint32_t l0 = qw[(MC + c) * QSW + j0], l1 = qw[(MC + c) * QSW + j0 + 4];
            mma_1688_tf32(acc[rt], ah[hf], b0, b1);
            mma_1688_tf32(acc[rt], al[hf], b0, b1);
            mma_1688_tf32(acc[rt], ah[hf], l0, l1);
          }
        }
      } else {
        // f16 / bf16 A fragment: a0 (g; 2t, 2t+1), a1 (g+8; 2t, 2t+1),
        // a2 (g; 2t+8, 2t+9), a3 (g+8; 2t+8, 2t+9)
        uint32_t ph[4];
        ph[0] = H::pack(v0.x, v0.y);
        ph[1] = H::pack(v1.x, v1.y);
        ph[2] = H::pack(v2.x, v2.y);
        ph[3] = H::pack(v3.x, v3.y);
#pragma unroll
        for (int rt = 0; rt < NRT; ++rt) {
          const int c = rt * 8 + g;
          const uint32_t b0 = qw[c * (QS / 2) + kk * 8 + t], b1 = qw[c * (QS / 2) + kk * 8 + t + 4];
          mma_16816<BF>(acc[rt], ph, b0, b1);
        }
      }
    }
    // f16 sums carry the 2^15 offset of the kernel values
    constexpr float unscale = (SPLIT || BF) ? 1.f : 1.f / 32768.f;
#pragma unroll
    for (int rt = 0; rt < NRT; ++rt)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        kahan_add(S[rt][e], C[rt][e], acc[rt][e] * unscale);
        acc[rt][e] = 0.f;
      }
    __syncthreads();
  }
  if (abort_flag) {
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % DT_RS], (r / DT_RS) & 1);
    __syncthreads();
    return;
  }
  // accumulator element e: row g + 8 (e >> 1), column 8 rt + 2t + (e & 1)
#pragma unroll
  for (int rt = 0; rt < NRT; ++rt)
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int c = rt * 8 + 2 * t + (e & 1);
      const int64_t i = row0 + g + 8 * (e >> 1);
      if (c < p.m && i < p.Nt_pad)
        p.part[((int64_t)blockIdx.y * p.m + c) * p.Nt_pad + i] = (double)S[rt][e] - (double)C[rt][e];
    }
}

template <int D, int NRT, bool SPLIT, bool BF, int KF>
cudaError_t dt_launch(const DtParams& p, int64_t nctas, int splits, cudaStream_t st, bool launch) {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  constexpr size_t shm = dt_smem_bytes<D, NRT, SPLIT>();
  static_assert(shm <= 227 * 1024, "shared memory");
  if (!(dev < 128 && done[dev])) {
    cudaError_t e = cudaFuncSetAttribute(mvp_dirtc_kernel<D, NRT, SPLIT, BF, KF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e) return e;
    if (dev < 128) done[dev] = true;
  }
  if (!launch) return cudaSuccess;
  mvp_dirtc_kernel<D, NRT, SPLIT, BF, KF><<<dim3((unsigned)nctas, (unsigned)splits), DT_THREADS, shm, st>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <int D, int KF>
cudaError_t dt_dispatch_d(const DtParams& p, int64_t nctas, int splits, krr_precision prec,
                          cudaStream_t st, bool launch) {
  const bool two = p.m > 8;
  if (KF != 0 || prec == KRR_FP32)
    return two ? dt_launch<D, 2, true, false, KF>(p, nctas, splits, st, launch)
               : dt_launch<D, 1, true, false, KF>(p, nctas, splits, st, launch);
  if constexpr (KF == 0) {
    if (prec == KRR_BF16)
      return two ? dt_launch<D, 2, false, true, 0>(p, nctas, splits, st, launch)
                 : dt_launch<D, 1, false, true, 0>(p, nctas, splits, st, launch);
    return two ? dt_launch<D, 2, false, false, 0>(p, nctas, splits, st, launch)
               : dt_launch<D, 1, false, false, 0>(p, nctas, splits, st, launch);
  }
  return cudaErrorNotSupported;
}

template <int KF>
cudaError_t dt_dispatch(const DtParams& p, int d, int64_t nctas, int splits, krr_precision prec,
                        cudaStream_t st, bool launch) {
  switch (d) {
    case 1: return dt_dispatch_d<1, KF>(p, nctas, splits, prec, st, launch);
    case 2: return dt_dispatch_d<2, KF>(p, nctas, splits, prec, st, launch);
    case 3: return dt_dispatch_d<3, KF>(p, nctas, splits, prec, st, launch);
    case 4: return dt_dispatch_d<4, KF>(p, nctas, splits, prec, st, launch);
    case 5: return dt_dispatch_d<5, KF>(p, nctas, splits, prec, st, launch);
    case 6: return dt_dispatch_d<6, KF>(p, nctas, splits, prec, st, launch);
    case 7: return dt_dispatch_d<7, KF>(p, nctas, splits, prec, st, launch);
    case 8: return dt_dispatch_d<8, KF>(p, nctas, splits, prec, st, launch);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace

cudaError_t mvp_dirtc_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* Q, int m,
                               krr_precision prec, int splits, int tiles_per_split, int64_t slot0,
                               const int* tn_exp, double* part, float* fac, const int* active,
                               cudaStream_t st, bool dry) {
  if (T.d < 1 || T.d > 8 || m < 1 || m > MAX_COLS) return cudaErrorNotSupported;
  DtParams p{};
  p.xt = T.xs;
  p.Nt = T.N;
  p.Nt_pad = T.Npad;
  p.torder = T.sb_order;
  p.tn_exp = tn_exp;
  p.nsb = T.nsb;
  p.slot0 = slot0;
  p.xs = S.xs;
  p.Q = Q;
  p.q_stride = S.Npad;
  p.m = m;
  p.ntiles = (int)(S.Npad / TS);
  p.tiles_per_split = tiles_per_split;
  p.part = part;
  p.fac = fac;
  p.err = c.d_err;
  p.s = S.scale;
  p.active = active;
  p.row_lo = c.row_lo;
  p.row_hi = c.row_hi;
  const int64_t nctas = std::max<int64_t>(1, T.nsb - slot0);
  if (T.kfam == KRR_KERNEL_MATERN32) return dt_dispatch<1>(p, T.d, nctas, splits, prec, st, !dry);
  if (T.kfam != KRR_KERNEL_GAUSSIAN) return cudaErrorNotSupported;
  return dt_dispatch<0>(p, T.d, nctas, splits, prec, st, !dry);
}

}  // namespace krr
