// Tensor-core kernel product for several right-hand sides and for the
// reduced-precision inner product (hot-path steps A3/A4):
//
//   Y[i, c] = sum_j 2^(-s^2 |x_i - x_j|^2) Q[j, c]        (Eqs. 1-2)
//
// over the expanded-form super-blocks of prep.cu (compact blocks of 256 targets with
// centre c, x^ = s (x - c), |x^_i|^2 <= EXPANDED_R2), written as two dense
// contractions on the tensor cores (mma.sync m16n8k16, f16 or bf16 inputs,
// f32 accumulation) around one special-function step:
//
//  1. E = A B^T with A_i = [x^_i, 1] and B_j = [2 x^_j, b_j], b_j = -|x^_j|^2,
//     so that E_ij = -|x^_i - x^_j|^2 + |x^_i|^2.  A and B are split into
//     f16 hi + lo parts stacked along the contraction (K) dimension,
//     A' = [Ah, Ah, Al, Al], B' = [Bh, Bl, Bh, Bl] (three terms when four do
//     not fit), so one MMA yields E to about 2^-33 relative: FP32-grade
//     exponents at d <= 3, about 2^-22 otherwise.
//  2. P = 2^E by MUFU.EX2 straight from the accumulator registers; the
//     accumulator fragment of the first MMA is the operand fragment of the
//     second (no shared-memory round trip); 2^(-|x^_i|^2) is applied by the
//     finalize kernel.
//  3. Y += P Q: in f16 for the reduced-precision product, or with P and Q
//     split hi + lo (three MMAs: Ph Qh + Pl Qh + Ph Ql) for float32-grade
//     results, folded into float32 Kahan sums every few source tiles.
//
// The tensor work per pair (2m flops for P Q plus 2 x 16 for E) is far below
// even the mma.sync peak; the kernel is bound by MUFU.EX2 and the f32->f16
// packing, and the accumulation into many right-hand sides is nearly free.
// Operands stay in registers, which is why mma.sync (register fragments) is
// used rather than tcgen05 (operands in shared or tensor memory).
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace krr {
namespace {

constexpr int RS = 2;  // raw stages

struct TcParams {
  const float* xt;    // targets (tile-blocked SoA, raw)
  int64_t Nt, Nt_pad;
  const float* tctr;  // warp-block centres
  const int* torder;
  const int* tn_exp;
  int64_t nblk;       // CTAs: the expanded-form super-blocks
  int WB;             // warp-block size (targets)
  const float* xs;    // sources (tile-blocked SoA, raw)
  const float* Q;     // sorted source weights, m columns of stride Ns_pad
  int64_t Ns_pad;
  int m;
  int ntiles, tiles_per_split;
  double* part;       // [split][col][Nt_pad]
  float* fac;         // [Nt_pad]
  int* err;
  float s;
  const int* active;
  // tcgen05 kernel: weights pre-split into f16 hi / lo, one 16 x 256 K-major
  // tile (8 KB) per source tile
  const uint16_t* qh_tiles;
  const uint16_t* ql_tiles;
  // sorted target rows computed (shard emulation): whole super-blocks outside
  // [row_lo, row_hi) are skipped
  int64_t row_lo = 0, row_hi = INT64_MAX;
};

// Terms of the split exponent: 4 (Ah Bh + Ah Bl + Al Bh + Al Bl) when 4(D+1)
// fits the contraction, else 3; contraction steps of 16.
template <int D>
struct ExpLayout {
  static constexpr int W = D + 1;
  static constexpr int TERMS = (4 * W <= 16 || (4 * W > 16 && 4 * W <= 32 && D > 4)) ? 4 : 3;
  static constexpr int KSTEPS = (TERMS * W + 15) / 16;
  static constexpr int KV = 16 * KSTEPS;              // halves per K-vector
  static constexpr int KV_STRIDE_W = KSTEPS == 1 ? 12 : 20;  // 32-bit words, bank-conflict free
};

template <bool BF>
struct Half;
template <>
struct Half<false> {
  using T = __half;
  using T2 = __half2;
  static __device__ __forceinline__ T from(float v) { return __float2half_rn(v); }
  static __device__ __forceinline__ float to(T v) { return __half2float(v); }
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    T2 h = __floats2half2_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 unpack(uint32_t u) {
    T2 h = *reinterpret_cast<T2*>(&u);
    return __half22float2(h);
  }
};
template <>
struct Half<true> {
  using T = __nv_bfloat16;
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ T from(float v) { return __float2bfloat16_rn(v); }
  static __device__ __forceinline__ float to(T v) { return __bfloat162float(v); }
  static __device__ __forceinline__ uint32_t pack(float lo, float hi) {
    T2 h = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&h);
  }
  static __device__ __forceinline__ float2 unpack(uint32_t u) {
    T2 h = *reinterpret_cast<T2*>(&u);
    return __bfloat1622float2(h);
  }
};

template <bool BF>
__device__ __forceinline__ void mma16816(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
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

// d = a b (zero accumulator input), f16 operands.
__device__ __forceinline__ void mma16816_z(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                           uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.f16.f16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%10,%10,%10,%10};"
      : "=f"(d[0]), "=f"(d[1]), "=f"(d[2]), "=f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1), "f"(0.f));
}

// Value of K-vector slot k for the split vector v (hi/lo per component):
// A' = [h, h, l, l] (operand A) or B' = [h, l, h, l] (operand B); 3-term
// layouts drop the last block.
template <int D>
__device__ __forceinline__ float kv_value(const float (&h)[D + 1], const float (&l)[D + 1], int k,
                                          bool is_a) {
  constexpr int W = D + 1;
  constexpr int TERMS = ExpLayout<D>::TERMS;
  const int term = k / W, comp = k % W;
  if (term >= TERMS) return 0.f;
  const bool lo = is_a ? (term >= 2) : (term & 1);
  float v = 0.f;
#pragma unroll
  for (int c = 0; c < W; ++c)
    if (c == comp) v = lo ? l[c] : h[c];
  return v;
}

template <int D, int MT, int NRT, bool SPLIT, bool BF>
__global__ void __launch_bounds__(256) mvp_tc_kernel(const TcParams p) {
  using L = ExpLayout<D>;
  using H = Half<BF>;
  constexpr int W = D + 1;
  constexpr int MC = 8 * NRT;  // padded right-hand sides
  constexpr int QSTRIDE_W = 132;  // words per column of a source tile (256 halves + pad)
  extern __shared__ __align__(128) float smem[];
  const int nthreads = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  __shared__ __align__(8) uint64_t bars[RS];
  __shared__ volatile int abort_flag;
  if (p.active && *p.active == 0) return;
  const int64_t nexp = *p.tn_exp;
  if ((int64_t)blockIdx.x >= nexp) return;  // direct-form blocks: CUDA-core kernel

  const int raw_floats = (D + p.m) * TS;
  float* raw = smem;                                                  // RS stages
  uint32_t* kvb = reinterpret_cast<uint32_t*>(smem + RS * raw_floats);  // 2 x TS x KV_STRIDE_W
  uint32_t* qb = kvb + 2 * TS * L::KV_STRIDE_W;                         // 2 x (SPLIT?2:1) x MC x QSTRIDE_W
  constexpr int QBUF_W = (SPLIT ? 2 : 1) * MC * QSTRIDE_W;

  const int64_t blk = p.torder[blockIdx.x];
  if (blk * SB < p.row_lo || blk * SB >= p.row_hi) return;  // outside the shard
  float ctr[D];
#pragma unroll
  for (int k = 0; k < D; ++k) ctr[k] = p.tctr[blk * D + k];

  // ---- operand A' of the exponent MMA for this warp's m-tiles (constant)
  uint32_t afr[MT][L::KSTEPS][4];
  const int64_t row0 = blk * p.WB + (int64_t)warp * 16 * MT;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {  // rows g and g + 8
      const int64_t i = row0 + mt * 16 + g + 8 * half;
      const int64_t ii = i < p.Nt ? i : p.Nt - 1;
      float ah[W], al[W];
      float r2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float x = p.xt[(ii / TS) * (int64_t)D * TS + (int64_t)k * TS + ii % TS];
        const float xh = p.s * (x - ctr[k]);
        r2 = fmaf(xh, xh, r2);
        ah[k] = H::to(H::from(xh));
        al[k] = xh - ah[k];
      }
      ah[D] = 1.f;
      al[D] = 0.f;
      if (blockIdx.y == 0 && t == 0 && i < p.Nt_pad) p.fac[i] = exp2f(-r2);
#pragma unroll
      for (int ks = 0; ks < L::KSTEPS; ++ks) {
        const int k0 = 16 * ks + 2 * t;
        afr[mt][ks][half] = H::pack(kv_value<D>(ah, al, k0, true), kv_value<D>(ah, al, k0 + 1, true));
        afr[mt][ks][half + 2] =
            H::pack(kv_value<D>(ah, al, k0 + 8, true), kv_value<D>(ah, al, k0 + 9, true));
      }
    }
  }

  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;

  float acc[MT][NRT][4];
  float S[MT][NRT][4], C[MT][NRT][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int rt = 0; rt < NRT; ++rt)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[mt][rt][e] = S[mt][rt][e] = C[mt][rt][e] = 0.f;

  auto issue = [&](int r) {
    const int stage = r % RS;
    const int64_t tile = t_begin + r;
    float* dst = raw + stage * raw_floats;
    mbar_arrive_expect_tx(&bars[stage], (uint32_t)raw_floats * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    for (int c = 0; c < p.m; ++c)
      bulk_g2s(dst + (D + c) * TS, p.Q + (int64_t)c * p.Ns_pad + tile * (int64_t)TS, TS * 4,
               &bars[stage]);
  };

  // CTA-wide transform of raw tile r into buffer b: source K-vectors and the
  // weights in half precision (hi, and lo when split)
  auto transform = [&](int r, int b) {
    const float* rs = raw + (r % RS) * raw_floats;
    uint32_t* kv = kvb + b * TS * L::KV_STRIDE_W;
    uint32_t* qq = qb + b * QBUF_W;
    for (int j = tid; j < TS; j += nthreads) {
      float bh[W], bl[W];
      float bb = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float xh = p.s * (rs[k * TS + j] - ctr[k]);
        bb = fmaf(-xh, xh, bb);
        const float v = 2.f * xh;
        bh[k] = H::to(H::from(v));
        bl[k] = v - bh[k];
      }
      if (bb < -30000.f) {  // farther than any target can see: contributes 0
#pragma unroll
        for (int k = 0; k < D; ++k) bh[k] = bl[k] = 0.f;
        bb = -30000.f;
      }
      bh[D] = H::to(H::from(bb));
      bl[D] = bb - bh[D];
      uint16_t hv[L::KV];
#pragma unroll
      for (int k = 0; k < L::KV; ++k) {
        const typename H::T hk = H::from(kv_value<D>(bh, bl, k, false));
        hv[k] = *reinterpret_cast<const uint16_t*>(&hk);
      }
#pragma unroll
      for (int w = 0; w < L::KV / 2; ++w)
        kv[j * L::KV_STRIDE_W + w] = (uint32_t)hv[2 * w] | ((uint32_t)hv[2 * w + 1] << 16);
    }
    // weights: column c of the tile as halves at qq[c*QSTRIDE_W*2 + j]
    uint16_t* qh = reinterpret_cast<uint16_t*>(qq);
    uint16_t* ql = qh + MC * QSTRIDE_W * 2;
    for (int e = tid; e < MC * TS; e += nthreads) {
      const int c = e / TS, j = e % TS;
      const float v = c < p.m ? rs[(D + c) * TS + j] : 0.f;
      const typename H::T h = H::from(v);
      qh[c * QSTRIDE_W * 2 + j] = *reinterpret_cast<const uint16_t*>(&h);
      if (SPLIT) {
        const typename H::T l = H::from(v - H::to(h));
        ql[c * QSTRIDE_W * 2 + j] = *reinterpret_cast<const uint16_t*>(&l);
      }
    }
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
  if (nt > 0) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[0], 0));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    }
    __syncthreads();
    if (!abort_flag) transform(0, 0);
    __syncthreads();
  }

  for (int r = 0; r < nt && !abort_flag; ++r) {
    // raw stage r % RS was consumed by transform(r); refill it with tile r + RS
    if (tid == 0 && r + RS < nt) {
      fence_proxy_async_smem();
      issue(r + RS);
      ++issued;
    }
    if (r + 1 < nt) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[(r + 1) % RS], ((r + 1) / RS) & 1));
      if (!ok) {
        abort_flag = 1;
        if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
      } else {
        transform(r + 1, (r + 1) & 1);
      }
    }
    const uint32_t* kv = kvb + (r & 1) * TS * L::KV_STRIDE_W;
    const uint32_t* qh = qb + (r & 1) * QBUF_W;
    const uint32_t* ql = qh + MC * QSTRIDE_W;
#pragma unroll 1
    for (int kk = 0; kk < TS / 16; ++kk) {
      // exponent operand B' for the two 8-source halves of this 16-source step
      uint32_t bfr[2][L::KSTEPS][2];
#pragma unroll
      for (int nt2 = 0; nt2 < 2; ++nt2) {
        const int j = kk * 16 + nt2 * 8 + g;
#pragma unroll
        for (int ks = 0; ks < L::KSTEPS; ++ks) {
          bfr[nt2][ks][0] = kv[j * L::KV_STRIDE_W + 8 * ks + t];
          bfr[nt2][ks][1] = kv[j * L::KV_STRIDE_W + 8 * ks + t + 4];
        }
      }
      // weights operand for each group of 8 right-hand sides
      uint32_t qfh[NRT][2], qfl[NRT][2];
#pragma unroll
      for (int rt = 0; rt < NRT; ++rt) {
        const int c = rt * 8 + g;
        qfh[rt][0] = qh[c * QSTRIDE_W + kk * 8 + t];
        qfh[rt][1] = qh[c * QSTRIDE_W + kk * 8 + t + 4];
        if (SPLIT) {
          qfl[rt][0] = ql[c * QSTRIDE_W + kk * 8 + t];
          qfl[rt][1] = ql[c * QSTRIDE_W + kk * 8 + t + 4];
        }
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        float e0[4] = {0.f, 0.f, 0.f, 0.f}, e1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int ks = 0; ks < L::KSTEPS; ++ks) {
          mma16816<BF>(e0, afr[mt][ks], bfr[0][ks][0], bfr[0][ks][1]);
          mma16816<BF>(e1, afr[mt][ks], bfr[1][ks][0], bfr[1][ks][1]);
        }
        // P = 2^E; accumulator layout (rows g, g+8; cols 2t, 2t+1) of the two
        // 8-source halves is the A-operand layout of the 16-source step
        float pv[8];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          pv[e] = ex2(e0[e]);
          pv[4 + e] = ex2(e1[e]);
        }
        uint32_t ph[4];
        ph[0] = H::pack(pv[0], pv[1]);
        ph[1] = H::pack(pv[2], pv[3]);
        ph[2] = H::pack(pv[4], pv[5]);
        ph[3] = H::pack(pv[6], pv[7]);
        uint32_t pl[4];
        if (SPLIT) {
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const float2 hv = H::unpack(ph[w]);
            pl[w] = H::pack(pv[2 * w] - hv.x, pv[2 * w + 1] - hv.y);
          }
        }
#pragma unroll
        for (int rt = 0; rt < NRT; ++rt) {
          mma16816<BF>(acc[mt][rt], ph, qfh[rt][0], qfh[rt][1]);
          if (SPLIT) {
            mma16816<BF>(acc[mt][rt], pl, qfh[rt][0], qfh[rt][1]);
            mma16816<BF>(acc[mt][rt], ph, qfl[rt][0], qfl[rt][1]);
          }
        }
      }
    }
    // fold the tile's sums into compensated float32 accumulators
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int rt = 0; rt < NRT; ++rt)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          kahan_add(S[mt][rt][e], C[mt][rt][e], acc[mt][rt][e]);
          acc[mt][rt][e] = 0.f;
        }
    __syncthreads();
  }
  if (abort_flag) {
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % RS], (r / RS) & 1);
    __syncthreads();
    return;
  }

  // ---- partials: rows g, g+8 of each m-tile, columns 2t, 2t+1 of each group
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t i = row0 + mt * 16 + g + 8 * half;
      if (i >= p.Nt_pad) continue;
#pragma unroll
      for (int rt = 0; rt < NRT; ++rt)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc) {
          const int c = rt * 8 + 2 * t + cc;
          if (c >= p.m) continue;
          const int e = 2 * half + cc;
          p.part[((int64_t)blockIdx.y * p.m + c) * p.Nt_pad + i] =
              (double)S[mt][rt][e] - (double)C[mt][rt][e];
        }
    }
}

// ------------------------------------------------------------------------
// Single-column float32-grade product: the exponent contraction E = A' B'^T
// on the tensor cores (split f16 operands as above), then per pair one
// MUFU.EX2 straight from the accumulator register and one float32 FMA with
// the source weight, so the CUDA cores carry 1 EX2 + 1 FMA per pair and the
// special-function unit is the only pipe near its limit (the all-CUDA-core
// product needs d + 1 FP32 operations per pair as well, which at d = 3 loads
// the FP32 pipe as fully as the EX2 loads MUFU).  One CTA per expanded-form
// super-block, MT m-tiles of 16 targets per warp; a thread accumulates the
// rows g and g+8 of each m-tile over its columns 2t, 2t+1 and the four
// threads of a row are summed at the end.
template <int D, int MT>
__global__ void __launch_bounds__(32 * (SB / (16 * MT))) mvp_tcx_kernel(const TcParams p) {
  using L = ExpLayout<D>;
  using H = Half<false>;
  constexpr int W = D + 1;
  constexpr int RAW = (D + 1) * TS;  // coordinates, weights
  extern __shared__ __align__(128) float smem[];
  const int nthreads = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  __shared__ __align__(8) uint64_t bars[RS];
  __shared__ volatile int abort_flag;
  if (p.active && *p.active == 0) return;
  const int64_t nexp = *p.tn_exp;
  if ((int64_t)blockIdx.x >= nexp) return;

  float* raw = smem;                                                   // RS stages
  uint32_t* kvb = reinterpret_cast<uint32_t*>(smem + RS * RAW);          // 2 x TS x KV_STRIDE_W
  float* qbuf = reinterpret_cast<float*>(kvb + 2 * TS * L::KV_STRIDE_W);  // 2 x TS weights

  const int64_t blk = p.torder[blockIdx.x];
  if (blk * SB < p.row_lo || blk * SB >= p.row_hi) return;  // outside the shard
  float ctr[D];
#pragma unroll
  for (int k = 0; k < D; ++k) ctr[k] = p.tctr[blk * D + k];

  uint32_t afr[MT][L::KSTEPS][4];
  const int64_t row0 = blk * p.WB + (int64_t)warp * 16 * MT;
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
#pragma unroll
    for (int half = 0; half < 2; ++half) {
      const int64_t i = row0 + mt * 16 + g + 8 * half;
      const int64_t ii = i < p.Nt ? i : p.Nt - 1;
      float ah[W], al[W];
      float r2 = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float x = p.xt[(ii / TS) * (int64_t)D * TS + (int64_t)k * TS + ii % TS];
        const float xh = p.s * (x - ctr[k]);
        r2 = fmaf(xh, xh, r2);
        ah[k] = H::to(H::from(xh));
        al[k] = xh - ah[k];
      }
      ah[D] = 1.f;
      al[D] = 0.f;
      if (blockIdx.y == 0 && t == 0 && i < p.Nt_pad) p.fac[i] = exp2f(-r2);
#pragma unroll
      for (int ks = 0; ks < L::KSTEPS; ++ks) {
        const int k0 = 16 * ks + 2 * t;
        afr[mt][ks][half] = H::pack(kv_value<D>(ah, al, k0, true), kv_value<D>(ah, al, k0 + 1, true));
        afr[mt][ks][half + 2] =
            H::pack(kv_value<D>(ah, al, k0 + 8, true), kv_value<D>(ah, al, k0 + 9, true));
      }
    }
  }

  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;
  float2 acc[MT][2], acc2[MT][2];
  float S[MT][2], C[MT][2];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      acc[mt][h] = acc2[mt][h] = make_float2(0.f, 0.f);
      S[mt][h] = C[mt][h] = 0.f;
    }

  auto issue = [&](int r) {
    const int stage = r % RS;
    const int64_t tile = t_begin + r;
    float* dst = raw + stage * RAW;
    mbar_arrive_expect_tx(&bars[stage], (uint32_t)RAW * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    bulk_g2s(dst + D * TS, p.Q + tile * (int64_t)TS, TS * 4, &bars[stage]);
  };
  // CTA-wide transform of raw tile r into buffer b: the split source
  // K-vectors, and the float32 weights (the raw stage is refilled while the
  // tile is still being used)
  auto transform = [&](int r, int b) {
    const float* rs = raw + (r % RS) * RAW;
    uint32_t* kv = kvb + b * TS * L::KV_STRIDE_W;
    for (int j = tid; j < TS; j += nthreads) {
      float bh[W], bl[W];
      float bb = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float xh = p.s * (rs[k * TS + j] - ctr[k]);
        bb = fmaf(-xh, xh, bb);
        const float v = 2.f * xh;
        bh[k] = H::to(H::from(v));
        bl[k] = v - bh[k];
      }
      if (bb < -30000.f) {  // farther than any target can see: contributes 0
#pragma unroll
        for (int k = 0; k < D; ++k) bh[k] = bl[k] = 0.f;
        bb = -30000.f;
      }
      bh[D] = H::to(H::from(bb));
      bl[D] = bb - bh[D];
      uint16_t hv[L::KV];
#pragma unroll
      for (int k = 0; k < L::KV; ++k) {
        const typename H::T hk = H::from(kv_value<D>(bh, bl, k, false));
        hv[k] = *reinterpret_cast<const uint16_t*>(&hk);
      }
#pragma unroll
      for (int w = 0; w < L::KV / 2; ++w)
        kv[j * L::KV_STRIDE_W + w] = (uint32_t)hv[2 * w] | ((uint32_t)hv[2 * w + 1] << 16);
      qbuf[b * TS + j] = rs[D * TS + j];
    }
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
  if (nt > 0) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[0], 0));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    }
    __syncthreads();
    if (!abort_flag) transform(0, 0);
    __syncthreads();
  }

  for (int r = 0; r < nt && !abort_flag; ++r) {
    if (tid == 0 && r + RS < nt) {
      fence_proxy_async_smem();
      issue(r + RS);
      ++issued;
    }
    if (r + 1 < nt) {
      const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[(r + 1) % RS], ((r + 1) / RS) & 1));
      if (!ok) {
        abort_flag = 1;
        if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
      } else {
        transform(r + 1, (r + 1) & 1);
      }
    }
    const uint32_t* kv = kvb + (r & 1) * TS * L::KV_STRIDE_W;
    const float* qv = qbuf + (r & 1) * TS;
#pragma unroll 1
    for (int kk = 0; kk < TS / 16; ++kk) {
      uint32_t bfr[2][L::KSTEPS][2];
#pragma unroll
      for (int nt2 = 0; nt2 < 2; ++nt2) {
        const int j = kk * 16 + nt2 * 8 + g;
#pragma unroll
        for (int ks = 0; ks < L::KSTEPS; ++ks) {
          bfr[nt2][ks][0] = kv[j * L::KV_STRIDE_W + 8 * ks + t];
          bfr[nt2][ks][1] = kv[j * L::KV_STRIDE_W + 8 * ks + t + 4];
        }
      }
      // weights of this thread's accumulator columns: sources 2t, 2t+1 of
      // each 8-source half
      const float2 q0 = *reinterpret_cast<const float2*>(qv + kk * 16 + 2 * t);
      const float2 q1 = *reinterpret_cast<const float2*>(qv + kk * 16 + 8 + 2 * t);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        float e0[4], e1[4];
        mma16816_z(e0, afr[mt][0], bfr[0][0][0], bfr[0][0][1]);
        mma16816_z(e1, afr[mt][0], bfr[1][0][0], bfr[1][0][1]);
#pragma unroll
        for (int ks = 1; ks < L::KSTEPS; ++ks) {
          mma16816<false>(e0, afr[mt][ks], bfr[0][ks][0], bfr[0][ks][1]);
          mma16816<false>(e1, afr[mt][ks], bfr[1][ks][0], bfr[1][ks][1]);
        }
        // rows g (elements 0, 1) and g+8 (elements 2, 3): the two columns of
        // a row and 8-source half share one packed FMA
        acc[mt][0] = ffma2(q0, make_float2(ex2(e0[0]), ex2(e0[1])), acc[mt][0]);
        acc2[mt][0] = ffma2(q1, make_float2(ex2(e1[0]), ex2(e1[1])), acc2[mt][0]);
        acc[mt][1] = ffma2(q0, make_float2(ex2(e0[2]), ex2(e0[3])), acc[mt][1]);
        acc2[mt][1] = ffma2(q1, make_float2(ex2(e1[2]), ex2(e1[3])), acc2[mt][1]);
      }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        kahan_add(S[mt][h], C[mt][h], (acc[mt][h].x + acc[mt][h].y) + (acc2[mt][h].x + acc2[mt][h].y));
        acc[mt][h] = acc2[mt][h] = make_float2(0.f, 0.f);
      }
    __syncthreads();
  }
  if (abort_flag) {
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % RS], (r / RS) & 1);
    __syncthreads();
    return;
  }
  // the four threads of a row hold its sums over columns 2t, 2t+1
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double v = (double)S[mt][h] - (double)C[mt][h];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      const int64_t i = row0 + mt * 16 + g + 8 * h;
      if (t == 0 && i < p.Nt_pad) p.part[(int64_t)blockIdx.y * p.Nt_pad + i] = v;
    }
}

// ------------------------------------------------------------------------
// High-dimensional single-column product (d = 16, 32, 48, 64: coordinates
// zero-padded), where the cross term -2 x^_i . x^_j is a real contraction:
// per pair 3 (d + 1) split-f16 products on the tensor cores instead of 2d + 2
// float32 operations on the CUDA cores.  Same factored form as
// mvp_tcx_kernel (compact super-blocks only: |x^_i - c|^2 <= 8 in scaled
// units bounds the cancellation error of the expanded form, whatever d):
//   E_ij = A_i . B_j, A_i = [u_i, 1], B_j = [2 v_j, -|v_j|^2], u, v = x^ - c,
// split three ways (A' = [Ah, Ah, Al], B' = [Bh, Bl, Bh]).
// Differences from the low-d kernel:
//  * the K-vectors are long (4 to 13 contraction steps), so the A fragments
//    of a warp cover MT = 2 m-tiles (d <= 32) or 1 (d >= 48), and the CTA has
//    SB / (16 MT) warps;
//  * targets and sources are written to shared memory as K-vector rows one
//    component at a time (three 16-bit stores each), without per-slot
//    selects; the target rows are read back once into the A fragments;
//  * one K-vector buffer (the d = 64 tile is 108 KB): a tile is transformed
//    from its raw stage between two barriers, and the raw stages (TMA bulk
//    copies) keep loading while the tensor cores work.
template <int D>
struct HighD {
  static constexpr int W = D + 1;
  static constexpr int KSTEPS = (3 * W + 15) / 16;
  static constexpr int STRIDE = 8 * KSTEPS + 4;    // words per K-vector row (fragment loads conflict-free)
  static constexpr int MT = KSTEPS <= 7 ? 2 : 1;   // m-tiles per warp
  static constexpr int WARPS = SB / (16 * MT);
  static constexpr int RSD = D <= 32 ? 2 : 1;      // raw source stages
};

template <int D>
constexpr size_t tch_smem_bytes() {
  using L = HighD<D>;
  return sizeof(float) * (L::RSD * (D + 1) * TS + TS) + sizeof(uint32_t) * TS * L::STRIDE;
}

template <int D>
__global__ void __launch_bounds__(32 * HighD<D>::WARPS) mvp_tch_kernel(const TcParams p) {
  using L = HighD<D>;
  using H = Half<false>;
  constexpr int W = D + 1, MT = L::MT, RSD = L::RSD, KS = L::KSTEPS, ST = L::STRIDE;
  constexpr int RAW = (D + 1) * TS;  // coordinates, weights
  extern __shared__ __align__(128) float smem[];
  float* raw = smem;                                       // RSD stages
  float* qbuf = smem + RSD * RAW;                          // TS weights
  uint32_t* kv = reinterpret_cast<uint32_t*>(qbuf + TS);   // TS rows x ST words
  const int nthreads = blockDim.x;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  __shared__ __align__(8) uint64_t bars[RSD];
  __shared__ volatile int abort_flag;
  __shared__ float ctr[D];
  if (p.active && *p.active == 0) return;
  const int64_t nexp = *p.tn_exp;
  if ((int64_t)blockIdx.x >= nexp) return;
  const int64_t blk = p.torder[blockIdx.x];
  if (blk * SB < p.row_lo || blk * SB >= p.row_hi) return;  // outside the shard
  const int64_t row0 = blk * p.WB;
  for (int k = tid; k < D; k += nthreads) ctr[k] = p.tctr[blk * D + k];
  for (int w = tid; w < TS * ST; w += nthreads) kv[w] = 0u;  // padding slots stay zero
  __syncthreads();

  // ---- target K-vectors A' = [uh, uh, ul] over [u, 1], then the A fragments
  for (int r = tid; r < SB; r += nthreads) {
    const int64_t i = row0 + r;
    const int64_t ii = i < p.Nt ? i : p.Nt - 1;
    uint16_t* row = reinterpret_cast<uint16_t*>(kv + r * ST);
    float r2 = 0.f;
#pragma unroll 4
    for (int k = 0; k < D; ++k) {
      const float u = p.s * (p.xt[(ii / TS) * (int64_t)D * TS + (int64_t)k * TS + ii % TS] - ctr[k]);
      r2 = fmaf(u, u, r2);
      const typename H::T uh = H::from(u);
      const typename H::T ul = H::from(u - H::to(uh));
      row[k] = *reinterpret_cast<const uint16_t*>(&uh);
      row[W + k] = *reinterpret_cast<const uint16_t*>(&uh);
      row[2 * W + k] = *reinterpret_cast<const uint16_t*>(&ul);
    }
    const typename H::T one = H::from(1.f), zero = H::from(0.f);
    row[D] = *reinterpret_cast<const uint16_t*>(&one);
    row[W + D] = *reinterpret_cast<const uint16_t*>(&one);
    row[2 * W + D] = *reinterpret_cast<const uint16_t*>(&zero);
    if (blockIdx.y == 0 && i < p.Nt_pad) p.fac[i] = exp2f(-r2);
  }
  __syncthreads();
  uint32_t afr[MT][KS][4];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt) {
    const int ra = (warp * MT + mt) * 16 + g, rb = ra + 8;
#pragma unroll
    for (int ks = 0; ks < KS; ++ks) {
      afr[mt][ks][0] = kv[ra * ST + 8 * ks + t];
      afr[mt][ks][1] = kv[rb * ST + 8 * ks + t];
      afr[mt][ks][2] = kv[ra * ST + 8 * ks + t + 4];
      afr[mt][ks][3] = kv[rb * ST + 8 * ks + t + 4];
    }
  }

  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;
  float2 acc[MT][2], acc2[MT][2];
  float S[MT][2], C[MT][2];
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      acc[mt][h] = acc2[mt][h] = make_float2(0.f, 0.f);
      S[mt][h] = C[mt][h] = 0.f;
    }

  auto issue = [&](int r) {
    const int stage = r % RSD;
    const int64_t tile = t_begin + r;
    float* dst = raw + stage * RAW;
    mbar_arrive_expect_tx(&bars[stage], (uint32_t)RAW * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    bulk_g2s(dst + D * TS, p.Q + tile * (int64_t)TS, TS * 4, &bars[stage]);
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < RSD; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();  // also: every warp holds its A fragments before kv is reused
  int issued = 0;
  if (tid == 0)
    for (; issued < min(RSD, nt); ++issued) issue(issued);

  for (int r = 0; r < nt; ++r) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[r % RSD], (r / RSD) & 1));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    }
    __syncthreads();  // the previous tile's products are done with kv
    if (abort_flag) break;
    // ---- source K-vectors B' = [Bh, Bl, Bh] over [2 v, -|v|^2] and weights
    const float* rs = raw + (r % RSD) * RAW;
    // with 2 TS threads, the two threads of a source write half of its
    // components each (both form |v|^2)
    const int parts = nthreads >= 2 * TS ? 2 : 1;
    const int part = parts == 2 ? tid / TS : 0;
    const int k_lo = part * (D / parts), k_hi = k_lo + D / parts;
    for (int j = parts == 2 ? tid % TS : tid; j < TS; j += (parts == 2 ? TS : nthreads)) {
      float bb = 0.f;
#pragma unroll 8
      for (int k = 0; k < D; ++k) {
        const float v = p.s * (rs[k * TS + j] - ctr[k]);
        bb = fmaf(-v, v, bb);
      }
      const bool far = bb < -30000.f;  // farther than any target can see: contributes 0
      uint16_t* row = reinterpret_cast<uint16_t*>(kv + j * ST);
#pragma unroll 4
      for (int k = k_lo; k < k_hi; ++k) {
        const float v = far ? 0.f : 2.f * p.s * (rs[k * TS + j] - ctr[k]);
        const typename H::T vh = H::from(v);
        const typename H::T vl = H::from(v - H::to(vh));
        row[k] = *reinterpret_cast<const uint16_t*>(&vh);
        row[W + k] = *reinterpret_cast<const uint16_t*>(&vl);
        row[2 * W + k] = *reinterpret_cast<const uint16_t*>(&vh);
      }
      if (part == parts - 1) {
        const float b = far ? -30000.f : bb;
        const typename H::T bh = H::from(b);
        const typename H::T bl = H::from(b - H::to(bh));
        row[D] = *reinterpret_cast<const uint16_t*>(&bh);
        row[W + D] = *reinterpret_cast<const uint16_t*>(&bl);
        row[2 * W + D] = *reinterpret_cast<const uint16_t*>(&bh);
        qbuf[j] = rs[D * TS + j];
      }
    }
    __syncthreads();  // kv ready; the raw stage may be refilled
    if (tid == 0 && r + RSD < nt) {
      fence_proxy_async_smem();
      issue(r + RSD);
      ++issued;
    }
#pragma unroll 1
    for (int kk = 0; kk < TS / 16; ++kk) {
      const int j0 = kk * 16 + g, j1 = j0 + 8;
      // even and odd contraction steps accumulate separately (twice the
      // independent MMA chains), summed before the exponential
      float e0[MT][4], e1[MT][4], o0[MT][4], o1[MT][4];
#pragma unroll
      for (int ks = 0; ks < KS; ++ks) {
        const uint32_t b00 = kv[j0 * ST + 8 * ks + t], b01 = kv[j0 * ST + 8 * ks + t + 4];
        const uint32_t b10 = kv[j1 * ST + 8 * ks + t], b11 = kv[j1 * ST + 8 * ks + t + 4];
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          if (ks == 0) {
            mma16816_z(e0[mt], afr[mt][0], b00, b01);
            mma16816_z(e1[mt], afr[mt][0], b10, b11);
          } else if (ks == 1) {
            mma16816_z(o0[mt], afr[mt][1], b00, b01);
            mma16816_z(o1[mt], afr[mt][1], b10, b11);
          } else if (ks & 1) {
            mma16816<false>(o0[mt], afr[mt][ks], b00, b01);
            mma16816<false>(o1[mt], afr[mt][ks], b10, b11);
          } else {
            mma16816<false>(e0[mt], afr[mt][ks], b00, b01);
            mma16816<false>(e1[mt], afr[mt][ks], b10, b11);
          }
        }
      }
#pragma unroll
      for (int mt = 0; mt < MT; ++mt)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          e0[mt][v] += o0[mt][v];
          e1[mt][v] += o1[mt][v];
        }
      const float2 q0 = *reinterpret_cast<const float2*>(qbuf + kk * 16 + 2 * t);
      const float2 q1 = *reinterpret_cast<const float2*>(qbuf + kk * 16 + 8 + 2 * t);
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        acc[mt][0] = ffma2(q0, make_float2(ex2(e0[mt][0]), ex2(e0[mt][1])), acc[mt][0]);
        acc2[mt][0] = ffma2(q1, make_float2(ex2(e1[mt][0]), ex2(e1[mt][1])), acc2[mt][0]);
        acc[mt][1] = ffma2(q0, make_float2(ex2(e0[mt][2]), ex2(e0[mt][3])), acc[mt][1]);
        acc2[mt][1] = ffma2(q1, make_float2(ex2(e1[mt][2]), ex2(e1[mt][3])), acc2[mt][1]);
      }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        kahan_add(S[mt][h], C[mt][h], (acc[mt][h].x + acc[mt][h].y) + (acc2[mt][h].x + acc2[mt][h].y));
        acc[mt][h] = acc2[mt][h] = make_float2(0.f, 0.f);
      }
  }
  if (abort_flag) {
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % RSD], (r / RSD) & 1);
    __syncthreads();
    return;
  }
#pragma unroll
  for (int mt = 0; mt < MT; ++mt)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      double v = (double)S[mt][h] - (double)C[mt][h];
      v += __shfl_xor_sync(0xffffffffu, v, 1);
      v += __shfl_xor_sync(0xffffffffu, v, 2);
      const int64_t i = row0 + (warp * MT + mt) * 16 + g + 8 * h;
      if (t == 0 && i < p.Nt_pad) p.part[(int64_t)blockIdx.y * p.Nt_pad + i] = v;
    }
}

// ------------------------------------------------------------------------
// Multi-column product on the 5th-generation tensor cores (tcgen05, TMEM
// accumulators): the same two contractions as mvp_tc_kernel, with the
// operands where the tcgen05 datapath wants them.
//
// One CTA = 128 targets (half of an expanded-form super-block) = the 128
// TMEM lanes, 9 warps: warp 8 issues the MMAs (one elected thread); warps 0-3
// and 4-7 form two chunk groups, each covering the 128 lanes (warp w serves
// lanes 32 (w % 4) .. + 31), that take alternate chunks of 64 sources.  Per
// source tile (256 sources) the groups build the f16 K-major source operand B
// in shared memory (half each), the weight columns Q arrive pre-split (hi,
// lo) by bulk copies, and for each chunk:
//   1. the elected thread issues S = A B^T (M = 128, N = 64, K = 16 per
//      instruction) into one of three TMEM buffers (fp32), two chunks ahead
//      of the P Q in hand, so the tensor cores work while the threads
//      exponentiate;
//   2. the chunk's group reads S (tcgen05.ld, 32 columns at a time), forms
//      P = 2^S with MUFU.EX2 and writes P as f16 (hi, and lo when split) over
//      the same TMEM columns (tcgen05.st); the other group meanwhile works on
//      its own chunk;
//   3. the elected thread issues Y += P Q with P read from TMEM (M = 128,
//      N = 16, K = 16 per instruction: Ph Qh + Pl Qh + Ph Ql when split).
// Each S buffer has its own mbarriers (a commit per chunk, the group's
// arrivals), Y its own; every barrier phase is awaited before the barrier can
// complete again.  Y lives in TMEM for a tile (two buffers by tile parity)
// and is folded into float32 Kahan sums one tile later, after which the
// tile's TMA stage (three stages) is refilled.  Shared operands use the
// canonical no-swizzle K-major layout: 8-row x 16-byte core matrices,
// adjacent along K 128 bytes apart (leading byte offset), 8-row groups
// KC*128 bytes apart (stride byte offset).
namespace umma {

constexpr int ROWS = 128;       // targets per CTA (MMA M)
constexpr int THREADS = 256;    // two warpgroups
constexpr int NC = 64;          // sources per chunk (N of the exponent MMA)
constexpr int NBUF = 3;         // S/P buffers of NC columns
constexpr int YN = 16;          // Y columns (N of the P Q MMA)
constexpr int TMEM_COLS = 256;  // S/P buffers at 0, 64, 128; Y buffers at 192, 208
constexpr int SMEM_FLOOR = 80 * 1024;  // at most two CTAs per SM (TMEM holds two)
constexpr int URS = 3;          // raw TMA stages (a tile's stage is refilled one tile after use)
constexpr int GROUP_WARPS = 4;  // compute warps per chunk group (all 128 TMEM lanes)

__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo) {
  return ((uint64_t)((saddr >> 4) & 0x3FFF)) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

// kind::f16 instruction descriptor: D f32, A/B f16 (bf = 0) or bf16 (1),
// both K-major, N and M as given.
__host__ __device__ constexpr uint32_t idesc(int bf, int n, int m) {
  return (1u << 4) | ((uint32_t)bf << 7) | ((uint32_t)bf << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t id, int acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}"
               :: "r"(d), "l"(a), "l"(b), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a_tmem, uint64_t b, uint32_t id, int acc) {
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}"
               :: "r"(d), "r"(a_tmem), "l"(b), "r"(id), "r"(acc) : "memory");
}

__device__ __forceinline__ void commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

__device__ __forceinline__ void ld8(uint32_t taddr, uint32_t (&v)[8]) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
               : "r"(taddr));
}

__device__ __forceinline__ void st16(uint32_t taddr, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
      :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
         "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}

__device__ __forceinline__ void wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

// Byte offset of element (row, k) in a K-major no-swizzle tile with kc
// k-chunks of 8 elements per 8-row group.
__device__ __forceinline__ uint32_t kmaj(int row, int k, int kc) {
  return (uint32_t)((((row >> 3) * kc + (k >> 3)) << 7) + ((row & 7) << 4) + ((k & 7) << 1));
}

// A stage: the tile's raw coordinates (D x 1 KB) and its weight tiles (hi,
// and lo when split: 8 KB each, read by the MMAs straight from the stage).
template <int D>
constexpr uint32_t stage_bytes(bool split) {
  return (uint32_t)(sizeof(float) * D * TS + 2 * YN * TS * (split ? 2 : 1));
}

template <int D>
constexpr size_t smem_bytes(bool split) {
  using L = ExpLayout<D>;
  const size_t need = URS * (size_t)stage_bytes<D>(split) + 2 * ROWS * L::KV + 2 * (2 * TS * L::KV);
  return need > SMEM_FLOOR ? need : SMEM_FLOOR;
}

}  // namespace umma

__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.release.cta.shared::cta.b64 _, [%0];" :: "r"(smem_addr(bar)) : "memory");
}

template <int D, bool SPLIT, bool BF>
__global__ void __launch_bounds__(umma::THREADS + 32) mvp_umma_kernel(const TcParams p) {
  using namespace umma;
  using L = ExpLayout<D>;
  using H = Half<BF>;
  constexpr int W = D + 1;
  constexpr int KC = L::KV / 8;      // k-chunks of a K-vector
  constexpr int QKC = TS / 8;        // k-chunks of a weight row (one tile)
  constexpr int NCW = THREADS / 32;  // compute warps (warp NCW issues the MMAs)
  constexpr int CPT = TS / NC;       // chunks per tile
  constexpr int AHEAD = NBUF - 1;    // exponent MMAs issued ahead of the P Q in hand
  constexpr uint32_t BBYTES = 2 * TS * L::KV;  // one B operand buffer
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[URS];       // TMA stages
  __shared__ __align__(8) uint64_t sfull[NBUF];     // S of buffer b complete (commit)
  __shared__ __align__(8) uint64_t pfull[NBUF];     // P of buffer b written (one chunk group)
  __shared__ __align__(8) uint64_t pdone[NBUF];     // P Q reading buffer b complete (commit)
  __shared__ __align__(8) uint64_t bready[2];       // B operand buffer written (compute warps)
  __shared__ __align__(8) uint64_t yfull[2];        // Y buffer complete for its tile (commit)
  __shared__ __align__(8) uint64_t yfree[2];        // Y buffer read (compute warps)
  __shared__ __align__(8) uint64_t dbar;            // after an abort: the MMAs issued are complete
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool mma_warp = warp == NCW;
  const int grp = (warp >> 2) & 1;  // chunk group of a compute warp: chunks c with c % 2 == grp
  if (p.active && *p.active == 0) return;
  const int64_t nexp = *p.tn_exp;
  const int64_t sb_slot = blockIdx.x >> 1;
  if (sb_slot >= nexp) return;
  constexpr uint32_t SBYTES = stage_bytes<D>(SPLIT);
  constexpr uint32_t QTILE = 2 * YN * TS;  // bytes of one weight tile
  unsigned char* stages = smem_raw;        // URS stages: coordinates, Qh, Ql
  unsigned char* sA = smem_raw + URS * SBYTES;
  unsigned char* sB = sA + 2 * ROWS * L::KV;  // two B buffers

  const int64_t blk = p.torder[sb_slot];
  if (blk * SB < p.row_lo || blk * SB >= p.row_hi) return;  // outside the shard
  float ctr[D];
#pragma unroll
  for (int k = 0; k < D; ++k) ctr[k] = p.tctr[blk * D + k];
  const int row = 32 * (warp & 3) + lane;                                  // TMEM lane of a compute thread
  const int64_t i = blk * SB + (int64_t)(blockIdx.x & 1) * ROWS + row;  // and its target

  // ---- operand A (first compute warpgroup): the row's split K-vector [x^, 1]
  if (warp < 4) {
    const int64_t ii = i < p.Nt ? i : p.Nt - 1;
    float ah[W], al[W];
    float r2 = 0.f;
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float x = p.xt[(ii / TS) * (int64_t)D * TS + (int64_t)k * TS + ii % TS];
      const float xh = p.s * (x - ctr[k]);
      r2 = fmaf(xh, xh, r2);
      ah[k] = H::to(H::from(xh));
      al[k] = xh - ah[k];
    }
    ah[D] = 1.f;
    al[D] = 0.f;
    if (blockIdx.y == 0 && i < p.Nt_pad) p.fac[i] = exp2f(-r2);
#pragma unroll
    for (int kc = 0; kc < KC; ++kc) {
      uint32_t w[4];
#pragma unroll
      for (int e = 0; e < 4; ++e)
        w[e] = H::pack(kv_value<D>(ah, al, 8 * kc + 2 * e, true), kv_value<D>(ah, al, 8 * kc + 2 * e + 1, true));
      *reinterpret_cast<uint4*>(sA + kmaj(row, 8 * kc, KC)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < URS; ++st) mbar_init(&bars[st], 1);
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&sfull[b], 1);
      mbar_init(&pfull[b], GROUP_WARPS);
      mbar_init(&pdone[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bready[b], NCW);
      mbar_init(&yfull[b], 1);
      mbar_init(&yfree[b], NCW);
    }
    mbar_init(&dbar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async_smem();
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  const uint32_t y_col = NBUF * NC;  // Y buffers at y_col and y_col + YN
  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;

  auto issue = [&](int r) {
    const int stage = r % URS;
    const int64_t tile = t_begin + r;
    unsigned char* dst = stages + stage * SBYTES;
    mbar_arrive_expect_tx(&bars[stage], SBYTES);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    bulk_g2s(dst + D * TS * 4, p.qh_tiles + tile * (int64_t)(YN * TS), QTILE, &bars[stage]);
    if (SPLIT) bulk_g2s(dst + D * TS * 4 + QTILE, p.ql_tiles + tile * (int64_t)(YN * TS), QTILE, &bars[stage]);
  };
  // a bounded wait that also gives up once the other role has aborted
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
      if (abort_flag || clock64() - t0 > WAIT_LIMIT_CLOCKS) return false;
    }
    return true;
  };

  int issued = 0;
  if (mma_warp) {
    // ================= MMA warp: one thread issues every tcgen05.mma, as a
    // stream of chunks: the exponent MMAs run AHEAD chunks in front of the
    // P Q in hand, across tile boundaries
    if (lane == 0) {
      const uint32_t id_s = idesc(BF ? 1 : 0, NC, ROWS);
      const uint32_t id_y = idesc(BF ? 1 : 0, YN, ROWS);
      const uint32_t a_addr = smem_addr(sA), b_addr = smem_addr(sB);
      uint32_t n_pd[NBUF] = {0, 0, 0}, w_pd[NBUF] = {0, 0, 0};  // pdone commits issued / awaited
      uint32_t n_pf[NBUF] = {0, 0, 0};                            // pfull phases awaited
      uint32_t n_br[2] = {0, 0}, n_yf[2] = {0, 0};                // bready / yfree phases awaited
      const int total = nt * CPT;
      int next_s = 0;
      bool ok = true;
      for (int c = 0; c < total && ok; ++c) {
        while (ok && next_s < total && next_s <= c + AHEAD) {
          const int r = next_s / CPT, q = next_s % CPT, b = next_s % NBUF, bb = r & 1;
          if (q == 0) {  // the tile's B operand: waited for only when this S is
                         // needed now, else the P Q in hand goes first
            if (next_s > c && !mbar_try_wait(&bready[bb], n_br[bb] & 1)) break;
            ok = wait(&bready[bb], n_br[bb] & 1);
            ++n_br[bb];
          }
          if (ok && n_pd[b] != w_pd[b]) {  // the last P Q that read buffer b
            ok = wait(&pdone[b], w_pd[b] & 1);
            ++w_pd[b];
          }
          if (!ok) break;
          fence_after();
#pragma unroll
          for (int ks = 0; ks < L::KSTEPS; ++ks)
            mma_ss(tmem + (uint32_t)(b * NC), sdesc(a_addr + 256u * ks, KC * 128),
                   sdesc(b_addr + (uint32_t)bb * BBYTES + (uint32_t)(8 * q * KC * 128) + 256u * ks, KC * 128),
                   id_s, ks > 0);
          commit(&sfull[b]);
          ++next_s;
        }
        if (!ok) break;
        const int r = c / CPT, q = c % CPT, b = c % NBUF, yb = r & 1;
        ok = wait(&pfull[b], n_pf[b] & 1);
        ++n_pf[b];
        if (ok && q == 0 && r >= 2) {  // Y buffer yb was read for tile r - 2
          ok = wait(&yfree[yb], n_yf[yb] & 1);
          ++n_yf[yb];
        }
        if (!ok) break;
        fence_after();
        const uint32_t qh_addr = smem_addr(stages + (r % URS) * SBYTES + D * TS * 4);
        const uint32_t ql_addr = qh_addr + QTILE;
        const uint32_t sbuf = tmem + (uint32_t)(b * NC);
        const uint32_t yd = tmem + y_col + (uint32_t)(YN * yb);
#pragma unroll
        for (int ks = 0; ks < NC / 16; ++ks) {
          const uint32_t qoff = (uint32_t)((NC / 8) * q + 2 * ks) * 128u;
          const uint32_t pa = sbuf + (uint32_t)(32 * (ks >> 1) + 8 * (ks & 1));
          const int acc = (q > 0 || ks > 0) ? 1 : 0;
          mma_ts(yd, pa, sdesc(qh_addr + qoff, QKC * 128), id_y, acc);
          if (SPLIT) {
            mma_ts(yd, pa + 16u, sdesc(qh_addr + qoff, QKC * 128), id_y, 1);
            mma_ts(yd, pa, sdesc(ql_addr + qoff, QKC * 128), id_y, 1);
          }
        }
        commit(&pdone[b]);
        ++n_pd[b];
        if (q == CPT - 1) commit(&yfull[yb]);
      }
      if (!ok) {
        // stop the compute warps, and let every MMA issued complete before
        // the tensor memory is released
        abort_flag = 1;
        commit(&dbar);
        mbar_wait_bounded(&dbar, 0);
      }
    }
    __syncwarp();  // the idle lanes wait for the issuing lane before the block barrier
  } else {
    // ================= compute warps: two groups of four (warps 0-3 and
    // 4-7, each covering the 128 TMEM lanes) take alternate chunks, a whole
    // chunk of 64 sources each, so that one group exponentiates while the
    // other waits on tensor memory.  After its first chunk of tile r a group
    // folds its half of tile r - 1's Y (that tile's MMAs are complete by then
    // or soon after) and builds its half of tile r + 1's B operand (one source
    // per thread); the stage of tile r - 1 is then refilled with tile
    // r - 1 + URS, one tile ahead of its use.
    if (tid == 0)
      for (; issued < min(URS, nt); ++issued) issue(issued);
    constexpr int YW = YN / 2;  // Y columns folded per group
    float Ssum[YW], Scomp[YW];
#pragma unroll
    for (int c = 0; c < YW; ++c) Ssum[c] = Scomp[c] = 0.f;
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;  // this warp's TMEM lanes
    // tile r's B operand into buffer r & 1 (its stage awaited first)
    auto make_b = [&](int r) -> bool {
      if (!__all_sync(0xffffffffu, wait(&bars[r % URS], (r / URS) & 1))) return false;
      const float* rs = reinterpret_cast<const float*>(stages + (r % URS) * SBYTES);
      unsigned char* bdst = sB + (r & 1) * BBYTES;
      const int j = tid;  // one source per thread: its K-vector as 16-byte rows
      float bh[W], bl[W];
      float bb = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float xh = p.s * (rs[k * TS + j] - ctr[k]);
        bb = fmaf(-xh, xh, bb);
        const float v = 2.f * xh;
        bh[k] = H::to(H::from(v));
        bl[k] = v - bh[k];
      }
      if (bb < -30000.f) {  // farther than any target can see: contributes 0
#pragma unroll
        for (int k = 0; k < D; ++k) bh[k] = bl[k] = 0.f;
        bb = -30000.f;
      }
      bh[D] = H::to(H::from(bb));
      bl[D] = bb - bh[D];
#pragma unroll
      for (int kc = 0; kc < KC; ++kc) {
        uint32_t w[4];
#pragma unroll
        for (int e = 0; e < 4; ++e)
          w[e] = H::pack(kv_value<D>(bh, bl, 8 * kc + 2 * e, false), kv_value<D>(bh, bl, 8 * kc + 2 * e + 1, false));
        *reinterpret_cast<uint4*>(bdst + kmaj(j, 8 * kc, KC)) = make_uint4(w[0], w[1], w[2], w[3]);
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&bready[r & 1]);
      return true;
    };
    // tile r's Y (this group's YW columns) into the Kahan sums; Y buffer r & 1
    // is handed back and, every MMA of tile r being complete, its stage refilled
    auto fold_y = [&](int r) -> bool {
      const int yb = r & 1;
      if (!__all_sync(0xffffffffu, wait(&yfull[yb], (r >> 1) & 1))) return false;
      fence_after();
      uint32_t yv[8];
      ld8(tmem + y_col + (uint32_t)(YN * yb) + lanes + (uint32_t)(YW * grp), yv);
      wait_ld();
#pragma unroll
      for (int c = 0; c < YW; ++c) kahan_add(Ssum[c], Scomp[c], __uint_as_float(yv[c]));
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&yfree[yb]);
      if (tid == 0 && r + URS < nt) {
        fence_proxy_async_smem();
        issue(r + URS);
        ++issued;
      }
      return true;
    };
    bool ok = nt > 0 ? make_b(0) : true;
    for (int r = 0; r < nt && ok; ++r) {
      for (int h2 = 0; h2 < CPT / 2 && ok; ++h2) {
        const int c = r * CPT + grp + 2 * h2, b = c % NBUF;
        ok = __all_sync(0xffffffffu, wait(&sfull[b], (c / NBUF) & 1));
        if (!ok) break;
        fence_after();
        // P = 2^S over the chunk's 64 columns, 32 at a time: hi in the first
        // 16 columns of each half, lo in the last 16 (each thread reads its
        // values before overwriting them); the second half's load overlaps the
        // first half's store
#pragma unroll 1
        for (int hf = 0; hf < 2; ++hf) {
          const uint32_t cols = tmem + (uint32_t)(b * NC) + lanes + (uint32_t)(32 * hf);
          uint32_t v[32];
          ld32(cols, v);
          wait_ld();
          uint32_t ph[16], pl[16];
#pragma unroll
          for (int w = 0; w < 16; ++w) {
            const float p0 = ex2(__uint_as_float(v[2 * w])), p1 = ex2(__uint_as_float(v[2 * w + 1]));
            ph[w] = H::pack(p0, p1);
            if (SPLIT) {
              const float2 hv = H::unpack(ph[w]);
              pl[w] = H::pack(p0 - hv.x, p1 - hv.y);
            }
          }
          st16(cols, ph);
          if (SPLIT) st16(cols + 16u, pl);
        }
        wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&pfull[b]);
        if (h2 == 0) {
          if (r >= 1 && !(ok = fold_y(r - 1))) break;
          if (r + 1 < nt && !(ok = make_b(r + 1))) break;
        }
      }
    }
    if (ok && nt > 0) ok = fold_y(nt - 1);
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    } else if (i < p.Nt_pad) {
#pragma unroll
      for (int c = 0; c < YW; ++c) {
        const int col = YW * grp + c;
        if (col < p.m) p.part[((int64_t)blockIdx.y * p.m + col) * p.Nt_pad + i] = (double)Ssum[c] - (double)Scomp[c];
      }
    }
  }
  __syncthreads();
  if (abort_flag) {
    // drain (bounded): copies in flight before the shared memory is released
    if (tid == 0)
      for (int rr = 0; rr < issued; ++rr) mbar_wait_bounded(&bars[rr % URS], (rr / URS) & 1);
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------------
// Multi-column product with the exponent on mma.sync and the weighted sum on
// tcgen05 (KRR_OPT_TCGEN05 = 1, mvp_umx_kernel).  The exponent E = A'B'^T
// is computed as in mvp_tcx_kernel, into registers; P = 2^E is split into
// f16 hi / lo there and written to tensor memory with tcgen05.st.16x256b,
// whose fragment (thread (g, t): lanes g and g + 8, columns 2t and 2t + 1)
// is the mma.sync accumulator fragment.  The source order of the exponent
// MMA's B fragment is permuted so that the four values of a row a thread
// holds per 16 sources, from two 8-source n-tiles, are sources 4t .. 4t + 3:
// the packed pairs (4t, 4t+1) and (4t+2, 4t+3) are then exactly the K-pairs
// of tensor-memory columns 2t and 2t + 1 that the P Q MMA reads.  So
// tensor memory is written once per P value and never read by the CUDA
// cores (the tensor-memory exponent kernel below loads S and stores P).
// Roles (per CTA of 128 targets, two per compact super-block):
//  * 8 compute warps in two chunk groups (warps 0-3 and 4-7, each covering
//    the 128 tensor-memory lanes: warp w takes lanes 32 (w mod 4) on as two
//    m-tiles of 16) take alternate 64-source chunks: wait until the P Q MMAs
//    that last read the chunk's P buffer are complete, exponentiate, store
//    P hi / lo, signal pfull.  After their first chunk of a tile they fold
//    the previous tile's Y into Kahan sums and build the next tile's source
//    K-vectors (one source per thread);
//  * 1 MMA warp (one elected thread): per chunk, once its P is stored,
//    Y += Ph Qh (+ Pl Qh + Ph Ql) with A from tensor memory and the weight
//    tiles (pre-split, as for the kernel below) from shared memory.
// Every wait is bounded; on abort the issued MMAs and copies are drained
// before tensor memory is freed.
namespace umx {
constexpr int NCW = umma::THREADS / 32;  // compute warps
constexpr int CPT = TS / umma::NC;       // chunks per tile
template <int D>
constexpr size_t smem_bytes(bool split) {
  const size_t need = umma::URS * (size_t)umma::stage_bytes<D>(split) +
                      sizeof(uint32_t) * 2 * TS * ExpLayout<D>::KV_STRIDE_W;
  return need > umma::SMEM_FLOOR ? need : umma::SMEM_FLOOR;
}
// Column n of n-tile nt in a 16-source block takes source 2n - (n mod 2) +
// 2 nt (see above).  Its inverse gives the shared-memory row of source j in
// its block, so that the B-fragment loads of an n-tile read 8 consecutive
// rows (bank-conflict free with the K-vector stride of ExpLayout).
__device__ __forceinline__ int src_slot(int j) { return 8 * ((j >> 1) & 1) + 2 * (j >> 2) + (j & 1); }
__device__ __forceinline__ void st_16x256b_x2(uint32_t taddr, const uint32_t (&v)[8]) {
  asm volatile("tcgen05.st.sync.aligned.16x256b.x2.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
               :: "r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]),
                  "r"(v[7])
               : "memory");
}
}  // namespace umx

template <int D, bool SPLIT, bool BF>
__global__ void __launch_bounds__(umma::THREADS + 32, 2) mvp_umx_kernel(const TcParams p) {
  using namespace umma;
  using L = ExpLayout<D>;
  using H = Half<BF>;      // P and weight operands
  using HE = Half<false>;  // split-f16 exponent operands
  constexpr int W = D + 1;
  constexpr int NCW = umx::NCW;
  constexpr int CPT = umx::CPT;
  constexpr uint32_t SBYTES = stage_bytes<D>(SPLIT);
  constexpr int QTILE = 2 * YN * TS;  // bytes of one weight tile
  constexpr int KVW = L::KV_STRIDE_W;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bars[URS];   // TMA stages
  __shared__ __align__(8) uint64_t pfull[NBUF];  // P of buffer b stored (one chunk group)
  __shared__ __align__(8) uint64_t pdone[NBUF];  // P Q reading buffer b complete (commit)
  __shared__ __align__(8) uint64_t kready[2];    // a tile's source K-vectors written (compute warps)
  __shared__ __align__(8) uint64_t yfull[2];     // Y buffer complete for its tile (commit)
  __shared__ __align__(8) uint64_t yfree[2];     // Y buffer read (compute warps)
  __shared__ __align__(8) uint64_t dbar;         // after an abort: the MMAs issued are complete
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const bool mma_warp = warp == NCW;
  const int grp = (warp >> 2) & 1;  // chunk group: chunks c with c % 2 == grp
  const int qw = warp & 3;          // tensor-memory lane quarter of a compute warp
  if (p.active && *p.active == 0) return;
  const int64_t nexp = *p.tn_exp;
  const int64_t sb_slot = blockIdx.x >> 1;
  if (sb_slot >= nexp) return;
  unsigned char* stages = smem_raw;  // URS stages: coordinates, Qh, Ql
  uint32_t* kvb = reinterpret_cast<uint32_t*>(smem_raw + URS * SBYTES);  // 2 x TS x KVW

  const int64_t blk = p.torder[sb_slot];
  if (blk * SB < p.row_lo || blk * SB >= p.row_hi) return;  // outside the shard
  float ctr[D];
#pragma unroll
  for (int k = 0; k < D; ++k) ctr[k] = p.tctr[blk * D + k];
  const int64_t row_base = blk * SB + (int64_t)(blockIdx.x & 1) * ROWS;

  // ---- operand A' of the exponent MMA: rows 32 qw + 16 mt + g (+ 8)
  uint32_t afr[2][L::KSTEPS][4];
  if (!mma_warp) {
#pragma unroll
    for (int mt = 0; mt < 2; ++mt) {
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int64_t i = row_base + 32 * qw + 16 * mt + g + 8 * half;
        const int64_t ii = i < p.Nt ? i : p.Nt - 1;
        float ah[W], al[W];
        float r2 = 0.f;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float x = p.xt[(ii / TS) * (int64_t)D * TS + (int64_t)k * TS + ii % TS];
          const float xh = p.s * (x - ctr[k]);
          r2 = fmaf(xh, xh, r2);
          ah[k] = HE::to(HE::from(xh));
          al[k] = xh - ah[k];
        }
        ah[D] = 1.f;
        al[D] = 0.f;
        if (grp == 0 && blockIdx.y == 0 && t == 0 && i < p.Nt_pad) p.fac[i] = exp2f(-r2);
#pragma unroll
        for (int ks = 0; ks < L::KSTEPS; ++ks) {
          const int k0 = 16 * ks + 2 * t;
          afr[mt][ks][half] = HE::pack(kv_value<D>(ah, al, k0, true), kv_value<D>(ah, al, k0 + 1, true));
          afr[mt][ks][half + 2] =
              HE::pack(kv_value<D>(ah, al, k0 + 8, true), kv_value<D>(ah, al, k0 + 9, true));
        }
      }
    }
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < URS; ++st) mbar_init(&bars[st], 1);
    for (int b = 0; b < NBUF; ++b) {
      mbar_init(&pfull[b], GROUP_WARPS);
      mbar_init(&pdone[b], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&kready[b], NCW);
      mbar_init(&yfull[b], 1);
      mbar_init(&yfree[b], NCW);
    }
    mbar_init(&dbar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&tmem_slot)), "r"(TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_before();
  __syncthreads();
  fence_after();
  const uint32_t tmem = tmem_slot;
  // Y buffers at y_col and y_col + YW2: with the split, each holds Ph Qh +
  // Pl Qh in its first YN columns and Ph Ql in the next YN (one N = 32 MMA
  // computes Ph [Qh | Ql]); the halves are added when Y is folded
  constexpr uint32_t YW2 = SPLIT ? 2 * YN : YN;
  static_assert(NBUF * NC + 2 * YW2 <= TMEM_COLS, "tensor-memory columns");
  const uint32_t y_col = NBUF * NC;
  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;

  auto issue = [&](int r) {
    const int stage = r % URS;
    const int64_t tile = t_begin + r;
    unsigned char* dst = stages + stage * SBYTES;
    mbar_arrive_expect_tx(&bars[stage], SBYTES);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    bulk_g2s(dst + D * TS * 4, p.qh_tiles + tile * (int64_t)(YN * TS), QTILE, &bars[stage]);
    if (SPLIT) bulk_g2s(dst + D * TS * 4 + QTILE, p.ql_tiles + tile * (int64_t)(YN * TS), QTILE, &bars[stage]);
  };
  // a bounded wait that also gives up once another role has aborted
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
      if (abort_flag || clock64() - t0 > WAIT_LIMIT_CLOCKS) return false;
    }
    return true;
  };

  int issued = 0;
  if (mma_warp) {
    // ================= MMA warp: chunk c's P Q once its P is stored
    if (lane == 0) {
      const uint32_t id_y = idesc(BF ? 1 : 0, YN, ROWS);
      const uint32_t id_y2 = idesc(BF ? 1 : 0, 2 * YN, ROWS);
      uint32_t n_yf[2] = {0, 0};
      const int total = nt * CPT;
      bool ok = true;
      for (int c = 0; c < total && ok; ++c) {
        const int r = c / CPT, q = c % CPT, b = c % NBUF, yb = r & 1;
        ok = wait(&pfull[b], (uint32_t)(c / NBUF) & 1);
        if (ok && q == 0 && r >= 2) {  // Y buffer yb was read for tile r - 2
          ok = wait(&yfree[yb], n_yf[yb] & 1);
          ++n_yf[yb];
        }
        if (!ok) break;
        fence_after();
        const uint32_t qh_addr = smem_addr(stages + (r % URS) * SBYTES + D * TS * 4);
        const uint32_t pbuf = tmem + (uint32_t)(b * NC);
        const uint32_t yd = tmem + y_col + YW2 * (uint32_t)yb;
#pragma unroll
        for (int ks = 0; ks < NC / 16; ++ks) {
          const uint32_t qoff = (uint32_t)((NC / 8) * q + 2 * ks) * 128u;
          const uint32_t pa = pbuf + (uint32_t)(32 * (ks >> 1) + 8 * (ks & 1));
          const int acc = (q > 0 || ks > 0) ? 1 : 0;
          if (SPLIT) {
            // B rows 0-15 are Qh, rows 16-31 the Ql tile that follows it (the
            // 8-row-group stride is a quarter of a tile): Ph [Qh | Ql]
            mma_ts(yd, pa, sdesc(qh_addr + qoff, (TS / 8) * 128), id_y2, acc);
            mma_ts(yd, pa + 16u, sdesc(qh_addr + qoff, (TS / 8) * 128), id_y, 1);
          } else {
            mma_ts(yd, pa, sdesc(qh_addr + qoff, (TS / 8) * 128), id_y, acc);
          }
        }
        commit(&pdone[b]);
        if (q == CPT - 1) commit(&yfull[yb]);
      }
      if (!ok) {
        // stop the compute warps, and let every MMA issued complete before
        // the tensor memory is released
        abort_flag = 1;
        commit(&dbar);
        mbar_wait_bounded(&dbar, 0);
      }
    }
    __syncwarp();  // the idle lanes wait for the issuing lane before the block barrier
  } else {
    // ================= compute warps
    if (tid == 0)
      for (; issued < min(URS, nt); ++issued) issue(issued);
    constexpr int YW = YN / 2;  // Y columns folded per group
    float Ssum[YW], Scomp[YW];
#pragma unroll
    for (int c = 0; c < YW; ++c) Ssum[c] = Scomp[c] = 0.f;
    const uint32_t lanes = (uint32_t)(32 * qw) << 16;  // this warp's tensor-memory lanes
    // tile r's source K-vectors into buffer r & 1 (its stage awaited first;
    // one source per thread)
    auto make_k = [&](int r) -> bool {
      if (!__all_sync(0xffffffffu, wait(&bars[r % URS], (r / URS) & 1))) return false;
      const float* rs = reinterpret_cast<const float*>(stages + (r % URS) * SBYTES);
      uint32_t* kv = kvb + (r & 1) * TS * KVW;
      const int j = tid;
      float bh[W], bl[W];
      float bb = 0.f;
#pragma unroll
      for (int k = 0; k < D; ++k) {
        const float xh = p.s * (rs[k * TS + j] - ctr[k]);
        bb = fmaf(-xh, xh, bb);
        const float v = 2.f * xh;
        bh[k] = HE::to(HE::from(v));
        bl[k] = v - bh[k];
      }
      if (bb < -30000.f) {  // farther than any target can see: contributes 0
#pragma unroll
        for (int k = 0; k < D; ++k) bh[k] = bl[k] = 0.f;
        bb = -30000.f;
      }
      bh[D] = HE::to(HE::from(bb));
      bl[D] = bb - bh[D];
      uint32_t kw[L::KV / 2];
#pragma unroll
      for (int w = 0; w < L::KV / 2; ++w)
        kw[w] = HE::pack(kv_value<D>(bh, bl, 2 * w, false), kv_value<D>(bh, bl, 2 * w + 1, false));
      // row of source j: its permuted slot within its 16-source block
      uint4* dst = reinterpret_cast<uint4*>(kv + ((j & ~15) + umx::src_slot(j & 15)) * KVW);
#pragma unroll
      for (int w = 0; w < L::KV / 8; ++w) dst[w] = make_uint4(kw[4 * w], kw[4 * w + 1], kw[4 * w + 2], kw[4 * w + 3]);
      __syncwarp();
      if (lane == 0) mbar_arrive1(&kready[r & 1]);
      return true;
    };
    // tile r's Y (this group's YW columns) into the Kahan sums; Y buffer r & 1
    // is handed back and, every MMA of tile r being complete, its stage refilled
    auto fold_y = [&](int r) -> bool {
      const int yb = r & 1;
      if (!__all_sync(0xffffffffu, wait(&yfull[yb], (r >> 1) & 1))) return false;
      fence_after();
      uint32_t yv[8], yl[8];
      const uint32_t ya = tmem + y_col + YW2 * (uint32_t)yb + lanes + (uint32_t)(YW * grp);
      ld8(ya, yv);
      if (SPLIT) ld8(ya + YN, yl);
      wait_ld();
#pragma unroll
      for (int c = 0; c < YW; ++c)
        kahan_add(Ssum[c], Scomp[c], SPLIT ? __uint_as_float(yv[c]) + __uint_as_float(yl[c]) : __uint_as_float(yv[c]));
      fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&yfree[yb]);
      if (tid == 0 && r + URS < nt) {
        fence_proxy_async_smem();
        issue(r + URS);
        ++issued;
      }
      return true;
    };
    // rows of this lane's B-fragment columns (sources src_perm(nt, g), stored
    // at slot 8 nt + g of their block)
    const int js0 = g, js1 = 8 + g;
    bool ok = nt > 0 ? make_k(0) : true;
    for (int r = 0; r < nt && ok; ++r) {
      ok = __all_sync(0xffffffffu, wait(&kready[r & 1], (uint32_t)(r >> 1) & 1));
      if (!ok) break;
      const uint32_t* kv = kvb + (r & 1) * TS * KVW;
      for (int h2 = 0; h2 < CPT / 2 && ok; ++h2) {
        const int c = r * CPT + grp + 2 * h2, b = c % NBUF, q = c % CPT;
        if (c >= NBUF) {  // the P Q MMAs that last read buffer b are complete
          ok = __all_sync(0xffffffffu, wait(&pdone[b], (uint32_t)(c / NBUF - 1) & 1));
          if (!ok) break;
        }
        fence_after();
#pragma unroll
        for (int hf = 0; hf < 2; ++hf) {  // 32 sources: tensor-memory columns 32 hf on
          // B fragments of the two 16-source blocks, shared by both m-tiles
          uint32_t bfr[2][2][L::KSTEPS][2];
#pragma unroll
          for (int k2 = 0; k2 < 2; ++k2) {
            const int j0 = NC * q + 32 * hf + 16 * k2;
#pragma unroll
            for (int ks = 0; ks < L::KSTEPS; ++ks) {
              bfr[k2][0][ks][0] = kv[(j0 + js0) * KVW + 8 * ks + t];
              bfr[k2][0][ks][1] = kv[(j0 + js0) * KVW + 8 * ks + t + 4];
              bfr[k2][1][ks][0] = kv[(j0 + js1) * KVW + 8 * ks + t];
              bfr[k2][1][ks][1] = kv[(j0 + js1) * KVW + 8 * ks + t + 4];
            }
          }
#pragma unroll
          for (int mt = 0; mt < 2; ++mt) {
            uint32_t ph[8], pl[8];
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
              float e0[4], e1[4];
              mma16816_z(e0, afr[mt][0], bfr[k2][0][0][0], bfr[k2][0][0][1]);
              mma16816_z(e1, afr[mt][0], bfr[k2][1][0][0], bfr[k2][1][0][1]);
#pragma unroll
              for (int ks = 1; ks < L::KSTEPS; ++ks) {
                mma16816<false>(e0, afr[mt][ks], bfr[k2][0][ks][0], bfr[k2][0][ks][1]);
                mma16816<false>(e1, afr[mt][ks], bfr[k2][1][ks][0], bfr[k2][1][ks][1]);
              }
              // registers of tcgen05.st.16x256b: (lane g, column 2t), (g, 2t+1),
              // (g+8, 2t), (g+8, 2t+1); the second 16 sources in the repeat
              const float v[4][2] = {{ex2(e0[0]), ex2(e0[1])}, {ex2(e1[0]), ex2(e1[1])},
                                     {ex2(e0[2]), ex2(e0[3])}, {ex2(e1[2]), ex2(e1[3])}};
#pragma unroll
              for (int e = 0; e < 4; ++e) {
                ph[4 * k2 + e] = H::pack(v[e][0], v[e][1]);
                if (SPLIT) {
                  const float2 lo = ffma2(H::unpack(ph[4 * k2 + e]), make_float2(-1.f, -1.f),
                                          make_float2(v[e][0], v[e][1]));
                  pl[4 * k2 + e] = H::pack(lo.x, lo.y);
                }
              }
            }
            const uint32_t cols = tmem + lanes + ((uint32_t)(16 * mt) << 16) + (uint32_t)(b * NC + 32 * hf);
            umx::st_16x256b_x2(cols, ph);
            if (SPLIT) umx::st_16x256b_x2(cols + 16u, pl);
          }
        }
        wait_st();
        fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive1(&pfull[b]);
        if (h2 == 0) {
          if (r >= 1 && !(ok = fold_y(r - 1))) break;
          if (r + 1 < nt && !(ok = make_k(r + 1))) break;
        }
      }
    }
    if (ok && nt > 0) ok = fold_y(nt - 1);
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    } else {
      const int64_t i = row_base + 32 * qw + lane;
      if (i < p.Nt_pad) {
#pragma unroll
        for (int c = 0; c < YW; ++c) {
          const int col = YW * grp + c;
          if (col < p.m) p.part[((int64_t)blockIdx.y * p.m + col) * p.Nt_pad + i] = (double)Ssum[c] - (double)Scomp[c];
        }
      }
    }
  }
  __syncthreads();
  if (abort_flag) {
    // drain (bounded): copies in flight before the shared memory is released
    if (tid == 0)
      for (int rr = 0; rr < issued; ++rr) mbar_wait_bounded(&bars[rr % URS], (rr / URS) & 1);
    __syncthreads();
  }
  fence_before();
  __syncthreads();
  fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TMEM_COLS) : "memory");
}

// ------------------------------------------------------------------------
// High-dimensional single-column product on the 5th-generation tensor cores
// (tcgen05; the default above 8 dimensions, KRR_OPT_HIGHD_TCGEN05): the
// contraction of mvp_tch_kernel, the
// split 3 (d + 1)-term K-vectors of 128 targets against 128 sources at a
// time, as KSTEPS tcgen05.mma (M = N = 128, K = 16, f16 in, f32 out) into
// tensor memory.  Warp-specialized pipeline over chunks of 128 sources:
//  * 8 worker warps: write the K-vectors of chunk c + 1 into the B operand
//    buffer (c + 1) & 1 (K-major core matrices, no swizzle; the two threads
//    of a source take half of its components each), then read S of chunk c
//    from tensor-memory buffer c & 1 (warp w: lanes 32 (w mod 4) on = target
//    rows, half of the columns) and add q_j 2^S_ij;
//  * 1 MMA warp: issues chunk c once its B operand is written and the
//    epilogue of chunk c - 2 has released the S buffer, and commits to
//    mdone[c & 1].
// A B buffer is rewritten only after the epilogue of its previous chunk,
// which waited for that chunk's MMAs.  Two CTAs per compact super-block (128
// targets each).  Raw source tiles arrive by TMA bulk copies; a tile's stage
// is refilled once the B operands of its last chunk are written (its weights
// are copied to a per-tile buffer first).  Every wait is bounded; on abort
// the issued MMAs and copies are drained before tensor memory is freed.
namespace uhd {
constexpr int ROWS = 128;     // targets per CTA (MMA M, tensor-memory lanes)
constexpr int WORKERS = 256;  // 8 worker warps; warp 8 issues the MMAs
// K-vector layout: three terms, each padded to W8 = round_up(d + 1, 8) slots,
// so that every 16-byte k-chunk holds 8 consecutive components of one term
// (one vector store each).
template <int D>
struct L {
  static constexpr int W = D + 1;
  static constexpr int W8 = (W + 7) / 8 * 8;
  static constexpr int G = W8 / 8;                 // k-chunks per term
  static constexpr int KSTEPS = (3 * G + 1) / 2;   // K = 16 per MMA
  static constexpr int KV = 16 * KSTEPS;           // halves per K-vector
  static constexpr int KC = KV / 8;                // 16-byte k-chunks
  // sources per chunk (MMA N) and raw stages, sized to the 227 KB of shared
  // memory: A, two B buffers, the raw tiles, two tiles' weights
  static constexpr int NC = D >= 64 ? 64 : 128;
  static constexpr int RSD = D <= 32 ? 2 : 1;
  static constexpr int TMEM_COLS = 2 * NC;
};
template <int D>
constexpr size_t smem_bytes() {
  using LL = L<D>;
  return (size_t)(ROWS + 2 * LL::NC) * LL::KV * 2 + sizeof(float) * ((size_t)LL::RSD * (D + 1) * TS + 2 * TS);
}
static_assert(smem_bytes<64>() <= 225 * 1024 && smem_bytes<48>() <= 225 * 1024, "shared memory");
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, %0;" :: "n"(WORKERS) : "memory"); }
}  // namespace uhd

template <int D>
__global__ void __launch_bounds__(uhd::WORKERS + 32) mvp_uhd_kernel(const TcParams p) {
  using LL = uhd::L<D>;
  using H = Half<false>;
  constexpr int KS = LL::KSTEPS, KC = LL::KC, RSD = LL::RSD;
  constexpr int ROWS = uhd::ROWS, NC = LL::NC, NW8 = uhd::WORKERS;
  constexpr int TPS = NW8 / NC;  // worker threads per source of a chunk
  constexpr int RAW = (D + 1) * TS;  // coordinates, weights
  constexpr int CPT = TS / NC;       // chunks per tile
  constexpr uint32_t BBYTES = NC * LL::KV * 2;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char* sA = smem_raw;
  unsigned char* sB = sA + ROWS * LL::KV * 2;  // two buffers
  float* raw = reinterpret_cast<float*>(sB + 2 * BBYTES);
  float* qbuf = raw + RSD * RAW;  // two tiles' weights
  __shared__ __align__(8) uint64_t bars[RSD];
  __shared__ __align__(8) uint64_t bready[2];  // B buffer written (worker warps)
  __shared__ __align__(8) uint64_t mdone[2];   // chunk's MMAs complete (commit)
  __shared__ __align__(8) uint64_t sfree[2];   // S buffer read (worker warps)
  __shared__ __align__(8) uint64_t dbar;       // after an abort: every MMA issued is complete
  __shared__ uint32_t tmem_slot;
  __shared__ volatile int abort_flag;
  __shared__ float ctr[D];
  __shared__ double red[ROWS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const bool mma_warp = warp == NW8 / 32;
  const int half = (tid / ROWS) & 1;  // worker: half of a source's components / of a row's columns
  if (p.active && *p.active == 0) return;
  const int64_t nexp = *p.tn_exp;
  const int64_t sb_slot = blockIdx.x >> 1;
  if (sb_slot >= nexp) return;
  const int64_t blk = p.torder[sb_slot];
  if (blk * SB < p.row_lo || blk * SB >= p.row_hi) return;  // outside the shard
  for (int k = tid; k < D; k += blockDim.x) ctr[k] = p.tctr[blk * D + k];
  for (int w = tid; w < (ROWS + 2 * NC) * LL::KV * 2 / 16; w += blockDim.x)
    reinterpret_cast<uint4*>(sA)[w] = make_uint4(0u, 0u, 0u, 0u);  // padding slots stay zero
  __syncthreads();
  const int row = tid % ROWS;
  const int64_t i = blk * SB + (int64_t)(blockIdx.x & 1) * ROWS + row;
  if (!mma_warp && half == 0) {  // operand A: this row's K-vector [uh | uh | ul] over [u, 1]
    const int64_t ii = i < p.Nt ? i : p.Nt - 1;
    const float* xr = p.xt + (ii / TS) * (int64_t)D * TS + ii % TS;
    float r2 = 0.f;
    for (int g = 0; g < LL::G; ++g) {
      uint32_t hw[4], lw[4];
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        float u2[2];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int k = 8 * g + 2 * e + h2;
          u2[h2] = k < D ? p.s * (xr[(int64_t)k * TS] - ctr[k]) : (k == D ? 1.f : 0.f);
          if (k < D) r2 = fmaf(u2[h2], u2[h2], r2);
        }
        hw[e] = H::pack(u2[0], u2[1]);
        const float2 hv = H::unpack(hw[e]);
        lw[e] = H::pack(u2[0] - hv.x, u2[1] - hv.y);
      }
      const uint4 hv4 = make_uint4(hw[0], hw[1], hw[2], hw[3]), lv4 = make_uint4(lw[0], lw[1], lw[2], lw[3]);
      *reinterpret_cast<uint4*>(sA + umma::kmaj(row, 8 * g, KC)) = hv4;
      *reinterpret_cast<uint4*>(sA + umma::kmaj(row, 8 * (LL::G + g), KC)) = hv4;
      *reinterpret_cast<uint4*>(sA + umma::kmaj(row, 8 * (2 * LL::G + g), KC)) = lv4;
    }
    if (blockIdx.y == 0 && i < p.Nt_pad) p.fac[i] = exp2f(-r2);
  }
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < RSD; ++st) mbar_init(&bars[st], 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&bready[b], NW8 / 32);
      mbar_init(&mdone[b], 1);
      mbar_init(&sfree[b], NW8 / 32);
    }
    mbar_init(&dbar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 :: "r"(smem_addr(&tmem_slot)), "r"(LL::TMEM_COLS) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  fence_proxy_async_smem();  // operand A: generic-proxy writes, read by the tensor cores
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = tmem_slot;
  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;
  const int total = nt * CPT;
  // a bounded wait that also gives up once the other role has aborted
  auto wait = [&](uint64_t* bar, uint32_t parity) -> bool {
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity)) {
      if (abort_flag || clock64() - t0 > WAIT_LIMIT_CLOCKS) return false;
    }
    return true;
  };
  auto issue = [&](int r) {
    const int stage = r % RSD;
    const int64_t tile = t_begin + r;
    float* dst = raw + stage * RAW;
    mbar_arrive_expect_tx(&bars[stage], (uint32_t)RAW * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    bulk_g2s(dst + D * TS, p.Q + tile * (int64_t)TS, TS * 4, &bars[stage]);
  };
  int issued = 0;
  float S = 0.f, C = 0.f;
  bool ok = true;
  if (mma_warp) {
    // ================= MMA warp (one lane issues)
    if (lane == 0) {
      const uint32_t id_s = umma::idesc(0, NC, ROWS);
      const uint32_t a_addr = smem_addr(sA), b_addr = smem_addr(sB);
      for (int c = 0; c < total && ok; ++c) {
        const int b = c & 1;
        ok = wait(&bready[b], (c >> 1) & 1);
        if (ok && c >= 2) ok = wait(&sfree[b], ((c - 2) >> 1) & 1);
        if (!ok) break;
        umma::fence_after();
#pragma unroll
        for (int ks = 0; ks < KS; ++ks)
          umma::mma_ss(tmem + (uint32_t)(b * NC), umma::sdesc(a_addr + 256u * ks, KC * 128),
                       umma::sdesc(b_addr + (uint32_t)b * BBYTES + 256u * ks, KC * 128), id_s, ks > 0);
        umma::commit(&mdone[b]);
      }
      if (!ok) {
        abort_flag = 1;
        umma::commit(&dbar);
        mbar_wait_bounded(&dbar, 0);
      }
    }
    __syncwarp();
  } else {
    // ================= worker warps
    if (tid == 0)
      for (; issued < min(RSD, nt); ++issued) issue(issued);
    const uint32_t lanes = (uint32_t)(32 * (warp & 3)) << 16;
    // chunk c's B operand (and, at a tile's first chunk, the tile's
    // weights).  Every worker calls it for every chunk, aborted or not, so
    // the named worker barriers always match.
    auto make_b = [&](int c) {
      const int r = c / CPT, q = c % CPT;
      if (q == 0) {
        if (!abort_flag && !wait(&bars[r % RSD], (r / RSD) & 1)) abort_flag = 1;
        uhd::workers_sync();
        if (!abort_flag) qbuf[(r & 1) * TS + tid] = raw[(r % RSD) * RAW + D * TS + tid];
      }
      if (!abort_flag) {
      const float* rs = raw + (r % RSD) * RAW;
      unsigned char* bdst = sB + (c & 1) * BBYTES;
      const int jr = tid % NC, j = q * NC + jr;
      // the TPS threads of a source take interleaved k-chunks of each term
      float bb = 0.f;
#pragma unroll 8
      for (int k = 0; k < D; ++k) {
        const float v = p.s * (rs[k * TS + j] - ctr[k]);
        bb = fmaf(-v, v, bb);
      }
      const bool far = bb < -30000.f;  // farther than any target can see: contributes 0
      const float b_aug = far ? -30000.f : bb;
      for (int g = tid / NC; g < LL::G; g += TPS) {
        uint32_t hw[4], lw[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          float v2[2];
#pragma unroll
          for (int h2 = 0; h2 < 2; ++h2) {
            const int k = 8 * g + 2 * e + h2;
            v2[h2] = k < D ? (far ? 0.f : 2.f * p.s * (rs[k * TS + j] - ctr[k])) : (k == D ? b_aug : 0.f);
          }
          hw[e] = H::pack(v2[0], v2[1]);
          const float2 hv = H::unpack(hw[e]);
          lw[e] = H::pack(v2[0] - hv.x, v2[1] - hv.y);
        }
        const uint4 hv4 = make_uint4(hw[0], hw[1], hw[2], hw[3]), lv4 = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        *reinterpret_cast<uint4*>(bdst + umma::kmaj(jr, 8 * g, KC)) = hv4;
        *reinterpret_cast<uint4*>(bdst + umma::kmaj(jr, 8 * (LL::G + g), KC)) = lv4;
        *reinterpret_cast<uint4*>(bdst + umma::kmaj(jr, 8 * (2 * LL::G + g), KC)) = hv4;
      }
      fence_proxy_async_smem();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&bready[c & 1]);
      }
      if (q == CPT - 1) {  // the tile's stage is no longer read: refill it
        uhd::workers_sync();
        if (tid == 0 && r + RSD < nt && !abort_flag) {
          fence_proxy_async_smem();
          issue(r + RSD);
          ++issued;
        }
      }
    };
    if (total > 0) make_b(0);
    for (int c = 0; c < total; ++c) {
      if (c + 1 < total) make_b(c + 1);
      if (abort_flag) continue;  // keep passing the worker barriers
      const int b = c & 1, r = c / CPT, q = c % CPT;
      if (!__all_sync(0xffffffffu, wait(&mdone[b], (c >> 1) & 1))) {
        abort_flag = 1;
        continue;
      }
      umma::fence_after();
      const float* qc0 = qbuf + (r & 1) * TS + q * NC;
#pragma unroll 1
      for (int cb = half * (NC / 2); cb < (half + 1) * (NC / 2); cb += 32) {
        uint32_t v[32];
        umma::ld32(tmem + lanes + (uint32_t)(b * NC + cb), v);
        umma::wait_ld();
        const float* qc = qc0 + cb;
        float2 acc = make_float2(0.f, 0.f);
#pragma unroll
        for (int e = 0; e < 32; e += 2)
          acc = ffma2(make_float2(qc[e], qc[e + 1]),
                      make_float2(ex2(__uint_as_float(v[e])), ex2(__uint_as_float(v[e + 1]))), acc);
        kahan_add(S, C, acc.x + acc.y);
      }
      umma::fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive1(&sfree[b]);
    }
    if (abort_flag && lane == 0) atomicExch(p.err, DEV_TIMEOUT);
  }
  __syncthreads();
  if (abort_flag) {
    if (tid == 0)
      for (int rr = 0; rr < issued; ++rr) mbar_wait_bounded(&bars[rr % RSD], (rr / RSD) & 1);
    __syncthreads();
  }
  // the two halves of each row
  if (!mma_warp && half == 1) red[row] = (double)S - (double)C;
  __syncthreads();
  if (!abort_flag && !mma_warp && half == 0 && i < p.Nt_pad)
    p.part[(int64_t)blockIdx.y * p.Nt_pad + i] = ((double)S - (double)C) + red[row];
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(LL::TMEM_COLS) : "memory");
}

// Weights Q (m columns, stride ld, sorted, zero padded) -> per source tile a
// 16 x 256 K-major f16 tile (core matrices 8 rows x 16 B): hi, and lo = the
// float32 remainder when split; rows m..15 zero.  One thread per 8 sources of
// one row (16-byte stores).
template <bool BF>
__global__ void q_split_kernel(const float* __restrict__ Q, int m, int64_t ld, int64_t ntiles,
                               uint16_t* __restrict__ qh, uint16_t* __restrict__ ql, const int* active) {
  using H = Half<BF>;
  if (active && *active == 0) return;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ntiles * 512) return;
  const int64_t tile = e >> 9;
  const int w = (int)(e & 511);
  const int c = (w & 7) + 8 * ((w >> 3) & 1);  // row (column of Y)
  const int seg = w >> 4;                      // 8 sources
  uint32_t h[4] = {0, 0, 0, 0}, l[4] = {0, 0, 0, 0};
  if (c < m) {
    const float* src = Q + (int64_t)c * ld + tile * TS + 8 * seg;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const float v0 = src[2 * k], v1 = src[2 * k + 1];
      h[k] = H::pack(v0, v1);
      const float2 hv = H::unpack(h[k]);
      if (ql) l[k] = H::pack(v0 - hv.x, v1 - hv.y);
    }
  }
  const int64_t off = tile * (int64_t)(umma::YN * TS) + (int64_t)(umma::kmaj(c, 8 * seg, TS / 8) >> 1);
  *reinterpret_cast<uint4*>(qh + off) = make_uint4(h[0], h[1], h[2], h[3]);
  if (ql) *reinterpret_cast<uint4*>(ql + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

template <int D, bool SPLIT, bool BF>
cudaError_t umma_launch_typed(const TcParams& p, int splits, cudaStream_t st, bool dry) {
  const size_t shm = umma::smem_bytes<D>(SPLIT);
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mvp_umma_kernel<D, SPLIT, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e) return e;
    done[dev] = true;
  }
  if (dry) return cudaSuccess;
  dim3 grid((unsigned)(2 * p.nblk), (unsigned)splits);
  mvp_umma_kernel<D, SPLIT, BF><<<grid, umma::THREADS + 32, shm, st>>>(p); count_launch();
  return cudaGetLastError();
}

template <int D, bool SPLIT, bool BF>
cudaError_t umx_launch_typed(const TcParams& p, int splits, cudaStream_t st, bool dry) {
  const size_t shm = umx::smem_bytes<D>(SPLIT);
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mvp_umx_kernel<D, SPLIT, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
    if (e) return e;
    done[dev] = true;
  }
  if (dry) return cudaSuccess;
  dim3 grid((unsigned)(2 * p.nblk), (unsigned)splits);
  mvp_umx_kernel<D, SPLIT, BF><<<grid, umma::THREADS + 32, shm, st>>>(p); count_launch();
  return cudaGetLastError();
}

template <int D>
cudaError_t umma_dispatch(const TcParams& p, int splits, bool split, bool bf, int kind, cudaStream_t st,
                          bool dry) {
  if (kind == 2) {
    if (split) return umma_launch_typed<D, true, false>(p, splits, st, dry);
    return bf ? umma_launch_typed<D, false, true>(p, splits, st, dry)
              : umma_launch_typed<D, false, false>(p, splits, st, dry);
  }
  if (split) return umx_launch_typed<D, true, false>(p, splits, st, dry);
  return bf ? umx_launch_typed<D, false, true>(p, splits, st, dry)
            : umx_launch_typed<D, false, false>(p, splits, st, dry);
}

constexpr int TCX_MT = 4;

template <int D>
constexpr size_t tcx_smem_bytes() {
  return sizeof(float) * RS * (D + 1) * TS + sizeof(uint32_t) * 2 * TS * ExpLayout<D>::KV_STRIDE_W +
         sizeof(float) * 2 * TS;
}

template <int D>
cudaError_t tcx_launch_typed(const TcParams& p, int splits, cudaStream_t st, bool dry) {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mvp_tcx_kernel<D, TCX_MT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tcx_smem_bytes<D>());
    if (e) return e;
    done[dev] = true;
  }
  if (dry) return cudaSuccess;
  dim3 grid((unsigned)p.nblk, (unsigned)splits);
  mvp_tcx_kernel<D, TCX_MT><<<grid, 32 * (SB / (16 * TCX_MT)), tcx_smem_bytes<D>(), st>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <int D>
cudaError_t uhd_launch_typed(const TcParams& p, int splits, cudaStream_t st, bool dry) {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mvp_uhd_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)uhd::smem_bytes<D>());
    if (e) return e;
    done[dev] = true;
  }
  if (dry) return cudaSuccess;
  dim3 grid((unsigned)(2 * p.nblk), (unsigned)splits);
  mvp_uhd_kernel<D><<<grid, uhd::WORKERS + 32, uhd::smem_bytes<D>(), st>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <int D>
cudaError_t tch_launch_typed(const TcParams& p, int splits, cudaStream_t st, bool dry) {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(mvp_tch_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)tch_smem_bytes<D>());
    if (e) return e;
    done[dev] = true;
  }
  if (dry) return cudaSuccess;
  dim3 grid((unsigned)p.nblk, (unsigned)splits);
  mvp_tch_kernel<D><<<grid, 32 * HighD<D>::WARPS, tch_smem_bytes<D>(), st>>>(p);
  count_launch();
  return cudaGetLastError();
}

template <int D, int MT, int NRT, bool SPLIT, bool BF>
cudaError_t launch(const TcParams& p, int splits, int warps, cudaStream_t st, bool dry) {
  using L = ExpLayout<D>;
  constexpr int MC = 8 * NRT;
  const size_t shm = sizeof(float) * RS * (D + p.m) * TS + sizeof(uint32_t) * 2 * TS * L::KV_STRIDE_W +
                     sizeof(uint32_t) * 2 * (SPLIT ? 2 : 1) * MC * 132;
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && !done[dev]) {
    // sized for the largest m of this instance
    const size_t shm_max = sizeof(float) * RS * (D + MC) * TS + sizeof(uint32_t) * 2 * TS * L::KV_STRIDE_W +
                           sizeof(uint32_t) * 2 * (SPLIT ? 2 : 1) * MC * 132;
    cudaError_t e = cudaFuncSetAttribute(mvp_tc_kernel<D, MT, NRT, SPLIT, BF>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm_max);
    if (e) return e;
    done[dev] = true;
  }
  if (dry) return cudaSuccess;
  dim3 grid((unsigned)p.nblk, (unsigned)splits);
  mvp_tc_kernel<D, MT, NRT, SPLIT, BF><<<grid, 32 * warps, shm, st>>>(p); count_launch();
  return cudaGetLastError();
}

template <int D, bool SPLIT, bool BF>
cudaError_t dispatch_m(const TcParams& p, int splits, cudaStream_t st, bool dry) {
  // m-tiles per warp: 4 (2 for two groups of right-hand sides with split
  // accumulators, keeping registers under 128); never beyond the block
  const int mt_max = p.WB / 16;
  if (p.m <= 8) {
    const int MT = std::min(4, mt_max);
    const int warps = p.WB / (16 * MT);
    if (MT == 4) return launch<D, 4, 1, SPLIT, BF>(p, splits, warps, st, dry);
    return launch<D, 2, 1, SPLIT, BF>(p, splits, warps, st, dry);
  }
  const int MT = std::min(2, mt_max);
  return launch<D, 2, 2, SPLIT, BF>(p, splits, p.WB / (16 * MT), st, dry);
}

template <int D>
cudaError_t dispatch_prec(const TcParams& p, int splits, bool split, bool bf, cudaStream_t st,
                          bool dry) {
  if (split)
    return bf ? dispatch_m<D, true, true>(p, splits, st, dry) : dispatch_m<D, true, false>(p, splits, st, dry);
  return bf ? dispatch_m<D, false, true>(p, splits, st, dry) : dispatch_m<D, false, false>(p, splits, st, dry);
}

}  // namespace

cudaError_t mvp_tc_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* Q, int m,
                            bool split, bool bf, int splits, int tiles_per_split, double* part,
                            float* fac, const int* active, cudaStream_t st, bool dry) {
  if (m < 1 || m > 16) return cudaErrorNotSupported;
  TcParams p{};
  p.xt = T.xs;
  p.Nt = T.N;
  p.Nt_pad = T.Npad;
  // one CTA per expanded-form super-block
  p.tctr = T.sb_ctr;
  p.torder = T.sb_order;
  p.tn_exp = T.sb_nexp;
  p.nblk = std::max<int64_t>(1, T.h_sb_nexp);
  p.WB = SB;
  p.xs = S.xs;
  p.Q = Q;
  p.Ns_pad = S.Npad;
  p.m = m;
  p.ntiles = (int)(S.Npad / TS);
  p.tiles_per_split = tiles_per_split;
  p.part = part;
  p.fac = fac;
  p.err = c.d_err;
  p.row_lo = c.row_lo;
  p.row_hi = c.row_hi;
  p.s = S.scale;
  p.active = active;
  switch (T.d) {
    case 1: return dispatch_prec<1>(p, splits, split, bf, st, dry);
    case 2: return dispatch_prec<2>(p, splits, split, bf, st, dry);
    case 3: return dispatch_prec<3>(p, splits, split, bf, st, dry);
    case 4: return dispatch_prec<4>(p, splits, split, bf, st, dry);
    case 5: return dispatch_prec<5>(p, splits, split, bf, st, dry);
    case 6: return dispatch_prec<6>(p, splits, split, bf, st, dry);
    case 7: return dispatch_prec<7>(p, splits, split, bf, st, dry);
    case 8: return dispatch_prec<8>(p, splits, split, bf, st, dry);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t mvp_tcx_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* q,
                             int splits, int tiles_per_split, double* part, float* fac,
                             const int* active, cudaStream_t st, bool dry) {
  TcParams p{};
  p.xt = T.xs;
  p.Nt = T.N;
  p.Nt_pad = T.Npad;
  p.tctr = T.sb_ctr;
  p.torder = T.sb_order;
  p.tn_exp = T.sb_nexp;
  p.nblk = std::max<int64_t>(1, T.h_sb_nexp);
  p.WB = SB;
  p.xs = S.xs;
  p.Q = q;
  p.Ns_pad = S.Npad;
  p.m = 1;
  p.ntiles = (int)(S.Npad / TS);
  p.tiles_per_split = tiles_per_split;
  p.part = part;
  p.fac = fac;
  p.err = c.d_err;
  p.row_lo = c.row_lo;
  p.row_hi = c.row_hi;
  p.s = S.scale;
  p.active = active;
  switch (T.d) {
    case 1: return tcx_launch_typed<1>(p, splits, st, dry);
    case 2: return tcx_launch_typed<2>(p, splits, st, dry);
    case 3: return tcx_launch_typed<3>(p, splits, st, dry);
    case 4: return tcx_launch_typed<4>(p, splits, st, dry);
    case 5: return tcx_launch_typed<5>(p, splits, st, dry);
    case 6: return tcx_launch_typed<6>(p, splits, st, dry);
    case 7: return tcx_launch_typed<7>(p, splits, st, dry);
    case 8: return tcx_launch_typed<8>(p, splits, st, dry);
    case 16: return c.highd_tcgen05 ? uhd_launch_typed<16>(p, splits, st, dry) : tch_launch_typed<16>(p, splits, st, dry);
    case 32: return c.highd_tcgen05 ? uhd_launch_typed<32>(p, splits, st, dry) : tch_launch_typed<32>(p, splits, st, dry);
    case 48: return c.highd_tcgen05 ? uhd_launch_typed<48>(p, splits, st, dry) : tch_launch_typed<48>(p, splits, st, dry);
    case 64: return c.highd_tcgen05 ? uhd_launch_typed<64>(p, splits, st, dry) : tch_launch_typed<64>(p, splits, st, dry);
    default: return cudaErrorNotSupported;
  }
}

cudaError_t mvp_umma_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* Q, int m,
                              bool split, bool bf, int splits, int tiles_per_split, double* part,
                              float* fac, const int* active, cudaStream_t st, bool dry) {
  if (m < 1 || m > umma::YN) return cudaErrorNotSupported;
  // the weights pre-split per source tile (workspace sized here, also in a
  // dry run, so that a captured launch allocates nothing)
  const int64_t ntiles = S.Npad / TS;
  void *qh = nullptr, *ql = nullptr;
  cudaError_t e = c.ws.get("umma.qh", sizeof(uint16_t) * umma::YN * TS * (size_t)ntiles, &qh);
  if (!e && split) e = c.ws.get("umma.ql", sizeof(uint16_t) * umma::YN * TS * (size_t)ntiles, &ql);
  if (e) return e;
  if (!dry) {
    const unsigned blocks = (unsigned)((ntiles * 512 + 255) / 256);
    if (bf) q_split_kernel<true><<<blocks, 256, 0, st>>>(Q, m, S.Npad, ntiles, (uint16_t*)qh, nullptr, active);
    else q_split_kernel<false><<<blocks, 256, 0, st>>>(Q, m, S.Npad, ntiles, (uint16_t*)qh,
                                                       split ? (uint16_t*)ql : nullptr, active);
    count_launch();
    if ((e = cudaGetLastError())) return e;
  }
  TcParams p{};
  p.qh_tiles = (const uint16_t*)qh;
  p.ql_tiles = (const uint16_t*)ql;
  p.xt = T.xs;
  p.Nt = T.N;
  p.Nt_pad = T.Npad;
  p.tctr = T.sb_ctr;
  p.torder = T.sb_order;
  p.tn_exp = T.sb_nexp;
  p.nblk = std::max<int64_t>(1, T.h_sb_nexp);
  p.WB = SB;
  p.xs = S.xs;
  p.Q = Q;
  p.Ns_pad = S.Npad;
  p.m = m;
  p.ntiles = (int)(S.Npad / TS);
  p.tiles_per_split = tiles_per_split;
  p.part = part;
  p.fac = fac;
  p.err = c.d_err;
  p.row_lo = c.row_lo;
  p.row_hi = c.row_hi;
  p.s = S.scale;
  p.active = active;
  switch (T.d) {
    case 1: return umma_dispatch<1>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    case 2: return umma_dispatch<2>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    case 3: return umma_dispatch<3>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    case 4: return umma_dispatch<4>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    case 5: return umma_dispatch<5>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    case 6: return umma_dispatch<6>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    case 7: return umma_dispatch<7>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    case 8: return umma_dispatch<8>(p, splits, split, bf, c.tcgen05_kind, st, dry);
    default: return cudaErrorNotSupported;
  }
}

}  // namespace krr
