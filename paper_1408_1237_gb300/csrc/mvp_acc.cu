// Accurate kernel product for the true residual of the outer solver
// (hot-path step A9: the cycle-start residual and the convergence test of
// Algorithm 1, r = b - K x):
//
//   out_i = cu u_i + cy (sum_j exp(-|x_i - x_j|^2 / (2 sigma^2)) q_j + shift q_i)
//
// The residual of a converged solve is a small difference of large sums, so
// the fast float32 product (relative error ~1e-7 per term) would put a floor
// near the 1e-6 target.  Here every pair that can matter is evaluated in
// float-float arithmetic (about 48-bit significands):
//   * r^2 = sum_k (x_ik - x_jk)^2 from the raw float32 coordinates with exact
//     differences (TwoSum), exact products (FMA error terms) and TwoSum
//     accumulation;
//   * e = -s^2 r^2 with s^2 = log2(e)/(2 sigma^2) split into float hi + lo;
//   * 2^e by Tang's table-driven reduction (ffexp2.h) e = n + k/64 + t,
//     |t| <= 1/128: 2^(k/64) from a 64-entry float-float table, 2^t = 1 + u
//     with u from the Taylor series of exp(t ln 2) to degree 4 (remainder
//     < 1e-13), u itself in float-float; relative error 5e-12 + 2e-7 |el| +
//     (ln 2 el)^2 / 2, below 6e-11 for the terms that matter (a bound
//     tests/test_ffexp2.py checks on the CPU);
//   * q_j (the FP64 iterate) arrives as float hi + lo; each product q_j Phi_ij
//     is split exactly (FMA error term) and summed with TwoSum.
// The Matern kernel of Sec. 6.1 (KF = 1) follows the same scheme: r^2 as
// above; r = sqrt(r^2) in float-float (the correctly rounded square root of
// the high part plus one Newton correction for the remainder); a = s r with
// s = sqrt(3)/h split hi + lo; 2^(-a log2 e) by the same table and series
// (log2 e split hi + lo); then (1 + a) times it in float-float.
// A (warp, source tile) pair whose bounding boxes are farther apart than
// s^2 d^2 > 30 (Gaussian; 625 for the Matern kernel, a > 25) contributes less
// than 2^-30 per term; it takes a plain float32 path into the low-order
// accumulator.  Each source split writes an FP64
// partial per target; the finalize kernel sums splits in fixed order and
// applies the epilogue in FP64 (deterministic).
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "ffexp2.h"
#include "internal.h"

namespace krr {
namespace {

constexpr int NT = 256;
constexpr int NW = NT / 32;
constexpr int RS = 3;
// s^2 dist^2 beyond which a tile is far: Gaussian 2^-30, Matern (1 + a) e^-a < 2^-30
template <int KF>
constexpr float far_e() { return KF == 0 ? 30.f : 625.f; }

struct AccConst : FFExp2Const {
  float s2h, s2l;  // s^2 = s2h + s2l
  float sh, sl;    // s = sh + sl (Matern: sqrt(3) / h)
  float l2eh, l2el;  // log2(e) = l2eh + l2el
};

struct AccParams {
  const float* xs;   // points, tile-blocked SoA (raw), targets = sources
  int64_t N, Npad;
  const float* qh;   // source weights hi (sorted, zero padded)
  const float* ql;   // source weights lo
  const float* tbox; // source tile boxes
  int ntiles, tiles_per_split;
  double* part;      // [columns][splits][Npad]
  int splits;
  int* err;
  // columns (blockIdx.z): qh, ql Npad apart; column c runs when its active
  // word (state_stride bytes after column c-1's) is nonzero
  const int* active;
  size_t state_stride;
  AccConst k;
};

// a - b exactly as s + e (Knuth's TwoSum on a and -b).
__device__ __forceinline__ void two_diff(float a, float b, float& s, float& e) {
  s = a - b;
  const float bb = s - a;
  e = (a - (s - bb)) - (b + bb);
}

// r^2 = sum_k (xi_k - xj_k)^2 as the float-float rh + rl, the differences
// exact (xj: source coordinates, TS apart).
template <int D>
__device__ __forceinline__ void acc_r2(const float (&xi)[D], const float* __restrict__ xj,
                                       float& rh, float& rl) {
  float dh, dl;
  two_diff(xi[0], xj[0], dh, dl);
  rh = dh * dh;
  rl = fmaf(dh, dh, -rh) + 2.f * dh * dl;
#pragma unroll
  for (int c = 1; c < D; ++c) {
    two_diff(xi[c], xj[c * TS], dh, dl);
    const float p = dh * dh;
    const float pe = fmaf(dh, dh, -p) + 2.f * dh * dl;
    float s, e;
    two_sum(rh, p, s, e);
    rh = s;
    rl += e + pe;
  }
}

// 2^(eh + el) as the float-float Hout + Lout (ffexp2.h).
__device__ __forceinline__ void acc_exp2(float eh, float el, const AccConst& k,
                                         const float* __restrict__ tab_h,
                                         const float* __restrict__ tab_l, float& Hout, float& Lout) {
  ff_exp2(eh, el, k, tab_h, tab_l, Hout, Lout);
}

// Kernel value of the pair (xi, xj) as the float-float Hout + Lout:
//   KF = 0: exp2(-s^2 r^2) (the Gaussian);
//   KF = 1: (1 + a) exp2(-a log2 e), a = s r (the Matern kernel, smoothness 3/2).
template <int D, int KF>
__device__ __forceinline__ void acc_kval(const float (&xi)[D], const float* __restrict__ xj,
                                         const AccConst& k, const float* __restrict__ tab_h,
                                         const float* __restrict__ tab_l, float& Hout, float& Lout) {
  float rh, rl;
  acc_r2<D>(xi, xj, rh, rl);
  if constexpr (KF == 0) {
    // e = -(s2h + s2l)(rh + rl)
    const float eh = -k.s2h * rh;
    const float el = fmaf(-k.s2h, rh, -eh) - fmaf(k.s2h, rl, k.s2l * rh);
    acc_exp2(eh, el, k, tab_h, tab_l, Hout, Lout);
  } else {
    // r = sqrt(rh + rl): uh the correctly rounded sqrt(rh), whose remainder
    // rh - uh^2 is exact by FMA; one Newton step gives the low part
    const float uh = __fsqrt_rn(rh);
    const float ul = uh > 0.f ? __fdividef(fmaf(-uh, uh, rh) + rl, 2.f * uh) : 0.f;
    // a = (sh + sl)(uh + ul)
    const float ah = k.sh * uh;
    const float al = fmaf(k.sh, uh, -ah) + fmaf(k.sh, ul, k.sl * uh);
    // e = -(l2eh + l2el)(ah + al)
    const float p = k.l2eh * ah;
    const float eh = -p;
    const float el = -(fmaf(k.l2eh, ah, -p) + fmaf(k.l2eh, al, k.l2el * ah));
    float Eh, El;
    acc_exp2(eh, el, k, tab_h, tab_l, Eh, El);
    // (1 + ah + al)(Eh + El)
    float oh, ol;
    two_sum(1.f, ah, oh, ol);
    ol += al;
    Hout = oh * Eh;
    Lout = fmaf(oh, Eh, -Hout) + fmaf(oh, El, ol * Eh);
  }
}

// Float32 kernel value of a far pair from its squared distance.
template <int KF>
__device__ __forceinline__ float far_value(float r2, const AccConst& k) {
  if constexpr (KF == 0) {
    return ex2(-k.s2h * r2);
  } else {
    const float a = k.sh * (r2 * rsqrtf(fmaxf(r2, 1e-30f)));
    const float e = ex2(-k.l2eh * a);
    return fmaf(a, e, e);
  }
}

// (qh + ql)(H + L2) added into (S, L): the product's high part exactly split
// (FMA error term) and added with TwoSum.
__device__ __forceinline__ void acc_fma(float qh, float ql, float H, float L2, float& S, float& L) {
  const float a = qh * H;
  const float ae = fmaf(qh, H, -a);
  float s, e;
  two_sum(S, a, s, e);
  S = s;
  L += e + ae + fmaf(qh, L2, ql * H);
}

// Accurate q * k(xi, xj) added into (S, L).
template <int D, int KF>
__device__ __forceinline__ void acc_pair(const float (&xi)[D], const float* __restrict__ xj,
                                         float qh, float ql, float& S, float& L,
                                         const AccConst& k, const float* __restrict__ tab_h,
                                         const float* __restrict__ tab_l) {
  float H, L2;
  acc_kval<D, KF>(xi, xj, k, tab_h, tab_l, H, L2);
  acc_fma(qh, ql, H, L2, S, L);
}

template <int D, int TA, int KF>
__global__ void __launch_bounds__(NT) mvp_acc_kernel(const AccParams p) {
  constexpr uint32_t kStageFloats = (D + 2) * TS;  // coordinates, qh, ql
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t bars[RS];
  __shared__ volatile int abort_flag;
  __shared__ float tab_h[64], tab_l[64];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int col = blockIdx.z;
  if (p.active && *(const int*)((const char*)p.active + col * p.state_stride) == 0) return;
  const float* qhc = p.qh + (int64_t)col * p.Npad;
  const float* qlc = p.ql + (int64_t)col * p.Npad;
  if (tid < 64) {
    tab_h[tid] = p.k.th[tid];
    tab_l[tid] = p.k.tl[tid];
  }

  // this warp's targets: 32*TA consecutive sorted points
  const int64_t t0 = ((int64_t)blockIdx.x * NW + warp) * 32 * TA;
  float xi[TA][D];
  bool valid[TA];
#pragma unroll
  for (int u = 0; u < TA; ++u) {
    const int64_t i = t0 + lane + 32 * u;
    valid[u] = i < p.N;
    const int64_t ii = valid[u] ? i : (p.N - 1);
#pragma unroll
    for (int c = 0; c < D; ++c) xi[u][c] = p.xs[(ii / TS) * (int64_t)D * TS + (int64_t)c * TS + ii % TS];
  }
  // warp box (centre, half-width) for the near/far test; above 8
  // dimensions every tile is treated as near (no box registers)
  constexpr bool BOX = D <= 8;
  constexpr int DB = BOX ? D : 1;
  float bc[DB], bh[DB];
  if constexpr (BOX) {
#pragma unroll
    for (int c = 0; c < D; ++c) {
      float lo = xi[0][c], hi = xi[0][c];
#pragma unroll
      for (int u = 1; u < TA; ++u) {
        lo = fminf(lo, xi[u][c]);
        hi = fmaxf(hi, xi[u][c]);
      }
      lo = warp_min(lo);
      hi = warp_max(hi);
      bc[c] = 0.5f * (lo + hi);
      bh[c] = 0.5f * (hi - lo);
    }
  }

  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;
  float S[TA], L[TA];
#pragma unroll
  for (int u = 0; u < TA; ++u) S[u] = L[u] = 0.f;

  auto issue = [&](int r) {
    const int stage = r % RS;
    const int64_t tile = t_begin + r;
    float* dst = smem + stage * kStageFloats;
    mbar_arrive_expect_tx(&bars[stage], kStageFloats * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    bulk_g2s(dst + D * TS, qhc + tile * (int64_t)TS, TS * 4, &bars[stage]);
    bulk_g2s(dst + (D + 1) * TS, qlc + tile * (int64_t)TS, TS * 4, &bars[stage]);
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < RS; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0)
    for (; issued < min(RS, nt); ++issued) issue(issued);
  const float s2h = p.k.s2h;

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
    } else {
      const float* st = smem + (r % RS) * kStageFloats;
      const float* sq = st + D * TS;
      const float* sl = st + (D + 1) * TS;
      // near/far test of this warp's box against the tile's box
      float dist2 = 0.f;
      if constexpr (BOX) {
        const float* tb = p.tbox + (int64_t)(t_begin + r) * 2 * D;
#pragma unroll
        for (int c = 0; c < D; ++c) {
          const float g = fmaxf(0.f, fabsf(bc[c] - tb[c]) - bh[c] - tb[D + c]);
          dist2 = fmaf(g, g, dist2);
        }
      }
      if (s2h * dist2 <= far_e<KF>()) {
#pragma unroll 2
        for (int j = 0; j < TS; ++j) {
          const float qh = sq[j], ql = sl[j];
#pragma unroll
          for (int u = 0; u < TA; ++u)
            acc_pair<D, KF>(xi[u], st + j, qh, ql, S[u], L[u], p.k, tab_h, tab_l);
        }
      } else {
        for (int j = 0; j < TS; ++j) {
          const float qh = sq[j];
#pragma unroll
          for (int u = 0; u < TA; ++u) {
            float r2 = 0.f;
#pragma unroll
            for (int c = 0; c < D; ++c) {
              const float dd = xi[u][c] - st[c * TS + j];
              r2 = fmaf(dd, dd, r2);
            }
            L[u] = fmaf(qh, far_value<KF>(r2, p.k), L[u]);
          }
        }
      }
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
  double* part = p.part + ((int64_t)col * p.splits + blockIdx.y) * p.Npad;
#pragma unroll
  for (int u = 0; u < TA; ++u) {
    const int64_t i = t0 + lane + 32 * u;
    if (valid[u]) part[i] = (double)S[u] + (double)L[u];
  }
}

// Several columns at once: the float-float exponential of a pair is formed
// once and applied to every active column (a near pair costs one
// exponential plus about a dozen operations per column instead of both per
// column).  One target per thread; per column a (S, L) accumulator pair;
// coordinates, qh and ql of up to AM columns per source tile in shared memory
// (RSM-stage TMA ring).  Columns that are inactive (or beyond m) are skipped
// uniformly across the CTA.
constexpr int AM = MAX_COLS;
constexpr int RSM = 2;

template <int D>
constexpr size_t accm_smem_bytes() {
  return sizeof(float) * RSM * (D + 2 * AM) * TS;
}

template <int D, int KF>
__global__ void __launch_bounds__(NT, (D > 8 ? 1 : 2)) mvp_accm_kernel(const AccParams p, int m) {
  constexpr uint32_t kStage = (D + 2 * AM) * TS;
  extern __shared__ __align__(128) float smem[];
  __shared__ __align__(8) uint64_t bars[RSM];
  __shared__ volatile int abort_flag;
  __shared__ float tab_h[64], tab_l[64];
  __shared__ unsigned act_s;
  const int tid = threadIdx.x, lane = tid & 31;
  if (tid < 64) {
    tab_h[tid] = p.k.th[tid];
    tab_l[tid] = p.k.tl[tid];
  }
  if (tid == 0) {
    unsigned a = 0u;
    for (int c = 0; c < m; ++c)
      if (!p.active || *(const int*)((const char*)p.active + c * p.state_stride) != 0) a |= 1u << c;
    act_s = a;
  }
  __syncthreads();
  const unsigned act = act_s;
  if (act == 0u) return;
  int na = 0;  // active columns, packed to the front of each stage
  int cols[AM];
#pragma unroll
  for (int c = 0; c < AM; ++c) cols[c] = 0;
  for (int c = 0; c < m; ++c)
    if (act & (1u << c)) cols[na++] = c;

  const int64_t i = (int64_t)blockIdx.x * NT + tid;
  const bool valid = i < p.N;
  const int64_t ii = valid ? i : (p.N - 1);
  float xi[D];
#pragma unroll
  for (int k = 0; k < D; ++k) xi[k] = p.xs[(ii / TS) * (int64_t)D * TS + (int64_t)k * TS + ii % TS];
  constexpr bool BOX = D <= 8;  // near/far test (above 8 dimensions: all near)
  constexpr int DB = BOX ? D : 1;
  float bc[DB], bh[DB];
  if constexpr (BOX) {
#pragma unroll
    for (int k = 0; k < D; ++k) {
      const float lo = warp_min(xi[k]), hi = warp_max(xi[k]);
      bc[k] = 0.5f * (lo + hi);
      bh[k] = 0.5f * (hi - lo);
    }
  }

  const int t_begin = blockIdx.y * p.tiles_per_split;
  const int nt = min(p.ntiles, t_begin + p.tiles_per_split) - t_begin;
  float S[AM], L[AM];
#pragma unroll
  for (int c = 0; c < AM; ++c) S[c] = L[c] = 0.f;

  auto issue = [&](int r) {
    const int stage = r % RSM;
    const int64_t tile = t_begin + r;
    float* dst = smem + stage * kStage;
    mbar_arrive_expect_tx(&bars[stage], (uint32_t)(D + 2 * na) * TS * 4);
    bulk_g2s(dst, p.xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    for (int a = 0; a < na; ++a) {
      const int64_t off = (int64_t)cols[a] * p.Npad + tile * (int64_t)TS;
      bulk_g2s(dst + (D + a) * TS, p.qh + off, TS * 4, &bars[stage]);
      bulk_g2s(dst + (D + AM + a) * TS, p.ql + off, TS * 4, &bars[stage]);
    }
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int s = 0; s < RSM; ++s) mbar_init(&bars[s], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0)
    for (; issued < min(RSM, nt); ++issued) issue(issued);
  const float s2h = p.k.s2h;

  for (int r = 0; r < nt; ++r) {
    if (tid == 0 && r >= 1 && r - 1 + RSM < nt) {
      fence_proxy_async_smem();
      issue(r - 1 + RSM);
      ++issued;
    }
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[r % RSM], (r / RSM) & 1));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(p.err, DEV_TIMEOUT);
    } else {
      const float* st = smem + (r % RSM) * kStage;
      const float* sq = st + D * TS;
      const float* sl = st + (D + AM) * TS;
      float dist2 = 0.f;
      if constexpr (BOX) {
        const float* tb = p.tbox + (int64_t)(t_begin + r) * 2 * D;
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float g = fmaxf(0.f, fabsf(bc[k] - tb[k]) - bh[k] - tb[D + k]);
          dist2 = fmaf(g, g, dist2);
        }
      }
      if (s2h * dist2 <= far_e<KF>()) {
#pragma unroll 1
        for (int j = 0; j < TS; ++j) {
          float H, L2;
          acc_kval<D, KF>(xi, st + j, p.k, tab_h, tab_l, H, L2);
#pragma unroll
          for (int a = 0; a < AM; ++a)
            if (a < na) acc_fma(sq[a * TS + j], sl[a * TS + j], H, L2, S[a], L[a]);
        }
      } else {
#pragma unroll 1
        for (int j = 0; j < TS; ++j) {
          float r2 = 0.f;
#pragma unroll
          for (int k = 0; k < D; ++k) {
            const float dd = xi[k] - st[k * TS + j];
            r2 = fmaf(dd, dd, r2);
          }
          const float E = far_value<KF>(r2, p.k);
#pragma unroll
          for (int a = 0; a < AM; ++a)
            if (a < na) L[a] = fmaf(sq[a * TS + j], E, L[a]);
        }
      }
    }
    __syncthreads();
    if (abort_flag) break;
  }
  if (abort_flag) {
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % RSM], (r / RSM) & 1);
    __syncthreads();
    return;
  }
  if (valid) {
#pragma unroll
    for (int a = 0; a < AM; ++a)
      if (a < na)
        p.part[((int64_t)cols[a] * p.splits + blockIdx.y) * p.Npad + i] = (double)S[a] + (double)L[a];
  }
}

struct AccFin {
  const double* part;
  int splits;
  int64_t N, Npad;
  const float* qh;
  const float* ql;
  double shift, cu, cy;
  const float* u;
  double* out;
  double* dot;
  double* dot_part;
  unsigned* dot_count;
  const int* active;
  size_t state_stride;
};

__global__ void __launch_bounds__(256) acc_finalize_kernel(const AccFin f) {
  __shared__ double red[8];
  __shared__ bool is_last;
  const int col = blockIdx.y;
  if (f.active && *(const int*)((const char*)f.active + col * f.state_stride) == 0) return;
  const int64_t cv = (int64_t)col * f.Npad;
  const double* part = f.part + cv * f.splits;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double o = 0.0;
  if (i < f.N) {
    double y = 0.0;
    for (int s = 0; s < f.splits; ++s) y += part[(int64_t)s * f.Npad + i];
    y += f.shift * ((double)f.qh[cv + i] + (double)f.ql[cv + i]);
    o = f.cy * y;
    if (f.u) o += f.cu * (double)f.u[cv + i];
  }
  if (i < f.Npad) f.out[cv + i] = o;
  if (f.dot) {
    double* dot_part = f.dot_part + (int64_t)col * gridDim.x;
    const double bs = block_sum(o * o, red);
    if (threadIdx.x == 0) {
      dot_part[blockIdx.x] = bs;
      __threadfence();
      is_last = atomicAdd(f.dot_count + col, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (is_last) {
      __threadfence();
      double t = 0.0;
      for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += dot_part[b];
      t = block_sum(t, red);
      if (threadIdx.x == 0) {
        *(double*)((char*)f.dot + col * f.state_stride) = t;
        f.dot_count[col] = 0u;
      }
    }
  }
}

// log2(e) in float-float, and the constants of the float-float 2^x.
AccConst make_consts() {
  AccConst k;
  ff_exp2_consts(k);
  const double ln2 = std::log(2.0);
  k.l2eh = (float)(1.0 / ln2);
  k.l2el = (float)(1.0 / ln2 - (double)k.l2eh);
  return k;
}

template <int D, int TA, int KF>
cudaError_t set_acc_attr() {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && done[dev]) return cudaSuccess;
  const size_t shm = sizeof(float) * RS * (D + 2) * TS;
  cudaError_t e = cudaFuncSetAttribute(mvp_acc_kernel<D, TA, KF>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm);
  if (!e && dev < 128) done[dev] = true;
  return e;
}

// Single-column accurate product (launch = false: only its attribute).
template <int D, int TA, int KF>
cudaError_t launch_acc(const AccParams& p, int splits, int ncols, cudaStream_t st, bool launch) {
  const size_t shm = sizeof(float) * RS * (D + 2) * TS;
  cudaError_t e = set_acc_attr<D, TA, KF>();
  if (e || !launch) return e;
  dim3 grid((unsigned)((p.N + NT * TA - 1) / (NT * TA)), (unsigned)splits, (unsigned)ncols);
  mvp_acc_kernel<D, TA, KF><<<grid, NT, shm, st>>>(p); count_launch();
  return cudaGetLastError();
}

constexpr int ACC_TA = 2;

template <int KF>
cudaError_t launch_acc_d(const AccParams& p, int d, int splits, int ncols, cudaStream_t st,
                         bool launch) {
  switch (d) {
    case 1: return launch_acc<1, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 2: return launch_acc<2, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 3: return launch_acc<3, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 4: return launch_acc<4, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 5: return launch_acc<5, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 6: return launch_acc<6, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 7: return launch_acc<7, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 8: return launch_acc<8, ACC_TA, KF>(p, splits, ncols, st, launch);
    case 16: return launch_acc<16, 1, KF>(p, splits, ncols, st, launch);
    case 32: return launch_acc<32, 1, KF>(p, splits, ncols, st, launch);
    case 48: return launch_acc<48, 1, KF>(p, splits, ncols, st, launch);
    case 64: return launch_acc<64, 1, KF>(p, splits, ncols, st, launch);
    default: return cudaErrorNotSupported;
  }
}

template <int D, int KF>
cudaError_t accm_attr_typed() {
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && done[dev]) return cudaSuccess;
  cudaError_t e = cudaFuncSetAttribute(mvp_accm_kernel<D, KF>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)accm_smem_bytes<D>());
  if (!e && dev < 128) done[dev] = true;
  return e;
}

// Multi-column accurate product (launch = false: only its attribute).
template <int D, int KF>
cudaError_t launch_accm_typed(const AccParams& p, int splits, int ncols, cudaStream_t st, bool launch) {
  cudaError_t e = accm_attr_typed<D, KF>();
  if (e || !launch) return e;
  dim3 grid((unsigned)((p.N + NT - 1) / NT), (unsigned)splits);
  mvp_accm_kernel<D, KF><<<grid, NT, accm_smem_bytes<D>(), st>>>(p, ncols); count_launch();
  return cudaGetLastError();
}

template <int KF>
cudaError_t launch_accm_d(const AccParams& p, int d, int splits, int ncols, cudaStream_t st,
                          bool launch) {
  switch (d) {
    case 1: return launch_accm_typed<1, KF>(p, splits, ncols, st, launch);
    case 2: return launch_accm_typed<2, KF>(p, splits, ncols, st, launch);
    case 3: return launch_accm_typed<3, KF>(p, splits, ncols, st, launch);
    case 4: return launch_accm_typed<4, KF>(p, splits, ncols, st, launch);
    case 5: return launch_accm_typed<5, KF>(p, splits, ncols, st, launch);
    case 6: return launch_accm_typed<6, KF>(p, splits, ncols, st, launch);
    case 7: return launch_accm_typed<7, KF>(p, splits, ncols, st, launch);
    case 8: return launch_accm_typed<8, KF>(p, splits, ncols, st, launch);
    case 16: return launch_accm_typed<16, KF>(p, splits, ncols, st, launch);
    case 32: return launch_accm_typed<32, KF>(p, splits, ncols, st, launch);
    case 48: return launch_accm_typed<48, KF>(p, splits, ncols, st, launch);
    case 64: return launch_accm_typed<64, KF>(p, splits, ncols, st, launch);
    default: return cudaErrorNotSupported;
  }
}

// The accurate product's kernel for the points' kernel family and column
// count (launch = false: only the shared-memory attribute).
cudaError_t launch_any(const AccParams& p, int d, int kf, int splits, int ncols, cudaStream_t st,
                       bool launch) {
  if (kf == KRR_KERNEL_MATERN32)
    return ncols > 1 ? launch_accm_d<1>(p, d, splits, ncols, st, launch)
                     : launch_acc_d<1>(p, d, splits, ncols, st, launch);
  if (kf != KRR_KERNEL_GAUSSIAN) return cudaErrorNotSupported;
  return ncols > 1 ? launch_accm_d<0>(p, d, splits, ncols, st, launch)
                   : launch_acc_d<0>(p, d, splits, ncols, st, launch);
}

struct AccPlan {
  int splits, tiles_per_split;
};

// scale: the autotuner's factor on the modelled split count (1: the model).
AccPlan acc_plan(const PointsDev& P, int num_sms, int plan_slots, int ncols, double scale) {
  const int ntiles = (int)(P.Npad / TS);
  // one target per thread in the multi-column kernel, ACC_TA otherwise
  const int ta = (ncols > 1 || P.d > 8) ? 1 : ACC_TA;
  const int64_t ctas = (P.N + NT * ta - 1) / (NT * ta);
  const int slots = plan_slots > 0 ? plan_slots : num_sms * 2;
  // fill the GPU about four times over, never below one tile per split
  int splits = (int)std::min<int64_t>(ntiles, std::max<int64_t>(1, (4LL * slots + ctas - 1) / ctas));
  if (scale != 1.0) splits = std::max(1, std::min({(int)std::lround(splits * scale), ntiles, 256}));
  AccPlan pl;
  pl.tiles_per_split = (ntiles + splits - 1) / splits;
  pl.splits = (ntiles + pl.tiles_per_split - 1) / pl.tiles_per_split;
  return pl;
}

// The autotuner of the accurate product (see autotune_mvp in mvp.cu): the
// real launch on scratch zero weights at each split scale, fastest kept.
cudaError_t autotune_acc(Ctx& c, const PointsDev& P, int ncols, cudaStream_t st, const std::string& key) {
  struct Restore {
    Ctx& c;
    ~Restore() { c.tuning = false; }
  } restore{c};
  c.tuning = true;
  void *qv, *yv;
  cudaError_t e;
  if ((e = c.ws.get("tune.aq", sizeof(float) * (size_t)ncols * P.Npad, &qv))) return e;
  if ((e = c.ws.get("tune.ay", sizeof(double) * (size_t)ncols * P.Npad, &yv))) return e;
  if ((e = cudaMemsetAsync(qv, 0, sizeof(float) * (size_t)ncols * P.Npad, st))) return e;
  cudaEvent_t ev[2];
  if ((e = cudaEventCreate(&ev[0]))) return e;
  if ((e = cudaEventCreate(&ev[1]))) {
    cudaEventDestroy(ev[0]);
    return e;
  }
  AccCols cols;
  cols.n = ncols;
  double best = 1.0;
  float best_ms = -1.f;
  for (double s : TUNE_SCALES) {
    c.tune_cache[key] = s;
    if (s > 1.0 &&
        8.0 * acc_plan(P, c.num_sms, c.plan_slots, ncols, s).splits * ncols * (double)P.Npad > TUNE_MAX_BYTES)
      continue;
    auto run = [&]() {
      return mvp_acc_launch(c, P, (const float*)qv, (const float*)qv, 0.f, 0.0, nullptr, 1.0, (double*)yv,
                            nullptr, st, cols);
    };
    if ((e = run())) break;
    float ms = 1e30f;
    for (int rep = 0; rep < 2 && !e; ++rep) {
      cudaEventRecord(ev[0], st);
      e = run();
      cudaEventRecord(ev[1], st);
      if (!e) e = cudaEventSynchronize(ev[1]);
      float t = 0.f;
      if (!e) cudaEventElapsedTime(&t, ev[0], ev[1]);
      ms = std::min(ms, t);
    }
    if (e) break;
    if (best_ms < 0.f || ms < 0.98f * best_ms) {
      best_ms = ms;
      best = s;
    }
  }
  cudaEventDestroy(ev[0]);
  cudaEventDestroy(ev[1]);
  c.tune_cache[key] = e ? 1.0 : best;
  return e;
}

}  // namespace

cudaError_t mvp_acc_reserve(Ctx& c, const PointsDev& P, cudaStream_t st, int ncols) {
  if (P.N == 0) return cudaSuccess;
  if (ncols < 1 || ncols > MAX_COLS) return cudaErrorNotSupported;
  const std::string key = tune_key(c, "acc", P, P, ncols, KRR_FP32);
  if (can_tune(c, st) && !c.tune_cache.count(key)) {
    cudaError_t te = autotune_acc(c, P, ncols, st, key);
    if (te) return te;
  }
  TuneScope scope(c, tuned_scale(c, key));
  const AccPlan pl = acc_plan(P, c.num_sms, c.plan_slots, ncols, c.split_scale);
  void* v;
  cudaError_t e;
  if ((e = c.ws.get("acc.part", sizeof(double) * ncols * pl.splits * (size_t)P.Npad, &v))) return e;
  const unsigned fin_blocks = (unsigned)((P.Npad + 255) / 256);
  if ((e = c.ws.get("acc.dotpart", sizeof(double) * MAX_COLS * fin_blocks, &v))) return e;
  const bool fresh = c.ws.slots.find("acc.dotcnt") == c.ws.slots.end();
  if ((e = c.ws.get("acc.dotcnt", sizeof(unsigned) * MAX_COLS, &v))) return e;
  if (fresh && (e = cudaMemsetAsync(v, 0, sizeof(unsigned) * MAX_COLS, st))) return e;
  AccParams p{};
  return launch_any(p, P.d, P.kfam, pl.splits, ncols, st, false);
}

cudaError_t mvp_acc_launch(Ctx& c, const PointsDev& P, const float* qh, const float* ql,
                           float shift, double cu, const float* u, double cy, double* out,
                           double* dot, cudaStream_t st, const AccCols& cols) {
  if (P.N == 0) return cudaSuccess;
  const int ncols = cols.n;
  const std::string key = tune_key(c, "acc", P, P, ncols, KRR_FP32);
  if (can_tune(c, st) && !c.tune_cache.count(key)) {
    cudaError_t te = autotune_acc(c, P, ncols, st, key);
    if (te) return te;
  }
  TuneScope scope(c, tuned_scale(c, key));
  cudaError_t e = mvp_acc_reserve(c, P, st, ncols);
  if (e) return e;
  AccParams p{};
  p.xs = P.xs;
  p.N = P.N;
  p.Npad = P.Npad;
  p.qh = qh;
  p.ql = ql;
  p.tbox = P.tbox;
  p.ntiles = (int)(P.Npad / TS);
  p.err = c.d_err;
  p.k = make_consts();
  // s^2 (Gaussian: log2(e) / (2 sigma^2); Matern: 3 / h^2) and s in
  // float-float from the double values
  p.k.s2h = (float)P.s2;
  p.k.s2l = (float)(P.s2 - (double)p.k.s2h);
  const double sd = std::sqrt(P.s2);
  p.k.sh = (float)sd;
  p.k.sl = (float)(sd - (double)p.k.sh);
  const AccPlan pl = acc_plan(P, c.num_sms, c.plan_slots, ncols, c.split_scale);
  p.tiles_per_split = pl.tiles_per_split;
  p.splits = pl.splits;
  p.active = cols.active;
  p.state_stride = cols.state_stride;
  void *part, *dpart, *dcnt;
  const unsigned fin_blocks = (unsigned)((P.Npad + 255) / 256);
  if ((e = c.ws.get("acc.part", sizeof(double) * ncols * pl.splits * (size_t)P.Npad, &part))) return e;
  if ((e = c.ws.get("acc.dotpart", sizeof(double) * MAX_COLS * fin_blocks, &dpart))) return e;
  if ((e = c.ws.get("acc.dotcnt", sizeof(unsigned) * MAX_COLS, &dcnt))) return e;
  p.part = (double*)part;
  e = launch_any(p, P.d, P.kfam, pl.splits, ncols, st, true);
  if (e) return e;
  AccFin f{};
  f.part = p.part;
  f.splits = pl.splits;
  f.N = P.N;
  f.Npad = P.Npad;
  f.qh = qh;
  f.ql = ql;
  f.shift = shift;
  f.cu = cu;
  f.cy = cy;
  f.u = u;
  f.out = out;
  f.dot = dot;
  f.dot_part = (double*)dpart;
  f.dot_count = (unsigned*)dcnt;
  f.active = cols.active;
  f.state_stride = cols.state_stride;
  acc_finalize_kernel<<<dim3(fin_blocks, (unsigned)ncols), 256, 0, st>>>(f); count_launch();
  return cudaGetLastError();
}

}  // namespace krr
