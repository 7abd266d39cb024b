// Gradient of the GP log-marginal likelihood (hot-path step A12; the
// maximum-likelihood fit of sigma and gamma that Sec. 2.1 and Sec. 6.1 call
// for, which the paper does not spell out):
//
//   L = -1/2 y^T K^-1 y - 1/2 log det K - N/2 log 2 pi,   K = K_hat + gamma I
//   dL/dtheta = 1/2 alpha^T (dK/dtheta) alpha - 1/2 tr(K^-1 dK/dtheta)
//
// with alpha = K^-1 y and the Hutchinson estimate K^-1 ~ (1/P) sum_p u_p z_p^T,
// u_p = K^-1 z_p, z_p Rademacher.  With W = 1/2 (alpha alpha^T - (1/P) U Z^T)
// and w_ij = W_ij + W_ji:
//
//   dL/dlog sigma = (1 / (2 sigma^2)) sum_i H_i,  H_i = sum_j w_ij Phi_ij r_ij^2
//   dL/dlog gamma = gamma tr(W)
//   dL/dx_i       = -(1 / sigma^2) G_i,          G_i = sum_j w_ij Phi_ij (x_i - x_j)
//
// w has rank 2P + 1: w_ij = sum_c a_ci b_cj over (alpha, alpha),
// (u_p, -z_p / 2P) and (z_p, -u_p / 2P).  The adjoint kernel computes, for
// each weight column b_c, the fused sums
//
//   A_ci = sum_j Phi_ij b_cj (x_i - x_j)   (d values)
//   R_ci = sum_j Phi_ij b_cj r_ij^2
//
// straight from the pair differences (no expansion of r^2, which would lose
// (|x|/sigma)^2 digits to cancellation); then G_i = sum_c a_ci A_ci and
// H_i = sum_c a_ci R_ci.  The solves use FGMRES with the paper's
// preconditioner.
#include <algorithm>
#include <cmath>
#include <vector>

#include "api_util.h"
#include "common.cuh"
#include "internal.h"

namespace krr {
namespace {

// SplitMix64 (Steele, Lea and Flood 2014): output number c+1 of the stream
// started from `seed`, used as a counter-based generator.
__device__ __forceinline__ uint64_t splitmix64(uint64_t seed, uint64_t c) {
  uint64_t z = seed + (c + 1) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// B (original order, N x (1 + P) column-major): column 0 = y, column 1 + p =
// Rademacher probe p, element (i, p) = -1 when the top bit of output
// p*N + i + 1 is set.
__global__ void rhs_kernel(const float* __restrict__ y, int64_t N, int P, uint64_t seed,
                           float* __restrict__ B) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < N * (1 + (int64_t)P);
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t col = e / N, i = e % N;
    if (col == 0) {
      B[i] = y[i];
    } else {
      const uint64_t r = splitmix64(seed, (uint64_t)(col - 1) * (uint64_t)N + (uint64_t)i);
      B[e] = (r >> 63) ? -1.f : 1.f;
    }
  }
}

// Weight columns in sorted order, one per weight vector c: alpha (c = 0),
// z_p (c = p), u_p (c = P + p).  Solutions Sol are FP64 original order
// (column 0 alpha, 1 + p: u_p); probes come from B.
__global__ void weights_kernel(const double* __restrict__ Sol, const float* __restrict__ B,
                               const int* __restrict__ perm, int64_t N, int64_t Np, int P,
                               float* __restrict__ WC) {
  const int ncols = 2 * P + 1;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const bool v = i < N;
    const int64_t oi = v ? perm[i] : 0;
    for (int c = 0; c < ncols; ++c) {
      float b = 0.f;
      if (v) {
        if (c == 0) b = (float)Sol[oi];
        else if (c <= P) b = B[(int64_t)c * N + oi];             // z_p
        else b = (float)Sol[(int64_t)(c - P) * N + oi];          // u_p
      }
      WC[(int64_t)c * Np + i] = b;
    }
  }
}

constexpr int ADJ_NT = 256;   // threads: one target each
constexpr int ADJ_RS = 2;     // raw stages

// Weight columns per pass and dimensions per pass: up to 8 dimensions all in
// one pass with 4 columns; above 8, passes over 8-dimension chunks with 2
// columns (each pass forms the full distance again).
template <int D>
constexpr int adj_mc() { return D <= 8 ? 4 : 2; }
template <int D>
constexpr int adj_dc() { return D <= 8 ? D : 8; }
template <int D>
constexpr size_t adj_smem() { return sizeof(float) * ADJ_RS * (D + adj_mc<D>()) * TS; }

// Adjoint sums for adj_mc weight columns starting at c0 and the dimensions
// k0 .. k0 + adj_dc - 1: for target i, out[(c * (D+1) + k) * Np + i] =
// sum_j Phi_ij b_cj (x_ik - x_jk), and (pass k0 = 0) out[(c * (D+1) + D) *
// Np + i] = sum_j Phi_ij b_cj r_ij^2, over this split's source tiles; float32
// per tile, Kahan-folded, FP64 partial per split.
template <int D>
__global__ void __launch_bounds__(ADJ_NT)
    adjoint_kernel(const float* __restrict__ xs, int64_t N, int64_t Np, const float* __restrict__ WC,
                   int c0, int mcols, float s2, int tiles_per_split, int ntiles,
                   double* __restrict__ out, int64_t split_stride, int* err, int k0) {
  constexpr int MC = adj_mc<D>();
  constexpr int DC = adj_dc<D>();
  constexpr int NO = MC * (DC + 1);
  constexpr int RAW = (D + MC) * TS;
  extern __shared__ __align__(128) float raw_dyn[];
  __shared__ __align__(8) uint64_t bars[ADJ_RS];
  __shared__ volatile int abort_flag;
  const int tid = threadIdx.x, lane = tid & 31;
  const int64_t i = (int64_t)blockIdx.x * ADJ_NT + tid;
  const int64_t ii = i < N ? i : N - 1;
  const bool with_r2 = k0 == 0;
  const int kc = k0 / DC;  // this pass's chunk of dimensions
  float xi[D];
#pragma unroll
  for (int k = 0; k < D; ++k) xi[k] = xs[(ii / TS) * (int64_t)D * TS + (int64_t)k * TS + ii % TS];
  float S[NO], C[NO], acc[NO];
#pragma unroll
  for (int o = 0; o < NO; ++o) S[o] = C[o] = acc[o] = 0.f;
  const int t_begin = blockIdx.y * tiles_per_split;
  const int nt = min(ntiles, t_begin + tiles_per_split) - t_begin;
  auto issue = [&](int r) {
    const int stage = r % ADJ_RS;
    const int64_t tile = t_begin + r;
    float* dst = raw_dyn + stage * RAW;
    mbar_arrive_expect_tx(&bars[stage], RAW * 4);
    bulk_g2s(dst, xs + tile * (int64_t)D * TS, D * TS * 4, &bars[stage]);
    for (int c = 0; c < MC; ++c) {
      const int cc = c0 + (c < mcols ? c : 0);  // unused slots reload column c0 (weights ignored)
      bulk_g2s(dst + (D + c) * TS, WC + (int64_t)cc * Np + tile * (int64_t)TS, TS * 4, &bars[stage]);
    }
  };
  if (tid == 0) {
    abort_flag = 0;
    for (int st = 0; st < ADJ_RS; ++st) mbar_init(&bars[st], 1);
    fence_barrier_init();
  }
  __syncthreads();
  int issued = 0;
  if (tid == 0)
    for (; issued < min(ADJ_RS, nt); ++issued) issue(issued);
  for (int r = 0; r < nt; ++r) {
    const bool ok = __all_sync(0xffffffffu, mbar_wait_bounded(&bars[r % ADJ_RS], (r / ADJ_RS) & 1));
    if (!ok) {
      abort_flag = 1;
      if (lane == 0) atomicExch(err, DEV_TIMEOUT);
    } else {
      const float* rs = raw_dyn + (r % ADJ_RS) * RAW;
      for (int j = 0; j < TS; ++j) {
        // full distance, and the differences of this pass's dimensions (kept
        // at compile-time register indices: chunk kc of 8 selected at run time)
        float r2 = 0.f;
        float dc[DC];
#pragma unroll
        for (int k = 0; k < D; ++k) {
          const float dk = xi[k] - rs[k * TS + j];
          r2 = fmaf(dk, dk, r2);
          if (DC == D) dc[k % DC] = dk;
          else if (k / DC == kc) dc[k % DC] = dk;
        }
        const float phi = ex2(-s2 * r2);
#pragma unroll
        for (int c = 0; c < MC; ++c) {
          const float w = (c < mcols) ? phi * rs[(D + c) * TS + j] : 0.f;
#pragma unroll
          for (int k = 0; k < DC; ++k) acc[c * (DC + 1) + k] = fmaf(w, dc[k], acc[c * (DC + 1) + k]);
          acc[c * (DC + 1) + DC] = fmaf(w, r2, acc[c * (DC + 1) + DC]);
        }
      }
#pragma unroll
      for (int o = 0; o < NO; ++o) {
        kahan_add(S[o], C[o], acc[o]);
        acc[o] = 0.f;
      }
    }
    __syncthreads();  // every thread is done with stage r % ADJ_RS
    if (abort_flag) break;
    if (tid == 0 && r + ADJ_RS < nt) {
      fence_proxy_async_smem();
      issue(r + ADJ_RS);
      ++issued;
    }
  }
  if (abort_flag) {
    if (tid == 0)
      for (int r = 0; r < issued; ++r) mbar_wait_bounded(&bars[r % ADJ_RS], (r / ADJ_RS) & 1);
    __syncthreads();
    return;
  }
  if (i < N) {
    double* o = out + (int64_t)blockIdx.y * split_stride;
#pragma unroll
    for (int c = 0; c < MC; ++c) {
      if (c >= mcols) break;
#pragma unroll
      for (int k = 0; k < DC; ++k)
        if (k0 + k < D)
          o[((int64_t)(c0 + c) * (D + 1) + k0 + k) * Np + i] =
              (double)S[c * (DC + 1) + k] - (double)C[c * (DC + 1) + k];
      if (with_r2)
        o[((int64_t)(c0 + c) * (D + 1) + D) * Np + i] =
            (double)S[c * (DC + 1) + DC] - (double)C[c * (DC + 1) + DC];
    }
  }
}

struct GradAcc {
  double h, aa, uz;
  unsigned ticket;
};

// Combine the adjoint sums into G_i, H_i; dX (original order) = -G / sigma^2;
// fixed-order grid sums of H, alpha^2 and u.z.  A holds `splits` partial
// copies of the (2P+1)(d+1) output columns.
__global__ void combine_kernel(const double* __restrict__ A, int splits, int64_t split_stride,
                               const float* __restrict__ WC, const int* __restrict__ perm,
                               int64_t N, int64_t Np, int d, int d_out, int P, double inv_s2,
                               float* __restrict__ dX, double* partials, GradAcc* acc) {
  __shared__ double red[8];
  __shared__ bool is_last;
  const int ncols = 2 * P + 1;
  double h_loc = 0.0, aa_loc = 0.0, uz_loc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double G[64];
    for (int k = 0; k < d; ++k) G[k] = 0.0;
    double H = 0.0;
    for (int c = 0; c < ncols; ++c) {
      // a_c for target i: alpha (c = 0); u_p for the z_p columns; z_p for the
      // u_p columns; the probe terms carry -1/(2P)
      double a;
      if (c == 0) a = WC[i];
      else if (c <= P) a = -0.5 / P * (double)WC[(int64_t)(c + P) * Np + i];
      else a = -0.5 / P * (double)WC[(int64_t)(c - P) * Np + i];
      for (int k = 0; k <= d; ++k) {
        double v = 0.0;
        for (int sp = 0; sp < splits; ++sp) v += A[sp * split_stride + ((int64_t)c * (d + 1) + k) * Np + i];
        if (k < d) G[k] += a * v;
        else H += a * v;
      }
    }
    const int64_t oi = perm[i];
    for (int k = 0; k < d_out; ++k) dX[oi * d_out + k] = (float)(-G[k] * inv_s2);
    h_loc += H;
    const double al = WC[i];
    aa_loc += al * al;
    for (int p = 1; p <= P; ++p)
      uz_loc += (double)WC[(int64_t)(p + P) * Np + i] * (double)WC[(int64_t)p * Np + i];
  }
  const double bh = block_sum(h_loc, red);
  const double ba = block_sum(aa_loc, red);
  const double bu = block_sum(uz_loc, red);
  if (threadIdx.x == 0) {
    partials[3 * blockIdx.x] = bh;
    partials[3 * blockIdx.x + 1] = ba;
    partials[3 * blockIdx.x + 2] = bu;
    __threadfence();
    is_last = atomicAdd(&acc->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    __threadfence();
    double th = 0.0, ta = 0.0, tu = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
      th += partials[3 * b];
      ta += partials[3 * b + 1];
      tu += partials[3 * b + 2];
    }
    acc->h = th;
    acc->aa = ta;
    acc->uz = tu;
    acc->ticket = 0u;
  }
}

template <int D>
cudaError_t launch_adjoint(const PointsDev& Pt, const float* WC, int ncols, int splits,
                           int tiles_per_split, double* out, int64_t split_stride, int* err,
                           cudaStream_t st) {
  constexpr int MC = adj_mc<D>(), DC = adj_dc<D>();
  static bool done[128] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 128 && !done[dev]) {
    cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)adj_smem<D>());
    if (e) return e;
    done[dev] = true;
  }
  const dim3 grid((unsigned)((Pt.N + ADJ_NT - 1) / ADJ_NT), (unsigned)splits);
  const float s2 = (float)Pt.s2;
  for (int c0 = 0; c0 < ncols; c0 += MC)
    for (int k0 = 0; k0 < D; k0 += DC) {
      adjoint_kernel<D><<<grid, ADJ_NT, adj_smem<D>(), st>>>(Pt.xs, Pt.N, Pt.Npad, WC, c0,
                                                             std::min(MC, ncols - c0), s2, tiles_per_split,
                                                             (int)(Pt.Npad / TS), out, split_stride, err, k0);
      count_launch();
      cudaError_t e = cudaGetLastError();
      if (e) return e;
    }
  return cudaSuccess;
}

}  // namespace
}  // namespace krr

using namespace krr;

extern "C" krr_status krr_mll_grad(krr_handle h, const float* X, int64_t N, int d, float sigma,
                                   float gamma, const float* y, int n_probes, uint64_t seed,
                                   const krr_fgmres_opts* opts, double* dlogsigma,
                                   double* dloggamma, float* dX, krr_solve_info* info,
                                   void* stream) {
  NvtxRange nvtx_range("krr_mll_grad");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_mll_grad";
  if (c.kernel_family != KRR_KERNEL_GAUSSIAN)
    return set_error(c, KRR_ERR_UNIMPLEMENTED, "%s: the gradient is built for the Gaussian kernel only", fn);
  krr_status s = check_points(c, fn, X, N, d, sigma);
  if (s) return s;
  if (!(gamma > 0.f) || !std::isfinite(gamma))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: gamma must be finite and > 0", fn);
  if (n_probes < 1 || n_probes > 256)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: n_probes out of range [1, 256]", fn);
  if (!dlogsigma || !dloggamma) return set_error(c, KRR_ERR_INVALID_ARG, "%s: scalar outputs are NULL", fn);
  if (N == 0) {
    *dlogsigma = *dloggamma = 0.0;
    return KRR_OK;
  }
  if (!y) return set_error(c, KRR_ERR_INVALID_ARG, "%s: y is NULL", fn);
  cudaStream_t st = (cudaStream_t)stream;
  const int P = n_probes, nrhs = 1 + P, ncols = 2 * P + 1;
  float *dXin, *dy, *ddX = nullptr;
  bool sX, sy, sdX = false;
  if ((s = device_view(c, "stage.X", X, (size_t)N * d, true, st, &dXin, &sX))) return s;
  if ((s = device_view(c, "stage.y", y, (size_t)N, true, st, &dy, &sy))) return s;
  if (dX && (s = device_view(c, "stage.dX", dX, (size_t)N * d, false, st, &ddX, &sdX))) return s;
  void *Bv, *Solv;
  cudaError_t e;
  if ((e = c.ws.get("mll.B", sizeof(float) * (size_t)N * nrhs, &Bv))) return cuda_error(c, e, fn);
  if ((e = c.ws.get("mll.sol", sizeof(double) * (size_t)N * nrhs, &Solv))) return cuda_error(c, e, fn);
  float* B = (float*)Bv;
  double* Sol = (double*)Solv;
  const unsigned vb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((N * nrhs + 255) / 256, 4LL * c.num_sms));
  rhs_kernel<<<vb, 256, 0, st>>>(dy, N, P, seed, B); count_launch();
  // alpha = K^-1 y, u_p = K^-1 z_p
  std::vector<krr_solve_info> infos(nrhs);
  krr_status ss = krr_fgmres_solve(h, dXin, N, d, sigma, gamma, B, nrhs, Sol, opts, infos.data(), st);
  if (info)
    for (int k = 0; k < nrhs; ++k) info[k] = infos[k];
  if (ss != KRR_OK && ss != KRR_NOT_CONVERGED) return ss;
  // adjoint sums
  PointsDev Pt;
  if ((e = prepare_points(c, dXin, N, d, sigma, "mll.pts", Pt, st))) return cuda_error(c, e, fn);
  const int ntiles = (int)(Pt.Npad / TS);
  const int64_t ctas = (N + ADJ_NT - 1) / ADJ_NT;
  int splits = (int)std::min<int64_t>(ntiles, std::max<int64_t>(1, (2LL * c.num_sms + ctas - 1) / ctas));
  const int tps = (ntiles + splits - 1) / splits;
  splits = (ntiles + tps - 1) / tps;
  const int64_t split_stride = (int64_t)ncols * (Pt.d + 1) * Pt.Npad;  // prepared (padded) dimension
  void *WCv, *Av, *partv, *accv;
  if ((e = c.ws.get("mll.wc", sizeof(float) * (size_t)ncols * Pt.Npad, &WCv))) return cuda_error(c, e, fn);
  if ((e = c.ws.get("mll.adj", sizeof(double) * (size_t)splits * split_stride, &Av))) return cuda_error(c, e, fn);
  if ((e = c.ws.get("mll.part", sizeof(double) * 3 * 1024, &partv))) return cuda_error(c, e, fn);
  const bool fresh = c.ws.slots.find("mll.acc") == c.ws.slots.end();
  if ((e = c.ws.get("mll.acc", sizeof(GradAcc), &accv))) return cuda_error(c, e, fn);
  if (fresh && (e = cudaMemsetAsync(accv, 0, sizeof(GradAcc), st))) return cuda_error(c, e, fn);
  float* WC = (float*)WCv;
  double* A = (double*)Av;
  const unsigned pb = (unsigned)std::max<int64_t>(1, std::min<int64_t>((Pt.Npad + 255) / 256, 1024));
  weights_kernel<<<pb, 256, 0, st>>>(Sol, B, Pt.perm, N, Pt.Npad, P, WC); count_launch();
  switch (Pt.d) {
    case 1: e = launch_adjoint<1>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 2: e = launch_adjoint<2>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 3: e = launch_adjoint<3>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 4: e = launch_adjoint<4>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 5: e = launch_adjoint<5>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 6: e = launch_adjoint<6>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 7: e = launch_adjoint<7>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 8: e = launch_adjoint<8>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 16: e = launch_adjoint<16>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 32: e = launch_adjoint<32>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 48: e = launch_adjoint<48>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    case 64: e = launch_adjoint<64>(Pt, WC, ncols, splits, tps, A, split_stride, c.d_err, st); break;
    default: e = cudaErrorNotSupported; break;
  }
  if (e) return cuda_error(c, e, fn);
  const double inv_s2 = 1.0 / ((double)sigma * (double)sigma);
  float* dXout = ddX;
  void* dummy = nullptr;
  if (!dXout) {
    if ((e = c.ws.get("mll.dxdummy", sizeof(float) * (size_t)N * d, &dummy))) return cuda_error(c, e, fn);
    dXout = (float*)dummy;
  }
  combine_kernel<<<pb, 256, 0, st>>>(A, splits, split_stride, WC, Pt.perm, N, Pt.Npad, Pt.d, d, P,
                                     inv_s2, dXout, (double*)partv, (GradAcc*)accv); count_launch();
  GradAcc ha;
  if ((e = cudaMemcpyAsync(&ha, accv, sizeof(GradAcc), cudaMemcpyDeviceToHost, st))) return cuda_error(c, e, fn);
  if (sdX && (e = cudaMemcpyAsync(dX, ddX, sizeof(float) * N * d, cudaMemcpyDeviceToHost, st)))
    return cuda_error(c, e, fn);
  if ((e = cudaStreamSynchronize(st))) return cuda_error(c, e, fn);
  *dlogsigma = 0.5 * ha.h * inv_s2;
  *dloggamma = 0.5 * (double)gamma * (ha.aa - ha.uz / P);
  krr_status de = read_device_error(c, st, fn);
  if (de) return de;
  return ss;
}
