// Krylov solvers (hot-path steps A5, A7-A10):
//   * krr_cg_solve     -- conjugate gradient (Sec. 3) on (K_hat + shift I) x = b
//   * krr_fgmres_solve -- Algorithm 1 (flexible GMRES(m), restarted) on
//                         K = K_hat + gamma I, right-preconditioned by truncated
//                         CG on M = K + delta I (Sec. 5)
//
// Everything runs on the device; the host only enqueues.  All scalars live in
// a device-resident KState.  Reductions are deterministic: every block writes
// a partial, and the last block to arrive (atomic ticket, no waiting) sums the
// partials in fixed order and performs the scalar step that follows (CG step
// lengths, Givens rotation, convergence tests).  Loop control is either
//   * a CUDA graph: the whole solve is captured once into nested conditional
//     WHILE nodes whose conditions the device sets (cudaGraphSetConditional),
//     so a solve is one graph launch with no host round trip; or
//   * a host loop that enqueues predicated iterations in batches and reads the
//     device flags between batches.
//
// Precision (the flexible outer iteration tolerates an inexact preconditioner,
// Sec. 5.1):
//   * inner products M p in the requested precision, CG vectors in float32,
//     dot products accumulated in FP64;
//   * outer products w = K z_j and the restart residuals with the compensated
//     float32 (float-float) product of mvp_acc.cu;
//   * Arnoldi orthogonalisation (CGS2: classical Gram-Schmidt applied twice,
//     which gives the same column as the modified Gram-Schmidt of Alg. 1 to
//     working precision while needing two grid reductions instead of j+1),
//     Hessenberg matrix, Givens rotations and least squares in FP64;
//   * the iterate x in float-float (two float32 arrays, returned as FP64) and the restart
//     residual r = b - K x (each cycle start of Alg. 1) from the accurate product of
//     mvp_acc.cu, so a restart acts as a step of iterative refinement and the
//     true residual reaches tolerances the float32 products alone cannot.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "api_util.h"
#include "common.cuh"
#include "internal.h"

namespace krr {
namespace {

constexpr int MMAX = 64;      // largest restart length
constexpr int VT = 256;       // threads of the vector kernels
constexpr int MAX_VBLOCKS = 1024;
// reduction partials per column: up to MMAX + 1 sums of up to MAX_VBLOCKS blocks
constexpr int64_t PSTRIDE = (int64_t)(MMAX + 1) * MAX_VBLOCKS;

// State of one right-hand side (one column of a block solve).
struct KState {
  // conjugate gradient
  double rho, rho0, pAp, alpha, beta, eps2;  // eps2 = (inner tol)^2
  int k, maxit, cg_cont, cg_brk;
  // Arnoldi / Givens
  int j, m, arn_cont, kcols, stepping;  // stepping: this column takes the current Arnoldi step
  double H[(MMAX + 1) * MMAX];  // column-major, leading dimension MMAX+1
  double cs[MMAX], sn[MMAX], g[MMAX + 1], y[MMAX];
  double h1[MMAX + 1], h2[MMAX + 1];
  double wnorm2;
  // restarts
  double rnorm2, bnorm, beta0, tol, tol_cycle;
  int cycles, max_cycles, restart_cont, lucky;
  // report
  int outer_total, inner_total, breakdowns, status;
  double relres_est, relres_true;
  // reduction scratch
  unsigned ticket;
};

// Loop control of one block solve (its columns advance in lockstep): the
// arrival ticket of group reductions and, per loop, whether some column
// still continues.
struct Group {
  unsigned ticket;
  int cg_any, arn_any, rst_any;
};

struct Cond {
  cudaGraphConditionalHandle h = 0;
  int use = 0;
};

__device__ __forceinline__ void set_cond(const Cond& c, int v) {
  if (c.use) cudaGraphSetConditional(c.h, (unsigned)v);
}

// Which columns a kernel works on.
enum Pred : int {
  PRED_ALL = 0,
  PRED_CG,    // the column's inner CG continues
  PRED_ARN,   // the column's Arnoldi process continues in this cycle
  PRED_STEP,  // the column takes the current Arnoldi step
  PRED_RST,   // the column is in a restart cycle (not yet converged)
};

__device__ __forceinline__ int col_flag(const KState* S, int pred) {
  switch (pred) {
    case PRED_CG: return *(const volatile int*)&S->cg_cont;
    case PRED_ARN: return *(const volatile int*)&S->arn_cont;
    case PRED_STEP: return *(const volatile int*)&S->stepping;
    case PRED_RST: return *(const volatile int*)&S->restart_cont;
    default: return 1;
  }
}

// One arrival per column, by one thread, once the column's flag `pred` is
// final.  The last column to arrive publishes whether any column's flag is
// set (in G and, when cc is in use, as the loop condition).
__device__ void group_arrive(const KState* S0, int ncols, Group* G, int pred, Cond cc) {
  __threadfence();
  if (atomicAdd(&G->ticket, 1u) != (unsigned)(ncols - 1)) return;
  __threadfence();
  int any = 0;
  for (int c = 0; c < ncols; ++c) any |= col_flag(S0 + c, pred);
  if (pred == PRED_CG) G->cg_any = any;
  else G->arn_any = any;
  G->ticket = 0u;
  set_cond(cc, any);
}

// Block partial -> per-block slot; returns true in the last block to arrive,
// where `total` then holds the fixed-order sum of all partials.
__device__ __forceinline__ bool grid_sum_last(double v, double* partials, unsigned* ticket,
                                              double* red, double& total) {
  __shared__ bool is_last;
  const double bs = block_sum(v, red);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = bs;
    __threadfence();
    is_last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  double t = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) t += partials[b];
  total = block_sum(t, red);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Vector kernels run on a grid (blocks, columns): column blockIdx.y has its
// state at S0 + blockIdx.y, its float / double vectors Np apart, its Arnoldi
// basis vstride apart, its Z basis zstride apart and its reduction partials
// PSTRIDE apart.
#define KRR_COL                                   \
  const int col = blockIdx.y;                     \
  KState* S = S0 + col;                           \
  const int64_t co = (int64_t)col * Np;           \
  (void)co

#define KRR_GRID_LOOP(i) \
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np; i += (int64_t)gridDim.x * blockDim.x)

// ------------------------------------------------------------------ CG ---
// For the columns selected by pred: z = 0 (z = v without preconditioner),
// r = p = v (v = V[j] in FP64, or the float vector vf), rho0 = rho = |v|^2.
// The other columns sit out this Arnoldi step.
__global__ void cg_init_kernel(KState* S0, const double* __restrict__ V, int64_t vstride,
                               const float* __restrict__ vf, int64_t Np, float* __restrict__ z,
                               float* __restrict__ r, float* __restrict__ p, double* partials,
                               int pred, Group* G, Cond cc) {
  __shared__ double red[8];
  KRR_COL;
  if (!col_flag(S, pred)) {
    if (blockIdx.x == 0 && threadIdx.x == 0) {
      S->cg_cont = 0;
      S->stepping = 0;
      group_arrive(S0, gridDim.y, G, PRED_CG, cc);
    }
    return;
  }
  const double* v = V ? V + (int64_t)col * vstride + (int64_t)S->j * Np : nullptr;
  const bool identity = S->maxit == 0;
  double acc = 0.0;
  KRR_GRID_LOOP(i) {
    const float vi = v ? (float)v[i] : vf[co + i];
    r[co + i] = vi;
    p[co + i] = vi;
    z[co + i] = identity ? vi : 0.f;
    acc += (double)vi * (double)vi;
  }
  double tot;
  if (grid_sum_last(acc, partials + col * PSTRIDE, &S->ticket, red, tot) && threadIdx.x == 0) {
    S->rho = tot;
    S->rho0 = tot;
    S->k = 0;
    S->cg_brk = 0;
    S->cg_cont = (!identity && tot > 0.0) ? 1 : 0;
    S->stepping = 1;
    group_arrive(S0, gridDim.y, G, PRED_CG, cc);
  }
}

// z += alpha p; r -= alpha Mp; rho' = |r|^2; beta = rho'/rho; continue test.
__global__ void cg_update_kernel(KState* S0, float* __restrict__ z, float* __restrict__ r,
                                 const float* __restrict__ p, const float* __restrict__ Mp,
                                 int64_t Np, double* partials, Group* G, Cond cc) {
  __shared__ double red[8];
  KRR_COL;
  if (!S->cg_cont) {
    if (blockIdx.x == 0 && threadIdx.x == 0) group_arrive(S0, gridDim.y, G, PRED_CG, cc);
    return;
  }
  const float a = (float)S->alpha;
  double acc = 0.0;
  KRR_GRID_LOOP(i) {
    z[co + i] = fmaf(a, p[co + i], z[co + i]);
    const float ri = fmaf(-a, Mp[co + i], r[co + i]);
    r[co + i] = ri;
    acc += (double)ri * (double)ri;
  }
  double tot;
  if (grid_sum_last(acc, partials + col * PSTRIDE, &S->ticket, red, tot) && threadIdx.x == 0) {
    S->beta = (S->rho > 0.0) ? tot / S->rho : 0.0;
    S->rho = tot;
    S->k += 1;
    S->inner_total += 1;
    if (S->cg_brk) S->breakdowns += 1;
    const bool more = !S->cg_brk && S->k < S->maxit && tot > S->eps2 * S->rho0 && isfinite(tot);
    S->cg_cont = more ? 1 : 0;
    group_arrive(S0, gridDim.y, G, PRED_CG, cc);
  }
}

// p = r + beta p for the columns whose CG continues.
__global__ void cg_p_kernel(KState* S0, const float* __restrict__ r, float* __restrict__ p,
                            int64_t Np) {
  KRR_COL;
  if (!S->cg_cont) return;
  const float b = (float)S->beta;
  KRR_GRID_LOOP(i) p[co + i] = fmaf(b, p[co + i], r[co + i]);
}

// ------------------------------------------------------------- Arnoldi ---
__global__ void store_z_kernel(KState* S0, const float* __restrict__ z, float* __restrict__ Z,
                               int64_t zstride, int64_t Np, int pred) {
  KRR_COL;
  if (!col_flag(S, pred)) return;
  float* zj = Z + (int64_t)col * zstride + (int64_t)S->j * Np;
  KRR_GRID_LOOP(i) zj[i] = z[co + i];
}

// h1[i] = (w, v_i), i = 0..j  (first Gram-Schmidt pass).
__global__ void cgs_dots_kernel(KState* S0, const double* __restrict__ V, int64_t vstride,
                                const double* __restrict__ w, int64_t Np, double* partials,
                                int pred) {
  __shared__ double red[8];
  __shared__ bool is_last;
  KRR_COL;
  if (!col_flag(S, pred)) return;
  V += (int64_t)col * vstride;
  w += co;
  partials += col * PSTRIDE;
  const int nj = S->j + 1;
  for (int c = 0; c < nj; ++c) {
    const double* vc = V + (int64_t)c * Np;
    double acc = 0.0;
    KRR_GRID_LOOP(i) acc += vc[i] * w[i];
    const double bs = block_sum(acc, red);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * (MMAX + 1) + c] = bs;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int c = 0; c < nj; ++c) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      t += partials[(int64_t)b * (MMAX + 1) + c];
    t = block_sum(t, red);
    if (threadIdx.x == 0) S->h1[c] = t;
  }
  if (threadIdx.x == 0) S->ticket = 0u;
}

// w -= sum_i h1[i] v_i; h2[i] = (w, v_i) (second pass); |w|^2; then, in the
// last block, the Hessenberg column, the Givens update of Alg. 1's least
// squares problem and the continuation test.
__global__ void cgs_update_kernel(KState* S0, const double* __restrict__ V, int64_t vstride,
                                  double* __restrict__ w, int64_t Np, double* partials, int pred) {
  __shared__ double red[8];
  __shared__ bool is_last;
  __shared__ double h1s[MMAX + 1];
  KRR_COL;
  if (!col_flag(S, pred)) return;
  V += (int64_t)col * vstride;
  w += co;
  partials += col * PSTRIDE;
  const int j = S->j, nj = j + 1;
  for (int c = threadIdx.x; c < nj; c += blockDim.x) h1s[c] = S->h1[c];
  __syncthreads();
  KRR_GRID_LOOP(i) {
    double wi = w[i];
    for (int c = 0; c < nj; ++c) wi -= h1s[c] * V[(int64_t)c * Np + i];
    w[i] = wi;
  }
  // second-pass dots and the norm of w, from this block's elements
  for (int c = 0; c <= nj; ++c) {
    double acc = 0.0;
    KRR_GRID_LOOP(i) acc += (c < nj) ? V[(int64_t)c * Np + i] * w[i] : w[i] * w[i];
    const double bs = block_sum(acc, red);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * (MMAX + 1) + c] = bs;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(&S->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int c = 0; c <= nj; ++c) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      t += partials[(int64_t)b * (MMAX + 1) + c];
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
      if (c < nj) S->h2[c] = t;
      else S->wnorm2 = t;
    }
  }
  if (threadIdx.x != 0) return;
  S->ticket = 0u;
  // |w - V h2|^2 = |w|^2 - |h2|^2 (V orthonormal)
  double hh = 0.0;
  for (int c = 0; c < nj; ++c) hh += S->h2[c] * S->h2[c];
  const double wn2 = fmax(S->wnorm2 - hh, 0.0);
  double* Hj = S->H + (int64_t)j * (MMAX + 1);
  for (int c = 0; c < nj; ++c) Hj[c] = S->h1[c] + S->h2[c];
  const double hnext = sqrt(wn2);
  Hj[nj] = hnext;
  // apply the previous rotations to the new column, then a new rotation that
  // zeroes H[j+1, j]
  for (int c = 0; c < j; ++c) {
    const double t0 = S->cs[c] * Hj[c] + S->sn[c] * Hj[c + 1];
    const double t1 = -S->sn[c] * Hj[c] + S->cs[c] * Hj[c + 1];
    Hj[c] = t0;
    Hj[c + 1] = t1;
  }
  const double a = Hj[j], b = Hj[j + 1];
  const double rr = hypot(a, b);
  const double cj = rr > 0.0 ? a / rr : 1.0, sj = rr > 0.0 ? b / rr : 0.0;
  S->cs[j] = cj;
  S->sn[j] = sj;
  Hj[j] = rr;
  Hj[j + 1] = 0.0;
  const double gj = S->g[j];
  S->g[j] = cj * gj;
  S->g[j + 1] = -sj * gj;
  S->relres_est = fabs(S->g[j + 1]) / S->bnorm;
  S->outer_total += 1;
  S->kcols = j + 1;
  // lucky breakdown: w lies in the span of V, the least-squares residual is exact
  const bool lucky = !(hnext > 1e-14 * rr) || !isfinite(hnext);
  S->lucky = lucky ? 1 : 0;
  S->wnorm2 = hnext;  // reused by cgs_final as the normaliser
  const bool more = !lucky && (j + 1 < S->m) && S->relres_est > S->tol_cycle;
  S->arn_cont = more ? 1 : 0;
}

// v_{j+1} = (w - V h2) / h_{j+1,j}
__global__ void cgs_final_kernel(KState* S0, double* __restrict__ V, int64_t vstride,
                                 const double* __restrict__ w, int64_t Np, int pred) {
  __shared__ double h2s[MMAX + 1];
  KRR_COL;
  if (!col_flag(S, pred)) return;
  const int j = S->j, nj = j + 1;
  if (S->lucky || j + 1 > S->m) return;
  V += (int64_t)col * vstride;
  w += co;
  for (int c = threadIdx.x; c < nj; c += blockDim.x) h2s[c] = S->h2[c];
  __syncthreads();
  const double inv = 1.0 / S->wnorm2;
  double* vn = V + (int64_t)nj * Np;
  KRR_GRID_LOOP(i) {
    double wi = w[i];
    for (int c = 0; c < nj; ++c) wi -= h2s[c] * V[(int64_t)c * Np + i];
    vn[i] = wi * inv;
  }
}

// One thread per column: advance the columns whose Arnoldi process
// continues; the loop goes on while any does.
__global__ void arn_advance_kernel(KState* S0, int ncols, Group* G, Cond ac) {
  int any = 0;
  for (int c = threadIdx.x; c < ncols; c += blockDim.x) {
    KState* S = S0 + c;
    if (S->arn_cont) {
      S->j += 1;
      any = 1;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    G->arn_any = any;
    set_cond(ac, any);
  }
}

// ---------------------------------------------------------- restarts -----
// One thread per column: back-substitution R y = g (R upper triangular after
// the rotations, kcols columns).
__global__ void lsq_kernel(KState* S0, int ncols, int pred) {
  for (int cix = threadIdx.x; cix < ncols; cix += blockDim.x) {
    KState* S = S0 + cix;
    if (!col_flag(S, pred)) continue;
    const int k = S->kcols;
    for (int r = k - 1; r >= 0; --r) {
      double t = S->g[r];
      for (int c = r + 1; c < k; ++c) t -= S->H[(int64_t)c * (MMAX + 1) + r] * S->y[c];
      const double d = S->H[(int64_t)r * (MMAX + 1) + r];
      S->y[r] = d != 0.0 ? t / d : 0.0;
    }
  }
}

// x += Z y in float-float.
__global__ void x_update_kernel(KState* S0, const float* __restrict__ Z, int64_t zstride,
                                int64_t Np, float* __restrict__ xh, float* __restrict__ xl,
                                int pred) {
  __shared__ double ys[MMAX];
  KRR_COL;
  if (!col_flag(S, pred)) return;
  Z += (int64_t)col * zstride;
  const int k = S->kcols;
  for (int c = threadIdx.x; c < k; c += blockDim.x) ys[c] = S->y[c];
  __syncthreads();
  KRR_GRID_LOOP(i) {
    double t = (double)xh[co + i] + (double)xl[co + i];
    for (int c = 0; c < k; ++c) t += ys[c] * (double)Z[(int64_t)c * Np + i];
    const float h = (float)t;
    xh[co + i] = h;
    xl[co + i] = (float)(t - (double)h);
  }
}

// One thread per column, after the accurate residual: convergence test and
// the next cycle's start (the restart test and cycle start of Alg. 1).  tol_stop < tol leaves
// room for rounding.  A column that has stopped keeps its verdict (its
// residual is not recomputed, so the test repeats it).
__global__ void restart_check_kernel(KState* S0, int ncols, Group* G, Cond rc, double tol_stop) {
  int any = 0;
  for (int cix = threadIdx.x; cix < ncols; cix += blockDim.x) {
    KState* S = S0 + cix;
    const double beta = sqrt(S->rnorm2);
    S->relres_true = S->bnorm > 0.0 ? beta / S->bnorm : 0.0;
    bool more = S->bnorm > 0.0 && S->relres_true > tol_stop && isfinite(beta);
    if (more && S->cycles >= S->max_cycles) {
      // out of cycles: converged if the true residual meets the tolerance
      // itself (tol_stop only leaves a margin while there are cycles left)
      more = false;
      if (S->relres_true > S->tol) S->status = KRR_NOT_CONVERGED;
    }
    if (!isfinite(beta)) S->status = KRR_ERR_NONFINITE;
    S->restart_cont = more ? 1 : 0;
    if (more) {
      S->cycles += 1;
      S->beta0 = beta;
      S->g[0] = beta;
      for (int c = 1; c <= MMAX; ++c) S->g[c] = 0.0;
      S->j = 0;
      S->kcols = 0;
      S->arn_cont = 1;
      S->lucky = 0;
      any = 1;
    }
  }
  any = __syncthreads_or(any);
  if (threadIdx.x == 0) {
    G->rst_any = any;
    set_cond(rc, any);
  }
}

// V[0] = r / beta0 for the columns in a cycle; re-arms the Arnoldi loop (a
// WHILE condition takes its default only once per graph launch).
__global__ void v0_kernel(KState* S0, const double* __restrict__ r, double* __restrict__ V,
                          int64_t vstride, int64_t Np, int pred, Group* G, Cond ac) {
  KRR_COL;
  if (blockIdx.x == 0 && col == 0 && threadIdx.x == 0) {
    G->arn_any = 1;
    set_cond(ac, 1);
  }
  if (!col_flag(S, pred)) return;
  const double inv = 1.0 / S->beta0;
  V += (int64_t)col * vstride;
  KRR_GRID_LOOP(i) V[i] = r[co + i] * inv;
}

// x = 0, r = b (the residual of x0 = 0), |b|^2.
__global__ void solve_init_kernel(KState* S0, const float* __restrict__ b, int64_t Np,
                                  float* __restrict__ xh, float* __restrict__ xl,
                                  double* __restrict__ r, double* partials) {
  __shared__ double red[8];
  KRR_COL;
  double acc = 0.0;
  KRR_GRID_LOOP(i) {
    xh[co + i] = 0.f;
    xl[co + i] = 0.f;
    const double bi = b[co + i];
    r[co + i] = bi;
    acc += bi * bi;
  }
  double tot;
  if (grid_sum_last(acc, partials + col * PSTRIDE, &S->ticket, red, tot) && threadIdx.x == 0) {
    S->rnorm2 = tot;
    S->bnorm = sqrt(tot);
  }
}

// x = x0 (FP64, original order, column c at x0 + c N; columns >= nx and the
// padding start at 0) in float-float, and |b| per column.  The residual
// r = b - K x follows from the accurate product (the start of a restart
// cycle of Alg. 1 with x0 <- the given guess).
__global__ void solve_init_x0_kernel(KState* S0, const float* __restrict__ b,
                                     const double* __restrict__ x0, const int* __restrict__ perm,
                                     int64_t N, int nx, int64_t Np, float* __restrict__ xh,
                                     float* __restrict__ xl, double* partials) {
  __shared__ double red[8];
  KRR_COL;
  double acc = 0.0;
  KRR_GRID_LOOP(i) {
    const double v = (col < nx && i < N) ? x0[(int64_t)col * N + perm[i]] : 0.0;
    const float h = (float)v;
    xh[co + i] = h;
    xl[co + i] = (float)(v - (double)h);
    const double bi = b[co + i];
    acc += bi * bi;
  }
  double tot;
  if (grid_sum_last(acc, partials + col * PSTRIDE, &S->ticket, red, tot) && threadIdx.x == 0)
    S->bnorm = sqrt(tot);
}

// CG restart setup: stop when the true relative residual meets tol_stop,
// else aim the next CG run at reducing |r| to tol_stop |b| (residual
// replacement: CG restarted on A z = r from the accurate residual).
__global__ void cg_cycle_kernel(KState* S, double tol_stop, int maxit_total) {
  const double rn = sqrt(S->rnorm2);
  S->relres_true = S->bnorm > 0.0 ? rn / S->bnorm : 0.0;
  const int left = maxit_total - S->inner_total;
  bool more = S->bnorm > 0.0 && S->relres_true > tol_stop && isfinite(rn);
  if (more && left <= 0) {
    more = false;
    S->status = KRR_NOT_CONVERGED;
  }
  if (!isfinite(rn)) S->status = KRR_ERR_NONFINITE;
  S->restart_cont = more ? 1 : 0;
  if (more) {
    S->cycles += 1;
    S->j = 0;
    S->maxit = left;
    const double target = 0.5 * tol_stop * S->bnorm / rn;  // relative to |r|
    S->eps2 = fmax(target, 1e-7) * fmax(target, 1e-7);
  }
}

// x += z in float-float
__global__ void x_add_kernel(const float* __restrict__ z, int64_t Np, float* __restrict__ xh,
                             float* __restrict__ xl) {
  KRR_GRID_LOOP(i) {
    const double t = (double)xh[i] + (double)xl[i] + (double)z[i];
    const float h = (float)t;
    xh[i] = h;
    xl[i] = (float)(t - (double)h);
  }
}

// x = x0 (FP64, original order) gathered to sorted float-float; padding 0
__global__ void x_from64_kernel(const double* __restrict__ x0, const int* __restrict__ perm,
                                int64_t N, int64_t Np, float* __restrict__ xh, float* __restrict__ xl) {
  KRR_GRID_LOOP(i) {
    const double v = i < N ? x0[perm[i]] : 0.0;
    const float h = (float)v;
    xh[i] = h;
    xl[i] = (float)(v - (double)h);
  }
}

__global__ void bnorm_kernel(KState* S, const float* __restrict__ b, int64_t Np, double* partials) {
  __shared__ double red[8];
  double acc = 0.0;
  KRR_GRID_LOOP(i) acc += (double)b[i] * (double)b[i];
  double tot;
  if (grid_sum_last(acc, partials, &S->ticket, red, tot) && threadIdx.x == 0) S->bnorm = sqrt(tot);
}

// Column blockIdx.y: out[col * N + perm[i]] = xh[i] + xl[i] (FP64, original order)
__global__ void scatter_x64_kernel(const float* __restrict__ xh, const float* __restrict__ xl,
                                   const int* __restrict__ perm, int64_t N, int64_t Np,
                                   double* __restrict__ out) {
  const int64_t co = (int64_t)blockIdx.y * Np;
  out += (int64_t)blockIdx.y * N;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    out[perm[i]] = (double)xh[co + i] + (double)xl[co + i];
}

__global__ void fill_zero_kernel(float* __restrict__ a, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    a[i] = 0.f;
}

#undef KRR_COL
#undef KRR_GRID_LOOP

// ------------------------------------------------------- flexible CG ---
// Flexible CG (Notay; the paper's second outer iteration, Sec. 4.2): step i
// takes the preconditioned residual z_i (truncated inner CG on M) and makes it
// A-orthogonal to the previous (at most mmax) directions,
//   d_i = z_i - sum_k beta_k d_k,  beta_k = (z_i . A d_k) / (d_k . A d_k),
// then alpha_i = (d_i . r_i) / (d_i . A d_i), x += alpha_i d_i,
// r -= alpha_i A d_i.  Directions and A d live in a circular window of
// W = mmax + 1 FP64 slots; slot `head` receives the new direction.
struct FState {
  double beta[MMAX + 1], dad[MMAX + 1];
  double alpha, rr, bnorm;
  int cnt, head, W, brk;
  unsigned ticket;
};

// beta_k for the cnt directions before head (multi-dot, last block divides)
__global__ void fcg_beta_kernel(FState* F, const float* __restrict__ z, const double* __restrict__ AD,
                                int64_t Np, double* partials) {
  __shared__ double red[8];
  __shared__ bool is_last;
  const int cnt = F->cnt, W = F->W, head = F->head;
  for (int c = 0; c < cnt; ++c) {
    const int slot = (head - 1 - c + W) % W;
    const double* adk = AD + (int64_t)slot * Np;
    double acc = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
         i += (int64_t)gridDim.x * blockDim.x)
      acc += (double)z[i] * adk[i];
    const double bs = block_sum(acc, red);
    if (threadIdx.x == 0) partials[(int64_t)blockIdx.x * (MMAX + 1) + c] = bs;
  }
  if (threadIdx.x == 0) {
    __threadfence();
    is_last = atomicAdd(&F->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  for (int c = 0; c < cnt; ++c) {
    double t = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x)
      t += partials[(int64_t)b * (MMAX + 1) + c];
    t = block_sum(t, red);
    if (threadIdx.x == 0) {
      const int slot = (head - 1 - c + W) % W;
      F->beta[slot] = F->dad[slot] > 0.0 ? t / F->dad[slot] : 0.0;
    }
  }
  if (threadIdx.x == 0) F->ticket = 0u;
}

// d = z - sum beta_k d_k into slot head (FP64) and as float-float (dh + dl)
__global__ void fcg_dir_kernel(const FState* F, const float* __restrict__ z, double* __restrict__ D,
                               int64_t Np, float* __restrict__ dh, float* __restrict__ dl) {
  __shared__ double bs[MMAX + 1];
  __shared__ int slots[MMAX + 1];
  const int cnt = F->cnt, W = F->W, head = F->head;
  for (int c = threadIdx.x; c < cnt; c += blockDim.x) {
    slots[c] = (head - 1 - c + W) % W;
    bs[c] = F->beta[slots[c]];
  }
  __syncthreads();
  double* dn = D + (int64_t)head * Np;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = z[i];
    for (int c = 0; c < cnt; ++c) v -= bs[c] * D[(int64_t)slots[c] * Np + i];
    dn[i] = v;
    const float h = (float)v;
    dh[i] = h;
    dl[i] = (float)(v - (double)h);
  }
}

// d . A d and d . r; the last block sets alpha (or flags a breakdown)
__global__ void fcg_alpha_kernel(FState* F, const double* __restrict__ D, const double* __restrict__ AD,
                                 const double* __restrict__ r, int64_t Np, double* partials) {
  __shared__ double red[8];
  __shared__ bool is_last;
  const int head = F->head;
  const double* d = D + (int64_t)head * Np;
  const double* ad = AD + (int64_t)head * Np;
  double a1 = 0.0, a2 = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
       i += (int64_t)gridDim.x * blockDim.x) {
    a1 += d[i] * ad[i];
    a2 += d[i] * r[i];
  }
  const double b1 = block_sum(a1, red);
  const double b2 = block_sum(a2, red);
  if (threadIdx.x == 0) {
    partials[2 * blockIdx.x] = b1;
    partials[2 * blockIdx.x + 1] = b2;
    __threadfence();
    is_last = atomicAdd(&F->ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!is_last || threadIdx.x != 0) return;
  __threadfence();
  double t1 = 0.0, t2 = 0.0;
  for (int b = 0; b < (int)gridDim.x; ++b) {
    t1 += partials[2 * b];
    t2 += partials[2 * b + 1];
  }
  F->dad[head] = t1;
  const bool good = t1 > 0.0 && isfinite(t1) && isfinite(t2);
  F->alpha = good ? t2 / t1 : 0.0;
  F->brk = good ? 0 : 1;
  F->ticket = 0u;
}

// x += alpha d (float-float), r -= alpha A d, |r|^2; the last block advances
// the window
__global__ void fcg_update_kernel(FState* F, const double* __restrict__ D, const double* __restrict__ AD,
                                  int64_t Np, float* __restrict__ xh, float* __restrict__ xl,
                                  double* __restrict__ r, double* partials, int mmax) {
  __shared__ double red[8];
  const int head = F->head;
  const double a = F->alpha;
  const double* d = D + (int64_t)head * Np;
  const double* ad = AD + (int64_t)head * Np;
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double t = (double)xh[i] + (double)xl[i] + a * d[i];
    const float h = (float)t;
    xh[i] = h;
    xl[i] = (float)(t - (double)h);
    const double ri = r[i] - a * ad[i];
    r[i] = ri;
    acc += ri * ri;
  }
  double tot;
  if (grid_sum_last(acc, partials, &F->ticket, red, tot) && threadIdx.x == 0) {
    F->rr = tot;
    F->cnt = min(F->cnt + 1, mmax);
    F->head = (head + 1) % F->W;
  }
}

__global__ void fcg_to_float_kernel(const double* __restrict__ r, int64_t Np, float* __restrict__ rf) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < Np;
       i += (int64_t)gridDim.x * blockDim.x)
    rf[i] = (float)r[i];
}

// ---------------------------------------------------------------- driver --
// One solve of mc right-hand sides of one problem in lockstep (a block
// solve): every column runs its own FGMRES (its own Krylov basis, Givens
// rotations and restarts), but each inner CG step applies the operator to
// all columns' search directions in one multi-column product, and the outer
// products and residuals of all columns go out in one launch.  Columns that
// have finished their CG, Arnoldi step or solve sit out (predicated per
// column) until the block's loop ends.
struct Solver {
  Ctx& c;
  cudaStream_t st;
  PointsDev P;
  int64_t Np = 0;
  unsigned vblocks = 1;
  float gamma = 0.f, mshift = 0.f;
  krr_precision inner_prec = KRR_FP32;
  int m = 30;   // restart length
  int mc = 1;   // columns
  // device buffers (column-major blocks of mc columns)
  KState* S = nullptr;
  Group* G = nullptr;
  float *b = nullptr, *xh = nullptr, *xl = nullptr, *zero = nullptr;
  double *r64 = nullptr, *V = nullptr, *w = nullptr, *partials = nullptr;
  float *Z = nullptr, *z = nullptr, *rr = nullptr, *p = nullptr, *Mp = nullptr;
  Cond cg_c, arn_c, rst_c;

  explicit Solver(Ctx& cc) : c(cc) {}

  int64_t vstride() const { return (int64_t)(m + 1) * Np; }
  int64_t zstride() const { return (int64_t)m * Np; }
  dim3 vgrid() const { return dim3(vblocks, (unsigned)mc); }

  cudaError_t alloc(int restart, int ncols) {
    cudaError_t e;
    void* v;
    const size_t n = (size_t)Np * ncols;
    m = restart;
    mc = ncols;
#define KRR_WS(name, ptr, bytes)                      \
  if ((e = c.ws.get(name, bytes, &v))) return e;       \
  ptr = (decltype(ptr))v;
    KRR_WS("kry.state", S, sizeof(KState) * mc);
    KRR_WS("kry.group", G, sizeof(Group));
    KRR_WS("kry.b", b, n * 4);
    KRR_WS("kry.xh", xh, n * 4);
    KRR_WS("kry.xl", xl, n * 4);
    KRR_WS("kry.zero", zero, n * 4);
    KRR_WS("kry.r64", r64, n * 8);
    KRR_WS("kry.V", V, n * 8 * (m + 1));
    KRR_WS("kry.w", w, n * 8);
    KRR_WS("kry.partials", partials, sizeof(double) * PSTRIDE * mc);
    KRR_WS("kry.Z", Z, n * 4 * m);
    KRR_WS("kry.z", z, n * 4);
    KRR_WS("kry.r", rr, n * 4);
    KRR_WS("kry.p", p, n * 4);
    KRR_WS("kry.Mp", Mp, n * 4);
#undef KRR_WS
    vblocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((Np + VT - 1) / VT, 4LL * c.num_sms));
    if (vblocks > (unsigned)MAX_VBLOCKS) vblocks = MAX_VBLOCKS;
    fill_zero_kernel<<<vblocks, VT, 0, st>>>(zero, (int64_t)n); count_launch();
    if ((e = cudaMemsetAsync(G, 0, sizeof(Group), st))) return e;
    return cudaGetLastError();
  }

  // Workspace and kernel attributes of every product this solver launches,
  // so that nothing allocates inside a graph capture.
  cudaError_t reserve() {
    cudaError_t e = mvp_reserve(c, P, P, st);
    if (!e && (mc > 1 || inner_prec != KRR_FP32)) e = mvp_multi_reserve(c, P, P, mc, inner_prec, st);
    if (!e) e = mvp_acc_reserve(c, P, st, mc);
    return e;
  }

  // ---- one CG iteration on the inner operator M p = K_hat p + mshift p,
  // for every column whose CG continues
  cudaError_t cg_iteration() {
    MvpOut o;
    o.out_f = Mp;
    o.dotw = p;
    o.dot = &S->pAp;
    o.ratio_num = &S->rho;
    o.ratio_out = &S->alpha;
    o.brk_flag = &S->cg_brk;
    o.active = &G->cg_any;
    o.col_active = &S->cg_cont;
    o.state_stride = sizeof(KState);
    cudaError_t e = mc == 1 ? mvp_launch(c, P, P, p, p, mshift, inner_prec, o, st)
                            : mvp_multi_launch(c, P, P, p, mc, p, mshift, inner_prec, o, st);
    if (e) return e;
    cg_update_kernel<<<vgrid(), VT, 0, st>>>(S, z, rr, p, Mp, Np, partials, G, cg_c); count_launch();
    cg_p_kernel<<<vgrid(), VT, 0, st>>>(S, rr, p, Np); count_launch();
    return cudaGetLastError();
  }

  // ---- Arnoldi step after the inner solve: Z[j] = z, w = K z, CGS2, Givens
  cudaError_t arnoldi_tail() {
    store_z_kernel<<<vgrid(), VT, 0, st>>>(S, z, Z, zstride(), Np, PRED_STEP); count_launch();
    // w = K z_j with the compensated product: its error enters the flexible
    // Arnoldi relation K Z = V Hbar, and through it the true residual
    AccCols cols;
    cols.n = mc;
    cols.active = &S->stepping;
    cols.state_stride = sizeof(KState);
    cudaError_t e = mvp_acc_launch(c, P, z, zero, gamma, 0.0, nullptr, 1.0, w, nullptr, st, cols);
    if (e) return e;
    cgs_dots_kernel<<<vgrid(), VT, 0, st>>>(S, V, vstride(), w, Np, partials, PRED_STEP); count_launch();
    cgs_update_kernel<<<vgrid(), VT, 0, st>>>(S, V, vstride(), w, Np, partials, PRED_STEP); count_launch();
    cgs_final_kernel<<<vgrid(), VT, 0, st>>>(S, V, vstride(), w, Np, PRED_STEP); count_launch();
    arn_advance_kernel<<<1, 32, 0, st>>>(S, mc, G, arn_c); count_launch();
    return cudaGetLastError();
  }

  cudaError_t cycle_tail(double tol_stop) {
    lsq_kernel<<<1, 32, 0, st>>>(S, mc, PRED_RST); count_launch();
    x_update_kernel<<<vgrid(), VT, 0, st>>>(S, Z, zstride(), Np, xh, xl, PRED_RST); count_launch();
    cudaError_t e = residual(true);
    if (e) return e;
    restart_check_kernel<<<1, 32, 0, st>>>(S, mc, G, rst_c, tol_stop); count_launch();
    return cudaGetLastError();
  }

  // Start of a solve: x = 0, r = b (x0 == null), or x = x0 (first nx
  // columns of x0, N apart) and r = b - K x0 from the accurate product
  cudaError_t init_solution(const double* x0, int64_t N, int nx) {
    if (!x0) {
      solve_init_kernel<<<vgrid(), VT, 0, st>>>(S, b, Np, xh, xl, r64, partials); count_launch();
      return cudaGetLastError();
    }
    solve_init_x0_kernel<<<vgrid(), VT, 0, st>>>(S, b, x0, P.perm, N, nx, Np, xh, xl, partials); count_launch();
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    return residual(false);
  }

  // r64 = b - K x (accurate), rnorm2 = |r|^2; only for the columns in a
  // restart cycle when in_cycle is set
  cudaError_t residual(bool in_cycle) {
    AccCols cols;
    cols.n = mc;
    cols.active = in_cycle ? &S->restart_cont : nullptr;
    cols.state_stride = sizeof(KState);
    return mvp_acc_launch(c, P, xh, xl, gamma, 1.0, b, -1.0, r64, &S->rnorm2, st, cols);
  }
};

cudaError_t read_state(Ctx& c, const KState* S, KState& h, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(&h, S, sizeof(KState), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  return e;
}

cudaError_t read_group(const Group* G, Group& h, cudaStream_t st) {
  cudaError_t e = cudaMemcpyAsync(&h, G, sizeof(Group), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  return e;
}

struct SolveCfg {
  int restart, max_cycles, inner_maxit;
  double tol, delta, inner_tol;
  krr_precision inner_prec;
  bool graph;
  bool x0_given;
};

// Host-side initial state for one right-hand side.
void init_state(KState& h, const SolveCfg& cfg) {
  memset(&h, 0, sizeof(h));
  h.maxit = cfg.inner_maxit;
  h.eps2 = cfg.inner_tol * cfg.inner_tol;
  h.m = cfg.restart;
  h.tol = cfg.tol;
  h.tol_cycle = 0.5 * cfg.tol;
  h.max_cycles = cfg.max_cycles;
  h.status = KRR_OK;
}

// Initial states of all columns of s (host copy, then one upload).
cudaError_t upload_states(Solver& s, const SolveCfg& cfg, std::vector<KState>& hs) {
  hs.resize(s.mc);
  for (auto& h : hs) init_state(h, cfg);
  cudaError_t e = cudaMemcpyAsync(s.S, hs.data(), sizeof(KState) * s.mc, cudaMemcpyHostToDevice, s.st);
  if (!e) e = cudaMemsetAsync(s.G, 0, sizeof(Group), s.st);
  if (!e) e = cudaStreamSynchronize(s.st);  // hs is pageable and reused
  return e;
}

std::vector<cudaGraphNode_t> sinks(cudaGraph_t g) {
  std::vector<cudaGraphNode_t> out;
  size_t n = 0;
  if (cudaGraphGetNodes(g, nullptr, &n) || n == 0) return out;
  std::vector<cudaGraphNode_t> all(n);
  cudaGraphGetNodes(g, all.data(), &n);
  for (auto nd : all) {
    size_t nout = 0;
    cudaGraphNodeGetDependentNodes(nd, nullptr, nullptr, &nout);
    if (nout == 0) out.push_back(nd);
  }
  return out;
}

// Append a WHILE node controlled by `h` after every sink of `parent`.
cudaError_t add_while(cudaGraph_t parent, cudaGraphConditionalHandle h, cudaGraph_t* body) {
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  std::vector<cudaGraphNode_t> deps = sinks(parent);
  cudaGraphNode_t node;
  cudaError_t e = cudaGraphAddNode(&node, parent, deps.data(), nullptr, deps.size(), &np);
  if (e) return e;
  *body = np.conditional.phGraph_out[0];
  return cudaSuccess;
}

// Capture the work enqueued by fn() into `into`, after its current sinks.
template <typename F>
cudaError_t capture_into(cudaStream_t st, cudaGraph_t into, F&& fn) {
  std::vector<cudaGraphNode_t> deps = sinks(into);
  cudaError_t e = cudaStreamBeginCaptureToGraph(st, into, deps.data(), nullptr, deps.size(),
                                                cudaStreamCaptureModeThreadLocal);
  if (e) return e;
  const cudaError_t fe = fn();
  cudaGraph_t out;
  e = cudaStreamEndCapture(st, &out);
  return fe ? fe : e;
}

// Fill the body of the restart WHILE node: v0; WHILE arnoldi { cg_init;
// WHILE cg { CG iteration }; Arnoldi step }; least squares, x update, true
// residual, restart check.
cudaError_t fill_restart_body(Solver& s, cudaGraph_t rbody, double tol_stop) {
  cudaError_t e;
  cudaGraph_t abody, cbody;
  if ((e = cudaGraphConditionalHandleCreate(&s.arn_c.h, rbody, 1, cudaGraphCondAssignDefault))) return e;
  s.arn_c.use = 1;
  if ((e = capture_into(s.st, rbody, [&]() -> cudaError_t {
         v0_kernel<<<s.vgrid(), VT, 0, s.st>>>(s.S, s.r64, s.V, s.vstride(), s.Np, PRED_RST, s.G,
                                                s.arn_c); count_launch();
         return cudaGetLastError();
       })))
    return e;
  if ((e = add_while(rbody, s.arn_c.h, &abody))) return e;
  if ((e = cudaGraphConditionalHandleCreate(&s.cg_c.h, abody, 0, cudaGraphCondAssignDefault))) return e;
  s.cg_c.use = 1;
  if ((e = capture_into(s.st, abody, [&]() -> cudaError_t {
         cg_init_kernel<<<s.vgrid(), VT, 0, s.st>>>(s.S, s.V, s.vstride(), nullptr, s.Np, s.z, s.rr,
                                                    s.p, s.partials, PRED_ARN, s.G, s.cg_c); count_launch();
         return cudaGetLastError();
       })))
    return e;
  if ((e = add_while(abody, s.cg_c.h, &cbody))) return e;
  if ((e = capture_into(s.st, cbody, [&]() -> cudaError_t { return s.cg_iteration(); }))) return e;
  if ((e = capture_into(s.st, abody, [&]() -> cudaError_t { return s.arnoldi_tail(); }))) return e;
  return capture_into(s.st, rbody, [&]() -> cudaError_t { return s.cycle_tail(tol_stop); });
}

// The whole FGMRES block solve (after solve_init and the first restart
// check) as one graph:  WHILE restart { restart body }.
cudaError_t build_graph(Solver& s, double tol_stop, cudaGraphExec_t* exec) {
  cudaError_t e;
  cudaGraph_t g, rbody;
  if ((e = cudaGraphCreate(&g, 0))) return e;
  auto fail = [&](cudaError_t ee) {
    cudaGraphDestroy(g);
    return ee;
  };
  if ((e = cudaGraphConditionalHandleCreate(&s.rst_c.h, g, 1, cudaGraphCondAssignDefault))) return fail(e);
  s.rst_c.use = 1;
  if ((e = add_while(g, s.rst_c.h, &rbody))) return fail(e);
  if ((e = fill_restart_body(s, rbody, tol_stop))) return fail(e);
  e = cudaGraphInstantiate(exec, g, 0);
  cudaGraphDestroy(g);
  return e;
}

// Capture fn() into graph g after `deps`; the nodes that end the captured
// work are returned in `frontier`.
template <typename F>
cudaError_t capture_after(cudaStream_t st, cudaGraph_t g, const std::vector<cudaGraphNode_t>& deps,
                          F&& fn, std::vector<cudaGraphNode_t>& frontier) {
  cudaError_t e = cudaStreamBeginCaptureToGraph(st, g, deps.data(), nullptr, deps.size(),
                                                cudaStreamCaptureModeThreadLocal);
  if (e) return e;
  const cudaError_t fe = fn();
  cudaStreamCaptureStatus status;
  const cudaGraphNode_t* d = nullptr;
  size_t nd = 0;
  cudaError_t ie = cudaStreamGetCaptureInfo(st, &status, nullptr, nullptr, &d, nullptr, &nd);
  if (!ie) frontier.assign(d, d + nd);
  cudaGraph_t out;
  e = cudaStreamEndCapture(st, &out);
  return fe ? fe : (ie ? ie : e);
}

// One independent branch of a batched graph: solve init (x0 = 0, or the
// guess in xout when x0_given) and first check,
// WHILE restart { ... }, scatter of the first `ncols_out` solution columns
// to `xout` (original order, columns N apart).
cudaError_t build_branch(cudaGraph_t g, Solver& s, double tol_stop, int64_t N, double* xout,
                         int ncols_out, bool x0_given) {
  cudaError_t e;
  if ((e = cudaGraphConditionalHandleCreate(&s.rst_c.h, g, 0, cudaGraphCondAssignDefault))) return e;
  s.rst_c.use = 1;
  std::vector<cudaGraphNode_t> f0, f1;
  if ((e = capture_after(s.st, g, {}, [&]() -> cudaError_t {
         cudaError_t ie = s.init_solution(x0_given ? xout : nullptr, N, ncols_out);
         if (ie) return ie;
         restart_check_kernel<<<1, 32, 0, s.st>>>(s.S, s.mc, s.G, s.rst_c, tol_stop); count_launch();
         return cudaGetLastError();
       }, f0)))
    return e;
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = s.rst_c.h;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t wnode;
  if ((e = cudaGraphAddNode(&wnode, g, f0.data(), nullptr, f0.size(), &np))) return e;
  if ((e = fill_restart_body(s, np.conditional.phGraph_out[0], tol_stop))) return e;
  return capture_after(s.st, g, {wnode}, [&]() -> cudaError_t {
    scatter_x64_kernel<<<dim3(s.vblocks, (unsigned)ncols_out), VT, 0, s.st>>>(s.xh, s.xl, s.P.perm, N,
                                                                                s.Np, xout); count_launch();
    return cudaGetLastError();
  }, f1);
}

// Columns per block for m right-hand sides: as few blocks of at most
// MAX_COLS columns as possible, all of the same width (the last one padded
// with zero right-hand sides, which stop at the first check).
int block_width(int m_rhs) {
  const int nblocks = (m_rhs + MAX_COLS - 1) / MAX_COLS;
  return (m_rhs + nblocks - 1) / nblocks;
}

// Sorted right-hand sides of columns [col0, col0 + ncols) of B (N x m, columns
// N apart) into s.b, the remaining columns of the block zero.
cudaError_t load_rhs(Solver& s, const float* B, int64_t N, int ncols) {
  cudaError_t e = gather_sorted(B, N, ncols, s.P.perm, s.Np, s.b, s.st);
  if (!e && ncols < s.mc) {
    fill_zero_kernel<<<s.vblocks, VT, 0, s.st>>>(s.b + (size_t)ncols * s.Np, (int64_t)(s.mc - ncols) * s.Np);
    count_launch();
    e = cudaGetLastError();
  }
  return e;
}

}  // namespace
}  // namespace krr

using namespace krr;

namespace {

krr_status resolve_opts(Ctx& c, const char* fn, const krr_fgmres_opts* opts, float gamma,
                        SolveCfg& cfg) {
  krr_fgmres_opts o;
  krr_fgmres_default_opts(&o);
  if (opts) o = *opts;
  if (o.restart < 1 || o.restart > MMAX)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: restart %d out of range [1, %d]", fn, o.restart, MMAX);
  if (o.max_cycles < 1) return set_error(c, KRR_ERR_INVALID_ARG, "%s: max_cycles < 1", fn);
  if (!(o.tol > 0.0) || !(o.tol < 1.0))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: tol must be in (0, 1)", fn);
  if (o.inner_maxit < 0 || o.inner_maxit > 100000)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: inner_maxit out of range", fn);
  if (o.inner_prec != KRR_FP32 && o.inner_prec != KRR_BF16 && o.inner_prec != KRR_FP16)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: unknown inner precision", fn);
  cfg.restart = o.restart;
  cfg.max_cycles = o.max_cycles;
  cfg.tol = o.tol;
  cfg.delta = o.delta >= 0.0 ? o.delta : (gamma > 0.f ? 10.0 * gamma : 1e-3);  // Sec. 6
  cfg.inner_tol = o.inner_tol >= 0.0 ? o.inner_tol : 10.0 * o.tol;             // Sec. 6
  cfg.inner_maxit = o.inner_maxit;
  cfg.inner_prec = o.inner_prec;
  cfg.graph = o.use_graph != 0;
  cfg.x0_given = o.x0_given != 0;
  if (!std::isfinite(cfg.delta) || !std::isfinite(cfg.inner_tol))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: delta / inner_tol not finite", fn);
  return KRR_OK;
}

void fill_info(const KState& h, float ms, krr_solve_info* info) {
  if (!info) return;
  info->outer_iters = h.outer_total;
  info->inner_iters = h.inner_total;
  info->cycles = h.cycles;
  info->breakdowns = h.breakdowns;
  info->relres_est = h.relres_est;
  info->relres_true = h.relres_true;
  info->time_ms = ms;
  info->status = (krr_status)h.status;
}

// One block solve of the sorted right-hand sides already in s.b (exec: the
// solve graph, or null for the host-driven loop); final states in hs.
krr_status fgmres_block(Solver& s, const SolveCfg& cfg, cudaGraphExec_t exec,
                        std::vector<KState>& hs, float* ms_out, const double* x0 = nullptr,
                        int64_t N = 0, int nx = 0) {
  Ctx& c = s.c;
  const char* fn = "krr_fgmres_solve";
  cudaError_t e;
  if ((e = upload_states(s, cfg, hs))) return cuda_error(c, e, fn);
  const double tol_stop = 0.5 * cfg.tol;
  cudaEventRecord(c.ev0, s.st);
  if ((e = s.init_solution(x0, N, nx))) return cuda_error(c, e, fn);
  // the first restart check turns x0, r0 = b - K x0 into the first cycle
  restart_check_kernel<<<1, 32, 0, s.st>>>(s.S, s.mc, s.G, Cond{}, tol_stop); count_launch();
  Group g;
  if (exec) {
    // the restart loop's default condition is 1: skip the graph when the
    // first check already stopped every column (b = 0)
    if ((e = read_group(s.G, g, s.st))) return cuda_error(c, e, fn);
    if (g.rst_any && (e = cudaGraphLaunch(exec, s.st))) return cuda_error(c, e, fn);
  } else {
    for (;;) {
      if ((e = read_group(s.G, g, s.st))) return cuda_error(c, e, fn);
      if (!g.rst_any) break;
      v0_kernel<<<s.vgrid(), VT, 0, s.st>>>(s.S, s.r64, s.V, s.vstride(), s.Np, PRED_RST, s.G, Cond{}); count_launch();
      for (;;) {
        cg_init_kernel<<<s.vgrid(), VT, 0, s.st>>>(s.S, s.V, s.vstride(), nullptr, s.Np, s.z, s.rr, s.p,
                                                   s.partials, PRED_ARN, s.G, Cond{}); count_launch();
        for (;;) {
          if ((e = read_group(s.G, g, s.st))) return cuda_error(c, e, fn);
          if (!g.cg_any) break;
          // predicated batch: iterations after convergence do nothing
          for (int b = 0; b < 8; ++b)
            if ((e = s.cg_iteration())) return cuda_error(c, e, fn);
        }
        if ((e = s.arnoldi_tail())) return cuda_error(c, e, fn);
        if ((e = read_group(s.G, g, s.st))) return cuda_error(c, e, fn);
        if (!g.arn_any) break;
      }
      if ((e = s.cycle_tail(tol_stop))) return cuda_error(c, e, fn);
    }
  }
  cudaEventRecord(c.ev1, s.st);
  if ((e = cudaEventSynchronize(c.ev1))) return cuda_error(c, e, fn);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c.ev0, c.ev1);
  *ms_out = ms;
  if ((e = cudaMemcpyAsync(hs.data(), s.S, sizeof(KState) * s.mc, cudaMemcpyDeviceToHost, s.st)) ||
      (e = cudaStreamSynchronize(s.st)))
    return cuda_error(c, e, fn);
  for (auto& h : hs)
    if (h.status == KRR_OK && h.relres_true > cfg.tol) h.status = KRR_NOT_CONVERGED;
  return KRR_OK;
}

// Enqueue the caller-stream join for the handle's work stream.
struct Join {
  Ctx& c;
  cudaStream_t ust;
  ~Join() {
    cudaEventRecord(c.ev_out, c.work);
    cudaStreamWaitEvent(ust, c.ev_out, 0);
  }
};

cudaError_t fork_work(Ctx& c, cudaStream_t ust) {
  cudaError_t e = cudaEventRecord(c.ev_in, ust);
  if (!e) e = cudaStreamWaitEvent(c.work, c.ev_in, 0);
  return e;
}

}  // namespace

extern "C" {

krr_status krr_fgmres_solve(krr_handle h, const float* X, int64_t N, int d, float sigma,
                            float gamma, const float* B, int m_rhs, double* Xsol,
                            const krr_fgmres_opts* opts, krr_solve_info* info, void* stream) {
  NvtxRange nvtx_range("krr_fgmres_solve");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_fgmres_solve";
  krr_status s = check_points(c, fn, X, N, d, sigma);
  if (s) return s;
  if (!(gamma >= 0.f) || !std::isfinite(gamma))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: gamma must be finite and >= 0", fn);
  if (m_rhs < 1 || m_rhs > 1024)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: m_rhs out of range [1, 1024]", fn);
  SolveCfg cfg;
  if ((s = resolve_opts(c, fn, opts, gamma, cfg))) return s;
  if (N == 0) return KRR_OK;
  if (!B || !Xsol) return set_error(c, KRR_ERR_INVALID_ARG, "%s: B or Xsol is NULL", fn);
  // all work on the handle's capturable stream, ordered after the caller's
  cudaStream_t ust = (cudaStream_t)stream;
  cudaStream_t st = c.work;
  {
    cudaError_t e0 = fork_work(c, ust);
    if (e0) return cuda_error(c, e0, fn);
  }
  Join join{c, ust};
  float *dX, *dB;
  double* dXs;
  bool sX, sB, sXs;
  if ((s = device_view(c, "stage.X", X, (size_t)N * d, true, st, &dX, &sX))) return s;
  if ((s = device_view(c, "stage.B", B, (size_t)N * m_rhs, true, st, &dB, &sB))) return s;
  if ((s = device_view_d(c, "stage.Xsol", Xsol, (size_t)N * m_rhs, cfg.x0_given, st, &dXs, &sXs)))
    return s;
  Solver sv(c);
  sv.st = st;
  cudaError_t e = prepare_points(c, dX, N, d, sigma, "kry.pts", sv.P, st);
  if (e) return cuda_error(c, e, fn);
  sv.Np = sv.P.Npad;
  sv.gamma = gamma;
  sv.mshift = (float)(gamma + cfg.delta);
  sv.inner_prec = cfg.inner_prec;
  const int width = block_width(m_rhs);
  if ((e = sv.alloc(cfg.restart, width))) return cuda_error(c, e, fn);
  // size every workspace buffer now: nothing may allocate inside a capture
  if ((e = sv.reserve())) return cuda_error(c, e, fn);
  cudaGraphExec_t exec = nullptr;
  sv.cg_c = sv.arn_c = sv.rst_c = Cond{};
  if (cfg.graph) {
    if ((e = build_graph(sv, 0.5 * cfg.tol, &exec))) {
      cudaGetLastError();
      return cuda_error(c, e, "krr_fgmres_solve (graph build)");
    }
  }
  struct ExecGuard {
    cudaGraphExec_t x;
    ~ExecGuard() {
      if (x) cudaGraphExecDestroy(x);
    }
  } guard{exec};
  krr_status worst = KRR_OK;
  std::vector<KState> hs;
  for (int col0 = 0; col0 < m_rhs; col0 += width) {
    const int ncols = std::min(width, m_rhs - col0);
    if ((e = load_rhs(sv, dB + (size_t)col0 * N, N, ncols))) return cuda_error(c, e, fn);
    float ms = 0.f;
    const double* x0 = cfg.x0_given ? dXs + (size_t)col0 * N : nullptr;
    if ((s = fgmres_block(sv, cfg, exec, hs, &ms, x0, N, ncols))) return s;
    scatter_x64_kernel<<<dim3(sv.vblocks, (unsigned)ncols), VT, 0, st>>>(sv.xh, sv.xl, sv.P.perm, N, sv.Np,
                                                                          dXs + (size_t)col0 * N); count_launch();
    if ((e = cudaGetLastError())) return cuda_error(c, e, fn);
    for (int k = 0; k < ncols; ++k) {
      if (info) fill_info(hs[k], ms, info + col0 + k);
      if (hs[k].status != KRR_OK && worst == KRR_OK) worst = (krr_status)hs[k].status;
    }
  }
  if (sXs && (e = cudaMemcpyAsync(Xsol, dXs, sizeof(double) * N * m_rhs, cudaMemcpyDeviceToHost, st)))
    return cuda_error(c, e, fn);
  krr_status de = read_device_error(c, st, fn);
  if (de) return de;
  if (worst == KRR_NOT_CONVERGED)
    set_error(c, worst, "%s: tolerance not reached in %d cycles", fn, cfg.max_cycles);
  else if (worst != KRR_OK)
    set_error(c, worst, "%s: solve failed", fn);
  return worst;
}

krr_status krr_fcg_solve(krr_handle h, const float* X, int64_t N, int d, float sigma, float gamma,
                         const float* B, int m_rhs, double* Xsol, const krr_fgmres_opts* opts,
                         krr_solve_info* info, void* stream) {
  NvtxRange nvtx_range("krr_fcg_solve");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_fcg_solve";
  krr_status s = check_points(c, fn, X, N, d, sigma);
  if (s) return s;
  if (!(gamma >= 0.f) || !std::isfinite(gamma))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: gamma must be finite and >= 0", fn);
  if (m_rhs < 1 || m_rhs > 1024)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: m_rhs out of range [1, 1024]", fn);
  SolveCfg cfg;
  if ((s = resolve_opts(c, fn, opts, gamma, cfg))) return s;
  if (N == 0) return KRR_OK;
  if (!B || !Xsol) return set_error(c, KRR_ERR_INVALID_ARG, "%s: B or Xsol is NULL", fn);
  cudaStream_t ust = (cudaStream_t)stream;
  cudaStream_t st = c.work;
  {
    cudaError_t e0 = fork_work(c, ust);
    if (e0) return cuda_error(c, e0, fn);
  }
  Join join{c, ust};
  float *dX, *dB;
  double* dXs;
  bool sX, sB, sXs;
  if ((s = device_view(c, "stage.X", X, (size_t)N * d, true, st, &dX, &sX))) return s;
  if ((s = device_view(c, "stage.B", B, (size_t)N * m_rhs, true, st, &dB, &sB))) return s;
  if ((s = device_view_d(c, "stage.Xsol", Xsol, (size_t)N * m_rhs, cfg.x0_given, st, &dXs, &sXs)))
    return s;
  Solver sv(c);
  sv.st = st;
  cudaError_t e = prepare_points(c, dX, N, d, sigma, "kry.pts", sv.P, st);
  if (e) return cuda_error(c, e, fn);
  sv.Np = sv.P.Npad;
  sv.gamma = gamma;
  sv.mshift = (float)(gamma + cfg.delta);
  sv.inner_prec = cfg.inner_prec;
  if ((e = sv.alloc(1, 1))) return cuda_error(c, e, fn);
  if ((e = sv.reserve())) return cuda_error(c, e, fn);
  const int mmax = cfg.restart, W = mmax + 1;
  const int64_t Np = sv.Np;
  void *Dv, *ADv, *dhv, *dlv, *rfv, *Fv;
  if ((e = c.ws.get("fcg.D", sizeof(double) * W * (size_t)Np, &Dv)) ||
      (e = c.ws.get("fcg.AD", sizeof(double) * W * (size_t)Np, &ADv)) ||
      (e = c.ws.get("fcg.dh", sizeof(float) * (size_t)Np, &dhv)) ||
      (e = c.ws.get("fcg.dl", sizeof(float) * (size_t)Np, &dlv)) ||
      (e = c.ws.get("fcg.rf", sizeof(float) * (size_t)Np, &rfv)) ||
      (e = c.ws.get("fcg.state", sizeof(FState), &Fv)))
    return cuda_error(c, e, fn);
  double *D = (double*)Dv, *AD = (double*)ADv;
  float *dh = (float*)dhv, *dl = (float*)dlv, *rf = (float*)rfv;
  FState* F = (FState*)Fv;
  const double tol_stop = 0.5 * cfg.tol;
  const int cap = cfg.restart * cfg.max_cycles;  // outer steps in total
  const unsigned vb = sv.vblocks;
  krr_status worst = KRR_OK;
  for (int col = 0; col < m_rhs; ++col) {
    if ((e = load_rhs(sv, dB + (size_t)col * N, N, 1))) return cuda_error(c, e, fn);
    std::vector<KState> hs;
    if ((e = upload_states(sv, cfg, hs))) return cuda_error(c, e, fn);  // inner CG settings
    FState hf;
    auto reset_window = [&](double bnorm) -> cudaError_t {
      memset(&hf, 0, sizeof(hf));
      hf.W = W;
      hf.bnorm = bnorm;
      cudaError_t ee = cudaMemcpyAsync(F, &hf, sizeof(FState), cudaMemcpyHostToDevice, st);
      if (!ee) ee = cudaStreamSynchronize(st);
      return ee;
    };
    cudaEventRecord(c.ev0, st);
    // x0 = 0 and r = b, or the given guess and r = b - K x0 (accurate)
    if ((e = sv.init_solution(cfg.x0_given ? dXs + (size_t)col * N : nullptr, N, 1)))
      return cuda_error(c, e, fn);
    KState ks;
    if ((e = read_state(c, sv.S, ks, st))) return cuda_error(c, e, fn);
    const double bnorm = ks.bnorm;
    if ((e = reset_window(bnorm))) return cuda_error(c, e, fn);
    double rr = ks.rnorm2, relres_true = bnorm > 0.0 ? std::sqrt(rr) / bnorm : 0.0;
    int it = 0, head = 0, cycles = 1;
    krr_status st_col = KRR_OK;
    bool done = bnorm == 0.0;
    while (!done) {
      if (rr <= tol_stop * tol_stop * bnorm * bnorm || it >= cap || hf.brk) {
        // the recursive residual met the tolerance (or the cap / a breakdown):
        // check the true one with the accurate product
        if ((e = sv.residual(false))) return cuda_error(c, e, fn);
        if ((e = read_state(c, sv.S, ks, st))) return cuda_error(c, e, fn);
        relres_true = std::sqrt(ks.rnorm2) / bnorm;
        if (!std::isfinite(relres_true)) {
          st_col = KRR_ERR_NONFINITE;
          break;
        }
        if (relres_true <= tol_stop) break;
        if (it >= cap || hf.brk) {
          st_col = KRR_NOT_CONVERGED;
          break;
        }
        // restart from the true residual with an empty window (a step of
        // iterative refinement)
        rr = ks.rnorm2;
        head = 0;
        ++cycles;
        if ((e = reset_window(bnorm))) return cuda_error(c, e, fn);
      }
      // z = M^-1 r by truncated CG (float32 right-hand side)
      fcg_to_float_kernel<<<vb, VT, 0, st>>>(sv.r64, Np, rf); count_launch();
      cg_init_kernel<<<vb, VT, 0, st>>>(sv.S, nullptr, 0, rf, Np, sv.z, sv.rr, sv.p, sv.partials, PRED_ALL,
                                        sv.G, Cond{}); count_launch();
      for (;;) {
        Group g;
        if ((e = read_group(sv.G, g, st))) return cuda_error(c, e, fn);
        if (!g.cg_any) break;
        for (int b = 0; b < 8; ++b)
          if ((e = sv.cg_iteration())) return cuda_error(c, e, fn);
      }
      // the new direction, its product and the step
      fcg_beta_kernel<<<vb, VT, 0, st>>>(F, sv.z, AD, Np, sv.partials); count_launch();
      fcg_dir_kernel<<<vb, VT, 0, st>>>(F, sv.z, D, Np, dh, dl); count_launch();
      if ((e = mvp_acc_launch(c, sv.P, dh, dl, gamma, 0.0, nullptr, 1.0, AD + (size_t)head * Np, nullptr, st)))
        return cuda_error(c, e, fn);
      fcg_alpha_kernel<<<vb, VT, 0, st>>>(F, D, AD, sv.r64, Np, sv.partials); count_launch();
      fcg_update_kernel<<<vb, VT, 0, st>>>(F, D, AD, Np, sv.xh, sv.xl, sv.r64, sv.partials, mmax); count_launch();
      if ((e = cudaGetLastError())) return cuda_error(c, e, fn);
      if ((e = cudaMemcpyAsync(&hf, F, sizeof(FState), cudaMemcpyDeviceToHost, st)) ||
          (e = cudaStreamSynchronize(st)))
        return cuda_error(c, e, fn);
      rr = hf.rr;
      head = hf.head;
      ++it;
    }
    cudaEventRecord(c.ev1, st);
    if ((e = cudaEventSynchronize(c.ev1))) return cuda_error(c, e, fn);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.ev0, c.ev1);
    if ((e = read_state(c, sv.S, ks, st))) return cuda_error(c, e, fn);
    scatter_x64_kernel<<<vb, VT, 0, st>>>(sv.xh, sv.xl, sv.P.perm, N, Np, dXs + (size_t)col * N); count_launch();
    if (info) {
      krr_solve_info& in = info[col];
      in.outer_iters = it;
      in.inner_iters = ks.inner_total;
      in.cycles = cycles;
      in.breakdowns = ks.breakdowns + hf.brk;
      in.relres_est = bnorm > 0.0 ? std::sqrt(rr) / bnorm : 0.0;
      in.relres_true = relres_true;
      in.time_ms = ms;
      in.status = st_col;
    }
    if (st_col != KRR_OK && worst == KRR_OK) worst = st_col;
  }
  if (sXs && (e = cudaMemcpyAsync(Xsol, dXs, sizeof(double) * N * m_rhs, cudaMemcpyDeviceToHost, st)))
    return cuda_error(c, e, fn);
  krr_status de = read_device_error(c, st, fn);
  if (de) return de;
  if (worst != KRR_OK) set_error(c, worst, "%s: a right-hand side did not reach the tolerance", fn);
  return worst;
}

krr_status krr_cg_solve(krr_handle h, const float* X, int64_t N, int d, float sigma, float shift,
                        const float* b, double* x, double tol, int maxit, krr_precision prec,
                        krr_solve_info* info, void* stream) {
  NvtxRange nvtx_range("krr_cg_solve");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_cg_solve";
  krr_status s = check_points(c, fn, X, N, d, sigma);
  if (s) return s;
  if (!(shift >= 0.f) || !std::isfinite(shift))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: shift must be finite and >= 0", fn);
  if (!(tol > 0.0) || !(tol < 1.0)) return set_error(c, KRR_ERR_INVALID_ARG, "%s: tol must be in (0, 1)", fn);
  if (maxit < 0) return set_error(c, KRR_ERR_INVALID_ARG, "%s: maxit < 0", fn);
  if (prec != KRR_FP32 && prec != KRR_BF16 && prec != KRR_FP16)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: unknown precision", fn);
  if (N == 0) return KRR_OK;
  if (!b || !x) return set_error(c, KRR_ERR_INVALID_ARG, "%s: b or x is NULL", fn);
  cudaStream_t ust = (cudaStream_t)stream;
  cudaStream_t st = c.work;
  {
    cudaError_t e0 = fork_work(c, ust);
    if (e0) return cuda_error(c, e0, fn);
  }
  Join join{c, ust};
  float *dX, *db;
  double* dx;
  bool sX, sb, sx;
  if ((s = device_view(c, "stage.X", X, (size_t)N * d, true, st, &dX, &sX))) return s;
  if ((s = device_view(c, "stage.B", b, (size_t)N, true, st, &db, &sb))) return s;
  if ((s = device_view_d(c, "stage.Xsol", x, (size_t)N, true, st, &dx, &sx))) return s;
  Solver sv(c);
  sv.st = st;
  cudaError_t e = prepare_points(c, dX, N, d, sigma, "kry.pts", sv.P, st);
  if (e) return cuda_error(c, e, fn);
  sv.Np = sv.P.Npad;
  sv.gamma = shift;   // the operator of this solve is K_hat + shift I throughout
  sv.mshift = shift;
  sv.inner_prec = prec;
  if ((e = sv.alloc(1, 1))) return cuda_error(c, e, fn);
  if ((e = sv.reserve())) return cuda_error(c, e, fn);
  KState hs;
  memset(&hs, 0, sizeof(hs));
  hs.status = KRR_OK;
  if ((e = cudaMemcpyAsync(sv.S, &hs, sizeof(KState), cudaMemcpyHostToDevice, st))) return cuda_error(c, e, fn);
  if ((e = cudaStreamSynchronize(st))) return cuda_error(c, e, fn);
  if ((e = gather_sorted(db, N, 1, sv.P.perm, sv.Np, sv.b, st))) return cuda_error(c, e, fn);
  cudaEventRecord(c.ev0, st);
  x_from64_kernel<<<sv.vblocks, VT, 0, st>>>(dx, sv.P.perm, N, sv.Np, sv.xh, sv.xl); count_launch();
  bnorm_kernel<<<sv.vblocks, VT, 0, st>>>(sv.S, sv.b, sv.Np, sv.partials); count_launch();
  if ((e = sv.residual(false))) return cuda_error(c, e, fn);
  const double tol_stop = tol;
  for (;;) {
    cg_cycle_kernel<<<1, 1, 0, st>>>(sv.S, tol_stop, maxit); count_launch();
    KState hcur;
    if ((e = read_state(c, sv.S, hcur, st))) return cuda_error(c, e, fn);
    if (!hcur.restart_cont) break;
    cg_init_kernel<<<sv.vblocks, VT, 0, st>>>(sv.S, sv.r64, 0, nullptr, sv.Np, sv.z, sv.rr, sv.p,
                                              sv.partials, PRED_ALL, sv.G, Cond{}); count_launch();
    Group g;
    for (;;) {
      for (int bt = 0; bt < 16; ++bt)
        if ((e = sv.cg_iteration())) return cuda_error(c, e, fn);
      if ((e = read_group(sv.G, g, st))) return cuda_error(c, e, fn);
      if (!g.cg_any) break;
    }
    x_add_kernel<<<sv.vblocks, VT, 0, st>>>(sv.z, sv.Np, sv.xh, sv.xl); count_launch();
    if ((e = sv.residual(false))) return cuda_error(c, e, fn);
  }
  cudaEventRecord(c.ev1, st);
  if ((e = cudaEventSynchronize(c.ev1))) return cuda_error(c, e, fn);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c.ev0, c.ev1);
  if ((e = read_state(c, sv.S, hs, st))) return cuda_error(c, e, fn);
  scatter_x64_kernel<<<sv.vblocks, VT, 0, st>>>(sv.xh, sv.xl, sv.P.perm, N, sv.Np, dx); count_launch();
  if (sx && (e = cudaMemcpyAsync(x, dx, sizeof(double) * N, cudaMemcpyDeviceToHost, st)))
    return cuda_error(c, e, fn);
  krr_status de = read_device_error(c, st, fn);
  if (de) return de;
  if (info) {
    info->outer_iters = hs.inner_total;
    info->inner_iters = 0;
    info->cycles = hs.cycles;
    info->breakdowns = hs.breakdowns;
    info->relres_est = sqrt(hs.rho) / (hs.bnorm > 0 ? hs.bnorm : 1.0);
    info->relres_true = hs.relres_true;
    info->time_ms = ms;
    info->status = (krr_status)hs.status;
  }
  if (hs.status != KRR_OK)
    return set_error(c, (krr_status)hs.status, "%s: tolerance not reached in %d iterations", fn, maxit);
  return KRR_OK;
}

krr_status krr_fgmres_solve_batched(krr_handle h, const krr_problem* probs, int nprob, int d,
                                    float sigma, int m_rhs, const krr_fgmres_opts* opts,
                                    krr_solve_info* info, void* stream) {
  NvtxRange nvtx_range("krr_fgmres_solve_batched");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_fgmres_solve_batched";
  if (nprob < 0 || nprob > 4096 || (nprob > 0 && !probs))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: nprob out of range [0, 4096] or probs NULL", fn);
  if (m_rhs < 1 || m_rhs > 64) return set_error(c, KRR_ERR_INVALID_ARG, "%s: m_rhs out of range [1, 64]", fn);
  if ((int64_t)nprob * m_rhs > 4096)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: nprob * m_rhs > 4096", fn);
  krr_status s;
  for (int k = 0; k < nprob; ++k) {
    if ((s = check_points(c, fn, probs[k].X, probs[k].N, d, sigma))) return s;
    if (!(probs[k].gamma >= 0.f) || !std::isfinite(probs[k].gamma))
      return set_error(c, KRR_ERR_INVALID_ARG, "%s: problem %d: gamma must be finite and >= 0", fn, k);
    if (probs[k].N > 0 && (!probs[k].B || !probs[k].Xsol || !is_device_ptr(c, probs[k].X) ||
                           !is_device_ptr(c, probs[k].B) || !is_device_ptr(c, probs[k].Xsol)))
      return set_error(c, KRR_ERR_INVALID_ARG, "%s: problem %d: arrays must be device arrays", fn, k);
  }
  SolveCfg cfg;
  if ((s = resolve_opts(c, fn, opts, 0.f, cfg))) return s;
  cudaStream_t ust = (cudaStream_t)stream;
  cudaStream_t st = c.work;
  {
    cudaError_t e0 = fork_work(c, ust);
    if (e0) return cuda_error(c, e0, fn);
  }
  Join join{c, ust};
  cudaError_t e;
  // One branch per (problem, block of right-hand sides): a block solve with
  // its own context; a problem's blocks share its prepared points.
  const int width = block_width(m_rhs);
  const int per_prob = (m_rhs + width - 1) / width;
  // graphs of at most BRANCHES_PER_GRAPH independent branches, launched in
  // turn (larger graphs of nested conditional loops are not used: one of
  // 1024 branches failed on the device)
  constexpr int BRANCHES_PER_GRAPH = 32;
  int nbr = 0;
  for (int k = 0; k < nprob; ++k)
    if (probs[k].N > 0) nbr += per_prob;
  if (nbr == 0) return KRR_OK;
  // concurrent branches share the SMs: plan each product for its share
  const int slots = std::max(16, 2 * c.num_sms * 4 / std::min(nbr, BRANCHES_PER_GRAPH));
  struct Branch {
    std::unique_ptr<Solver> sv;
    int prob, col0, ncols;
    Ctx* ctx;
  };
  std::vector<Branch> br;
  std::vector<PointsDev> pts(nprob);
  for (int k = 0; k < nprob; ++k) {
    const krr_problem& pr = probs[k];
    if (pr.N == 0) continue;
    const double delta = opts && opts->delta >= 0.0 ? opts->delta : (pr.gamma > 0.f ? 10.0 * pr.gamma : 1e-3);
    for (int col0 = 0; col0 < m_rhs; col0 += width) {
      Ctx* bc;
      if ((e = sub_context(c, br.size(), &bc))) return cuda_error(c, e, fn);
      bc->plan_slots = slots;
      bc->use_tcgen05 = c.use_tcgen05;
      bc->tcgen05_kind = c.tcgen05_kind;
      bc->tcgen05_auto = c.tcgen05_auto;
      bc->kernel_family = c.kernel_family;
      bc->autotune = c.autotune;
      bc->highd_tcgen05 = c.highd_tcgen05;
      bc->direct_tensor = c.direct_tensor;
      if (col0 == 0 && (e = prepare_points(*bc, pr.X, pr.N, d, sigma, "bat.pts", pts[k], st)))
        return cuda_error(c, e, fn);
      auto so = std::make_unique<Solver>(*bc);
      so->st = st;
      so->P = pts[k];
      so->Np = pts[k].Npad;
      so->gamma = pr.gamma;
      so->mshift = (float)(pr.gamma + delta);
      so->inner_prec = cfg.inner_prec;
      const int ncols = std::min(width, m_rhs - col0);
      if ((e = so->alloc(cfg.restart, width))) return cuda_error(c, e, fn);
      if ((e = so->reserve())) return cuda_error(c, e, fn);
      std::vector<KState> hs;
      if ((e = upload_states(*so, cfg, hs))) return cuda_error(c, e, fn);
      if ((e = load_rhs(*so, pr.B + (size_t)col0 * pr.N, pr.N, ncols))) return cuda_error(c, e, fn);
      br.push_back(Branch{std::move(so), k, col0, ncols, bc});
    }
  }
  // Graphs run one after another and each lasts as long as its slowest
  // branch, so branches are grouped by their expected cost: N^2 pairs per
  // product times about 1 / sqrt(gamma) Krylov steps (the conditioning of
  // K_hat + gamma I, Sec. 3), most expensive first.
  std::stable_sort(br.begin(), br.end(), [&](const Branch& a, const Branch& b) {
    auto cost = [&](const Branch& x) {
      const double n = (double)probs[x.prob].N;
      return n * n / std::sqrt(std::max((double)probs[x.prob].gamma, 1e-12));
    };
    return cost(a) > cost(b);
  });
  float ms = 0.f;
  for (size_t b0 = 0; b0 < br.size(); b0 += BRANCHES_PER_GRAPH) {
    const size_t b1 = std::min(br.size(), b0 + (size_t)BRANCHES_PER_GRAPH);
    cudaGraph_t g;
    if ((e = cudaGraphCreate(&g, 0))) return cuda_error(c, e, fn);
    for (size_t b = b0; b < b1; ++b) {
      const Branch& x = br[b];
      const krr_problem& pr = probs[x.prob];
      if ((e = build_branch(g, *x.sv, 0.5 * cfg.tol, pr.N, pr.Xsol + (size_t)x.col0 * pr.N, x.ncols,
                            cfg.x0_given))) {
        cudaGraphDestroy(g);
        cudaGetLastError();
        return cuda_error(c, e, "krr_fgmres_solve_batched (graph build)");
      }
    }
    cudaGraphExec_t exec;
    e = cudaGraphInstantiate(&exec, g, 0);
    cudaGraphDestroy(g);
    if (e) return cuda_error(c, e, "krr_fgmres_solve_batched (graph instantiate)");
    cudaEventRecord(c.ev0, st);
    e = cudaGraphLaunch(exec, st);
    cudaEventRecord(c.ev1, st);
    if (!e) e = cudaEventSynchronize(c.ev1);
    cudaGraphExecDestroy(exec);
    if (e) return cuda_error(c, e, fn);
    float part_ms = 0.f;
    cudaEventElapsedTime(&part_ms, c.ev0, c.ev1);
    ms += part_ms;
  }
  krr_status worst = KRR_OK;
  for (const Branch& x : br) {
    std::vector<KState> hs(x.sv->mc);
    if ((e = cudaMemcpyAsync(hs.data(), x.sv->S, sizeof(KState) * x.sv->mc, cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
      return cuda_error(c, e, fn);
    for (int k = 0; k < x.ncols; ++k) {
      KState& hk = hs[k];
      if (hk.status == KRR_OK && hk.relres_true > cfg.tol) hk.status = KRR_NOT_CONVERGED;
      if (info) fill_info(hk, ms, info + (size_t)x.prob * m_rhs + x.col0 + k);
      if (hk.status != KRR_OK && worst == KRR_OK) worst = (krr_status)hk.status;
    }
  }
  // device error words of the branches' contexts (read through this handle's
  // pinned status word)
  for (const Branch& x : br) {
    if ((e = cudaMemcpyAsync(c.h_status, x.ctx->d_err, sizeof(int), cudaMemcpyDeviceToHost, st)) ||
        (e = cudaStreamSynchronize(st)))
      return cuda_error(c, e, fn);
    if (*c.h_status != DEV_OK) {
      const int v = *c.h_status;
      cudaMemsetAsync(x.ctx->d_err, 0, sizeof(int), st);
      return set_error(c, v == DEV_TIMEOUT ? KRR_ERR_TIMEOUT : KRR_ERR_NONFINITE,
                       "%s: problem %d: device error %d", fn, x.prob, v);
    }
  }
  if (worst != KRR_OK) set_error(c, worst, "%s: a problem did not reach the tolerance", fn);
  return worst;
}

}  // extern "C"
