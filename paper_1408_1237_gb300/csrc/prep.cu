// Point preparation (hot-path step A1): Morton-order sort, scaling and
// tile-blocked packing of the points.
//
// The Gaussian of Eq. 2 becomes a base-2 exponential of scaled points:
//   exp(-|x_i - x_j|^2 / (2 sigma^2)) = 2^(-s^2 |x_i - x_j|^2),
//   s = sqrt(log2(e) / (2 sigma^2)),
// so the product kernels evaluate it with one MUFU.EX2 per pair.  (Under the
// Matern kernel of Sec. 6.1 the scale is s = sqrt(3) / h and the kernels form
// a = s |x_i - x_j|; every block takes the direct form.)  The packed
// copy keeps the caller's float32 coordinates unscaled: the kernels scale
// only after recentring or differencing, where no significant digits are
// lost (scaling first would round s*x at the magnitude of s*x).  Sorting the
// points along a Morton (Z-order) curve makes every block of consecutive
// points spatially compact, which the product kernels use to recentre their
// arithmetic (see mvp.cu).  K is invariant under a simultaneous permutation of
// rows and columns, so the solvers work in sorted order throughout and only
// the right-hand sides and solutions are permuted in and out.
#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "internal.h"

namespace krr {

namespace {

constexpr int BBOX_THREADS = 256;
constexpr int SORT_THREADS = 256;
constexpr int SORT_ITEMS = 8;
constexpr int SORT_CHUNK = SORT_THREADS * SORT_ITEMS;  // elements per sort block
constexpr int SCAN_THREADS = 1024;

// Per-block partial bounding boxes: part[b*2d + k] = min, part[b*2d + d + k] = max.
// Non-finite coordinates raise DEV_NONFINITE.
__global__ void bbox_partial_kernel(const float* __restrict__ X, int64_t N, int d,
                                    float* __restrict__ part, int* err) {
  extern __shared__ float sh[];  // 2 * d * (BBOX_THREADS/32)
  const int nw = blockDim.x >> 5, w = threadIdx.x >> 5, l = threadIdx.x & 31;
  for (int k = 0; k < d; ++k) {
    float lo = INFINITY, hi = -INFINITY;
    bool bad = false;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
         i += (int64_t)gridDim.x * blockDim.x) {
      const float v = X[i * d + k];
      if (!isfinite(v)) bad = true;
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
    if (bad) atomicExch(err, DEV_NONFINITE);
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (l == 0) {
      sh[k * nw + w] = lo;
      sh[(d + k) * nw + w] = hi;
    }
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 2 * d; t += blockDim.x) {
    const bool is_min = t < d;
    float v = is_min ? INFINITY : -INFINITY;
    for (int ww = 0; ww < nw; ++ww) v = is_min ? fminf(v, sh[t * nw + ww]) : fmaxf(v, sh[t * nw + ww]);
    part[(int64_t)blockIdx.x * 2 * d + t] = v;
  }
}

__global__ void bbox_final_kernel(const float* __restrict__ part, int nblocks, int d,
                                  float* __restrict__ bbox) {
  for (int t = threadIdx.x; t < 2 * d; t += blockDim.x) {
    const bool is_min = t < d;
    float v = is_min ? INFINITY : -INFINITY;
    for (int b = 0; b < nblocks; ++b) {
      const float u = part[(int64_t)b * 2 * d + t];
      v = is_min ? fminf(v, u) : fmaxf(v, u);
    }
    bbox[t] = v;
  }
}

// Morton key over the first dk = min(d, 30) coordinates, `bits` bits each,
// bit b of coordinate k placed at key bit b*dk + k.
__global__ void morton_kernel(const float* __restrict__ X, int64_t N, int d, int dk, int bits,
                              const float* __restrict__ bbox, uint32_t* __restrict__ keys,
                              int* __restrict__ vals) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const uint32_t cells = 1u << bits;
  uint32_t key = 0;
  for (int k = 0; k < dk; ++k) {
    const float lo = bbox[k], hi = bbox[d + k];
    const float ext = hi - lo;
    uint32_t u = 0;
    if (ext > 0.f) {
      float f = (X[i * d + k] - lo) / ext * (float)cells;
      f = fminf(fmaxf(f, 0.f), (float)(cells - 1));
      u = (uint32_t)f;
    }
    for (int b = 0; b < bits; ++b) key |= ((u >> b) & 1u) << (b * dk + k);
  }
  keys[i] = key;
  vals[i] = (int)i;
}

// Radix sort pass 1: digit histogram of each chunk, stored digit-major:
// hist[digit * nchunks + chunk].
__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t N, int shift,
                                  uint32_t* __restrict__ hist, int nchunks) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
  for (int e = threadIdx.x; e < SORT_CHUNK; e += SORT_THREADS) {
    const int64_t i = base + e;
    if (i < N) atomicAdd(&h[(keys[i] >> shift) & 0xFFu], 1u);
  }
  __syncthreads();
  hist[(int64_t)threadIdx.x * nchunks + blockIdx.x] = h[threadIdx.x];
}

// Radix sort pass 2: exclusive scan of the digit-major histogram (one block).
__global__ void radix_scan_kernel(uint32_t* __restrict__ hist, int64_t L) {
  __shared__ uint32_t sums[SCAN_THREADS];
  const int64_t per = (L + SCAN_THREADS - 1) / SCAN_THREADS;
  const int64_t lo = threadIdx.x * per, hi = min(L, lo + per);
  uint32_t s = 0;
  for (int64_t e = lo; e < hi; ++e) s += hist[e];
  sums[threadIdx.x] = s;
  __syncthreads();
  // Hillis-Steele inclusive scan over the per-thread sums
  for (int o = 1; o < SCAN_THREADS; o <<= 1) {
    const uint32_t v = threadIdx.x >= o ? sums[threadIdx.x - o] : 0u;
    __syncthreads();
    sums[threadIdx.x] += v;
    __syncthreads();
  }
  uint32_t run = threadIdx.x ? sums[threadIdx.x - 1] : 0u;
  for (int64_t e = lo; e < hi; ++e) {
    const uint32_t v = hist[e];
    hist[e] = run;
    run += v;
  }
}

// Radix sort pass 3: stable scatter.  Thread t owns digit t and walks the
// chunk in order, so equal digits keep their relative order.
__global__ void radix_scatter_kernel(const uint32_t* __restrict__ keys_in,
                                     const int* __restrict__ vals_in, int64_t N, int shift,
                                     const uint32_t* __restrict__ offs, int nchunks,
                                     uint32_t* __restrict__ keys_out, int* __restrict__ vals_out) {
  __shared__ uint32_t sk[SORT_CHUNK];
  __shared__ int sv[SORT_CHUNK];
  const int64_t base = (int64_t)blockIdx.x * SORT_CHUNK;
  const int n = (int)min((int64_t)SORT_CHUNK, N - base);
  for (int e = threadIdx.x; e < n; e += SORT_THREADS) {
    sk[e] = keys_in[base + e];
    sv[e] = vals_in[base + e];
  }
  __syncthreads();
  const uint32_t digit = threadIdx.x;
  uint32_t pos = offs[(int64_t)digit * nchunks + blockIdx.x];
  for (int e = 0; e < n; ++e) {
    const uint32_t k = sk[e];
    if (((k >> shift) & 0xFFu) == digit) {
      keys_out[pos] = k;
      vals_out[pos] = sv[e];
      ++pos;
    }
  }
}

// Tile-blocked pack: xs[(i/TS)*d*TS + k*TS + i%TS] = X[perm[i]*d + k]; the
// padded points i >= N repeat the last sorted point (their weights are zero),
// so every coordinate the product kernels meet is finite and nearby.
__global__ void pack_kernel(const float* __restrict__ X, int64_t N, int64_t Npad, int d_in, int d,
                            const int* __restrict__ perm, float* __restrict__ xs) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  const int64_t tile = i / TS, lane = i % TS;
  float* dst = xs + tile * (int64_t)d * TS + lane;
  const int64_t src = (int64_t)perm[i < N ? i : N - 1] * d_in;
  for (int k = 0; k < d; ++k) dst[(int64_t)k * TS] = k < d_in ? X[src + k] : 0.f;  // padding: 0
}

__global__ void gather_kernel(const float* __restrict__ in, int64_t N, int m,
                              const int* __restrict__ perm, int64_t Npad, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= Npad) return;
  const int64_t p = i < N ? perm[i] : -1;
  for (int c = 0; c < m; ++c) out[(int64_t)c * Npad + i] = p >= 0 ? in[(int64_t)c * N + p] : 0.f;
}

__global__ void scatter_kernel(const float* __restrict__ in, int64_t Npad, int64_t N, int m,
                               const int* __restrict__ perm, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= N) return;
  const int64_t p = perm[i];
  for (int c = 0; c < m; ++c) out[(int64_t)c * N + p] = in[(int64_t)c * Npad + i];
}

// Warp-block metadata: one warp per block of WB = 32*T sorted points.
// ctr = centre of the bounding box of the block's valid points (raw
// coordinates); flag = 1 when every valid point lies within squared radius
// EXPANDED_R2 of the centre in scaled units s (x - c).
__global__ void blkinfo_kernel(const float* __restrict__ xs, int64_t N, int d, int T, float s,
                               int64_t nblk, float* __restrict__ ctr, int* __restrict__ flag,
                               int allow_expanded) {
  const int64_t b = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (b >= nblk) return;
  float r2max = 0.f;
  float c[64];
  for (int k = 0; k < d; ++k) {
    float lo = INFINITY, hi = -INFINITY;
    for (int u = 0; u < T; ++u) {
      const int64_t i = b * 32 * T + lane + 32 * u;
      if (i < N) {
        const float v = xs[(i / TS) * (int64_t)d * TS + (int64_t)k * TS + (i % TS)];
        lo = fminf(lo, v);
        hi = fmaxf(hi, v);
      }
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    c[k] = 0.5f * (lo + hi);
    if (lane == 0) ctr[b * d + k] = c[k];
  }
  for (int u = 0; u < T; ++u) {
    const int64_t i = b * 32 * T + lane + 32 * u;
    if (i < N) {
      float a = 0.f;
      for (int k = 0; k < d; ++k) {
        const float v = s * (xs[(i / TS) * (int64_t)d * TS + (int64_t)k * TS + (i % TS)] - c[k]);
        a = fmaf(v, v, a);
      }
      r2max = fmaxf(r2max, a);
    }
  }
  r2max = warp_max(r2max);
  if (lane == 0) flag[b] = (allow_expanded && r2max <= EXPANDED_R2) ? 1 : 0;
}

// Stable partition of the warp blocks: expanded-form blocks first (one block
// of SCAN_THREADS threads).  n_exp = number of expanded-form blocks.
__global__ void order_kernel(const int* __restrict__ flag, int64_t nblk, int* __restrict__ order,
                             int* __restrict__ n_exp) {
  __shared__ int sums[SCAN_THREADS];
  const int64_t per = (nblk + SCAN_THREADS - 1) / SCAN_THREADS;
  const int64_t lo = threadIdx.x * per, hi = min(nblk, lo + per);
  int cnt = 0;
  for (int64_t b = lo; b < hi; ++b) cnt += flag[b];
  sums[threadIdx.x] = cnt;
  __syncthreads();
  for (int o = 1; o < SCAN_THREADS; o <<= 1) {
    const int v = threadIdx.x >= o ? sums[threadIdx.x - o] : 0;
    __syncthreads();
    sums[threadIdx.x] += v;
    __syncthreads();
  }
  const int total = sums[SCAN_THREADS - 1];
  int e = threadIdx.x ? sums[threadIdx.x - 1] : 0;  // expanded blocks before lo
  int64_t dpos = total + (lo - e);                   // direct blocks before lo, after all expanded
  for (int64_t b = lo; b < hi; ++b) {
    if (flag[b]) order[e++] = (int)b;
    else order[dpos++] = (int)b;
  }
  if (threadIdx.x == 0) *n_exp = total;
}

// Bounding box of every source tile of TS sorted points (padded points repeat
// the last real one, so including them leaves the box unchanged): one warp
// per tile; tbox[t*2d + k] = centre, tbox[t*2d + d + k] = half-width.
__global__ void tilebox_kernel(const float* __restrict__ xs, int64_t ntiles, int d,
                               float* __restrict__ tbox) {
  const int64_t t = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= ntiles) return;
  for (int k = 0; k < d; ++k) {
    float lo = INFINITY, hi = -INFINITY;
    for (int j = lane; j < TS; j += 32) {
      const float v = xs[t * (int64_t)d * TS + (int64_t)k * TS + j];
      lo = fminf(lo, v);
      hi = fmaxf(hi, v);
    }
    lo = warp_min(lo);
    hi = warp_max(hi);
    if (lane == 0) {
      tbox[t * 2 * d + k] = 0.5f * (lo + hi);
      tbox[t * 2 * d + d + k] = 0.5f * (hi - lo);
    }
  }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t gather_sorted(const float* in, int64_t N, int m, const int* perm, int64_t Npad,
                          float* out, cudaStream_t st) {
  if (Npad == 0) return cudaSuccess;
  gather_kernel<<<blocks_for(Npad, 256), 256, 0, st>>>(in, N, m, perm, Npad, out); count_launch();
  return cudaGetLastError();
}

cudaError_t scatter_orig(const float* in, int64_t Npad, int64_t N, int m, const int* perm,
                         float* out, cudaStream_t st) {
  if (N == 0) return cudaSuccess;
  scatter_kernel<<<blocks_for(N, 256), 256, 0, st>>>(in, Npad, N, m, perm, out); count_launch();
  return cudaGetLastError();
}

cudaError_t prepare_points(Ctx& c, const float* X, int64_t N, int d, float sigma,
                           const char* tag, PointsDev& P, cudaStream_t st) {
  const std::string t(tag);
  const int d_in = d;
  d = padded_dim(d_in);
  P.N = N;
  P.d = d;
  P.d_in = d_in;
  P.Npad = round_up(std::max<int64_t>(N, 1), PAD);
  P.kfam = c.kernel_family;
  if (P.kfam == KRR_KERNEL_MATERN32)
    P.s2 = 3.0 / ((double)sigma * (double)sigma);  // (sqrt(3) / h)^2
  else
    P.s2 = 1.0 / (std::log(2.0) * 2.0 * (double)sigma * (double)sigma);  // log2(e) / (2 sigma^2)
  P.scale = (float)std::sqrt(P.s2);
  cudaError_t e;
  void *xs, *perm, *ka, *kb, *va, *vb, *hist, *bbp, *bb;
  const int nbb = (int)std::min<int64_t>(blocks_for(N, BBOX_THREADS), 256);
  // the expanded form factors the Gaussian; other kernels take the direct
  // form.  Warp blocks (the packed CUDA-core kernel, d <= 8) and super-blocks
  // (the tensor-core kernels, d <= 64) are classified separately.
  const bool gauss = P.kfam == KRR_KERNEL_GAUSSIAN;
  const int allow_expanded = (d <= 8 && gauss) ? 1 : 0;
  const int allow_expanded_sb = gauss ? 1 : 0;
  const int nchunks = (int)blocks_for(N, SORT_CHUNK);
  if ((e = c.ws.get(t + ".xs", sizeof(float) * P.Npad * d, &xs))) return e;
  if ((e = c.ws.get(t + ".perm", sizeof(int) * P.Npad, &perm))) return e;
  if ((e = c.ws.get("sort.ka", sizeof(uint32_t) * N, &ka))) return e;
  if ((e = c.ws.get("sort.kb", sizeof(uint32_t) * N, &kb))) return e;
  if ((e = c.ws.get("sort.va", sizeof(int) * N, &va))) return e;
  if ((e = c.ws.get("sort.vb", sizeof(int) * N, &vb))) return e;
  if ((e = c.ws.get("sort.hist", sizeof(uint32_t) * 256 * (size_t)nchunks, &hist))) return e;
  if ((e = c.ws.get("sort.bbp", sizeof(float) * 2 * d_in * (size_t)nbb, &bbp))) return e;
  if ((e = c.ws.get("sort.bb", sizeof(float) * 2 * d_in, &bb))) return e;
  P.xs = (float*)xs;
  P.perm = (int*)perm;

  bbox_partial_kernel<<<nbb, BBOX_THREADS, sizeof(float) * 2 * d_in * (BBOX_THREADS / 32), st>>>(
      X, N, d_in, (float*)bbp, c.d_err); count_launch();
  bbox_final_kernel<<<1, 128, 0, st>>>((const float*)bbp, nbb, d_in, (float*)bb); count_launch();
  const int dk = std::min(d_in, 30);
  const int bits = std::max(1, std::min(16, 30 / dk));
  morton_kernel<<<blocks_for(N, 256), 256, 0, st>>>(X, N, d_in, dk, bits, (const float*)bb,
                                                    (uint32_t*)ka, (int*)va); count_launch();
  const int key_bits = bits * dk;
  uint32_t *kin = (uint32_t*)ka, *kout = (uint32_t*)kb;
  int *vin = (int*)va, *vout = (int*)vb;
  for (int shift = 0; shift < key_bits; shift += 8) {
    radix_hist_kernel<<<nchunks, SORT_THREADS, 0, st>>>(kin, N, shift, (uint32_t*)hist, nchunks); count_launch();
    radix_scan_kernel<<<1, SCAN_THREADS, 0, st>>>((uint32_t*)hist, 256LL * nchunks); count_launch();
    radix_scatter_kernel<<<nchunks, SORT_THREADS, 0, st>>>(kin, vin, N, shift,
                                                           (const uint32_t*)hist, nchunks, kout,
                                                           vout); count_launch();
    std::swap(kin, kout);
    std::swap(vin, vout);
  }
  if ((e = cudaMemcpyAsync(P.perm, vin, sizeof(int) * N, cudaMemcpyDeviceToDevice, st))) return e;
  pack_kernel<<<blocks_for(P.Npad, 256), 256, 0, st>>>(X, N, P.Npad, d_in, d, P.perm, P.xs); count_launch();

  P.T = mvp_targets_per_thread(d, N);
  P.nblk = (N + 32 * P.T - 1) / (32 * P.T);
  void *ctr, *flag, *order, *nexp;
  if ((e = c.ws.get(t + ".ctr", sizeof(float) * P.nblk * d, &ctr))) return e;
  if ((e = c.ws.get(t + ".order", sizeof(int) * P.nblk, &order))) return e;
  if ((e = c.ws.get(t + ".nexp", sizeof(int), &nexp))) return e;
  if ((e = c.ws.get("sort.flag", sizeof(int) * P.nblk, &flag))) return e;
  P.ctr = (float*)ctr;
  P.order = (int*)order;
  P.n_exp = (int*)nexp;
  blkinfo_kernel<<<blocks_for(P.nblk, 8), 256, 0, st>>>(P.xs, N, d, P.T, P.scale, P.nblk, P.ctr,
                                                       (int*)flag, allow_expanded); count_launch();
  order_kernel<<<1, SCAN_THREADS, 0, st>>>((const int*)flag, P.nblk, P.order, P.n_exp); count_launch();
  // super-blocks of SB targets (nsb <= nblk: the flag scratch fits)
  P.nsb = (N + SB - 1) / SB;
  if ((e = c.ws.get(t + ".sbctr", sizeof(float) * P.nsb * d, &ctr))) return e;
  if ((e = c.ws.get(t + ".sborder", sizeof(int) * P.nsb, &order))) return e;
  if ((e = c.ws.get(t + ".sbnexp", sizeof(int), &nexp))) return e;
  if ((e = c.ws.get(t + ".sbflag", sizeof(int) * P.nsb, &flag))) return e;
  P.sb_ctr = (float*)ctr;
  P.sb_order = (int*)order;
  P.sb_nexp = (int*)nexp;
  P.sb_flag = (int*)flag;
  blkinfo_kernel<<<blocks_for(P.nsb, 8), 256, 0, st>>>(P.xs, N, d, SB / 32, P.scale, P.nsb, P.sb_ctr,
                                                       P.sb_flag, allow_expanded_sb); count_launch();
  order_kernel<<<1, SCAN_THREADS, 0, st>>>(P.sb_flag, P.nsb, P.sb_order, P.sb_nexp); count_launch();
  const int64_t ntiles = P.Npad / TS;
  void* tbox;
  if ((e = c.ws.get(t + ".tbox", sizeof(float) * 2 * d * ntiles, &tbox))) return e;
  P.tbox = (float*)tbox;
  tilebox_kernel<<<blocks_for(ntiles, 8), 256, 0, st>>>(P.xs, ntiles, d, P.tbox); count_launch();
  if ((e = cudaGetLastError())) return e;
  // the block counts size the product grids: read them once (a short wait
  // for the preparation; never inside a graph capture)
  int counts[2] = {0, 0};
  if ((e = cudaMemcpyAsync(&counts[0], P.n_exp, sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaMemcpyAsync(&counts[1], P.sb_nexp, sizeof(int), cudaMemcpyDeviceToHost, st))) return e;
  if ((e = cudaStreamSynchronize(st))) return e;
  P.h_nexp = counts[0];
  P.h_sb_nexp = counts[1];
  return cudaSuccess;
}

}  // namespace krr
