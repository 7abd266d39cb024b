// Internal host-side interfaces of libkrr (not part of the public ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/libkrr.h"

namespace krr {

constexpr int PAD = 2048;  // prepared arrays are padded to a multiple of PAD points
// Most columns one multi-column product (and one block of a block solve) takes.
constexpr int MAX_COLS = 16;

inline int64_t round_up(int64_t n, int64_t m) { return (n + m - 1) / m * m; }

struct Buf {
  void* p = nullptr;
  size_t bytes = 0;
};

// Grow-only device workspace addressed by name.  A fixed workspace (slots laid
// out over memory the caller owns) never allocates: a request for a name it
// does not hold, or for more bytes than that slot has, fails with
// cudaErrorMemoryAllocation before any kernel could use the buffer.
struct Workspace {
  std::unordered_map<std::string, Buf> slots;
  bool fixed = false;
  cudaError_t get(const std::string& name, size_t bytes, void** out);
  void release_all();
  // frees the buffers whose names start with prefix
  void release_prefix(const std::string& prefix);
};

// Targets are handled in warp blocks of WB = 32*T consecutive sorted points
// (T targets per thread).  prep.cu computes, per warp block, the centre of its
// bounding box and whether it is compact enough for the expanded exponent
// form, and orders the blocks so that the expanded ones come first.
// Coordinates per point in the prepared layout: d itself up to 8, else d
// rounded up to 16, 32, 48 or 64 with zero coordinates (which leave every
// distance unchanged).  Above 8 every block takes the direct form.
inline int padded_dim(int d) { return d <= 8 ? d : (int)round_up(d, 16); }

struct PointsDev {
  int64_t N = 0, Npad = 0;
  int d = 0;            // prepared coordinates per point (padded_dim of d_in)
  int d_in = 0;         // the caller's dimension
  // kernel family (KRR_KERNEL_*) and its scale s, with x^ = s x:
  //   Gaussian:   s = sqrt(log2(e) / (2 sigma^2)), value 2^(-|x^_i - x^_j|^2)
  //   Matern 3/2: s = sqrt(3) / h,                 value (1 + a) 2^(-a log2(e)),
  //               a = |x^_i - x^_j|
  int kfam = 0;
  float scale = 0.f;
  double s2 = 0.0;      // s^2 in double
  float* xs = nullptr;  // tile-blocked SoA of the raw coordinates, Npad*d floats
  int* perm = nullptr;  // sorted position -> original index
  int T = 1;            // targets per thread of the product kernels
  int64_t nblk = 0;     // warp blocks: ceil(N / (32*T))
  float* ctr = nullptr; // nblk x d block centres (raw coordinates)
  int* order = nullptr; // nblk block indices, expanded-form blocks first
  int* n_exp = nullptr; // device scalar: number of expanded-form blocks
  float* tbox = nullptr;// Npad/TS source tiles x 2d: centre, then half-width per dim
  // the same per super-block of SB = 256 consecutive targets (the target
  // blocks of the multi-column products: one CTA each)
  int64_t nsb = 0;
  float* sb_ctr = nullptr;
  int* sb_order = nullptr;
  int* sb_nexp = nullptr;
  int* sb_flag = nullptr;  // nsb flags: 1 = expanded form
  // host copies of *n_exp and *sb_nexp (read once by prepare_points)
  int64_t h_nexp = 0, h_sb_nexp = 0;
};

// Targets per super-block.
constexpr int SB = 256;

// Targets per thread the product kernels use for N targets in d dimensions.
int mvp_targets_per_thread(int d, int64_t N);
// Squared radius (scaled units) up to which a warp block uses the expanded form.
constexpr float EXPANDED_R2 = 8.0f;

struct Ctx {
  int device = 0;
  int num_sms = 0;
  Workspace ws;
  int* d_err = nullptr;        // device error word (DevErr)
  int* h_status = nullptr;     // pinned host mirror for status reads
  std::string last_error;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  // solver work runs on this non-blocking stream (capturable), joined to the
  // caller's stream by ev_in / ev_out
  cudaStream_t work = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  // concurrent branches of a batched solve each get a sub-context with its
  // own workspace and error word (sub-contexts own no streams or events)
  std::vector<Ctx*> subs;
  // CTA slots the product kernels plan for (0: 2 per SM); a batched solve
  // lowers it so that concurrent small problems are not over-split
  int plan_slots = 0;
  // single-column float32 products may take the tensor-core exponent path
  // (the no-allocation entry point keeps to the CUDA-core kernel, whose
  // scratch its fixed array holds)
  bool allow_tcx = true;
  // multi-column tensor-core products on the tcgen05 / tensor-memory kernel
  // instead of the mma.sync kernel (krr_set_option)
  bool use_tcgen05 = false;
  // which tcgen05 multi-column kernel: 1 = exponent by mma.sync into
  // registers, P stored to tensor memory (mvp_umx_kernel); 2 = exponent by
  // tcgen05 into tensor memory, loaded, exponentiated and stored back
  // (mvp_umma_kernel)
  int tcgen05_kind = 1;
  // the default: float32 multi-column products on mvp_umx_kernel, reduced-
  // precision ones on the mma.sync kernel (the faster of each on GB300);
  // cleared when KRR_OPT_TCGEN05 picks one kernel for all
  bool tcgen05_auto = true;
  // single-column products above 8 dimensions on the tcgen05 kernel
  // (mvp_uhd_kernel; false: the mma.sync kernel mvp_tch_kernel)
  bool highd_tcgen05 = true;
  // direct-form super-blocks of multi-column products up to 8 dimensions:
  // kernel values on the CUDA cores, the weighted sum on the tensor cores
  // (mvp_dirtc_kernel); false: the all-CUDA-core kernel mvp_dirm_kernel
  bool direct_tensor = true;
  // kernel function of every product and solve (KRR_KERNEL_*, krr_set_option)
  int kernel_family = 0;
  // autotuning of the products' source splits (KRR_OPT_AUTOTUNE): the first
  // reserve or launch of a product shape outside a graph capture times the
  // real launch at several scales of the modelled split count and keeps the
  // fastest; split_scale is the scale in force for the product being planned
  bool autotune = false;
  bool tuning = false;
  // target-row shard emulation (KRR_OPT_SHARD_COUNT / _INDEX): the products
  // of krr_kernel_mvp compute and write only sorted target rows
  // [row_lo, row_hi) (whole super-blocks); elsewhere the range is everything
  int shard_count = 1, shard_index = 0;
  int64_t row_lo = 0, row_hi = INT64_MAX;
  int prod_depth = 0;
  double split_scale = 1.0;
  std::unordered_map<std::string, double> tune_cache;
  // the kernel variant the autotuner picked per product shape (TuneVariant
  // bits; absent: the handle's own settings)
  std::unordered_map<std::string, int> tune_variant;
  // profiling of the fast product kernel (krr_profile_enable / _read)
  bool profiling = false;
  std::vector<cudaEvent_t> prof_ev;  // pairs: start, stop
  size_t prof_used = 0;              // events in use (even)
  double prof_pairs = 0.0;
  int prof_tensor_exp = 0;           // timed launches on the tensor-core exponent path
};

// Product shape key of the autotuner: kind ("mvp" or "acc"), sizes, columns,
// precision, kernel family and the planning context.
std::string tune_key(const Ctx& c, const char* kind, const PointsDev& Tp, const PointsDev& Sp, int m,
                     int prec);
// The tuned split scale of a shape (1 when untuned).
inline double tuned_scale(const Ctx& c, const std::string& key) {
  const auto it = c.tune_cache.find(key);
  return it == c.tune_cache.end() ? 1.0 : it->second;
}
// Whether a product entry point may run the tuner now: enabled, not already
// tuning, not nested in another product entry point, and the stream is not
// being captured into a graph.
bool can_tune(const Ctx& c, cudaStream_t st);
// Sets c.split_scale for one product entry point and counts the nesting.
struct TuneScope {
  Ctx& c;
  double old;
  TuneScope(Ctx& cc, double s) : c(cc), old(cc.split_scale) {
    c.split_scale = s;
    ++c.prod_depth;
  }
  ~TuneScope() {
    c.split_scale = old;
    --c.prod_depth;
  }
};
// Kernel variants of a product shape (KRR_OPT_AUTOTUNE picks one per shape):
// which kernel, hence which CTA shape and targets per thread, carries each
// kind of target block.
enum TuneVariant : int {
  TV_TCGEN05 = 1,        // compact blocks of multi-column products: tcgen05 kernel (128-target CTAs)
                         // instead of mma.sync (256-target CTAs)
  TV_DIRECT_TENSOR = 2,  // direct-form blocks of multi-column products: tensor-core P Q (512-thread
                         // CTAs) instead of one target per thread on the CUDA cores
  TV_TENSOR_EXP = 4,     // single-column float32 products may take the tensor-core exponent path
                         // (128-thread CTAs per super-block) instead of the packed CUDA-core kernel
};
// Whether the compact blocks of an m-column product of precision prec over
// the targets Tp take a tcgen05 kernel (c.tcgen05_kind) rather than the
// mma.sync kernel.  The automatic choice (measured on GB300, 16 columns,
// compact blocks) takes mvp_umx_kernel for float32 products of more than
// TC5_AUTO_MIN_COLS columns, where the mma.sync kernel's three split P Q
// MMAs per column tile bound it, once there are enough targets: from 65536
// at d >= 5 (two exponent contraction steps; 1.25-1.46x at 65536 and
// 262144, 0.84-0.91x at 16384) and from 131072 at d <= 4 (1.08-1.14x at
// 262144, 0.90-1.02x at 65536, 0.57-1.0x at 16384).  The solvers refine it
// per shape by timing both kernels (mvp_multi_reserve).
constexpr int TC5_AUTO_MIN_COLS = 8;
constexpr int64_t TC5_AUTO_MIN_N_HIGH_D = 65536, TC5_AUTO_MIN_N_LOW_D = 131072;
inline bool tc5_auto_choice(int prec, int m, const PointsDev& Tp) {
  return prec == KRR_FP32 && m > TC5_AUTO_MIN_COLS &&
         Tp.N >= (Tp.d >= 5 ? TC5_AUTO_MIN_N_HIGH_D : TC5_AUTO_MIN_N_LOW_D);
}
inline bool tc5_on(const Ctx& c, int prec, int m, const PointsDev& Tp) {
  return c.tcgen05_auto ? tc5_auto_choice(prec, m, Tp) : c.use_tcgen05;
}
inline int current_variant(const Ctx& c, int prec, int m, const PointsDev& Tp) {
  return (tc5_on(c, prec, m, Tp) ? TV_TCGEN05 : 0) | (c.direct_tensor ? TV_DIRECT_TENSOR : 0) |
         (c.allow_tcx ? TV_TENSOR_EXP : 0);
}
// Applies the tuned variant of a shape for one product entry point (and puts
// the handle's settings back after it).
struct VariantScope {
  Ctx& c;
  bool tc5, tc5_auto, dt, tcx;
  int tc5_kind;
  VariantScope(Ctx& cc, const std::string& key)
      : c(cc), tc5(cc.use_tcgen05), tc5_auto(cc.tcgen05_auto), dt(cc.direct_tensor), tcx(cc.allow_tcx),
        tc5_kind(cc.tcgen05_kind) {
    const auto it = c.tune_variant.find(key);
    if (it == c.tune_variant.end()) return;
    c.tcgen05_auto = false;
    c.use_tcgen05 = (it->second & TV_TCGEN05) != 0;
    if (tc5_auto) c.tcgen05_kind = 1;  // the automatic choice's tcgen05 kernel
    c.direct_tensor = (it->second & TV_DIRECT_TENSOR) != 0;
    c.allow_tcx = tcx && (it->second & TV_TENSOR_EXP) != 0;  // never where the handle forbids it
  }
  ~VariantScope() {
    c.use_tcgen05 = tc5;
    c.tcgen05_auto = tc5_auto;
    c.tcgen05_kind = tc5_kind;
    c.direct_tensor = dt;
    c.allow_tcx = tcx;
  }
};
// Split scales the tuner tries, the modelled one first.
constexpr double TUNE_SCALES[] = {1.0, 0.5, 2.0, 0.25, 4.0};
// Largest partial-sum buffer a tuning candidate may ask for.
constexpr double TUNE_MAX_BYTES = 1073741824.0;

// Sub-context k of c (created on first use; freed with the handle).
cudaError_t sub_context(Ctx& c, size_t k, Ctx** out);
void release_context(Ctx& c);

// ---- prep.cu
// Sort X (N x d row-major, device) along a Morton curve and pack the scaled,
// tile-blocked structure-of-arrays copy.  `tag` names the workspace slots.
cudaError_t prepare_points(Ctx& c, const float* X, int64_t N, int d, float sigma,
                           const char* tag, PointsDev& P, cudaStream_t st);
// out[i] = in[perm[i]] (float columns, m of them, column stride N / Npad);
// padded tail of each column set to zero.
cudaError_t gather_sorted(const float* in, int64_t N, int m, const int* perm, int64_t Npad,
                          float* out, cudaStream_t st);
// out[perm[i]] = in[i]
cudaError_t scatter_orig(const float* in, int64_t Npad, int64_t N, int m, const int* perm,
                         float* out, cudaStream_t st);

// ---- mvp_acc.cu
// Accurate product for true residuals: out = cu * u + cy * (K_hat q + shift q)
// in FP64 (sorted order), q given as float-float (qh + ql), with the fused
// squared norm *dot += |out|^2 when dot != null.  Per-term relative error
// about 3e-12 on near tiles.
//
// Several columns at once (cols.n <= MAX_COLS, one grid z-slice each): qh,
// ql, u and out hold cols.n columns Npad apart; column c's dot and active
// word sit cols.state_stride bytes after column c-1's, and a column whose
// active word is 0 is skipped.
struct AccCols {
  int n = 1;
  const int* active = nullptr;
  size_t state_stride = 0;
};
cudaError_t mvp_acc_launch(Ctx& c, const PointsDev& P, const float* qh, const float* ql,
                           float shift, double cu, const float* u, double cy, double* out,
                           double* dot, cudaStream_t st, const AccCols& cols = AccCols{});

// ---- mvp.cu
struct MvpOut {
  // y = alpha * (K_hat q + shift q) + beta * u, sorted order
  float alpha = 1.f, beta = 0.f;
  const float* u = nullptr;
  float* out_f = nullptr;       // sorted-order float output (may be null)
  double* out_d = nullptr;      // sorted-order double output (may be null)
  const int* perm = nullptr;    // if set with out_orig: scatter to original order
  float* out_orig = nullptr;
  const float* dotw = nullptr;  // if set: *dot = sum_i y_i * dotw_i (assigned)
  double* dot = nullptr;
  // CG step length, applied once the dot is complete: *ratio_out =
  // *ratio_num / *dot when the dot is positive and finite, else 0 with
  // *brk_flag set to 1.
  const double* ratio_num = nullptr;
  double* ratio_out = nullptr;
  int* brk_flag = nullptr;
  // predication: when non-null and *active == 0 the launch does nothing
  const int* active = nullptr;
  // several columns (mvp_multi_launch): column c's scalars (dot, ratio_num,
  // ratio_out, brk_flag, col_active) sit state_stride bytes after column
  // c-1's; a column whose *col_active is 0 writes nothing
  const int* col_active = nullptr;
  size_t state_stride = 0;
};

// Allocate the workspace and set the kernel attributes a later mvp_launch /
// mvp_acc_launch on these point sets needs, so that launches captured into a
// CUDA graph allocate nothing.
cudaError_t mvp_reserve(Ctx& c, const PointsDev& T, const PointsDev& S, cudaStream_t st);
cudaError_t mvp_acc_reserve(Ctx& c, const PointsDev& P, cudaStream_t st, int ncols = 1);

// Several right-hand sides at once: Y[:, c] = (K_hat + shift I) Q[:, c] for
// c < m (m <= MAX_COLS), Q sorted with column stride S.Npad, qdiag, u, dotw
// with column stride T.Npad.  Output per column c: out_f + c*T.Npad (sorted)
// and/or out_orig + c*T.N (original order); the dot / step-length epilogue
// applies to every column, with the column scalars o.state_stride bytes apart.
// Expanded-form warp blocks run on the tensor cores (prec KRR_FP32 with
// hi/lo-split operands, float32-grade; KRR_FP16 / KRR_BF16 with single
// half-precision operands), direct-form blocks on a multi-column float32
// CUDA-core kernel (one exponential per pair shared by all columns).
cudaError_t mvp_multi_launch(Ctx& c, const PointsDev& T, const PointsDev& S, const float* Q, int m,
                             const float* qdiag, float shift, krr_precision prec, const MvpOut& o,
                             cudaStream_t st);
// ---- mvp_tc.cu: tensor-core partial sums of the expanded-form warp blocks
// dry = true only sets the kernel attributes (before any graph capture).
cudaError_t mvp_tc_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* Q, int m,
                            bool split, bool bf, int splits, int tiles_per_split, double* part,
                            float* fac, const int* active, cudaStream_t st, bool dry = false);
// ---- mvp_tc.cu: single-column float32-grade partial sums of the
// expanded-form super-blocks (exponent on the tensor cores, EX2 + FMA per
// pair on the CUDA cores); part: [splits][T.Npad].
cudaError_t mvp_tcx_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* q,
                             int splits, int tiles_per_split, double* part, float* fac,
                             const int* active, cudaStream_t st, bool dry = false);
// ---- mvp_tc.cu: the same partial sums on the 5th-generation tensor cores
// (tcgen05.mma, accumulators in tensor memory), two CTAs per super-block.
cudaError_t mvp_umma_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* Q, int m,
                              bool split, bool bf, int splits, int tiles_per_split, double* part,
                              float* fac, const int* active, cudaStream_t st, bool dry = false);
// ---- mvp_dirtc.cu: partial sums of the direct-form super-blocks (slots
// [slot0, nsb) of T.sb_order, checked against the device count tn_exp) of a
// multi-column product, d <= 8: kernel values on the CUDA cores, the weighted
// sum P Q on the tensor cores (split f16 for KRR_FP32, single f16 / bf16
// otherwise; the Matern kernel always split); part: [splits][m][T.Npad].
cudaError_t mvp_dirtc_partials(Ctx& c, const PointsDev& T, const PointsDev& S, const float* Q, int m,
                               krr_precision prec, int splits, int tiles_per_split, int64_t slot0,
                               const int* tn_exp, double* part, float* fac, const int* active,
                               cudaStream_t st, bool dry = false);
// Workspace and attributes of mvp_multi_launch with m columns and prec.
cudaError_t mvp_multi_reserve(Ctx& c, const PointsDev& T, const PointsDev& S, int m,
                              krr_precision prec, cudaStream_t st);

// Single right-hand side product over prepared targets T and sources S
// (the same object for the square product).  q: sorted source weights
// (length S.Npad, zero padded); qdiag: sorted target weights for the shift
// term (may be null when shift == 0).
cudaError_t mvp_launch(Ctx& c, const PointsDev& T, const PointsDev& S, const float* q,
                       const float* qdiag, float shift, krr_precision prec, const MvpOut& o,
                       cudaStream_t st);

}  // namespace krr
