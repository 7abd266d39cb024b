// C-ABI entry points of libkrr: handle, workspace, argument checks, host
// array staging and the kernel-product calls.  The solvers live in krylov.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "api_util.h"
#include "common.cuh"
#include "internal.h"

namespace krr {

std::atomic<long long> g_launches{0};

cudaError_t Workspace::get(const std::string& name, size_t bytes, void** out) {
  bytes = std::max<size_t>(bytes, 256);
  auto it = slots.find(name);
  if (it != slots.end() && it->second.bytes >= bytes) {
    *out = it->second.p;
    return cudaSuccess;
  }
  if (fixed) return cudaErrorMemoryAllocation;
  if (it != slots.end()) {
    // cudaFree waits for the device, so work queued on the old buffer is done
    cudaFree(it->second.p);
    it->second = Buf{};
  }
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return e;
  }
  slots[name] = Buf{p, bytes};
  *out = p;
  return cudaSuccess;
}

void Workspace::release_all() {
  for (auto& kv : slots) cudaFree(kv.second.p);
  slots.clear();
}

void Workspace::release_prefix(const std::string& prefix) {
  for (auto it = slots.begin(); it != slots.end();) {
    if (it->first.compare(0, prefix.size(), prefix) == 0) {
      cudaFree(it->second.p);
      it = slots.erase(it);
    } else {
      ++it;
    }
  }
}

std::string tune_key(const Ctx& c, const char* kind, const PointsDev& Tp, const PointsDev& Sp, int m,
                     int prec) {
  char buf[256];
  snprintf(buf, sizeof(buf), "%s|%lld|%lld|%d|%d|%d|%d|%d|%d|%lld|%lld", kind, (long long)Tp.N,
           (long long)Sp.N, Tp.d, Tp.kfam, m, prec, c.plan_slots, c.tcgen05_auto ? 3 : c.use_tcgen05 ? c.tcgen05_kind : 0,
           (long long)Tp.h_nexp, (long long)Tp.h_sb_nexp);
  return buf;
}

// The product over prepared points (both krr_kernel_mvp and
// krr_kernel_mvp_points): gather Q into sorted order, then one single-column
// launch or multi-column passes of at most MAX_COLS, each writing its
// columns of Y in original order.  Row shards as set on the handle.  No host
// synchronisation.
cudaError_t product_prepared(Ctx& c, const PointsDev& P, const float* dQ, int m, float gamma,
                             krr_precision prec, float* dY, cudaStream_t st) {
  struct RowRange {
    Ctx& c;
    ~RowRange() {
      c.row_lo = 0;
      c.row_hi = INT64_MAX;
    }
  } row_range{c};
  if (c.shard_count > 1) {
    c.row_lo = (int64_t)SB * (P.nsb * c.shard_index / c.shard_count);
    c.row_hi = (int64_t)SB * (P.nsb * (c.shard_index + 1) / c.shard_count);
  }
  const int64_t N = P.N;
  void* qs;
  cudaError_t e;
  if ((e = c.ws.get("mvp.qs", sizeof(float) * P.Npad * m, &qs))) return e;
  if ((e = gather_sorted(dQ, N, m, P.perm, P.Npad, (float*)qs, st))) return e;
  if (m == 1) {
    MvpOut o;
    o.perm = P.perm;
    o.out_orig = dY;
    return mvp_launch(c, P, P, (const float*)qs, (const float*)qs, gamma, prec, o, st);
  }
  // columns in as few passes of at most MAX_COLS as possible: each kernel
  // value serves every column of a pass
  const int passes = (m + MAX_COLS - 1) / MAX_COLS;
  const int width = (m + passes - 1) / passes;
  for (int col0 = 0; col0 < m; col0 += width) {
    const int mc = std::min(width, m - col0);
    const float* qc = (const float*)qs + (size_t)col0 * P.Npad;
    MvpOut o;
    o.perm = P.perm;
    o.out_orig = dY + (size_t)col0 * N;
    if ((e = mvp_multi_launch(c, P, P, qc, mc, qc, gamma, prec, o, st))) return e;
  }
  return cudaSuccess;
}

bool can_tune(const Ctx& c, cudaStream_t st) {
  if (!c.autotune || c.tuning || c.prod_depth > 0) return false;
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) return false;
  return cs == cudaStreamCaptureStatusNone;
}

cudaError_t sub_context(Ctx& c, size_t k, Ctx** out) {
  while (c.subs.size() <= k) {
    Ctx* s = new (std::nothrow) Ctx();
    if (!s) return cudaErrorMemoryAllocation;
    s->device = c.device;
    s->num_sms = c.num_sms;
    cudaError_t e = cudaMalloc(&s->d_err, sizeof(int));
    if (!e) e = cudaMemset(s->d_err, 0, sizeof(int));
    if (e) {
      delete s;
      return e;
    }
    c.subs.push_back(s);
  }
  *out = c.subs[k];
  return cudaSuccess;
}

void release_context(Ctx& c) {
  for (Ctx* s : c.subs) {
    release_context(*s);
    s->ws.release_all();
    cudaFree(s->d_err);
    delete s;
  }
  c.subs.clear();
}

krr_status set_error(Ctx& c, krr_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  c.last_error = buf;
  return s;
}

krr_status cuda_error(Ctx& c, cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return set_error(c, KRR_ERR_OOM, "%s: out of device memory", what);
  if (e == cudaErrorNotSupported)
    return set_error(c, KRR_ERR_UNIMPLEMENTED, "%s: configuration not built", what);
  return set_error(c, KRR_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool is_device_ptr(const Ctx& c, const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) &&
         a.device == c.device;
}

// Read and clear the device error word (waits for `st`).
krr_status read_device_error(Ctx& c, cudaStream_t st, const char* what) {
  cudaError_t e = cudaMemcpyAsync(c.h_status, c.d_err, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (!e) e = cudaStreamSynchronize(st);
  if (e) return cuda_error(c, e, what);
  const int v = *c.h_status;
  if (v == DEV_OK) return KRR_OK;
  cudaMemsetAsync(c.d_err, 0, sizeof(int), st);
  cudaStreamSynchronize(st);
  if (v == DEV_TIMEOUT) return set_error(c, KRR_ERR_TIMEOUT, "%s: a bounded device wait ran out", what);
  if (v == DEV_NONFINITE) return set_error(c, KRR_ERR_NONFINITE, "%s: non-finite input", what);
  if (v == DEV_BREAKDOWN) return set_error(c, KRR_ERR_BREAKDOWN, "%s: Krylov breakdown", what);
  return set_error(c, KRR_ERR_CUDA, "%s: device error %d", what, v);
}

krr_status check_points(Ctx& c, const char* fn, const float* X, int64_t N, int d, float sigma) {
  if (N < 0 || N > (int64_t(1) << 30))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: N = %lld out of range [0, 2^30]", fn, (long long)N);
  if (d < 1 || d > 64) return set_error(c, KRR_ERR_INVALID_ARG, "%s: d = %d out of range [1, 64]", fn, d);
  if (!(sigma > 0.f) || !std::isfinite(sigma))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: sigma must be finite and > 0", fn);
  if (N > 0 && X == nullptr) return set_error(c, KRR_ERR_INVALID_ARG, "%s: X is NULL", fn);
  return KRR_OK;
}

// Device view of a caller array: the array itself when it is on the handle's
// device, else a staged copy in the workspace (copied in when `in`).
krr_status device_view(Ctx& c, const char* slot, const float* p, size_t count, bool in,
                       cudaStream_t st, float** out, bool* staged) {
  if (p == nullptr || count == 0 || is_device_ptr(c, p)) {
    *out = const_cast<float*>(p);
    *staged = false;
    return KRR_OK;
  }
  void* d;
  cudaError_t e = c.ws.get(slot, count * sizeof(float), &d);
  if (e) return cuda_error(c, e, slot);
  if (in && (e = cudaMemcpyAsync(d, p, count * sizeof(float), cudaMemcpyHostToDevice, st)))
    return cuda_error(c, e, slot);
  *out = (float*)d;
  *staged = true;
  return KRR_OK;
}

krr_status device_view_d(Ctx& c, const char* slot, const double* p, size_t count, bool in,
                         cudaStream_t st, double** out, bool* staged) {
  if (p == nullptr || count == 0 || is_device_ptr(c, p)) {
    *out = const_cast<double*>(p);
    *staged = false;
    return KRR_OK;
  }
  void* d;
  cudaError_t e = c.ws.get(slot, count * sizeof(double), &d);
  if (e) return cuda_error(c, e, slot);
  if (in && (e = cudaMemcpyAsync(d, p, count * sizeof(double), cudaMemcpyHostToDevice, st)))
    return cuda_error(c, e, slot);
  *out = (double*)d;
  *staged = true;
  return KRR_OK;
}

}  // namespace krr

using namespace krr;

extern "C" {

int krr_version(void) { return 300; }

const char* krr_status_string(krr_status s) {
  switch (s) {
    case KRR_OK: return "KRR_OK";
    case KRR_ERR_INVALID_ARG: return "KRR_ERR_INVALID_ARG";
    case KRR_ERR_CUDA: return "KRR_ERR_CUDA";
    case KRR_ERR_OOM: return "KRR_ERR_OOM";
    case KRR_ERR_NONFINITE: return "KRR_ERR_NONFINITE";
    case KRR_NOT_CONVERGED: return "KRR_NOT_CONVERGED";
    case KRR_ERR_BREAKDOWN: return "KRR_ERR_BREAKDOWN";
    case KRR_ERR_TIMEOUT: return "KRR_ERR_TIMEOUT";
    case KRR_ERR_UNIMPLEMENTED: return "KRR_ERR_UNIMPLEMENTED";
    case KRR_ERR_SIZE_LIMIT: return "KRR_ERR_SIZE_LIMIT";
  }
  return "KRR_UNKNOWN";
}

void krr_fgmres_default_opts(krr_fgmres_opts* o) {
  if (!o) return;
  o->restart = 30;
  o->max_cycles = 50;
  o->tol = 1e-6;
  o->delta = -1.0;
  o->inner_tol = -1.0;
  o->inner_maxit = 100;
  o->inner_prec = KRR_FP32;
  o->use_graph = 1;
  o->x0_given = 0;
}

krr_status krr_create(krr_handle* out) {
  if (!out) return KRR_ERR_INVALID_ARG;
  *out = nullptr;
  krr_handle h = new (std::nothrow) krr_handle_s();
  if (!h) return KRR_ERR_OOM;
  Ctx& c = h->ctx;
  cudaError_t e = cudaGetDevice(&c.device);
  if (!e) e = cudaDeviceGetAttribute(&c.num_sms, cudaDevAttrMultiProcessorCount, c.device);
  if (!e) e = cudaMalloc(&c.d_err, sizeof(int));
  if (!e) e = cudaMemset(c.d_err, 0, sizeof(int));
  if (!e) e = cudaMallocHost(&c.h_status, 64 * sizeof(int));
  if (!e) e = cudaEventCreate(&c.ev0);
  if (!e) e = cudaEventCreate(&c.ev1);
  if (!e) e = cudaStreamCreateWithFlags(&c.work, cudaStreamNonBlocking);
  if (!e) e = cudaEventCreateWithFlags(&c.ev_in, cudaEventDisableTiming);
  if (!e) e = cudaEventCreateWithFlags(&c.ev_out, cudaEventDisableTiming);
  if (e) {
    cudaGetLastError();
    if (c.d_err) cudaFree(c.d_err);
    if (c.h_status) cudaFreeHost(c.h_status);
    for (cudaEvent_t ev : {c.ev0, c.ev1, c.ev_in, c.ev_out})
      if (ev) cudaEventDestroy(ev);
    if (c.work) cudaStreamDestroy(c.work);
    cudaGetLastError();
    delete h;
    return e == cudaErrorMemoryAllocation ? KRR_ERR_OOM : KRR_ERR_CUDA;
  }
  *out = h;
  return KRR_OK;
}

krr_status krr_destroy(krr_handle h) {
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  cudaDeviceSynchronize();
  release_context(c);
  c.ws.release_all();
  cudaFree(c.d_err);
  cudaFreeHost(c.h_status);
  cudaEventDestroy(c.ev0);
  cudaEventDestroy(c.ev1);
  cudaEventDestroy(c.ev_in);
  cudaEventDestroy(c.ev_out);
  for (auto ev : c.prof_ev) cudaEventDestroy(ev);
  cudaStreamDestroy(c.work);
  delete h;
  return KRR_OK;
}

const char* krr_last_error(krr_handle h) { return h ? h->ctx.last_error.c_str() : "NULL handle"; }

krr_status krr_set_option(krr_handle h, int option, int value) {
  if (!h) return KRR_ERR_INVALID_ARG;
  switch (option) {
    case KRR_OPT_TCGEN05:
      if (value < 0 || value > 3)
        return set_error(h->ctx, KRR_ERR_INVALID_ARG, "krr_set_option: tcgen05 kernel %d out of [0, 3]", value);
      h->ctx.tcgen05_auto = value == 3;
      h->ctx.use_tcgen05 = value == 1 || value == 2;
      h->ctx.tcgen05_kind = value == 2 ? 2 : 1;
      return KRR_OK;
    case KRR_OPT_AUTOTUNE:
      h->ctx.autotune = value != 0;
      return KRR_OK;
    case KRR_OPT_HIGHD_TCGEN05:
      h->ctx.highd_tcgen05 = value != 0;
      return KRR_OK;
    case KRR_OPT_DIRECT_TENSOR:
      h->ctx.direct_tensor = value != 0;
      return KRR_OK;
    case KRR_OPT_SHARD_COUNT:
      if (value < 1 || value > 4096)
        return set_error(h->ctx, KRR_ERR_INVALID_ARG, "krr_set_option: shard count %d out of [1, 4096]", value);
      h->ctx.shard_count = value;
      return KRR_OK;
    case KRR_OPT_SHARD_INDEX:
      if (value < 0)
        return set_error(h->ctx, KRR_ERR_INVALID_ARG, "krr_set_option: shard index %d < 0", value);
      h->ctx.shard_index = value;
      return KRR_OK;
    case KRR_OPT_KERNEL:
      if (value != KRR_KERNEL_GAUSSIAN && value != KRR_KERNEL_MATERN32)
        return set_error(h->ctx, KRR_ERR_INVALID_ARG, "krr_set_option: unknown kernel family %d", value);
      h->ctx.kernel_family = value;
      return KRR_OK;
    default:
      return set_error(h->ctx, KRR_ERR_INVALID_ARG, "krr_set_option: unknown option %d", option);
  }
}

// Tuning cache file: "krr-tune 1 sms <n>", then per shape
// "<key>\t<split scale>\t<variant or -1>" (keys hold no tabs or newlines).
krr_status krr_tune_save(krr_handle h, const char* path) {
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  if (!path) return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_save: path is NULL");
  FILE* f = std::fopen(path, "w");
  if (!f) return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_save: cannot write %s", path);
  bool ok = std::fprintf(f, "krr-tune 1 sms %d\n", c.num_sms) > 0;
  for (const auto& kv : c.tune_cache) {
    const auto it = c.tune_variant.find(kv.first);
    ok = ok && std::fprintf(f, "%s\t%.17g\t%d\n", kv.first.c_str(), kv.second,
                            it == c.tune_variant.end() ? -1 : it->second) > 0;
  }
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_save: write to %s failed", path);
  return KRR_OK;
}

krr_status krr_tune_load(krr_handle h, const char* path) {
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  if (!path) return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_load: path is NULL");
  FILE* f = std::fopen(path, "r");
  if (!f) return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_load: cannot read %s", path);
  char line[1024];
  int sms = -1;
  if (!std::fgets(line, sizeof line, f) || std::sscanf(line, "krr-tune 1 sms %d", &sms) != 1) {
    std::fclose(f);
    return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_load: %s is not a tuning cache file", path);
  }
  if (sms != c.num_sms) {
    std::fclose(f);
    return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_load: %s was tuned on %d SMs, this device has %d",
                     path, sms, c.num_sms);
  }
  std::vector<std::pair<std::string, std::pair<double, int>>> entries;
  bool ok = true;
  while (std::fgets(line, sizeof line, f)) {
    const size_t n = std::strlen(line);
    if (n == 0 || line[n - 1] != '\n') {
      ok = false;  // over-long or truncated line
      break;
    }
    line[n - 1] = 0;
    char* t1 = std::strchr(line, '\t');
    char* t2 = t1 ? std::strchr(t1 + 1, '\t') : nullptr;
    if (!t1 || !t2 || t1 == line) {
      ok = false;
      break;
    }
    *t1 = *t2 = 0;
    char* end1 = nullptr;
    char* end2 = nullptr;
    const double scale = std::strtod(t1 + 1, &end1);
    const long variant = std::strtol(t2 + 1, &end2, 10);
    if (*end1 || *end2 || !(scale > 0.0 && scale <= 256.0) || variant < -1 || variant > 7) {
      ok = false;
      break;
    }
    entries.push_back({std::string(line), {scale, (int)variant}});
  }
  std::fclose(f);
  if (!ok) return set_error(c, KRR_ERR_INVALID_ARG, "krr_tune_load: malformed line in %s", path);
  for (const auto& e : entries) {
    c.tune_cache[e.first] = e.second.first;
    if (e.second.second >= 0) c.tune_variant[e.first] = e.second.second;
    else c.tune_variant.erase(e.first);
  }
  return KRR_OK;
}

krr_status krr_profile_enable(krr_handle h, int enable) {
  if (!h) return KRR_ERR_INVALID_ARG;
  h->ctx.profiling = enable != 0;
  h->ctx.prof_used = 0;
  h->ctx.prof_pairs = 0.0;
  h->ctx.prof_tensor_exp = 0;
  return KRR_OK;
}

krr_status krr_profile_read(krr_handle h, krr_profile* out) {
  if (!h || !out) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  out->launches = g_launches.load();
  out->product_launches = (int)(c.prof_used / 2);
  out->product_ms = 0.0;
  out->product_pairs = c.prof_pairs;
  out->tensor_exponent_launches = c.prof_tensor_exp;
  for (size_t k = 0; k + 1 < c.prof_used; k += 2) {
    cudaError_t e = cudaEventSynchronize(c.prof_ev[k + 1]);
    if (e) return cuda_error(c, e, "krr_profile_read");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.prof_ev[k], c.prof_ev[k + 1]);
    out->product_ms += ms;
  }
  c.prof_used = 0;
  c.prof_pairs = 0.0;
  c.prof_tensor_exp = 0;
  return KRR_OK;
}

krr_status krr_kernel_mvp(krr_handle h, const float* X, int64_t N, int d, float sigma, float gamma,
                          const float* Q, int m, float* Y, krr_precision prec, void* stream) {
  NvtxRange nvtx_range("krr_kernel_mvp");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_kernel_mvp";
  krr_status s = check_points(c, fn, X, N, d, sigma);
  if (s) return s;
  if (!(gamma >= 0.f) || !std::isfinite(gamma))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: gamma must be finite and >= 0", fn);
  if (m < 1 || m > 64) return set_error(c, KRR_ERR_INVALID_ARG, "%s: m = %d out of range [1, 64]", fn, m);
  if (prec != KRR_FP32 && prec != KRR_BF16 && prec != KRR_FP16)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: unknown precision %d", fn, (int)prec);
  if (N == 0) return KRR_OK;
  if (!Q || !Y) return set_error(c, KRR_ERR_INVALID_ARG, "%s: Q or Y is NULL", fn);
  if (Y == Q || (const void*)Y == (const void*)X)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: Y aliases an input", fn);
  const bool sharded = c.shard_count > 1;
  if (c.shard_index >= c.shard_count)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: shard index %d >= shard count %d", fn, c.shard_index,
                     c.shard_count);
  cudaStream_t st = (cudaStream_t)stream;
  float *dX, *dQ, *dY;
  bool sX, sQ, sY;
  if ((s = device_view(c, "stage.X", X, (size_t)N * d, true, st, &dX, &sX))) return s;
  if ((s = device_view(c, "stage.Q", Q, (size_t)N * m, true, st, &dQ, &sQ))) return s;
  // a shard leaves the other rows of Y as they were: a host Y goes up first
  if ((s = device_view(c, "stage.Y", Y, (size_t)N * m, sharded, st, &dY, &sY))) return s;
  PointsDev P;
  cudaError_t e = prepare_points(c, dX, N, d, sigma, "pts", P, st);
  if (e) return cuda_error(c, e, fn);
  if ((e = product_prepared(c, P, dQ, m, gamma, prec, dY, st))) return cuda_error(c, e, fn);
  if (sY) {
    if ((e = cudaMemcpyAsync(Y, dY, sizeof(float) * N * m, cudaMemcpyDeviceToHost, st)))
      return cuda_error(c, e, fn);
  }
  if (sX || sQ || sY) return read_device_error(c, st, fn);
  return KRR_OK;
}

// The handle's product options, copied into a point set's own context.
static void copy_product_options(Ctx& dst, const Ctx& src) {
  dst.allow_tcx = src.allow_tcx;
  dst.use_tcgen05 = src.use_tcgen05;
  dst.tcgen05_kind = src.tcgen05_kind;
  dst.tcgen05_auto = src.tcgen05_auto;
  dst.highd_tcgen05 = src.highd_tcgen05;
  dst.direct_tensor = src.direct_tensor;
  dst.kernel_family = src.kernel_family;
  dst.autotune = src.autotune;
  dst.shard_count = src.shard_count;
  dst.shard_index = src.shard_index;
}

static void free_points(krr_points_s* pts) {
  release_context(pts->ctx);
  pts->ctx.ws.release_all();
  cudaFree(pts->ctx.d_err);
  delete pts;
}

krr_status krr_points_create(krr_handle h, const float* X, int64_t N, int d, float sigma, krr_points* out,
                             void* stream) {
  NvtxRange nvtx_range("krr_points_create");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_points_create";
  if (!out) return set_error(c, KRR_ERR_INVALID_ARG, "%s: out is NULL", fn);
  *out = nullptr;
  krr_status s = check_points(c, fn, X, N, d, sigma);
  if (s) return s;
  if (N == 0) return set_error(c, KRR_ERR_INVALID_ARG, "%s: empty point set", fn);
  cudaStream_t st = (cudaStream_t)stream;
  float* dX;
  bool sX;
  if ((s = device_view(c, "stage.X", X, (size_t)N * d, true, st, &dX, &sX))) return s;
  krr_points_s* pts = new (std::nothrow) krr_points_s;
  if (!pts) return set_error(c, KRR_ERR_OOM, "%s: out of host memory", fn);
  pts->h = h;
  Ctx& pc = pts->ctx;
  pc.device = c.device;
  pc.num_sms = c.num_sms;
  copy_product_options(pc, c);
  cudaError_t e = cudaMalloc(&pc.d_err, sizeof(int));
  if (!e) e = cudaMemsetAsync(pc.d_err, 0, sizeof(int), st);
  if (!e) e = prepare_points(pc, dX, N, d, sigma, "points", pts->P, st);  // waits once
  if (e) {
    free_points(pts);
    return cuda_error(c, e, fn);
  }
  pc.ws.release_prefix("sort.");  // the sort's scratch is not needed again
  pc.h_status = c.h_status;       // the handle's pinned status word, for this one read
  s = read_device_error(pc, st, fn);
  pc.h_status = nullptr;
  if (s) {
    c.last_error = pc.last_error;
    free_points(pts);
    return s;
  }
  *out = pts;
  return KRR_OK;
}

krr_status krr_kernel_mvp_points(krr_handle h, krr_points P, const float* Q, int m, float gamma, float* Y,
                                 krr_precision prec, void* stream) {
  NvtxRange nvtx_range("krr_kernel_mvp_points");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_kernel_mvp_points";
  if (!P || P->h != h) return set_error(c, KRR_ERR_INVALID_ARG, "%s: point set of another handle", fn);
  if (!(gamma >= 0.f) || !std::isfinite(gamma))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: gamma must be finite and >= 0", fn);
  if (m < 1 || m > 64) return set_error(c, KRR_ERR_INVALID_ARG, "%s: m = %d out of range [1, 64]", fn, m);
  if (prec != KRR_FP32 && prec != KRR_BF16 && prec != KRR_FP16)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: unknown precision %d", fn, (int)prec);
  if (!Q || !Y) return set_error(c, KRR_ERR_INVALID_ARG, "%s: Q or Y is NULL", fn);
  if ((const void*)Y == (const void*)Q) return set_error(c, KRR_ERR_INVALID_ARG, "%s: Y aliases Q", fn);
  if (!is_device_ptr(c, Q) || !is_device_ptr(c, Y))
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: Q and Y must be device arrays", fn);
  if (c.shard_index >= c.shard_count)
    return set_error(c, KRR_ERR_INVALID_ARG, "%s: shard index %d >= shard count %d", fn, c.shard_index,
                     c.shard_count);
  Ctx& pc = P->ctx;
  copy_product_options(pc, c);
  cudaError_t e = product_prepared(pc, P->P, Q, m, gamma, prec, Y, (cudaStream_t)stream);
  if (e) return cuda_error(c, e, fn);
  return KRR_OK;
}

krr_status krr_points_destroy(krr_handle h, krr_points P) {
  if (!h) return KRR_ERR_INVALID_ARG;
  if (!P) return KRR_OK;
  if (P->h != h) return set_error(h->ctx, KRR_ERR_INVALID_ARG, "krr_points_destroy: point set of another handle");
  cudaDeviceSynchronize();  // products in flight finish before their buffers go
  int err = DEV_OK;
  cudaMemcpy(&err, P->ctx.d_err, sizeof(int), cudaMemcpyDeviceToHost);
  free_points(P);
  if (err == DEV_TIMEOUT)
    return set_error(h->ctx, KRR_ERR_TIMEOUT, "krr_points_destroy: a product's bounded device wait ran out");
  if (err != DEV_OK) return set_error(h->ctx, KRR_ERR_CUDA, "krr_points_destroy: device error %d", err);
  return KRR_OK;
}

krr_status krr_kernel_mvp_rect(krr_handle h, const float* Xt, int64_t Nt, const float* Xs,
                               int64_t Ns, int d, float sigma, const float* Q, int m, float* Y,
                               krr_precision prec, void* stream) {
  NvtxRange nvtx_range("krr_kernel_mvp_rect");
  if (!h) return KRR_ERR_INVALID_ARG;
  Ctx& c = h->ctx;
  const char* fn = "krr_kernel_mvp_rect";
  krr_status s = check_points(c, fn, Xt, Nt, d, sigma);
  if (s) return s;
  if ((s = check_points(c, fn, Xs, Ns, d, sigma))) return s;
  if (m < 1 || m > 64) return set_error(c, KRR_ERR_INVALID_ARG, "%s: m = %d out of range [1, 64]", fn, m);
  if (Nt == 0) return KRR_OK;
  if (!Y) return set_error(c, KRR_ERR_INVALID_ARG, "%s: Y is NULL", fn);
  cudaStream_t st = (cudaStream_t)stream;
  float *dXt, *dXs, *dQ, *dY;
  bool s1, s2, s3, s4;
  if ((s = device_view(c, "stage.Xt", Xt, (size_t)Nt * d, true, st, &dXt, &s1))) return s;
  if ((s = device_view(c, "stage.Xs", Xs, (size_t)Ns * d, true, st, &dXs, &s2))) return s;
  if ((s = device_view(c, "stage.Q", Q, (size_t)Ns * m, true, st, &dQ, &s3))) return s;
  if ((s = device_view(c, "stage.Y", Y, (size_t)Nt * m, false, st, &dY, &s4))) return s;
  cudaError_t e;
  if (Ns == 0) {
    if ((e = cudaMemsetAsync(dY, 0, sizeof(float) * Nt * m, st))) return cuda_error(c, e, fn);
  } else {
    if (!Q) return set_error(c, KRR_ERR_INVALID_ARG, "%s: Q is NULL", fn);
    PointsDev T, S;
    if ((e = prepare_points(c, dXt, Nt, d, sigma, "pts_t", T, st))) return cuda_error(c, e, fn);
    if ((e = prepare_points(c, dXs, Ns, d, sigma, "pts_s", S, st))) return cuda_error(c, e, fn);
    void* qs;
    if ((e = c.ws.get("mvp.qs", sizeof(float) * S.Npad * m, &qs))) return cuda_error(c, e, fn);
    if ((e = gather_sorted(dQ, Ns, m, S.perm, S.Npad, (float*)qs, st))) return cuda_error(c, e, fn);
    for (int col = 0; col < m; ++col) {
      MvpOut o;
      o.perm = T.perm;
      o.out_orig = dY + (size_t)col * Nt;
      if ((e = mvp_launch(c, T, S, (const float*)qs + (size_t)col * S.Npad, nullptr, 0.f, prec, o, st)))
        return cuda_error(c, e, fn);
    }
  }
  if (s4 && (e = cudaMemcpyAsync(Y, dY, sizeof(float) * Nt * m, cudaMemcpyDeviceToHost, st)))
    return cuda_error(c, e, fn);
  if (s1 || s2 || s3 || s4) return read_device_error(c, st, fn);
  return KRR_OK;
}

}  // extern "C"
