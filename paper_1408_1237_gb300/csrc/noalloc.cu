// krr_kernel_mvp_noalloc: the kernel product for callers that cannot
// allocate device memory.
//
// Who needs it: a process whose device memory pool belongs to another
// framework (an inference server, a game engine) that forbids foreign
// cudaMalloc calls or would be fragmented by them, and code on a
// latency-bound path where cudaMalloc's implicit device synchronisation is
// not acceptable.  Such a caller cannot create a krr_handle either (the handle
// grows its workspace with cudaMalloc).
//
// Limits: device arrays only, N <= 16384 points, d <= 8, m <= 16 columns.
//
// How: every scratch buffer the product needs (sorting keys, the packed
// points, block metadata, split partial sums, counters, the error word) is
// carved out of one file-scope device array of KRR_NOALLOC_SCRATCH_BYTES.
// The array exists on every GPU that loads the library, from load to exit.
// In host code its name is only a host-side stand-in, so its device address
// is looked up with cudaGetSymbolAddress, once per device, by the first call
// made with that device current; that first call should therefore come
// before any stream capture.  The carved-up workspace is presented to the
// same prep and product code as a handle's workspace, marked fixed: each
// region is recorded with its real size, and a request for more than a
// region holds (or for a buffer the table does not list) fails with
// KRR_ERR_OOM before any kernel could write past the region.
//
// The call is not asynchronous: the point preparation reads two block counts
// back to the host to size the product grids, so the call waits for `stream`
// up to that point.  It must therefore not be made while `stream` is being
// captured into a graph (it returns KRR_ERR_INVALID_ARG then), nor from a
// host function enqueued on a stream (CUDA forbids CUDA calls there).
//
// Every call on a device shares the one array and it keeps the previous
// call's contents; the counters that must start at zero are cleared by each
// call.  Calls that overlap on the GPU (different streams, or different host
// threads) race on the array and give wrong results: serialise them.
#include <cmath>
#include <mutex>

#include "api_util.h"
#include "common.cuh"
#include "internal.h"

namespace krr {
namespace {

constexpr int64_t NA_MAX_N = 16384;  // points
constexpr int NA_MAX_D = 8;
constexpr int NA_MAX_M = 16;          // right-hand sides
constexpr int NA_MAX_DEV = 64;

// Upper bounds of every buffer the prep and product code requests for
// N <= NA_MAX_N, d <= NA_MAX_D, m <= NA_MAX_M (see prep.cu and mvp.cu).
constexpr int64_t NPAD = NA_MAX_N;                 // multiple of PAD
constexpr int64_t NCHUNK = NA_MAX_N / 2048;         // radix-sort chunks
constexpr int64_t NBLK = NA_MAX_N / 32;             // warp blocks (T >= 1)
constexpr int64_t NTILE = NPAD / 256;               // source tiles
constexpr int64_t MAX_SPLITS = 64;

struct Region {
  const char* name;
  size_t bytes;
};

constexpr Region kRegions[] = {
    {"na.xs", sizeof(float) * NPAD * NA_MAX_D},
    {"na.perm", sizeof(int) * NPAD},
    {"sort.ka", sizeof(uint32_t) * NA_MAX_N},
    {"sort.kb", sizeof(uint32_t) * NA_MAX_N},
    {"sort.va", sizeof(int) * NA_MAX_N},
    {"sort.vb", sizeof(int) * NA_MAX_N},
    {"sort.hist", sizeof(uint32_t) * 256 * NCHUNK},
    {"sort.bbp", sizeof(float) * 2 * NA_MAX_D * 256},
    {"sort.bb", sizeof(float) * 2 * NA_MAX_D},
    {"na.ctr", sizeof(float) * NBLK * NA_MAX_D},
    {"na.order", sizeof(int) * NBLK},
    {"na.nexp", sizeof(int)},
    {"sort.flag", sizeof(int) * NBLK},
    {"na.tbox", sizeof(float) * 2 * NA_MAX_D * NTILE},
    {"na.sbctr", sizeof(float) * (NA_MAX_N / SB) * NA_MAX_D},
    {"na.sborder", sizeof(int) * (NA_MAX_N / SB)},
    {"na.sbnexp", sizeof(int)},
    {"na.sbflag", sizeof(int) * (NA_MAX_N / SB)},
    {"mvp.qs", sizeof(float) * NPAD * NA_MAX_M},
    {"mvp.part", sizeof(double) * MAX_SPLITS * NPAD},
    {"mvp.fac", sizeof(float) * NPAD},
    {"mvp.dotpart", sizeof(double) * MAX_COLS * (NPAD / 256)},
    {"mvp.dotcnt", sizeof(unsigned) * MAX_COLS},
    {"na.err", sizeof(int)},
};

constexpr size_t align256(size_t b) { return (b + 255) / 256 * 256; }

constexpr size_t total_bytes() {
  size_t t = 0;
  for (const Region& r : kRegions) t += align256(r.bytes);
  return t;
}

}  // namespace
}  // namespace krr

#define KRR_NOALLOC_SCRATCH_BYTES (krr::total_bytes())

// The scratch array: 10,415,872 bytes (about 10 MB).  Host code must not take its address
// directly: use the pointer from cudaGetSymbolAddress.
static_assert(KRR_NOALLOC_SCRATCH_BYTES == 10415872, "the documented scratch size");
static __device__ __align__(256) unsigned char g_noalloc_scratch[KRR_NOALLOC_SCRATCH_BYTES];

namespace krr {
namespace {

struct DeviceScratch {
  bool ready = false;
  unsigned char* base = nullptr;
  Ctx ctx;
  std::mutex mu;
};

DeviceScratch g_dev[NA_MAX_DEV];
std::mutex g_setup_mu;

// Once per device, with that device current: find the array's device address
// and lay the workspace out over it.
krr_status setup_device(int dev, DeviceScratch*& out) {
  if (dev < 0 || dev >= NA_MAX_DEV) return KRR_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(g_setup_mu);
  DeviceScratch& d = g_dev[dev];
  if (!d.ready) {
    void* base = nullptr;
    if (cudaGetSymbolAddress(&base, g_noalloc_scratch) != cudaSuccess || base == nullptr) {
      cudaGetLastError();
      return KRR_ERR_CUDA;
    }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
      cudaGetLastError();
      return KRR_ERR_CUDA;
    }
    d.base = (unsigned char*)base;
    d.ctx.device = dev;
    d.ctx.num_sms = sms;
    d.ctx.allow_tcx = false;
    d.ctx.tcgen05_auto = false;  // the regions are laid out for the mma.sync kernels
    d.ctx.use_tcgen05 = false;
    size_t off = 0;
    for (const Region& r : kRegions) {
      // each region with its real (256-byte rounded) size; the workspace is
      // fixed, so a larger request fails instead of allocating
      d.ctx.ws.slots[r.name] = Buf{d.base + off, align256(r.bytes)};
      off += align256(r.bytes);
    }
    d.ctx.ws.fixed = true;
    d.ctx.d_err = (int*)d.ctx.ws.slots["na.err"].p;
    d.ready = true;
  }
  out = &d;
  return KRR_OK;
}

bool on_device(int dev, const void* p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

}  // namespace
}  // namespace krr

using namespace krr;

extern "C" krr_status krr_kernel_mvp_noalloc(const float* X, int64_t N, int d, float sigma,
                                             float gamma, const float* Q, int m, float* Y,
                                             void* stream) {
  if (N > NA_MAX_N || d > NA_MAX_D || m > NA_MAX_M) return KRR_ERR_SIZE_LIMIT;
  if (N < 0 || d < 1 || m < 1) return KRR_ERR_INVALID_ARG;
  if (!(sigma > 0.f) || !std::isfinite(sigma) || !(gamma >= 0.f) || !std::isfinite(gamma))
    return KRR_ERR_INVALID_ARG;
  if (N == 0) return KRR_OK;
  if (!X || !Q || !Y || (const void*)Y == (const void*)Q || (const void*)Y == (const void*)X)
    return KRR_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)stream;
  // the preparation waits for the stream, which a capture does not allow
  // (checked before any other CUDA call of this entry point)
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(st, &cs) != cudaSuccess) {
    cudaGetLastError();
    return KRR_ERR_INVALID_ARG;
  }
  if (cs != cudaStreamCaptureStatusNone) return KRR_ERR_INVALID_ARG;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return KRR_ERR_CUDA;
  }
  DeviceScratch* ds = nullptr;
  krr_status s = setup_device(dev, ds);
  if (s) return s;
  Ctx& c = ds->ctx;
  std::lock_guard<std::mutex> lk(ds->mu);
  // device arrays only: staging host arrays would need an allocation
  if (!on_device(dev, X) || !on_device(dev, Q) || !on_device(dev, Y)) return KRR_ERR_INVALID_ARG;
  const size_t nslots = c.ws.slots.size();
  // counters that must start at zero: the error word and the dot ticket
  cudaError_t e = cudaMemsetAsync(c.d_err, 0, sizeof(int), st);
  if (!e) e = cudaMemsetAsync(c.ws.slots["mvp.dotcnt"].p, 0, sizeof(unsigned) * MAX_COLS, st);
  if (e) return cuda_error(c, e, "krr_kernel_mvp_noalloc");
  PointsDev P;
  if ((e = prepare_points(c, X, N, d, sigma, "na", P, st))) return cuda_error(c, e, "krr_kernel_mvp_noalloc");

  float* qs = (float*)c.ws.slots["mvp.qs"].p;
  if ((e = gather_sorted(Q, N, m, P.perm, P.Npad, qs, st))) return cuda_error(c, e, "krr_kernel_mvp_noalloc");
  for (int col = 0; col < m; ++col) {
    const float* qc = qs + (size_t)col * P.Npad;
    MvpOut o;
    o.perm = P.perm;
    o.out_orig = Y + (size_t)col * N;
    if ((e = mvp_launch(c, P, P, qc, qc, gamma, KRR_FP32, o, st)))
      return cuda_error(c, e, "krr_kernel_mvp_noalloc");
  }
  // every buffer must have come from the carved regions
  if (c.ws.slots.size() != nslots) return KRR_ERR_CUDA;
  return KRR_OK;
}
