// Helpers shared by the C-ABI translation units (defined in krr_api.cu).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "internal.h"

namespace krr {

// NVTX range over an entry point (host side; shown by profilers that read
// NVTX, free otherwise: the header-only NVTX v3 only forwards when a tool is
// attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

krr_status set_error(Ctx& c, krr_status s, const char* fmt, ...);
krr_status cuda_error(Ctx& c, cudaError_t e, const char* what);
bool is_device_ptr(const Ctx& c, const void* p);
krr_status read_device_error(Ctx& c, cudaStream_t st, const char* what);
krr_status check_points(Ctx& c, const char* fn, const float* X, int64_t N, int d, float sigma);
krr_status device_view(Ctx& c, const char* slot, const float* p, size_t count, bool in,
                       cudaStream_t st, float** out, bool* staged);
krr_status device_view_d(Ctx& c, const char* slot, const double* p, size_t count, bool in,
                         cudaStream_t st, double** out, bool* staged);

}  // namespace krr

struct krr_handle_s {
  krr::Ctx ctx;
};

// A prepared point set (krr_points_create).  It owns a context of its own:
// the sorted layout, block metadata and every scratch buffer of its products
// live in that context's workspace, so work on the handle never reallocates
// what a captured graph of its products refers to.  The handle's product
// options are copied into it at each call.
struct krr_points_s {
  krr_handle_s* h = nullptr;
  krr::Ctx ctx;
  krr::PointsDev P;
};
