// Krylov solvers (hot-path steps A5, A7-A10): truncated CG, FGMRES with
// modified Gram-Schmidt Arnoldi and Givens least squares, device-side control.
#include "api_util.h"
#include "common.cuh"
#include "internal.h"

using namespace krr;

extern "C" {

krr_status krr_cg_solve(krr_handle h, const float*, int64_t, int, float, float, const float*,
                        float*, double, int, krr_precision, krr_solve_info*, void*) {
  if (!h) return KRR_ERR_INVALID_ARG;
  return set_error(h->ctx, KRR_ERR_UNIMPLEMENTED, "krr_cg_solve: not built yet");
}

krr_status krr_fgmres_solve(krr_handle h, const float*, int64_t, int, float, float, const float*,
                            int, float*, const krr_fgmres_opts*, krr_solve_info*, void*) {
  if (!h) return KRR_ERR_INVALID_ARG;
  return set_error(h->ctx, KRR_ERR_UNIMPLEMENTED, "krr_fgmres_solve: not built yet");
}

krr_status krr_fgmres_solve_batched(krr_handle h, const krr_problem*, int, int, float, int,
                                    const krr_fgmres_opts*, krr_solve_info*, void*) {
  if (!h) return KRR_ERR_INVALID_ARG;
  return set_error(h->ctx, KRR_ERR_UNIMPLEMENTED, "krr_fgmres_solve_batched: not built yet");
}

krr_status krr_mll_grad(krr_handle h, const float*, int64_t, int, float, float, const float*, int,
                        uint64_t, const krr_fgmres_opts*, double*, double*, float*,
                        krr_solve_info*, void*) {
  if (!h) return KRR_ERR_INVALID_ARG;
  return set_error(h->ctx, KRR_ERR_UNIMPLEMENTED, "krr_mll_grad: not built yet");
}

}  // extern "C"
