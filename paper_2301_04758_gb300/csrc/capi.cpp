// Status strings and per-thread error messages of the C ABI.
#include <string>

#include "common.h"

namespace vef {

static thread_local std::string g_last_error;

void set_last_error(const std::string& msg) { g_last_error = msg; }

vef_status cuda_fail(cudaError_t err, const char* what) {
  set_last_error(std::string(what) + ": " + cudaGetErrorString(err));
  cudaGetLastError();
  return err == cudaErrorMemoryAllocation ? VEF_ERR_OOM : VEF_ERR_CUDA;
}

}  // namespace vef

extern "C" const char* vef_status_string(vef_status s) {
  switch (s) {
    case VEF_OK: return "VEF_OK";
    case VEF_ERR_INVALID_ARG: return "VEF_ERR_INVALID_ARG";
    case VEF_ERR_CUDA: return "VEF_ERR_CUDA";
    case VEF_ERR_OOM: return "VEF_ERR_OOM";
    case VEF_ERR_TIMEOUT: return "VEF_ERR_TIMEOUT";
    case VEF_ERR_NOT_CONVERGED: return "VEF_ERR_NOT_CONVERGED";
    case VEF_ERR_NONPOSITIVE_DENOM: return "VEF_ERR_NONPOSITIVE_DENOM";
    case VEF_ERR_NOT_IMPLEMENTED: return "VEF_ERR_NOT_IMPLEMENTED";
  }
  return "VEF_ERR_UNKNOWN";
}

extern "C" const char* vef_last_error(void) { return vef::g_last_error.c_str(); }
