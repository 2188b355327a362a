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

static cudaEvent_t take_event(Mesh* m) {
  if (!m->event_pool.empty()) {
    cudaEvent_t e = m->event_pool.back();
    m->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

KTimer::KTimer(Mesh* m, int k, cudaStream_t s) : m_(m), k_(k), s_(s) {
  m_->kstat[k_].launches++;
  if (m_->prof_on) {
    e0_ = take_event(m_);
    if (e0_) cudaEventRecord(e0_, s_);
  }
}

KTimer::~KTimer() {
  if (!e0_) return;
  cudaEvent_t e1 = take_event(m_);
  if (!e1) return;
  cudaEventRecord(e1, s_);
  m_->kstat[k_].events.push_back({e0_, e1});
}

static void release_events(Mesh& M) {
  for (auto& ks : M.kstat) {
    for (auto& pr : ks.events) {
      M.event_pool.push_back(pr.first);
      M.event_pool.push_back(pr.second);
    }
    ks.events.clear();
  }
}

void destroy_events(Mesh& M) {
  release_events(M);
  for (cudaEvent_t e : M.event_pool) cudaEventDestroy(e);
  M.event_pool.clear();
}

}  // namespace vef

using namespace vef;

extern "C" vef_status vef_profile(vef_mesh mesh, int enable) {
  if (!mesh) { set_last_error("mesh is NULL"); return VEF_ERR_INVALID_ARG; }
  Mesh& M = mesh->impl;
  VEF_CUDA_TRY(cudaDeviceSynchronize());
  release_events(M);
  for (auto& ks : M.kstat) ks.launches = 0;
  M.prof_on = enable != 0;
  return VEF_OK;
}

extern "C" vef_status vef_profile_read(vef_mesh mesh, vef_kernel_stat* out) {
  if (!mesh || !out) { set_last_error("NULL argument"); return VEF_ERR_INVALID_ARG; }
  Mesh& M = mesh->impl;
  for (int k = 0; k < VEF_K_COUNT; ++k) {
    double ms = 0.0;
    for (auto& pr : M.kstat[k].events) {
      VEF_CUDA_TRY(cudaEventSynchronize(pr.second));
      float t = 0.f;
      VEF_CUDA_TRY(cudaEventElapsedTime(&t, pr.first, pr.second));
      ms += t;
    }
    out[k].launches = M.kstat[k].launches;
    out[k].ms = ms;
  }
  return VEF_OK;
}

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
    case VEF_ERR_BOUNDS: return "VEF_ERR_BOUNDS";
  }
  return "VEF_ERR_UNKNOWN";
}

extern "C" const char* vef_last_error(void) { return vef::g_last_error.c_str(); }

extern "C" int vef_build_checked(void) {
#ifdef VEF_CHECKED
  return 1;
#else
  return 0;
#endif
}
