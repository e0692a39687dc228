// CUDA driver API entry points used by the runtime (module loading and
// kernel launch of NVRTC-compiled cubins), resolved through the CUDA runtime
// at first use.  The library therefore loads on machines without a GPU
// driver (planning and NVRTC compilation need none); only running fails.
#include <mutex>

#include "dcp_internal.h"

namespace dcp {

namespace {
Driver g_drv;
bool g_ok = false;
std::once_flag g_once;
std::string g_err;

template <class F>
bool get(const char* name, F& fn) {
  void* p = nullptr;
  cudaDriverEntryPointQueryResult q;
  cudaError_t e = cudaGetDriverEntryPointByVersion(name, &p, 13000, cudaEnableDefault, &q);
  if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !p) {
    g_err = std::string("driver entry point ") + name + " unavailable: " + cudaGetErrorString(e);
    return false;
  }
  fn = reinterpret_cast<F>(p);
  return true;
}
}  // namespace

const Driver& drv() {
  std::call_once(g_once, [] {
    g_ok = get("cuCtxGetCurrent", g_drv.ctxGetCurrent) &&
           get("cuModuleLoadData", g_drv.moduleLoadData) &&
           get("cuModuleGetFunction", g_drv.moduleGetFunction) &&
           get("cuFuncGetAttribute", g_drv.funcGetAttribute) &&
           get("cuFuncSetAttribute", g_drv.funcSetAttribute) &&
           get("cuOccupancyMaxActiveBlocksPerMultiprocessor", g_drv.occupancy) &&
           get("cuLaunchKernel", g_drv.launchKernel) &&
           get("cuLaunchCooperativeKernel", g_drv.launchCooperative) &&
           get("cuGetErrorString", g_drv.getErrorString);
  });
  if (!g_ok) fail(DCP_E_CUDA, g_err.empty() ? "CUDA driver unavailable" : g_err);
  return g_drv;
}

void check_cu(CUresult r, const char* what) {
  if (r != CUDA_SUCCESS) {
    const char* s = nullptr;
    if (g_ok && g_drv.getErrorString) g_drv.getErrorString(r, &s);
    std::string msg = std::string(what) + ": " + (s ? s : ("CUDA driver error " + std::to_string((int)r)));
    if (r == CUDA_ERROR_OUT_OF_MEMORY) fail(DCP_E_OOM, msg);
    fail(DCP_E_CUDA, msg);
  }
}

}  // namespace dcp
