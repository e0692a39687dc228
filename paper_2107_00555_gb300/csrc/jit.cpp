// Run-time compilation of generated kernels (Sec. 3.3: compile the
// specialised program once, then call it like a function).  NVRTC compiles
// straight to an sm_103a cubin; cubins are cached in memory by source hash
// and, when DCP_NVRTC_CACHE names a directory, on disk.  Modules are loaded
// into the calling thread's current CUDA context on first use.
#include <nvrtc.h>

#include <chrono>
#include <cinttypes>
#include <cstdio>
#include <cstdlib>
#include <fstream>
#include <mutex>
#include <unordered_map>

#include "dcp_internal.h"

namespace dcp {

namespace {

std::mutex g_mu;
std::unordered_map<uint64_t, std::shared_ptr<const std::vector<char>>> g_cubins;  // hash -> cubin
struct Loaded {
  CUcontext ctx;
  CUmodule mod;
  CUfunction fn;
  int regs;
};
std::unordered_map<uint64_t, Loaded> g_loaded;              // (hash) -> function in ctx

const char* kOpts[] = {"--gpu-architecture=sm_103a", "-std=c++17", "-lineinfo",
                       "--extra-device-vectorization", "-DDCP_RTC=1"};

std::string disk_path(uint64_t h) {
  const char* dir = std::getenv("DCP_NVRTC_CACHE");
  if (!dir || !*dir) return "";
  char name[64];
  std::snprintf(name, sizeof name, "/dcp_%016" PRIx64 ".cubin", h);
  return std::string(dir) + name;
}

}  // namespace

CubinRef nvrtc_compile(const std::string& src, const std::string& name, double* ms,
                       std::string* log_out) {
  uint64_t h = fnv1a(src);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_cubins.find(h);
    if (it != g_cubins.end()) {
      if (ms) *ms = 0.0;
      return it->second;
    }
  }
  std::string dp = disk_path(h);
  if (!dp.empty()) {
    std::ifstream f(dp, std::ios::binary);
    if (f) {
      std::vector<char> c((std::istreambuf_iterator<char>(f)), std::istreambuf_iterator<char>());
      if (!c.empty()) {
        auto ref = std::make_shared<const std::vector<char>>(std::move(c));
        std::lock_guard<std::mutex> lk(g_mu);
        g_cubins[h] = ref;
        if (ms) *ms = 0.0;
        return ref;
      }
    }
  }
  auto t0 = std::chrono::steady_clock::now();
  const char* hdr_src[] = {device_header_source(), kernel_map_source(), kernel_stencil2d_source(),
                           kernel_stencil3d_source(), kernel_stream_source(), kernel_axis_source(),
                           kernel_math64_source(), kernel_adj_source(), kernel_coop_source()};
  const char* hdr_name[] = {"dcp_device.cuh", "k_map.cuh", "k_stencil2d.cuh", "k_stencil3d.cuh",
                            "k_stencil2d_stream.cuh", "k_axis.cuh", "k_math64.cuh",
                            "k_stencil_adj.cuh", "k_stencil2d_coop.cuh"};
  nvrtcProgram prog;
  nvrtcResult r = nvrtcCreateProgram(&prog, src.c_str(), (name + ".cu").c_str(), 9, hdr_src,
                                     hdr_name);
  if (r != NVRTC_SUCCESS) fail(DCP_E_COMPILE, std::string("nvrtcCreateProgram: ") + nvrtcGetErrorString(r));
  // DCP_PTXAS_VERBOSE=1 prints the assembler's register / spill report of
  // every compiled kernel to stderr (a diagnostic; needs no GPU)
  const char* verbose = std::getenv("DCP_PTXAS_VERBOSE");
  const bool vb = verbose && *verbose == '1';
  std::vector<const char*> opts(kOpts, kOpts + sizeof kOpts / sizeof kOpts[0]);
  if (vb) opts.push_back("--ptxas-options=-v");
  r = nvrtcCompileProgram(prog, (int)opts.size(), opts.data());
  size_t logsz = 0;
  nvrtcGetProgramLogSize(prog, &logsz);
  std::string log(logsz, '\0');
  if (logsz) nvrtcGetProgramLog(prog, &log[0]);
  if (log_out) *log_out = log;
  if (vb && r == NVRTC_SUCCESS) std::fprintf(stderr, "[dcp] %s:\n%s\n", name.c_str(), log.c_str());
  if (r != NVRTC_SUCCESS) {
    nvrtcDestroyProgram(&prog);
    fail(DCP_E_COMPILE, "NVRTC failed for " + name + ": " + log);
  }
  size_t n = 0;
  nvrtcGetCUBINSize(prog, &n);
  std::vector<char> cubin(n);
  nvrtcGetCUBIN(prog, cubin.data());
  nvrtcDestroyProgram(&prog);
  auto t1 = std::chrono::steady_clock::now();
  if (ms) *ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
  if (!dp.empty()) {
    std::string tmp = dp + ".tmp" + std::to_string((long)std::rand());
    std::ofstream f(tmp, std::ios::binary);
    if (f) {
      f.write(cubin.data(), (std::streamsize)cubin.size());
      f.close();
      std::rename(tmp.c_str(), dp.c_str());
    }
  }
  auto ref = std::make_shared<const std::vector<char>>(std::move(cubin));
  std::lock_guard<std::mutex> lk(g_mu);
  g_cubins[h] = ref;
  return ref;
}

CUfunction load_function(const std::string& src, const std::string& name, double* ms, int* regs) {
  uint64_t h = fnv1a(src);
  CUcontext ctx = nullptr;
  check_cu(drv().ctxGetCurrent(&ctx), "cuCtxGetCurrent");
  if (!ctx) fail(DCP_E_CUDA, "no current CUDA context");
  {
    std::lock_guard<std::mutex> lk(g_mu);
    auto it = g_loaded.find(h);
    if (it != g_loaded.end() && it->second.ctx == ctx) {
      if (regs) *regs = it->second.regs;
      return it->second.fn;
    }
  }
  CubinRef cubin = nvrtc_compile(src, name, ms, nullptr);
  CUmodule mod;
  check_cu(drv().moduleLoadData(&mod, cubin->data()), "cuModuleLoadData");
  CUfunction fn;
  check_cu(drv().moduleGetFunction(&fn, mod, name.c_str()), "cuModuleGetFunction");
  int nregs = 0;
  drv().funcGetAttribute(&nregs, CU_FUNC_ATTRIBUTE_NUM_REGS, fn);
  if (regs) *regs = nregs;
  std::lock_guard<std::mutex> lk(g_mu);
  g_loaded[h] = Loaded{ctx, mod, fn, nregs};
  return fn;
}

}  // namespace dcp
