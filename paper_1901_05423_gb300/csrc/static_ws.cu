// rtf_build_static: the single-distribution build with its scratch memory in
// a fixed array inside the library instead of a caller-supplied workspace.
//
// Some callers cannot allocate device memory at the point where they need a
// build: a plugin that runs inside a host application which owns the whole
// device memory budget, a real-time loop that forbids allocation after
// start-up, or a foreign runtime that hands over raw pointers but has no way
// to reach an allocator.  This entry point lets them build without ever
// allocating; they still pass the weights and the forest buffers.
//
// The scratch is one file-scope device array of kStaticBytes (10 MiB), enough
// for n <= 2^20 weights and m <= 16 guide bits.  Every GPU that loads the
// library holds it until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "rtf.h"

namespace {

constexpr int64_t kStaticMaxElems = int64_t(1) << 20;
constexpr int32_t kStaticMaxBits = 16;
constexpr size_t kStaticBytes = size_t(10) << 20;
constexpr int kMaxContexts = 64;

// Every build clears or writes each part of its workspace that it reads, so
// the array's leftover contents from the previous call do no harm.
static __device__ __align__(256) unsigned char g_rtf_static_ws[kStaticBytes];

// Device address of the array per CUDA context.  The array lives in the
// library's module, which every context loads separately, so the address is
// looked up once per context, with that context current.  (The primary
// context of a device keeps its handle across cudaDeviceReset, so an address
// cached before a reset is not looked up again: rtf_build_static is not
// supported after cudaDeviceReset in the same process.)
struct CtxEntry {
  CUcontext ctx;
  void* ptr;
};

std::mutex g_setup_lock;
CtxEntry g_entries[kMaxContexts] = {};
int g_num_entries = 0;

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_get_current = nullptr;

rtf_status current_context(CUcontext* ctx) {
  if (g_ctx_get_current == nullptr) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || fn == nullptr)
      return RTF_ECUDA;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(fn);
  }
  *ctx = nullptr;
  if (g_ctx_get_current(ctx) != CUDA_SUCCESS) return RTF_ECUDA;
  return RTF_OK;
}

// Device address of the array in the current context.  Host code must not
// pass the symbol itself to a kernel: on the host it only names a stand-in.
rtf_status static_workspace(void** out) {
  std::lock_guard<std::mutex> guard(g_setup_lock);
  CUcontext ctx = nullptr;
  rtf_status s = current_context(&ctx);
  if (s != RTF_OK) return s;
  if (ctx == nullptr) {
    // no context on this thread yet: cudaSetDevice makes the current device's
    // primary context current (it allocates nothing)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaSetDevice(dev) != cudaSuccess) return RTF_ECUDA;
    if ((s = current_context(&ctx)) != RTF_OK) return s;
    if (ctx == nullptr) return RTF_ECUDA;
  }
  for (int k = 0; k < g_num_entries; ++k) {
    if (g_entries[k].ctx == ctx) {
      *out = g_entries[k].ptr;
      return RTF_OK;
    }
  }
  if (g_num_entries == kMaxContexts) return RTF_ECUDA;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_rtf_static_ws) != cudaSuccess || p == nullptr)
    return RTF_ECUDA;
  g_entries[g_num_entries++] = CtxEntry{ctx, p};
  *out = p;
  return RTF_OK;
}

}  // namespace

extern "C" rtf_status rtf_build_static(const float* w, int64_t n, int32_t m, rtf_forest* f,
                                       void* stream) {
  if (n > kStaticMaxElems || m > kStaticMaxBits) return RTF_EWORKSPACE;
  if (rtf_build_workspace_size(n, 1, int64_t(1) << (m < 0 ? 0 : m)) > kStaticBytes)
    return RTF_EWORKSPACE;
  void* ws = nullptr;
  rtf_status s = static_workspace(&ws);
  if (s != RTF_OK) return s;
  return rtf_build(w, n, m, f, ws, kStaticBytes, stream);
}
