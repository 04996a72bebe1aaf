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
#include <cstdint>
#include <mutex>

#include "rtf.h"

namespace {

constexpr int64_t kStaticMaxElems = int64_t(1) << 20;
constexpr int32_t kStaticMaxBits = 16;
constexpr size_t kStaticBytes = size_t(10) << 20;
constexpr int kMaxDevices = 64;

// Every build clears or writes each part of its workspace that it reads, so
// the array's leftover contents from the previous call do no harm.
static __device__ __align__(256) unsigned char g_rtf_static_ws[kStaticBytes];

std::mutex g_setup_lock;
void* g_static_ptr[kMaxDevices] = {};

// Device address of the array on the current device (looked up once per
// device, with that device current).  Host code must not pass the symbol
// itself to a kernel: on the host it only names a stand-in.
rtf_status static_workspace(void** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return RTF_ECUDA;
  std::lock_guard<std::mutex> guard(g_setup_lock);
  if (g_static_ptr[dev] == nullptr) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_rtf_static_ws) != cudaSuccess || p == nullptr)
      return RTF_ECUDA;
    g_static_ptr[dev] = p;
  }
  *out = g_static_ptr[dev];
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
