// Host-streamed sampling: the samples are copied to the device, mapped and
// the results copied back chunk by chunk, with the copies of one chunk in
// flight while another is sampled (rtf_sample_pipelined in include/rtf.h).
//
// The caller's stream runs the sampling kernels; two copy streams per device
// (created once, never destroyed) run the host-to-device and device-to-host
// copies.  Events order them: the copy streams start after the work already
// on the caller's stream, the kernel of chunk k waits for its input copy, the
// output copy of chunk k waits for its kernel, and the caller's stream waits
// for the last output copy, so that synchronising it makes the host results
// visible (or, when the caller passes an event, that event is recorded after
// the last output copy instead, and the caller's stream waits only for the
// input copies: later work on it then overlaps the copies back).  An event is re-recorded for every chunk: a wait takes the record
// most recent at the time it is enqueued.  The pattern is a fork and join of
// the caller's stream, which stream capture turns into graph edges.
#include <cstdint>
#include <mutex>

#include "rtf.h"
#include "rtf_device.cuh"

namespace rtf {

cudaError_t launch_sample(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                          int64_t count, int mode, int32_t* idx_out, float* pos_out,
                          cudaStream_t st);

namespace {

constexpr int kMaxDevices = 64;

struct CopyStreams {
  bool ready = false;
  cudaStream_t in = nullptr, out = nullptr;
  cudaEvent_t start = nullptr, in_done = nullptr, kernel_done = nullptr, out_done = nullptr;
};

CopyStreams g_streams[kMaxDevices];
std::mutex g_streams_mu;

cudaError_t copy_streams(CopyStreams** cs) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_streams_mu);
  CopyStreams& c = g_streams[dev];
  if (!c.ready) {
    const unsigned ef = cudaEventDisableTiming;
    if ((e = cudaStreamCreateWithFlags(&c.in, cudaStreamNonBlocking)) ||
        (e = cudaStreamCreateWithFlags(&c.out, cudaStreamNonBlocking)) ||
        (e = cudaEventCreateWithFlags(&c.start, ef)) ||
        (e = cudaEventCreateWithFlags(&c.in_done, ef)) ||
        (e = cudaEventCreateWithFlags(&c.kernel_done, ef)) ||
        (e = cudaEventCreateWithFlags(&c.out_done, ef)))
      return e;
    c.ready = true;
  }
  *cs = &c;
  return cudaSuccess;
}

}  // namespace

cudaError_t launch_sample_pipelined(const rtf_forest* f, const uint32_t* u_host, uint32_t* u_dev,
                                    const int32_t* dist_host, int32_t* dist_dev, int64_t count,
                                    int mode, int32_t* idx_dev, float* pos_dev,
                                    int32_t* idx_host, float* pos_host, int64_t chunk,
                                    cudaEvent_t done, cudaStream_t st) {
  if (count == 0) return done ? cudaEventRecord(done, st) : cudaSuccess;
  CopyStreams* cs = nullptr;
  cudaError_t e = copy_streams(&cs);
  if (e != cudaSuccess) return e;
  const int per = (mode & 0xFF) == RTF_SAMPLE_2D ? 2 : 1;  // values per sample
  const bool copy_in = u_host != nullptr || dist_host != nullptr;
  const bool copy_out = idx_host != nullptr || pos_host != nullptr;
  // the copies start after the work already queued on the caller's stream
  if ((e = cudaEventRecord(cs->start, st))) return e;
  if (copy_in && (e = cudaStreamWaitEvent(cs->in, cs->start, 0))) return e;
  if (copy_out && (e = cudaStreamWaitEvent(cs->out, cs->start, 0))) return e;
  for (int64_t off = 0; off < count; off += chunk) {
    const int64_t n = count - off < chunk ? count - off : chunk;
    const size_t v0 = (size_t)(off * per), nv = (size_t)(n * per);
    if (copy_in) {
      if (u_host && (e = cudaMemcpyAsync(u_dev + v0, u_host + v0, 4 * nv, cudaMemcpyHostToDevice,
                                         cs->in)))
        return e;
      if (dist_host && (e = cudaMemcpyAsync(dist_dev + off, dist_host + off, 4 * (size_t)n,
                                            cudaMemcpyHostToDevice, cs->in)))
        return e;
      if ((e = cudaEventRecord(cs->in_done, cs->in))) return e;
      if ((e = cudaStreamWaitEvent(st, cs->in_done, 0))) return e;
    }
    if ((e = launch_sample(f, u_dev + v0, dist_dev ? dist_dev + off : nullptr, n, mode,
                           idx_dev + v0, pos_dev + v0, st)))
      return e;
    if (copy_out) {
      if ((e = cudaEventRecord(cs->kernel_done, st))) return e;
      if ((e = cudaStreamWaitEvent(cs->out, cs->kernel_done, 0))) return e;
      if (idx_host && (e = cudaMemcpyAsync(idx_host + v0, idx_dev + v0, 4 * nv,
                                           cudaMemcpyDeviceToHost, cs->out)))
        return e;
      if (pos_host && (e = cudaMemcpyAsync(pos_host + v0, pos_dev + v0, 4 * nv,
                                           cudaMemcpyDeviceToHost, cs->out)))
        return e;
    }
  }
  // join: the caller's stream waits for the last copies of both directions,
  // or the caller's event marks the end of the copies back
  if (copy_out) {
    if (done) {
      if ((e = cudaEventRecord(done, cs->out))) return e;
    } else {
      if ((e = cudaEventRecord(cs->out_done, cs->out))) return e;
      if ((e = cudaStreamWaitEvent(st, cs->out_done, 0))) return e;
    }
  } else if (done && (e = cudaEventRecord(done, st))) {
    return e;
  }
  if (copy_in) {
    if ((e = cudaEventRecord(cs->in_done, cs->in))) return e;
    if ((e = cudaStreamWaitEvent(st, cs->in_done, 0))) return e;
  }
  return cudaGetLastError();
}

}  // namespace rtf
