// C interface (include/rtf.h): argument checks, workspace carving and the
// launch sequences.  No allocation, no synchronisation: every call is a
// sequence of stream-ordered launches and memsets.
#include <cstdint>
#include <cstring>

#include "rtf.h"
#include "rtf_device.cuh"

namespace rtf {
cudaError_t launch_build(const float* w, int64_t N, int64_t Nw, int D, int marginal,
                         const int64_t* offsets, const int32_t* m_arr, const int64_t* goff,
                         int64_t n_single, int m_single, const rtf_forest* f, void* ws,
                         cudaStream_t st);
cudaError_t launch_sample(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                          int64_t count, int mode, int32_t* idx_out, float* pos_out,
                          cudaStream_t st);
cudaError_t launch_sample_pipelined(const rtf_forest* f, const uint32_t* u_host, uint32_t* u_dev,
                                    const int32_t* dist_host, int32_t* dist_dev, int64_t count,
                                    int mode, int32_t* idx_dev, float* pos_dev,
                                    int32_t* idx_host, float* pos_host, int64_t chunk,
                                    cudaEvent_t done, cudaStream_t st);
cudaError_t launch_sample_loads(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                                int64_t count, int mode, int32_t* loads_out, cudaStream_t st);
size_t backward_ws_bytes(int64_t N, int32_t D);
cudaError_t launch_build_quad(const rtf_forest* f, rtf_quad_rec* quad, cudaStream_t st);
cudaError_t launch_wait_probe(uint32_t* status, uint64_t* scratch, cudaStream_t st);
void set_launch_shape(const int32_t* v);
void get_launch_shape(int32_t* v);
cudaError_t launch_sample_quad(const rtf_forest* f, const rtf_quad_rec* quad, const uint32_t* u,
                               const int32_t* dist_id, int64_t count, int mode, int32_t* idx_out,
                               float* pos_out, int32_t* loads_out, cudaStream_t st);
cudaError_t launch_backward_begin(const rtf_forest* f, void* ws, cudaStream_t st);
cudaError_t launch_backward_accumulate(const rtf_forest* f, const int32_t* dist_id,
                                       const int32_t* idx, const float* pos, const float* gpos,
                                       int64_t count, int mode, void* ws, cudaStream_t st);
cudaError_t launch_backward_finish(const rtf_forest* f, const float* w, int mode, float* grad_w,
                                   void* ws, cudaStream_t st);
cudaError_t launch_backward(const rtf_forest* f, const float* w, const uint32_t* u,
                            const int32_t* dist_id, const int32_t* idx, const float* pos,
                            const float* gpos, int64_t count, int mode, float* grad_w, void* ws,
                            cudaStream_t st);
}  // namespace rtf

namespace {

constexpr int64_t kMaxElems = (int64_t(1) << 31) - (int64_t(1) << 16);

bool aligned(const void* p, uintptr_t a) { return (reinterpret_cast<uintptr_t>(p) & (a - 1)) == 0; }

bool forest_ok(const rtf_forest* f) {
  return f && f->nodes && f->guide && f->dists && f->status && f->guide_recs &&
         aligned(f->guide_recs, 32) && f->num_dists >= 1 &&
         f->num_elems >= 1 && f->num_elems <= kMaxElems && f->num_cells >= 1 &&
         f->num_cells < (int64_t(1) << 31) &&
         f->max_m >= 0 && f->max_m <= 30 && aligned(f->nodes, 16) && aligned(f->status, 4);
}

rtf_status cuda_status(cudaError_t e) { return e == cudaSuccess ? RTF_OK : RTF_ECUDA; }

}  // namespace

extern "C" {

const char* rtf_version(void) { return "rtf 0.2.0 (sm_103a)"; }

const char* rtf_status_string(rtf_status s) {
  switch (s) {
    case RTF_OK:
      return "ok";
    case RTF_EINVAL:
      return "invalid argument";
    case RTF_EWORKSPACE:
      return "workspace too small";
    case RTF_ECUDA:
      return "CUDA error";
  }
  return "unknown status";
}

size_t rtf_build_workspace_size(int64_t num_elems, int32_t num_dists, int64_t num_cells) {
  if (num_elems < 1 || num_dists < 1 || num_cells < 1) return 0;
  return rtf::ws_layout(num_elems, num_dists, num_cells).total;
}

rtf_status rtf_build(const float* w, int64_t n, int32_t m, rtf_forest* f, void* ws,
                     size_t ws_bytes, void* stream) {
  if (!w || !ws || !forest_ok(f)) return RTF_EINVAL;
  if (n < 1 || n > kMaxElems || m < 0 || m > 30) return RTF_EINVAL;
  if (f->num_dists != 1 || f->num_elems != n || f->num_cells != (int64_t(1) << m) ||
      f->max_m != m || f->flags != 0)
    return RTF_EINVAL;
  if (!aligned(w, 4) || !aligned(ws, 256)) return RTF_EINVAL;
  if (ws_bytes < rtf_build_workspace_size(n, 1, int64_t(1) << m)) return RTF_EWORKSPACE;
  return cuda_status(rtf::launch_build(w, n, n, 1, 0, nullptr, nullptr, nullptr, n, m, f, ws,
                                       static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_build_batched(const float* w, const int64_t* offsets, const int32_t* m,
                             const int64_t* guide_offsets, rtf_forest* f, void* ws,
                             size_t ws_bytes, void* stream) {
  if (!w || !offsets || !m || !guide_offsets || !ws || !forest_ok(f)) return RTF_EINVAL;
  const int D = f->num_dists;
  const int marginal = (f->flags & RTF_FOREST_MARGINAL) ? 1 : 0;
  if (f->flags & ~RTF_FOREST_MARGINAL) return RTF_EINVAL;
  if (marginal && D < 2) return RTF_EINVAL;
  if (!aligned(w, 4) || !aligned(ws, 256) || !aligned(offsets, 8) || !aligned(guide_offsets, 8))
    return RTF_EINVAL;
  const int64_t N = f->num_elems;
  const int64_t Nw = marginal ? N - (D - 1) : N;
  if (Nw < D - marginal) return RTF_EINVAL;
  if (ws_bytes < rtf_build_workspace_size(N, D, f->num_cells)) return RTF_EWORKSPACE;
  return cuda_status(rtf::launch_build(w, N, Nw, D, marginal, offsets, m, guide_offsets, 0, 0, f,
                                       ws, static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_sample(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                      int64_t count, int32_t mode, int32_t* idx_out, float* pos_out,
                      void* stream) {
  if (!forest_ok(f) || count < 0) return RTF_EINVAL;
  if (count == 0) return RTF_OK;
  if (!u || !idx_out || !pos_out) return RTF_EINVAL;
  if (!aligned(u, 16) || !aligned(idx_out, 16) || !aligned(pos_out, 16)) return RTF_EINVAL;
  if (mode & ~(0xFF | RTF_SAMPLE_BSEARCH | RTF_SAMPLE_COHERENT)) return RTF_EINVAL;
  const int32_t base = mode & 0xFF;
  if (base == RTF_SAMPLE_2D) {
    if (!(f->flags & RTF_FOREST_MARGINAL) || dist_id) return RTF_EINVAL;
  } else if (base != RTF_SAMPLE_1D) {
    return RTF_EINVAL;
  }
  return cuda_status(rtf::launch_sample(f, u, dist_id, count, mode, idx_out, pos_out,
                                        static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_sample_pipelined(const rtf_forest* f, const uint32_t* u_host, uint32_t* u_dev,
                                const int32_t* dist_id_host, int32_t* dist_id_dev, int64_t count,
                                int32_t mode, int32_t* idx_dev, float* pos_dev,
                                int32_t* idx_host, float* pos_host, int64_t chunk,
                                void* done_event, void* stream) {
  if (!forest_ok(f) || count < 0 || chunk < 4 || (chunk & 3)) return RTF_EINVAL;
  if (mode & ~(0xFF | RTF_SAMPLE_BSEARCH | RTF_SAMPLE_COHERENT)) return RTF_EINVAL;
  const int32_t base = mode & 0xFF;
  if (base == RTF_SAMPLE_2D) {
    if (!(f->flags & RTF_FOREST_MARGINAL) || dist_id_dev || dist_id_host) return RTF_EINVAL;
  } else if (base != RTF_SAMPLE_1D) {
    return RTF_EINVAL;
  }
  if (count == 0) return RTF_OK;
  if (!u_dev || !idx_dev || !pos_dev) return RTF_EINVAL;
  if (!aligned(u_dev, 16) || !aligned(idx_dev, 16) || !aligned(pos_dev, 16)) return RTF_EINVAL;
  if (dist_id_host && !dist_id_dev) return RTF_EINVAL;
  if (dist_id_dev && !aligned(dist_id_dev, 4)) return RTF_EINVAL;
  return cuda_status(rtf::launch_sample_pipelined(
      f, u_host, u_dev, dist_id_host, dist_id_dev, count, mode, idx_dev, pos_dev, idx_host,
      pos_host, chunk, static_cast<cudaEvent_t>(done_event), static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_sample_loads(const rtf_forest* f, const uint32_t* u, const int32_t* dist_id,
                            int64_t count, int32_t mode, int32_t* loads_out, void* stream) {
  if (!forest_ok(f) || count < 0) return RTF_EINVAL;
  if (mode != RTF_SAMPLE_1D && mode != (RTF_SAMPLE_1D | RTF_SAMPLE_BSEARCH)) return RTF_EINVAL;
  if (count == 0) return RTF_OK;
  if (!u || !loads_out || !aligned(u, 4) || !aligned(loads_out, 4)) return RTF_EINVAL;
  if (dist_id && !aligned(dist_id, 4)) return RTF_EINVAL;
  return cuda_status(rtf::launch_sample_loads(f, u, dist_id, count, mode, loads_out,
                                              static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_build_quad(const rtf_forest* f, rtf_quad_rec* quad, void* stream) {
  if (!forest_ok(f) || !quad || !aligned(quad, 32)) return RTF_EINVAL;
  return cuda_status(rtf::launch_build_quad(f, quad, static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_sample_quad(const rtf_forest* f, const rtf_quad_rec* quad, const uint32_t* u,
                           const int32_t* dist_id, int64_t count, int32_t mode, int32_t* idx_out,
                           float* pos_out, int32_t* loads_out, void* stream) {
  if (!forest_ok(f) || !quad || !aligned(quad, 32) || count < 0) return RTF_EINVAL;
  if (mode & ~(0xFF | RTF_SAMPLE_COHERENT)) return RTF_EINVAL;
  const int32_t base = mode & 0xFF;
  if (base == RTF_SAMPLE_2D) {
    if (!(f->flags & RTF_FOREST_MARGINAL) || dist_id) return RTF_EINVAL;
  } else if (base != RTF_SAMPLE_1D) {
    return RTF_EINVAL;
  }
  if (count == 0) return RTF_OK;
  if (!u || !idx_out || !pos_out) return RTF_EINVAL;
  if (!aligned(u, 16) || !aligned(idx_out, 16) || !aligned(pos_out, 16)) return RTF_EINVAL;
  if (dist_id && !aligned(dist_id, 4)) return RTF_EINVAL;
  if (loads_out && !aligned(loads_out, 8)) return RTF_EINVAL;
  return cuda_status(rtf::launch_sample_quad(f, quad, u, dist_id, count, mode, idx_out, pos_out,
                                             loads_out, static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_set_launch_shape(const rtf_launch_shape* shape) {
  if (!shape) {
    rtf::set_launch_shape(nullptr);
    return RTF_OK;
  }
  const int32_t v[4] = {shape->single_large, shape->single, shape->tagged, shape->pairs};
  for (int k = 0; k < 4; ++k)
    if (v[k] < 0 || v[k] > 64) return RTF_EINVAL;
  rtf::set_launch_shape(v);
  return RTF_OK;
}

rtf_status rtf_get_launch_shape(rtf_launch_shape* shape) {
  if (!shape) return RTF_EINVAL;
  int32_t v[4];
  rtf::get_launch_shape(v);
  shape->single_large = v[0];
  shape->single = v[1];
  shape->tagged = v[2];
  shape->pairs = v[3];
  return RTF_OK;
}

rtf_status rtf_check_bounded_wait(uint32_t* status, uint64_t* scratch, void* stream) {
  if (!status || !scratch || !aligned(status, 4) || !aligned(scratch, 8)) return RTF_EINVAL;
  return cuda_status(rtf::launch_wait_probe(status, scratch, static_cast<cudaStream_t>(stream)));
}

size_t rtf_backward_workspace_size(int64_t num_elems, int32_t num_dists) {
  if (num_elems < 1 || num_dists < 1) return 0;
  return rtf::backward_ws_bytes(num_elems, num_dists);
}

rtf_status rtf_sample_backward(const rtf_forest* f, const float* w, const uint32_t* u,
                               const int32_t* dist_id, const int32_t* idx, const float* pos,
                               const float* grad_pos, int64_t count, int32_t mode,
                               float* grad_w, void* ws, size_t ws_bytes, void* stream) {
  if (!forest_ok(f) || !w || !grad_w || !ws || count < 0) return RTF_EINVAL;
  if (count > 0 && (!u || !idx || !pos || !grad_pos)) return RTF_EINVAL;
  if (mode == RTF_SAMPLE_2D) {
    if (!(f->flags & RTF_FOREST_MARGINAL) || dist_id) return RTF_EINVAL;
    if (count > 0 && (!aligned(u, 8) || !aligned(idx, 8) || !aligned(pos, 8) ||
                      !aligned(grad_pos, 8)))
      return RTF_EINVAL;
  } else if (mode != RTF_SAMPLE_1D) {
    return RTF_EINVAL;
  }
  if (!aligned(ws, 256)) return RTF_EINVAL;
  if (ws_bytes < rtf_backward_workspace_size(f->num_elems, f->num_dists)) return RTF_EWORKSPACE;
  return cuda_status(rtf::launch_backward(f, w, u, dist_id, idx, pos, grad_pos, count, mode,
                                          grad_w, ws, static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_backward_begin(const rtf_forest* f, void* ws, size_t ws_bytes, void* stream) {
  if (!forest_ok(f) || !ws || !aligned(ws, 256)) return RTF_EINVAL;
  if (ws_bytes < rtf_backward_workspace_size(f->num_elems, f->num_dists)) return RTF_EWORKSPACE;
  return cuda_status(rtf::launch_backward_begin(f, ws, static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_backward_accumulate(const rtf_forest* f, const int32_t* dist_id,
                                   const int32_t* idx, const float* pos, const float* grad_pos,
                                   int64_t count, int32_t mode, void* ws, size_t ws_bytes,
                                   void* stream) {
  if (!forest_ok(f) || !ws || !aligned(ws, 256) || count < 0) return RTF_EINVAL;
  if (count > 0 && (!idx || !pos || !grad_pos)) return RTF_EINVAL;
  if (mode == RTF_SAMPLE_2D) {
    if (!(f->flags & RTF_FOREST_MARGINAL) || dist_id) return RTF_EINVAL;
    if (count > 0 && (!aligned(idx, 8) || !aligned(pos, 8) || !aligned(grad_pos, 8)))
      return RTF_EINVAL;
  } else if (mode != RTF_SAMPLE_1D) {
    return RTF_EINVAL;
  }
  if (ws_bytes < rtf_backward_workspace_size(f->num_elems, f->num_dists)) return RTF_EWORKSPACE;
  return cuda_status(rtf::launch_backward_accumulate(f, dist_id, idx, pos, grad_pos, count, mode,
                                                     ws, static_cast<cudaStream_t>(stream)));
}

rtf_status rtf_backward_finish(const rtf_forest* f, const float* w, int32_t mode, float* grad_w,
                               void* ws, size_t ws_bytes, void* stream) {
  if (!forest_ok(f) || !w || !grad_w || !ws || !aligned(ws, 256)) return RTF_EINVAL;
  if (mode == RTF_SAMPLE_2D) {
    if (!(f->flags & RTF_FOREST_MARGINAL)) return RTF_EINVAL;
  } else if (mode != RTF_SAMPLE_1D) {
    return RTF_EINVAL;
  }
  if (ws_bytes < rtf_backward_workspace_size(f->num_elems, f->num_dists)) return RTF_EWORKSPACE;
  return cuda_status(
      rtf::launch_backward_finish(f, w, mode, grad_w, ws, static_cast<cudaStream_t>(stream)));
}

}  // extern "C"
