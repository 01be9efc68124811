// res2tac_compute_static: the pipeline of res2tac_compute on a fixed device array instead of a
// context's allocated scratch, for callers that must not allocate device memory while running
// (see include/res2tac.h). The paper has no counterpart.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <mutex>

#include "../../include/res2tac.h"
#include "launch.h"
#include "layout.h"

namespace {

// The scratch of every res2tac_compute_static call. Host code only sees a stand-in for it: the
// device address is looked up with cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_static_scratch[RES2TAC_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices];  // device address of g_static_scratch on each device

int reject(int code, const char* fmt, ...) {
  char msg[384];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(msg, sizeof(msg), fmt, ap);
  va_end(ap);
  return r2t::report_error(code, msg);
}

}  // namespace

extern "C" int res2tac_compute_static(const res2tac_params* p, const uint8_t* left,
                                      const uint8_t* right, int64_t in_pitch, uint16_t* disp,
                                      int64_t out_pitch, res2tac_stream_t s) {
  if (!p || res2tac_workspace_bytes(p) == 0)
    return reject(RES2TAC_EINVAL, "res2tac_compute_static: invalid parameters");
  if (!left || !right || !disp)
    return reject(RES2TAC_EINVAL, "res2tac_compute_static: NULL image or output pointer");
  if (in_pitch < p->width || out_pitch < 2 * (int64_t)p->width || (out_pitch & 1) ||
      (reinterpret_cast<uintptr_t>(disp) & 1))
    return reject(RES2TAC_EINVAL, "res2tac_compute_static: bad pitch or output alignment");
  const int W = p->width, H = p->height, D = p->max_disp;
  const bool wide = p->num_paths * (255 + p->p2) > 65535;
  // the same buffers a context allocates, at their offsets inside the array
  const r2t::Layout lay = r2t::layout_for(W, H, D, wide, (p->flags & RES2TAC_EXACT_CC) != 0,
                                          (p->flags & RES2TAC_NCC) != 0);
  if (lay.total > RES2TAC_STATIC_SCRATCH_BYTES)
    return reject(RES2TAC_ENOMEM,
                  "res2tac_compute_static: %dx%d with D=%d needs %zu bytes of scratch, more than "
                  "the fixed array of %zu bytes",
                  W, H, D, lay.total, (size_t)RES2TAC_STATIC_SCRATCH_BYTES);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return reject(RES2TAC_ECUDA, "res2tac_compute_static: cudaGetDevice: %s",
                  cudaGetErrorString(e));
  char* base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_setup_mu);
    if (!g_scratch_addr[dev]) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_static_scratch);
      if (e != cudaSuccess || !ptr) {
        cudaGetLastError();
        return reject(RES2TAC_ECUDA, "res2tac_compute_static: cudaGetSymbolAddress: %s",
                      cudaGetErrorString(e));
      }
      g_scratch_addr[dev] = ptr;
    }
    base = static_cast<char*>(g_scratch_addr[dev]);
  }
  // the aggregated volume and the right-disparity keys are reset by the cost stage of each call
  r2t::Problem pb = r2t::problem_at(base, lay, W, H, D);
  pb.left = left;
  pb.right = right;
  pb.in_pitch = in_pitch;
  pb.disp = disp;
  pb.out_pitch = out_pitch;
  r2t::Method mt;
  mt.cw = p->census_w;
  mt.ch = p->census_h;
  mt.P1 = p->p1;
  mt.P2 = p->p2;
  mt.num_paths = p->num_paths;
  mt.flags = p->flags;
  mt.lr_threshold = p->lr_threshold;
  mt.wide = wide ? 1 : 0;
  int launches = 0;
  e = r2t::run_pipeline(pb, mt, r2t::default_tuning(D), (cudaStream_t)s, &launches, nullptr);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return reject(RES2TAC_ECUDA, "res2tac_compute_static: launch failed: %s",
                  cudaGetErrorString(e));
  }
  return RES2TAC_OK;
}
