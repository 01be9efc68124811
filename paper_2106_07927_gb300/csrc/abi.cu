// C ABI of the SGM stereo library: context management, validation, scratch layout, dispatch.
#include <cuda_runtime.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/res2tac.h"
#include "../../include/res2tac_measure.h"
#include "batch.h"
#include "launch.h"
#include "layout.h"

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return code;
}

int fail_cuda(cudaError_t e, const char* what) {
  cudaGetLastError();  // clear a sticky launch error of this thread
  return fail(e == cudaErrorMemoryAllocation ? RES2TAC_ENOMEM : RES2TAC_ECUDA, "%s: %s (%s)", what,
              cudaGetErrorName(e), cudaGetErrorString(e));
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

bool shape_ok(int W, int H, int D) {
  return W >= 1 && W <= 16384 && H >= 1 && H <= 16384 && D >= 16 && D <= 256 && D % 16 == 0;
}

const char* params_error(const res2tac_params* p) {
  if (!p) return "params is NULL";
  if (!shape_ok(p->width, p->height, p->max_disp))
    return "need 1 <= width, height <= 16384 and 16 <= max_disp <= 256, max_disp % 16 == 0";
  if (p->flags & RES2TAC_NCC) {
    if (!((p->census_w == 5 && p->census_h == 5) || (p->census_w == 9 && p->census_h == 9)))
      return "NCC patch must be 5x5 or 9x9";
  } else if (!((p->census_w == 5 && p->census_h == 5) || (p->census_w == 9 && p->census_h == 7))) {
    return "census window must be 5x5 or 9x7";
  }
  if (p->p1 < 0 || p->p2 < p->p1 || p->p2 > 16384) return "need 0 <= p1 <= p2 <= 16384";
  if (p->num_paths != 4 && p->num_paths != 8) return "num_paths must be 4 or 8";
  if (p->flags & ~(RES2TAC_LR_CHECK | RES2TAC_MEDIAN | RES2TAC_EXACT_CC | RES2TAC_NCC))
    return "unknown flag bits";
  if (p->lr_threshold < 0 || p->lr_threshold > 255) return "lr_threshold must be in 0..255";
  return nullptr;
}

bool needs_wide(const res2tac_params* p) { return p->num_paths * (255 + p->p2) > 65535; }

using r2t::Layout;
using r2t::layout_for;
using r2t::problem_at;

r2t::Method method_of(const res2tac_params& p) {
  r2t::Method m;
  m.cw = p.census_w;
  m.ch = p.census_h;
  m.P1 = p.p1;
  m.P2 = p.p2;
  m.num_paths = p.num_paths;
  m.flags = p.flags;
  m.lr_threshold = p.lr_threshold;
  m.wide = needs_wide(&p) ? 1 : 0;
  return m;
}

}  // namespace

namespace r2t {
// Records msg as the calling thread's last error (read by res2tac_last_error) and returns code.
int report_error(int code, const char* msg) { return fail(code, "%s", msg); }
}  // namespace r2t

struct res2tac_ctx {
  res2tac_params p;
  r2t::Method method;
  r2t::Tuning tuning;
  int device;
  Layout lay;
  char* scratch;       // per-pair scratch of the context's own shape
  uint8_t* stage_in;   // device staging of res2tac_compute_host: left, right (pitch W)
  uint16_t* stage_out; // device staging of the output map (pitch 2W bytes)
  float* maps;         // rectification maps mapx_l, mapy_l, mapx_r, mapy_r (W x H each), or NULL
  int raw_w, raw_h;    // raw image size the maps sample
  int last_launches;
  r2t::BatchEngine* batch;
  int profiling;
  cudaEvent_t ev[8];  // stage boundaries of the last profiled compute (8 with the exact check)
  r2t::Fork fork;     // second stream for the concurrent aggregation kernels
};


extern "C" {

const char* res2tac_strerror(int code) {
  switch (code) {
    case RES2TAC_OK: return "ok";
    case RES2TAC_EINVAL: return "invalid argument";
    case RES2TAC_ENOMEM: return "out of device memory";
    case RES2TAC_ECUDA: return "CUDA error";
    case RES2TAC_ETIMEOUT: return "device-side wait timed out";
    default: return "unknown error";
  }
}

const char* res2tac_last_error(void) { return g_err; }

size_t res2tac_workspace_bytes(const res2tac_params* p) {
  if (params_error(p)) return 0;
  const size_t npx = (size_t)p->width * p->height;
  return layout_for(p->width, p->height, p->max_disp, needs_wide(p),
                    (p->flags & RES2TAC_EXACT_CC) != 0, (p->flags & RES2TAC_NCC) != 0).total +
         npx * 2 + npx * 2 + 1024;
}

int res2tac_create(const res2tac_params* p, res2tac_t* out) {
  if (!out) return fail(RES2TAC_EINVAL, "out is NULL");
  *out = nullptr;
  if (const char* why = params_error(p)) return fail(RES2TAC_EINVAL, "res2tac_create: %s", why);
  res2tac_ctx* h = new (std::nothrow) res2tac_ctx;
  if (!h) return fail(RES2TAC_ENOMEM, "host allocation failed");
  memset(h, 0, sizeof(*h));
  h->p = *p;
  h->method = method_of(*p);
  h->tuning = r2t::default_tuning(p->max_disp);
  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    delete h;
    return fail_cuda(e, "cudaGetDevice");
  }
  h->lay = layout_for(p->width, p->height, p->max_disp, h->method.wide != 0,
                      (p->flags & RES2TAC_EXACT_CC) != 0, (p->flags & RES2TAC_NCC) != 0);
  const size_t npx = (size_t)p->width * p->height;
  e = cudaMalloc(&h->scratch, h->lay.total);
  if (e == cudaSuccess) e = cudaMemset(h->scratch + h->lay.fault, 0, 16);  // range-check record
  if (e == cudaSuccess) e = cudaMalloc(&h->stage_in, align_up(npx * 2, 256));
  if (e == cudaSuccess) e = cudaMalloc(&h->stage_out, align_up(npx * 2, 256));
  if (e == cudaSuccess) e = r2t::fork_create(&h->fork);
  if (e != cudaSuccess) {
    int rc = fail_cuda(e, "cudaMalloc of the context scratch");
    res2tac_destroy(h);
    return rc;
  }
  *out = h;
  return RES2TAC_OK;
}

void res2tac_destroy(res2tac_t h) {
  if (!h) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  r2t::batch_destroy(h->batch);
  r2t::fork_destroy(&h->fork);
  for (int i = 0; i < 8; i++)
    if (h->ev[i]) cudaEventDestroy(h->ev[i]);
  cudaFree(h->scratch);
  cudaFree(h->stage_in);
  cudaFree(h->stage_out);
  cudaFree(h->maps);
  if (cur >= 0 && cur != h->device) cudaSetDevice(cur);
  delete h;
}

static int check_io(res2tac_t h, const void* left, const void* right, int64_t in_pitch,
                    const void* disp, int64_t out_pitch) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
  if (!left || !right || !disp) return fail(RES2TAC_EINVAL, "NULL image or output pointer");
  if (in_pitch < h->p.width) return fail(RES2TAC_EINVAL, "in_pitch < width");
  if (out_pitch < 2 * (int64_t)h->p.width || (out_pitch & 1))
    return fail(RES2TAC_EINVAL, "out_pitch must be even and >= 2 * width");
  if ((reinterpret_cast<uintptr_t>(disp) & 1) != 0)
    return fail(RES2TAC_EINVAL, "disp must be 2-byte aligned");
  return RES2TAC_OK;
}

int res2tac_compute(res2tac_t h, const uint8_t* left, const uint8_t* right, int64_t in_pitch,
                    uint16_t* disp, int64_t out_pitch, res2tac_stream_t s) {
  int rc = check_io(h, left, right, in_pitch, disp, out_pitch);
  if (rc) return rc;
  r2t::Problem pb = problem_at(h->scratch, h->lay, h->p.width, h->p.height, h->p.max_disp);
  pb.left = left;
  pb.right = right;
  pb.in_pitch = in_pitch;
  pb.disp = disp;
  pb.out_pitch = out_pitch;
  int n = 0;
  cudaError_t e = r2t::run_pipeline(pb, h->method, h->tuning, (cudaStream_t)s, &n,
                                    h->profiling ? h->ev : nullptr, &h->fork);
  h->last_launches = n;
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_compute launch");
  return RES2TAC_OK;
}

// Device address of a host buffer the GPU can read and write in place (pinned, mapped host
// memory: over NVLink-C2C on a Grace system), or NULL for memory that needs a copy.
static void* device_alias(const void* host) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int res2tac_compute_host(res2tac_t h, const uint8_t* left, const uint8_t* right,
                         int64_t in_pitch, uint16_t* disp, int64_t out_pitch,
                         res2tac_stream_t s) {
  int rc = check_io(h, left, right, in_pitch, disp, out_pitch);
  if (rc) return rc;
  const int W = h->p.width, H = h->p.height;
  cudaStream_t st = (cudaStream_t)s;
  {
    // pinned host buffers: the kernels read the images and write the map in place, so the
    // transfers overlap the computation instead of running as separate copies
    const void* al = device_alias(left);
    const void* ar = device_alias(right);
    void* ad = device_alias(disp);
    if (al && ar && ad) {
      rc = res2tac_compute(h, static_cast<const uint8_t*>(al), static_cast<const uint8_t*>(ar),
                           in_pitch, static_cast<uint16_t*>(ad), out_pitch, s);
      if (rc) return rc;
      cudaError_t e = cudaStreamSynchronize(st);
      if (e != cudaSuccess) return fail_cuda(e, "res2tac_compute_host");
      return RES2TAC_OK;
    }
  }
  uint8_t* dl = h->stage_in;
  uint8_t* dr = h->stage_in + (size_t)W * H;
  cudaError_t e = cudaMemcpy2DAsync(dl, W, left, in_pitch, W, H, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpy2DAsync(dr, W, right, in_pitch, W, H, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_compute_host upload");
  rc = res2tac_compute(h, dl, dr, W, h->stage_out, 2 * (int64_t)W, s);
  if (rc) return rc;
  e = cudaMemcpy2DAsync(disp, out_pitch, h->stage_out, 2 * (size_t)W, 2 * (size_t)W, H,
                        cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_compute_host download");
  return RES2TAC_OK;
}

int res2tac_rectify(const uint8_t* raw, int64_t raw_pitch, int32_t raw_w, int32_t raw_h,
                    const float* mapx, const float* mapy, int64_t map_pitch, uint8_t* out,
                    int64_t out_pitch, int32_t width, int32_t height, res2tac_stream_t s) {
  if (!raw || !mapx || !mapy || !out) return fail(RES2TAC_EINVAL, "NULL pointer");
  if (raw_w < 1 || raw_h < 1 || width < 1 || height < 1 || raw_w > 65536 || raw_h > 65536 ||
      width > 65536 || height > 65536)
    return fail(RES2TAC_EINVAL, "image sizes must be 1 .. 65536");
  if (raw_pitch < raw_w || out_pitch < width || map_pitch < 4 * (int64_t)width || (map_pitch & 3) ||
      (reinterpret_cast<uintptr_t>(mapx) & 3) || (reinterpret_cast<uintptr_t>(mapy) & 3))
    return fail(RES2TAC_EINVAL, "bad pitch or map alignment");
  r2t::RectifyJob j{raw, raw_pitch, raw_w, raw_h, mapx, mapy, map_pitch, out, out_pitch, width,
                    height};
  cudaError_t e = r2t::launch_rectify(&j, 1, (cudaStream_t)s);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_rectify launch");
  return RES2TAC_OK;
}

int res2tac_set_rectification(res2tac_t h, const float* mapx_l, const float* mapy_l,
                              const float* mapx_r, const float* mapy_r, int64_t map_pitch,
                              int32_t raw_w, int32_t raw_h, res2tac_stream_t s) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
  if (!mapx_l || !mapy_l || !mapx_r || !mapy_r) return fail(RES2TAC_EINVAL, "NULL map");
  const int W = h->p.width, H = h->p.height;
  if (raw_w < 1 || raw_h < 1 || raw_w > 65536 || raw_h > 65536)
    return fail(RES2TAC_EINVAL, "raw size must be 1 .. 65536");
  if (map_pitch < 4 * (int64_t)W || (map_pitch & 3)) return fail(RES2TAC_EINVAL, "bad map pitch");
  const size_t plane = (size_t)W * H * 4;
  if (!h->maps) {
    cudaError_t e = cudaMalloc(&h->maps, 4 * plane);
    if (e != cudaSuccess) {
      h->maps = nullptr;
      cudaGetLastError();
      return fail(RES2TAC_ENOMEM, "rectification maps of %zu bytes could not be allocated",
                  4 * plane);
    }
  }
  const float* src[4] = {mapx_l, mapy_l, mapx_r, mapy_r};
  for (int i = 0; i < 4; i++) {
    cudaError_t e = cudaMemcpy2DAsync(reinterpret_cast<uint8_t*>(h->maps) + i * plane, 4 * (size_t)W,
                                      src[i], (size_t)map_pitch, 4 * (size_t)W, H,
                                      cudaMemcpyDeviceToDevice, (cudaStream_t)s);
    if (e != cudaSuccess) return fail_cuda(e, "res2tac_set_rectification copy");
  }
  h->raw_w = raw_w;
  h->raw_h = raw_h;
  return RES2TAC_OK;
}

int res2tac_compute_raw(res2tac_t h, const uint8_t* raw_left, const uint8_t* raw_right,
                        int64_t raw_pitch, uint16_t* disp, int64_t out_pitch,
                        res2tac_stream_t s) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
  if (!h->maps) return fail(RES2TAC_EINVAL, "no rectification maps: call res2tac_set_rectification");
  if (!raw_left || !raw_right) return fail(RES2TAC_EINVAL, "NULL raw image");
  if (raw_pitch < h->raw_w) return fail(RES2TAC_EINVAL, "raw_pitch < raw width");
  const int W = h->p.width, H = h->p.height;
  const size_t plane = (size_t)W * H;
  const float* m = h->maps;
  r2t::RectifyJob j[2] = {
      {raw_left, raw_pitch, h->raw_w, h->raw_h, m, m + plane, 4 * (int64_t)W, h->stage_in, W, W,
       H},
      {raw_right, raw_pitch, h->raw_w, h->raw_h, m + 2 * plane, m + 3 * plane, 4 * (int64_t)W,
       h->stage_in + plane, W, W, H}};
  cudaError_t e = r2t::launch_rectify(j, 2, (cudaStream_t)s);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_compute_raw rectification");
  int rc = res2tac_compute(h, h->stage_in, h->stage_in + plane, W, disp, out_pitch, s);
  if (rc == RES2TAC_OK) h->last_launches += 1;
  return rc;
}

int res2tac_compute_subpixel(res2tac_t h, const uint8_t* left, const uint8_t* right,
                             int64_t in_pitch, float* disp, int64_t out_pitch,
                             res2tac_stream_t s) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
  if (!left || !right || !disp) return fail(RES2TAC_EINVAL, "NULL image or output pointer");
  if (in_pitch < h->p.width) return fail(RES2TAC_EINVAL, "in_pitch < width");
  if (out_pitch < 4 * (int64_t)h->p.width || (out_pitch & 3))
    return fail(RES2TAC_EINVAL, "out_pitch must be a multiple of 4 and >= 4 * width");
  if ((reinterpret_cast<uintptr_t>(disp) & 3) != 0)
    return fail(RES2TAC_EINVAL, "disp must be 4-byte aligned");
  r2t::Problem pb = problem_at(h->scratch, h->lay, h->p.width, h->p.height, h->p.max_disp);
  pb.left = left;
  pb.right = right;
  pb.in_pitch = in_pitch;
  pb.disp = nullptr;
  pb.disp_f = disp;
  pb.out_pitch = out_pitch;
  int n = 0;
  cudaError_t e = r2t::run_pipeline(pb, h->method, h->tuning, (cudaStream_t)s, &n,
                                    h->profiling ? h->ev : nullptr, &h->fork);
  h->last_launches = n;
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_compute_subpixel launch");
  return RES2TAC_OK;
}

int res2tac_debug_subpixel(res2tac_t h, float* dl_sub, res2tac_stream_t s) {
  if (!h || !dl_sub) return fail(RES2TAC_EINVAL, "NULL argument");
  r2t::Problem pb = problem_at(h->scratch, h->lay, h->p.width, h->p.height, h->p.max_disp);
  cudaError_t e = r2t::copy_subpixel(pb, h->method.wide != 0, dl_sub, (cudaStream_t)s);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_debug_subpixel");
  return RES2TAC_OK;
}

int res2tac_debug_outputs(res2tac_t h, uint8_t* cost, uint16_t* agg, uint16_t* dl, uint16_t* dr,
                          uint8_t* mask, res2tac_stream_t s) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
  r2t::Problem pb = problem_at(h->scratch, h->lay, h->p.width, h->p.height, h->p.max_disp);
  cudaStream_t st = (cudaStream_t)s;
  const size_t npx = (size_t)pb.W * pb.H;
  cudaError_t e = cudaSuccess;
  if (cost && e == cudaSuccess) e = r2t::copy_cost(pb, cost, st);
  if (agg && e == cudaSuccess) e = r2t::copy_agg_u16(pb, h->method.wide != 0, agg, st);
  if (dl && e == cudaSuccess) e = cudaMemcpyAsync(dl, pb.dl, npx * 2, cudaMemcpyDeviceToDevice, st);
  if (dr && e == cudaSuccess) e = cudaMemcpyAsync(dr, pb.dr, npx * 2, cudaMemcpyDeviceToDevice, st);
  if (mask && e == cudaSuccess) e = cudaMemcpyAsync(mask, pb.mask, npx, cudaMemcpyDeviceToDevice, st);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_debug_outputs");
  return RES2TAC_OK;
}

int res2tac_get_tuning(res2tac_t h, res2tac_tuning* t) {
  if (!h || !t) return fail(RES2TAC_EINVAL, "NULL argument");
  t->agg_dpl = h->tuning.agg_dpl;
  t->agg_warps = h->tuning.agg_warps;
  t->wta_chunk = h->tuning.wta_chunk;
  t->shear_dpl = h->tuning.shear_dpl;
  t->row_mode = h->tuning.row_split ? 2 : 1;
  t->shear_cpl = h->tuning.shear_cpl;
  t->cost_mode = h->tuning.cost_mode + 1;
  t->row_cost = h->tuning.row_cost + 1;
  return RES2TAC_OK;
}

int res2tac_set_tuning(res2tac_t h, const res2tac_tuning* t) {
  if (!h || !t) return fail(RES2TAC_EINVAL, "NULL argument");
  r2t::Tuning n = r2t::default_tuning(h->p.max_disp);
  if (t->agg_dpl) n.agg_dpl = t->agg_dpl;
  if (t->agg_warps) n.agg_warps = t->agg_warps;
  if (t->wta_chunk) n.wta_chunk = t->wta_chunk;
  if (t->shear_dpl) n.shear_dpl = t->shear_dpl;
  if (t->row_mode) n.row_split = t->row_mode == 2 ? 1 : (t->row_mode == 1 ? 0 : -1);
  if (t->shear_cpl) n.shear_cpl = t->shear_cpl;
  if (t->cost_mode) n.cost_mode = t->cost_mode - 1;
  if (t->row_cost) n.row_cost = t->row_cost - 1;
  if (!r2t::tuning_valid(n, h->p.max_disp))
    return fail(RES2TAC_EINVAL,
                "tuning (dpl %d, warps %d, chunk %d, shear dpl %d, row mode %d, shear cpl %d, "
                "cost mode %d) invalid for D = %d",
                n.agg_dpl, n.agg_warps, n.wta_chunk, n.shear_dpl, t->row_mode, n.shear_cpl,
                t->cost_mode, h->p.max_disp);
  h->tuning = n;
  return RES2TAC_OK;
}

int res2tac_autotune(res2tac_t h, const uint8_t* left, const uint8_t* right, int64_t in_pitch,
                     uint16_t* disp, int64_t out_pitch, res2tac_stream_t s,
                     res2tac_tuning* best) {
  int rc = check_io(h, left, right, in_pitch, disp, out_pitch);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)s;
  std::vector<r2t::Tuning> cands;
  const int dpls[3] = {2, 4, 8}, warps[3] = {2, 4, 8}, chunks[3] = {64, 128, 256};
  const int sdpls[3] = {8, 16, 32};
  for (int a : dpls)
    for (int w : warps)
      for (int c : chunks)
        for (int sd : sdpls)
          for (int split = 0; split < 2; split++)
            for (int cpl = 1; cpl <= 2; cpl++) {
              r2t::Tuning t{a, w, c, sd, split, cpl, 0, 0};
              if (r2t::tuning_valid(t, h->p.max_disp)) cands.push_back(t);
            }
  if (cands.empty()) return fail(RES2TAC_EINVAL, "no valid tuning");
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(RES2TAC_ECUDA, "cudaEventCreate failed");
  const r2t::Tuning keep = h->tuning;
  float best_ms = 1e30f;
  r2t::Tuning best_t = keep;
  // times t (two warm-up calls, then 5 calls) and keeps it when it is the fastest so far
  auto try_tuning = [&](const r2t::Tuning& t) {
    h->tuning = t;
    for (int rep = 0; rep < 2 && !rc; rep++)  // warm-up
      rc = res2tac_compute(h, left, right, in_pitch, disp, out_pitch, s);
    if (rc) return;
    cudaEventRecord(e0, st);
    const int reps = 5;
    for (int rep = 0; rep < reps && !rc; rep++)
      rc = res2tac_compute(h, left, right, in_pitch, disp, out_pitch, s);
    cudaEventRecord(e1, st);
    if (rc) return;
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      rc = fail(RES2TAC_ECUDA, "autotune synchronisation failed");
      return;
    }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) {
      best_ms = ms;
      best_t = t;
    }
  };
  for (const r2t::Tuning& t : cands) {
    try_tuning(t);
    if (rc) break;
  }
  r2t::Problem shape{};
  shape.D = h->p.max_disp;
  if (!rc && r2t::cost_mma_ok(shape, h->method)) {  // the other cost kernel with the best setting
    r2t::Tuning t = best_t;
    t.cost_mode = 1 - t.cost_mode;
    try_tuning(t);
  }
  {  // the row kernel recomputing its costs, with the best setting so far
    r2t::Tuning t = best_t;
    t.row_cost = 1;
    if (!rc && r2t::rows_recompute_ok(shape, h->method, t)) try_tuning(t);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->tuning = rc ? keep : best_t;
  if (rc) return rc;
  if (best) res2tac_get_tuning(h, best);
  return RES2TAC_OK;
}

int res2tac_last_launch_count(res2tac_t h) { return h ? h->last_launches : 0; }

int res2tac_set_profiling(res2tac_t h, int enable) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
  if (enable && !h->ev[0]) {
    for (int i = 0; i < 8; i++) {
      cudaError_t e = cudaEventCreate(&h->ev[i]);
      if (e != cudaSuccess) return fail_cuda(e, "cudaEventCreate");
    }
  }
  h->profiling = enable ? 1 : 0;
  return RES2TAC_OK;
}

int res2tac_stage_times(res2tac_t h, float* ms, int n) {
  if (!h || !ms || n < 0) return fail(RES2TAC_EINVAL, "NULL argument");
  if (!h->profiling || !h->ev[0]) return fail(RES2TAC_EINVAL, "profiling is not enabled");
  const bool exact = (h->method.flags & RES2TAC_EXACT_CC) != 0;
  cudaError_t e = cudaEventSynchronize(h->ev[exact ? 7 : 4]);
  if (e != cudaSuccess) return fail_cuda(e, "cudaEventSynchronize");
  // event intervals of each stage; with the exact check a stage runs once per pass (the flip
  // counts to the first cost stage)
  static const int kPlain[4][4] = {{0, 1, -1, -1}, {1, 2, -1, -1}, {2, 3, -1, -1}, {3, 4, -1, -1}};
  static const int kExact[4][4] = {{0, 1, 3, 4}, {1, 2, 4, 5}, {2, 3, 5, 6}, {6, 7, -1, -1}};
  const int(*iv)[4] = exact ? kExact : kPlain;
  for (int i = 0; i < n && i < 4; i++) {
    ms[i] = 0;
    for (int k = 0; k < 4 && iv[i][k] >= 0; k += 2) {
      float t = 0;
      e = cudaEventElapsedTime(&t, h->ev[iv[i][k]], h->ev[iv[i][k + 1]]);
      if (e != cudaSuccess) return fail_cuda(e, "cudaEventElapsedTime");
      ms[i] += t;
    }
  }
  return RES2TAC_OK;
}

int res2tac_probe_red_peak(int64_t bytes, int32_t passes, res2tac_stream_t s, double* bytes_per_s) {
  if (bytes < 1024 || passes < 1 || !bytes_per_s) return fail(RES2TAC_EINVAL, "bad probe arguments");
  cudaError_t e = r2t::probe_red_peak(bytes, passes, (cudaStream_t)s, bytes_per_s);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_probe_red_peak");
  return RES2TAC_OK;
}

int res2tac_probe_popc_rate(int iters, res2tac_stream_t s, double* popc_per_s) {
  if (iters < 1 || !popc_per_s) return fail(RES2TAC_EINVAL, "bad probe arguments");
  cudaError_t e = r2t::probe_popc_rate(iters, (cudaStream_t)s, popc_per_s);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_probe_popc_rate");
  return RES2TAC_OK;
}

int res2tac_probe_int_peak(int iters, res2tac_stream_t s, double* lane_ops_per_s) {
  if (iters < 1 || !lane_ops_per_s) return fail(RES2TAC_EINVAL, "bad probe arguments");
  cudaError_t e = r2t::probe_int_peak(iters, (cudaStream_t)s, lane_ops_per_s);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_probe_int_peak");
  return RES2TAC_OK;
}

size_t res2tac_batch_workspace_bytes(const res2tac_params* p, const res2tac_pair* pairs,
                                     int32_t n) {
  if (params_error(p) || !pairs || n < 1) return 0;
  const bool wide = needs_wide(p);
  size_t total = 0;
  for (int i = 0; i < n; i++) {
    if (!shape_ok(pairs[i].width, pairs[i].height, pairs[i].max_disp)) return 0;
    total += layout_for(pairs[i].width, pairs[i].height, pairs[i].max_disp, wide).total;
  }
  return total + r2t::batch_fixed_bytes(n);
}

int res2tac_batch_reserve(res2tac_t h, size_t scratch_bytes, int32_t max_pairs) {
  if (!h || max_pairs < 1) return fail(RES2TAC_EINVAL, "bad batch reservation");
  int rc = r2t::batch_reserve(&h->batch, scratch_bytes, max_pairs);
  if (rc == -2) return fail(RES2TAC_ENOMEM, "batch reservation of %zu bytes failed", scratch_bytes);
  if (rc) return fail(RES2TAC_ECUDA, "batch reservation: %s", r2t::batch_error(h->batch));
  return RES2TAC_OK;
}

int res2tac_compute_batch(res2tac_t h, const res2tac_pair* pairs, int32_t n, res2tac_stream_t s) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
  if (!pairs || n < 1) return fail(RES2TAC_EINVAL, "empty batch");
  if (h->method.flags & (RES2TAC_EXACT_CC | RES2TAC_NCC))
    return fail(RES2TAC_EINVAL,
                "the exact consistency check and the NCC cost run per pair (res2tac_compute)");
  std::vector<r2t::Problem> probs((size_t)n);
  std::vector<size_t> offs((size_t)n);
  size_t total = 0;
  const bool wide = h->method.wide != 0;
  for (int i = 0; i < n; i++) {
    const res2tac_pair& q = pairs[i];
    if (!shape_ok(q.width, q.height, q.max_disp))
      return fail(RES2TAC_EINVAL, "pair %d: invalid shape %dx%d D=%d", i, q.width, q.height,
                  q.max_disp);
    if (!q.left || !q.right || !q.disp) return fail(RES2TAC_EINVAL, "pair %d: NULL pointer", i);
    if (q.in_pitch < q.width || q.out_pitch < 2 * (int64_t)q.width || (q.out_pitch & 1))
      return fail(RES2TAC_EINVAL, "pair %d: bad pitch", i);
    offs[i] = total;
    total += layout_for(q.width, q.height, q.max_disp, wide).total;
  }
  int rc = r2t::batch_reserve(&h->batch, total, n);
  if (rc == -2) return fail(RES2TAC_ENOMEM, "batch scratch of %zu bytes could not be allocated", total);
  if (rc) return fail(RES2TAC_ECUDA, "batch engine setup failed: %s", r2t::batch_error(h->batch));
  char* base = r2t::batch_scratch(h->batch);
  for (int i = 0; i < n; i++) {
    const res2tac_pair& q = pairs[i];
    Layout l = layout_for(q.width, q.height, q.max_disp, wide);
    r2t::Problem pb = problem_at(base + offs[i], l, q.width, q.height, q.max_disp);
    pb.left = q.left;
    pb.right = q.right;
    pb.in_pitch = q.in_pitch;
    pb.disp = q.disp;
    pb.out_pitch = q.out_pitch;
    probs[i] = pb;
  }
  int launches = 0;
  rc = r2t::batch_run(h->batch, probs.data(), n, h->method, (cudaStream_t)s, &launches);
  h->last_launches = launches;
  if (rc == -4) return fail(RES2TAC_ETIMEOUT, "batch work queue wait timed out");
  if (rc) return fail(RES2TAC_ECUDA, "batch run failed: %s", r2t::batch_error(h->batch));
  return RES2TAC_OK;
}

static int bucket_of(const res2tac_batch_tuning* t) {
  if (!t || t->max_disp < 16 || t->max_disp > 256 || t->max_disp % 16 || (t->large & ~1)) return -1;
  return 2 * (t->max_disp / 16) + t->large;
}

static int ensure_engine(res2tac_t h) {
  if (h->batch) return RES2TAC_OK;
  int rc = r2t::batch_reserve(&h->batch, 0, 1);
  if (rc == -2) return fail(RES2TAC_ENOMEM, "batch engine setup: out of memory");
  if (rc) return fail(RES2TAC_ECUDA, "batch engine setup failed: %s", r2t::batch_error(h->batch));
  return RES2TAC_OK;
}

int res2tac_set_batch_tuning(res2tac_t h, const res2tac_batch_tuning* t, int32_t n) {
  if (!h || !t || n < 0) return fail(RES2TAC_EINVAL, "NULL argument");
  for (int i = 0; i < n; i++) {
    const int b = bucket_of(&t[i]);
    r2t::BatchTune v;
    memset(&v, 0, sizeof(v));
    v.row_dpl = (signed char)t[i].row_dpl;
    v.shear_dpl = (signed char)t[i].shear_dpl;
    v.shear_cpl = (signed char)t[i].shear_cpl;
    v.wta_px = (short)t[i].wta_px;
    if (b < 0 || t[i].row_dpl != v.row_dpl || t[i].shear_dpl != v.shear_dpl ||
        t[i].shear_cpl != v.shear_cpl || t[i].wta_px != v.wta_px || !r2t::batch_tune_valid(b, v))
      return fail(RES2TAC_EINVAL,
                  "batch tuning %d (D %d, large %d: row dpl %d, shear %d x %d, wta %d) invalid", i,
                  t[i].max_disp, t[i].large, t[i].row_dpl, t[i].shear_dpl, t[i].shear_cpl,
                  t[i].wta_px);
  }
  int rc = ensure_engine(h);
  if (rc) return rc;
  for (int i = 0; i < n; i++) {
    r2t::BatchTune v;
    memset(&v, 0, sizeof(v));
    v.row_dpl = (signed char)t[i].row_dpl;
    v.shear_dpl = (signed char)t[i].shear_dpl;
    v.shear_cpl = (signed char)t[i].shear_cpl;
    v.wta_px = (short)t[i].wta_px;
    r2t::batch_set_tune(h->batch, bucket_of(&t[i]), v);
  }
  return RES2TAC_OK;
}

int res2tac_get_batch_tuning(res2tac_t h, res2tac_batch_tuning* t) {
  if (!h || !t) return fail(RES2TAC_EINVAL, "NULL argument");
  const int b = bucket_of(t);
  if (b < 0) return fail(RES2TAC_EINVAL, "bucket D %d large %d invalid", t->max_disp, t->large);
  const r2t::BatchTune v = r2t::batch_get_tune(h->batch, b);
  t->row_dpl = v.row_dpl;
  t->shear_dpl = v.shear_dpl;
  t->shear_cpl = v.shear_cpl;
  t->wta_px = v.wta_px;
  return RES2TAC_OK;
}

// Median time of 3 batch runs after one warm-up (ms), or a negative RES2TAC code.
static float time_batch(res2tac_t h, const res2tac_pair* pairs, int32_t n, cudaStream_t st,
                        cudaEvent_t e0, cudaEvent_t e1, int* rc) {
  *rc = res2tac_compute_batch(h, pairs, n, st);
  if (*rc) return -1.0f;
  float ms[3];
  for (int r = 0; r < 3; r++) {
    cudaEventRecord(e0, st);
    *rc = res2tac_compute_batch(h, pairs, n, st);
    if (*rc) return -1.0f;
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess) {
      *rc = fail(RES2TAC_ECUDA, "autotune synchronisation failed");
      return -1.0f;
    }
    cudaEventElapsedTime(&ms[r], e0, e1);
  }
  std::sort(ms, ms + 3);
  return ms[1];
}

int res2tac_autotune_batch(res2tac_t h, const res2tac_pair* pairs, int32_t n, res2tac_stream_t s,
                           res2tac_batch_tuning* table, int32_t cap, int32_t* count,
                           float* ms_default, float* ms_tuned) {
  if (!h || !pairs || n < 1) return fail(RES2TAC_EINVAL, "empty batch");
  cudaStream_t st = (cudaStream_t)s;
  // buckets present, by their total work
  std::vector<std::pair<double, int>> work;
  for (int i = 0; i < n; i++) {
    if (!shape_ok(pairs[i].width, pairs[i].height, pairs[i].max_disp))
      return fail(RES2TAC_EINVAL, "pair %d: invalid shape", i);
    const int b = r2t::tune_bucket(pairs[i].width, pairs[i].height, pairs[i].max_disp);
    const double de = (double)pairs[i].width * pairs[i].height * pairs[i].max_disp;
    bool found = false;
    for (auto& w : work)
      if (w.second == b) {
        w.first += de;
        found = true;
      }
    if (!found) work.push_back({de, b});
  }
  std::sort(work.begin(), work.end(), [](const auto& a, const auto& b) { return a.first > b.first; });
  int rc = ensure_engine(h);
  if (rc) return rc;
  for (const auto& w : work) r2t::batch_set_tune(h->batch, w.second, r2t::batch_default_tune(w.second));
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(RES2TAC_ECUDA, "cudaEventCreate failed");
  float best = time_batch(h, pairs, n, st, e0, e1, &rc);
  const float first = best;
  const int rows[3] = {2, 4, 8}, sdpl[2] = {16, 16}, scpl[2] = {1, 2};
  const int wpx[3] = {64, 128, 256};
  for (size_t wi = 0; wi < work.size() && !rc; wi++) {
    const int b = work[wi].second;
    for (int param = 0; param < 3 && !rc; param++) {
      const int ncand = param == 1 ? 2 : 3;
      r2t::BatchTune keep = r2t::batch_get_tune(h->batch, b);
      for (int c = 0; c < ncand && !rc; c++) {
        r2t::BatchTune t = keep;
        if (param == 0) t.row_dpl = (signed char)rows[c];
        if (param == 1) {
          t.shear_dpl = (signed char)sdpl[c];
          t.shear_cpl = (signed char)scpl[c];
        }
        if (param == 2) t.wta_px = (short)wpx[c];
        if (memcmp(&t, &keep, sizeof(t)) == 0 || !r2t::batch_tune_valid(b, t)) continue;
        const r2t::BatchTune prev = r2t::batch_get_tune(h->batch, b);
        r2t::batch_set_tune(h->batch, b, t);
        const float ms = time_batch(h, pairs, n, st, e0, e1, &rc);
        if (!rc && ms < best) {
          best = ms;
        } else {
          r2t::batch_set_tune(h->batch, b, prev);
        }
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  int k = 0;
  for (size_t wi = 0; wi < work.size() && table && k < cap; wi++, k++) {
    const int b = work[wi].second;
    const r2t::BatchTune v = r2t::batch_get_tune(h->batch, b);
    table[k].max_disp = 16 * (b / 2);
    table[k].large = b & 1;
    table[k].row_dpl = v.row_dpl;
    table[k].shear_dpl = v.shear_dpl;
    table[k].shear_cpl = v.shear_cpl;
    table[k].wta_px = v.wta_px;
  }
  if (count) *count = k;
  if (ms_default) *ms_default = first;
  if (ms_tuned) *ms_tuned = best;
  return RES2TAC_OK;
}

int res2tac_bounds_status(res2tac_t h, int32_t* checked, int32_t* site, int64_t* offset) {
  if (!h) return fail(RES2TAC_EINVAL, "handle is NULL");
#ifdef RES2TAC_CHECK_BOUNDS
  const int on = 1;
#else
  const int on = 0;
#endif
  long long rec[2] = {0, 0};
  cudaError_t e = cudaMemcpy(rec, h->scratch + h->lay.fault, 16, cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return fail_cuda(e, "res2tac_bounds_status");
  if (checked) *checked = on;
  if (site) *site = (int32_t)(rec[0] & 0xFFFFFFFFll);
  if (offset) *offset = rec[1];
  return RES2TAC_OK;
}

}  // extern "C"
