// Batch engine: every stage of the pipeline runs as a persistent kernel over all pairs of the
// batch. A block (or, in the aggregation, a warp) claims its next work item from a device queue
// with one atomic increment and maps it to (pair, item of that pair) through prefix tables; no
// block ever waits for another, so the queues need no device-side spin. Stage order is kept by
// the launch order on one stream; the two aggregation kernels (row paths and sheared-column
// paths) run concurrently on a forked stream inside the graph. The descriptor upload, the queue
// reset and the stage kernels are recorded once into a CUDA graph and replayed while the
// capacities last.
//
// Aggregation work is described by segments, two per pair: its rows (one warp item per group of
// rows) and its sheared columns (one warp item per group of adjacent chains of one kind). Each
// queue is ordered by the chain length of its segments across the whole batch (longest first),
// so the sequential chains that bound the batch's duration start earliest.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "aggregate.cuh"
#include "batch.h"
#include "batch_dev.cuh"
#include "census_cost.cuh"
#include "launch.h"
#include "post.cuh"

namespace r2t {


__global__ void __launch_bounds__(256) batch_census_kernel(const BatchHeader* hd,
                                                           const Problem* probs,
                                                           const int* prefix, Method mt,
                                                           unsigned* counters) {
  __shared__ CensusSmem sm;
  __shared__ int s_item;
  const int total = hd->total[kStCensus], n = hd->n;
  for (;;) {
    const int item = claim_block(&counters[kStCensus], &s_item);
    if (item >= total) break;
    const int p = find_slot(prefix, n, item);
    const Problem pb = probs[p];
    census_tile_dispatch(pb, mt, item - prefix[p], sm);
  }
}

__global__ void __launch_bounds__(256) batch_cost_kernel(const BatchHeader* hd,
                                                         const Problem* probs, const int* prefix,
                                                         Method mt, unsigned* counters) {
  __shared__ CostSmem sm;
  __shared__ int s_item;
  const int total = hd->total[kStCost], n = hd->n;
  for (;;) {
    const int item = claim_block(&counters[kStCost], &s_item);
    if (item >= total) break;
    const int p = find_slot(prefix, n, item);
    const Problem pb = probs[p];
    cost_tile_dispatch(pb, mt, item - prefix[p], sm);
  }
}


template <bool WIDE>
__global__ void __launch_bounds__(256) batch_wta_kernel(const BatchHeader* hd, const Problem* probs,
                                                        const int* prefix, unsigned* counters) {
  extern __shared__ __align__(16) uint8_t wsm[];
  __shared__ int s_item;
  const int total = hd->total[kStWta], n = hd->n;
  for (;;) {
    // (the barrier inside claim_block also ends the previous item's use of the shared memory)
    const int item = claim_block(&counters[kStWta], &s_item);
    if (item >= total) break;
    const int p = find_slot(prefix, n, item);
    const Problem pb = probs[p];
    const int T = wta_staged_px(pb.D, WIDE, hd->tune[tune_bucket(pb.W, pb.H, pb.D)].wta_px);
    wta_dr_staged<WIDE>(pb, item - prefix[p], wsm, T);
  }
}

__global__ void __launch_bounds__(256) batch_median_kernel(const BatchHeader* hd,
                                                           const Problem* probs, const int* prefix,
                                                           Method mt, unsigned* counters) {
  __shared__ MedianSmem sm;
  __shared__ int s_item;
  const int total = hd->total[kStMedian], n = hd->n;
  for (;;) {
    const int item = claim_block(&counters[kStMedian], &s_item);
    if (item >= total) break;
    const int p = find_slot(prefix, n, item);
    const Problem pb = probs[p];
    lr_median_tile<false, false>(pb, mt, item - prefix[p], sm);
  }
}

struct BatchEngine {
  char* scratch = nullptr;
  size_t scratch_cap = 0;
  char* d_desc = nullptr;  // descriptor block (device)
  char* h_desc = nullptr;  // its pinned host image
  size_t desc_bytes = 0;
  int cap_pairs = 0;
  unsigned* d_counters = nullptr;
  cudaStream_t cap_stream = nullptr;
  Fork fork = {nullptr, nullptr, nullptr};
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t copied = nullptr;  // recorded in the graph after the descriptor upload
  bool copy_pending = false;
  Method graph_method;
  int graph_wta_smem = 0;
  int graph_shear_smem = 0;  // per warp
  int graph_launches = 0;
  BatchTune tune[kTuneBuckets];
  char err[256];
};

static size_t probs_offset() { return (sizeof(BatchHeader) + 255) / 256 * 256; }
static size_t prefix_offset(int cap) { return probs_offset() + (size_t)cap * sizeof(Problem); }
static size_t segs_offset(int cap, int q) {  // q = 0 rows, 1 sheared columns
  const size_t base = (prefix_offset(cap) + 4 * sizeof(int) * (size_t)(cap + 1) + 15) / 16 * 16;
  const size_t per = ((size_t)cap * sizeof(AggSeg) + sizeof(int) * (size_t)(cap + 1) + 15) / 16 * 16;
  return base + q * per;
}
static size_t seg_prefix_offset(int cap, int q) { return segs_offset(cap, q) + (size_t)cap * sizeof(AggSeg); }
static size_t desc_size(int cap) { return segs_offset(cap, 2); }

size_t batch_fixed_bytes(int n) { return desc_size(n) + 4096; }

static int set_err(BatchEngine* e, cudaError_t c, const char* what) {
  cudaGetLastError();
  snprintf(e->err, sizeof(e->err), "%s: %s", what, cudaGetErrorString(c));
  return c == cudaErrorMemoryAllocation ? -2 : -3;
}

static int grow_desc(BatchEngine* e, int n) {
  if (n <= e->cap_pairs) return 0;
  const int cap = std::max(n, 2 * e->cap_pairs);
  if (e->copy_pending) cudaEventSynchronize(e->copied);
  cudaDeviceSynchronize();  // the old descriptor block may still be read by a running batch
  cudaFree(e->d_desc);
  cudaFreeHost(e->h_desc);
  e->d_desc = nullptr;
  e->h_desc = nullptr;
  e->desc_bytes = desc_size(cap);
  cudaError_t c = cudaMalloc(&e->d_desc, e->desc_bytes);
  if (c == cudaSuccess) c = cudaMallocHost(&e->h_desc, e->desc_bytes);
  if (c != cudaSuccess) {
    e->cap_pairs = 0;
    return set_err(e, c, "descriptor allocation");
  }
  e->cap_pairs = cap;
  e->copy_pending = false;
  if (e->exec) {  // the graph holds the old descriptor addresses
    cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
  }
  return 0;
}

int batch_reserve(BatchEngine** pe, size_t scratch_bytes, int n) {
  if (!*pe) {
    BatchEngine* e = new BatchEngine();
    for (int b = 0; b < kTuneBuckets; b++) e->tune[b] = batch_default_tune(b);
    e->err[0] = 0;
    memset(&e->graph_method, 0, sizeof(Method));
    *pe = e;
    cudaError_t c = cudaMalloc(&e->d_counters, 64);
    if (c == cudaSuccess) c = cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking);
    if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->copied, cudaEventDisableTiming);
    if (c == cudaSuccess) c = fork_create(&e->fork);
    if (c != cudaSuccess) return set_err(e, c, "batch engine setup");
  }
  BatchEngine* e = *pe;
  if (!e->d_counters || !e->fork.aux)
    return set_err(e, cudaErrorInitializationError, "batch engine setup");
  if (scratch_bytes > e->scratch_cap) {
    // the previous batch may still run on its stream: wait before freeing its scratch
    cudaDeviceSynchronize();
    cudaFree(e->scratch);
    e->scratch = nullptr;
    e->scratch_cap = 0;
    cudaError_t c = cudaMalloc(&e->scratch, scratch_bytes);
    if (c != cudaSuccess) return set_err(e, c, "batch scratch allocation");
    e->scratch_cap = scratch_bytes;
  }
  return grow_desc(e, n);
}

char* batch_scratch(BatchEngine* e) { return e ? e->scratch : nullptr; }
const char* batch_error(BatchEngine* e) { return e ? e->err : "no batch engine"; }

BatchTune batch_default_tune(int bucket) {
  const int D = 16 * (bucket / 2);
  BatchTune t;
  memset(&t, 0, sizeof(t));
  t.row_dpl = (signed char)long_dpl_default(D);
  t.shear_dpl = 16;
  t.shear_cpl = 1;
  t.wta_px = 128;
  return t;
}

bool batch_tune_valid(int bucket, const BatchTune& t) {
  const int D = 16 * (bucket / 2);
  if (bucket < 2 || bucket >= kTuneBuckets) return false;
  if (t.row_dpl != 2 && t.row_dpl != 4 && t.row_dpl != 8) return false;
  if (D % t.row_dpl != 0 || D / t.row_dpl > 32) return false;
  if (!batch_shear_ok(t.shear_dpl, t.shear_cpl) || D % t.shear_dpl != 0) return false;
  return t.wta_px == 64 || t.wta_px == 128 || t.wta_px == 256;
}

int batch_set_tune(BatchEngine* e, int bucket, const BatchTune& t) {
  if (!e || !batch_tune_valid(bucket, t)) return -1;
  e->tune[bucket] = t;
  return 0;
}

BatchTune batch_get_tune(BatchEngine* e, int bucket) {
  return (e && bucket >= 0 && bucket < kTuneBuckets) ? e->tune[bucket] : batch_default_tune(bucket);
}

void batch_destroy(BatchEngine* e) {
  if (!e) return;
  if (e->exec) cudaGraphExecDestroy(e->exec);
  if (e->copied) cudaEventDestroy(e->copied);
  if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
  fork_destroy(&e->fork);
  cudaFree(e->scratch);
  cudaFree(e->d_desc);
  cudaFreeHost(e->h_desc);
  cudaFree(e->d_counters);
  delete e;
}

template <class K>
static int persistent_grid(K kernel, size_t smem) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, 256, smem);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

template <bool WIDE>
static int capture_t(BatchEngine* e, const Method& mt, int wta_smem, int warp_smem) {
  const int cap = e->cap_pairs;
  const BatchHeader* hd = reinterpret_cast<const BatchHeader*>(e->d_desc);
  const Problem* probs = reinterpret_cast<const Problem*>(e->d_desc + probs_offset());
  const int* prefix = reinterpret_cast<const int*>(e->d_desc + prefix_offset(cap));
  const int stride = cap + 1;
  const AggSeg* lsegs = reinterpret_cast<const AggSeg*>(e->d_desc + segs_offset(cap, 0));
  const int* lpre = reinterpret_cast<const int*>(e->d_desc + seg_prefix_offset(cap, 0));
  const AggSeg* bsegs = reinterpret_cast<const AggSeg*>(e->d_desc + segs_offset(cap, 1));
  const int* bpre = reinterpret_cast<const int*>(e->d_desc + seg_prefix_offset(cap, 1));
  // launch shapes and attributes are settled before the capture starts
  cudaFuncSetAttribute(batch_wta_kernel<WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       wta_smem);
  const int g_census = persistent_grid(batch_census_kernel, 0);
  const int g_cost = persistent_grid(batch_cost_kernel, 0);
  const void* k_rows = batch_row_kernel_fn<WIDE>();
  const void* k_shear = batch_shear_kernel_fn<WIDE>();
  const int g_rows = persistent_grid(k_rows, 0);
  const int shear_smem = 8 * warp_smem;  // 8 warps per block
  cudaFuncSetAttribute(k_shear, cudaFuncAttributeMaxDynamicSharedMemorySize, shear_smem);
  const int g_shear = persistent_grid(k_shear, shear_smem);
  const int g_wta = persistent_grid(batch_wta_kernel<WIDE>, wta_smem);
  const int g_med = persistent_grid(batch_median_kernel, 0);
  cudaError_t c = cudaGetLastError();
  if (c != cudaSuccess) return set_err(e, c, "kernel attributes");
  cudaStream_t cs = e->cap_stream;
  cudaGraph_t g = nullptr;
  c = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (c != cudaSuccess) return set_err(e, c, "begin capture");
  cudaMemcpyAsync(e->d_desc, e->h_desc, e->desc_bytes, cudaMemcpyHostToDevice, cs);
  // an external record node, so the host can wait for the upload of each replay
  cudaEventRecordWithFlags(e->copied, cs, cudaEventRecordExternal);
  cudaMemsetAsync(e->d_counters, 0, 64, cs);
  batch_census_kernel<<<g_census, 256, 0, cs>>>(hd, probs, prefix + 3 * stride, mt, e->d_counters);
  batch_cost_kernel<<<g_cost, 256, 0, cs>>>(hd, probs, prefix + 0 * stride, mt, e->d_counters);
  cudaEventRecord(e->fork.fork, cs);
  cudaStreamWaitEvent(e->fork.aux, e->fork.fork, 0);
  {
    int nseg = cap;
    Method m = mt;
    unsigned* counters = e->d_counters;
    int wsm = warp_smem;
    void* rargs[] = {(void*)&hd, (void*)&probs, (void*)&lsegs, (void*)&lpre, (void*)&nseg,
                     (void*)&m, (void*)&counters, (void*)&wsm};
    void* sargs[] = {(void*)&hd, (void*)&probs, (void*)&bsegs, (void*)&bpre, (void*)&nseg,
                     (void*)&m, (void*)&counters, (void*)&wsm};
    // the row kernel holds the batch's longest chains: its node keeps the highest priority so
    // its blocks are dispatched ahead of the sheared kernel's
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributePriority;
    attr[0].val.priority = hi;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g_rows);
    cfg.blockDim = dim3(256);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = e->fork.aux;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaLaunchKernelExC(&cfg, k_rows, rargs);
    cudaLaunchKernel(k_shear, dim3(g_shear), dim3(256), sargs, shear_smem, cs);
  }
  cudaEventRecord(e->fork.join, e->fork.aux);
  cudaStreamWaitEvent(cs, e->fork.join, 0);
  batch_wta_kernel<WIDE><<<g_wta, 256, wta_smem, cs>>>(hd, probs, prefix + 1 * stride,
                                                       e->d_counters);
  batch_median_kernel<<<g_med, 256, 0, cs>>>(hd, probs, prefix + 2 * stride, mt, e->d_counters);
  c = cudaStreamEndCapture(cs, &g);
  if (c != cudaSuccess) return set_err(e, c, "end capture");
  c = cudaGraphInstantiate(&e->exec, g, 0);
  cudaGraphDestroy(g);
  if (c != cudaSuccess) return set_err(e, c, "graph instantiate");
  e->graph_method = mt;
  e->graph_wta_smem = wta_smem;
  e->graph_shear_smem = warp_smem;
  e->graph_launches = 6;
  return 0;
}

static int capture(BatchEngine* e, const Method& mt, int wta_smem, int warp_smem) {
  if (e->exec) {
    cudaGraphExecDestroy(e->exec);
    e->exec = nullptr;
  }
  return mt.wide ? capture_t<true>(e, mt, wta_smem, warp_smem)
                 : capture_t<false>(e, mt, wta_smem, warp_smem);
}

struct Keyed {
  AggSeg s;
  int len;
};

// Writes one queue's segments, sorted by their chain length, and its prefix table.
static int write_queue(std::vector<Keyed>& kv, AggSeg* segs, int* pre, int cap) {
  std::stable_sort(kv.begin(), kv.end(), [](const Keyed& a, const Keyed& b) { return a.len > b.len; });
  int items = 0;
  const int n = (int)kv.size();
  for (int i = 0; i < n; i++) {
    segs[i] = kv[i].s;
    pre[i] = items;
    items += (kv[i].s.end - kv[i].s.begin + kv[i].s.group - 1) / kv[i].s.group;
  }
  for (int i = n; i <= cap; i++) pre[i] = items;  // padding slots never match an item
  return items;
}

int batch_run(BatchEngine* e, const Problem* probs, int n, const Method& mt, cudaStream_t s,
              int* launches) {
  int rc = grow_desc(e, n);
  if (rc) return rc;
  const int cap = e->cap_pairs;
  // the previous replay must have consumed the pinned descriptors before they are rewritten
  if (e->copy_pending) {
    cudaError_t c = cudaEventSynchronize(e->copied);
    if (c != cudaSuccess) return set_err(e, c, "descriptor upload wait");
    e->copy_pending = false;
  }
  BatchHeader* hd = reinterpret_cast<BatchHeader*>(e->h_desc);
  memset(hd, 0, sizeof(BatchHeader));
  Problem* hp = reinterpret_cast<Problem*>(e->h_desc + probs_offset());
  int* prefix = reinterpret_cast<int*>(e->h_desc + prefix_offset(cap));
  const int stride = cap + 1;
  int tot[4] = {0, 0, 0, 0};
  int wta_smem = 0, warp_smem = 0;
  std::vector<Keyed> lk, bk;
  lk.reserve(n);
  bk.reserve(n);
  for (int p = 0; p < n; p++) {
    const Problem& pb = probs[p];
    const BatchTune& tn = e->tune[tune_bucket(pb.W, pb.H, pb.D)];
    hp[p] = pb;
    prefix[0 * stride + p] = tot[0];
    prefix[1 * stride + p] = tot[1];
    prefix[2 * stride + p] = tot[2];
    prefix[3 * stride + p] = tot[3];
    tot[0] += cost_items(pb.W, pb.H);
    tot[3] += 2 * census_items(pb.W, pb.H);
    const int wt = wta_staged_px(pb.D, mt.wide != 0, tn.wta_px);
    tot[1] += wta_items(pb.W, pb.H, wt);
    tot[2] += median_items(pb.W, pb.H);
    wta_smem = std::max(wta_smem, (int)wta_staged_smem_bytes(pb.D, mt.wide != 0, wt));
    warp_smem = std::max(warp_smem, shear_smem_bytes(tn.shear_dpl, mt.wide != 0, tn.shear_cpl));
    lk.push_back(Keyed{AggSeg{p, 0, row_units(pb.H, true), 32 / long_lanes(pb.D, tn.row_dpl)},
                       pb.W});
    bk.push_back(Keyed{AggSeg{p, 0, shear_items(pb.W, pb.D, tn.shear_dpl, mt.num_paths,
                                                tn.shear_cpl), 1}, pb.H});
  }
  for (int k = 0; k < 4; k++) prefix[k * stride + n] = tot[k];
  const int nrows = write_queue(lk, reinterpret_cast<AggSeg*>(e->h_desc + segs_offset(cap, 0)),
                                reinterpret_cast<int*>(e->h_desc + seg_prefix_offset(cap, 0)), cap);
  const int nshear = write_queue(bk, reinterpret_cast<AggSeg*>(e->h_desc + segs_offset(cap, 1)),
                                reinterpret_cast<int*>(e->h_desc + seg_prefix_offset(cap, 1)), cap);
  hd->n = n;
  hd->total[kStCost] = tot[0];
  hd->total[kStRows] = nrows;
  hd->total[kStShear] = nshear;
  hd->total[kStWta] = tot[1];
  hd->total[kStMedian] = tot[2];
  hd->total[kStCensus] = tot[3];
  memcpy(hd->tune, e->tune, sizeof(hd->tune));
  if (!e->exec || memcmp(&e->graph_method, &mt, sizeof(Method)) != 0 ||
      wta_smem > e->graph_wta_smem || warp_smem > e->graph_shear_smem) {
    rc = capture(e, mt, std::max(wta_smem, e->graph_wta_smem),
                 std::max(warp_smem, e->graph_shear_smem));
    if (rc) return rc;
  }
  cudaError_t c = cudaGraphLaunch(e->exec, s);
  if (c != cudaSuccess) return set_err(e, c, "graph launch");
  e->copy_pending = true;
  if (launches) *launches = e->graph_launches;
  return 0;
}

}  // namespace r2t
