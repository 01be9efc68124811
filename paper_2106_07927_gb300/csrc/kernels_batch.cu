// Batch engine: many pairs of uneven W, H, D run as persistent stage kernels fed by device work
// queues, recorded into a CUDA graph and replayed while the batch layout lasts.
//
// Groups. The pairs are sorted by their memory footprint (cost volume + aggregated volume) and
// cut into groups whose footprint stays within kGroupBytes (a larger pair is a group of its own).
// Each group runs the six stages - census, cost, the two aggregation kernels (concurrently, on
// a forked stream), WTA, LR check + median - as persistent kernels over its own pairs, so a
// group's volumes are still in L2 when its next stage reads them, as they are for a pair run
// alone, while the pairs of a group fill the GPU together. Groups rotate over kSlots slots of
// streams, so one group's latency-bound aggregation overlaps the next groups' other stages
// (measured on the 64-pair mix: 0.80 of per-pair launches with one slot, 0.985 with two, 1.013
// with four; aggregation blocks of two warps, as the single-pair kernels use, rather than
// eight: 0.977 -> 0.985 with two slots).
//
// A block (or, in the aggregation, a warp) claims its next work item from its group's queue
// with one atomic increment and maps it to (pair, item of that pair) through prefix tables; no
// block ever waits for another, so the queues need no device-side spin. Aggregation work is
// described by segments, two per pair: its rows (one warp item per group of rows) and its
// sheared columns (one warp item per group of adjacent chains of one kind); each group's queue
// is ordered by chain length (longest first), so the sequential chains that bound the group's
// duration start earliest.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <numeric>
#include <vector>

#include "aggregate.cuh"
#include "batch.h"
#include "batch_dev.cuh"
#include "census_cost.cuh"
#include "launch.h"
#include "post.cuh"

namespace r2t {


// Footprint bound of one group (bytes of cost and aggregated volumes) and its pair count.
constexpr size_t kGroupBytes = 96u << 20;
constexpr int kGroupMaxPairs = 32;
constexpr int kSlots = 4;  // groups in flight
constexpr int kAggWarps = 2;  // warps per block of the persistent aggregation kernels
// Blocks per SM of the persistent aggregation kernels. Their warps claim chains with atomics;
// a grid of every block that fits lets the SMs that start first take most of a group's long row
// chains, which then share their schedulers while other SMs idle (a single 1242x375 pair: row
// kernel 228 us against 121 us for the single-pair launch, whose blocks the hardware spreads).
constexpr int kRowBlocksPerSM = 3, kShearBlocksPerSM = 8;

// Block-claimed stage kernels of one group: item = lo + claim, pair found among the group's.
#define R2T_GROUP_LOOP(STAGE, BODY)                                                  \
  __shared__ int s_item;                                                             \
  const int p0 = gd->p0, np = gd->np, lo = gd->lo[STAGE], hi = gd->hi[STAGE];       \
  for (;;) {                                                                         \
    const int item = lo + claim_block(&counters[STAGE], &s_item);                   \
    if (item >= hi) break;                                                           \
    const int p = p0 + find_slot(prefix + p0, np, item);                             \
    const Problem pb = probs[p];                                                     \
    BODY;                                                                            \
  }

__global__ void __launch_bounds__(256) batch_census_kernel(const GroupDesc* gd,
                                                           const Problem* probs,
                                                           const int* prefix, Method mt,
                                                           unsigned* counters) {
  __shared__ CensusSmem sm;
  R2T_GROUP_LOOP(kStCensus, census_tile_dispatch(pb, mt, item - prefix[p], sm))
}

// (at least 5 blocks per SM: the population counts need the warps to hide their pipe's queue)
__global__ void __launch_bounds__(256, 5) batch_cost_kernel(const GroupDesc* gd,
                                                         const Problem* probs, const int* prefix,
                                                         Method mt, unsigned* counters) {
  __shared__ CostSmem sm;
  R2T_GROUP_LOOP(kStCost, cost_tile_dispatch(pb, mt, item - prefix[p], sm))
}

// (the barrier inside claim_block also ends the previous item's use of the shared memory)
template <bool WIDE>
__global__ void __launch_bounds__(256) batch_wta_kernel(const BatchHeader* hd, const GroupDesc* gd,
                                                        const Problem* probs, const int* prefix,
                                                        unsigned* counters) {
  extern __shared__ __align__(16) uint8_t wsm[];
  R2T_GROUP_LOOP(kStWta,
                 wta_dr_staged<WIDE>(pb, item - prefix[p], wsm,
                                     wta_staged_px(pb.D, WIDE,
                                                   hd->tune[tune_bucket(pb.W, pb.H, pb.D)].wta_px)))
}

__global__ void __launch_bounds__(256) batch_median_kernel(const GroupDesc* gd,
                                                           const Problem* probs, const int* prefix,
                                                           Method mt, unsigned* counters) {
  __shared__ MedianSmem sm;
  R2T_GROUP_LOOP(kStMedian, (lr_median_tile<false, false>(pb, mt, item - prefix[p], sm)))
}
#undef R2T_GROUP_LOOP

struct BatchEngine {
  char* scratch = nullptr;
  size_t scratch_cap = 0;
  char* d_desc = nullptr;  // descriptor block (device)
  char* h_desc = nullptr;  // its pinned host image
  size_t desc_bytes = 0;
  int cap_pairs = 0;
  unsigned* d_counters = nullptr;  // kCountersPerGroup per group, cap_pairs groups
  cudaStream_t main[kSlots] = {};  // main[0] is the capture origin
  cudaStream_t aux[kSlots] = {};   // row-path kernels of each slot
  cudaEvent_t ev_fork[kSlots] = {}, ev_join[kSlots] = {};
  cudaEvent_t ev_start = nullptr, ev_end = nullptr;
  // captured graphs by group count (index G), all for graph_method and the shared-memory sizes
  std::vector<cudaGraphExec_t> execs;
  cudaEvent_t copied = nullptr;  // recorded in the graph after the descriptor upload
  bool copy_pending = false;
  Method graph_method;
  int graph_wta_smem = 0;
  int graph_shear_smem = 0;  // per warp
  BatchTune tune[kTuneBuckets];
  char err[256];
};

// Descriptor block: BatchHeader | Problem[cap] | int prefix[4][cap + 1] (cost, wta, median,
// census items) | for the row and the sheared queue AggSeg[cap], int seg_prefix[cap + 1] |
// GroupDesc[cap].
static size_t probs_offset() { return (sizeof(BatchHeader) + 255) / 256 * 256; }
static size_t prefix_offset(int cap) { return probs_offset() + (size_t)cap * sizeof(Problem); }
static size_t segs_offset(int cap, int q) {  // q = 0 rows, 1 sheared columns, 2 groups
  const size_t base = (prefix_offset(cap) + 4 * sizeof(int) * (size_t)(cap + 1) + 15) / 16 * 16;
  const size_t per = ((size_t)cap * sizeof(AggSeg) + sizeof(int) * (size_t)(cap + 1) + 15) / 16 * 16;
  return base + q * per;
}
static size_t seg_prefix_offset(int cap, int q) { return segs_offset(cap, q) + (size_t)cap * sizeof(AggSeg); }
static size_t groups_offset(int cap) { return segs_offset(cap, 2); }
static size_t desc_size(int cap) { return groups_offset(cap) + (size_t)cap * sizeof(GroupDesc); }

size_t batch_fixed_bytes(int n) {
  return desc_size(n) + (size_t)n * kCountersPerGroup * sizeof(unsigned) + 4096;
}

static int set_err(BatchEngine* e, cudaError_t c, const char* what) {
  cudaGetLastError();
  snprintf(e->err, sizeof(e->err), "%s: %s", what, cudaGetErrorString(c));
  return c == cudaErrorMemoryAllocation ? -2 : -3;
}

static void drop_graphs(BatchEngine* e) {
  for (cudaGraphExec_t& x : e->execs)
    if (x) cudaGraphExecDestroy(x);
  e->execs.clear();
}

static int grow_desc(BatchEngine* e, int n) {
  if (n <= e->cap_pairs) return 0;
  const int cap = std::max(n, 2 * e->cap_pairs);
  if (e->copy_pending) cudaEventSynchronize(e->copied);
  cudaDeviceSynchronize();  // the old descriptor block may still be read by a running batch
  cudaFree(e->d_desc);
  cudaFreeHost(e->h_desc);
  cudaFree(e->d_counters);
  e->d_desc = nullptr;
  e->h_desc = nullptr;
  e->d_counters = nullptr;
  e->desc_bytes = desc_size(cap);
  cudaError_t c = cudaMalloc(&e->d_desc, e->desc_bytes);
  if (c == cudaSuccess) c = cudaMallocHost(&e->h_desc, e->desc_bytes);
  if (c == cudaSuccess)
    c = cudaMalloc(&e->d_counters, (size_t)cap * kCountersPerGroup * sizeof(unsigned));
  if (c != cudaSuccess) {
    e->cap_pairs = 0;
    return set_err(e, c, "descriptor allocation");
  }
  e->cap_pairs = cap;
  e->copy_pending = false;
  drop_graphs(e);  // the graphs hold the old descriptor addresses
  return 0;
}

int batch_reserve(BatchEngine** pe, size_t scratch_bytes, int n) {
  if (!*pe) {
    BatchEngine* e = new BatchEngine();
    for (int b = 0; b < kTuneBuckets; b++) e->tune[b] = batch_default_tune(b);
    e->err[0] = 0;
    memset(&e->graph_method, 0, sizeof(Method));
    *pe = e;
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);
    cudaError_t c = cudaSuccess;
    for (int k = 0; k < kSlots && c == cudaSuccess; k++) {
      c = cudaStreamCreateWithFlags(&e->main[k], cudaStreamNonBlocking);
      if (c == cudaSuccess) c = cudaStreamCreateWithPriority(&e->aux[k], cudaStreamNonBlocking, hi);
      if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->ev_fork[k], cudaEventDisableTiming);
      if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->ev_join[k], cudaEventDisableTiming);
    }
    if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->ev_start, cudaEventDisableTiming);
    if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->ev_end, cudaEventDisableTiming);
    if (c == cudaSuccess) c = cudaEventCreateWithFlags(&e->copied, cudaEventDisableTiming);
    if (c != cudaSuccess) return set_err(e, c, "batch engine setup");
  }
  BatchEngine* e = *pe;
  if (!e->main[0] || !e->copied)
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
  drop_graphs(e);
  if (e->copied) cudaEventDestroy(e->copied);
  for (int k = 0; k < kSlots; k++) {
    if (e->main[k]) cudaStreamDestroy(e->main[k]);
    if (e->aux[k]) cudaStreamDestroy(e->aux[k]);
    if (e->ev_fork[k]) cudaEventDestroy(e->ev_fork[k]);
    if (e->ev_join[k]) cudaEventDestroy(e->ev_join[k]);
  }
  if (e->ev_start) cudaEventDestroy(e->ev_start);
  if (e->ev_end) cudaEventDestroy(e->ev_end);
  cudaFree(e->scratch);
  cudaFree(e->d_desc);
  cudaFreeHost(e->h_desc);
  cudaFree(e->d_counters);
  delete e;
}

static int sm_count() {
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  return sms > 0 ? sms : 1;
}

template <class K>
static int persistent_grid(K kernel, size_t smem, int threads = 256) {
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  if (per_sm < 1) per_sm = 1;
  return sms * per_sm;
}

// Records the graph for G groups: the descriptor upload and the counter reset on main[0], then
// group g's six stage kernels on slot g % kSlots (its row-path kernel forked onto the slot's
// aux stream), and the join of every stream back into main[0].
template <bool WIDE>
static int capture_t(BatchEngine* e, const Method& mt, int wta_smem, int warp_smem, int G) {
  const int cap = e->cap_pairs;
  const BatchHeader* hd = reinterpret_cast<const BatchHeader*>(e->d_desc);
  const Problem* probs = reinterpret_cast<const Problem*>(e->d_desc + probs_offset());
  const int* prefix = reinterpret_cast<const int*>(e->d_desc + prefix_offset(cap));
  const int stride = cap + 1;
  const AggSeg* lsegs = reinterpret_cast<const AggSeg*>(e->d_desc + segs_offset(cap, 0));
  const int* lpre = reinterpret_cast<const int*>(e->d_desc + seg_prefix_offset(cap, 0));
  const AggSeg* bsegs = reinterpret_cast<const AggSeg*>(e->d_desc + segs_offset(cap, 1));
  const int* bpre = reinterpret_cast<const int*>(e->d_desc + seg_prefix_offset(cap, 1));
  const GroupDesc* groups = reinterpret_cast<const GroupDesc*>(e->d_desc + groups_offset(cap));
  // launch shapes and attributes are settled before the capture starts
  cudaFuncSetAttribute(batch_wta_kernel<WIDE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       wta_smem);
  const int g_census = persistent_grid(batch_census_kernel, 0);
  const int g_cost = persistent_grid(batch_cost_kernel, 0);
  const void* k_rows = batch_row_kernel_fn<WIDE>();
  const void* k_shear = batch_shear_kernel_fn<WIDE>();
  const int g_rows = std::min(persistent_grid(k_rows, 0, 32 * kAggWarps), sm_count() * kRowBlocksPerSM);
  const int shear_smem = kAggWarps * warp_smem;
  cudaFuncSetAttribute(k_shear, cudaFuncAttributeMaxDynamicSharedMemorySize, shear_smem);
  const int g_shear = std::min(persistent_grid(k_shear, shear_smem, 32 * kAggWarps),
                               sm_count() * kShearBlocksPerSM);
  const int g_wta = persistent_grid(batch_wta_kernel<WIDE>, wta_smem);
  const int g_med = persistent_grid(batch_median_kernel, 0);
  cudaError_t c = cudaGetLastError();
  if (c != cudaSuccess) return set_err(e, c, "kernel attributes");
  int lo = 0, hi = 0;
  cudaDeviceGetStreamPriorityRange(&lo, &hi);
  cudaStream_t cs = e->main[0];
  cudaGraph_t g = nullptr;
  c = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (c != cudaSuccess) return set_err(e, c, "begin capture");
  cudaMemcpyAsync(e->d_desc, e->h_desc, e->desc_bytes, cudaMemcpyHostToDevice, cs);
  // an external record node, so the host can wait for the upload of each replay
  cudaEventRecordWithFlags(e->copied, cs, cudaEventRecordExternal);
  cudaMemsetAsync(e->d_counters, 0, (size_t)G * kCountersPerGroup * sizeof(unsigned), cs);
  cudaEventRecord(e->ev_start, cs);
  for (int k = 1; k < kSlots; k++) cudaStreamWaitEvent(e->main[k], e->ev_start, 0);
  for (int gi = 0; gi < G; gi++) {
    const int sl = gi % kSlots;
    cudaStream_t m = e->main[sl], a = e->aux[sl];
    const GroupDesc* gd = groups + gi;
    unsigned* cnt = e->d_counters + (size_t)gi * kCountersPerGroup;
    batch_census_kernel<<<g_census, 256, 0, m>>>(gd, probs, prefix + 3 * stride, mt, cnt);
    batch_cost_kernel<<<g_cost, 256, 0, m>>>(gd, probs, prefix + 0 * stride, mt, cnt);
    cudaEventRecord(e->ev_fork[sl], m);
    cudaStreamWaitEvent(a, e->ev_fork[sl], 0);
    {
      Method mm = mt;
      int wsm = warp_smem;
      void* rargs[] = {(void*)&hd, (void*)&gd, (void*)&probs, (void*)&lsegs, (void*)&lpre,
                       (void*)&mm, (void*)&cnt, (void*)&wsm};
      void* sargs[] = {(void*)&hd, (void*)&gd, (void*)&probs, (void*)&bsegs, (void*)&bpre,
                       (void*)&mm, (void*)&cnt, (void*)&wsm};
      // the row kernel holds the group's longest chains: its node keeps the highest priority so
      // its blocks are dispatched ahead of the sheared kernel's
      cudaLaunchAttribute attr[1];
      attr[0].id = cudaLaunchAttributePriority;
      attr[0].val.priority = hi;
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(g_rows);
      cfg.blockDim = dim3(32 * kAggWarps);
      cfg.dynamicSmemBytes = 0;
      cfg.stream = a;
      cfg.attrs = attr;
      cfg.numAttrs = 1;
      cudaLaunchKernelExC(&cfg, k_rows, rargs);
      cudaLaunchKernel(k_shear, dim3(g_shear), dim3(32 * kAggWarps), sargs, shear_smem, m);
    }
    cudaEventRecord(e->ev_join[sl], a);
    cudaStreamWaitEvent(m, e->ev_join[sl], 0);
    batch_wta_kernel<WIDE><<<g_wta, 256, wta_smem, m>>>(hd, gd, probs, prefix + 1 * stride, cnt);
    batch_median_kernel<<<g_med, 256, 0, m>>>(gd, probs, prefix + 2 * stride, mt, cnt);
  }
  for (int k = 1; k < kSlots; k++) {
    cudaEventRecord(e->ev_end, e->main[k]);
    cudaStreamWaitEvent(cs, e->ev_end, 0);
  }
  c = cudaStreamEndCapture(cs, &g);
  if (c != cudaSuccess) return set_err(e, c, "end capture");
  cudaGraphExec_t x = nullptr;
  c = cudaGraphInstantiate(&x, g, 0);
  cudaGraphDestroy(g);
  if (c != cudaSuccess) return set_err(e, c, "graph instantiate");
  if ((int)e->execs.size() <= G) e->execs.resize((size_t)G + 1, nullptr);
  e->execs[(size_t)G] = x;
  return 0;
}

// The graph for G groups, captured when missing; every cached graph is dropped first when the
// method or a shared-memory size changes.
static int graph_for(BatchEngine* e, const Method& mt, int wta_smem, int warp_smem, int G,
                     cudaGraphExec_t* out) {
  if (memcmp(&e->graph_method, &mt, sizeof(Method)) != 0 || wta_smem > e->graph_wta_smem ||
      warp_smem > e->graph_shear_smem) {
    drop_graphs(e);
    e->graph_method = mt;
    e->graph_wta_smem = std::max(wta_smem, e->graph_wta_smem);
    e->graph_shear_smem = std::max(warp_smem, e->graph_shear_smem);
  }
  if ((int)e->execs.size() <= G || !e->execs[(size_t)G]) {
    const int rc = mt.wide ? capture_t<true>(e, mt, e->graph_wta_smem, e->graph_shear_smem, G)
                           : capture_t<false>(e, mt, e->graph_wta_smem, e->graph_shear_smem, G);
    if (rc) return rc;
  }
  *out = e->execs[(size_t)G];
  return 0;
}

struct Keyed {
  AggSeg s;
  int len;
};

// Writes one group's queue segments at segs[0 .. k), sorted by their chain length, with item
// prefixes continuing from base; returns the queue's item count after the group.
static int write_queue(std::vector<Keyed>& kv, AggSeg* segs, int* pre, int base) {
  std::stable_sort(kv.begin(), kv.end(), [](const Keyed& a, const Keyed& b) { return a.len > b.len; });
  int items = base;
  for (size_t i = 0; i < kv.size(); i++) {
    segs[i] = kv[i].s;
    pre[i] = items;
    items += (kv[i].s.end - kv[i].s.begin + kv[i].s.group - 1) / kv[i].s.group;
  }
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
  const size_t bpe = mt.wide ? 4 : 2;
  // pairs by footprint, largest first, then cut into groups
  std::vector<int> order((size_t)n);
  std::iota(order.begin(), order.end(), 0);
  auto fp = [&](int p) { return (size_t)probs[p].W * probs[p].H * probs[p].D * (1 + bpe); };
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return fp(a) > fp(b); });
  std::vector<int> gstart;
  for (int i = 0; i < n;) {
    gstart.push_back(i);
    size_t bytes = fp(order[i]);
    int k = 1;
    i++;
    while (i < n && k < kGroupMaxPairs && bytes + fp(order[i]) <= kGroupBytes) {
      bytes += fp(order[i]);
      k++;
      i++;
    }
  }
  const int G = (int)gstart.size();
  gstart.push_back(n);

  BatchHeader* hd = reinterpret_cast<BatchHeader*>(e->h_desc);
  memset(hd, 0, sizeof(BatchHeader));
  Problem* hp = reinterpret_cast<Problem*>(e->h_desc + probs_offset());
  int* prefix = reinterpret_cast<int*>(e->h_desc + prefix_offset(cap));
  AggSeg* lsegs = reinterpret_cast<AggSeg*>(e->h_desc + segs_offset(cap, 0));
  int* lpre = reinterpret_cast<int*>(e->h_desc + seg_prefix_offset(cap, 0));
  AggSeg* bsegs = reinterpret_cast<AggSeg*>(e->h_desc + segs_offset(cap, 1));
  int* bpre = reinterpret_cast<int*>(e->h_desc + seg_prefix_offset(cap, 1));
  GroupDesc* groups = reinterpret_cast<GroupDesc*>(e->h_desc + groups_offset(cap));
  const int stride = cap + 1;
  int tot[4] = {0, 0, 0, 0};
  int wta_smem = 0, warp_smem = 0, nrows = 0, nshear = 0;
  for (int gi = 0; gi < G; gi++) {
    const int p0 = gstart[gi], p1 = gstart[gi + 1];
    GroupDesc& gd = groups[gi];
    memset(&gd, 0, sizeof(gd));
    gd.p0 = p0;
    gd.np = p1 - p0;
    gd.lo[kStCost] = tot[0];
    gd.lo[kStWta] = tot[1];
    gd.lo[kStMedian] = tot[2];
    gd.lo[kStCensus] = tot[3];
    std::vector<Keyed> lk, bk;
    for (int i = p0; i < p1; i++) {
      const Problem& pb = probs[order[i]];
      const BatchTune& tn = e->tune[tune_bucket(pb.W, pb.H, pb.D)];
      hp[i] = pb;
      prefix[0 * stride + i] = tot[0];
      prefix[1 * stride + i] = tot[1];
      prefix[2 * stride + i] = tot[2];
      prefix[3 * stride + i] = tot[3];
      tot[0] += cost_items(pb.W, pb.H);
      const int wt = wta_staged_px(pb.D, mt.wide != 0, tn.wta_px);
      tot[1] += wta_items(pb.W, pb.H, wt);
      tot[2] += median_items(pb.W, pb.H);
      tot[3] += 2 * census_items(pb.W, pb.H);
      wta_smem = std::max(wta_smem, (int)wta_staged_smem_bytes(pb.D, mt.wide != 0, wt));
      warp_smem = std::max(warp_smem, shear_smem_bytes(tn.shear_dpl, mt.wide != 0, tn.shear_cpl));
      lk.push_back(Keyed{AggSeg{i, 0, row_units(pb.H, true), 32 / long_lanes(pb.D, tn.row_dpl)},
                         pb.W});
      bk.push_back(Keyed{AggSeg{i, 0, shear_items(pb.W, pb.D, tn.shear_dpl, mt.num_paths,
                                                  tn.shear_cpl), 1}, pb.H});
    }
    gd.hi[kStCost] = tot[0];
    gd.hi[kStWta] = tot[1];
    gd.hi[kStMedian] = tot[2];
    gd.hi[kStCensus] = tot[3];
    gd.lo[kStRows] = nrows;
    nrows = write_queue(lk, lsegs + p0, lpre + p0, nrows);
    gd.hi[kStRows] = nrows;
    gd.lo[kStShear] = nshear;
    nshear = write_queue(bk, bsegs + p0, bpre + p0, nshear);
    gd.hi[kStShear] = nshear;
  }
  for (int k = 0; k < 4; k++) prefix[k * stride + n] = tot[k];
  lpre[n] = nrows;
  bpre[n] = nshear;
  hd->n = n;
  hd->total[kStCost] = tot[0];
  hd->total[kStRows] = nrows;
  hd->total[kStShear] = nshear;
  hd->total[kStWta] = tot[1];
  hd->total[kStMedian] = tot[2];
  hd->total[kStCensus] = tot[3];
  memcpy(hd->tune, e->tune, sizeof(hd->tune));
  cudaGraphExec_t exec = nullptr;
  rc = graph_for(e, mt, wta_smem, warp_smem, G, &exec);
  if (rc) return rc;
  cudaError_t c = cudaGraphLaunch(exec, s);
  if (c != cudaSuccess) return set_err(e, c, "graph launch");
  e->copy_pending = true;
  if (launches) *launches = 6 * G;
  return 0;
}

}  // namespace r2t
