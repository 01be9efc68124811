// The Hamming matching cost of the 9 x 7 census (Eq. image_matching) as a contraction on the
// tensor cores (tcgen05, fp8 operands, fp32 accumulators in tensor memory).
//
// For 62-bit descriptors a (left pixel x) and b (right pixel x'), with a_k, b_k in {0, 1},
//   popcount(a ^ b) = sum_k (a_k + b_k - 2 a_k b_k) = |a| + |b| - 2 a.b,
// a dot product over k plus two terms. One tile is row y, left pixels x0 .. x0 + 127 (the M = 128
// rows of A) against right pixels x0 - 128 .. x0 + 127 (the N = 256 rows of B), K = 64:
//   A row x : -2 a_0 .. -2 a_61, 1, 1
//   B row x': b_0 .. b_61, h, l      with |b| = h + l, h = |b| & 56, l = |b| & 7
// so that the accumulator holds v(x, x') = |b| - 2 a.b, and popcount(a ^ b) = v + |a|. Every
// value is an integer representable in e4m3 (0, 1, -2, 0..7, 8..56 in steps of 8); the products
// and every partial sum are integers of magnitude below 2^8, so the fp32 accumulation is exact in
// any order. The epilogue adds |a| + 2^23 in fp32 (exact) and takes the low byte of the result's
// bits, which is the cost. C(x, d) is the accumulator entry (x, x - d): a band of D of the 256
// columns of row x, shifted by one column from one row to the next; each lane moves its row's
// band into place with a funnel shift and four conditional word moves, then stores it.
// Costs where x - d < 0 are 255 (the B rows left of the image are zero and are not used).
//
// Persistent blocks, one per SM, each taking a contiguous run of tiles, in three roles:
// - warps 8 - 15 (producers) expand the descriptors of tile i into operand stage i % 2 (canonical
//   K-major layout without swizzle: 8-row x 16-byte core matrices, 128 bytes apart along K, 512
//   bytes apart along M / N) and clear the tile's aggregated sums and right-disparity keys;
// - warp 16 owns the tensor memory (512 columns: two 256-column accumulators) and one of its
//   threads issues the two K = 32 MMAs of tile i into accumulator i % 2;
// - warps 0 - 7 (epilogue) read accumulator i % 2 back (warp w: lanes 32 (w % 4) .., half w / 4
//   of the disparities) and store the costs.
// The hand-offs are mbarriers: stage full (producers -> MMA), stage empty and accumulator full
// (MMA completion, tcgen05.commit), accumulator empty (epilogue -> MMA). Every wait polls at most
// kSpinLimit times; a wait that gives up records fault site 8 and makes the block stop taking
// tiles, so the kernel always ends. The block holds all 512 tensor-memory columns of its SM: when
// a kernel of another library (a tensor-core GEMM on another stream) holds columns on that SM,
// the allocation waits until that kernel frees them.
#include <stdint.h>

#include <algorithm>

#include "census_cost.cuh"
#include "launch.h"

namespace r2t {

namespace {

constexpr int kMmaM = 128, kMmaN = 256, kMmaK = 64;  // bytes per operand row (e4m3)
constexpr int kTileA = kMmaM * kMmaK, kTileB = kMmaN * kMmaK, kStageBytes = kTileA + kTileB;
constexpr int kBarOff = 2 * kStageBytes;  // 8 mbarriers, the tensor-memory address, abort flag
constexpr int kShiftOff = kBarOff + 128;  // per epilogue warp: 32 rows of a shift buffer
constexpr int kSmemRequest = 120 << 10;   // one block per SM: it holds all 512 columns
constexpr int kProdWarps = 8, kProdThreads = kProdWarps * 32;
constexpr int kEpq = 2;  // epilogue warps per lane quarter (at most D / 32)
// Warps of the kernel for D: kEpq epilogue warps per lane quarter (D / kEpq disparities each),
// then the producers, then the MMA warp.
template <int D>
struct MmaWarps {
  static constexpr int kEpiQ = kEpq < D / 32 ? kEpq : D / 32;
  static constexpr int kDh = D / kEpiQ;               // disparities per epilogue warp
  static constexpr int kNp = (kDh + 32) / 4;          // packed words read per lane
  static constexpr int kRow = kNp + 1;                // shift-buffer words per lane (odd)
  static constexpr int kEpiWarps = 4 * kEpiQ, kEpiThreads = kEpiWarps * 32;
  static constexpr int kMmaWarp = kEpiWarps + kProdWarps, kThreads = (kMmaWarp + 1) * 32;
  static constexpr int kSmemUsed = kShiftOff + kEpiThreads * kRow * 4;
};
// A wait polls the mbarrier with a suspend-time hint (the thread sleeps until the phase
// completes or the hint runs out, so waiting warps take no issue slots) at most kSpinLimit times.
constexpr uint32_t kSuspendNs = 20000;
constexpr uint32_t kSpinLimit = 1u << 16;
constexpr uint32_t kTmemCols = 512;

// e4m3 code of a small non-negative integer with at most 4 significant bits (0 .. 7, 8 .. 56 in
// steps of 8): v = 2^e (1 + m / 8) is ((e + 7) << 3) | m.
__device__ __forceinline__ uint32_t e4m3_small_int(uint32_t v) {
  if (v == 0) return 0;
  const int e = 31 - __clz(v);
  const uint32_t m = ((v << 3) >> e) & 7u;
  return ((uint32_t)(e + 7) << 3) | m;
}

// Byte offset of element (row r, byte k) of an operand tile: 8 x 16-byte core matrices.
__device__ __forceinline__ uint32_t tile_off(int r, int k) {
  return (uint32_t)((r >> 3) * 512 + (k >> 4) * 128 + (r & 7) * 16 + (k & 15));
}

// Shared-memory matrix descriptor: start address, leading (K) and stride (M / N) byte offsets,
// descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)(128 >> 4) << 16) |
         ((uint64_t)(512 >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::f8f6f4: fp32 accumulator, A and B e4m3, both K-major,
// N = 256, M = 128.
constexpr uint32_t kIdesc =
    (1u << 4) | ((uint32_t)(kMmaN >> 3) << 17) | ((uint32_t)(kMmaM >> 4) << 24);

// 16 bits of a descriptor as 16 bytes of value `one` (bit set) or 0, in bit order.
__device__ __forceinline__ uint4 expand16(uint32_t bits, uint32_t one) {
  uint4 r;
  r.x = ((((bits >> 0) & 15u) * 0x00204081u) & 0x01010101u) * one;
  r.y = ((((bits >> 4) & 15u) * 0x00204081u) & 0x01010101u) * one;
  r.z = ((((bits >> 8) & 15u) * 0x00204081u) & 0x01010101u) * one;
  r.w = ((((bits >> 12) & 15u) * 0x00204081u) & 0x01010101u) * one;
  return r;
}

// 32 consecutive accumulator columns of the warp's 32 lanes (lane l: row lane base + l).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, "
      "%12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, "
      "%30, %31}, [%32];"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
        "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]),
        "=r"(v[14]), "=r"(v[15]), "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]),
        "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]),
        "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(taddr));
}

// Polls the mbarrier at `bar` until the phase of parity `par` has completed; false after
// kSpinLimit polls, or earlier once another role has given up (*abort set; abort == nullptr: no
// early end).
__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t par, volatile int* abort) {
  for (uint32_t it = 0; it < kSpinLimit; it++) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        "selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(bar), "r"(par), "r"(kSuspendNs)
        : "memory");
    if (done) return true;
    if (abort && *abort) return false;
  }
  return false;
}
__device__ __forceinline__ void bar_arrive(uint32_t bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void give_up(const Problem& pb, volatile int* abort) {
  *abort = 1;
  if (pb.fault) atomicCAS(pb.fault, 0u, 8u);
}

// Tile t of the pair: row y, left pixels x0 .. x0 + 127.
struct TilePos {
  int y, x0;
};
__device__ __forceinline__ TilePos tile_pos(int t, int ntx) {
  const int y = t / ntx;
  return {y, (t - y * ntx) * kCostTX};
}

// bpe: bytes per aggregated sum (2, or 4 when wide)
template <int D>
__global__ void __launch_bounds__(MmaWarps<D>::kThreads, 1) cost_mma_kernel(Problem pb, int bpe) {
  constexpr int kEpiWarps = MmaWarps<D>::kEpiWarps, kEpiThreads = MmaWarps<D>::kEpiThreads;
  constexpr int kMmaWarp = MmaWarps<D>::kMmaWarp;
  extern __shared__ __align__(1024) uint8_t msm[];
  const int W = pb.W;
  const int ntx = (W + kCostTX - 1) / kCostTX;
  const int ntiles = pb.H * ntx;
  const int t0 = (int)((int64_t)ntiles * blockIdx.x / gridDim.x);
  const int t1 = (int)((int64_t)ntiles * (blockIdx.x + 1) / gridDim.x);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t sbase = (uint32_t)__cvta_generic_to_shared(msm);
  // mbarriers: full[2], empty[2] (operand stages), tfull[2], tempty[2] (accumulators)
  const uint32_t bars = sbase + kBarOff;
  auto full = [&](int s) { return bars + 8u * s; };
  auto empty = [&](int s) { return bars + 16u + 8u * s; };
  auto tfull = [&](int b) { return bars + 32u + 8u * b; };
  auto tempty = [&](int b) { return bars + 48u + 8u * b; };
  volatile int* abort = reinterpret_cast<volatile int*>(msm + kBarOff + 72);
  const uint64_t* ctl = pb.ct;
  const uint64_t* ctr = pb.ct + (int64_t)W * pb.H;

  if (warp == kMmaWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     bars + 64),
                 "r"(kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < 2; s++) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(full(s)), "r"(kProdThreads));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(empty(s)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tfull(s)));
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(tempty(s)), "r"(kEpiThreads));
    }
    *abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *reinterpret_cast<volatile uint32_t*>(msm + kBarOff + 64);

  if (warp >= kEpiWarps && warp < kMmaWarp) {
    // ---------------------------------------------------------------- producers
    // thread pt expands chunks c0, c0 + 1 (c0 = 2 (pt & 1)) of row pt / 2 of A and of rows
    // pt / 2, pt / 2 + 128 of B; the three descriptors of the next tile are loaded while this one
    // is expanded
    static_assert(kProdThreads == 2 * kMmaM, "two producer threads per row of A");
    const int pt = threadIdx.x - kEpiThreads, pr = pt >> 1, c0 = 2 * (pt & 1);
    auto fetch = [&](int t, uint64_t (&d)[3]) {
      const TilePos tp = tile_pos(t, ntx);
      const int xa = tp.x0 + pr, xb = tp.x0 - kMmaM + pr;
      d[0] = xa < W ? ctl[(int64_t)tp.y * W + xa] : 0ull;
      d[1] = xb >= 0 ? ctr[(int64_t)tp.y * W + xb] : 0ull;
      d[2] = xa < W ? ctr[(int64_t)tp.y * W + xa] : 0ull;
    };
    uint64_t nxt[3] = {0, 0, 0};
    if (t0 < t1) fetch(t0, nxt);
    for (int t = t0, i = 0; t < t1; t++, i++) {
      const int s = i & 1;
      uint64_t cur[3] = {nxt[0], nxt[1], nxt[2]};
      if (t + 1 < t1) fetch(t + 1, nxt);
      if (!bar_wait(empty(s), ((i >> 1) & 1) ^ 1, abort)) {
        give_up(pb, abort);
        break;
      }
      const TilePos tp = tile_pos(t, ntx);
      uint8_t* stage = msm + s * kStageBytes;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        const bool is_a = k == 0;
        const int j = k == 2 ? pr + kMmaM : pr;  // row of its tile
        const uint64_t dsc = cur[k];             // 0 outside the image
        uint8_t* base = stage + (is_a ? 0 : kTileA);
#pragma unroll
        for (int cc = 0; cc < 2; cc++) {
          const int c = c0 + cc;
          uint4 v = expand16((uint32_t)(dsc >> (16 * c)) & 0xFFFFu, is_a ? 0xC0u : 0x38u);
          // bytes 62, 63: 1, 1 in A; h, l of |b| in B (rows outside the image give entries
          // that are not used: x >= W is not stored, x - d < 0 is 255)
          if (c == 3) {
            if (is_a) {
              v.w |= 0x38380000u;
            } else {
              const uint32_t nb = (uint32_t)__popcll(dsc);
              v.w |= (e4m3_small_int(nb & 56u) << 16) | (e4m3_small_int(nb & 7u) << 24);
            }
          }
          *reinterpret_cast<uint4*>(base + tile_off(j, 16 * c)) = v;
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      bar_arrive(full(s));
      // the tile's aggregated sums start at 0, its right-disparity keys at their maximum
      const int npx = min(kCostTX, W - tp.x0);
      const int nv = npx * D * bpe / 16;
      uint4* z = reinterpret_cast<uint4*>(reinterpret_cast<uint8_t*>(pb.agg) +
                                          ((int64_t)tp.y * W + tp.x0) * D * bpe);
      for (int k = pt; k < nv; k += kProdThreads) z[k] = make_uint4(0, 0, 0, 0);
      for (int k = pt; k < npx; k += kProdThreads)
        pb.kr[(int64_t)tp.y * W + tp.x0 + k] = 0xFFFFFFFFu;
    }
  } else if (warp == kMmaWarp) {
    // ---------------------------------------------------------------- MMA issue
    if (lane == 0) {
      int issued = 0;  // tiles whose MMAs were issued
      for (int t = t0, i = 0; t < t1; t++, i++) {
        const int s = i & 1;
        const uint32_t par = (i >> 1) & 1;
        if (!bar_wait(full(s), par, abort) || !bar_wait(tempty(s), par ^ 1, abort)) {
          give_up(pb, abort);
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = sbase + s * kStageBytes, b0 = a0 + kTileA;
        const uint32_t acc = tmem + (uint32_t)(s * kMmaN);
#pragma unroll
        for (int k = 0; k < kMmaK / 32; k++)
          asm volatile(
              "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
              "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}" ::"r"(acc),
              "l"(smem_desc(a0 + k * 256)), "l"(smem_desc(b0 + k * 256)), "r"(kIdesc), "r"(k));
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                empty(s)));
        asm volatile(
            "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                tfull(s)));
        issued = i + 1;
      }
      // the tensor memory is freed below: wait for the last MMAs to complete, also when another
      // role gave up before reading them (their phase has completed already otherwise)
      if (issued > 0 && !bar_wait(tfull((issued - 1) & 1), ((issued - 1) >> 1) & 1, nullptr))
        give_up(pb, abort);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- epilogue
    // TMEM lanes 32 q .. 32 q + 31 (tile rows), disparities dh0 .. dh0 + DH - 1
    constexpr int DH = MmaWarps<D>::kDh, NP = MmaWarps<D>::kNp, NQ = DH / 4;
    static_assert(NP % 8 == 0 && DH % 32 == 0, "32-column loads at multiples of 32");
    const int q = warp & 3, h = warp >> 2;
    const int ti = 32 * q + lane, dh0 = h * DH;
    const int ca = 32 * q + kMmaM - dh0 - DH;  // first column read: offset o <-> column ca + o
    // row ti, column j holds x' = x0 - 128 + j, i.e. d = ti + 128 - j; lane l needs offsets
    // l + 1 .. l + DH: its packed row P shifted left by s = l + 1 bytes, taken through its row of
    // the warp's shift buffer (word shift ws, then a funnel shift of bs bits)
    const int sh = lane + 1, bs = 8 * (sh & 3), ws = sh >> 2;
    uint32_t* row = reinterpret_cast<uint32_t*>(msm + kShiftOff) +
                    (warp * 32 + lane) * MmaWarps<D>::kRow;
    row[NP] = 0;
    // |a| of the lane's pixel, loaded one tile ahead
    auto popa = [&](int t) {
      const TilePos tp = tile_pos(t, ntx);
      return (uint32_t)__popcll(ctl[(int64_t)tp.y * W + min(tp.x0 + ti, W - 1)]);
    };
    uint32_t la_next = t0 < t1 ? popa(t0) : 0u;
    for (int t = t0, i = 0; t < t1; t++, i++) {
      const int b = i & 1;
      const TilePos tp = tile_pos(t, ntx);
      const int x = tp.x0 + ti;
      const float bias = (float)la_next + 8388608.0f;  // + 2^23: the low byte is the sum
      if (t + 1 < t1) la_next = popa(t + 1);
      // the lanes leave together: the tensor-memory loads below are warp-wide
      if (!__all_sync(0xFFFFFFFFu, bar_wait(tfull(b), (i >> 1) & 1, abort))) {
        give_up(pb, abort);
        break;
      }
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
#pragma unroll
      for (int c = 0; c < NP / 8; c++) {  // columns ca + 32 c .. + 31 (ca is a multiple of 32)
        uint32_t v[32];
        tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kMmaN + ca + 32 * c), v);
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (c == NP / 8 - 1) {  // the accumulator is free for the MMA of tile i + 2
          asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
          bar_arrive(tempty(b));
        }
#pragma unroll
        for (int k = 0; k < 8; k++) {
          const uint32_t b0 = __float_as_uint(__uint_as_float(v[4 * k + 0]) + bias);
          const uint32_t b1 = __float_as_uint(__uint_as_float(v[4 * k + 1]) + bias);
          const uint32_t b2 = __float_as_uint(__uint_as_float(v[4 * k + 2]) + bias);
          const uint32_t b3 = __float_as_uint(__uint_as_float(v[4 * k + 3]) + bias);
          row[8 * c + k] =
              __byte_perm(__byte_perm(b0, b1, 0x0040), __byte_perm(b2, b3, 0x0040), 0x5410);
        }
      }
      __syncwarp();
      // output word k (d = dh0 + 4k .. + 3): the four bytes at offsets s + 4 (NQ - 1 - k) ..,
      // reversed
      uint32_t o[NQ];
      uint32_t w1 = row[ws + NQ];
#pragma unroll
      for (int n = NQ - 1; n >= 0; n--) {
        const uint32_t w0 = row[ws + n];
        o[NQ - 1 - n] = __byte_perm(__funnelshift_r(w0, w1, bs), 0, 0x0123);
        w1 = w0;
      }
      __syncwarp();  // the row is rewritten for the next tile
      if (x < dh0 + DH - 1) {  // d > x: outside the right image
#pragma unroll
        for (int k = 0; k < NQ; k++) {
          const int nv = x - dh0 - 4 * k + 1;  // valid bytes of word k
          if (nv <= 0)
            o[k] = 0xFFFFFFFFu;
          else if (nv < 4)
            o[k] |= 0xFFFFFFFFu << (8 * nv);
        }
      }
      if (x < W) {
        uint4* dst = reinterpret_cast<uint4*>(pb.cost + ((int64_t)tp.y * W + x) * D + dh0);
#pragma unroll
        for (int k = 0; k < NQ / 4; k++)
          dst[k] = make_uint4(o[4 * k], o[4 * k + 1], o[4 * k + 2], o[4 * k + 3]);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == kMmaWarp) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(kTmemCols));
  }
}

int g_sms = 0;  // SMs of the device (one persistent block each)

template <int D>
cudaError_t launch_t(const Problem& pb, int bpe, cudaStream_t s) {
  if (g_sms == 0) {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    g_sms = n > 0 ? n : 1;
  }
  cudaFuncSetAttribute(cost_mma_kernel<D>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                       kSmemRequest);
  const int grid = std::min(g_sms, cost_items(pb.W, pb.H));
  cost_mma_kernel<D><<<grid, MmaWarps<D>::kThreads, kSmemRequest, s>>>(pb, bpe);
  return cudaGetLastError();
}

static_assert(MmaWarps<128>::kSmemUsed <= kSmemRequest && MmaWarps<64>::kSmemUsed <= kSmemRequest,
              "shared memory");

}  // namespace

bool cost_mma_ok(const Problem& pb, const Method& mt) {
  return mt.cw == 9 && mt.ch == 7 && !(mt.flags & 8) && (pb.D == 64 || pb.D == 128);
}

cudaError_t launch_cost_mma(const Problem& pb, const Method& mt, cudaStream_t s) {
  const int bpe = mt.wide ? 4 : 2;
  return pb.D == 128 ? launch_t<128>(pb, bpe, s) : launch_t<64>(pb, bpe, s);
}

}  // namespace r2t
