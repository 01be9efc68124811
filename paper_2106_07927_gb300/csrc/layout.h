// Scratch layout of one pair: byte offsets of every buffer inside one allocation (host code).
#pragma once
#include <stddef.h>
#include <string.h>

#include "common.cuh"

namespace r2t {

struct Layout {
  size_t cost, ct, agg, dl, dr, kr, mask, flip, dp, nst, nsv, fault, total;  // 0: buffer not used
};

inline size_t align256(size_t v) { return (v + 255) / 256 * 256; }

// Cost 1 B/DE, aggregated volume 2 B/DE (4 when wide), census descriptors of both images
// 16 B/px, D^L and D^R 2 B/px each, right-disparity keys 4 B/px, LR mask 1 B/px: 3 B per DE +
// 25 B per pixel. The exact
// consistency check adds the swapped, flipped pair (2 B/px) and its D^L (2 B/px); the NCC cost
// the patch statistics of both images (16 B/px) and their exact patch variances (8 B/px).
inline Layout layout_for(int W, int H, int D, bool wide, bool exact = false, bool ncc = false) {
  const size_t npx = (size_t)W * H, nde = npx * D;
  Layout l;
  size_t o = 0;
  l.cost = o; o = align256(o + nde);
  l.ct = o; o = align256(o + npx * 16);
  l.agg = o; o = align256(o + nde * (wide ? 4 : 2));
  l.dl = o; o = align256(o + npx * 2);
  l.dr = o; o = align256(o + npx * 2);
  l.kr = o; o = align256(o + npx * 4);
  l.mask = o; o = align256(o + npx);
  l.fault = o; o = align256(o + 16);  // range-check record of the debug build
  l.flip = l.dp = 0;
  if (exact) {
    l.flip = o; o = align256(o + npx * 2);
    l.dp = o; o = align256(o + npx * 2);
  }
  l.nst = l.nsv = 0;
  if (ncc) {  // 2 KB of slack in front (reads at a matching pixel x - d < 0 stay inside)
    l.nst = o + 2048; o = align256(o + 2048 + npx * 16);
    l.nsv = o; o = align256(o + npx * 8);
  }
  l.total = o;
  return l;
}

inline Problem problem_at(char* base, const Layout& l, int W, int H, int D) {
  Problem pb;
  memset(&pb, 0, sizeof(pb));
  pb.W = W;
  pb.H = H;
  pb.D = D;
  pb.cost = reinterpret_cast<uint8_t*>(base + l.cost);
  pb.ct = reinterpret_cast<uint64_t*>(base + l.ct);
  pb.agg = base + l.agg;
  pb.dl = reinterpret_cast<uint16_t*>(base + l.dl);
  pb.dr = reinterpret_cast<uint16_t*>(base + l.dr);
  pb.kr = reinterpret_cast<uint32_t*>(base + l.kr);
  pb.mask = reinterpret_cast<uint8_t*>(base + l.mask);
  pb.disp_f = nullptr;
  pb.flip = l.flip ? reinterpret_cast<uint8_t*>(base + l.flip) : nullptr;
  pb.dp = l.dp ? reinterpret_cast<uint16_t*>(base + l.dp) : nullptr;
  pb.nst = l.nst ? reinterpret_cast<uint2*>(base + l.nst) : nullptr;
  pb.nsv = l.nsv ? reinterpret_cast<int32_t*>(base + l.nsv) : nullptr;
  pb.fault = reinterpret_cast<unsigned*>(base + l.fault);
  return pb;
}

}  // namespace r2t
