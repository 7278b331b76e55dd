// sweep.cuh -- device building blocks shared by the sweep, min-marginal and
// adjoint kernels: per-warp shared-memory staging of one tile and the
// per-lane min-sum passes over one BDD.
//
// Execution model: one warp owns one tile of up to 32 BDDs and lane b owns
// BDD b.  A lane walks its BDD level by level (App. B: SP(root, v) and
// SP(v, top) by min-sum over the 0- and 1-arcs).  Everything a tile holds is
// interleaved by lane (element 32 n + b belongs to lane b), so the 32 lanes of
// a warp always touch 32 different shared-memory banks and read global memory
// in coalesced segments.  Node numbers 0 and 1 are the top (cost 0) and
// bottom (cost +inf) terminals, so arcs into terminals need no branch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_internal.h"

namespace dg {

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

__device__ __forceinline__ int desc_width(uint32_t ds) { return (int)(ds >> 8); }
__device__ __forceinline__ int desc_first(uint32_t ds) { return (int)(ds & 0xFFu); }

// Shared-memory image of one tile (one warp's slice).
struct TileSmem {
  float* full;     // [32 * nmax] costs of the first pass (all levels), lane-interleaved
  float* ring;     // [32 * ring] costs of the sweep direction, two levels live
  float* lam;      // [32 * nh]
  float* sg;       // [32 * nh] averaging term of the slot's variable
  float* om;       // [32 * nh] omega_ij (mode 1)
  float* al;       // [32 * nh] alpha_ij (mode 1)
  uint16_t* desc;  // [32 * nh]
  uint16_t* code;       // child codes, biased: element 32 n + lane is node number n
  uint16_t* code_base;  // [32 * (nmax - 2)] the staged codes of nodes 2 .. nmax-1
  uint16_t* meta;       // recording sweeps: argmin record per node, biased like code
  int nmax, nh, rmask;
};

// RING: the sweep-direction costs live in a ring of T.ring node numbers;
// otherwise in a second whole array (s.ring then indexed by node number).
// REC: an argmin record per node follows the child codes.
template <int MODE, bool RING, bool REC = false>
__device__ __forceinline__ TileSmem carve(unsigned char* p, const Tile& T) {
  TileSmem s;
  s.nmax = T.nmax;
  s.nh = T.nhops;
  const int ns = s.nh * kWarp;
  s.rmask = T.ring - 1;
  s.full = (float*)p;
  p += (size_t)s.nmax * kWarp * 4;
  s.ring = (float*)p;
  p += (size_t)(RING ? T.ring : s.nmax) * kWarp * 4;
  s.lam = (float*)p;
  p += (size_t)ns * 4;
  s.sg = (float*)p;
  p += (size_t)ns * 4;
  if (MODE == 1) {
    s.om = (float*)p;
    p += (size_t)ns * 4;
    s.al = (float*)p;
    p += (size_t)ns * 4;
  } else {
    s.om = s.al = nullptr;
  }
  s.desc = (uint16_t*)p;
  p += (size_t)ns * 2;
  s.code_base = (uint16_t*)p;
  s.code = s.code_base - 2 * kWarp;
  s.meta = REC ? s.code + (size_t)(s.nmax - 2) * kWarp : nullptr;
  return s;
}

// Argmin record of node number n >= 2 (recording sweeps).
#define DG_META(s, n) (s).meta[(n) * kWarp + lane]
constexpr uint32_t kHiChoice = 1u << 9;  // SP(v, top) leaves v by its 1-arc
constexpr uint32_t kInHi = 1u << 8;      // SP(root, v) enters v by a 1-arc

// Cost arrays of lane `lane`: DG_F is the element of node number n in the
// first-pass array (numbers 0 and 1 hold the terminal costs 0 and +inf);
// DG_R the ring element of node number n >= 2 (the two live levels always
// occupy fewer than `ring` consecutive node numbers).
#define DG_F(s, n) (s).full[(n) * kWarp + lane]
#define DG_R(s, n) (s).ring[(((int)(n)) & (s).rmask) * kWarp + lane]
// second whole array (backward sweeps): element of node number n
#define DG_W(s, n) (s).ring[(n) * kWarp + lane]

// Child codes (lo | hi << 8) of node number n >= 2 of my BDD.
__device__ __forceinline__ uint32_t node_code(const uint16_t* code, int n, int lane) {
  return code[n * kWarp + lane];
}
__device__ __forceinline__ uint32_t node_code(const TileSmem& s, int n, int lane) {
  return node_code(s.code, n, lane);
}

// L2 eviction priority of the staged tile arrays: a sweep streams them
// through L2 once, several times the L2's size, so they are marked
// evict_first and leave the lines the sweep writes (lambda and M, which the S
// reduction after it reads) in place.
__device__ __forceinline__ uint64_t l2_evict_first() {
  uint64_t p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}

// Asynchronous 16-byte global -> shared copy (cp.async) with an L2 policy.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, uint64_t pol) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void copy_async(void* dst, const void* src, int bytes, int lane) {
  char* d = reinterpret_cast<char*>(dst);
  const char* g = reinterpret_cast<const char*>(src);
  const uint64_t pol = l2_evict_first();
  for (int o = lane * 16; o < bytes; o += kWarp * 16) cp_async16(d + o, g + o, pol);
}

// Warp-cooperative staging of the tile: child codes, slot descriptors,
// lambda and, with WITH_S, the averaging term of every slot (A.slot_avg, as
// the S reduction before the sweep left it) plus omega and alpha in mode 1,
// all by asynchronous copies; returns once they have landed.  With costs
// non-null, the costs of nodes 2 .. nmax-1 (per node and lane, in the layout
// of the child codes) are staged into s.full as well.
template <bool WITH_S, int MODE>
__device__ __forceinline__ void load_tile(const DevArena& A, const Tile& T, TileSmem& s, const float* lam,
                                          const float* omega, const float* alpha, int lane,
                                          const float* costs = nullptr) {
  const int ns = s.nh * kWarp;
  copy_async(s.code_base, A.lohi8 + T.node_base, (s.nmax - 2) * kWarp * 2, lane);
  if (costs) copy_async(s.full + 2 * kWarp, costs + T.node_base, (s.nmax - 2) * kWarp * 4, lane);
  copy_async(s.desc, A.desc + T.slot_base, ns * 2, lane);
  copy_async(s.lam, lam + T.slot_base, ns * 4, lane);
  if (WITH_S) {
    copy_async(s.sg, A.slot_avg + T.slot_base, ns * 4, lane);
    if (MODE == 1) {
      copy_async(s.om, omega + T.slot_base, ns * 4, lane);
      copy_async(s.al, alpha + T.slot_base, ns * 4, lane);
    }
  }
  cp_async_commit();
  DG_F(s, kTopCode) = 0.0f;
  DG_F(s, kBotCode) = f_inf();
  cp_async_wait_all();
  __syncwarp();
}

// Writes the costs of nodes 2 .. nmax-1 held in `src` (a lane-interleaved
// cost array of the tile's shared memory) to dst, in the layout load_tile
// reads them back in: one bulk asynchronous copy (TMA engine) issued by lane
// 0, which waits for its completion before the warp's shared memory can go.
// Both addresses are 16-byte aligned (slices start on 128 bytes, node_base
// is a multiple of 32) and the size is a multiple of 128 bytes.
__device__ __forceinline__ void store_costs(float* dst, const float* src, int nmax, int lane) {
  // the lanes' shared-memory stores, ordered before the async proxy reads them
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncwarp();
  if (lane == 0) {
    const unsigned s = (unsigned)__cvta_generic_to_shared(src + 2 * kWarp);
    const unsigned bytes = (unsigned)(nmax - 2) * kWarp * 4u;
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(dst), "r"(s), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
  }
}

// The term a sweep adds to lambda_ij of slot q: alpha_ij * S_i.
template <int MODE>
__device__ __forceinline__ float slot_avg(const TileSmem& s, int q) {
  return MODE == 1 ? s.al[q] * s.sg[q] : s.sg[q];
}

// SP(v, top) of every node of my BDD under s.lam into s.full (levels
// bottom-up).
__device__ __forceinline__ void lane_cost_to_top(TileSmem& s, int lane) {
  for (int h = s.nh - 1; h >= 0; --h) {
    const uint32_t ds = s.desc[h * kWarp + lane];
    const int w = desc_width(ds);
    if (w == 0) continue;
    const int fn = desc_first(ds);
    const float l = s.lam[h * kWarp + lane];
    #pragma unroll 2
    for (int r = 0; r < w; ++r) {
      const int n = fn + r;
      const uint32_t c = node_code(s, n, lane);
      DG_F(s, n) = fminf(DG_F(s, c & 0xFFu), l + DG_F(s, c >> 8));
    }
  }
}

// lane_cost_to_top that also records per node whether the minimum leaves by
// the 1-arc (kHiChoice; the 0-arc wins ties), the rest of the record cleared.
__device__ __forceinline__ void lane_cost_to_top_rec(TileSmem& s, int lane) {
  for (int h = s.nh - 1; h >= 0; --h) {
    const uint32_t ds = s.desc[h * kWarp + lane];
    const int w = desc_width(ds);
    if (w == 0) continue;
    const int fn = desc_first(ds);
    const float l = s.lam[h * kWarp + lane];
    #pragma unroll 2
    for (int r = 0; r < w; ++r) {
      const int n = fn + r;
      const uint32_t c = node_code(s, n, lane);
      const float tl = DG_F(s, c & 0xFFu), th = l + DG_F(s, c >> 8);
      const bool take0 = (c & 0xFFu) != kBotCode && tl <= th;
      DG_F(s, n) = take0 ? tl : th;
      DG_META(s, n) = take0 ? 0 : kHiChoice;
    }
  }
}

// SP(root, v) of every node of my BDD under s.lam into s.full (levels
// top-down).
__device__ __forceinline__ void lane_cost_from_root(TileSmem& s, int lane) {
  if (desc_width(s.desc[lane]) == 0) return;
  DG_F(s, 2) = 0.0f;
  for (int h = 0; h + 1 < s.nh; ++h) {
    const uint32_t ds = s.desc[h * kWarp + lane];
    const uint32_t dn = s.desc[(h + 1) * kWarp + lane];
    const int w = desc_width(ds), wn = desc_width(dn);
    if (wn == 0) break;
    const int fn = desc_first(ds), fnn = desc_first(dn);
    const float l = s.lam[h * kWarp + lane];
    #pragma unroll 2
    for (int r = 0; r < wn; ++r) DG_F(s, fnn + r) = f_inf();
    #pragma unroll 2
    for (int r = 0; r < w; ++r) {
      const int n = fn + r;
      const uint32_t c = node_code(s, n, lane);
      const uint32_t lo = c & 0xFFu, hi = c >> 8;
      const float dv = DG_F(s, n);
      // arcs into the bottom terminal write its entry, which this pass never reads
      DG_F(s, lo) = fminf(DG_F(s, lo), dv);
      DG_F(s, hi) = fminf(DG_F(s, hi), dv + l);
    }
  }
}

// lane_cost_from_root that also records per node its argmin in-arc: the
// parent's node number | kInHi for a 1-arc; the first strictly smaller
// candidate wins (parents in node order, the 0-arc before the 1-arc).
__device__ __forceinline__ void lane_cost_from_root_rec(TileSmem& s, int lane) {
  if (desc_width(s.desc[lane]) == 0) return;
  DG_F(s, 2) = 0.0f;
  DG_META(s, 2) = 0;
  for (int h = 0; h + 1 < s.nh; ++h) {
    const uint32_t ds = s.desc[h * kWarp + lane];
    const uint32_t dn = s.desc[(h + 1) * kWarp + lane];
    const int w = desc_width(ds), wn = desc_width(dn);
    if (wn == 0) break;
    const int fn = desc_first(ds), fnn = desc_first(dn);
    const float l = s.lam[h * kWarp + lane];
    #pragma unroll 2
    for (int r = 0; r < wn; ++r) DG_F(s, fnn + r) = f_inf();
    #pragma unroll 2
    for (int r = 0; r < w; ++r) {
      const int n = fn + r;
      const uint32_t c = node_code(s, n, lane);
      const uint32_t lo = c & 0xFFu, hi = c >> 8;
      const float dv = DG_F(s, n);
      if (lo >= 2 && dv < DG_F(s, lo)) {
        DG_F(s, lo) = dv;
        DG_META(s, lo) = (uint16_t)n;
      }
      if (hi >= 2 && dv + l < DG_F(s, hi)) {
        DG_F(s, hi) = dv + l;
        DG_META(s, hi) = (uint16_t)(n | kInHi);
      }
    }
  }
}

}  // namespace dg
