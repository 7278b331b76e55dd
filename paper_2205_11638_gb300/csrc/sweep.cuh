// sweep.cuh -- device building blocks shared by the sweep, min-marginal and
// adjoint kernels: shared-memory tile staging, warp-segmented reductions over
// BDD levels and the per-hop min-sum passes.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "dg_internal.h"

namespace dg {

constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ float f_inf() { return __int_as_float(0x7f800000); }

// Monotone map float -> int so that shared-memory atomicMin on ints is a min
// on floats (no NaNs occur: bottom arcs are skipped, never added).
__device__ __forceinline__ int ford(float f) {
  int i = __float_as_int(f);
  return i >= 0 ? i : i ^ 0x7FFFFFFF;
}
__device__ __forceinline__ float funord(int i) { return __int_as_float(i >= 0 ? i : i ^ 0x7FFFFFFF); }

__device__ __forceinline__ unsigned lanemask_le(int lane) { return kFull >> (31 - lane); }

// Lane of the first node of my level inside the warp row.
__device__ __forceinline__ int head_lane(unsigned head, int lane) { return 31 - __clz(head & lanemask_le(lane)); }

// Tile-local slot of the level my lane belongs to.
__device__ __forceinline__ int lane_slot(const RowMeta& rm, int lane) {
  return (int)(rm.info & 0xFFFFu) + __popc(rm.head & lanemask_le(lane)) - 1;
}
__device__ __forceinline__ int row_valid(const RowMeta& rm) { return (int)(rm.info >> 16); }

// Segmented min towards the first lane of every level: after the call the
// head lane of a level holds the min over the level's lanes.  `width_pow`
// bounds the level width (power of two >= widest level of the tile).
__device__ __forceinline__ void seg_min2(float& a, float& b, unsigned head, int lane, int width_pow) {
  const unsigned long long hm = (unsigned long long)head | (1ull << 32);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    if (off >= width_pow) break;
    float oa = __shfl_down_sync(kFull, a, off);
    float ob = __shfl_down_sync(kFull, b, off);
    unsigned long long between = (hm >> (lane + 1)) & ((1ull << off) - 1ull);
    if (between == 0ull) {
      a = fminf(a, oa);
      b = fminf(b, ob);
    }
  }
}

// Segmented sum towards the head lane (same segments as seg_min2); the sum
// order is fixed by the layout, so the result is deterministic.
__device__ __forceinline__ float seg_sum(float a, unsigned head, int lane, int width_pow) {
  const unsigned long long hm = (unsigned long long)head | (1ull << 32);
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    if (off >= width_pow) break;
    float o = __shfl_down_sync(kFull, a, off);
    unsigned long long between = (hm >> (lane + 1)) & ((1ull << off) - 1ull);
    if (between == 0ull) a += o;
  }
  return a;
}

__device__ __forceinline__ int pow2_ceil(int w) {
  int p = 1;
  while (p < w) p <<= 1;
  return p;
}

__device__ __forceinline__ uint32_t hop_rows(const uint32_t* s_hop, int h) { return s_hop[h] & 0xFFFFu; }
__device__ __forceinline__ uint32_t hop_slots(const uint32_t* s_hop, int h) { return s_hop[h] >> 16; }

// Shared-memory image of one tile.
struct TileSmem {
  uint32_t* lohi;  // [nn]
  float* t;        // [nn] SP(v, top)
  int* d;          // [nn] SP(root, v) as ordered ints
  RowMeta* meta;   // [nrows]
  uint32_t* hop;   // [nhops + 1]
  float* lam;      // [ns]
  float* as;       // [ns] alpha_ij * S_i  (sweeps) / scratch
  float* M;        // [ns] M out / m0 / seeds
  float* om;       // [ns] omega per slot (mode 1) / m1
  int nn, ns, nrows, nhops, wpow;
};

__device__ __forceinline__ TileSmem carve(unsigned char* smem, const Tile& T) {
  TileSmem s;
  s.nn = T.nrows * kWarp;
  s.ns = T.nslots;
  s.nrows = T.nrows;
  s.nhops = T.nhops;
  s.wpow = pow2_ceil(T.maxw);
  unsigned char* p = smem;
  s.lohi = (uint32_t*)p;
  p += (size_t)s.nn * 4;
  s.t = (float*)p;
  p += (size_t)s.nn * 4;
  s.d = (int*)p;
  p += (size_t)s.nn * 4;
  s.lam = (float*)p;
  p += (size_t)s.ns * 4;
  s.as = (float*)p;
  p += (size_t)s.ns * 4;
  s.M = (float*)p;
  p += (size_t)s.ns * 4;
  s.om = (float*)p;
  p += (size_t)s.ns * 4;
  s.meta = (RowMeta*)p;
  p += (size_t)s.nrows * 8;
  s.hop = (uint32_t*)p;
  return s;
}

// Stages the structure of tile T (child indices, row metadata, hop table).
__device__ __forceinline__ void load_structure(const DevArena& A, const Tile& T, TileSmem& s) {
  const uint4* src = reinterpret_cast<const uint4*>(A.lohi + (size_t)T.row_base * kWarp);
  uint4* dst = reinterpret_cast<uint4*>(s.lohi);
  for (int i = threadIdx.x; i < s.nn / 4; i += blockDim.x) dst[i] = __ldg(src + i);
  const uint2* msrc = reinterpret_cast<const uint2*>(A.rows + T.row_base);
  uint2* mdst = reinterpret_cast<uint2*>(s.meta);
  for (int i = threadIdx.x; i < s.nrows; i += blockDim.x) mdst[i] = __ldg(msrc + i);
  for (int i = threadIdx.x; i <= s.nhops; i += blockDim.x) s.hop[i] = __ldg(A.hoptab + T.hop_base + i);
}

__device__ __forceinline__ float child_cost(const float* t, uint32_t c) {
  return c == kTop ? 0.0f : t[c];
}

// SP(v, top) for every node of the tile under s.lam (levels bottom-up).
__device__ __forceinline__ void pass_cost_to_top(TileSmem& s) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int h = s.nhops - 1; h >= 0; --h) {
    const int r0 = hop_rows(s.hop, h), r1 = hop_rows(s.hop, h + 1);
    for (int r = r0 + warp; r < r1; r += nw) {
      const RowMeta rm = s.meta[r];
      if (lane < row_valid(rm)) {
        const int v = r * kWarp + lane;
        const uint32_t lh = s.lohi[v];
        const uint32_t lo = lh & 0xFFFFu, hi = lh >> 16;
        float best = f_inf();
        if (lo != kBot) best = child_cost(s.t, lo);
        if (hi != kBot) best = fminf(best, s.lam[lane_slot(rm, lane)] + child_cost(s.t, hi));
        s.t[v] = best;
      }
    }
    __syncthreads();
  }
}

// d = ordered(+inf) everywhere, 0 at the roots (the nodes of hop 0).
__device__ __forceinline__ void init_from_root(TileSmem& s) {
  const int nroot = hop_rows(s.hop, 1) * kWarp;
  const int zero = ford(0.0f), inf = ford(f_inf());
  for (int v = threadIdx.x; v < s.nn; v += blockDim.x) s.d[v] = v < nroot ? zero : inf;
  __syncthreads();
}

// SP(root, v) for every node under s.lam (levels top-down, push relaxation).
__device__ __forceinline__ void pass_cost_from_root(TileSmem& s) {
  init_from_root(s);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int h = 0; h + 1 < s.nhops; ++h) {
    const int r0 = hop_rows(s.hop, h), r1 = hop_rows(s.hop, h + 1);
    for (int r = r0 + warp; r < r1; r += nw) {
      const RowMeta rm = s.meta[r];
      if (lane < row_valid(rm)) {
        const int v = r * kWarp + lane;
        const uint32_t lh = s.lohi[v];
        const uint32_t lo = lh & 0xFFFFu, hi = lh >> 16;
        const float dv = funord(s.d[v]);
        if (lo < kTop) atomicMin(&s.d[lo], ford(dv));
        if (hi < kTop) atomicMin(&s.d[hi], ford(dv + s.lam[lane_slot(rm, lane)]));
      }
    }
    __syncthreads();
  }
}

}  // namespace dg
