// kernels_sweep.cu -- the sweeps of Alg. 1 (generalized min-marginal
// averaging, Sec. 3.2 of DOGE-Train) over tiles of BDDs, plus the kernels
// that evaluate min-marginals, subproblem energies and minimising
// assignments on the same layout.
//
// One CTA owns one tile for the whole sweep: the tile's structure and slot
// state are staged in shared memory, the hop loop runs there (one thread per
// BDD node of the current hop, one warp segment per BDD level), and only the
// updated lambda and M go back to global memory.  The shortest-path costs of
// the direction opposite to the sweep (SP(.,T) for a forward sweep, SP(r,.)
// for a backward one) are recomputed from lambda inside the CTA instead of
// being kept in HBM between sweeps; they equal the values the previous sweep
// left, bit for bit, because the same FP32 operations run on the same inputs.
#include "kernels.h"
#include "sweep.cuh"

namespace dg {

template <int KIND>
__global__ void __launch_bounds__(512) k_sweep(DevArena A, SweepArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const Tile T = A.tiles[blockIdx.x];
  TileSmem s = carve(smem, T);
  load_structure(A, T, s);
  // slot state
  {
    const float4* lam4 = reinterpret_cast<const float4*>(a.lam + T.slot_base);
    const int4* var4 = reinterpret_cast<const int4*>(A.slot_var + T.slot_base);
    for (int q = threadIdx.x; q < s.ns / 4; q += blockDim.x) {
      float4 l = lam4[q];
      reinterpret_cast<float4*>(s.lam)[q] = l;
      reinterpret_cast<float4*>(s.M)[q] = make_float4(0.f, 0.f, 0.f, 0.f);
      if (KIND == kFwd || KIND == kBwd) {
        int4 v = __ldg(var4 + q);
        int vv[4] = {v.x, v.y, v.z, v.w};
        float as[4];
        float4 al = make_float4(0.f, 0.f, 0.f, 0.f);
        if (a.mode == 1) al = __ldg(reinterpret_cast<const float4*>(a.alpha + T.slot_base) + q);
        float alv[4] = {al.x, al.y, al.z, al.w};
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int var = vv[e];
          float w = 0.f;
          if (var >= 0) w = (a.mode == 1 ? alv[e] : __ldg(A.invdeg + var)) * A.S[var];
          as[e] = w;
        }
        reinterpret_cast<float4*>(s.as)[q] = make_float4(as[0], as[1], as[2], as[3]);
        if (a.mode == 1)
          reinterpret_cast<float4*>(s.om)[q] = __ldg(reinterpret_cast<const float4*>(a.omega + T.slot_base) + q);
      }
    }
  }
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;

  if (KIND == kFwd || KIND == kMinMarg) {
    // ---- SP(., T) under lambda at sweep start, then the forward sweep -----
    pass_cost_to_top(s);
    init_from_root(s);
    for (int h = 0; h < s.nhops; ++h) {
      const int r0 = hop_rows(s.hop, h), r1 = hop_rows(s.hop, h + 1);
      for (int r = r0 + warp; r < r1; r += nw) {
        const RowMeta rm = s.meta[r];
        const bool valid = lane < row_valid(rm);
        const int v = r * kWarp + lane;
        const uint32_t lh = valid ? s.lohi[v] : 0xFFFFFFFFu;
        const uint32_t lo = lh & 0xFFFFu, hi = lh >> 16;
        const int slot = lane_slot(rm, lane);
        const float dv = valid ? funord(s.d[v]) : f_inf();
        float a0 = lo != kBot ? dv + child_cost(s.t, lo) : f_inf();
        float a1 = hi != kBot ? dv + child_cost(s.t, hi) : f_inf();
        seg_min2(a0, a1, rm.head, lane, s.wpow);
        float lnew = 0.f;
        if (valid && ((rm.head >> lane) & 1u)) {
          const float l = s.lam[slot];
          const float m0 = a0, m1 = l + a1;
          if (KIND == kMinMarg) {
            s.M[slot] = m0;
            s.om[slot] = m1;
            lnew = l;
          } else {
            const float om = a.mode == 1 ? s.om[slot] : a.omega0;
            const float Mn = om * (m1 - m0);
            lnew = l - Mn + s.as[slot];
            s.lam[slot] = lnew;
            s.M[slot] = Mn;
          }
        }
        lnew = __shfl_sync(kFull, lnew, head_lane(rm.head, lane));
        if (valid && h + 1 < s.nhops) {
          if (lo < kTop) atomicMin(&s.d[lo], ford(dv));
          if (hi < kTop) atomicMin(&s.d[hi], ford(dv + lnew));
        }
      }
      __syncthreads();
    }
  } else if (KIND == kBwd) {
    // ---- SP(r, .) under lambda at sweep start, then the backward sweep ----
    pass_cost_from_root(s);
    for (int h = s.nhops - 1; h >= 0; --h) {
      const int r0 = hop_rows(s.hop, h), r1 = hop_rows(s.hop, h + 1);
      for (int r = r0 + warp; r < r1; r += nw) {
        const RowMeta rm = s.meta[r];
        const bool valid = lane < row_valid(rm);
        const int v = r * kWarp + lane;
        const uint32_t lh = valid ? s.lohi[v] : 0xFFFFFFFFu;
        const uint32_t lo = lh & 0xFFFFu, hi = lh >> 16;
        const int slot = lane_slot(rm, lane);
        const float dv = valid ? funord(s.d[v]) : f_inf();
        const float tl = lo != kBot ? child_cost(s.t, lo) : f_inf();
        const float th = hi != kBot ? child_cost(s.t, hi) : f_inf();
        float a0 = lo != kBot ? dv + tl : f_inf();
        float a1 = hi != kBot ? dv + th : f_inf();
        seg_min2(a0, a1, rm.head, lane, s.wpow);
        float lnew = 0.f;
        if (valid && ((rm.head >> lane) & 1u)) {
          const float l = s.lam[slot];
          const float m0 = a0, m1 = l + a1;
          const float om = a.mode == 1 ? s.om[slot] : a.omega0;
          const float Mn = om * (m1 - m0);
          lnew = l - Mn + s.as[slot];
          s.lam[slot] = lnew;
          s.M[slot] = Mn;
        }
        lnew = __shfl_sync(kFull, lnew, head_lane(rm.head, lane));
        if (valid) s.t[v] = fminf(tl, hi != kBot ? lnew + th : f_inf());
      }
      __syncthreads();
    }
  } else {
    // kEnergy / kSeed: SP(., T) under lambda
    pass_cost_to_top(s);
  }

  if (KIND == kSeed) {
    // walk the minimising path from every root: 0-arc on ties
    for (int v = threadIdx.x; v < s.nn; v += blockDim.x) s.d[v] = v < (int)hop_rows(s.hop, 1) * kWarp ? 1 : 0;
    __syncthreads();
    for (int h = 0; h < s.nhops; ++h) {
      const int r0 = hop_rows(s.hop, h), r1 = hop_rows(s.hop, h + 1);
      for (int r = r0 + warp; r < r1; r += nw) {
        const RowMeta rm = s.meta[r];
        const int v = r * kWarp + lane;
        if (lane < row_valid(rm) && s.d[v]) {
          const uint32_t lh = s.lohi[v];
          const uint32_t lo = lh & 0xFFFFu, hi = lh >> 16;
          const int slot = lane_slot(rm, lane);
          bool take0 = false;
          if (lo != kBot) take0 = hi == kBot || child_cost(s.t, lo) <= s.lam[slot] + child_cost(s.t, hi);
          s.M[slot] = take0 ? 0.f : 1.f;
          const uint32_t ch = take0 ? lo : hi;
          if (ch < kTop) s.d[ch] = 1;
        }
      }
      __syncthreads();
    }
  }

  if ((KIND == kBwd || KIND == kEnergy) && a.E != nullptr) {
    // hop-0 nodes are the roots; SP(root, T) = E^j
    const int r1 = hop_rows(s.hop, 1);
    for (int v = threadIdx.x; v < r1 * kWarp; v += blockDim.x) {
      const RowMeta rm = s.meta[v >> 5];
      const int ln = v & 31;
      if (ln < row_valid(rm)) {
        const int row = __ldg(A.slot_row + T.slot_base + lane_slot(rm, ln));
        a.E[row] = s.t[v];
      }
    }
  }

  // write back
  if (KIND == kFwd || KIND == kBwd) {
    float4* lam4 = reinterpret_cast<float4*>(a.lam + T.slot_base);
    float4* M4 = reinterpret_cast<float4*>(a.M + T.slot_base);
    for (int q = threadIdx.x; q < s.ns / 4; q += blockDim.x) {
      lam4[q] = reinterpret_cast<const float4*>(s.lam)[q];
      M4[q] = reinterpret_cast<const float4*>(s.M)[q];
    }
  } else if (KIND == kMinMarg) {
    float4* m0 = reinterpret_cast<float4*>(a.M + T.slot_base);
    float4* m1 = reinterpret_cast<float4*>(a.out2 + T.slot_base);
    for (int q = threadIdx.x; q < s.ns / 4; q += blockDim.x) {
      m0[q] = reinterpret_cast<const float4*>(s.M)[q];
      m1[q] = reinterpret_cast<const float4*>(s.om)[q];
    }
  } else if (KIND == kSeed) {
    float4* g = reinterpret_cast<float4*>(a.M + T.slot_base);
    for (int q = threadIdx.x; q < s.ns / 4; q += blockDim.x) g[q] = reinterpret_cast<const float4*>(s.M)[q];
  }
}

cudaError_t set_sweep_smem_limit(size_t bytes) {
  cudaError_t e = cudaSuccess;
  int b = (int)bytes;
  if ((e = cudaFuncSetAttribute(k_sweep<kFwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep<kBwd>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep<kMinMarg>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep<kEnergy>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  if ((e = cudaFuncSetAttribute(k_sweep<kSeed>, cudaFuncAttributeMaxDynamicSharedMemorySize, b))) return e;
  return e;
}

void launch_sweep(int kind, const DevArena& A, const SweepArgs& a, int threads, size_t smem, cudaStream_t st) {
  if (A.num_tiles == 0) return;
  dim3 grid(A.num_tiles), block(threads);
  switch (kind) {
    case kFwd: k_sweep<kFwd><<<grid, block, smem, st>>>(A, a); break;
    case kBwd: k_sweep<kBwd><<<grid, block, smem, st>>>(A, a); break;
    case kMinMarg: k_sweep<kMinMarg><<<grid, block, smem, st>>>(A, a); break;
    case kEnergy: k_sweep<kEnergy><<<grid, block, smem, st>>>(A, a); break;
    default: k_sweep<kSeed><<<grid, block, smem, st>>>(A, a); break;
  }
}

}  // namespace dg
