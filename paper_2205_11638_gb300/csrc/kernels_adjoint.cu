// kernels_adjoint.cu -- backpropagation through one sweep of Alg. 1
// (Alg. 2 "BlockUpdate backpropagation", Prop. 2, and the shortest-path
// formulation of App. B: gradients of min-marginals flow along the argmin
// arcs of the min-sum recursions).
//
// One warp per tile, one lane per BDD, as in the forward sweeps.  The sweep
// being differentiated was run as a recording sweep (k_sweep<kFwdRec/kBwdRec>
// with the same FP32 operations as the plain sweep), which left per node the
// argmin in-arc of SP(r, .) (smallest (parent rank, beta) on ties) and the
// argmin out-arc of SP(., T) (0-arc on ties), and per level the argmin nodes
// of m0 and m1 (smallest rank on ties) and m1 - m0.  A lane stages those
// records and runs the reverse of the sweep level by level:
//   lambda^new = lambda^old - M^new + alpha S^in,  M^new = omega (m1 - m0)
// gives   S-dot contribution alpha * g, alpha-dot += g S^in,
//         Mt = M-dot - g, omega-dot += Mt (m1 - m0),
//         m1-dot = omega Mt, m0-dot = -omega Mt, lambda^old-dot = g + m1-dot
// (g = gradient of lambda^new), and the min-marginal gradients are routed to
// SP(r, .) and SP(., T) of the argmin nodes and from there, arc by arc, to the
// lambdas on the argmin paths.  This equals Alg. 2's minimiser-vector formula
// (the argmin paths are the minimisers s^j(i, beta)) at O(arcs) per sweep.
#include "kernels.h"
#include "sweep.cuh"

namespace dg {

namespace {

// Shared-memory image of one tile in the adjoint kernels: what the level
// loops walk node by node.  The per-slot inputs of the update's reverse
// (S^in, alpha, omega, M-dot, the recorded argmins and m1 - m0, and the
// running omega-dot / alpha-dot sums) are read from global memory into
// registers one level ahead instead (see LevelIn), which keeps a tile's
// footprint small enough for more warps per SM; the per-variable ones come
// laid out per slot (AdjArgs::slot_in), so no read depends on another.
struct AdjSmem {
  float* a1;       // [32 * nmax] gradient of SP(., T)
  float* a2;       // [32 * nmax] gradient of SP(r, .)
  uint16_t* meta;  // [32 * nmax] parent node | beta << 8 | hi-choice << 9 (recorded)
  uint16_t* code;  // [32 * (nmax - 2)]
  uint16_t* desc;  // [32 * nh]
  float* gl;       // [32 * nh] lambda gradient (new -> old)
  int nmax, nh;
};

#define A1(n) s.a1[(n) * kWarp + lane]
#define A2(n) s.a2[(n) * kWarp + lane]
#define META(n) s.meta[(n) * kWarp + lane]

__device__ __forceinline__ AdjSmem carve_adj(unsigned char* p, const Tile& T) {
  AdjSmem s;
  s.nmax = T.nmax;
  s.nh = T.nhops;
  const int nn = s.nmax * kWarp, ns = s.nh * kWarp;
  s.a1 = (float*)p;
  p += (size_t)nn * 4;
  s.a2 = (float*)p;
  p += (size_t)nn * 4;
  s.gl = (float*)p;
  p += (size_t)ns * 4;
  s.meta = (uint16_t*)p;
  p += (size_t)nn * 2;
  s.desc = (uint16_t*)p;
  p += (size_t)ns * 2;
  s.code = (uint16_t*)p - 2 * kWarp;  // biased: element 32 n + lane is node number n
  return s;
}

// The per-slot inputs of one level's reverse step, for lane `lane`.
struct LevelIn {
  float S, al, om, md, diff, ga, go;
  uint32_t amin;
};

template <int MODE>
__device__ __forceinline__ LevelIn load_level(const DevArena& A, const AdjArgs& a, const AdjSmem& s, int64_t sb,
                                              int h, int lane) {
  LevelIn r;
  const int q = h * kWarp + lane;
  const float2 in = a.slot_in[sb + q];
  r.diff = a.rec_diff[sb + q];
  r.amin = a.rec_amin[sb + q];
  r.S = in.y;
  r.al = MODE == 1 ? a.alpha[sb + q] : A.slot_invdeg[sb + q];
  r.om = MODE == 1 ? a.omega[sb + q] : a.omega0;
  const float seed = a.seed_M ? a.seed_M[sb + q] : 0.0f;
  r.md = seed + in.x;  // gradient of M^new
  r.ga = a.g_alpha ? a.g_alpha[sb + q] : 0.0f;
  r.go = a.g_omega ? a.g_omega[sb + q] : 0.0f;
  return r;
}

}  // namespace

template <int FWD, int MODE>
__global__ void __launch_bounds__(128) k_adjoint(DevArena A, AdjArgs a, int region_bytes, int tile0, int tile1) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = tile0 + blockIdx.x * (blockDim.x >> 5) + warp;
  if (tile >= tile1) return;
  const Tile T = A.tiles[tile];
  AdjSmem s = carve_adj(smem + (size_t)warp * region_bytes, T);
  const int ns = s.nh * kWarp;
  const int64_t sb = T.slot_base;

  // ---- staging: child codes, the sweep's node records, the gradients -----
  copy_async(s.code + 2 * kWarp, A.lohi8 + T.node_base, (s.nmax - 2) * kWarp * 2, lane);
  copy_async(s.meta + 2 * kWarp, a.rec_meta + T.node_base, (s.nmax - 2) * kWarp * 2, lane);
  copy_async(s.desc, A.desc + sb, ns * 2, lane);
  copy_async(s.gl, a.g_lam + sb, ns * 4, lane);
  cp_async_commit();
  // gradient accumulators of SP(., T) and SP(r, .)
  for (int n = 0; n < s.nmax; ++n) {
    A1(n) = 0.0f;
    A2(n) = 0.0f;
  }
  cp_async_wait_all();
  __syncwarp();

  // ---- reverse ------------------------------------------------------------
  // one step of the reverse: the update and the min-marginal argmins of level h
  auto reverse_level = [&](int h, const LevelIn& in) {
    const int q = h * kWarp + lane;
    const float g = s.gl[q];
    const float Mt = in.md - g;
    a.sdot[sb + q] = in.al * g;                              // contribution to S-dot
    if (a.g_alpha) a.g_alpha[sb + q] = in.ga + g * in.S;
    if (a.g_omega) a.g_omega[sb + q] = in.go + Mt * in.diff;
    const float dm1 = in.om * Mt, dm0 = -in.om * Mt;
    s.gl[q] = g + dm1;                                       // gradient of lambda^old
    const int v0 = in.amin & 0xFFu, v1 = in.amin >> 8;
    const uint32_t c0 = node_code(s.code, v0, lane), c1 = node_code(s.code, v1, lane);
    A2(v0) += dm0;
    A1(c0 & 0xFFu) += dm0;  // terminals absorb into their unused entries
    A2(v1) += dm1;
    A1(c1 >> 8) += dm1;
  };
  if (FWD) {
    LevelIn cur = load_level<MODE>(A, a, s, sb, s.nh - 1, lane);
    for (int h = s.nh - 1; h >= 0; --h) {
      // the next level's inputs are loaded while this level is worked on
      const LevelIn nxt = load_level<MODE>(A, a, s, sb, h > 0 ? h - 1 : 0, lane);
      const uint32_t ds = s.desc[h * kWarp + lane];
      if (desc_width(ds) > 0) {
        const int q = h * kWarp + lane;
        const uint32_t dn = h + 1 < s.nh ? s.desc[(h + 1) * kWarp + lane] : 0u;
        const int wn = desc_width(dn), fnn = desc_first(dn);
        // SP(r, .) of level h+1 was relaxed from level h with lambda^new_h
        float g = s.gl[q];
        for (int r = 0; r < wn; ++r) {
          const int wnode = fnn + r;
          const float gd = A2(wnode);
          const uint32_t mt = META(wnode);
          A2(mt & 0xFFu) += gd;
          if (mt & (1u << 8)) g += gd;
        }
        s.gl[q] = g;
        reverse_level(h, cur);
      }
      cur = nxt;
    }
    // SP(., T) under lambda^old: route its gradient top-down along argmin out-arcs
    for (int h = 0; h < s.nh; ++h) {
      const uint32_t ds = s.desc[h * kWarp + lane];
      const int w = desc_width(ds);
      if (w == 0) break;
      const int fn = desc_first(ds);
      const int q = h * kWarp + lane;
      float g = s.gl[q];
      for (int r = 0; r < w; ++r) {
        const int n = fn + r;
        const float gt = A1(n);
        const uint32_t c = node_code(s.code, n, lane);
        if (META(n) & (1u << 9)) {
          A1(c >> 8) += gt;
          g += gt;
        } else {
          A1(c & 0xFFu) += gt;
        }
      }
      s.gl[q] = g;
    }
  } else {
    LevelIn cur = load_level<MODE>(A, a, s, sb, 0, lane);
    for (int h = 0; h < s.nh; ++h) {
      const uint32_t ds = s.desc[h * kWarp + lane];
      const int w = desc_width(ds);
      if (w == 0) break;
      const LevelIn nxt = load_level<MODE>(A, a, s, sb, h + 1 < s.nh ? h + 1 : h, lane);
      const int fn = desc_first(ds);
      const int q = h * kWarp + lane;
      // SP(., T) of level h was recomputed with lambda^new_h
      float g = s.gl[q];
      for (int r = 0; r < w; ++r) {
        const int n = fn + r;
        const float gt = A1(n);
        const uint32_t c = node_code(s.code, n, lane);
        if (META(n) & (1u << 9)) {
          A1(c >> 8) += gt;
          g += gt;
        } else {
          A1(c & 0xFFu) += gt;
        }
      }
      s.gl[q] = g;
      reverse_level(h, cur);
      cur = nxt;
    }
    // SP(r, .) under lambda^old: route its gradient bottom-up along argmin in-arcs
    for (int h = s.nh - 1; h >= 1; --h) {
      const uint32_t ds = s.desc[h * kWarp + lane];
      const int w = desc_width(ds);
      if (w == 0) continue;
      const int fn = desc_first(ds);
      const int qp = (h - 1) * kWarp + lane;
      float g = s.gl[qp];
      for (int r = 0; r < w; ++r) {
        const int n = fn + r;
        const float gd = A2(n);
        const uint32_t mt = META(n);
        A2(mt & 0xFFu) += gd;
        if (mt & (1u << 8)) g += gd;
      }
      s.gl[qp] = g;
    }
  }
  __syncwarp();
  // ---- outputs ----------------------------------------------------------
  for (int q = lane; q < ns; q += kWarp) {
    if (desc_width(s.desc[q]) == 0) continue;
    a.g_lam[sb + q] = s.gl[q];
  }
}

template <int FWD>
static cudaError_t set_adj_attr(int b) {
  cudaError_t e = cudaFuncSetAttribute(k_adjoint<FWD, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_adjoint<FWD, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

cudaError_t set_adjoint_smem_limit(size_t bytes) {
  cudaError_t e = set_adj_attr<1>((int)bytes);
  if (e == cudaSuccess) e = set_adj_attr<0>((int)bytes);
  return e;
}

template <int FWD, int MODE>
static void launch_adj(const DevArena& A, const AdjArgs& a, const AdjGroup* groups, int num_groups, size_t cap,
                       const StreamSet& ss) {
  const bool fork = num_groups + (A.num_long > 0 ? 1 : 0) > 1 && ss.ready;
  if (fork) ss.begin();
  launch_long_adjoint(FWD != 0, A, a, fork ? ss.of(A.long_stream) : ss.main);
  for (int g = 0; g < num_groups; ++g) {
    const AdjGroup& G = groups[g];
    const size_t region = (size_t)G.region;
    const int wpc = best_warps_per_cta(region, 4, cap);
    const int nt = G.tile1 - G.tile0;
    k_adjoint<FWD, MODE><<<(nt + wpc - 1) / wpc, wpc * kWarp, region * wpc, fork ? ss.of(G.stream) : ss.main>>>(
        A, a, (int)region, G.tile0, G.tile1);
  }
  if (fork) ss.end();
}

void launch_adjoint_sweep(bool forward, const DevArena& A, const AdjArgs& a, const AdjGroup* groups, int num_groups,
                          size_t cta_smem_cap, const StreamSet& st) {
  if (forward)
    a.mode == 1 ? launch_adj<1, 1>(A, a, groups, num_groups, cta_smem_cap, st)
                : launch_adj<1, 0>(A, a, groups, num_groups, cta_smem_cap, st);
  else
    a.mode == 1 ? launch_adj<0, 1>(A, a, groups, num_groups, cta_smem_cap, st)
                : launch_adj<0, 0>(A, a, groups, num_groups, cta_smem_cap, st);
}

}  // namespace dg
