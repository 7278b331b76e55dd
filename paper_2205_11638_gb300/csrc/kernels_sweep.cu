// kernels_sweep.cu -- the sweeps of Alg. 1 (generalized min-marginal
// averaging, Sec. 3.2 of DOGE-Train) over tiles of BDDs, plus the kernels
// that evaluate min-marginals, subproblem energies and minimising
// assignments on the same layout.
//
// One warp owns one tile (up to 32 BDDs, BDD b on lane b).  The warp stages
// the tile's slot descriptors, lambda and alpha*S in its slice of shared
// memory; every lane then runs BlockUpdate level by level on its own BDD (a
// forward sweep visits B_1..B_u, a backward sweep B_u..B_1) and writes the new
// lambda and M of each level straight to global memory (the lanes of a warp
// write 32 consecutive slots).  The shortest-path costs of the direction
// opposite to the sweep (SP(.,T) for a forward sweep, SP(r,.) for a backward
// one) are recomputed from lambda in shared memory instead of being kept in
// HBM between sweeps; they equal the values the previous sweep left, bit for
// bit, because the same FP32 operations run on the same inputs.
#include "kernels.h"
#include "sweep.cuh"

namespace dg {

static size_t g_cta_smem_cap = 227 * 1024;

// Nodes of a level whose child costs the backward sweeps keep in registers
// between the level's two passes (most levels are this narrow).  The forward
// sweeps measured faster without such a cache (register pressure).
constexpr int kCacheFwd = 0;
constexpr int kCacheBwd = 4;

template <int KIND, int MODE>
__global__ void __launch_bounds__(128) k_sweep(DevArena A, SweepArgs a, int region_bytes, int tile0, int tile1) {
  // kFwdRec / kBwdRec are kFwd / kBwd that also record the argmins of their
  // recursions for the adjoint: strict comparisons in node order instead of
  // fminf (the same values, plus the winner), and the records written out
  constexpr bool REC = KIND == kFwdRec || KIND == kBwdRec;
  constexpr bool FWD = KIND == kFwd || KIND == kFwdRec;
  constexpr bool BWD = KIND == kBwd || KIND == kBwdRec;
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = tile0 + blockIdx.x * (blockDim.x >> 5) + warp;
  if (tile >= tile1) return;  // whole warp leaves; no CTA-wide barrier follows
  const Tile T = A.tiles[tile];
  TileSmem s = carve<MODE, !BWD, REC>(smem + (size_t)warp * region_bytes, T);
  // a plain sweep may take the opposite-direction costs from the sweep before it
  const float* cost_in = (FWD || BWD) ? a.cost_in : nullptr;
  load_tile<FWD || BWD, MODE>(A, T, s, a.lam, a.omega, a.alpha, lane, cost_in);
  // a recording sweep that takes the costs also takes the records the
  // recording sweep before it made in the same comparisons: the out-arc
  // choices of SP(., T) (for a forward sweep) or the in-arcs of SP(r, .)
  // (for a backward one); the rest of each record is rewritten below
  if (REC && cost_in) {
    copy_async(s.meta + 2 * kWarp, a.meta_in + T.node_base, (s.nmax - 2) * kWarp * 2, lane);
    cp_async_commit();
    cp_async_wait_all();
    __syncwarp();
    if (FWD && desc_width(s.desc[lane]) > 0) DG_META(s, 2) &= kHiChoice;  // the root has no in-arc
  }
  const int64_t sbase = T.slot_base;

  if (FWD || KIND == kMinMarg) {
    // ---- SP(., T) under lambda at sweep start, then the forward sweep -----
    if (!cost_in) {
      if (REC)
        lane_cost_to_top_rec(s, lane);
      else
        lane_cost_to_top(s, lane);
    }
    if (desc_width(s.desc[lane]) > 0) DG_R(s, 2) = 0.0f;
    for (int h = 0; h < s.nh; ++h) {
      const uint32_t ds = s.desc[h * kWarp + lane];
      const int w = desc_width(ds);
      if (w == 0) break;
      const int fn = desc_first(ds);
      const uint32_t dn = h + 1 < s.nh ? s.desc[(h + 1) * kWarp + lane] : 0u;
      const int wn = desc_width(dn), fnn = desc_first(dn);
      float b0 = f_inf(), b1 = f_inf();
      int v0 = fn, v1 = fn;
      // the codes and costs of the level's first kCacheFwd nodes stay in
      // registers for the relaxation below
      constexpr int CF = REC ? 0 : kCacheFwd;
      uint32_t cc[CF > 0 ? CF : 1];
      float dd[CF > 0 ? CF : 1];
      #pragma unroll
      for (int i = 0; i < CF; ++i) {
        cc[i] = 0u;
        dd[i] = 0.0f;
        if (i < w) {
          cc[i] = node_code(s, fn + i, lane);
          dd[i] = DG_R(s, fn + i);
          if (FWD) DG_F(s, fn + i) = dd[i];
          b0 = fminf(b0, dd[i] + DG_F(s, cc[i] & 0xFFu));
          b1 = fminf(b1, dd[i] + DG_F(s, cc[i] >> 8));
        }
      }
      #pragma unroll 2
      for (int r = CF; r < w; ++r) {
        const int n = fn + r;
        const uint32_t c = node_code(s, n, lane);
        const float dv = DG_R(s, n);
        const float x0 = dv + DG_F(s, c & 0xFFu), x1 = dv + DG_F(s, c >> 8);
        // SP(r, n) is final here and SP(n, T) is not read again: the whole
        // array ends the sweep holding SP(r, .) under the new lambda
        if (FWD) DG_F(s, n) = dv;
        if (REC) {
          if (x0 < b0) { b0 = x0; v0 = n; }
          if (x1 < b1) { b1 = x1; v1 = n; }
        } else {
          b0 = fminf(b0, x0);
          b1 = fminf(b1, x1);
        }
      }
      const int q = h * kWarp + lane;
      const float l = s.lam[q];
      const float m0 = b0, m1 = l + b1;
      float ln = l;
      if (KIND == kMinMarg) {
        a.M[sbase + q] = m0;
        a.out2[sbase + q] = m1;
      } else {
        const float om = MODE == 1 ? s.om[q] : a.omega0;
        const float Mn = om * (m1 - m0);
        ln = l - Mn + slot_avg<MODE>(s, q);
        a.lam[sbase + q] = ln;
        a.M[sbase + q] = Mn;
        if (REC) {
          a.rec_amin[sbase + q] = (uint16_t)(v0 | (v1 << 8));
          a.rec_diff[sbase + q] = m1 - m0;
        }
      }
      if (wn > 0) {
        #pragma unroll 2
        for (int r = 0; r < wn; ++r) DG_R(s, fnn + r) = f_inf();
        #pragma unroll
        for (int i = 0; i < CF; ++i) {
          if (i < w) {
            const uint32_t lo = cc[i] & 0xFFu, hi = cc[i] >> 8;
            if (lo != kBotCode) DG_R(s, lo) = fminf(DG_R(s, lo), dd[i]);
            if (hi != kBotCode) DG_R(s, hi) = fminf(DG_R(s, hi), dd[i] + ln);
          }
        }
        #pragma unroll 2
        for (int r = CF; r < w; ++r) {
          const int n = fn + r;
          const uint32_t c = node_code(s, n, lane);
          const uint32_t lo = c & 0xFFu, hi = c >> 8;
          const float dv = DG_R(s, n);
          if (REC) {
            if (lo >= 2 && dv < DG_R(s, lo)) {
              DG_R(s, lo) = dv;
              DG_META(s, lo) = (uint16_t)((DG_META(s, lo) & kHiChoice) | n);
            }
            if (hi >= 2 && dv + ln < DG_R(s, hi)) {
              DG_R(s, hi) = dv + ln;
              DG_META(s, hi) = (uint16_t)((DG_META(s, hi) & kHiChoice) | n | kInHi);
            }
          } else {
            if (lo != kBotCode) DG_R(s, lo) = fminf(DG_R(s, lo), dv);
            if (hi != kBotCode) DG_R(s, hi) = fminf(DG_R(s, hi), dv + ln);
          }
        }
      }
    }
    if (FWD && a.cost_out) store_costs(a.cost_out + T.node_base, s.full, s.nmax, lane);
  } else if (BWD) {
    // ---- SP(r, .) under lambda at sweep start, then the backward sweep ----
    if (!cost_in) {
      if (REC)
        lane_cost_from_root_rec(s, lane);
      else
        lane_cost_from_root(s, lane);
    }
    DG_W(s, kTopCode) = 0.0f;
    DG_W(s, kBotCode) = f_inf();
    for (int h = s.nh - 1; h >= 0; --h) {
      const uint32_t ds = s.desc[h * kWarp + lane];
      const int w = desc_width(ds);
      if (w == 0) continue;
      const int fn = desc_first(ds);
      float b0 = f_inf(), b1 = f_inf();
      int v0 = fn, v1 = fn;
      // the child costs of the level's first kCacheBwd nodes stay in registers
      // for the level's own costs below
      constexpr int CB = REC ? 0 : kCacheBwd;
      float wl[CB > 0 ? CB : 1], wh[CB > 0 ? CB : 1];
      #pragma unroll
      for (int i = 0; i < CB; ++i) {
        wl[i] = wh[i] = 0.0f;
        if (i < w) {
          const uint32_t c = node_code(s, fn + i, lane);
          const float dv = DG_F(s, fn + i);
          wl[i] = DG_W(s, c & 0xFFu);
          wh[i] = DG_W(s, c >> 8);
          b0 = fminf(b0, dv + wl[i]);
          b1 = fminf(b1, dv + wh[i]);
        }
      }
      #pragma unroll 2
      for (int r = CB; r < w; ++r) {
        const int n = fn + r;
        const uint32_t c = node_code(s, n, lane);
        const float dv = DG_F(s, n);
        const float x0 = dv + DG_W(s, c & 0xFFu), x1 = dv + DG_W(s, c >> 8);
        if (REC) {
          if (x0 < b0) { b0 = x0; v0 = n; }
          if (x1 < b1) { b1 = x1; v1 = n; }
        } else {
          b0 = fminf(b0, x0);
          b1 = fminf(b1, x1);
        }
      }
      const int q = h * kWarp + lane;
      const float l = s.lam[q];
      const float m0 = b0, m1 = l + b1;
      const float om = MODE == 1 ? s.om[q] : a.omega0;
      const float Mn = om * (m1 - m0);
      const float ln = l - Mn + slot_avg<MODE>(s, q);
      a.lam[sbase + q] = ln;
      a.M[sbase + q] = Mn;
      if (REC) {
        a.rec_amin[sbase + q] = (uint16_t)(v0 | (v1 << 8));
        a.rec_diff[sbase + q] = m1 - m0;
      }
      #pragma unroll
      for (int i = 0; i < CB; ++i)
        if (i < w) DG_W(s, fn + i) = fminf(wl[i], ln + wh[i]);
      #pragma unroll 2
      for (int r = CB; r < w; ++r) {
        const int n = fn + r;
        const uint32_t c = node_code(s, n, lane);
        if (REC) {
          const float tl = DG_W(s, c & 0xFFu), th = ln + DG_W(s, c >> 8);
          const bool take0 = (c & 0xFFu) != kBotCode && tl <= th;
          DG_W(s, n) = take0 ? tl : th;
          DG_META(s, n) = (uint16_t)((DG_META(s, n) & 0x1FFu) | (take0 ? 0u : kHiChoice));
        } else {
          DG_W(s, n) = fminf(DG_W(s, c & 0xFFu), ln + DG_W(s, c >> 8));
        }
      }
    }
    // the second whole array ends the sweep holding SP(., T) under the new lambda
    if (BWD && a.cost_out) store_costs(a.cost_out + T.node_base, s.ring, s.nmax, lane);
  } else {
    // kEnergy / kSeed: SP(., T) under lambda
    lane_cost_to_top(s, lane);
  }

  if (KIND == kSeed) {
    // walk the minimising path from my root: 0-arc on ties
    int n = 2;
    for (int h = 0; h < s.nh; ++h) {
      if (desc_width(s.desc[h * kWarp + lane]) == 0) break;
      const uint32_t c = node_code(s, n, lane);
      const uint32_t lo = c & 0xFFu, hi = c >> 8;
      const int q = h * kWarp + lane;
      const bool take0 = lo != kBotCode && (hi == kBotCode || DG_F(s, lo) <= s.lam[q] + DG_F(s, hi));
      a.M[sbase + q] = take0 ? 0.f : 1.f;
      n = (int)(take0 ? lo : hi);
    }
  }

  if (REC) {
    // the records of nodes 2 .. nmax-1, in the layout of the child codes
    __syncwarp();
    const uint32_t* src = reinterpret_cast<const uint32_t*>(s.meta + 2 * kWarp);
    uint32_t* dst = reinterpret_cast<uint32_t*>(a.rec_meta + T.node_base);
    for (int o = lane; o < (s.nmax - 2) * (kWarp / 2); o += kWarp) dst[o] = src[o];
  }

  if ((BWD || KIND == kEnergy) && a.E != nullptr && lane < T.nbdd) {
    // SP(root, T) = E^j of my BDD
    const int row = __ldg(A.slot_row + sbase + lane);
    a.E[row] = BWD ? DG_W(s, 2) : DG_F(s, 2);
  }
}

// log(exp(x) + exp(y)) with -inf as the empty sum.
__device__ __forceinline__ float lse2(float x, float y) {
  const float m = fmaxf(x, y);
  if (m == -f_inf()) return m;
  return m + log1pf(expf(-fabsf(x - y)));
}

// Smoothed subproblems (the feature table's smoothed dual, read as the
// soft-min E_a = -a log sum_{x in X_j} exp(-<lambda, x>/a)) and their
// gradients, the marginals P(x_i = 1), by log-sum-exp over the BDD paths:
// B(v) over v-T paths, F(v) over r-v paths, log Z = B(root).
__global__ void __launch_bounds__(128) k_smoothed(DevArena A, const float* lam, float a_s, float* E_a, float* marg,
                                                  int region_bytes, int tile0, int tile1) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int tile = tile0 + blockIdx.x * (blockDim.x >> 5) + warp;
  if (tile >= tile1) return;
  const Tile T = A.tiles[tile];
  TileSmem s = carve<0, false>(smem + (size_t)warp * region_bytes, T);
  load_tile<false, 0>(A, T, s, lam, nullptr, nullptr, lane);
  const int64_t sbase = T.slot_base;
  const float inv_a = 1.0f / a_s;
  DG_F(s, kBotCode) = -f_inf();  // B of the terminals: log 1 = 0 for top, log 0 for bottom
  for (int h = s.nh - 1; h >= 0; --h) {
    const uint32_t ds = s.desc[h * kWarp + lane];
    const int w = desc_width(ds);
    if (w == 0) continue;
    const int fn = desc_first(ds);
    const float wgt = -s.lam[h * kWarp + lane] * inv_a;
    #pragma unroll 2
    for (int r = 0; r < w; ++r) {
      const int n = fn + r;
      const uint32_t c = node_code(s, n, lane);
      DG_F(s, n) = lse2(DG_F(s, c & 0xFFu), wgt + DG_F(s, c >> 8));
    }
  }
  if (desc_width(s.desc[lane]) == 0) return;
  const float logZ = DG_F(s, 2);
  if (E_a) E_a[__ldg(A.slot_row + sbase + lane)] = -a_s * logZ;
  DG_W(s, 2) = 0.0f;
  for (int h = 0; h < s.nh; ++h) {
    const uint32_t ds = s.desc[h * kWarp + lane];
    const int w = desc_width(ds);
    if (w == 0) break;
    const int fn = desc_first(ds);
    const uint32_t dn = h + 1 < s.nh ? s.desc[(h + 1) * kWarp + lane] : 0u;
    const int wn = desc_width(dn), fnn = desc_first(dn);
    const float wgt = -s.lam[h * kWarp + lane] * inv_a;
    #pragma unroll 2
    for (int r = 0; r < wn; ++r) DG_W(s, fnn + r) = -f_inf();
    float acc = -f_inf();
    #pragma unroll 2
    for (int r = 0; r < w; ++r) {
      const int n = fn + r;
      const uint32_t c = node_code(s, n, lane);
      const uint32_t lo = c & 0xFFu, hi = c >> 8;
      const float f = DG_W(s, n);
      acc = lse2(acc, f + wgt + DG_F(s, hi));
      if (wn > 0) {
        DG_W(s, lo) = lse2(DG_W(s, lo), f);  // bottom's entry is scratch
        DG_W(s, hi) = lse2(DG_W(s, hi), f + wgt);
      }
    }
    marg[sbase + h * kWarp + lane] = expf(acc - logZ);
  }
}

void launch_smoothed(const DevArena& A, const float* lam, float a_s, float* E_a, float* marg, const LaunchGroup* groups,
                     int num_groups, const StreamSet& ss) {
  const bool fork = num_groups + (A.num_long > 0 ? 1 : 0) > 1 && ss.ready;
  if (fork) ss.begin();
  launch_long_smoothed(A, lam, a_s, E_a, marg, fork ? ss.of(A.long_stream) : ss.main);
  for (int g = 0; g < num_groups; ++g) {
    const LaunchGroup& G = groups[g];
    const size_t region = (size_t)G.region_bwd0;
    const int wpc = best_warps_per_cta(region, 4, g_cta_smem_cap);
    const int nt = G.tile1 - G.tile0;
    k_smoothed<<<(nt + wpc - 1) / wpc, wpc * kWarp, region * wpc, fork ? ss.of(G.stream) : ss.main>>>(
        A, lam, a_s, E_a, marg, (int)region, G.tile0, G.tile1);
  }
  if (fork) ss.end();
}

template <int KIND>
static cudaError_t set_attr(int b) {
  cudaError_t e = cudaFuncSetAttribute(k_sweep<KIND, 0>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(k_sweep<KIND, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  return e;
}

cudaError_t set_sweep_smem_limit(size_t bytes) {
  const int b = (int)bytes;
  cudaError_t e = cudaFuncSetAttribute(k_smoothed, cudaFuncAttributeMaxDynamicSharedMemorySize, b);
  if (e == cudaSuccess) e = set_attr<kFwd>(b);
  if (e == cudaSuccess) e = set_attr<kBwd>(b);
  if (e == cudaSuccess) e = set_attr<kMinMarg>(b);
  if (e == cudaSuccess) e = set_attr<kEnergy>(b);
  if (e == cudaSuccess) e = set_attr<kSeed>(b);
  if (e == cudaSuccess) e = set_attr<kFwdRec>(b);
  if (e == cudaSuccess) e = set_attr<kBwdRec>(b);
  return e;
}

void set_cta_smem_cap(size_t bytes) { g_cta_smem_cap = bytes; }

// Warps per CTA for a per-warp slice of `region` bytes: the CTA size (1, 2
// or 4 warps, at most `max_wpc`) that lets the most warps share one SM (228 KB
// of shared memory, 1 KB reserved per CTA, at most 32 CTAs and 64 warps).
int best_warps_per_cta(size_t region, int max_wpc, size_t cta_cap) {
  const size_t sm_smem = 228 * 1024;
  int best = 1, best_warps = -1;
  for (int w = 1; w <= max_wpc; w *= 2) {
    const size_t cta = region * w;
    if (cta > cta_cap) break;
    int ctas = (int)(sm_smem / (cta + 1024));
    if (ctas > 32) ctas = 32;
    int warps = ctas * w;
    if (warps > 64) warps = 64;
    if (warps >= best_warps) {
      best_warps = warps;
      best = w;
    }
  }
  return best;
}

void StreamSet::begin() const {
  if (!ready || n <= 1) return;
  cudaEventRecord(fork, main);
  for (int k = 0; k < n - 1; ++k) cudaStreamWaitEvent(aux[k], fork, 0);
}

void StreamSet::end() const {
  if (!ready || n <= 1) return;
  for (int k = 0; k < n - 1; ++k) {
    cudaEventRecord(join[k], aux[k]);
    cudaStreamWaitEvent(main, join[k], 0);
  }
}

template <int KIND, int MODE>
static void launch_groups(const DevArena& A, const SweepArgs& a, int threads, const LaunchGroup* groups,
                          int num_groups, const StreamSet& ss) {
  const bool fork = num_groups + (A.num_long > 0 ? 1 : 0) > 1 && ss.ready;
  if (fork) ss.begin();
  // the long BDDs first: their launch is a few warps walking long chains
  launch_long_sweep(KIND, A, a, fork ? ss.of(A.long_stream) : ss.main);
  for (int g = 0; g < num_groups; ++g) {
    const LaunchGroup& G = groups[g];
    constexpr bool REC = KIND == kFwdRec || KIND == kBwdRec;
    constexpr bool BWD = KIND == kBwd || KIND == kBwdRec;
    const size_t region = (size_t)(BWD ? (MODE == 1 ? G.region_bwd1 : G.region_bwd0)
                                       : (MODE == 1 ? G.region_bytes : G.region_bytes0)) +
                          (REC ? (size_t)G.meta_bytes : 0);
    int wpc = threads / kWarp;
    if (wpc > 4) wpc = 4;  // __launch_bounds__(128)
    const int tuned = REC ? 0 : (BWD ? G.wpc_bwd : G.wpc_fwd);
    if (tuned > 0 && region * tuned <= g_cta_smem_cap)
      wpc = tuned;
    else
      wpc = best_warps_per_cta(region, wpc, g_cta_smem_cap);
    const int nt = G.tile1 - G.tile0;
    dim3 grid((nt + wpc - 1) / wpc), block(wpc * kWarp);
    k_sweep<KIND, MODE><<<grid, block, region * wpc, fork ? ss.of(G.stream) : ss.main>>>(A, a, (int)region, G.tile0,
                                                                                          G.tile1);
  }
  if (fork) ss.end();
}

// One launch per launch group; threads = warps per CTA * 32, every warp
// sweeps one tile with its own slice of the group's shared memory.  Only
// the update sweeps read omega/alpha, so only they have a mode-1 variant.
void launch_sweep(int kind, const DevArena& A, const SweepArgs& a, int threads, const LaunchGroup* groups,
                  int num_groups, const StreamSet& st) {
  const bool m1 = a.mode == 1;
  switch (kind) {
    case kFwd:
      m1 ? launch_groups<kFwd, 1>(A, a, threads, groups, num_groups, st)
         : launch_groups<kFwd, 0>(A, a, threads, groups, num_groups, st);
      break;
    case kBwd:
      m1 ? launch_groups<kBwd, 1>(A, a, threads, groups, num_groups, st)
         : launch_groups<kBwd, 0>(A, a, threads, groups, num_groups, st);
      break;
    case kFwdRec:
      m1 ? launch_groups<kFwdRec, 1>(A, a, threads, groups, num_groups, st)
         : launch_groups<kFwdRec, 0>(A, a, threads, groups, num_groups, st);
      break;
    case kBwdRec:
      m1 ? launch_groups<kBwdRec, 1>(A, a, threads, groups, num_groups, st)
         : launch_groups<kBwdRec, 0>(A, a, threads, groups, num_groups, st);
      break;
    case kMinMarg: launch_groups<kMinMarg, 0>(A, a, threads, groups, num_groups, st); break;
    case kEnergy: launch_groups<kEnergy, 0>(A, a, threads, groups, num_groups, st); break;
    default: launch_groups<kSeed, 0>(A, a, threads, groups, num_groups, st); break;
  }
}

}  // namespace dg
