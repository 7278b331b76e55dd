// kernels_long.cu -- the sweeps of Alg. 1, their recording variants, the
// energies, minimising assignments and smoothed subproblems, and the adjoint
// of a sweep (Alg. 2) for BDDs beyond the lane-per-BDD tiles (LongBdd: more
// than 254 nodes or a level wider than 128).  The paper names long
// subproblems as the sequential part of the method (its conclusion): App. B's
// recursions over one BDD visit its levels one after another.
//
// Execution model: one warp per BDD; the nodes of a level are spread over the
// lanes (node f + lane, f + lane + 32, ...), the levels are walked in turn
// with a __syncwarp between them.  The min-marginals of a level (App. B:
// m^beta = min over the level's nodes of SP(r, v) + SP(s^beta(v), T), plus
// lambda for beta = 1) are lane minima combined by warp shuffles; SP(r, .)
// of a level is a pull over each node's in-arc list, SP(., T) over its two
// children, so no two lanes write the same node and nothing needs atomics.
// Path costs live in the arena's scratch (long_d, long_t, indexed by node
// number: 0 top, 1 bottom, own nodes from 2), read and written through L1.
// A sweep leaves there the costs of its own direction under the new lambda,
// so a sweep handed the costs (SweepArgs::cost_in, set when the tiles' costs
// are handed on) skips its first pass: they are already in place.
//
// The plain forward and backward sweeps of the long BDDs whose levels have
// at most 32 nodes (long cardinality and assignment rows) run in
// k_long_narrow instead: several such BDDs to a warp, G lanes each, the
// costs of the sweep direction in registers (see narrow_down / narrow_up).
// The recording sweeps, energies, seeds, min-marginals, smoothed
// subproblems and adjoints keep one warp per BDD.
//
// The arithmetic is the lane kernels': the same FP32 operations per arc;
// minima are exact, so values do not depend on the order of the reduction;
// argmins follow the same tie rules (smallest node number for the
// min-marginals, smallest (parent, beta) in-arc for SP(r, .), the 0-arc for
// SP(., T)).  Sums of gradients over a level (warp shuffles) round in another
// order than the lane kernels' sequential sums.
#include <climits>

#include "kernels.h"
#include "sweep.cuh"

namespace dg {

namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
// argmin record of a node in the recording sweeps: parent << 2 | beta << 1 |
// hi-choice, i.e. the in-arc (parent << 1 | beta) shifted left by one
constexpr int32_t kLHi = 1;
constexpr int32_t kLBeta = 2;

__device__ __forceinline__ float warp_sum(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(kFull, x, o);
  return x;
}

__device__ __forceinline__ float warp_min(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// (value, node) minimum, the smaller node on equal values; every lane gets it
__device__ __forceinline__ void warp_argmin(float& v, int& n) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float v2 = __shfl_xor_sync(kFull, v, o);
    const int n2 = __shfl_xor_sync(kFull, n, o);
    if (v2 < v || (v2 == v && n2 < n)) {
      v = v2;
      n = n2;
    }
  }
}

// log(exp(x) + exp(y)) with -inf as the empty sum (symmetric in x, y)
__device__ __forceinline__ float lse2(float x, float y) {
  const float m = fmaxf(x, y);
  if (m == -f_inf()) return m;
  return m + log1pf(expf(-fabsf(x - y)));
}

__device__ __forceinline__ float warp_lse(float x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = lse2(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// One warp's view of its BDD; every array is indexed by node number.
struct LongCtx {
  LongBdd B;
  const int2* code;     // children of node n >= 2
  const int32_t* lvl;   // first node number of level h (h = 0..k)
  const int32_t* inp;   // in-arcs of node n >= 2: in[inp[n] .. inp[n + 1])
  const int32_t* in;    // parent << 1 | beta
  float* d;             // SP(r, .)
  float* t;             // SP(., T)
};

__device__ __forceinline__ LongCtx long_ctx(const DevArena& A, int b) {
  LongCtx c;
  c.B = A.longs[b];
  c.code = A.long_code + c.B.code_base - 2;
  c.lvl = A.long_lvl + c.B.lvl_base;
  c.inp = A.long_in_ptr + c.B.code_base - 2;
  c.in = A.long_in;
  c.d = A.long_d + c.B.cost_base;
  c.t = A.long_t + c.B.cost_base;
  return c;
}

// lambda^new = lambda - M^new + (alpha_ij S_i in mode 1, S_i / |J_i| in mode
// 0; the per-slot term the S reduction before the sweep wrote), with every
// rounding spelled out: M^new = omega (m1 - m0) is rounded on its own (the
// value stored as M), the mode-1 term enters by one fused multiply-add.  The
// general level loop and the narrow one (which loads the inputs levels ahead)
// therefore round alike whatever the compiler would contract.
template <int MODE>
__device__ __forceinline__ float long_lambda_new(float l, float Mn, float al, float av) {
  const float r = l - Mn;
  return MODE == 1 ? __fmaf_rn(al, av, r) : r + av;
}

// The records of a recording sweep handed the costs: the choices the
// recording sweep before it made in the same comparisons (keep: kLHi, the
// out-arc choices of SP(., T), for a forward sweep; the in-arcs of SP(r, .)
// for a backward one), the rest cleared for the sweep to write.
__device__ __forceinline__ void long_take_records(const LongCtx& c, const int32_t* prev, int32_t* meta, int32_t keep,
                                                  int lane) {
  const int e = c.lvl[c.B.k];
  for (int n = 2 + lane; n < e; n += kWarp) meta[n] = prev[n] & keep;
  __syncwarp();
}

// SP(., T) of every node under lam, levels bottom-up.  REC: the record of
// every node is rewritten with its hi-choice (0-arc on ties).
template <bool REC>
__device__ void long_cost_to_top(const LongCtx& c, const float* lam, int32_t* meta, int lane) {
  if (lane == 0) {
    c.t[kTopCode] = 0.0f;
    c.t[kBotCode] = f_inf();
  }
  __syncwarp();
  for (int h = c.B.k - 1; h >= 0; --h) {
    const float l = lam[c.B.slot_base + h];
    const int e = c.lvl[h + 1];
    for (int n = c.lvl[h] + lane; n < e; n += kWarp) {
      const int2 cc = c.code[n];
      const float tl = c.t[cc.x], th = l + c.t[cc.y];
      if (REC) {
        const bool take0 = cc.x != (int)kBotCode && tl <= th;
        c.t[n] = take0 ? tl : th;
        meta[n] = take0 ? 0 : kLHi;
      } else {
        c.t[n] = fminf(tl, th);
      }
    }
    __syncwarp();
  }
}

// SP(r, n) from the in-arcs of n (l = lambda of the parents' level).  REC:
// the argmin in-arc (first strictly smaller in (parent, beta) order) goes
// into n's record, whose hi-choice bit is kept when KEEP_HI.
template <bool REC, bool KEEP_HI>
__device__ __forceinline__ void relax_pull(const LongCtx& c, int n, float l, int32_t* meta) {
  float best = f_inf();
  int32_t arg = 0;
  const int e = c.inp[n + 1];
  for (int i = c.inp[n]; i < e; ++i) {
    const int32_t in = c.in[i];
    const float x = (in & 1) ? c.d[in >> 1] + l : c.d[in >> 1];
    if (REC) {
      if (x < best) {
        best = x;
        arg = in;
      }
    } else {
      best = fminf(best, x);
    }
  }
  c.d[n] = best;
  if (REC) meta[n] = (KEEP_HI ? (meta[n] & kLHi) : 0) | (arg << 1);
}

// SP(r, .) of every node under lam, levels top-down.  REC: records rewritten
// with the argmin in-arc (hi-choice cleared; the backward sweep sets it).
template <bool REC>
__device__ void long_cost_from_root(const LongCtx& c, const float* lam, int32_t* meta, int lane) {
  if (lane == 0) {
    c.d[2] = 0.0f;
    if (REC) meta[2] = 0;
  }
  __syncwarp();
  for (int h = 0; h + 1 < c.B.k; ++h) {
    const float l = lam[c.B.slot_base + h];
    const int e = c.lvl[h + 2];
    for (int n = c.lvl[h + 1] + lane; n < e; n += kWarp) relax_pull<REC, false>(c, n, l, meta);
    __syncwarp();
  }
}

// m0, m1 of level h: minima over its nodes of SP(r, v) + SP(child, T) by the
// 0- and the 1-arc (lambda not yet added); REC: argmin nodes v0, v1.
template <bool REC>
__device__ __forceinline__ void level_minima(const LongCtx& c, int h, int lane, float& b0, float& b1, int& v0,
                                             int& v1) {
  b0 = b1 = f_inf();
  v0 = v1 = INT_MAX;
  const int e = c.lvl[h + 1];
  for (int n = c.lvl[h] + lane; n < e; n += kWarp) {
    const int2 cc = c.code[n];
    const float dv = c.d[n];
    const float x0 = dv + c.t[cc.x], x1 = dv + c.t[cc.y];
    if (REC) {
      if (x0 < b0) {
        b0 = x0;
        v0 = n;
      }
      if (x1 < b1) {
        b1 = x1;
        v1 = n;
      }
    } else {
      b0 = fminf(b0, x0);
      b1 = fminf(b1, x1);
    }
  }
  if (REC) {
    warp_argmin(b0, v0);
    warp_argmin(b1, v1);
    // a level without a finite candidate cannot occur in a planned arena (it
    // would force a variable); the first node keeps the record in range
    if (v0 == INT_MAX) v0 = c.lvl[h];
    if (v1 == INT_MAX) v1 = c.lvl[h];
  } else {
    b0 = warp_min(b0);
    b1 = warp_min(b1);
  }
}

// ---- plain sweeps of narrow long BDDs --------------------------------------
// A long BDD whose levels all have at most 32 nodes (a long cardinality or
// assignment row) is swept by a segment of G lanes (G a power of two at least
// its widest level, 32 / G BDDs to a warp): node lvl[h] + s of level h
// belongs to the segment's lane s.  The costs of the sweep direction stay in
// a register, a pull reads a parent's (forward) or a child's (backward) by a
// shuffle inside the segment, minima are shuffles inside the segment, and
// what does not change during the sweep (level bounds, child codes, in-arcs,
// the opposite costs, lambda, omega, alpha, the averaging term) is loaded
// two levels ahead.  The general loop gives a whole warp to one level and
// reads every cost back through L2 after the lane that wrote it.  The FP32
// operations and their order (in-arcs ascending; minima are exact) are the
// general loop's, so the results are bit-identical; the costs still go to
// long_d / long_t for the sweep after.  The segments of a warp walk their
// own BDDs side by side; one whose BDD has fewer levels idles at the end.

// What lane s of a segment needs of one level (node f + s when s < w).
struct NarrowLevel {
  int f, w;         // first node number, width (0 outside the BDD's levels)
  int2 cc;          // children of node f + s (the bottom terminal twice off the level)
  int i0, deg;      // forward: its in-arcs in[i0 .. i0 + deg)
  int32_t in0, in1; // ... the first two of them
  float c0, c1;     // forward: SP(child, T) by the 0- / 1-arc; backward: SP(r, f + s) in c0
  float l, om, al, av;  // lambda, omega, alpha (mode 1) and the averaging term of the level's slot
};

// The lanes of one segment: the first lane, the lane within it, its size.
struct Seg {
  int base, s, G;
};

__device__ __forceinline__ float seg_min(float x, int G) {
  for (int o = G >> 1; o > 0; o >>= 1) x = fminf(x, __shfl_xor_sync(kFull, x, o));
  return x;
}

// First half of a level's loads: its node range and the codes (and, forward,
// the in-arc range) of node f + s.  L outside 0 .. k - 1 (k the segment's
// level count, 0 for a segment without a BDD) gives an empty level.  Loads
// are predicated into the fields (no select waits on them).
template <bool FWD>
__device__ __forceinline__ void narrow_nodes(const LongCtx& c, NarrowLevel& r, int L, int f, int e, int s, int k) {
  r.f = f;
  r.w = L >= 0 && L < k ? e - f : 0;
  const bool on = s < r.w;
  r.cc = make_int2((int)kBotCode, (int)kBotCode);
  if (on) r.cc = c.code[f + s];
  if (FWD) {
    r.i0 = 0;
    int i1 = 0;
    if (on) {
      r.i0 = c.inp[f + s];
      i1 = c.inp[f + s + 1];
    }
    r.deg = i1 - r.i0;
  } else {
    r.c0 = f_inf();
    if (on) r.c0 = c.d[f + s];
    r.c1 = 0.0f;
  }
}

// Second half: what depends on the first (forward: the children's SP(., T),
// the first two in-arcs) and the level's per-slot inputs (clamped to the
// BDD's levels; unused outside them).
template <bool FWD, int MODE>
__device__ __forceinline__ void narrow_inputs(const DevArena& A, const SweepArgs& a, const LongCtx& c,
                                              NarrowLevel& r, int L) {
  if (FWD) {
    r.in0 = 0;
    r.in1 = 0;
    if (r.deg > 0) r.in0 = c.in[r.i0];
    if (r.deg > 1) r.in1 = c.in[r.i0 + 1];
    r.c0 = c.t[r.cc.x];
    r.c1 = c.t[r.cc.y];
  }
  const int64_t q = c.B.slot_base + min(max(L, 0), c.B.k - 1);
  r.l = a.lam[q];
  r.om = MODE == 1 ? a.omega[q] : a.omega0;
  r.al = MODE == 1 ? a.alpha[q] : 0.0f;
  r.av = A.slot_avg[q];
}

// The update of one level from its minima (the general loop's arithmetic);
// the segment's lane 0 stores lambda and M when `store`.  Returns lambda^new.
template <int MODE>
__device__ __forceinline__ float narrow_update(const SweepArgs& a, const NarrowLevel& r, int64_t q, float x0,
                                               float x1, int G, bool store) {
  const float m0 = seg_min(x0, G), m1 = r.l + seg_min(x1, G);
  const float Mn = __fmul_rn(r.om, m1 - m0);
  const float ln = long_lambda_new<MODE>(r.l, Mn, r.al, r.av);
  if (store) {
    a.lam[q] = ln;
    a.M[q] = Mn;
  }
  return ln;
}

// Top-down over the levels: with UPD the forward sweep (min-marginals, the
// update, SP(r, .) under the new lambda; SP(., T) in long_t already), without
// it SP(r, .) under lambda alone (the first pass of a backward sweep that
// was not handed the costs).  Leaves SP(r, .) in long_d.  Every load that
// another load's address depends on is issued two levels before it is
// needed: while level h is worked on, level h + 2 receives its dependent
// loads (children's SP(., T), in-arcs, per-slot inputs), level h + 4 its
// node loads, and the end of level h + 6 is read.  Five level records take
// turns; the loop is unrolled by five so that they rotate by name (a
// register copy would wait for the loads in flight).  k: the segment's
// levels; kmax: the warp's.
template <int MODE, bool UPD>
__device__ __forceinline__ void narrow_down(const DevArena& A, const SweepArgs& a, const LongCtx& c, const Seg& g,
                                            int k, int kmax) {
  NarrowLevel r0, r1, r2, r3, r4;
  int st = k > 0 ? c.lvl[0] : 0;
  int en = k > 0 ? c.lvl[1] : st;  // levels 0 .. 3: node loads, 0 and 1 also the rest
  narrow_nodes<true>(c, r0, 0, st, en, g.s, k);
  narrow_inputs<true, MODE>(A, a, c, r0, 0);
  st = en;
  en = k > 1 ? c.lvl[2] : st;
  narrow_nodes<true>(c, r1, 1, st, en, g.s, k);
  narrow_inputs<true, MODE>(A, a, c, r1, 1);
  st = en;
  en = k > 2 ? c.lvl[3] : st;
  narrow_nodes<true>(c, r2, 2, st, en, g.s, k);
  st = en;
  en = k > 3 ? c.lvl[4] : st;
  narrow_nodes<true>(c, r3, 3, st, en, g.s, k);
  int eA = k > 4 ? c.lvl[5] : en;  // end of level h + 4
  int eB = k > 5 ? c.lvl[6] : eA;  // end of level h + 5
  float dreg = g.s == 0 ? 0.0f : f_inf();  // SP(r, .) of level h (level 0 is the root)
  if (g.s == 0 && k > 0) c.d[2] = 0.0f;
  auto level = [&](int h, NarrowLevel& s0, NarrowLevel& s1, NarrowLevel& s2, NarrowLevel& s3, NarrowLevel& s4) {
    narrow_inputs<true, MODE>(A, a, c, s2, h + 2);
    narrow_nodes<true>(c, s4, h + 4, s3.f + s3.w, eA, g.s, k);
    eA = eB;
    if (h + 7 <= k) eB = c.lvl[h + 7];
    const int maxdeg = (int)__reduce_max_sync(kFull, (unsigned)s1.deg);
    const float ln = UPD ? narrow_update<MODE>(a, s0, c.B.slot_base + h, dreg + s0.c0, dreg + s0.c1, g.G,
                                               g.s == 0 && h < k)
                         : s0.l;
    if (h + 1 < kmax) {
      // SP(r, .) of level h + 1: its in-arcs ascending, each parent's cost from the parent's lane
      float best = f_inf();
      for (int j = 0; j < maxdeg; ++j) {
        const bool has = j < s1.deg;
        int32_t in = j == 0 ? s1.in0 : s1.in1;
        if (j >= 2 && has) in = c.in[s1.i0 + j];
        const float dp = __shfl_sync(kFull, dreg, g.base + (((in >> 1) - s0.f) & (g.G - 1)));
        if (has) best = fminf(best, (in & 1) ? dp + ln : dp);
      }
      const bool on = g.s < s1.w;
      if (on) c.d[s1.f + g.s] = best;
      dreg = on ? best : f_inf();
    }
  };
  for (int h = 0; h < kmax; h += 5) {
    level(h, r0, r1, r2, r3, r4);
    if (h + 1 < kmax) level(h + 1, r1, r2, r3, r4, r0);
    if (h + 2 < kmax) level(h + 2, r2, r3, r4, r0, r1);
    if (h + 3 < kmax) level(h + 3, r3, r4, r0, r1, r2);
    if (h + 4 < kmax) level(h + 4, r4, r0, r1, r2, r3);
  }
}

// Bottom-up over the levels: with UPD the backward sweep (SP(r, .) in long_d
// already), without it SP(., T) under lambda alone (the first pass of a
// forward sweep that was not handed the costs).  Leaves SP(., T) in long_t
// (the terminals' entries are the caller's).  The children's costs come from
// the lanes of the level below, so only the level bounds feed addresses:
// while level h is worked on, level h - 3 receives its loads and the start
// of level h - 5 is read.  Four records take turns (the loop unrolled by
// four); step t of the warp is level k - 1 - t of each segment.
template <int MODE, bool UPD>
__device__ __forceinline__ void narrow_up(const DevArena& A, const SweepArgs& a, const LongCtx& c, const Seg& g,
                                          int k, int kmax) {
  NarrowLevel r0, r1, r2, r3;
  int en = k > 0 ? c.lvl[k] : 0;
  int st = k > 0 ? c.lvl[k - 1] : en;  // levels k - 1 .. k - 3 loaded before the loop
  narrow_nodes<false>(c, r0, k - 1, st, en, g.s, k);
  narrow_inputs<false, MODE>(A, a, c, r0, k - 1);
  en = st;
  st = k > 1 ? c.lvl[k - 2] : en;
  narrow_nodes<false>(c, r1, k - 2, st, en, g.s, k);
  narrow_inputs<false, MODE>(A, a, c, r1, k - 2);
  en = st;
  st = k > 2 ? c.lvl[k - 3] : en;
  narrow_nodes<false>(c, r2, k - 3, st, en, g.s, k);
  narrow_inputs<false, MODE>(A, a, c, r2, k - 3);
  int fA = k > 3 ? c.lvl[k - 4] : st;  // start of level h - 3
  int fB = k > 4 ? c.lvl[k - 5] : fA;  // start of level h - 4
  float treg = f_inf();                // SP(., T) of level h + 1 (none below the last level)
  auto level = [&](int t, NarrowLevel& s0, NarrowLevel& s1, NarrowLevel& s2, NarrowLevel& s3) {
    const int h = k - 1 - t;  // the segment's level (negative once its BDD is done)
    narrow_nodes<false>(c, s3, h - 3, fA, s2.f, g.s, k);
    narrow_inputs<false, MODE>(A, a, c, s3, h - 3);
    fA = fB;
    if (h >= 5) fB = c.lvl[h - 5];
    // the children's SP(., T): level h + 1 from its lanes, the terminals by code
    const int fn = s0.f + s0.w;
    float tlo = __shfl_sync(kFull, treg, g.base + ((s0.cc.x - fn) & (g.G - 1)));
    float thi = __shfl_sync(kFull, treg, g.base + ((s0.cc.y - fn) & (g.G - 1)));
    if (s0.cc.x < 2) tlo = s0.cc.x == (int)kTopCode ? 0.0f : f_inf();
    if (s0.cc.y < 2) thi = s0.cc.y == (int)kTopCode ? 0.0f : f_inf();
    const float ln = UPD ? narrow_update<MODE>(a, s0, c.B.slot_base + h, s0.c0 + tlo, s0.c0 + thi, g.G,
                                               g.s == 0 && h >= 0)
                         : s0.l;
    const float tn = fminf(tlo, ln + thi);
    const bool on = g.s < s0.w;
    if (on) c.t[s0.f + g.s] = tn;
    treg = on ? tn : f_inf();
  };
  for (int t = 0; t < kmax; t += 4) {
    level(t, r0, r1, r2, r3);
    if (t + 1 < kmax) level(t + 1, r1, r2, r3, r0);
    if (t + 2 < kmax) level(t + 2, r2, r3, r0, r1);
    if (t + 3 < kmax) level(t + 3, r3, r0, r1, r2);
  }
}

}  // namespace

template <int KIND, int MODE>
__global__ void __launch_bounds__(128) k_long_sweep(DevArena A, SweepArgs a) {
  constexpr bool REC = KIND == kFwdRec || KIND == kBwdRec;
  constexpr bool FWD = KIND == kFwd || KIND == kFwdRec;
  constexpr bool BWD = KIND == kBwd || KIND == kBwdRec;
  const int lane = threadIdx.x & 31;
  int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (KIND == kFwd || KIND == kBwd) {
    // the plain sweeps take the wide long BDDs here (k_long_narrow the others)
    if (b >= A.num_long - A.num_long_narrow) return;  // whole warp leaves
    b = A.long_order[A.num_long_narrow + b];
  } else if (b >= A.num_long) {
    return;
  }
  const LongCtx c = long_ctx(A, b);
  const int64_t sb = c.B.slot_base;
  const int k = c.B.k;
  int32_t* meta = REC ? a.rec_lmeta + c.B.cost_base : nullptr;
  const bool handed = (FWD || BWD) && a.cost_in != nullptr;

  if (FWD || KIND == kMinMarg) {
    if (!handed)
      long_cost_to_top<REC>(c, a.lam, meta, lane);
    else if (REC)
      long_take_records(c, a.lmeta_in + c.B.cost_base, meta, kLHi, lane);
    if (lane == 0) c.d[2] = 0.0f;
    __syncwarp();
    for (int h = 0; h < k; ++h) {
      float b0, b1;
      int v0, v1;
      level_minima<REC>(c, h, lane, b0, b1, v0, v1);
      const int64_t q = sb + h;
      const float l = a.lam[q];
      const float m0 = b0, m1 = l + b1;
      float ln = l;
      if (KIND == kMinMarg) {
        if (lane == 0) {
          a.M[q] = m0;
          a.out2[q] = m1;
        }
      } else {
        const float om = MODE == 1 ? a.omega[q] : a.omega0;
        const float Mn = __fmul_rn(om, m1 - m0);
        ln = long_lambda_new<MODE>(l, Mn, MODE == 1 ? a.alpha[q] : 0.0f, A.slot_avg[q]);
        if (lane == 0) {
          a.lam[q] = ln;
          a.M[q] = Mn;
          if (REC) {
            a.rec_lamin[q - A.long_slot_base] = make_int2(v0, v1);
            a.rec_diff[q] = m1 - m0;
          }
        }
      }
      if (h + 1 < k) {
        const int e = c.lvl[h + 2];
        for (int n = c.lvl[h + 1] + lane; n < e; n += kWarp) relax_pull<REC, true>(c, n, ln, meta);
      }
      __syncwarp();
    }
  } else if (BWD) {
    if (!handed)
      long_cost_from_root<REC>(c, a.lam, meta, lane);
    else if (REC)
      long_take_records(c, a.lmeta_in + c.B.cost_base, meta, ~kLHi, lane);
    if (lane == 0) {
      c.t[kTopCode] = 0.0f;
      c.t[kBotCode] = f_inf();
    }
    __syncwarp();
    for (int h = k - 1; h >= 0; --h) {
      float b0, b1;
      int v0, v1;
      level_minima<REC>(c, h, lane, b0, b1, v0, v1);
      const int64_t q = sb + h;
      const float l = a.lam[q];
      const float m0 = b0, m1 = l + b1;
      const float om = MODE == 1 ? a.omega[q] : a.omega0;
      const float Mn = __fmul_rn(om, m1 - m0);
      const float ln = long_lambda_new<MODE>(l, Mn, MODE == 1 ? a.alpha[q] : 0.0f, A.slot_avg[q]);
      if (lane == 0) {
        a.lam[q] = ln;
        a.M[q] = Mn;
        if (REC) {
          a.rec_lamin[q - A.long_slot_base] = make_int2(v0, v1);
          a.rec_diff[q] = m1 - m0;
        }
      }
      const int e = c.lvl[h + 1];
      for (int n = c.lvl[h] + lane; n < e; n += kWarp) {
        const int2 cc = c.code[n];
        const float tl = c.t[cc.x], th = ln + c.t[cc.y];
        if (REC) {
          const bool take0 = cc.x != (int)kBotCode && tl <= th;
          c.t[n] = take0 ? tl : th;
          meta[n] = (meta[n] & ~kLHi) | (take0 ? 0 : kLHi);
        } else {
          c.t[n] = fminf(tl, th);
        }
      }
      __syncwarp();
    }
  } else {
    // kEnergy / kSeed: SP(., T) under lambda
    long_cost_to_top<false>(c, a.lam, nullptr, lane);
  }

  if (KIND == kSeed && lane == 0) {
    // walk the minimising path from the root: 0-arc on ties
    int n = 2;
    for (int h = 0; h < k; ++h) {
      const int2 cc = c.code[n];
      const bool take0 = cc.x != (int)kBotCode &&
                         (cc.y == (int)kBotCode || c.t[cc.x] <= a.lam[sb + h] + c.t[cc.y]);
      a.M[sb + h] = take0 ? 0.f : 1.f;
      n = take0 ? cc.x : cc.y;
    }
  }
  if ((BWD || KIND == kEnergy) && a.E != nullptr && lane == 0) a.E[c.B.row] = c.t[2];  // E^j = SP(r, T)
}

// Plain forward / backward sweep of the narrow long BDDs (the head of
// long_order), 32 / G of them to a warp, G = A.long_lanes lanes each (see
// narrow_down / narrow_up).  A sweep not handed the costs first computes the
// opposite ones the same way.
template <int KIND, int MODE>
__global__ void __launch_bounds__(128) k_long_narrow(DevArena A, SweepArgs a) {
  constexpr bool FWD = KIND == kFwd;
  const int lane = threadIdx.x & 31;
  const int G = A.long_lanes;
  const int first = (blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5)) * (kWarp / G);
  if (first >= A.num_long_narrow) return;  // whole warp leaves
  Seg g;
  g.s = lane & (G - 1);
  g.base = lane - g.s;
  g.G = G;
  const int i = first + lane / G;
  const bool act = i < A.num_long_narrow;  // segments past the list sweep nothing
  const LongCtx c = long_ctx(A, A.long_order[act ? i : first]);
  const int k = act ? c.B.k : 0;
  const int kmax = (int)__reduce_max_sync(kFull, (unsigned)k);
  const bool handed = a.cost_in != nullptr;
  if (FWD) {
    if (!handed) {
      if (g.s == 0 && act) {
        c.t[kTopCode] = 0.0f;
        c.t[kBotCode] = f_inf();
      }
      narrow_up<MODE, false>(A, a, c, g, k, kmax);
      __syncwarp();
    }
    narrow_down<MODE, true>(A, a, c, g, k, kmax);
  } else {
    if (!handed) {
      narrow_down<MODE, false>(A, a, c, g, k, kmax);
      __syncwarp();
    }
    if (g.s == 0 && act) {
      c.t[kTopCode] = 0.0f;
      c.t[kBotCode] = f_inf();
    }
    narrow_up<MODE, true>(A, a, c, g, k, kmax);
    if (a.E != nullptr && g.s == 0 && act) a.E[c.B.row] = c.t[2];  // E^j = SP(r, T), written by this lane
  }
}

// Smoothed subproblem (soft-min reading) and its marginals P(x_i = 1):
// B(v) = log-sum-exp over v-T paths (in long_t), F(v) over r-v paths (in
// long_d), log Z = B(root).
__global__ void __launch_bounds__(128) k_long_smoothed(DevArena A, const float* lam, float a_s, float* E_a,
                                                       float* marg) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= A.num_long) return;
  const LongCtx c = long_ctx(A, b);
  const int64_t sb = c.B.slot_base;
  const int k = c.B.k;
  const float inv_a = 1.0f / a_s;
  if (lane == 0) {
    c.t[kTopCode] = 0.0f;  // log 1
    c.t[kBotCode] = -f_inf();
  }
  __syncwarp();
  for (int h = k - 1; h >= 0; --h) {
    const float wgt = -lam[sb + h] * inv_a;
    const int e = c.lvl[h + 1];
    for (int n = c.lvl[h] + lane; n < e; n += kWarp) {
      const int2 cc = c.code[n];
      c.t[n] = lse2(c.t[cc.x], wgt + c.t[cc.y]);
    }
    __syncwarp();
  }
  const float logZ = c.t[2];
  if (E_a && lane == 0) E_a[c.B.row] = -a_s * logZ;
  if (lane == 0) c.d[2] = 0.0f;
  __syncwarp();
  for (int h = 0; h < k; ++h) {
    const float wgt = -lam[sb + h] * inv_a;
    float acc = -f_inf();
    const int e = c.lvl[h + 1];
    for (int n = c.lvl[h] + lane; n < e; n += kWarp) acc = lse2(acc, c.d[n] + wgt + c.t[c.code[n].y]);
    acc = warp_lse(acc);
    if (lane == 0) marg[sb + h] = expf(acc - logZ);
    if (h + 1 < k) {
      const int e2 = c.lvl[h + 2];
      for (int n = c.lvl[h + 1] + lane; n < e2; n += kWarp) {
        float f = -f_inf();
        const int ie = c.inp[n + 1];
        for (int i = c.inp[n]; i < ie; ++i) {
          const int32_t in = c.in[i];
          f = lse2(f, (in & 1) ? c.d[in >> 1] + wgt : c.d[in >> 1]);
        }
        c.d[n] = f;
      }
    }
    __syncwarp();
  }
}

// Adjoint of one sweep over a long BDD (the reverse of k_long_sweep<kFwdRec
// or kBwdRec>, whose records it reads): the steps of k_adjoint with the
// gradients of SP(., T) and SP(r, .) per node in the backward workspace
// (long_a1, long_a2) and every routing step a pull (each node gathers from
// its two children or its in-arcs).
template <int FWD, int MODE>
__global__ void __launch_bounds__(128) k_long_adjoint(DevArena A, AdjArgs a) {
  const int lane = threadIdx.x & 31;
  const int b = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (b >= A.num_long) return;
  const LongCtx c = long_ctx(A, b);
  const int64_t sb = c.B.slot_base;
  const int k = c.B.k;
  const int32_t* meta = a.rec_lmeta + c.B.cost_base;
  float* A1 = a.long_a1 + c.B.cost_base;  // gradient of SP(., T)
  float* A2 = a.long_a2 + c.B.cost_base;  // gradient of SP(r, .)
  for (int n = lane; n < c.B.nn + 2; n += kWarp) {
    A1[n] = 0.0f;
    A2[n] = 0.0f;
  }
  __syncwarp();

  // the update of level h reversed (g = gradient of lambda^new_h with the
  // path-cost contributions of its level added); lane 0 writes
  auto reverse_level = [&](int h, float g) {
    const int64_t q = sb + h;
    const int v = __ldg(A.slot_var + q);
    const float S = a.S_in[v];
    const float al = MODE == 1 ? a.alpha[q] : __ldg(A.invdeg + v);
    const float om = MODE == 1 ? a.omega[q] : a.omega0;
    const float md = (a.seed_M ? a.seed_M[q] : 0.0f) + (a.sdot_next ? a.sdot_next[v] : 0.0f);
    const float Mt = md - g;
    const float dm1 = om * Mt, dm0 = -om * Mt;
    if (lane == 0) {
      const int2 am = a.rec_lamin[q - A.long_slot_base];
      a.sdot[q] = al * g;
      if (a.g_alpha) a.g_alpha[q] = a.g_alpha[q] + g * S;
      if (a.g_omega) a.g_omega[q] = a.g_omega[q] + Mt * a.rec_diff[q];
      a.g_lam[q] = g + dm1;
      A2[am.x] += dm0;
      A1[c.code[am.x].x] += dm0;  // terminals absorb into their unused entries
      A2[am.y] += dm1;
      A1[c.code[am.y].y] += dm1;
    }
    __syncwarp();
  };
  // gradients of SP(., T) of level h leave along the argmin out-arcs: those
  // of the 1-arcs are returned (their sum), level h + 1 pulls them in
  auto route_out = [&](int h) -> float {
    float part = 0.0f;
    const int e = c.lvl[h + 1];
    for (int n = c.lvl[h] + lane; n < e; n += kWarp)
      if (meta[n] & kLHi) part += A1[n];
    if (h + 1 < k) {
      const int e2 = c.lvl[h + 2];
      for (int w = c.lvl[h + 1] + lane; w < e2; w += kWarp) {
        float acc = A1[w];
        const int ie = c.inp[w + 1];
        for (int i = c.inp[w]; i < ie; ++i) {
          const int32_t in = c.in[i];
          if ((meta[in >> 1] & kLHi) == (in & 1)) acc += A1[in >> 1];
        }
        A1[w] = acc;
      }
    }
    return warp_sum(part);
  };
  // gradients of SP(r, .) of level h (>= 1) go to the argmin parents on level
  // h - 1 (pull over the parents' children, ascending); those entering by a
  // 1-arc are returned (their sum)
  auto route_in = [&](int h) -> float {
    float part = 0.0f;
    const int e = c.lvl[h + 1];
    for (int n = c.lvl[h] + lane; n < e; n += kWarp)
      if (meta[n] & kLBeta) part += A2[n];
    const int ep = c.lvl[h];
    for (int n = c.lvl[h - 1] + lane; n < ep; n += kWarp) {
      const int2 cc = c.code[n];
      float acc = A2[n];
      const bool tlo = cc.x >= 2 && (meta[cc.x] >> 1) == (n << 1);
      const bool thi = cc.y >= 2 && (meta[cc.y] >> 1) == ((n << 1) | 1);
      if (cc.x <= cc.y) {
        if (tlo) acc += A2[cc.x];
        if (thi) acc += A2[cc.y];
      } else {
        if (thi) acc += A2[cc.y];
        if (tlo) acc += A2[cc.x];
      }
      A2[n] = acc;
    }
    return warp_sum(part);
  };

  if (FWD) {
    for (int h = k - 1; h >= 0; --h) {
      float g = a.g_lam[sb + h];
      // SP(r, .) of level h+1 was relaxed from level h with lambda^new_h
      if (h + 1 < k) g += route_in(h + 1);
      __syncwarp();
      reverse_level(h, g);
    }
    // SP(., T) under lambda^old: its gradient flows top-down
    for (int h = 0; h < k; ++h) {
      const float part = route_out(h);
      if (lane == 0) a.g_lam[sb + h] += part;
      __syncwarp();
    }
  } else {
    for (int h = 0; h < k; ++h) {
      // SP(., T) of level h was recomputed with lambda^new_h
      const float g = a.g_lam[sb + h] + route_out(h);
      __syncwarp();
      reverse_level(h, g);
    }
    // SP(r, .) under lambda^old: its gradient flows bottom-up
    for (int h = k - 1; h >= 1; --h) {
      const float part = route_in(h);
      if (lane == 0) a.g_lam[sb + h - 1] += part;
      __syncwarp();
    }
  }
}

namespace {

constexpr int kLongWarps = 4;  // BDDs (warps) per CTA

int long_grid(const DevArena& A) { return (A.num_long + kLongWarps - 1) / kLongWarps; }

template <int KIND>
void launch_long_kind(const DevArena& A, const SweepArgs& a, cudaStream_t st) {
  int grid = long_grid(A);
  if constexpr (KIND == kFwd || KIND == kBwd) {
    if (A.num_long_narrow > 0) {
      const int per = kWarp / A.long_lanes;
      const int warps = (A.num_long_narrow + per - 1) / per;
      const int ng = (warps + kLongWarps - 1) / kLongWarps;
      if (a.mode == 1)
        k_long_narrow<KIND, 1><<<ng, kLongWarps * kWarp, 0, st>>>(A, a);
      else
        k_long_narrow<KIND, 0><<<ng, kLongWarps * kWarp, 0, st>>>(A, a);
    }
    grid = (A.num_long - A.num_long_narrow + kLongWarps - 1) / kLongWarps;
    if (grid == 0) return;
  }
  if (a.mode == 1)
    k_long_sweep<KIND, 1><<<grid, kLongWarps * kWarp, 0, st>>>(A, a);
  else
    k_long_sweep<KIND, 0><<<grid, kLongWarps * kWarp, 0, st>>>(A, a);
}

}  // namespace

void launch_long_sweep(int kind, const DevArena& A, const SweepArgs& a, cudaStream_t st) {
  if (A.num_long == 0) return;
  switch (kind) {
    case kFwd: launch_long_kind<kFwd>(A, a, st); break;
    case kBwd: launch_long_kind<kBwd>(A, a, st); break;
    case kFwdRec: launch_long_kind<kFwdRec>(A, a, st); break;
    case kBwdRec: launch_long_kind<kBwdRec>(A, a, st); break;
    case kMinMarg: k_long_sweep<kMinMarg, 0><<<long_grid(A), kLongWarps * kWarp, 0, st>>>(A, a); break;
    case kEnergy: k_long_sweep<kEnergy, 0><<<long_grid(A), kLongWarps * kWarp, 0, st>>>(A, a); break;
    default: k_long_sweep<kSeed, 0><<<long_grid(A), kLongWarps * kWarp, 0, st>>>(A, a); break;
  }
}

void launch_long_smoothed(const DevArena& A, const float* lam, float a_s, float* E_a, float* marg, cudaStream_t st) {
  if (A.num_long == 0) return;
  k_long_smoothed<<<long_grid(A), kLongWarps * kWarp, 0, st>>>(A, lam, a_s, E_a, marg);
}

void launch_long_adjoint(bool forward, const DevArena& A, const AdjArgs& a, cudaStream_t st) {
  if (A.num_long == 0) return;
  const int g = long_grid(A), t = kLongWarps * kWarp;
  if (forward)
    a.mode == 1 ? k_long_adjoint<1, 1><<<g, t, 0, st>>>(A, a) : k_long_adjoint<1, 0><<<g, t, 0, st>>>(A, a);
  else
    a.mode == 1 ? k_long_adjoint<0, 1><<<g, t, 0, st>>>(A, a) : k_long_adjoint<0, 0><<<g, t, 0, st>>>(A, a);
}

}  // namespace dg
