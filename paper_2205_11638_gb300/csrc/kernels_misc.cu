// kernels_misc.cu -- per-variable and per-instance kernels around the sweeps:
// the deferred min-marginal sums S_i (Alg. 1, lambda update), the FP64
// re-projection onto the dual constraint of (D), the initial split of c and
// the FP64 lower bound (Def. 2 with the unary term of the deferred
// min-marginals).
#include "kernels.h"

namespace dg {

// S_i = sum_{j in J_i} M_ij over the variable's slots in fixed order.  With
// renorm the same pass re-projects lambda onto sum_j (lambda_ij + M_ij) = c_i
// (the invariant of the proof of Prop. 1): the FP64 residual
// r_i = c_i - sum_j (lambda_ij + M_ij) is spread with the averaging weights.
// With SCATTER every slot of the variable also receives the averaging term
// the sweeps add (Sbar_i = S_i / |J_i| in mode 0, S_i in mode 1, which they
// multiply by alpha_ij), so that a sweep reads it with the slot's other
// inputs instead of gathering it per variable.
template <bool RENORM, bool SCATTER>
__global__ void __launch_bounds__(256) k_reduce_S(DevArena A, const float* __restrict__ M, float* lam,
                                                   const float* __restrict__ alpha, int mode) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  float s = 0.f;
  if (!RENORM) {
    // the first kEll slots come from the ELL columns (coalesced, no var_ptr
    // needed), all loaded before their M values, which are all loaded before
    // the first addition; the order of additions is the plain loop's
    int q[kEll];
#pragma unroll
    for (int r = 0; r < kEll; ++r) q[r] = __ldg(A.var_ell + (int64_t)r * A.n + i);
    const bool more = q[kEll - 1] <= -2;
    if (more) q[kEll - 1] = -2 - q[kEll - 1];
    float mv[kEll];
#pragma unroll
    for (int r = 0; r < kEll; ++r) mv[r] = q[r] >= 0 ? M[q[r]] : 0.f;
#pragma unroll
    for (int r = 0; r < kEll; ++r)
      if (q[r] >= 0) s += mv[r];
    int b = 0, e = 0;
    if (more) {
      b = __ldg(A.var_ptr + i) + kEll;
      e = __ldg(A.var_ptr + i + 1);
      if (e - b > kWide - kEll) return;  // a wide variable: k_reduce_wide's
      for (int k = b; k < e; ++k) s += M[__ldg(A.var_slots + k)];
    }
    const float sbar = __ldg(A.invdeg + i) * s;
    A.S[i] = s;
    A.Sbar[i] = sbar;
    if (SCATTER) {
      const float t = mode == 1 ? s : sbar;
#pragma unroll
      for (int r = 0; r < kEll; ++r)
        if (q[r] >= 0) A.slot_avg[q[r]] = t;
      for (int k = b; k < e; ++k) A.slot_avg[__ldg(A.var_slots + k)] = t;
    }
    return;
  }
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  double tot = 0.0;
  for (int k = b; k < e; ++k) {
    const int q = __ldg(A.var_slots + k);
    const float mk = M[q];
    s += mk;
    tot += (double)lam[q] + (double)mk;
  }
  const float sbar = __ldg(A.invdeg + i) * s;
  A.S[i] = s;
  A.Sbar[i] = sbar;
  if (e > b) {
    const double r = A.c[i] - tot;
    const float inv = __ldg(A.invdeg + i);
    const float t = mode == 1 ? s : sbar;
    for (int k = b; k < e; ++k) {
      const int q = __ldg(A.var_slots + k);
      const double w = mode == 1 ? (double)alpha[q] : (double)inv;
      lam[q] = (float)((double)lam[q] + w * r);
      if (SCATTER) A.slot_avg[q] = t;
    }
  }
}

// k_reduce_S<false, SCATTER> for the wide variables (more than kWide slots),
// one warp each: the lanes load 32 of the variable's M values at a time and
// every lane adds them in slot order (the plain loop's order, so S is the
// same to the bit); lane 0 stores S.
template <bool SCATTER>
__global__ void __launch_bounds__(256) k_reduce_wide(DevArena A, const float* __restrict__ M, int mode) {
  constexpr unsigned kAll = 0xffffffffu;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (w >= A.num_wide) return;  // the whole warp
  const int i = __ldg(A.wide_vars + w);
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  float s = 0.f;
  for (int c = b; c < e; c += 32) {
    const float v = c + lane < e ? M[__ldg(A.var_slots + c + lane)] : 0.f;
    const int cnt = min(32, e - c);
    for (int j = 0; j < cnt; ++j) s += __shfl_sync(kAll, v, j);
  }
  const float sbar = __ldg(A.invdeg + i) * s;
  if (lane == 0) {
    A.S[i] = s;
    A.Sbar[i] = sbar;
  }
  if (SCATTER) {
    const float t = mode == 1 ? s : sbar;
    for (int k = b + lane; k < e; k += 32) A.slot_avg[__ldg(A.var_slots + k)] = t;
  }
}

__global__ void k_init(DevArena A, float* lam, float* M) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.num_slots) return;
  const int var = __ldg(A.slot_var + q);
  float l = 0.f;
  if (var >= 0) {
    const int deg = __ldg(A.var_ptr + var + 1) - __ldg(A.var_ptr + var);
    l = (float)(A.c[var] / (double)deg);
  }
  lam[q] = l;
  M[q] = 0.f;
}

// One partial sum per chunk: rows contribute E^j, variables min(0, S_i)
// (variables no row covers add min(0, c_i), a constant per instance that
// k_lb_final adds).  FP64 arithmetic is slow on this
// part, so every thread accumulates its float32 terms with Knuth's TwoSum
// (an error-free transformation: the running sum and its exact rounding
// error, both float32), and only the per-thread results are combined in
// FP64, in a fixed order (deterministic for a given layout).
__global__ void __launch_bounds__(256) k_lb_partial(DevArena A) {
  const int4 ch = __ldg(A.lb_chunks + blockIdx.x);
  float hi = 0.f, lo = 0.f;
  // variables no row covers have S_i = 0 (an empty sum), so min(0, S_i) adds
  // nothing for them; their cost term is the per-instance constant inst_unc
  const bool rows = ch.y == 0;
  const float* src = rows ? A.E : A.S;
  constexpr int kU = 4;  // loads of kU elements are issued before their sums
  for (int x0 = ch.z + threadIdx.x; x0 < ch.w; x0 += kU * blockDim.x) {
    float v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int x = x0 + u * blockDim.x;
      const float y = x < ch.w ? src[x] : 0.f;
      v[u] = rows ? y : fminf(0.f, y);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const float s = hi + v[u];
      const float bp = s - hi;
      lo += (hi - (s - bp)) + (v[u] - bp);
      hi = s;
    }
  }
  // float-float tree over the block (TwoSum at every step), one conversion
  // to float64 per block: FP64 arithmetic is slow on this part
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_down_sync(0xFFFFFFFFu, hi, o);
    const float l2 = __shfl_down_sync(0xFFFFFFFFu, lo, o);
    const float s = hi + h2;
    const float bp = s - hi;
    lo = lo + l2 + ((hi - (s - bp)) + (h2 - bp));
    hi = s;
  }
  __shared__ float rh[8], rl[8];
  if ((threadIdx.x & 31) == 0) {
    rh[threadIdx.x >> 5] = hi;
    rl[threadIdx.x >> 5] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += (double)rh[w] + (double)rl[w];
    A.lb_part[blockIdx.x] = t;
  }
}

// One CTA per instance sums the instance's chunk partials (strided per
// thread, then a fixed tree): deterministic for a given layout.
__global__ void __launch_bounds__(256) k_lb_final(DevArena A, double* lb) {
  const int k = blockIdx.x;
  double t = 0.0;
  for (int c = A.inst_chunk_ptr[k] + threadIdx.x; c < A.inst_chunk_ptr[k + 1]; c += blockDim.x) t += A.lb_part[c];
  __shared__ double red[8];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = t;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    lb[k] = s + A.inst_unc[k];
  }
}

__global__ void k_seed_M(DevArena A, float* gM) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.num_slots) return;
  const int var = __ldg(A.slot_var + q);
  gM[q] = (var >= 0 && A.S[var] < 0.f) ? 1.f : 0.f;
}

// Between two adjoint sweeps: the S-dot of a variable (sum of its slots'
// contributions) and the per-slot inputs of the next adjoint sweep.
__global__ void __launch_bounds__(256) k_slot_inputs(DevArena A, const float* __restrict__ x,
                                                      const float* __restrict__ sd_in, float* out_var,
                                                      const float* __restrict__ S_var, float2* slot_in) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n) return;
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  if (e - b > kWide) return;  // a wide variable: k_slot_inputs_wide's
  float s = 0.f;
  if (x)
    for (int k = b; k < e; ++k) s += x[__ldg(A.var_slots + k)];
  else if (sd_in)
    s = sd_in[i];
  if (out_var) out_var[i] = s;
  if (slot_in) {
    const float2 t = make_float2(s, S_var ? S_var[i] : 0.f);
    for (int k = b; k < e; ++k) slot_in[__ldg(A.var_slots + k)] = t;
  }
}

// k_slot_inputs for the wide variables, one warp each (the sum in slot order
// as in k_reduce_wide).
__global__ void __launch_bounds__(256) k_slot_inputs_wide(DevArena A, const float* __restrict__ x,
                                                           const float* __restrict__ sd_in, float* out_var,
                                                           const float* __restrict__ S_var, float2* slot_in) {
  constexpr unsigned kAll = 0xffffffffu;
  const int w = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  if (w >= A.num_wide) return;  // the whole warp
  const int i = __ldg(A.wide_vars + w);
  const int b = __ldg(A.var_ptr + i), e = __ldg(A.var_ptr + i + 1);
  float s = 0.f;
  if (x) {
    for (int c = b; c < e; c += 32) {
      const float v = c + lane < e ? x[__ldg(A.var_slots + c + lane)] : 0.f;
      const int cnt = min(32, e - c);
      for (int j = 0; j < cnt; ++j) s += __shfl_sync(kAll, v, j);
    }
  } else if (sd_in) {
    s = sd_in[i];
  }
  if (out_var && lane == 0) out_var[i] = s;
  if (slot_in) {
    const float2 t = make_float2(s, S_var ? S_var[i] : 0.f);
    for (int k = b + lane; k < e; k += 32) slot_in[__ldg(A.var_slots + k)] = t;
  }
}

__global__ void k_slot_invdeg(DevArena A) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.num_slots) return;
  const int var = __ldg(A.slot_var + q);
  A.slot_invdeg[q] = var >= 0 ? __ldg(A.invdeg + var) : 0.f;
}

void launch_fill_slot_invdeg(const DevArena& A, cudaStream_t st) {
  const int T = 256;
  const int64_t G = (A.num_slots + T - 1) / T;
  if (G > 0) k_slot_invdeg<<<(unsigned)G, T, 0, st>>>(A);
}

__global__ void k_gather_var(DevArena A, const float* __restrict__ v, float* out) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= A.num_slots) return;
  const int var = __ldg(A.slot_var + q);
  out[q] = var >= 0 ? v[var] : 0.f;
}

void launch_slot_inputs(const DevArena& A, const float* x, const float* sd_in, float* out_var, const float* S_var,
                        float2* slot_in, cudaStream_t st) {
  const int T = 256;
  const int G = (A.n + T - 1) / T;
  if (G > 0) k_slot_inputs<<<G, T, 0, st>>>(A, x, sd_in, out_var, S_var, slot_in);
  if (A.num_wide > 0)
    k_slot_inputs_wide<<<(A.num_wide + 7) / 8, 256, 0, st>>>(A, x, sd_in, out_var, S_var, slot_in);
}

void launch_gather_var(const DevArena& A, const float* v, float* out_slot, cudaStream_t st) {
  const int T = 256;
  const int64_t G = (A.num_slots + T - 1) / T;
  if (G > 0) k_gather_var<<<(unsigned)G, T, 0, st>>>(A, v, out_slot);
}

void launch_reduce_S(const DevArena& A, const float* M, float* lam, const float* alpha, int mode, bool renorm,
                     cudaStream_t st, bool for_sweep) {
  const int T = 256;
  const int G = (A.n + T - 1) / T;
  if (G == 0) return;
  if (renorm)
    for_sweep ? k_reduce_S<true, true><<<G, T, 0, st>>>(A, M, lam, alpha, mode)
              : k_reduce_S<true, false><<<G, T, 0, st>>>(A, M, lam, alpha, mode);
  else {
    for_sweep ? k_reduce_S<false, true><<<G, T, 0, st>>>(A, M, lam, alpha, mode)
              : k_reduce_S<false, false><<<G, T, 0, st>>>(A, M, lam, alpha, mode);
    if (A.num_wide > 0)
      for_sweep ? k_reduce_wide<true><<<(A.num_wide + 7) / 8, 256, 0, st>>>(A, M, mode)
                : k_reduce_wide<false><<<(A.num_wide + 7) / 8, 256, 0, st>>>(A, M, mode);
  }
}

void launch_init(const DevArena& A, float* lam, float* M, cudaStream_t st) {
  const int T = 256;
  const int64_t G = (A.num_slots + T - 1) / T;
  if (G > 0) k_init<<<(unsigned)G, T, 0, st>>>(A, lam, M);
}

void launch_lower_bound(const DevArena& A, double* lb, cudaStream_t st) {
  if (A.num_lb_chunks > 0) k_lb_partial<<<A.num_lb_chunks, 256, 0, st>>>(A);
  k_lb_final<<<A.num_inst, 256, 0, st>>>(A, lb);
}

void launch_seed_M(const DevArena& A, float* gM, cudaStream_t st) {
  const int T = 256;
  const int64_t G = (A.num_slots + T - 1) / T;
  if (G > 0) k_seed_M<<<(unsigned)G, T, 0, st>>>(A, gM);
}

}  // namespace dg
