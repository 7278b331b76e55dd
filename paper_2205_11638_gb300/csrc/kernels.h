// kernels.h -- host-side launchers of the libdg kernels (internal).
#pragma once

#include <cuda_runtime.h>

#include "dg_internal.h"

namespace dg {

// kFwdRec / kBwdRec: the update sweeps that also record, for the adjoint,
// the argmins of their min-sum recursions (see SweepArgs::rec_*).
enum SweepKind : int { kFwd = 0, kBwd = 1, kMinMarg = 2, kEnergy = 3, kSeed = 4, kFwdRec = 5, kBwdRec = 6 };

struct SweepArgs {
  float* lam;          // in/out (read-only for kMinMarg/kEnergy/kSeed)
  float* M;            // out: M (kFwd/kBwd), m0 (kMinMarg), g_lam (kSeed)
  float* out2;         // out: m1 (kMinMarg)
  const float* omega;  // mode 1
  const float* alpha;  // mode 1
  float omega0;        // mode 0
  int mode;
  float* E;            // nullable: E^j per original row (kBwd, kEnergy)
  // Hand-off of App. B's path costs from one update sweep (plain or
  // recording) to the next (per node and lane of the tiles, in the layout of
  // the child codes; both nullable).  cost_out: the costs of the sweep's own
  // direction under the outgoing lambda, which it computes anyway (SP(r, .)
  // after a forward sweep, SP(., T) after a backward one).  cost_in: the
  // costs opposite to the sweep direction under the incoming lambda (SP(., T)
  // for a forward sweep, SP(r, .) for a backward one), read instead of
  // recomputed; valid when lambda has not changed since the sweep that wrote
  // them.  The two may be the same array: each warp stages its tile's part
  // before it writes it.
  float* cost_out;
  const float* cost_in;
  // kFwdRec / kBwdRec with cost_in: the node records (rec_meta, and
  // rec_lmeta for the long BDDs) of the recording sweep that wrote the costs
  const uint16_t* meta_in;
  const int32_t* lmeta_in;
  // argmin records (kFwdRec, kBwdRec), read back by the adjoint of the sweep:
  uint16_t* rec_meta;  // per node (layout of the child codes): in-arc parent | beta << 8 | hi-choice << 9
  uint16_t* rec_amin;  // per slot: argmin node of m0 | argmin node of m1 << 8
  float* rec_diff;     // per slot: m1 - m0
  // ... for the long BDDs: per node (cost scratch index) in-arc << 1 |
  // hi-choice, per long slot (from long_slot_base) the argmin nodes of m0, m1
  int32_t* rec_lmeta;
  int2* rec_lamin;
};

// The caller's stream plus kStreams - 1 auxiliary streams of an arena: the
// launch groups of one sweep fork from the caller's stream, run on their
// assigned streams concurrently, and join back before the next step.
struct StreamSet {
  cudaStream_t main = nullptr;
  cudaStream_t aux[kStreams - 1] = {};
  cudaEvent_t fork = nullptr;
  cudaEvent_t join[kStreams - 1] = {};
  bool ready = false;
  int n = kStreams;  // streams in use (1: everything on main)
  cudaStream_t of(int k) const {
    const int j = n > 0 ? k % n : 0;
    return j == 0 || !ready ? main : aux[j - 1];
  }
  void begin() const;  // fork
  void end() const;    // join
};

cudaError_t set_sweep_smem_limit(size_t bytes);
// Dynamic shared memory one CTA may use; launchers put fewer warps in a CTA
// when their tiles need more.
void set_cta_smem_cap(size_t bytes);
int best_warps_per_cta(size_t region, int max_wpc, size_t cta_cap);
void launch_sweep(int kind, const DevArena& A, const SweepArgs& a, int threads, const LaunchGroup* groups,
                  int num_groups, const StreamSet& ss);

// S_i = sum_{k in J_i} M_ik in fixed slot order; with renorm, also
// lambda_ij += alpha_ij * (c_i - sum_k (lambda_ik + M_ik)) computed in FP64.
// With for_sweep, also the mode's averaging term of every slot into
// A.slot_avg, where the next sweeps read it.
void launch_reduce_S(const DevArena& A, const float* M, float* lam, const float* alpha, int mode, bool renorm,
                     cudaStream_t st, bool for_sweep);
void launch_init(const DevArena& A, float* lam, float* M, cudaStream_t st);
// per-instance FP64 lower bound from A.E and A.S
void launch_lower_bound(const DevArena& A, double* lb_out, cudaStream_t st);
void launch_seed_M(const DevArena& A, float* g_M, cudaStream_t st);

// Backpropagation through one sweep (kernels_adjoint.cu).
struct AdjArgs {
  const uint16_t* rec_meta;  // the records of the sweep (SweepArgs::rec_*)
  const uint16_t* rec_amin;
  const float* rec_diff;
  const float* S_in;       // S at the start of the sweep (per variable)
  const float* omega;      // mode 1
  const float* alpha;      // mode 1
  float omega0;            // mode 0
  int mode;
  const float* seed_M;     // nullable: gradient of the sweep's M output (per slot)
  const float* sdot_next;  // nullable: S-dot of the next sweep (per variable)
  // per slot: {S-dot of the next sweep, S at the sweep's start} of the
  // slot's variable (launch_slot_inputs), what the tiles' reverse reads
  // instead of gathering per variable (with DevArena::slot_invdeg for the
  // weights of mode 0); the long BDDs use the per-variable arrays above
  const float2* slot_in;
  float* g_lam;            // in: gradient of lambda after the sweep; out: before
  float* g_omega;          // accumulated (nullable: not computed)
  float* g_alpha;          // accumulated (nullable: not computed)
  float* sdot;             // out: alpha * (gradient of lambda after the sweep), per slot
  // long BDDs: the records of the sweep and per-node gradient scratch of
  // SP(., T) and SP(r, .)
  const int32_t* rec_lmeta;
  const int2* rec_lamin;
  float* long_a1;
  float* long_a2;
};
cudaError_t set_adjoint_smem_limit(size_t bytes);
void launch_adjoint_sweep(bool forward, const DevArena& A, const AdjArgs& a, const AdjGroup* groups, int num_groups,
                          size_t cta_smem_cap, const StreamSet& ss);
// Per variable i: s_i = sum over the slots q of i of x[q] (fixed order), or
// sd_in[i] when x is NULL (0 when both are); out_var[i] = s_i (nullable);
// and, when slot_in is not NULL, slot_in[q] = {s_i, S_var[i] (0 if NULL)}
// for every slot q of i.
void launch_slot_inputs(const DevArena& A, const float* x, const float* sd_in, float* out_var, const float* S_var,
                        float2* slot_in, cudaStream_t st);
// A.slot_invdeg[q] = 1/|J_i| of the variable of slot q (0 for padding)
void launch_fill_slot_invdeg(const DevArena& A, cudaStream_t st);
// out_slot[q] = v[variable of q] (0 for padding slots)
void launch_gather_var(const DevArena& A, const float* v, float* out_slot, cudaStream_t st);

// smoothed subproblems (soft-min reading) and their marginals
void launch_smoothed(const DevArena& A, const float* lam, float a_s, float* E_a, float* marg, const LaunchGroup* groups,
                     int num_groups, const StreamSet& ss);

// eq. 2 and the output transforms of Alg. 3 (kernels_params.cu)
void launch_nonparam(const DevArena& A, float* lam, const float* theta, cudaStream_t st);
void launch_center(const DevArena& A, const float* x, float* out, cudaStream_t st);
void launch_param_transform(const DevArena& A, const float* ah, const float* wh, const float* th, float* alpha,
                            float* omega, float* theta, cudaStream_t st);
void launch_param_transform_bwd(const DevArena& A, const float* alpha, const float* omega, const float* ga,
                                const float* gw, const float* gt, float* gah, float* gwh, float* gth, cudaStream_t st);

// Long BDDs, one warp per BDD (kernels_long.cu); each is a single launch on
// the given stream, or nothing when the arena has no long BDDs.
void launch_long_sweep(int kind, const DevArena& A, const SweepArgs& a, cudaStream_t st);
void launch_long_smoothed(const DevArena& A, const float* lam, float a_s, float* E_a, float* marg, cudaStream_t st);
void launch_long_adjoint(bool forward, const DevArena& A, const AdjArgs& a, cudaStream_t st);

// dg_lower_bound with its intermediates in a static device array (noalloc.cu).
dg_status lower_bound_noalloc(const DevArena& arena, const LaunchGroup* groups, int num_groups, int threads,
                              const StreamSet& ss, const float* lam, const float* M, double* lb);

}  // namespace dg
