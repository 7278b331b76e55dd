// api.cu -- the C ABI of libdg (declared in include/dg.h): status codes,
// two-phase build (host plan, device bind), the solver calls, the CUDA graph
// of the iteration loop.
#include <algorithm>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <string>
#include <thread>

#include "kernels.h"

namespace dg {

static thread_local std::string g_err;

dg_status fail(dg_status st, const std::string& msg) {
  g_err = msg;
  return st;
}
void clear_error() { g_err.clear(); }

static dg_status cuda_fail(cudaError_t e, const char* where) {
  return fail(DG_ECUDA, std::string(where) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
}

}  // namespace dg

using namespace dg;

struct dg_arena_s {
  DevArena dev{};
  StreamSet streams;  // auxiliary streams and events for concurrent launch groups
  std::vector<LaunchGroup> groups;
  std::vector<AdjGroup> adj_groups;
  size_t cta_smem_cap = 0;
  dg_sizes sizes{};
  dg_stats stats{};
  size_t smem_sweep = 0, smem_adjoint = 0;
  int device = 0;
  int max_tile_rows = 0, max_tile_slots = 0, max_tile_hops = 0;
  // mode of the averaging terms the last S reduction for a sweep wrote into
  // the per-slot array (-1: none yet, the array holds zeros)
  int avg_mode = -1;
  // path costs handed from one dg_sweep to the next (DG_SWEEP_COSTS_*): every
  // API call advances `epoch`; the sweep that wrote the costs records its
  // epoch, direction and lambda, and only dg_sum_M without re-projection and
  // dg_bound_from_energies may run in between
  uint64_t epoch = 0, costs_epoch = 0;
  int costs_dir = -1;  // 1 forward, 0 backward
  const float* costs_lam = nullptr;
};

struct dg_graph_s {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the arena the graph iterates, and its mode: a replay rewrites the
  // arena's per-slot averaging terms and handed-on path costs
  dg_arena* arena = nullptr;
  int mode = 0;
};

namespace {

int threads_of(const dg_options* o) {
  int t = o && o->block_threads > 0 ? o->block_threads : 128;
  t = (t + 31) / 32 * 32;
  return t < 32 ? 32 : (t > 512 ? 512 : t);
}
float omega_of(const dg_options* o) { return o && o->omega > 0.f ? o->omega : 0.5f; }

StreamSet streams_for(const dg_arena* ar, cudaStream_t main) {
  StreamSet s = ar->streams;
  s.main = main;
  return s;
}

dg_status check_launch(const char* where) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, where);
  return DG_OK;
}

// Enqueues `iters` iterations (forward sweep, S, backward sweep, S per
// iteration) on st.  The first S reduction makes the snapshot of the
// incoming M.
dg_status enqueue_iterate(dg_arena* ar, cudaStream_t st, float* lam, float* M, const float* omega, const float* alpha,
                          int mode, int iters, double* lb_out, const dg_options* opts) {
  const DevArena& A = ar->dev;
  const int threads = threads_of(opts);
  const int renorm = opts ? opts->renorm_every : 0;
  SweepArgs a{};
  a.lam = lam;
  a.M = M;
  a.omega = omega;
  a.alpha = alpha;
  a.omega0 = omega_of(opts);
  a.mode = mode;
  ar->avg_mode = mode;
  launch_reduce_S(A, M, lam, alpha, mode, false, st, true);
  // every sweep hands its path costs to the next one (the S reductions
  // between them leave lambda alone), except into the first sweep, whose
  // lambda comes from the caller, and across a re-projection
  bool handed = false;
  for (int it = 0; it < iters; ++it) {
    const bool rn = renorm > 0 && ((it + 1) % renorm == 0);
    a.E = nullptr;
    a.cost_out = A.nodecost;
    a.cost_in = handed ? A.nodecost : nullptr;
    launch_sweep(kFwd, A, a, threads, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
    launch_reduce_S(A, M, lam, alpha, mode, false, st, true);
    if (lb_out && it == iters - 1) a.E = A.E;
    handed = it + 1 < iters && !rn;
    a.cost_out = handed ? A.nodecost : nullptr;
    a.cost_in = A.nodecost;
    launch_sweep(kBwd, A, a, threads, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
    launch_reduce_S(A, M, lam, alpha, mode, rn, st, it + 1 < iters);
  }
  if (lb_out) {
    if (iters == 0) {
      SweepArgs e{};
      e.lam = lam;
      e.E = A.E;
      launch_sweep(kEnergy, A, e, threads, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
    }
    launch_lower_bound(A, lb_out, st);
  }
  return check_launch("dg_iterate");
}

// The recording sweeps keep an argmin record per node on top of the sweep's
// shared memory; every launch group's tiles must still fit one CTA.
dg_status check_recording_fits(const dg_arena* ar, int mode, const char* where) {
  for (const LaunchGroup& g : ar->groups)
    if ((size_t)(mode ? g.region_bwd1 : g.region_bwd0) + (size_t)g.meta_bytes > ar->cta_smem_cap ||
        (size_t)(mode ? g.region_bytes : g.region_bytes0) + (size_t)g.meta_bytes > ar->cta_smem_cap)
      return fail(DG_EINVAL, std::string(where) + ": a tile's recording sweep does not fit one CTA's shared memory");
  return DG_OK;
}

// A state vector may be NULL only when the arena has no slots (no rows).
bool missing(const dg_arena* ar, const void* p) { return p == nullptr && ar->sizes.num_slots > 0; }

dg_status check_state(const dg_arena* ar) {
  if (!ar) return fail(DG_ESTATE, "null arena");
  ++const_cast<dg_arena*>(ar)->epoch;
  return DG_OK;
}

// For the calls that leave lambda and the arena's handed-on path costs alone.
void keep_costs(dg_arena* ar) {
  if (ar->costs_epoch + 1 == ar->epoch) ar->costs_epoch = ar->epoch;
}

// Arena-order vectors are read and written as float4: 16-byte alignment.
bool aligned16(const void* p) { return p == nullptr || ((uintptr_t)p & 15u) == 0; }
dg_status check_vectors(const char* where, const void* a, const void* b, const void* c = nullptr,
                        const void* d = nullptr) {
  if (!aligned16(a) || !aligned16(b) || !aligned16(c) || !aligned16(d))
    return fail(DG_EINVAL, std::string(where) + ": state vectors must be 16-byte aligned");
  return DG_OK;
}

}  // namespace

extern "C" {

const char* dg_last_error(void) { return g_err.c_str(); }

dg_status dg_plan(const dg_rows* rows, const dg_options* opts, dg_plan_t** out, dg_sizes* sizes) {
  clear_error();
  if (!out) return fail(DG_EINVAL, "dg_plan: null out");
  *out = nullptr;
  dg_plan_t* p = nullptr;
  try {
    p = new dg_plan_t();
    dg_status st = build_plan(rows, opts, p->p);
    if (st != DG_OK) {
      delete p;
      return st;
    }
  } catch (const std::bad_alloc&) {
    delete p;
    return fail(DG_ENOMEM, "dg_plan: host allocation failed");
  } catch (const std::exception& e) {
    delete p;
    return fail(DG_EINVAL, std::string("dg_plan: ") + e.what());
  }
  if (p->p.smem_sweep > 227 * 1024) {
    // a single BDD larger than one CTA's shared memory
    delete p;
    return fail(DG_EINVAL, "dg_plan: a BDD does not fit one tile's shared memory");
  }
  if (sizes) *sizes = p->p.sizes;
  *out = p;
  return DG_OK;
}

dg_status dg_build(const dg_rows* rows, const dg_options* opts, dg_plan_t** out, dg_sizes* sizes) {
  return dg_plan(rows, opts, out, sizes);
}

void dg_plan_free(dg_plan_t* plan) { delete plan; }

dg_status dg_get_sizes(const dg_plan_t* plan, dg_sizes* sizes) {
  if (!plan || !sizes) return fail(DG_EINVAL, "dg_get_sizes: null argument");
  *sizes = plan->p.sizes;
  return DG_OK;
}

dg_status dg_launch_group(const dg_plan_t* plan, int32_t g, int32_t* tile0, int32_t* tile1, int32_t* region_bytes,
                          int32_t* stream) {
  if (!plan) return fail(DG_EINVAL, "dg_launch_group: null plan");
  if (g < 0 || g >= (int32_t)plan->p.groups.size()) return fail(DG_EINVAL, "dg_launch_group: group out of range");
  const LaunchGroup& G = plan->p.groups[g];
  if (tile0) *tile0 = G.tile0;
  if (tile1) *tile1 = G.tile1;
  if (region_bytes) *region_bytes = G.region_bytes0;
  if (stream) *stream = G.stream;
  return DG_OK;
}

dg_status dg_plan_validate(const dg_plan_t* plan) {
  if (!plan) return fail(DG_EINVAL, "dg_plan_validate: null plan");
  return validate_plan(plan->p);
}

dg_status dg_slot_map(const dg_plan_t* plan, int64_t* out) {
  if (!plan || !out) return fail(DG_EINVAL, "dg_slot_map: null argument");
  std::memcpy(out, plan->p.slot_to_csr.data(), plan->p.slot_to_csr.size() * sizeof(int64_t));
  return DG_OK;
}

dg_status dg_bdd_export(const dg_plan_t* plan, int64_t j, int32_t* level_start, int32_t* lo, int32_t* hi,
                        int32_t* num_nodes) {
  if (!plan) return fail(DG_EINVAL, "dg_bdd_export: null plan");
  const Plan& P = plan->p;
  if (j < 0 || j >= P.sizes.m) return fail(DG_EINVAL, "dg_bdd_export: row out of range");
  if (P.long_of_row[j] >= 0) {
    // a long BDD: levels from its level table, child ranks as stored
    const int b = P.long_of_row[j];
    const LongBdd& L = P.longs[b];
    if (num_nodes) *num_nodes = L.nn;
    if (!level_start || !lo || !hi) return DG_OK;
    const int32_t* lvl = P.long_lvl.data() + L.lvl_base;
    for (int h = 0; h <= L.k; ++h) level_start[h] = lvl[h] - 2;
    const int64_t r0 = P.long_rank_ptr[b];
    for (int v = 0; v < L.nn; ++v) {
      lo[v] = P.long_lo[r0 + v];
      hi[v] = P.long_hi[r0 + v];
    }
    return DG_OK;
  }
  const int64_t nb = P.node_ptr[j], ne = P.node_ptr[j + 1];
  if (num_nodes) *num_nodes = (int32_t)(ne - nb);
  if (!level_start || !lo || !hi) return DG_OK;
  // level widths from the tile layout are not kept; recount from the child
  // ranks: level h+1 has as many nodes as the largest rank referenced + 1,
  // and every level's nodes are contiguous in node order.
  const int k = (int)(P.row_ptr[j + 1] - P.row_ptr[j]);
  int pos = 0;
  level_start[0] = 0;
  int width = 1;  // root level
  for (int h = 0; h < k; ++h) {
    level_start[h + 1] = pos + width;
    int next = 0;
    for (int r = 0; r < width; ++r) {
      lo[pos + r] = P.lo8[nb + pos + r];
      hi[pos + r] = P.hi8[nb + pos + r];
      next = std::max(next, std::max((int)lo[pos + r], (int)hi[pos + r]) + 1);
    }
    pos += width;
    width = next;
  }
  return DG_OK;
}

dg_status dg_bind(const dg_plan_t* plan, void* arena_dev, size_t arena_bytes, void* stream, dg_arena** out) {
  clear_error();
  if (!plan || !out) return fail(DG_EINVAL, "dg_bind: null argument");
  *out = nullptr;
  const Plan& P = plan->p;
  if (!arena_dev || arena_bytes < P.off.total) return fail(DG_EINVAL, "dg_bind: arena buffer too small");
  if (((uintptr_t)arena_dev & 255u) != 0) return fail(DG_EINVAL, "dg_bind: arena buffer must be 256-byte aligned");
  cudaStream_t st = (cudaStream_t)stream;
  // host image of everything up to the scratch area
  const size_t image = P.off.S;
  std::vector<unsigned char> h(image, 0);
  auto cp = [&](size_t off, const void* src, size_t bytes) {
    if (bytes) std::memcpy(h.data() + off, src, bytes);
  };
  cp(P.off.tiles, P.tiles.data(), P.tiles.size() * sizeof(Tile));
  cp(P.off.desc, P.desc.data(), P.desc.size() * 2);
  cp(P.off.lohi8, P.lohi8.data(), P.lohi8.size() * 2);
  cp(P.off.slot_var, P.slot_var.data(), P.slot_var.size() * 4);
  cp(P.off.slot_row, P.slot_row.data(), P.slot_row.size() * 4);
  cp(P.off.var_ptr, P.var_ptr.data(), P.var_ptr.size() * 4);
  cp(P.off.var_slots, P.var_slots.data(), P.var_slots.size() * 4);
  cp(P.off.var_ell, P.var_ell.data(), P.var_ell.size() * 4);
  cp(P.off.wide_vars, P.wide_vars.data(), P.wide_vars.size() * 4);
  cp(P.off.c, P.c.data(), P.c.size() * 8);
  cp(P.off.invdeg, P.invdeg.data(), P.invdeg.size() * 4);
  cp(P.off.inst_row_ptr, P.inst_row_ptr.data(), P.inst_row_ptr.size() * 8);
  cp(P.off.inst_var_ptr, P.inst_var_ptr.data(), P.inst_var_ptr.size() * 4);
  cp(P.off.lb_chunks, P.lb_chunks.data(), P.lb_chunks.size() * 4);
  cp(P.off.inst_chunk_ptr, P.inst_chunk_ptr.data(), P.inst_chunk_ptr.size() * 4);
  cp(P.off.inst_unc, P.inst_unc.data(), P.inst_unc.size() * 8);
  cp(P.off.longs, P.longs.data(), P.longs.size() * sizeof(LongBdd));
  cp(P.off.long_code, P.long_code.data(), P.long_code.size() * sizeof(int2));
  cp(P.off.long_lvl, P.long_lvl.data(), P.long_lvl.size() * 4);
  cp(P.off.long_in_ptr, P.long_in_ptr.data(), P.long_in_ptr.size() * 4);
  cp(P.off.long_in, P.long_in.data(), P.long_in.size() * 4);
  cp(P.off.long_order, P.long_order.data(), P.long_order.size() * 4);
  cudaError_t e = cudaMemcpyAsync(arena_dev, h.data(), image, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync((char*)arena_dev + P.off.S, 0, P.off.total - P.off.S, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e, "dg_bind upload");
  {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e, "dg_bind: device attribute");
    if ((size_t)optin < P.smem_sweep) return fail(DG_EINVAL, "dg_bind: tiles need more shared memory than a CTA has");
    e = set_sweep_smem_limit((size_t)optin);  // same limit for every arena of the process
    if (e == cudaSuccess) e = set_adjoint_smem_limit((size_t)optin);
    set_cta_smem_cap((size_t)optin);
    if (e != cudaSuccess) return cuda_fail(e, "dg_bind: shared-memory limit");
  }
  dg_arena* ar = new dg_arena();
  cudaGetDevice(&ar->device);
  {
    bool ok = cudaEventCreateWithFlags(&ar->streams.fork, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; ok && k < kStreams - 1; ++k) {
      ok = cudaStreamCreateWithFlags(&ar->streams.aux[k], cudaStreamNonBlocking) == cudaSuccess &&
           cudaEventCreateWithFlags(&ar->streams.join[k], cudaEventDisableTiming) == cudaSuccess;
    }
    if (!ok) {
      delete ar;
      return fail(DG_ECUDA, "dg_bind: stream or event creation failed");
    }
    ar->streams.ready = true;
  }
  {
    int optin = 0;
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, ar->device);
    ar->cta_smem_cap = (size_t)optin;
  }
  char* b = (char*)arena_dev;
  DevArena& A = ar->dev;
  A.tiles = (const Tile*)(b + P.off.tiles);
  A.desc = (const uint16_t*)(b + P.off.desc);
  A.lohi8 = (const uint16_t*)(b + P.off.lohi8);
  A.slot_var = (const int32_t*)(b + P.off.slot_var);
  A.slot_row = (const int32_t*)(b + P.off.slot_row);
  A.var_ptr = (const int32_t*)(b + P.off.var_ptr);
  A.var_slots = (const int32_t*)(b + P.off.var_slots);
  A.var_ell = (const int32_t*)(b + P.off.var_ell);
  A.wide_vars = (const int32_t*)(b + P.off.wide_vars);
  A.num_wide = (int32_t)P.wide_vars.size();
  A.c = (const double*)(b + P.off.c);
  A.invdeg = (const float*)(b + P.off.invdeg);
  A.inst_row_ptr = (const int64_t*)(b + P.off.inst_row_ptr);
  A.inst_var_ptr = (const int32_t*)(b + P.off.inst_var_ptr);
  A.lb_chunks = (const int4*)(b + P.off.lb_chunks);
  A.inst_chunk_ptr = (const int32_t*)(b + P.off.inst_chunk_ptr);
  A.inst_unc = (const double*)(b + P.off.inst_unc);
  A.longs = (const LongBdd*)(b + P.off.longs);
  A.long_code = (const int2*)(b + P.off.long_code);
  A.long_lvl = (const int32_t*)(b + P.off.long_lvl);
  A.long_in_ptr = (const int32_t*)(b + P.off.long_in_ptr);
  A.long_in = (const int32_t*)(b + P.off.long_in);
  A.long_order = (const int32_t*)(b + P.off.long_order);
  A.long_d = (float*)(b + P.off.long_d);
  A.long_t = (float*)(b + P.off.long_t);
  A.nodecost = (float*)(b + P.off.nodecost);
  A.slot_invdeg = (float*)(b + P.off.slot_invdeg);
  A.S = (float*)(b + P.off.S);
  A.Sbar = (float*)(b + P.off.Sbar);
  A.slot_avg = (float*)(b + P.off.slot_avg);
  A.E = (float*)(b + P.off.E);
  A.lb_part = (double*)(b + P.off.lb_part);
  A.n = P.sizes.n;
  A.num_inst = P.sizes.num_inst;
  A.m = P.sizes.m;
  A.num_slots = P.sizes.num_slots;
  A.num_tiles = P.sizes.num_tiles;
  A.num_lb_chunks = (int32_t)(P.lb_chunks.size() / 4);
  A.num_long = (int32_t)P.longs.size();
  A.long_slot_base = P.long_slot_base;
  A.long_cost_size = P.long_cost_size;
  A.long_stream = P.long_stream;
  A.num_long_narrow = P.num_long_narrow;
  {
    // lanes per narrow long BDD: the widest level's power of two (or the
    // option's, if larger); by default doubled (fewer BDDs per warp) while
    // that leaves fewer than four warps per SM
    int G = 1, maxw = 1, sms = 1;
    for (int32_t i = 0; i < P.num_long_narrow; ++i) maxw = std::max(maxw, P.longs[P.long_order[i]].maxw);
    while (G < maxw) G <<= 1;
    if (P.long_lanes > 0) {
      G = std::max(G, (int)P.long_lanes);
    } else {
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, ar->device);
      while (G < kWarp && (int64_t)(P.num_long_narrow + kWarp / G - 1) / (kWarp / G) < 4LL * sms) G <<= 1;
    }
    A.long_lanes = G;
  }
  // the per-slot weights of mode 0 the adjoint reads, laid out once
  launch_fill_slot_invdeg(A, st);
  e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) {
    dg_destroy(ar);
    return cuda_fail(e, "dg_bind: per-slot weights");
  }
  ar->sizes = P.sizes;
  ar->smem_sweep = P.smem_sweep;
  ar->groups = P.groups;
  ar->adj_groups = P.adj_groups;
  ar->smem_adjoint = P.smem_adjoint;
  ar->max_tile_rows = P.max_tile_rows;
  ar->max_tile_slots = P.max_tile_slots;
  ar->max_tile_hops = P.max_tile_hops;
  dg_stats& S = ar->stats;
  S.sizes = P.sizes;
  S.num_arcs = 2 * P.sizes.num_nodes;
  const double Nv = (double)P.sizes.num_nodes, Nl = (double)P.sizes.num_lambda, n = (double)P.sizes.n;
  S.bytes_per_iter = 32.0 * Nv + 48.0 * Nl + 16.0 * n;
  const double NVp = (double)P.sizes.num_nodes_padded, ns = (double)P.sizes.num_slots;
  // per sweep (the path costs handed on, as inside dg_iterate): children
  // 2 B and the costs read and written 8 B per node; descriptor, lambda read
  // and write, M write, averaging term 18 B per slot; alpha 4 B per lambda
  // (mode 1).  Per S reduction: M read and averaging term written 8 B per
  // lambda, ELL columns 16 B and S, S/|J_i| 8 B per variable.
  // long BDDs per sweep: children 8 B, in-arcs ~8 B and the path costs 8 B
  // per node
  S.actual_bytes_per_iter = 2.0 * (10.0 * NVp + 18.0 * ns + 4.0 * Nl) + 2.0 * (24.0 * n + 8.0 * Nl) +
                            2.0 * 24.0 * (double)P.sizes.num_long_nodes;
  for (int i = 0; i < 64; ++i) S.hop_histogram[i] = P.hop_histogram[i];
  *out = ar;
  return DG_OK;
}

void dg_destroy(dg_arena* arena) {
  if (!arena) return;
  if (arena->streams.ready) {
    cudaEventDestroy(arena->streams.fork);
    for (int k = 0; k < kStreams - 1; ++k) {
      cudaStreamDestroy(arena->streams.aux[k]);
      cudaEventDestroy(arena->streams.join[k]);
    }
  }
  delete arena;
}

dg_status dg_get_stats(const dg_arena* arena, dg_stats* stats) {
  if (!arena || !stats) return fail(DG_EINVAL, "dg_get_stats: null argument");
  *stats = arena->stats;
  return DG_OK;
}

dg_status dg_init_lambda(dg_arena* ar, void* stream, float* lam, float* M) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, M)) return fail(DG_EINVAL, "dg_init_lambda: null state");
  launch_init(ar->dev, lam, M, (cudaStream_t)stream);
  return check_launch("dg_init_lambda");
}

dg_status dg_iterate(dg_arena* ar, void* stream, float* lam, float* M, const float* omega, const float* alpha,
                     int32_t mode, int32_t iters, double* lb_out, const dg_options* opts) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, M)) return fail(DG_EINVAL, "dg_iterate: null state");
  if (mode != 0 && mode != 1) return fail(DG_EINVAL, "dg_iterate: mode must be 0 or 1");
  if (mode == 1 && (!omega || !alpha)) return fail(DG_EINVAL, "dg_iterate: mode 1 needs omega and alpha");
  if (iters < 0) return fail(DG_EINVAL, "dg_iterate: negative iteration count");
  if (opts && opts->block_threads != 0 && (opts->block_threads % 32 != 0 || opts->block_threads > 512))
    return fail(DG_EINVAL, "dg_iterate: block_threads must be a multiple of 32 in [32, 512]");
  if (dg_status s = check_vectors("dg_iterate", lam, M, omega, alpha)) return s;
  return enqueue_iterate(ar, (cudaStream_t)stream, lam, M, omega, alpha, mode, iters, lb_out, opts);
}

dg_status dg_autotune(dg_arena* ar, void* stream, float* lam, float* M, int32_t reps, float* tuned_ms) {
  if (dg_status s = check_state(ar)) return s;
  if (!lam || !M) return fail(DG_EINVAL, "dg_autotune: null work buffers");
  if (dg_status s = check_vectors("dg_autotune", lam, M)) return s;
  reps = std::max(1, std::min(reps, 100));
  cudaStream_t st = (cudaStream_t)stream;
  const DevArena& A = ar->dev;
  SweepArgs a{};
  a.lam = lam;
  a.M = M;
  a.omega0 = 0.5f;
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
    return fail(DG_ECUDA, "dg_autotune: event creation failed");
  auto timed = [&](auto&& body) -> float {
    body();  // warm-up
    cudaEventRecord(e0, st);
    for (int r = 0; r < reps; ++r) body();
    cudaEventRecord(e1, st);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms / reps;
  };
  ar->avg_mode = 0;
  launch_reduce_S(A, M, nullptr, nullptr, 0, false, st, true);
  // timed as dg_iterate runs them after its first sweep: each sweep takes
  // its opposite-direction costs from the one before
  a.cost_out = A.nodecost;
  launch_sweep(kFwd, A, a, 128, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
  a.cost_in = A.nodecost;
  launch_sweep(kBwd, A, a, 128, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
  auto pair = [&] {
    launch_sweep(kFwd, A, a, 128, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
    launch_sweep(kBwd, A, a, 128, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
  };
  // start from the occupancy choice, made explicit
  for (LaunchGroup& G : ar->groups) {
    G.wpc_fwd = (int8_t)best_warps_per_cta((size_t)G.region_bytes0, 4, ar->cta_smem_cap);
    G.wpc_bwd = (int8_t)best_warps_per_cta((size_t)G.region_bwd0, 4, ar->cta_smem_cap);
  }
  float best = 3.0e38f;
  int bestn = kStreams;
  for (int nstr : {1, 2, kStreams}) {
    ar->streams.n = nstr;
    const float ms = timed(pair);
    if (ms < best) {
      best = ms;
      bestn = nstr;
    }
  }
  ar->streams.n = bestn;
  best = timed(pair);
  for (LaunchGroup& G : ar->groups) {
    for (int dir = 0; dir < 2; ++dir) {
      int8_t& cur = dir == 0 ? G.wpc_fwd : G.wpc_bwd;
      const size_t region = (size_t)(dir == 0 ? G.region_bytes0 : G.region_bwd0);
      const int8_t keep = cur;
      for (int w = 1; w <= 4; w *= 2) {
        if (w == keep || region * w > ar->cta_smem_cap) continue;
        cur = (int8_t)w;
        const float ms = timed(pair);
        if (ms < best * 0.995f) {
          best = ms;
          break;
        }
        cur = keep;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (tuned_ms) *tuned_ms = best;
  return check_launch("dg_autotune");
}

dg_status dg_wait(void* stream, int32_t timeout_ms) {
  const auto t0 = std::chrono::steady_clock::now();
  for (;;) {
    const cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
    if (e == cudaSuccess) return DG_OK;
    if (e != cudaErrorNotReady) return cuda_fail(e, "dg_wait");
    const auto ms = std::chrono::duration_cast<std::chrono::milliseconds>(std::chrono::steady_clock::now() - t0).count();
    if (ms >= timeout_ms) return fail(DG_ETIMEOUT, "dg_wait: work still running after " + std::to_string(timeout_ms) + " ms");
    std::this_thread::sleep_for(std::chrono::microseconds(50));
  }
}

int32_t dg_iterate_launches(const dg_arena* ar, int32_t iters, int32_t want_lb, const dg_options* opts) {
  (void)opts;
  const int32_t g = ar ? (int32_t)ar->groups.size() + (ar->dev.num_long > 0 ? 1 : 0) : 1;
  int32_t l = 1 + iters * (2 * g + 2);
  if (want_lb) l += 2 + (iters == 0 ? g : 0);
  return l;
}

dg_status dg_sum_M(dg_arena* ar, void* stream, const float* M, float* lam, const float* alpha, int32_t mode,
                   int32_t renorm) {
  if (dg_status s = check_state(ar)) return s;
  if (!M || (renorm && !lam)) return fail(DG_EINVAL, "dg_sum_M: null pointer");
  if (renorm && mode == 1 && !alpha) return fail(DG_EINVAL, "dg_sum_M: mode 1 needs alpha");
  ar->avg_mode = mode;
  // a reduction without re-projection leaves lambda, so a hand-off survives it
  if (!renorm) keep_costs(ar);
  launch_reduce_S(ar->dev, M, lam, alpha, mode, renorm != 0, (cudaStream_t)stream, true);
  return check_launch("dg_sum_M");
}

dg_status dg_sweep(dg_arena* ar, void* stream, float* lam, float* M, const float* omega, const float* alpha,
                   int32_t mode, int32_t forward, int32_t flags, const dg_options* opts) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, M)) return fail(DG_EINVAL, "dg_sweep: null state");
  if (mode != 0 && mode != 1) return fail(DG_EINVAL, "dg_sweep: mode must be 0 or 1");
  if (mode == 1 && (!omega || !alpha)) return fail(DG_EINVAL, "dg_sweep: mode 1 needs omega and alpha");
  if (flags & ~(DG_SWEEP_ENERGY | DG_SWEEP_COSTS_OUT | DG_SWEEP_COSTS_IN))
    return fail(DG_EINVAL, "dg_sweep: unknown flag");
  const bool want_energy = (flags & DG_SWEEP_ENERGY) != 0;
  if (forward && want_energy) return fail(DG_EINVAL, "dg_sweep: energies come from backward sweeps");
  const int dir = forward ? 1 : 0;
  if ((flags & DG_SWEEP_COSTS_IN) &&
      (ar->costs_epoch + 1 != ar->epoch || ar->costs_dir != 1 - dir || ar->costs_lam != lam))
    return fail(DG_EINVAL, "dg_sweep: DG_SWEEP_COSTS_IN needs the arena's previous call to be a sweep in the other "
                           "direction on the same lambda with DG_SWEEP_COSTS_OUT (only dg_sum_M without renorm and "
                           "dg_bound_from_energies may run in between)");
  if (ar->avg_mode >= 0 && ar->avg_mode != mode)
    return fail(DG_EINVAL, "dg_sweep: mode differs from the one the arena's last S reduction (dg_sum_M) was run in");
  if (dg_status s = check_vectors("dg_sweep", lam, M, omega, alpha)) return s;
  SweepArgs a{};
  a.lam = lam;
  a.M = M;
  a.omega = omega;
  a.alpha = alpha;
  a.omega0 = omega_of(opts);
  a.mode = mode;
  a.E = want_energy ? ar->dev.E : nullptr;
  a.cost_out = (flags & DG_SWEEP_COSTS_OUT) ? ar->dev.nodecost : nullptr;
  a.cost_in = (flags & DG_SWEEP_COSTS_IN) ? ar->dev.nodecost : nullptr;
  launch_sweep(forward ? kFwd : kBwd, ar->dev, a, threads_of(opts), ar->groups.data(), (int)ar->groups.size(),
               streams_for(ar, (cudaStream_t)stream));
  if (flags & DG_SWEEP_COSTS_OUT) {
    ar->costs_epoch = ar->epoch;
    ar->costs_dir = dir;
    ar->costs_lam = lam;
  }
  return check_launch("dg_sweep");
}

dg_status dg_bound_from_energies(dg_arena* ar, void* stream, double* lb_out) {
  if (dg_status s = check_state(ar)) return s;
  if (!lb_out) return fail(DG_EINVAL, "dg_bound_from_energies: null output");
  keep_costs(ar);
  launch_lower_bound(ar->dev, lb_out, (cudaStream_t)stream);
  return check_launch("dg_bound_from_energies");
}

dg_status dg_min_marginals(dg_arena* ar, void* stream, const float* lam, float* m0, float* m1) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, m0) || missing(ar, m1)) return fail(DG_EINVAL, "dg_min_marginals: null pointer");
  if (dg_status s = check_vectors("dg_min_marginals", lam, m0, m1)) return s;
  SweepArgs a{};
  a.lam = const_cast<float*>(lam);
  a.M = m0;
  a.out2 = m1;
  launch_sweep(kMinMarg, ar->dev, a, threads_of(nullptr), ar->groups.data(), (int)ar->groups.size(),
               streams_for(ar, (cudaStream_t)stream));
  return check_launch("dg_min_marginals");
}

dg_status dg_lower_bound(dg_arena* ar, void* stream, const float* lam, const float* M, double* lb, float* E_per_row) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, M) || !lb) return fail(DG_EINVAL, "dg_lower_bound: null pointer");
  if (dg_status s = check_vectors("dg_lower_bound", lam, M)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  SweepArgs a{};
  a.lam = const_cast<float*>(lam);
  a.E = ar->dev.E;
  launch_sweep(kEnergy, ar->dev, a, threads_of(nullptr), ar->groups.data(), (int)ar->groups.size(),
               streams_for(ar, st));
  launch_reduce_S(ar->dev, M, nullptr, nullptr, 0, false, st, false);
  launch_lower_bound(ar->dev, lb, st);
  if (E_per_row) {
    cudaError_t e = cudaMemcpyAsync(E_per_row, ar->dev.E, (size_t)ar->dev.m * 4, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "dg_lower_bound copy");
  }
  return check_launch("dg_lower_bound");
}

dg_status dg_lower_bound_noalloc(dg_arena* ar, void* stream, const float* lam, const float* M, double* lb) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, M) || !lb) return fail(DG_EINVAL, "dg_lower_bound_noalloc: null pointer");
  if (dg_status s = check_vectors("dg_lower_bound_noalloc", lam, M)) return s;
  return lower_bound_noalloc(ar->dev, ar->groups.data(), (int)ar->groups.size(), threads_of(nullptr),
                             streams_for(ar, (cudaStream_t)stream), lam, M, lb);
}

dg_status dg_lb_seed(dg_arena* ar, void* stream, const float* lam, const float* M, float* g_lam, float* g_M) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, M) || missing(ar, g_lam) || missing(ar, g_M))
    return fail(DG_EINVAL, "dg_lb_seed: null pointer");
  if (dg_status s = check_vectors("dg_lb_seed", lam, g_lam)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  SweepArgs a{};
  a.lam = const_cast<float*>(lam);
  a.M = g_lam;
  launch_sweep(kSeed, ar->dev, a, threads_of(nullptr), ar->groups.data(), (int)ar->groups.size(),
               streams_for(ar, st));
  launch_reduce_S(ar->dev, M, nullptr, nullptr, 0, false, st, false);
  launch_seed_M(ar->dev, g_M, st);
  return check_launch("dg_lb_seed");
}

dg_status dg_smoothed_dual(dg_arena* ar, void* stream, const float* lam, float a, float* E_per_row, float* marginals) {
  if (dg_status s = check_state(ar)) return s;
  if (!lam || !marginals) return fail(DG_EINVAL, "dg_smoothed_dual: null pointer");
  if (!(a > 0.0f)) return fail(DG_EINVAL, "dg_smoothed_dual: smoothing factor must be positive");
  if (dg_status s = check_vectors("dg_smoothed_dual", lam, marginals)) return s;
  launch_smoothed(ar->dev, lam, a, E_per_row, marginals, ar->groups.data(), (int)ar->groups.size(),
                  streams_for(ar, (cudaStream_t)stream));
  return check_launch("dg_smoothed_dual");
}

dg_status dg_nonparam_update(dg_arena* ar, void* stream, float* lam, const float* theta) {
  if (dg_status s = check_state(ar)) return s;
  if (!lam || !theta) return fail(DG_EINVAL, "dg_nonparam_update: null pointer");
  launch_nonparam(ar->dev, lam, theta, (cudaStream_t)stream);
  return check_launch("dg_nonparam_update");
}

dg_status dg_nonparam_backward(dg_arena* ar, void* stream, const float* g_lam, float* g_theta) {
  if (dg_status s = check_state(ar)) return s;
  if (!g_lam || !g_theta) return fail(DG_EINVAL, "dg_nonparam_backward: null pointer");
  launch_center(ar->dev, g_lam, g_theta, (cudaStream_t)stream);
  return check_launch("dg_nonparam_backward");
}

dg_status dg_param_transform(dg_arena* ar, void* stream, const float* alpha_hat, const float* omega_hat,
                             const float* theta_hat, float* alpha, float* omega, float* theta) {
  if (dg_status s = check_state(ar)) return s;
  if ((!alpha_hat) != (!alpha) || (!omega_hat) != (!omega) || (!theta_hat) != (!theta))
    return fail(DG_EINVAL, "dg_param_transform: every input needs its output");
  launch_param_transform(ar->dev, alpha_hat, omega_hat, theta_hat, alpha, omega, theta, (cudaStream_t)stream);
  return check_launch("dg_param_transform");
}

dg_status dg_param_transform_backward(dg_arena* ar, void* stream, const float* alpha, const float* omega,
                                      const float* g_alpha, const float* g_omega, const float* g_theta,
                                      float* g_alpha_hat, float* g_omega_hat, float* g_theta_hat) {
  if (dg_status s = check_state(ar)) return s;
  if ((g_alpha_hat && (!alpha || !g_alpha)) || (g_omega_hat && (!omega || !g_omega)) || (g_theta_hat && !g_theta))
    return fail(DG_EINVAL, "dg_param_transform_backward: missing input for a requested gradient");
  launch_param_transform_bwd(ar->dev, alpha, omega, g_alpha, g_omega, g_theta, g_alpha_hat, g_omega_hat, g_theta_hat,
                             (cudaStream_t)stream);
  return check_launch("dg_param_transform_backward");
}

dg_status dg_graph_create(dg_arena* ar, void* stream, float* lam, float* M, const float* omega, const float* alpha,
                          int32_t mode, int32_t iters, double* lb_out, const dg_options* opts, dg_graph_t** out) {
  if (dg_status s = check_state(ar)) return s;
  if (!out) return fail(DG_EINVAL, "dg_graph_create: null out");
  *out = nullptr;
  if (!lam || !M) return fail(DG_EINVAL, "dg_graph_create: null state");
  if (mode == 1 && (!omega || !alpha)) return fail(DG_EINVAL, "dg_graph_create: mode 1 needs omega and alpha");
  if (dg_status s = check_vectors("dg_graph_create", lam, M, omega, alpha)) return s;
  cudaStream_t st = (cudaStream_t)stream;
  if (!st) return fail(DG_EINVAL, "dg_graph_create: capture needs a non-default stream");
  cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return cuda_fail(e, "dg_graph_create: begin capture");
  dg_status s = enqueue_iterate(ar, st, lam, M, omega, alpha, mode, iters, lb_out, opts);
  cudaGraph_t g = nullptr;
  e = cudaStreamEndCapture(st, &g);
  if (s != DG_OK) {
    if (g) cudaGraphDestroy(g);
    return s;
  }
  if (e != cudaSuccess) return cuda_fail(e, "dg_graph_create: end capture");
  cudaGraphExec_t x = nullptr;
  e = cudaGraphInstantiate(&x, g, 0);
  if (e != cudaSuccess) {
    cudaGraphDestroy(g);
    return cuda_fail(e, "dg_graph_create: instantiate");
  }
  dg_graph_t* G = new dg_graph_t();
  G->graph = g;
  G->exec = x;
  G->arena = ar;
  G->mode = mode;
  *out = G;
  return DG_OK;
}

dg_status dg_graph_replay(dg_graph_t* g, void* stream) {
  if (!g) return fail(DG_EINVAL, "dg_graph_replay: null graph");
  if (g->arena) {
    // no hand-off across the replay; the per-slot terms are now the graph's
    ++g->arena->epoch;
    g->arena->avg_mode = g->mode;
  }
  cudaError_t e = cudaGraphLaunch(g->exec, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "dg_graph_replay");
  return DG_OK;
}

void dg_graph_destroy(dg_graph_t* g) {
  if (!g) return;
  if (g->exec) cudaGraphExecDestroy(g->exec);
  if (g->graph) cudaGraphDestroy(g->graph);
  delete g;
}

namespace {

struct BwdLayout {
  size_t ck_lam, ck_M, rec_meta, rec_amin, rec_diff, seg_S, w_lam, w_M, sdot, sd_a, sd_b, slot_in, rec_lmeta,
      rec_lamin, long_a1, long_a2, total;
  size_t meta_stride;   // bytes of one sweep's node records
  size_t lmeta_stride;  // ... of the long BDDs' node records
  size_t lamin_stride;  // ... of the long BDDs' slot records
  int nseg, k;
};

BwdLayout backward_layout(const dg_arena* ar, int iters, int ckpt_every) {
  BwdLayout L{};
  const size_t NS = (size_t)ar->sizes.num_slots, n = (size_t)ar->sizes.n;
  L.k = ckpt_every > 0 ? std::min(ckpt_every, std::max(iters, 1)) : std::max(iters, 1);
  L.nseg = iters > 0 ? (iters + L.k - 1) / L.k : 0;
  size_t o = 0;
  auto put = [&](size_t bytes) {
    size_t at = o;
    o = (o + bytes + 255) / 256 * 256;
    return at;
  };
  L.ck_lam = put((size_t)L.nseg * NS * 4);
  L.ck_M = put((size_t)L.nseg * NS * 4);
  // argmin records of every sweep of one segment (recording sweeps)
  L.meta_stride = (size_t)ar->sizes.num_nodes_padded * 2;
  L.rec_meta = put((size_t)2 * L.k * L.meta_stride);
  L.rec_amin = put((size_t)2 * L.k * NS * 2);
  L.rec_diff = put((size_t)2 * L.k * NS * 4);
  L.seg_S = put((size_t)2 * L.k * n * 4);
  L.w_lam = put(NS * 4);
  L.w_M = put(NS * 4);
  L.sdot = put(NS * 4);
  L.sd_a = put(n * 4);
  L.sd_b = put(n * 4);
  L.slot_in = put(NS * 8);  // float2 per slot: the adjoint sweep's per-variable inputs
  // long BDDs: node and slot records of every sweep of one segment, and the
  // per-node gradients of the adjoint
  const size_t lcost = (size_t)ar->dev.long_cost_size, lslots = NS - (size_t)ar->dev.long_slot_base;
  L.lmeta_stride = lcost * 4;
  L.lamin_stride = lslots * 8;
  L.rec_lmeta = put((size_t)2 * L.k * L.lmeta_stride);
  L.rec_lamin = put((size_t)2 * L.k * L.lamin_stride);
  L.long_a1 = put(lcost * 4);
  L.long_a2 = put(lcost * 4);
  L.total = o;
  return L;
}

// Runs `k` iterations from (lam, M) as recording sweeps: before sweep sw the
// S snapshot is taken and kept in seg_S[sw], the sweep's argmin records go to
// record slot sw of the workspace.  The same kernels in the same order as
// enqueue_iterate (the recording sweeps compute the same values), so lam, M
// and the bound are bit-identical to k plain iterations.  With lb_out the last
// backward sweep writes the energies and the bound follows.
dg_status enqueue_recorded_segment(dg_arena* ar, cudaStream_t st, float* lam, float* M, const float* omega,
                                   const float* alpha, int mode, int k, const BwdLayout& L, char* w, double* lb_out,
                                   const dg_options* opts) {
  const DevArena& A = ar->dev;
  const size_t NS = (size_t)ar->sizes.num_slots, n = (size_t)ar->sizes.n;
  SweepArgs fa{};
  fa.lam = lam;
  fa.M = M;
  fa.omega = omega;
  fa.alpha = alpha;
  fa.omega0 = omega_of(opts);
  fa.mode = mode;
  cudaError_t e = cudaSuccess;
  ar->avg_mode = mode;
  for (int sw = 0; sw < 2 * k; ++sw) {
    launch_reduce_S(A, M, nullptr, nullptr, mode, false, st, true);
    if (e == cudaSuccess && n)
      e = cudaMemcpyAsync(w + L.seg_S + (size_t)sw * n * 4, A.S, n * 4, cudaMemcpyDeviceToDevice, st);
    SweepArgs ra = fa;
    ra.rec_meta = (uint16_t*)(w + L.rec_meta + (size_t)sw * L.meta_stride);
    ra.rec_amin = (uint16_t*)(w + L.rec_amin) + (size_t)sw * NS;
    ra.rec_diff = (float*)(w + L.rec_diff) + (size_t)sw * NS;
    ra.rec_lmeta = (int32_t*)(w + L.rec_lmeta + (size_t)sw * L.lmeta_stride);
    ra.rec_lamin = (int2*)(w + L.rec_lamin + (size_t)sw * L.lamin_stride);
    // each recording sweep hands its path costs (and records) to the next
    ra.cost_out = A.nodecost;
    if (sw > 0) {
      ra.cost_in = A.nodecost;
      ra.meta_in = (const uint16_t*)(w + L.rec_meta + (size_t)(sw - 1) * L.meta_stride);
      ra.lmeta_in = (const int32_t*)(w + L.rec_lmeta + (size_t)(sw - 1) * L.lmeta_stride);
    }
    if (lb_out && sw == 2 * k - 1) ra.E = A.E;
    launch_sweep(sw % 2 == 0 ? kFwdRec : kBwdRec, A, ra, threads_of(opts), ar->groups.data(), (int)ar->groups.size(),
                 streams_for(ar, st));
  }
  launch_reduce_S(A, M, nullptr, nullptr, mode, false, st, false);
  if (lb_out) launch_lower_bound(A, lb_out, st);
  if (e != cudaSuccess) return cuda_fail(e, "recorded segment copies");
  return check_launch("recorded segment");
}

}  // namespace

size_t dg_backward_workspace_bytes(const dg_arena* ar, int32_t iters, int32_t ckpt_every) {
  if (!ar || iters < 0) return 0;
  return backward_layout(ar, iters, ckpt_every).total;
}

namespace {

// dg_backward and dg_backward_checkpointed.  With lam0 == nullptr the
// checkpoints are already in the workspace (dg_iterate_checkpointed) and the
// forward pass is skipped.
dg_status backward_impl(dg_arena* ar, void* stream, const float* lam0, const float* M0, const float* omega,
                        const float* alpha, int32_t mode, int32_t iters, int32_t ckpt_every, const float* g_lam_T,
                        const float* g_M_T, float* g_lam0, float* g_M0, float* g_omega, float* g_alpha,
                        void* workspace, size_t ws_bytes, const dg_options* opts) {
  const bool have_ckpt = lam0 == nullptr;
  if (dg_status s = check_state(ar)) return s;
  if ((!have_ckpt && !M0) || !g_lam_T || !g_M_T || !g_lam0 || !g_M0)
    return fail(DG_EINVAL, "dg_backward: null pointer");
  if (mode != 0 && mode != 1) return fail(DG_EINVAL, "dg_backward: mode must be 0 or 1");
  if (mode == 1 && (!omega || !alpha)) return fail(DG_EINVAL, "dg_backward: mode 1 needs omega and alpha");
  if (iters < 0) return fail(DG_EINVAL, "dg_backward: negative iteration count");
  if (opts && opts->renorm_every > 0)
    return fail(DG_EINVAL, "dg_backward: the adjoint does not differentiate the FP64 re-projection "
                           "(renorm_every must be 0)");
  if (dg_status s = check_vectors("dg_backward", lam0, M0, omega, alpha)) return s;
  if (dg_status s = check_vectors("dg_backward", g_lam_T, g_M_T, g_lam0, g_M0)) return s;
  if (dg_status s = check_vectors("dg_backward", g_omega, g_alpha)) return s;
  for (const AdjGroup& g : ar->adj_groups)
    if ((size_t)g.region > ar->cta_smem_cap)
      return fail(DG_EINVAL, "dg_backward: a tile's adjoint state does not fit one CTA's shared memory");
  if (dg_status s = check_recording_fits(ar, mode, "dg_backward")) return s;
  const BwdLayout L = backward_layout(ar, iters, ckpt_every);
  if (iters > 0 && (!workspace || ws_bytes < L.total))
    return fail(DG_EINVAL, "dg_backward: workspace smaller than dg_backward_workspace_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  const DevArena& A = ar->dev;
  if (iters > 0) ar->avg_mode = mode;
  const size_t NS = (size_t)ar->sizes.num_slots, n = (size_t)ar->sizes.n;
  const size_t bNS = NS * 4, bn = n * 4;
  cudaError_t e = cudaSuccess;
  auto cpy = [&](void* d, const void* src, size_t bytes) {
    if (e == cudaSuccess && bytes) e = cudaMemcpyAsync(d, src, bytes, cudaMemcpyDeviceToDevice, st);
  };
  if (g_omega) e = cudaMemsetAsync(g_omega, 0, bNS, st);
  if (e == cudaSuccess && g_alpha) e = cudaMemsetAsync(g_alpha, 0, bNS, st);
  if (iters == 0) {
    cpy(g_lam0, g_lam_T, bNS);
    cpy(g_M0, g_M_T, bNS);
    if (e != cudaSuccess) return cuda_fail(e, "dg_backward");
    return DG_OK;
  }
  char* w = (char*)workspace;
  float* ck_lam = (float*)(w + L.ck_lam);
  float* ck_M = (float*)(w + L.ck_M);
  char* rec_meta = w + L.rec_meta;
  uint16_t* rec_amin = (uint16_t*)(w + L.rec_amin);
  float* rec_diff = (float*)(w + L.rec_diff);
  float* seg_S = (float*)(w + L.seg_S);
  float* w_lam = (float*)(w + L.w_lam);
  float* w_M = (float*)(w + L.w_M);
  float* sdot = (float*)(w + L.sdot);
  float* sd_next = (float*)(w + L.sd_a);
  float* sd_cur = (float*)(w + L.sd_b);
  float2* slot_in = (float2*)(w + L.slot_in);
  const int threads = threads_of(opts);
  SweepArgs fa{};
  fa.lam = w_lam;
  fa.M = w_M;
  fa.omega = omega;
  fa.alpha = alpha;
  fa.omega0 = omega_of(opts);
  fa.mode = mode;
  // 1. forward pass keeping a checkpoint of (lambda, M) every k iterations
  //    (already done by dg_iterate_checkpointed when have_ckpt)
  if (!have_ckpt) {
    cpy(w_lam, lam0, bNS);
    cpy(w_M, M0, bNS);
  }
  bool handed = false;  // the sweeps hand their path costs on as in dg_iterate
  for (int c = 0; c < (have_ckpt ? 0 : L.nseg); ++c) {
    cpy(ck_lam + (size_t)c * NS, w_lam, bNS);
    cpy(ck_M + (size_t)c * NS, w_M, bNS);
    if (c + 1 == L.nseg) {
      // the last segment runs as recording sweeps right away
      if (e != cudaSuccess) return cuda_fail(e, "dg_backward copies");
      if (dg_status s = enqueue_recorded_segment(ar, st, w_lam, w_M, omega, alpha, mode, iters - c * L.k, L, w,
                                                 nullptr, opts))
        return s;
      break;
    }
    for (int it = 0; it < L.k; ++it) {
      SweepArgs f = fa, b = fa;
      f.cost_out = b.cost_out = A.nodecost;
      f.cost_in = handed ? A.nodecost : nullptr;
      b.cost_in = A.nodecost;
      handed = true;
      launch_reduce_S(A, w_M, nullptr, nullptr, mode, false, st, true);
      launch_sweep(kFwd, A, f, threads, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
      launch_reduce_S(A, w_M, nullptr, nullptr, mode, false, st, true);
      launch_sweep(kBwd, A, b, threads, ar->groups.data(), (int)ar->groups.size(), streams_for(ar, st));
    }
  }
  // 2. segments newest first: recompute every sweep of the segment as a
  //    recording sweep (its argmins and S at its start kept; the last
  //    segment's are already there from the forward pass), then run the
  //    adjoint sweeps backwards
  cpy(g_lam0, g_lam_T, bNS);
  AdjArgs aa{};
  aa.omega = omega;
  aa.alpha = alpha;
  aa.omega0 = omega_of(opts);
  aa.mode = mode;
  aa.g_lam = g_lam0;
  aa.g_omega = g_omega;
  aa.g_alpha = g_alpha;
  aa.sdot = sdot;
  aa.slot_in = slot_in;
  // padding slots belong to no variable: their inputs stay 0
  if (e == cudaSuccess && iters > 0) e = cudaMemsetAsync(slot_in, 0, NS * 8, st);
  aa.long_a1 = (float*)(w + L.long_a1);
  aa.long_a2 = (float*)(w + L.long_a2);
  const int last_sweep = 2 * iters - 1;
  for (int c = L.nseg - 1; c >= 0; --c) {
    const int it0 = c * L.k, it1 = std::min(iters, it0 + L.k);
    const int nsw = 2 * (it1 - it0);
    const bool recorded = c + 1 == L.nseg;
    if (!recorded) {
      cpy(w_lam, ck_lam + (size_t)c * NS, bNS);
      cpy(w_M, ck_M + (size_t)c * NS, bNS);
    }
    for (int sw = 0; sw < (recorded ? 0 : nsw); ++sw) {
      launch_reduce_S(A, w_M, nullptr, nullptr, mode, false, st, true);
      cpy(seg_S + (size_t)sw * n, A.S, bn);
      SweepArgs ra = fa;
      ra.rec_meta = (uint16_t*)(rec_meta + (size_t)sw * L.meta_stride);
      ra.rec_amin = rec_amin + (size_t)sw * NS;
      ra.rec_diff = rec_diff + (size_t)sw * NS;
      ra.rec_lmeta = (int32_t*)(w + L.rec_lmeta + (size_t)sw * L.lmeta_stride);
      ra.rec_lamin = (int2*)(w + L.rec_lamin + (size_t)sw * L.lamin_stride);
      ra.cost_out = A.nodecost;  // handed on from recording sweep to recording sweep
      if (sw > 0) {
        ra.cost_in = A.nodecost;
        ra.meta_in = (const uint16_t*)(rec_meta + (size_t)(sw - 1) * L.meta_stride);
        ra.lmeta_in = (const int32_t*)(w + L.rec_lmeta + (size_t)(sw - 1) * L.lmeta_stride);
      }
      launch_sweep(sw % 2 == 0 ? kFwdRec : kBwdRec, A, ra, threads, ar->groups.data(), (int)ar->groups.size(),
                   streams_for(ar, st));
    }
    // the per-slot inputs of the segment's last sweep: the S-dot handed over
    // from the adjoint of the segment after it (none after the last sweep)
    launch_slot_inputs(A, nullptr, 2 * it0 + nsw - 1 == last_sweep ? nullptr : sd_next, nullptr,
                       seg_S + (size_t)(nsw - 1) * n, slot_in, st);
    for (int sw = nsw - 1; sw >= 0; --sw) {
      const int gsw = 2 * it0 + sw;
      aa.rec_meta = (const uint16_t*)(rec_meta + (size_t)sw * L.meta_stride);
      aa.rec_amin = rec_amin + (size_t)sw * NS;
      aa.rec_diff = rec_diff + (size_t)sw * NS;
      aa.rec_lmeta = (const int32_t*)(w + L.rec_lmeta + (size_t)sw * L.lmeta_stride);
      aa.rec_lamin = (const int2*)(w + L.rec_lamin + (size_t)sw * L.lamin_stride);
      aa.S_in = seg_S + (size_t)sw * n;
      aa.seed_M = gsw == last_sweep ? g_M_T : nullptr;
      aa.sdot_next = gsw == last_sweep ? nullptr : sd_next;
      launch_adjoint_sweep(sw % 2 == 0, A, aa, ar->adj_groups.data(), (int)ar->adj_groups.size(), ar->cta_smem_cap,
                           streams_for(ar, st));
      // S-dot of this sweep, and the next adjoint sweep's per-slot inputs
      launch_slot_inputs(A, sdot, nullptr, sd_cur, sw > 0 ? seg_S + (size_t)(sw - 1) * n : nullptr,
                         sw > 0 ? slot_in : nullptr, st);
      std::swap(sd_next, sd_cur);
    }
  }
  // 3. M0 only enters through the first snapshot S_i = sum_j M0_ij
  launch_gather_var(A, sd_next, g_M0, st);
  if (e != cudaSuccess) return cuda_fail(e, "dg_backward copies");
  return check_launch("dg_backward");
}

}  // namespace

dg_status dg_backward(dg_arena* ar, void* stream, const float* lam0, const float* M0, const float* omega,
                      const float* alpha, int32_t mode, int32_t iters, int32_t ckpt_every, const float* g_lam_T,
                      const float* g_M_T, float* g_lam0, float* g_M0, float* g_omega, float* g_alpha, void* workspace,
                      size_t ws_bytes, const dg_options* opts) {
  if (dg_status s = check_state(ar)) return s;
  if (!lam0 || !M0) return fail(DG_EINVAL, "dg_backward: null pointer");
  return backward_impl(ar, stream, lam0, M0, omega, alpha, mode, iters, ckpt_every, g_lam_T, g_M_T, g_lam0, g_M0,
                       g_omega, g_alpha, workspace, ws_bytes, opts);
}

dg_status dg_backward_checkpointed(dg_arena* ar, void* stream, const float* omega, const float* alpha, int32_t mode,
                                   int32_t iters, int32_t ckpt_every, const float* g_lam_T, const float* g_M_T,
                                   float* g_lam0, float* g_M0, float* g_omega, float* g_alpha, void* workspace,
                                   size_t ws_bytes, const dg_options* opts) {
  return backward_impl(ar, stream, nullptr, nullptr, omega, alpha, mode, iters, ckpt_every, g_lam_T, g_M_T, g_lam0,
                       g_M0, g_omega, g_alpha, workspace, ws_bytes, opts);
}

dg_status dg_iterate_checkpointed(dg_arena* ar, void* stream, float* lam, float* M, const float* omega,
                                  const float* alpha, int32_t mode, int32_t iters, int32_t ckpt_every,
                                  void* workspace, size_t ws_bytes, double* lb_out, const dg_options* opts) {
  if (dg_status s = check_state(ar)) return s;
  if (missing(ar, lam) || missing(ar, M)) return fail(DG_EINVAL, "dg_iterate_checkpointed: null state");
  if (mode != 0 && mode != 1) return fail(DG_EINVAL, "dg_iterate_checkpointed: mode must be 0 or 1");
  if (mode == 1 && (!omega || !alpha)) return fail(DG_EINVAL, "dg_iterate_checkpointed: mode 1 needs omega and alpha");
  if (iters < 0) return fail(DG_EINVAL, "dg_iterate_checkpointed: negative iteration count");
  if (opts && opts->renorm_every > 0)
    return fail(DG_EINVAL, "dg_iterate_checkpointed: the adjoint does not differentiate the FP64 re-projection "
                           "(renorm_every must be 0)");
  if (opts && opts->block_threads != 0 && (opts->block_threads % 32 != 0 || opts->block_threads > 512))
    return fail(DG_EINVAL, "dg_iterate_checkpointed: block_threads must be a multiple of 32 in [32, 512]");
  if (dg_status s = check_vectors("dg_iterate_checkpointed", lam, M, omega, alpha)) return s;
  if (dg_status s = check_recording_fits(ar, mode, "dg_iterate_checkpointed")) return s;
  const BwdLayout L = backward_layout(ar, iters, ckpt_every);
  if (iters > 0 && (!workspace || ws_bytes < L.total))
    return fail(DG_EINVAL, "dg_iterate_checkpointed: workspace smaller than dg_backward_workspace_bytes()");
  cudaStream_t st = (cudaStream_t)stream;
  const size_t bNS = (size_t)ar->sizes.num_slots * 4;
  char* w = (char*)workspace;
  for (int c = 0; c < L.nseg; ++c) {
    cudaError_t e = cudaMemcpyAsync(w + L.ck_lam + (size_t)c * bNS, lam, bNS, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(w + L.ck_M + (size_t)c * bNS, M, bNS, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e, "dg_iterate_checkpointed copies");
    const int k = std::min(L.k, iters - c * L.k);
    if (c + 1 == L.nseg) {
      // the last segment's argmin records stay in the workspace, so that
      // dg_backward_checkpointed does not recompute that segment
      if (dg_status s = enqueue_recorded_segment(ar, st, lam, M, omega, alpha, mode, k, L, w, lb_out, opts)) return s;
    } else if (dg_status s = enqueue_iterate(ar, st, lam, M, omega, alpha, mode, k, nullptr, opts)) {
      return s;
    }
  }
  if (iters == 0) return enqueue_iterate(ar, st, lam, M, omega, alpha, mode, 0, lb_out, opts);
  return DG_OK;
}

}  // extern "C"
