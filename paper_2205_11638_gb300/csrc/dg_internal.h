// dg_internal.h -- layout of the device arena and declarations shared by the
// host builder, the kernels and the C ABI of libdg.  Not installed.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "dg.h"

namespace dg {

// Node numbers inside a BDD: 0 is the top terminal, 1 the bottom terminal,
// the BDD's own nodes are 2, 3, ... level by level (at most kMaxNodesPerBdd).
// A node's children are stored as node numbers (8 bits each).
constexpr uint32_t kTopCode = 0u;
constexpr uint32_t kBotCode = 1u;
constexpr int kMaxNodesPerBdd = 254;
constexpr int kWarp = 32;
constexpr int kMaxWidth = 128;  // nodes of one BDD level (child ranks are 8-bit)
constexpr int kStreams = 4;    // streams one sweep's launch groups run on
// The first kEll slots of every variable are also stored column by column
// (var_ell[r * n + i], ELLPACK layout) so that the S reduction reads them
// without first reading var_ptr; -1 marks "no slot", and a variable with more
// than kEll slots stores its last ELL entry as -2 - slot, the rest coming
// from var_slots[var_ptr[i] + kEll ..].
constexpr int kEll = 4;
// Variables with more slots than this ("wide") are reduced by a warp each in
// the per-variable kernels, listed in wide_vars; the others by a thread each.
constexpr int kWide = 32;

// One tile = up to 32 BDDs swept by one warp, BDD b by lane b.  Per-tile
// arrays are interleaved by lane: slot (h, b) is slot_base + 32 h + b (its
// descriptor holds the first node number of level h and the level's width, 0
// when BDD b has no level h) and node n >= 2 of lane b has its child codes at
// node_base + 32 (n - 2) + b.
struct Tile {
  int32_t node_base;  // first child-code entry (multiple of 32)
  int32_t slot_base;  // first slot (multiple of 32)
  int32_t nmax;       // node numbers per lane, terminals included
  int32_t nhops;      // longest BDD of the tile
  int32_t nbdd;       // BDDs (lanes in use)
  int32_t maxw;       // widest level
  int32_t ring;       // ring size (power of two >= 2 * maxw) of the sweep-direction costs
  int32_t pad1;
};
static_assert(sizeof(Tile) == 32, "Tile is 32 bytes");

inline int ring_size(int maxw) {
  int r = 2;
  while (r < 2 * maxw) r <<= 1;
  return r;
}

// A BDD beyond the limits of the lane-per-BDD tiles (more than
// kMaxNodesPerBdd nodes, or a level wider than kMaxWidth): swept by one warp
// with a level's nodes spread over the lanes.  Its levels are consecutive
// arena slots; its nodes are numbered like a tile lane's (0 top, 1 bottom,
// own nodes from 2 level by level) with 32-bit child numbers, and every node
// lists its in-arcs (parent number << 1 | beta, ascending) for the pulls of
// SP(r, .).
struct LongBdd {
  int32_t slot_base;  // arena slot of level 0
  int32_t k;          // levels
  int32_t code_base;  // long_code / long_in_ptr index of node number 2
  int32_t nn;         // own nodes
  int32_t lvl_base;   // long_lvl index: k + 1 entries, first node number of each level, then nn + 2
  int32_t cost_base;  // per-node scratch index of node number 0 (nn + 2 entries)
  int32_t row;        // original row
  int32_t maxw;       // widest level
};
static_assert(sizeof(LongBdd) == 32, "LongBdd is 32 bytes");

// Device view of an arena (all pointers inside the caller's buffer).
struct DevArena {
  const Tile* tiles;
  const uint16_t* desc;     // per slot: first node number | width << 8
  const uint16_t* lohi8;    // per node and lane: lo code | hi code << 8
  const int32_t* slot_var;  // variable of a slot, -1 for padding
  const int32_t* slot_row;  // original row of a slot, -1 for padding
  const int32_t* var_ptr;   // CSR over variables: slots of variable i
  const int32_t* var_slots; // arena slots, grouped by variable, rows ascending
  const int32_t* var_ell;   // [kEll * n] the first kEll slots of each variable (see kEll)
  const int32_t* wide_vars; // the variables with more than kWide slots, ascending
  int32_t num_wide;
  const double* c;          // objective, float64[n]
  const float* invdeg;      // 1/|J_i| (0 for uncovered variables)
  const int64_t* inst_row_ptr;
  const int32_t* inst_var_ptr;
  const int4* lb_chunks;    // {instance, kind (0 rows, 1 vars), begin, end}
  const int32_t* inst_chunk_ptr;
  const double* inst_unc;   // per instance: sum of min(0, c_i) over variables no row covers
  // BDDs swept one warp per BDD (see LongBdd)
  const LongBdd* longs;
  const int2* long_code;     // per own node: lo, hi node numbers
  const int32_t* long_lvl;
  const int32_t* long_in_ptr;  // CSR of in-arcs over own nodes (global index)
  const int32_t* long_in;      // parent node number << 1 | beta
  // the long BDDs whose levels have at most 32 nodes ("narrow"; longest
  // first), then the others (ascending): indices into `longs`
  const int32_t* long_order;
  float* long_d;               // scratch per node of long BDDs: SP(r, .)
  float* long_t;               // ... SP(., T)
  // scratch per node and lane of the tiles (layout of lohi8): SP(r, .) as a
  // forward sweep leaves it for the backward sweep after it (see SweepArgs)
  float* nodecost;
  // per slot: 1/|J_i| of its variable (0 for padding), filled when the arena
  // is bound; the adjoint's alpha in mode 0
  float* slot_invdeg;
  float* S;                 // scratch: per-variable sum of M (snapshot)
  float* Sbar;              // scratch: S_i / |J_i| (the mode-0 averaging term)
  float* slot_avg;          // scratch per slot: the averaging term of its variable (Sbar_i in mode 0,
                            // S_i in mode 1) as the last S reduction before a sweep left it; 0 for padding
  float* E;                 // scratch: E^j per original row
  double* lb_part;          // scratch: one partial sum per lb chunk
  int32_t n;
  int32_t num_inst;
  int64_t m;
  int64_t num_slots;
  int32_t num_tiles;
  int32_t num_lb_chunks;
  int32_t num_long;
  int32_t long_slot_base;   // first slot of the long BDDs (after every tile's slots)
  int32_t long_cost_size;   // entries of long_d / long_t
  int32_t long_stream;      // stream of the fork/join set the long BDDs run on
  int32_t num_long_narrow;  // narrow long BDDs (the head of long_order)
  int32_t long_lanes;       // lanes per narrow BDD in the plain sweeps (a power of two, set at bind)
};

// Tiles that one kernel launch sweeps: consecutive tiles whose shared-memory
// footprints are within a fixed ratio, so that a launch's per-warp slice of
// shared memory (the largest footprint of its tiles) wastes little.
struct LaunchGroup {
  int32_t tile0, tile1;
  int32_t region_bytes;   // per-slot omega staged (mode 1)
  int32_t region_bytes0;  // without omega (mode 0)
  int32_t region_bwd1;    // backward sweeps (two full cost arrays), mode 1
  int32_t region_bwd0;    // ... mode 0
  int64_t work;           // estimated cost: sum over tiles of 32 * nmax * nhops
  int32_t stream;         // stream of the fork/join set the group runs on
  int8_t wpc_fwd;         // tuned warps per CTA (0: choose by occupancy)
  int8_t wpc_bwd;
  int8_t pad[2];
  int32_t meta_bytes;     // argmin records of the recording sweeps: 64 (nmax - 2), largest tile
};

// Tiles of one adjoint launch (the sweep's launch groups with the adjoint's
// shared-memory footprint).
struct AdjGroup {
  int32_t tile0, tile1;
  int32_t region;  // per-warp slice (the same in both modes)
  int32_t stream;
};

struct Plan {
  // sizes
  dg_sizes sizes{};
  int64_t hop_histogram[64]{};
  // host images of the device arrays
  std::vector<Tile> tiles;
  std::vector<LaunchGroup> groups;
  std::vector<AdjGroup> adj_groups;
  std::vector<uint16_t> desc;
  std::vector<uint16_t> lohi8;
  std::vector<int32_t> slot_var, slot_row;
  std::vector<int32_t> var_ptr, var_slots, var_ell, wide_vars;
  std::vector<double> c;
  std::vector<float> invdeg;
  std::vector<int64_t> inst_row_ptr;
  std::vector<int32_t> inst_var_ptr;
  std::vector<int32_t> lb_chunks;  // 4 ints per chunk
  std::vector<int32_t> inst_chunk_ptr;
  std::vector<double> inst_unc;    // per instance: sum of min(0, c_i) over its uncovered variables
  std::vector<int64_t> slot_to_csr;
  // canonical BDDs (for dg_bdd_export): per CSR slot the level width, per
  // node the child ranks (-2 bottom, -1 top)
  std::vector<int64_t> row_ptr;
  std::vector<int64_t> node_ptr;  // per row, first node
  std::vector<int8_t> lo8, hi8;
  // long BDDs: per row the index into `longs` (-1 for tile rows), their
  // device arrays, and for export their levels' widths and child ranks
  std::vector<int32_t> long_of_row;
  std::vector<LongBdd> longs;
  std::vector<int2> long_code;
  std::vector<int32_t> long_lvl, long_in_ptr, long_in;
  std::vector<int32_t> long_order;  // see DevArena::long_order
  int32_t num_long_narrow = 0;
  int32_t long_lanes = 0;           // dg_options::long_lanes (0: chosen at bind)
  std::vector<int64_t> long_rank_ptr;  // per long BDD, first entry of long_lo / long_hi
  std::vector<int32_t> long_lo, long_hi;  // child ranks as in lo8 / hi8 (-2 bottom, -1 top)
  int32_t long_slot_base = 0, long_cost_size = 0, long_stream = 0;
  // byte offsets of every array inside the arena
  struct Off {
    size_t tiles, desc, lohi8, slot_var, slot_row, var_ptr, var_slots, var_ell, wide_vars, c, invdeg, inst_row_ptr,
        inst_var_ptr,
        lb_chunks, inst_chunk_ptr, inst_unc, longs, long_code, long_lvl, long_in_ptr, long_in, long_order, S, Sbar, slot_avg, E, lb_part,
        long_d, long_t, nodecost, slot_invdeg, total;
  } off{};
  size_t smem_sweep = 0;   // dynamic smem of the sweep kernels
  size_t smem_adjoint = 0; // dynamic smem of the adjoint kernels
  int32_t max_tile_rows = 0, max_tile_slots = 0, max_tile_hops = 0;
};

// Shared-memory footprint of one tile (one warp's slice) in the sweep
// kernels: the costs of the first pass (32 x nmax floats), a ring of two
// levels for the costs of the sweep direction (32 x ring floats), the child
// codes of 32 x (nmax - 2) nodes, and per slot its descriptor, lambda, the
// averaging term and (mode 1) omega and alpha.
inline size_t sweep_smem_bytes(int nmax, int nhops, int mode, int ring) {
  size_t b = (size_t)nmax * kWarp * 4 + (size_t)ring * kWarp * 4 + (size_t)(nmax - 2) * kWarp * 2 +
             (size_t)nhops * kWarp * (mode ? 18 : 10);
  return (b + 127) / 128 * 128;
}
// The backward sweeps keep both cost arrays whole (the ring would need a
// test for terminal children on every arc): as above with ring = nmax.
inline size_t sweep_smem_bytes_bwd(int nmax, int nhops, int mode) {
  return sweep_smem_bytes(nmax, nhops, mode, nmax);
}
// ... and in the adjoint kernels: two gradient arrays, the argmin record and
// the child codes per node; per slot the descriptor and the lambda gradient
// (the other per-slot inputs of the reverse are read into registers a level
// ahead, the same in both modes).
inline size_t adjoint_smem_bytes(int nmax, int nhops) {
  const size_t nn = (size_t)nmax * kWarp, ns = (size_t)nhops * kWarp;
  size_t b = nn * 10 + ns * 6 + (size_t)(nmax - 2) * kWarp * 2;
  return (b + 127) / 128 * 128;
}

dg_status build_plan(const dg_rows* rows, const dg_options* opts, Plan& plan);
dg_status validate_plan(const Plan& plan);

// error reporting
dg_status fail(dg_status st, const std::string& msg);
void clear_error();

}  // namespace dg

struct dg_plan_s {
  dg::Plan p;
};
