// dg_internal.h -- layout of the device arena and declarations shared by the
// host builder, the kernels and the C ABI of libdg.  Not installed.
#pragma once

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include <vector_types.h>

#include "../../include/dg.h"

namespace dg {

// Child codes of a node inside a tile (16-bit tile-local node index or a
// terminal).
constexpr uint32_t kBot = 0xFFFFu;
constexpr uint32_t kTop = 0xFFFEu;
constexpr int kWarp = 32;
constexpr int kMaxWidth = 32;  // nodes of one BDD level; a level is one warp segment

// One tile = the BDDs one CTA sweeps.  Its nodes are stored hop-major in warp
// rows of 32 lanes; a BDD level ("layer", one Lagrange slot) never straddles
// two rows.  Slots are hop-major in the same order as the layers.
struct Tile {
  int32_t row_base;   // first global warp row (node base = 32 * row_base)
  int32_t slot_base;  // first arena slot (multiple of 4)
  int32_t hop_base;   // offset of the tile's hop table (nhops + 1 entries)
  int32_t nrows;      // warp rows
  int32_t nslots;     // slots, padded to a multiple of 4
  int32_t nhops;      // longest BDD of the tile
  int32_t maxw;       // widest level of the tile (bounds the segmented min)
  int32_t nbdd;
};
static_assert(sizeof(Tile) == 32, "Tile is 32 bytes");

// Per warp row: bit l of head marks lane l as the first node of a layer;
// info = first tile-local slot of the row | (valid lanes << 16).
struct RowMeta {
  uint32_t head;
  uint32_t info;
};

// Device view of an arena (all pointers inside the caller's buffer).
struct DevArena {
  const Tile* tiles;
  const uint32_t* hoptab;   // row_off | slot_off << 16 (tile-local)
  const RowMeta* rows;
  const uint32_t* lohi;     // lo | hi << 16 per node
  const int32_t* slot_var;  // variable of a slot, -1 for padding
  const int32_t* slot_row;  // original row of a slot, -1 for padding
  const int32_t* var_ptr;   // CSR over variables: slots of variable i
  const int32_t* var_slots; // arena slots, grouped by variable, rows ascending
  const double* c;          // objective, float64[n]
  const float* invdeg;      // 1/|J_i| (0 for uncovered variables)
  const int64_t* inst_row_ptr;
  const int32_t* inst_var_ptr;
  const int4* lb_chunks;    // {instance, kind (0 rows, 1 vars), begin, end}
  const int32_t* inst_chunk_ptr;
  float* S;                 // scratch: per-variable sum of M (snapshot)
  float* E;                 // scratch: E^j per original row
  double* lb_part;          // scratch: one partial sum per lb chunk
  int32_t n;
  int32_t num_inst;
  int64_t m;
  int64_t num_slots;
  int32_t num_tiles;
  int32_t num_lb_chunks;
};

struct Plan {
  // sizes
  dg_sizes sizes{};
  int64_t hop_histogram[64]{};
  // host images of the device arrays
  std::vector<Tile> tiles;
  std::vector<uint32_t> hoptab;
  std::vector<RowMeta> rows;
  std::vector<uint32_t> lohi;
  std::vector<int32_t> slot_var, slot_row;
  std::vector<int32_t> var_ptr, var_slots;
  std::vector<double> c;
  std::vector<float> invdeg;
  std::vector<int64_t> inst_row_ptr;
  std::vector<int32_t> inst_var_ptr;
  std::vector<int32_t> lb_chunks;  // 4 ints per chunk
  std::vector<int32_t> inst_chunk_ptr;
  std::vector<int64_t> slot_to_csr;
  // canonical BDDs (for dg_bdd_export): per CSR slot the level width, per
  // node the child ranks (-2 bottom, -1 top)
  std::vector<int64_t> row_ptr;
  std::vector<int64_t> node_ptr;  // per row, first node
  std::vector<int8_t> lo8, hi8;
  // byte offsets of every array inside the arena
  struct Off {
    size_t tiles, hoptab, rows, lohi, slot_var, slot_row, var_ptr, var_slots, c, invdeg, inst_row_ptr, inst_var_ptr,
        lb_chunks, inst_chunk_ptr, S, E, lb_part, total;
  } off{};
  size_t smem_sweep = 0;   // dynamic smem of the sweep kernels
  size_t smem_adjoint = 0; // dynamic smem of the adjoint kernels
  int32_t max_tile_rows = 0, max_tile_slots = 0, max_tile_hops = 0;
};

// Shared-memory footprint of one tile in the sweep kernels.
inline size_t sweep_smem_bytes(int nrows, int nslots, int nhops) {
  size_t nn = (size_t)nrows * kWarp;
  return nn * 12 + (size_t)nrows * 8 + (size_t)(nhops + 1) * 4 + (size_t)nslots * 16 + 64;
}
// ... and in the adjoint kernels (adds per-node adjoints, argmin codes and
// per-slot recomputed quantities).
inline size_t adjoint_smem_bytes(int nrows, int nslots, int nhops) {
  size_t nn = (size_t)nrows * kWarp;
  return nn * 24 + (size_t)nrows * 8 + (size_t)(nhops + 1) * 4 + (size_t)nslots * 40 + 64;
}

dg_status build_plan(const dg_rows* rows, const dg_options* opts, Plan& plan);

// error reporting
dg_status fail(dg_status st, const std::string& msg);
void clear_error();

}  // namespace dg

struct dg_plan_s {
  dg::Plan p;
};
