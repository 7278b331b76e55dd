// Host-only harness for the plan validator: builds the plan of a small
// instance with the library's own builder, then corrupts one invariant at a
// time and prints, per case, the status and message of validate_plan.
// Compiled and run by tests/test_lib_cpu.py together with builder.cpp; it
// supplies the error-reporting functions that api.cu defines in the library.
#include <cstdio>
#include <functional>
#include <string>
#include <vector>

#include "dg_internal.h"

namespace dg {
static std::string g_msg;
dg_status fail(dg_status st, const std::string& msg) {
  g_msg = msg;
  return st;
}
void clear_error() { g_msg.clear(); }
}  // namespace dg

int main() {
  using namespace dg;
  // 12 variables, 9 rows of 2..5 variables (<=, >=, =), one instance; fewer
  // than 32 rows, so the only tile has padding lanes
  const int n = 12;
  std::vector<std::vector<int>> rows = {{0, 1, 2},    {1, 3, 4, 5}, {2, 5, 6},     {0, 7},       {3, 8, 9, 10, 11},
                                        {4, 6, 8},    {7, 9},       {1, 10, 11},   {2, 3, 4, 5, 6}};
  std::vector<int8_t> sense = {0, 0, 1, 0, 0, 2, 1, 0, 0};
  std::vector<int32_t> rhs = {1, 2, 1, 1, 2, 1, 1, 1, 3};
  std::vector<int64_t> row_ptr = {0};
  std::vector<int32_t> col, coef;
  for (auto& r : rows) {
    for (int v : r) {
      col.push_back(v);
      coef.push_back(1);
    }
    row_ptr.push_back((int64_t)col.size());
  }
  std::vector<double> c(n);
  for (int i = 0; i < n; ++i) c[i] = (i % 3) - 1.0 + 0.1 * i;
  dg_rows R{};
  R.num_inst = 1;
  R.n = n;
  R.m = (int64_t)rows.size();
  R.row_ptr = row_ptr.data();
  R.col = col.data();
  R.coef = coef.data();
  R.sense = sense.data();
  R.rhs = rhs.data();
  R.c = c.data();
  dg_options o{};
  Plan P;
  if (build_plan(&R, &o, P) != DG_OK) {
    std::printf("build failed: %s\n", g_msg.c_str());
    return 1;
  }
  auto run = [&](const char* name, const std::function<void(Plan&)>& corrupt) {
    Plan Q = P;
    corrupt(Q);
    g_msg.clear();
    const dg_status st = validate_plan(Q);
    std::printf("%s|%d|%s\n", name, (int)st, g_msg.c_str());
  };
  // first real slot and node of lane 0, and a padding lane of tile 0
  const int pad_lane = P.tiles[0].nbdd;
  run("intact", [](Plan&) {});
  run("child_outside_next_level", [](Plan& Q) { Q.lohi8[0] = (uint16_t)(200 | (200 << 8)); });
  run("descriptor_first", [](Plan& Q) { Q.desc[kWarp] = (uint16_t)(Q.desc[kWarp] + 1); });
  run("padding_in_use", [&](Plan& Q) { Q.slot_var[pad_lane] = 0; });
  run("variable_out_of_range", [&](Plan& Q) { Q.slot_var[0] = n; });
  run("slot_map_duplicate", [](Plan& Q) { Q.slot_to_csr[1] = Q.slot_to_csr[0]; });
  run("variable_slot_list", [](Plan& Q) { std::swap(Q.var_slots[0], Q.var_slots[Q.var_slots.size() - 1]); });
  run("ell_column", [](Plan& Q) { Q.var_ell[0] = -1; });
  run("group_shared_memory", [](Plan& Q) { Q.groups[0].region_bytes = 0; });
  run("bound_chunk_gap", [](Plan& Q) { Q.lb_chunks[3] -= 1; });
  run("tile_bases", [](Plan& Q) { Q.tiles[0].slot_base = kWarp; });
  run("wide_variable_list", [](Plan& Q) { Q.wide_vars.push_back(0); });
  run("long_bdd_order", [](Plan& Q) { Q.long_order.push_back(0); });
  return 0;
}
