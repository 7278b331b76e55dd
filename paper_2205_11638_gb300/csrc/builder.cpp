// builder.cpp -- host side of dg_plan: rows -> canonical quasi-reduced BDDs
// -> tiles -> the structure-of-arrays image of the device arena.
//
// BDDs (App. B of DOGE-Train): one per constraint row; level h holds the nodes
// of the row's h-th variable (ascending variable id), every root-to-top path
// meets one node per level and the paths are exactly the feasible
// assignments.  A node is identified with the set of feasible completions of
// the partial sums that reach it; nodes of a level are ordered by
// (lo rank, hi rank) with bottom = -2 < top = -1 < ranks, so that the
// minimal quasi-reduced BDD of a row is one fixed table.
#include <algorithm>
#include <atomic>
#include <cstring>
#include <numeric>
#include <thread>

#include "dg_internal.h"

namespace dg {

namespace {

constexpr int kCodeBot = -2;
constexpr int kCodeTop = -1;
constexpr size_t kMaxStatesPerRow = size_t(1) << 22;

struct RowResult {
  int status = 0;  // dg_status
  std::string msg;
};

// Scratch reused across the rows one host thread builds.
struct RowScratch {
  std::vector<int64_t> sums;      // reachable partial sums (clamped), level by level
  std::vector<int64_t> rem_lo, rem_hi;  // per level: least / largest sum of the remaining terms
  std::vector<size_t> lvl;        // level offsets into sums
  std::vector<int32_t> code;      // code of every (level, sum)
  std::vector<uint64_t> keys;     // (lo+2) << 32 | (hi+2) per sum of a level
  std::vector<std::vector<uint64_t>> level_keys;  // per level: its nodes' keys, ascending
  int64_t nodes = 0;
  int maxw = 0;
};

inline bool row_holds(int64_t act, int sense, int64_t rhs) {
  switch (sense) {
    case 0: return act <= rhs;
    case 1: return act >= rhs;
    default: return act == rhs;
  }
}

inline int key_lo(uint64_t key) { return int(key >> 32) - 2; }
inline int key_hi(uint64_t key) { return int(key & 0xFFFFFFFFu) - 2; }

// Builds the BDD of one row: on success sc.level_keys[h] holds the nodes of
// level h in canonical order as keys (lo code + 2) << 32 | (hi code + 2),
// codes being ranks on level h + 1 with bottom = -2 and top = -1.
RowResult build_row(const int32_t* a, int k, int sense, int64_t rhs, RowScratch& sc) {
  RowResult res;
  // 1. partial sums reachable from the root, per level (sorted, unique).  A
  // partial sum s of level g behaves like any other sum outside the window
  // [rhs - rem_hi[g] - 1, rhs - rem_lo[g] + 1] on the same side of it (below
  // it every completion is feasible for '<=' and none for '>=' and '='; above
  // it the reverse), and adding a term keeps it outside, so sums are clamped
  // to the window: the same residual functions, hence the same BDD, from
  // O(k * window) partial sums instead of every reachable one.
  sc.rem_lo.assign(k + 1, 0);
  sc.rem_hi.assign(k + 1, 0);
  for (int h = k - 1; h >= 0; --h) {
    sc.rem_lo[h] = sc.rem_lo[h + 1] + std::min<int64_t>(0, a[h]);
    sc.rem_hi[h] = sc.rem_hi[h + 1] + std::max<int64_t>(0, a[h]);
  }
  auto clamp = [&](int64_t v, int g) {
    return std::min(std::max(v, rhs - sc.rem_hi[g] - 1), rhs - sc.rem_lo[g] + 1);
  };
  sc.sums.clear();
  sc.lvl.assign(1, 0);
  sc.sums.push_back(clamp(0, 0));
  sc.lvl.push_back(1);
  for (int h = 0; h < k; ++h) {
    size_t b = sc.lvl[h], e = sc.lvl[h + 1];
    size_t p = b, q = b;
    while (p < e || q < e) {  // merge {s} and {s + a_h}, both ascending (clamping is monotone)
      int64_t x = p < e ? clamp(sc.sums[p], h + 1) : INT64_MAX;
      int64_t y = q < e ? clamp(sc.sums[q] + a[h], h + 1) : INT64_MAX;
      int64_t v = std::min(x, y);
      if (x == v) ++p;
      if (y == v) ++q;
      if (sc.sums.size() == e || sc.sums.back() != v) sc.sums.push_back(v);
    }
    sc.lvl.push_back(sc.sums.size());
    if (sc.sums.size() > kMaxStatesPerRow) {
      res.status = DG_EINVAL;
      res.msg = "row has too many distinct partial sums for the BDD builder";
      return res;
    }
  }
  // 2. codes bottom-up
  sc.code.assign(sc.sums.size(), kCodeBot);
  for (size_t q = sc.lvl[k]; q < sc.lvl[k + 1]; ++q) sc.code[q] = row_holds(sc.sums[q], sense, rhs) ? kCodeTop : kCodeBot;
  if (sc.level_keys.size() < (size_t)k) sc.level_keys.resize(k);
  for (int h = k - 1; h >= 0; --h) {
    const size_t b = sc.lvl[h], e = sc.lvl[h + 1];
    const size_t nb = sc.lvl[h + 1], ne = sc.lvl[h + 2];
    const int64_t* nxt = sc.sums.data() + nb;
    const size_t nn = ne - nb;
    sc.keys.resize(e - b);
    for (size_t q = b; q < e; ++q) {
      const int64_t s = sc.sums[q];
      size_t i0 = std::lower_bound(nxt, nxt + nn, clamp(s, h + 1)) - nxt;
      size_t i1 = std::lower_bound(nxt, nxt + nn, clamp(s + a[h], h + 1)) - nxt;
      const int c0 = sc.code[nb + i0], c1 = sc.code[nb + i1];
      sc.keys[q - b] = (uint64_t(uint32_t(c0 + 2)) << 32) | uint64_t(uint32_t(c1 + 2));
    }
    std::vector<uint64_t>& uniq = sc.level_keys[h];
    uniq.assign(sc.keys.begin(), sc.keys.end());
    std::sort(uniq.begin(), uniq.end());
    uniq.erase(std::unique(uniq.begin(), uniq.end()), uniq.end());
    if (!uniq.empty() && uniq.front() == 0u) uniq.erase(uniq.begin());  // (bottom, bottom)
    for (size_t q = b; q < e; ++q) {
      const uint64_t key = sc.keys[q - b];
      sc.code[q] = key == 0u ? kCodeBot : int(std::lower_bound(uniq.begin(), uniq.end(), key) - uniq.begin());
    }
  }
  if (sc.code[0] == kCodeBot) {
    res.status = DG_EINFEASIBLE;
    res.msg = "row has no feasible assignment";
    return res;
  }
  sc.nodes = 0;
  sc.maxw = 0;
  for (int h = 0; h < k; ++h) {
    bool zero_ok = false, one_ok = false;
    for (uint64_t key : sc.level_keys[h]) {
      zero_ok |= key_lo(key) != kCodeBot;
      one_ok |= key_hi(key) != kCodeBot;
    }
    if (!zero_ok || !one_ok) {
      res.status = DG_EFORCED;
      res.msg = "row fixes one of its variables (presolve it away)";
      return res;
    }
    sc.nodes += (int64_t)sc.level_keys[h].size();
    sc.maxw = std::max<int>(sc.maxw, (int)sc.level_keys[h].size());
  }
  return res;
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

dg_status build_plan(const dg_rows* R, const dg_options* opts, Plan& P) {
  if (!R || !R->row_ptr || !R->col || !R->coef || !R->sense || !R->rhs || !R->c)
    return fail(DG_EINVAL, "dg_plan: null row array");
  const int32_t n = R->n;
  const int64_t m = R->m;
  if (n < 0 || m < 0) return fail(DG_EINVAL, "dg_plan: negative sizes");
  if (opts && opts->long_lanes != 0 &&
      (opts->long_lanes < 0 || opts->long_lanes > kWarp || (opts->long_lanes & (opts->long_lanes - 1)) != 0))
    return fail(DG_EINVAL, "dg_plan: long_lanes must be 0 or a power of two up to 32");
  if (R->row_ptr[0] != 0) return fail(DG_EINVAL, "dg_plan: row_ptr[0] must be 0");
  const int64_t nnz = R->row_ptr[m];
  if (nnz > (int64_t)INT32_MAX / 2) return fail(DG_EINVAL, "dg_plan: too many nonzeros");
  for (int64_t j = 0; j < m; ++j) {
    const int64_t b = R->row_ptr[j], e = R->row_ptr[j + 1];
    if (e <= b) return fail(DG_EINVAL, "dg_plan: empty row " + std::to_string(j));
    if (e - b > 4096) return fail(DG_EINVAL, "dg_plan: row longer than 4096 variables");
    if (R->sense[j] < 0 || R->sense[j] > 2) return fail(DG_EINVAL, "dg_plan: sense must be 0, 1 or 2");
    for (int64_t s = b; s < e; ++s) {
      if (R->col[s] < 0 || R->col[s] >= n || (s > b && R->col[s] <= R->col[s - 1]))
        return fail(DG_EINVAL, "dg_plan: columns of row " + std::to_string(j) + " must be ascending ids in [0,n)");
    }
  }
  for (int32_t i = 0; i < n; ++i)
    if (!(R->c[i] == R->c[i]) || R->c[i] == 1.0 / 0.0 || R->c[i] == -1.0 / 0.0)
      return fail(DG_EINVAL, "dg_plan: non-finite cost");
  // instances
  int32_t ni = R->num_inst <= 1 || !R->inst_row_ptr || !R->inst_var_ptr ? 1 : R->num_inst;
  P.inst_row_ptr.resize(ni + 1);
  P.inst_var_ptr.resize(ni + 1);
  if (ni == 1) {
    P.inst_row_ptr = {0, m};
    P.inst_var_ptr = {0, n};
  } else {
    for (int k = 0; k <= ni; ++k) {
      P.inst_row_ptr[k] = R->inst_row_ptr[k];
      P.inst_var_ptr[k] = R->inst_var_ptr[k];
    }
    if (P.inst_row_ptr[0] != 0 || P.inst_row_ptr[ni] != m || P.inst_var_ptr[0] != 0 || P.inst_var_ptr[ni] != n)
      return fail(DG_EINVAL, "dg_plan: instance pointers must span all rows and variables");
    for (int k = 0; k < ni; ++k) {
      if (P.inst_row_ptr[k + 1] < P.inst_row_ptr[k] || P.inst_var_ptr[k + 1] < P.inst_var_ptr[k])
        return fail(DG_EINVAL, "dg_plan: instance pointers must be non-decreasing");
      for (int64_t j = P.inst_row_ptr[k]; j < P.inst_row_ptr[k + 1]; ++j)
        for (int64_t s = R->row_ptr[j]; s < R->row_ptr[j + 1]; ++s)
          if (R->col[s] < P.inst_var_ptr[k] || R->col[s] >= P.inst_var_ptr[k + 1])
            return fail(DG_EINVAL, "dg_plan: row uses a variable of another instance");
    }
  }

  // ---- 1. BDDs, in parallel over contiguous row ranges --------------------
  int nthreads = opts && opts->num_threads > 0 ? opts->num_threads : (int)std::thread::hardware_concurrency();
  nthreads = std::max(1, std::min<int>(nthreads, (int)std::max<int64_t>(1, std::min<int64_t>(m / 64, nnz / 16384))));
  struct Part {
    std::vector<uint8_t> width;
    std::vector<int8_t> lo, hi;
    std::vector<int32_t> nodes_of_row;
    // rows whose BDD exceeds the tile limits: row, level widths, child ranks
    std::vector<int64_t> long_rows;
    std::vector<int32_t> lwidth, llo, lhi;
    RowResult err;
    int64_t err_row = -1;
  };
  std::vector<Part> parts(nthreads);
  std::vector<int64_t> cut(nthreads + 1);
  for (int t = 0; t <= nthreads; ++t) cut[t] = m * t / nthreads;
  auto worker = [&](int t) {
    RowScratch sc;
    Part& pt = parts[t];
    pt.nodes_of_row.reserve(cut[t + 1] - cut[t]);
    for (int64_t j = cut[t]; j < cut[t + 1]; ++j) {
      const int64_t b = R->row_ptr[j];
      const int k = (int)(R->row_ptr[j + 1] - b);
      RowResult r = build_row(R->coef + b, k, R->sense[j], R->rhs[j], sc);
      if (r.status != 0) {
        pt.err = r;
        pt.err_row = j;
        return;
      }
      if (sc.nodes <= kMaxNodesPerBdd && sc.maxw <= kMaxWidth) {
        for (int h = 0; h < k; ++h) {
          pt.width.push_back((uint8_t)sc.level_keys[h].size());
          for (uint64_t key : sc.level_keys[h]) {
            pt.lo.push_back((int8_t)key_lo(key));
            pt.hi.push_back((int8_t)key_hi(key));
          }
        }
        pt.nodes_of_row.push_back((int32_t)sc.nodes);
      } else {
        pt.width.insert(pt.width.end(), (size_t)k, (uint8_t)0);
        pt.nodes_of_row.push_back(0);
        pt.long_rows.push_back(j);
        for (int h = 0; h < k; ++h) {
          pt.lwidth.push_back((int32_t)sc.level_keys[h].size());
          for (uint64_t key : sc.level_keys[h]) {
            pt.llo.push_back(key_lo(key));
            pt.lhi.push_back(key_hi(key));
          }
        }
      }
    }
  };
  if (nthreads == 1) {
    worker(0);
  } else {
    std::vector<std::thread> th;
    for (int t = 0; t < nthreads; ++t) th.emplace_back(worker, t);
    for (auto& x : th) x.join();
  }
  for (int t = 0; t < nthreads; ++t)
    if (parts[t].err.status != 0)
      return fail((dg_status)parts[t].err.status, "dg_plan: row " + std::to_string(parts[t].err_row) + ": " +
                                                      parts[t].err.msg);
  std::vector<uint8_t> width;
  width.reserve(nnz);
  P.node_ptr.assign(m + 1, 0);
  std::vector<int64_t> long_rows;
  std::vector<int32_t> long_width;  // level widths of the long BDDs, in row order
  {
    int64_t j = 0;
    for (int t = 0; t < nthreads; ++t) {
      width.insert(width.end(), parts[t].width.begin(), parts[t].width.end());
      P.lo8.insert(P.lo8.end(), parts[t].lo.begin(), parts[t].lo.end());
      P.hi8.insert(P.hi8.end(), parts[t].hi.begin(), parts[t].hi.end());
      for (int32_t c : parts[t].nodes_of_row) {
        P.node_ptr[j + 1] = P.node_ptr[j] + c;
        ++j;
      }
      long_rows.insert(long_rows.end(), parts[t].long_rows.begin(), parts[t].long_rows.end());
      long_width.insert(long_width.end(), parts[t].lwidth.begin(), parts[t].lwidth.end());
      P.long_lo.insert(P.long_lo.end(), parts[t].llo.begin(), parts[t].llo.end());
      P.long_hi.insert(P.long_hi.end(), parts[t].lhi.begin(), parts[t].lhi.end());
      std::vector<uint8_t>().swap(parts[t].width);
      std::vector<int8_t>().swap(parts[t].lo);
      std::vector<int8_t>().swap(parts[t].hi);
      std::vector<int32_t>().swap(parts[t].llo);
      std::vector<int32_t>().swap(parts[t].lhi);
    }
  }
  P.row_ptr.assign(R->row_ptr, R->row_ptr + m + 1);
  P.long_of_row.assign(m, -1);
  for (size_t b = 0; b < long_rows.size(); ++b) P.long_of_row[long_rows[b]] = (int32_t)b;
  const int64_t num_long_nodes = (int64_t)P.long_lo.size();
  const int64_t num_nodes = P.node_ptr[m] + num_long_nodes;

  // ---- 2. tiles: 32 BDDs per tile, one per lane ---------------------------
  // Rows are cut into chunks of consecutive rows (so that a tile's variables,
  // and the S values its lanes gather, stay close together); inside a chunk
  // BDDs are sorted by hop count and node count, longest first, and every 32
  // consecutive BDDs form a tile.  Inside a tile everything is interleaved by
  // lane: slot (h, b) is slot_base + 32 h + b and node number n of lane b is
  // element 32 n + b of the per-tile arrays.  Node numbers 0 and 1 stand for
  // the top and bottom terminals, the BDD's own nodes are numbered 2, 3, ...
  // level by level; child codes are node numbers (8 bits).
  // Rows of the long BDDs take no tile (they are laid out after the tiles).
  const int64_t kChunkRows = opts && opts->chunk_rows > 0 ? opts->chunk_rows : 16384;
  std::vector<int64_t> order;
  order.reserve(m - (int64_t)long_rows.size());
  for (int64_t j = 0; j < m; ++j)
    if (P.long_of_row[j] < 0) order.push_back(j);
  const int64_t m_tiles = (int64_t)order.size();
  std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) {
    const int64_t cx = x / kChunkRows, cy = y / kChunkRows;
    if (cx != cy) return cx < cy;
    int64_t kx = R->row_ptr[x + 1] - R->row_ptr[x], ky = R->row_ptr[y + 1] - R->row_ptr[y];
    if (kx != ky) return kx > ky;
    return (P.node_ptr[x + 1] - P.node_ptr[x]) > (P.node_ptr[y + 1] - P.node_ptr[y]);
  });
  int max_hops = 0, max_width = 0;
  for (int64_t j = 0; j < m; ++j) {
    int k = (int)(R->row_ptr[j + 1] - R->row_ptr[j]);
    max_hops = std::max(max_hops, k);
    P.hop_histogram[std::min(k, 63)]++;
  }
  for (uint8_t w : width) max_width = std::max<int>(max_width, w);
  for (int32_t w : long_width) max_width = std::max<int>(max_width, w);

  const int T = (int)((m_tiles + kWarp - 1) / kWarp);
  if (opts && opts->host_mb_limit > 0) {
    // host bytes of the arena image about to be built: child codes, slot
    // arrays (descriptor, variable, row, CSR position), variable CSR and ELL
    const double est = 2.0 * (double)num_nodes * 1.1 + 18.0 * (double)nnz * 1.1 + 8.0 * (double)nnz +
                       (16.0 + 4.0 * kEll) * (double)n + 40.0 * (double)T;
    if (est > (double)opts->host_mb_limit * 1048576.0)
      return fail(DG_ENOMEM, "dg_plan: the arena image needs about " + std::to_string((long long)(est / 1048576.0)) +
                                 " MiB of host memory, more than host_mb_limit");
  }
  // tile t takes BDDs order[32 t .. 32 t + 31]; tiles are then laid out by
  // shared-memory footprint, largest first, so that tiles of one launch group
  // are contiguous (and the longest tiles start first)
  std::vector<int> tile_nh(T, 0), tile_nmax(T, 2), tile_maxw(T, 1), tile_order(T);
  for (int t = 0; t < T; ++t) {
    for (int64_t q = (int64_t)t * kWarp; q < std::min<int64_t>(m_tiles, (int64_t)(t + 1) * kWarp); ++q) {
      const int64_t j = order[q];
      tile_nh[t] = std::max<int>(tile_nh[t], (int)(R->row_ptr[j + 1] - R->row_ptr[j]));
      tile_nmax[t] = std::max<int>(tile_nmax[t], 2 + (int)(P.node_ptr[j + 1] - P.node_ptr[j]));
      for (int64_t c = R->row_ptr[j]; c < R->row_ptr[j + 1]; ++c) tile_maxw[t] = std::max<int>(tile_maxw[t], width[c]);
    }
    tile_order[t] = t;
  }
  auto tile_smem = [&](int t) { return sweep_smem_bytes(tile_nmax[t], tile_nh[t], 1, ring_size(tile_maxw[t])); };
  std::stable_sort(tile_order.begin(), tile_order.end(), [&](int x, int y) { return tile_smem(x) > tile_smem(y); });
  P.tiles.resize(T);
  P.slot_to_csr.clear();
  std::vector<int64_t> slot_of_csr(nnz, -1);
  int64_t node_base = 0, slot_base = 0;
  size_t smem_max = 0, smem_adj_max = 0;
  for (int t = 0; t < T; ++t) {
    const int src = tile_order[t];
    const int64_t q0 = (int64_t)src * kWarp, q1 = std::min<int64_t>(m_tiles, q0 + kWarp);
    const int nb = (int)(q1 - q0);
    const int nh = tile_nh[src], nmax = tile_nmax[src];
    const int64_t tslots = (int64_t)nh * kWarp;
    Tile& tile = P.tiles[t];
    tile.node_base = (int32_t)node_base;
    tile.slot_base = (int32_t)slot_base;
    tile.nmax = nmax;
    tile.nhops = nh;
    tile.nbdd = nb;
    int maxw = 1;
    P.desc.resize(slot_base + tslots, 0);
    P.slot_var.resize(slot_base + tslots, -1);
    P.slot_row.resize(slot_base + tslots, -1);
    P.slot_to_csr.resize(slot_base + tslots, -1);
    P.lohi8.resize(node_base + (int64_t)(nmax - 2) * kWarp, 0x0101u);
    for (int bb = 0; bb < nb; ++bb) {
      const int64_t j = order[q0 + bb];
      const int k = (int)(R->row_ptr[j + 1] - R->row_ptr[j]);
      const int64_t nbj = P.node_ptr[j];
      int first = 2;
      for (int h = 0; h < k; ++h) {
        const int64_t csr = R->row_ptr[j] + h;
        const int w = width[csr];
        maxw = std::max(maxw, w);
        const int64_t sl = slot_base + (int64_t)h * kWarp + bb;
        P.desc[sl] = (uint16_t)(first | (w << 8));
        P.slot_var[sl] = R->col[csr];
        P.slot_row[sl] = (int32_t)j;
        P.slot_to_csr[sl] = csr;
        slot_of_csr[csr] = sl;
        const int first_next = first + w;
        for (int r = 0; r < w; ++r) {
          auto code = [&](int8_t cc) -> uint32_t {
            return cc == kCodeBot ? kBotCode : (cc == kCodeTop ? kTopCode : (uint32_t)(first_next + cc));
          };
          const int64_t nidx = nbj + (first - 2) + r;
          P.lohi8[node_base + (int64_t)(first - 2 + r) * kWarp + bb] =
              (uint16_t)(code(P.lo8[nidx]) | (code(P.hi8[nidx]) << 8));
        }
        first = first_next;
      }
    }
    tile.maxw = maxw;
    tile.ring = ring_size(maxw);
    smem_max = std::max(smem_max, sweep_smem_bytes(nmax, nh, 1, tile.ring));
    smem_adj_max = std::max(smem_adj_max, adjoint_smem_bytes(nmax, nh));
    P.max_tile_rows = std::max(P.max_tile_rows, nmax);
    P.max_tile_slots = std::max<int32_t>(P.max_tile_slots, (int32_t)tslots);
    P.max_tile_hops = std::max(P.max_tile_hops, nh);
    node_base += (int64_t)(nmax - 2) * kWarp;
    slot_base += tslots;
  }
  // launch groups: consecutive tiles whose footprints stay within 1/kGroupRatio
  // of the group's largest one
  {
    const double kGroupRatio =
        opts && opts->group_ratio_pct > 0 && opts->group_ratio_pct <= 100 ? opts->group_ratio_pct / 100.0 : 0.85;
    int32_t t0 = 0;
    size_t gmax = 0, gmax0 = 0;
    for (int t = 0; t < T; ++t) {
      const size_t r = sweep_smem_bytes(P.tiles[t].nmax, P.tiles[t].nhops, 1, P.tiles[t].ring);
      if (t > t0 && (double)r < kGroupRatio * (double)gmax) {
        P.groups.push_back({t0, t, (int32_t)gmax, (int32_t)gmax0, 0, 0, 0, 0, 0, 0, {0, 0}});
        t0 = t;
        gmax = 0;
        gmax0 = 0;
      }
      gmax = std::max(gmax, r);
      gmax0 = std::max(gmax0, sweep_smem_bytes(P.tiles[t].nmax, P.tiles[t].nhops, 0, P.tiles[t].ring));
    }
    if (T > 0) P.groups.push_back({t0, T, (int32_t)gmax, (int32_t)gmax0, 0, 0, 0, 0, 0, 0, {0, 0}});
    for (LaunchGroup& g : P.groups)
      for (int t = g.tile0; t < g.tile1; ++t) {
        g.region_bwd1 = std::max<int32_t>(g.region_bwd1, (int32_t)sweep_smem_bytes_bwd(P.tiles[t].nmax, P.tiles[t].nhops, 1));
        g.region_bwd0 = std::max<int32_t>(g.region_bwd0, (int32_t)sweep_smem_bytes_bwd(P.tiles[t].nmax, P.tiles[t].nhops, 0));
        g.meta_bytes = std::max<int32_t>(g.meta_bytes, (P.tiles[t].nmax - 2) * kWarp * 2);
        smem_max = std::max<size_t>(smem_max, (size_t)g.region_bwd1);
      }
    // work estimate per group, then longest-processing-time assignment of the
    // groups to the kStreams streams that run one sweep's launches concurrently
    for (LaunchGroup& g : P.groups)
      for (int t = g.tile0; t < g.tile1; ++t) g.work += (int64_t)kWarp * P.tiles[t].nmax * P.tiles[t].nhops;
    // the long BDDs are one more launch (index -1 here): a warp walks each
    // level in turn, estimated like a tile level of 16 nodes per level
    int64_t long_work = 0;
    for (size_t b = 0; b < long_rows.size(); ++b)
      long_work += (int64_t)kWarp * 16 * (R->row_ptr[long_rows[b] + 1] - R->row_ptr[long_rows[b]]);
    auto work_of = [&](int x) { return x < 0 ? long_work : P.groups[x].work; };
    std::vector<int> idx(P.groups.size());
    std::iota(idx.begin(), idx.end(), 0);
    if (!long_rows.empty()) idx.push_back(-1);
    std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return work_of(x) > work_of(y); });
    std::vector<int64_t> load(kStreams, 0);
    for (int gi : idx) {
      int best = 0;
      for (int k = 1; k < kStreams; ++k)
        if (load[k] < load[best]) best = k;
      if (gi < 0)
        P.long_stream = best;
      else
        P.groups[gi].stream = best;
      load[best] += work_of(gi);
    }
  }
  for (const LaunchGroup& g : P.groups) {
    AdjGroup a{g.tile0, g.tile1, 0, g.stream};
    for (int t = g.tile0; t < g.tile1; ++t)
      a.region = std::max<int32_t>(a.region, (int32_t)adjoint_smem_bytes(P.tiles[t].nmax, P.tiles[t].nhops));
    P.adj_groups.push_back(a);
  }
  // ---- 2b. long BDDs: levels as consecutive slots after the tiles (each
  // BDD's range padded to a multiple of 32), nodes numbered 2, 3, ... level
  // by level with 32-bit children (0 top, 1 bottom), and per node its
  // in-arcs in (parent, beta) order
  P.long_slot_base = (int32_t)slot_base;
  {
    int64_t lslot = slot_base, code_base = 0, lvl_base = 0, cost_base = 0, wpos = 0, rpos = 0;
    P.longs.resize(long_rows.size());
    P.long_rank_ptr.assign(long_rows.size() + 1, 0);
    P.long_code.resize(num_long_nodes);
    P.long_in_ptr.assign(num_long_nodes + 1, 0);
    std::vector<int32_t> first;
    for (size_t b = 0; b < long_rows.size(); ++b) {
      const int64_t j = long_rows[b];
      const int k = (int)(R->row_ptr[j + 1] - R->row_ptr[j]);
      LongBdd& L = P.longs[b];
      L.slot_base = (int32_t)lslot;
      L.k = k;
      L.code_base = (int32_t)code_base;
      L.lvl_base = (int32_t)lvl_base;
      L.cost_base = (int32_t)cost_base;
      L.row = (int32_t)j;
      L.maxw = 0;
      first.assign(k + 1, 2);
      for (int h = 0; h < k; ++h) {
        const int w = long_width[wpos + h];
        first[h + 1] = first[h] + w;
        L.maxw = std::max(L.maxw, w);
      }
      L.nn = first[k] - 2;
      P.long_lvl.insert(P.long_lvl.end(), first.begin(), first.end());
      const int64_t tslots = ((int64_t)k + kWarp - 1) / kWarp * kWarp;
      P.desc.resize(lslot + tslots, 0);
      P.slot_var.resize(lslot + tslots, -1);
      P.slot_row.resize(lslot + tslots, -1);
      P.slot_to_csr.resize(lslot + tslots, -1);
      for (int h = 0; h < k; ++h) {
        const int64_t csr = R->row_ptr[j] + h, sl = lslot + h;
        P.slot_var[sl] = R->col[csr];
        P.slot_row[sl] = (int32_t)j;
        P.slot_to_csr[sl] = csr;
        slot_of_csr[csr] = sl;
      }
      // children as node numbers; in-degree counts
      P.long_rank_ptr[b] = rpos;
      for (int h = 0; h < k; ++h)
        for (int r = 0; r < long_width[wpos + h]; ++r) {
          auto num = [&](int32_t rank) -> int32_t {
            return rank == kCodeBot ? (int32_t)kBotCode : (rank == kCodeTop ? (int32_t)kTopCode : first[h + 1] + rank);
          };
          const int32_t lo = num(P.long_lo[rpos]), hi = num(P.long_hi[rpos]);
          int2& cc = P.long_code[code_base + (first[h] - 2) + r];
          cc.x = lo;
          cc.y = hi;
          if (lo >= 2) P.long_in_ptr[code_base + (lo - 2) + 1]++;
          if (hi >= 2) P.long_in_ptr[code_base + (hi - 2) + 1]++;
          ++rpos;
        }
      wpos += k;
      lslot += tslots;
      code_base += L.nn;
      lvl_base += k + 1;
      cost_base += L.nn + 2;
    }
    P.long_rank_ptr[long_rows.size()] = rpos;
    for (int64_t g = 0; g < num_long_nodes; ++g) P.long_in_ptr[g + 1] += P.long_in_ptr[g];
    P.long_in.assign(P.long_in_ptr[num_long_nodes], 0);
    std::vector<int32_t> fill(P.long_in_ptr.begin(), P.long_in_ptr.end() - 1);
    for (const LongBdd& L : P.longs)  // parents ascending, the 0-arc first
      for (int n = 2; n < L.nn + 2; ++n) {
        const int2 c = P.long_code[L.code_base + n - 2];
        if (c.x >= 2) P.long_in[fill[L.code_base + c.x - 2]++] = n << 1;
        if (c.y >= 2) P.long_in[fill[L.code_base + c.y - 2]++] = (n << 1) | 1;
      }
    slot_base = lslot;
    if (cost_base >= (int64_t)INT32_MAX || P.long_in_ptr[num_long_nodes] >= (int64_t)INT32_MAX)
      return fail(DG_EINVAL, "dg_plan: long BDDs exceed 2^31 nodes or arcs");
    P.long_cost_size = (int32_t)cost_base;
    // the plain sweeps pack the narrow long BDDs several to a warp: list them
    // first, longest first (a warp's BDDs then take about as many levels)
    P.long_order.clear();
    for (size_t b = 0; b < P.longs.size(); ++b)
      if (P.longs[b].maxw <= kWarp) P.long_order.push_back((int32_t)b);
    std::stable_sort(P.long_order.begin(), P.long_order.end(),
                     [&](int32_t x, int32_t y) { return P.longs[x].k > P.longs[y].k; });
    P.num_long_narrow = (int32_t)P.long_order.size();
    P.long_lanes = opts ? opts->long_lanes : 0;
    for (size_t b = 0; b < P.longs.size(); ++b)
      if (P.longs[b].maxw > kWarp) P.long_order.push_back((int32_t)b);
  }
  const int64_t num_slots = slot_base;
  if (num_slots >= (int64_t)INT32_MAX || node_base >= (int64_t)INT32_MAX)
    return fail(DG_EINVAL, "dg_plan: arena exceeds 2^31 slots or nodes");

  // ---- 3. variable CSR (slots of each variable, rows ascending) -----------
  P.var_ptr.assign(n + 1, 0);
  for (int64_t s = 0; s < nnz; ++s) P.var_ptr[R->col[s] + 1]++;
  for (int32_t i = 0; i < n; ++i) P.var_ptr[i + 1] += P.var_ptr[i];
  P.var_slots.assign(nnz, 0);
  {
    std::vector<int32_t> cur(P.var_ptr.begin(), P.var_ptr.end() - 1);
    for (int64_t s = 0; s < nnz; ++s) P.var_slots[cur[R->col[s]]++] = (int32_t)slot_of_csr[s];
  }
  P.c.assign(R->c, R->c + n);
  P.var_ell.assign((size_t)kEll * n, -1);
  P.wide_vars.clear();
  for (int32_t i = 0; i < n; ++i) {
    const int d = P.var_ptr[i + 1] - P.var_ptr[i];
    for (int r = 0; r < std::min(d, kEll); ++r) P.var_ell[(size_t)r * n + i] = P.var_slots[P.var_ptr[i] + r];
    if (d > kEll) P.var_ell[(size_t)(kEll - 1) * n + i] = -2 - P.var_ell[(size_t)(kEll - 1) * n + i];
    if (d > kWide) P.wide_vars.push_back(i);
  }
  P.invdeg.assign(n, 0.0f);
  for (int32_t i = 0; i < n; ++i) {
    int d = P.var_ptr[i + 1] - P.var_ptr[i];
    P.invdeg[i] = d > 0 ? (float)(1.0 / d) : 0.0f;
  }
  // ---- 4. lower-bound chunks: per instance its rows, then its variables ----
  const int kChunk = 4096;
  P.inst_chunk_ptr.assign(ni + 1, 0);
  for (int k = 0; k < ni; ++k) {
    for (int kind = 0; kind < 2; ++kind) {
      int64_t b = kind == 0 ? P.inst_row_ptr[k] : P.inst_var_ptr[k];
      int64_t e = kind == 0 ? P.inst_row_ptr[k + 1] : P.inst_var_ptr[k + 1];
      for (int64_t x = b; x < e; x += kChunk) {
        P.lb_chunks.insert(P.lb_chunks.end(), {k, kind, (int32_t)x, (int32_t)std::min<int64_t>(e, x + kChunk)});
      }
    }
    P.inst_chunk_ptr[k + 1] = (int32_t)(P.lb_chunks.size() / 4);
  }
  // variables no row covers keep their cost: their term of the bound is the
  // constant min(0, c_i) (their S_i is an empty sum, 0, so the kernels may add
  // min(0, S_i) = 0 for them as for every other variable)
  P.inst_unc.assign(ni, 0.0);
  for (int k = 0; k < ni; ++k)
    for (int32_t i = P.inst_var_ptr[k]; i < P.inst_var_ptr[k + 1]; ++i)
      if (P.var_ptr[i + 1] == P.var_ptr[i]) P.inst_unc[k] += std::min(0.0, P.c[i]);
  const int num_chunks = (int)(P.lb_chunks.size() / 4);

  // ---- 5. arena offsets ----------------------------------------------------
  size_t o = 0;
  auto put = [&](size_t bytes) {
    size_t at = o;
    o = align_up(o + std::max<size_t>(bytes, 1), 256);
    return at;
  };
  P.off.tiles = put(P.tiles.size() * sizeof(Tile));
  P.off.desc = put(P.desc.size() * 2);
  P.off.lohi8 = put(P.lohi8.size() * 2);
  P.off.slot_var = put(num_slots * 4);
  P.off.slot_row = put(num_slots * 4);
  P.off.var_ptr = put((size_t)(n + 1) * 4);
  P.off.var_slots = put((size_t)nnz * 4);
  P.off.var_ell = put((size_t)kEll * n * 4);
  P.off.wide_vars = put(P.wide_vars.size() * 4);
  P.off.c = put((size_t)n * 8);
  P.off.invdeg = put((size_t)n * 4);
  P.off.inst_row_ptr = put((size_t)(ni + 1) * 8);
  P.off.inst_var_ptr = put((size_t)(ni + 1) * 4);
  P.off.lb_chunks = put((size_t)num_chunks * 16);
  P.off.inst_chunk_ptr = put((size_t)(ni + 1) * 4);
  P.off.inst_unc = put((size_t)ni * 8);
  P.off.longs = put(P.longs.size() * sizeof(LongBdd));
  P.off.long_code = put(P.long_code.size() * sizeof(int2));
  P.off.long_lvl = put(P.long_lvl.size() * 4);
  P.off.long_in_ptr = put(P.long_in_ptr.size() * 4);
  P.off.long_in = put(P.long_in.size() * 4);
  P.off.long_order = put(P.long_order.size() * 4);
  P.off.S = put((size_t)n * 4);
  P.off.Sbar = put((size_t)n * 4);
  P.off.slot_avg = put((size_t)num_slots * 4);
  P.off.E = put((size_t)m * 4);
  P.off.lb_part = put((size_t)num_chunks * 8);
  P.off.long_d = put((size_t)P.long_cost_size * 4);
  P.off.long_t = put((size_t)P.long_cost_size * 4);
  P.off.nodecost = put(P.lohi8.size() * 4);
  P.off.slot_invdeg = put((size_t)num_slots * 4);
  P.off.total = o;
  P.smem_sweep = align_up(smem_max, 16);
  P.smem_adjoint = align_up(smem_adj_max, 16);

  dg_sizes& z = P.sizes;
  z.arena_bytes = P.off.total;
  z.num_slots = num_slots;
  z.num_lambda = nnz;
  z.num_nodes = num_nodes;
  z.num_nodes_padded = node_base;
  z.n = n;
  z.m = m;
  z.num_inst = ni;
  z.num_tiles = T;
  z.max_hops = max_hops;
  z.max_width = max_width;
  z.smem_bytes = P.smem_sweep;
  z.num_launch_groups = (int32_t)P.groups.size();
  z.num_long_bdds = (int64_t)P.longs.size();
  z.num_long_nodes = num_long_nodes;
  return DG_OK;
}

// Structural invariants of the arena image, checked on the host (the kernels
// index shared and global memory with these numbers without bounds checks).
dg_status validate_plan(const Plan& P) {
  auto bad = [](const std::string& m) { return fail(DG_EINVAL, "dg_plan_validate: " + m); };
  const int32_t n = P.sizes.n;
  const int64_t m = P.sizes.m, NS = P.sizes.num_slots, NL = P.sizes.num_lambda;
  const int64_t T = (int64_t)P.tiles.size();
  if ((int64_t)P.desc.size() != NS || (int64_t)P.slot_var.size() != NS || (int64_t)P.slot_row.size() != NS ||
      (int64_t)P.slot_to_csr.size() != NS || (int64_t)P.lohi8.size() != P.sizes.num_nodes_padded)
    return bad("array sizes disagree with the plan sizes");
  // tiles: contiguous bases, sane shapes, every lane's BDD well formed
  int64_t node_base = 0, slot_base = 0, real_nodes = 0, real_slots = 0;
  std::vector<int64_t> csr_seen(NL, 0);
  for (int64_t t = 0; t < T; ++t) {
    const Tile& tl = P.tiles[t];
    const std::string at = "tile " + std::to_string(t) + ": ";
    if (tl.node_base != node_base || tl.slot_base != slot_base) return bad(at + "bases not contiguous");
    if (tl.nbdd < 1 || tl.nbdd > kWarp || tl.nhops < 1 || tl.nmax < 3 || tl.nmax > kMaxNodesPerBdd + 2 ||
        tl.maxw < 1 || tl.maxw > kMaxWidth || tl.ring != ring_size(tl.maxw))
      return bad(at + "shape out of range");
    for (int b = 0; b < kWarp; ++b) {
      int first = 2, level_w = 0, last_h = -1, row = -1;
      for (int h = 0; h < tl.nhops; ++h) {
        const int64_t q = slot_base + (int64_t)h * kWarp + b;
        const int f = P.desc[q] & 0xFF, w = P.desc[q] >> 8;
        if (b >= tl.nbdd || last_h >= 0) {
          if (P.desc[q] != 0 || P.slot_var[q] != -1 || P.slot_to_csr[q] != -1)
            return bad(at + "padding slot in use");
          continue;
        }
        if (w == 0) {
          if (h == 0) return bad(at + "lane without a BDD");
          last_h = h - 1;
          if (P.slot_var[q] != -1 || P.slot_to_csr[q] != -1) return bad(at + "padding slot in use");
          continue;
        }
        if (f != first || (h == 0 && w != 1) || w > tl.maxw || f + w > tl.nmax)
          return bad(at + "level descriptor inconsistent");
        if (P.slot_var[q] < 0 || P.slot_var[q] >= n) return bad(at + "variable id out of range");
        if (row < 0) row = P.slot_row[q];
        if (P.slot_row[q] != row || row < 0 || row >= m) return bad(at + "slot rows of a lane differ");
        const int64_t c = P.slot_to_csr[q];
        if (c < 0 || c >= NL || csr_seen[c]++) return bad(at + "slot map not a bijection");
        first = f + w;
        level_w = w;
        real_slots++;
        real_nodes += w;
      }
      if (b >= tl.nbdd) continue;
      if (last_h < 0) last_h = tl.nhops - 1;
      // children: next level's nodes (no level skipped) or the bottom; the
      // last level only the terminals; at least one child not the bottom
      int f = 2;
      for (int h = 0; h <= last_h; ++h) {
        const int64_t q = slot_base + (int64_t)h * kWarp + b;
        const int w = P.desc[q] >> 8;
        const int fn = f + w;
        const int wn = h < last_h ? (P.desc[q + kWarp] >> 8) : 0;
        for (int r = 0; r < w; ++r) {
          const uint32_t code = P.lohi8[node_base + (int64_t)(f + r - 2) * kWarp + b];
          const uint32_t ch[2] = {code & 0xFFu, code >> 8};
          if (ch[0] == (uint32_t)kBotCode && ch[1] == (uint32_t)kBotCode) return bad(at + "node with no path to top");
          for (uint32_t c : ch) {
            const bool term = c == (uint32_t)kTopCode || c == (uint32_t)kBotCode;
            if (h == last_h ? !term : (c == (uint32_t)kTopCode || (!term && (c < (uint32_t)fn || c >= (uint32_t)(fn + wn)))))
              return bad(at + "child code outside the next level");
          }
        }
        f = fn;
      }
      (void)level_w;
    }
    node_base += (int64_t)(tl.nmax - 2) * kWarp;
    slot_base += (int64_t)tl.nhops * kWarp;
  }
  if (node_base != P.sizes.num_nodes_padded || slot_base != P.long_slot_base) return bad("tiles do not cover the arrays");
  // long BDDs: consecutive slot ranges after the tiles, levels and children
  // consistent, in-arc lists exactly the arcs into each node in (parent,
  // beta) order
  {
    int64_t lslot = P.long_slot_base, code_base = 0, lvl_base = 0, cost_base = 0;
    for (size_t b = 0; b < P.longs.size(); ++b) {
      const LongBdd& L = P.longs[b];
      const std::string at = "long BDD " + std::to_string(b) + ": ";
      if (L.slot_base != lslot || L.code_base != code_base || L.lvl_base != lvl_base || L.cost_base != cost_base ||
          L.k < 1 || L.nn < 1 || L.row < 0 || L.row >= m || P.long_of_row[L.row] != (int32_t)b)
        return bad(at + "bases or shape inconsistent");
      const int32_t* lvl = P.long_lvl.data() + L.lvl_base;
      if ((size_t)(L.lvl_base + L.k + 1) > P.long_lvl.size() || lvl[0] != 2 || lvl[1] != 3 || lvl[L.k] != L.nn + 2)
        return bad(at + "level table inconsistent");
      const int64_t tslots = ((int64_t)L.k + kWarp - 1) / kWarp * kWarp;
      int row = -1;
      for (int64_t q = lslot; q < lslot + tslots; ++q) {
        const int h = (int)(q - lslot);
        if (h >= L.k) {
          if (P.slot_var[q] != -1 || P.slot_to_csr[q] != -1) return bad(at + "padding slot in use");
          continue;
        }
        if (lvl[h + 1] <= lvl[h]) return bad(at + "empty level");
        if (P.slot_var[q] < 0 || P.slot_var[q] >= n) return bad(at + "variable id out of range");
        if (row < 0) row = P.slot_row[q];
        if (P.slot_row[q] != row || row != L.row) return bad(at + "slot rows differ");
        const int64_t c = P.slot_to_csr[q];
        if (c < 0 || c >= NL || csr_seen[c]++) return bad(at + "slot map not a bijection");
        real_slots++;
      }
      real_nodes += L.nn;
      std::vector<int32_t> indeg(L.nn + 2, 0);
      for (int h = 0; h < L.k; ++h)
        for (int v = lvl[h]; v < lvl[h + 1]; ++v) {
          const int2 c = P.long_code[L.code_base + v - 2];
          if (c.x == (int)kBotCode && c.y == (int)kBotCode) return bad(at + "node with no path to top");
          for (int ch : {c.x, c.y}) {
            const bool term = ch == (int)kTopCode || ch == (int)kBotCode;
            const bool in_next = h + 1 < L.k && ch >= lvl[h + 1] && ch < lvl[h + 2];
            if (h + 1 == L.k ? !term : !(ch == (int)kBotCode || in_next)) return bad(at + "child outside the next level");
            if (ch >= 2) indeg[ch]++;
          }
        }
      for (int v = 2; v < L.nn + 2; ++v) {
        const int32_t b0 = P.long_in_ptr[L.code_base + v - 2], b1 = P.long_in_ptr[L.code_base + v - 1];
        if (b1 - b0 != indeg[v] || (v > 2 && indeg[v] == 0)) return bad(at + "in-arc list size wrong");
        int32_t prev = -1;
        for (int32_t i = b0; i < b1; ++i) {
          const int32_t e = P.long_in[i], par = e >> 1;
          if (e <= prev || par < 2 || par >= v) return bad(at + "in-arc list not ascending");
          const int2 c = P.long_code[L.code_base + par - 2];
          if ((e & 1 ? c.y : c.x) != v) return bad(at + "in-arc is not an arc");
          prev = e;
        }
      }
      lslot += tslots;
      code_base += L.nn;
      lvl_base += L.k + 1;
      cost_base += L.nn + 2;
    }
    if (lslot != NS || cost_base != P.long_cost_size || code_base != P.sizes.num_long_nodes)
      return bad("long BDDs do not cover the arrays");
    // the order list: a permutation, the narrow BDDs (levels within a warp) first
    if (P.long_order.size() != P.longs.size() || P.num_long_narrow < 0 ||
        P.num_long_narrow > (int32_t)P.longs.size())
      return bad("long BDD order malformed");
    if (P.long_lanes < 0 || P.long_lanes > kWarp || (P.long_lanes & (P.long_lanes - 1)) != 0)
      return bad("lanes per narrow long BDD not a power of two up to 32");
    std::vector<char> listed(P.longs.size(), 0);
    for (size_t i = 0; i < P.long_order.size(); ++i) {
      const int32_t b = P.long_order[i];
      if (b < 0 || b >= (int32_t)P.longs.size() || listed[b]++) return bad("long BDD order not a permutation");
      if ((P.longs[b].maxw <= kWarp) != ((int32_t)i < P.num_long_narrow))
        return bad("long BDD order: narrow and wide BDDs mixed");
    }
  }
  if (real_slots != NL || real_nodes != P.sizes.num_nodes) return bad("slot or node count mismatch");
  // variables: CSR and ELL columns point back at their own slots, rows ascending
  if ((int64_t)P.var_ptr.size() != (int64_t)n + 1 || P.var_ptr[0] != 0 || P.var_ptr[n] != NL)
    return bad("variable pointers malformed");
  size_t next_wide = 0;
  for (int32_t i = 0; i < n; ++i) {
    if (P.var_ptr[i + 1] < P.var_ptr[i]) return bad("variable pointers not monotone");
    int prev_row = -1;
    for (int32_t k = P.var_ptr[i]; k < P.var_ptr[i + 1]; ++k) {
      const int32_t q = P.var_slots[k];
      if (q < 0 || q >= NS || P.slot_var[q] != i) return bad("variable " + std::to_string(i) + ": slot list wrong");
      if (P.slot_row[q] <= prev_row) return bad("variable " + std::to_string(i) + ": rows not ascending");
      prev_row = P.slot_row[q];
    }
    const int d = P.var_ptr[i + 1] - P.var_ptr[i];
    for (int r = 0; r < kEll; ++r) {
      int32_t e = P.var_ell[(size_t)r * n + i];
      if (d > kEll && r == kEll - 1) {
        if (e > -2) return bad("variable " + std::to_string(i) + ": ELL overflow mark missing");
        e = -2 - e;
      }
      const int32_t want = r < d ? P.var_slots[P.var_ptr[i] + r] : -1;
      if (e != want) return bad("variable " + std::to_string(i) + ": ELL column disagrees with the slot list");
    }
    if (d > kWide) {
      if (next_wide >= P.wide_vars.size() || P.wide_vars[next_wide] != i)
        return bad("variable " + std::to_string(i) + ": missing from the wide-variable list");
      ++next_wide;
    }
  }
  if (next_wide != P.wide_vars.size()) return bad("wide-variable list lists a narrow variable");
  // launch groups cover the tiles in order
  int32_t t0 = 0;
  for (const LaunchGroup& g : P.groups) {
    if (g.tile0 != t0 || g.tile1 <= g.tile0 || g.stream < 0 || g.stream >= kStreams) return bad("launch groups malformed");
    for (int32_t t = g.tile0; t < g.tile1; ++t) {
      const Tile& tl = P.tiles[t];
      if ((size_t)g.region_bytes < sweep_smem_bytes(tl.nmax, tl.nhops, 1, tl.ring) ||
          (size_t)g.region_bwd1 < sweep_smem_bytes_bwd(tl.nmax, tl.nhops, 1) ||
          g.meta_bytes < (tl.nmax - 2) * kWarp * 2)
        return bad("launch group " + std::to_string(t0) + ": shared memory smaller than a tile needs");
    }
    t0 = g.tile1;
  }
  if (t0 != T) return bad("launch groups do not cover the tiles");
  // bound chunks: per instance its rows, then its variables, in order
  const int ni = P.sizes.num_inst;
  for (int k = 0; k < ni; ++k) {
    int64_t rows_at = P.inst_row_ptr[k], vars_at = P.inst_var_ptr[k];
    for (int32_t c = P.inst_chunk_ptr[k]; c < P.inst_chunk_ptr[k + 1]; ++c) {
      const int32_t* ch = &P.lb_chunks[(size_t)c * 4];
      if (ch[0] != k || ch[3] <= ch[2]) return bad("bound chunk malformed");
      int64_t& at = ch[1] == 0 ? rows_at : vars_at;
      if (ch[2] != at) return bad("bound chunks leave a gap");
      at = ch[3];
    }
    if (rows_at != P.inst_row_ptr[k + 1] || vars_at != P.inst_var_ptr[k + 1]) return bad("bound chunks do not cover an instance");
  }
  return DG_OK;
}

}  // namespace dg
