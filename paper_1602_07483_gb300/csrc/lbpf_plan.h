// lbpf_plan.h -- work decomposition of the step kernels (host code, plain C++).
//
// A step kernel block covers TILE_X interior columns and `by - 2` interior rows (one row
// for the one-row blocks of the 2D lattices) of the xy plane over a z-chunk of planes; a
// work item names one such tile.  This header also plans the one-launch step: the order
// in which the blocks of that launch take the phase-field and U/theta tiles, and which
// phase-field tiles each U/theta tile waits for.  It has no CUDA dependency, so the
// planner can be checked by a host program.
#pragma once

#include <algorithm>
#include <vector>

namespace lbpf {

constexpr int TILE_X = 30;  // interior columns per block row (block x = 32)

struct WorkItem {
  int sim;
  int x0, y0;  // first interior column of the tile
  int z0, z1;  // planes [z0, z1) written by this block
};

// Tiles of one simulation for blocks of `by` rows and z-chunks of `zchunk` planes, z-chunk
// major, then rows, then columns.
inline void build_items(int sim_index, int nx, int ny, int nz, int by, int zchunk, std::vector<WorkItem>& out) {
  const int ty = by == 1 ? 1 : by - 2;  // interior rows per block: one-row blocks (2D) have no y halo
  for (int z0 = 0; z0 < nz; z0 += zchunk)
    for (int y0 = 0; y0 < ny; y0 += ty)
      for (int x0 = 0; x0 < nx; x0 += TILE_X) out.push_back(WorkItem{sim_index, x0, y0, z0, std::min(nz, z0 + zchunk)});
}

struct TileGeom {
  int nx, ny, nz, zchunk;
};

// Ticket order and dependency lists of the one-launch step over `items` (tiles of TILE_X
// columns and ty rows, z-chunks of geo[sim].zchunk planes, as build_items makes them).  The
// U/theta tile of item j reads phi^{n+1} on columns [x0-2, x0+31], rows [y0-2, y0+by-1] and
// planes [z0-2, z1+1] (clamped to the grid): it depends on every phase-field tile that writes
// part of that box.  Phase-field tickets go by simulation, row tile, z-chunk, then column
// tile, so that the tiles a U/theta tile needs are close together in the order; each U/theta
// ticket follows the last of its phase-field tiles by `lag` phase-field tickets.  False if a
// tile of the box has no work item (a tiling that build_items did not make).
inline bool plan_one_launch(const std::vector<WorkItem>& items, const std::vector<TileGeom>& geo, int by, int lag,
                     std::vector<int>& order, std::vector<int>& dep_off, std::vector<int>& dep) {
  const int ty = by == 1 ? 1 : by - 2;
  const size_t ns = geo.size();
  std::vector<long long> base(ns + 1, 0);
  std::vector<int> nxt(ns), nyt(ns), nct(ns);
  for (size_t k = 0; k < ns; ++k) {
    nxt[k] = (geo[k].nx + TILE_X - 1) / TILE_X;
    nyt[k] = (geo[k].ny + ty - 1) / ty;
    nct[k] = (geo[k].nz + geo[k].zchunk - 1) / geo[k].zchunk;
    base[k + 1] = base[k] + (long long)nxt[k] * nyt[k] * nct[k];
  }
  auto cell = [&](int sim, int c, int r, int q) { return base[sim] + ((long long)r * nct[sim] + c) * nxt[sim] + q; };
  const int n = (int)items.size();
  std::vector<int> at((size_t)base[ns], -1);
  for (int j = 0; j < n; ++j) {
    const WorkItem& w = items[j];
    at[cell(w.sim, w.z0 / geo[w.sim].zchunk, w.y0 / ty, w.x0 / TILE_X)] = j;
  }
  // rank of each item's phase-field ticket: the cell order above
  std::vector<int> rank(n, -1), phi_order;
  phi_order.reserve(n);
  for (int a : at)
    if (a >= 0) {
      rank[a] = (int)phi_order.size();
      phi_order.push_back(a);
    }
  if ((int)phi_order.size() != n) return false;
  dep_off.assign(n + 1, 0);
  dep.clear();
  std::vector<std::vector<int>> after(n);
  for (int j = 0; j < n; ++j) {
    const WorkItem& w = items[j];
    const TileGeom& g = geo[w.sim];
    const int q0 = std::max(w.x0 - 2, 0) / TILE_X, q1 = std::min(w.x0 + 31, g.nx - 1) / TILE_X;
    const int ylo = std::max(w.y0 - 2, 0);
    const int r0 = ylo / ty, r1 = (by == 1 ? ylo : std::min(w.y0 + by - 1, g.ny - 1)) / ty;
    const int c0 = std::max(w.z0 - 2, 0) / g.zchunk, c1 = std::min(w.z1 + 1, g.nz - 1) / g.zchunk;
    int last = 0;
    for (int c = c0; c <= c1; ++c)
      for (int r = r0; r <= r1; ++r)
        for (int q = q0; q <= q1; ++q) {
          const int d = at[cell(w.sim, c, r, q)];
          if (d < 0) return false;
          dep.push_back(d);
          last = std::max(last, rank[d]);
        }
    dep_off[j + 1] = (int)dep.size();
    after[std::min(last + lag, n - 1)].push_back(j);
  }
  order.clear();
  order.reserve(2 * (size_t)n);
  for (int k = 0; k < n; ++k) {
    order.push_back(phi_order[k]);
    for (int j : after[k]) order.push_back(~j);
  }
  return true;
}

}  // namespace lbpf
