// Host check of the one-launch step planner (lbpf_plan.h), built by tests/test_one_launch_plan.py.
//
// Usage: plan_check by lag batch_order  nx ny nz zchunk  [nx ny nz zchunk ...]
// Builds the work items of each simulation as the library does (batch_order = 1: sorted by
// descending z-chunk length, as for a batch), plans the one-launch step and checks, against
// a brute-force recomputation from the kernels' own index ranges:
//   - every item appears exactly once as a phase-field ticket and once as a U/theta ticket;
//   - each U/theta tile's dependency list is exactly the set of phase-field tiles of its
//     simulation whose phi^{n+1} writes meet the region its ring reads;
//   - every one of those phase-field tickets precedes the U/theta ticket (so no block waits
//     for a ticket that has not been taken, and every wait ends).
// Prints "ok" and exits 0, or prints the first violation and exits 1.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <set>
#include <vector>

#include "../paper_1602_07483_gb300/csrc/lbpf_plan.h"

using lbpf::TileGeom;
using lbpf::WorkItem;

namespace {

struct Box {
  int x0, x1, y0, y1, z0, z1;  // inclusive bounds
  bool meets(const Box& o) const {
    return x0 <= o.x1 && o.x0 <= x1 && y0 <= o.y1 && o.y0 <= y1 && z0 <= o.z1 && o.z0 <= z1;
  }
};

int clampi(int v, int lo, int hi) { return std::min(std::max(v, lo), hi); }

// Nodes whose phi^{n+1} the phase-field tile writes: lanes 1..30 of the block row
// (x = x0 - 1 + lane), rows 1..by-2 (one row for one-row blocks), planes [z0, z1).
Box written(const WorkItem& w, const TileGeom& g, int by) {
  const int ty = by == 1 ? 1 : by - 2;
  return Box{w.x0, std::min(w.x0 + 29, g.nx - 1), w.y0, std::min(w.y0 + ty - 1, g.ny - 1), w.z0, w.z1 - 1};
}

// Nodes whose phi^{n+1} the U/theta tile's ring reads: 34 columns from x0 - 2, by + 2 rows
// from y0 - 2 (one row for one-row blocks), planes zlo - 1 .. zhi + 1 with
// zlo = max(z0 - 1, 0) and zhi = min(z1, nz - 1); every coordinate clamped to the grid.
Box ring_read(const WorkItem& w, const TileGeom& g, int by) {
  const int rows = by == 1 ? 1 : by + 2;
  const int zlo = std::max(w.z0 - 1, 0), zhi = std::min(w.z1, g.nz - 1);
  return Box{clampi(w.x0 - 2, 0, g.nx - 1), clampi(w.x0 + 31, 0, g.nx - 1),
             clampi(w.y0 - 2, 0, g.ny - 1), clampi(w.y0 - 2 + rows - 1, 0, g.ny - 1),
             clampi(zlo - 1, 0, g.nz - 1),  clampi(zhi + 1, 0, g.nz - 1)};
}

int fail(const char* what, int j) {
  std::printf("violation: %s (item %d)\n", what, j);
  return 1;
}

}  // namespace

int main(int argc, char** argv) {
  if (argc < 8 || (argc - 4) % 4 != 0) {
    std::printf("usage: plan_check by lag batch_order nx ny nz zchunk [...]\n");
    return 2;
  }
  const int by = std::atoi(argv[1]), lag = std::atoi(argv[2]), batch_order = std::atoi(argv[3]);
  std::vector<TileGeom> geo;
  std::vector<WorkItem> items;
  for (int a = 4; a < argc; a += 4) {
    const TileGeom g{std::atoi(argv[a]), std::atoi(argv[a + 1]), std::atoi(argv[a + 2]), std::atoi(argv[a + 3])};
    lbpf::build_items((int)geo.size(), g.nx, g.ny, g.nz, by, g.zchunk, items);
    geo.push_back(g);
  }
  if (batch_order)
    std::stable_sort(items.begin(), items.end(),
                     [](const WorkItem& a, const WorkItem& c) { return (a.z1 - a.z0) > (c.z1 - c.z0); });
  std::vector<int> order, dep_off, dep;
  if (!lbpf::plan_one_launch(items, geo, by, lag, order, dep_off, dep)) return fail("planner refused the tiling", -1);
  const int n = (int)items.size();
  if ((int)order.size() != 2 * n) return fail("ticket count is not twice the item count", -1);
  std::vector<int> phi_pos(n, -1), uth_pos(n, -1);
  for (int t = 0; t < 2 * n; ++t) {
    const int w = order[t];
    const int j = w >= 0 ? w : ~w;
    if (j < 0 || j >= n) return fail("ticket names no item", j);
    int& pos = w >= 0 ? phi_pos[j] : uth_pos[j];
    if (pos >= 0) return fail("item appears twice in one phase", j);
    pos = t;
  }
  for (int j = 0; j < n; ++j) {
    const WorkItem& w = items[j];
    const TileGeom& g = geo[w.sim];
    const Box need = ring_read(w, g, by);
    std::set<int> expect;
    for (int p = 0; p < n; ++p)
      if (items[p].sim == w.sim && written(items[p], g, by).meets(need)) expect.insert(p);
    const std::set<int> got(dep.begin() + dep_off[j], dep.begin() + dep_off[j + 1]);
    if ((int)got.size() != dep_off[j + 1] - dep_off[j]) return fail("duplicate dependency", j);
    if (got != expect) return fail("dependency list differs from the ring's region", j);
    for (int p : got)
      if (phi_pos[p] >= uth_pos[j]) return fail("a dependency's ticket does not precede the U/theta ticket", j);
  }
  std::printf("ok %d items %zu deps\n", n, dep.size());
  return 0;
}
