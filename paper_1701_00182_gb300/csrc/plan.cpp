// Planner: the 2D planar bisection cluster tree of one n x n plane
// (Section 3.1: planes are clustered by binary space partitioning of the 2D
// plane; Section 2.1.1: cluster tree and weak admissibility).
//
// Split rule: halve the longer side of the rectangle, the x side when both
// sides are equal, until a cluster holds `leaf` points.  Leaves list their
// points in lexicographic order (x fastest), so every cluster is a contiguous
// range of the permuted index.  For every node the grid edges crossing its
// bisection are enumerated along the cut: they are the exact rank-one terms of
// the off-diagonal blocks of the 5-point in-plane operator.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "acr_internal.h"

namespace acr {

int plan_geometry(int n, int leaf, Geometry& g) {
  if (n < 2 || n > 1024 || (n & (n - 1))) return 1;
  const int m = n * n;
  if (leaf < 4 || leaf > 128 || m % leaf) return 1;
  int nleaf = m / leaf;
  if (nleaf & (nleaf - 1)) return 1;
  int L = 0;
  while ((1 << L) < nleaf) ++L;
  if (L >= MAXL) return 1;
  g.n = n; g.m = m; g.leaf = leaf; g.L = L;
  using Rect = std::array<int, 4>;  // x0, x1, y0, y1
  std::vector<std::vector<Rect>> rects(L + 1);
  rects[0].push_back({0, n, 0, n});
  for (int l = 0; l < L; ++l) {
    for (const Rect& r : rects[l]) {
      int w = r[1] - r[0], h = r[3] - r[2];
      if (w >= h) {
        int xm = r[0] + w / 2;
        rects[l + 1].push_back({r[0], xm, r[2], r[3]});
        rects[l + 1].push_back({xm, r[1], r[2], r[3]});
      } else {
        int ym = r[2] + h / 2;
        rects[l + 1].push_back({r[0], r[1], r[2], ym});
        rects[l + 1].push_back({r[0], r[1], ym, r[3]});
      }
    }
  }
  g.perm.clear();
  g.perm.reserve(m);
  for (const Rect& r : rects[L]) {
    if ((r[1] - r[0]) * (r[3] - r[2]) != leaf) return 1;
    for (int y = r[2]; y < r[3]; ++y)
      for (int x = r[0]; x < r[1]; ++x) g.perm.push_back(x + n * y);
  }
  std::vector<int> pos(m);
  for (int p = 0; p < m; ++p) pos[g.perm[p]] = p;
  g.ncut.assign(L, 0);
  g.cutp.assign(L, {});
  g.cutq.assign(L, {});
  for (int l = 0; l < L; ++l) {
    int nc = -1;
    for (size_t t = 0; t < rects[l].size(); ++t) {
      const Rect& r = rects[l][t];
      const Rect& a = rects[l + 1][2 * t];
      std::vector<int> cp, cq;
      if (a[1] < r[1]) {
        for (int y = r[2]; y < r[3]; ++y) {
          cp.push_back(pos[(a[1] - 1) + n * y]);
          cq.push_back(pos[a[1] + n * y]);
        }
      } else {
        for (int x = r[0]; x < r[1]; ++x) {
          cp.push_back(pos[x + n * (a[3] - 1)]);
          cq.push_back(pos[x + n * a[3]]);
        }
      }
      if (nc < 0) nc = (int)cp.size();
      if ((int)cp.size() != nc) return 1;
      g.cutp[l].insert(g.cutp[l].end(), cp.begin(), cp.end());
      g.cutq[l].insert(g.cutq[l].end(), cq.begin(), cq.end());
    }
    g.ncut[l] = nc;
  }
  return 0;
}

// Block cluster tree of one plane (Section 2.1: index set, cluster tree,
// block cluster tree, admissibility condition).  Clusters are the rectangles
// of the bisection tree above; a cluster holds the grid nodes x0 <= i < x1,
// y0 <= j < y1, whose convex hull is the rectangle with corners (x0, y0) and
// (x1 - 1, y1 - 1) in grid steps.  Standard admissibility: the pair (t, s) of
// one level is stored low rank when min(diam t, diam s) <= eta dist(t, s);
// both sides scale with the grid step, so the test is taken in grid steps and
// squared (exact integers on the left) -- a cluster is never admissible with
// itself.  An inadmissible pair is split into the four pairs of its children
// (row child first, then column child); pairs of leaves stay dense.  eta < 0:
// weak admissibility (siblings low rank, only diagonal pairs recurse).
int plan_blocks(int n, int leaf, double eta, std::vector<std::array<int, 4>>& out) {
  out.clear();
  if (!std::isfinite(eta)) return 1;
  Geometry g;
  if (plan_geometry(n, leaf, g)) return 1;
  const int L = g.L;
  using Rect = std::array<int, 4>;
  std::vector<std::vector<Rect>> rects(L + 1);
  rects[0].push_back({0, n, 0, n});
  for (int l = 0; l < L; ++l)
    for (const Rect& r : rects[l]) {
      const int w = r[1] - r[0], h = r[3] - r[2];
      if (w >= h) {
        const int xm = r[0] + w / 2;
        rects[l + 1].push_back({r[0], xm, r[2], r[3]});
        rects[l + 1].push_back({xm, r[1], r[2], r[3]});
      } else {
        const int ym = r[2] + h / 2;
        rects[l + 1].push_back({r[0], r[1], r[2], ym});
        rects[l + 1].push_back({r[0], r[1], ym, r[3]});
      }
    }
  auto diam2 = [](const Rect& r) -> long {
    const long a = r[1] - 1 - r[0], b = r[3] - 1 - r[2];
    return a * a + b * b;
  };
  auto dist2 = [](const Rect& a, const Rect& b) -> long {
    const long dx = std::max({0, b[0] - (a[1] - 1), a[0] - (b[1] - 1)});
    const long dy = std::max({0, b[2] - (a[3] - 1), a[2] - (b[3] - 1)});
    return dx * dx + dy * dy;
  };
  const bool weak = eta < 0;
  // explicit stack in the order of the recursion: the children pushed in reverse
  std::vector<std::array<int, 3>> stack{{0, 0, 0}};
  while (!stack.empty()) {
    const auto [l, t, s] = stack.back();
    stack.pop_back();
    bool lowrank;
    if (weak) {
      lowrank = t != s;
    } else {
      const long d2 = dist2(rects[l][t], rects[l][s]);
      lowrank = d2 > 0 && (double)std::min(diam2(rects[l][t]), diam2(rects[l][s])) <= eta * eta * (double)d2;
    }
    if (lowrank || l == L) {
      out.push_back({l, t, s, lowrank ? 1 : 0});
      continue;
    }
    for (int a = 1; a >= 0; --a)
      for (int b = 1; b >= 0; --b) stack.push_back({l + 1, 2 * t + a, 2 * s + b});
  }
  return 0;
}

}  // namespace acr
