// Nested dissection of a general graph with vertex coordinates (Sec. 3.1, Alg. 1), on the host:
// the ordering of a finite-element-like graph, for callers whose matrix is not a regular grid.
// (The factorization kernels of this library take regular grids, spalu_nd_build_grid.)
//
// Each part is cut by the separator walk of Sec. 3.1: the centre c is the vertex nearest the
// coordinate median; the direction d is +x when the part's bounding box is narrower than tall,
// else +y; from c the walk moves to the unvisited neighbour u maximising
//   D(u, v, c, d) = <u - v, d> / |u - v| + theta <u - c, d> / |u - c|,   theta = 0.1
// (Eq. (degreebias)), first along +d and then along -d.  Conventions where the paper is
// silent: a walk also ends at the first vertex on the part's boundary (a neighbour outside
// the part, or the domain's boundary); D values within 1e-12 count as equal (first neighbour
// in adjacency order wins) and D <= 1e-12 ends the walk; the remaining vertices' connected
// components go to the side of the separator where their lowest-numbered vertex lies; a part
// with one side empty, or with at most leaf_size vertices, is a leaf.  Order I: leaves (each
// in increasing vertex id) in depth-first order, then the separators by level L..1, depth
// first within a level, each in walk order.
#include <algorithm>
#include <cmath>
#include <map>
#include <vector>

#include "spalu_internal.h"

namespace {

constexpr double ND_THETA = 0.1;
constexpr double ND_TOL = 1e-12;

struct GraphND {
  int n = 0;
  const int* rowptr = nullptr;
  const int* colind = nullptr;
  const double* xy = nullptr;
  std::vector<char> dom_bd;        // domain boundary flags
  int leaf = 1;
  std::vector<int> level;
  std::vector<std::vector<int>> leaves;
  std::map<int, std::vector<std::vector<int>>> seps;
  std::vector<char> inpart, insep, bd, seen, comp;

  double x(int v) const { return xy[2 * (size_t)v]; }
  double y(int v) const { return xy[2 * (size_t)v + 1]; }

  // walk from c along (dx, dy); the vertices of `taken` (the other walk) are not revisited
  void walk(int c, double dx, double dy, const std::vector<int>& taken, std::vector<int>& path) {
    int v = c;
    std::vector<int> visited{c};
    seen[c] = 1;
    for (int u : taken) { seen[u] = 1; visited.push_back(u); }
    for (;;) {
      int bestu = -1;
      double best = 0.0;
      for (int p = rowptr[v]; p < rowptr[v + 1]; ++p) {
        const int u = colind[p];
        if (u == v || !inpart[u] || seen[u]) continue;
        const double ax = x(u) - x(v), ay = y(u) - y(v);
        const double bx = x(u) - x(c), by = y(u) - y(c);
        const double na = std::sqrt(ax * ax + ay * ay);
        const double nb = std::sqrt(bx * bx + by * by);
        const double t1 = (ax * dx + ay * dy) / na;
        const double t2 = nb == 0.0 ? 0.0 : (bx * dx + by * dy) / nb;
        const double val = t1 + ND_THETA * t2;
        if (bestu < 0 || val > best + ND_TOL) {
          best = val;
          bestu = u;
        }
      }
      if (bestu < 0 || best <= ND_TOL) break;
      path.push_back(bestu);
      seen[bestu] = 1;
      visited.push_back(bestu);
      if (bd[bestu]) break;
      v = bestu;
    }
    for (int u : visited) seen[u] = 0;
  }

  void rec(std::vector<int> part, int l) {
    std::sort(part.begin(), part.end());
    if ((int)part.size() <= leaf) {
      leaves.push_back(part);
      return;
    }
    for (int v : part) inpart[v] = 1;
    // centre: the vertex nearest the coordinate median (first within the tolerance)
    std::vector<double> xs, ys;
    xs.reserve(part.size());
    ys.reserve(part.size());
    double xmin = x(part[0]), xmax = xmin, ymin = y(part[0]), ymax = ymin;
    for (int v : part) {
      xs.push_back(x(v));
      ys.push_back(y(v));
      xmin = std::min(xmin, x(v)); xmax = std::max(xmax, x(v));
      ymin = std::min(ymin, y(v)); ymax = std::max(ymax, y(v));
    }
    auto median = [](std::vector<double>& a) {
      const size_t m = a.size() / 2;
      std::nth_element(a.begin(), a.begin() + m, a.end());
      const double hi = a[m];
      if (a.size() % 2) return hi;
      const double lo = *std::max_element(a.begin(), a.begin() + m);
      return (lo + hi) / 2.0;
    };
    const double mx = median(xs), my = median(ys);
    std::vector<double> d2(part.size());
    double dmin = 0.0;
    for (size_t i = 0; i < part.size(); ++i) {
      const double ex = x(part[i]) - mx, ey = y(part[i]) - my;
      d2[i] = ex * ex + ey * ey;
      if (i == 0 || d2[i] < dmin) dmin = d2[i];
    }
    int c = part[0];
    for (size_t i = 0; i < part.size(); ++i)
      if (d2[i] <= dmin + ND_TOL * std::max(dmin, 1.0)) { c = part[i]; break; }
    const bool alongx = (xmax - xmin) < (ymax - ymin);
    const double dx = alongx ? 1.0 : 0.0, dy = alongx ? 0.0 : 1.0;
    for (int v : part) {
      bool b = dom_bd[v] != 0;
      for (int p = rowptr[v]; p < rowptr[v + 1] && !b; ++p)
        if (colind[p] != v && !inpart[colind[p]]) b = true;
      bd[v] = b ? 1 : 0;
    }
    std::vector<int> fwd, bwd;
    walk(c, dx, dy, {}, fwd);
    walk(c, -dx, -dy, fwd, bwd);
    std::vector<int> sep(bwd.rbegin(), bwd.rend());
    sep.push_back(c);
    sep.insert(sep.end(), fwd.begin(), fwd.end());
    for (int v : sep) insep[v] = 1;
    // sides: connected components of the rest, by the side of their lowest vertex
    std::vector<int> side[2];
    const double cacross = alongx ? y(c) : x(c);
    for (int v : part) {
      if (insep[v] || comp[v]) continue;
      std::vector<int> members, stack{v};
      comp[v] = 1;
      while (!stack.empty()) {
        const int t = stack.back();
        stack.pop_back();
        members.push_back(t);
        for (int p = rowptr[t]; p < rowptr[t + 1]; ++p) {
          const int u = colind[p];
          if (inpart[u] && !insep[u] && !comp[u]) {
            comp[u] = 1;
            stack.push_back(u);
          }
        }
      }
      const int first = *std::min_element(members.begin(), members.end());
      const double a = alongx ? y(first) : x(first);
      side[a < cacross ? 0 : 1].insert(side[a < cacross ? 0 : 1].end(), members.begin(), members.end());
    }
    for (int v : part) { inpart[v] = 0; comp[v] = 0; bd[v] = 0; }
    for (int v : sep) insep[v] = 0;
    if (side[0].empty() || side[1].empty()) {
      leaves.push_back(part);
      return;
    }
    for (int v : sep) level[v] = l;
    seps[l].push_back(sep);
    rec(std::move(side[0]), l + 1);
    rec(std::move(side[1]), l + 1);
  }
};

}  // namespace

extern "C" spalu_status spalu_nd_order_csr(int n, const int* rowptr, const int* colind, const double* xy,
                                           const unsigned char* boundary, int leaf_size, int* perm, int* level) {
  if (n < 0 || (n > 0 && (!rowptr || !colind || !xy || !perm)) || leaf_size < 1) return SPALU_ERR_ARG;
  if (n == 0) return SPALU_OK;
  if (rowptr[0] != 0) return SPALU_ERR_ARG;
  for (int v = 0; v < n; ++v) {
    if (rowptr[v + 1] < rowptr[v]) return SPALU_ERR_ARG;
    if (!std::isfinite(xy[2 * (size_t)v]) || !std::isfinite(xy[2 * (size_t)v + 1])) return SPALU_ERR_ARG;
  }
  for (int p = 0; p < rowptr[n]; ++p)
    if (colind[p] < 0 || colind[p] >= n) return SPALU_ERR_ARG;
  GraphND g;
  g.n = n; g.rowptr = rowptr; g.colind = colind; g.xy = xy; g.leaf = leaf_size;
  g.level.assign(n, 0);
  g.inpart.assign(n, 0); g.insep.assign(n, 0); g.bd.assign(n, 0); g.seen.assign(n, 0); g.comp.assign(n, 0);
  g.dom_bd.assign(n, 0);
  if (boundary) {
    for (int v = 0; v < n; ++v) g.dom_bd[v] = boundary[v] ? 1 : 0;
  } else {
    int maxdeg = 0;
    std::vector<int> deg(n, 0);
    for (int v = 0; v < n; ++v) {
      for (int p = rowptr[v]; p < rowptr[v + 1]; ++p) deg[v] += colind[p] != v;
      maxdeg = std::max(maxdeg, deg[v]);
    }
    for (int v = 0; v < n; ++v) g.dom_bd[v] = deg[v] < maxdeg;
  }
  std::vector<int> all(n);
  for (int v = 0; v < n; ++v) all[v] = v;
  g.rec(std::move(all), 1);
  size_t k = 0;
  for (const auto& leaf : g.leaves)
    for (int v : leaf) perm[k++] = v;
  for (auto it = g.seps.rbegin(); it != g.seps.rend(); ++it)
    for (const auto& sep : it->second)
      for (int v : sep) perm[k++] = v;
  if (k != (size_t)n) return SPALU_ERR_ARG;       // a vertex listed twice in a walk (not a simple graph)
  if (level) std::copy(g.level.begin(), g.level.end(), level);
  return SPALU_OK;
}
