// Bandwidth-reducing node order for the banded direct solve (host code).
//
// Three candidate orders of a node graph, the one of smallest bandwidth kept: the graph's own
// numbering, and two reverse Cuthill-McKee orders (Cuthill and McKee 1969; reversed as George and
// Liu describe). Cuthill-McKee numbers the nodes breadth first, queueing the unnumbered neighbours
// of each node in order of increasing degree; the reverse of that numbering has the same bandwidth
// and less fill. One start is a pseudo-peripheral node (breadth-first searches repeated from a node
// of least degree in the last level while the number of levels grows), the other the whole last
// level of that node's level structure: on an elongated lattice the corner's levels are shells of
// up to three faces, while the last level is an end face and the levels from it are cross-sections.
// Further connected parts start from a node of least degree each.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <vector>

#include "band_order.h"

namespace vms {

int band_order_host(int64_t nodes, const int32_t* start, const int32_t* adj, int32_t* perm_out) {
  if (nodes <= 0) return 0;
  auto deg = [&](int64_t a) { return start[a + 1] - start[a]; };
  auto bandwidth = [&](const std::vector<int32_t>& perm) {
    int bw = 0;
    for (int64_t a = 0; a < nodes; ++a)
      for (int32_t t = start[a]; t < start[a + 1]; ++t) bw = std::max(bw, std::abs(perm[a] - perm[adj[t]]));
    return bw;
  };
  // breadth-first levels from a set of nodes: the depth; the last level's nodes into lastv and the
  // visited nodes in visiting order into `queue`
  std::vector<int32_t> level(nodes), queue;
  auto levels = [&](const std::vector<int32_t>& src, std::vector<int32_t>& lastv) {
    std::fill(level.begin(), level.end(), -1);
    queue.assign(src.begin(), src.end());
    for (int32_t a : src) level[a] = 0;
    int depth = 0;
    for (size_t h = 0; h < queue.size(); ++h) {
      const int32_t a = queue[h];
      depth = level[a];
      for (int32_t t = start[a]; t < start[a + 1]; ++t)
        if (level[adj[t]] < 0) {
          level[adj[t]] = level[a] + 1;
          queue.push_back(adj[t]);
        }
    }
    lastv.clear();
    for (int32_t a : queue)
      if (level[a] == depth) lastv.push_back(a);
    return depth;
  };
  // reverse Cuthill-McKee numbering from a set of start nodes; returns perm (node -> position)
  std::vector<char> placed(nodes);
  std::vector<int32_t> order, nb;
  auto rcm = [&](std::vector<int32_t> src) {
    std::fill(placed.begin(), placed.end(), 0);
    order.clear();
    for (int64_t next = 0;;) {
      std::stable_sort(src.begin(), src.end(), [&](int32_t x, int32_t y) { return deg(x) < deg(y); });
      const size_t h0 = order.size();
      for (int32_t a : src) {
        placed[a] = 1;
        order.push_back(a);
      }
      for (size_t h = h0; h < order.size(); ++h) {
        const int32_t a = order[h];
        nb.clear();
        for (int32_t t = start[a]; t < start[a + 1]; ++t)
          if (!placed[adj[t]]) {
            placed[adj[t]] = 1;
            nb.push_back(adj[t]);
          }
        std::stable_sort(nb.begin(), nb.end(), [&](int32_t x, int32_t y) { return deg(x) < deg(y); });
        for (int32_t x : nb) order.push_back(x);
      }
      if ((int64_t)order.size() == nodes) break;
      while (placed[next]) ++next;
      int32_t r = (int32_t)next;
      for (int64_t a = next; a < nodes; ++a)
        if (!placed[a] && deg(a) < deg(r)) r = (int32_t)a;
      src.assign(1, r);
    }
    std::vector<int32_t> perm(nodes);
    for (int64_t k = 0; k < nodes; ++k) perm[order[k]] = (int32_t)(nodes - 1 - k);
    return perm;
  };
  std::vector<int32_t> best(nodes);
  for (int64_t a = 0; a < nodes; ++a) best[a] = (int32_t)a;
  int bw = bandwidth(best);
  // a pseudo-peripheral node r of the part holding node 0, and the last level of its levels
  int32_t r = 0;
  std::vector<int32_t> last, lc;
  levels(std::vector<int32_t>(1, 0), last);
  for (int32_t a : queue)
    if (deg(a) < deg(r)) r = a;
  int depth = levels(std::vector<int32_t>(1, r), last);
  for (int it = 0; it < 8; ++it) {
    int32_t c = last[0];
    for (int32_t a : last)
      if (deg(a) < deg(c)) c = a;
    const int dc = levels(std::vector<int32_t>(1, c), lc);
    if (dc <= depth) break;
    r = c;
    depth = dc;
    last.swap(lc);
  }
  for (int variant = 0; variant < 2; ++variant) {
    std::vector<int32_t> perm = rcm(variant == 0 ? std::vector<int32_t>(1, r) : last);
    const int b = bandwidth(perm);
    if (b < bw) {
      bw = b;
      best.swap(perm);
    }
  }
  std::copy(best.begin(), best.end(), perm_out);
  return bw;
}

}  // namespace vms
