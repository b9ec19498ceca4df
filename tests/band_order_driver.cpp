// Reads node graphs (CSR adjacency) from stdin and prints, for each, the bandwidth and the order
// band_order_host returns. Input per graph: nodes nnz, then nodes + 1 offsets, then nnz columns.
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../paper_0809_4802_gb300/csrc/band_order.h"

int main() {
  long long nodes = 0, nnz = 0;
  while (std::scanf("%lld %lld", &nodes, &nnz) == 2) {
    std::vector<int32_t> start(nodes + 1), adj(nnz), perm(nodes > 0 ? nodes : 1);
    for (auto& v : start)
      if (std::scanf("%d", &v) != 1) return 1;
    for (auto& v : adj)
      if (std::scanf("%d", &v) != 1) return 1;
    const int bw = vms::band_order_host(nodes, start.data(), adj.data(), perm.data());
    std::printf("%d", bw);
    for (long long a = 0; a < nodes; ++a) std::printf(" %d", perm[a]);
    std::printf("\n");
  }
  return 0;
}
