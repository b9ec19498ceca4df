// Bandwidth-reducing node order for the banded direct solve (host code, band_order.cpp).
#pragma once

#include <stdint.h>

namespace vms {

// Order of a node graph given as CSR adjacency (start[nodes + 1], adj; no self loops):
// perm[a] = position of node a in the order of smallest bandwidth among the graph's own numbering
// and two reverse Cuthill-McKee orders. Returns that bandwidth (the largest |perm[a] - perm[b]|
// over the edges).
int band_order_host(int64_t nodes, const int32_t* start, const int32_t* adj, int32_t* perm);

}  // namespace vms
