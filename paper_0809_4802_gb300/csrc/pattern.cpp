// Once-per-mesh host work: CSR pattern of the condensed coarse system, element -> CSR block map,
// element colouring and Dirichlet bookkeeping. The assembly operator of Section 5 (Eq.
// SchurUpdate) sums element matrices (32x32 for the hexahedron, 16x16 for the tetrahedron) over
// elements; this file fixes where each element's npe x npe node blocks of 4x4 values land, so the
// device scatter is a plain indexed add.
//
// Layout: node-major dofs 4*node+c. Row 4n+i holds, for every neighbour m of node n in increasing
// order, the four columns 4m..4m+3, so the 4x4 block (n,m) occupies four runs of four contiguous
// values: value index rowptr[4n] + i*rowlen[n] + 4*pos(n,m) + k for entry (4n+i, 4m+k).
#include <algorithm>
#include <cstring>
#include <string>
#include <vector>

#include "vms_internal.h"

namespace vms {

std::string build_pattern(int64_t n_nodes, int64_t n_elems, const int32_t* conn, int64_t n_dir,
                          const int64_t* dir_dof, HostPattern& out, int npe) {
  if (n_nodes <= 0 || n_elems <= 0) return "mesh must have nodes and elements";
  if (npe != 4 && npe != 8) return "elements must have 4 or 8 nodes";
  for (int64_t i = 0; i < n_elems * npe; ++i)
    if (conn[i] < 0 || conn[i] >= n_nodes) return "connectivity index out of range";
  for (int64_t e = 0; e < n_elems; ++e)
    for (int a = 0; a < npe; ++a)
      for (int b = a + 1; b < npe; ++b)
        if (conn[e * npe + a] == conn[e * npe + b]) return "element with a repeated node";

  // node -> element incidence (counting sort)
  std::vector<int64_t> nstart(n_nodes + 1, 0);
  for (int64_t i = 0; i < n_elems * npe; ++i) nstart[conn[i] + 1]++;
  for (int64_t n = 0; n < n_nodes; ++n) nstart[n + 1] += nstart[n];
  std::vector<int32_t> nelem(nstart[n_nodes]);
  {
    std::vector<int64_t> fill(nstart.begin(), nstart.end() - 1);
    for (int64_t e = 0; e < n_elems; ++e)
      for (int a = 0; a < npe; ++a) nelem[fill[conn[e * npe + a]]++] = (int32_t)e;
  }

  // sorted neighbour lists
  std::vector<int64_t> adj_start(n_nodes + 1, 0);
  std::vector<int32_t> adj;
  adj.reserve((size_t)n_nodes * 27);
  std::vector<int32_t> cand;
  cand.reserve(512);
  for (int64_t n = 0; n < n_nodes; ++n) {
    cand.clear();
    for (int64_t k = nstart[n]; k < nstart[n + 1]; ++k) {
      const int32_t* c = conn + (int64_t)nelem[k] * npe;
      cand.insert(cand.end(), c, c + npe);
    }
    std::sort(cand.begin(), cand.end());
    cand.erase(std::unique(cand.begin(), cand.end()), cand.end());
    adj.insert(adj.end(), cand.begin(), cand.end());
    adj_start[n + 1] = (int64_t)adj.size();
  }

  // rowptr / colidx
  int64_t nnz = 16 * (int64_t)adj.size();
  if (nnz >= (int64_t)INT32_MAX) return "matrix has 2^31 or more nonzeros (int32 indices)";
  out.rowptr.assign(4 * n_nodes + 1, 0);
  out.rowlen.assign(n_nodes, 0);
  out.colidx.resize(nnz);
  int64_t pos = 0;
  for (int64_t n = 0; n < n_nodes; ++n) {
    int64_t deg = adj_start[n + 1] - adj_start[n];
    out.rowlen[n] = (int32_t)(4 * deg);
    for (int i = 0; i < 4; ++i) {
      out.rowptr[4 * n + i] = (int32_t)pos;
      for (int64_t k = adj_start[n]; k < adj_start[n + 1]; ++k)
        for (int c = 0; c < 4; ++c) out.colidx[pos++] = 4 * adj[k] + c;
    }
  }
  out.rowptr[4 * n_nodes] = (int32_t)pos;

  auto find_pos = [&](int32_t n, int32_t m) -> int64_t {
    const int32_t* b = adj.data() + adj_start[n];
    const int32_t* e = adj.data() + adj_start[n + 1];
    const int32_t* it = std::lower_bound(b, e, m);
    return (int64_t)(it - b);
  };

  // element block map: npe x npe blocks per element
  const int nb = npe * npe;
  out.blk.resize((size_t)n_elems * nb);
  for (int64_t e = 0; e < n_elems; ++e) {
    const int32_t* c = conn + e * npe;
    for (int a = 0; a < npe; ++a)
      for (int b = 0; b < npe; ++b)
        out.blk[e * nb + a * npe + b] = out.rowptr[4 * c[a]] + (int32_t)(4 * find_pos(c[a], c[b]));
  }

  // greedy colouring: no two elements of one colour share a node (at most 128 colours)
  constexpr int MAXC = 128;
  out.colour.assign(n_elems, -1);
  int n_col = 0;
  for (int64_t e = 0; e < n_elems; ++e) {
    uint64_t used[MAXC / 64] = {0, 0};
    for (int a = 0; a < npe; ++a) {
      int32_t n = conn[e * npe + a];
      for (int64_t k = nstart[n]; k < nstart[n + 1]; ++k) {
        int32_t o = out.colour[nelem[k]];
        if (o >= 0) used[o >> 6] |= (1ull << (o & 63));
      }
    }
    int col = 0;
    while (col < MAXC && (used[col >> 6] >> (col & 63) & 1ull)) ++col;
    if (col >= MAXC) return "element colouring needs more than 128 colours";
    out.colour[e] = col;
    n_col = std::max(n_col, col + 1);
  }
  out.n_colours = n_col;
  out.colour_start.assign(n_col + 1, 0);
  for (int64_t e = 0; e < n_elems; ++e) out.colour_start[out.colour[e] + 1]++;
  for (int c = 0; c < n_col; ++c) out.colour_start[c + 1] += out.colour_start[c];
  out.colour_order.resize(n_elems);
  {
    std::vector<int32_t> fill(out.colour_start.begin(), out.colour_start.end() - 1);
    for (int64_t e = 0; e < n_elems; ++e) out.colour_order[fill[out.colour[e]]++] = (int32_t)e;
  }

  // Dirichlet bookkeeping
  std::vector<uint8_t> constrained(4 * n_nodes, 0);
  out.diag_pos.resize(n_dir);
  for (int64_t k = 0; k < n_dir; ++k) {
    int64_t d = dir_dof[k];
    if (d < 0 || d >= 4 * n_nodes) return "Dirichlet dof out of range";
    constrained[d] = 1;
    int32_t n = (int32_t)(d / 4);
    int c = (int)(d % 4);
    out.diag_pos[k] = (int64_t)out.rowptr[d] + 4 * find_pos(n, n) + c;
  }
  out.dir_mask.assign(n_elems, 0u);
  for (int64_t e = 0; e < n_elems; ++e) {
    uint32_t m = 0;
    for (int a = 0; a < npe; ++a)
      for (int c = 0; c < 4; ++c)
        if (constrained[4 * (int64_t)conn[e * npe + a] + c]) m |= 1u << (4 * a + c);
    out.dir_mask[e] = m;
  }
  return "";
}

}  // namespace vms
