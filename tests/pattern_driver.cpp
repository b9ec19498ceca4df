// Test driver for the host CSR-pattern builder of the library (row a0): reads a mesh from stdin and
// prints what build_pattern produced, one labelled line per array. Compiled and run by
// tests/test_pattern_host.py; not part of the library.
//
// Input: n_nodes n_elems npe n_dir, then n_elems * npe node indices, then n_dir constrained dofs.
#include <cstdio>
#include <string>
#include <vector>

#include "../paper_0809_4802_gb300/csrc/vms_internal.h"

template <typename T>
static void put(const char* name, const std::vector<T>& v) {
  std::printf("%s %zu", name, v.size());
  for (const T& x : v) std::printf(" %lld", (long long)x);
  std::printf("\n");
}

int main() {
  long long nn = 0, ne = 0, nd = 0;
  int npe = 0;
  if (std::scanf("%lld %lld %d %lld", &nn, &ne, &npe, &nd) != 4) return 2;
  std::vector<int32_t> conn((size_t)(ne * npe));
  for (auto& c : conn)
    if (std::scanf("%d", &c) != 1) return 2;
  std::vector<int64_t> dir((size_t)nd);
  for (auto& d : dir) {
    long long x = 0;
    if (std::scanf("%lld", &x) != 1) return 2;
    d = x;
  }
  vms::HostPattern P;
  const std::string err =
      vms::build_pattern(nn, ne, conn.data(), nd, nd ? dir.data() : nullptr, P, npe);
  if (!err.empty()) {
    std::printf("error %s\n", err.c_str());
    return 0;
  }
  put("rowptr", P.rowptr);
  put("colidx", P.colidx);
  put("blk", P.blk);
  put("rowlen", P.rowlen);
  put("colour", P.colour);
  put("colour_order", P.colour_order);
  put("colour_start", P.colour_start);
  put("diag_pos", P.diag_pos);
  put("dir_mask", P.dir_mask);
  std::printf("n_colours %d\n", P.n_colours);
  return 0;
}
