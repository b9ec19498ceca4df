// Test driver for the host-side plan of the FP64 tangent's factorised sums: prints, for the 2- and
// 3-point Gauss rules, the one-dimensional basis rows and the plan ts_tables builds. Compiled and
// run by tests/test_ts_plan_host.py; not part of the library.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <vector>

namespace vms {
bool ts_tables(int n1, const double* x, std::vector<double>& basis, std::vector<uint32_t>& plan);
}

int main() {
  for (int n1 = 2; n1 <= 3; ++n1) {
    std::vector<double> x(n1);
    if (n1 == 2) {
      x[0] = -1.0 / std::sqrt(3.0);
      x[1] = -x[0];
    } else {
      x[0] = -std::sqrt(0.6);
      x[1] = 0.0;
      x[2] = std::sqrt(0.6);
    }
    std::vector<double> b;
    std::vector<uint32_t> p;
    const bool ok = vms::ts_tables(n1, x.data(), b, p);
    std::printf("rule %d %d %zu %zu\n", n1, ok ? 1 : 0, b.size(), p.size());
    for (double v : b) std::printf("%.17g\n", v);
    for (uint32_t v : p) std::printf("%u\n", v);
  }
  return 0;
}
