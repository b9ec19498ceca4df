// Host-side plan of the FP64 tangent's factorised sums (Section 4.2, Eq. NewtonUpdate2; the sums
// themselves are described in tangent_ts.cuh): the one-dimensional basis rows at the Gauss points
// and, for the six steps (three directions for the fields of the coarse blocks, then three for
// the fields of the couplings), the list of n1-term partial sums with their places in the warp's
// work area. Plain C++, built by the host compiler.
#include <algorithm>
#include <cstdint>
#include <utility>
#include <vector>

#include "ts_layout.h"

namespace vms {

bool ts_tables(int n1, const double* x, std::vector<double>& basis, std::vector<uint32_t>& plan);

bool ts_tables(int n1, const double* x, std::vector<double>& basis, std::vector<uint32_t>& plan) {
  const int nq = n1 * n1 * n1, ld = ts_ld(nq), fbase = TS_SUMS, total = TS_SUMS + TS_FIELDS * ld;
  auto phi = [](int b, double t) { return b ? 0.5 * (1.0 + t) : 0.5 * (1.0 - t); };
  basis.assign(4 * TS_BASIS_ROWS, 0.0);
  for (int i = 0; i < n1; ++i) {
    for (int sm = 0; sm < 3; ++sm)
      basis[4 * (TS_ROW_PSI + sm) + i] = phi(sm == 2, x[i]) * phi(sm >= 1, x[i]);
    for (int b = 0; b < 2; ++b) basis[4 * (TS_ROW_PHI + b) + i] = phi(b, x[i]);
    basis[4 * TS_ROW_ONE + i] = 1.0;
    basis[4 * TS_ROW_X + i] = x[i];
  }
  // one factorised sum family: a field, per direction the first basis row, the row count and the
  // stride of that direction's index in the sums, and where the sums start
  struct Task { int field, out, row[3], m[3], st[3]; };
  struct Dir { int row, m, st; };
  const Dir PSI{TS_ROW_PSI, 3, 0}, PHI{TS_ROW_PHI, 2, 0}, ONE{TS_ROW_ONE, 1, 0};
  auto task = [](int field, int out, Dir d0, Dir d1, Dir d2, int s0, int s1, int s2) {
    return Task{field, out, {d0.row, d1.row, d2.row}, {d0.m, d1.m, d2.m}, {s0, s1, s2}};
  };
  // direction al gets (da, sa), the two others in increasing order (db, sb) and (dc, sc)
  auto by_dir = [&](int field, int out, int al, Dir da, int sa, Dir db, int sb, Dir dc, int sc) {
    Dir d[3]; int st[3];
    d[al] = da; st[al] = sa;
    d[ts_d1(al)] = db; st[ts_d1(al)] = sb;
    d[ts_d2(al)] = dc; st[ts_d2(al)] = sc;
    return task(field, out, d[0], d[1], d[2], st[0], st[1], st[2]);
  };
  std::vector<Task> ga, gb;  // fields 0..26 (coarse blocks) and 27..56 (couplings)
  for (int f = 0; f < 9; ++f) ga.push_back(task(TF_L + f, TJ_L + 27 * f, PSI, PSI, PSI, 1, 3, 9));
  for (int al = 0; al < 3; ++al)
    for (int fl = 0; fl < 4; ++fl)
      ga.push_back(by_dir(fl == 0 ? TF_ADV + al : TF_VP + 3 * al + fl - 1, TJ_VP + 72 * al + 18 * fl,
                          al, PHI, 1, PSI, 2, PSI, 6));
  for (int al = 0; al < 3; ++al) ga.push_back(by_dir(TF_G + al, TJ_DD + 9 * al, al, ONE, 0, PSI, 1, PSI, 3));
  for (int pp = 0; pp < 3; ++pp) {
    const int al = pp == 2 ? 1 : 0, be = pp == 0 ? 1 : 2, gm = 2 - pp;
    Dir d[3]; int st[3];
    d[al] = PHI; st[al] = 1;
    d[be] = PHI; st[be] = 2;
    d[gm] = PSI; st[gm] = 4;
    ga.push_back(task(TF_G + 3 + pp, TJ_OD + 12 * pp, d[0], d[1], d[2], st[0], st[1], st[2]));
  }
  for (int f = 0; f < 12; ++f) {
    gb.push_back(task(TF_YCF + f, TJ_CFN + 8 * f, PHI, PHI, PHI, 1, 2, 4));
    gb.push_back(task(TF_YFC + f, TJ_FCN + 8 * f, PHI, PHI, PHI, 1, 2, 4));
  }
  for (int al = 0; al < 3; ++al) {
    gb.push_back(by_dir(TF_ZCF + al, TJ_CFD + 4 * al, al, ONE, 0, PHI, 1, PHI, 2));
    gb.push_back(by_dir(TF_ZFC + al, TJ_FCD + 4 * al, al, ONE, 0, PHI, 1, PHI, 2));
  }
  // first fit of `size` doubles avoiding the busy intervals [a, b)
  auto place = [&](int size, std::vector<std::pair<int, int>> busy) {
    std::sort(busy.begin(), busy.end());
    int at = 0;
    for (auto& iv : busy) {
      if (iv.first - at >= size) break;
      at = std::max(at, iv.second);
    }
    return at + size <= total ? at : -1;
  };
  plan.assign(TS_PLAN_HEAD, 0u);
  auto entry = [&](int in, int out, int row) {
    plan.push_back((uint32_t)in | (uint32_t)out << 12 | (uint32_t)row << 24);
  };
  const std::vector<Task>* groups[2] = {&ga, &gb};
  const int f_hi[2] = {27, TS_FIELDS}, t_lo[2] = {0, TJ_CFN}, t_hi[2] = {TJ_CFN, TS_SUMS};
  if (total > 4096) return false;
  int step = 0;
  for (int g = 0; g < 2; ++g) {
    const auto& ts = *groups[g];
    const std::pair<int, int> later{fbase + f_hi[g] * ld, total}, done{0, t_lo[g]};
    int n1sz = 0, n2sz = 0;
    for (auto& t : ts) { n1sz += t.m[0] * n1 * n1; n2sz += t.m[0] * t.m[1] * n1; }
    const int s1 = place(n1sz, {{fbase + (g ? 27 : 0) * ld, total}, done});
    if (s1 < 0) return false;
    const int s2 = place(n2sz, {{s1, s1 + n1sz}, later, done, {t_lo[g], t_hi[g]}});
    if (s2 < 0) return false;
    // step 1: direction 0 of the point fields into s1 (per task and t0: n1^2 partial sums)
    plan[step++] = (uint32_t)plan.size();
    int p1 = s1;
    for (auto& t : ts)
      for (int t0 = 0; t0 < t.m[0]; ++t0)
        for (int i12 = 0; i12 < n1 * n1; ++i12) entry(fbase + t.field * ld + n1 * i12, p1++, t.row[0] + t0);
    // step 2: direction 1 (per task, t0, t1: n1 partial sums)
    plan[step++] = (uint32_t)plan.size();
    p1 = s1;
    int p2 = s2;
    for (auto& t : ts)
      for (int t0 = 0; t0 < t.m[0]; ++t0, p1 += n1 * n1)
        for (int t1 = 0; t1 < t.m[1]; ++t1)
          for (int i2 = 0; i2 < n1; ++i2) entry(p1 + n1 * i2, p2++, t.row[1] + t1);
    // step 3: direction 2 into the sums
    plan[step++] = (uint32_t)plan.size();
    p2 = s2;
    for (auto& t : ts)
      for (int t0 = 0; t0 < t.m[0]; ++t0)
        for (int t1 = 0; t1 < t.m[1]; ++t1, p2 += n1)
          for (int t2 = 0; t2 < t.m[2]; ++t2)
            entry(p2, t.out + t0 * t.st[0] + t1 * t.st[1] + t2 * t.st[2], t.row[2] + t2);
  }
  plan[step] = (uint32_t)plan.size();
  return true;
}

}  // namespace vms
