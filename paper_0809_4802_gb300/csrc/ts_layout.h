// Layout of the FP64 tangent's factorised sums (tangent_ts.cuh): the per-point fields, the 738
// sums and the one-dimensional basis rows, shared by the device code and the host-side plan
// builder (ts_plan.cpp).
#pragma once

#ifndef __CUDACC__
#ifndef __host__
#define __host__
#endif
#ifndef __device__
#define __device__
#endif
#endif

namespace vms {

constexpr int TS_FIELDS = 57, TS_SUMS = 738;
constexpr int TS_ENGINE = 3;
constexpr int TS_STEPS = 6, TS_PLAN_HEAD = 8;
// rows of the one-dimensional basis table: psi_0..2, phi_0..1, the constant 1, and the Gauss points
constexpr int TS_ROW_PSI = 0, TS_ROW_PHI = 3, TS_ROW_ONE = 5, TS_ROW_X = 6, TS_BASIS_ROWS = 8;
// field slots
constexpr int TF_L = 0, TF_ADV = 9, TF_VP = 12, TF_G = 21, TF_YCF = 27, TF_YFC = 39, TF_ZCF = 51,
              TF_ZFC = 54;
// ranges of the sums
constexpr int TJ_L = 0, TJ_VP = 243, TJ_DD = 459, TJ_OD = 486, TJ_CFN = 522, TJ_FCN = 618,
              TJ_CFD = 714, TJ_FCD = 726;

// point-field stride (odd: conflict-free column reads across lanes)
__host__ __device__ constexpr int ts_ld(int nq) { return nq | 1; }

// the two directions other than al, in increasing order
__host__ __device__ inline int ts_d1(int al) { return al == 0 ? 1 : 0; }
__host__ __device__ inline int ts_d2(int al) { return al == 2 ? 1 : 2; }

}  // namespace vms
