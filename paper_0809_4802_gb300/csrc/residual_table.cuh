// Shared-memory coefficient store and quadrature table of the FP64 residual kernels (used by the
// residual kernel and by the fused assembly kernel).
#pragma once

#include "vms_internal.h"

namespace vms {

// Monomial coefficients live in shared memory, one column per thread (conflict-free).
template <int THREADS>
struct SmemStore {
  double (*sc)[THREADS];
  int tid;
  __device__ __forceinline__ double get(int k) const { return sc[k][tid]; }
  __device__ __forceinline__ void set(int k, double v) const { sc[k][tid] = v; }
};

// Per-point table in global memory; every thread of a warp reads the same row (broadcast).
struct GlobalTable {
  const QpRow* __restrict__ t;
  __device__ __forceinline__ double xi(int q) const { return __ldg(&t[q].xi); }
  __device__ __forceinline__ double eta(int q) const { return __ldg(&t[q].eta); }
  __device__ __forceinline__ double zeta(int q) const { return __ldg(&t[q].zeta); }
  __device__ __forceinline__ double ez(int q) const { return __ldg(&t[q].ez); }
  __device__ __forceinline__ double b(int q) const { return __ldg(&t[q].b); }
  __device__ __forceinline__ double db(int q, int al) const {
    return al == 0 ? __ldg(&t[q].db0) : (al == 1 ? __ldg(&t[q].db1) : __ldg(&t[q].db2));
  }
  __device__ __forceinline__ double w(int q) const { return __ldg(&t[q].w); }
};

}  // namespace vms
