// af_device.cuh -- index maps and array views shared by the forward and
// adjoint kernels of libaf (internal).
#pragma once
#include <cuda_runtime.h>

#include "af_internal.h"

namespace {

__device__ __forceinline__ int wrapi(int i, int n) { return i < 0 ? i + n : (i >= n ? i - n : i); }
// boundary maps: periodic wrap; outflow mirrors the DoFs across the boundary
// face without sign changes (cell -1 <- 0, face -1 <- face 1)
__device__ __forceinline__ int mcell(int i, int n, int bc) {
  if (bc == 0) return wrapi(i, n);
  return i < 0 ? -1 - i : (i >= n ? 2 * n - 1 - i : i);
}
__device__ __forceinline__ int mface(int f, int n, int bc) {
  if (bc == 0) return wrapi(f, n);
  return f < 0 ? -f : (f > n ? 2 * n - f : f);
}

struct SV {   // one DoF class of a state: component k at (i,j) is p[k*cs + j*ex + i]
  const double *p;
  size_t cs;
  int ex;
  __device__ __forceinline__ double operator()(int i, int j, int k) const {
    return __ldg(p + (size_t)k * cs + (size_t)j * ex + i);
  }
};
__device__ __forceinline__ SV sview(const double *p, const AfGrid &g, int c) {
  SV v;
  v.p = p;
  v.cs = (size_t)g.ex[c] * g.ey[c];
  v.ex = g.ex[c];
  return v;
}
struct WV {   // a work array [q][nya][nxa]
  const double *p;
  size_t PS;
  int nxa;
  __device__ __forceinline__ double operator()(int i, int j, int q) const {
    return __ldg(p + (size_t)q * PS + (size_t)j * nxa + i);
  }
};
__device__ __forceinline__ WV wview(const double *p, const AfGrid &g) {
  WV v;
  v.p = p;
  v.PS = (size_t)g.nxa * g.nya;
  v.nxa = g.nxa;
  return v;
}

// F-slot of component k in the stored F1 (skip B1, l = 0) or F2 (skip B2, l = 1)
__device__ __forceinline__ int fslot(int l, int k) { return k < 4 + l ? k : k - 1; }


}  // namespace
