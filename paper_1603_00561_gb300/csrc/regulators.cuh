// FP64 regulators of the DSRG-MRPT2 amplitudes and a deterministic block sum.
#pragma once

#include <cuda_runtime.h>

namespace dsrg {

// (1 - exp(-s D^2)) / D of the first-order amplitudes (Eqs. (12), (13));
// its D -> 0 limit is 0 (Sec. II.B, Maclaurin form t ~ v s D).
__device__ __forceinline__ double reg_t(double D, double s) {
  return D == 0.0 ? 0.0 : -expm1(-s * D * D) / D;
}

// 1 + exp(-s D^2) of the modified integrals and Fock elements (Eqs. (14), (15)).
__device__ __forceinline__ double reg_v(double D, double s) { return 1.0 + exp(-s * D * D); }

// (1 - exp(-2 s D^2)) / D: product of the two above for diagram F1 (Eq. (23)).
__device__ __forceinline__ double reg_f1(double D, double s) {
  return D == 0.0 ? 0.0 : -expm1(-2.0 * s * D * D) / D;
}

// Sum of one double per thread over a CTA of NT threads, in a fixed order
// (warp butterfly, then the warp sums in index order by warp 0). The result
// is valid in thread 0. `sh` needs NT/32 doubles.
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) sh[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x < 32) {
    r = (l < NT / 32) ? sh[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
  }
  __syncthreads();
  return r;
}

}  // namespace dsrg
