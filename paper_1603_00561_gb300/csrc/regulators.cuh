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

// ---------------------------------------------------------------------------
// Regulator values and derivatives. x = s D^2.
//   Rt = (1 - e^{-x})/D, dRt/dD = (2 x e^{-x} + expm1(-x))/D^2, dRt/ds = D e^{-x}
//   Rv = 1 + e^{-x},     dRv/dD = -2 s D e^{-x},              dRv/ds = -D^2 e^{-x}
// For x < 1e-4 the Maclaurin series of Sec. II.B is used:
//   Rt = s D (1 - x/2 + x^2/6), dRt/dD = s (1 - 3x/2 + 5x^2/6).
// The F1 regulator is Rt with s -> 2s (and dR/ds doubles).
// ---------------------------------------------------------------------------
struct RegD {
  double v, dD, ds;
};

__device__ __forceinline__ RegD rt_d(double D, double s) {
  const double x = s * D * D;
  const double g = exp(-x);
  RegD r;
  if (x < 1e-4) {
    r.v = s * D * (1.0 - 0.5 * x + x * x / 6.0);
    r.dD = s * (1.0 - 1.5 * x + 5.0 / 6.0 * x * x);
  } else {
    // for x > 1/2, e^{-x} < 0.61 and e^{-x} - 1 has no cancellation: one exponential
    const double em = x > 0.5 ? g - 1.0 : expm1(-x);
    const double inv = 1.0 / D;
    r.v = -em * inv;
    r.dD = (2.0 * x * g + em) * inv * inv;
  }
  r.ds = D * g;
  return r;
}

__device__ __forceinline__ RegD rv_d(double D, double s) {
  const double g = exp(-s * D * D);
  return RegD{1.0 + g, -2.0 * s * D * g, -D * D * g};
}

__device__ __forceinline__ RegD rf1_d(double D, double s) {
  RegD r = rt_d(D, 2.0 * s);
  r.ds *= 2.0;
  return r;
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
