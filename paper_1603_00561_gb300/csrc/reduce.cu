// Deterministic compensated reduction of the per-CTA partial sums into the
// block energies, and the pair energies of diagram F1 (Eq. (23)).
#include "internal.cuh"

namespace dsrg {

// Neumaier's compensated sum: (s, c) += x.
__device__ __forceinline__ void neumaier_add(double& s, double& c, double x) {
  const double t = s + x;
  if (fabs(s) >= fabs(x))
    c += (s - t) + x;
  else
    c += (x - t) + s;
  s = t;
}

// One CTA of 256 threads. Each thread sums a fixed strided subset of each
// block's segments; the 256 (sum, compensation) pairs are then folded in
// index order by thread 0. out[0..3] = blocks, out[4] = their total.
__global__ void __launch_bounds__(256) final_reduce_kernel(const double* __restrict__ partials,
                                                           const Segment* __restrict__ segs,
                                                           int nseg, double* __restrict__ out) {
  __shared__ double sh_s[256], sh_c[256];
  __shared__ double blk[4];
  for (int b = 0; b < 4; ++b) {
    double s = 0.0, c = 0.0;
    for (int g = 0; g < nseg; ++g) {
      if (segs[g].block != b) continue;
      const double* p = partials + segs[g].begin;
      for (int k = threadIdx.x; k < segs[g].count; k += 256) neumaier_add(s, c, p[k]);
    }
    sh_s[threadIdx.x] = s;
    sh_c[threadIdx.x] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
      double S = 0.0, C = 0.0;
      for (int k = 0; k < 256; ++k) {
        neumaier_add(S, C, sh_s[k]);
        C += sh_c[k];
      }
      blk[b] = S + C;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int b = 0; b < 4; ++b) {
      out[b] = blk[b];
      neumaier_add(S, C, blk[b]);
    }
    out[4] = S + C;
  }
}

cudaError_t launch_final_reduce(dsrg_plan* p, double* out) {
  final_reduce_kernel<<<1, 256, 0, p->stream>>>(p->d_partials, p->d_segs, (int)p->segs.size(), out);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// Pair energies e[i][j] from the CCVV partials: items are pair-major, n_tp per
// pair; a pair i<j carries e_ij + e_ji = 2 e_ij.
__global__ void pair_energies_kernel(const double* __restrict__ part, const int2* __restrict__ pairs,
                                     int n_pairs, int n_tp, int nC, double* __restrict__ out) {
  const int pidx = blockIdx.x * blockDim.x + threadIdx.x;
  if (pidx >= n_pairs) return;
  double s = 0.0, c = 0.0;
  for (int k = 0; k < n_tp; ++k) neumaier_add(s, c, part[(size_t)pidx * n_tp + k]);
  const double tot = s + c;
  const int2 ij = pairs[pidx];
  if (ij.x == ij.y) {
    out[ij.x * nC + ij.y] = tot;
  } else {
    out[ij.x * nC + ij.y] = 0.5 * tot;
    out[ij.y * nC + ij.x] = 0.5 * tot;
  }
}

cudaError_t launch_pair_energies(dsrg_plan* p, double* pairs) {
  const Segment& sg = p->segs[p->seg_ccvv];
  const int n_tp = sg.count / p->n_pairs;
  pair_energies_kernel<<<(p->n_pairs + 127) / 128, 128, 0, p->stream>>>(
      p->d_partials + sg.begin, p->d_pairs, p->n_pairs, n_tp, p->z.nC, pairs);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

}  // namespace dsrg
