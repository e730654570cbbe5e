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

// Level 1: one CTA of 256 threads per chunk of RED_CHUNK partials of one
// segment. Each thread sums a fixed strided subset with Neumaier compensation;
// warp 0 then folds the 256 (sum, compensation) pairs in a fixed order: lane l
// takes pairs 8l .. 8l+7 in index order, and the 32 lane results meet in a
// fixed butterfly of compensated additions (lane l with lane l ^ o). Every lane
// ends with the same (sum, compensation); lane 0 stores the chunk's pair.
__global__ void __launch_bounds__(256) reduce_chunks_kernel(const double* __restrict__ partials,
                                                            const Segment* __restrict__ segs,
                                                            const int2* __restrict__ chunks,
                                                            double* __restrict__ red) {
  __shared__ double sh_s[256], sh_c[256];
  const int2 ch = chunks[blockIdx.x];
  const Segment sg = segs[ch.x];
  const int k0 = ch.y * RED_CHUNK;
  const int k1 = min(sg.count, k0 + RED_CHUNK);
  const double* p = partials + sg.begin;
  double s = 0.0, c = 0.0;
  for (int k = k0 + threadIdx.x; k < k1; k += 256) neumaier_add(s, c, p[k]);
  sh_s[threadIdx.x] = s;
  sh_c[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x < 32) {
    double S = 0.0, C = 0.0;
    for (int k = 8 * threadIdx.x; k < 8 * threadIdx.x + 8; ++k) {
      neumaier_add(S, C, sh_s[k]);
      C += sh_c[k];
    }
    for (int o = 1; o < 32; o <<= 1) {
      // the lower lane of each pair adds the upper one's sum, and vice versa: both
      // get the same operands in the same order (a + b with b from the higher lane)
      const double oS = __shfl_xor_sync(0xffffffffu, S, o);
      const double oC = __shfl_xor_sync(0xffffffffu, C, o);
      const bool low = (threadIdx.x & o) == 0;
      double a = low ? S : oS, b = low ? oS : S;
      const double ca = low ? C : oC, cb = low ? oC : C;
      double cc = ca + cb;
      neumaier_add(a, cc, b);
      S = a;
      C = cc;
    }
    if (threadIdx.x == 0) {
      red[2 * blockIdx.x] = S;
      red[2 * blockIdx.x + 1] = C;
    }
  }
}

// Level 2 (one CTA): the chunk pairs and their block ids are staged in shared
// memory, then one thread folds the chunk pairs of each block in chunk order.
// out[0..3] = blocks, out[4] = their total.
constexpr int RED2_MAX = 2048;  // chunks staged in shared memory
__global__ void reduce_blocks_kernel(const Segment* __restrict__ segs, const int2* __restrict__ chunks,
                                     int nchunks, const double* __restrict__ red,
                                     double* __restrict__ out) {
  __shared__ double sr[2 * RED2_MAX];
  __shared__ int sb[RED2_MAX];
  const bool staged = nchunks <= RED2_MAX;
  if (staged)
    for (int k = threadIdx.x; k < nchunks; k += blockDim.x) {
      sb[k] = segs[chunks[k].x].block;
      sr[2 * k] = red[2 * k];
      sr[2 * k + 1] = red[2 * k + 1];
    }
  __syncthreads();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double T = 0.0, TC = 0.0;
  for (int b = 0; b < 4; ++b) {
    double S = 0.0, C = 0.0;
    for (int k = 0; k < nchunks; ++k) {
      const int kb = staged ? sb[k] : segs[chunks[k].x].block;
      if (kb != b) continue;
      neumaier_add(S, C, staged ? sr[2 * k] : red[2 * k]);
      C += staged ? sr[2 * k + 1] : red[2 * k + 1];
    }
    out[b] = S + C;
    neumaier_add(T, TC, out[b]);
  }
  out[4] = T + TC;
}

cudaError_t launch_final_reduce(dsrg_plan* p, double* out) {
  if (p->n_chunks > 0) {
    reduce_chunks_kernel<<<p->n_chunks, 256, 0, p->stream>>>(p->d_partials, p->d_segs, p->d_chunks,
                                                            p->d_red);
    DSRG_LAUNCH_CHECK(p);
  }
  reduce_blocks_kernel<<<1, 256, 0, p->stream>>>(p->d_segs, p->d_chunks, p->n_chunks, p->d_red, out);
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
