// The integral factorisations of Sec. II.C, in FP64.
//
// Density fitting in the MO basis:
//   (pq|P) = sum_{mu nu} C_{mu p} (mu nu|P) C_{nu q}             (two GEMMs per P)
//   B^Q_pq = sum_P [W]_QP (pq|P),  W W^T = J^{-1}
// The paper writes W = J^{-1/2}; any W with W W^T = J^{-1} gives the same
// integrals (pq|rs) = sum_Q B^Q_pq B^Q_rs and hence the same energy, and this
// code takes W = L^{-1} from the Cholesky factor J = L L^T (one forward
// elimination instead of an eigendecomposition of the metric). The factors
// then differ from the J^{-1/2} ones by an orthogonal rotation of Q.
//
// Cholesky decomposition of the integrals: the matrix M[(pq),(rs)] = (pq|rs)
// is given implicitly by factors F^k_pq (M = sum_k F^k (F^k)^T); the pivoted
// incomplete Cholesky decomposition (outer-product form with diagonal
// pivoting, Golub & Van Loan) picks at step k the pair p with the largest
// remaining diagonal d_p, forms L[:,k] = (M[:,p] - sum_{j<k} L[:,j] L[p,j]) /
// sqrt(d_p) and subtracts L[:,k]^2 from d, until max d < tau. The whole loop
// runs on the device (a flag stops the remaining steps); the host reads the
// rank at the end.
#include <cmath>
#include <new>
#include <vector>

#include "internal.cuh"

namespace dsrg {
namespace {

// ---------------------------- Cholesky of the metric ----------------------------
// Right-looking column Cholesky on the lower triangle of A, one column per
// step: column k below the diagonal is divided by sqrt(A[k][k]) (the diagonal
// itself keeps the squared value until chol_diag_kernel takes the roots at the
// end, so no thread of a step reads an element another thread of the step
// writes); then A[i][j] -= L[i][k] L[j][k] for k < j <= i. A non-positive
// pivot sets *bad.
__global__ void chol_col_kernel(double* __restrict__ A, int n, int k, int* __restrict__ bad) {
  const int i = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const double akk = A[(size_t)k * n + k];
  if (!(akk > 0.0)) {
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicExch(bad, 1);
    return;
  }
  if (i >= n) return;
  A[(size_t)i * n + k] /= sqrt(akk);
}

__global__ void chol_update_kernel(double* __restrict__ A, int n, int k) {
  const int j = k + 1 + blockIdx.x * blockDim.x + threadIdx.x;
  const int i = k + 1 + blockIdx.y;
  if (j > i || i >= n) return;  // lower triangle only
  A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
}

__global__ void chol_diag_kernel(double* __restrict__ A, int n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n) A[(size_t)k * n + k] = sqrt(A[(size_t)k * n + k]);
}

// Row i of L^{-1} (lower triangular) by forward substitution, all its columns
// c <= i at once: Li[i][c] = (delta_ic - sum_{c <= k < i} L[i][k] Li[k][c]) / L[i][i]
// (rows above i are complete from the earlier launches).
__global__ void tri_row_kernel(const double* __restrict__ L, int n, int i, double* __restrict__ Li) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c > i) return;
  double v = (i == c) ? 1.0 : 0.0;
  for (int k = c; k < i; ++k) v = fma(-L[(size_t)i * n + k], Li[(size_t)k * n + c], v);
  Li[(size_t)i * n + c] = v / L[(size_t)i * n + i];
}

// ------------------------------ pivoted Cholesky ------------------------------
struct CdState {
  int pivot;   // pivot of the current step
  int rank;    // vectors accepted so far
  int done;    // 1 once the largest remaining diagonal fell below tau
  double dmax;
};

// d[p] = M_pp = sum_k F[k][p]^2 (p over the N = n^2 pairs)
__global__ void cd_diag_kernel(const double* __restrict__ F, int K0, size_t N, double* __restrict__ d) {
  const size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= N) return;
  double acc = 0.0;
  for (int k = 0; k < K0; ++k) {
    const double f = F[(size_t)k * N + p];
    acc = fma(f, f, acc);
  }
  d[p] = acc;
}

// argmax of d (one CTA); stops the decomposition when the maximum is below tau
// or the maximum rank is reached. Ties: the lowest index.
__global__ void __launch_bounds__(1024) cd_pivot_kernel(const double* __restrict__ d, size_t N,
                                                        double tau, int max_rank,
                                                        CdState* __restrict__ st) {
  __shared__ double sv[1024];
  __shared__ long long si[1024];
  if (st->done) return;
  double best = -1.0;
  long long bi = 0;
  for (size_t p = threadIdx.x; p < N; p += 1024) {
    const double v = d[p];
    if (v > best) {
      best = v;
      bi = (long long)p;
    }
  }
  sv[threadIdx.x] = best;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int s = 512; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      const double a = sv[threadIdx.x], b = sv[threadIdx.x + s];
      const long long ia = si[threadIdx.x], ib = si[threadIdx.x + s];
      if (b > a || (b == a && ib < ia)) {
        sv[threadIdx.x] = b;
        si[threadIdx.x] = ib;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->dmax = sv[0];
    if (sv[0] < tau || st->rank >= max_rank) {
      st->done = 1;
    } else {
      st->pivot = (int)si[0];
    }
  }
}

// L[:, k] = (M[:, p] - sum_{j<k} L[:, j] L[p, j]) / sqrt(d_p), then d -= L[:, k]^2
// (L stored as [rank][N]: vector k contiguous).
__global__ void cd_column_kernel(const double* __restrict__ F, int K0, size_t N,
                                 double* __restrict__ L, double* __restrict__ d,
                                 CdState* __restrict__ st) {
  if (st->done) return;
  const size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= N) return;
  const int p = st->pivot, k = st->rank;
  double m = 0.0;
  for (int kk = 0; kk < K0; ++kk) m = fma(F[(size_t)kk * N + q], F[(size_t)kk * N + p], m);
  for (int j = 0; j < k; ++j) m = fma(-L[(size_t)j * N + q], L[(size_t)j * N + p], m);
  const double v = m / sqrt(st->dmax);
  L[(size_t)k * N + q] = v;
  d[q] = (q == (size_t)p) ? 0.0 : d[q] - v * v;
}

__global__ void cd_advance_kernel(CdState* __restrict__ st) {
  if (!st->done) st->rank += 1;
}

}  // namespace
}  // namespace dsrg

using namespace dsrg;

extern "C" {

dsrg_status_t dsrg_df_mo_transform(const double* ao3, const double* C, const double* metric,
                                   int32_t nbf, int32_t nmo, int32_t naux, int32_t p0, int32_t np,
                                   int32_t q0, int32_t nq, double* B_out, double* work,
                                   size_t work_bytes, void* cuda_stream) {
  if (!ao3 || !C || !metric || !B_out || !work) return DSRG_ERR_INVALID_ARG;
  if (nbf < 1 || nmo < 1 || naux < 1 || np < 1 || nq < 1 || p0 < 0 || q0 < 0 || p0 + np > nmo ||
      q0 + nq > nmo)
    return DSRG_ERR_INVALID_ARG;
  if (((uintptr_t)ao3 | (uintptr_t)C | (uintptr_t)metric | (uintptr_t)B_out | (uintptr_t)work) & 7u)
    return DSRG_ERR_INVALID_ARG;
  const size_t need = dsrg_df_mo_transform_work_bytes(nbf, naux, np, nq);
  if (work_bytes < need) return DSRG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* Y = work;                                        // [naux][np][nbf]
  double* Z = Y + (size_t)naux * np * nbf;                 // [naux][np][nq]
  double* Lm = Z + (size_t)naux * np * nq;                 // [naux][naux] metric -> L
  double* Li = Lm + (size_t)naux * naux;                   // [naux][naux] L^{-1}
  int* bad = (int*)(Li + (size_t)naux * naux);
  cudaError_t e;
  // Y[P][p][nu] = sum_mu C[mu][p0 + p] ao3[P][mu][nu]
  GemmArgs g1 = batched(mk(np, nbf, nbf, 1, C + p0, 1, nmo, 0, ao3, nbf, 0, 1, Y, nbf, 1, 1.0), naux,
                        0, (long long)nbf * nbf, (long long)np * nbf);
  g1.accumulate = 0;
  // Z[P][p][q] = sum_nu Y[P][p][nu] C[nu][q0 + q]
  GemmArgs g2 = batched(mk(np, nq, nbf, 1, Y, nbf, 1, 0, C + q0, nmo, 0, 1, Z, nq, 1, 1.0), naux,
                        (long long)np * nbf, 0, (long long)np * nq);
  g2.accumulate = 0;
  if ((e = launch_gemm_fp64(st, g1)) != cudaSuccess || (e = launch_gemm_fp64(st, g2)) != cudaSuccess)
    return DSRG_ERR_CUDA;
  // J = L L^T, then L^{-1}
  if (cudaMemcpyAsync(Lm, metric, (size_t)naux * naux * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess ||
      cudaMemsetAsync(bad, 0, sizeof(int), st) != cudaSuccess)
    return DSRG_ERR_CUDA;
  for (int k = 0; k < naux; ++k) {
    chol_col_kernel<<<(naux - k + 255) / 256, 256, 0, st>>>(Lm, naux, k, bad);
    if (k + 1 < naux) {
      dim3 g((naux - k - 1 + 255) / 256, naux - k - 1);
      chol_update_kernel<<<g, 256, 0, st>>>(Lm, naux, k);
    }
  }
  chol_diag_kernel<<<(naux + 255) / 256, 256, 0, st>>>(Lm, naux);
  if (cudaGetLastError() != cudaSuccess) return DSRG_ERR_CUDA;
  if (cudaMemsetAsync(Li, 0, (size_t)naux * naux * 8, st) != cudaSuccess) return DSRG_ERR_CUDA;
  for (int i = 0; i < naux; ++i) tri_row_kernel<<<(i + 256) / 256, 256, 0, st>>>(Lm, naux, i, Li);
  if (cudaGetLastError() != cudaSuccess) return DSRG_ERR_CUDA;
  // B[Q][pq] = sum_P Li[Q][P] Z[P][pq]  (Li lower triangular; the GEMM reads it whole)
  const long long npq = (long long)np * nq;
  GemmArgs g3 = mk(naux, (int)npq, naux, 1, Li, naux, 1, 0, Z, npq, 0, 1, B_out, npq, 1, 1.0);
  g3.accumulate = 0;
  if ((e = launch_gemm_fp64(st, g3)) != cudaSuccess) return DSRG_ERR_CUDA;
  int hbad = 0;
  if (cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DSRG_ERR_CUDA;
  return hbad ? DSRG_ERR_INVALID_ARG : DSRG_OK;
}

size_t dsrg_df_mo_transform_work_bytes(int32_t nbf, int32_t naux, int32_t np, int32_t nq) {
  return ((size_t)naux * np * nbf + (size_t)naux * np * nq + 2 * (size_t)naux * naux) * 8 + 64;
}

dsrg_status_t dsrg_cd_factors(const double* F, int32_t nfac, int32_t n, double tau,
                              int32_t max_rank, double* L_out, int32_t* rank_out, double* work,
                              size_t work_bytes, void* cuda_stream) {
  if (!F || !L_out || !rank_out || !work || nfac < 1 || n < 1 || max_rank < 1 || !(tau > 0.0))
    return DSRG_ERR_INVALID_ARG;
  if (((uintptr_t)F | (uintptr_t)L_out | (uintptr_t)work) & 7u) return DSRG_ERR_INVALID_ARG;
  const size_t N = (size_t)n * n;
  if (work_bytes < dsrg_cd_factors_work_bytes(n)) return DSRG_ERR_INVALID_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  double* d = work;
  CdState* cs = (CdState*)(d + N);
  if (cudaMemsetAsync(cs, 0, sizeof(CdState), st) != cudaSuccess) return DSRG_ERR_CUDA;
  const unsigned gb = (unsigned)((N + 255) / 256);
  cd_diag_kernel<<<gb, 256, 0, st>>>(F, nfac, N, d);
  for (int k = 0; k < max_rank; ++k) {
    cd_pivot_kernel<<<1, 1024, 0, st>>>(d, N, tau, max_rank, cs);
    cd_column_kernel<<<gb, 256, 0, st>>>(F, nfac, N, L_out, d, cs);
    cd_advance_kernel<<<1, 1, 0, st>>>(cs);
  }
  if (cudaGetLastError() != cudaSuccess) return DSRG_ERR_CUDA;
  CdState h{};
  if (cudaMemcpyAsync(&h, cs, sizeof(CdState), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
      cudaStreamSynchronize(st) != cudaSuccess)
    return DSRG_ERR_CUDA;
  *rank_out = h.rank;
  return DSRG_OK;
}

size_t dsrg_cd_factors_work_bytes(int32_t n) {
  return (size_t)n * n * 8 + sizeof(CdState) + 64;
}

}  // extern "C"
