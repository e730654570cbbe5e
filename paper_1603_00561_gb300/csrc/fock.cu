// Generalized Fock matrix and semicanonical orbitals (Sec. II.B, Eq. (8);
// Sec. III, steps 2-3 of the procedure), all FP64.
//
//   f_pq = h_pq + sum_rs D_rs [(pq|rs) - 1/2 (ps|rq)],  (pq|rs) = sum_Q B^Q_pq B^Q_rs
//
// with D the spin-summed density of the reference (2 on the core diagonal, G on
// the active block, 0 on the virtuals): Eq. (8) summed over spin for a
// spin-free density. The Coulomb part is a contraction of the factors with
// w_Q = sum_rs B^Q_rs D_rs; the exchange part K_pq = sum_{Q, r in H}
// X^Q_pr B^Q_rq, X^Q_pr = sum_{s in H} B^Q_ps D_sr, is one GEMM over the
// composite index (Q, r).
//
// The core, active and virtual blocks of f are then diagonalised separately by
// a parallel cyclic Jacobi method (round-robin pairing, m/2 disjoint rotations
// per step; the rotation of each pair as in Golub & Van Loan, Matrix
// Computations, Sec. 8.5, "symmetric Schur decomposition" of a 2 x 2 block).
// Eigenvalues are sorted ascending within each block and each eigenvector's
// largest component is made positive. U = blockdiag(U_C, U_A, U_V) gives
//   eps = diag(U^T f U), f^(1) = hole x particle block of U^T f U (its active x
//   active part, which belongs to the diagonal block, set to 0),
//   B'^Q = U_H^T B^Q_HP U_P, G' = U_A^T G U_A, lambda2' and lambda3' rotated
//   on every active index.
#include <algorithm>
#include <cmath>
#include <new>
#include <numeric>
#include <vector>

#include "internal.cuh"

struct dsrg_sc_plan {
  dsrg::Sizes z{};
  int device = 0;
  cudaStream_t stream = nullptr;
  std::string last_error;
  std::vector<void*> allocs;
  size_t ws_bytes = 0;
  double *w = nullptr;      // [naux]
  double *J = nullptr;      // [n][n]
  double *K = nullptr;      // [n][n]
  double *X = nullptr;      // [naux][n][nH]
  double *f = nullptr;      // [n][n]
  double *U = nullptr;      // [n][n]
  double *T = nullptr;      // [n][n]
  double *A = nullptr;      // [mmax][mmax] Jacobi work matrix
  double *V = nullptr;      // [mmax][mmax] Jacobi eigenvectors
  double2 *cs = nullptr;    // [mmax/2 + 1] rotation (c, s) per pair
  double *off = nullptr;    // [2] off-diagonal and total squared norms
  double *Bhp = nullptr;    // [naux][nH][nP] gathered hole x particle factors
  double *Bt = nullptr;     // [naux][nH][nP] after the particle rotation
  int *perm = nullptr;      // [mmax]
  double *L3t = nullptr;    // [(2 nA)^6] intermediate of the lambda3 rotation
  int mmax = 0;
  int sweeps_last = 0;
};

namespace dsrg {
namespace {

bool sc_alloc(dsrg_sc_plan* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (cudaMalloc(ptr, bytes ? bytes : 8) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return false;
  }
  p->allocs.push_back(*ptr);
  p->ws_bytes += bytes;
  return true;
}

// w_Q = sum_rs B^Q_rs D_rs = 2 sum_m B^Q_mm + sum_uv B^Q_{nC+u, nC+v} G_uv (one warp per Q).
__global__ void fock_w_kernel(const double* __restrict__ B, const double* __restrict__ G, Sizes z,
                              double* __restrict__ w) {
  const int q = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (q >= z.Q) return;
  const size_t n = (size_t)z.n;
  const double* Bq = B + (size_t)q * n * n;
  double acc = 0.0;
  for (int m = lane; m < z.nC; m += 32) acc += 2.0 * Bq[(size_t)m * n + m];
  for (int k = lane; k < z.nA * z.nA; k += 32) {
    const int u = k / z.nA, v = k % z.nA;
    acc = fma(Bq[(size_t)(z.nC + u) * n + z.nC + v], G[k], acc);
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) w[q] = acc;
}

// J_pq = sum_Q B^Q_pq w_Q: one thread per (p, q), Q outer (coalesced along q).
__global__ void fock_j_kernel(const double* __restrict__ B, const double* __restrict__ w, Sizes z,
                              double* __restrict__ J) {
  const size_t nn = (size_t)z.n * z.n;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nn) return;
  double acc = 0.0;
  for (int q = 0; q < z.Q; ++q) acc = fma(B[(size_t)q * nn + k], w[q], acc);
  J[k] = acc;
}

// X^Q_pr = sum_{s in H} B^Q_ps D_sr for r in H: 2 B^Q_pm (core m), sum_u B^Q_{p,nC+u} G_uv.
__global__ void fock_x_kernel(const double* __restrict__ B, const double* __restrict__ G, Sizes z,
                              double* __restrict__ X) {
  const size_t total = (size_t)z.Q * z.n * z.nH;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  const int r = (int)(k % z.nH);
  const size_t qp = k / z.nH;  // q * n + p
  const double* row = B + qp * z.n;
  double v;
  if (r < z.nC) {
    v = 2.0 * row[r];
  } else {
    const int vv = r - z.nC;
    v = 0.0;
    for (int u = 0; u < z.nA; ++u) v = fma(row[z.nC + u], G[u * z.nA + vv], v);
  }
  X[k] = v;
}

// f = h + J - K / 2, symmetrised (the two halves round differently only in K)
__global__ void fock_sum_kernel(const double* __restrict__ h, const double* __restrict__ J,
                                const double* __restrict__ K, int n, double* __restrict__ f) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)n * n) return;
  const int p = (int)(k / n), q = (int)(k % n);
  const size_t kt = (size_t)q * n + p;
  const double a = fma(-0.5, K[k], h[k] + J[k]);
  const double b = fma(-0.5, K[kt], h[kt] + J[kt]);
  f[k] = 0.5 * (a + b);
}

// ---------------------------- Jacobi eigensolver ----------------------------
// Round-robin pairing of mp (even) positions: at step t position 0 stays and
// the others rotate; pair k couples slots k and mp-1-k.
__device__ __forceinline__ int rr_slot(int k, int t, int mp) {
  return k == 0 ? 0 : 1 + (k - 1 + t) % (mp - 1);
}

__global__ void jac_copy_kernel(const double* __restrict__ f, int n, int lo, int m,
                                double* __restrict__ A, double* __restrict__ V) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m * m) return;
  const int i = k / m, j = k % m;
  A[k] = f[(size_t)(lo + i) * n + lo + j];
  V[k] = (i == j) ? 1.0 : 0.0;
}

// (c, s) of every pair of step t: the 2 x 2 symmetric Schur decomposition.
__global__ void jac_params_kernel(const double* __restrict__ A, int m, int mp, int t,
                                  double2* __restrict__ cs) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= mp / 2) return;
  const int p = rr_slot(k, t, mp), q = rr_slot(mp - 1 - k, t, mp);
  double c = 1.0, s = 0.0;
  if (p < m && q < m) {
    const double apq = A[(size_t)p * m + q];
    if (apq != 0.0) {
      const double app = A[(size_t)p * m + p], aqq = A[(size_t)q * m + q];
      const double tau = (aqq - app) / (2.0 * apq);
      const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
      c = 1.0 / sqrt(1.0 + tt * tt);
      s = tt * c;
    }
  }
  cs[k] = make_double2(c, s);
}

// rows p, q of A <- J^T A (all pairs of the step at once; they are disjoint)
__global__ void jac_rows_kernel(double* __restrict__ A, int m, int mp, int t,
                                const double2* __restrict__ cs) {
  const int k = blockIdx.y;
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int p = rr_slot(k, t, mp), q = rr_slot(mp - 1 - k, t, mp);
  if (p >= m || q >= m) return;
  const double c = cs[k].x, s = cs[k].y;
  if (s == 0.0) return;
  const double ap = A[(size_t)p * m + j], aq = A[(size_t)q * m + j];
  A[(size_t)p * m + j] = c * ap - s * aq;
  A[(size_t)q * m + j] = s * ap + c * aq;
}

// columns p, q of A and of V <- (.) J
__global__ void jac_cols_kernel(double* __restrict__ A, double* __restrict__ V, int m, int mp,
                                int t, const double2* __restrict__ cs) {
  const int k = blockIdx.y;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int p = rr_slot(k, t, mp), q = rr_slot(mp - 1 - k, t, mp);
  if (p >= m || q >= m) return;
  const double c = cs[k].x, s = cs[k].y;
  if (s == 0.0) return;
  double ap = A[(size_t)i * m + p], aq = A[(size_t)i * m + q];
  A[(size_t)i * m + p] = c * ap - s * aq;
  A[(size_t)i * m + q] = s * ap + c * aq;
  ap = V[(size_t)i * m + p];
  aq = V[(size_t)i * m + q];
  V[(size_t)i * m + p] = c * ap - s * aq;
  V[(size_t)i * m + q] = s * ap + c * aq;
}

// off[0] = sum_{i != j} A_ij^2, off[1] = sum A_ij^2 (one CTA)
__global__ void __launch_bounds__(256) jac_norm_kernel(const double* __restrict__ A, int m,
                                                       double* __restrict__ off) {
  __shared__ double s0[256], s1[256];
  double a = 0.0, b = 0.0;
  for (size_t k = threadIdx.x; k < (size_t)m * m; k += 256) {
    const double x = A[k];
    b = fma(x, x, b);
    if (k / m != k % m) a = fma(x, x, a);
  }
  s0[threadIdx.x] = a;
  s1[threadIdx.x] = b;
  __syncthreads();
  for (int st = 128; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      s0[threadIdx.x] += s0[threadIdx.x + st];
      s1[threadIdx.x] += s1[threadIdx.x + st];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    off[0] = s0[0];
    off[1] = s1[0];
  }
}

// U block and eps from the converged A, V: column perm[k] of V becomes column
// lo+k of U, with its largest-magnitude component made positive (first one on ties).
__global__ void jac_store_kernel(const double* __restrict__ A, const double* __restrict__ V, int m,
                                 const int* __restrict__ perm, int n, int lo,
                                 double* __restrict__ U, double* __restrict__ eps) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= m) return;
  const int c = perm[k];
  int imax = 0;
  double vmax = -1.0;
  for (int i = 0; i < m; ++i) {
    const double a = fabs(V[(size_t)i * m + c]);
    if (a > vmax) {
      vmax = a;
      imax = i;
    }
  }
  const double sg = V[(size_t)imax * m + c] < 0.0 ? -1.0 : 1.0;
  for (int i = 0; i < m; ++i) U[(size_t)(lo + i) * n + lo + k] = sg * V[(size_t)i * m + c];
  eps[lo + k] = A[(size_t)c * m + c];
}

// ------------------------------ transformations ------------------------------
// Bhp[Q][i][a] = B^Q[i][nC + a] (hole rows, particle columns)
__global__ void gather_hp_kernel(const double* __restrict__ B, Sizes z, double* __restrict__ Bhp) {
  const size_t total = (size_t)z.Q * z.nH * z.nP;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  const int a = (int)(k % z.nP);
  const size_t qi = k / z.nP;
  const int i = (int)(qi % z.nH);
  const size_t q = qi / z.nH;
  Bhp[k] = B[(q * z.n + i) * z.n + z.nC + a];
}

// f1 = hole x particle block of T = U^T f U with the active x active part 0
__global__ void f1_kernel(const double* __restrict__ T, Sizes z, double* __restrict__ f1) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= z.nH * z.nP) return;
  const int i = k / z.nP, a = k % z.nP;
  f1[k] = (i >= z.nC && a < z.nA) ? 0.0 : T[(size_t)i * z.n + z.nC + a];
}

// G' = UA^T G UA and lambda2' = L rotated on every index (one thread per output)
__global__ void rot_active_kernel(const double* __restrict__ U, const double* __restrict__ G,
                                  const double* __restrict__ L, Sizes z, double* __restrict__ Go,
                                  double* __restrict__ Lo) {
  const int nA = z.nA, nA2 = nA * nA, nA4 = nA2 * nA2;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  auto ua = [&](int a, int u) { return U[(size_t)(z.nC + a) * z.n + z.nC + u]; };
  if (k < nA2) {
    const int u = k / nA, v = k % nA;
    double acc = 0.0;
    for (int a = 0; a < nA; ++a)
      for (int b = 0; b < nA; ++b) acc = fma(ua(a, u) * ua(b, v), G[a * nA + b], acc);
    Go[k] = acc;
  } else if (k < nA2 + nA4) {
    const int r = k - nA2;
    const int y = r % nA, x = (r / nA) % nA, v = (r / nA2) % nA, u = r / (nA2 * nA);
    double acc = 0.0;
    for (int a = 0; a < nA; ++a)
      for (int b = 0; b < nA; ++b)
        for (int c = 0; c < nA; ++c)
          for (int d = 0; d < nA; ++d)
            acc = fma(ua(a, u) * ua(b, v) * ua(c, x) * ua(d, y), L[((a * nA + b) * nA + c) * nA + d],
                      acc);
    Lo[r] = acc;
  }
}

// One index of the spin-orbital three-body cumulant rotated by Us = UA (x) I2:
// out[..., X_ax, ...] = sum_a Us[a][X] in[..., a, ...] on axis `ax` (0..5).
__global__ void rot_l3_axis_kernel(const double* __restrict__ U, Sizes z, int ax,
                                   const double* __restrict__ in, double* __restrict__ out) {
  const int n2 = 2 * z.nA;
  size_t total = 1;
  for (int d = 0; d < 6; ++d) total *= (size_t)n2;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= total) return;
  size_t stride = 1;
  for (int d = 5; d > ax; --d) stride *= (size_t)n2;
  const int X = (int)((k / stride) % n2);
  const size_t base = k - (size_t)X * stride;
  double acc = 0.0;
  for (int a = X & 1; a < n2; a += 2) {  // spin conserved: a and X of the same spin
    const double us = U[(size_t)(z.nC + (a >> 1)) * z.n + z.nC + (X >> 1)];
    acc = fma(us, in[base + (size_t)a * stride], acc);
  }
  out[k] = acc;
}

cudaError_t sc_check(dsrg_sc_plan* p) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) p->last_error = cudaGetErrorString(e);
  return e;
}

// Diagonalise the block [lo, lo + m) of f (symmetric); writes U and eps there.
cudaError_t jacobi_block(dsrg_sc_plan* p, int lo, int m, double* eps) {
  if (m == 0) return cudaSuccess;
  cudaStream_t st = p->stream;
  const int n = p->z.n;
  const int mp = m + (m & 1);
  cudaError_t e;
  jac_copy_kernel<<<(m * m + 255) / 256, 256, 0, st>>>(p->f, n, lo, m, p->A, p->V);
  if ((e = sc_check(p)) != cudaSuccess) return e;
  int sweeps = 0;
  if (m > 1) {
    for (; sweeps < 30; ++sweeps) {
      jac_norm_kernel<<<1, 256, 0, st>>>(p->A, m, p->off);
      if ((e = sc_check(p)) != cudaSuccess) return e;
      double off[2] = {0.0, 0.0};
      if ((e = cudaMemcpyAsync(off, p->off, 2 * sizeof(double), cudaMemcpyDeviceToHost, st)) !=
          cudaSuccess)
        return e;
      if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
      if (off[0] <= 1e-30 * off[1] || off[0] == 0.0) break;
      for (int t = 0; t < mp - 1; ++t) {
        jac_params_kernel<<<(mp / 2 + 127) / 128, 128, 0, st>>>(p->A, m, mp, t, p->cs);
        dim3 g((m + 127) / 128, mp / 2);
        jac_rows_kernel<<<g, 128, 0, st>>>(p->A, m, mp, t, p->cs);
        jac_cols_kernel<<<g, 128, 0, st>>>(p->A, p->V, m, mp, t, p->cs);
      }
      if ((e = sc_check(p)) != cudaSuccess) return e;
    }
  }
  p->sweeps_last = std::max(p->sweeps_last, sweeps);
  // sort the eigenvalues ascending (host: m values)
  std::vector<double> diag(m);
  std::vector<double> Ah((size_t)m * m);
  if ((e = cudaMemcpyAsync(Ah.data(), p->A, (size_t)m * m * sizeof(double), cudaMemcpyDeviceToHost,
                           st)) != cudaSuccess)
    return e;
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  for (int i = 0; i < m; ++i) diag[i] = Ah[(size_t)i * m + i];
  std::vector<int> perm(m);
  std::iota(perm.begin(), perm.end(), 0);
  std::stable_sort(perm.begin(), perm.end(), [&](int a, int b) { return diag[a] < diag[b]; });
  if ((e = cudaMemcpyAsync(p->perm, perm.data(), m * sizeof(int), cudaMemcpyHostToDevice, st)) !=
      cudaSuccess)
    return e;
  jac_store_kernel<<<(m + 127) / 128, 128, 0, st>>>(p->A, p->V, m, p->perm, n, lo, p->U, eps);
  if ((e = sc_check(p)) != cudaSuccess) return e;
  // the host vectors above must outlive the copy
  return cudaStreamSynchronize(st);
}

cudaError_t build_fock(dsrg_sc_plan* p, const double* h, const double* B, const double* G) {
  const Sizes& z = p->z;
  cudaStream_t st = p->stream;
  cudaError_t e;
  const size_t nn = (size_t)z.n * z.n;
  fock_w_kernel<<<(unsigned)(((size_t)z.Q * 32 + 255) / 256), 256, 0, st>>>(B, G, z, p->w);
  if ((e = sc_check(p)) != cudaSuccess) return e;
  fock_j_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(B, p->w, z, p->J);
  if ((e = sc_check(p)) != cudaSuccess) return e;
  const size_t nx = (size_t)z.Q * z.n * z.nH;
  fock_x_kernel<<<(unsigned)((nx + 255) / 256), 256, 0, st>>>(B, G, z, p->X);
  if ((e = sc_check(p)) != cudaSuccess) return e;
  // K[p][q] = sum_{Q, r in H} X[Q][p][r] B[Q][r][q]
  GemmArgs g = mk(z.n, z.n, z.Q, z.nH, p->X, z.nH, (long long)z.n * z.nH, 1, B,
                  (long long)nn, z.n, 1, p->K, z.n, 1, 1.0);
  g.accumulate = 0;
  if ((e = launch_gemm_fp64(st, g)) != cudaSuccess) return e;
  fock_sum_kernel<<<(unsigned)((nn + 255) / 256), 256, 0, st>>>(h, p->J, p->K, z.n, p->f);
  return sc_check(p);
}

}  // namespace
}  // namespace dsrg

using namespace dsrg;

extern "C" {

dsrg_status_t dsrg_sc_plan_create(dsrg_sc_plan_t** out, const dsrg_sizes_t* sz, void* cuda_stream) {
  if (!out) return DSRG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!sz || sz->ncore < 0 || sz->nactive < 0 || sz->nvirt < 0 || sz->naux < 1 ||
      sz->ncore + sz->nactive + sz->nvirt < 1)
    return DSRG_ERR_INVALID_ARG;
  if (sz->nactive > NA_MAX) return DSRG_ERR_UNSUPPORTED;
  const long long n = (long long)sz->ncore + sz->nactive + sz->nvirt;
  if (n > (1 << 15) || (long long)sz->naux * n * n > (1ll << 36)) return DSRG_ERR_UNSUPPORTED;
  dsrg_sc_plan* p = new (std::nothrow) dsrg_sc_plan();
  if (!p) return DSRG_ERR_OOM;
  Sizes& z = p->z;
  z.nC = sz->ncore;
  z.nA = sz->nactive;
  z.nV = sz->nvirt;
  z.Q = sz->naux;
  z.nH = z.nC + z.nA;
  z.nP = z.nA + z.nV;
  z.n = z.nC + z.nA + z.nV;
  p->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&p->device);
  p->mmax = std::max(z.nC, std::max(z.nA, z.nV));
  const size_t nn = (size_t)z.n * z.n, mm = (size_t)p->mmax * p->mmax;
  const size_t nhp = (size_t)z.Q * z.nH * z.nP;
  bool ok = sc_alloc(p, (void**)&p->w, (size_t)z.Q * 8) && sc_alloc(p, (void**)&p->J, nn * 8) &&
            sc_alloc(p, (void**)&p->K, nn * 8) &&
            sc_alloc(p, (void**)&p->X, (size_t)z.Q * z.n * z.nH * 8) &&
            sc_alloc(p, (void**)&p->f, nn * 8) && sc_alloc(p, (void**)&p->U, nn * 8) &&
            sc_alloc(p, (void**)&p->T, nn * 8) && sc_alloc(p, (void**)&p->A, mm * 8) &&
            sc_alloc(p, (void**)&p->V, mm * 8) &&
            sc_alloc(p, (void**)&p->cs, ((size_t)p->mmax / 2 + 2) * sizeof(double2)) &&
            sc_alloc(p, (void**)&p->off, 16) && sc_alloc(p, (void**)&p->Bhp, nhp * 8) &&
            sc_alloc(p, (void**)&p->Bt, nhp * 8) &&
            sc_alloc(p, (void**)&p->perm, ((size_t)p->mmax + 1) * sizeof(int));
  size_t n3 = 1;
  for (int d = 0; d < 6; ++d) n3 *= (size_t)(2 * z.nA);
  ok = ok && (z.nA == 0 || sc_alloc(p, (void**)&p->L3t, n3 * 8));
  if (!ok) {
    for (void* a : p->allocs) cudaFree(a);
    delete p;
    return DSRG_ERR_OOM;
  }
  *out = p;
  return DSRG_OK;
}

dsrg_status_t dsrg_sc_plan_destroy(dsrg_sc_plan_t* p) {
  if (!p) return DSRG_OK;
  cudaStreamSynchronize(p->stream);
  for (void* a : p->allocs) cudaFree(a);
  delete p;
  return DSRG_OK;
}

const char* dsrg_sc_last_error(const dsrg_sc_plan_t* p) { return p ? p->last_error.c_str() : "no plan"; }

int32_t dsrg_sc_last_sweeps(const dsrg_sc_plan_t* p) { return p ? p->sweeps_last : -1; }

dsrg_status_t dsrg_generalized_fock(dsrg_sc_plan_t* p, const double* h, const double* Bfull,
                                   const double* gamma1, double* f_dev) {
  if (!p || !h || !Bfull || !f_dev || (p->z.nA > 0 && !gamma1)) return DSRG_ERR_INVALID_ARG;
  if (((uintptr_t)h | (uintptr_t)Bfull | (uintptr_t)gamma1 | (uintptr_t)f_dev) & 7u)
    return DSRG_ERR_INVALID_ARG;
  if (build_fock(p, h, Bfull, gamma1) != cudaSuccess) return DSRG_ERR_CUDA;
  const size_t nn = (size_t)p->z.n * p->z.n;
  if (cudaMemcpyAsync(f_dev, p->f, nn * 8, cudaMemcpyDeviceToDevice, p->stream) != cudaSuccess)
    return DSRG_ERR_CUDA;
  return DSRG_OK;
}

dsrg_status_t dsrg_semicanonicalize(dsrg_sc_plan_t* p, const double* h, const double* Bfull,
                                    const double* gamma1, const double* lambda2,
                                    const double* lambda3, double* eps_out, double* B_out,
                                    double* f1_out, double* gamma1_out, double* lambda2_out,
                                    double* lambda3_out, double* U_out) {
  if (!p || !h || !Bfull || !eps_out || !B_out || !f1_out) return DSRG_ERR_INVALID_ARG;
  const Sizes& z = p->z;
  if (z.nA > 0 && (!gamma1 || !lambda2 || !gamma1_out || !lambda2_out)) return DSRG_ERR_INVALID_ARG;
  if (lambda3 && z.nA > 0 && !lambda3_out) return DSRG_ERR_INVALID_ARG;
  const uintptr_t mis = (uintptr_t)h | (uintptr_t)Bfull | (uintptr_t)gamma1 | (uintptr_t)lambda2 |
                        (uintptr_t)lambda3 | (uintptr_t)eps_out | (uintptr_t)B_out |
                        (uintptr_t)f1_out | (uintptr_t)gamma1_out | (uintptr_t)lambda2_out |
                        (uintptr_t)lambda3_out | (uintptr_t)U_out;
  if (mis & 7u) return DSRG_ERR_INVALID_ARG;
  cudaStream_t st = p->stream;
  const size_t nn = (size_t)z.n * z.n;
  p->sweeps_last = 0;
  if (build_fock(p, h, Bfull, gamma1) != cudaSuccess) return DSRG_ERR_CUDA;
  if (cudaMemsetAsync(p->U, 0, nn * 8, st) != cudaSuccess) return DSRG_ERR_CUDA;
  if (jacobi_block(p, 0, z.nC, eps_out) != cudaSuccess ||
      jacobi_block(p, z.nC, z.nA, eps_out) != cudaSuccess ||
      jacobi_block(p, z.nH, z.nV, eps_out) != cudaSuccess)
    return DSRG_ERR_CUDA;
  cudaError_t e;
  // T = f U, then T <- U^T T (written to K): U^T f U
  GemmArgs g1 = mk(z.n, z.n, z.n, 1, p->f, z.n, 1, 0, p->U, z.n, 0, 1, p->T, z.n, 1, 1.0);
  g1.accumulate = 0;
  GemmArgs g2 = mk(z.n, z.n, z.n, 1, p->U, 1, z.n, 0, p->T, z.n, 0, 1, p->K, z.n, 1, 1.0);
  g2.accumulate = 0;
  if ((e = launch_gemm_fp64(st, g1)) != cudaSuccess || (e = launch_gemm_fp64(st, g2)) != cudaSuccess)
    return DSRG_ERR_CUDA;
  f1_kernel<<<(z.nH * z.nP + 255) / 256, 256, 0, st>>>(p->K, z, f1_out);
  if (sc_check(p) != cudaSuccess) return DSRG_ERR_CUDA;
  // B' = U_H^T B_HP U_P: gather, particle rotation over all (Q, i) rows, hole rotation per Q
  const size_t nhp = (size_t)z.Q * z.nH * z.nP;
  gather_hp_kernel<<<(unsigned)((nhp + 255) / 256), 256, 0, st>>>(Bfull, z, p->Bhp);
  if (sc_check(p) != cudaSuccess) return DSRG_ERR_CUDA;
  const double* UP = p->U + (size_t)z.nC * z.n + z.nC;  // U[nC + a'][nC + a], row pitch n
  GemmArgs g3 = mk(z.Q * z.nH, z.nP, z.nP, 1, p->Bhp, z.nP, 1, 0, UP, z.n, 0, 1, p->Bt, z.nP, 1, 1.0);
  g3.accumulate = 0;
  // B'[Q][i][a] = sum_i' U[i'][i] Bt[Q][i'][a]
  GemmArgs g4 = batched(mk(z.nH, z.nP, z.nH, 1, p->U, 1, z.n, 0, p->Bt, z.nP, 0, 1, B_out, z.nP, 1,
                           1.0),
                        z.Q, 0, (long long)z.nH * z.nP, (long long)z.nH * z.nP);
  g4.accumulate = 0;
  if ((e = launch_gemm_fp64(st, g3)) != cudaSuccess || (e = launch_gemm_fp64(st, g4)) != cudaSuccess)
    return DSRG_ERR_CUDA;
  if (z.nA > 0) {
    const int n4 = z.nA * z.nA * z.nA * z.nA + z.nA * z.nA;
    rot_active_kernel<<<(n4 + 127) / 128, 128, 0, st>>>(p->U, gamma1, lambda2, z, gamma1_out,
                                                        lambda2_out);
    if (sc_check(p) != cudaSuccess) return DSRG_ERR_CUDA;
    if (lambda3) {
      // six one-index rotations, alternating between the scratch and lambda3_out
      size_t total = 1;
      for (int d = 0; d < 6; ++d) total *= (size_t)(2 * z.nA);
      const double* src = lambda3;
      for (int ax = 0; ax < 6; ++ax) {
        double* dst = (ax % 2 == 0) ? p->L3t : lambda3_out;
        rot_l3_axis_kernel<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(p->U, z, ax, src, dst);
        if (sc_check(p) != cudaSuccess) return DSRG_ERR_CUDA;
        src = dst;
      }
    }
  }
  if (U_out && cudaMemcpyAsync(U_out, p->U, nn * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess)
    return DSRG_ERR_CUDA;
  return DSRG_OK;
}

}  // extern "C"
