// FP64 CUDA-core kernels for the two pair contractions of the DSRG-MRPT2
// energy: diagram F1 (CCVV, Eq. (23)) and diagram F2 (CAVV, Table 2).
//
// Both are DF products over the auxiliary index Q (Eq. (19)) feeding a fused
// epilogue; no four-index quantity is stored (Sec. III).
#include "internal.cuh"
#include "regulators.cuh"

namespace dsrg {

// ---------------------------------------------------------------------------
// F1 (CCVV). Work item = (core pair i<=j, virtual tile pair A<=B), 64x64 tiles.
// The CTA forms x = v^{ij}[A,B] (x_ab = (ia|jb)) and, for i<j, y = v^{ji}[A,B]
// (y_ab = (ja|ib) = x_ba of the same pair). The pair energies of i,j obey
//   e_ij + e_ji = sum_ab 2 (x^2 - x y + y^2) R_ab   (i < j)
//   e_ii        = sum_ab x^2 R_ab                  (y = x)
// with R = (1 - exp(-2 s D^2))/D and D = e_i + e_j - e_a - e_b; an
// off-diagonal tile A<B stands for itself and its mirror (B,A) (weight 2).
// One FP64 partial per CTA.
// ---------------------------------------------------------------------------
constexpr int T64 = 64, KC64 = 16;

__global__ void __launch_bounds__(256) ccvv_fp64_kernel(
    const double* __restrict__ B, const double* __restrict__ eps, double s, Sizes z,
    const int2* __restrict__ pairs, const int2* __restrict__ tps, int n_tp,
    double* __restrict__ partials, int shard_rank, int shard_world) {
  __shared__ double sIA[KC64][T64], sJB[KC64][T64], sJA[KC64][T64], sIB[KC64][T64];
  __shared__ double red[8];
  const int item = blockIdx.x;
  if (!pair_in_shard(item / n_tp, shard_rank, shard_world)) {
    if (threadIdx.x == 0) partials[item] = 0.0;  // another rank's pair
    return;
  }
  const int2 ij = pairs[item / n_tp];
  const int2 ab = tps[item % n_tp];
  const int i = ij.x, j = ij.y;
  const bool same = (i == j);
  const int a0 = ab.x * T64, b0 = ab.y * T64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int pv = z.nA;  // particle index of the first virtual

  double x[4][4], y[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) x[r][c] = y[r][c] = 0.0;

  for (int q0 = 0; q0 < z.Q; q0 += KC64) {
    for (int e = threadIdx.x; e < KC64 * T64; e += 256) {
      const int qq = e / T64, c = e % T64, q = q0 + qq;
      const bool qok = q < z.Q;
      const int a = a0 + c, b = b0 + c;
      const bool aok = qok && a < z.nV, bok = qok && b < z.nV;
      sIA[qq][c] = aok ? B[bidx(z, q, i, pv + a)] : 0.0;
      sJB[qq][c] = bok ? B[bidx(z, q, j, pv + b)] : 0.0;
      sJA[qq][c] = aok ? B[bidx(z, q, j, pv + a)] : 0.0;
      sIB[qq][c] = bok ? B[bidx(z, q, i, pv + b)] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int qq = 0; qq < KC64; ++qq) {
      double ra[4], rb[4], sa[4], sb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        ra[r] = sIA[qq][ty * 4 + r];
        rb[r] = sJB[qq][tx * 4 + r];
        sa[r] = sJA[qq][ty * 4 + r];
        sb[r] = sIB[qq][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          x[r][c] = fma(ra[r], rb[c], x[r][c]);
          if (!same) y[r][c] = fma(sa[r], sb[c], y[r][c]);
        }
    }
    __syncthreads();
  }

  const double E = eps[i] + eps[j];
  const int ve = z.nC + z.nA;  // orbital index of the first virtual
  double acc = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = a0 + ty * 4 + r;
    if (a >= z.nV) continue;
    const double Ea = E - eps[ve + a];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int b = b0 + tx * 4 + c;
      if (b >= z.nV) continue;
      const double D = Ea - eps[ve + b];
      const double xv = x[r][c];
      const double yv = same ? xv : y[r][c];
      const double qv = fma(xv, xv - yv, yv * yv);  // x^2 - x y + y^2
      acc = fma(qv, reg_f1(D, s), acc);
    }
  }
  const double w = (same ? 1.0 : 2.0) * (ab.x < ab.y ? 2.0 : 1.0);
  const double tot = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[item] = w * tot;
}

int ccvv_fp64_blocks(const dsrg_plan* p) { return p->n_pairs * p->n_tp_ccvv; }

cudaError_t launch_ccvv_fp64(dsrg_plan* p, const double* B, const double* eps, double s) {
  const Segment& sg = p->segs[p->seg_ccvv];
  ccvv_fp64_kernel<<<sg.count, 256, 0, p->stream>>>(B, eps, s, p->z, p->d_pairs, p->d_tp_ccvv,
                                                    p->n_tp_ccvv, p->d_partials + sg.begin,
                                                    p->shard_rank, p->shard_world);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// F2 (CAVV), spin-adapted:
//   F2 = sum_m sum_{u,v} G_uv sum_ef X_u[e,f] (2 X_v[e,f] - X_v[f,e]) Rv_u Rt_v
//   X_u[e,f] = (me|uf), D_u = e_m + e_u - e_e - e_f,
//   Rv_u = 1 + exp(-s D_u^2) (Eq. (15)), Rt_v = (1 - exp(-s D_v^2))/D_v (Eq. (13)).
// Work item = (core m, virtual tile pair A<=B) with 32x32 tiles; the CTA holds
// X_u[A,B] and X_u[B,A]^T for all active u. An off-diagonal tile adds the
// mirror term with X and X^T exchanged.
// ---------------------------------------------------------------------------
constexpr int T32 = 32, KC32 = 8;

template <int NA>
__global__ void __launch_bounds__(256) cavv_fp64_kernel(
    const double* __restrict__ B, const double* __restrict__ eps, const double* __restrict__ G,
    double s, Sizes z, const int2* __restrict__ tps, int n_tp, double* __restrict__ partials) {
  __shared__ double sMA[KC32][T32], sMB[KC32][T32];
  __shared__ double sUA[NA][KC32][T32], sUB[NA][KC32][T32];
  __shared__ double sG[NA][NA];
  __shared__ double red[8];
  const int item = blockIdx.x;
  const int m = item / n_tp;
  const int2 ab = tps[item % n_tp];
  const int a0 = ab.x * T32, b0 = ab.y * T32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // col b = tx, rows a = ty*4 + r
  const int pv = z.nA;
  if (threadIdx.x < NA * NA) sG[threadIdx.x / NA][threadIdx.x % NA] = G[threadIdx.x];

  double X[NA][4], Xt[NA][4];
#pragma unroll
  for (int u = 0; u < NA; ++u)
#pragma unroll
    for (int r = 0; r < 4; ++r) X[u][r] = Xt[u][r] = 0.0;

  for (int q0 = 0; q0 < z.Q; q0 += KC32) {
    for (int e = threadIdx.x; e < KC32 * T32; e += 256) {
      const int qq = e / T32, c = e % T32, q = q0 + qq;
      const bool qok = q < z.Q;
      const int a = a0 + c, b = b0 + c;
      const bool aok = qok && a < z.nV, bok = qok && b < z.nV;
      sMA[qq][c] = aok ? B[bidx(z, q, m, pv + a)] : 0.0;
      sMB[qq][c] = bok ? B[bidx(z, q, m, pv + b)] : 0.0;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        sUA[u][qq][c] = aok ? B[bidx(z, q, z.nC + u, pv + a)] : 0.0;
        sUB[u][qq][c] = bok ? B[bidx(z, q, z.nC + u, pv + b)] : 0.0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int qq = 0; qq < KC32; ++qq) {
      const double mb = sMB[qq][tx];
      double ma[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) ma[r] = sMA[qq][ty * 4 + r];
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        const double ub = sUB[u][qq][tx];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          X[u][r] = fma(ma[r], ub, X[u][r]);                   // (m a | u b)
          Xt[u][r] = fma(sUA[u][qq][ty * 4 + r], mb, Xt[u][r]);  // (m b | u a)
        }
      }
    }
    __syncthreads();
  }

  const int ve = z.nC + z.nA;
  const bool mirror = ab.x < ab.y;
  double acc = 0.0;
  const int b = b0 + tx;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = a0 + ty * 4 + r;
    if (a >= z.nV || b >= z.nV) continue;
    const double base = eps[m] - eps[ve + a] - eps[ve + b];
    double Rv[NA], Rt[NA];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const double D = base + eps[z.nC + u];
      Rv[u] = reg_v(D, s);
      Rt[u] = reg_t(D, s);
    }
    double t1 = 0.0, t2 = 0.0;
#pragma unroll
    for (int v = 0; v < NA; ++v) {
      const double A1 = (2.0 * X[v][r] - Xt[v][r]) * Rt[v];
      const double A2 = (2.0 * Xt[v][r] - X[v][r]) * Rt[v];
      double c1 = 0.0, c2 = 0.0;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        c1 = fma(sG[u][v] * Rv[u], X[u][r], c1);
        c2 = fma(sG[u][v] * Rv[u], Xt[u][r], c2);
      }
      t1 = fma(c1, A1, t1);
      t2 = fma(c2, A2, t2);
    }
    acc += mirror ? (t1 + t2) : t1;
  }
  const double tot = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[item] = tot;
}

int cavv_fp64_blocks(const dsrg_plan* p) { return p->z.nA > 0 ? p->z.nC * p->n_tp_cavv : 0; }

cudaError_t launch_cavv_fp64(dsrg_plan* p, const double* B, const double* eps, const double* G,
                             double s) {
  const Segment& sg = p->segs[p->seg_cavv];
  if (sg.count == 0) return cudaSuccess;
  double* out = p->d_partials + sg.begin;
#define CAVV_CASE(NA_)                                                                   \
  case NA_:                                                                              \
    cavv_fp64_kernel<NA_><<<sg.count, 256, 0, p->stream>>>(B, eps, G, s, p->z,            \
                                                           p->d_tp_cavv, p->n_tp_cavv, out); \
    break;
  switch (p->z.nA) {
    CAVV_CASE(1)
    CAVV_CASE(2)
    CAVV_CASE(3)
    CAVV_CASE(4)
    CAVV_CASE(5)
    CAVV_CASE(6)
    CAVV_CASE(7)
    CAVV_CASE(8)
    default:
      return cudaErrorInvalidValue;
  }
#undef CAVV_CASE
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

}  // namespace dsrg
