// Adjoint of the DSRG-MRPT2 energy: dE_total/dB, dE_total/deps, dE_total/ds.
//
// FP64 plans: all adjoint arithmetic is FP64 on CUDA cores. Pair quantities
// are recomputed per core row rather than stored: for a fixed core orbital k
// the kernel forms v^{kj} for every j tile by tile and keeps only
// W^{kj} = dE/dv^{kj}, which a GEMM turns into dB.
// Split-precision plans: the CCVV pair blocks are recomputed on the tensor
// cores by the CCVV kernel's adjoint epilogue (tc_split.cu), the CAVV / CCAV
// integrals X, Z in FP32 (round to nearest) on CUDA cores; the adjoints of all
// integrals then form one symmetric matrix S and one tensor-core GEMM turns it
// into dB (tc_adjoint.cu). Regulators, their derivatives and every epilogue
// stay FP64. dB is assembled with one thread per element (fixed order,
// bit-reproducible); deps and ds use FP64 atomics.
//
// Derivatives (closed-shell spin-adapted forms of Table 2, Eqs. (12)-(15), (23)):
//  F1: E = sum_{ij} sum_ab v_ab (2 v_ab - v_ba) R(D),  R = (1 - exp(-2 s D^2))/D
//      dE/dv^{kj}_cb = W^{kj}_cb = (4 v_cb - 2 v_bc) R,
//      dE/dB[Q,k,c] = 2 sum_{j,b} W^{kj}_cb B[Q,j,b]
//  F2: dE/dX_u = Rv_u sum_v G_uv (2 X_v - X_v^T) Rt_v + Rt_u sum_w G_wu Rv_w (2 X_w - X_w^T)
//  F3: dE/dZ_w = Rv_w sum_u Hh_wu (2 Z_u - Z_u^T) Rt_u + Rt_w sum_v Hh_vw Rv_v (2 Z_v - Z_v^T)
//  active block: reverse pass through the term sums, T1 / modified Fock, the
//      dressed T of term I, the (A,A|V,V) spin sums and the spin-orbital tables.
#include <type_traits>

#include "internal.cuh"
#include "regulators.cuh"

namespace dsrg {

// ---------------------------------------------------------------------------
// Generic FP64 GEMM with composite K index:
//   C[i*ci + j*cj] (+)= alpha * sum_{l1<L1, l2<L2} A[i*ai + l1*a1 + l2*a2] * Bm[l1*b1 + l2*b2 + j*bj]
// 64 x 64 tiles, 256 threads, K chunks of 16 over l = l1*L2 + l2.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) gemm_fp64_kernel(GemmArgs g) {
  __shared__ double sA[16][65], sB[16][65];
  g.A += blockIdx.z * g.sa;
  g.Bm += blockIdx.z * g.sb;
  g.C += blockIdx.z * g.sc;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const long long L = (long long)g.L1 * g.L2;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (long long l0 = 0; l0 < L; l0 += 16) {
    for (int e = threadIdx.x; e < 16 * 64; e += 256) {
      const int ll = e / 64, c = e % 64;
      const long long l = l0 + ll;
      double va = 0.0, vb = 0.0;
      if (l < L) {
        const long long l1 = l / g.L2, l2 = l % g.L2;
        if (i0 + c < g.M) va = g.A[(long long)(i0 + c) * g.ai + l1 * g.a1 + l2 * g.a2];
        if (j0 + c < g.N) vb = g.Bm[l1 * g.b1 + l2 * g.b2 + (long long)(j0 + c) * g.bj];
      }
      sA[ll][c] = va;
      sB[ll][c] = vb;
    }
    __syncthreads();
#pragma unroll 4
    for (int ll = 0; ll < 16; ++ll) {
      double ra[4], rb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        ra[r] = sA[ll][ty * 4 + r];
        rb[r] = sB[ll][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(ra[r], rb[c], acc[r][c]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int i = i0 + ty * 4 + r;
    if (i >= g.M) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + tx * 4 + c;
      if (j >= g.N) continue;
      double* p = g.C + (long long)i * g.ci + (long long)j * g.cj;
      *p = g.accumulate ? fma(g.alpha, acc[r][c], *p) : g.alpha * acc[r][c];
    }
  }
}

// Gradient workspace (DSRG_PLAN_GRAD).
struct GradWs {
  double* Wk = nullptr;   // [kgroup][nC][nVp][nVp]
  int nVp = 0;
  int kgroup = 1;         // core rows whose W^{kj} are formed before one batched GEMM
  size_t nB = 0;          // elements of B
  double* dX = nullptr;   // [nC][nA][nV][nV]
  double* dZ = nullptr;   // [nA][nC][nC][nV]
  double *dW1Vt = nullptr, *dW1T = nullptr, *dTi = nullptr, *dV1 = nullptr;
  double *dW2Vt = nullptr, *dW2T = nullptr, *dV2 = nullptr;
  double *dt1 = nullptr, *dft = nullptr, *dS = nullptr, *dP12 = nullptr;
  double *dK1 = nullptr, *dK2 = nullptr, *dK3 = nullptr, *dM = nullptr;
};

cudaError_t launch_gemm_fp64(cudaStream_t st, const GemmArgs& g) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.nb);
  gemm_fp64_kernel<<<grid, 256, 0, st>>>(g);
  return cudaGetLastError();
}

// The FP64 plans' GEMMs (split plans assemble dB on the tensor cores).
static cudaError_t gemm(dsrg_plan* p, const GemmArgs& g) {
  if (g.M <= 0 || g.N <= 0) return cudaSuccess;
  dim3 grid((g.N + 63) / 64, (g.M + 63) / 64, g.nb);
  gemm_fp64_kernel<<<grid, 256, 0, p->stream>>>(g);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// F1 adjoint for one core row k: items (j, tile pair A<=B), 64 x 64 tiles.
// Writes W^{kj}[c][b] into Wk[j][c][b] (row pitch nVp) and adds to deps, ds.
// ---------------------------------------------------------------------------
constexpr int GT = 64;

template <typename T>
__global__ void __launch_bounds__(256) ccvv_adj_kernel(const double* __restrict__ B,
                                                       const double* __restrict__ eps, double s,
                                                       Sizes z, int k, const int2* __restrict__ tps,
                                                       int n_tp, int nVp, double* __restrict__ Wk,
                                                       double* __restrict__ deps,
                                                       double* __restrict__ ds) {
  __shared__ T sKA[16][GT], sJB[16][GT], sJA[16][GT], sKB[16][GT];
  __shared__ double rowacc[GT], colacc[GT];
  __shared__ double red[8];
  const int j = blockIdx.x / n_tp;
  const int2 ab = tps[blockIdx.x % n_tp];
  const int a0 = ab.x * GT, b0 = ab.y * GT;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int pv = z.nA, ve = z.nC + z.nA;
  if (threadIdx.x < GT) {
    rowacc[threadIdx.x] = 0.0;
    colacc[threadIdx.x] = 0.0;
  }
  T x[4][4], y[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) x[r][c] = y[r][c] = (T)0;
  for (int q0 = 0; q0 < z.Q; q0 += 16) {
    for (int e = threadIdx.x; e < 16 * GT; e += 256) {
      const int qq = e / GT, c = e % GT, q = q0 + qq;
      const bool qok = q < z.Q;
      const int a = a0 + c, b = b0 + c;
      const bool aok = qok && a < z.nV, bok = qok && b < z.nV;
      sKA[qq][c] = aok ? (T)B[bidx(z, q, k, pv + a)] : (T)0;
      sJB[qq][c] = bok ? (T)B[bidx(z, q, j, pv + b)] : (T)0;
      sJA[qq][c] = aok ? (T)B[bidx(z, q, j, pv + a)] : (T)0;
      sKB[qq][c] = bok ? (T)B[bidx(z, q, k, pv + b)] : (T)0;
    }
    __syncthreads();
#pragma unroll 4
    for (int qq = 0; qq < 16; ++qq) {
      T ra[4], rb[4], sa[4], sb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        ra[r] = sKA[qq][ty * 4 + r];
        rb[r] = sJB[qq][tx * 4 + r];
        sa[r] = sJA[qq][ty * 4 + r];
        sb[r] = sKB[qq][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          x[r][c] = fma(ra[r], rb[c], x[r][c]);
          y[r][c] = fma(sa[r], sb[c], y[r][c]);
        }
    }
    __syncthreads();
  }
  const double E = eps[k] + eps[j];
  const bool mirror = ab.x < ab.y;
  const double wt = mirror ? 2.0 : 1.0;
  double dk = 0.0, dss = 0.0;
  double racc[4] = {0, 0, 0, 0}, cacc[4] = {0, 0, 0, 0};
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = a0 + ty * 4 + r;
    if (a >= z.nV) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int b = b0 + tx * 4 + c;
      if (b >= z.nV) continue;
      const double D = E - eps[ve + a] - eps[ve + b];
      const RegD R = rf1_d(D, s);
      const double xv = (double)x[r][c], yv = (double)y[r][c];
      Wk[((size_t)j * nVp + a) * nVp + b] = (4.0 * xv - 2.0 * yv) * R.v;
      if (mirror) Wk[((size_t)j * nVp + b) * nVp + a] = (4.0 * yv - 2.0 * xv) * R.v;
      const double q = fma(xv, xv - yv, yv * yv);
      dk = fma(2.0 * wt * q, R.dD, dk);
      dss = fma(wt * q, R.ds, dss);
      const double gv = -2.0 * q * R.dD;
      racc[r] += gv;
      if (mirror) cacc[c] += gv;
    }
  }
#pragma unroll
  for (int r = 0; r < 4; ++r) atomicAdd(&rowacc[ty * 4 + r], racc[r]);
  if (mirror) {
#pragma unroll
    for (int c = 0; c < 4; ++c) atomicAdd(&colacc[tx * 4 + c], cacc[c]);
  }
  const double tk = block_sum<256>(dk, red);
  const double ts = block_sum<256>(dss, red);
  if (threadIdx.x == 0) {
    atomicAdd(&deps[k], tk);
    atomicAdd(ds, ts);
  }
  if (threadIdx.x < GT) {
    const int a = a0 + threadIdx.x, b = b0 + threadIdx.x;
    if (a < z.nV) atomicAdd(&deps[ve + a], rowacc[threadIdx.x]);
    if (mirror && b < z.nV) atomicAdd(&deps[ve + b], colacc[threadIdx.x]);
  }
}


// ---------------------------------------------------------------------------
// F2 adjoint: items (m, tile pair A<=B), 32 x 32 tiles; writes dX[m][u][e][f].
// ---------------------------------------------------------------------------
template <int NA, typename T>
__global__ void __launch_bounds__(256) cavv_adj_kernel(
    const double* __restrict__ B, const double* __restrict__ eps, const double* __restrict__ G,
    double s, Sizes z, const int2* __restrict__ tps, int n_tp, int nVp, double* __restrict__ dX,
    double* __restrict__ deps, double* __restrict__ ds) {
  __shared__ T sMA[8][32], sMB[8][32];
  __shared__ T sUA[NA][8][32], sUB[NA][8][32];
  __shared__ double sG[NA][NA];
  __shared__ double rowacc[32], colacc[32], uacc[NA];
  __shared__ double red[8];
  const int m = blockIdx.x / n_tp;
  const int2 ab = tps[blockIdx.x % n_tp];
  const int a0 = ab.x * 32, b0 = ab.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int pv = z.nA, ve = z.nC + z.nA;
  if (threadIdx.x < NA * NA) sG[threadIdx.x / NA][threadIdx.x % NA] = G[threadIdx.x];
  if (threadIdx.x < 32) {
    rowacc[threadIdx.x] = 0.0;
    colacc[threadIdx.x] = 0.0;
  }
  if (threadIdx.x < NA) uacc[threadIdx.x] = 0.0;
  T Xa[NA][4], Xta[NA][4];
#pragma unroll
  for (int u = 0; u < NA; ++u)
#pragma unroll
    for (int r = 0; r < 4; ++r) Xa[u][r] = Xta[u][r] = (T)0;
  for (int q0 = 0; q0 < z.Q; q0 += 8) {
    for (int e = threadIdx.x; e < 8 * 32; e += 256) {
      const int qq = e / 32, c = e % 32, q = q0 + qq;
      const bool qok = q < z.Q;
      const int a = a0 + c, b = b0 + c;
      const bool aok = qok && a < z.nV, bok = qok && b < z.nV;
      sMA[qq][c] = aok ? (T)B[bidx(z, q, m, pv + a)] : (T)0;
      sMB[qq][c] = bok ? (T)B[bidx(z, q, m, pv + b)] : (T)0;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        sUA[u][qq][c] = aok ? (T)B[bidx(z, q, z.nC + u, pv + a)] : (T)0;
        sUB[u][qq][c] = bok ? (T)B[bidx(z, q, z.nC + u, pv + b)] : (T)0;
      }
    }
    __syncthreads();
#pragma unroll
    for (int qq = 0; qq < 8; ++qq) {
      const T mb = sMB[qq][tx];
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        const T ub = sUB[u][qq][tx];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          Xa[u][r] = fma(sMA[qq][ty * 4 + r], ub, Xa[u][r]);
          Xta[u][r] = fma(sUA[u][qq][ty * 4 + r], mb, Xta[u][r]);
        }
      }
    }
    __syncthreads();
  }
  double X[NA][4], Xt[NA][4];
#pragma unroll
  for (int u = 0; u < NA; ++u)
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      X[u][r] = (double)Xa[u][r];
      Xt[u][r] = (double)Xta[u][r];
    }
  const bool mirror = ab.x < ab.y;
  const int b = b0 + tx;
  double dm = 0.0, dss = 0.0, cacc = 0.0;
  double du[NA];
#pragma unroll
  for (int u = 0; u < NA; ++u) du[u] = 0.0;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int a = a0 + ty * 4 + r;
    if (a >= z.nV || b >= z.nV) continue;
    const double base = eps[m] - eps[ve + a] - eps[ve + b];
    RegD Rv[NA], Rt[NA];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const double D = base + eps[z.nC + u];
      Rv[u] = rv_d(D, s);
      Rt[u] = rt_d(D, s);
    }
    double P[NA], Pt[NA];  // 2 X - X^T at (a,b) and at (b,a)
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      P[u] = 2.0 * X[u][r] - Xt[u][r];
      Pt[u] = 2.0 * Xt[u][r] - X[u][r];
    }
    double gsum = 0.0;
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      double s1 = 0.0, s2 = 0.0, s1t = 0.0, s2t = 0.0;
#pragma unroll
      for (int v = 0; v < NA; ++v) {
        s1 = fma(sG[u][v] * Rt[v].v, P[v], s1);
        s2 = fma(sG[v][u] * Rv[v].v, P[v], s2);
        s1t = fma(sG[u][v] * Rt[v].v, Pt[v], s1t);
        s2t = fma(sG[v][u] * Rv[v].v, Pt[v], s2t);
      }
      const double dxab = Rv[u].v * s1 + Rt[u].v * s2;
      dX[(((size_t)m * NA + u) * nVp + a) * nVp + b] = dxab;
      if (mirror) dX[(((size_t)m * NA + u) * nVp + b) * nVp + a] = Rv[u].v * s1t + Rt[u].v * s2t;
      // dE/dD_u and dE/ds at (a,b) (+ mirror): y_uv = G_uv X_u P_v
      double gD = X[u][r] * (Rv[u].dD * s1 + 0.0);
      double gs = X[u][r] * Rv[u].ds * s1;
      // Rt'_u part: sum_w G_wu X_w Rv_w P_u
      double cw = 0.0, cwt = 0.0;
#pragma unroll
      for (int w = 0; w < NA; ++w) {
        cw = fma(sG[w][u] * Rv[w].v, X[w][r], cw);
        cwt = fma(sG[w][u] * Rv[w].v, Xt[w][r], cwt);
      }
      gD = fma(cw * P[u], Rt[u].dD, gD);
      gs = fma(cw * P[u], Rt[u].ds, gs);
      if (mirror) {
        gD = fma(Xt[u][r] * s1t, Rv[u].dD, gD);
        gs = fma(Xt[u][r] * s1t, Rv[u].ds, gs);
        gD = fma(cwt * Pt[u], Rt[u].dD, gD);
        gs = fma(cwt * Pt[u], Rt[u].ds, gs);
      }
      du[u] += gD;
      gsum += gD;
      dss += gs;
    }
    dm += gsum;
    atomicAdd(&rowacc[ty * 4 + r], -gsum);
    cacc -= gsum;
  }
  atomicAdd(&colacc[tx], cacc);
  const double tm = block_sum<256>(dm, red);
  const double ts = block_sum<256>(dss, red);
  for (int u = 0; u < NA; ++u) {
    const double t = block_sum<256>(du[u], red);
    if (threadIdx.x == 0) atomicAdd(&deps[z.nC + u], t);
  }
  if (threadIdx.x == 0) {
    atomicAdd(&deps[m], tm);
    atomicAdd(ds, ts);
  }
  if (threadIdx.x < 32) {
    const int a = a0 + threadIdx.x, bb = b0 + threadIdx.x;
    if (a < z.nV) atomicAdd(&deps[ve + a], rowacc[threadIdx.x]);
    if (bb < z.nV) atomicAdd(&deps[ve + bb], colacc[threadIdx.x]);
  }
}

// ---------------------------------------------------------------------------
// F3 adjoint: one CTA per virtual e; writes dZ[w][m][n][e].
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) ccav_adj_kernel(
    const double* __restrict__ B, const double* __restrict__ eps, const double* __restrict__ G,
    double s, Sizes z, double* __restrict__ dZ, double* __restrict__ deps, double* __restrict__ ds) {
  extern __shared__ double smem[];
  const int nC = z.nC, nA = z.nA;
  double* accm = smem;                 // [nC]  deps of core orbitals
  double* accu = accm + nC;            // [nA]
  T* Z = (T*)(accu + nA);              // [nA][nC][nC]
  T* sBe = Z + nA * nC * nC;           // [8][nC]
  T* sBu = sBe + 8 * nC;               // [8][nC][nA]
  __shared__ double red[8];
  const int e = blockIdx.x;
  const int nz = nA * nC * nC;
  for (int k = threadIdx.x; k < nz; k += 256) Z[k] = (T)0;
  for (int k = threadIdx.x; k < nC + nA; k += 256) accm[k] = 0.0;
  for (int q0 = 0; q0 < z.Q; q0 += 8) {
    __syncthreads();
    for (int k = threadIdx.x; k < 8 * nC * (1 + nA); k += 256) {
      const int qq = k / (nC * (1 + nA)), r = k % (nC * (1 + nA)), q = q0 + qq;
      T v = (T)0;
      if (r < nC) {
        if (q < z.Q) v = (T)B[bidx(z, q, r, nA + e)];
        sBe[qq * nC + r] = v;
      } else {
        const int nu = r - nC, n = nu / nA, u = nu % nA;
        if (q < z.Q) v = (T)B[bidx(z, q, n, u)];
        sBu[(qq * nC + n) * nA + u] = v;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nz; k += 256) {
      const int u = k / (nC * nC), mn = k % (nC * nC), m = mn / nC, n = mn % nC;
      T acc = Z[k];
#pragma unroll
      for (int qq = 0; qq < 8; ++qq) acc = fma(sBe[qq * nC + m], sBu[(qq * nC + n) * nA + u], acc);
      Z[k] = acc;
    }
  }
  __syncthreads();
  const double ee = eps[nC + nA + e];
  double de = 0.0, dss = 0.0;
  for (int mn = threadIdx.x; mn < nC * nC; mn += 256) {
    const int m = mn / nC, n = mn % nC;
    const double base = eps[m] + eps[n] - ee;
    RegD Rv[NA_MAX], Rt[NA_MAX];
    double P[NA_MAX];
    for (int u = 0; u < nA; ++u) {
      const double D = base - eps[nC + u];
      Rv[u] = rv_d(D, s);
      Rt[u] = rt_d(D, s);
      P[u] = 2.0 * (double)Z[(u * nC + m) * nC + n] - (double)Z[(u * nC + n) * nC + m];
    }
    double gsum = 0.0;
    for (int w = 0; w < nA; ++w) {
      double s1 = 0.0, s2 = 0.0, cw = 0.0;
      for (int u = 0; u < nA; ++u) {
        const double Hwu = (w == u ? 2.0 : 0.0) - G[w * nA + u];
        const double Huw = (u == w ? 2.0 : 0.0) - G[u * nA + w];
        s1 = fma(Hwu * Rt[u].v, P[u], s1);
        s2 = fma(Huw * Rv[u].v, P[u], s2);
        cw = fma(Huw * Rv[u].v, (double)Z[(u * nC + m) * nC + n], cw);
      }
      const double zw = (double)Z[(w * nC + m) * nC + n];
      dZ[(((size_t)w * nC + m) * nC + n) * z.nV + e] = Rv[w].v * s1 + Rt[w].v * s2;
      // dE/dD_w: y_wu Rv'_w Rt_u + y_vw Rv_v Rt'_w
      const double gD = zw * s1 * Rv[w].dD + cw * P[w] * Rt[w].dD;
      dss += zw * s1 * Rv[w].ds + cw * P[w] * Rt[w].ds;
      gsum += gD;
      atomicAdd(&accu[w], -gD);
    }
    atomicAdd(&accm[m], gsum);
    atomicAdd(&accm[n], gsum);
    de -= gsum;
  }
  __syncthreads();
  const double te = block_sum<256>(de, red);
  const double ts = block_sum<256>(dss, red);
  if (threadIdx.x == 0) {
    atomicAdd(&deps[nC + nA + e], te);
    atomicAdd(ds, ts);
  }
  for (int k = threadIdx.x; k < nC; k += 256) atomicAdd(&deps[k], accm[k]);
  for (int k = threadIdx.x; k < nA; k += 256) atomicAdd(&deps[nC + k], accu[k]);
}

}  // namespace dsrg

namespace dsrg {

// ---------------------------------------------------------------------------
// Active block adjoint. Index conventions as in the forward (active.cu):
// W1[I][U][A][X] = <iu||ax> (I hole spin orbital, U active hole, A particle
// spin orbital, X active particle), W2[I][J][X][Y] = <ij||xy>, spin orbital
// 2p + sigma; gamma/eta sparse (identity on core / virtual).
// ---------------------------------------------------------------------------
struct AD {
  int nC2, nA2, nH2, nP2, nV2;
};
__device__ __forceinline__ AD adims(const Sizes& z) {
  return AD{2 * z.nC, 2 * z.nA, 2 * z.nH, 2 * z.nP, 2 * z.nV};
}
__device__ __forceinline__ size_t W1(const AD& d, int I, int U, int A, int X) {
  return (((size_t)I * d.nA2 + U) * d.nP2 + A) * d.nA2 + X;
}
__device__ __forceinline__ size_t W2(const AD& d, int I, int J, int X, int Y) {
  return (((size_t)I * d.nH2 + J) * d.nA2 + X) * d.nA2 + Y;
}
__device__ __forceinline__ int LM(const AD& d, int U, int V, int X, int Y) {
  return ((U * d.nA2 + V) * d.nA2 + X) * d.nA2 + Y;
}
__device__ __forceinline__ double gH(const AD& d, const double* gA, int K, int I) {
  if (K < d.nC2 || I < d.nC2) return (K == I) ? 1.0 : 0.0;
  return gA[(K - d.nC2) * d.nA2 + (I - d.nC2)];
}
__device__ __forceinline__ double eP(const AD& d, const double* gA, int A, int Bp) {
  if (A >= d.nA2 || Bp >= d.nA2) return (A == Bp) ? 1.0 : 0.0;
  return (A == Bp ? 1.0 : 0.0) - gA[A * d.nA2 + Bp];
}
__device__ __forceinline__ double gAA(const AD& d, const double* gA, int U, int V) {
  return gA[U * d.nA2 + V];
}
__device__ __forceinline__ double eAA(const AD& d, const double* gA, int U, int V) {
  return (U == V ? 1.0 : 0.0) - gA[U * d.nA2 + V];
}

struct ActAdjArgs {
  Sizes z;
  double s;
  const double* eps;
  const double *K1, *K2, *K3, *W1V, *W1T, *W1Vt, *W2V, *W2T, *W2Vt, *Ti, *lam, *gA, *t1, *ft, *M;
  double *dW1Vt, *dW1T, *dTi, *dW2Vt, *dW2T, *dt1, *dft, *dP12, *dS, *dV1, *dV2, *dK1, *dK2, *dK3,
      *dM;
  double *deps, *ds;
  size_t w1n, w2n;
  const double* lam3;  // [2nA]^6 spin-orbital three-body cumulant (terms J, K), or null
  const double* f1;    // [nH][nP] off-diagonal Fock block (Eqs. (12), (14)), or null
};

__device__ __forceinline__ size_t L3I(int n2, int U, int V, int W, int X, int Y, int Z) {
  return (((((size_t)U * n2 + V) * n2 + W) * n2 + X) * n2 + Y) * n2 + Z;
}

// (A1) term adjoints landing on W1-shaped tables: d(vt), d(t) direct, d(Ti).
__global__ void adj_w1_terms_kernel(ActAdjArgs a) {
  const AD d = adims(a.z);
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.w1n) return;
  const int X = (int)(k % d.nA2);
  const int A = (int)((k / d.nA2) % d.nP2);
  const int U = (int)((k / ((size_t)d.nA2 * d.nP2)) % d.nA2);
  const int I = (int)(k / ((size_t)d.nA2 * d.nP2 * d.nA2));
  const bool Iact = I >= d.nC2, Avir = A >= d.nA2;
  const double* lam = a.lam;
  const double* gA = a.gA;
  double dvt = 0.0, dt = 0.0, dti = 0.0;
  // term I (all elements): vt_{jx}^{bu} at (J=I, x=U, b=A, u=X); Ti at (J=I, V=U, B=A, Y=X)
  for (int V = 0; V < d.nA2; ++V)
    for (int Y = 0; Y < d.nA2; ++Y) dvt = fma(a.Ti[W1(d, I, V, A, Y)], lam[LM(d, X, V, U, Y)], dvt);
  for (int Uu = 0; Uu < d.nA2; ++Uu)
    for (int Xx = 0; Xx < d.nA2; ++Xx)
      dti = fma(a.W1Vt[W1(d, I, Xx, A, Uu)], lam[LM(d, Uu, U, Xx, X)], dti);
  if (Iact && Avir) {
    const int Xa = I - d.nC2;  // the active hole of the first slot
    // B: 1/2 vt[Xa,Y=U,e,V=X] t1[U',e] lam[U',V,Xa,Y]
    for (int Uu = 0; Uu < d.nA2; ++Uu)
      dvt = fma(0.5 * a.t1[(size_t)(d.nC2 + Uu) * d.nP2 + A], lam[LM(d, Uu, X, Xa, U)], dvt);
    // GVA: 1/4 sum lam[U',V',Xa,Y] W1Vt[Xa,Y,e,C] tg[U',V',C], tg = sum_A' eta[C][A'] W1T[U',V',e,A']
    for (int Uu = 0; Uu < d.nA2; ++Uu)
      for (int Vv = 0; Vv < d.nA2; ++Vv) {
        double tg = 0.0;
        for (int Ap = 0; Ap < d.nA2; ++Ap)
          tg = fma(eAA(d, gA, X, Ap), a.W1T[W1(d, d.nC2 + Uu, Vv, A, Ap)], tg);
        dvt = fma(0.25 * lam[LM(d, Uu, Vv, Xa, U)], tg, dvt);
      }
    // D: 1/2 ft[Xx,e] t[Ua=Xa, V=U, e, Y=X] lam[Ua,V,Xx,Y]  -> d(t)
    for (int Xx = 0; Xx < d.nA2; ++Xx)
      dt = fma(0.5 * a.ft[(size_t)(d.nC2 + Xx) * d.nP2 + A], lam[LM(d, Xa, U, Xx, X)], dt);
    // GVA -> d(t) at (Ua=Xa, Vv=U, e, A'=X): sum_C eta[C][A'] dtg[Ua,Vv,C]
    for (int C = 0; C < d.nA2; ++C) {
      const double ec = eAA(d, gA, C, X);
      if (ec == 0.0) continue;
      double dtg = 0.0;
      for (int Xx = 0; Xx < d.nA2; ++Xx)
        for (int Y = 0; Y < d.nA2; ++Y)
          dtg = fma(lam[LM(d, Xa, U, Xx, Y)], a.W1Vt[W1(d, d.nC2 + Xx, Y, A, C)], dtg);
      dt = fma(0.25 * ec, dtg, dt);
    }
    // F7: vt[Ya, Z=U, e, V=X]: 1/2 sum gA[Ya,W] gA[Z,X'] eta[U',V] W1T[W, X', e, U']
    for (int W = 0; W < d.nA2; ++W) {
      const double g1 = gAA(d, gA, Xa, W);
      if (g1 == 0.0) continue;
      for (int Xx = 0; Xx < d.nA2; ++Xx) {
        const double g2 = gAA(d, gA, U, Xx);
        if (g2 == 0.0) continue;
        for (int Uu = 0; Uu < d.nA2; ++Uu)
          dvt = fma(0.5 * g1 * g2 * eAA(d, gA, Uu, X), a.W1T[W1(d, d.nC2 + W, Xx, A, Uu)], dvt);
      }
    }
    // F7 -> d(t) at (Wa=Xa, X'=U, e, U'=X): 1/2 sum gA[Y,Wa] gA[Z,X'] eta[U',V] W1Vt[Y, Z, e, V]
    for (int Y = 0; Y < d.nA2; ++Y) {
      const double g1 = gAA(d, gA, Y, Xa);
      if (g1 == 0.0) continue;
      for (int Z = 0; Z < d.nA2; ++Z) {
        const double g2 = gAA(d, gA, Z, U);
        if (g2 == 0.0) continue;
        for (int V = 0; V < d.nA2; ++V)
          dt = fma(0.5 * g1 * g2 * eAA(d, gA, X, V), a.W1Vt[W1(d, d.nC2 + Y, Z, A, V)], dt);
      }
    }
  }
  if (!Iact && !Avir) {
    // C: -1/2 vt[M, Y=U, U'=A, V=X] t1[M, X'] lam[A, X, X', U]
    for (int Xx = 0; Xx < d.nA2; ++Xx)
      dvt = fma(-0.5 * a.t1[(size_t)I * d.nP2 + Xx], lam[LM(d, A, X, Xx, U)], dvt);
    // F8: vt[M, W=U, V'=A, Y=X]: 1/2 sum gA[W,Z] eta[U',V'] eta[X',Y] W1T[M, Z, U', X']
    for (int Z = 0; Z < d.nA2; ++Z) {
      const double g = gAA(d, gA, U, Z);
      if (g == 0.0) continue;
      for (int Uu = 0; Uu < d.nA2; ++Uu)
        for (int Xx = 0; Xx < d.nA2; ++Xx)
          dvt = fma(0.5 * g * eAA(d, gA, Uu, A) * eAA(d, gA, Xx, X), a.W1T[W1(d, I, Z, Uu, Xx)], dvt);
    }
    // F8 -> d(t) at (M, Z=U, U'=A, X'=X): 1/2 sum gA[W,Z] eta[U',V'] eta[X',Y] W1Vt[M, W, V', Y]
    for (int W = 0; W < d.nA2; ++W) {
      const double g = gAA(d, gA, W, U);
      if (g == 0.0) continue;
      for (int V = 0; V < d.nA2; ++V)
        for (int Y = 0; Y < d.nA2; ++Y)
          dt = fma(0.5 * g * eAA(d, gA, A, V) * eAA(d, gA, X, Y), a.W1Vt[W1(d, I, W, V, Y)], dt);
    }
  }
  if (a.lam3 && !Iact && !Avir) {
    // J = 1/4 vt[M,Z,U',V] t[M,W,X',Y] lam3[U',V,W,X',Y,Z]
    //  -> d(vt) at (M=I, Z=U, U'=A, V=X); d(t) at (M=I, W=U, X'=A, Y=X)
    const int n2 = d.nA2;
    for (int W = 0; W < n2; ++W)
      for (int Xx = 0; Xx < n2; ++Xx) {
        const int sy = (I & 1) + (W & 1) - (Xx & 1);  // <I W||X' Y> conserves spin
        if (sy < 0 || sy > 1) continue;
        for (int y = 0; y < d.nA2 / 2; ++y) {
          const int Y = 2 * y + sy;
          dvt = fma(0.25 * a.W1T[W1(d, I, W, Xx, Y)], a.lam3[L3I(n2, A, X, W, Xx, Y, U)], dvt);
        }
      }
    for (int Z = 0; Z < n2; ++Z)
      for (int Up = 0; Up < n2; ++Up) {
        const int sv = (I & 1) + (Z & 1) - (Up & 1);  // <I Z||U' V> conserves spin
        if (sv < 0 || sv > 1) continue;
        for (int v = 0; v < d.nA2 / 2; ++v) {
          const int V = 2 * v + sv;
          dt = fma(0.25 * a.W1Vt[W1(d, I, Z, Up, V)], a.lam3[L3I(n2, Up, V, U, A, X, Z)], dt);
        }
      }
  }
  if (a.lam3 && Iact && Avir) {
    // K = -1/4 vt[C2+X',Y,E,W] t[C2+U',V,E,Z] lam3[U',V,W,X',Y,Z]
    //  -> d(vt) at (X'=Ia, Y=U, E=A, W=X); d(t) at (U'=Ia, V=U, E=A, Z=X)
    const int n2 = d.nA2, Ia = I - d.nC2;
    for (int Up = 0; Up < n2; ++Up)
      for (int Vv = 0; Vv < n2; ++Vv) {
        const int sz = (Up & 1) + (Vv & 1) - (A & 1);  // <U' V||E Z> conserves spin
        if (sz < 0 || sz > 1) continue;
        for (int zz = 0; zz < d.nA2 / 2; ++zz) {
          const int Z = 2 * zz + sz;
          dvt = fma(-0.25 * a.W1T[W1(d, d.nC2 + Up, Vv, A, Z)], a.lam3[L3I(n2, Up, Vv, X, Ia, U, Z)],
                    dvt);
        }
      }
    for (int Xp = 0; Xp < n2; ++Xp)
      for (int Yp = 0; Yp < n2; ++Yp) {
        const int sw = (Xp & 1) + (Yp & 1) - (A & 1);  // <X' Y||E W> conserves spin
        if (sw < 0 || sw > 1) continue;
        for (int ww = 0; ww < d.nA2 / 2; ++ww) {
          const int W = 2 * ww + sw;
          dt = fma(-0.25 * a.W1Vt[W1(d, d.nC2 + Xp, Yp, A, W)], a.lam3[L3I(n2, Ia, U, W, Xp, Yp, X)],
                   dt);
        }
      }
  }
  if (!Iact && Avir) {
    // F6: vt[M, X'=U, e, V'=X]: sum gA[X',Y] eta[U',V'] W1T[M, Y, e, U']
    for (int Y = 0; Y < d.nA2; ++Y) {
      const double g = gAA(d, gA, U, Y);
      if (g == 0.0) continue;
      for (int Uu = 0; Uu < d.nA2; ++Uu)
        dvt = fma(g * eAA(d, gA, Uu, X), a.W1T[W1(d, I, Y, A, Uu)], dvt);
    }
    // F6 -> d(t) at (M, Y=U, e, U'=X): sum gA[X',Y] eta[U',V'] W1Vt[M, X', e, V']
    for (int Xx = 0; Xx < d.nA2; ++Xx) {
      const double g = gAA(d, gA, Xx, U);
      if (g == 0.0) continue;
      for (int V = 0; V < d.nA2; ++V) dt = fma(g * eAA(d, gA, X, V), a.W1Vt[W1(d, I, Xx, A, V)], dt);
    }
  }
  a.dW1Vt[k] = dvt;
  a.dW1T[k] = dt;
  a.dTi[k] = dti;
}

// (A2) term adjoints on W2-shaped tables (E, H, F5).
__global__ void adj_w2_terms_kernel(ActAdjArgs a) {
  const AD d = adims(a.z);
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.w2n) return;
  const int Y = (int)(k % d.nA2);
  const int X = (int)((k / d.nA2) % d.nA2);
  const int J = (int)((k / ((size_t)d.nA2 * d.nA2)) % d.nH2);
  const int I = (int)(k / ((size_t)d.nA2 * d.nA2 * d.nH2));
  const double* lam = a.lam;
  const double* gA = a.gA;
  double dvt = 0.0, dt = 0.0;
  // H: vt[K=I, L=J, U=X, V=Y] * Th[K,L,X',Y'] lam[U,V,X',Y'] / 8
  {
    const int i0 = (I < d.nC2) ? I : d.nC2, i1 = (I < d.nC2) ? I + 1 : d.nH2;
    const int j0 = (J < d.nC2) ? J : d.nC2, j1 = (J < d.nC2) ? J + 1 : d.nH2;
    for (int Xx = 0; Xx < d.nA2; ++Xx)
      for (int Yy = 0; Yy < d.nA2; ++Yy) {
        double th = 0.0;
        for (int I2 = i0; I2 < i1; ++I2)
          for (int J2 = j0; J2 < j1; ++J2)
            th = fma(gH(d, gA, I, I2) * gH(d, gA, J, J2), a.W2T[W2(d, I2, J2, Xx, Yy)], th);
        dvt = fma(0.125 * th, lam[LM(d, X, Y, Xx, Yy)], dvt);
      }
    // H -> d(t) at (I'=I, J'=J, X'=X, Y'=Y): sum_{K,L} gamma[K,I] gamma[L,J] dTh[K,L,X,Y]
    for (int K = i0; K < i1; ++K)
      for (int L = j0; L < j1; ++L) {
        const double gg = gH(d, gA, K, I) * gH(d, gA, L, J);
        if (gg == 0.0) continue;
        double dth = 0.0;
        for (int U = 0; U < d.nA2; ++U)
          for (int V = 0; V < d.nA2; ++V) dth = fma(a.W2Vt[W2(d, K, L, U, V)], lam[LM(d, U, V, X, Y)], dth);
        dt = fma(0.125 * gg, dth, dt);
      }
  }
  // E: -1/2 ft[M, V] t[U, M, X, Y] lam[U,V,X,Y]  (I active hole U, J core M)
  if (I >= d.nC2 && J < d.nC2) {
    const int Ua = I - d.nC2;
    for (int V = 0; V < d.nA2; ++V)
      dt = fma(-0.5 * a.ft[(size_t)J * d.nP2 + V], lam[LM(d, Ua, V, X, Y)], dt);
  }
  // F5: 1/4 vt[M,N,V,Y] t[M,N,U,X] eta[U,V] eta[X,Y] (both core)
  if (I < d.nC2 && J < d.nC2) {
    for (int U = 0; U < d.nA2; ++U)
      for (int Xx = 0; Xx < d.nA2; ++Xx)
        dvt = fma(0.25 * eAA(d, gA, U, X) * eAA(d, gA, Xx, Y), a.W2T[W2(d, I, J, U, Xx)], dvt);
    for (int V = 0; V < d.nA2; ++V)
      for (int Yy = 0; Yy < d.nA2; ++Yy)
        dt = fma(0.25 * eAA(d, gA, X, V) * eAA(d, gA, Y, Yy), a.W2Vt[W2(d, I, J, V, Yy)], dt);
  }
  a.dW2Vt[k] = dvt;
  a.dW2T[k] = dt;
}

// (A3) term adjoints on t1 and ft ([2nH][2nP]) from terms A-E.
__global__ void adj_t1ft_terms_kernel(ActAdjArgs a) {
  const AD d = adims(a.z);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.nH2 * d.nP2) return;
  const int I = k / d.nP2, A = k % d.nP2;
  const double* lam = a.lam;
  const double* gA = a.gA;
  double dt1 = 0.0, dft = 0.0;
  // A: dft[I,A] = sum_J gamma[J,I] te[J,A], te[J,A] = sum_A' eta[A',A] t1[J,A']
  //    dt1[I,A] = sum_B eta[A,B] gf[I,B], gf[I,B] = sum_K gamma[I,K] ft[K,B]
  {
    const int j0 = (I < d.nC2) ? I : d.nC2, j1 = (I < d.nC2) ? I + 1 : d.nH2;
    const int b0 = (A < d.nA2) ? 0 : A, b1 = (A < d.nA2) ? d.nA2 : A + 1;
    for (int J = j0; J < j1; ++J) {
      const double g = gH(d, gA, J, I);
      if (g == 0.0) continue;
      double te = 0.0;
      for (int Ap = b0; Ap < b1; ++Ap) te = fma(eP(d, gA, Ap, A), a.t1[(size_t)J * d.nP2 + Ap], te);
      dft = fma(g, te, dft);
    }
    for (int Bp = b0; Bp < b1; ++Bp) {
      const double e = eP(d, gA, A, Bp);
      if (e == 0.0) continue;
      double gf = 0.0;
      for (int K = j0; K < j1; ++K) gf = fma(gH(d, gA, I, K), a.ft[(size_t)K * d.nP2 + Bp], gf);
      dt1 = fma(e, gf, dt1);
    }
  }
  if (I >= d.nC2 && A >= d.nA2) {
    const int Ua = I - d.nC2;
    // B: dt1[Ua, e] = 1/2 sum vt[X, Y, e, V] lam[Ua, V, X, Y]
    for (int X = 0; X < d.nA2; ++X)
      for (int Y = 0; Y < d.nA2; ++Y)
        for (int V = 0; V < d.nA2; ++V)
          dt1 = fma(0.5 * a.W1Vt[W1(d, d.nC2 + X, Y, A, V)], lam[LM(d, Ua, V, X, Y)], dt1);
    // D: dft[Xa, e] = 1/2 sum t[U, V, e, Y] lam[U, V, Xa, Y]
    for (int U = 0; U < d.nA2; ++U)
      for (int V = 0; V < d.nA2; ++V)
        for (int Y = 0; Y < d.nA2; ++Y)
          dft = fma(0.5 * a.W1T[W1(d, d.nC2 + U, V, A, Y)], lam[LM(d, U, V, Ua, Y)], dft);
  }
  if (I < d.nC2 && A < d.nA2) {
    // C: dt1[M, X] = -1/2 sum vt[M, Y, U, V] lam[U, V, X, Y]
    for (int Y = 0; Y < d.nA2; ++Y)
      for (int U = 0; U < d.nA2; ++U)
        for (int V = 0; V < d.nA2; ++V)
          dt1 = fma(-0.5 * a.W1Vt[W1(d, I, Y, U, V)], lam[LM(d, U, V, A, Y)], dt1);
    // E: dft[M, V] = -1/2 sum t[U, M, X, Y] lam[U, V, X, Y]
    for (int U = 0; U < d.nA2; ++U)
      for (int X = 0; X < d.nA2; ++X)
        for (int Y = 0; Y < d.nA2; ++Y)
          dft = fma(-0.5 * a.W2T[W2(d, d.nC2 + U, I, X, Y)], lam[LM(d, U, A, X, Y)], dft);
  }
  a.dt1[k] = dt1;
  a.dft[k] = dft;
}

// (A4) adjoint of P1, P2 from terms G (two virtual particles) and F4.
__global__ void adj_p12_kernel(ActAdjArgs a) {
  const AD d = adims(a.z);
  const int nA = a.z.nA, nA4 = nA * nA * nA * nA;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nA4) return;
  const int p3 = c % nA, p2 = (c / nA) % nA, p1 = (c / (nA * nA)) % nA, p0 = c / (nA * nA * nA);
  double d1 = 0.0, d2 = 0.0;
  for (int sg = 0; sg < 16; ++sg) {
    const int s0 = sg & 1, s1 = (sg >> 1) & 1, s2 = (sg >> 2) & 1, s3 = (sg >> 3) & 1;
    const int A0 = 2 * p0 + s0, A1 = 2 * p1 + s1, A2 = 2 * p2 + s2, A3 = 2 * p3 + s3;
    // G: 1/8 lam[U,V,X,Y] S[(X,Y),(U,V)] with (X,Y,U,V) = (A0,A1,A2,A3)
    const double lg = a.lam[LM(d, A2, A3, A0, A1)];
    if (s0 == s2 && s1 == s3) d1 += 0.25 * lg;
    if (s0 == s3 && s1 == s2) d2 -= 0.25 * lg;
    // F4: 1/4 gA[X,Y] gA[U,V] S[(X,U),(Y,V)] with (X,U,Y,V) = (A0,A1,A2,A3)
    const double gg = gAA(d, a.gA, A0, A2) * gAA(d, a.gA, A1, A3);
    if (s0 == s2 && s1 == s3) d1 += 0.5 * gg;
    if (s0 == s3 && s1 == s2) d2 -= 0.5 * gg;
  }
  a.dP12[c] = d1;
  a.dP12[nA4 + c] = d2;
}

// (B1) t1/ft -> S, with the eps and s dependence of their regulators.
// Per-block accumulation of the eps / s derivatives: entries 0..n-1 of the
// shared array are the orbitals, entry n is s. These kernels touch few distinct
// orbitals per block (often the few active ones in every thread), and direct
// global atomics on those addresses serialised them; the block adds in shared
// memory and flushes one global atomic per non-zero entry.
__device__ __forceinline__ void dacc_init(double* sh, int n) {
  for (int k = threadIdx.x; k <= n; k += blockDim.x) sh[k] = 0.0;
  __syncthreads();
}
__device__ __forceinline__ void dacc_flush(const double* sh, int n, double* deps, double* ds) {
  __syncthreads();
  for (int k = threadIdx.x; k < n; k += blockDim.x)
    if (sh[k] != 0.0) atomicAdd(&deps[k], sh[k]);
  if (threadIdx.x == 0 && sh[n] != 0.0) atomicAdd(ds, sh[n]);
}

__device__ __forceinline__ void adj_t1_chain_kernel_body(ActAdjArgs a, double* sacc_) {
  const AD d = adims(a.z);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.nH2 * d.nP2) return;
  const int I = k / d.nP2, A = k % d.nP2;
  const Sizes& z = a.z;
  double S = 0.0;
  for (int U = 0; U < d.nA2; ++U)
    for (int X = 0; X < d.nA2; ++X) {
      const double g = a.gA[U * d.nA2 + X];
      if (g == 0.0) continue;
      S = fma((a.eps[z.nC + (X >> 1)] - a.eps[z.nC + (U >> 1)]) * g, a.W1T[W1(d, I, U, A, X)], S);
    }
  const double D1 = a.eps[I >> 1] - a.eps[z.nC + (A >> 1)];
  const bool internal = (I >= d.nC2) && (A < d.nA2);
  const RegD rt = rt_d(D1, a.s);
  const double ex = exp(-a.s * D1 * D1);
  const double dt1 = internal ? 0.0 : a.dt1[k];
  const double dft = a.dft[k];
  a.dS[k] = dt1 * rt.v + dft * ex;
  // t1 = (F + S) Rt(D1), ft = F (1 + e^{-s D1^2}) + S e^{-s D1^2}: both regulators
  // multiply F + S
  const double F = (a.f1 && !internal && (I & 1) == (A & 1))
                       ? a.f1[(size_t)(I >> 1) * z.nP + (A >> 1)]
                       : 0.0;
  const double FS = F + S;
  const double dD = FS * (dt1 * rt.dD + dft * (-2.0 * a.s * D1 * ex));
  const double dss = FS * (dt1 * rt.ds + dft * (-D1 * D1 * ex));
  if (dD != 0.0) {
    atomicAdd(&sacc_[I >> 1], dD);
    atomicAdd(&sacc_[z.nC + (A >> 1)], -dD);
  }
  if (dss != 0.0) atomicAdd(&sacc_[a.z.n], dss);
}

__global__ void adj_t1_chain_kernel(ActAdjArgs a) {
  extern __shared__ double sacc_[];
  dacc_init(sacc_, a.z.n);
  adj_t1_chain_kernel_body(a, sacc_);
  dacc_flush(sacc_, a.z.n, a.deps, a.ds);
}

// (B2) W1: total d(t) (direct + via Ti + via S), then through the regulators to d(V).
__device__ __forceinline__ void adj_w1_chain_kernel_body(ActAdjArgs a, double* sacc_) {
  const AD d = adims(a.z);
  const Sizes& z = a.z;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.w1n) return;
  const int X = (int)(k % d.nA2);
  const int A = (int)((k / d.nA2) % d.nP2);
  const int U = (int)((k / ((size_t)d.nA2 * d.nP2)) % d.nA2);
  const int I = (int)(k / ((size_t)d.nA2 * d.nP2 * d.nA2));
  double dt = a.dW1T[k];
  // via Ti[J][U][Bp][X] = sum_{I,A} gamma[J,I] eta[A,Bp] T[I,U,A,X]
  {
    const int j0 = (I < d.nC2) ? I : d.nC2, j1 = (I < d.nC2) ? I + 1 : d.nH2;
    const int b0 = (A < d.nA2) ? 0 : A, b1 = (A < d.nA2) ? d.nA2 : A + 1;
    for (int J = j0; J < j1; ++J) {
      const double g = gH(d, a.gA, J, I);
      if (g == 0.0) continue;
      for (int Bp = b0; Bp < b1; ++Bp) dt = fma(g * eP(d, a.gA, A, Bp), a.dTi[W1(d, J, U, Bp, X)], dt);
    }
  }
  // via S[I,A] = sum (e_X - e_U) gamma[U][X] T[I,U,A,X]
  const double gux = a.gA[U * d.nA2 + X];
  const double eX = a.eps[z.nC + (X >> 1)], eU = a.eps[z.nC + (U >> 1)];
  const double dS = a.dS[(size_t)I * d.nP2 + A];
  dt = fma(dS * (eX - eU), gux, dt);
  const double T = a.W1T[k];
  if (gux != 0.0 && dS != 0.0 && T != 0.0) {
    atomicAdd(&sacc_[z.nC + (X >> 1)], dS * gux * T);
    atomicAdd(&sacc_[z.nC + (U >> 1)], -dS * gux * T);
  }
  // regulators: T = V Rt(D) (zero if internal), Vt = V Rv(D)
  const double V = a.W1V[k];
  const double D = a.eps[I >> 1] + a.eps[z.nC + (U >> 1)] - a.eps[z.nC + (A >> 1)] - eX;
  const bool internal = (I >= d.nC2) && (A < d.nA2);
  const RegD rt = rt_d(D, a.s), rv = rv_d(D, a.s);
  const double dvt = a.dW1Vt[k];
  const double dtt = internal ? 0.0 : dt;
  a.dV1[k] = dtt * rt.v + dvt * rv.v;
  const double dD = V * (dtt * rt.dD + dvt * rv.dD);
  const double dss = V * (dtt * rt.ds + dvt * rv.ds);
  if (dD != 0.0) {
    atomicAdd(&sacc_[I >> 1], dD);
    atomicAdd(&sacc_[z.nC + (U >> 1)], dD);
    atomicAdd(&sacc_[z.nC + (A >> 1)], -dD);
    atomicAdd(&sacc_[z.nC + (X >> 1)], -dD);
  }
  if (dss != 0.0) atomicAdd(&sacc_[a.z.n], dss);
}

__global__ void adj_w1_chain_kernel(ActAdjArgs a) {
  extern __shared__ double sacc_[];
  dacc_init(sacc_, a.z.n);
  adj_w1_chain_kernel_body(a, sacc_);
  dacc_flush(sacc_, a.z.n, a.deps, a.ds);
}

// (B3) W2 through its regulators to d(V).
__device__ __forceinline__ void adj_w2_chain_kernel_body(ActAdjArgs a, double* sacc_) {
  const AD d = adims(a.z);
  const Sizes& z = a.z;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.w2n) return;
  const int Y = (int)(k % d.nA2);
  const int X = (int)((k / d.nA2) % d.nA2);
  const int J = (int)((k / ((size_t)d.nA2 * d.nA2)) % d.nH2);
  const int I = (int)(k / ((size_t)d.nA2 * d.nA2 * d.nH2));
  const double V = a.W2V[k];
  const double D = a.eps[I >> 1] + a.eps[J >> 1] - a.eps[z.nC + (X >> 1)] - a.eps[z.nC + (Y >> 1)];
  const bool internal = (I >= d.nC2) && (J >= d.nC2);
  const RegD rt = rt_d(D, a.s), rv = rv_d(D, a.s);
  const double dt = internal ? 0.0 : a.dW2T[k];
  const double dvt = a.dW2Vt[k];
  a.dV2[k] = dt * rt.v + dvt * rv.v;
  const double dD = V * (dt * rt.dD + dvt * rv.dD);
  const double dss = V * (dt * rt.ds + dvt * rv.ds);
  if (dD != 0.0) {
    atomicAdd(&sacc_[I >> 1], dD);
    atomicAdd(&sacc_[J >> 1], dD);
    atomicAdd(&sacc_[z.nC + (X >> 1)], -dD);
    atomicAdd(&sacc_[z.nC + (Y >> 1)], -dD);
  }
  if (dss != 0.0) atomicAdd(&sacc_[a.z.n], dss);
}

__global__ void adj_w2_chain_kernel(ActAdjArgs a) {
  extern __shared__ double sacc_[];
  dacc_init(sacc_, a.z.n);
  adj_w2_chain_kernel_body(a, sacc_);
  dacc_flush(sacc_, a.z.n, a.deps, a.ds);
}

// (B4) spin sums back to the spatial integrals K1, K2 (from W1) and K3 (from W2).
__global__ void adj_k_kernel(ActAdjArgs a) {
  const AD d = adims(a.z);
  const Sizes& z = a.z;
  const size_t n12 = (size_t)z.nH * z.nA * z.nA * z.nP;
  const size_t n3 = (size_t)z.nH * z.nA * z.nH * z.nA;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n12) {
    const int ap = (int)(k % z.nP);
    const int x = (int)((k / z.nP) % z.nA);
    const int u = (int)((k / ((size_t)z.nP * z.nA)) % z.nA);
    const int i = (int)(k / ((size_t)z.nP * z.nA * z.nA));
    double d1 = 0.0, d2 = 0.0;
    for (int sg = 0; sg < 16; ++sg) {
      const int si = sg & 1, su = (sg >> 1) & 1, sa = (sg >> 2) & 1, sx = (sg >> 3) & 1;
      const double g = a.dV1[W1(d, 2 * i + si, 2 * u + su, 2 * ap + sa, 2 * x + sx)];
      if (si == sa && su == sx) d1 += g;
      if (si == sx && su == sa) d2 -= g;
    }
    a.dK1[k] = d1;
    a.dK2[k] = d2;
  } else if (k < n12 + n3) {
    const size_t r = k - n12;
    const int y = (int)(r % z.nA);
    const int j = (int)((r / z.nA) % z.nH);
    const int x = (int)((r / ((size_t)z.nA * z.nH)) % z.nA);
    const int i = (int)(r / ((size_t)z.nA * z.nH * z.nA));
    double d3 = 0.0;
    for (int sg = 0; sg < 16; ++sg) {
      const int si = sg & 1, sj = (sg >> 1) & 1, s1 = (sg >> 2) & 1, s2 = (sg >> 3) & 1;
      // coulomb (ix|jy) of <IJ||XY> with X = (x, s1), Y = (y, s2)
      if (si == s1 && sj == s2) d3 += a.dV2[W2(d, 2 * i + si, 2 * j + sj, 2 * x + s1, 2 * y + s2)];
      // exchange -(ix|jy) of <IJ||X'Y'> with X' = (y, s1), Y' = (x, s2): -(iY'|jX')
      if (si == s2 && sj == s1) d3 -= a.dV2[W2(d, 2 * i + si, 2 * j + sj, 2 * y + s1, 2 * x + s2)];
    }
    a.dK3[r] = d3;
  }
}

// (B5) adjoint of P1/P2 -> dM[x][u][e][f] (one thread per virtual pair (e,f)), eps, s.
template <int NA>
__device__ __forceinline__ void adj_m_kernel_body(ActAdjArgs a, const double* __restrict__ dP12, double* sacc_) {
  const Sizes& z = a.z;
  const size_t nV2 = (size_t)z.nV * z.nV;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nV2) return;
  const int e = (int)(k / z.nV), f = (int)(k % z.nV);
  constexpr int NA2 = NA * NA, NA4 = NA2 * NA2;
  const int ve = z.nC + z.nA;
  const double ef = a.eps[ve + e] + a.eps[ve + f];
  double m[NA2], dm[NA2], dDp[NA2];
  RegD rv[NA2], rt[NA2];
#pragma unroll
  for (int p = 0; p < NA2; ++p) {
    m[p] = a.M[(size_t)p * nV2 + k];
    dm[p] = 0.0;
    dDp[p] = 0.0;
    const double D = a.eps[z.nC + p / NA] + a.eps[z.nC + p % NA] - ef;
    rv[p] = rv_d(D, a.s);
    rt[p] = rt_d(D, a.s);
  }
  double dss = 0.0;
#pragma unroll
  for (int p = 0; p < NA2; ++p) {        // p = (x, u)
#pragma unroll
    for (int q = 0; q < NA2; ++q) {      // q = (y, v)
      const int qt = (q % NA) * NA + q / NA;  // (v, y)
      const double d1 = dP12[p * NA2 + q], d2 = dP12[NA4 + p * NA2 + q];
      const double R = rv[p].v * rt[q].v;
      dm[p] += (d1 * m[q] + d2 * m[qt]) * R;
      dm[q] += d1 * m[p] * R;
      dm[qt] += d2 * m[p] * R;
      const double dR = m[p] * (d1 * m[q] + d2 * m[qt]);
      dDp[p] += dR * rv[p].dD * rt[q].v;
      dDp[q] += dR * rv[p].v * rt[q].dD;
      dss += dR * (rv[p].ds * rt[q].v + rv[p].v * rt[q].ds);
    }
  }
  double dsum = 0.0;
#pragma unroll
  for (int p = 0; p < NA2; ++p) {
    a.dM[(size_t)p * nV2 + k] = dm[p];
    dsum += dDp[p];
    if (dDp[p] != 0.0) {
      atomicAdd(&sacc_[z.nC + p / NA], dDp[p]);
      atomicAdd(&sacc_[z.nC + p % NA], dDp[p]);
    }
  }
  if (dsum != 0.0) {
    atomicAdd(&sacc_[ve + e], -dsum);
    atomicAdd(&sacc_[ve + f], -dsum);
  }
  if (dss != 0.0) atomicAdd(&sacc_[a.z.n], dss);
}

template <int NA>
__global__ void adj_m_kernel(ActAdjArgs a, const double* __restrict__ dP12) {
  extern __shared__ double sacc_[];
  dacc_init(sacc_, a.z.n);
  adj_m_kernel_body<NA>(a, dP12, sacc_);
  dacc_flush(sacc_, a.z.n, a.deps, a.ds);
}

// (B6) dK1, dK2, dK3 -> dB (gather, one thread per dB element; adds).
__global__ void adj_k_to_b_kernel(ActAdjArgs a, const double* __restrict__ B, double* __restrict__ dB) {
  const Sizes& z = a.z;
  const size_t n = (size_t)z.Q * z.nH * z.nP;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int p = (int)(k % z.nP);
  const int h = (int)((k / z.nP) % z.nH);
  const int q = (int)(k / ((size_t)z.nP * z.nH));
  auto K1i = [&](int i, int u, int x, int ap) { return (((size_t)i * z.nA + u) * z.nA + x) * z.nP + ap; };
  auto K3i = [&](int i, int x, int j, int y) { return (((size_t)i * z.nA + x) * z.nH + j) * z.nA + y; };
  double acc = 0.0;
  // K1[i,u,x,a] = sum_Q B[Q,i,a] B[Q,nC+u,x]
  for (int u = 0; u < z.nA; ++u)
    for (int x = 0; x < z.nA; ++x) acc = fma(a.dK1[K1i(h, u, x, p)], B[bidx(z, q, z.nC + u, x)], acc);
  if (h >= z.nC && p < z.nA) {
    const int u = h - z.nC, x = p;
    for (int i = 0; i < z.nH; ++i)
      for (int ap = 0; ap < z.nP; ++ap) acc = fma(a.dK1[K1i(i, u, x, ap)], B[bidx(z, q, i, ap)], acc);
  }
  // K2[i,u,x,a] = sum_Q B[Q,i,x] B[Q,nC+u,a]
  if (p < z.nA) {
    const int x = p;
    for (int u = 0; u < z.nA; ++u)
      for (int ap = 0; ap < z.nP; ++ap)
        acc = fma(a.dK2[K1i(h, u, x, ap)], B[bidx(z, q, z.nC + u, ap)], acc);
  }
  if (h >= z.nC) {
    const int u = h - z.nC;
    for (int i = 0; i < z.nH; ++i)
      for (int x = 0; x < z.nA; ++x) acc = fma(a.dK2[K1i(i, u, x, p)], B[bidx(z, q, i, x)], acc);
  }
  // K3[i,x,j,y] = sum_Q B[Q,i,x] B[Q,j,y]
  if (p < z.nA) {
    for (int j = 0; j < z.nH; ++j)
      for (int y = 0; y < z.nA; ++y) {
        acc = fma(a.dK3[K3i(h, p, j, y)], B[bidx(z, q, j, y)], acc);
        acc = fma(a.dK3[K3i(j, y, h, p)], B[bidx(z, q, j, y)], acc);
      }
  }
  dB[k] += acc;
}

}  // namespace dsrg

namespace dsrg {

// Generic-nA fallback of adj_m_kernel for active spaces above 4 orbitals.
__device__ __forceinline__ void adj_m_generic_kernel_body(ActAdjArgs a, const double* __restrict__ dP12, double* sacc_) {
  const Sizes& z = a.z;
  const int NA = z.nA, NA2 = NA * NA, NA4 = NA2 * NA2;
  const size_t nV2 = (size_t)z.nV * z.nV;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nV2) return;
  const int e = (int)(k / z.nV), f = (int)(k % z.nV);
  const int ve = z.nC + z.nA;
  const double ef = a.eps[ve + e] + a.eps[ve + f];
  double dsum = 0.0, dss = 0.0;
  for (int p = 0; p < NA2; ++p) {
    const double mp = a.M[(size_t)p * nV2 + k];
    const RegD rvp = rv_d(a.eps[z.nC + p / NA] + a.eps[z.nC + p % NA] - ef, a.s);
    const RegD rtp = rt_d(a.eps[z.nC + p / NA] + a.eps[z.nC + p % NA] - ef, a.s);
    double dm = 0.0, dDp = 0.0;
    for (int q = 0; q < NA2; ++q) {
      const int qt = (q % NA) * NA + q / NA;
      const double mq = a.M[(size_t)q * nV2 + k], mqt = a.M[(size_t)qt * nV2 + k];
      const RegD rvq = rv_d(a.eps[z.nC + q / NA] + a.eps[z.nC + q % NA] - ef, a.s);
      const RegD rtq = rt_d(a.eps[z.nC + q / NA] + a.eps[z.nC + q % NA] - ef, a.s);
      // p in the first slot of P1/P2
      {
        const double d1 = dP12[p * NA2 + q], d2 = dP12[NA4 + p * NA2 + q];
        dm += (d1 * mq + d2 * mqt) * rvp.v * rtq.v;
        const double dR = mp * (d1 * mq + d2 * mqt);
        dDp += dR * rvp.dD * rtq.v;
        dss += dR * (rvp.ds * rtq.v + rvp.v * rtq.ds);
      }
      // p in the second slot: P1[q, p] with M_p, and P2[q, pt] with M_p (pt = transposed p)
      {
        const double d1 = dP12[q * NA2 + p];
        dm += d1 * mq * rvq.v * rtp.v;
        dDp += d1 * mq * mp * rvq.v * rtp.dD;
        const int pt = (p % NA) * NA + p / NA;
        const double d2 = dP12[NA4 + q * NA2 + pt];
        const RegD rtpt = rt_d(a.eps[z.nC + pt / NA] + a.eps[z.nC + pt % NA] - ef, a.s);
        dm += d2 * mq * rvq.v * rtpt.v;
        const double dR2 = d2 * mq * mp;
        if (dR2 != 0.0) {
          atomicAdd(&sacc_[z.nC + pt / NA], dR2 * rvq.v * rtpt.dD);
          atomicAdd(&sacc_[z.nC + pt % NA], dR2 * rvq.v * rtpt.dD);
          dsum += dR2 * rvq.v * rtpt.dD;
        }
      }
    }
    a.dM[(size_t)p * nV2 + k] = dm;
    if (dDp != 0.0) {
      atomicAdd(&sacc_[z.nC + p / NA], dDp);
      atomicAdd(&sacc_[z.nC + p % NA], dDp);
    }
    dsum += dDp;
  }
  if (dsum != 0.0) {
    atomicAdd(&sacc_[ve + e], -dsum);
    atomicAdd(&sacc_[ve + f], -dsum);
  }
  if (dss != 0.0) atomicAdd(&sacc_[a.z.n], dss);
}

__global__ void adj_m_generic_kernel(ActAdjArgs a, const double* __restrict__ dP12) {
  extern __shared__ double sacc_[];
  dacc_init(sacc_, a.z.n);
  adj_m_generic_kernel_body(a, dP12, sacc_);
  dacc_flush(sacc_, a.z.n, a.deps, a.ds);
}


bool grad_alloc(dsrg_plan* p) {
  const Sizes& z = p->z;
  GradWs* g = new GradWs();
  p->grad = g;
  g->nVp = (z.nV + GT - 1) / GT * GT;
  g->nB = (size_t)z.Q * z.nH * z.nP;
  bool ok = true;
  if (p->prec == DSRG_PREC_FP64) {
    // as many rows as fit in 2 GiB of W (at least one)
    const size_t per_w = (size_t)z.nC * g->nVp * g->nVp * 8;
    const size_t kmax = ((size_t)2 << 30) / per_w;
    g->kgroup = (int)(kmax < 1 ? 1 : (kmax > (size_t)z.nC ? (size_t)z.nC : kmax));
    ok = plan_alloc(p, (void**)&g->Wk, per_w * g->kgroup);
  } else {
    // split plans: S and B^T planes of the tensor-core assembly (tc_adjoint.cu)
    ok = tc_adj_alloc(p);
  }
  if (z.nA > 0) {
    const size_t w1n = p->act.w1n, w2n = p->act.w2n;
    const size_t nHP2 = (size_t)4 * z.nH * z.nP;
    const size_t n12 = (size_t)z.nH * z.nA * z.nA * z.nP, n3 = (size_t)z.nH * z.nA * z.nH * z.nA;
    const size_t nA4 = (size_t)z.nA * z.nA * z.nA * z.nA;
    ok = ok && plan_alloc(p, (void**)&g->dX, (size_t)z.nC * z.nA * z.nV * z.nV * 8) &&
         plan_alloc(p, (void**)&g->dZ, (size_t)z.nA * z.nC * z.nC * z.nV * 8) &&
         plan_alloc(p, (void**)&g->dW1Vt, w1n * 8) && plan_alloc(p, (void**)&g->dW1T, w1n * 8) &&
         plan_alloc(p, (void**)&g->dTi, w1n * 8) && plan_alloc(p, (void**)&g->dV1, w1n * 8) &&
         plan_alloc(p, (void**)&g->dW2Vt, w2n * 8) && plan_alloc(p, (void**)&g->dW2T, w2n * 8) &&
         plan_alloc(p, (void**)&g->dV2, w2n * 8) && plan_alloc(p, (void**)&g->dt1, nHP2 * 8) &&
         plan_alloc(p, (void**)&g->dft, nHP2 * 8) && plan_alloc(p, (void**)&g->dS, nHP2 * 8) &&
         plan_alloc(p, (void**)&g->dP12, 2 * nA4 * 8) && plan_alloc(p, (void**)&g->dK1, n12 * 8) &&
         plan_alloc(p, (void**)&g->dK2, n12 * 8) && plan_alloc(p, (void**)&g->dK3, n3 * 8) &&
         plan_alloc(p, (void**)&g->dM, (size_t)z.nA * z.nA * z.nV * z.nV * 8);
  }
  return ok;
}

void grad_free(dsrg_plan* p) {
  delete p->grad;
  p->grad = nullptr;
  tc_adj_free(p);
}

GemmArgs mk(int M, int N, int L1, int L2, const double* A, long long ai, long long a1,
                   long long a2, const double* Bm, long long b1, long long b2, long long bj,
                   double* C, long long ci, long long cj, double alpha) {
  GemmArgs g;
  g.M = M; g.N = N; g.L1 = L1; g.L2 = L2;
  g.A = A; g.ai = ai; g.a1 = a1; g.a2 = a2;
  g.Bm = Bm; g.b1 = b1; g.b2 = b2; g.bj = bj;
  g.C = C; g.ci = ci; g.cj = cj;
  g.alpha = alpha;
  g.accumulate = 1;
  g.nb = 1;
  g.sa = g.sb = g.sc = 0;
  g.A32 = g.B32 = nullptr;
  return g;
}

// The same GEMM for nb problems whose A, Bm, C start sa, sb, sc elements apart.
GemmArgs batched(GemmArgs g, int nb, long long sa, long long sb, long long sc) {
  g.nb = nb;
  g.sa = sa;
  g.sb = sb;
  g.sc = sc;
  return g;
}

static size_t ccav_adj_smem(const Sizes& z) {
  return sizeof(double) * ((size_t)z.nA * z.nC * z.nC + 8 * (size_t)z.nC * (1 + z.nA) + z.nC + z.nA);
}

// Gradient of E_total (the energy itself must have been computed on the same
// stream just before: the active-block tables of the forward pass are reused).
// Term A with no active orbitals (f^(1) singles): E = 2 sum_{m,e} f^2 (1 + g) Rt,
// g = exp(-s D^2), D = e_m - e_e; its eps and s derivatives (f^(1) is an input
// of its own, B does not enter).
__device__ __forceinline__ void singles_adj_kernel_body(const double* __restrict__ eps, double s, Sizes z,
                                   const double* __restrict__ f1, double* __restrict__ deps,
                                   double* __restrict__ ds, double* sacc_) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= z.nC * z.nP) return;
  const int m = k / z.nP, e = k % z.nP;
  const double f = f1[k];
  const double D = eps[m] - eps[z.nC + e];
  const RegD rt = rt_d(D, s);
  const double g = exp(-s * D * D);
  const double w = 2.0 * f * f;
  const double dD = w * ((-2.0 * s * D * g) * rt.v + (1.0 + g) * rt.dD);
  const double dss = w * ((-D * D * g) * rt.v + (1.0 + g) * rt.ds);
  if (dD != 0.0) {
    atomicAdd(&sacc_[m], dD);
    atomicAdd(&sacc_[z.nC + e], -dD);
  }
  if (dss != 0.0) atomicAdd(&sacc_[z.n], dss);
}

__global__ void singles_adj_kernel(const double* __restrict__ eps, double s, Sizes z,
                                   const double* __restrict__ f1, double* __restrict__ deps,
                                   double* __restrict__ ds) {
  extern __shared__ double sacc_[];
  dacc_init(sacc_, z.n);
  singles_adj_kernel_body(eps, s, z, f1, deps, ds, sacc_);
  dacc_flush(sacc_, z.n, deps, ds);
}

cudaError_t launch_grad(dsrg_plan* p, const double* B, const double* eps, const double* G,
                        const double* L, const double* L3, const double* F1, double s, double* dB,
                        double* deps, double* ds) {
  (void)L;
  const Sizes& z = p->z;
  GradWs* w = p->grad;
  cudaStream_t st = p->stream;
  cudaError_t e;
  const long long HP = (long long)z.nH * z.nP;
  // FP64 plans: FP64 adjoints and GEMMs. Split plans: the adjoints of the
  // integrals, then one tensor-core GEMM of their symmetric matrix S with B^T
  // (tc_adjoint.cu), which writes every element of dB.
  const bool fp64 = p->prec == DSRG_PREC_FP64;
  if (fp64 && (e = cudaMemsetAsync(dB, 0, (size_t)z.Q * HP * 8, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(deps, 0, (size_t)z.n * 8, st)) != cudaSuccess) return e;
  if ((e = cudaMemsetAsync(ds, 0, 8, st)) != cudaSuccess) return e;
  if (!fp64) {
    // ---- F1: the core x core block of S and the eps / s derivatives (this rank's pairs)
    if ((e = tc_adj_ccvv(p, B, eps, s, deps, ds)) != cudaSuccess) return e;
    if (p->shard_rank != 0 || z.nA == 0) {
      if (p->shard_rank == 0 && F1) {
        const int n = z.nC * z.nP;
        singles_adj_kernel<<<(n + 255) / 256, 256, ((size_t)z.n + 1) * 8, st>>>(eps, s, z, F1, deps, ds);
        DSRG_LAUNCH_CHECK(p);
      }
      return tc_adj_assemble(p, B, dB);
    }
  }
  // ---- F1 (FP64 plans): per core row k, W^{kj} then dB[:, k, V] += 2 sum_j B_j W^{kj T}
  const int n_tp = p->n_tp_ccvv;  // 64-wide tile pairs of the FP64 work list
  // rows k in groups of w->kgroup: W^{kj} of the group, then one batched GEMM
  const long long nVp = w->nVp, wstride = (long long)z.nC * nVp * nVp;
  for (int k0 = 0, grp = 0; fp64 && k0 < z.nC; k0 += w->kgroup, ++grp) {
    const int kg = (z.nC - k0) < w->kgroup ? (z.nC - k0) : w->kgroup;
    // multi-GPU share: groups of core rows dealt round-robin (their dB rows are disjoint)
    if (!pair_in_shard(grp, p->shard_rank, p->shard_world)) continue;
    for (int k = k0; k < k0 + kg; ++k) {
      ccvv_adj_kernel<double><<<z.nC * n_tp, 256, 0, st>>>(B, eps, s, z, k, p->d_tp_ccvv, n_tp,
                                                           w->nVp, w->Wk + (k - k0) * wstride,
                                                           deps, ds);
      DSRG_LAUNCH_CHECK(p);
    }
    GemmArgs gw = batched(mk(z.Q, z.nV, z.nC, z.nV, B + z.nA, HP, z.nP, 1, w->Wk, nVp * nVp, 1, nVp,
                             dB + (long long)k0 * z.nP + z.nA, HP, 1, 2.0),
                          kg, 0, wstride, z.nP);
    if ((e = gemm(p, gw)) != cudaSuccess) return e;
  }
  if (p->shard_rank != 0) return cudaSuccess;  // the other blocks' adjoints: rank 0
  if (z.nA == 0) {
    if (F1) {
      const int n = z.nC * z.nP;
      singles_adj_kernel<<<(n + 255) / 256, 256, ((size_t)z.n + 1) * 8, st>>>(eps, s, z, F1, deps, ds);
      DSRG_LAUNCH_CHECK(p);
    }
    return cudaSuccess;
  }
  const long long nV = z.nV, nV2 = nV * nV;

  // ---- F2
  {
#define CAVV_ADJ(NA_)                                                                            \
  case NA_:                                                                                      \
    if (fp64)                                                                                    \
      cavv_adj_kernel<NA_, double><<<z.nC * p->n_tp_cavv, 256, 0, st>>>(                         \
          B, eps, G, s, z, p->d_tp_cavv, p->n_tp_cavv, z.nV, w->dX, deps, ds);                   \
    else                                                                                         \
      cavv_adj_kernel<NA_, float><<<z.nC * p->n_tp_cavv, 256, 0, st>>>(                          \
          B, eps, G, s, z, p->d_tp_cavv, p->n_tp_cavv, z.nV, w->dX, deps, ds);                   \
    break;
    if (!fp64 && p->rest_tc) {
      // X from the energy call's tensor-core GEMM output
      if ((e = launch_split_cavv_adjoint(p, eps, G, s, w->dX, deps, ds)) != cudaSuccess) return e;
    } else {
      switch (z.nA) {
        CAVV_ADJ(1) CAVV_ADJ(2) CAVV_ADJ(3) CAVV_ADJ(4) CAVV_ADJ(5) CAVV_ADJ(6) CAVV_ADJ(7) CAVV_ADJ(8)
        default: return cudaErrorInvalidValue;
      }
      DSRG_LAUNCH_CHECK(p);
    }
#undef CAVV_ADJ
  }
  if (fp64) {
    e = gemm(p, batched(mk(z.Q, z.nV, z.nA, z.nV, B + (long long)z.nC * z.nP + z.nA, HP, z.nP, 1,
                           w->dX, nV2, 1, nV, dB + z.nA, HP, 1, 1.0),
                        z.nC, 0, (long long)z.nA * nV2, z.nP));
    if (e != cudaSuccess) return e;
    e = gemm(p, batched(mk(z.Q, z.nV, z.nC, z.nV, B + z.nA, HP, z.nP, 1, w->dX,
                           (long long)z.nA * nV2, nV, 1, dB + (long long)z.nC * z.nP + z.nA, HP, 1,
                           1.0),
                        z.nA, 0, nV2, z.nP));
    if (e != cudaSuccess) return e;
  }
  // ---- F3
  {
    const size_t sm = ccav_adj_smem(z);
    if (fp64) {
      raise_smem_limit((const void*)ccav_adj_kernel<double>, sm);
      ccav_adj_kernel<double><<<z.nV, 256, sm, st>>>(B, eps, G, s, z, w->dZ, deps, ds);
    } else {
      raise_smem_limit((const void*)ccav_adj_kernel<float>, sm);
      ccav_adj_kernel<float><<<z.nV, 256, sm, st>>>(B, eps, G, s, z, w->dZ, deps, ds);
    }
    DSRG_LAUNCH_CHECK(p);
  }
  if (fp64) {
    const long long nCV = (long long)z.nC * nV, nCCV = (long long)z.nC * nCV;
    e = gemm(p, batched(mk(z.Q, z.nV, z.nC, z.nA, B, HP, z.nP, 1, w->dZ, nV, nCCV, 1, dB + z.nA, HP,
                           1, 1.0),
                        z.nC, 0, nCV, z.nP));
    if (e != cudaSuccess) return e;
    e = gemm(p, batched(mk(z.Q, z.nC, z.nC, z.nV, B + z.nA, HP, z.nP, 1, w->dZ, nCV, 1, nV, dB, HP,
                           z.nP, 1.0),
                        z.nA, 0, nCCV, 1));
    if (e != cudaSuccess) return e;
  }
  // ---- active block
  {
    ActiveWs& A = p->act;
    ActAdjArgs a;
    a.z = z;
    a.s = s;
    a.eps = eps;
    a.K1 = A.K1; a.K2 = A.K2; a.K3 = A.K3;
    a.W1V = A.W1; a.W1T = A.W1 + A.w1n; a.W1Vt = A.W1 + 2 * A.w1n;
    a.W2V = A.W2; a.W2T = A.W2 + A.w2n; a.W2Vt = A.W2 + 2 * A.w2n;
    a.Ti = A.Ti; a.lam = A.lam; a.gA = A.gA; a.t1 = A.t1; a.ft = A.ft; a.M = A.M;
    a.dW1Vt = w->dW1Vt; a.dW1T = w->dW1T; a.dTi = w->dTi; a.dW2Vt = w->dW2Vt; a.dW2T = w->dW2T;
    a.dt1 = w->dt1; a.dft = w->dft; a.dP12 = w->dP12; a.dS = w->dS; a.dV1 = w->dV1; a.dV2 = w->dV2;
    a.dK1 = w->dK1; a.dK2 = w->dK2; a.dK3 = w->dK3; a.dM = w->dM;
    a.deps = deps;
    a.ds = ds;
    a.w1n = A.w1n;
    a.w2n = A.w2n;
    a.lam3 = L3;
    a.f1 = F1;
    const int nHP2 = 4 * z.nH * z.nP;
    const int nA4 = z.nA * z.nA * z.nA * z.nA;
    auto blocks = [](size_t n) { return (unsigned)((n + 255) / 256); };
    const size_t dsm = ((size_t)z.n + 1) * 8;  // block sums of deps and ds
    adj_w1_terms_kernel<<<blocks(A.w1n), 256, 0, st>>>(a);
    DSRG_LAUNCH_CHECK(p);
    adj_w2_terms_kernel<<<blocks(A.w2n), 256, 0, st>>>(a);
    DSRG_LAUNCH_CHECK(p);
    adj_t1ft_terms_kernel<<<blocks(nHP2), 256, 0, st>>>(a);
    DSRG_LAUNCH_CHECK(p);
    adj_p12_kernel<<<blocks(nA4), 256, 0, st>>>(a);
    DSRG_LAUNCH_CHECK(p);
    adj_t1_chain_kernel<<<blocks(nHP2), 256, dsm, st>>>(a);
    DSRG_LAUNCH_CHECK(p);
    adj_w1_chain_kernel<<<blocks(A.w1n), 256, dsm, st>>>(a);
    DSRG_LAUNCH_CHECK(p);
    adj_w2_chain_kernel<<<blocks(A.w2n), 256, dsm, st>>>(a);
    DSRG_LAUNCH_CHECK(p);
    {
      const size_t n = 2 * (size_t)z.nH * z.nA * z.nA * z.nP + (size_t)z.nH * z.nA * z.nH * z.nA;
      adj_k_kernel<<<blocks(n), 256, 0, st>>>(a);
      DSRG_LAUNCH_CHECK(p);
    }
    switch (z.nA) {
      case 1: adj_m_kernel<1><<<blocks(nV2), 256, dsm, st>>>(a, w->dP12); break;
      case 2: adj_m_kernel<2><<<blocks(nV2), 256, dsm, st>>>(a, w->dP12); break;
      case 3: adj_m_kernel<3><<<blocks(nV2), 256, dsm, st>>>(a, w->dP12); break;
      case 4: adj_m_kernel<4><<<blocks(nV2), 256, dsm, st>>>(a, w->dP12); break;
      default: adj_m_generic_kernel<<<blocks(nV2), 256, dsm, st>>>(a, w->dP12); break;
    }
    DSRG_LAUNCH_CHECK(p);
    if (!fp64) {
      // every adjoint of an integral is formed: S outside the core block, then dB
      if ((e = tc_adj_rest(p, w->dX, w->dZ, w->dM, w->dK1, w->dK2, w->dK3)) != cudaSuccess) return e;
      return tc_adj_assemble(p, B, dB);
    }
    adj_k_to_b_kernel<<<blocks((size_t)z.Q * HP), 256, 0, st>>>(a, B, dB);
    DSRG_LAUNCH_CHECK(p);
    const long long CP = (long long)z.nC * z.nP;
    e = gemm(p, batched(mk(z.Q, z.nV, z.nA, z.nV, B + CP + z.nA, HP, z.nP, 1, w->dM, nV2, 1, nV,
                           dB + (long long)z.nC * z.nP + z.nA, HP, 1, 1.0),
                        z.nA, 0, (long long)z.nA * nV2, z.nP));
    if (e != cudaSuccess) return e;
    e = gemm(p, batched(mk(z.Q, z.nV, z.nA, z.nV, B + CP + z.nA, HP, z.nP, 1, w->dM,
                           (long long)z.nA * nV2, nV, 1, dB + (long long)z.nC * z.nP + z.nA, HP, 1,
                           1.0),
                        z.nA, 0, nV2, z.nP));
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace dsrg
