// FP64 kernels for diagram F3 (CCAV) and for the active block of the
// DSRG-MRPT2 energy: Table 1 terms A-E, G-I and Table 2 diagrams F4-F8.
//
// The active block works in spin orbitals (spin orbital 2p + sigma) on the
// integral blocks that carry at least two active indices, which the paper
// forms explicitly (Sec. III, steps 4-6):
//   W1 = <iu||ax>   i in H, u active hole, a in P, x active particle
//   W2 = <ij||xy>   i, j in H, x, y active particles
// and the (A,A|V,V) integrals M_xu[e,f] = (xe|uf) in spatial orbitals, whose
// spin sums P1, P2 feed terms G and F4.
//
// Amplitudes and modified integrals (Eqs. (12)-(15)), with D = hole energies
// minus particle energies: t = v (1 - exp(-s D^2))/D (zero when all four
// indices are active), vt = v (1 + exp(-s D^2)); the T1 amplitude of Eq. (12)
// with f^(1) = 0 is t_a^i = S_ia (1 - exp(-s D_ia^2))/D_ia with
// S_ia = sum_{ux} (e_x - e_u) t_{ax}^{iu} gamma_u^x, and the modified Fock
// element of Eq. (14) is ft_a^i = S_ia exp(-s D_ia^2); Table 1's ft_j^b is the
// Hermitian element ft_b^j.
//
// Densities (Fig. 1): gamma = 1 on core, G/2 per spin on the active block;
// eta = 1 - gamma on particles (1 on virtuals). Cumulant from the opposite-
// spin input L: same spin L[u,v,x,y] - L[u,v,y,x]; (alpha beta|alpha beta)
// L[u,v,x,y]; (beta alpha|beta alpha) L[v,u,y,x]; (alpha beta|beta alpha)
// -L[u,v,y,x]; (beta alpha|alpha beta) -L[v,u,x,y].
#include <type_traits>

#include "internal.cuh"
#include "regulators.cuh"

namespace dsrg {

// ---------------------------------------------------------------------------
// F3 (CCAV), spin-adapted:
//   F3 = sum_{u,v} Hh_uv sum_{m,n,e} Z_v[m,n,e] (2 Z_u[m,n,e] - Z_u[n,m,e])
//        (1 + exp(-s D_v^2)) (1 - exp(-s D_u^2))/D_u,
//   Z_u[m,n,e] = (me|nu), D_u = e_m + e_n - e_e - e_u, Hh = 2 I - G.
// One CTA per virtual e holds Z_u[m,n,e] for all m, n, u in shared memory.
// ---------------------------------------------------------------------------
constexpr int KC_CCAV = 8;

__global__ void __launch_bounds__(256) ccav_fp64_kernel(
    const double* __restrict__ B, const double* __restrict__ eps, const double* __restrict__ G,
    double s, Sizes z, double* __restrict__ partials) {
  extern __shared__ double smem[];
  const int nC = z.nC, nA = z.nA;
  double* Z = smem;                          // [nA][nC][nC]
  double* sBe = Z + nA * nC * nC;            // [KC][nC]
  double* sBu = sBe + KC_CCAV * nC;          // [KC][nC][nA]
  __shared__ double red[8];
  const int e = blockIdx.x;
  const int nz = nA * nC * nC;
  for (int k = threadIdx.x; k < nz; k += 256) Z[k] = 0.0;
  for (int q0 = 0; q0 < z.Q; q0 += KC_CCAV) {
    __syncthreads();
    for (int k = threadIdx.x; k < KC_CCAV * nC * (1 + nA); k += 256) {
      const int qq = k / (nC * (1 + nA)), r = k % (nC * (1 + nA)), q = q0 + qq;
      double v = 0.0;
      if (r < nC) {
        if (q < z.Q) v = B[bidx(z, q, r, nA + e)];
        sBe[qq * nC + r] = v;
      } else {
        const int nu = r - nC, n = nu / nA, u = nu % nA;
        if (q < z.Q) v = B[bidx(z, q, n, u)];
        sBu[(qq * nC + n) * nA + u] = v;
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < nz; k += 256) {
      const int u = k / (nC * nC), mn = k % (nC * nC), m = mn / nC, n = mn % nC;
      double acc = Z[k];
#pragma unroll
      for (int qq = 0; qq < KC_CCAV; ++qq) acc = fma(sBe[qq * nC + m], sBu[(qq * nC + n) * nA + u], acc);
      Z[k] = acc;
    }
  }
  __syncthreads();
  const double ee = eps[nC + nA + e];
  double acc = 0.0;
  for (int mn = threadIdx.x; mn < nC * nC; mn += 256) {
    const int m = mn / nC, n = mn % nC;
    const double base = eps[m] + eps[n] - ee;
    double Rv[NA_MAX], Rt[NA_MAX];
    for (int u = 0; u < nA; ++u) {
      const double D = base - eps[nC + u];
      Rv[u] = reg_v(D, s);
      Rt[u] = reg_t(D, s);
    }
    for (int u = 0; u < nA; ++u) {
      const double zu = 2.0 * Z[(u * nC + m) * nC + n] - Z[(u * nC + n) * nC + m];
      double c = 0.0;
      for (int v = 0; v < nA; ++v) {
        const double Hh = (u == v ? 2.0 : 0.0) - G[u * nA + v];
        c = fma(Hh * Rv[v], Z[(v * nC + m) * nC + n], c);
      }
      acc = fma(c, zu * Rt[u], acc);
    }
  }
  const double tot = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[e] = tot;
}

static size_t ccav_smem(const Sizes& z) {
  return sizeof(double) * ((size_t)z.nA * z.nC * z.nC + (size_t)KC_CCAV * z.nC * (1 + z.nA));
}

int ccav_fp64_blocks(const dsrg_plan* p) { return p->z.nA == 0 ? 0 : p->z.nV; }

cudaError_t launch_ccav_fp64(dsrg_plan* p, const double* B, const double* eps, const double* G,
                             double s) {
  const Segment& sg = p->segs[p->seg_ccav];
  if (sg.count == 0) return cudaSuccess;
  const size_t sm = ccav_smem(p->z);
  raise_smem_limit((const void*)ccav_fp64_kernel, sm);
  ccav_fp64_kernel<<<sg.count, 256, sm, p->stream>>>(B, eps, G, s, p->z,
                                                     p->d_partials + sg.begin);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Active block: tables.
// ---------------------------------------------------------------------------
struct ActDims {
  int nC2, nA2, nH2, nP2, nV2;
};

__host__ __device__ __forceinline__ ActDims act_dims(const Sizes& z) {
  return ActDims{2 * z.nC, 2 * z.nA, 2 * z.nH, 2 * z.nP, 2 * z.nV};
}

// W1 flat index: [I in 2nH][U in 2nA][A in 2nP][X in 2nA]
__device__ __forceinline__ size_t w1i(const ActDims& d, int I, int U, int A, int X) {
  return (((size_t)I * d.nA2 + U) * d.nP2 + A) * d.nA2 + X;
}
// W2 flat index: [I in 2nH][J in 2nH][X in 2nA][Y in 2nA]
__device__ __forceinline__ size_t w2i(const ActDims& d, int I, int J, int X, int Y) {
  return (((size_t)I * d.nH2 + J) * d.nA2 + X) * d.nA2 + Y;
}
__device__ __forceinline__ int lami(const ActDims& d, int U, int V, int X, int Y) {
  return ((U * d.nA2 + V) * d.nA2 + X) * d.nA2 + Y;
}

// Spatial integrals K1 = (ia|ux), K2 = (ix|ua) [nH][nA][nA][nP], K3 = (ix|jy) [nH][nA][nH][nA].
__global__ void small_ints_kernel(const double* __restrict__ B, Sizes z, double* __restrict__ K1,
                                  double* __restrict__ K2, double* __restrict__ K3) {
  const size_t n12 = (size_t)z.nH * z.nA * z.nA * z.nP;
  const size_t n3 = (size_t)z.nH * z.nA * z.nH * z.nA;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < 2 * n12) {
    const bool second = k >= n12;
    const size_t r = second ? k - n12 : k;
    const int a = (int)(r % z.nP);
    const int x = (int)((r / z.nP) % z.nA);
    const int u = (int)((r / ((size_t)z.nP * z.nA)) % z.nA);
    const int i = (int)(r / ((size_t)z.nP * z.nA * z.nA));
    double acc = 0.0;
    if (!second) {
      for (int q = 0; q < z.Q; ++q) acc = fma(B[bidx(z, q, i, a)], B[bidx(z, q, z.nC + u, x)], acc);
      K1[r] = acc;
    } else {
      for (int q = 0; q < z.Q; ++q) acc = fma(B[bidx(z, q, i, x)], B[bidx(z, q, z.nC + u, a)], acc);
      K2[r] = acc;
    }
  } else if (k < 2 * n12 + n3) {
    const size_t r = k - 2 * n12;
    const int y = (int)(r % z.nA);
    const int j = (int)((r / z.nA) % z.nH);
    const int x = (int)((r / ((size_t)z.nA * z.nH)) % z.nA);
    const int i = (int)(r / ((size_t)z.nA * z.nH * z.nA));
    double acc = 0.0;
    for (int q = 0; q < z.Q; ++q) acc = fma(B[bidx(z, q, i, x)], B[bidx(z, q, j, y)], acc);
    K3[r] = acc;
  }
}

// Spin-orbital W1, W2 (V, T, Vt), cumulant and active gamma. One thread per
// spatial quadruple of W1 / W2: the regulators depend on the spatial orbitals
// only, so they are evaluated once and the 16 spin combinations written.
__global__ void build_tables_kernel(const double* __restrict__ eps, const double* __restrict__ G,
                                    const double* __restrict__ L, double s, Sizes z,
                                    const double* __restrict__ K1, const double* __restrict__ K2,
                                    const double* __restrict__ K3, double* __restrict__ W1,
                                    double* __restrict__ W2, double* __restrict__ lam,
                                    double* __restrict__ gA, size_t w1n, size_t w2n) {
  const ActDims d = act_dims(z);
  const size_t n1 = (size_t)z.nH * z.nA * z.nP * z.nA;   // spatial (i, u, a, x)
  const size_t n2 = (size_t)z.nH * z.nH * z.nA * z.nA;   // spatial (i, j, x, y)
  const size_t nl = (size_t)d.nA2 * d.nA2 * d.nA2 * d.nA2;
  const size_t ng = (size_t)d.nA2 * d.nA2;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n1) {
    const int x = (int)(k % z.nA);
    const int a = (int)((k / z.nA) % z.nP);
    const int u = (int)((k / ((size_t)z.nA * z.nP)) % z.nA);
    const int i = (int)(k / ((size_t)z.nA * z.nP * z.nA));
    const size_t kk = (((size_t)i * z.nA + u) * z.nA + x) * z.nP + a;
    const double k1 = K1[kk], k2 = K2[kk];
    const double D = eps[i] + eps[z.nC + u] - eps[z.nC + a] - eps[z.nC + x];
    const double rt = reg_t(D, s), rv = reg_v(D, s);
    const bool internal = (i >= z.nC) && (a < z.nA);
    for (int sp = 0; sp < 16; ++sp) {
      const int si = sp >> 3, su = (sp >> 2) & 1, sa = (sp >> 1) & 1, sx = sp & 1;
      double V = 0.0;
      if (si == sa && su == sx) V += k1;
      if (si == sx && su == sa) V -= k2;
      const size_t o = w1i(d, 2 * i + si, 2 * u + su, 2 * a + sa, 2 * x + sx);
      W1[o] = V;
      W1[w1n + o] = internal ? 0.0 : V * rt;
      W1[2 * w1n + o] = V * rv;
    }
  } else if (k < n1 + n2) {
    const size_t r = k - n1;
    const int y = (int)(r % z.nA);
    const int x = (int)((r / z.nA) % z.nA);
    const int j = (int)((r / ((size_t)z.nA * z.nA)) % z.nH);
    const int i = (int)(r / ((size_t)z.nA * z.nA * z.nH));
    const double kxy = K3[(((size_t)i * z.nA + x) * z.nH + j) * z.nA + y];
    const double kyx = K3[(((size_t)i * z.nA + y) * z.nH + j) * z.nA + x];
    const double D = eps[i] + eps[j] - eps[z.nC + x] - eps[z.nC + y];
    const double rt = reg_t(D, s), rv = reg_v(D, s);
    const bool internal = (i >= z.nC) && (j >= z.nC);
    for (int sp = 0; sp < 16; ++sp) {
      const int si = sp >> 3, sj = (sp >> 2) & 1, sx = (sp >> 1) & 1, sy = sp & 1;
      double V = 0.0;
      if (si == sx && sj == sy) V += kxy;
      if (si == sy && sj == sx) V -= kyx;
      const size_t o = w2i(d, 2 * i + si, 2 * j + sj, 2 * x + sx, 2 * y + sy);
      W2[o] = V;
      W2[w2n + o] = internal ? 0.0 : V * rt;
      W2[2 * w2n + o] = V * rv;
    }
  } else if (k < n1 + n2 + nl) {
    const int r = (int)(k - n1 - n2);
    const int Y = r % d.nA2, X = (r / d.nA2) % d.nA2, V = (r / (d.nA2 * d.nA2)) % d.nA2,
              U = r / (d.nA2 * d.nA2 * d.nA2);
    const int u = U >> 1, v = V >> 1, x = X >> 1, y = Y >> 1;
    const int su = U & 1, sv = V & 1, sx = X & 1, sy = Y & 1;
    const int nA = z.nA;
    auto Lf = [&](int p0, int p1, int p2, int p3) { return L[((p0 * nA + p1) * nA + p2) * nA + p3]; };
    double val = 0.0;
    if (su == sv && sv == sx && sx == sy) {
      val = Lf(u, v, x, y) - Lf(u, v, y, x);
    } else if (su == sx && sv == sy) {
      val = (su == 0) ? Lf(u, v, x, y) : Lf(v, u, y, x);
    } else if (su == sy && sv == sx) {
      val = (su == 0) ? -Lf(u, v, y, x) : -Lf(v, u, x, y);
    }
    lam[r] = val;
  } else if (k < n1 + n2 + nl + ng) {
    const int r = (int)(k - n1 - n2 - nl);
    const int U = r / d.nA2, V = r % d.nA2;
    gA[r] = ((U & 1) == (V & 1)) ? 0.5 * G[(U >> 1) * z.nA + (V >> 1)] : 0.0;
  }
}

// T1 amplitudes and modified Fock elements over spin orbitals [2nH][2nP]
// (Eqs. (12), (14)); f1 is the optional off-diagonal Fock block [nH][nP]
// (spatial, spin-diagonal; its active x active entries are not read).
__global__ void t1_kernel(const double* __restrict__ eps, double s, Sizes z,
                          const double* __restrict__ W1T, const double* __restrict__ gA,
                          const double* __restrict__ f1, double* __restrict__ t1,
                          double* __restrict__ ft) {
  const ActDims d = act_dims(z);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= d.nH2 * d.nP2) return;
  const int I = k / d.nP2, A = k % d.nP2;
  double S = 0.0;
  for (int U = 0; U < d.nA2; ++U)
    for (int X = 0; X < d.nA2; ++X) {
      const double g = gA[U * d.nA2 + X];
      if (g == 0.0) continue;
      const double Dux = eps[z.nC + (X >> 1)] - eps[z.nC + (U >> 1)];
      S = fma(Dux * g, W1T[w1i(d, I, U, A, X)], S);
    }
  const double D1 = eps[I >> 1] - eps[z.nC + (A >> 1)];
  const bool internal = (I >= d.nC2) && (A < d.nA2);
  const double F = (f1 && !internal && (I & 1) == (A & 1)) ? f1[(size_t)(I >> 1) * z.nP + (A >> 1)]
                                                           : 0.0;
  const double g = exp(-s * D1 * D1);
  t1[k] = internal ? 0.0 : (F + S) * reg_t(D1, s);
  ft[k] = fma(F, 1.0 + g, S * g);
}

// Term A with no active orbitals (the only term then, from f^(1)): per core
// orbital m, 2 sum_e f_me^2 (1 + exp(-s D^2)) (1 - exp(-s D^2)) / D, D = e_m - e_e
// (the factor 2 is the spin sum). f1 == null: 0.
__global__ void __launch_bounds__(128) singles_kernel(const double* __restrict__ eps, double s,
                                                      Sizes z, const double* __restrict__ f1,
                                                      double* __restrict__ partials) {
  __shared__ double red[4];
  const int m = blockIdx.x;
  double acc = 0.0;
  if (f1) {
    for (int e = threadIdx.x; e < z.nP; e += 128) {
      const double D = eps[m] - eps[z.nC + e];
      const double f = f1[(size_t)m * z.nP + e];
      acc = fma(f * f * (1.0 + exp(-s * D * D)), reg_t(D, s), acc);
    }
  }
  const double tot = block_sum<128>(acc, red);
  if (threadIdx.x == 0) partials[m] = 2.0 * tot;
}

// gamma (over holes) and eta (over particles) as sparse row lookups.
__device__ __forceinline__ double gam_h(const ActDims& d, const double* gA, int K, int I) {
  if (K < d.nC2 || I < d.nC2) return (K == I) ? 1.0 : 0.0;
  return gA[(K - d.nC2) * d.nA2 + (I - d.nC2)];
}
__device__ __forceinline__ double eta_p(const ActDims& d, const double* gA, int A, int Bp) {
  if (A >= d.nA2 || Bp >= d.nA2) return (A == Bp) ? 1.0 : 0.0;
  return (A == Bp ? 1.0 : 0.0) - gA[A * d.nA2 + Bp];
}

// Ti[J][V][B][Y] = sum_{I,A} gamma_I^J eta_B^A t_{AY}^{IV}  (the dressed T of term I).
__global__ void ti_kernel(Sizes z, const double* __restrict__ W1T, const double* __restrict__ gA,
                          double* __restrict__ Ti, size_t w1n) {
  const ActDims d = act_dims(z);
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= w1n) return;
  const int Y = (int)(k % d.nA2);
  const int Bp = (int)((k / d.nA2) % d.nP2);
  const int V = (int)((k / ((size_t)d.nA2 * d.nP2)) % d.nA2);
  const int J = (int)(k / ((size_t)d.nA2 * d.nP2 * d.nA2));
  const int i0 = (J < d.nC2) ? J : d.nC2, i1 = (J < d.nC2) ? J + 1 : d.nH2;
  const int a0 = (Bp < d.nA2) ? 0 : Bp, a1 = (Bp < d.nA2) ? d.nA2 : Bp + 1;
  double acc = 0.0;
  for (int I = i0; I < i1; ++I) {
    const double g = gam_h(d, gA, J, I);
    if (g == 0.0) continue;
    for (int A = a0; A < a1; ++A) acc = fma(g * eta_p(d, gA, A, Bp), W1T[w1i(d, I, V, A, Y)], acc);
  }
  Ti[k] = acc;
}

// (A,A|V,V) integrals M[x][u][e][f] = (xe|uf), 64x64 tiles, FP64.
__global__ void __launch_bounds__(256) gram_aavv_kernel(const double* __restrict__ B, Sizes z,
                                                       int ntile, double* __restrict__ M) {
  __shared__ double sX[16][64], sU[16][64];
  const int nT2 = ntile * ntile;
  const int xu = blockIdx.x / nT2, t = blockIdx.x % nT2;
  const int x = xu / z.nA, u = xu % z.nA;
  const int e0 = (t / ntile) * 64, f0 = (t % ntile) * 64;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  double acc[4][4];
#pragma unroll
  for (int r = 0; r < 4; ++r)
#pragma unroll
    for (int c = 0; c < 4; ++c) acc[r][c] = 0.0;
  for (int q0 = 0; q0 < z.Q; q0 += 16) {
    for (int k = threadIdx.x; k < 16 * 64; k += 256) {
      const int qq = k / 64, c = k % 64, q = q0 + qq;
      const int e = e0 + c, f = f0 + c;
      sX[qq][c] = (q < z.Q && e < z.nV) ? B[bidx(z, q, z.nC + x, z.nA + e)] : 0.0;
      sU[qq][c] = (q < z.Q && f < z.nV) ? B[bidx(z, q, z.nC + u, z.nA + f)] : 0.0;
    }
    __syncthreads();
#pragma unroll 4
    for (int qq = 0; qq < 16; ++qq) {
      double ra[4], rb[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        ra[r] = sX[qq][ty * 4 + r];
        rb[r] = sU[qq][tx * 4 + r];
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[r][c] = fma(ra[r], rb[c], acc[r][c]);
    }
    __syncthreads();
  }
  const size_t base = (size_t)xu * z.nV * z.nV;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const int e = e0 + ty * 4 + r;
    if (e >= z.nV) continue;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int f = f0 + tx * 4 + c;
      if (f < z.nV) M[base + (size_t)e * z.nV + f] = acc[r][c];
    }
  }
}

// P1[xu][yv] = sum_ef M_xu[ef] M_yv[ef] R, P2[xu][yv] = sum_ef M_xu[ef] M_vy[ef] R
// (M_vy[e,f] = M_yv[f,e]) with R = (1 + exp(-s D_xu^2)) (1 - exp(-s D_yv^2))/D_yv.
constexpr int ACTVV_BLOCKS = 152;
constexpr int ACTVV_CH = 64;      // positions (e, f) per chunk of the active VV sums

// Factor tables of exp(-s D_p^2), D_p = E_p - e_e - e_f for the active pairs
// p = (x, u), E_p = e_x + e_u: exp(-s E_p^2) exp(2 s E_p e_e) exp(2 s E_p e_f)
// exp(-s (e_e + e_f)^2). alpha == nullptr: evaluate exp directly.
struct ActFact {
  const double* alpha;  // [nA^2][ld]  exp(2 s E_p e_e)
  const double* pinfo;  // [nA^2][4]   E_p, exp(-s E_p^2), factorisable flag
  const double* tau;    // [ld][ld]    exp(-s (e_e + e_f)^2)
  int ld;
};

// Rv = 1 + exp(-s D^2), Rt = (1 - exp(-s D^2)) / D in FP64; g = exp(-s D^2)
// from the factor tables when fact, 1/D as an FP32 seed and one Newton step;
// |D| < 1/4 takes expm1 and an FP64 divide.
__device__ __forceinline__ void reg_pair(double D, double s, bool fact, double g, double& rv,
                                         double& rt) {
  if (fact && fabs(D) >= 0.25) {
    float r0f;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0f) : "f"((float)D));
    const double r0 = (double)r0f;
    const double en = fma(-D, r0, 1.0);
    const double R0 = fma(-g, r0, r0);
    rt = fma(R0, en, R0);
    rv = 1.0 + g;
  } else {
    rt = reg_t(D, s);
    rv = reg_v(D, s);
  }
}

__global__ void __launch_bounds__(256) actvv_kernel(const double* __restrict__ eps, double s,
                                                    Sizes z, const double* __restrict__ M,
                                                    double* __restrict__ part) {
  __shared__ double red[8];
  const int nA = z.nA, nA4 = nA * nA * nA * nA;
  const int c = blockIdx.y;
  const int v = c % nA, y = (c / nA) % nA, u = (c / (nA * nA)) % nA, x = c / (nA * nA * nA);
  const size_t nV2 = (size_t)z.nV * z.nV;
  const double* Mxu = M + (size_t)(x * nA + u) * nV2;
  const double* Myv = M + (size_t)(y * nA + v) * nV2;
  const double* Mvy = M + (size_t)(v * nA + y) * nV2;
  const int ve = z.nC + z.nA;
  const double Exu = eps[z.nC + x] + eps[z.nC + u], Eyv = eps[z.nC + y] + eps[z.nC + v];
  double p1 = 0.0, p2 = 0.0;
  for (size_t k = (size_t)blockIdx.x * 256 + threadIdx.x; k < nV2; k += (size_t)gridDim.x * 256) {
    const int e = (int)(k / z.nV), f = (int)(k % z.nV);
    const double ef = eps[ve + e] + eps[ve + f];
    const double R = reg_v(Exu - ef, s) * reg_t(Eyv - ef, s);
    const double m = Mxu[k] * R;
    p1 = fma(m, Myv[k], p1);
    p2 = fma(m, Mvy[k], p2);
  }
  const double t1 = block_sum<256>(p1, red);
  const double t2 = block_sum<256>(p2, red);
  if (threadIdx.x == 0) {
    part[((size_t)blockIdx.x * 2 + 0) * nA4 + c] = t1;
    part[((size_t)blockIdx.x * 2 + 1) * nA4 + c] = t2;
  }
}

// Same sums for small active spaces, with the regulators of each active pair
// evaluated once per (e,f): Rv(D_xu) and Rt(D_yv) for the nA^2 pairs, then the
// nA^4 products P1 += (M_xu Rv_xu)(M_yv Rt_yv), P2 += (M_xu Rv_xu)(M_vy Rt_yv).
// F32 (split-precision plans, as actvv_gen_kernel): the regulated factors are
// rounded to FP32 and each thread's sums over up to ACTVV_CH positions run in
// FP32 with round-to-nearest, the chunk sums in FP64; the regulators stay FP64.
template <int NA, bool F32>
__global__ void __launch_bounds__(256) actvv_small_kernel(const double* __restrict__ eps, double s,
                                                          Sizes z, const double* __restrict__ M,
                                                          ActFact F, double* __restrict__ part) {
  constexpr int NA2 = NA * NA, NA4 = NA2 * NA2;
  __shared__ double red[8];
  const size_t nV2 = (size_t)z.nV * z.nV;
  const int ve = z.nC + z.nA;
  double Ep[NA2], Bp[NA2];
  bool fact = F.alpha != nullptr;
#pragma unroll
  for (int p = 0; p < NA2; ++p) {
    Ep[p] = eps[z.nC + p / NA] + eps[z.nC + p % NA];
    Bp[p] = fact ? F.pinfo[4 * p + 1] : 0.0;
    fact = fact && F.pinfo[4 * p + 2] != 0.0;
  }
  double acc1[NA4], acc2[NA4];
  float f1[NA4], f2[NA4];
  int cnt = 0;
#pragma unroll
  for (int c = 0; c < NA4; ++c) {
    acc1[c] = acc2[c] = 0.0;
    f1[c] = f2[c] = 0.0f;
  }
  for (size_t k = (size_t)blockIdx.x * 256 + threadIdx.x; k < nV2; k += (size_t)gridDim.x * 256) {
    const int e = (int)(k / z.nV), f = (int)(k % z.nV);
    const double ef = eps[ve + e] + eps[ve + f];
    const double tau = fact ? F.tau[(size_t)e * F.ld + f] : 0.0;
    double mr[NA2], mq[NA2], m[NA2];
#pragma unroll
    for (int p = 0; p < NA2; ++p) m[p] = M[(size_t)p * nV2 + k];
#pragma unroll
    for (int p = 0; p < NA2; ++p) {
      const double D = Ep[p] - ef;
      const double g = fact ? Bp[p] * F.alpha[(size_t)p * F.ld + e] * F.alpha[(size_t)p * F.ld + f] * tau : 0.0;
      double rv, rt;
      reg_pair(D, s, fact, g, rv, rt);
      mr[p] = m[p] * rv;
      mq[p] = rt;
    }
    if constexpr (F32) {
      float a[NA2], b[NA2], c[NA2];
#pragma unroll
      for (int p = 0; p < NA2; ++p) {
        const int pt = (p % NA) * NA + p / NA;
        a[p] = (float)mr[p];
        b[p] = (float)(m[p] * mq[p]);
        c[p] = (float)(m[pt] * mq[p]);
      }
#pragma unroll
      for (int p = 0; p < NA2; ++p)
#pragma unroll
        for (int q = 0; q < NA2; ++q) {
          f1[p * NA2 + q] = fmaf(a[p], b[q], f1[p * NA2 + q]);
          f2[p * NA2 + q] = fmaf(a[p], c[q], f2[p * NA2 + q]);
        }
      if (++cnt == ACTVV_CH) {
        cnt = 0;
#pragma unroll
        for (int o = 0; o < NA4; ++o) {
          acc1[o] += (double)f1[o];
          acc2[o] += (double)f2[o];
          f1[o] = f2[o] = 0.0f;
        }
      }
    } else {
#pragma unroll
      for (int p = 0; p < NA2; ++p)
#pragma unroll
        for (int q = 0; q < NA2; ++q) {
          const int qt = (q % NA) * NA + q / NA;
          acc1[p * NA2 + q] = fma(mr[p], m[q] * mq[q], acc1[p * NA2 + q]);
          acc2[p * NA2 + q] = fma(mr[p], m[qt] * mq[q], acc2[p * NA2 + q]);
        }
    }
  }
  if constexpr (F32) {
#pragma unroll
    for (int o = 0; o < NA4; ++o) {
      acc1[o] += (double)f1[o];
      acc2[o] += (double)f2[o];
    }
  }
#pragma unroll
  for (int c = 0; c < NA4; ++c) {
    const double t1 = block_sum<256>(acc1[c], red);
    const double t2 = block_sum<256>(acc2[c], red);
    if (threadIdx.x == 0) {
      part[((size_t)blockIdx.x * 2 + 0) * NA4 + c] = t1;
      part[((size_t)blockIdx.x * 2 + 1) * NA4 + c] = t2;
    }
  }
}

// The same sums for any active space: per chunk of ACTVV_CH positions (e,f)
// the CTA first forms, for every active pair p = (x,u) and its transpose
// p' = (u,x), a_p = M_p Rv_p, b_p = M_p Rt_p and c_p = M_p' Rt_p in shared memory
// (nA^2 regulator pairs per position; D_p' = D_p), then accumulates
// P1[p][q] += a_p b_q and P2[p][q] += a_p c_q (M_vy = M_(yv)') over the chunk,
// each thread holding a fixed set of (p, q).

// F32 (split-precision plans): the regulated factors are rounded to FP32 and each
// 64-term chunk of the sum over (e, f) runs in FP32 on CUDA cores (round to
// nearest), the chunk sums in FP64; the regulators themselves stay FP64.
template <int NA, bool F32>
__global__ void __launch_bounds__(256) actvv_gen_kernel(const double* __restrict__ eps, double s,
                                                        Sizes z, const double* __restrict__ M,
                                                        ActFact F, double* __restrict__ part) {
  using T = typename std::conditional<F32, float, double>::type;
  constexpr int NA2 = NA * NA, NA4 = NA2 * NA2;
  constexpr int PER = (NA4 + 255) / 256;  // (p,q) outputs per thread
  extern __shared__ double avs[];
  T* sa = (T*)avs;                         // [NA2][CH]
  T* sb = sa + NA2 * ACTVV_CH;             // [NA2][CH]
  T* sc = sb + NA2 * ACTVV_CH;             // [NA2][CH]
  __shared__ double red[8];
  const size_t nV2 = (size_t)z.nV * z.nV;
  const int ve = z.nC + z.nA;
  bool fact = F.alpha != nullptr;
  for (int p = 0; fact && p < NA2; ++p) fact = F.pinfo[4 * p + 2] != 0.0;
  double acc1[PER], acc2[PER];
#pragma unroll
  for (int r = 0; r < PER; ++r) acc1[r] = acc2[r] = 0.0;
  const size_t nchunks = (nV2 + ACTVV_CH - 1) / ACTVV_CH;
  for (size_t ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const size_t k0 = ch * ACTVV_CH;
    __syncthreads();
    for (int it = threadIdx.x; it < NA2 * ACTVV_CH; it += 256) {
      const int pidx = it / ACTVV_CH, kk = it % ACTVV_CH;
      const size_t k = k0 + kk;
      double a = 0.0, b = 0.0, c = 0.0;
      if (k < nV2) {
        const int x = pidx / NA, u = pidx % NA;
        const int e = (int)(k / z.nV), f = (int)(k % z.nV);
        const double D = eps[z.nC + x] + eps[z.nC + u] - eps[ve + e] - eps[ve + f];
        const double m = M[(size_t)pidx * nV2 + k];
        const double mt = M[(size_t)(u * NA + x) * nV2 + k];
        const double g = fact ? F.pinfo[4 * pidx + 1] * F.alpha[(size_t)pidx * F.ld + e] *
                                    F.alpha[(size_t)pidx * F.ld + f] * F.tau[(size_t)e * F.ld + f]
                              : 0.0;
        double rv, rt;
        reg_pair(D, s, fact, g, rv, rt);
        a = m * rv;
        b = m * rt;
        c = mt * rt;
      }
      sa[it] = (T)a;
      sb[it] = (T)b;
      sc[it] = (T)c;
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < PER; ++r) {
      const int o = threadIdx.x + 256 * r;
      if (o < NA4) {
        const T* ap = sa + (o / NA2) * ACTVV_CH;
        const T* bq = sb + (o % NA2) * ACTVV_CH;
        const T* cq = sc + (o % NA2) * ACTVV_CH;
        if constexpr (F32) {
          float t1 = 0.f, t2 = 0.f;
#pragma unroll 8
          for (int kk = 0; kk < ACTVV_CH; ++kk) {
            t1 = fmaf(ap[kk], bq[kk], t1);
            t2 = fmaf(ap[kk], cq[kk], t2);
          }
          acc1[r] += (double)t1;
          acc2[r] += (double)t2;
        } else {
          double t1 = acc1[r], t2 = acc2[r];
#pragma unroll 8
          for (int kk = 0; kk < ACTVV_CH; ++kk) {
            t1 = fma(ap[kk], bq[kk], t1);
            t2 = fma(ap[kk], cq[kk], t2);
          }
          acc1[r] = t1;
          acc2[r] = t2;
        }
      }
    }
  }
  // per-CTA partials: thread-owned outputs need no block reduction
#pragma unroll
  for (int r = 0; r < PER; ++r) {
    const int o = threadIdx.x + 256 * r;
    if (o < NA4) {
      part[((size_t)blockIdx.x * 2 + 0) * NA4 + o] = acc1[r];
      part[((size_t)blockIdx.x * 2 + 1) * NA4 + o] = acc2[r];
    }
  }
  (void)red;
}

__global__ void actvv_reduce_kernel(int nA4, int nblk, const double* __restrict__ part,
                                    double* __restrict__ P12) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= 2 * nA4) return;
  double acc = 0.0;
  for (int b = 0; b < nblk; ++b) acc += part[(size_t)b * 2 * nA4 + k];
  P12[k] = acc;
}

// ---------------------------------------------------------------------------
// Active block: one kernel, one term per blockIdx.y, one outer index per thread.
// ---------------------------------------------------------------------------
enum Term {
  T_A = 0, T_B, T_C, T_D, T_E, T_GVA, T_GVV, T_H, T_I, T_F4, T_F5, T_F6, T_F7, T_F8, T_J, T_K,
  N_TERMS
};

struct TermArgs {
  const double *W1V, *W1T, *W1Vt, *W2V, *W2T, *W2Vt, *Ti, *lam, *gA, *t1, *ft, *P12;
  const double* lam3;  // [2nA]^6 spin-orbital three-body cumulant, or null (J = K = 0)
};

// Index of lambda_{UVW}^{XYZ} in the spin-orbital three-body cumulant.
__device__ __forceinline__ size_t lam3i(int n2, int U, int V, int W, int X, int Y, int Z) {
  return (((((size_t)U * n2 + V) * n2 + W) * n2 + X) * n2 + Y) * n2 + Z;
}

__device__ __forceinline__ double ga(const ActDims& d, const double* gA, int U, int V) {
  return gA[U * d.nA2 + V];
}
__device__ __forceinline__ double ea(const ActDims& d, const double* gA, int U, int V) {
  return (U == V ? 1.0 : 0.0) - gA[U * d.nA2 + V];
}

// S[(X,U),(Y,V)] = sum_{E,F} vt_{XU}^{EF} t_{EF}^{YV} over virtual spin orbitals.
__device__ __forceinline__ double s_vv(const ActDims& d, int nA, const double* P12, int X, int U,
                                       int Y, int V) {
  const int nA4 = nA * nA * nA * nA;
  const int c = (((X >> 1) * nA + (U >> 1)) * nA + (Y >> 1)) * nA + (V >> 1);
  double r = 0.0;
  if ((X & 1) == (Y & 1) && (U & 1) == (V & 1)) r += 2.0 * P12[c];
  if ((X & 1) == (V & 1) && (U & 1) == (Y & 1)) r -= 2.0 * P12[nA4 + c];
  return r;
}

// Every term is a full sum over its spin-orbital indices; a thread takes one
// value of the leading indices (the "outer" index o of that term) and loops
// over the rest. gamma and eta are spin-diagonal, the cumulant is non-zero
// only for {s_u, s_v} = {s_x, s_y} and t1, ft conserve spin, so the inner loops
// run over spatial orbitals of the one spin that can give a non-zero product.
__device__ __forceinline__ long term_count(int term, const ActDims& d) {
  const long a2 = (long)d.nA2 * d.nA2;
  switch (term) {
    case T_A: return (long)d.nH2 * d.nP2;
    case T_B: return (long)d.nV2 * a2;
    case T_C: return (long)d.nC2 * a2;
    case T_D: return (long)d.nV2 * a2;
    case T_E: return (long)d.nC2 * a2;
    case T_GVA: return (long)d.nV2 * a2;
    case T_GVV: return a2 * a2;
    case T_H: return (long)d.nH2 * d.nH2 * a2;
    case T_I: return (long)d.nH2 * d.nP2 * a2;
    case T_F4: return a2 * a2;
    case T_F5: return (long)d.nC2 * d.nC2 * a2;
    case T_F6: return (long)d.nC2 * d.nV2 * a2;
    case T_F7: return (long)d.nV2 * a2 * d.nA2;
    case T_F8: return (long)d.nC2 * a2 * d.nA2;
    case T_J: return (long)d.nC2 * a2 * d.nA2;
    case T_K: return (long)d.nV2 * a2 * d.nA2;
  }
  return 0;
}

__device__ double term_value(int term, long o, const Sizes& z, const ActDims& d,
                             const TermArgs& t) {
  const int nA2 = d.nA2, nA = z.nA;
  const int C2 = d.nC2;  // first active hole spin orbital
  double acc = 0.0;
  switch (term) {
    case T_A: {  // ft_j^b t_a^i gamma_i^j eta_b^a, outer (J, Bp)
      const int J = (int)(o / d.nP2), Bp = (int)(o % d.nP2);
      double gf = 0.0, te = 0.0;
      const int k0 = (J < C2) ? J : C2, k1 = (J < C2) ? J + 1 : d.nH2;
      for (int K = k0; K < k1; ++K) gf = fma(gam_h(d, t.gA, J, K), t.ft[(size_t)K * d.nP2 + Bp], gf);
      const int a0 = (Bp < nA2) ? 0 : Bp, a1 = (Bp < nA2) ? nA2 : Bp + 1;
      for (int A = a0; A < a1; ++A) te = fma(eta_p(d, t.gA, A, Bp), t.t1[(size_t)J * d.nP2 + A], te);
      return gf * te;
    }
    case T_B: {  // 1/2 vt_{xy}^{ev} t_e^u lambda_{uv}^{xy}, outer (E, X, Y)
      const int Y = (int)(o % nA2), X = (int)((o / nA2) % nA2);
      const int Ap = nA2 + (int)(o / ((long)nA2 * nA2));
      const int su = Ap & 1;  // t_e^u conserves spin
      for (int V = 0; V < nA2; ++V) {
        const double vt = t.W1Vt[w1i(d, C2 + X, Y, Ap, V)];
        if (vt == 0.0) continue;
        for (int u = 0; u < nA; ++u) {
          const int U = 2 * u + su;
          acc = fma(vt * t.t1[(size_t)(C2 + U) * d.nP2 + Ap], t.lam[lami(d, U, V, X, Y)], acc);
        }
      }
      return 0.5 * acc;
    }
    case T_C: {  // -1/2 vt_{my}^{uv} t_x^m lambda_{uv}^{xy}, outer (M, Y, U)
      const int U = (int)(o % nA2), Y = (int)((o / nA2) % nA2), M = (int)(o / ((long)nA2 * nA2));
      const int sx = M & 1;
      for (int V = 0; V < nA2; ++V) {
        const double vt = t.W1Vt[w1i(d, M, Y, U, V)];
        if (vt == 0.0) continue;
        for (int x = 0; x < nA; ++x) {
          const int X = 2 * x + sx;
          acc = fma(vt * t.t1[(size_t)M * d.nP2 + X], t.lam[lami(d, U, V, X, Y)], acc);
        }
      }
      return -0.5 * acc;
    }
    case T_D: {  // 1/2 ft_x^e t_{ey}^{uv} lambda_{uv}^{xy}, outer (E, U, V)
      const int V = (int)(o % nA2), U = (int)((o / nA2) % nA2);
      const int Ap = nA2 + (int)(o / ((long)nA2 * nA2));
      const int sx = Ap & 1;
      for (int Y = 0; Y < nA2; ++Y) {
        const double tt = t.W1T[w1i(d, C2 + U, V, Ap, Y)];
        if (tt == 0.0) continue;
        for (int x = 0; x < nA; ++x) {
          const int X = 2 * x + sx;
          acc = fma(tt * t.ft[(size_t)(C2 + X) * d.nP2 + Ap], t.lam[lami(d, U, V, X, Y)], acc);
        }
      }
      return 0.5 * acc;
    }
    case T_E: {  // -1/2 ft_m^v t_{xy}^{um} lambda_{uv}^{xy}, outer (M, U, X)
      const int X = (int)(o % nA2), U = (int)((o / nA2) % nA2), M = (int)(o / ((long)nA2 * nA2));
      const int sv = M & 1;
      for (int Y = 0; Y < nA2; ++Y) {
        const double tt = t.W2T[w2i(d, C2 + U, M, X, Y)];
        if (tt == 0.0) continue;
        for (int v = 0; v < nA; ++v) {
          const int V = 2 * v + sv;
          acc = fma(tt * t.ft[(size_t)M * d.nP2 + V], t.lam[lami(d, U, V, X, Y)], acc);
        }
      }
      return -0.5 * acc;
    }
    case T_GVA: {  // G with one virtual and one active particle, outer (E, U, V)
      const int V = (int)(o % nA2), U = (int)((o / nA2) % nA2);
      const int Ap = nA2 + (int)(o / ((long)nA2 * nA2));
      for (int Cc = 0; Cc < nA2; ++Cc) {
        double tg = 0.0;  // sum_a eta_c^a t_{a e}^{uv}, with the particle pair reversed
        for (int a = 0; a < nA; ++a) {
          const int A = 2 * a + (Cc & 1);
          tg = fma(ea(d, t.gA, Cc, A), t.W1T[w1i(d, C2 + U, V, Ap, A)], tg);
        }
        if (tg == 0.0) continue;
        for (int X = 0; X < nA2; ++X) {
          const int sy = (U & 1) + (V & 1) - (X & 1);  // cumulant spin rule
          if (sy < 0 || sy > 1) continue;
          for (int y = 0; y < nA; ++y) {
            const int Y = 2 * y + sy;
            acc = fma(t.W1Vt[w1i(d, C2 + X, Y, Ap, Cc)] * tg, t.lam[lami(d, U, V, X, Y)], acc);
          }
        }
      }
      return 0.25 * acc;
    }
    case T_GVV: {  // G with two virtual particles, outer (X, Y, U, V)
      const int V = (int)(o % nA2), U = (int)((o / nA2) % nA2), Y = (int)((o / (nA2 * nA2)) % nA2),
                X = (int)(o / (nA2 * nA2 * nA2));
      return 0.125 * t.lam[lami(d, U, V, X, Y)] * s_vv(d, z.nA, t.P12, X, Y, U, V);
    }
    case T_H: {  // 1/8 vt_{kl}^{uv} t_{xy}^{ij} gamma_i^k gamma_j^l lambda_{uv}^{xy}, outer (K, L, X, Y)
      const int Y = (int)(o % nA2), X = (int)((o / nA2) % nA2);
      const long kl = o / ((long)nA2 * nA2);
      const int K = (int)(kl / d.nH2), L = (int)(kl % d.nH2);
      double th = 0.0;
      const int ni = (K < C2) ? 1 : nA, nj = (L < C2) ? 1 : nA;
      for (int ii = 0; ii < ni; ++ii) {
        const int I = (K < C2) ? K : C2 + 2 * ii + (K & 1);
        const double gk = gam_h(d, t.gA, K, I);
        if (gk == 0.0) continue;
        for (int jj = 0; jj < nj; ++jj) {
          const int J = (L < C2) ? L : C2 + 2 * jj + (L & 1);
          th = fma(gk * gam_h(d, t.gA, L, J), t.W2T[w2i(d, I, J, X, Y)], th);
        }
      }
      if (th == 0.0) return 0.0;
      for (int U = 0; U < nA2; ++U) {
        const int sv = (X & 1) + (Y & 1) - (U & 1);
        if (sv < 0 || sv > 1) continue;
        for (int v = 0; v < nA; ++v) {
          const int V = 2 * v + sv;
          acc = fma(t.W2Vt[w2i(d, K, L, U, V)] * th, t.lam[lami(d, U, V, X, Y)], acc);
        }
      }
      return 0.125 * acc;
    }
    case T_I: {  // vt_{jx}^{bu} t_{ay}^{iv} gamma_i^j eta_b^a lambda_{uv}^{xy}, outer (J, Bp, U, X)
      const int X = (int)(o % nA2), U = (int)((o / nA2) % nA2);
      const long jb = o / ((long)nA2 * nA2);
      const int J = (int)(jb / d.nP2), Bp = (int)(jb % d.nP2);
      const double vt = t.W1Vt[w1i(d, J, X, Bp, U)];
      if (vt == 0.0) return 0.0;
      double c = 0.0;
      for (int V = 0; V < nA2; ++V) {
        const int sy = (U & 1) + (V & 1) - (X & 1);
        if (sy < 0 || sy > 1) continue;
        for (int y = 0; y < nA; ++y) {
          const int Y = 2 * y + sy;
          c = fma(t.Ti[w1i(d, J, V, Bp, Y)], t.lam[lami(d, U, V, X, Y)], c);
        }
      }
      return vt * c;
    }
    case T_J: {  // 1/4 vt_{mz}^{uv} t_{xy}^{mw} lambda_{uvw}^{xyz}, outer (M, W, X, Y)
      if (!t.lam3) return 0.0;
      const int Y = (int)(o % nA2), X = (int)((o / nA2) % nA2), W = (int)((o / (nA2 * nA2)) % nA2);
      const int M = (int)(o / ((long)nA2 * nA2 * nA2));
      const double tt = t.W1T[w1i(d, M, W, X, Y)];
      if (tt == 0.0) return 0.0;
      for (int Z = 0; Z < nA2; ++Z)
        for (int U = 0; U < nA2; ++U) {
          // <M Z||U V> conserves spin: s_V = s_M + s_Z - s_U
          const int sv = (M & 1) + (Z & 1) - (U & 1);
          if (sv < 0 || sv > 1) continue;
          // the cumulant conserves spin: s_U + s_V + s_W = s_X + s_Y + s_Z
          if ((U & 1) + sv + (W & 1) != (X & 1) + (Y & 1) + (Z & 1)) continue;
          for (int v = 0; v < nA; ++v) {
            const int V = 2 * v + sv;
            acc = fma(t.W1Vt[w1i(d, M, Z, U, V)], t.lam3[lam3i(nA2, U, V, W, X, Y, Z)], acc);
          }
        }
      return 0.25 * tt * acc;
    }
    case T_K: {  // 1/4 vt_{xy}^{we} t_{ez}^{uv} lambda_{uvw}^{xyz}, outer (E, U, V, Z)
      // vt_{xy}^{we} = <xy||we> = -<xy||ew> = -W1Vt[x, y, e, w]; t_{ez}^{uv} = W1T[u, v, e, z]
      if (!t.lam3) return 0.0;
      const int Z = (int)(o % nA2), V = (int)((o / nA2) % nA2), U = (int)((o / (nA2 * nA2)) % nA2);
      const int Ap = nA2 + (int)(o / ((long)nA2 * nA2 * nA2));
      const double tt = t.W1T[w1i(d, C2 + U, V, Ap, Z)];
      if (tt == 0.0) return 0.0;
      for (int X = 0; X < nA2; ++X)
        for (int Y = 0; Y < nA2; ++Y) {
          // <X Y||E W> conserves spin: s_W = s_X + s_Y - s_E
          const int sw = (X & 1) + (Y & 1) - (Ap & 1);
          if (sw < 0 || sw > 1) continue;
          if ((U & 1) + (V & 1) + sw != (X & 1) + (Y & 1) + (Z & 1)) continue;
          for (int w = 0; w < nA; ++w) {
            const int W = 2 * w + sw;
            acc = fma(t.W1Vt[w1i(d, C2 + X, Y, Ap, W)], t.lam3[lam3i(nA2, U, V, W, X, Y, Z)], acc);
          }
        }
      return -0.25 * tt * acc;
    }
    case T_F4: {  // 1/4 vt_{xu}^{ef} t_{ef}^{yv} gamma_y^x gamma_v^u, outer (X, U, Y, V)
      const int V = (int)(o % nA2), Y = (int)((o / nA2) % nA2), U = (int)((o / (nA2 * nA2)) % nA2),
                X = (int)(o / (nA2 * nA2 * nA2));
      return 0.25 * ga(d, t.gA, X, Y) * ga(d, t.gA, U, V) * s_vv(d, z.nA, t.P12, X, U, Y, V);
    }
    case T_F5: {  // 1/4 vt_{mn}^{vy} t_{ux}^{mn} eta_v^u eta_y^x, outer (M, N, V, Y)
      const int Y = (int)(o % nA2), V = (int)((o / nA2) % nA2);
      const long mn = o / ((long)nA2 * nA2);
      const int M = (int)(mn / C2), N = (int)(mn % C2);
      const double vt = t.W2Vt[w2i(d, M, N, V, Y)];
      if (vt == 0.0) return 0.0;
      for (int u = 0; u < nA; ++u) {
        const int U = 2 * u + (V & 1);
        const double eu = ea(d, t.gA, U, V);
        for (int x = 0; x < nA; ++x) {
          const int X = 2 * x + (Y & 1);
          acc = fma(eu * ea(d, t.gA, X, Y), t.W2T[w2i(d, M, N, U, X)], acc);
        }
      }
      return 0.25 * vt * acc;
    }
    case T_F6: {  // vt_{mx}^{ve} t_{ue}^{my} gamma_y^x eta_v^u, outer (M, E, X, V)
      const int V = (int)(o % nA2), X = (int)((o / nA2) % nA2);
      const long me = o / ((long)nA2 * nA2);
      const int M = (int)(me / d.nV2), Ap = nA2 + (int)(me % d.nV2);
      const double vt = t.W1Vt[w1i(d, M, X, Ap, V)];
      if (vt == 0.0) return 0.0;
      for (int y = 0; y < nA; ++y) {
        const int Y = 2 * y + (X & 1);
        const double gy = ga(d, t.gA, X, Y);
        for (int u = 0; u < nA; ++u) {
          const int U = 2 * u + (V & 1);
          acc = fma(gy * ea(d, t.gA, U, V), t.W1T[w1i(d, M, Y, Ap, U)], acc);
        }
      }
      return vt * acc;
    }
    case T_F7: {  // 1/2 vt_{yz}^{ve} t_{ue}^{wx} gamma_w^y gamma_x^z eta_v^u, outer (E, Y, Z, V)
      const int V = (int)(o % nA2), Z = (int)((o / nA2) % nA2), Y = (int)((o / (nA2 * nA2)) % nA2);
      const int Ap = nA2 + (int)(o / ((long)nA2 * nA2 * nA2));
      const double vt = t.W1Vt[w1i(d, C2 + Y, Z, Ap, V)];
      if (vt == 0.0) return 0.0;
      for (int w = 0; w < nA; ++w) {
        const int W = 2 * w + (Y & 1);
        const double gw = ga(d, t.gA, Y, W);
        for (int x = 0; x < nA; ++x) {
          const int X = 2 * x + (Z & 1);
          const double gg = gw * ga(d, t.gA, Z, X);
          if (gg == 0.0) continue;
          for (int u = 0; u < nA; ++u) {
            const int U = 2 * u + (V & 1);
            acc = fma(gg * ea(d, t.gA, U, V), t.W1T[w1i(d, C2 + W, X, Ap, U)], acc);
          }
        }
      }
      return 0.5 * vt * acc;
    }
    case T_F8: {  // 1/2 vt_{mw}^{vy} t_{ux}^{mz} gamma_z^w eta_v^u eta_y^x, outer (M, W, V, Y)
      const int Y = (int)(o % nA2), V = (int)((o / nA2) % nA2), W = (int)((o / (nA2 * nA2)) % nA2);
      const int M = (int)(o / ((long)nA2 * nA2 * nA2));
      const double vt = t.W1Vt[w1i(d, M, W, V, Y)];
      if (vt == 0.0) return 0.0;
      for (int zz = 0; zz < nA; ++zz) {
        const int Z = 2 * zz + (W & 1);
        const double g = ga(d, t.gA, W, Z);
        if (g == 0.0) continue;
        for (int u = 0; u < nA; ++u) {
          const int U = 2 * u + (V & 1);
          const double ge = g * ea(d, t.gA, U, V);
          for (int x = 0; x < nA; ++x) {
            const int X = 2 * x + (Y & 1);
            acc = fma(ge * ea(d, t.gA, X, Y), t.W1T[w1i(d, M, Z, U, X)], acc);
          }
        }
      }
      return 0.5 * vt * acc;
    }
  }
  return 0.0;
}

constexpr int TERM_NT = 128;
constexpr int TERM_BLOCKS = 608;  // CTAs per term, grid-stride over its outer index

__global__ void __launch_bounds__(TERM_NT) terms_kernel(Sizes z, TermArgs t,
                                                        double* __restrict__ partials) {
  __shared__ double red[TERM_NT / 32];
  const ActDims d = act_dims(z);
  const int term = blockIdx.y;
  if (term == T_F6 || term == T_F7) return;  // term_f6_kernel, term_f7_kernel
  if (term == T_I && z.nA <= 6) return;      // term_i_kernel
  const long n = term_count(term, d);
  double v = 0.0;
  for (long o = (long)blockIdx.x * TERM_NT + threadIdx.x; o < n; o += (long)gridDim.x * TERM_NT)
    v += term_value(term, o, z, d, t);
  const double tot = block_sum<TERM_NT>(v, red);
  if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = tot;
}

static int term_blocks(const Sizes&) { return TERM_BLOCKS; }

// Terms F6 and F7 (Table 2) factorised. Their sums over spin orbitals are
// contractions of small active-index tensors with the spin-diagonal gamma and
// eta, so per virtual (and core) index they are evaluated as chains of matrix
// products in shared memory instead of one nested loop per output entry:
//   F7 = 1/2 sum_E sum_{Y,Z,V} vt[Y,Z,V] S3[Y,Z,V],   vt[Y,Z,V] = Vt_{yz}^{ve},
//        S1[W,X,V] = sum_U t[W,X,U] eta_v^u,  t[W,X,U] = T_{wx}^{ue},
//        S2[W,Z,V] = sum_X gamma_x^z S1[W,X,V],  S3[Y,Z,V] = sum_W gamma_w^y S2[W,Z,V];
//   F6 = sum_{M,E} sum_{X,V} vt[X,V] Q[X,V],   vt[X,V] = Vt_{mx}^{ve},
//        P[X,U] = sum_Y gamma_y^x T_{my}^{ue},  Q[X,V] = sum_U P[X,U] eta_v^u.
// gamma and eta vanish between spin orbitals of different spin, so each sum runs
// over the nA orbitals of one spin. The CTA count and partial slots are those of
// terms_kernel (TERM_BLOCKS per term), which skips these two terms.
template <int NA>
__global__ void __launch_bounds__(TERM_NT) term_f7_kernel(Sizes z, TermArgs t,
                                                          double* __restrict__ partials) {
  constexpr int A2 = 2 * NA, A3 = A2 * A2 * A2;
  extern __shared__ double f7s[];
  double* sa = f7s;        // [A3]
  double* sb = f7s + A3;   // [A3]
  __shared__ double sg[A2 * A2], se[A2 * A2], red[TERM_NT / 32];
  const ActDims d = act_dims(z);
  const int C2 = d.nC2;
  for (int k = threadIdx.x; k < A2 * A2; k += TERM_NT) {
    sg[k] = t.gA[k];
    se[k] = ((k / A2) == (k % A2) ? 1.0 : 0.0) - t.gA[k];
  }
  double acc = 0.0;
  for (int e = blockIdx.x; e < d.nV2; e += gridDim.x) {
    const int Ap = A2 + e;
    __syncthreads();
    for (int k = threadIdx.x; k < A3; k += TERM_NT) {  // t[W,X,U], U fastest
      const int U = k % A2, X = (k / A2) % A2, W = k / (A2 * A2);
      sa[k] = t.W1T[w1i(d, C2 + W, X, Ap, U)];
    }
    __syncthreads();
    for (int k = threadIdx.x; k < A3; k += TERM_NT) {  // S1[W,X,V] = sum_U t[W,X,U] eta[U,V]
      const int V = k % A2, WX = k / A2;
      double v = 0.0;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        const int U = 2 * u + (V & 1);
        v = fma(sa[WX * A2 + U], se[U * A2 + V], v);
      }
      sb[k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < A3; k += TERM_NT) {  // S2[W,Z,V] = sum_X gamma[Z,X] S1[W,X,V]
      const int V = k % A2, Z = (k / A2) % A2, W = k / (A2 * A2);
      double v = 0.0;
#pragma unroll
      for (int x = 0; x < NA; ++x) {
        const int X = 2 * x + (Z & 1);
        v = fma(sg[Z * A2 + X], sb[(W * A2 + X) * A2 + V], v);
      }
      sa[k] = v;
    }
    __syncthreads();
    for (int k = threadIdx.x; k < A3; k += TERM_NT) {  // vt[Y,Z,V] * sum_W gamma[Y,W] S2[W,Z,V]
      const int V = k % A2, Z = (k / A2) % A2, Y = k / (A2 * A2);
      double v = 0.0;
#pragma unroll
      for (int w = 0; w < NA; ++w) {
        const int W = 2 * w + (Y & 1);
        v = fma(sg[Y * A2 + W], sa[(W * A2 + Z) * A2 + V], v);
      }
      acc = fma(t.W1Vt[w1i(d, C2 + Y, Z, Ap, V)], v, acc);
    }
  }
  const double tot = block_sum<TERM_NT>(0.5 * acc, red);
  if (threadIdx.x == 0) partials[(size_t)T_F7 * gridDim.x + blockIdx.x] = tot;
}

template <int NA>
__global__ void __launch_bounds__(TERM_NT) term_f6_kernel(Sizes z, TermArgs t,
                                                          double* __restrict__ partials) {
  constexpr int A2 = 2 * NA, NW = TERM_NT / 32;
  __shared__ double sT[NW][A2 * A2], sP[NW][A2 * A2];
  __shared__ double sg[A2 * A2], se[A2 * A2], red[NW];
  const ActDims d = act_dims(z);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < A2 * A2; k += TERM_NT) {
    sg[k] = t.gA[k];
    se[k] = ((k / A2) == (k % A2) ? 1.0 : 0.0) - t.gA[k];
  }
  __syncthreads();
  double acc = 0.0;
  const long n = (long)d.nC2 * d.nV2;
  for (long me = (long)blockIdx.x * NW + warp; me < n; me += (long)gridDim.x * NW) {
    const int M = (int)(me / d.nV2), Ap = A2 + (int)(me % d.nV2);
    for (int k = lane; k < A2 * A2; k += 32)  // T[Y,U] = T_{my}^{ue}
      sT[warp][k] = t.W1T[w1i(d, M, k / A2, Ap, k % A2)];
    __syncwarp();
    for (int k = lane; k < A2 * A2; k += 32) {  // P[X,U] = sum_Y gamma[X,Y] T[Y,U]
      const int X = k / A2, U = k % A2;
      double v = 0.0;
#pragma unroll
      for (int y = 0; y < NA; ++y) {
        const int Y = 2 * y + (X & 1);
        v = fma(sg[X * A2 + Y], sT[warp][Y * A2 + U], v);
      }
      sP[warp][k] = v;
    }
    __syncwarp();
    for (int k = lane; k < A2 * A2; k += 32) {  // vt[X,V] * sum_U P[X,U] eta[U,V]
      const int X = k / A2, V = k % A2;
      double v = 0.0;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        const int U = 2 * u + (V & 1);
        v = fma(sP[warp][X * A2 + U], se[U * A2 + V], v);
      }
      acc = fma(t.W1Vt[w1i(d, M, X, Ap, V)], v, acc);
    }
    __syncwarp();
  }
  const double tot = block_sum<TERM_NT>(acc, red);
  if (threadIdx.x == 0) partials[(size_t)T_F6 * gridDim.x + blockIdx.x] = tot;
}

// Term I, vt_{jx}^{bu} Ti_{jv}^{by} lambda_{uv}^{xy} summed over (J, B, U, X, V, Y),
// for nA <= 6: the spin-orbital cumulant is staged once per CTA in shared memory,
// transposed to [V][Y][U][X] so that the lanes (consecutive X) read consecutive
// entries, and the dressed Ti rows of TI_ROWS (J, B) pairs at a time beside it.
constexpr int TI_ROWS = 8, TI_NT = 256;
template <int NA>
__global__ void __launch_bounds__(TI_NT) term_i_kernel(Sizes z, TermArgs t,
                                                       double* __restrict__ partials) {
  constexpr int A2 = 2 * NA, AA = A2 * A2, A4 = AA * AA;
  extern __shared__ double ism[];
  double* lamT = ism;       // [V][Y][U][X]
  double* sTi = ism + A4;   // [TI_ROWS][V][Y]
  __shared__ double red[TI_NT / 32];
  const ActDims d = act_dims(z);
  for (int k = threadIdx.x; k < A4; k += TI_NT) {
    const int X = k % A2, U = (k / A2) % A2, Y = (k / AA) % A2, V = k / (AA * A2);
    lamT[k] = t.lam[lami(d, U, V, X, Y)];
  }
  double acc = 0.0;
  const long n = (long)d.nH2 * d.nP2;
  for (long r0 = (long)blockIdx.x * TI_ROWS; r0 < n; r0 += (long)gridDim.x * TI_ROWS) {
    __syncthreads();  // the previous rows' reads are done (and the cumulant is staged)
    for (int k = threadIdx.x; k < TI_ROWS * AA; k += TI_NT) {
      const long r = r0 + k / AA;
      double v = 0.0;
      if (r < n) {
        const int J = (int)(r / d.nP2), Bp = (int)(r % d.nP2), V = (k % AA) / A2, Y = k % A2;
        v = t.Ti[w1i(d, J, V, Bp, Y)];
      }
      sTi[k] = v;
    }
    __syncthreads();
    // only spin-allowed (U, X): vt_{jx}^{bu} conserves spin, s_J + s_X = s_B + s_U, so a
    // row with s_J = s_B has 2 nA^2 pairs (U and X alike) and any other row nA^2
    // (U of spin s_J, X of spin s_B)
    constexpr int NUX = 2 * NA * NA;
    for (int k = threadIdx.x; k < TI_ROWS * NUX; k += TI_NT) {
      const long r = r0 + k / NUX;
      if (r >= n) break;
      const int J = (int)(r / d.nP2), Bp = (int)(r % d.nP2);
      const int sJ = J & 1, sB = Bp & 1, m = k % NUX;
      int U, X;
      if (sJ == sB) {
        const int mm = m % (NA * NA), sp = m / (NA * NA);
        U = 2 * (mm / NA) + sp;
        X = 2 * (mm % NA) + sp;
      } else {
        if (m >= NA * NA) continue;
        U = 2 * (m / NA) + sJ;
        X = 2 * (m % NA) + sB;
      }
      const double vt = t.W1Vt[w1i(d, J, X, Bp, U)];
      if (vt == 0.0) continue;
      const double* ti = sTi + (k / NUX) * AA;
      double c = 0.0;
#pragma unroll
      for (int V = 0; V < A2; ++V) {
        const int sy = (U & 1) + (V & 1) - (X & 1);  // cumulant spin rule
        if (sy < 0 || sy > 1) continue;
#pragma unroll
        for (int y = 0; y < NA; ++y) {
          const int Y = 2 * y + sy;
          c = fma(ti[V * A2 + Y], lamT[((V * A2 + Y) * A2 + U) * A2 + X], c);
        }
      }
      acc = fma(vt, c, acc);
    }
  }
  const double tot = block_sum<TI_NT>(acc, red);
  if (threadIdx.x == 0) partials[(size_t)T_I * gridDim.x + blockIdx.x] = tot;
}

static size_t ti_smem_bytes(int nA) {
  const size_t aa = 4 * (size_t)nA * nA;
  return (aa * aa + TI_ROWS * aa) * sizeof(double);
}

static size_t f7_smem_bytes(int nA) {
  const size_t a2 = 2 * (size_t)nA;
  return 2 * a2 * a2 * a2 * sizeof(double);
}

bool active_alloc(dsrg_plan* p) {
  const Sizes& z = p->z;
  if (z.nA == 0) return true;
  const ActDims d = act_dims(z);
  ActiveWs& w = p->act;
  w.w1n = (size_t)d.nH2 * d.nA2 * d.nP2 * d.nA2;
  w.w2n = (size_t)d.nH2 * d.nH2 * d.nA2 * d.nA2;
  const size_t n12 = (size_t)z.nH * z.nA * z.nA * z.nP;
  const size_t n3 = (size_t)z.nH * z.nA * z.nH * z.nA;
  const size_t nA4 = (size_t)z.nA * z.nA * z.nA * z.nA;
  w.actvv_blocks = ACTVV_BLOCKS;
  bool ok = true;
  ok = ok && plan_alloc(p, (void**)&w.K1, n12 * 8);
  ok = ok && plan_alloc(p, (void**)&w.K2, n12 * 8);
  ok = ok && plan_alloc(p, (void**)&w.K3, n3 * 8);
  ok = ok && plan_alloc(p, (void**)&w.W1, 3 * w.w1n * 8);
  ok = ok && plan_alloc(p, (void**)&w.W2, 3 * w.w2n * 8);
  ok = ok && plan_alloc(p, (void**)&w.Ti, w.w1n * 8);
  ok = ok && plan_alloc(p, (void**)&w.lam, (size_t)d.nA2 * d.nA2 * d.nA2 * d.nA2 * 8);
  ok = ok && plan_alloc(p, (void**)&w.gA, (size_t)d.nA2 * d.nA2 * 8);
  ok = ok && plan_alloc(p, (void**)&w.t1, (size_t)d.nH2 * d.nP2 * 8);
  ok = ok && plan_alloc(p, (void**)&w.ft, (size_t)d.nH2 * d.nP2 * 8);
  ok = ok && plan_alloc(p, (void**)&w.M, (size_t)z.nA * z.nA * z.nV * z.nV * 8);
  ok = ok && plan_alloc(p, (void**)&w.P12, 2 * nA4 * 8);
  ok = ok && plan_alloc(p, (void**)&w.P12part, (size_t)ACTVV_BLOCKS * 2 * nA4 * 8);
  return ok;
}

int active_plan(dsrg_plan* p, int first_partial) {
  if (p->z.nA == 0) {
    // no active orbitals: one partial per core orbital for the f^(1) singles
    p->segs.push_back(Segment{first_partial, p->z.nC, BLK_ACTIVE});
    p->seg_active.push_back((int)p->segs.size() - 1);
    return p->z.nC;
  }
  const int nb = term_blocks(p->z) * N_TERMS;
  p->segs.push_back(Segment{first_partial, nb, BLK_ACTIVE});
  p->seg_active.push_back((int)p->segs.size() - 1);
  return nb;
}

cudaError_t launch_gram_aavv_fp64(dsrg_plan* p, const double* B) {
  const Sizes& z = p->z;
  if (z.nA == 0) return cudaSuccess;
  const int nt = (z.nV + 63) / 64;
  gram_aavv_kernel<<<z.nA * z.nA * nt * nt, 256, 0, p->stream>>>(B, z, nt, p->act.M);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

cudaError_t launch_active(dsrg_plan* p, const double* B, const double* eps, const double* G,
                          const double* L, const double* L3, const double* F1, double s,
                          bool ints_ready) {
  const Sizes& z = p->z;
  if (z.nA == 0) {
    const Segment& sg = p->segs[p->seg_active[0]];
    singles_kernel<<<z.nC, 128, 0, p->stream>>>(eps, s, z, F1, p->d_partials + sg.begin);
    DSRG_LAUNCH_CHECK(p);
    return cudaSuccess;
  }
  ActiveWs& w = p->act;
  const ActDims d = act_dims(z);
  cudaStream_t st = p->stream;
  if (!ints_ready) {
    const size_t n = 2 * (size_t)z.nH * z.nA * z.nA * z.nP + (size_t)z.nH * z.nA * z.nH * z.nA;
    small_ints_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(B, z, w.K1, w.K2, w.K3);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    const size_t n = w.w1n / 16 + w.w2n / 16 + (size_t)d.nA2 * d.nA2 * d.nA2 * d.nA2 +
                     (size_t)d.nA2 * d.nA2;
    build_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(
        eps, G, L, s, z, w.K1, w.K2, w.K3, w.W1, w.W2, w.lam, w.gA, w.w1n, w.w2n);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    const int n = d.nH2 * d.nP2;
    t1_kernel<<<(n + 255) / 256, 256, 0, st>>>(eps, s, z, w.W1 + w.w1n, w.gA, F1, w.t1, w.ft);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    ti_kernel<<<(unsigned)((w.w1n + 255) / 256), 256, 0, st>>>(z, w.W1 + w.w1n, w.gA, w.Ti, w.w1n);
    DSRG_LAUNCH_CHECK(p);
  }
  if (!ints_ready) {
    cudaError_t e = launch_gram_aavv_fp64(p, B);
    if (e != cudaSuccess) return e;
  }
  const int nA4 = z.nA * z.nA * z.nA * z.nA;
  {
    const size_t smg = (size_t)3 * z.nA * z.nA * ACTVV_CH * sizeof(double);
    // factor tables of the split path (tc_rest.cu) when this call formed them
    ActFact F{nullptr, nullptr, nullptr, 0};
    if (ints_ready) rest_act_tables(p, &F.alpha, &F.pinfo, &F.tau, &F.ld);
#define ACTVV_GEN(NA_)                                                                       \
  case NA_:                                                                                  \
    if (ints_ready) {                                                                        \
      raise_smem_limit((const void*)actvv_gen_kernel<NA_, true>, smg);                       \
      actvv_gen_kernel<NA_, true><<<ACTVV_BLOCKS, 256, smg, st>>>(eps, s, z, w.M, F, w.P12part); \
    } else {                                                                                 \
      raise_smem_limit((const void*)actvv_gen_kernel<NA_, false>, smg);                      \
      actvv_gen_kernel<NA_, false><<<ACTVV_BLOCKS, 256, smg, st>>>(eps, s, z, w.M, F, w.P12part); \
    }                                                                                        \
    break;
    switch (z.nA) {
      case 1:
        if (ints_ready)
          actvv_small_kernel<1, true><<<ACTVV_BLOCKS, 256, 0, st>>>(eps, s, z, w.M, F, w.P12part);
        else
          actvv_small_kernel<1, false><<<ACTVV_BLOCKS, 256, 0, st>>>(eps, s, z, w.M, F, w.P12part);
        break;
      case 2:
        if (ints_ready)
          actvv_small_kernel<2, true><<<ACTVV_BLOCKS, 256, 0, st>>>(eps, s, z, w.M, F, w.P12part);
        else
          actvv_small_kernel<2, false><<<ACTVV_BLOCKS, 256, 0, st>>>(eps, s, z, w.M, F, w.P12part);
        break;
      ACTVV_GEN(3) ACTVV_GEN(4) ACTVV_GEN(5) ACTVV_GEN(6) ACTVV_GEN(7) ACTVV_GEN(8)
      default: {
        dim3 grid(ACTVV_BLOCKS, nA4);
        actvv_kernel<<<grid, 256, 0, st>>>(eps, s, z, w.M, w.P12part);
      }
    }
#undef ACTVV_GEN
    DSRG_LAUNCH_CHECK(p);
    actvv_reduce_kernel<<<(2 * nA4 + 127) / 128, 128, 0, st>>>(nA4, ACTVV_BLOCKS, w.P12part, w.P12);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    TermArgs ta;
    ta.W1V = w.W1;
    ta.W1T = w.W1 + w.w1n;
    ta.W1Vt = w.W1 + 2 * w.w1n;
    ta.W2V = w.W2;
    ta.W2T = w.W2 + w.w2n;
    ta.W2Vt = w.W2 + 2 * w.w2n;
    ta.Ti = w.Ti;
    ta.lam = w.lam;
    ta.gA = w.gA;
    ta.t1 = w.t1;
    ta.ft = w.ft;
    ta.P12 = w.P12;
    ta.lam3 = L3;
    const Segment& sg = p->segs[p->seg_active[0]];
    dim3 grid(term_blocks(z), N_TERMS);
    terms_kernel<<<grid, TERM_NT, 0, st>>>(z, ta, p->d_partials + sg.begin);
    DSRG_LAUNCH_CHECK(p);
    const size_t smf7 = f7_smem_bytes(z.nA), smti = ti_smem_bytes(z.nA);
#define F67_LAUNCH(NA_)                                                                        \
  case NA_:                                                                                    \
    raise_smem_limit((const void*)term_f7_kernel<NA_>, smf7);                                  \
    term_f7_kernel<NA_><<<term_blocks(z), TERM_NT, smf7, st>>>(z, ta, p->d_partials + sg.begin); \
    DSRG_LAUNCH_CHECK(p);                                                                      \
    term_f6_kernel<NA_><<<term_blocks(z), TERM_NT, 0, st>>>(z, ta, p->d_partials + sg.begin);   \
    if (NA_ <= 6) {                                                                            \
      DSRG_LAUNCH_CHECK(p);                                                                    \
      raise_smem_limit((const void*)term_i_kernel<(NA_ <= 6 ? NA_ : 6)>, smti);                \
      term_i_kernel<(NA_ <= 6 ? NA_ : 6)><<<term_blocks(z), TI_NT, smti, st>>>(                \
          z, ta, p->d_partials + sg.begin);                                                     \
    }                                                                                          \
    break;
    switch (z.nA) {
      F67_LAUNCH(1) F67_LAUNCH(2) F67_LAUNCH(3) F67_LAUNCH(4)
      F67_LAUNCH(5) F67_LAUNCH(6) F67_LAUNCH(7) F67_LAUNCH(8)
      default: return cudaErrorInvalidValue;
    }
#undef F67_LAUNCH
    DSRG_LAUNCH_CHECK(p);
  }
  return cudaSuccess;
}

bool ccav_supported(const Sizes& z) { return ccav_smem(z) <= 200 * 1024; }

}  // namespace dsrg
