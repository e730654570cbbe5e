// Split-precision CAVV (diagram F2), CCAV (diagram F3) and the integrals of
// the active block from one tensor-core GEMM over the hi/lo planes of CCVV.
//
// Every one of these quantities is a product of two rows of the hole x
// particle factors B: (ge|uf), (ge|hx), (hx|h'y) with g, h holes, u an
// active hole, e, f virtuals and x, y active particles. The planes already
// hold the rows (g, e) for every hole g and virtual e (K-major over Q); the
// rows (h, x) of the active particles are appended to them (nH*nA rows,
// padded to 64). One GEMM
//     Y = P[(g,e)] . P[(u,f) ; (h,x)]^T       (hi.hi + hi.lo + lo.hi, FP32 accumulation,
//                                              + lo.lo on tiles where the rows overlap;
//                                              the first 32 auxiliary functions are added
//                                              in the epilogue in FP32 round-to-nearest)
// then holds, at row (g, e):
//     columns u*nVpad + f   ->  (ge|uf) = X_u[e,f] of F2 for g = m core,
//                               M_xu[e,f] = (xe|uf) for g = x active
//     columns XC + h*nA + x ->  (ge|hx): Z_u[m,n,e] = (me|nu) of F3, and the
//                               virtual parts of (ia|ux), (ix|ua)
// (Sec. III step 4: the integrals with active indices are formed explicitly,
// then contracted). FP64 kernels then evaluate the F2 and F3 energies with
// FP64 regulators, and gather the active-block integrals; (hx|h'y), which
// has no virtual index, is formed in FP64 from B directly.
//
// The GEMM kernel (one CTA per SM, persistent, tiles 128 x 256):
//   warp 0      TMA producer (one elected thread)
//   warp 1      TMEM allocator and MMA issuer (one elected thread)
//   warps 2-5   epilogue: TMEM -> registers -> FP32 stores of Y
// Shared memory: 4 stages x (A 128 rows + B 256 rows) x 2 planes x 64 B, 64-byte
// swizzle. TMEM: 2 buffers x 256 columns. Every wait is bounded (about 2 s).
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "regulators.cuh"
#include "tc_common.cuh"

namespace dsrg {

constexpr int G_BM = 128, G_BN = 256;
constexpr int G_KB = 64;                              // K bytes per row per stage
constexpr int G_STAGES = 4;
constexpr int G_A_BYTES = G_BM * G_KB;                // 8 KB per plane
constexpr int G_B_BYTES = G_BN * G_KB;                // 16 KB per plane
constexpr int G_STAGE_BYTES = 2 * (G_A_BYTES + G_B_BYTES);
constexpr int G_THREADS = 192;
constexpr uint32_t G_TMEM_COLS = 512;
constexpr int XROW_ALIGN = 64;
constexpr int F2_T = 32;                              // F2 epilogue tile edge

struct TcGemmArgs {
  int a_row0;        // row r of Y is plane row a_row0 + r
  int b_row0;        // column c of Y is plane row b_row0 + c
  int m_tiles, n_tiles;
  int kblocks;        // K stages on the tensor cores: Q from kq0 to the padded end
  int kq0;            // = TAIL_Q: Q < kq0 is added in the epilogue from `tail`
  const float* tail;  // [plane rows + TAIL_PAD][TAIL_Q] fl32(B) of Q < TAIL_Q
  float* Y;
  long long ldy;
  int* status;
};

__host__ __device__ constexpr uint32_t idesc_mn(bool bf16, uint32_t m, uint32_t n) {
  return (1u << 4) | ((bf16 ? 1u : 2u) << 7) | ((bf16 ? 1u : 2u) << 10) | ((n >> 3) << 17) |
         ((m >> 4) << 24);
}

// The MMAs of one K stage of one tile (two K steps). K runs from the last
// auxiliary function to the first and the cross products go before hi*hi: the
// FP32 accumulator truncates toward zero at every instruction, and with
// factors that decrease along Q this keeps it small until the largest terms
// arrive. GRAM (the tile's A rows and B rows overlap, so its diagonal holds
// squares sum_Q P_r^2) also keeps lo*lo, whose omission would bias them low.
template <bool BF16, bool GRAM>
__device__ __forceinline__ void gemm_stage_mmas(uint32_t d, uint32_t sa, uint32_t sb, int kb) {
  constexpr uint32_t idesc = idesc_mn(BF16, G_BM, G_BN);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint32_t off = (uint32_t)((1 - k) * 32);
    const uint64_t ah = desc_sw64(sa + off), al = desc_sw64(sa + G_A_BYTES + off);
    const uint64_t bh = desc_sw64(sb + off), bl = desc_sw64(sb + G_B_BYTES + off);
    const uint32_t acc0 = (kb > 0 || k > 0) ? 1u : 0u;
    if (GRAM) {
      tc_mma<BF16>(d, al, bl, idesc, acc0);
      tc_mma<BF16>(d, al, bh, idesc, 1u);
    } else {
      tc_mma<BF16>(d, al, bh, idesc, acc0);
    }
    tc_mma<BF16, 1>(d, ah, bl, idesc, 1u);
    tc_mma<BF16, 2>(d, ah, bh, idesc, 1u);
  }
}

template <bool BF16>
__global__ void __launch_bounds__(G_THREADS, 1)
    split_gemm_kernel(const __grid_constant__ CUtensorMap map_hi,
                      const __grid_constant__ CUtensorMap map_lo, const TcGemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* tiles = smem;
  uint64_t* full = (uint64_t*)(smem + G_STAGES * G_STAGE_BYTES);
  uint64_t* empty = full + G_STAGES;
  uint64_t* tfull = empty + G_STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = a.m_tiles * a.n_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < G_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 4);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(G_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_hi) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_lo) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        const int arow = a.a_row0 + (it / a.n_tiles) * G_BM;
        const int brow = a.b_row0 + (it % a.n_tiles) * G_BN;
        for (int kb = 0; kb < a.kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.status)) {
            ok = false;
            break;
          }
          uint8_t* st = tiles + stage * G_STAGE_BYTES;
          mbar_expect_tx(&full[stage], (uint32_t)G_STAGE_BYTES);
          // the last auxiliary functions first (see the K order of the MMA issuer)
          const int kq = a.kq0 + (a.kblocks - 1 - kb) * (G_KB / (BF16 ? 2 : 4));
          tma_load_2d(st, &map_hi, &full[stage], kq, arow);
          tma_load_2d(st + G_A_BYTES, &map_lo, &full[stage], kq, arow);
          uint8_t* sb = st + 2 * G_A_BYTES;
          tma_load_2d(sb, &map_hi, &full[stage], kq, brow);
          tma_load_2d(sb + G_A_BYTES, &map_hi, &full[stage], kq, brow + G_BM);
          tma_load_2d(sb + G_B_BYTES, &map_lo, &full[stage], kq, brow);
          tma_load_2d(sb + G_B_BYTES + G_A_BYTES, &map_lo, &full[stage], kq, brow + G_BM);
          if (++stage == G_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        int s = stage;
        uint32_t ph = phase;
        for (int k = 0; k < G_STAGES; ++k) {
          if (--s < 0) {
            s = G_STAGES - 1;
            ph ^= 1u;
          }
          const unsigned long long t0 = gtimer();
          while (!mbar_try(&full[s], ph) && gtimer() - t0 < TC_WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      int tbuf = 0;
      uint32_t tphase = 0;
      bool ok = true, issued = false;
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        if (!mbar_wait(&tempty[tbuf], tphase ^ 1u, abort_flag, a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t d = tmem_base + (uint32_t)(tbuf * G_BN);
        const int arow = a.a_row0 + (it / a.n_tiles) * G_BM;
        const int brow = a.b_row0 + (it % a.n_tiles) * G_BN;
        const bool gram = arow < brow + G_BN && brow < arow + G_BM;
        for (int kb = 0; kb < a.kblocks; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sa = su32(tiles + stage * G_STAGE_BYTES);
          const uint32_t sb = sa + 2 * G_A_BYTES;
          if (gram)
            gemm_stage_mmas<BF16, true>(d, sa, sb, kb);
          else
            gemm_stage_mmas<BF16, false>(d, sa, sb, kb);
          issued = true;
          tc_commit(&empty[stage]);
          if (++stage == G_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(&tfull[tbuf]);
        if (++tbuf == 2) {
          tbuf = 0;
          tphase ^= 1u;
        }
      }
      if (!ok && issued) {
        tc_commit(drain);
        const unsigned long long t0 = gtimer();
        while (!mbar_try(drain, 0) && gtimer() - t0 < TC_WAIT_NS) {
        }
      }
    }
  } else {
    // epilogue: warp w reads TMEM lanes 32*(w%4).. (its row of the tile)
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    int tbuf = 0;
    uint32_t tphase = 0;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
      const bool ok = mbar_wait(&tfull[tbuf], tphase, abort_flag, a.status);
      tc_fence_after();
      if (ok) {
        const uint32_t t = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tbuf * G_BN);
        float* y = a.Y + (size_t)((it / a.n_tiles) * G_BM + row) * a.ldy + (it % a.n_tiles) * G_BN;
        const float* ta = a.tail + (size_t)(a.a_row0 + (it / a.n_tiles) * G_BM + row) * TAIL_Q;
        const float* tb = a.tail + (size_t)(a.b_row0 + (it % a.n_tiles) * G_BN) * TAIL_Q;
        for (int c0 = 0; c0 < G_BN; c0 += 32) {
          uint32_t r0[16], r1[16];
          tmem_ld16(t + c0, r0);
          tmem_ld16(t + c0 + 16, r1);
          tmem_ld_wait();
          // the first TAIL_Q auxiliary functions in FP32 round-to-nearest
          tail_add16(ta, tb + (size_t)c0 * TAIL_Q, r0);
          tail_add16(ta, tb + (size_t)(c0 + 16) * TAIL_Q, r1);
          float4* o = (float4*)(y + c0);
#pragma unroll
          for (int q = 0; q < 4; ++q)
            o[q] = make_float4(__uint_as_float(r0[4 * q]), __uint_as_float(r0[4 * q + 1]),
                               __uint_as_float(r0[4 * q + 2]), __uint_as_float(r0[4 * q + 3]));
#pragma unroll
          for (int q = 0; q < 4; ++q)
            o[4 + q] = make_float4(__uint_as_float(r1[4 * q]), __uint_as_float(r1[4 * q + 1]),
                                   __uint_as_float(r1[4 * q + 2]), __uint_as_float(r1[4 * q + 3]));
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[tbuf]);
      if (++tbuf == 2) {
        tbuf = 0;
        tphase ^= 1u;
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(G_TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Active-particle rows of the planes and their FP64 copy.
//   plane row xrow0 + h*nA + x  =  B[Q][h][x]  (split like the main rows)
//   Xq[(h*nA + x) * Q + q]      =  B[q][h][x]  (FP64)
// ---------------------------------------------------------------------------
template <bool BF16>
__global__ void xrows_kernel(const double* __restrict__ B, Sizes z, long long xrow0, int Qld,
                             void* __restrict__ hi, void* __restrict__ lo, double* __restrict__ Xq,
                             float* __restrict__ tail) {
  const int T = z.nH * z.nA;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)T * z.Q) return;
  const int t = (int)(k / z.Q), q = (int)(k % z.Q);
  const int h = t / z.nA, x = t % z.nA;
  const double v = B[bidx(z, q, h, x)];
  Xq[k] = v;
  const size_t o = (size_t)(xrow0 + t) * Qld + q;
  // the same split of fl32(B) as the main plane rows
  const float vf = (float)v;
  if (q < TAIL_Q) tail[(size_t)(xrow0 + t) * TAIL_Q + q] = vf;
  if (BF16) {
    const __nv_bfloat16 vh = __float2bfloat16_rn(vf);
    ((__nv_bfloat16*)hi)[o] = vh;
    ((__nv_bfloat16*)lo)[o] = __float2bfloat16_rn(vf - __bfloat162float(vh));
  } else {
    uint32_t u = __float_as_uint(vf);
    if ((u & 0x7f800000u) != 0x7f800000u) u = (u + 0xfffu + ((u >> 13) & 1u)) & 0xffffe000u;
    const float vh = __uint_as_float(u);
    uint32_t w = __float_as_uint(vf - vh);
    if ((w & 0x7f800000u) != 0x7f800000u) w = (w + 0xfffu + ((w >> 13) & 1u)) & 0xffffe000u;
    ((float*)hi)[o] = vh;
    ((float*)lo)[o] = __uint_as_float(w);
  }
}

// (hx|h'y) in FP64: one warp per pair t1 <= t2 of active-particle rows.
__global__ void xx_gram_kernel(const double* __restrict__ Xq, int T, int Q, double* __restrict__ Gxx) {
  const int w = (int)(((size_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5), lane = threadIdx.x & 31;
  const int npair = T * (T + 1) / 2;
  if (w >= npair) return;
  int t1 = 0, r = w;
  while (r >= T - t1) {
    r -= T - t1;
    ++t1;
  }
  const int t2 = t1 + r;
  const double* a = Xq + (size_t)t1 * Q;
  const double* b = Xq + (size_t)t2 * Q;
  double acc = 0.0;
  for (int q = lane; q < Q; q += 32) acc = fma(a[q], b[q], acc);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if (lane == 0) {
    Gxx[(size_t)t1 * T + t2] = acc;
    Gxx[(size_t)t2 * T + t1] = acc;
  }
}

// Factors of exp(-s D_u^2), D_u = E_mu - e_a - e_b, E_mu = e_m + e_u, for the
// pairs mu = (m core, u active) and then (x active, u active) (the active VV
// sums of the active block).
__global__ void cavv_tables_kernel(const double* __restrict__ eps, double s, Sizes z, int nVpad,
                                   double* __restrict__ alpha, double* __restrict__ pinfo,
                                   double* __restrict__ tau1, const double* __restrict__ vmaxp) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ve = z.nC + z.nA;
  const int nmu = (z.nC + z.nA) * z.nA;
  const size_t na = (size_t)nmu * nVpad, nt = (size_t)nVpad * nVpad;
  if (k < na) {
    const int mu = (int)(k / nVpad), b = (int)(k % nVpad);
    const int m = mu / z.nA, u = mu % z.nA;  // m < nC: core; m >= nC: active x = m - nC
    const double E = eps[m] + eps[z.nC + u];
    alpha[k] = (b < z.nV) ? exp(2.0 * s * E * eps[ve + b]) : 0.0;
    if (b == 0) {
      const double vmax = *vmaxp;  // max |e_v| over the virtual orbitals
      // factors are multiplied left to right (pair, row, column, table); the partial
      // products carry -sE^2 + 2sE e_e (+ 2sE e_f), bounded by the sum of magnitudes
      const bool ok = (s * E * E + 4.0 * s * fabs(E) * vmax <= 700.0) &&
                      (4.0 * s * vmax * vmax <= 700.0);
      pinfo[4 * mu + 0] = E;
      pinfo[4 * mu + 1] = exp(-s * E * E);
      pinfo[4 * mu + 2] = ok ? 1.0 : 0.0;
      pinfo[4 * mu + 3] = 0.0;
    }
  } else if (k < na + nt) {
    const size_t r = k - na;
    const int aa = (int)(r / nVpad), bb = (int)(r % nVpad);
    double v = 0.0;
    if (aa < z.nV && bb < z.nV) {
      const double t = eps[ve + aa] + eps[ve + bb];
      v = exp(-s * t * t);
    }
    tau1[r] = v;
  }
}

// ---------------------------------------------------------------------------
// F2 (CAVV), spin-adapted (closed-shell spin sum of Table 2's F2):
//   F2 = sum_m sum_{u,v} G_uv sum_ef X_u[e,f] (2 X_v[e,f] - X_v[f,e]) Rv_u Rt_v,
//   X_u[e,f] = (me|uf), D_u = e_m + e_u - e_e - e_f,
//   Rv_u = 1 + exp(-s D_u^2) (Eq. (15)), Rt_v = (1 - exp(-s D_v^2)) / D_v (Eq. (13)).
// One CTA per (m, 32 x 32 tile pair E <= F); for E < F each position (e,f) also
// adds its mirror (f,e), whose X_u[f,e] is the same CTA's transposed tile.
// exp(-s D_u^2) = exp(-s E^2) exp(2 s E e_e) exp(2 s E e_f) exp(-s (e_e + e_f)^2);
// 1/D_u is an FP32 seed with one FP64 Newton step; |D_u| < 1/4 (or a pair whose
// factors could overflow) takes expm1 and an FP64 divide.
// ---------------------------------------------------------------------------
template <int NA>
__global__ void __launch_bounds__(256) cavv_f2_kernel(const float* __restrict__ Y, long long ldy,
                                                      int nVpad, const double* __restrict__ eps,
                                                      const double* __restrict__ G, double s, Sizes z,
                                                      const int2* __restrict__ tps, int n_tp,
                                                      const double* __restrict__ alpha,
                                                      const double* __restrict__ pinfo,
                                                      const double* __restrict__ tau1,
                                                      double* __restrict__ partials,
                                                      unsigned long long* __restrict__ counts) {
  extern __shared__ float f2s[];
  float* sX = f2s;                              // [NA][32][33]   X_u[e,f]
  float* sXt = sX + NA * F2_T * (F2_T + 1);     // [NA][32][33]   X_u[f,e]
  // sBAe = beta_u * alpha_u(e): the row factor of exp(-s D^2) with the pair factor folded in
  __shared__ double sBAe[NA][F2_T], sAf[NA][F2_T], sEe[F2_T], sEf[F2_T], sG[NA * NA];
  __shared__ double sE[NA];
  // FP32 copies: e_e + e_f and E_u for the path test and the reciprocal seed;
  // G as FP32 head + FP32 remainder for the far path's FP32 sums
  __shared__ float sEeF[F2_T], sEfF[F2_T], sEF[NA], sGh[NA * NA], sGl[NA * NA];
  __shared__ int sFact, sFar;
  __shared__ double red[8];
  const int m = blockIdx.x / n_tp;
  const int2 ab = tps[blockIdx.x % n_tp];
  const int E0 = ab.x * F2_T, F0 = ab.y * F2_T;
  const int ve = z.nC + z.nA;
  const float* Ym = Y + (size_t)m * nVpad * ldy;
  for (int k = threadIdx.x; k < NA * F2_T * F2_T; k += 256) {
    const int u = k / (F2_T * F2_T), r = (k / F2_T) % F2_T, c = k % F2_T;
    sX[(u * F2_T + r) * (F2_T + 1) + c] = Ym[(size_t)(E0 + r) * ldy + u * nVpad + F0 + c];
    sXt[(u * F2_T + c) * (F2_T + 1) + r] = Ym[(size_t)(F0 + r) * ldy + u * nVpad + E0 + c];
  }
  if (threadIdx.x < F2_T) {
    const int t = threadIdx.x;
    const int e = E0 + t, f = F0 + t;
    sEe[t] = e < z.nV ? eps[ve + e] : 0.0;
    sEf[t] = f < z.nV ? eps[ve + f] : 0.0;
    sEeF[t] = (float)sEe[t];
    sEfF[t] = (float)sEf[t];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const double* al = alpha + (size_t)(m * z.nA + u) * nVpad;
      sBAe[u][t] = pinfo[4 * (m * z.nA + u) + 1] * al[E0 + t];
      sAf[u][t] = al[F0 + t];
    }
  }
  if (threadIdx.x < NA * NA) {
    const double g = G[threadIdx.x];
    sG[threadIdx.x] = g;
    sGh[threadIdx.x] = (float)g;
    sGl[threadIdx.x] = (float)(g - (double)(float)g);
  }
  if (threadIdx.x == 0) {
    int fact = 1;
    for (int u = 0; u < NA; ++u) {
      sE[u] = pinfo[4 * (m * z.nA + u)];
      sEF[u] = (float)sE[u];
      fact = fact && (pinfo[4 * (m * z.nA + u) + 2] != 0.0);
    }
    sFact = fact;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // every D_u of the tile pair so far from 0 that exp(-s D_u^2) < 2^-63:
    // then Rv = 1 and Rt = 1/D_u to FP64 precision
    double elo = 1e300, flo = 1e300, ehi = -1e300, fhi = -1e300;
    for (int t = 0; t < F2_T; ++t) {
      if (E0 + t < z.nV) elo = fmin(elo, sEe[t]), ehi = fmax(ehi, sEe[t]);
      if (F0 + t < z.nV) flo = fmin(flo, sEf[t]), fhi = fmax(fhi, sEf[t]);
    }
    int far = 1;
    for (int u = 0; u < NA; ++u) {
      const double dhi = sE[u] - elo - flo, dlo = sE[u] - ehi - fhi;
      const double dn = dhi <= 0.0 ? dhi : (dlo >= 0.0 ? dlo : 0.0);
      far = far && (dhi <= -0.25 || dlo >= 0.25) && s * dn * dn > 44.0;
    }
    sFar = far;
  }
  __syncthreads();
  const bool mirror = ab.x < ab.y;
  const bool fact = sFact != 0;
  const bool tile_far = sFar != 0;
  const int c = threadIdx.x & 31;
  const int f = F0 + c;
  double acc = 0.0;
  unsigned long long near = 0;  // positions of this thread on the expm1 path
  if (threadIdx.x == 0 && !fact) atomicAdd(&counts[DSRG_COUNT_CAVV_UNFACTORABLE], 1ull);
  if (f < z.nV) {
    for (int r = threadIdx.x >> 5; r < F2_T; r += 8) {
      const int e = E0 + r;
      if (e >= z.nV) break;
      const double tau = (fact && !tile_far) ? tau1[(size_t)e * nVpad + f] : 0.0;
      const double eef = sEe[r] + sEf[c];
      const float eeff = sEeF[r] + sEfF[c];
      float X[NA], Xt[NA];
      bool far = fact;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        X[u] = sX[(u * F2_T + r) * (F2_T + 1) + c];
        Xt[u] = sXt[(u * F2_T + r) * (F2_T + 1) + c];
        // D_u in FP32 (a few ulp): the path test, whose threshold is not sharp
        // (both paths are accurate near it), and below the reciprocal seed
        far = far && fabsf(sEF[u] - eeff) >= 0.25f;
      }
      if (far || tile_far) {
        // every D_u away from 0 (|D_u| >= 1/4): Rt_u = (1 - g_u) / D_u in FP64
        // (g_u = exp(-s D_u^2) from the factor tables, or 0 where it is below FP64
        // precision; 1/D_u an FP32 seed and one FP64 Newton step). The exchange
        // combination Q_uv = X_u (2 X_v - Xt_v) [+ mirror], the smooth factor
        // Rv_u = 1 + g_u in [1, 2) and the u sums with G_uv run in FP32 with
        // round-to-nearest (unbiased; G as head + remainder, so its own rounding
        // is not a systematic error); each v sum meets Rt_v in FP64. The
        // remainder sums take Rt in FP32 (they are 2^-24 of the head sums).
        double Rt[NA];
        float a[NA], at[NA], rtf[NA];
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          const double D = sE[u] - eef;
          const double g = tile_far ? 0.0 : sBAe[u][r] * sAf[u][c] * tau;
          float r0f;
          asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0f) : "f"(sEF[u] - eeff));
          const double r0 = (double)r0f;
          const double en = fma(-D, r0, 1.0);
          const double R0 = fma(-g, r0, r0);
          Rt[u] = fma(R0, en, R0);
          const float gf = (float)g;
          const float w = 1.0f + gf;
          a[u] = w * X[u];
          at[u] = w * Xt[u];
          rtf[u] = (1.0f - gf) * r0f;
        }
        // sum_u G_uv Rv_u Q_uv = (2 X_v - Xt_v) sum_u G_uv Rv_u X_u
        //                       [+ (2 Xt_v - X_v) sum_u G_uv Rv_u Xt_u for the mirror]
        double t = 0.0;
        float tl = 0.0f;
#pragma unroll
        for (int v = 0; v < NA; ++v) {
          float zh = 0.0f, zl = 0.0f, zth = 0.0f, ztl = 0.0f;
#pragma unroll
          for (int u = 0; u < NA; ++u) {
            // volatile: reloaded per position instead of held in 2 NA^2 registers
            const float gh = ((volatile float*)sGh)[u * NA + v];
            const float gl = ((volatile float*)sGl)[u * NA + v];
            zh = fmaf(gh, a[u], zh);
            zl = fmaf(gl, a[u], zl);
            if (mirror) {
              zth = fmaf(gh, at[u], zth);
              ztl = fmaf(gl, at[u], ztl);
            }
          }
          const float dv = 2.0f * X[v] - Xt[v], dtv = 2.0f * Xt[v] - X[v];
          const float ch = mirror ? fmaf(dv, zh, dtv * zth) : dv * zh;
          const float cl = mirror ? fmaf(dv, zl, dtv * ztl) : dv * zl;
          t = fma((double)ch, Rt[v], t);
          tl = fmaf(cl, rtf[v], tl);
        }
        acc += t + (double)tl;
      } else {
        // a D_u near 0 (or a pair whose factors could overflow): expm1 regulators
        // and the exchange combination in FP64
        ++near;
        double Rv[NA], Rt[NA];
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          const double D = sE[u] - eef;
          Rt[u] = reg_t(D, s);
          Rv[u] = reg_v(D, s);
        }
        double t1 = 0.0, t2 = 0.0;
#pragma unroll
        for (int v = 0; v < NA; ++v) {
          double c1 = 0.0, c2 = 0.0;
#pragma unroll
          for (int u = 0; u < NA; ++u) {
            const double w = sG[u * NA + v] * Rv[u];
            c1 = fma(w, (double)X[u], c1);
            c2 = fma(w, (double)Xt[u], c2);
          }
          t1 = fma(c1, (2.0 * (double)X[v] - (double)Xt[v]) * Rt[v], t1);
          t2 = fma(c2, (2.0 * (double)Xt[v] - (double)X[v]) * Rt[v], t2);
        }
        acc += mirror ? (t1 + t2) : t1;
      }
    }
  }
  if (near) atomicAdd(&counts[DSRG_COUNT_CAVV_NEAR], near);
  const double tot = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[blockIdx.x] = tot;
}

// ---------------------------------------------------------------------------
// Adjoint of F2 for the gradient of split plans: X_u from the GEMM output Y of
// the energy call just made (its error, about 1e-8 relative, is far below the
// gradient's), regulators from the same factor tables. Per position (e, f)
// (and its mirror (f, e) for E < F), with P_v = 2 X_v[e,f] - X_v[f,e]:
//   dE/dX_u[e,f] = Rv_u s1_u + Rt_u s2_u,
//   s1_u = sum_v G_uv Rt_v P_v,  s2_u = sum_v G_vu Rv_v P_v,
// and the derivative of the summand with respect to D_u,
//   X_u Rv_u' s1_u + (sum_w G_wu Rv_w X_w) P_u Rt_u',
// goes to e_m and e_u (+) and to e_e, e_f (-); the s derivative likewise.
// ---------------------------------------------------------------------------
template <int NA>
__global__ void __launch_bounds__(256) cavv_adj_tc_kernel(
    const float* __restrict__ Y, long long ldy, int nVpad, const double* __restrict__ eps,
    const double* __restrict__ G, double s, Sizes z, const int2* __restrict__ tps, int n_tp,
    const double* __restrict__ alpha, const double* __restrict__ pinfo,
    const double* __restrict__ tau1, double* __restrict__ dX, double* __restrict__ deps,
    double* __restrict__ ds) {
  extern __shared__ float f2s[];
  float* sX = f2s;                              // [NA][32][33]   X_u[e,f]
  float* sXt = sX + NA * F2_T * (F2_T + 1);     // [NA][32][33]   X_u[f,e]
  __shared__ double sBAe[NA][F2_T], sAf[NA][F2_T], sEe[F2_T], sEf[F2_T], sG[NA * NA];
  __shared__ double sE[NA];
  __shared__ int sFact, sFar;
  __shared__ double rowacc[F2_T], colacc[F2_T], uacc[NA];
  __shared__ double red[8];
  const int m = blockIdx.x / n_tp;
  const int2 ab = tps[blockIdx.x % n_tp];
  const int E0 = ab.x * F2_T, F0 = ab.y * F2_T;
  const int ve = z.nC + z.nA;
  const float* Ym = Y + (size_t)m * nVpad * ldy;
  for (int k = threadIdx.x; k < NA * F2_T * F2_T; k += 256) {
    const int u = k / (F2_T * F2_T), r = (k / F2_T) % F2_T, c = k % F2_T;
    sX[(u * F2_T + r) * (F2_T + 1) + c] = Ym[(size_t)(E0 + r) * ldy + u * nVpad + F0 + c];
    sXt[(u * F2_T + c) * (F2_T + 1) + r] = Ym[(size_t)(F0 + r) * ldy + u * nVpad + E0 + c];
  }
  if (threadIdx.x < F2_T) {
    const int t = threadIdx.x;
    const int e = E0 + t, f = F0 + t;
    sEe[t] = e < z.nV ? eps[ve + e] : 0.0;
    sEf[t] = f < z.nV ? eps[ve + f] : 0.0;
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const double* al = alpha + (size_t)(m * z.nA + u) * nVpad;
      sBAe[u][t] = pinfo[4 * (m * z.nA + u) + 1] * al[E0 + t];
      sAf[u][t] = al[F0 + t];
    }
    rowacc[t] = 0.0;
    colacc[t] = 0.0;
  }
  if (threadIdx.x < NA * NA) sG[threadIdx.x] = G[threadIdx.x];
  if (threadIdx.x < NA) uacc[threadIdx.x] = 0.0;
  if (threadIdx.x == 0) {
    int fact = 1;
    for (int u = 0; u < NA; ++u) {
      sE[u] = pinfo[4 * (m * z.nA + u)];
      fact = fact && (pinfo[4 * (m * z.nA + u) + 2] != 0.0);
    }
    sFact = fact;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // every D_u of the tile pair so far from 0 that exp(-s D_u^2) < 2^-63
    double elo = 1e300, flo = 1e300, ehi = -1e300, fhi = -1e300;
    for (int t = 0; t < F2_T; ++t) {
      if (E0 + t < z.nV) elo = fmin(elo, sEe[t]), ehi = fmax(ehi, sEe[t]);
      if (F0 + t < z.nV) flo = fmin(flo, sEf[t]), fhi = fmax(fhi, sEf[t]);
    }
    int far = 1;
    for (int u = 0; u < NA; ++u) {
      const double dhi = sE[u] - elo - flo, dlo = sE[u] - ehi - fhi;
      const double dn = dhi <= 0.0 ? dhi : (dlo >= 0.0 ? dlo : 0.0);
      far = far && (dhi <= -0.25 || dlo >= 0.25) && s * dn * dn > 44.0;
    }
    sFar = far;
  }
  __syncthreads();
  const bool mirror = ab.x < ab.y;
  const bool fact = sFact != 0;
  const bool tile_far = sFar != 0;
  const int c = threadIdx.x & 31;
  const int f = F0 + c;
  double dm = 0.0, dss = 0.0, cacc = 0.0;
  double du[NA];
#pragma unroll
  for (int u = 0; u < NA; ++u) du[u] = 0.0;
  if (f < z.nV) {
    for (int r = threadIdx.x >> 5; r < F2_T; r += 8) {
      const int e = E0 + r;
      if (e >= z.nV) break;
      const double tau = (fact && !tile_far) ? tau1[(size_t)e * nVpad + f] : 0.0;
      const double eef = sEe[r] + sEf[c];
      RegD Rv[NA], Rt[NA];
      double X[NA], Xt[NA], Dd[NA];
      bool far = fact;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        X[u] = sX[(u * F2_T + r) * (F2_T + 1) + c];
        Xt[u] = sXt[(u * F2_T + r) * (F2_T + 1) + c];
        Dd[u] = sE[u] - eef;
        far = far && fabs(Dd[u]) >= 0.25;
      }
      if (far || tile_far) {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          const double D = Dd[u];
          const double g = tile_far ? 0.0 : sBAe[u][r] * sAf[u][c] * tau;
          float r0f;
          asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0f) : "f"((float)D));
          const double r0 = (double)r0f;
          const double en = fma(-D, r0, 1.0);
          const double inv = fma(r0, en, r0);
          const double R0 = fma(-g, r0, r0);
          const double x = s * D * D;
          Rt[u].v = fma(R0, en, R0);                        // (1 - g) / D
          Rt[u].dD = fma(2.0 * x, g, g - 1.0) * inv * inv;  // (2 x g + e^{-x} - 1) / D^2
          Rt[u].ds = D * g;
          Rv[u].v = 1.0 + g;
          Rv[u].dD = -2.0 * s * D * g;
          Rv[u].ds = -D * D * g;
        }
      } else {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          Rt[u] = rt_d(Dd[u], s);
          Rv[u] = rv_d(Dd[u], s);
        }
      }
      double P[NA], Pt[NA];
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        P[u] = 2.0 * X[u] - Xt[u];
        Pt[u] = 2.0 * Xt[u] - X[u];
      }
      double gsum = 0.0;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        double s1 = 0.0, s2 = 0.0, s1t = 0.0, s2t = 0.0, cw = 0.0, cwt = 0.0;
#pragma unroll
        for (int v = 0; v < NA; ++v) {
          const double gt = sG[u * NA + v] * Rt[v].v, gv = sG[v * NA + u] * Rv[v].v;
          s1 = fma(gt, P[v], s1);
          s2 = fma(gv, P[v], s2);
          s1t = fma(gt, Pt[v], s1t);
          s2t = fma(gv, Pt[v], s2t);
          cw = fma(gv, X[v], cw);
          cwt = fma(gv, Xt[v], cwt);
        }
        dX[(((size_t)m * NA + u) * z.nV + e) * z.nV + f] = Rv[u].v * s1 + Rt[u].v * s2;
        if (mirror) dX[(((size_t)m * NA + u) * z.nV + f) * z.nV + e] = Rv[u].v * s1t + Rt[u].v * s2t;
        double gD = X[u] * Rv[u].dD * s1 + cw * P[u] * Rt[u].dD;
        double gs = X[u] * Rv[u].ds * s1 + cw * P[u] * Rt[u].ds;
        if (mirror) {
          gD += Xt[u] * Rv[u].dD * s1t + cwt * Pt[u] * Rt[u].dD;
          gs += Xt[u] * Rv[u].ds * s1t + cwt * Pt[u] * Rt[u].ds;
        }
        du[u] += gD;
        gsum += gD;
        dss += gs;
      }
      dm += gsum;
      atomicAdd(&rowacc[r], -gsum);
      cacc -= gsum;
    }
  }
  atomicAdd(&colacc[c], cacc);
  const double tm = block_sum<256>(dm, red);
  const double ts = block_sum<256>(dss, red);
#pragma unroll
  for (int u = 0; u < NA; ++u) {
    const double t = block_sum<256>(du[u], red);
    if (threadIdx.x == 0) uacc[u] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    atomicAdd(&deps[m], tm);
    atomicAdd(ds, ts);
    for (int u = 0; u < NA; ++u) atomicAdd(&deps[z.nC + u], uacc[u]);
  }
  if (threadIdx.x < F2_T) {
    const int e = E0 + threadIdx.x, ff = F0 + threadIdx.x;
    if (e < z.nV) atomicAdd(&deps[ve + e], rowacc[threadIdx.x]);
    if (ff < z.nV) atomicAdd(&deps[ve + ff], colacc[threadIdx.x]);
  }
}

// ---------------------------------------------------------------------------
// F3 (CCAV), spin-adapted:
//   F3 = sum_{u,v} Hh_uv sum_{m,n,e} Z_v[m,n,e] (2 Z_u[m,n,e] - Z_u[n,m,e])
//        (1 + exp(-s D_v^2)) (1 - exp(-s D_u^2))/D_u,
//   Z_u[m,n,e] = (me|nu) = Y[(m,e), XC + n*nA + u], D_u = e_m + e_n - e_e - e_u,
//   Hh = 2 I - G. One CTA per virtual e.
// ---------------------------------------------------------------------------
template <int NA>
__global__ void __launch_bounds__(256) ccav_f3_kernel(const float* __restrict__ Y, long long ldy,
                                                      int nVpad, long long xc,
                                                      const double* __restrict__ eps,
                                                      const double* __restrict__ G, double s, Sizes z,
                                                      double* __restrict__ partials) {
  extern __shared__ float f3s[];  // [nC][nC*NA]: Z_u[m,n,e] at m*(nC*NA) + n*NA + u
  __shared__ double sH[NA * NA];
  __shared__ double red[8];
  const int e = blockIdx.x, nC = z.nC, w = nC * NA;
  for (int k = threadIdx.x; k < nC * w; k += 256) {
    const int m = k / w, r = k % w;
    f3s[k] = Y[(size_t)(m * nVpad + e) * ldy + xc + r];
  }
  if (threadIdx.x < NA * NA) {
    const int u = threadIdx.x / NA, v = threadIdx.x % NA;
    sH[threadIdx.x] = (u == v ? 2.0 : 0.0) - G[threadIdx.x];
  }
  __syncthreads();
  const double ee = eps[nC + z.nA + e];
  double acc = 0.0;
  for (int mn = threadIdx.x; mn < nC * nC; mn += 256) {
    const int m = mn / nC, n = mn % nC;
    const double base = eps[m] + eps[n] - ee;
    double Rv[NA], Rt[NA], Zmn[NA], Znm[NA];
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const double D = base - eps[nC + u];
      // one exponential for both regulators: for s D^2 > 1/2, 1 - exp(-s D^2) > 0.39
      // has no cancellation; below, expm1
      const double x = s * D * D;
      const double g = exp(-x);
      const double em = x > 0.5 ? g - 1.0 : expm1(-x);
      Rv[u] = 1.0 + g;
      Rt[u] = D == 0.0 ? 0.0 : -em / D;
      Zmn[u] = (double)f3s[m * w + n * NA + u];
      Znm[u] = (double)f3s[n * w + m * NA + u];
    }
#pragma unroll
    for (int v = 0; v < NA; ++v) Rv[v] *= Zmn[v];  // Rv_v Z_v[m,n,e]
#pragma unroll
    for (int u = 0; u < NA; ++u) {
      const double zu = 2.0 * Zmn[u] - Znm[u];
      double cc = 0.0;
#pragma unroll
      for (int v = 0; v < NA; ++v) cc = fma(sH[u * NA + v], Rv[v], cc);
      acc = fma(cc, zu * Rt[u], acc);
    }
  }
  const double tot = block_sum<256>(acc, red);
  if (threadIdx.x == 0) partials[e] = tot;
}

// ---------------------------------------------------------------------------
// Active-block integrals from Y (virtual indices) and Gxx (active particles):
//   K1[i][u][x][a] = (ia|ux), K2[i][u][x][a] = (ix|ua)   [nH][nA][nA][nP]
//   K3[i][x][j][y] = (ix|jy)                              [nH][nA][nH][nA]
//   M[x][u][e][f]  = (xe|uf)                              [nA][nA][nV][nV]
// ---------------------------------------------------------------------------
__global__ void act_gather_kernel(const float* __restrict__ Y, long long ldy, int nVpad,
                                  long long xc, const double* __restrict__ Gxx, Sizes z,
                                  double* __restrict__ K1, double* __restrict__ K2,
                                  double* __restrict__ K3, double* __restrict__ M) {
  const int nA = z.nA, nC = z.nC, T = z.nH * nA;
  const size_t n12 = (size_t)z.nH * nA * nA * z.nP;
  const size_t n3 = (size_t)T * T;
  const size_t nm = (size_t)nA * nA * z.nV * z.nV;
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k < 2 * n12) {
    const bool second = k >= n12;
    const size_t r = second ? k - n12 : k;
    const int a = (int)(r % z.nP);
    const int x = (int)((r / z.nP) % nA);
    const int u = (int)((r / ((size_t)z.nP * nA)) % nA);
    const int i = (int)(r / ((size_t)z.nP * nA * nA));
    double v;
    if (!second) {  // (ia|ux)
      v = (a < nA) ? Gxx[(size_t)(i * nA + a) * T + (nC + u) * nA + x]
                   : (double)Y[(size_t)(i * nVpad + a - nA) * ldy + xc + (nC + u) * nA + x];
      K1[r] = v;
    } else {        // (ix|ua)
      v = (a < nA) ? Gxx[(size_t)(i * nA + x) * T + (nC + u) * nA + a]
                   : (double)Y[(size_t)((nC + u) * nVpad + a - nA) * ldy + xc + i * nA + x];
      K2[r] = v;
    }
  } else if (k < 2 * n12 + n3) {
    const size_t r = k - 2 * n12;  // [i][x][j][y] = Gxx[(i,x)][(j,y)]
    K3[r] = Gxx[r];
  } else if (k < 2 * n12 + n3 + nm) {
    const size_t r = k - 2 * n12 - n3;
    const int f = (int)(r % z.nV);
    const int e = (int)((r / z.nV) % z.nV);
    const int u = (int)((r / ((size_t)z.nV * z.nV)) % nA);
    const int x = (int)(r / ((size_t)z.nV * z.nV * nA));
    M[r] = (double)Y[(size_t)((nC + x) * nVpad + e) * ldy + (size_t)u * nVpad + f];
  }
}

// ------------------------------- host side -------------------------------
struct RestState {
  int nVpad = 0, XR = 0, ncols = 0, n_tiles = 0, m_tiles = 0, grid = 0;
  long long ldy = 0, xc = 0;
  float* Y = nullptr;
  double* Xq = nullptr;
  double* Gxx = nullptr;
  double* alpha = nullptr;
  double* pinfo = nullptr;
  double* tau1 = nullptr;
  double* vmax = nullptr;  // max |e_v| over the virtual orbitals
  int2* d_tp = nullptr;
  int n_tp = 0;
  // tau1 was written by the pair tables of the CCVV kernel (split_stage_tables)
  // queued before this call's CAVV tables: those skip it
  bool tau1_staged = false;
};

int rest_xrows(const Sizes& z) {
  if (z.nA == 0) return 0;
  return (z.nH * z.nA + XROW_ALIGN - 1) / XROW_ALIGN * XROW_ALIGN;
}

static void rest_dims(const Sizes& z, RestState* st) {
  st->nVpad = (z.nV + G_BM - 1) / G_BM * G_BM;
  st->XR = rest_xrows(z);
  st->ncols = z.nA * st->nVpad + st->XR;
  st->n_tiles = (st->ncols + G_BN - 1) / G_BN;
  st->m_tiles = z.nH * st->nVpad / G_BM;
  st->ldy = (long long)st->n_tiles * G_BN;
  st->xc = (long long)z.nA * st->nVpad;
  const int nt = (z.nV + F2_T - 1) / F2_T;
  st->n_tp = nt * (nt + 1) / 2;
}

size_t rest_y_bytes(const Sizes& z) {
  if (z.nA == 0) return 0;
  RestState st;
  rest_dims(z, &st);
  return (size_t)z.nH * st.nVpad * st.ldy * sizeof(float);
}

bool rest_split_used(const dsrg_plan* p) { return p->prec != DSRG_PREC_FP64 && p->z.nA > 0; }

int rest_cavv_blocks(const dsrg_plan* p) {
  RestState st;
  rest_dims(p->z, &st);
  return p->z.nC * st.n_tp;
}

int rest_ccav_blocks(const dsrg_plan* p) { return p->z.nV; }

static size_t gemm_smem_bytes() { return (size_t)G_STAGES * G_STAGE_BYTES + 1024 + 256; }
static size_t f2_smem_bytes(int na) { return (size_t)2 * na * F2_T * (F2_T + 1) * sizeof(float); }
static size_t f3_smem_bytes(const Sizes& z) { return (size_t)z.nC * z.nC * z.nA * sizeof(float); }

bool rest_supported(const Sizes& z) {
  return z.nA <= NA_MAX && f3_smem_bytes(z) <= 200 * 1024;
}

bool rest_alloc(dsrg_plan* p, float* shared_y) {
  const Sizes& z = p->z;
  RestState* st = new RestState();
  p->rest = st;
  rest_dims(z, st);
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  const int items = st->m_tiles * st->n_tiles;
  st->grid = items < nsm ? items : nsm;
  const int T = z.nH * z.nA;
  bool ok = true;
  if (shared_y)
    st->Y = shared_y;
  else
    ok = plan_alloc(p, (void**)&st->Y, rest_y_bytes(z));
  ok = ok && plan_alloc(p, (void**)&st->Xq, (size_t)T * z.Q * 8) &&
       plan_alloc(p, (void**)&st->Gxx, (size_t)T * T * 8) &&
       plan_alloc(p, (void**)&st->alpha, (size_t)z.nH * z.nA * st->nVpad * 8) &&
       plan_alloc(p, (void**)&st->pinfo, (size_t)z.nH * z.nA * 4 * 8) &&
       plan_alloc(p, (void**)&st->tau1, (size_t)st->nVpad * st->nVpad * 8) &&
       plan_alloc(p, (void**)&st->vmax, 8) &&
       plan_alloc(p, (void**)&st->d_tp, (size_t)st->n_tp * sizeof(int2));
  if (!ok) return false;
  const int nt = (z.nV + F2_T - 1) / F2_T;
  std::vector<int2> tp;
  for (int A = 0; A < nt; ++A)
    for (int B = A; B < nt; ++B) tp.push_back(make_int2(A, B));
  return cudaMemcpy(st->d_tp, tp.data(), tp.size() * sizeof(int2), cudaMemcpyHostToDevice) ==
         cudaSuccess;
}

// tau1 for the CCVV pair tables to fill (exp(-s t^2), whose square is their
// own exp(-2 s t^2)); the next CAVV tables of this plan then skip it.
double* rest_take_tau1(dsrg_plan* p) {
  RestState* st = p->rest;
  if (!st) return nullptr;
  st->tau1_staged = true;
  return st->tau1;
}

void rest_act_tables(const dsrg_plan* p, const double** alpha, const double** pinfo,
                     const double** tau, int* ld) {
  const RestState* st = p->rest;
  if (!st) return;
  const size_t off = (size_t)p->z.nC * p->z.nA;  // the (x, u) pairs follow the (m, u) pairs
  *alpha = st->alpha + off * st->nVpad;
  *pinfo = st->pinfo + off * 4;
  *tau = st->tau1;
  *ld = st->nVpad;
}

void rest_free(dsrg_plan* p) {
  delete p->rest;
  p->rest = nullptr;
}

// CAVV and CCAV partials and the active-block integrals K1, K2, K3, M of this
// call (requires the planes staged by the CCVV launch of the same call).
cudaError_t launch_split_rest(dsrg_plan* p, const double* B, const double* eps, const double* G,
                              double s) {
  RestState* st = p->rest;
  const Sizes& z = p->z;
  const bool bf16 = p->prec == DSRG_PREC_BF16X3;
  cudaStream_t stream = p->stream;
  const int T = z.nH * z.nA;
  const long long xrow0 = (long long)z.nH * st->nVpad;
  {
    const size_t n = (size_t)T * z.Q;
    void* hi = split_plane_ptr(p, true);
    void* lo = split_plane_ptr(p, false);
    float* tail = (float*)split_tail_ptr(p);
    const int Qld = split_qld(p);
    if (bf16)
      xrows_kernel<true><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(B, z, xrow0, Qld, hi, lo,
                                                                         st->Xq, tail);
    else
      xrows_kernel<false><<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(B, z, xrow0, Qld, hi, lo,
                                                                          st->Xq, tail);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    TcGemmArgs a;
    a.a_row0 = 0;
    a.b_row0 = z.nC * st->nVpad;
    a.m_tiles = st->m_tiles;
    a.n_tiles = st->n_tiles;
    a.kq0 = TAIL_Q;
    a.kblocks = (split_qpad(p) - TAIL_Q) / (G_KB / (bf16 ? 2 : 4));
    a.tail = split_tail_ptr(p);
    a.Y = st->Y;
    a.ldy = st->ldy;
    a.status = p->d_status;
    const size_t sm = gemm_smem_bytes();
    const CUtensorMap* mh = split_map(p, true);
    const CUtensorMap* ml = split_map(p, false);
    if (bf16) {
      raise_smem_limit((const void*)split_gemm_kernel<true>, sm);
      split_gemm_kernel<true><<<st->grid, G_THREADS, sm, stream>>>(*mh, *ml, a);
    } else {
      raise_smem_limit((const void*)split_gemm_kernel<false>, sm);
      split_gemm_kernel<false><<<st->grid, G_THREADS, sm, stream>>>(*mh, *ml, a);
    }
    DSRG_LAUNCH_CHECK(p);
  }
  {
    // the pair-independent table tau1 comes with the CCVV pair tables when they were
    // staged for this call
    const size_t n = (size_t)z.nH * z.nA * st->nVpad +
                     (st->tau1_staged ? 0 : (size_t)st->nVpad * st->nVpad);
    st->tau1_staged = false;
    abs_max_kernel<<<1, 256, 0, stream>>>(eps + z.nC + z.nA, z.nV, st->vmax);
    DSRG_LAUNCH_CHECK(p);
    cavv_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
        eps, s, z, st->nVpad, st->alpha, st->pinfo, st->tau1, st->vmax);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    const Segment& sg = p->segs[p->seg_cavv];
    const size_t sm = f2_smem_bytes(z.nA);
#define F2_LAUNCH(NA_)                                                                             \
  case NA_:                                                                                        \
    raise_smem_limit((const void*)cavv_f2_kernel<NA_>, sm); \
    cavv_f2_kernel<NA_><<<sg.count, 256, sm, stream>>>(st->Y, st->ldy, st->nVpad, eps, G, s, z,       \
                                                      st->d_tp, st->n_tp, st->alpha, st->pinfo,   \
                                                      st->tau1, p->d_partials + sg.begin,         \
                                                      p->d_counts);                               \
    break;
    switch (z.nA) {
      F2_LAUNCH(1) F2_LAUNCH(2) F2_LAUNCH(3) F2_LAUNCH(4)
      F2_LAUNCH(5) F2_LAUNCH(6) F2_LAUNCH(7) F2_LAUNCH(8)
      default: return cudaErrorInvalidValue;
    }
#undef F2_LAUNCH
    DSRG_LAUNCH_CHECK(p);
  }
  {
    const Segment& sg = p->segs[p->seg_ccav];
    const size_t sm = f3_smem_bytes(z);
#define F3_LAUNCH(NA_)                                                                             \
  case NA_:                                                                                        \
    raise_smem_limit((const void*)ccav_f3_kernel<NA_>, sm); \
    ccav_f3_kernel<NA_><<<sg.count, 256, sm, stream>>>(st->Y, st->ldy, st->nVpad, st->xc, eps, G, s, \
                                                      z, p->d_partials + sg.begin);              \
    break;
    switch (z.nA) {
      F3_LAUNCH(1) F3_LAUNCH(2) F3_LAUNCH(3) F3_LAUNCH(4)
      F3_LAUNCH(5) F3_LAUNCH(6) F3_LAUNCH(7) F3_LAUNCH(8)
      default: return cudaErrorInvalidValue;
    }
#undef F3_LAUNCH
    DSRG_LAUNCH_CHECK(p);
  }
  {
    const int npair = T * (T + 1) / 2;
    xx_gram_kernel<<<(npair + 7) / 8, 256, 0, stream>>>(st->Xq, T, z.Q, st->Gxx);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    const size_t n = 2 * (size_t)z.nH * z.nA * z.nA * z.nP + (size_t)T * T +
                     (size_t)z.nA * z.nA * z.nV * z.nV;
    act_gather_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(
        st->Y, st->ldy, st->nVpad, st->xc, st->Gxx, z, p->act.K1, p->act.K2, p->act.K3, p->act.M);
    DSRG_LAUNCH_CHECK(p);
  }
  return cudaSuccess;
}

// Adjoint of F2 for split plans (the gradient), after the energy call on the
// same stream: writes dX [nC][nA][nV][nV] and adds to deps, ds.
cudaError_t launch_split_cavv_adjoint(dsrg_plan* p, const double* eps, const double* G, double s,
                                      double* dX, double* deps, double* ds) {
  RestState* st = p->rest;
  const Sizes& z = p->z;
  const size_t sm = f2_smem_bytes(z.nA);
  const unsigned grid = (unsigned)(z.nC * st->n_tp);
  if (grid == 0) return cudaSuccess;
#define F2A_LAUNCH(NA_)                                                                     \
  case NA_:                                                                                 \
    raise_smem_limit((const void*)cavv_adj_tc_kernel<NA_>, sm);                             \
    cavv_adj_tc_kernel<NA_><<<grid, 256, sm, p->stream>>>(st->Y, st->ldy, st->nVpad, eps, G, s, z, \
                                                        st->d_tp, st->n_tp, st->alpha,      \
                                                        st->pinfo, st->tau1, dX, deps, ds); \
    break;
  switch (z.nA) {
    F2A_LAUNCH(1) F2A_LAUNCH(2) F2A_LAUNCH(3) F2A_LAUNCH(4)
    F2A_LAUNCH(5) F2A_LAUNCH(6) F2A_LAUNCH(7) F2A_LAUNCH(8)
    default: return cudaErrorInvalidValue;
  }
#undef F2A_LAUNCH
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

}  // namespace dsrg
