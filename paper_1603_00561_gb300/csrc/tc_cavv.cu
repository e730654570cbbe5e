// Split-precision CAVV (diagram F2 of Table 2) and the (A,A|V,V) integrals of
// the active block on the tensor cores, from the same hi/lo planes as CCVV.
//
// Spin-adapted F2 (closed-shell spin sum of Table 2's F2):
//   F2 = sum_m sum_{u,v} G_uv sum_ef X_u[e,f] (2 X_v[e,f] - X_v[f,e]) Rv_u Rt_v,
//   X_u[e,f] = (me|uf), D_u = e_m + e_u - e_e - e_f,
//   Rv_u = 1 + exp(-s D_u^2) (Eq. (15)), Rt_v = (1 - exp(-s D_v^2)) / D_v (Eq. (13)).
// Work item = (hole row g, virtual tile pair A <= B), 128 x 128. For every
// active u the CTA accumulates X_u[A,B] = P_g[A] P_u[B]^T and its mirror
// Xt_u[A,B] = X_u[B,A]^T = P_u[A] P_g[B]^T in TMEM (2 nA accumulators of 128
// columns, nA <= 2). For a core row g the FP64 epilogue adds the F2
// contribution of the positions (a,b) and, for A < B, of their mirrors (b,a).
// For an active row g = x it stores M_xu[a,b] = (xa|ub) (Sec. III step 4:
// integrals with active indices are formed explicitly) for the active block.
//
// exp(-s D_u^2) = exp(-s E^2) exp(2 s E e_a) exp(2 s E e_b) exp(-s (e_a + e_b)^2)
// with E = e_m + e_u: per-(m,u) tables, one pair-independent table; 1/D_u is an
// FP32 seed with one FP64 Newton step; |D_u| < 1/4 takes expm1 and an FP64 divide.
#include <cuda.h>
#include <cudaTypedefs.h>

#include "internal.cuh"
#include "regulators.cuh"
#include "tc_common.cuh"

namespace dsrg {

constexpr int CT = 128;
constexpr int C_KB = 64;                  // K bytes per row per stage
constexpr int C_SLOT = CT * C_KB;         // 8 KB
constexpr int C_STAGES = 2;
constexpr int C_MAXSLOTS = 6;             // (g,A) (g,B) (u,A) (u,B) for u < 2
constexpr int C_STAGE_BYTES = C_MAXSLOTS * 2 * C_SLOT;  // 96 KB
constexpr int C_THREADS = 192;

struct CavvArgs {
  const double* eps;
  const double* G;
  double s;
  Sizes z;
  int nVpad, kblocks, n_tp, n_items;
  const int2* tps;
  const double* alpha;   // [nC*nA][nVpad] exp(2 s E_mu e_b)
  const double* pinfo;   // [nC*nA][4] E_mu, exp(-s E_mu^2), flag
  const double* tau1;    // [nVpad][nVpad] exp(-s (e_a + e_b)^2)
  double* partials;      // [nC * n_tp]
  double* M;             // [nA][nA][nV][nV]
  int* status;
};

template <bool BF16, int NA>
__global__ void __launch_bounds__(C_THREADS, 1)
    cavv_split_kernel(const __grid_constant__ CUtensorMap map_hi,
                      const __grid_constant__ CUtensorMap map_lo, const CavvArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* tiles = smem;
  uint64_t* full = (uint64_t*)(smem + C_STAGES * C_STAGE_BYTES);
  uint64_t* empty = full + C_STAGES;
  uint64_t* tfull = empty + C_STAGES;
  uint64_t* tempty = tfull + 1;
  uint64_t* drain = tempty + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  double* sEps = (double*)(smem + C_STAGES * C_STAGE_BYTES + 256);
  double* sAlpha = sEps + CT;          // [NA][CT]
  double* sRed = sAlpha + NA * CT;
  double* sG = sRed + 8;               // [NA][NA]

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Sizes& z = a.z;
  constexpr uint32_t NCOLS = 512;

  if (threadIdx.x == 0) {
    for (int s = 0; s < C_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(tfull, 1);
    mbar_init(tempty, 4);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (threadIdx.x < NA * NA) sG[threadIdx.x] = a.G[threadIdx.x];
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(NCOLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < a.n_items; item += gridDim.x) {
        const int g = item / a.n_tp;
        const int2 ab = a.tps[item % a.n_tp];
        const bool dt = ab.x == ab.y;
        const int nload = dt ? 1 + NA : 2 + 2 * NA;
        for (int kb = 0; kb < a.kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.status)) {
            ok = false;
            break;
          }
          uint8_t* st = tiles + stage * C_STAGE_BYTES;
          mbar_expect_tx(&full[stage], (uint32_t)(nload * 2 * C_SLOT));
          const int kq = kb * (C_KB / (BF16 ? 2 : 4));
          // slot 0: (g, A); slot 1: (g, B); slot 2+2u: (u, A); slot 3+2u: (u, B)
          for (int sl = 0; sl < 2 + 2 * NA; ++sl) {
            if (dt && (sl & 1)) continue;
            const int h = (sl < 2) ? g : z.nC + (sl - 2) / 2;
            const int tile = (sl & 1) ? ab.y : ab.x;
            const int row = h * a.nVpad + tile * CT;
            tma_load_2d(st + (sl * 2 + 0) * C_SLOT, &map_hi, &full[stage], kq, row);
            tma_load_2d(st + (sl * 2 + 1) * C_SLOT, &map_lo, &full[stage], kq, row);
          }
          if (++stage == C_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        int s = stage;
        uint32_t ph = phase;
        for (int k = 0; k < C_STAGES; ++k) {
          if (--s < 0) {
            s = C_STAGES - 1;
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
      constexpr uint32_t idesc = idesc_128x128<BF16>();
      int stage = 0;
      uint32_t phase = 0;
      uint32_t tphase = 0;
      bool ok = true, issued = false;
      for (int item = blockIdx.x; ok && item < a.n_items; item += gridDim.x) {
        const int2 ab = a.tps[item % a.n_tp];
        const bool dt = ab.x == ab.y;
        if (!mbar_wait(tempty, tphase ^ 1u, abort_flag, a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        for (int kb = 0; kb < a.kblocks; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = su32(tiles + stage * C_STAGE_BYTES);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint32_t off = (uint32_t)(k * 32);
            const uint32_t acc0 = (kb > 0 || k > 0) ? 1u : 0u;
            const int sgA = 0, sgB = dt ? 0 : 1;
#pragma unroll
            for (int u = 0; u < NA; ++u) {
              const int suA = 2 + 2 * u, suB = dt ? 2 + 2 * u : 3 + 2 * u;
              const uint32_t dX = tmem_base + (uint32_t)(2 * u * 128);
              const uint32_t dXt = dX + 128;
              // X_u = (g, A) . (u, B)^T
              {
                const uint64_t ah = desc_sw64(sb + (sgA * 2 + 0) * C_SLOT + off);
                const uint64_t al = desc_sw64(sb + (sgA * 2 + 1) * C_SLOT + off);
                const uint64_t bh = desc_sw64(sb + (suB * 2 + 0) * C_SLOT + off);
                const uint64_t bl = desc_sw64(sb + (suB * 2 + 1) * C_SLOT + off);
                tc_mma<BF16>(dX, ah, bh, idesc, acc0);
                tc_mma<BF16>(dX, ah, bl, idesc, 1u);
                tc_mma<BF16>(dX, al, bh, idesc, 1u);
              }
              // Xt_u = (u, A) . (g, B)^T
              {
                const uint64_t ah = desc_sw64(sb + (suA * 2 + 0) * C_SLOT + off);
                const uint64_t al = desc_sw64(sb + (suA * 2 + 1) * C_SLOT + off);
                const uint64_t bh = desc_sw64(sb + (sgB * 2 + 0) * C_SLOT + off);
                const uint64_t bl = desc_sw64(sb + (sgB * 2 + 1) * C_SLOT + off);
                tc_mma<BF16>(dXt, ah, bh, idesc, acc0);
                tc_mma<BF16>(dXt, ah, bl, idesc, 1u);
                tc_mma<BF16>(dXt, al, bh, idesc, 1u);
              }
            }
          }
          issued = true;
          tc_commit(&empty[stage]);
          if (++stage == C_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
        if (!ok) break;
        tc_commit(tfull);
        tphase ^= 1u;
      }
      if (!ok && issued) {
        tc_commit(drain);
        const unsigned long long t0 = gtimer();
        while (!mbar_try(drain, 0) && gtimer() - t0 < TC_WAIT_NS) {
        }
      }
    }
  } else {
    const int et = threadIdx.x - 64;
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int ve = z.nC + z.nA;
    uint32_t tphase = 0;
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
      const int g = item / a.n_tp;
      const int2 ab = a.tps[item % a.n_tp];
      const bool core = g < z.nC;
      const bool mirror = ab.x < ab.y;
      const int arow = ab.x * CT + row;
      const bool rok = arow < z.nV;
      const int ncols = min(CT, z.nV - ab.y * CT);
      named_bar(1, 128);
      {
        const int b = ab.y * CT + et;
        sEps[et] = (b < z.nV) ? a.eps[ve + b] : 0.0;
        if (core) {
#pragma unroll
          for (int u = 0; u < NA; ++u)
            sAlpha[u * CT + et] = (b < z.nV) ? a.alpha[(size_t)(g * z.nA + u) * a.nVpad + b] : 0.0;
        }
      }
      named_bar(1, 128);
      double cu[NA], hu[NA];
      bool fact = true;
      const double ea = rok ? a.eps[ve + arow] : 0.0;
#pragma unroll
      for (int u = 0; u < NA; ++u) {
        if (core) {
          const double* pi = a.pinfo + 4 * (g * z.nA + u);
          cu[u] = pi[0] - ea;
          hu[u] = rok ? pi[1] * a.alpha[(size_t)(g * z.nA + u) * a.nVpad + arow] : 0.0;
          fact = fact && (pi[2] != 0.0);
        } else {
          cu[u] = 0.0;
          hu[u] = 0.0;
        }
      }
      const double s = a.s;
      const bool ok = mbar_wait(tfull, tphase, abort_flag, a.status);
      tc_fence_after();
      double acc = 0.0;
      if (ok) {
        const uint32_t tb = tmem_base + ((uint32_t)(quarter * 32) << 16);
        for (int c0 = 0; c0 < ncols; c0 += 16) {
          uint32_t xr[NA][16], tr[NA][16];
#pragma unroll
          for (int u = 0; u < NA; ++u) {
            tmem_ld16(tb + (uint32_t)(2 * u * 128 + c0), xr[u]);
            tmem_ld16(tb + (uint32_t)(2 * u * 128 + 128 + c0), tr[u]);
          }
          tmem_ld_wait();
          if (!rok) continue;
          if (!core) {
            // store M_xu[a][b] (and the mirror block for A < B)
            const int x = g - z.nC;
#pragma unroll
            for (int u = 0; u < NA; ++u) {
              double* Mxu = a.M + (size_t)(x * z.nA + u) * z.nV * z.nV;
#pragma unroll
              for (int k = 0; k < 16; ++k) {
                const int b = ab.y * CT + c0 + k;
                if (c0 + k >= ncols) break;
                Mxu[(size_t)arow * z.nV + b] = (double)__uint_as_float(xr[u][k]);
                if (mirror) Mxu[(size_t)b * z.nV + arow] = (double)__uint_as_float(tr[u][k]);
              }
            }
            continue;
          }
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int cb = c0 + k;
            if (cb >= ncols) break;
            const double eb = sEps[cb];
            const double tau = fact ? a.tau1[(size_t)(ab.y * CT + cb) * a.nVpad + arow] : 0.0;
            double Rv[NA], Rt[NA], X[NA], Xt[NA];
#pragma unroll
            for (int u = 0; u < NA; ++u) {
              X[u] = (double)__uint_as_float(xr[u][k]);
              Xt[u] = (double)__uint_as_float(tr[u][k]);
              const double D = cu[u] - eb;
              if (fabs(D) >= 0.25) {
                const double gg = fact ? hu[u] * sAlpha[u * CT + cb] * tau : exp(-s * D * D);
                float r0f;
                asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0f) : "f"((float)D));
                const double r0 = (double)r0f;
                const double e = fma(-D, r0, 1.0);
                const double R0 = (1.0 - gg) * r0;
                Rt[u] = fma(R0, e, R0);
                Rv[u] = 1.0 + gg;
              } else {
                Rt[u] = reg_t(D, s);
                Rv[u] = reg_v(D, s);
              }
            }
            double t1 = 0.0, t2 = 0.0;
#pragma unroll
            for (int v = 0; v < NA; ++v) {
              double c1 = 0.0, c2 = 0.0;
#pragma unroll
              for (int u = 0; u < NA; ++u) {
                const double w = sG[u * NA + v] * Rv[u];
                c1 = fma(w, X[u], c1);
                c2 = fma(w, Xt[u], c2);
              }
              t1 = fma(c1, (2.0 * X[v] - Xt[v]) * Rt[v], t1);
              t2 = fma(c2, (2.0 * Xt[v] - X[v]) * Rt[v], t2);
            }
            acc += mirror ? (t1 + t2) : t1;
          }
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(tempty);
      tphase ^= 1u;
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sRed[warp - 2] = acc;
      named_bar(1, 128);
      if (et == 0 && core) a.partials[item] = ok ? (((sRed[0] + sRed[1]) + sRed[2]) + sRed[3]) : 0.0;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(NCOLS)
                 : "memory");
  }
}

// Factors of exp(-s D_u^2), D_u = E_mu - e_a - e_b, E_mu = e_m + e_u.
__global__ void cavv_tables_kernel(const double* __restrict__ eps, double s, Sizes z, int nVpad,
                                   double* __restrict__ alpha, double* __restrict__ pinfo,
                                   double* __restrict__ tau1) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ve = z.nC + z.nA;
  const int nmu = z.nC * z.nA;
  const size_t na = (size_t)nmu * nVpad, nt = (size_t)nVpad * nVpad;
  if (k < na) {
    const int mu = (int)(k / nVpad), b = (int)(k % nVpad);
    const int m = mu / z.nA, u = mu % z.nA;
    const double E = eps[m] + eps[z.nC + u];
    alpha[k] = (b < z.nV) ? exp(2.0 * s * E * eps[ve + b]) : 0.0;
    if (b == 0) {
      double vmax = 0.0;
      for (int v = 0; v < z.nV; ++v) vmax = fmax(vmax, fabs(eps[ve + v]));
      const bool ok = (s * E * E <= 700.0) && (2.0 * s * fabs(E) * vmax <= 700.0) &&
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

// ------------------------------- host side -------------------------------
bool cavv_split_supported(const dsrg_plan* p) { return p->z.nA >= 1 && p->z.nA <= 2; }

int cavv_split_blocks(const dsrg_plan* p) {
  const int nT = (p->z.nV + CT - 1) / CT;
  return p->z.nC * (nT * (nT + 1) / 2);
}

struct CavvState {
  double* alpha;
  double* pinfo;
  double* tau1;
  int2* d_tp;
  int n_tp, nVpad;
};

static CavvState* g_state_of(dsrg_plan* p) { return (CavvState*)p->cavv_state; }

bool cavv_split_alloc(dsrg_plan* p) {
  if (!cavv_split_supported(p)) return true;
  const Sizes& z = p->z;
  CavvState* st = new CavvState();
  p->cavv_state = st;
  const int nT = (z.nV + CT - 1) / CT;
  st->nVpad = nT * CT;
  st->n_tp = nT * (nT + 1) / 2;
  bool ok = plan_alloc(p, (void**)&st->alpha, (size_t)z.nC * z.nA * st->nVpad * 8) &&
            plan_alloc(p, (void**)&st->pinfo, (size_t)z.nC * z.nA * 4 * 8) &&
            plan_alloc(p, (void**)&st->tau1, (size_t)st->nVpad * st->nVpad * 8) &&
            plan_alloc(p, (void**)&st->d_tp, (size_t)st->n_tp * sizeof(int2));
  if (!ok) return false;
  std::vector<int2> tp;
  for (int A = 0; A < nT; ++A)
    for (int B = A; B < nT; ++B) tp.push_back(make_int2(A, B));
  return cudaMemcpy(st->d_tp, tp.data(), tp.size() * sizeof(int2), cudaMemcpyHostToDevice) ==
         cudaSuccess;
}

void cavv_split_free(dsrg_plan* p) {
  delete g_state_of(p);
  p->cavv_state = nullptr;
}

static size_t cavv_smem_bytes(int na) {
  return (size_t)C_STAGES * C_STAGE_BYTES + 1024 + 256 + (size_t)(CT + na * CT + 8 + na * na) * 8 + 64;
}

// Requires the hi/lo planes of this call (launch_split_ccvv stages them first).
cudaError_t launch_split_cavv(dsrg_plan* p, const double* eps, const double* G, double s) {
  CavvState* st = g_state_of(p);
  const Sizes& z = p->z;
  const bool bf16 = p->prec == DSRG_PREC_BF16X3;
  {
    const size_t n = (size_t)z.nC * z.nA * st->nVpad + (size_t)st->nVpad * st->nVpad;
    cavv_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(eps, s, z, st->nVpad,
                                                                         st->alpha, st->pinfo,
                                                                         st->tau1);
    DSRG_LAUNCH_CHECK(p);
  }
  CavvArgs a;
  a.eps = eps;
  a.G = G;
  a.s = s;
  a.z = z;
  a.nVpad = st->nVpad;
  a.kblocks = split_qpad(p) / (C_KB / (bf16 ? 2 : 4));
  a.n_tp = st->n_tp;
  a.n_items = (z.nC + z.nA) * st->n_tp;
  a.tps = st->d_tp;
  a.alpha = st->alpha;
  a.pinfo = st->pinfo;
  a.tau1 = st->tau1;
  a.partials = p->d_partials + p->segs[p->seg_cavv].begin;
  a.M = p->act.M;
  a.status = p->d_status;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  const int grid = a.n_items < nsm ? a.n_items : nsm;
  const size_t sm = cavv_smem_bytes(z.nA);
  const CUtensorMap* mh = split_map(p, true);
  const CUtensorMap* ml = split_map(p, false);
#define CAVV_LAUNCH(BF, NA_)                                                                   \
  do {                                                                                         \
    cudaFuncSetAttribute(cavv_split_kernel<BF, NA_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                         (int)sm);                                                             \
    cavv_split_kernel<BF, NA_><<<grid, C_THREADS, sm, p->stream>>>(*mh, *ml, a);               \
  } while (0)
  if (bf16) {
    if (z.nA == 1) CAVV_LAUNCH(true, 1); else CAVV_LAUNCH(true, 2);
  } else {
    if (z.nA == 1) CAVV_LAUNCH(false, 1); else CAVV_LAUNCH(false, 2);
  }
#undef CAVV_LAUNCH
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

}  // namespace dsrg
