// dE/dB of split-precision plans on the tensor cores.
//
// Every term of the energy depends on the factors B only through integrals
// (r|c) = sum_Q B^Q_r B^Q_c between two rows r, c of the hole x particle block
// (the CCVV pair blocks v, the CAVV and CCAV integrals X and Z, and the
// active-block integrals K1, K2, K3, M of Sec. III step 4). With the plane rows
// r = (h, e) for every hole h and virtual e, then (h, x) for every hole h and
// active particle x (the row order of the split planes), the gradient is
//     dE/dB^Q_r = sum_c S_rc B^Q_c,   S = dE/d(r|c) + dE/d(c|r)   (symmetric),
// one GEMM of S [rows x rows] with B^T [Q x rows]. The CCVV block of S (core
// rows x core rows) comes from the adjoint epilogue of the CCVV kernel; the
// rest is gathered here from the adjoints dX, dZ, dM, dK1, dK2, dK3.
//
// The GEMM runs on tcgen05 with S and B^T split into BF16 hi + lo planes
// (three products, as the energy). Its K index runs over plane rows whose
// terms do not decay, so the truncating FP32 accumulator of the tensor cores
// must not carry the whole sum: every K stage (32 values) is its own
// accumulation in TMEM every AG_CH = 2 stages (64 values, 12 MMAs), which the
// epilogue adds in FP32 round-to-nearest into registers; every AG_L1 of those
// the register sums go into a second FP32 sum in shared memory, and the two
// are added in FP64 at the end.
//
// Roles (one CTA per SM, persistent): warp 0 TMA producer, warp 1 TMEM
// allocator and MMA issuer, warps 2-9 epilogue (two warps per TMEM lane
// quarter, 64 columns each). Shared memory: 4 stages x (S tile, B^T tile) x
// (hi, lo) x 128 rows x 64 bytes, 64-byte swizzle; 64 KB of second-level sums.
// TMEM: 4 buffers x 128 columns. Every wait is bounded (about 2 s).
#include <cuda.h>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "tc_common.cuh"

namespace dsrg {

constexpr int AG_BM = 128, AG_BN = 128;
constexpr int AG_KB = 64;                     // K bytes per row per stage: 32 BF16, two MMA K steps
constexpr int AG_STAGES = 4;
constexpr int AG_TILE = AG_BM * AG_KB;        // 8 KB: one operand tile of one plane
constexpr int AG_STAGE_BYTES = 4 * AG_TILE;   // S hi, S lo, B^T hi, B^T lo
constexpr int AG_THREADS = 320;
constexpr int AG_EPI = 8;
constexpr int AG_NBUF = 4;                    // TMEM accumulators
constexpr int AG_CH = 2;                      // K stages per TMEM accumulation (12 MMAs)
constexpr int AG_L1 = 16;                     // accumulations summed in registers before the shared-memory sum
constexpr uint32_t AG_TMEM_COLS = AG_NBUF * AG_BN;
constexpr int AG_BAND = 12;                   // m tiles per band of the item order

struct TcAdjWs {
  int rows = 0;        // plane rows (the order of the split planes)
  int lds = 0;         // row pitch of S and B^T (elements; = rows, a multiple of 64)
  int Qt = 0;          // B^T rows: Q rounded up to 128
  int cv_rows = 0;     // core x virtual rows: nC * nVpad
  int nVpad = 0, xr0 = 0;
  uint16_t *s_hi = nullptr, *s_lo = nullptr;    // [rows][lds]
  uint16_t *bt_hi = nullptr, *bt_lo = nullptr;  // [Qt][lds]
  CUtensorMap map_s_hi, map_s_lo, map_bt_hi, map_bt_lo;
  int m_tiles = 0, n_tiles = 0, grid = 0;
};

struct AdjGemmArgs {
  int m_tiles, n_tiles, kblocks;
  int Q, nH, nA, nV, nP, nVpad, xr0;
  long long HP;
  double* dB;
  int* status;
};

// Plane row r -> (hole, particle) of the [nH][nP] block, or -1 for padding.
__device__ __forceinline__ int row_hp(int r, int nH, int nA, int nV, int nVpad, int xr0, int* h,
                                      int* p) {
  if (r < xr0) {
    const int e = r % nVpad;
    if (e >= nV) return -1;
    *h = r / nVpad;
    *p = nA + e;
    return 0;
  }
  const int t = r - xr0;
  if (t >= nH * nA) return -1;
  *h = t / nA;
  *p = t % nA;
  return 0;
}

// ---------------------------------------------------------------------------
// B^T planes: BT[q][r] = B^Q of plane row r (0 for padding), split into BF16
// hi + lo of fl32(B).
// ---------------------------------------------------------------------------
__global__ void adj_bt_kernel(const double* __restrict__ B, Sizes z, int Qt, int lds, int nVpad,
                              int xr0, uint16_t* __restrict__ hi, uint16_t* __restrict__ lo) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (size_t)Qt * lds) return;
  const int q = (int)(k / lds), r = (int)(k % lds);
  int h, p;
  float v = 0.f;
  if (q < z.Q && row_hp(r, z.nH, z.nA, z.nV, nVpad, xr0, &h, &p) == 0) v = (float)B[bidx(z, q, h, p)];
  const __nv_bfloat16 bh = __float2bfloat16_rn(v);
  hi[k] = __bfloat16_as_ushort(bh);
  lo[k] = __bfloat16_as_ushort(__float2bfloat16_rn(v - __bfloat162float(bh)));
}

// ---------------------------------------------------------------------------
// S outside the core x core block: rows r >= nC*nVpad (active-hole rows (u, f)
// and the active-particle rows (h, x)) against every column c, and the
// transposed block (core rows, those columns). Each integral family adds
// its adjoint at (r, c) and (c, r):
//   X  (F2)   (m e | u f)   dX[m][u][e][f]
//   M         (x e | u f)   dM[x][u][e][f]
//   Z  (F3)   (m e | n u)   dZ[u][m][n][e]     (n u): row of active particle u
//   K1        (i p | u x)   dK1[i][u][x][p]    p any particle, (u x) active rows
//   K2        (i x | u p)   dK2[i][u][x][p]
//   K3        (i x | j y)   dK3[i][x][j][y]
// (u, v as rows are active holes nC + u.) One thread per position, 32 x 32
// tiles through shared memory so that both orientations are written coalesced.
// ---------------------------------------------------------------------------
struct SRestArgs {
  Sizes z;
  int nVpad, xr0, cv_rows, lds;
  const double *dX, *dZ, *dM, *dK1, *dK2, *dK3;
  uint16_t *hi, *lo;
};

__device__ __forceinline__ double s_rest_value(const SRestArgs& a, int r, int c) {
  const Sizes& z = a.z;
  int hr, pr, hc, pc;
  if (row_hp(r, z.nH, z.nA, z.nV, a.nVpad, a.xr0, &hr, &pr) != 0) return 0.0;
  if (row_hp(c, z.nH, z.nA, z.nV, a.nVpad, a.xr0, &hc, &pc) != 0) return 0.0;
  const int nC = z.nC, nA = z.nA, nV = z.nV, nP = z.nP, nH = z.nH;
  const bool rx = pr < nA, cx = pc < nA;  // active-particle rows
  double v = 0.0;
  // X: (m e) core-virtual, (u f) active-virtual
  if (!rx && !cx) {
    if (hr >= nC && hc < nC)
      v += a.dX[(((size_t)hc * nA + (hr - nC)) * nV + (pc - nA)) * nV + (pr - nA)];
    if (hc >= nC && hr < nC)
      v += a.dX[(((size_t)hr * nA + (hc - nC)) * nV + (pr - nA)) * nV + (pc - nA)];
    // M: both active-virtual
    if (hr >= nC && hc >= nC) {
      const int u1 = hr - nC, u2 = hc - nC, e1 = pr - nA, e2 = pc - nA;
      v += a.dM[(((size_t)u1 * nA + u2) * nV + e1) * nV + e2];
      v += a.dM[(((size_t)u2 * nA + u1) * nV + e2) * nV + e1];
    }
  }
  // Z: (m e) core-virtual, (n u) core active-particle
  if (rx && !cx && hr < nC && hc < nC)
    v += a.dZ[(((size_t)pr * nC + hc) * nC + hr) * nV + (pc - nA)];
  if (cx && !rx && hc < nC && hr < nC)
    v += a.dZ[(((size_t)pc * nC + hr) * nC + hc) * nV + (pr - nA)];
  // K1: (i p | u x), the second row an active-hole active-particle row
  if (cx && hc >= nC) v += a.dK1[(((size_t)hr * nA + (hc - nC)) * nA + pc) * nP + pr];
  if (rx && hr >= nC) v += a.dK1[(((size_t)hc * nA + (hr - nC)) * nA + pr) * nP + pc];
  // K2: (i x | u p), the first row active-particle, the second an active-hole row
  if (rx && hc >= nC) v += a.dK2[(((size_t)hr * nA + (hc - nC)) * nA + pr) * nP + pc];
  if (cx && hr >= nC) v += a.dK2[(((size_t)hc * nA + (hr - nC)) * nA + pc) * nP + pr];
  // K3: both active-particle rows
  if (rx && cx) {
    v += a.dK3[(((size_t)hr * nA + pr) * nH + hc) * nA + pc];
    v += a.dK3[(((size_t)hc * nA + pc) * nH + hr) * nA + pr];
  }
  return v;
}

__global__ void __launch_bounds__(256) adj_s_rest_kernel(SRestArgs a) {
  __shared__ float t[32][33];  // t[c][r]
  const int r0 = a.cv_rows + blockIdx.y * 32, c0 = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  // lanes along r: the adjoint arrays are read along their last index where it is r's
  for (int k = ty; k < 32; k += 8) t[k][tx] = (float)s_rest_value(a, r0 + tx, c0 + k);
  __syncthreads();
  for (int k = ty; k < 32; k += 8) {
    const size_t o = (size_t)(r0 + k) * a.lds + c0 + tx;
    const float f = t[tx][k];
    const __nv_bfloat16 bh = __float2bfloat16_rn(f);
    a.hi[o] = __bfloat16_as_ushort(bh);
    a.lo[o] = __bfloat16_as_ushort(__float2bfloat16_rn(f - __bfloat162float(bh)));
  }
  if (c0 < a.cv_rows) {
    // S is symmetric: the same tile transposed in the core-virtual rows
    for (int k = ty; k < 32; k += 8) {
      const size_t o = (size_t)(c0 + k) * a.lds + r0 + tx;
      const float f = t[k][tx];
      const __nv_bfloat16 bh = __float2bfloat16_rn(f);
      a.hi[o] = __bfloat16_as_ushort(bh);
      a.lo[o] = __bfloat16_as_ushort(__float2bfloat16_rn(f - __bfloat162float(bh)));
    }
  }
}

// ---------------------------------------------------------------------------
// dB = S . B^T on the tensor cores (see the file comment).
// ---------------------------------------------------------------------------
__device__ __forceinline__ void ag_item(int it, int m_tiles, int n_tiles, int* mt, int* nt) {
  // bands of AG_BAND m tiles; within a band, n tiles outer: the CTAs running at
  // the same time share the S tiles of one band and the B^T tiles of a few n
  const int per_band = AG_BAND * n_tiles;
  const int band = it / per_band, rem = it % per_band;
  const int bm = min(AG_BAND, m_tiles - band * AG_BAND);
  *nt = rem / bm;
  *mt = band * AG_BAND + rem % bm;
}

__global__ void __launch_bounds__(AG_THREADS, 1)
    adj_gemm_kernel(const __grid_constant__ CUtensorMap map_s_hi,
                    const __grid_constant__ CUtensorMap map_s_lo,
                    const __grid_constant__ CUtensorMap map_bt_hi,
                    const __grid_constant__ CUtensorMap map_bt_lo, const AdjGemmArgs g) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* tiles = smem;
  float* sL2 = (float*)(smem + AG_STAGES * AG_STAGE_BYTES);  // [64][256] second-level sums
  uint64_t* full = (uint64_t*)(sL2 + 64 * 256);
  uint64_t* empty = full + AG_STAGES;
  uint64_t* tfull = empty + AG_STAGES;
  uint64_t* tempty = tfull + AG_NBUF;
  uint64_t* drain = tempty + AG_NBUF;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_items = g.m_tiles * g.n_tiles;

  if (threadIdx.x == 0) {
    for (int s = 0; s < AG_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < AG_NBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], AG_EPI);
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(tmem_slot)),
                 "r"(AG_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_s_hi) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_s_lo) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_bt_hi) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_bt_lo) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        int mt, nt;
        ag_item(it, g.m_tiles, g.n_tiles, &mt, &nt);
        for (int kb = 0; kb < g.kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, g.status)) {
            ok = false;
            break;
          }
          uint8_t* st = tiles + stage * AG_STAGE_BYTES;
          mbar_expect_tx(&full[stage], (uint32_t)AG_STAGE_BYTES);
          const int kq = kb * (AG_KB / 2);
          tma_load_2d(st, &map_s_hi, &full[stage], kq, mt * AG_BM);
          tma_load_2d(st + AG_TILE, &map_s_lo, &full[stage], kq, mt * AG_BM);
          tma_load_2d(st + 2 * AG_TILE, &map_bt_hi, &full[stage], kq, nt * AG_BN);
          tma_load_2d(st + 3 * AG_TILE, &map_bt_lo, &full[stage], kq, nt * AG_BN);
          if (++stage == AG_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        int s = stage;
        uint32_t ph = phase;
        for (int k = 0; k < AG_STAGES; ++k) {
          if (--s < 0) {
            s = AG_STAGES - 1;
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
      constexpr uint32_t idesc = idesc_128x128<true>();
      int stage = 0, tb = 0;
      uint32_t phase = 0, tphase = 0;
      bool ok = true, issued = false;
      for (int it = blockIdx.x; ok && it < n_items; it += gridDim.x) {
        for (int kb = 0; kb < g.kblocks; ++kb) {
          const int sub = kb % AG_CH;  // stage within the TMEM accumulation
          if ((sub == 0 && !mbar_wait(&tempty[tb], tphase ^ 1u, abort_flag, g.status)) ||
              !mbar_wait(&full[stage], phase, abort_flag, g.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t d = tmem_base + (uint32_t)(tb * AG_BN);
          const uint32_t sa = su32(tiles + stage * AG_STAGE_BYTES);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint32_t off = (uint32_t)(k * 32);
            const uint64_t ah = desc_sw64(sa + off), al = desc_sw64(sa + AG_TILE + off);
            const uint64_t bh = desc_sw64(sa + 2 * AG_TILE + off);
            const uint64_t bl = desc_sw64(sa + 3 * AG_TILE + off);
            // a fresh accumulation every AG_CH stages: lo.hi, hi.lo (keeps A), hi.hi (reuses it)
            tc_mma<true>(d, al, bh, idesc, (sub > 0 || k > 0) ? 1u : 0u);
            tc_mma<true, 1>(d, ah, bl, idesc, 1u);
            tc_mma<true, 2>(d, ah, bh, idesc, 1u);
          }
          issued = true;
          tc_commit(&empty[stage]);
          if (++stage == AG_STAGES) {
            stage = 0;
            phase ^= 1u;
          }
          if (sub == AG_CH - 1) {
            tc_commit(&tfull[tb]);
            if (++tb == AG_NBUF) {
              tb = 0;
              tphase ^= 1u;
            }
          }
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
    const int et = threadIdx.x - 64;        // 0..255
    const int quarter = warp & 3;
    const int row = quarter * 32 + lane;
    const int half = (warp - 2) >> 2;       // columns 64*half ..
    int tb = 0;
    uint32_t tphase = 0;
    bool ok = true;
    for (int it = blockIdx.x; it < n_items; it += gridDim.x) {
      int mt, nt;
      ag_item(it, g.m_tiles, g.n_tiles, &mt, &nt);
      float l1[64];
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        l1[c] = 0.f;
        sL2[c * 256 + et] = 0.f;
      }
      int nl1 = 0;
      for (int kc = 0; kc < g.kblocks / AG_CH; ++kc) {
        if (ok) ok = mbar_wait(&tfull[tb], tphase, abort_flag, g.status);
        tc_fence_after();
        if (ok) {
          const uint32_t t = tmem_base + ((uint32_t)(quarter * 32) << 16) +
                             (uint32_t)(tb * AG_BN + half * 64);
          uint32_t r[4][16];
          tmem_ld16(t, r[0]);
          tmem_ld16(t + 16, r[1]);
          tmem_ld16(t + 32, r[2]);
          tmem_ld16(t + 48, r[3]);
          tmem_ld_wait();
          tc_fence_before();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[tb]);
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 16; ++c) l1[16 * j + c] += __uint_as_float(r[j][c]);
          if (++nl1 == AG_L1) {
#pragma unroll
            for (int c = 0; c < 64; ++c) {
              sL2[c * 256 + et] += l1[c];
              l1[c] = 0.f;
            }
            nl1 = 0;
          }
        }
        if (++tb == AG_NBUF) {
          tb = 0;
          tphase ^= 1u;
        }
      }
      if (!ok) continue;
      // the row of dB this thread holds: (h, p) of plane row mt*128 + row
      int h, p;
      if (row_hp(mt * AG_BM + row, g.nH, g.nA, g.nV, g.nVpad, g.xr0, &h, &p) != 0) continue;
      double* out = g.dB + (size_t)h * g.nP + p;
      const int q0 = nt * AG_BN + half * 64;
#pragma unroll
      for (int c = 0; c < 64; ++c) {
        const int q = q0 + c;
        if (q < g.Q) out[(size_t)q * g.HP] = (double)sL2[c * 256 + et] + (double)l1[c];
      }
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(AG_TMEM_COLS)
                 : "memory");
  }
}

static size_t ag_smem_bytes() {
  return 1024 + (size_t)AG_STAGES * AG_STAGE_BYTES + 64 * 256 * 4 +
         (2 * AG_STAGES + 2 * AG_NBUF + 1) * 8 + 16;
}

// ------------------------------- host side -------------------------------
bool tc_adj_alloc(dsrg_plan* p) {
  const Sizes& z = p->z;
  TcAdjWs* w = new TcAdjWs();
  p->tcadj = w;
  w->nVpad = (z.nV + AG_BM - 1) / AG_BM * AG_BM;
  w->xr0 = z.nH * w->nVpad;
  w->rows = split_plane_rows(z);
  w->lds = (w->rows + 63) / 64 * 64;
  w->Qt = (z.Q + AG_BN - 1) / AG_BN * AG_BN;
  w->cv_rows = z.nC * w->nVpad;
  const size_t s_bytes = (size_t)w->rows * w->lds * 2, bt_bytes = (size_t)w->Qt * w->lds * 2;
  if (!plan_alloc(p, (void**)&w->s_hi, s_bytes) || !plan_alloc(p, (void**)&w->s_lo, s_bytes) ||
      !plan_alloc(p, (void**)&w->bt_hi, bt_bytes) || !plan_alloc(p, (void**)&w->bt_lo, bt_bytes))
    return false;
  // padding positions of S are never written: zero once
  if (cudaMemset(w->s_hi, 0, s_bytes) != cudaSuccess || cudaMemset(w->s_lo, 0, s_bytes) != cudaSuccess)
    return false;
  if (!split_make_map(&w->map_s_hi, w->s_hi, true, w->rows, w->lds, AG_KB, AG_BM) ||
      !split_make_map(&w->map_s_lo, w->s_lo, true, w->rows, w->lds, AG_KB, AG_BM) ||
      !split_make_map(&w->map_bt_hi, w->bt_hi, true, w->Qt, w->lds, AG_KB, AG_BN) ||
      !split_make_map(&w->map_bt_lo, w->bt_lo, true, w->Qt, w->lds, AG_KB, AG_BN))
    return false;
  w->m_tiles = (w->rows + AG_BM - 1) / AG_BM;
  w->n_tiles = w->Qt / AG_BN;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  const int items = w->m_tiles * w->n_tiles;
  w->grid = items < nsm ? items : nsm;
  return split_adj_alloc(p);
}

void tc_adj_free(dsrg_plan* p) {
  delete p->tcadj;
  p->tcadj = nullptr;
}

cudaError_t tc_adj_clear(dsrg_plan* p) {
  TcAdjWs* w = p->tcadj;
  if (!w) return cudaSuccess;
  const size_t s_bytes = (size_t)w->rows * w->lds * 2;
  cudaError_t e = cudaMemsetAsync(w->s_hi, 0, s_bytes, p->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(w->s_lo, 0, s_bytes, p->stream);
  return e;
}

cudaError_t tc_adj_ccvv(dsrg_plan* p, const double* B, const double* eps, double s, double* deps,
                        double* ds) {
  TcAdjWs* w = p->tcadj;
  return split_launch_ccvv_adjoint(p, B, eps, s, w->s_hi, w->s_lo, w->lds, deps, ds);
}

cudaError_t tc_adj_rest(dsrg_plan* p, const double* dX, const double* dZ, const double* dM,
                        const double* dK1, const double* dK2, const double* dK3) {
  TcAdjWs* w = p->tcadj;
  SRestArgs a;
  a.z = p->z;
  a.nVpad = w->nVpad;
  a.xr0 = w->xr0;
  a.cv_rows = w->cv_rows;
  a.lds = w->lds;
  a.dX = dX;
  a.dZ = dZ;
  a.dM = dM;
  a.dK1 = dK1;
  a.dK2 = dK2;
  a.dK3 = dK3;
  a.hi = w->s_hi;
  a.lo = w->s_lo;
  const int nrest = w->rows - w->cv_rows;  // a multiple of 64
  dim3 grid(w->lds / 32, nrest / 32);
  adj_s_rest_kernel<<<grid, 256, 0, p->stream>>>(a);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

cudaError_t tc_adj_assemble(dsrg_plan* p, const double* B, double* dB) {
  TcAdjWs* w = p->tcadj;
  const Sizes& z = p->z;
  {
    const size_t n = (size_t)w->Qt * w->lds;
    adj_bt_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(B, z, w->Qt, w->lds, w->nVpad,
                                                                      w->xr0, w->bt_hi, w->bt_lo);
    DSRG_LAUNCH_CHECK(p);
  }
  AdjGemmArgs g;
  g.m_tiles = w->m_tiles;
  g.n_tiles = w->n_tiles;
  g.kblocks = w->lds / (AG_KB / 2);  // lds is a multiple of 64: an even number of stages
  if (g.kblocks % AG_CH != 0) return cudaErrorInvalidValue;
  g.Q = z.Q;
  g.nH = z.nH;
  g.nA = z.nA;
  g.nV = z.nV;
  g.nP = z.nP;
  g.nVpad = w->nVpad;
  g.xr0 = w->xr0;
  g.HP = (long long)z.nH * z.nP;
  g.dB = dB;
  g.status = p->d_status;
  const size_t sm = ag_smem_bytes();
  raise_smem_limit((const void*)adj_gemm_kernel, sm);
  adj_gemm_kernel<<<w->grid, AG_THREADS, sm, p->stream>>>(w->map_s_hi, w->map_s_lo, w->map_bt_hi,
                                                          w->map_bt_lo, g);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

}  // namespace dsrg
