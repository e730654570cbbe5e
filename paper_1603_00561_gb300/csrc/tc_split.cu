// Split-precision CCVV (diagram F1, Eq. (23)) on the 5th-generation tensor
// cores: TMA -> shared memory -> tcgen05.mma -> TMEM -> FP64 epilogue.
//
// The DF factors of the core x virtual block are split once per call into
// two planes, B = hi + lo (TF32 or BF16), laid out K-major (K = the auxiliary
// index Q). For a core pair i<=j and a virtual tile pair A<=B (128 x 128) a
// CTA accumulates in TMEM
//     x = v^{ij}[A,B],  x_ab = sum_Q B_ia B_jb  ~ hi.hi + hi.lo + lo.hi
//     y = v^{ji}[A,B],  y_ab = sum_Q B_ja B_ib  (= v^{ij}_{ba})
// with FP32 accumulation, then an FP64 epilogue adds
//     w * sum_ab (x^2 - x y + y^2) R_ab,   R = (1 - exp(-2 s D^2)) / D,
// D = e_i + e_j - e_a - e_b, w = (2 if i<j) * (2 if A<B); for i = j only x is
// formed (y = x). The regulator is FP64 throughout: exp(-2 s D^2) is the
// product of four exponentials (one per pair, one per row, one per column,
// one pair-independent table), 1/D is an FP32 seed refined by one FP64
// Newton-Raphson step; positions with |D| < 1/4 (never the case for core ->
// virtual excitations of a normal spectrum) take expm1 and an FP64 exchange
// combination instead.
//
// Roles (one CTA per SM, persistent over the work list):
//   warp 0      TMA producer (one elected thread)
//   warp 1      TMEM allocator and MMA issuer (one elected thread)
//   warps 2-5   epilogue: 128 threads, thread = TMEM lane = tile row
// Shared memory: 3 stages x 4 operand slots x 2 planes x (128 rows x 64 B),
// 64-byte swizzle. TMEM: 2 buffers x (x, y) x 128 columns = 512 columns.
// Every wait is bounded (about 2 s); on expiry the CTA records a status word,
// drains what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include "internal.cuh"
#include "regulators.cuh"
#include "tc_common.cuh"

namespace dsrg {

constexpr int TT = 128;                      // tile edge (rows = TMEM lanes, columns)
constexpr int KB_BYTES = 64;                 // K bytes per row per stage (64-byte swizzle span)
constexpr int STAGES = 3;
constexpr int SLOT_BYTES = TT * KB_BYTES;    // one operand tile of one plane: 8 KB
constexpr int STAGE_BYTES = 4 * 2 * SLOT_BYTES;
constexpr int SPLIT_THREADS = 192;
constexpr int TMEM_COLS = 512;

struct SplitWs {
  int elt = 4, kb_elems = 16;
  int nVpad = 0, Qpad = 0, rows = 0, nT = 0, n_tp = 0, n_items = 0, grid = 0;
  void* hi = nullptr;
  void* lo = nullptr;
  CUtensorMap map_hi, map_lo;
  double* alpha = nullptr;  // [n_pairs][nVpad]  exp(4 s E_p e_b)
  double* pinfo = nullptr;  // [n_pairs][4]      E_p, exp(-2 s E_p^2), factorisable flag
  double* tau = nullptr;    // [nVpad][nVpad]    exp(-2 s (e_a + e_b)^2)
  int2* d_tp = nullptr;
};

struct SplitArgs {
  const double* eps;
  double s;
  Sizes z;
  int nVpad, kblocks, n_tp, n_items;
  const int2* pairs;
  const int2* tps;
  const double* alpha;
  const double* pinfo;
  const double* tau;
  double* partials;
  int* status;
};

// Operand slots of one stage: 0 = rows (i, A), 1 = (j, B), 2 = (j, A), 3 = (i, B).
// x = slot g1a . slot g1b^T, y = slot g2a . slot g2b^T; duplicate tiles are
// loaded once (i = j: y not formed; A = B: (j,B) = (j,A), (i,B) = (i,A)).
struct ItemPlan {
  int i, j, A, Bt, p;
  bool two;             // form y
  int nload;            // slots to load: 0 .. nload-1 of the list `load`
  int load[4];          // slot ids to load
  int g1a, g1b, g2a, g2b;
};

__device__ __forceinline__ ItemPlan plan_item(const SplitArgs& a, int item) {
  ItemPlan ip;
  ip.p = item / a.n_tp;
  const int2 ij = a.pairs[ip.p];
  const int2 ab = a.tps[item % a.n_tp];
  ip.i = ij.x;
  ip.j = ij.y;
  ip.A = ab.x;
  ip.Bt = ab.y;
  ip.two = ip.i != ip.j;
  const bool dt = ip.A == ip.Bt;
  if (ip.two && !dt) {
    ip.nload = 4;
    ip.load[0] = 0; ip.load[1] = 1; ip.load[2] = 2; ip.load[3] = 3;
    ip.g1a = 0; ip.g1b = 1; ip.g2a = 2; ip.g2b = 3;
  } else if (ip.two && dt) {
    ip.nload = 2;
    ip.load[0] = 0; ip.load[1] = 2;
    ip.g1a = 0; ip.g1b = 2; ip.g2a = 2; ip.g2b = 0;
  } else if (!dt) {
    ip.nload = 2;
    ip.load[0] = 0; ip.load[1] = 1;
    ip.g1a = 0; ip.g1b = 1; ip.g2a = 0; ip.g2b = 1;
  } else {
    ip.nload = 1;
    ip.load[0] = 0;
    ip.g1a = 0; ip.g1b = 0; ip.g2a = 0; ip.g2b = 0;
  }
  return ip;
}

__device__ __forceinline__ int slot_row(const ItemPlan& ip, int slot, int nVpad) {
  switch (slot) {
    case 0: return ip.i * nVpad + ip.A * TT;
    case 1: return ip.j * nVpad + ip.Bt * TT;
    case 2: return ip.j * nVpad + ip.A * TT;
    default: return ip.i * nVpad + ip.Bt * TT;
  }
}

template <bool BF16>
__global__ void __launch_bounds__(SPLIT_THREADS, 1)
    ccvv_split_kernel(const __grid_constant__ CUtensorMap map_hi,
                      const __grid_constant__ CUtensorMap map_lo, const SplitArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint8_t* tiles = smem;
  uint64_t* full = (uint64_t*)(smem + STAGES * STAGE_BYTES);
  uint64_t* empty = full + STAGES;
  uint64_t* tfull = empty + STAGES;
  uint64_t* tempty = tfull + 2;
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);
  double* sEps = (double*)(smem + STAGES * STAGE_BYTES + 256);
  double* sAlpha = sEps + TT;
  double* sRed = sAlpha + TT;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Sizes& z = a.z;

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
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
                 "r"(TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem_base = *tmem_slot;

  if (warp == 0) {
    // ------------------------------ TMA producer ------------------------------
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_hi) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_lo) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      for (int item = blockIdx.x; ok && item < a.n_items; item += gridDim.x) {
        const ItemPlan ip = plan_item(a, item);
        for (int kb = 0; kb < a.kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.status)) {
            ok = false;
            break;
          }
          uint8_t* st = tiles + stage * STAGE_BYTES;
          mbar_expect_tx(&full[stage], (uint32_t)(ip.nload * 2 * SLOT_BYTES));
          const int kq = kb * (KB_BYTES / (BF16 ? 2 : 4));
          for (int l = 0; l < ip.nload; ++l) {
            const int sl = ip.load[l];
            const int row = slot_row(ip, sl, a.nVpad);
            tma_load_2d(st + (sl * 2 + 0) * SLOT_BYTES, &map_hi, &full[stage], kq, row);
            tma_load_2d(st + (sl * 2 + 1) * SLOT_BYTES, &map_lo, &full[stage], kq, row);
          }
          if (++stage == STAGES) {
            stage = 0;
            phase ^= 1u;
          }
        }
      }
      if (!ok) {
        // drain: wait (bounded) until the copies of the stages still in flight have landed
        int s = stage;
        uint32_t ph = phase;
        for (int k = 0; k < STAGES; ++k) {
          if (--s < 0) {
            s = STAGES - 1;
            ph ^= 1u;
          }
          const unsigned long long t0 = gtimer();
          while (!mbar_try(&full[s], ph) && gtimer() - t0 < TC_WAIT_NS) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------ MMA issuer ------------------------------
    if (lane == 0) {
      constexpr uint32_t idesc = idesc_128x128<BF16>();
      int stage = 0;
      uint32_t phase = 0;
      int tbuf = 0;
      uint32_t tphase = 0;
      bool ok = true;
      bool issued = false;
      for (int item = blockIdx.x; ok && item < a.n_items; item += gridDim.x) {
        const ItemPlan ip = plan_item(a, item);
        if (!mbar_wait(&tempty[tbuf], tphase ^ 1u, abort_flag, a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dx = tmem_base + (uint32_t)(tbuf * 256);
        const uint32_t dy = dx + 128;
        for (int kb = 0; kb < a.kblocks; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = su32(tiles + stage * STAGE_BYTES);
#pragma unroll
          for (int k = 0; k < 2; ++k) {
            const uint32_t off = (uint32_t)(k * 32);
            const uint64_t a1h = desc_sw64(sb + (ip.g1a * 2 + 0) * SLOT_BYTES + off);
            const uint64_t a1l = desc_sw64(sb + (ip.g1a * 2 + 1) * SLOT_BYTES + off);
            const uint64_t b1h = desc_sw64(sb + (ip.g1b * 2 + 0) * SLOT_BYTES + off);
            const uint64_t b1l = desc_sw64(sb + (ip.g1b * 2 + 1) * SLOT_BYTES + off);
            const uint32_t acc0 = (kb > 0 || k > 0) ? 1u : 0u;
            tc_mma<BF16>(dx, a1h, b1h, idesc, acc0);
            tc_mma<BF16>(dx, a1h, b1l, idesc, 1u);
            tc_mma<BF16>(dx, a1l, b1h, idesc, 1u);
            if (ip.two) {
              const uint64_t a2h = desc_sw64(sb + (ip.g2a * 2 + 0) * SLOT_BYTES + off);
              const uint64_t a2l = desc_sw64(sb + (ip.g2a * 2 + 1) * SLOT_BYTES + off);
              const uint64_t b2h = desc_sw64(sb + (ip.g2b * 2 + 0) * SLOT_BYTES + off);
              const uint64_t b2l = desc_sw64(sb + (ip.g2b * 2 + 1) * SLOT_BYTES + off);
              tc_mma<BF16>(dy, a2h, b2h, idesc, acc0);
              tc_mma<BF16>(dy, a2h, b2l, idesc, 1u);
              tc_mma<BF16>(dy, a2l, b2h, idesc, 1u);
            }
          }
          issued = true;
          tc_commit(&empty[stage]);
          if (++stage == STAGES) {
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
        // drain: every MMA issued so far completes before the TMEM is released
        tc_commit(drain);
        const unsigned long long t0 = gtimer();
        while (!mbar_try(drain, 0) && gtimer() - t0 < TC_WAIT_NS) {
        }
      }
    }
  } else {
    // ------------------------------ epilogue ------------------------------
    const int et = threadIdx.x - 64;          // 0..127
    const int quarter = warp & 3;              // TMEM lanes this warp may access
    const int row = quarter * 32 + lane;       // tile row held by this thread
    const int ve = z.nC + z.nA;
    int tbuf = 0;
    uint32_t tphase = 0;
    for (int item = blockIdx.x; item < a.n_items; item += gridDim.x) {
      const ItemPlan ip = plan_item(a, item);
      const double* pi = a.pinfo + 4 * ip.p;
      const double E = pi[0], beta = pi[1];
      const bool fact = pi[2] != 0.0;
      const double* alpha = a.alpha + (size_t)ip.p * a.nVpad;
      named_bar(1, 128);
      {
        const int b = ip.Bt * TT + et;
        sEps[et] = (b < z.nV) ? a.eps[ve + b] : 0.0;
        sAlpha[et] = (b < z.nV) ? alpha[b] : 0.0;
      }
      named_bar(1, 128);
      const int arow = ip.A * TT + row;
      const bool rok = arow < z.nV;
      const double ea = rok ? a.eps[ve + arow] : 0.0;
      const double ca = E - ea;
      const double ha = rok ? beta * alpha[arow] : 0.0;
      const int ncols = min(TT, z.nV - ip.Bt * TT);
      const double s = a.s;

      bool ok = mbar_wait(&tfull[tbuf], tphase, abort_flag, a.status);
      tc_fence_after();
      double acc = 0.0;
      if (ok) {
        const uint32_t tx = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tbuf * 256);
        const uint32_t ty = tx + 128;
        for (int c0 = 0; c0 < ncols; c0 += 16) {
          uint32_t xr[16], yr[16];
          tmem_ld16(tx + c0, xr);
          if (ip.two) tmem_ld16(ty + c0, yr);
          tmem_ld_wait();
          if (!rok) continue;
#pragma unroll
          for (int k = 0; k < 16; ++k) {
            const int cb = c0 + k;
            if (cb >= ncols) break;
            const float xf = __uint_as_float(xr[k]);
            const float yf = ip.two ? __uint_as_float(yr[k]) : xf;
            const double D = ca - sEps[cb];
            double R, q;
            if (fabs(D) >= 0.25) {
              const double g = fact ? ha * sAlpha[cb] * a.tau[(size_t)(ip.Bt * TT + cb) * a.nVpad + arow]
                                    : exp(-2.0 * s * D * D);
              float r0f;
              asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r0f) : "f"((float)D));
              const double r0 = (double)r0f;
              const double e = fma(-D, r0, 1.0);
              const double R0 = (1.0 - g) * r0;
              R = fma(R0, e, R0);
              q = (double)fmaf(xf, xf - yf, yf * yf);
            } else {
              R = reg_f1(D, s);
              const double xd = xf, yd = yf;
              q = fma(xd, xd - yd, yd * yd);
            }
            acc = fma(q, R, acc);
          }
        }
      }
      // release this TMEM buffer to the MMA issuer
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[tbuf]);
      if (++tbuf == 2) {
        tbuf = 0;
        tphase ^= 1u;
      }
      // fixed-order CTA sum of the item's contribution
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sRed[warp - 2] = acc;
      named_bar(1, 128);
      if (et == 0) {
        const double w = (ip.two ? 2.0 : 1.0) * (ip.A < ip.Bt ? 2.0 : 1.0);
        a.partials[item] = ok ? w * (((sRed[0] + sRed[1]) + sRed[2]) + sRed[3]) : 0.0;
      }
      // after an abort the loop keeps running without waits, so that all four
      // epilogue warps keep meeting at the same named barriers
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 1) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem_base),
                 "r"(TMEM_COLS)
                 : "memory");
  }
}

// ---------------------------------------------------------------------------
// Staging: B[Q][h][nA + a] (FP64) -> hi/lo planes [h * nVpad + a][Qpad], K-major.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float tf32_rne(float x) {
  uint32_t u = __float_as_uint(x);
  if ((u & 0x7f800000u) == 0x7f800000u) return x;  // inf / nan unchanged
  u += 0xfffu + ((u >> 13) & 1u);
  u &= 0xffffe000u;
  return __uint_as_float(u);
}

template <bool BF16>
__global__ void split_planes_kernel(const double* __restrict__ B, Sizes z, int nVpad, int Qpad,
                                    void* __restrict__ hi, void* __restrict__ lo) {
  __shared__ double t[32][33];
  const int q0 = blockIdx.x * 32, a0 = blockIdx.y * 32, h = blockIdx.z;
  const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int q = q0 + r, a = a0 + tx;
    t[r][tx] = (q < z.Q && a < z.nV) ? B[bidx(z, q, h, z.nA + a)] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int a = a0 + r, q = q0 + tx;
    const double x = t[tx][r];
    const size_t o = ((size_t)h * nVpad + a) * Qpad + q;
    if (BF16) {
      const __nv_bfloat16 xh = __float2bfloat16_rn((float)x);
      const __nv_bfloat16 xl = __float2bfloat16_rn((float)(x - (double)__bfloat162float(xh)));
      ((__nv_bfloat16*)hi)[o] = xh;
      ((__nv_bfloat16*)lo)[o] = xl;
    } else {
      const float xh = tf32_rne((float)x);
      const float xl = tf32_rne((float)(x - (double)xh));
      ((float*)hi)[o] = xh;
      ((float*)lo)[o] = xl;
    }
  }
}

// Per-pair factors of exp(-2 s D^2) with D = E - e_a - e_b:
//   exp(-2 s E^2) * exp(4 s E e_a) * exp(4 s E e_b) * exp(-2 s (e_a + e_b)^2).
// A pair is factorisable when every exponent stays within +-700.
__global__ void split_tables_kernel(const double* __restrict__ eps, double s, Sizes z,
                                    const int2* __restrict__ pairs, int n_pairs, int nVpad,
                                    double* __restrict__ alpha, double* __restrict__ pinfo,
                                    double* __restrict__ tau) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ve = z.nC + z.nA;
  const size_t na = (size_t)n_pairs * nVpad, nt = (size_t)nVpad * nVpad;
  if (k < na) {
    const int p = (int)(k / nVpad), b = (int)(k % nVpad);
    const int2 ij = pairs[p];
    const double E = eps[ij.x] + eps[ij.y];
    alpha[k] = (b < z.nV) ? exp(4.0 * s * E * eps[ve + b]) : 0.0;
    if (b == 0) {
      double vmax = 0.0;
      for (int v = 0; v < z.nV; ++v) vmax = fmax(vmax, fabs(eps[ve + v]));
      const bool ok = (2.0 * s * E * E <= 700.0) && (4.0 * s * fabs(E) * vmax <= 700.0) &&
                      (8.0 * s * vmax * vmax <= 700.0);
      pinfo[4 * p + 0] = E;
      pinfo[4 * p + 1] = exp(-2.0 * s * E * E);
      pinfo[4 * p + 2] = ok ? 1.0 : 0.0;
      pinfo[4 * p + 3] = 0.0;
    }
  } else if (k < na + nt) {
    const size_t r = k - na;
    const int a = (int)(r / nVpad), b = (int)(r % nVpad);
    double v = 0.0;
    if (a < z.nV && b < z.nV) {
      const double t = eps[ve + a] + eps[ve + b];
      v = exp(-2.0 * s * t * t);
    }
    tau[r] = v;
  }
}

// ------------------------------- host side -------------------------------
static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  if (!fn) {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)f;
  }
  return fn;
}

bool split_supported(const dsrg_plan* p, std::string* why) {
  const Sizes& z = p->z;
  const long long nVpad = (z.nV + TT - 1) / TT * TT;
  if ((long long)z.nH * nVpad >= (1ll << 31)) {
    if (why) *why = "too many rows for 32-bit TMA coordinates";
    return false;
  }
  return true;
}

static bool make_map(CUtensorMap* m, void* ptr, bool bf16, int rows, int Qpad, int kb_elems) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int elt = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)Qpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Qpad * elt};
  cuuint32_t box[2] = {(cuuint32_t)kb_elems, (cuuint32_t)TT};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                  CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

int split_ccvv_blocks(const dsrg_plan* p) {
  const int nT = (p->z.nV + TT - 1) / TT;
  return p->n_pairs * (nT * (nT + 1) / 2);
}

bool split_alloc(dsrg_plan* p) {
  const Sizes& z = p->z;
  SplitWs* w = new SplitWs();
  p->split = w;
  const bool bf16 = p->prec == DSRG_PREC_BF16X3;
  w->elt = bf16 ? 2 : 4;
  w->kb_elems = KB_BYTES / w->elt;
  w->nT = (z.nV + TT - 1) / TT;
  w->nVpad = w->nT * TT;
  w->Qpad = (z.Q + 63) / 64 * 64;
  w->rows = z.nH * w->nVpad;
  w->n_tp = w->nT * (w->nT + 1) / 2;
  w->n_items = p->n_pairs * w->n_tp;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  w->grid = w->n_items < nsm ? w->n_items : nsm;
  const size_t plane = (size_t)w->rows * w->Qpad * w->elt;
  bool ok = plan_alloc(p, &w->hi, plane) && plan_alloc(p, &w->lo, plane) &&
            plan_alloc(p, (void**)&w->alpha, (size_t)p->n_pairs * w->nVpad * 8) &&
            plan_alloc(p, (void**)&w->pinfo, (size_t)p->n_pairs * 4 * 8) &&
            plan_alloc(p, (void**)&w->tau, (size_t)w->nVpad * w->nVpad * 8) &&
            plan_alloc(p, (void**)&w->d_tp, (size_t)w->n_tp * sizeof(int2));
  if (!ok) return false;
  std::vector<int2> tp;
  for (int A = 0; A < w->nT; ++A)
    for (int B = A; B < w->nT; ++B) tp.push_back(make_int2(A, B));
  if (cudaMemcpy(w->d_tp, tp.data(), tp.size() * sizeof(int2), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  // zero the planes once: padding rows/columns stay zero
  if (cudaMemset(w->hi, 0, plane) != cudaSuccess || cudaMemset(w->lo, 0, plane) != cudaSuccess)
    return false;
  if (!make_map(&w->map_hi, w->hi, bf16, w->rows, w->Qpad, w->kb_elems)) return false;
  if (!make_map(&w->map_lo, w->lo, bf16, w->rows, w->Qpad, w->kb_elems)) return false;
  return true;
}

int split_qpad(const dsrg_plan* p) { return p->split->Qpad; }

const CUtensorMap* split_map(const dsrg_plan* p, bool hi) {
  return hi ? &p->split->map_hi : &p->split->map_lo;
}

void split_free(dsrg_plan* p) {
  delete p->split;
  p->split = nullptr;
}

static size_t split_smem_bytes() { return (size_t)STAGES * STAGE_BYTES + 1024 + 256 + 3 * TT * 8 + 64; }

cudaError_t launch_split_ccvv(dsrg_plan* p, const double* B, const double* eps, double s) {
  SplitWs* w = p->split;
  const Sizes& z = p->z;
  const bool bf16 = p->prec == DSRG_PREC_BF16X3;
  {
    dim3 grid(w->Qpad / 32, w->nVpad / 32, z.nH), block(32, 8);
    if (bf16)
      split_planes_kernel<true><<<grid, block, 0, p->stream>>>(B, z, w->nVpad, w->Qpad, w->hi, w->lo);
    else
      split_planes_kernel<false><<<grid, block, 0, p->stream>>>(B, z, w->nVpad, w->Qpad, w->hi, w->lo);
    DSRG_LAUNCH_CHECK(p);
  }
  {
    const size_t n = (size_t)p->n_pairs * w->nVpad + (size_t)w->nVpad * w->nVpad;
    split_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(
        eps, s, z, p->d_pairs, p->n_pairs, w->nVpad, w->alpha, w->pinfo, w->tau);
    DSRG_LAUNCH_CHECK(p);
  }
  SplitArgs a;
  a.eps = eps;
  a.s = s;
  a.z = z;
  a.nVpad = w->nVpad;
  a.kblocks = w->Qpad / w->kb_elems;
  a.n_tp = w->n_tp;
  a.n_items = w->n_items;
  a.pairs = p->d_pairs;
  a.tps = w->d_tp;
  a.alpha = w->alpha;
  a.pinfo = w->pinfo;
  a.tau = w->tau;
  a.partials = p->d_partials + p->segs[p->seg_ccvv].begin;
  a.status = p->d_status;
  const size_t sm = split_smem_bytes();
  if (bf16) {
    cudaFuncSetAttribute(ccvv_split_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ccvv_split_kernel<true><<<w->grid, SPLIT_THREADS, sm, p->stream>>>(w->map_hi, w->map_lo, a);
  } else {
    cudaFuncSetAttribute(ccvv_split_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    ccvv_split_kernel<false><<<w->grid, SPLIT_THREADS, sm, p->stream>>>(w->map_hi, w->map_lo, a);
  }
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

}  // namespace dsrg
