// Split-precision CCVV (diagram F1, Eq. (23)) on the 5th-generation tensor
// cores: TMA -> shared memory -> tcgen05.mma -> TMEM -> FP64 epilogue.
//
// The DF factors of the core x virtual block are split once per call into
// two planes, B = hi + lo (TF32 or BF16), laid out K-major (K = the auxiliary
// index Q). For a core pair i<=j and a virtual tile pair A<=B (128 x 128) a
// CTA accumulates in TMEM
//     x = v^{ij}[A,B],  x_ab = sum_Q B_ia B_jb  ~ hi.hi + hi.lo + lo.hi
//     y = v^{ji}[A,B],  y_ab = sum_Q B_ja B_ib  (= v^{ij}_{ba})
// with FP32 accumulation over Q >= 32; the epilogue adds the terms of the
// first 32 auxiliary functions (the largest) in FP32 with round-to-nearest from
// fl32(B) rows, because the tensor-core accumulator truncates toward zero and
// its bias would otherwise be set by the largest partial sums. Then it adds
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
//   warps 2-9   epilogue: 256 threads; warp w reads TMEM lanes 32*(w%4).. and
//               columns 64*((w-2)/4).. of the tile (two warps per lane quarter)
// Shared memory: 3 stages x 4 operand slots x 2 planes x (128 rows x 64 B),
// 64-byte swizzle (two MMA K steps per stage). The last virtual tile is as wide
// as the virtual space leaves it (N = its width rounded up to 16); when that is
// at most 64, the slots read only as B operands load 64 rows. TMEM: 2 buffers
// x (x, y) x 128 columns = 512 columns.
// Every wait is bounded (about 2 s); on expiry the CTA records a status word,
// drains what it issued, frees its TMEM and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>

#include "internal.cuh"
#include "regulators.cuh"
#include "tc_common.cuh"

namespace dsrg {

constexpr int TT = 128;                      // tile edge (rows = TMEM lanes, columns)
constexpr int KB_BYTES = 64;                 // K bytes per row per stage: two MMA K steps (64-byte swizzle span)
constexpr int STAGES = 3;
constexpr int SLOT_BYTES = TT * KB_BYTES;    // one operand tile of one plane: 8 KB
constexpr int STAGE_BYTES = 4 * 2 * SLOT_BYTES;
constexpr int GEMM_KB_BYTES = 64;            // K bytes per box of the tc_rest GEMM's maps (64-byte swizzle)
constexpr int SPLIT_THREADS = 320;  // warps 0-1 roles, warps 2-9 epilogue
constexpr int EPI_WARPS = 8;
constexpr int TMEM_COLS = 512;

struct SplitWs {
  int elt = 4, kb_elems = 16;
  int nVpad = 0, Qpad = 0, Qld = 0, rows = 0, nT = 0, n_tp = 0, n_items = 0, grid = 0;
  long long row_base = 0;   // first row of this molecule in a shared (batched) plane buffer
  void* hi = nullptr;
  void* lo = nullptr;
  float* tail = nullptr;    // [rows + TAIL_PAD][TAIL_Q]  fl32(B) of the first TAIL_Q auxiliary functions
  CUtensorMap map_hi, map_lo;  // 64-byte swizzled maps of the tc_rest GEMM
  CcvvMaps cmaps;              // 32-byte swizzled maps of the CCVV kernel
  double* alpha = nullptr;  // [n_pairs][nVpad]  exp(4 s E_p e_b)
  double* pinfo = nullptr;  // [n_pairs][4]      E_p, exp(-2 s E_p^2), factorisable flag
  double* tau = nullptr;    // [nVpad][nVpad]    exp(-2 s (e_a + e_b)^2)
  double* trange = nullptr; // [nT][2]           min, max of e over the virtuals of a tile
  double* vmax = nullptr;   // max |e_v| over the virtual orbitals (pair tables)
  void* d_mol = nullptr;    // device MolDesc of this molecule
  int4* d_items = nullptr;  // single-molecule schedule
  int* d_begin = nullptr;
  int order = 0;            // item order of that schedule (split_item_list)
  // The same items split by the core row j of their pair (i <= j) into groups of
  // consecutive rows [h0, h1): a group's items read only rows < h1, so they can
  // run as soon as those rows are staged (the host-buffer entry's pipeline).
  struct Group {
    int h0 = 0, h1 = 0, n = 0, grid = 0;
    int4* d_items = nullptr;
    int* d_begin = nullptr;
  };
  std::vector<Group> groups;
  // The adjoint's recompute of x and y (TF32x3 whatever the plan's precision;
  // for BF16 plans TF32 planes of the core rows of its own): maps and descriptor
  bool adj_ready = false;
  void* adj_hi = nullptr;
  void* adj_lo = nullptr;
  CcvvMaps adj_maps;
  void* d_mol_adj = nullptr;
};

// One molecule of a (possibly batched) CCVV launch.
struct MolDesc {
  const double* eps;      // orbital energies [core | active | virtual]
  double s;
  int nC, nA, nV, nVpad, row0, n_tp;
  int kblocks;            // K stages on the tensor cores: Q from kq0 to the padded end
  int kq0;                // first Q of the tensor-core stages (TAIL_Q)
  const float* tail;      // [plane rows][TAIL_Q] fl32(B) of Q < TAIL_Q (rows local to the molecule)
  const double* alpha;    // [pairs][nVpad]  exp(4 s E_p e_b)
  const double* pinfo;    // [pairs][4]      E_p, exp(-2 s E_p^2), factorisable flag
  const double* tau;      // [nVpad][nVpad]  exp(-2 s (e_a + e_b)^2)
  const double* trange;   // [tiles][2]      min, max of e over the virtuals of a tile
  double* partials;       // one FP64 partial per work item of this molecule
};

// Work item: x = molecule, y = i << 16 | j, z = A << 16 | B, w = item index within
// the molecule (pair-major; pair = w / n_tp). Items are stored CTA by CTA
// (the host scheduler's order); CTA b processes [cta_begin[b], cta_begin[b+1]).
struct SplitArgs {
  const MolDesc* mols;
  const int4* items;
  const int* cta_begin;
  int* status;
  unsigned long long* counts;  // epilogue branch counters (DSRG_COUNT_CCVV_*)
  int prefetch;  // K stages ahead to prefetch into L2 (0: off)
  // adjoint launches only: the core x virtual block of S = 2 dE/dv (BF16 hi
  // and lo planes, row pitch lds elements) and the eps / s derivatives
  uint16_t* s_hi;
  uint16_t* s_lo;
  long long lds;
  double* deps;
  double* ds;
};

// Operand slots of one stage: 0 = rows (i, A), 1 = (j, B), 2 = (j, A), 3 = (i, B).
// x = slot g1a . slot g1b^T, y = slot g2a . slot g2b^T; duplicate tiles are
// loaded once (i = j: y not formed; A = B: (j,B) = (j,A), (i,B) = (i,A)).
struct ItemPlan {
  int i, j, A, Bt, p, slot, mol;
  bool two;             // form y
  int nload;            // slots to load: 0 .. nload-1 of the list `load`
  int load[4];          // slot ids to load
  int g1a, g1b, g2a, g2b;
  int nB;               // MMA N: the item's columns rounded up to 16
  int ncols;            // the item's valid columns (virtual orbitals of tile Bt from cofs)
  int cofs;             // first column of the item within tile Bt (0 or 64)
  int boff;             // byte offset of the B operand rows in an A slot (diagonal tile pairs)
  bool narrow;          // B-only slots (1, 3) of this item load 64 rows (nB <= 64, A != Bt)
};

// HALVES: the launch's items may be column halves (bits 14-15 of z); without
// it every item is a whole tile and the column shape folds to constants.
template <bool HALVES>
__device__ __forceinline__ ItemPlan plan_item(const SplitArgs& a, int idx, const MolDesc** mdp) {
  ItemPlan ip;
  const int4 it = a.items[idx];
  const MolDesc* md = a.mols + it.x;
  *mdp = md;
  ip.mol = it.x;
  ip.i = it.y >> 16;
  ip.j = it.y & 0xffff;
  ip.A = it.z >> 16;
  ip.Bt = it.z & 0x3fff;
  // column shape (bits 14-15): 0 the whole tile Bt, 1 its columns 0-63, 2 its columns 64-127
  const int hc = HALVES ? (it.z >> 14) & 3 : 0;
  ip.cofs = hc == 2 ? 64 : 0;
  ip.slot = it.w;
  ip.p = it.w / md->n_tp;
  ip.two = ip.i != ip.j;
  const bool dt = ip.A == ip.Bt;
  const int nb = min(hc == 0 ? TT : TT / 2, md->nV - ip.Bt * TT - ip.cofs);
  ip.nB = (nb + 15) & ~15;
  ip.ncols = nb;
  // a diagonal tile pair reads its B operand from the A slots, cofs rows in
  // (a whole number of 512-byte swizzle atoms)
  ip.boff = dt ? ip.cofs * KB_BYTES : 0;
  // slots 1 = (j, B) and 3 = (i, B) of an off-diagonal tile pair are read only as
  // B operands (N rows); on a diagonal tile pair every slot is also an A operand
  ip.narrow = !dt && ip.nB <= 64;
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
    case 1: return ip.j * nVpad + ip.Bt * TT + ip.cofs;
    case 2: return ip.j * nVpad + ip.A * TT;
    default: return ip.i * nVpad + ip.Bt * TT + ip.cofs;
  }
}

// The MMAs of one K stage of one item (two K steps of 16 BF16 / 8 TF32 values).
// K runs from the last auxiliary function to the first and the small cross
// products go before hi*hi: the accumulator truncates toward zero at every
// instruction, and with the factors' magnitudes decreasing along Q this keeps
// the accumulator small until the largest terms arrive, so few truncations act
// on the full-size sum. hi*lo and hi*hi share their A operand, which the second
// takes from the collector buffer. N is the item's tile width (nB).
template <bool BF16>
__device__ __forceinline__ void ccvv_stage_mmas(uint32_t dx, uint32_t dy, uint32_t sb,
                                                const ItemPlan& ip, int kb) {
  const uint32_t idesc = idesc_128xn<BF16>((uint32_t)ip.nB);
#pragma unroll
  for (int k = 0; k < 2; ++k) {
    const uint32_t off = (uint32_t)((1 - k) * 32);
    const uint64_t a1h = desc_sw64(sb + (ip.g1a * 2 + 0) * SLOT_BYTES + off);
    const uint64_t a1l = desc_sw64(sb + (ip.g1a * 2 + 1) * SLOT_BYTES + off);
    const uint64_t b1h = desc_sw64(sb + (ip.g1b * 2 + 0) * SLOT_BYTES + ip.boff + off);
    const uint64_t b1l = desc_sw64(sb + (ip.g1b * 2 + 1) * SLOT_BYTES + ip.boff + off);
    const uint32_t acc0 = (kb > 0 || k > 0) ? 1u : 0u;
    tc_mma<BF16>(dx, a1l, b1h, idesc, acc0);
    tc_mma<BF16, 1>(dx, a1h, b1l, idesc, 1u);
    tc_mma<BF16, 2>(dx, a1h, b1h, idesc, 1u);
    if (ip.two) {
      const uint64_t a2h = desc_sw64(sb + (ip.g2a * 2 + 0) * SLOT_BYTES + off);
      const uint64_t a2l = desc_sw64(sb + (ip.g2a * 2 + 1) * SLOT_BYTES + off);
      const uint64_t b2h = desc_sw64(sb + (ip.g2b * 2 + 0) * SLOT_BYTES + ip.boff + off);
      const uint64_t b2l = desc_sw64(sb + (ip.g2b * 2 + 1) * SLOT_BYTES + ip.boff + off);
      tc_mma<BF16>(dy, a2l, b2h, idesc, acc0);
      tc_mma<BF16, 1>(dy, a2h, b2l, idesc, 1u);
      tc_mma<BF16, 2>(dy, a2h, b2h, idesc, 1u);
    }
  }
}

// Split of one FP32 value into BF16 hi + lo (f - hi is exact in FP32).
__device__ __forceinline__ void bf16_split(float f, uint32_t& h, uint32_t& l) {
  const __nv_bfloat16 bh = __float2bfloat16_rn(f);
  h = __bfloat16_as_ushort(bh);
  l = __bfloat16_as_ushort(__float2bfloat16_rn(f - __bfloat162float(bh)));
}

// 16 consecutive values of S (32-byte aligned offset) into the hi and lo planes.
__device__ __forceinline__ void store_split16(uint16_t* hi, uint16_t* lo, long long off,
                                              const float (&v)[16]) {
  uint32_t ph[8], pl[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) {
    uint32_t h0, l0, h1, l1;
    bf16_split(v[2 * k], h0, l0);
    bf16_split(v[2 * k + 1], h1, l1);
    ph[k] = h0 | (h1 << 16);
    pl[k] = l0 | (l1 << 16);
  }
  uint4* dh = (uint4*)(hi + off);
  uint4* dl = (uint4*)(lo + off);
  dh[0] = make_uint4(ph[0], ph[1], ph[2], ph[3]);
  dh[1] = make_uint4(ph[4], ph[5], ph[6], ph[7]);
  dl[0] = make_uint4(pl[0], pl[1], pl[2], pl[3]);
  dl[1] = make_uint4(pl[4], pl[5], pl[6], pl[7]);
}

// One 16-column chunk of the adjoint epilogue (F1 part of the gradient).
// For the item's x_ab = v^{ij}_ab and y_ab = v^{ij}_ba (ordered pairs (i, j) and
// (j, i) are both terms of Eq. (23)), the derivative of E_F1 with respect to
// v^{ij}_ab is W^{ij}_ab = (4 x - 2 y) R and with respect to v^{ij}_ba it is
// (4 y - 2 x) R; v^{ji} holds the same values transposed. dE/dB^Q_{ia} =
// sum_{jb} 2 W^{ij}_ab B^Q_{jb}, so the chunk writes S = 2 W at the four
// positions of the symmetric matrix S over the plane rows (i a), (j b):
//   S[(i,a)][(j,b)] = S[(j,b)][(i,a)] = P = 2 (4x - 2y) R,
//   S[(j,a)][(i,b)] = S[(i,b)][(j,a)] = Q = 2 (4y - 2x) R
// (the duplicates of i = j or A = B are skipped). It adds q R'(D), q = x^2 -
// x y + y^2, to the row sum `racc` and the column sums `colacc`, and q dR/ds
// to `sacc` (the item's weight is applied once at its end).
__device__ __forceinline__ void adjoint_chunk(
    const SplitArgs& a, const ItemPlan& ip, uint32_t (&xr)[16], uint32_t (&yr)[16], bool rok,
    int pth, int c0, int cend, int cbeg, int arow, int nVpad, double ca, double ha, double s,
    const double* sEps, const double* sAlpha, const double* taucol, const float* tail,
    const float* tail_ia, const float* tail_ja, double* colacc, int lane, double& racc,
    double& sacc) {
  if (rok) {
    // the first TAIL_Q auxiliary functions in FP32 round-to-nearest
    tail_add16(tail_ia, tail + (size_t)(ip.j * nVpad + ip.Bt * TT + ip.cofs + c0) * TAIL_Q, xr);
    if (ip.two)
      tail_add16(tail_ja, tail + (size_t)(ip.i * nVpad + ip.Bt * TT + ip.cofs + c0) * TAIL_Q, yr);
  }
  float P[16], Qv[16];
  double gd[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int cb = c0 + k;
    const bool cok = rok && cb < cend;
    const float xf = __uint_as_float(xr[k]);
    const float yf = ip.two ? __uint_as_float(yr[k]) : xf;
    const double D = ca - sEps[cb];
    double Rv, RdD, Rds;
    if (pth == 2) {
      const RegD r = rf1_d(D, s);
      Rv = r.v;
      RdD = r.dD;
      Rds = r.ds;
    } else {
      double r0;
      asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(D));  // 1/D, seed
      const double inv = fma(r0, fma(-D, r0, 1.0), r0);      // one Newton step
      if (pth == 0) {
        // exp(-2 s D^2) < 2^-63: R = 1/D, R' = -1/D^2, dR/ds = 2 D e^{-2sD^2} ~ 0
        Rv = inv;
        RdD = -inv * inv;
        Rds = 0.0;
      } else {
        // |D| >= 1/4: g = exp(-2 s D^2) from the factor tables, 1 - g without cancellation
        const double g = ha * sAlpha[cb] * taucol[(size_t)cb * nVpad];
        const double em = g - 1.0;
        const double x2 = 2.0 * s * D * D;
        Rv = -em * inv;
        RdD = fma(2.0 * x2, g, em) * inv * inv;
        Rds = 2.0 * D * g;
      }
    }
    // S is stored as BF16 hi + lo (16 bits): P and Q in FP32 with the FP64 regulator
    // rounded once; q as in the energy's epilogue, its products with R' and dR/ds in FP64
    const float rvf = (float)Rv;
    P[k] = cok ? 2.f * fmaf(4.f, xf, -2.f * yf) * rvf : 0.f;
    Qv[k] = cok ? 2.f * fmaf(4.f, yf, -2.f * xf) * rvf : 0.f;
    const double q = (double)fmaf(xf, xf - yf, yf * yf);
    const double g1 = cok ? q * RdD : 0.0;
    gd[k] = g1;
    racc += g1;
    sacc += cok ? q * Rds : 0.0;
  }
  // column sums over the warp's 32 rows: a transposing butterfly halves the
  // values per lane at each step; lane l ends with column
  // 8 b4 + 4 b3 + 2 b2 + b1 (b_k = bit k of l), duplicated in lanes l and l ^ 1
  double v8[8], v4[4], v2[2], v1;
  {
    const bool up = (lane & 16) != 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const double send = up ? gd[k] : gd[k + 8];
      v8[k] = (up ? gd[k + 8] : gd[k]) + __shfl_xor_sync(0xffffffffu, send, 16);
    }
  }
  {
    const bool up = (lane & 8) != 0;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const double send = up ? v8[k] : v8[k + 4];
      v4[k] = (up ? v8[k + 4] : v8[k]) + __shfl_xor_sync(0xffffffffu, send, 8);
    }
  }
  {
    const bool up = (lane & 4) != 0;
#pragma unroll
    for (int k = 0; k < 2; ++k) {
      const double send = up ? v4[k] : v4[k + 2];
      v2[k] = (up ? v4[k + 2] : v4[k]) + __shfl_xor_sync(0xffffffffu, send, 4);
    }
  }
  {
    const bool up = (lane & 2) != 0;
    const double send = up ? v2[0] : v2[1];
    v1 = (up ? v2[1] : v2[0]) + __shfl_xor_sync(0xffffffffu, send, 2);
  }
  v1 += __shfl_xor_sync(0xffffffffu, v1, 1);
  if ((lane & 1) == 0) {
    const int col = ((lane >> 4) & 1) * 8 + ((lane >> 3) & 1) * 4 + ((lane >> 2) & 1) * 2 +
                    ((lane >> 1) & 1);
    colacc[c0 - cbeg + col] += v1;
  }
  if (!rok) return;
  const long long lds = a.lds;
  const int colb = ip.Bt * TT + ip.cofs + c0;
  store_split16(a.s_hi, a.s_lo, (long long)(ip.i * nVpad + arow) * lds + ip.j * nVpad + colb, P);
  if (ip.two)
    store_split16(a.s_hi, a.s_lo, (long long)(ip.j * nVpad + arow) * lds + ip.i * nVpad + colb, Qv);
  if (ip.A != ip.Bt) {
    // the transposed positions: one row per column b, the warp's 32 rows a contiguous
#pragma unroll
    for (int k = 0; k < 16; ++k) {
      if (c0 + k >= cend) break;
      uint32_t h, l;
      bf16_split(Qv[k], h, l);
      const long long o1 = (long long)(ip.i * nVpad + colb + k) * lds + ip.j * nVpad + arow;
      a.s_hi[o1] = (uint16_t)h;
      a.s_lo[o1] = (uint16_t)l;
      if (ip.two) {
        bf16_split(P[k], h, l);
        const long long o2 = (long long)(ip.j * nVpad + colb + k) * lds + ip.i * nVpad + arow;
        a.s_hi[o2] = (uint16_t)h;
        a.s_lo[o2] = (uint16_t)l;
      }
    }
  }
}

template <bool BF16, bool ADJ, bool HALVES>
__global__ void __launch_bounds__(SPLIT_THREADS, 1)
    ccvv_split_kernel(const __grid_constant__ CUtensorMap map_hi,
                      const __grid_constant__ CUtensorMap map_lo,
                      const __grid_constant__ CUtensorMap map_hi64,
                      const __grid_constant__ CUtensorMap map_lo64, const SplitArgs a) {
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
  double* sRed = sAlpha + TT;                 // [EPI_WARPS] warp sums
  float* sEpsF = (float*)(sRed + EPI_WARPS);
  float* sCr = sEpsF + TT;  // [TT/16][2]: min, max of e over the valid columns of each 16-column chunk
  unsigned* sCnt = (unsigned*)(sCr + 2 * (TT / 16));  // [EPI_WARPS][3] epilogue blocks by regulator path
  // adjoint epilogue: column sums per warp [EPI_WARPS][64], row sums per column
  // half [2][TT], and the block sums of the pair and s derivatives [2][EPI_WARPS]
  double* sColAcc = (double*)(sCnt + 3 * EPI_WARPS);
  double* sRowAcc = sColAcc + EPI_WARPS * 64;
  double* sRed2 = sRowAcc + 2 * TT;

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int it0 = a.cta_begin[blockIdx.x], it1 = a.cta_begin[blockIdx.x + 1];

  if (threadIdx.x == 0) {
    for (int s = 0; s < STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], EPI_WARPS);
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
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_hi64) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((unsigned long long)&map_lo64) : "memory");
      int stage = 0;
      uint32_t phase = 0;
      bool ok = true;
      constexpr int KE = KB_BYTES / (BF16 ? 2 : 4);
      for (int idx = it0; ok && idx < it1; ++idx) {
        const MolDesc* md;
        const ItemPlan ip = plan_item<HALVES>(a, idx, &md);
        const int kblocks = md->kblocks, row0 = md->row0, nVpad = md->nVpad;
        if (a.prefetch == 0) {
          // The common path. The producer thread is close to the critical path (8
          // TMA issues per stage against 12 MMAs), so everything that does not
          // change along K is set up once per item: rows, maps, shared-memory
          // offsets, L2 policies of the loaded slots and the stage's bytes.
          const int nl = ip.nload;
          int srow[4];
          uint32_t soff[4];
          const CUtensorMap* mh[4];
          const CUtensorMap* ml[4];
          uint32_t bytes = 0;
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            const int sl = l < nl ? ip.load[l] : 0;
            // B-only slots (odd ids) of a narrow tile: 64 rows
            const bool half = ip.narrow && (sl & 1);
            srow[l] = row0 + slot_row(ip, sl, nVpad);
            soff[l] = (uint32_t)(sl * 2 * SLOT_BYTES);
            mh[l] = half ? &map_hi64 : &map_hi;
            ml[l] = half ? &map_lo64 : &map_lo;
            if (l < nl) bytes += half ? SLOT_BYTES : 2 * SLOT_BYTES;
          }
          const int kq0 = md->kq0 + (kblocks - 1) * KE;
          for (int kb = 0; kb < kblocks; ++kb) {
            if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.status)) {
              ok = false;
              break;
            }
            uint8_t* st = tiles + stage * STAGE_BYTES;
            mbar_expect_tx(&full[stage], bytes);
            const int kq = kq0 - kb * KE;
#pragma unroll
            for (int l = 0; l < 4; ++l) {
              if (l >= nl) break;
              tma_load_2d(st + soff[l], mh[l], &full[stage], kq, srow[l]);
              tma_load_2d(st + soff[l] + SLOT_BYTES, ml[l], &full[stage], kq, srow[l]);
            }
            if (++stage == STAGES) {
              stage = 0;
              phase ^= 1u;
            }
          }
          continue;
        }
        // with L2 prefetch (a schedule option the autotuner has never kept)
        // the next item of this CTA, for prefetches that run past this one
        const MolDesc* mdn = md;
        ItemPlan ipn = ip;
        const bool has_next = idx + 1 < it1;
        if (has_next) ipn = plan_item<HALVES>(a, idx + 1, &mdn);
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&empty[stage], phase ^ 1u, abort_flag, a.status)) {
            ok = false;
            break;
          }
          uint8_t* st = tiles + stage * STAGE_BYTES;
          uint32_t bytes = 0;
          for (int l = 0; l < ip.nload; ++l)
            bytes += (ip.narrow && (ip.load[l] & 1)) ? SLOT_BYTES : 2 * SLOT_BYTES;
          mbar_expect_tx(&full[stage], bytes);
          const int kq = md->kq0 + (kblocks - 1 - kb) * KE;
          for (int l = 0; l < ip.nload; ++l) {
            const int sl = ip.load[l];
            const int row = row0 + slot_row(ip, sl, nVpad);
            // B-only slots (odd ids) of a narrow tile: 64 rows
            const bool half = ip.narrow && (sl & 1);
            tma_load_2d(st + (sl * 2 + 0) * SLOT_BYTES, half ? &map_hi64 : &map_hi, &full[stage], kq,
                        row);
            tma_load_2d(st + (sl * 2 + 1) * SLOT_BYTES, half ? &map_lo64 : &map_lo, &full[stage], kq,
                        row);
          }
          if (a.prefetch > 0) {
            // L2 prefetch of the stage `prefetch` ahead (in this item or the next)
            const int kf = kb + a.prefetch;
            if (kf < kblocks) {
              const int kqf = md->kq0 + (kblocks - 1 - kf) * KE;
              for (int l = 0; l < ip.nload; ++l) {
                const int row = row0 + slot_row(ip, ip.load[l], nVpad);
                tma_prefetch_2d(&map_hi, kqf, row);
                tma_prefetch_2d(&map_lo, kqf, row);
              }
            } else if (has_next && kf - kblocks < mdn->kblocks) {
              const int kqf = mdn->kq0 + (mdn->kblocks - 1 - (kf - kblocks)) * KE;
              for (int l = 0; l < ipn.nload; ++l) {
                const int row = mdn->row0 + slot_row(ipn, ipn.load[l], mdn->nVpad);
                tma_prefetch_2d(&map_hi, kqf, row);
                tma_prefetch_2d(&map_lo, kqf, row);
              }
            }
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
      int stage = 0;
      uint32_t phase = 0;
      int tbuf = 0;
      uint32_t tphase = 0;
      bool ok = true;
      bool issued = false;
      for (int idx = it0; ok && idx < it1; ++idx) {
        const MolDesc* md;
        const ItemPlan ip = plan_item<HALVES>(a, idx, &md);
        const int kblocks = md->kblocks;
        if (!mbar_wait(&tempty[tbuf], tphase ^ 1u, abort_flag, a.status)) {
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dx = tmem_base + (uint32_t)(tbuf * 256);
        const uint32_t dy = dx + 128;
        for (int kb = 0; kb < kblocks; ++kb) {
          if (!mbar_wait(&full[stage], phase, abort_flag, a.status)) {
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t sb = su32(tiles + stage * STAGE_BYTES);
          ccvv_stage_mmas<BF16>(dx, dy, sb, ip, kb);
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
    const int et = threadIdx.x - 64;           // 0..255
    const int quarter = warp & 3;              // TMEM lanes this warp may access
    const int row = quarter * 32 + lane;       // tile row held by this thread
    const int wh = (warp - 2) >> 2;            // this warp's half of the item's columns
    int tbuf = 0;
    uint32_t tphase = 0;
    // 32-row x 16-column blocks of this warp by regulator path (lane 0 counts
    // in shared memory; the first barrier of the item loop orders the clearing)
    if (et < 3 * EPI_WARPS) sCnt[et] = 0u;
    for (int idx = it0; idx < it1; ++idx) {
      const MolDesc* md;
      const ItemPlan ip = plan_item<HALVES>(a, idx, &md);
      const int nV = md->nV, nVpad = md->nVpad;
      const int ve = md->nC + md->nA;
      const double* eps = md->eps;
      const double* pi = md->pinfo + 4 * ip.p;
      const double E = pi[0], beta = pi[1];
      const double* alpha = md->alpha + (size_t)ip.p * nVpad;
      const bool factorisable = pi[2] != 0.0;
      named_bar(1, 32 * EPI_WARPS);
      // warp half wh takes the item's columns 64 wh .. 64 wh + 63 (a half item: half 0 alone)
      const int cbeg = wh * 64;
      if (et < TT) {
        const int b = ip.Bt * TT + ip.cofs + et;
        const double eb = (b < nV) ? eps[ve + b] : 0.0;
        sEps[et] = eb;
        sEpsF[et] = (float)eb;
        sAlpha[et] = (b < nV) ? alpha[b] : 0.0;
      }
      named_bar(1, 32 * EPI_WARPS);
      if (et < TT / 16) {
        // range of e over the valid columns of chunk et (FP32: it only picks a path)
        float lo = 3.0e38f, hi = -3.0e38f;
        for (int c = 16 * et; c < 16 * et + 16 && c < ip.ncols; ++c) {
          lo = fminf(lo, sEpsF[c]);
          hi = fmaxf(hi, sEpsF[c]);
        }
        sCr[2 * et] = lo;
        sCr[2 * et + 1] = hi;
      }
      named_bar(1, 32 * EPI_WARPS);
      const int arow = ip.A * TT + row;
      const bool rok = arow < nV;
      const double ea = rok ? eps[ve + arow] : 0.0;
      const double ca = E - ea;
      const float caf = (float)ca;
      const double ha = rok ? beta * alpha[arow] : 0.0;
      const int cend = min(cbeg + 64, ip.ncols);
      const double s = md->s;
      const double* taucol = md->tau + (size_t)(ip.Bt * TT + ip.cofs) * nVpad + arow;
      const float* tail_ia = md->tail + (size_t)(ip.i * nVpad + arow) * TAIL_Q;
      const float* tail_ja = md->tail + (size_t)(ip.j * nVpad + arow) * TAIL_Q;
      // range of E - e_a over this warp's valid rows (FP32)
      float clo = rok ? caf : 3.0e38f, chi = rok ? caf : -3.0e38f;
      for (int o = 16; o > 0; o >>= 1) {
        clo = fminf(clo, __shfl_xor_sync(0xffffffffu, clo, o));
        chi = fmaxf(chi, __shfl_xor_sync(0xffffffffu, chi, o));
      }
      // exp(-2 s D^2) < 2^-63 for every D of a block when 2 s D^2 > 44 (the FP32
      // range carries a margin: 46)
      const float far_d2 = 46.0f / (2.0f * (float)s);
      // adjoint: this thread's sums of q R'(D) over its columns (row a) and of q dR/ds
      double racc = 0.0, sacc = 0.0;
      if constexpr (ADJ) {
        sColAcc[(warp - 2) * 64 + lane] = 0.0;
        sColAcc[(warp - 2) * 64 + 32 + lane] = 0.0;
        __syncwarp();
      }

      bool ok = mbar_wait(&tfull[tbuf], tphase, abort_flag, a.status);
      tc_fence_after();
      double acc = 0.0;
      if (ok) {
        const uint32_t tx = tmem_base + ((uint32_t)(quarter * 32) << 16) + (uint32_t)(tbuf * 256);
        const uint32_t ty = tx + 128;
        for (int c0 = cbeg; c0 < cend; c0 += 16) {
          uint32_t xr[16], yr[16];
          tmem_ld16(tx + c0, xr);
          if (ip.two) tmem_ld16(ty + c0, yr);
          tmem_ld_wait();
          // The regulator path of this warp's 32 rows and the 16 columns from c0
          // (the same for the whole warp): every |D| so large that
          // exp(-2 s D^2) < 2^-63 -> R = 1/D; every |D| >= 1/4 with factorisable
          // exponentials -> the factor tables; else expm1 per element.
          const float dlo = clo - sCr[2 * (c0 >> 4) + 1], dhi = chi - sCr[2 * (c0 >> 4)];
          const bool away = dhi <= -0.25f || dlo >= 0.25f;
          const float dn = dhi <= 0.0f ? dhi : dlo;
          const int pth = !away ? 2 : (dn * dn > far_d2 ? 0 : (factorisable ? 1 : 2));
          if constexpr (ADJ) {
            adjoint_chunk(a, ip, xr, yr, rok, pth, c0, cend, cbeg, arow, nVpad, ca, ha, s, sEps,
                          sAlpha, taucol, md->tail, tail_ia, tail_ja, sColAcc + (warp - 2) * 64,
                          lane, racc, sacc);
            continue;
          }
          if (lane == 0) sCnt[3 * (warp - 2) + pth] += 1u;
          if (!rok) continue;
          // the first TAIL_Q auxiliary functions, the largest terms, in FP32
          // round-to-nearest (the tensor cores took the rest)
          tail_add16(tail_ia, md->tail + (size_t)(ip.j * nVpad + ip.Bt * TT + ip.cofs + c0) * TAIL_Q,
                     xr);
          if (ip.two)
            tail_add16(tail_ja,
                       md->tail + (size_t)(ip.i * nVpad + ip.Bt * TT + ip.cofs + c0) * TAIL_Q, yr);
          if (pth == 0) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int cb = c0 + k;
              if (cb >= cend) break;
              const float xf = __uint_as_float(xr[k]);
              const float yf = ip.two ? __uint_as_float(yr[k]) : xf;
              const double D = ca - sEps[cb];
              double r0;
              asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(D));  // 1/D, seed
              const double R = fma(r0, fma(-D, r0, 1.0), r0);       // one Newton step
              acc = fma((double)fmaf(xf, xf - yf, yf * yf), R, acc);
            }
          } else if (pth == 1) {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int cb = c0 + k;
              if (cb >= cend) break;
              const float xf = __uint_as_float(xr[k]);
              const float yf = ip.two ? __uint_as_float(yr[k]) : xf;
              const double D = ca - sEps[cb];
              const double g = ha * sAlpha[cb] * taucol[(size_t)cb * nVpad];
              double r0;
              asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r0) : "d"(D));  // 1/D, seed
              const double e = fma(-D, r0, 1.0);         // Newton-Raphson residual
              const double R0 = fma(-g, r0, r0);         // (1 - g) / D, seed accuracy
              const double R = fma(R0, e, R0);           // one Newton step
              acc = fma((double)fmaf(xf, xf - yf, yf * yf), R, acc);
            }
          } else {
#pragma unroll
            for (int k = 0; k < 16; ++k) {
              const int cb = c0 + k;
              if (cb >= cend) break;
              const double xd = __uint_as_float(xr[k]);
              const double yd = ip.two ? (double)__uint_as_float(yr[k]) : xd;
              const double D = ca - sEps[cb];
              acc = fma(fma(xd, xd - yd, yd * yd), reg_f1(D, s), acc);
            }
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
      if constexpr (ADJ) {
        // D = e_i + e_j - e_a - e_b: the item's sums of q R'(D) go to e_i and e_j with
        // the sign +, to e_a (its rows) and e_b (its columns) with the sign -
        const int half = (warp - 2) >> 2;
        sRowAcc[half * TT + row] = racc;
        double tr = racc, ts = sacc;
        for (int o = 16; o > 0; o >>= 1) {
          tr += __shfl_xor_sync(0xffffffffu, tr, o);
          ts += __shfl_xor_sync(0xffffffffu, ts, o);
        }
        if (lane == 0) {
          sRed2[warp - 2] = tr;
          sRed2[EPI_WARPS + warp - 2] = ts;
        }
        named_bar(1, 32 * EPI_WARPS);
        if (ok) {
          const double w = (ip.two ? 2.0 : 1.0) * (ip.A < ip.Bt ? 2.0 : 1.0);
          if (et < TT) {
            const int ra = ip.A * TT + et;
            if (ra < nV) atomicAdd(&a.deps[ve + ra], -w * (sRowAcc[et] + sRowAcc[TT + et]));
            // item column et: warp half et / 64, position et % 64 in its warps' sums
            if (et < ip.ncols) {
              const int hb = et >> 6, cc = et & 63;
              double t = 0.0;
              for (int q = 0; q < 4; ++q) t += sColAcc[(4 * hb + q) * 64 + cc];
              atomicAdd(&a.deps[ve + ip.Bt * TT + ip.cofs + et], -w * t);
            }
          } else if (et == TT) {
            double tp = 0.0, tsum = 0.0;
            for (int k = 0; k < EPI_WARPS; ++k) {
              tp += sRed2[k];
              tsum += sRed2[EPI_WARPS + k];
            }
            atomicAdd(&a.deps[ip.i], w * tp);
            atomicAdd(&a.deps[ip.j], w * tp);
            atomicAdd(a.ds, w * tsum);
          }
        }
        // the sums are read before the next item clears them
        named_bar(1, 32 * EPI_WARPS);
        continue;
      }
      // fixed-order sums of the item's 64-column halves: warp butterfly, then the
      // four warps of each warp half in index order. A half item is processed by
      // warp half 0 alone, so the sum of a tile's column half does not depend on
      // whether the tile ran whole or as halves. Partial slot 2 * (pair tile-pair
      // index) + (column half of the tile).
      for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
      if (lane == 0) sRed[warp - 2] = acc;
      named_bar(1, 32 * EPI_WARPS);
      if (et == 0) {
        if (pi[2] == 0.0 && ip.cofs == 0) atomicAdd(&a.counts[DSRG_COUNT_CCVV_UNFACTORABLE], 1ull);
        const double w = (ip.two ? 2.0 : 1.0) * (ip.A < ip.Bt ? 2.0 : 1.0);
        const double t0 = sRed[0] + sRed[1] + sRed[2] + sRed[3];
        const double t1 = sRed[4] + sRed[5] + sRed[6] + sRed[7];
        double* part = md->partials + 2 * ip.slot;
        part[ip.cofs / 64] = ok ? w * t0 : 0.0;
        if (!HALVES) part[1] = ok ? w * t1 : 0.0;
      }
      // after an abort the loop keeps running without waits, so that all
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
  if (threadIdx.x >= 64 && threadIdx.x < 64 + 3 * EPI_WARPS && it1 > it0) {
    const unsigned c = sCnt[threadIdx.x - 64];
    const int slot = (threadIdx.x - 64) % 3;
    if (c)
      atomicAdd(&a.counts[slot == 0 ? DSRG_COUNT_CCVV_FAR
                                    : (slot == 1 ? DSRG_COUNT_CCVV_FACTORED : DSRG_COUNT_CCVV_DIRECT)],
                (unsigned long long)c);
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

// One thread per plane row (h, a) and 16 consecutive Q: the lanes of a warp take
// 32 consecutive a, so every load of one Q is 256 contiguous bytes of B, and each
// thread then writes its row's 16 values per plane as 16-byte stores (no shared
// memory, no barrier: each thread keeps 16 loads in flight). A block is 32 rows
// by 8 Q chunks of 16. The split is of fl32(B): hi = rn(fl32(B)),
// lo = rn(fl32(B) - hi); the difference from splitting B itself is below 2^-24
// relative, under the dropped lo*lo product.
template <bool BF16>
__global__ void __launch_bounds__(256) split_planes_kernel(const double* __restrict__ B, Sizes z,
                                                           int nVpad, int Qld,
                                                           void* __restrict__ hi,
                                                           void* __restrict__ lo,
                                                           float* __restrict__ tail, int h0) {
  const int lane = threadIdx.x & 31;
  const int a = blockIdx.y * 32 + lane;
  const int q0 = (blockIdx.x * 8 + (threadIdx.x >> 5)) * 16;
  const int h = h0 + blockIdx.z;
  if (q0 >= Qld) return;
  double x[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    const int q = q0 + k;
    x[k] = (q < z.Q && a < z.nV) ? B[bidx(z, q, h, z.nA + a)] : 0.0;
  }
  // one FP64 operation per element (the FP64 pipe is the scarce one): xf = fl32(x)
  float xf[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) xf[k] = (float)x[k];
  const size_t row = (size_t)h * nVpad + a;
  if (q0 < TAIL_Q) {
    // fl32(B) of the first TAIL_Q auxiliary functions, row-major per plane row
    float4* tr = (float4*)(tail + row * TAIL_Q + q0);
#pragma unroll
    for (int j = 0; j < 4; ++j) tr[j] = make_float4(xf[4 * j], xf[4 * j + 1], xf[4 * j + 2], xf[4 * j + 3]);
  }
  const size_t o = row * Qld + q0;
  if (BF16) {
    // hi = bf16(xf); xf - hi is exact in FP32; lo = bf16(xf - hi)
    uint32_t ph[8], pl[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      uint32_t wh = 0, wl = 0;
#pragma unroll
      for (int k = 0; k < 2; ++k) {
        const float f = xf[2 * j + k];
        const __nv_bfloat16 xh = __float2bfloat16_rn(f);
        const __nv_bfloat16 xl = __float2bfloat16_rn(f - __bfloat162float(xh));
        wh |= (uint32_t)__bfloat16_as_ushort(xh) << (16 * k);
        wl |= (uint32_t)__bfloat16_as_ushort(xl) << (16 * k);
      }
      ph[j] = wh;
      pl[j] = wl;
    }
    uint4* dh = (uint4*)((__nv_bfloat16*)hi + o);
    uint4* dl = (uint4*)((__nv_bfloat16*)lo + o);
    dh[0] = make_uint4(ph[0], ph[1], ph[2], ph[3]);
    dh[1] = make_uint4(ph[4], ph[5], ph[6], ph[7]);
    dl[0] = make_uint4(pl[0], pl[1], pl[2], pl[3]);
    dl[1] = make_uint4(pl[4], pl[5], pl[6], pl[7]);
  } else {
    float4* dh = (float4*)((float*)hi + o);
    float4* dl = (float4*)((float*)lo + o);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float vh[4], vl[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        vh[k] = tf32_rne(xf[4 * j + k]);
        vl[k] = tf32_rne(xf[4 * j + k] - vh[k]);  // exact in FP32
      }
      dh[j] = make_float4(vh[0], vh[1], vh[2], vh[3]);
      dl[j] = make_float4(vl[0], vl[1], vl[2], vl[3]);
    }
  }
}

// max |x_k| over n values into *out: one CTA, strided per-thread maxima and a
// tree (a maximum is exact, so the order does not matter). NaN entries are
// skipped, as fmax does.
__global__ void __launch_bounds__(256) abs_max_kernel(const double* __restrict__ x, int n,
                                                      double* __restrict__ out) {
  __shared__ double sm[256];
  double m = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) m = fmax(m, fabs(x[k]));
  sm[threadIdx.x] = m;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sm[0];
}

// Per-pair factors of exp(-2 s D^2) with D = E - e_a - e_b:
//   exp(-2 s E^2) * exp(4 s E e_a) * exp(4 s E e_b) * exp(-2 s (e_a + e_b)^2).
// A pair is factorisable when every partial product of these factors, taken in
// the epilogue's order, stays within exp(+-700).
__global__ void split_tables_kernel(const double* __restrict__ eps, double s, Sizes z,
                                    const int2* __restrict__ pairs, int n_pairs, int nVpad,
                                    double* __restrict__ alpha, double* __restrict__ pinfo,
                                    double* __restrict__ tau, double* __restrict__ trange,
                                    double* __restrict__ tau_s, const double* __restrict__ vmaxp) {
  const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int ve = z.nC + z.nA;
  const size_t na = (size_t)n_pairs * nVpad, nt = (size_t)nVpad * nVpad;
  if (k < na) {
    const int p = (int)(k / nVpad), b = (int)(k % nVpad);
    const int2 ij = pairs[p];
    const double E = eps[ij.x] + eps[ij.y];
    alpha[k] = (b < z.nV) ? exp(4.0 * s * E * eps[ve + b]) : 0.0;
    if (b == 0) {
      const double vmax = *vmaxp;  // max |e_v| over the virtual orbitals
      // the epilogue multiplies left to right, exp(-2sE^2) * alpha_a * alpha_b * tau:
      // the partial products carry the exponents -2sE^2 + 4sE e_a (+ 4sE e_b), which
      // for E e > 0 grow past each single factor's, so their sum of magnitudes is bounded
      const bool ok = (2.0 * s * E * E + 8.0 * s * fabs(E) * vmax <= 700.0) &&
                      (8.0 * s * vmax * vmax <= 700.0);
      pinfo[4 * p + 0] = E;
      pinfo[4 * p + 1] = exp(-2.0 * s * E * E);
      pinfo[4 * p + 2] = ok ? 1.0 : 0.0;
      pinfo[4 * p + 3] = 0.0;
    }
  } else if (k < na + nt) {
    const size_t r = k - na;
    const int a = (int)(r / nVpad), b = (int)(r % nVpad);
    double v = 0.0, v1 = 0.0;
    if (a < z.nV && b < z.nV) {
      const double t = eps[ve + a] + eps[ve + b];
      if (tau_s) {
        // the CAVV tables' exp(-s t^2) as well; this table is its square
        v1 = exp(-s * t * t);
        v = v1 * v1;
      } else {
        v = exp(-2.0 * s * t * t);
      }
    }
    tau[r] = v;
    if (tau_s) tau_s[r] = v1;
  } else if (k < na + nt + (size_t)(nVpad / TT)) {
    const int t = (int)(k - na - nt);
    double lo = 1e300, hi = -1e300;
    for (int b = t * TT; b < min((t + 1) * TT, z.nV); ++b) {
      lo = fmin(lo, eps[ve + b]);
      hi = fmax(hi, eps[ve + b]);
    }
    trange[2 * t] = lo;
    trange[2 * t + 1] = hi;
  }
}

// Per-call inputs of the molecules of a launch (eps pointers and s values).
constexpr int MOL_PER_UPDATE = 64;
struct MolInputs {
  const double* eps[MOL_PER_UPDATE];
  double s[MOL_PER_UPDATE];
};
__global__ void mol_inputs_kernel(MolDesc* mols, int first, int n, MolInputs in) {
  const int k = threadIdx.x;
  if (k < n) {
    mols[first + k].eps = in.eps[k];
    mols[first + k].s = in.s[k];
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
  if ((long long)z.nH * nVpad >= (1ll << 31) || z.nC >= 65536 || nVpad / TT >= 65536) {
    if (why) *why = "too many rows for the 32-bit TMA coordinates";
    return false;
  }
  return true;
}

bool split_make_map(CUtensorMap* m, void* ptr, bool bf16, long long rows, int Qld, int kb_bytes,
                    int box_rows) {
  auto fn = encode_fn();
  if (!fn) return false;
  const int elt = bf16 ? 2 : 4;
  cuuint64_t dims[2] = {(cuuint64_t)Qld, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)Qld * elt};
  cuuint32_t box[2] = {(cuuint32_t)(kb_bytes / elt), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  const CUtensorMapSwizzle sw =
      kb_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B : CU_TENSOR_MAP_SWIZZLE_64B;
  CUresult r = fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                  ptr, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, sw,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

bool split_make_ccvv_maps(CcvvMaps* m, void* hi, void* lo, bool bf16, long long rows, int Qld) {
  return split_make_map(&m->hi, hi, bf16, rows, Qld, KB_BYTES, TT) &&
         split_make_map(&m->lo, lo, bf16, rows, Qld, KB_BYTES, TT) &&
         split_make_map(&m->hi64, hi, bf16, rows, Qld, KB_BYTES, TT / 2) &&
         split_make_map(&m->lo64, lo, bf16, rows, Qld, KB_BYTES, TT / 2);
}

// Partial slots of the CCVV energy: one per 64-column half of every (pair,
// tile pair), 2 per tile pair, so that a half's sum is the same whether its
// tile runs whole or as column halves.
int split_ccvv_blocks(const dsrg_plan* p) {
  const int nT = (p->z.nV + TT - 1) / TT;
  return p->n_pairs * (nT * (nT + 1) / 2) * 2;
}

// Rows of one molecule's planes: (h, e) for every hole h and padded virtual e,
// then the active-particle rows (h, x) of tc_rest.cu.
int split_plane_rows(const Sizes& z) { return z.nH * ((z.nV + TT - 1) / TT * TT) + rest_xrows(z); }
int split_plane_qpad(const Sizes& z) { return (z.Q + 63) / 64 * 64; }
// FP32 rows of the first TAIL_Q auxiliary functions: one per plane row plus
// TAIL_PAD zero rows, so that a GEMM tile running past the last plane row
// reads zeros as its TMA loads do.
size_t split_tail_bytes(const Sizes& z) {
  return ((size_t)split_plane_rows(z) + TAIL_PAD) * TAIL_Q * sizeof(float);
}

// Static schedule: items in their global order (molecule, pair, tile pair) are
// dealt to the CTA with the least accumulated cost (ties: lowest index), which
// is round-robin for uniform costs (operand tiles of one pair stay close in
// time, so they are re-read from L2) and balances uneven molecules. Cost of an
// item: its K stages times its GEMM count, plus a fixed epilogue share.
void split_schedule(const std::vector<int4>& items, const std::vector<double>& cost, int ncta,
                    std::vector<int4>& out, std::vector<int>& begin) {
  std::vector<double> load(ncta, 0.0);
  std::vector<std::vector<int>> lists(ncta);
  for (size_t k = 0; k < items.size(); ++k) {
    int best = 0;
    for (int c = 1; c < ncta; ++c)
      if (load[c] < load[best]) best = c;
    load[best] += cost[k];
    lists[best].push_back((int)k);
  }
  out.clear();
  begin.assign(ncta + 1, 0);
  for (int c = 0; c < ncta; ++c) {
    begin[c] = (int)out.size();
    for (int k : lists[c]) out.push_back(items[k]);
  }
  begin[ncta] = (int)out.size();
}

// Work items of one molecule in the order given by `order` (the item's slot,
// which indexes its partial sum, is the same in every order):
//   0           pair-major: (i, j) then tile pairs (A, B)
//   2G + 0      core orbitals in blocks of G; per block pair (I <= J): tile
//               pairs outer, the pairs of the block inner
//   2G + 1      the same blocks; pairs outer, tile pairs inner
// Consecutive items run at the same time on different SMs, so the order sets
// which operand tiles share the L2 at any moment.
void split_item_list(const Sizes& z, int mol, int kblocks, std::vector<int4>& items,
                     std::vector<double>& cost, int code, int rank, int world) {
  const int nT = (z.nV + TT - 1) / TT, nC = z.nC;
  const int n_tp = nT * (nT + 1) / 2;
  const int order = code & 0xffff;
  const bool halves = split_code_halves(code);
  auto pair_index = [&](int i, int j) { return i * nC - i * (i - 1) / 2 + (j - i); };
  auto tp_index = [&](int A, int B) { return A * nT - A * (A - 1) / 2 + (B - A); };
  auto push = [&](int i, int j, int A, int B) {
    if (!pair_in_shard(pair_index(i, j), rank, world)) return;
    const int y = (i << 16) | j;
    const int slot = pair_index(i, j) * n_tp + tp_index(A, B);
    // MMA work: one GEMM for i = j, else two; plus a fixed share for the
    // epilogue. The narrower last tile is not weighted down: equal costs keep
    // the deal round-robin, so that the items running at the same time share
    // operand slabs in L2 (weighting it by width measured 7% slower)
    const double c = ((double)kblocks * (i == j ? 1.0 : 2.0) + 24.0) * (halves ? 0.5 : 1.0);
    // column shape in bits 14-15 of z (halves only): a tile of more than 64
    // columns as two half items, a narrower one as one
    const int width = z.nV - B * TT < TT ? z.nV - B * TT : TT;
    if (halves) {
      items.push_back(make_int4(mol, y, (A << 16) | (1 << 14) | B, slot));
      cost.push_back(c);
      if (width > TT / 2) {
        items.push_back(make_int4(mol, y, (A << 16) | (2 << 14) | B, slot));
        cost.push_back(c);
      }
    } else {
      items.push_back(make_int4(mol, y, (A << 16) | B, slot));
      cost.push_back(c);
    }
  };
  const int G = order >> 1;
  if (G <= 0) {
    for (int i = 0; i < nC; ++i)
      for (int j = i; j < nC; ++j)
        for (int A = 0; A < nT; ++A)
          for (int B = A; B < nT; ++B) push(i, j, A, B);
    return;
  }
  const bool pairs_outer = (order & 1) != 0;
  for (int I0 = 0; I0 < nC; I0 += G)
    for (int J0 = I0; J0 < nC; J0 += G) {
      std::vector<int2> pr;
      for (int i = I0; i < I0 + G && i < nC; ++i)
        for (int j = (J0 > i ? J0 : i); j < J0 + G && j < nC; ++j) pr.push_back(make_int2(i, j));
      if (pairs_outer) {
        for (const int2& ij : pr)
          for (int A = 0; A < nT; ++A)
            for (int B = A; B < nT; ++B) push(ij.x, ij.y, A, B);
      } else {
        for (int A = 0; A < nT; ++A)
          for (int B = A; B < nT; ++B)
            for (const int2& ij : pr) push(ij.x, ij.y, A, B);
      }
    }
}

// Schedule codes the autotuner tries: item order (low 16 bits, pair-major
// first), L2 prefetch distance in K stages (bits 16-23) and column halves
// (bit 24; without prefetch only: prefetching has never paid).
#define DSRG_ORDERS(PF) (PF << 16), (PF << 16) | (2 << 1), (PF << 16) | (4 << 1), (PF << 16) | (8 << 1), \
    (PF << 16) | (4 << 1) | 1, (PF << 16) | (8 << 1) | 1, (PF << 16) | (64 << 1)
const int SPLIT_ORDERS[] = {DSRG_ORDERS(0), DSRG_ORDERS(1 << 8), DSRG_ORDERS(4), DSRG_ORDERS(12)};
#undef DSRG_ORDERS

bool split_code_valid(long long c) { return c >= 0 && (c >> 25) == 0 && ((c >> 16) & 0xff) <= 64; }
int split_code_prefetch(int c) { return (c >> 16) & 0xff; }
bool split_code_halves(int c) { return ((c >> 24) & 1) != 0; }
const int N_SPLIT_ORDERS = sizeof(SPLIT_ORDERS) / sizeof(SPLIT_ORDERS[0]);

bool split_alloc_at(dsrg_plan* p, void* hi, void* lo, int Qld, long long row_base,
                    const CUtensorMap* shared_hi, const CUtensorMap* shared_lo) {
  const Sizes& z = p->z;
  SplitWs* w = new SplitWs();
  p->split = w;
  const bool bf16 = p->prec == DSRG_PREC_BF16X3;
  w->elt = bf16 ? 2 : 4;
  w->kb_elems = KB_BYTES / w->elt;
  w->nT = (z.nV + TT - 1) / TT;
  w->nVpad = w->nT * TT;
  w->Qpad = split_plane_qpad(z);
  w->rows = split_plane_rows(z);
  w->n_tp = w->nT * (w->nT + 1) / 2;
  w->n_items = p->n_pairs * w->n_tp;
  w->Qld = Qld;
  w->row_base = row_base;
  const size_t plane = (size_t)w->rows * Qld * w->elt;
  bool ok = true;
  if (hi) {
    w->hi = hi;
    w->lo = lo;
  } else {
    ok = plan_alloc(p, &w->hi, plane) && plan_alloc(p, &w->lo, plane);
  }
  ok = ok && plan_alloc(p, (void**)&w->alpha, (size_t)p->n_pairs * w->nVpad * 8) &&
       plan_alloc(p, (void**)&w->pinfo, (size_t)p->n_pairs * 4 * 8) &&
       plan_alloc(p, (void**)&w->tau, (size_t)w->nVpad * w->nVpad * 8) &&
       plan_alloc(p, (void**)&w->trange, (size_t)w->nT * 2 * 8) &&
       plan_alloc(p, (void**)&w->vmax, 8) &&
       plan_alloc(p, (void**)&w->d_mol, sizeof(MolDesc)) &&
       plan_alloc(p, (void**)&w->tail, split_tail_bytes(z));
  if (!ok) return false;
  if (cudaMemset(w->tail, 0, split_tail_bytes(z)) != cudaSuccess) return false;
  if (!hi && (cudaMemset(w->hi, 0, plane) != cudaSuccess || cudaMemset(w->lo, 0, plane) != cudaSuccess))
    return false;
  // this molecule's own maps: the tc_rest GEMM's, and the single-molecule CCVV kernel's
  if (!split_make_map(&w->map_hi, w->hi, bf16, w->rows, Qld, GEMM_KB_BYTES, TT)) return false;
  if (!split_make_map(&w->map_lo, w->lo, bf16, w->rows, Qld, GEMM_KB_BYTES, TT)) return false;
  if (!split_make_ccvv_maps(&w->cmaps, w->hi, w->lo, bf16, w->rows, Qld)) return false;
  (void)shared_hi;
  (void)shared_lo;
  // descriptor (eps and s are filled per call)
  MolDesc md;
  md.eps = nullptr;
  md.s = 0.0;
  md.nC = z.nC;
  md.nA = z.nA;
  md.nV = z.nV;
  md.nVpad = w->nVpad;
  md.row0 = 0;
  md.kq0 = TAIL_Q;
  md.kblocks = (w->Qpad - TAIL_Q) / w->kb_elems;
  md.tail = w->tail;
  md.n_tp = w->n_tp;
  md.alpha = w->alpha;
  md.pinfo = w->pinfo;
  md.tau = w->tau;
  md.trange = w->trange;
  md.partials = p->d_partials + p->segs[p->seg_ccvv].begin;
  if (cudaMemcpy(w->d_mol, &md, sizeof(MolDesc), cudaMemcpyHostToDevice) != cudaSuccess) return false;
  // single-molecule schedule
  std::vector<int4> items, sched;
  std::vector<double> cost;
  std::vector<int> begin;
  // sized for the larger item list (every tile in column halves)
  split_item_list(z, 0, md.kblocks, items, cost, 1 << 24);
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  w->grid = (int)items.size() < nsm ? (int)items.size() : nsm;
  ok = plan_alloc(p, (void**)&w->d_items, items.size() * sizeof(int4)) &&
       plan_alloc(p, (void**)&w->d_begin, (w->grid + 1) * sizeof(int));
  if (!ok) return false;
  return split_set_order(p, 0) == cudaSuccess;
}

// Rebuild the single-molecule schedule for item order `order`.
cudaError_t split_set_order(dsrg_plan* p, int order) {
  SplitWs* w = p->split;
  std::vector<int4> items, sched;
  std::vector<double> cost;
  std::vector<int> begin;
  split_item_list(p->z, 0, w->Qpad / w->kb_elems, items, cost, order, p->shard_rank,
                  p->shard_world);
  split_schedule(items, cost, w->grid, sched, begin);
  cudaError_t e = cudaMemcpy(w->d_items, sched.data(), sched.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(w->d_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice);
  for (SplitWs::Group& g : w->groups) {
    if (e != cudaSuccess) break;
    std::vector<int4> gi;
    std::vector<double> gc;
    for (size_t k = 0; k < items.size(); ++k) {
      const int j = items[k].y & 0xffff;
      if (j >= g.h0 && j < g.h1) {
        gi.push_back(items[k]);
        gc.push_back(cost[k]);
      }
    }
    split_schedule(gi, gc, g.grid, sched, begin);
    e = cudaMemcpy(g.d_items, sched.data(), sched.size() * sizeof(int4), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
      e = cudaMemcpy(g.d_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) w->order = order;
  return e;
}

// Split the core rows into groups of consecutive rows for the host-buffer
// pipeline (bounds[0] = 0 < ... < bounds.back() = nC) and build their schedules
// (item order of the plan).
bool split_alloc_groups(dsrg_plan* p, const std::vector<int>& bounds) {
  SplitWs* w = p->split;
  const int ngroups = (int)bounds.size() - 1;
  if (ngroups < 1) return true;
  int nsm = 148;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  std::vector<int4> items;
  std::vector<double> cost;
  // group sizes for the larger item list (every tile in column halves)
  split_item_list(p->z, 0, w->Qpad / w->kb_elems, items, cost, 1 << 24, p->shard_rank,
                  p->shard_world);
  w->groups.resize(ngroups);
  for (int g = 0; g < ngroups; ++g) {
    SplitWs::Group& G = w->groups[g];
    G.h0 = bounds[g];
    G.h1 = bounds[g + 1];
    G.n = 0;
    for (const int4& it : items) {
      const int j = it.y & 0xffff;
      G.n += (j >= G.h0 && j < G.h1) ? 1 : 0;
    }
    G.grid = G.n < nsm ? G.n : nsm;
    if (G.n == 0) continue;
    if (!plan_alloc(p, (void**)&G.d_items, (size_t)G.n * sizeof(int4)) ||
        !plan_alloc(p, (void**)&G.d_begin, (size_t)(G.grid + 1) * sizeof(int)))
      return false;
  }
  return split_set_order(p, w->order) == cudaSuccess;
}

int split_n_groups(const dsrg_plan* p) { return p->split ? (int)p->split->groups.size() : 0; }

void split_group_rows(const dsrg_plan* p, int g, int* h0, int* h1) {
  *h0 = p->split->groups[g].h0;
  *h1 = p->split->groups[g].h1;
}

// The CCVV items of row group g (planes of rows < its h1 and the tables staged).
cudaError_t split_launch_group(dsrg_plan* p, int g) {
  SplitWs* w = p->split;
  const SplitWs::Group& G = w->groups[g];
  if (G.n == 0) return cudaSuccess;
  return split_launch_ccvv(p, w->cmaps, w->d_mol, G.d_items, G.d_begin, G.grid,
                           p->prec == DSRG_PREC_BF16X3, w->order);
}

int split_order(const dsrg_plan* p) { return p->split ? p->split->order : -1; }

// Average duration of the CCVV kernel alone (planes and tables staged by the
// caller), `reps` launches between two events on the plan's stream.
cudaError_t split_time_ccvv(dsrg_plan* p, int reps, float* ms) {
  SplitWs* w = p->split;
  cudaEvent_t e0, e1;
  cudaError_t e = cudaEventCreate(&e0);
  if (e != cudaSuccess) return e;
  if ((e = cudaEventCreate(&e1)) != cudaSuccess) {
    cudaEventDestroy(e0);
    return e;
  }
  const bool bf16 = p->prec == DSRG_PREC_BF16X3;
  e = cudaEventRecord(e0, p->stream);
  for (int r = 0; e == cudaSuccess && r < reps; ++r)
    e = split_launch_ccvv(p, w->cmaps, w->d_mol, w->d_items, w->d_begin, w->grid, bf16,
                          w->order);
  if (e == cudaSuccess) e = cudaEventRecord(e1, p->stream);
  if (e == cudaSuccess) e = cudaEventSynchronize(e1);
  if (e == cudaSuccess) {
    float t = 0.f;
    e = cudaEventElapsedTime(&t, e0, e1);
    *ms = t / (float)(reps > 0 ? reps : 1);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return e;
}

bool split_alloc(dsrg_plan* p) {
  return split_alloc_at(p, nullptr, nullptr, split_plane_qpad(p->z), 0, nullptr, nullptr);
}

int split_qpad(const dsrg_plan* p) { return p->split->Qpad; }
int split_qld(const dsrg_plan* p) { return p->split->Qld; }
void* split_plane_ptr(const dsrg_plan* p, bool hi) { return hi ? p->split->hi : p->split->lo; }
const float* split_tail_ptr(const dsrg_plan* p) { return p->split->tail; }

const CUtensorMap* split_map(const dsrg_plan* p, bool hi) {
  return hi ? &p->split->map_hi : &p->split->map_lo;
}

void split_free(dsrg_plan* p) {
  delete p->split;
  p->split = nullptr;
}

static size_t split_smem_bytes() {
  return (size_t)STAGES * STAGE_BYTES + 1024 + 256 + (2 * TT + EPI_WARPS) * 8 + TT * 4 +
         2 * (TT / 16) * 4 + 3 * EPI_WARPS * 4 + 64;
}

// Planes (and FP32 tail rows) of the hole rows h0 <= h < h1 of B.
cudaError_t split_stage_rows(dsrg_plan* p, const double* B, int h0, int h1) {
  SplitWs* w = p->split;
  const Sizes& z = p->z;
  if (h1 <= h0) return cudaSuccess;
  dim3 grid((w->Qpad + 127) / 128, w->nVpad / 32, h1 - h0);
  if (p->prec == DSRG_PREC_BF16X3)
    split_planes_kernel<true><<<grid, 256, 0, p->stream>>>(B, z, w->nVpad, w->Qld, w->hi, w->lo,
                                                           w->tail, h0);
  else
    split_planes_kernel<false><<<grid, 256, 0, p->stream>>>(B, z, w->nVpad, w->Qld, w->hi, w->lo,
                                                            w->tail, h0);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// Pair tables of the regulator (they read eps only).
cudaError_t split_stage_tables(dsrg_plan* p, const double* eps, double s) {
  SplitWs* w = p->split;
  abs_max_kernel<<<1, 256, 0, p->stream>>>(eps + p->z.nC + p->z.nA, p->z.nV, w->vmax);
  DSRG_LAUNCH_CHECK(p);
  const size_t n = (size_t)p->n_pairs * w->nVpad + (size_t)w->nVpad * w->nVpad + w->nT;
  double* tau_s = p->rest ? rest_take_tau1(p) : nullptr;
  split_tables_kernel<<<(unsigned)((n + 255) / 256), 256, 0, p->stream>>>(
      eps, s, p->z, p->d_pairs, p->n_pairs, w->nVpad, w->alpha, w->pinfo, w->tau, w->trange, tau_s,
      w->vmax);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// Stage this molecule's planes and pair tables (no CCVV launch).
cudaError_t split_stage(dsrg_plan* p, const double* B, const double* eps, double s) {
  cudaError_t e = split_stage_rows(p, B, 0, p->z.nH);
  if (e == cudaSuccess) e = split_stage_tables(p, eps, s);
  return e;
}

// Self-test of the timeout path of the kernels' bounded waits: one thread waits,
// through the same mbar_wait, on an mbarrier that nothing arrives on. After the
// bound (TC_WAIT_NS) it records the status word and the kernel returns.
__global__ void wait_selftest_kernel(int* status) {
  __shared__ uint64_t bar;
  __shared__ int abort_flag;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) (void)mbar_wait(&bar, 0u, (volatile int*)&abort_flag, status);
}

cudaError_t launch_wait_selftest(dsrg_plan* p) {
  wait_selftest_kernel<<<1, 32, 0, p->stream>>>(p->d_status);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

size_t split_mol_desc_bytes() { return sizeof(MolDesc); }
int split_kb_elems(bool bf16) { return KB_BYTES / (bf16 ? 2 : 4); }

// Descriptor of plan p's molecule for a launch over a shared plane buffer in
// which its rows start at row0.
void split_fill_mol_desc(const dsrg_plan* p, long long row0, void* out) {
  const SplitWs* w = p->split;
  MolDesc md;
  md.eps = nullptr;
  md.s = 0.0;
  md.nC = p->z.nC;
  md.nA = p->z.nA;
  md.nV = p->z.nV;
  md.nVpad = w->nVpad;
  md.row0 = (int)row0;
  md.kq0 = TAIL_Q;
  md.kblocks = (w->Qpad - TAIL_Q) / w->kb_elems;
  md.tail = w->tail;
  md.n_tp = w->n_tp;
  md.alpha = w->alpha;
  md.pinfo = w->pinfo;
  md.tau = w->tau;
  md.trange = w->trange;
  md.partials = p->d_partials + p->segs[p->seg_ccvv].begin;
  memcpy(out, &md, sizeof(MolDesc));
}

cudaError_t split_set_inputs(dsrg_plan* p, void* d_mols_v, int first, int n,
                             const double* const* eps, const double* s) {
  MolDesc* d_mols = (MolDesc*)d_mols_v;
  for (int b = 0; b < n; b += MOL_PER_UPDATE) {
    MolInputs in;
    const int m = (n - b) < MOL_PER_UPDATE ? (n - b) : MOL_PER_UPDATE;
    for (int k = 0; k < m; ++k) {
      in.eps[k] = eps[b + k];
      in.s[k] = s[b + k];
    }
    mol_inputs_kernel<<<1, MOL_PER_UPDATE, 0, p->stream>>>(d_mols, first + b, m, in);
    DSRG_LAUNCH_CHECK(p);
  }
  return cudaSuccess;
}

template <bool BF16, bool ADJ, bool HALVES>
static void launch_ccvv_instance(dsrg_plan* p, const CcvvMaps& m, int grid, size_t sm,
                                 const SplitArgs& a) {
  raise_smem_limit((const void*)ccvv_split_kernel<BF16, ADJ, HALVES>, sm);
  ccvv_split_kernel<BF16, ADJ, HALVES><<<grid, SPLIT_THREADS, sm, p->stream>>>(m.hi, m.lo, m.hi64,
                                                                              m.lo64, a);
}

cudaError_t split_launch_ccvv(dsrg_plan* p, const CcvvMaps& maps, const void* d_mols,
                              const int4* d_items, const int* d_begin, int grid, bool bf16,
                              int code) {
  const int prefetch = split_code_prefetch(code);
  const bool halves = split_code_halves(code);
  SplitArgs a;
  a.mols = (const MolDesc*)d_mols;
  a.items = d_items;
  a.cta_begin = d_begin;
  a.status = p->d_status;
  a.counts = p->d_counts;
  a.prefetch = prefetch;
  a.s_hi = a.s_lo = nullptr;
  a.lds = 0;
  a.deps = a.ds = nullptr;
  const size_t sm = split_smem_bytes();
  if (bf16 && halves)
    launch_ccvv_instance<true, false, true>(p, maps, grid, sm, a);
  else if (bf16)
    launch_ccvv_instance<true, false, false>(p, maps, grid, sm, a);
  else if (halves)
    launch_ccvv_instance<false, false, true>(p, maps, grid, sm, a);
  else
    launch_ccvv_instance<false, false, false>(p, maps, grid, sm, a);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// The adjoint's recompute of the CCVV pair blocks needs TF32 operands: a BF16x3
// product carries each factor to 16 bits, and the element-wise errors of x and
// y (which the energy averages away) would reach dE/dB. TF32x3 plans reuse
// their planes and descriptor; BF16x3 plans get TF32 planes of the core rows.
bool split_adj_alloc(dsrg_plan* p) {
  SplitWs* w = p->split;
  const Sizes& z = p->z;
  if (p->prec != DSRG_PREC_BF16X3) {
    w->adj_maps = w->cmaps;
    w->d_mol_adj = w->d_mol;
    w->adj_ready = true;
    return true;
  }
  const long long rows = (long long)z.nC * w->nVpad;
  const size_t plane = (size_t)rows * w->Qpad * 4;
  if (!plan_alloc(p, &w->adj_hi, plane) || !plan_alloc(p, &w->adj_lo, plane) ||
      !plan_alloc(p, &w->d_mol_adj, sizeof(MolDesc)))
    return false;
  if (cudaMemset(w->adj_hi, 0, plane) != cudaSuccess || cudaMemset(w->adj_lo, 0, plane) != cudaSuccess)
    return false;
  if (!split_make_ccvv_maps(&w->adj_maps, w->adj_hi, w->adj_lo, false, rows, w->Qpad)) return false;
  MolDesc md;
  if (cudaMemcpy(&md, w->d_mol, sizeof(MolDesc), cudaMemcpyDeviceToHost) != cudaSuccess) return false;
  md.kblocks = (w->Qpad - TAIL_Q) / (KB_BYTES / 4);
  if (cudaMemcpy(w->d_mol_adj, &md, sizeof(MolDesc), cudaMemcpyHostToDevice) != cudaSuccess)
    return false;
  w->adj_ready = true;
  return true;
}

// F1's part of the gradient for the plan's pairs: S (core x virtual block),
// deps and ds (added to). The planes, tail rows and pair tables of the energy
// call just made on the stream (same B, eps, s) are reused.
cudaError_t split_launch_ccvv_adjoint(dsrg_plan* p, const double* B, const double* eps, double s,
                                      uint16_t* s_hi, uint16_t* s_lo, long long lds, double* deps,
                                      double* ds) {
  SplitWs* w = p->split;
  const Sizes& z = p->z;
  if (!w->adj_ready) return cudaErrorInvalidValue;
  if (p->prec == DSRG_PREC_BF16X3) {
    dim3 grid((w->Qpad + 127) / 128, w->nVpad / 32, z.nC);
    // the tail rows are rewritten with the same fl32(B) values
    split_planes_kernel<false><<<grid, 256, 0, p->stream>>>(B, z, w->nVpad, w->Qpad, w->adj_hi,
                                                            w->adj_lo, w->tail, 0);
    DSRG_LAUNCH_CHECK(p);
    cudaError_t e = split_set_inputs(p, w->d_mol_adj, 0, 1, &eps, &s);
    if (e != cudaSuccess) return e;
  }
  SplitArgs a;
  a.mols = (const MolDesc*)w->d_mol_adj;
  a.items = w->d_items;
  a.cta_begin = w->d_begin;
  a.status = p->d_status;
  a.counts = p->d_counts;
  a.prefetch = 0;
  a.s_hi = s_hi;
  a.s_lo = s_lo;
  a.lds = lds;
  a.deps = deps;
  a.ds = ds;
  const size_t sm = split_smem_bytes() + (EPI_WARPS * 64 + 2 * TT + 2 * EPI_WARPS) * 8;
  if (split_code_halves(w->order))
    launch_ccvv_instance<false, true, true>(p, w->adj_maps, w->grid, sm, a);
  else
    launch_ccvv_instance<false, true, false>(p, w->adj_maps, w->grid, sm, a);
  DSRG_LAUNCH_CHECK(p);
  return cudaSuccess;
}

// Per-call inputs (eps, s) of the single-molecule descriptor.
cudaError_t split_prepare_single(dsrg_plan* p, const double* eps, double s) {
  return split_set_inputs(p, p->split->d_mol, 0, 1, &eps, &s);
}

cudaError_t launch_split_ccvv(dsrg_plan* p, const double* B, const double* eps, double s) {
  SplitWs* w = p->split;
  cudaError_t e = split_stage(p, B, eps, s);
  if (e != cudaSuccess) return e;
  if ((e = split_prepare_single(p, eps, s)) != cudaSuccess) return e;
  return split_launch_ccvv(p, w->cmaps, w->d_mol, w->d_items,
                           w->d_begin, w->grid, p->prec == DSRG_PREC_BF16X3, w->order);
}

}  // namespace dsrg
