// Internal declarations of the DSRG-MRPT2 CUDA library (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "dsrg.h"

namespace dsrg {

constexpr int NA_MAX = 8;  // largest active space the kernels are built for

struct Sizes {
  int nC, nA, nV, Q;  // core, active, virtual, auxiliary
  int nH, nP, n;      // holes nC+nA, particles nA+nV, orbitals
};

// Index of B^Q_{h p} in the [naux][nH][nP] hole x particle layout.
__host__ __device__ __forceinline__ size_t bidx(const Sizes& z, int q, int h, int p) {
  return ((size_t)q * z.nH + h) * z.nP + p;
}

// Segments of the partial-sum buffer: every kernel that contributes to the
// energy writes one FP64 partial per CTA into its own segment; a final
// kernel adds the segments of each block in a fixed order.
enum Block { BLK_CCVV = 0, BLK_CAVV = 1, BLK_CCAV = 2, BLK_ACTIVE = 3 };

struct Segment {
  int begin, count, block;
};
constexpr int RED_CHUNK = 4096;  // partials per CTA of the first reduction level

// Active-block workspace (spin-orbital tables and spatial integrals).
struct ActiveWs {
  double* K1 = nullptr;   // (ia|ux)  [nH][nA][nA][nP]
  double* K2 = nullptr;   // (ix|ua)  [nH][nA][nA][nP]
  double* K3 = nullptr;   // (ix|jy)  [nH][nA][nH][nA]
  double* W1 = nullptr;   // 3 x [2nH][2nA][2nP][2nA]  (V, T, Vt)   <iu||ax>
  double* W2 = nullptr;   // 3 x [2nH][2nH][2nA][2nA]  (V, T, Vt)   <ij||xy>
  double* Ti = nullptr;   // [2nH][2nA][2nP][2nA]  gamma/eta-dressed T of W1
  double* lam = nullptr;  // [2nA]^4 spin-orbital cumulant
  double* gA = nullptr;   // [2nA][2nA]
  double* t1 = nullptr;   // [2nH][2nP]
  double* ft = nullptr;   // [2nH][2nP]
  double* M = nullptr;    // (xe|uf) [nA][nA][nV][nV]
  double* P12 = nullptr;  // P1, P2 [2][nA^4]
  double* P12part = nullptr;  // per-CTA partials of P1/P2 [nblk][2][nA^4]
  size_t w1n = 0, w2n = 0;
  int actvv_blocks = 0;
};

struct SplitWs;    // tensor-core path workspace (tc_split.cu)
struct RestState;  // tensor-core CAVV / CCAV / active integrals (tc_rest.cu)
struct GradWs;   // gradient workspace (grad.cu)
struct TcAdjWs;  // tensor-core assembly of dE/dB for split plans (tc_adjoint.cu)

}  // namespace dsrg

struct dsrg_plan {
  dsrg::Sizes z{};
  dsrg_precision_t prec = DSRG_PREC_FP64;
  cudaStream_t stream = nullptr;
  uint32_t flags = 0;
  int device = 0;
  std::string last_error;
  int launches = 0;
  size_t ws_bytes = 0;
  std::vector<void*> allocs;

  // CCVV (F1) work list: pairs i<=j and tile pairs A<=B
  int tile_ccvv = 64;
  int n_pairs = 0, n_tp_ccvv = 0;
  int2* d_pairs = nullptr;     // [n_pairs] (i, j)
  int2* d_tp_ccvv = nullptr;   // [n_tp_ccvv] (A, B)
  // CAVV (F2) work list: tile pairs with 32-wide tiles
  int tile_cavv = 32;
  int n_tp_cavv = 0;
  int2* d_tp_cavv = nullptr;

  // partial sums and segments
  double* d_partials = nullptr;
  int n_partials = 0;
  std::vector<dsrg::Segment> segs;
  dsrg::Segment* d_segs = nullptr;
  int n_chunks = 0;             // (segment, chunk) pairs of the first reduction level
  int2* d_chunks = nullptr;
  double* d_red = nullptr;      // [n_chunks][2] chunk sums and compensations
  int seg_ccvv = -1, seg_cavv = -1, seg_ccav = -1;
  std::vector<int> seg_active;
  double* d_pairbuf = nullptr;  // [nC*nC] pair energies (scratch for the pairs entry)

  dsrg::ActiveWs act;
  dsrg::SplitWs* split = nullptr;
  dsrg::RestState* rest = nullptr;  // split CAVV / CCAV / active integrals (tc_rest.cu)
  dsrg::GradWs* grad = nullptr;  // gradient workspace (DSRG_PLAN_GRAD)
  dsrg::TcAdjWs* tcadj = nullptr;  // split plans' S and B^T planes of the gradient
  bool rest_tc = false;        // CAVV, CCAV and the active integrals from the tensor-core GEMM

  // device staging of dsrg_mrpt2_energy_host (DSRG_PLAN_HOST_IO)
  double *st_B = nullptr, *st_eps = nullptr, *st_g = nullptr, *st_l = nullptr, *st_out = nullptr;
  // split plans: B is copied in groups of core rows on st_copy while the CCVV
  // items of the groups already staged run; st_ev[g] marks group g copied,
  // st_ev[G] the active rows, st_ev[G + 1] the previous call done with st_B
  cudaStream_t st_copy = nullptr;
  std::vector<cudaEvent_t> st_ev;

  // multi-GPU share of this plan (dsrg_plan_set_shard): CCVV pairs with index
  // = shard_rank (mod shard_world); the other blocks only on rank 0
  int shard_rank = 0, shard_world = 1;

  // device status word (bounded waits)
  int* d_status = nullptr;
  // counters of the epilogue branches taken by the split kernels (DSRG_COUNT_*)
  unsigned long long* d_counts = nullptr;
};

namespace dsrg {

// Allocation helper: records the pointer in the plan; returns false on failure.
bool plan_alloc(dsrg_plan* p, void** ptr, size_t bytes);

// Raise (never lower) a kernel's dynamic shared-memory limit on the current
// device. A launch captured in a CUDA graph keeps its own size; lowering the
// limit afterwards for a smaller problem would invalidate that launch.
cudaError_t raise_smem_limit(const void* func, size_t bytes);

// Launchers (each returns cudaSuccess or the launch error; adds to p->launches).
cudaError_t launch_ccvv_fp64(dsrg_plan* p, const double* B, const double* eps, double s);
cudaError_t launch_cavv_fp64(dsrg_plan* p, const double* B, const double* eps, const double* G,
                             double s);
cudaError_t launch_ccav_fp64(dsrg_plan* p, const double* B, const double* eps, const double* G,
                             double s);
// ints_ready: K1, K2, K3 and M are already formed (split path); otherwise they
// are formed here in FP64 from B. L3 (spin-orbital three-body cumulant) and F1
// (off-diagonal Fock block) may be null (read as 0).
cudaError_t launch_active(dsrg_plan* p, const double* B, const double* eps, const double* G,
                          const double* L, const double* L3, const double* F1, double s,
                          bool ints_ready);
cudaError_t launch_gram_aavv_fp64(dsrg_plan* p, const double* B);
cudaError_t launch_final_reduce(dsrg_plan* p, double* out);
cudaError_t launch_pair_energies(dsrg_plan* p, double* pairs);

// Sizes of the per-launch grids, used to lay out partial segments at plan time.
int ccvv_fp64_blocks(const dsrg_plan* p);
int cavv_fp64_blocks(const dsrg_plan* p);
int ccav_fp64_blocks(const dsrg_plan* p);
// Active block: fills the segment list (one per term kernel) and returns the partial count.
int active_plan(dsrg_plan* p, int first_partial);
bool active_alloc(dsrg_plan* p);

// Tensor-core split path (tc_split.cu).
bool split_supported(const dsrg_plan* p, std::string* why);
bool split_alloc(dsrg_plan* p);
void split_free(dsrg_plan* p);
int split_ccvv_blocks(const dsrg_plan* p);
cudaError_t launch_split_ccvv(dsrg_plan* p, const double* B, const double* eps, double s);
int split_qpad(const dsrg_plan* p);
const CUtensorMap* split_map(const dsrg_plan* p, bool hi);

// Plan construction and the energy pipeline (api.cu), reused by batches.
struct SplitShare {
  void* hi;
  void* lo;
  int Qld;
  long long row_base;
  float* y;  // GEMM output of tc_rest.cu shared by the molecules (NULL: the plan owns one)
};
dsrg_status_t create_plan(dsrg_plan_t** out, const dsrg_sizes_t* sz, dsrg_precision_t prec,
                          void* cuda_stream, uint32_t flags, const SplitShare* share);
dsrg_status_t run_rest(dsrg_plan* p, const double* B, const double* eps, const double* G,
                       const double* L, const double* L3, const double* F1, double s, double* out);
dsrg_status_t run_blocks(dsrg_plan* p, const double* B, const double* eps, const double* G,
                         const double* L, const double* L3, const double* F1, double s);
dsrg_status_t run_reduce(dsrg_plan* p, double* out);

// Split planes shared by several molecules (tc_split.cu).
bool split_alloc_at(dsrg_plan* p, void* hi, void* lo, int Qld, long long row_base,
                    const CUtensorMap* shared_hi, const CUtensorMap* shared_lo);
// Tensor map of a plane buffer [rows][Qld]: boxes of kb_bytes of K by box_rows
// rows, with the swizzle of the same span (32 or 64 bytes).
bool split_make_map(CUtensorMap* m, void* ptr, bool bf16, long long rows, int Qld, int kb_bytes,
                    int box_rows);
// Maps of the CCVV kernel over one pair of planes: 128-row boxes, and 64-row
// boxes for the B operand of a last virtual tile of at most 64 columns.
struct CcvvMaps {
  CUtensorMap hi, lo, hi64, lo64;
};
bool split_make_ccvv_maps(CcvvMaps* m, void* hi, void* lo, bool bf16, long long rows, int Qld);
int split_plane_rows(const Sizes& z);
int split_plane_qpad(const Sizes& z);
int split_kb_elems(bool bf16);
size_t split_mol_desc_bytes();
void split_fill_mol_desc(const dsrg_plan* p, long long row0, void* out);
cudaError_t split_stage(dsrg_plan* p, const double* B, const double* eps, double s);
// one bounded wait that runs out (about 2 s) and records DSRG_ERR_TIMEOUT's status word
cudaError_t launch_wait_selftest(dsrg_plan* p);
cudaError_t split_stage_rows(dsrg_plan* p, const double* B, int h0, int h1);
cudaError_t split_stage_tables(dsrg_plan* p, const double* eps, double s);
// host-buffer pipeline: CCVV items grouped by the core row j of their pair
bool split_alloc_groups(dsrg_plan* p, const std::vector<int>& bounds);
int split_n_groups(const dsrg_plan* p);
void split_group_rows(const dsrg_plan* p, int g, int* h0, int* h1);
cudaError_t split_launch_group(dsrg_plan* p, int g);
cudaError_t split_set_inputs(dsrg_plan* p, void* d_mols, int first, int n,
                             const double* const* eps, const double* s);
// `code`: the schedule code of the items (its prefetch and shape fields are used)
cudaError_t split_launch_ccvv(dsrg_plan* p, const CcvvMaps& maps, const void* d_mols,
                              const int4* d_items, const int* d_begin, int grid, bool bf16,
                              int code);
// items of pairs whose index is not = rank (mod world) are left out; `code` is a
// schedule code (its order and column-halves fields are used)
void split_item_list(const Sizes& z, int mol, int kblocks, std::vector<int4>& items,
                     std::vector<double>& cost, int code, int rank = 0, int world = 1);
// the shard of core pair index k (pairs i <= j in row-major order)
__host__ __device__ inline bool pair_in_shard(int k, int rank, int world) {
  return world <= 1 || k % world == rank;
}
extern const int SPLIT_ORDERS[];
extern const int N_SPLIT_ORDERS;
// Schedule code: item order (bits 0-15), L2 prefetch distance in K stages
// (bits 16-23, at most 64), every virtual tile split into column halves (bit 24).
bool split_code_valid(long long code);
int split_code_prefetch(int code);
bool split_code_halves(int code);
cudaError_t split_set_order(dsrg_plan* p, int order);
int split_order(const dsrg_plan* p);
cudaError_t split_time_ccvv(dsrg_plan* p, int reps, float* ms);
cudaError_t split_prepare_single(dsrg_plan* p, const double* eps, double s);
void split_schedule(const std::vector<int4>& items, const std::vector<double>& cost, int ncta,
                    std::vector<int4>& out, std::vector<int>& begin);

// Generic GEMM with a composite K index (grad.cu):
//   C[i*ci + j*cj] (+)= alpha * sum_{l1<L1, l2<L2} A[i*ai + l1*a1 + l2*a2] * Bm[l1*b1 + l2*b2 + j*bj]
// for nb problems whose A, Bm, C start sa, sb, sc elements apart.
struct GemmArgs {
  int M, N, L1, L2;
  const double* A;
  long long ai, a1, a2;
  const double* Bm;
  long long b1, b2, bj;
  double* C;
  long long ci, cj;
  double alpha;
  int accumulate;
  int nb;                // independent problems in one launch (blockIdx.z);
  long long sa, sb, sc;  // their offsets of A, Bm, C
  // FP32 copies of A and Bm (same element offsets) for the FP32 GEMM, or null
  const float* A32;
  const float* B32;
};
GemmArgs mk(int M, int N, int L1, int L2, const double* A, long long ai, long long a1, long long a2,
            const double* Bm, long long b1, long long b2, long long bj, double* C, long long ci,
            long long cj, double alpha);
GemmArgs batched(GemmArgs g, int nb, long long sa, long long sb, long long sc);
// FP64 (64 x 64 tiles, FP64 FMA) on stream st; accumulate = 1 adds to C.
cudaError_t launch_gemm_fp64(cudaStream_t st, const GemmArgs& g);

// Persisted autotuner choices (tune_cache.cu): a flat JSON object in the file
// named by DSRG_AUTOTUNE_CACHE. get: 1 found, 0 absent, -1 malformed file.
int tune_cache_get(const char* path, const char* key, long long* value);
bool tune_cache_put(const char* path, const char* key, long long value);
const char* tune_cache_path();  // NULL: no cache
std::string tune_gpu_name(int device);
std::string tune_size_class(const Sizes& z, int kblocks, int world);

// Gradient (grad.cu).
bool grad_alloc(dsrg_plan* p);
void grad_free(dsrg_plan* p);
cudaError_t launch_grad(dsrg_plan* p, const double* B, const double* eps, const double* G,
                        const double* L, const double* L3, const double* F1, double s, double* dB,
                        double* deps, double* ds);

// Tensor-core assembly of dE/dB for split plans (tc_adjoint.cu): S is the
// symmetric matrix of the adjoints of every integral (r|c) over the plane rows;
// dB = S . B^T. tc_adj_ccvv forms its core x core block (and adds to deps, ds),
// tc_adj_rest the rest from the adjoints dX, dZ, dM, dK1, dK2, dK3,
// tc_adj_assemble writes every element of dB.
bool tc_adj_alloc(dsrg_plan* p);
void tc_adj_free(dsrg_plan* p);
cudaError_t tc_adj_clear(dsrg_plan* p);
cudaError_t tc_adj_ccvv(dsrg_plan* p, const double* B, const double* eps, double s, double* deps,
                        double* ds);
cudaError_t tc_adj_rest(dsrg_plan* p, const double* dX, const double* dZ, const double* dM,
                        const double* dK1, const double* dK2, const double* dK3);
cudaError_t tc_adj_assemble(dsrg_plan* p, const double* B, double* dB);
// The CCVV kernel's adjoint epilogue (tc_split.cu), TF32x3 recompute.
bool split_adj_alloc(dsrg_plan* p);
cudaError_t split_launch_ccvv_adjoint(dsrg_plan* p, const double* B, const double* eps, double s,
                                      uint16_t* s_hi, uint16_t* s_lo, long long lds, double* deps,
                                      double* ds);

// Split-path CAVV, CCAV and active-block integrals (tc_rest.cu); needs the
// planes staged by the CCVV launch of the same call.
int rest_xrows(const Sizes& z);
size_t rest_y_bytes(const Sizes& z);
bool rest_supported(const Sizes& z);
int rest_cavv_blocks(const dsrg_plan* p);
int rest_ccav_blocks(const dsrg_plan* p);
bool rest_alloc(dsrg_plan* p, float* shared_y);
void rest_free(dsrg_plan* p);
cudaError_t launch_split_rest(dsrg_plan* p, const double* B, const double* eps, const double* G,
                              double s);
void* split_plane_ptr(const dsrg_plan* p, bool hi);
const float* split_tail_ptr(const dsrg_plan* p);  // [plane rows + 256][32] fl32(B), Q < 32
size_t split_tail_bytes(const Sizes& z);
// Factor tables of exp(-s D^2) for the active pairs and the pair-independent
// table, formed by launch_split_rest of the same call.
__global__ void abs_max_kernel(const double* __restrict__ x, int n, double* __restrict__ out);
double* rest_take_tau1(dsrg_plan* p);
void rest_act_tables(const dsrg_plan* p, const double** alpha, const double** pinfo,
                     const double** tau, int* ld);
int split_qld(const dsrg_plan* p);
// Adjoint of F2 from the energy call's GEMM output and factor tables (split
// plans with the tensor-core rest): dX [nC][nA][nV][nV], adds to deps, ds.
cudaError_t launch_split_cavv_adjoint(dsrg_plan* p, const double* eps, const double* G, double s,
                                      double* dX, double* deps, double* ds);

}  // namespace dsrg

#define DSRG_LAUNCH_CHECK(p)                 \
  do {                                       \
    (p)->launches++;                         \
    cudaError_t e_ = cudaGetLastError();     \
    if (e_ != cudaSuccess) return e_;        \
  } while (0)
