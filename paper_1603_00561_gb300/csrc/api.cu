// C ABI of the DSRG-MRPT2 library: plans, argument checks, dispatch.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>

#include "internal.cuh"

namespace dsrg {
bool ccav_supported(const Sizes& z);

// Allocation-failure injection for tests: DSRG_FAIL_ALLOC_AFTER=k makes the
// (k+1)-th device allocation of a plan fail as if the device were full.
static int fail_after() {
  const char* e = std::getenv("DSRG_FAIL_ALLOC_AFTER");
  return e ? std::atoi(e) : -1;
}

bool plan_alloc(dsrg_plan* p, void** ptr, size_t bytes) {
  *ptr = nullptr;
  if (bytes == 0) bytes = 8;
  const int fa = fail_after();
  if (fa >= 0 && (int)p->allocs.size() >= fa) return false;
  if (cudaMalloc(ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    *ptr = nullptr;
    return false;
  }
  p->allocs.push_back(*ptr);
  p->ws_bytes += bytes;
  return true;
}

cudaError_t raise_smem_limit(const void* func, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<const void*, int>, size_t> cur;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  size_t& c = cur[std::make_pair(func, dev)];
  if (bytes <= c) return cudaSuccess;
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) c = bytes;
  return e;
}

static void tile_pairs(int n, int tile, std::vector<int2>& out) {
  const int nt = (n + tile - 1) / tile;
  out.clear();
  for (int a = 0; a < nt; ++a)
    for (int b = a; b < nt; ++b) out.push_back(make_int2(a, b));
}

}  // namespace dsrg

using namespace dsrg;

static dsrg_status_t fail(dsrg_plan* p, dsrg_status_t st, const std::string& msg) {
  if (p) p->last_error = msg;
  return st;
}

static dsrg_status_t cuda_fail(dsrg_plan* p, cudaError_t e, const char* where) {
  return fail(p, DSRG_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

// Row groups of the host-buffer entry's copy/compute pipeline (split plans).
// Group g's copy takes c per core row; its CCVV launch takes q per pair (i <= j)
// with j in the group, plus a fixed o per launch, and starts when both the
// previous launch and its own copy are done. The bounds minimise the finish time
// of the last launch over at most HOST_IO_MAX_GROUPS groups (dynamic program over
// the last row of each group). The rates are rough estimates (host link about
// 200 GB/s, tensor cores about 1 PFLOP/s on the three split products); they only
// place the group bounds, never the result.
constexpr int HOST_IO_MAX_GROUPS = 8;

static std::vector<int> host_io_bounds(const Sizes& z) {
  const int nC = z.nC;
  const double c = (double)z.Q * z.nP * 8.0 / 200e9;
  const double q = 6.0 * z.Q * (double)z.nV * z.nV / 1e15;
  const double o = 120e-6;
  const int G = nC < HOST_IO_MAX_GROUPS ? nC : HOST_IO_MAX_GROUPS;
  const double inf = 1e300;
  // t[g][h]: earliest finish of the launch of group g when it ends at row h
  std::vector<std::vector<double>> t(G + 1, std::vector<double>(nC + 1, inf));
  std::vector<std::vector<int>> from(G + 1, std::vector<int>(nC + 1, -1));
  t[0][0] = 0.0;
  auto pairs = [](int h0, int h1) {  // pairs i <= j with h0 <= j < h1
    return 0.5 * ((double)h1 * (h1 + 1) - (double)h0 * (h0 + 1));
  };
  for (int g = 1; g <= G; ++g)
    for (int h = g; h <= nC; ++h)
      for (int h0 = g - 1; h0 < h; ++h0) {
        if (t[g - 1][h0] >= inf) continue;
        const double start = t[g - 1][h0] > c * h ? t[g - 1][h0] : c * h;
        const double fin = start + q * pairs(h0, h) + o;
        if (fin < t[g][h]) {
          t[g][h] = fin;
          from[g][h] = h0;
        }
      }
  int best = 1;
  for (int g = 2; g <= G; ++g)
    if (t[g][nC] < t[best][nC]) best = g;
  std::vector<int> b(best + 1);
  b[best] = nC;
  for (int g = best; g > 0; --g) b[g - 1] = from[g][b[g]];
  return b;
}

static void free_all(dsrg_plan* p) {
  for (cudaEvent_t ev : p->st_ev) cudaEventDestroy(ev);
  p->st_ev.clear();
  if (p->st_copy) cudaStreamDestroy(p->st_copy);
  p->st_copy = nullptr;
  if (p->split) split_free(p);
  if (p->rest) rest_free(p);
  if (p->grad) grad_free(p);
  for (void* a : p->allocs) cudaFree(a);
  p->allocs.clear();
}

extern "C" {

const char* dsrg_status_string(dsrg_status_t st) {
  switch (st) {
    case DSRG_OK: return "ok";
    case DSRG_ERR_INVALID_ARG: return "invalid argument";
    case DSRG_ERR_CUDA: return "CUDA runtime error";
    case DSRG_ERR_OOM: return "device workspace allocation failed";
    case DSRG_ERR_TIMEOUT: return "a bounded device-side wait ran out";
    case DSRG_ERR_NONFINITE: return "non-finite flow parameter";
    case DSRG_ERR_UNSUPPORTED: return "unsupported size or mode";
  }
  return "unknown status";
}

const char* dsrg_plan_last_error(const dsrg_plan_t* plan) {
  return plan ? plan->last_error.c_str() : "no plan";
}

int32_t dsrg_plan_last_launch_count(const dsrg_plan_t* plan) { return plan ? plan->launches : -1; }

size_t dsrg_plan_workspace_bytes(const dsrg_plan_t* plan) { return plan ? plan->ws_bytes : 0; }

}  // extern "C"

namespace dsrg {
dsrg_status_t create_plan(dsrg_plan_t** out, const dsrg_sizes_t* sz, dsrg_precision_t prec,
                          void* cuda_stream, uint32_t flags, const SplitShare* share) {
  if (!out) return DSRG_ERR_INVALID_ARG;
  *out = nullptr;
  if (!sz) return DSRG_ERR_INVALID_ARG;
  if (sz->ncore < 1 || sz->nvirt < 1 || sz->naux < 1 || sz->nactive < 0)
    return DSRG_ERR_INVALID_ARG;
  if (prec != DSRG_PREC_FP64 && prec != DSRG_PREC_TF32X3 && prec != DSRG_PREC_BF16X3)
    return DSRG_ERR_INVALID_ARG;
  if (sz->nactive > NA_MAX) return DSRG_ERR_UNSUPPORTED;
  // index arithmetic of the kernels uses int for per-space sizes and size_t for B
  if ((long long)sz->ncore + sz->nactive + sz->nvirt > (1 << 20) || sz->naux > (1 << 24))
    return DSRG_ERR_UNSUPPORTED;

  dsrg_plan* p = new (std::nothrow) dsrg_plan();
  if (!p) return DSRG_ERR_OOM;
  Sizes& z = p->z;
  z.nC = sz->ncore;
  z.nA = sz->nactive;
  z.nV = sz->nvirt;
  z.Q = sz->naux;
  z.nH = z.nC + z.nA;
  z.nP = z.nA + z.nV;
  z.n = z.nC + z.nA + z.nV;
  p->prec = prec;
  p->stream = (cudaStream_t)cuda_stream;
  p->flags = flags;
  cudaGetDevice(&p->device);
  if (!ccav_supported(z)) {
    delete p;
    return DSRG_ERR_UNSUPPORTED;
  }
  std::string why;
  if (prec != DSRG_PREC_FP64 && !split_supported(p, &why)) {
    delete p;
    return DSRG_ERR_UNSUPPORTED;
  }

  // work lists
  std::vector<int2> pairs;
  for (int i = 0; i < z.nC; ++i)
    for (int j = i; j < z.nC; ++j) pairs.push_back(make_int2(i, j));
  p->n_pairs = (int)pairs.size();
  std::vector<int2> tp64, tp32;
  tile_pairs(z.nV, p->tile_ccvv, tp64);
  tile_pairs(z.nV, p->tile_cavv, tp32);
  p->n_tp_ccvv = (int)tp64.size();
  p->n_tp_cavv = (int)tp32.size();

  // partial-sum segments
  int np = 0;
  const int nccvv = (prec == DSRG_PREC_FP64) ? ccvv_fp64_blocks(p) : split_ccvv_blocks(p);
  p->segs.push_back(Segment{np, nccvv, BLK_CCVV});
  p->seg_ccvv = 0;
  np += nccvv;
  p->rest_tc = (prec != DSRG_PREC_FP64) && z.nA > 0 && rest_supported(z);
  const int ncavv = p->rest_tc ? rest_cavv_blocks(p) : cavv_fp64_blocks(p);
  p->segs.push_back(Segment{np, ncavv, BLK_CAVV});
  p->seg_cavv = 1;
  np += ncavv;
  const int nccav = p->rest_tc ? rest_ccav_blocks(p) : ccav_fp64_blocks(p);
  p->segs.push_back(Segment{np, nccav, BLK_CCAV});
  p->seg_ccav = 2;
  np += nccav;
  np += active_plan(p, np);
  p->n_partials = np;

  bool ok = true;
  ok = ok && plan_alloc(p, (void**)&p->d_pairs, pairs.size() * sizeof(int2));
  ok = ok && plan_alloc(p, (void**)&p->d_tp_ccvv, tp64.size() * sizeof(int2));
  ok = ok && plan_alloc(p, (void**)&p->d_tp_cavv, tp32.size() * sizeof(int2));
  ok = ok && plan_alloc(p, (void**)&p->d_partials, (size_t)np * sizeof(double));
  ok = ok && plan_alloc(p, (void**)&p->d_segs, p->segs.size() * sizeof(Segment));
  std::vector<int2> chunks;
  for (int g = 0; g < (int)p->segs.size(); ++g)
    for (int c = 0; c * RED_CHUNK < p->segs[g].count; ++c) chunks.push_back(make_int2(g, c));
  p->n_chunks = (int)chunks.size();
  ok = ok && plan_alloc(p, (void**)&p->d_chunks, chunks.size() * sizeof(int2)) &&
       plan_alloc(p, (void**)&p->d_red, chunks.size() * 2 * sizeof(double));
  ok = ok && plan_alloc(p, (void**)&p->d_status, sizeof(int));
  ok = ok && plan_alloc(p, (void**)&p->d_counts, DSRG_NCOUNTERS * sizeof(unsigned long long));
  ok = ok && active_alloc(p);
  if (ok && prec != DSRG_PREC_FP64)
    ok = share ? split_alloc_at(p, share->hi, share->lo, share->Qld, share->row_base, nullptr, nullptr)
               : split_alloc(p);
  if (ok && p->rest_tc) ok = rest_alloc(p, share ? share->y : nullptr);
  if (ok && (flags & DSRG_PLAN_GRAD)) ok = grad_alloc(p);
  if (ok && (flags & DSRG_PLAN_HOST_IO)) {
    const size_t nb = (size_t)z.Q * z.nH * z.nP;
    const size_t ne = (size_t)z.n, ng = (size_t)z.nA * z.nA, nl = ng * ng;
    double* base = nullptr;
    ok = ok && plan_alloc(p, (void**)&base, (nb + ne + ng + nl + 5) * sizeof(double));
    if (ok) {
      p->st_B = base;
      p->st_eps = base + nb;
      p->st_g = p->st_eps + ne;
      p->st_l = p->st_g + ng;
      p->st_out = p->st_l + nl;
    }
    if (ok && p->rest_tc && !share) {
      // pipeline of the host-buffer entry over groups of core rows
      const std::vector<int> bounds = host_io_bounds(z);
      const int ngroups = (int)bounds.size() - 1;
      ok = cudaStreamCreateWithFlags(&p->st_copy, cudaStreamNonBlocking) == cudaSuccess;
      for (int g = 0; ok && g < ngroups + 2; ++g) {
        cudaEvent_t ev = nullptr;
        ok = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) == cudaSuccess;
        if (ok) p->st_ev.push_back(ev);
      }
      ok = ok && split_alloc_groups(p, bounds);
    }
  }
  if (!ok) {
    free_all(p);
    delete p;
    return DSRG_ERR_OOM;
  }
  cudaError_t e = cudaSuccess;
  e = cudaMemcpy(p->d_pairs, pairs.data(), pairs.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_tp_ccvv, tp64.data(), tp64.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_tp_cavv, tp32.data(), tp32.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_segs, p->segs.data(), p->segs.size() * sizeof(Segment),
                   cudaMemcpyHostToDevice);
  if (e == cudaSuccess && !chunks.empty())
    e = cudaMemcpy(p->d_chunks, chunks.data(), chunks.size() * sizeof(int2), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaMemset(p->d_counts, 0, DSRG_NCOUNTERS * sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemset(p->d_partials, 0, (size_t)np * sizeof(double));
  if (e != cudaSuccess) {
    free_all(p);
    delete p;
    return DSRG_ERR_CUDA;
  }
  *out = p;
  return DSRG_OK;
}

}  // namespace dsrg

extern "C" {

dsrg_status_t dsrg_df_plan(dsrg_plan_t** out, const dsrg_sizes_t* sz, dsrg_precision_t prec,
                           void* cuda_stream, uint32_t flags) {
  return create_plan(out, sz, prec, cuda_stream, flags, nullptr);
}

dsrg_status_t dsrg_plan_destroy(dsrg_plan_t* plan) {
  if (!plan) return DSRG_OK;
  cudaStreamSynchronize(plan->stream);
  free_all(plan);
  delete plan;
  return DSRG_OK;
}

dsrg_status_t dsrg_plan_set_stream(dsrg_plan_t* plan, void* cuda_stream) {
  if (!plan) return DSRG_ERR_INVALID_ARG;
  plan->stream = (cudaStream_t)cuda_stream;
  return DSRG_OK;
}

static dsrg_status_t check_common(dsrg_plan* p, const double* B, const double* eps,
                                  const double* g, const double* l, double s, bool need_active) {
  if (!p) return DSRG_ERR_INVALID_ARG;
  if (std::isnan(s) || std::isinf(s)) return fail(p, DSRG_ERR_NONFINITE, "s is not finite");
  if (s < 0.0) return fail(p, DSRG_ERR_INVALID_ARG, "s must be >= 0");
  if (!B || !eps) return fail(p, DSRG_ERR_INVALID_ARG, "B and eps must not be NULL");
  if (need_active && p->z.nA > 0 && (!g || !l))
    return fail(p, DSRG_ERR_INVALID_ARG, "gamma1 and lambda2 must not be NULL when nactive > 0");
  const uintptr_t mis = ((uintptr_t)B | (uintptr_t)eps | (uintptr_t)g | (uintptr_t)l) & 7u;
  if (mis) return fail(p, DSRG_ERR_INVALID_ARG, "arrays must be 8-byte aligned");
  return DSRG_OK;
}

}  // extern "C"

namespace dsrg {
// The blocks besides CCVV: CAVV, CCAV and the active block (they do not read
// the CCVV partials, so they may run beside the CCVV launch).
dsrg_status_t run_blocks(dsrg_plan* p, const double* B, const double* eps, const double* G,
                         const double* L, const double* L3, const double* F1, double s) {
  cudaError_t e;
  // on a shard of rank > 0 another rank's plan computes these blocks; this
  // rank's segments of them stay at the zeros set by dsrg_plan_set_shard
  if (p->shard_rank != 0) return DSRG_OK;
  if (p->rest_tc) {
    // one tensor-core GEMM feeds CAVV, CCAV and the active-block integrals
    if ((e = launch_split_rest(p, B, eps, G, s)) != cudaSuccess) return cuda_fail(p, e, "cavv/ccav");
  } else {
    if ((e = launch_cavv_fp64(p, B, eps, G, s)) != cudaSuccess) return cuda_fail(p, e, "cavv");
    if ((e = launch_ccav_fp64(p, B, eps, G, s)) != cudaSuccess) return cuda_fail(p, e, "ccav");
  }
  if ((e = launch_active(p, B, eps, G, L, L3, F1, s, p->rest_tc)) != cudaSuccess)
    return cuda_fail(p, e, "active");
  return DSRG_OK;
}

// The final reduction of every block's partials into out[5].
dsrg_status_t run_reduce(dsrg_plan* p, double* out) {
  const cudaError_t e = launch_final_reduce(p, out);
  return e == cudaSuccess ? DSRG_OK : cuda_fail(p, e, "reduce");
}

// Everything after the CCVV launch: CAVV, CCAV, active block, final reduction.
dsrg_status_t run_rest(dsrg_plan* p, const double* B, const double* eps, const double* G,
                       const double* L, const double* L3, const double* F1, double s, double* out) {
  const dsrg_status_t st = run_blocks(p, B, eps, G, L, L3, F1, s);
  return st != DSRG_OK ? st : run_reduce(p, out);
}
}  // namespace dsrg

static dsrg_status_t run_energy(dsrg_plan* p, const double* B, const double* eps, const double* G,
                                const double* L, const double* L3, const double* F1, double s,
                                double* out) {
  cudaError_t e;
  if (p->prec == DSRG_PREC_FP64)
    e = launch_ccvv_fp64(p, B, eps, s);
  else
    e = launch_split_ccvv(p, B, eps, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "ccvv");
  return run_rest(p, B, eps, G, L, L3, F1, s, out);
}

extern "C" {

dsrg_status_t dsrg_mrpt2_energy_ext(dsrg_plan_t* p, const double* B, const double* eps,
                                    const double* gamma1, const double* lambda2,
                                    const double* lambda3, const double* f1, double s,
                                    double* out_dev) {
  dsrg_status_t st = check_common(p, B, eps, gamma1, lambda2, s, true);
  if (st != DSRG_OK) return st;
  if (!out_dev || ((uintptr_t)out_dev & 7u)) return fail(p, DSRG_ERR_INVALID_ARG, "bad out pointer");
  if (((uintptr_t)lambda3 | (uintptr_t)f1) & 7u)
    return fail(p, DSRG_ERR_INVALID_ARG, "lambda3 and f1 must be 8-byte aligned");
  if (p->z.nA == 0) lambda3 = nullptr;
  p->launches = 0;
  return run_energy(p, B, eps, gamma1, lambda2, lambda3, f1, s, out_dev);
}

dsrg_status_t dsrg_mrpt2_energy(dsrg_plan_t* p, const double* B, const double* eps,
                                const double* gamma1, const double* lambda2, double s,
                                double* out_dev) {
  return dsrg_mrpt2_energy_ext(p, B, eps, gamma1, lambda2, nullptr, nullptr, s, out_dev);
}

dsrg_status_t dsrg_ccvv_pair_energies(dsrg_plan_t* p, const double* B, const double* eps, double s,
                                      double* pairs_dev) {
  dsrg_status_t st = check_common(p, B, eps, nullptr, nullptr, s, false);
  if (st != DSRG_OK) return st;
  if (!pairs_dev || ((uintptr_t)pairs_dev & 7u))
    return fail(p, DSRG_ERR_INVALID_ARG, "bad pairs pointer");
  p->launches = 0;
  cudaError_t e;
  if (p->prec == DSRG_PREC_FP64)
    e = launch_ccvv_fp64(p, B, eps, s);
  else
    e = launch_split_ccvv(p, B, eps, s);
  if (e != cudaSuccess) return cuda_fail(p, e, "ccvv");
  if ((e = launch_pair_energies(p, pairs_dev)) != cudaSuccess) return cuda_fail(p, e, "pairs");
  return DSRG_OK;
}

dsrg_status_t dsrg_mrpt2_energy_grad_ext(dsrg_plan_t* p, const double* B, const double* eps,
                                         const double* gamma1, const double* lambda2,
                                         const double* lambda3, const double* f1, double s,
                                         double* out_dev, double* dB_dev, double* deps_dev,
                                         double* ds_dev) {
  dsrg_status_t st = check_common(p, B, eps, gamma1, lambda2, s, true);
  if (((uintptr_t)lambda3 | (uintptr_t)f1) & 7u)
    return fail(p, DSRG_ERR_INVALID_ARG, "lambda3 and f1 must be 8-byte aligned");
  if (p && p->z.nA == 0) lambda3 = nullptr;
  if (st != DSRG_OK) return st;
  if (!p->grad) return fail(p, DSRG_ERR_INVALID_ARG, "plan was created without DSRG_PLAN_GRAD");
  if (!out_dev || !dB_dev || !deps_dev || !ds_dev)
    return fail(p, DSRG_ERR_INVALID_ARG, "gradient outputs must not be NULL");
  if (((uintptr_t)out_dev | (uintptr_t)dB_dev | (uintptr_t)deps_dev | (uintptr_t)ds_dev) & 7u)
    return fail(p, DSRG_ERR_INVALID_ARG, "outputs must be 8-byte aligned");
  p->launches = 0;
  st = run_energy(p, B, eps, gamma1, lambda2, lambda3, f1, s, out_dev);
  if (st != DSRG_OK) return st;
  // the adjoint reads the active-block tables the energy call left (split plans:
  // from the tensor-core integrals, whose error is far below the gradient's own)
  cudaError_t e = launch_grad(p, B, eps, gamma1, lambda2, lambda3, f1, s, dB_dev, deps_dev,
                              ds_dev);
  if (e != cudaSuccess) return cuda_fail(p, e, "gradient");
  return DSRG_OK;
}

dsrg_status_t dsrg_mrpt2_energy_grad(dsrg_plan_t* p, const double* B, const double* eps,
                                     const double* gamma1, const double* lambda2, double s,
                                     double* out_dev, double* dB_dev, double* deps_dev,
                                     double* ds_dev) {
  return dsrg_mrpt2_energy_grad_ext(p, B, eps, gamma1, lambda2, nullptr, nullptr, s, out_dev,
                                    dB_dev, deps_dev, ds_dev);
}

dsrg_status_t dsrg_plan_time_ccvv(dsrg_plan_t* p, const double* B, const double* eps, double s,
                                  int32_t reps, float* ms) {
  dsrg_status_t st = check_common(p, B, eps, nullptr, nullptr, s, false);
  if (st != DSRG_OK) return st;
  if (!ms || reps < 1) return fail(p, DSRG_ERR_INVALID_ARG, "ms must not be NULL and reps >= 1");
  if (p->prec == DSRG_PREC_FP64) return fail(p, DSRG_ERR_UNSUPPORTED, "FP64 plans have no split kernel");
  cudaError_t e = split_stage(p, B, eps, s);
  if (e == cudaSuccess) e = split_prepare_single(p, eps, s);
  float warm = 0.f;
  if (e == cudaSuccess) e = split_time_ccvv(p, 1, &warm);
  if (e == cudaSuccess) e = split_time_ccvv(p, reps, ms);
  if (e != cudaSuccess) return cuda_fail(p, e, "ccvv timing");
  return dsrg_plan_sync(p);
}

dsrg_status_t dsrg_plan_autotune(dsrg_plan_t* p, const double* B, const double* eps, double s,
                                 int32_t reps, int32_t* chosen) {
  dsrg_status_t st = check_common(p, B, eps, nullptr, nullptr, s, false);
  if (st != DSRG_OK) return st;
  if (reps < 1) return fail(p, DSRG_ERR_INVALID_ARG, "reps must be >= 1");
  if (chosen) *chosen = -1;
  if (p->prec == DSRG_PREC_FP64) return DSRG_OK;
  // a choice stored for this GPU, precision and size class is applied without timing
  const char* cache = tune_cache_path();
  std::string key;
  if (cache) {
    const int kblocks = (split_qpad(p) - 32) / split_kb_elems(p->prec == DSRG_PREC_BF16X3);
    key = std::string("ccvv-schedule|") + tune_gpu_name(p->device) + "|" +
          (p->prec == DSRG_PREC_BF16X3 ? "bf16x3" : "tf32x3") + "|" +
          tune_size_class(p->z, kblocks, p->shard_world);
    long long v = -1;
    if (tune_cache_get(cache, key.c_str(), &v) == 1 && split_code_valid(v)) {
      cudaError_t ec = split_set_order(p, (int)v);
      if (ec != cudaSuccess) return cuda_fail(p, ec, "autotune (cached)");
      if (chosen) *chosen = (int32_t)v;
      return DSRG_OK;
    }
  }
  cudaError_t e = split_stage(p, B, eps, s);
  if (e == cudaSuccess) e = split_prepare_single(p, eps, s);
  float best_ms = 0.f;
  int best = 0;
  for (int c = 0; c < N_SPLIT_ORDERS && e == cudaSuccess; ++c) {
    float warm = 0.f, ms = 0.f;
    e = split_set_order(p, SPLIT_ORDERS[c]);
    if (e == cudaSuccess) e = split_time_ccvv(p, 1, &warm);
    if (e == cudaSuccess) e = split_time_ccvv(p, reps, &ms);
    if (e == cudaSuccess && (c == 0 || ms < best_ms)) {
      best_ms = ms;
      best = SPLIT_ORDERS[c];
    }
  }
  if (e == cudaSuccess) e = split_set_order(p, best);
  if (e != cudaSuccess) return cuda_fail(p, e, "autotune");
  st = dsrg_plan_sync(p);
  if (st != DSRG_OK) return st;
  if (cache) tune_cache_put(cache, key.c_str(), best);  // best effort: a read-only path is no error
  if (chosen) *chosen = best;
  return DSRG_OK;
}

int32_t dsrg_plan_item_order(const dsrg_plan_t* p) { return p ? split_order(p) : -1; }

dsrg_status_t dsrg_plan_set_item_order(dsrg_plan_t* p, int32_t order) {
  if (!p || !split_code_valid(order)) return DSRG_ERR_INVALID_ARG;
  if (p->prec == DSRG_PREC_FP64) return DSRG_OK;
  cudaError_t e = split_set_order(p, order);
  return e == cudaSuccess ? DSRG_OK : cuda_fail(p, e, "item order");
}

dsrg_status_t dsrg_mrpt2_energy_host(dsrg_plan_t* p, const double* B_host, const double* eps_host,
                                     const double* gamma1_host, const double* lambda2_host,
                                     double s, double* out_host) {
  if (!p) return DSRG_ERR_INVALID_ARG;
  if (!(p->flags & DSRG_PLAN_HOST_IO) || !p->st_B)
    return fail(p, DSRG_ERR_INVALID_ARG, "plan was created without DSRG_PLAN_HOST_IO");
  dsrg_status_t st = check_common(p, B_host, eps_host, gamma1_host, lambda2_host, s, true);
  if (st != DSRG_OK) return st;
  if (!out_host) return fail(p, DSRG_ERR_INVALID_ARG, "out_host must not be NULL");
  const Sizes& z = p->z;
  const size_t nb = (size_t)z.Q * z.nH * z.nP, ng = (size_t)z.nA * z.nA;
  const int G = split_n_groups(p);
  cudaError_t e = cudaMemcpyAsync(p->st_eps, eps_host, (size_t)z.n * 8, cudaMemcpyHostToDevice,
                                  p->stream);
  if (e == cudaSuccess && ng)
    e = cudaMemcpyAsync(p->st_g, gamma1_host, ng * 8, cudaMemcpyHostToDevice, p->stream);
  if (e == cudaSuccess && ng)
    e = cudaMemcpyAsync(p->st_l, lambda2_host, ng * ng * 8, cudaMemcpyHostToDevice, p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "host to device copy");
  p->launches = 0;
  if (G > 0 && p->st_copy) {
    // Split plans: B goes over in groups of core rows on the copy stream, and the
    // CCVV items of a group (pairs i <= j with j in the group) start as soon as
    // its rows are staged, while later groups are still on the way. The partial
    // sums and their reduction are those of dsrg_mrpt2_energy: same result bits.
    const size_t pitch = (size_t)z.nH * z.nP * 8;
    auto copy_rows = [&](int h0, int h1) {
      return cudaMemcpy2DAsync(p->st_B + (size_t)h0 * z.nP, pitch, B_host + (size_t)h0 * z.nP,
                               pitch, (size_t)(h1 - h0) * z.nP * 8, (size_t)z.Q,
                               cudaMemcpyHostToDevice, p->st_copy);
    };
    // the copies must not overwrite st_B while work queued earlier still reads it
    e = cudaEventRecord(p->st_ev[G + 1], p->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->st_copy, p->st_ev[G + 1], 0);
    for (int g = 0; e == cudaSuccess && g < G; ++g) {
      int h0 = 0, h1 = 0;
      split_group_rows(p, g, &h0, &h1);
      e = copy_rows(h0, h1);
      if (e == cudaSuccess) e = cudaEventRecord(p->st_ev[g], p->st_copy);
    }
    if (e == cudaSuccess && z.nH > z.nC) e = copy_rows(z.nC, z.nH);
    if (e == cudaSuccess) e = cudaEventRecord(p->st_ev[G], p->st_copy);
    if (e != cudaSuccess) return cuda_fail(p, e, "host to device copy");
    if ((e = split_stage_tables(p, p->st_eps, s)) == cudaSuccess)
      e = split_prepare_single(p, p->st_eps, s);
    for (int g = 0; e == cudaSuccess && g < G; ++g) {
      int h0 = 0, h1 = 0;
      split_group_rows(p, g, &h0, &h1);
      e = cudaStreamWaitEvent(p->stream, p->st_ev[g], 0);
      if (e == cudaSuccess) e = split_stage_rows(p, p->st_B, h0, h1);
      if (e == cudaSuccess) e = split_launch_group(p, g);
    }
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->stream, p->st_ev[G], 0);
    if (e == cudaSuccess) e = split_stage_rows(p, p->st_B, z.nC, z.nH);
    if (e != cudaSuccess) return cuda_fail(p, e, "ccvv");
    st = run_rest(p, p->st_B, p->st_eps, p->st_g, p->st_l, nullptr, nullptr, s, p->st_out);
  } else {
    e = cudaMemcpyAsync(p->st_B, B_host, nb * 8, cudaMemcpyHostToDevice, p->stream);
    if (e != cudaSuccess) return cuda_fail(p, e, "host to device copy");
    st = run_energy(p, p->st_B, p->st_eps, p->st_g, p->st_l, nullptr, nullptr, s, p->st_out);
  }
  if (st != DSRG_OK) return st;
  e = cudaMemcpyAsync(out_host, p->st_out, 5 * 8, cudaMemcpyDeviceToHost, p->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "device to host copy");
  return DSRG_OK;
}

dsrg_status_t dsrg_plan_selftest_wait_timeout(dsrg_plan_t* p) {
  if (!p) return DSRG_ERR_INVALID_ARG;
  p->launches = 0;
  cudaError_t e = launch_wait_selftest(p);
  if (e != cudaSuccess) return cuda_fail(p, e, "wait self-test");
  return DSRG_OK;
}

int32_t dsrg_shard_pairs(int32_t ncore, int32_t rank, int32_t world, int32_t* pairs_out) {
  if (ncore < 1 || world < 1 || rank < 0 || rank >= world) return -1;
  int32_t n = 0, k = 0;
  for (int i = 0; i < ncore; ++i)
    for (int j = i; j < ncore; ++j, ++k)
      if (pair_in_shard(k, rank, world)) {
        if (pairs_out) {
          pairs_out[2 * n] = i;
          pairs_out[2 * n + 1] = j;
        }
        ++n;
      }
  return n;
}

dsrg_status_t dsrg_plan_set_shard(dsrg_plan_t* p, int32_t rank, int32_t world) {
  if (!p || world < 1 || rank < 0 || rank >= world) return DSRG_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "set shard");
  p->shard_rank = rank;
  p->shard_world = world;
  // every partial slot starts at zero: the slots of another rank's work are
  // never written again
  e = cudaMemset(p->d_partials, 0, (size_t)p->n_partials * sizeof(double));
  if (e == cudaSuccess && p->split) e = split_set_order(p, split_order(p));
  // the gradient's S: positions of another rank's pairs are never written again
  if (e == cudaSuccess) e = tc_adj_clear(p);
  if (e == cudaSuccess) e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "set shard");
  return DSRG_OK;
}

dsrg_status_t dsrg_plan_branch_counts(dsrg_plan_t* p, uint64_t* counts, int32_t reset) {
  if (!p || !counts) return DSRG_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  unsigned long long c[DSRG_NCOUNTERS] = {};
  if (e == cudaSuccess)
    e = cudaMemcpy(c, p->d_counts, sizeof(c), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(p->d_counts, 0, sizeof(c));
  if (e != cudaSuccess) return cuda_fail(p, e, "branch counts");
  for (int k = 0; k < DSRG_NCOUNTERS; ++k) counts[k] = (uint64_t)c[k];
  return DSRG_OK;
}

dsrg_status_t dsrg_plan_sync(dsrg_plan_t* p) {
  if (!p) return DSRG_ERR_INVALID_ARG;
  cudaError_t e = cudaStreamSynchronize(p->stream);
  if (e != cudaSuccess) return cuda_fail(p, e, "sync");
  int st = 0;
  e = cudaMemcpy(&st, p->d_status, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(p, e, "status read");
  if (st != 0) {
    cudaMemset(p->d_status, 0, sizeof(int));
    return fail(p, DSRG_ERR_TIMEOUT, "a device-side wait ran out");
  }
  return DSRG_OK;
}

}  // extern "C"
