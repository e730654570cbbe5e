// Batched energies of many molecules of uneven size.
//
// One plan per molecule provides the workspace of its blocks. In the split
// precision modes all molecules' hi/lo planes live in one shared buffer
// (molecule m's rows start at row_base[m], common row pitch = the largest
// padded naux), so a single persistent tcgen05 launch covers the CCVV work of
// every molecule: its work list holds (molecule, pair, tile pair) items, dealt
// to the CTAs by the cost-balancing scheduler of tc_split.cu. The whole call
// (staging, the batched CCVV launch, every molecule's remaining blocks and
// reductions) is captured once into a CUDA graph and replayed while the input
// pointers and flow parameters stay the same. After the batched CCVV launch the
// molecules' other blocks are independent of each other: the graph forks them
// into up to BATCH_MAX_BRANCHES concurrent branches (molecule m on branch
// m mod K), so that the small per-molecule kernels fill the GPU together; each
// branch has its own GEMM output buffer.
#include <cmath>
#include <cstring>
#include <new>
#include <string>

#include "internal.cuh"

constexpr int BATCH_MAX_BRANCHES = 8;

struct dsrg_batch {
  int nmol = 0;
  int branches = 1;      // concurrent branches of the per-molecule blocks (1, 2, 4 or 8)
  int max_branches = 1;  // branches the GEMM output buffers allow (a power of 2)
  cudaStream_t side[BATCH_MAX_BRANCHES] = {};
  cudaEvent_t ev_fork = nullptr;
  cudaEvent_t ev_ccvv = nullptr;  // the CCVV work of every molecule is done
  cudaEvent_t ev_staged[BATCH_MAX_BRANCHES] = {};  // a branch's molecules staged
  cudaEvent_t ev_join[BATCH_MAX_BRANCHES] = {};
  dsrg_precision_t prec = DSRG_PREC_FP64;
  cudaStream_t user_stream = nullptr;
  cudaStream_t cap_stream = nullptr;
  std::vector<dsrg_plan*> plans;
  std::vector<void*> allocs;
  void* hi = nullptr;
  void* lo = nullptr;
  float* ybuf = nullptr;  // GEMM outputs of the CAVV/CCAV/active stage, one per branch
  size_t ybytes = 0;      // bytes of one of them
  dsrg::CcvvMaps maps;
  void* d_mols = nullptr;
  int4* d_items = nullptr;
  int* d_begin = nullptr;
  int grid = 0;
  int order = 0;  // item order of the batched CCVV schedule
  std::string tune_class;  // size class of the batch in the autotuners' cache keys
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::vector<uintptr_t> key;
  std::string last_error;
  int launches = 0;
  size_t ws_bytes = 0;
};

namespace {

bool balloc(dsrg_batch* b, void** p, size_t bytes) {
  *p = nullptr;
  if (cudaMalloc(p, bytes ? bytes : 8) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return false;
  }
  b->allocs.push_back(*p);
  b->ws_bytes += bytes;
  return true;
}

void bfree(dsrg_batch* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  for (dsrg_plan* p : b->plans)
    if (p) dsrg_plan_destroy(p);
  b->plans.clear();
  for (void* a : b->allocs) cudaFree(a);
  b->allocs.clear();
  if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
  b->cap_stream = nullptr;
  for (int k = 0; k < BATCH_MAX_BRANCHES; ++k) {
    if (b->side[k]) cudaStreamDestroy(b->side[k]);
    if (b->ev_join[k]) cudaEventDestroy(b->ev_join[k]);
    if (b->ev_staged[k]) cudaEventDestroy(b->ev_staged[k]);
    b->side[k] = nullptr;
    b->ev_join[k] = nullptr;
    b->ev_staged[k] = nullptr;
  }
  if (b->ev_fork) cudaEventDestroy(b->ev_fork);
  b->ev_fork = nullptr;
  if (b->ev_ccvv) cudaEventDestroy(b->ev_ccvv);
  b->ev_ccvv = nullptr;
}

dsrg_status_t bfail(dsrg_batch* b, dsrg_status_t st, const std::string& m) {
  b->last_error = m;
  return st;
}

}  // namespace

extern "C" {

dsrg_status_t dsrg_batch_plan(dsrg_batch_t** out, int32_t nmol, const dsrg_sizes_t* sizes,
                              dsrg_precision_t prec, void* cuda_stream, uint32_t flags) {
  if (!out) return DSRG_ERR_INVALID_ARG;
  *out = nullptr;
  if (nmol < 1 || !sizes) return DSRG_ERR_INVALID_ARG;
  if (prec != DSRG_PREC_FP64 && prec != DSRG_PREC_TF32X3 && prec != DSRG_PREC_BF16X3)
    return DSRG_ERR_INVALID_ARG;
  dsrg_batch* b = new (std::nothrow) dsrg_batch();
  if (!b) return DSRG_ERR_OOM;
  b->nmol = nmol;
  b->prec = prec;
  b->user_stream = (cudaStream_t)cuda_stream;
  if (cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    delete b;
    return DSRG_ERR_CUDA;
  }
  b->max_branches = 1;
  while (b->max_branches * 2 <= BATCH_MAX_BRANCHES && b->max_branches * 2 <= nmol) b->max_branches *= 2;
  b->branches = b->max_branches;
  bool streams_ok = cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventCreateWithFlags(&b->ev_ccvv, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; streams_ok && k < b->max_branches; ++k)
    streams_ok = cudaStreamCreateWithFlags(&b->side[k], cudaStreamNonBlocking) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_join[k], cudaEventDisableTiming) == cudaSuccess &&
                 cudaEventCreateWithFlags(&b->ev_staged[k], cudaEventDisableTiming) == cudaSuccess;
  if (!streams_ok) {
    bfree(b);
    delete b;
    return DSRG_ERR_CUDA;
  }
  const bool split = prec != DSRG_PREC_FP64;
  const bool bf16 = prec == DSRG_PREC_BF16X3;
  std::vector<long long> row_base(nmol, 0);
  long long rows = 0;
  int Qld = 64;
  for (int m = 0; m < nmol; ++m) {
    const dsrg_sizes_t& s = sizes[m];
    if (s.ncore < 1 || s.nvirt < 1 || s.naux < 1 || s.nactive < 0 || s.nactive > dsrg::NA_MAX) {
      bfree(b);
      delete b;
      return DSRG_ERR_INVALID_ARG;
    }
    dsrg::Sizes z{s.ncore, s.nactive, s.nvirt, s.naux, s.ncore + s.nactive, s.nactive + s.nvirt,
                  s.ncore + s.nactive + s.nvirt};
    row_base[m] = rows;
    rows += dsrg::split_plane_rows(z);
    const int qp = dsrg::split_plane_qpad(z);
    Qld = qp > Qld ? qp : Qld;
  }
  if (split && rows >= (1ll << 31)) {
    bfree(b);
    delete b;
    return DSRG_ERR_UNSUPPORTED;
  }
  const int elt = bf16 ? 2 : 4;
  if (split) {
    // one GEMM output buffer per branch: molecule m uses buffer m mod max_branches,
    // and the molecules of one branch run one after another
    size_t ybytes = 0;
    for (int m = 0; m < nmol; ++m) {
      const dsrg_sizes_t& s = sizes[m];
      dsrg::Sizes z{s.ncore, s.nactive, s.nvirt, s.naux, s.ncore + s.nactive, s.nactive + s.nvirt,
                    s.ncore + s.nactive + s.nvirt};
      const size_t yb = dsrg::rest_supported(z) ? dsrg::rest_y_bytes(z) : 0;
      ybytes = yb > ybytes ? yb : ybytes;
    }
    ybytes = (ybytes + 255) / 256 * 256;
    if (ybytes > 0 && !balloc(b, (void**)&b->ybuf, ybytes * b->max_branches)) {
      bfree(b);
      delete b;
      return DSRG_ERR_OOM;
    }
    b->ybytes = ybytes;
    const size_t plane = (size_t)rows * Qld * elt;
    if (!balloc(b, &b->hi, plane) || !balloc(b, &b->lo, plane)) {
      bfree(b);
      delete b;
      return DSRG_ERR_OOM;
    }
    if (cudaMemset(b->hi, 0, plane) != cudaSuccess || cudaMemset(b->lo, 0, plane) != cudaSuccess ||
        !dsrg::split_make_ccvv_maps(&b->maps, b->hi, b->lo, bf16, rows, Qld)) {
      bfree(b);
      delete b;
      return DSRG_ERR_CUDA;
    }
  }
  b->plans.assign(nmol, nullptr);
  for (int m = 0; m < nmol; ++m) {
    dsrg::SplitShare sh;
    sh.hi = split ? (char*)b->hi + (size_t)row_base[m] * Qld * elt : nullptr;
    sh.lo = split ? (char*)b->lo + (size_t)row_base[m] * Qld * elt : nullptr;
    sh.Qld = Qld;
    sh.row_base = row_base[m];
    sh.y = b->ybuf ? b->ybuf + (m % b->max_branches) * (b->ybytes / sizeof(float)) : nullptr;
    dsrg_status_t st =
        dsrg::create_plan(&b->plans[m], &sizes[m], prec, b->cap_stream, flags, split ? &sh : nullptr);
    if (st != DSRG_OK) {
      bfree(b);
      delete b;
      return st;
    }
    b->ws_bytes += dsrg_plan_workspace_bytes(b->plans[m]);
  }
  if (split) {
    const size_t mdb = dsrg::split_mol_desc_bytes();
    std::vector<char> mols(mdb * nmol);
    std::vector<int4> items, sched;
    std::vector<double> cost;
    std::vector<int> begin;
    for (int m = 0; m < nmol; ++m) {
      dsrg::split_fill_mol_desc(b->plans[m], row_base[m], mols.data() + m * mdb);
      const int kblocks = dsrg::split_plane_qpad(b->plans[m]->z) / dsrg::split_kb_elems(bf16);
      dsrg::split_item_list(b->plans[m]->z, m, kblocks, items, cost, 0);
    }
    int nsm = 148, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    b->grid = (int)items.size() < nsm ? (int)items.size() : nsm;
    b->tune_class = "n" + std::to_string(nmol) + "-i" + std::to_string((items.size() + 255) / 256 * 256) +
                    "-q" + std::to_string(Qld);
    dsrg::split_schedule(items, cost, b->grid, sched, begin);
    // the item array is sized for the larger list of the column-halves shape
    size_t max_items = 0;
    {
      std::vector<int4> it2;
      std::vector<double> c2;
      for (int m = 0; m < nmol; ++m) {
        const int kblocks = dsrg::split_plane_qpad(b->plans[m]->z) / dsrg::split_kb_elems(bf16);
        dsrg::split_item_list(b->plans[m]->z, m, kblocks, it2, c2, 1 << 24);
      }
      max_items = it2.size();
    }
    if (!balloc(b, &b->d_mols, mols.size()) ||
        !balloc(b, (void**)&b->d_items, max_items * sizeof(int4)) ||
        !balloc(b, (void**)&b->d_begin, begin.size() * sizeof(int)) ||
        cudaMemcpy(b->d_mols, mols.data(), mols.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(b->d_items, sched.data(), sched.size() * sizeof(int4), cudaMemcpyHostToDevice) !=
            cudaSuccess ||
        cudaMemcpy(b->d_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice) !=
            cudaSuccess) {
      bfree(b);
      delete b;
      return DSRG_ERR_OOM;
    }
  }
  *out = b;
  return DSRG_OK;
}

}  // extern "C"

namespace {
// Key of an autotuner choice for this batch in the persisted cache.
std::string batch_key(const dsrg_batch* b, const char* what) {
  int dev = 0;
  cudaGetDevice(&dev);
  const char* prec = b->prec == DSRG_PREC_BF16X3 ? "bf16x3" : (b->prec == DSRG_PREC_TF32X3 ? "tf32x3" : "fp64");
  std::string cls = b->tune_class;
  if (cls.empty()) cls = "n" + std::to_string(b->nmol);
  return std::string(what) + "|" + dsrg::tune_gpu_name(dev) + "|" + prec + "|" + cls;
}

// Rebuild the batched CCVV schedule for item order `order` (same item count).
cudaError_t batch_set_order(dsrg_batch* b, int order) {
  const bool bf16 = b->prec == DSRG_PREC_BF16X3;
  std::vector<int4> items, sched;
  std::vector<double> cost;
  std::vector<int> begin;
  for (int m = 0; m < b->nmol; ++m) {
    const int kblocks = dsrg::split_plane_qpad(b->plans[m]->z) / dsrg::split_kb_elems(bf16);
    dsrg::split_item_list(b->plans[m]->z, m, kblocks, items, cost, order);
  }
  dsrg::split_schedule(items, cost, b->grid, sched, begin);
  cudaError_t e = cudaMemcpy(b->d_items, sched.data(), sched.size() * sizeof(int4), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_begin, begin.data(), begin.size() * sizeof(int), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) b->order = order;
  return e;
}
}  // namespace

extern "C" {

dsrg_status_t dsrg_batch_autotune(dsrg_batch_t* b, const double* const* B, const double* const* eps,
                                  const double* s, int32_t reps, int32_t* chosen) {
  if (!b || !B || !eps || !s || reps < 1) return DSRG_ERR_INVALID_ARG;
  if (chosen) *chosen = -1;
  if (b->prec == DSRG_PREC_FP64) return DSRG_OK;
  const int n = b->nmol;
  for (int m = 0; m < n; ++m) {
    if (!B[m] || !eps[m]) return bfail(b, DSRG_ERR_INVALID_ARG, "B and eps must not be NULL");
    if (std::isnan(s[m]) || std::isinf(s[m]) || s[m] < 0.0)
      return bfail(b, DSRG_ERR_INVALID_ARG, "bad s");
  }
  const char* cache = dsrg::tune_cache_path();
  const std::string key = cache ? batch_key(b, "batch-ccvv-schedule") : std::string();
  if (cache) {
    long long v = -1;
    if (dsrg::tune_cache_get(cache, key.c_str(), &v) == 1 && dsrg::split_code_valid(v)) {
      if (b->user_stream) cudaStreamSynchronize(b->user_stream);
      cudaError_t ec = batch_set_order(b, (int)v);
      if (ec != cudaSuccess) return bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(ec));
      if (chosen) *chosen = (int32_t)v;
      return DSRG_OK;
    }
  }
  cudaStream_t st = b->user_stream;
  dsrg_plan* p0 = b->plans[0];
  cudaError_t e = cudaSuccess;
  for (int m = 0; m < n && e == cudaSuccess; ++m) {
    b->plans[m]->stream = st;
    e = dsrg::split_stage(b->plans[m], B[m], eps[m], s[m]);
  }
  if (e == cudaSuccess) e = dsrg::split_set_inputs(p0, b->d_mols, 0, n, eps, s);
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  float best_ms = 0.f;
  int best = 0;
  const bool bf16 = b->prec == DSRG_PREC_BF16X3;
  for (int c = 0; c < dsrg::N_SPLIT_ORDERS && e == cudaSuccess; ++c) {
    e = batch_set_order(b, dsrg::SPLIT_ORDERS[c]);
    // one untimed launch, then `reps` timed ones
    for (int r = 0; e == cudaSuccess && r <= reps; ++r) {
      if (r == 1) e = cudaEventRecord(e0, st);
      if (e == cudaSuccess)
        e = dsrg::split_launch_ccvv(p0, b->maps, b->d_mols, b->d_items, b->d_begin,
                                    b->grid, bf16, b->order);
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && (c == 0 || ms < best_ms)) {
      best_ms = ms;
      best = dsrg::SPLIT_ORDERS[c];
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e == cudaSuccess) e = batch_set_order(b, best);
  if (e != cudaSuccess) return bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
  for (dsrg_plan* p : b->plans) {
    dsrg_status_t stt = dsrg_plan_sync(p);
    if (stt != DSRG_OK) return bfail(b, stt, "a device-side wait ran out");
  }
  // the schedule arrays keep their addresses: a captured graph stays valid
  if (cache) dsrg::tune_cache_put(cache, key.c_str(), best);
  if (chosen) *chosen = best;
  return DSRG_OK;
}

int32_t dsrg_batch_item_order(const dsrg_batch_t* b) {
  return (b && b->prec != DSRG_PREC_FP64) ? b->order : -1;
}

dsrg_status_t dsrg_batch_set_item_order(dsrg_batch_t* b, int32_t order) {
  if (!b || !dsrg::split_code_valid(order)) return DSRG_ERR_INVALID_ARG;
  if (b->prec == DSRG_PREC_FP64) return DSRG_OK;
  if (b->user_stream) cudaStreamSynchronize(b->user_stream);
  cudaError_t e = batch_set_order(b, order);
  return e == cudaSuccess ? DSRG_OK : bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
}

dsrg_status_t dsrg_batch_destroy(dsrg_batch_t* b) {
  if (!b) return DSRG_OK;
  if (b->user_stream) cudaStreamSynchronize(b->user_stream);
  cudaStreamSynchronize(b->cap_stream);
  bfree(b);
  delete b;
  return DSRG_OK;
}

const char* dsrg_batch_last_error(const dsrg_batch_t* b) {
  return b ? b->last_error.c_str() : "no batch";
}

dsrg_status_t dsrg_mrpt2_energy_batched(dsrg_batch_t* b, const double* const* B,
                                        const double* const* eps, const double* const* gamma1,
                                        const double* const* lambda2, const double* s,
                                        double* out_dev) {
  if (!b) return DSRG_ERR_INVALID_ARG;
  if (!B || !eps || !s || !out_dev) return bfail(b, DSRG_ERR_INVALID_ARG, "NULL argument");
  const int n = b->nmol;
  std::vector<uintptr_t> key;
  key.reserve(6 * n + 1);
  for (int m = 0; m < n; ++m) {
    const dsrg_plan* p = b->plans[m];
    const double* g = gamma1 ? gamma1[m] : nullptr;
    const double* l = lambda2 ? lambda2[m] : nullptr;
    if (std::isnan(s[m]) || std::isinf(s[m])) return bfail(b, DSRG_ERR_NONFINITE, "s is not finite");
    if (s[m] < 0.0) return bfail(b, DSRG_ERR_INVALID_ARG, "s must be >= 0");
    if (!B[m] || !eps[m]) return bfail(b, DSRG_ERR_INVALID_ARG, "B and eps must not be NULL");
    if (p->z.nA > 0 && (!g || !l))
      return bfail(b, DSRG_ERR_INVALID_ARG, "gamma1 and lambda2 must not be NULL when nactive > 0");
    if (((uintptr_t)B[m] | (uintptr_t)eps[m] | (uintptr_t)g | (uintptr_t)l) & 7u)
      return bfail(b, DSRG_ERR_INVALID_ARG, "arrays must be 8-byte aligned");
    uint64_t sbits;
    memcpy(&sbits, &s[m], 8);
    key.push_back((uintptr_t)B[m]);
    key.push_back((uintptr_t)eps[m]);
    key.push_back((uintptr_t)g);
    key.push_back((uintptr_t)l);
    key.push_back((uintptr_t)sbits);
  }
  if ((uintptr_t)out_dev & 7u) return bfail(b, DSRG_ERR_INVALID_ARG, "bad out pointer");
  key.push_back((uintptr_t)out_dev);
  cudaError_t e;
  if (!b->exec || key != b->key) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    b->launches = 0;
    e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeRelaxed);
    if (e != cudaSuccess) return bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
    dsrg_status_t st = DSRG_OK;
    const bool split = b->prec != DSRG_PREC_FP64;
    // The work is forked into K branches, molecule m on branch m mod K: each branch
    // stages its molecules (split: planes and pair tables; FP64: the CCVV kernel
    // itself). The batched CCVV launch waits for every branch's staging. CAVV, CCAV
    // and the active block read only the staged planes and write their own
    // partials, so they start beside the CCVV launch; each branch waits for it
    // only before its molecules' final reductions.
    const int K = b->branches;
    if (K > 1) {
      e = cudaEventRecord(b->ev_fork, b->cap_stream);
      for (int k = 0; k < K && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->ev_fork, 0);
      if (e != cudaSuccess) st = DSRG_ERR_CUDA;
    }
    for (int m = 0; m < n && st == DSRG_OK; ++m) {
      dsrg_plan* p = b->plans[m];
      p->stream = K > 1 ? b->side[m % K] : b->cap_stream;
      p->launches = 0;
      e = split ? dsrg::split_stage(p, B[m], eps[m], s[m]) : dsrg::launch_ccvv_fp64(p, B[m], eps[m], s[m]);
      if (e != cudaSuccess) st = DSRG_ERR_CUDA;
    }
    if (st == DSRG_OK && split && K > 1) {
      for (int k = 0; k < K && e == cudaSuccess; ++k) {
        e = cudaEventRecord(b->ev_staged[k], b->side[k]);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(b->cap_stream, b->ev_staged[k], 0);
      }
      if (e != cudaSuccess) st = DSRG_ERR_CUDA;
    }
    if (st == DSRG_OK && split) {
      dsrg_plan* p0 = b->plans[0];
      p0->stream = b->cap_stream;
      e = dsrg::split_set_inputs(p0, b->d_mols, 0, n, eps, s);
      if (e == cudaSuccess)
        e = dsrg::split_launch_ccvv(p0, b->maps, b->d_mols, b->d_items, b->d_begin,
                                    b->grid, b->prec == DSRG_PREC_BF16X3, b->order);
      if (e != cudaSuccess) st = DSRG_ERR_CUDA;
    }
    if (st == DSRG_OK && K > 1 && cudaEventRecord(b->ev_ccvv, b->cap_stream) != cudaSuccess)
      st = DSRG_ERR_CUDA;
    for (int m = 0; m < n && st == DSRG_OK; ++m) {
      dsrg_plan* p = b->plans[m];
      p->stream = K > 1 ? b->side[m % K] : b->cap_stream;
      st = dsrg::run_blocks(p, B[m], eps[m], gamma1 ? gamma1[m] : nullptr,
                            lambda2 ? lambda2[m] : nullptr, nullptr, nullptr, s[m]);
    }
    for (int k = 0; st == DSRG_OK && k < K && K > 1; ++k)
      if (cudaStreamWaitEvent(b->side[k], b->ev_ccvv, 0) != cudaSuccess) st = DSRG_ERR_CUDA;
    for (int m = 0; m < n && st == DSRG_OK; ++m) {
      dsrg_plan* p = b->plans[m];
      p->stream = K > 1 ? b->side[m % K] : b->cap_stream;
      st = dsrg::run_reduce(p, out_dev + 5 * m);
    }
    if (K > 1) {
      // join every branch that was forked, also after a failure, so that the capture ends
      for (int k = 0; k < K; ++k) {
        cudaError_t ej = cudaEventRecord(b->ev_join[k], b->side[k]);
        if (ej == cudaSuccess) ej = cudaStreamWaitEvent(b->cap_stream, b->ev_join[k], 0);
        if (ej != cudaSuccess && st == DSRG_OK) st = DSRG_ERR_CUDA;
      }
    }
    for (int m = 0; m < n; ++m) b->launches += b->plans[m]->launches;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(b->cap_stream, &graph);
    if (st != DSRG_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return bfail(b, st != DSRG_OK ? st : DSRG_ERR_CUDA, "graph capture failed");
    }
    b->graph = graph;
    e = cudaGraphInstantiate(&b->exec, graph, 0);
    if (e != cudaSuccess) {
      b->exec = nullptr;
      return bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
    }
    b->key = key;
  }
  e = cudaGraphLaunch(b->exec, b->user_stream);
  if (e != cudaSuccess) return bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
  return DSRG_OK;
}

int32_t dsrg_batch_launch_count(const dsrg_batch_t* b) { return b ? b->launches : -1; }

int32_t dsrg_batch_branches(const dsrg_batch_t* b) { return b ? b->branches : -1; }

dsrg_status_t dsrg_batch_set_branches(dsrg_batch_t* b, int32_t k) {
  if (!b || (k != 1 && k != 2 && k != 4 && k != 8) || k > b->max_branches) return DSRG_ERR_INVALID_ARG;
  if (k == b->branches) return DSRG_OK;
  if (b->user_stream) cudaStreamSynchronize(b->user_stream);
  // the next call captures a new graph
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
  b->key.clear();
  b->branches = k;
  return DSRG_OK;
}

dsrg_status_t dsrg_batch_autotune_branches(dsrg_batch_t* b, const double* const* B,
                                           const double* const* eps,
                                           const double* const* gamma1,
                                           const double* const* lambda2, const double* s,
                                           double* out_dev, int32_t reps, int32_t* chosen) {
  if (!b || reps < 1) return DSRG_ERR_INVALID_ARG;
  if (chosen) *chosen = -1;
  const char* cache = dsrg::tune_cache_path();
  const std::string key = cache ? batch_key(b, "batch-branches") : std::string();
  if (cache) {
    long long v = -1;
    if (dsrg::tune_cache_get(cache, key.c_str(), &v) == 1 && (v == 1 || v == 2 || v == 4 || v == 8) &&
        v <= b->max_branches) {
      dsrg_status_t rc = dsrg_batch_set_branches(b, (int32_t)v);
      if (rc == DSRG_OK && chosen) *chosen = (int32_t)v;
      return rc;
    }
  }
  cudaStream_t st = b->user_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  if (e != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
  }
  dsrg_status_t rs = DSRG_OK;
  float best_ms = 0.f;
  int best = b->branches;
  bool first = true;
  for (int k = 1; k <= b->max_branches && rs == DSRG_OK; k *= 2) {
    rs = dsrg_batch_set_branches(b, k);
    // the first call captures the graph; then one untimed and `reps` timed replays
    for (int r = 0; rs == DSRG_OK && r <= reps + 1; ++r) {
      if (r == 2 && cudaEventRecord(e0, st) != cudaSuccess) rs = DSRG_ERR_CUDA;
      if (rs == DSRG_OK) rs = dsrg_mrpt2_energy_batched(b, B, eps, gamma1, lambda2, s, out_dev);
    }
    if (rs != DSRG_OK) break;
    float ms = 0.f;
    e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rs = bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
      break;
    }
    if (first || ms < best_ms) {
      best_ms = ms;
      best = k;
    }
    first = false;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != DSRG_OK) return rs;
  rs = dsrg_batch_set_branches(b, best);
  if (rs == DSRG_OK) rs = dsrg_batch_sync(b);
  if (rs == DSRG_OK && cache) dsrg::tune_cache_put(cache, key.c_str(), best);
  if (rs == DSRG_OK && chosen) *chosen = best;
  return rs;
}

dsrg_status_t dsrg_batch_sync(dsrg_batch_t* b) {
  if (!b) return DSRG_ERR_INVALID_ARG;
  cudaError_t e = b->user_stream ? cudaStreamSynchronize(b->user_stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) return bfail(b, DSRG_ERR_CUDA, cudaGetErrorString(e));
  for (dsrg_plan* p : b->plans) {
    dsrg_status_t st = dsrg_plan_sync(p);
    if (st != DSRG_OK) return bfail(b, st, "a device-side wait ran out");
  }
  return DSRG_OK;
}

}  // extern "C"
