// E_CCVV (diagram F1) in FP64 without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a memory pool or
// allocator it does not own, host frameworks that forbid allocation on the hot
// path (allocation would synchronise the device or break a stream capture taken
// elsewhere), and embedded/plug-in hosts that hand out only their own buffers.
// This entry point serves them: the caller passes inputs and the output, and
// the work lists and per-item partial sums live in one file-scope device array
// that the library holds for every GPU it is loaded on, until the process
// exits. The arithmetic is that of the FP64 CCVV kernel (fp64_pairs.cu); only
// where its scratch lives differs.
#include <cudaTypedefs.h>

#include <mutex>

#include "internal.cuh"

namespace dsrg {
// The FP64 CCVV kernel of fp64_pairs.cu (pair/tile lists and partials are arguments).
__global__ void ccvv_fp64_kernel(const double* __restrict__ B, const double* __restrict__ eps,
                                 double s, Sizes z, const int2* __restrict__ pairs,
                                 const int2* __restrict__ tps, int n_tp,
                                 double* __restrict__ partials, int shard_rank, int shard_world);
}  // namespace dsrg

namespace {

// Scratch layout (in doubles): partials [NA_ITEMS] | pair list [NA_PAIRS] | tile-pair list [NA_TPS]
// (an int2 fits in one double slot). Total 147456 doubles = 1.125 MiB per GPU.
constexpr int NA_ITEMS = 1 << 17;   // core pairs x virtual tile pairs
constexpr int NA_PAIRS = 8192;      // core pairs i <= j   (nC <= 127)
constexpr int NA_TPS = 8192;        // 64-wide virtual tile pairs A <= B (nV <= 8128)
constexpr int NA_TILE = 64;
constexpr size_t NA_DOUBLES = (size_t)NA_ITEMS + NA_PAIRS + NA_TPS;

static __device__ __align__(256) double g_noalloc_scratch[NA_DOUBLES];

constexpr int MAX_DEV = 64;
std::mutex g_mu;
// Per device: the address of the scratch array in the context it was looked up
// in, keyed by that context's unique id. A context that is destroyed and made
// again (cudaDeviceReset, a re-created primary context) loads the module anew
// at a new address and gets a new id, so the address is looked up again.
struct ScratchSlot {
  unsigned long long ctx_id = 0;
  double* addr = nullptr;
};
ScratchSlot g_slot[MAX_DEV];

PFN_cuCtxGetCurrent_v4000 g_get_ctx = nullptr;
PFN_cuCtxGetId_v12000 g_get_id = nullptr;

bool driver_entry_points() {
  if (g_get_ctx && g_get_id) return true;
  void* f = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f, 4000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return false;
  g_get_ctx = (PFN_cuCtxGetCurrent_v4000)f;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &f, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      q != cudaDriverEntryPointSuccess)
    return false;
  g_get_id = (PFN_cuCtxGetId_v12000)f;
  return true;
}

__global__ void noalloc_lists_kernel(double* scratch, int nC, int nT, int n_pairs, int n_tp) {
  int2* pairs = (int2*)(scratch + NA_ITEMS);
  int2* tps = (int2*)(scratch + NA_ITEMS + NA_PAIRS);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_pairs) {
    // k-th pair (i, j), i <= j, in row-major order of the upper triangle
    int i = 0, r = k;
    while (r >= nC - i) {
      r -= nC - i;
      ++i;
    }
    pairs[k] = make_int2(i, i + r);
  }
  if (k < n_tp) {
    int a = 0, r = k;
    while (r >= nT - a) {
      r -= nT - a;
      ++a;
    }
    tps[k] = make_int2(a, a + r);
  }
}

// Fixed-order compensated sum of the partials into out[0] (one CTA).
__global__ void __launch_bounds__(256) noalloc_reduce_kernel(const double* scratch, int n,
                                                             double* out) {
  __shared__ double sh_s[256], sh_c[256];
  double s = 0.0, c = 0.0;
  for (int k = threadIdx.x; k < n; k += 256) {
    const double x = scratch[k];
    const double t = s + x;
    c += (fabs(s) >= fabs(x)) ? (s - t) + x : (x - t) + s;
    s = t;
  }
  sh_s[threadIdx.x] = s;
  sh_c[threadIdx.x] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    double S = 0.0, C = 0.0;
    for (int k = 0; k < 256; ++k) {
      const double x = sh_s[k];
      const double t = S + x;
      C += (fabs(S) >= fabs(x)) ? (S - t) + x : (x - t) + S;
      S = t;
      C += sh_c[k];
    }
    out[0] = S + C;
  }
}

// Device address of the scratch array in the current device's current context.
// Looked up with cudaGetSymbolAddress the first time a context is seen (this also
// creates the device's primary context if the runtime has not done so yet), then
// taken from the slot while the context id stays the same.
cudaError_t scratch_address(double** ptr) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEV) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!driver_entry_points()) return cudaErrorNotSupported;
  CUcontext ctx = nullptr;
  if (g_get_ctx(&ctx) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  void* p = nullptr;
  if (!ctx) {
    // no context current yet: the symbol lookup makes the primary context current
    if ((e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
    if (g_get_ctx(&ctx) != CUDA_SUCCESS || !ctx) return cudaErrorDeviceUninitialized;
  }
  unsigned long long id = 0;
  if (g_get_id(ctx, &id) != CUDA_SUCCESS) return cudaErrorDeviceUninitialized;
  ScratchSlot& sl = g_slot[dev];
  if (sl.addr && sl.ctx_id == id) {
    *ptr = sl.addr;
    return cudaSuccess;
  }
  if (!p && (e = cudaGetSymbolAddress(&p, g_noalloc_scratch)) != cudaSuccess) return e;
  sl.ctx_id = id;
  sl.addr = (double*)p;
  *ptr = sl.addr;
  return cudaSuccess;
}

}  // namespace

extern "C" dsrg_status_t dsrg_ccvv_energy_noalloc(const dsrg_sizes_t* sz, const double* B,
                                                  const double* eps, double s, double* out_dev,
                                                  void* cuda_stream) {
  if (!sz || !B || !eps || !out_dev) return DSRG_ERR_INVALID_ARG;
  if (sz->ncore < 1 || sz->nvirt < 1 || sz->naux < 1 || sz->nactive < 0) return DSRG_ERR_INVALID_ARG;
  if (s != s || s - s != 0.0) return DSRG_ERR_NONFINITE;
  if (s < 0.0) return DSRG_ERR_INVALID_ARG;
  if (((uintptr_t)B | (uintptr_t)eps | (uintptr_t)out_dev) & 7u) return DSRG_ERR_INVALID_ARG;
  const long long nC = sz->ncore, nT = (sz->nvirt + NA_TILE - 1) / NA_TILE;
  const long long n_pairs = nC * (nC + 1) / 2, n_tp = nT * (nT + 1) / 2;
  // sizes beyond the fixed scratch are rejected (no fallback allocation)
  if (n_pairs > NA_PAIRS || n_tp > NA_TPS || n_pairs * n_tp > NA_ITEMS) return DSRG_ERR_UNSUPPORTED;
  // an error left pending by the caller's earlier work is reported, not consumed:
  // it stays for the caller to read
  if (cudaPeekAtLastError() != cudaSuccess) return DSRG_ERR_CUDA;
  double* scratch = nullptr;
  if (scratch_address(&scratch) != cudaSuccess) return DSRG_ERR_CUDA;
  cudaStream_t st = (cudaStream_t)cuda_stream;
  dsrg::Sizes z;
  z.nC = sz->ncore;
  z.nA = sz->nactive;
  z.nV = sz->nvirt;
  z.Q = sz->naux;
  z.nH = z.nC + z.nA;
  z.nP = z.nA + z.nV;
  z.n = z.nC + z.nA + z.nV;
  const int nl = (int)(n_pairs > n_tp ? n_pairs : n_tp);
  noalloc_lists_kernel<<<(nl + 255) / 256, 256, 0, st>>>(scratch, (int)nC, (int)nT, (int)n_pairs,
                                                        (int)n_tp);
  if (cudaGetLastError() != cudaSuccess) return DSRG_ERR_CUDA;
  const int2* pairs = (const int2*)(scratch + NA_ITEMS);
  const int2* tps = (const int2*)(scratch + NA_ITEMS + NA_PAIRS);
  dsrg::ccvv_fp64_kernel<<<(unsigned)(n_pairs * n_tp), 256, 0, st>>>(B, eps, s, z, pairs, tps,
                                                                     (int)n_tp, scratch, 0, 1);
  if (cudaGetLastError() != cudaSuccess) return DSRG_ERR_CUDA;
  noalloc_reduce_kernel<<<1, 256, 0, st>>>(scratch, (int)(n_pairs * n_tp), out_dev);
  if (cudaGetLastError() != cudaSuccess) return DSRG_ERR_CUDA;
  return DSRG_OK;
}
