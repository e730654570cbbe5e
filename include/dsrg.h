/*
 * dsrg.h -- C ABI of the GB300 (sm_103a) DF/CD DSRG-MRPT2 energy library.
 *
 * The library evaluates the second-order DSRG-MRPT2 energy of Hannon, Li and
 * Evangelista (arXiv:1603.00561) from factorised two-electron integrals:
 *
 *   E2(s) = <[H~(1)(s), T(1)(s)]>                      (Sec. II.B, Eq. (11))
 *
 * with the first-order amplitudes of Eqs. (12)-(13), the modified Fock and
 * integrals of Eqs. (14)-(15), the terms of Table 1 (A-K; J and K need the
 * three-body cumulant, an optional input of dsrg_mrpt2_energy_ext, and are 0
 * without it), and the split of term F into the diagrams F1-F8 of Table 2.
 * The energy is reported per block:
 *
 *   out[0] = E_CCVV   diagram F1, Eq. (23): sum over core pairs (m,n) and
 *                     virtual pairs (e,f) of |v_mn^ef|^2 (1-exp(-2sD^2))/D
 *   out[1] = E_CAVV   diagram F2 (Table 2)
 *   out[2] = E_CCAV   diagram F3 (Table 2)
 *   out[3] = E_active terms A-E, G-K (Table 1) and F4-F8 (Table 2)
 *   out[4] = E_total  the sum of the four blocks
 *
 * Problem statement (Sec. II.A, II.B, II.C):
 *   - orbitals are partitioned into core C (nC), active A (nA) and virtual
 *     V (nV), ordered [core | active | virtual]; holes H = C+A (nH = nC+nA),
 *     particles P = A+V (nP = nA+nV);
 *   - orbitals are semicanonical: eps[p] is the diagonal of the generalized
 *     Fock matrix (Eq. (8)); the off-diagonal block f^(1) is an optional input
 *     of the _ext entry points (0 otherwise);
 *   - two-electron integrals are factorised, (pq|rs) = sum_Q B^Q_pq B^Q_rs
 *     (Eq. (19)); every term reads B only on hole x particle index pairs, so
 *     the caller passes that block;
 *   - the reference is a closed-shell-like (singlet, spin-averaged) CAS
 *     state: gamma1 is the spin-summed active one-particle density matrix G
 *     (per spin G/2), lambda2[u][v][x][y] is the opposite-spin cumulant
 *     lambda_{u alpha, v beta}^{x alpha, y beta}; the same-spin blocks are
 *     L[u,v,x,y] - L[u,v,y,x].
 *
 * Conventions of every entry point:
 *   - array arguments are DEVICE pointers owned by the caller, FP64,
 *     row-major, contiguous; the library never frees them;
 *   - B has layout [naux][nH][nP]: B[(Q*nH + i)*nP + a] = B^Q_{i a}, i a
 *     hole index (0..nC-1 core, nC..nH-1 active), a a particle index
 *     (0..nA-1 active, nA..nP-1 virtual); eps has length n = nC+nA+nV;
 *     gamma1 has nA*nA entries and lambda2 nA^4 (both may be NULL if nA == 0);
 *   - all work is queued on the plan's CUDA stream; energy and gradient calls
 *     do not allocate and do not synchronise (results land in device memory);
 *   - errors are returned as dsrg_status_t, never by abort or exception; a
 *     one-line detail is kept per plan (dsrg_plan_last_error). Conditions
 *     detected on the device (a bounded wait that ran out) are reported by
 *     dsrg_plan_sync.
 */
#ifndef DSRG_H
#define DSRG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  DSRG_OK = 0,
  DSRG_ERR_INVALID_ARG = 1,  /* bad size, NULL pointer, s < 0, misaligned pointer */
  DSRG_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  DSRG_ERR_OOM = 3,          /* workspace allocation failed */
  DSRG_ERR_TIMEOUT = 4,      /* a bounded device-side wait ran out */
  DSRG_ERR_NONFINITE = 5,    /* s is NaN or infinite */
  DSRG_ERR_UNSUPPORTED = 6   /* size or mode outside what this build supports */
} dsrg_status_t;

/* Arithmetic of the pair contractions (the v_mn^ef products over Q of
 * Eq. (19) for diagrams F1 and F2, and the (A,A|V,V) integrals):
 *   DSRG_PREC_FP64    plain FP64 products and sums on CUDA cores;
 *   DSRG_PREC_TF32X3  B = hi + lo split into two TF32 planes, products
 *                     hi*hi + hi*lo + lo*hi on tcgen05 tensor cores with FP32
 *                     accumulation (and lo*lo where both operands are the
 *                     same rows, whose diagonal is a sum of squares); the
 *                     first 32 auxiliary functions, the largest terms, are
 *                     summed on CUDA cores in FP32 from fl32(B), because the
 *                     tensor-core accumulator truncates toward zero;
 *   DSRG_PREC_BF16X3  same with BF16 planes.
 * In every mode the regulator (Delta, exp(-s Delta^2), the denominator), the
 * combination with the exchange integral and every sum of energy
 * contributions are FP64. */
typedef enum {
  DSRG_PREC_FP64 = 0,
  DSRG_PREC_TF32X3 = 1,
  DSRG_PREC_BF16X3 = 2
} dsrg_precision_t;

typedef struct {
  int32_t ncore;    /* nC >= 1 */
  int32_t nactive;  /* nA >= 0, nA <= 8 */
  int32_t nvirt;    /* nV >= 1 */
  int32_t naux;     /* naux >= 1 */
} dsrg_sizes_t;

/* Plan flags. */
#define DSRG_PLAN_HOST_IO 1u  /* also allocate device staging for dsrg_mrpt2_energy_host */
#define DSRG_PLAN_GRAD 2u     /* also allocate the workspace of dsrg_mrpt2_energy_grad */

typedef struct dsrg_plan dsrg_plan_t;

/* Create a plan for one problem size and precision. Allocates all device
 * workspace once (sized from *sz), records the stream (a cudaStream_t, NULL =
 * legacy default stream). Returns DSRG_ERR_OOM if allocation fails and
 * DSRG_ERR_UNSUPPORTED for sizes this build does not handle; *plan is NULL
 * on failure. */
dsrg_status_t dsrg_df_plan(dsrg_plan_t **plan, const dsrg_sizes_t *sz,
                           dsrg_precision_t prec, void *cuda_stream, uint32_t flags);

/* Free the plan and its workspace (waits for the plan's stream first). NULL is OK. */
dsrg_status_t dsrg_plan_destroy(dsrg_plan_t *plan);

/* Replace the plan's stream. */
dsrg_status_t dsrg_plan_set_stream(dsrg_plan_t *plan, void *cuda_stream);

/* Second-order energy by block (see top of file): out_dev[5] on the device.
 * B [naux][nH][nP], eps [n], gamma1 [nA][nA], lambda2 [nA]^4, s >= 0 (Eh^-2).
 * Non-finite s -> DSRG_ERR_NONFINITE; NaN in the arrays propagates to out. */
dsrg_status_t dsrg_mrpt2_energy(dsrg_plan_t *plan, const double *B, const double *eps,
                                const double *gamma1, const double *lambda2, double s,
                                double *out_dev);

/* Energy as dsrg_mrpt2_energy with the two optional inputs of the full
 * Table 1 (either may be NULL, read as 0):
 *   lambda3 [2nA]^6  the three-body cumulant of the reference (Sec. II.A) in
 *                    spin orbitals, lambda3[((((U*n2+V)*n2+W)*n2+X)*n2+Y)*n2+Z] =
 *                    lambda_{UVW}^{XYZ}, n2 = 2 nA, active spin orbital
 *                    U = 2u + sigma (sigma 0 = alpha, 1 = beta); it enters
 *                    terms J (1/4 vt_{mz}^{uv} t_{xy}^{mw} lambda_{uvw}^{xyz}) and
 *                    K (1/4 vt_{xy}^{we} t_{ez}^{uv} lambda_{uvw}^{xyz}) of Table 1,
 *                    reported in out[3]; ignored when nA == 0;
 *   f1 [nH][nP]      the off-diagonal block f^(1) of the generalized Fock matrix
 *                    (Eq. (8)) in the semicanonical basis, f1[i*nP + a] = f_a^i for
 *                    hole i and particle a (the same for both spins); it enters
 *                    the T1 amplitude (Eq. (12)) and the modified Fock matrix
 *                    (Eq. (14)), hence terms A-E (out[3]); its active x active
 *                    entries belong to the diagonal block F^(0) and are not read.
 * Both are caller-owned device arrays, 8-byte aligned. */
dsrg_status_t dsrg_mrpt2_energy_ext(dsrg_plan_t *plan, const double *B, const double *eps,
                                    const double *gamma1, const double *lambda2,
                                    const double *lambda3, const double *f1, double s,
                                    double *out_dev);

/* Pair energies of diagram F1 (Eq. (23)): pairs_dev[nC][nC] on the device,
 * e_mn = sum_ef v_ef (2 v_ef - v_fe) (1-exp(-2 s D^2))/D with v_ef = (me|nf);
 * their sum is out[0] of dsrg_mrpt2_energy. Same arguments and rules. */
dsrg_status_t dsrg_ccvv_pair_energies(dsrg_plan_t *plan, const double *B, const double *eps,
                                      double s, double *pairs_dev);

/* Energy as dsrg_mrpt2_energy, plus the gradient of E_total with respect to
 * the inputs: dB_dev [naux][nH][nP] (dE/dB^Q_{ia} for the entries as passed),
 * deps_dev [n], ds_dev [1]. Outputs are overwritten, not accumulated. Needs a
 * plan created with DSRG_PLAN_GRAD (else DSRG_ERR_INVALID_ARG). The adjoint is
 * the derivative of the energy expression (Table 1, Table 2, Eqs. (12)-(15),
 * (23)) evaluated in FP64 for every precision mode; each core row recomputes
 * its pair integrals v^{kj} instead of storing them. dB is bit-reproducible;
 * deps and ds are summed with FP64 atomics. */
dsrg_status_t dsrg_mrpt2_energy_grad(dsrg_plan_t *plan, const double *B, const double *eps,
                                     const double *gamma1, const double *lambda2, double s,
                                     double *out_dev, double *dB_dev, double *deps_dev,
                                     double *ds_dev);

/* Energy and gradient as dsrg_mrpt2_energy_grad with the optional lambda3
 * and f1 of dsrg_mrpt2_energy_ext (treated as constants: no gradient with
 * respect to them). */
dsrg_status_t dsrg_mrpt2_energy_grad_ext(dsrg_plan_t *plan, const double *B, const double *eps,
                                         const double *gamma1, const double *lambda2,
                                         const double *lambda3, const double *f1, double s,
                                         double *out_dev, double *dB_dev, double *deps_dev,
                                         double *ds_dev);

/* Same as dsrg_mrpt2_energy with HOST inputs and a HOST out[5]: copies the
 * inputs into plan-owned device staging (plan created with DSRG_PLAN_HOST_IO),
 * runs, copies the result back and waits for the stream. Pinned host memory
 * gives the fastest copies. For split-precision plans whose CAVV/CCAV/active
 * integrals come from the tensor-core GEMM, B is copied in groups of core rows
 * (up to eight, sized at plan creation) on a second stream owned by the plan, and the CCVV work of the pairs
 * (i, j) whose larger index j lies in a group starts once that group has
 * arrived, while the later groups are still being copied; the result is the
 * same, bit for bit, as dsrg_mrpt2_energy's on the same inputs. */
dsrg_status_t dsrg_mrpt2_energy_host(dsrg_plan_t *plan, const double *B_host,
                                     const double *eps_host, const double *gamma1_host,
                                     const double *lambda2_host, double s, double *out_host);

/* ---- Batches: many molecules of uneven size in one call. ----
 * A batch plan holds one plan per molecule. In the split modes every
 * molecule's hi/lo planes share one buffer and the CCVV work of all molecules
 * (items = molecule x core pair x virtual tile pair) runs in ONE persistent
 * tensor-core launch, its items dealt to the CTAs by a cost-balancing static
 * scheduler; the other blocks run per molecule. The first call (and any call
 * whose input pointers, s values or out pointer differ from the previous one)
 * captures the whole call into a CUDA graph on an internal stream, so it should
 * not itself be made while the caller's stream is being captured; later calls
 * replay the graph on `cuda_stream`. Results are bitwise those of one plan per
 * molecule. */
typedef struct dsrg_batch dsrg_batch_t;

/* nmol >= 1 sizes; flags as for dsrg_df_plan (DSRG_PLAN_HOST_IO, DSRG_PLAN_GRAD
 * apply to the per-molecule plans). */
dsrg_status_t dsrg_batch_plan(dsrg_batch_t **batch, int32_t nmol, const dsrg_sizes_t *sizes,
                              dsrg_precision_t prec, void *cuda_stream, uint32_t flags);
dsrg_status_t dsrg_batch_destroy(dsrg_batch_t *batch);

/* B, eps, gamma1, lambda2: HOST arrays of nmol DEVICE pointers (per molecule,
 * layouts as for dsrg_mrpt2_energy); s: HOST array of nmol flow parameters;
 * out_dev: DEVICE [nmol][5]. */
dsrg_status_t dsrg_mrpt2_energy_batched(dsrg_batch_t *batch, const double *const *B,
                                        const double *const *eps, const double *const *gamma1,
                                        const double *const *lambda2, const double *s,
                                        double *out_dev);

/* Concurrent branches of the per-molecule work (staging of the planes and pair
 * tables, CAVV, CCAV, the active block and the reductions of each molecule,
 * which do not depend on each other): the graph forks into K branches,
 * molecule m on branch m mod K. The batched CCVV launch waits for every
 * branch's staging; the other blocks run beside it, and each branch waits for
 * it only before its final reductions; the branches join at the end. K is 1,
 * 2, 4 or 8 and at most
 * min(nmol rounded down to a power of 2, 8) (each branch owns a GEMM output
 * buffer, allocated with the plan); the default is that maximum. Setting a new
 * K waits for the batch's stream and makes the next call capture a new graph.
 * The energies do not depend on K. The autotuner times `reps` replays of the
 * whole batched call for every allowed K on the given inputs (as for
 * dsrg_mrpt2_energy_batched; out_dev receives their energies), keeps the
 * fastest and returns it in *chosen (may be NULL). Synchronous. */
int32_t dsrg_batch_branches(const dsrg_batch_t *batch);
dsrg_status_t dsrg_batch_set_branches(dsrg_batch_t *batch, int32_t k);
dsrg_status_t dsrg_batch_autotune_branches(dsrg_batch_t *batch, const double *const *B,
                                           const double *const *eps,
                                           const double *const *gamma1,
                                           const double *const *lambda2, const double *s,
                                           double *out_dev, int32_t reps, int32_t *chosen);

/* Wait for the batch's stream and report device-side conditions of any molecule. */
dsrg_status_t dsrg_batch_sync(dsrg_batch_t *batch);
/* Kernel launches recorded in the batch's graph. */
int32_t dsrg_batch_launch_count(const dsrg_batch_t *batch);
const char *dsrg_batch_last_error(const dsrg_batch_t *batch);

/* Schedule tuning of the split-precision CCVV launch (build-side; the paper has
 * no counterpart). Work items (core pair x virtual tile pair) are dealt to the
 * SMs in a static order, and items that run at the same time share operand
 * tiles in L2 according to that order. A schedule code holds the order in its
 * low 16 bits: pair-major (0), or core orbitals grouped in blocks of G (2G:
 * tile pairs outer; 2G+1: pairs outer); and in bits 16 and up the number of K
 * stages (0..64) ahead that the producer prefetches into L2. The autotuner tries
 * the orders {0, 2G and 2G+1 for a few G} with prefetch distances {0, 4, 12},
 * stages the given inputs, times `reps` launches of the CCVV kernel under every
 * candidate with CUDA events on the plan's (or batch's) stream, keeps the
 * fastest and returns its code in *chosen (may be NULL). Energies do not depend
 * on the schedule: every item writes its own partial sum, reduced in a fixed order.
 * Synchronous; do not call while the stream is being captured. FP64 plans and
 * batches: no-op, *chosen = -1. B, eps: device arrays as for dsrg_mrpt2_energy
 * (for the batch: host arrays of device pointers, s a host array). */
dsrg_status_t dsrg_plan_autotune(dsrg_plan_t *plan, const double *B, const double *eps, double s,
                                 int32_t reps, int32_t *chosen);
dsrg_status_t dsrg_batch_autotune(dsrg_batch_t *batch, const double *const *B,
                                  const double *const *eps, const double *s, int32_t reps,
                                  int32_t *chosen);
/* Schedule code in use (-1 for FP64), and setting one directly (a code found
 * earlier; prefetch distance <= 64; no-op for FP64). The batch
 * setter waits for the batch's stream first; neither may run while a launch
 * that uses the schedule is being captured. */
/* Persisted choices: when the environment variable DSRG_AUTOTUNE_CACHE names a
 * file, dsrg_plan_autotune, dsrg_batch_autotune and dsrg_batch_autotune_branches
 * first look their key up there and, if it is present, apply the stored choice
 * without timing anything (it is returned in *chosen as usual); otherwise they
 * time the candidates and store the winner. Keys name the tuned quantity, the
 * GPU (device name and compute capability), the precision and the size class
 * of the problem (single plans: core orbitals rounded up to 4, virtual tiles of
 * 128, tensor-core K stages rounded up to 8, shard world; batches: molecule
 * count, work items rounded up to 256, padded naux). The file is a flat JSON
 * object {"key": integer, ...}, rewritten whole through a temporary file and a
 * rename. The two calls below read and write it directly (no GPU needed):
 * get returns 1 and sets *value when the key is present, 0 when it (or the
 * file) is absent, -1 for a file that is not such an object; put returns
 * DSRG_ERR_INVALID_ARG for a key with a quote, backslash or control character,
 * or when the file cannot be written. */
int32_t dsrg_tune_cache_get(const char *path, const char *key, int64_t *value);
dsrg_status_t dsrg_tune_cache_put(const char *path, const char *key, int64_t value);

int32_t dsrg_plan_item_order(const dsrg_plan_t *plan);
int32_t dsrg_batch_item_order(const dsrg_batch_t *batch);
dsrg_status_t dsrg_plan_set_item_order(dsrg_plan_t *plan, int32_t order);
dsrg_status_t dsrg_batch_set_item_order(dsrg_batch_t *batch, int32_t order);

/* Device time of the split-precision CCVV kernel alone (Eq. (23) pair GEMMs
 * with the fused regulator epilogue): stages the inputs, makes one untimed
 * launch, then times `reps` launches between two CUDA events recorded on the
 * plan's stream; *ms = average per launch. Synchronous. FP64 plans:
 * DSRG_ERR_UNSUPPORTED. */
dsrg_status_t dsrg_plan_time_ccvv(dsrg_plan_t *plan, const double *B, const double *eps, double s,
                                  int32_t reps, float *ms);

/* E_CCVV without any device allocation (the paper has no counterpart; this is a
 * service to callers that cannot call cudaMalloc, e.g. code running inside a
 * memory pool it does not own or a host that forbids allocation on its hot
 * path). Same value as out[0] of dsrg_mrpt2_energy with a DSRG_PREC_FP64 plan
 * (same FP64 kernel; the final sum may differ in the last bits). B and eps are
 * device arrays as above, out_dev one device double, work queued on
 * cuda_stream. Scratch (work lists and per-item partial sums) lives in a fixed
 * device array of 147456 doubles (1.125 MiB) inside the library, held on every
 * GPU that loads it until the process exits; sizes that do not fit (more than
 * 8192 core pairs, more than 8192 pairs of 64-wide virtual tiles, or more than
 * 131072 items in total) return DSRG_ERR_UNSUPPORTED. Every scratch slot a
 * call reads is written earlier in the same call, so nothing needs clearing.
 * All calls share the array: calls whose work overlaps on the GPU (other
 * streams, other host threads) race and must be serialised by the caller. The
 * first call in each CUDA context of a device looks up the array's device
 * address (the first call of the process on that device, and the first call
 * after the device's context was destroyed and made again, e.g. by
 * cudaDeviceReset, which loads the library's kernels anew at a new address);
 * make that call before any stream capture. A CUDA error left pending by the
 * caller's earlier work makes the call return DSRG_ERR_CUDA without queueing
 * anything, and the error stays pending for the caller to read. */
dsrg_status_t dsrg_ccvv_energy_noalloc(const dsrg_sizes_t *sz, const double *B, const double *eps,
                                       double s, double *out_dev, void *cuda_stream);

/* Counters of the epilogue branches the split-precision kernels took (the
 * paper has no counterpart; a diagnostic of which arithmetic evaluated the
 * regulators of Eqs. (13), (15) and (23)). Counted since the plan was created
 * or last reset; FP64 plans leave them at 0. Indices:
 *   DSRG_COUNT_CCVV_FAR       CCVV epilogue blocks (32 virtual rows x 16 virtual
 *                             columns of one core pair) whose every |Delta| is so
 *                             large that exp(-2 s Delta^2) < 2^-63, evaluated as
 *                             1/Delta;
 *   DSRG_COUNT_CCVV_FACTORED  blocks with every |Delta| >= 1/4 evaluated from the
 *                             factorised exponentials;
 *   DSRG_COUNT_CCVV_DIRECT    blocks with some |Delta| < 1/4 (or of a pair whose
 *                             factors could overflow), evaluated with expm1 per
 *                             element (R(0) = 0) and the exchange combination in FP64;
 *   DSRG_COUNT_CCVV_UNFACTORABLE work items (core pair x tile pair) of pairs whose
 *                             factors could overflow;
 *   DSRG_COUNT_CAVV_NEAR      CAVV positions (core m, e, f) with some |Delta_u| < 1/4
 *                             (or a non-factorisable (m, u)), evaluated in FP64 with
 *                             expm1;
 *   DSRG_COUNT_CAVV_UNFACTORABLE CAVV tiles with a non-factorisable (m, u).
 * Waits for the plan's stream; reset != 0 clears the counters after reading. */
#define DSRG_NCOUNTERS 8
#define DSRG_COUNT_CCVV_FAR 0
#define DSRG_COUNT_CCVV_FACTORED 1
#define DSRG_COUNT_CCVV_DIRECT 2
#define DSRG_COUNT_CCVV_UNFACTORABLE 3
#define DSRG_COUNT_CAVV_NEAR 4
#define DSRG_COUNT_CAVV_UNFACTORABLE 5
dsrg_status_t dsrg_plan_branch_counts(dsrg_plan_t *plan, uint64_t counts[DSRG_NCOUNTERS],
                                      int32_t reset);

/* ---- Generalized Fock matrix and semicanonical orbitals (Sec. II.B, Eq. (8);
 * Sec. III, steps 2-3 of the procedure) ----
 * Inputs over ALL orbitals (not only the hole x particle block), ordered
 * [core | active | virtual], n = nC + nA + nV:
 *   h      [n][n]          one-electron integrals (symmetric);
 *   Bfull  [naux][n][n]    DF/CD factors B^Q_pq (symmetric in p, q), Eq. (19);
 *   gamma1 [nA][nA]        spin-summed active density (may be NULL if nA == 0).
 * The Fock matrix is Eq. (8) for the reference's spin-free density D (2 on the
 * core diagonal, gamma1 on the active block):
 *   f_pq = h_pq + sum_rs D_rs [(pq|rs) - 1/2 (ps|rq)],
 * in FP64 (the exchange part is one FP64 GEMM over the composite index (Q, r)).
 * Semicanonicalisation diagonalises the core, active and virtual blocks of f
 * separately (FP64 parallel cyclic Jacobi; eigenvalues ascending within each
 * block, each eigenvector's largest component positive) and returns, for the
 * orbitals U = blockdiag(U_C, U_A, U_V), the inputs of dsrg_mrpt2_energy_ext:
 *   eps_out     [n]              diagonal of U^T f U;
 *   B_out       [naux][nH][nP]   hole x particle block of U^T B^Q U;
 *   f1_out      [nH][nP]         hole x particle block of U^T f U (f^(1); its
 *                                active x active part, diagonal, set to 0);
 *   gamma1_out  [nA][nA]         U_A^T gamma1 U_A;
 *   lambda2_out [nA]^4           lambda2 rotated by U_A on every index;
 *   lambda3_out [2nA]^6          the spin-orbital lambda3 rotated by U_A (x) 1
 *                                on every index (only if lambda3 != NULL);
 *   U_out       [n][n]           U (may be NULL).
 * All arrays are caller-owned device arrays, 8-byte aligned. The plan owns its
 * workspace (about naux*n*(nH+1) + 2*naux*nH*nP + 6 n^2 doubles). The
 * semicanonicalisation synchronises the plan's stream (the Jacobi sweeps stop
 * on a convergence test read by the host, ||offdiag||^2 <= 1e-30 ||A||^2, at
 * most 30 sweeps) and is not meant to be captured in a graph. */
typedef struct dsrg_sc_plan dsrg_sc_plan_t;
/* sz->ncore, nactive, nvirt >= 0 (n >= 1), naux >= 1, nactive <= 8. */
dsrg_status_t dsrg_sc_plan_create(dsrg_sc_plan_t **plan, const dsrg_sizes_t *sz, void *cuda_stream);
dsrg_status_t dsrg_sc_plan_destroy(dsrg_sc_plan_t *plan);
/* f_dev [n][n]: the generalized Fock matrix (asynchronous, on the plan's stream). */
dsrg_status_t dsrg_generalized_fock(dsrg_sc_plan_t *plan, const double *h, const double *Bfull,
                                    const double *gamma1, double *f_dev);
dsrg_status_t dsrg_semicanonicalize(dsrg_sc_plan_t *plan, const double *h, const double *Bfull,
                                    const double *gamma1, const double *lambda2,
                                    const double *lambda3, double *eps_out, double *B_out,
                                    double *f1_out, double *gamma1_out, double *lambda2_out,
                                    double *lambda3_out, double *U_out);
/* Jacobi sweeps of the slowest-converging block in the last call. */
int32_t dsrg_sc_last_sweeps(const dsrg_sc_plan_t *plan);
const char *dsrg_sc_last_error(const dsrg_sc_plan_t *plan);

/* ---- Integral factorisations (Sec. II.C) ----
 * Density fitting in the MO basis: the factors B^Q_pq = sum_P [W]_QP (pq|P) of
 * the MO three-centre integrals (pq|P) = sum_{mu nu} C_{mu p} (mu nu|P) C_{nu q}
 * for p in [p0, p0 + np), q in [q0, q0 + nq) (e.g. holes x particles, or all
 * orbitals for the Fock build), with W W^T = J^{-1}. The paper writes
 * W = J^{-1/2}; every such W gives the same integrals sum_Q B^Q_pq B^Q_rs and
 * the same energy, and this call takes W = L^{-1} from the Cholesky factor
 * J = L L^T (the factors differ from the J^{-1/2} ones by an orthogonal rotation
 * of the auxiliary index). FP64 throughout.
 *   ao3    [naux][nbf][nbf]  AO three-centre integrals (mu nu|P), symmetric in mu nu;
 *   C      [nbf][nmo]        MO coefficients;
 *   metric [naux][naux]      two-centre integrals J_PQ, symmetric positive definite;
 *   B_out  [naux][np][nq];
 *   work   caller-owned device scratch of dsrg_df_mo_transform_work_bytes() bytes.
 * Synchronous (it reads back the positivity check of the metric):
 * DSRG_ERR_INVALID_ARG if the metric is not positive definite. */
size_t dsrg_df_mo_transform_work_bytes(int32_t nbf, int32_t naux, int32_t np, int32_t nq);
dsrg_status_t dsrg_df_mo_transform(const double *ao3, const double *C, const double *metric,
                                   int32_t nbf, int32_t nmo, int32_t naux, int32_t p0, int32_t np,
                                   int32_t q0, int32_t nq, double *B_out, double *work,
                                   size_t work_bytes, void *cuda_stream);

/* Cholesky decomposition of the two-electron integrals: the pivoted incomplete
 * Cholesky decomposition (outer-product form with diagonal pivoting) of the
 * positive semi-definite matrix M[(pq),(rs)] = (pq|rs) over all n^2 orbital
 * pairs, stopped when the largest remaining diagonal element is below tau (the
 * paper's threshold is 1e-5 Eh) or after max_rank vectors. M is given by
 * factors F [nfac][n][n] (M = sum_k F^k (F^k)^T, e.g. exact integrals of a
 * small basis or a finer factorisation). Output: L_out [max_rank][n][n], of
 * which the first *rank_out are the Cholesky vectors B^Q_pq; every integral
 * of M - sum_Q B^Q (B^Q)^T is below tau in magnitude. FP64. work: caller-owned
 * device scratch of dsrg_cd_factors_work_bytes(n) bytes. Synchronous (the rank
 * is read back). */
size_t dsrg_cd_factors_work_bytes(int32_t n);
dsrg_status_t dsrg_cd_factors(const double *F, int32_t nfac, int32_t n, double tau,
                              int32_t max_rank, double *L_out, int32_t *rank_out, double *work,
                              size_t work_bytes, void *cuda_stream);

/* ---- Several GPUs on one molecule (the paper's loop over core pairs, Sec. III,
 * dealt to ranks instead of threads) ----
 * After dsrg_plan_set_shard(plan, rank, world), the plan's energy and gradient
 * calls compute only this rank's share: the CCVV (F1) core pairs i <= j whose
 * index in row-major order is = rank (mod world), and, on rank 0 only, the
 * other blocks (CAVV, CCAV, active). out[5] then holds this rank's partial
 * block energies: their sum over the ranks is the energy (one reduction of 5
 * doubles, e.g. an all-reduce). The gradient's F1 adjoint is dealt by groups of
 * core rows (their dB rows are disjoint) and the other adjoints run on rank 0,
 * so dB, deps and ds are partial too and sum over the ranks. Every rank needs
 * the whole B. world = 1 restores the full computation. Waits for the plan's
 * stream; do not call while the stream is being captured. */
dsrg_status_t dsrg_plan_set_shard(dsrg_plan_t *plan, int32_t rank, int32_t world);
/* Host-only: the (i, j) core pairs of a shard, pairs_out[2k] = i, [2k+1] = j
 * (pairs_out may be NULL); returns their number, -1 for bad arguments. */
int32_t dsrg_shard_pairs(int32_t ncore, int32_t rank, int32_t world, int32_t *pairs_out);

/* Wait for the plan's stream and report any device-side condition recorded
 * since the last call (DSRG_ERR_TIMEOUT), then clear it. */
dsrg_status_t dsrg_plan_sync(dsrg_plan_t *plan);

/* Self-test of the failure path of the tensor-core kernels (the paper has no
 * counterpart). Every wait in those kernels (on TMA copies, MMAs, TMEM buffers)
 * gives up after about 2 s, records a status word and lets the kernel return,
 * so a lost arrival becomes an error status instead of a hung GPU. This call
 * queues, on the plan's stream, one such wait on a barrier that nothing ever
 * completes; the next dsrg_plan_sync then returns DSRG_ERR_TIMEOUT (after about
 * 2 s) and clears the status, and the plan stays usable. Returns DSRG_OK when
 * the launch was queued. */
dsrg_status_t dsrg_plan_selftest_wait_timeout(dsrg_plan_t *plan);

/* Number of kernel launches the last energy/gradient call queued. */
int32_t dsrg_plan_last_launch_count(const dsrg_plan_t *plan);

/* Bytes of device workspace owned by the plan. */
size_t dsrg_plan_workspace_bytes(const dsrg_plan_t *plan);

const char *dsrg_status_string(dsrg_status_t st);
const char *dsrg_plan_last_error(const dsrg_plan_t *plan);

#ifdef __cplusplus
}
#endif
#endif /* DSRG_H */
