/*
 * gse.h -- C ABI of the GB300 library for group-shared-exponent (GSE) sparse
 * matrices: encoding, SpMV at precision level k, and the stepped
 * mixed-precision CG / GMRES solvers of "Precision-Aware Iterative Algorithms
 * Based on Group-Shared Exponents of Floating-Point Numbers" (Gao et al.,
 * arXiv 2411.04686).
 *
 * Conventions shared by every call:
 *  - Every function returns an int status: GSE_OK (0), a positive solver
 *    outcome (GSE_MAXITER, GSE_BREAKDOWN, GSE_NONFINITE, GSE_TIMEOUT) or a
 *    negative error.  gse_strerror() names it.  No C++ exception crosses the ABI.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Work is enqueued on it; calls that return host data synchronise it.
 *  - Vector arguments (x, y, b) are DEVICE pointers to contiguous FP64 arrays
 *    owned by the caller, unless a parameter says otherwise.
 *  - A handle owns all device memory it allocates.  Calls on one handle must
 *    not overlap in time (the SpMV keeps per-handle scratch for rows that span
 *    work chunks); distinct handles are independent.
 *  - Matrix limits: nnz < 2^31, n_rows < 2^31, column indices in int32.
 */
#ifndef GSE_H
#define GSE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------- */
#define GSE_OK              0
#define GSE_MAXITER         1   /* solve stopped at max_iter; info is filled      */
#define GSE_BREAKDOWN       2   /* p.Ap <= 0 at k_max (CG) or a singular Hessenberg */
#define GSE_NONFINITE       3   /* a solver scalar became Inf/NaN                 */
#define GSE_TIMEOUT         4   /* a bounded device-side wait gave up             */
#define GSE_ERR_INVALID    -1   /* bad argument or malformed CSR                  */
#define GSE_ERR_NONFINITE  -2   /* encode input holds Inf/NaN                     */
#define GSE_ERR_OOM        -3   /* device allocation failed                       */
#define GSE_ERR_CUDA       -4   /* a CUDA runtime call failed                     */
#define GSE_ERR_UNSUPPORTED -5  /* parameter outside what the kernels implement  */

/* Level selectors beyond the GSE levels 1..n_seg: the plain CSR baselines
 * (values attached with gse_attach_values). */
#define GSE_LEVEL_FP64     64
#define GSE_LEVEL_FP32     32
#define GSE_LEVEL_FP16     16   /* IEEE binary16 values (Sec. IV-C baseline) */
#define GSE_LEVEL_BF16     17   /* bfloat16 values (Sec. IV-C baseline)      */

/* Step-policy flags. */
#define GSE_POLICY_NO_STAGNATION 1  /* never evaluate Conditions 1-3              */
#define GSE_POLICY_FLOOR         2  /* also step when the recurrence residual falls
                                       below the level's perturbation floor
                                       (an addition beyond the paper)             */

typedef struct gse_matrix* gse_handle;

/* Input CSR (Sec. III-C, "Sparse Matrix Representation"): RowPtr, ColIdx, Val.
 * Columns must be sorted within each row.  The caller keeps ownership; the
 * arrays are copied.  on_device != 0 means the three pointers are device
 * pointers, else host pointers. */
typedef struct {
    int64_t n_rows, n_cols, nnz;
    const int32_t* row_ptr;
    const int32_t* col_idx;
    const double* val;
    int on_device;
} gse_csr;

/* Parameters of the precision-step policy (Sec. III-D; values used in the
 * paper are listed in Sec. IV-D).  l: iterations before the first check;
 * t: history window; m: check period; rsd_limit / ndec_limit / reldec_limit:
 * thresholds of Conditions 1-3 (ndec_limit <= 0 means t/2); max_iter: total
 * iteration cap; restart: GMRES cycle length (<= 64); k_start / k_max: first and
 * last precision level (1..n_seg, or GSE_LEVEL_FP64 / GSE_LEVEL_FP32 for both to
 * run the plain CSR baseline); flags: GSE_POLICY_*. */
typedef struct {
    int l, t, m;
    double rsd_limit;
    int ndec_limit;
    double reldec_limit;
    int max_iter, restart, k_start, k_max, flags;
} gse_step_policy;

/* Outcome of a solve.  switch_iter[i]: iteration at which level i+1 became
 * active (-1 if never).  rel_res_rec: last recurrence residual / ||b||;
 * rel_res_true: ||b - A_kmax x|| / ||b|| recomputed at the end; seconds: wall
 * time from entry to return. */
typedef struct {
    int status, iters, k_final;
    int switch_iter[3];
    double rel_res_rec, rel_res_true;
    double seconds;
} gse_solve_info;

/* Static description of an encoded matrix. */
typedef struct {
    int64_t n_rows, n_cols, nnz, n_groups, n_empty_rows;
    int group_size, n_seg, seg_bits[3];
    int max_row_len;
    double mean_row_len;
    int schedule;                 /* 1, 2, 4 (nonzero split) or GSE_SCHEDULE_ROWS */
    int64_t bytes_level[3];       /* algorithmic bytes read+written by one SpMV   */
    int num_exp;                  /* table format: shared exponents in the table;
                                     0 for the per-group format                   */
    int64_t overflow16;           /* finite values that became infinite when FP16
                                     values were attached (the paper's FP16
                                     arithmetic overflow); 0 otherwise            */
    int index_in_head;            /* table format: 1 when the exponent index sits
                                     in the head (GSE_INDEX_VALUE), 0 when it sits
                                     in the column index or there is no table     */
} gse_matrix_info;

/* Error name for a status code (static string). */
const char* gse_strerror(int status);

/*
 * Encode a CSR matrix in the group-shared-exponent format (Sec. III-B, Alg. 1,
 * Fig. 3), one shared exponent per group of `group_size` consecutive nonzeros
 * in CSR order (groups may straddle rows; the last one may be partial):
 *   E_g = max biased exponent in the group + 1 (0 for an all-zero group);
 *   M   = floor(|v| * 2^(W - (E_g - 1023))), W = (s1 - 1) + s2 + s3;
 *   head = sign << (s1-1) | top s1-1 bits of M; tail1 = next s2 bits;
 *   tail2 = last s3 bits.
 * group_size: 8, 16 or 32.  seg_bits[0..n_seg-1]: s1 in [2,16] (includes the
 * sign), s2 in [1,16], s3 in [1,16] or {20, 24, 32}.  n_seg in 1..3.
 * Also builds the row-end mask and chunk metadata the SpMV needs, measures
 * row-length statistics and picks a schedule.
 * Errors: GSE_ERR_INVALID (bad sizes, row_ptr not monotone, column out of
 * range), GSE_ERR_NONFINITE (Inf/NaN value), GSE_ERR_UNSUPPORTED, GSE_ERR_OOM.
 * On success *out owns everything; release with gse_free.
 */
int gse_encode(const gse_csr* csr, int group_size, const int* seg_bits, int n_seg,
               void* stream, gse_handle* out);

/* Attach plain CSR values to a handle for a baseline SpMV and solvers:
 * bits = GSE_LEVEL_FP64 (64), GSE_LEVEL_FP32 (32), GSE_LEVEL_FP16 (16, IEEE
 * binary16) or GSE_LEVEL_BF16 (17, bfloat16); the narrower formats round each
 * value to nearest even once from FP64 (Sec. IV-C stores the nonzeros in FP16 or
 * BF16 and widens them to FP64 for the multiply-accumulate).  FP16 overflow is
 * kept as infinity and counted in gse_matrix_info.overflow16.  csr must have the
 * structure the handle was encoded from. */
int gse_attach_values(gse_handle h, const gse_csr* csr, int bits, void* stream);

/*
 * y = A_k x (Sec. III-C, Alg. 2 and the two tail variants): A_k is rebuilt
 * from the first k segments (M_k = M >> (W - W_k), value = +-M_k *
 * 2^(E_g - 1023 - W_k)), multiplied and accumulated in FP64.  k in 1..n_seg,
 * or GSE_LEVEL_FP64 / GSE_LEVEL_FP32 for the attached baseline values.
 * x: n_cols doubles, y: n_rows doubles (device, must not alias).
 * Errors: GSE_ERR_INVALID (k out of range, NULL pointers).
 */
int gse_spmv(gse_handle h, int k, const double* x, double* y, void* stream);

/*
 * Stepped mixed-precision CG (Alg. 3 with the step policy of Sec. III-D,
 * Eqs. 3-6, Conditions 1-3; FP64 vector operations as in Sec. IV-D).
 * Starts at k_start; at a step the level rises by one, the residual is
 * recomputed as b - A_k x and the search direction restarts.  When the
 * recurrence residual falls below tol, the true residual with A_kmax decides:
 * below tol ends the solve, otherwise the level steps (or, at k_max, the
 * recurrence restarts from the true residual).
 * b: n_rows doubles; x: initial guess in, solution out (device).  info may be
 * NULL.  Returns GSE_OK, GSE_MAXITER, GSE_BREAKDOWN, GSE_NONFINITE or an error.
 */
int gse_cg(gse_handle h, const double* b, double* x, double tol, const gse_step_policy* policy,
           gse_solve_info* info, void* stream);

/*
 * Stepped mixed-precision restarted GMRES(restart) (Alg. 3, Sec. III-D), in
 * FP64 on the device: Arnoldi by classical Gram-Schmidt with one conditional
 * re-orthogonalisation pass (taken when the norm of w falls below 0.7 of its
 * value before the projection), Givens rotations and the least-squares
 * residual.  The paper does not name an orthogonalisation; the result equals
 * modified Gram-Schmidt's up to rounding.  The level changes only at cycle
 * boundaries; the monitored residual is the least-squares residual of each
 * inner iteration.  Arguments as gse_cg.
 */
int gse_gmres(gse_handle h, const double* b, double* x, double tol, const gse_step_policy* policy,
              gse_solve_info* info, void* stream);

/*
 * Batched stepped CG: nsys independent systems (each with its own handle,
 * right-hand side and initial guess) solved concurrently, their kernels
 * interleaved on one stream.  The paper solves one system at a time; batching
 * is a deployment addition, and each system's result is bit-identical to its
 * solo gse_cg.  infos: nsys entries (may be NULL).  b and x are host arrays of
 * nsys device pointers.  Returns the first non-OK status.
 */
int gse_batch_cg(int nsys, const gse_handle* hs, const double* const* b, double* const* x,
                 double tol, const gse_step_policy* policy, gse_solve_info* infos, void* stream);

/*
 * Continuous-batching CG engine: the batched solver above, exposed step by
 * step so that systems can join and leave while others run (serving).  Each
 * submitted system occupies a slot; gse_engine_run advances every active
 * system by up to max_slots iteration slots (one slot = one CG iteration, or
 * one restart / true-residual step) with one set of kernel launches per slot
 * for all of them; gse_engine_poll hands back finished systems and frees their
 * slots.  A handle may occupy at most one slot at a time (its workspace holds
 * the Krylov vectors).  Results of a system do not depend on what else runs.
 * The paper has no counterpart (it solves one system at a time).
 */
typedef struct gse_cg_engine* gse_engine;
int gse_engine_create(int capacity, void* stream, gse_engine* out);
int gse_engine_submit(gse_engine e, gse_handle h, const double* b, double* x, double tol,
                      const gse_step_policy* policy, int* slot);
int gse_engine_run(gse_engine e, int max_slots, int batch, int* n_running);
int gse_engine_poll(gse_engine e, int* done_slots, gse_solve_info* infos, int max_done, int* n_done);
int gse_engine_cancel(gse_engine e, int slot, gse_solve_info* info);
void gse_engine_destroy(gse_engine e);

/*
 * gse_engine_run in two halves, so the host can work while the device solves.
 * gse_engine_launch queues max_slots iteration slots (in CUDA-graph batches of
 * `batch`) and one copy of every system's state on the engine's stream, and
 * returns without waiting.  gse_engine_wait blocks until that launch has
 * finished, updates the host view of the states and sets *n_running (may be
 * NULL) to the active systems not yet done.  A launch runs all max_slots slots
 * (gse_engine_run stops early once nothing runs).  Between the two calls the
 * caller may do any other work, including encoding new matrices on other
 * streams; every other engine call (submit, run, poll, cancel, destroy) first
 * waits for a pending launch itself.  Errors: GSE_ERR_INVALID (NULL engine,
 * max_slots < 0), GSE_ERR_CUDA.
 */
int gse_engine_launch(gse_engine e, int max_slots, int batch);
int gse_engine_wait(gse_engine e, int* n_running);

/*
 * gse_cg_noalloc: the stepped CG of gse_cg for callers that cannot allocate
 * device memory once their set-up is done (a real-time loop with a fixed
 * memory budget, code under an allocator that forbids new allocations, a
 * thread that must not let cudaMalloc/cudaFree synchronise the device).  The
 * paper has no counterpart; this is a deployment variant.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library call.
 *    Its Krylov vectors, history, reduction scratch, descriptor and state live
 *    in one fixed device array inside the library (about 1.7 MB, held by every
 *    GPU that loads the library until the process exits).
 *  - Limit: h must have at most 65536 rows; larger systems and the
 *    GSE_POLICY_FLOOR flag are rejected with GSE_ERR_UNSUPPORTED.
 *  - The first call on a device looks up that array's device address (once
 *    per device, with the device current); make that first call before any
 *    stream capture.
 *  - All calls share the array and each call re-initialises it; calls whose
 *    GPU work overlaps (two threads, two streams) race and corrupt each other.
 * Arguments, results and status codes as gse_cg; the solution, iteration
 * counts and switch iterations equal gse_cg's bit for bit, and so does
 * rel_res_true of a converged solve (the true residual both compute on the
 * device at the convergence check).  For a solve that stops without
 * converging, rel_res_true is recomputed here by a one-block device sum and
 * agrees with gse_cg's (a host sum) to rounding only.
 */
int gse_cg_noalloc(gse_handle h, const double* b, double* x, double tol, const gse_step_policy* policy,
                   gse_solve_info* info, void* stream);

/* Host copies of the logical segments (tests): head[nnz], tail1[nnz],
 * tail2[nnz] (the s3-bit field, widened to 32 bits), gexp[n_groups].  Any
 * pointer may be NULL to skip that array.  Synchronises the device.  gexp must
 * be NULL for a table-format handle (GSE_ERR_INVALID otherwise). */
int gse_export(gse_handle h, uint16_t* head, uint16_t* tail1, uint32_t* tail2, int16_t* gexp);

/*
 * The paper's default layout: ONE table of shared exponents for the whole
 * matrix (Sec. III-B "Shared Exponents Extraction" and "Denormalized
 * Representation", Alg. 1), the exponent index of each nonzero stored in the
 * top bits of its column index (Sec. III-C, Alg. 2):
 *   table = the num_exp most frequent biased exponents, each + 1, ordered by
 *           count (equal counts: larger exponent first); max exponent + 1 is
 *           always an entry (it replaces the last kept one if it missed the cut);
 *   a value with exponent e uses the entry e + 1 when present (d = 1), else the
 *           nearest larger entry T (d = T - e);
 *   M = floor(|v| * 2^(W - (T - 1023))), split into head / tail1 / tail2 as in
 *           gse_encode (zeros and subnormals: M = 0, index 0).
 * num_exp in [1, 64].  The index takes b = ceil(log2(entries)) bits.  It goes
 * in the column index while n_cols <= 2^(32 - b); otherwise, as Sec. III-C
 * allows, into the value (GSE_INDEX_VALUE of gse_encode_table_ex).  Every other
 * call (SpMV at any level, baselines, solvers, decode, footprint) accepts the
 * handle.  Errors as gse_encode.
 */
int gse_encode_table(const gse_csr* csr, int num_exp, const int* seg_bits, int n_seg, void* stream,
                     gse_handle* out);

/* Where the exponent index of a table-format nonzero is kept. */
#define GSE_INDEX_AUTO   0   /* column index if its spare bits hold it, else the head */
#define GSE_INDEX_COL    1   /* top b bits of the column index (Sec. III-C, Alg. 2);
                                GSE_ERR_UNSUPPORTED when n_cols > 2^(32 - b)       */
#define GSE_INDEX_VALUE  2   /* the b head bits right below the sign (Sec. III-C,
                                for column counts without spare bits): every level
                                keeps b magnitude bits fewer, W_k' = W_k - b, and
                                M = floor(|v| * 2^(W' - (T - 1023)));
                                head = sign << (s1-1) | index << (s1-1-b) |
                                top s1-1-b bits of M.  Needs b <= s1 - 2
                                (GSE_ERR_UNSUPPORTED otherwise).                   */

/*
 * gse_encode_table with the placement of the index and, optionally, the
 * sampled exponent extraction of Sec. III-B.
 *   index_place: GSE_INDEX_AUTO / GSE_INDEX_COL / GSE_INDEX_VALUE.
 *   block_rows:  0 counts every nonzero (the exact extraction).  > 0 cuts the
 *                rows into blocks of block_rows rows (the last may be shorter)
 *                and counts only the nonzeros of one row per block,
 *                sample_rows[b] (host array of ceil(n_rows / block_rows)
 *                row indices, each inside its block; the caller draws them).
 *                Each counts as many times as its block has rows.  The entries
 *                are then chosen from these counts as in gse_encode_table.
 *                max exponent + 1 is still taken over all values, so every
 *                value has an entry at or above its exponent.
 * Errors: GSE_ERR_INVALID (as gse_encode; num_exp outside [1, 64]; a bad
 * index_place; block_rows < 0; a sample row outside its block or NULL
 * sample_rows), GSE_ERR_UNSUPPORTED (the chosen place cannot hold the index),
 * GSE_ERR_NONFINITE, GSE_ERR_OOM.  sample_rows is read before the call returns.
 */
int gse_encode_table_ex(const gse_csr* csr, int num_exp, const int* seg_bits, int n_seg, int index_place,
                        int64_t block_rows, const int64_t* sample_rows, void* stream, gse_handle* out);

/* Table-format handle (tests): the table (at most 64 int16 entries, host),
 * its entry count, and the index of every nonzero (idx[nnz], host; read from
 * the column words or the heads, wherever it is kept).  Any pointer may be
 * NULL.  GSE_ERR_INVALID for a per-group handle.  gse_export returns the heads
 * as stored, index bits included. */
int gse_export_table(gse_handle h, int16_t* table, int* n_table, uint8_t* idx);

/* vals[nnz] (device) = the FP64 values of A_k in CSR order (tests). */
int gse_decode(gse_handle h, int k, double* vals, void* stream);

/* Describes the handle. */
int gse_matrix_get_info(gse_handle h, gse_matrix_info* info);

/* Force the SpMV schedule: 1, 2 or 4 = nonzero split, that many units of 8
 * consecutive nonzeros per lane (the table format always runs 1);
 * GSE_SCHEDULE_ROWS = one row per lane, 256 consecutive rows per CTA (only for
 * matrices whose 256-row blocks span at most 4096 nonzeros, else
 * GSE_ERR_UNSUPPORTED); 0 restores the automatic choice. */
#define GSE_SCHEDULE_ROWS 8
int gse_set_schedule(gse_handle h, int schedule);

/* Time each schedule on this matrix at level k (CUDA events, a few reps) and
 * keep the fastest. */
int gse_autotune(gse_handle h, int k, void* stream);

/* Device bytes held by the handle, solver workspace included. */
size_t gse_footprint(gse_handle h);

/* Device bytes a CG (method 0) or GMRES (method 1) solve of this handle will
 * hold in total, encoded matrix included (admission control). */
size_t gse_solve_footprint(gse_handle h, int method, int restart);

/* Releases the handle and all its device memory (NULL is a no-op).  Waits for
 * the device to finish queued work first (the buffers may still be in use).
 * Handle and workspace memory comes from a stream-ordered pool the library
 * keeps per device: freed blocks stay cached there for later handles and are
 * not returned to the driver before the process exits, so a server that
 * encodes and frees one matrix per request never calls cudaMalloc/cudaFree. */
void gse_free(gse_handle h);

/* Test hook for the bounded waits (no counterpart in the paper).  The staged
 * kernels (the 256-row row schedule of the table format and of other segment
 * layouts, and the 2- and 4-unit nonzero split) wait on shared-memory barriers
 * for their bulk copies, and every wait gives up after a bounded number of
 * tries and records GSE_TIMEOUT in the handle, which the next solve on the
 * handle reports.  With on != 0 these kernels of handle h issue no copy and
 * wait with a short bound, so each wait runs out at once with nothing in
 * flight: the path a real expiry takes, without a fault or a hang.  on = 0
 * restores normal work; each solve starts with the record cleared.  Blocks
 * until the flag is on the device.  Errors: GSE_ERR_INVALID (NULL handle),
 * GSE_ERR_CUDA. */
int gse_test_timeout(gse_handle h, int on);

/* Machine probes (no counterpart in the paper: they measure the GPU the
 * kernels run on).  On GB300 two floors of the SpMV are not HBM: the FP64 FMA
 * rate (one DFMA per nonzero) and, for scattered columns, the rate at which
 * random 8-byte x gathers are served.  gse_probe runs one probe on `stream`
 * and waits for it; out[0] receives the result, out[1] the kernel time in ms
 * (where timed):
 *   GSE_PROBE_DFMA_RATE     FP64 FMAs per second, full occupancy, 8 chains
 *                           per thread (param unused);
 *   GSE_PROBE_DFMA_CHAINS   FP64 FMAs per second with `param` warps per SM
 *                           (1..64), one dependent chain per thread;
 *   GSE_PROBE_DFMA_LATENCY  SM clock cycles per dependent DFMA, one thread;
 *   GSE_PROBE_GATHER_L1 /   random 8-byte loads per second from `table`
 *   GSE_PROBE_GATHER_L2     (device, `param` doubles, a power of two in
 *                           [2^10, 2^32], owned by the caller), 8 in flight
 *                           per thread, through L1 (ld.global.nc) or L2 only.
 * The probe allocates 16 bytes of device scratch per call.  Errors:
 * GSE_ERR_INVALID (unknown probe, bad param or table), GSE_ERR_OOM,
 * GSE_ERR_CUDA. */
#define GSE_PROBE_DFMA_RATE    1
#define GSE_PROBE_DFMA_CHAINS  2
#define GSE_PROBE_DFMA_LATENCY 3
#define GSE_PROBE_GATHER_L1    4
#define GSE_PROBE_GATHER_L2    5
int gse_probe(int which, int64_t param, const double* table, double* out, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* GSE_H */
