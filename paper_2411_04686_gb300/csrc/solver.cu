// solver.cu -- the stepped mixed-precision CG (Alg. 3 with the policy of
// Sec. III-D) as a device-resident, multi-system engine.
//
// Every system carries a small state machine in device memory; one iteration
// "slot" is three kernels that each process all active systems:
//   P1  SpMV phase   ITER:    q = A_k p and p.q          (fused epilogue); the
//                             last block: alpha = rho / p.q and the breakdown test
//                    RESID_R: r = b - A_k x              (restart at level k)
//                    RESID_T: q = b - A_kmax x           (true-residual check)
//   P2  vector 1     ITER:    r -= alpha q, rho' = r.r, then (last block) the
//                             residual history, Eqs. 3-6, Conditions 1-3, the
//                             convergence check and the next mode
//                    RESID_R: rho = r.r      RESID_T: ||q||, decide
//   P3  vector 2     x += alpha p (the x update is folded here, one pass) and
//                    p = r + beta p, or p = r / r = p = q after a restart;
//                    under the floor rule also ||x_j|| and (last block) the
//                    floor decision
// The host only enqueues slots (batches of them replayed from a captured CUDA
// graph) and reads the state array once per batch, so a single solve runs
// without a host round trip per iteration, and a batch of systems shares each
// launch.  gse_engine_launch / gse_engine_wait split a batch so the host can
// work (encode the next requests) while it runs.  Each system's blocks, chunks
// and reduction order depend on its own size only, so a system gives
// bit-identical results alone and inside any batch.
#include <chrono>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <type_traits>
#include <vector>

#include "pool.cuh"
#include "solver_internal.cuh"

namespace gse {

// ---- helpers --------------------------------------------------------------

// Sum over a system's blocks: the last block (per-system counter) gets the total
// (in every thread) and returns true.
__device__ __forceinline__ bool sys_grid_sum(double v, double* partial, unsigned* counter, int lb,
                                             int nblk, double* red, double* total) {
    __shared__ bool last;
    __shared__ double tot;
    const double s = block_sum(v, red);
    if (threadIdx.x == 0) {
        partial[lb] = s;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double a = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) a += __ldcg(partial + i);
    a = block_sum(a, red);
    if (threadIdx.x == 0) {
        tot = a;
        *counter = 0;
    }
    __syncthreads();
    *total = tot;
    return true;
}

// Two sums at once (partials of the second at partial + nblk).
__device__ __forceinline__ bool sys_grid_sum2(double v, double w, double* partial, unsigned* counter, int lb,
                                              int nblk, double* red, double* total_v, double* total_w) {
    __shared__ bool last;
    __shared__ double tv, tw;
    const double s1 = block_sum(v, red);
    const double s2 = block_sum(w, red);
    if (threadIdx.x == 0) {
        partial[lb] = s1;
        partial[nblk + lb] = s2;
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (!last) return false;
    __threadfence();
    double a = 0.0, b = 0.0;
    for (int i = threadIdx.x; i < nblk; i += blockDim.x) {
        a += __ldcg(partial + i);
        b += __ldcg(partial + nblk + i);
    }
    a = block_sum(a, red);
    b = block_sum(b, red);
    if (threadIdx.x == 0) {
        tv = a;
        tw = b;
        *counter = 0;
    }
    __syncthreads();
    *total_v = tv;
    *total_w = tw;
    return true;
}

// Same block bookkeeping without a sum: true in the last block of the system.
__device__ __forceinline__ bool sys_grid_last(unsigned* counter, int nblk) {
    __shared__ bool last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(counter, 1u) == (unsigned)nblk - 1;
    }
    __syncthreads();
    if (!last) return false;
    if (threadIdx.x == 0) *counter = 0;
    return true;
}

// ITER: q = A p with the p.q epilogue; RESID: y = b - A x, no dot.  The engine
// runs one unit of 8 nonzeros per lane (chunks of 256), ENG_WARPS chunks per stage.
// ITER: q = A p with the p.q epilogue; RESID: y = b - A x, no dot.  The
// nonzero split runs the direct-load chunk loop (no stage ring): warp w of the
// system's CTAs takes chunks w, w + W, ...
template <bool ITER>
__device__ __forceinline__ double eng_pipe(int k, const MatView& m, const double* x, const Epi& e, int64_t w0,
                                           int64_t ws, int64_t nch) {
    switch (k) {
        case 1: return spmv_chunks_direct<1, 0, ITER, !ITER>(m, x, e, w0, ws, nch);
        case 2: return spmv_chunks_direct<2, 0, ITER, !ITER>(m, x, e, w0, ws, nch);
        case 3:
            if (m.r_lo == 4) return spmv_chunks_direct<3, 4, ITER, !ITER>(m, x, e, w0, ws, nch);
            return spmv_chunks_direct<3, -1, ITER, !ITER>(m, x, e, w0, ws, nch);
        case SRC_FP32: return spmv_chunks_direct<SRC_FP32, 0, ITER, !ITER>(m, x, e, w0, ws, nch);
        case SRC_FP16: return spmv_chunks_direct<SRC_FP16, 0, ITER, !ITER>(m, x, e, w0, ws, nch);
        case SRC_BF16: return spmv_chunks_direct<SRC_BF16, 0, ITER, !ITER>(m, x, e, w0, ws, nch);
        default: return spmv_chunks_direct<SRC_FP64, 0, ITER, !ITER>(m, x, e, w0, ws, nch);
    }
}

template <bool ITER>
__device__ __forceinline__ double eng_rows(int k, const MatView& m, const double* x, const Epi& e, int64_t sb0,
                                           int64_t sbs, int64_t nsb, int span, unsigned char* smem, int* err) {
    if (m.tbl) {                      // table format: the shared exponent comes with each col word
        switch (k) {
            case 1: return spmv_rows_block<1, 0, ITER, !ITER, ENG_ROW_STAGES, true>(m, x, e, sb0, sbs, nsb, row_stage_layout<1, 0>(span, m.r_lo), smem, err);
            case 2: return spmv_rows_block<2, 0, ITER, !ITER, ENG_ROW_STAGES, true>(m, x, e, sb0, sbs, nsb, row_stage_layout<2, 0>(span, m.r_lo), smem, err);
            case 3: return spmv_rows_block<3, -1, ITER, !ITER, ENG_ROW_STAGES, true>(m, x, e, sb0, sbs, nsb, row_stage_layout<3, -1>(span, m.r_lo), smem, err);
            default: break;
        }
    }
    switch (k) {
        case 1: return spmv_rows_block<1, 0, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<1, 0>(span, m.r_lo), smem, err);
        case 2: return spmv_rows_block<2, 0, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<2, 0>(span, m.r_lo), smem, err);
        case 3:
            if (m.r_lo == 4)
                return spmv_rows_block<3, 4, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<3, -1>(span, m.r_lo), smem, err);
            return spmv_rows_block<3, -1, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<3, -1>(span, m.r_lo), smem, err);
        case SRC_FP32: return spmv_rows_block<SRC_FP32, 0, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<SRC_FP32, 0>(span, m.r_lo), smem, err);
        case SRC_FP16: return spmv_rows_block<SRC_FP16, 0, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<SRC_FP16, 0>(span, m.r_lo), smem, err);
        case SRC_BF16: return spmv_rows_block<SRC_BF16, 0, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<SRC_BF16, 0>(span, m.r_lo), smem, err);
        default: return spmv_rows_block<SRC_FP64, 0, ITER, !ITER, ENG_ROW_STAGES>(m, x, e, sb0, sbs, nsb, row_stage_layout<SRC_FP64, 0>(span, m.r_lo), smem, err);
    }
}

// ---- P1: SpMV phase -------------------------------------------------------
// Two kernels, one per schedule, so the row kernel keeps the register budget
// and CTA shape (8 warps, 256-row super-blocks) of the standalone row SpMV.

template <bool ROWS>
__device__ __forceinline__ void p1_body(const SysDesc* __restrict__ sys, const int2* __restrict__ map,
                                        unsigned char* smem, double* red) {
    const int2 bm = map[blockIdx.x];
    const SysDesc& S = sys[bm.x];
    CgState* st = S.st;
    const int mode = st->mode;
    if (mode == MODE_DONE) return;
    const int lb = bm.y, nblk = S.nblk_spmv;
    const MatView m = S.m;
    Epi e;
    const double* x;
    int k;
    if (mode == MODE_ITER) {
        e.kind = EPI_CG_PQ; e.y = S.q; e.b = nullptr; e.p = S.p; x = S.p; k = st->k;
    } else if (mode == MODE_RESID_R) {
        e.kind = EPI_RESID; e.y = S.r; e.b = S.b; e.p = nullptr; x = S.x; k = st->k;
    } else {
        e.kind = EPI_RESID; e.y = S.q; e.b = S.b; e.p = nullptr; x = S.x; k = S.prm.kmax;
    }
    const int64_t nsb = (S.n + 32 * ENG_ROW_WARPS - 1) / (32 * ENG_ROW_WARPS);
    if (!ROWS) fill_empty_rows(m, e, (int64_t)lb * blockDim.x + threadIdx.x, (int64_t)nblk * blockDim.x);
    if (mode == MODE_ITER) {
        const int64_t w0 = (int64_t)lb * ENG_WARPS + (threadIdx.x >> 5), ws = (int64_t)nblk * ENG_WARPS;
        const double dot = ROWS ? eng_rows<true>(k, m, x, e, lb, nblk, nsb, S.row_span, smem, S.err)
                                : eng_pipe<true>(k, m, x, e, w0, ws, S.n_chunks);
        double total;
        if (sys_grid_sum(dot, S.partial, S.counter, lb, nblk, red, &total) && threadIdx.x == 0) {
            // alpha = rho / p.Ap once per system here, not in every thread of P2
            const double alpha = st->rho / total;
            st->pq = total;
            st->alpha = alpha;
            st->brk = !(total > 0.0) || !isfinite(total) || !isfinite(alpha);
        }
    } else {
        if (ROWS) eng_rows<false>(k, m, x, e, lb, nblk, nsb, S.row_span, smem, S.err);
        else eng_pipe<false>(k, m, x, e, (int64_t)lb * ENG_WARPS + (threadIdx.x >> 5), (int64_t)nblk * ENG_WARPS,
                             S.n_chunks);
    }
}

__global__ void __launch_bounds__(ENG_WARPS * 32) k_cg_p1(const SysDesc* __restrict__ sys,
                                                           const int2* __restrict__ map) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double red[32];
    p1_body<false>(sys, map, smem, red);
}

__global__ void __launch_bounds__(ENG_ROW_WARPS * 32, 4) k_cg_p1_rows(const SysDesc* __restrict__ sys,
                                                                    const int2* __restrict__ map) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double red[32];
    p1_body<true>(sys, map, smem, red);
}

// One lane-row pass as a separate (not inlined) function, so that the
// p.Ap pass and the residual pass of a kernel get their registers each.
template <int K, bool DOT, bool RESID, int TBL = 0>
__device__ __noinline__ double eng_lr_pass(const MatView& m, const double* x, const Epi& e, int64_t w0, int64_t ws,
                                           int64_t ntile, unsigned char* wsm) {
    return lr_loop<K, DOT, RESID, 1, TBL>(m, x, e, w0, ws, ntile, wsm);
}

// Lane-row SpMV phase: warp w of a system's CTAs takes the 32-row tiles w,
// w + W, ... through its own two-stage ring in shared memory, at the level
// its system runs.  Each level's pass is a separate function with its own
// registers; the kernel itself holds little besides the system's matrix
// view, which it stages in shared memory once per block.
// TBL: the system's table kind (lr_tbl); the plain CSR baselines of a table
// handle only mask their columns, so they take kind 1.
template <bool ITER, int TBL = 0>
__device__ __forceinline__ double eng_lanerow(int k, const MatView& m, const double* x, const Epi& e, int64_t w0,
                                              int64_t ws, int64_t ntile, unsigned char* smem) {
    const int warp = threadIdx.x >> 5;
    constexpr int TB = TBL ? 1 : 0;
    switch (k) {
#define GSE_LR_CASE(KK, T) \
    case KK: return eng_lr_pass<KK, ITER, !ITER, T>(m, x, e, w0, ws, ntile, smem + warp * LR_STAGES * LrLayout<KK, 1>::BYTES);
        GSE_LR_CASE(1, TBL)
        GSE_LR_CASE(2, TBL)
        GSE_LR_CASE(3, TBL)
        GSE_LR_CASE(SRC_FP32, TB)
        GSE_LR_CASE(SRC_FP16, TB)
        GSE_LR_CASE(SRC_BF16, TB)
        GSE_LR_CASE(SRC_FP64, TB)
#undef GSE_LR_CASE
        default: return 0.0;
    }
}

template <bool ITER>
__device__ __forceinline__ double eng_lanerow_kind(int tbl, int k, const MatView& m, const double* x, const Epi& e,
                                                   int64_t w0, int64_t ws, int64_t ntile, unsigned char* smem) {
    if (tbl == 2) return eng_lanerow<ITER, 2>(k, m, x, e, w0, ws, ntile, smem);
    if (tbl == 1) return eng_lanerow<ITER, 1>(k, m, x, e, w0, ws, ntile, smem);
    return eng_lanerow<ITER, 0>(k, m, x, e, w0, ws, ntile, smem);
}

__global__ void __launch_bounds__(ENG_LR_WARPS * 32, 4) k_cg_p1_lr(const SysDesc* __restrict__ sys,
                                                                    const int2* __restrict__ map) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double red[32];
    __shared__ MatView mv;
    const int2 bm = map[blockIdx.x];
    const SysDesc& S = sys[bm.x];
    CgState* st = S.st;
    const int mode = st->mode;
    if (mode == MODE_DONE) return;
    const int lb = bm.y, nblk = S.nblk_spmv;
    static_assert(sizeof(MatView) % 8 == 0, "word copy");
    if (threadIdx.x < sizeof(MatView) / 8)
        reinterpret_cast<long long*>(&mv)[threadIdx.x] = reinterpret_cast<const long long*>(&S.m)[threadIdx.x];
    __syncthreads();
    Epi e;
    const double* x;
    int k;
    if (mode == MODE_ITER) {
        e.kind = EPI_CG_PQ; e.y = S.q; e.b = nullptr; e.p = S.p; x = S.p; k = st->k;
    } else if (mode == MODE_RESID_R) {
        e.kind = EPI_RESID; e.y = S.r; e.b = S.b; e.p = nullptr; x = S.x; k = st->k;
    } else {
        e.kind = EPI_RESID; e.y = S.q; e.b = S.b; e.p = nullptr; x = S.x; k = S.prm.kmax;
    }
    const int64_t ntile = (S.n + 31) / 32;      // one row per lane in the engine
    const int64_t w0 = (int64_t)lb * ENG_LR_WARPS + (threadIdx.x >> 5), ws = (int64_t)nblk * ENG_LR_WARPS;
    if (mode == MODE_ITER) {
        const double dot = eng_lanerow_kind<true>(S.lr_tbl, k, mv, x, e, w0, ws, ntile, smem);
        double total;
        if (sys_grid_sum(dot, S.partial, S.counter, lb, nblk, red, &total) && threadIdx.x == 0) {
            const double alpha = st->rho / total;
            st->pq = total;
            st->alpha = alpha;
            st->brk = !(total > 0.0) || !isfinite(total) || !isfinite(alpha);
        }
    } else {
        eng_lanerow_kind<false>(S.lr_tbl, k, mv, x, e, w0, ws, ntile, smem);
    }
}

// The p.Ap pass of one system whose matrix view is the kernel's parameter:
// every level's loop inlined, so the view's fields are read from the
// parameter bank as in the standalone SpMV kernel, not from registers.
__device__ __forceinline__ double solo_lr_iter(int k, const MatView& m, const double* x, const Epi& e, int64_t w0,
                                               int64_t ws, int64_t ntile, unsigned char* smem) {
    const int warp = threadIdx.x >> 5;
    switch (k) {
#define GSE_LR_SOLO(KK) \
    case KK: return lr_loop<KK, true, false, 1>(m, x, e, w0, ws, ntile, smem + warp * LR_STAGES * LrLayout<KK, 1>::BYTES);
        GSE_LR_SOLO(1)
        GSE_LR_SOLO(2)
        GSE_LR_SOLO(3)
        GSE_LR_SOLO(SRC_FP32)
        GSE_LR_SOLO(SRC_FP16)
        GSE_LR_SOLO(SRC_BF16)
        GSE_LR_SOLO(SRC_FP64)
#undef GSE_LR_SOLO
        default: return 0.0;
    }
}

// k_cg_p1_lr for an engine that holds one lane-row system: the same
// partition (grid = the system's P1 blocks, block b = its block b), the same
// passes and the same sums, so its results are bit-identical; only the
// matrix view travels as a launch parameter.  The residual passes (a few per
// solve) take the shared-memory copy and the separate pass functions.
__global__ void __launch_bounds__(ENG_LR_WARPS * 32, 4) k_cg_p1_lr_solo(const __grid_constant__ MatView m,
                                                                         const SysDesc* __restrict__ sys) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ double red[32];
    __shared__ MatView mv;
    const SysDesc& S = *sys;
    CgState* st = S.st;
    const int mode = st->mode;
    if (mode == MODE_DONE) return;
    const int lb = blockIdx.x, nblk = S.nblk_spmv;
    const int64_t ntile = (S.n + 31) / 32;
    const int64_t w0 = (int64_t)lb * ENG_LR_WARPS + (threadIdx.x >> 5), ws = (int64_t)nblk * ENG_LR_WARPS;
    Epi e;
    if (mode == MODE_ITER) {
        e.kind = EPI_CG_PQ; e.y = S.q; e.b = nullptr; e.p = S.p;
        const double dot = S.lr_tbl ? eng_lanerow_kind<true>(S.lr_tbl, st->k, m, S.p, e, w0, ws, ntile, smem)
                                    : solo_lr_iter(st->k, m, S.p, e, w0, ws, ntile, smem);
        double total;
        if (sys_grid_sum(dot, S.partial, S.counter, lb, nblk, red, &total) && threadIdx.x == 0) {
            const double alpha = st->rho / total;
            st->pq = total;
            st->alpha = alpha;
            st->brk = !(total > 0.0) || !isfinite(total) || !isfinite(alpha);
        }
        return;
    }
    if (threadIdx.x < sizeof(MatView) / 8)
        reinterpret_cast<long long*>(&mv)[threadIdx.x] = reinterpret_cast<const long long*>(&m)[threadIdx.x];
    __syncthreads();
    int k;
    if (mode == MODE_RESID_R) {
        e.kind = EPI_RESID; e.y = S.r; e.b = S.b; e.p = nullptr; k = st->k;
    } else {
        e.kind = EPI_RESID; e.y = S.q; e.b = S.b; e.p = nullptr; k = S.prm.kmax;
    }
    eng_lanerow_kind<false>(S.lr_tbl, k, mv, S.x, e, w0, ws, ntile, smem);
}

// Dynamic shared memory of the lane-row P1 kernel for systems that run
// levels up to `widest` (the kernel's limit is set at the engine's creation).
int p1_lr_occupancy(size_t smem) {
    cudaFuncSetAttribute((const void*)k_cg_p1_lr_solo, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         lanerow_smem_k<1>(SRC_FP64, ENG_LR_WARPS));
    cudaFuncSetAttribute((const void*)k_cg_p1_lr, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         lanerow_smem_k<1>(SRC_FP64, ENG_LR_WARPS));
    int v = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, (const void*)k_cg_p1_lr, ENG_LR_WARPS * 32, smem) !=
            cudaSuccess || v < 1) {
        cudaGetLastError();
        v = 1;
    }
    return v;
}

// ---- P1b: rows that cross chunks (after P1) --------------------------------

__global__ void __launch_bounds__(256) k_cg_fix(const SysDesc* __restrict__ sys, const int2* __restrict__ map) {
    const int2 bm = map[blockIdx.x];
    const SysDesc& S = sys[bm.x];
    const int mode = S.st->mode;
    if (mode == MODE_DONE || S.n_chunks < 2 || S.sched == GSE_SCHEDULE_ROWS) return;
    Epi e;
    if (mode == MODE_ITER) {
        e.kind = EPI_CG_PQ; e.y = S.q; e.b = nullptr; e.p = S.p;
    } else {
        e.kind = EPI_RESID; e.y = mode == MODE_RESID_R ? S.r : S.q; e.b = S.b; e.p = nullptr;
    }
    const MatView m = S.m;
    const int64_t tid = (int64_t)bm.y * blockDim.x + threadIdx.x, nt = (int64_t)S.nblk_vec * blockDim.x;
    if (S.upl == 1) fix_split_rows<256>(m, e, S.n_chunks, tid, nt);
    else fix_split_rows<512>(m, e, S.n_chunks, tid, nt);
}

// ---- P2: residual update, history, policy, next mode ----------------------

// Metrics of Eqs. 3-6 over the ring (oldest .. newest = t + 1 entries), with the
// block's threads; results valid in thread 0.
__device__ void ring_metrics(const double* ring, int t, int hpos, double* red, double* rsd, int* ndec,
                             double* reldec) {
    const int cap = t + 1;
    double s = 0.0;
    for (int i = threadIdx.x; i < t; i += blockDim.x) s += ring[(hpos + i) % cap];
    s = block_sum(s, red);
    __shared__ double avg_sh;
    if (threadIdx.x == 0) avg_sh = s / t;
    __syncthreads();
    const double avg = avg_sh;
    double v = 0.0, nd = 0.0;
    for (int i = threadIdx.x; i < t; i += blockDim.x) {
        const double a = ring[(hpos + i) % cap], b = ring[(hpos + i + 1) % cap];
        v += (a - avg) * (a - avg);
        nd += a > b ? 1.0 : 0.0;
    }
    v = block_sum(v, red);
    nd = block_sum(nd, red);
    if (threadIdx.x == 0) {
        *rsd = sqrt(v / t) / avg;
        *ndec = (int)nd;
        const double first = ring[hpos % cap], prev = ring[(hpos + t - 1) % cap];
        *reldec = (first - prev) / first;
    }
}

__device__ __forceinline__ bool conditions(const CgParams& P, double rsd, int ndec, double reldec) {
    const double thr = P.ndec_limit > 0 ? (double)P.ndec_limit : 0.5 * P.t;
    const bool c1 = rsd > P.rsd_limit && (double)ndec < thr;
    const bool c2 = (double)ndec >= thr && reldec < P.reldec_limit;
    const bool c3 = ndec == 0;
    return c1 || c2 || c3;
}

__device__ __forceinline__ void step_level(CgState* st) {
    st->k = st->k + 1;
    st->sw[st->k - 1] = st->j;
}

__global__ void __launch_bounds__(256) k_cg_p2(const SysDesc* __restrict__ sys, const int2* __restrict__ map) {
    __shared__ double red[32];
    __shared__ int need_metrics;
    __shared__ double m_rsd, m_reldec;
    __shared__ int m_ndec;
    const int2 bm = map[blockIdx.x];
    const SysDesc& S = sys[bm.x];
    CgState* st = S.st;
    const int mode = st->mode;
    if (mode == MODE_DONE) return;
    const int lb = bm.y, nblk = S.nblk_vec;
    const int64_t n = S.n;
    double acc = 0.0, alpha = 0.0;
    bool brk = false;
    const int64_t t0 = (int64_t)lb * blockDim.x + threadIdx.x, di = (int64_t)nblk * blockDim.x;
    if (mode == MODE_ITER) {
        alpha = st->alpha;
        brk = st->brk != 0;
        if (!brk) {
            double* __restrict__ r = S.r;
            const double* __restrict__ q = S.q;
            int64_t i0 = 0;
            if (S.vec2) {
                // pairs of elements (16-byte loads), two pairs in flight per thread
                const int64_t n2 = n >> 1;
                double2* __restrict__ r2 = reinterpret_cast<double2*>(r);
                const double2* __restrict__ q2 = reinterpret_cast<const double2*>(q);
                int64_t i = t0;
                for (; i + di < n2; i += 2 * di) {
                    const double2 ra = r2[i], qa = q2[i], rb = r2[i + di], qb = q2[i + di];
                    const double2 na = make_double2(fma(-alpha, qa.x, ra.x), fma(-alpha, qa.y, ra.y));
                    const double2 nb = make_double2(fma(-alpha, qb.x, rb.x), fma(-alpha, qb.y, rb.y));
                    r2[i] = na;
                    r2[i + di] = nb;
                    acc = fma(na.x, na.x, acc);
                    acc = fma(na.y, na.y, acc);
                    acc = fma(nb.x, nb.x, acc);
                    acc = fma(nb.y, nb.y, acc);
                }
                if (i < n2) {
                    const double2 ra = r2[i], qa = q2[i];
                    const double2 na = make_double2(fma(-alpha, qa.x, ra.x), fma(-alpha, qa.y, ra.y));
                    r2[i] = na;
                    acc = fma(na.x, na.x, acc);
                    acc = fma(na.y, na.y, acc);
                }
                i0 = 2 * n2;
            }
            // the scalar loop: every element, or (pairs above) an odd last one
            const int64_t s0 = S.vec2 ? (t0 == 0 ? i0 : n) : t0;
            for (int64_t i = s0; i < n; i += di) {
                const double ri = fma(-alpha, q[i], r[i]);
                r[i] = ri;
                acc = fma(ri, ri, acc);
            }
        }
    } else {
        const double* __restrict__ v = mode == MODE_RESID_R ? S.r : S.q;
        for (int64_t i = t0; i < n; i += di) acc = fma(v[i], v[i], acc);
    }
    double total;
    if (!sys_grid_sum(acc, S.partial, S.counter + 1, lb, nblk, red, &total)) return;
    // ---- last block of this system: the decisions ----
    // The state and parameters are brought into shared memory with one
    // parallel load, decided on there, and written back with one parallel
    // store: no chain of dependent global round trips in the serial part.
    __shared__ CgState ss;
    __shared__ CgParams sp;
    static_assert(sizeof(CgState) % 8 == 0 && sizeof(CgParams) % 8 == 0, "word copies");
    constexpr int NS = sizeof(CgState) / 8, NP = sizeof(CgParams) / 8;
    if (threadIdx.x < NS) reinterpret_cast<long long*>(&ss)[threadIdx.x] = __ldcg(reinterpret_cast<const long long*>(S.st) + threadIdx.x);
    else if (threadIdx.x < NS + NP)
        reinterpret_cast<long long*>(&sp)[threadIdx.x - NS] = reinterpret_cast<const long long*>(&S.prm)[threadIdx.x - NS];
    __syncthreads();
    st = &ss;
    const CgParams& P = sp;
    if (threadIdx.x == 0) {
        need_metrics = 0;
        if (mode == MODE_ITER) {
            st->alpha = alpha;
            if (brk) {
                const double pq = st->pq;
                if (!isfinite(pq) || !isfinite(alpha)) {
                    st->mode = MODE_DONE; st->status = GSE_NONFINITE; st->p_action = PA_NONE;
                } else if (st->k < P.kmax) {
                    step_level(st); st->mode = MODE_RESID_R; st->p_action = PA_NONE;
                } else {
                    st->mode = MODE_DONE; st->status = GSE_BREAKDOWN; st->p_action = PA_NONE;
                }
            } else {
                const double res = sqrt(total) / st->nb;
                st->j = st->j + 1;
                st->res = res;
                const int cap = P.t + 1;
                S.ring[st->hpos] = res;
                st->hpos = (st->hpos + 1) % cap;
                if (st->hlen < cap) st->hlen = st->hlen + 1;
                st->p_action = PA_XONLY;
                if (!isfinite(res)) {
                    st->mode = MODE_DONE; st->status = GSE_NONFINITE; st->p_action = PA_NONE;
                } else if (res < P.tol) {
                    st->mode = MODE_RESID_T;
                } else {
                    // the floor rule (GSE_POLICY_FLOOR) is decided in P3, which
                    // forms x_j; every outcome decided here leaves it to P3
                    if (st->k < P.kmax && !(P.flags & GSE_POLICY_NO_STAGNATION) && P.m > 0 &&
                        st->j >= P.l && st->j % P.m == 0 && st->hlen >= cap)
                        need_metrics = 1;
                    if (!need_metrics) {
                        if (st->j >= P.max_iter) {
                            st->mode = MODE_DONE; st->status = GSE_MAXITER;
                        } else {
                            st->beta = total / st->rho; st->rho = total; st->p_action = PA_UPDATE;
                        }
                    }
                }
                st->pq = total;   // keep rho' until the metrics decide
            }
        } else if (mode == MODE_RESID_R) {
            st->rho = total;
            st->res = sqrt(total) / st->nb;
            st->hlen = 0; st->hpos = 0;
            if (st->res < P.tol) {
                if (st->k >= P.kmax) { st->mode = MODE_DONE; st->status = GSE_OK; st->true_res = st->res; st->p_action = PA_NONE; }
                else { st->mode = MODE_RESID_T; st->p_action = PA_NONE; }
            } else {
                st->mode = MODE_ITER; st->p_action = PA_COPY_R;
            }
        } else {  // MODE_RESID_T
            const double tr = sqrt(total) / st->nb;
            st->true_res = tr;
            if (tr < P.tol) {
                st->mode = MODE_DONE; st->status = GSE_OK; st->p_action = PA_NONE;
            } else {
                if (st->k < P.kmax) step_level(st);
                if (st->k >= P.kmax) {
                    st->rho = total; st->res = tr; st->hlen = 0; st->hpos = 0;
                    st->mode = MODE_ITER; st->p_action = PA_COPY_Q;
                } else {
                    st->mode = MODE_RESID_R; st->p_action = PA_NONE;
                }
                if (st->j >= P.max_iter) { st->mode = MODE_DONE; st->status = GSE_MAXITER; st->p_action = PA_NONE; }
            }
        }
    }
    __syncthreads();
    if (need_metrics) {
        ring_metrics(S.ring, P.t, st->hpos, red, &m_rsd, &m_ndec, &m_reldec);
        if (threadIdx.x == 0) {
            const double rho_new = st->pq;
            if (conditions(P, m_rsd, m_ndec, m_reldec)) {
                step_level(st); st->mode = MODE_RESID_R;
            } else if (st->j >= P.max_iter) {
                st->mode = MODE_DONE; st->status = GSE_MAXITER;
            } else {
                st->beta = rho_new / st->rho; st->rho = rho_new; st->p_action = PA_UPDATE;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x < NS) reinterpret_cast<long long*>(S.st)[threadIdx.x] = reinterpret_cast<const long long*>(&ss)[threadIdx.x];
}

// ---- P3: x and p updates --------------------------------------------------

// x += alpha p (and p = r + beta p when upd) over the block's share, element
// pairs when the vectors allow it; with FLOOR, returns the block's share of
// ||x_j||^2 of the x it stores.
template <bool FLOOR>
__device__ __forceinline__ double p3_update(const SysDesc& S, bool upd, double alpha, double beta, int64_t i0,
                                            int64_t di) {
    const int64_t n = S.n;
    double* __restrict__ x = S.x;
    double* __restrict__ p = S.p;
    const double* __restrict__ r = S.r;
    double xacc = 0.0;
    int64_t j0 = 0;
    if (S.vec2) {
        // pairs of elements (16-byte loads), two pairs in flight per thread
        const int64_t n2 = n >> 1;
        double2* __restrict__ x2 = reinterpret_cast<double2*>(x);
        double2* __restrict__ p2 = reinterpret_cast<double2*>(p);
        const double2* __restrict__ r2 = reinterpret_cast<const double2*>(r);
        int64_t i = i0;
        for (; i + di < n2; i += 2 * di) {
            const double2 pa2 = p2[i], xa = x2[i], pb = p2[i + di], xb = x2[i + di];
            const double2 na = make_double2(fma(alpha, pa2.x, xa.x), fma(alpha, pa2.y, xa.y));
            const double2 nb = make_double2(fma(alpha, pb.x, xb.x), fma(alpha, pb.y, xb.y));
            x2[i] = na;
            x2[i + di] = nb;
            if constexpr (FLOOR) {
                xacc = fma(na.x, na.x, xacc);
                xacc = fma(na.y, na.y, xacc);
                xacc = fma(nb.x, nb.x, xacc);
                xacc = fma(nb.y, nb.y, xacc);
            }
            if (upd) {
                const double2 ra = r2[i], rb = r2[i + di];
                p2[i] = make_double2(fma(beta, pa2.x, ra.x), fma(beta, pa2.y, ra.y));
                p2[i + di] = make_double2(fma(beta, pb.x, rb.x), fma(beta, pb.y, rb.y));
            }
        }
        if (i < n2) {
            const double2 pa2 = p2[i], xa = x2[i];
            const double2 na = make_double2(fma(alpha, pa2.x, xa.x), fma(alpha, pa2.y, xa.y));
            x2[i] = na;
            if constexpr (FLOOR) {
                xacc = fma(na.x, na.x, xacc);
                xacc = fma(na.y, na.y, xacc);
            }
            if (upd) {
                const double2 ra = r2[i];
                p2[i] = make_double2(fma(beta, pa2.x, ra.x), fma(beta, pa2.y, ra.y));
            }
        }
        j0 = 2 * n2;
    }
    // the scalar loop: every element, or (pairs above) an odd last one
    for (int64_t i = S.vec2 ? (i0 == 0 ? j0 : n) : i0; i < n; i += di) {
        const double pi = p[i];
        const double xi = fma(alpha, pi, x[i]);
        x[i] = xi;
        if constexpr (FLOOR) xacc = fma(xi, xi, xacc);
        if (upd) p[i] = fma(beta, pi, r[i]);
    }
    return xacc;
}

__global__ void __launch_bounds__(256, 5) k_cg_p3(const SysDesc* __restrict__ sys, const int2* __restrict__ map) {
    const int2 bm = map[blockIdx.x];
    const SysDesc& S = sys[bm.x];
    CgState* st = S.st;
    const int pa = st->p_action;
    if (pa == PA_NONE) return;
    const int lb = bm.y, nblk = S.nblk_vec;
    const int64_t n = S.n;
    const double alpha = st->alpha, beta = st->beta;
    double* __restrict__ x = S.x;
    double* __restrict__ p = S.p;
    double* __restrict__ r = S.r;
    const double* __restrict__ q = S.q;
    const int64_t i0 = (int64_t)lb * blockDim.x + threadIdx.x, di = (int64_t)nblk * blockDim.x;
    // The floor rule (GSE_POLICY_FLOOR, checked before the stagnation test in
    // the iteration's order) compares res_j with eta_k ||x_j|| / ||b||, x_j the
    // iterate this pass stores.  It is due when P2 let the iteration continue
    // (p is updated) or stopped it at max_iter; a stagnation step, a
    // convergence check or a breakdown decided in P2 comes first.  Uniform
    // over the system's blocks (all read the same state).
    const bool floor_due = (S.prm.flags & GSE_POLICY_FLOOR) && st->k < S.prm.kmax &&
                           (pa == PA_UPDATE || (pa == PA_XONLY && st->mode == MODE_DONE && st->status == GSE_MAXITER));
    if (floor_due) {
        const double xacc = p3_update<true>(S, pa == PA_UPDATE, alpha, beta, i0, di);
        __shared__ double red[32];
        double total_x;
        if (!sys_grid_sum(xacc, S.partial, S.counter + 2, lb, nblk, red, &total_x)) return;
        if (threadIdx.x == 0) {
            st->p_action = PA_NONE;
            if (total_x > 0.0 && st->res <= S.prm.eta[st->k] * sqrt(total_x) / st->nb) {
                step_level(st);
                if (st->mode != MODE_DONE) st->mode = MODE_RESID_R;   // at max_iter: the level only
            }
        }
        return;
    }
    if (pa == PA_UPDATE || pa == PA_XONLY) {
        p3_update<false>(S, pa == PA_UPDATE, alpha, beta, i0, di);
    } else if (pa == PA_COPY_R) {
        for (int64_t i = i0; i < n; i += di) p[i] = r[i];
    } else if (pa == PA_COPY_Q) {
        for (int64_t i = i0; i < n; i += di) {
            const double v = q[i];
            r[i] = v;
            p[i] = v;
        }
    } else {
        for (int64_t i = i0; i < n; i += di) x[i] = 0.0;
    }
    if (!sys_grid_last(S.counter + 2, nblk)) return;
    if (threadIdx.x == 0) st->p_action = PA_NONE;
}

// ---- P0: ||b|| and the initial state --------------------------------------

__global__ void __launch_bounds__(256) k_cg_init(const SysDesc* __restrict__ sys, const int2* __restrict__ map) {
    __shared__ double red[32];
    const int2 bm = map[blockIdx.x];
    const SysDesc& S = sys[bm.x];
    CgState* st = S.st;
    if (st->mode != MODE_RESID_R || st->j != -1) return;   // only freshly submitted systems
    const int lb = bm.y, nblk = S.nblk_vec;
    double acc = 0.0;
    for (int64_t i = (int64_t)lb * blockDim.x + threadIdx.x; i < S.n; i += (int64_t)nblk * blockDim.x)
        acc = fma(S.b[i], S.b[i], acc);
    double total;
    if (!sys_grid_sum(acc, S.partial, S.counter + 1, lb, nblk, red, &total)) return;
    if (threadIdx.x == 0) {
        st->nb = sqrt(total);
        st->j = 0;
        if (!(total > 0.0)) {
            st->mode = MODE_DONE; st->status = isfinite(total) ? GSE_OK : GSE_NONFINITE;
            st->res = 0.0; st->true_res = 0.0; st->p_action = PA_ZERO_X;
        } else if (!isfinite(total)) {
            st->mode = MODE_DONE; st->status = GSE_NONFINITE; st->p_action = PA_NONE;
        }
    }
}

// ---- floor coefficients (GSE_POLICY_FLOOR) --------------------------------
// eta_k = max_i sum_j |a3_ij - ak_ij|: the infinity norm of the truncation
// A_kmax - A_k, so that ||(A_kmax - A_k) x|| <~ eta_k ||x||.
__global__ void k_row_absdiff_max(const int32_t* row_ptr, int64_t n, const double* a, const double* b,
                                  unsigned long long* out) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int32_t e = row_ptr[r]; e < row_ptr[r + 1]; e++) s += fabs(a[e] - b[e]);
        atomicMax(out, (unsigned long long)__double_as_longlong(s));
    }
}

}  // namespace gse

using namespace gse;

// ---- workspace --------------------------------------------------------------

void gse_free_workspace(gse_matrix* h) {
    if (!h->ws) return;
    Workspace* w = h->ws;
    void* bufs[] = {w->r, w->p, w->q, w->ring, w->partial, w->counter, w->V, w->gm_scratch};
    for (void* b : bufs) pool_free(b);
    if (w->gm_host) cudaFreeHost(w->gm_host);
    delete w;
    h->ws = nullptr;
    h->bytes_ws = 0;
}

static int ensure_cg_workspace(gse_matrix* h, cudaStream_t s) {
    if (!h->ws) h->ws = new Workspace();
    Workspace* w = h->ws;
    const int64_t n = h->v.n_rows;
    if (!w->r) {
        size_t acc = 0;
        if (pool_alloc(&w->r, (size_t)n + 1, &acc, s) != GSE_OK || pool_alloc(&w->p, (size_t)n + 1, &acc, s) != GSE_OK ||
            pool_alloc(&w->q, (size_t)n + 1, &acc, s) != GSE_OK)
            return GSE_ERR_OOM;
        h->bytes_ws += acc;
        w->n = n;
    }
    if (!w->ring) {
        if (pool_alloc(&w->ring, RING_MAX + 1, &h->bytes_ws, s) != GSE_OK) return GSE_ERR_OOM;
    }
    if (!w->partial) {
        w->partial_cap = h->num_sms * 64;
        if (pool_alloc(&w->partial, (size_t)w->partial_cap, &h->bytes_ws, s) != GSE_OK ||
            pool_alloc(&w->counter, 8, &h->bytes_ws, s) != GSE_OK)
            return GSE_ERR_OOM;
        cudaMemsetAsync(w->counter, 0, 8 * sizeof(unsigned), s);
    }
    return GSE_OK;
}

extern "C" size_t gse_solve_footprint(gse_handle h, int method, int restart) {
    if (!h) return 0;
    const size_t n = (size_t)h->v.n_rows + 1;
    size_t ws = 3 * n * sizeof(double) + (RING_MAX + 1) * sizeof(double) + (size_t)h->num_sms * 64 * sizeof(double);
    if (method == 1) ws += (size_t)(restart + 2) * n * sizeof(double);
    return h->bytes_matrix + ws;
}

static int compute_eta(gse_matrix* h, int kmax, cudaStream_t s) {
    Workspace* w = h->ws;
    if (w->eta_ready) return GSE_OK;
    if (kmax < 1 || kmax > h->n_seg) return GSE_OK;
    const int64_t nnz = h->v.nnz;
    double *a = nullptr, *b = nullptr;
    unsigned long long* d = nullptr;
    if (cudaMalloc(&a, (nnz + 1) * sizeof(double)) != cudaSuccess || cudaMalloc(&b, (nnz + 1) * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&d, 4 * sizeof(unsigned long long)) != cudaSuccess) {
        cudaGetLastError();
        if (a) cudaFree(a);
        if (b) cudaFree(b);
        return GSE_ERR_OOM;
    }
    gse_decode(h, kmax, b, s);
    for (int k = 1; k < kmax; k++) {
        gse_decode(h, k, a, s);
        cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
        k_row_absdiff_max<<<1024, 256, 0, s>>>(h->v.row_ptr, h->v.n_rows, b, a, d);
        unsigned long long bits = 0;
        cudaMemcpyAsync(&bits, d, sizeof(bits), cudaMemcpyDeviceToHost, s);
        cudaStreamSynchronize(s);
        double e;
        memcpy(&e, &bits, sizeof(e));
        w->eta[k] = e;
    }
    cudaFree(a);
    cudaFree(b);
    cudaFree(d);
    w->eta_ready = true;
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

// ---- the engine (host side) --------------------------------------------------

struct EngineSlot {
    bool active = false;
    bool done_reported = true;
    gse_matrix* h = nullptr;
    std::chrono::steady_clock::time_point t0;
    int status_final = 0;
};

struct gse_cg_engine {
    int capacity = 0;
    cudaStream_t user = nullptr;    // the caller's stream: each call starts after its work and ends before its next
    cudaStream_t stream = nullptr;  // the engine's own stream (capturable; all engine work runs here)
    cudaEvent_t join = nullptr;
    // a batch of iteration slots captured once as a CUDA graph and replayed
    // (re-captured when the set of systems changes)
    cudaGraphExec_t graph = nullptr;
    int graph_slots = 0;
    bool graph_ok = true;
    int device = 0;
    int num_sms = 1;
    SysDesc* d_sys = nullptr;
    CgState* d_state = nullptr;
    CgState* h_state = nullptr;    // pinned mirror (latest completed batch)
    CgState* h_stage[2] = {nullptr, nullptr};  // pinned landing buffers, one per batch in flight
    int2* d_map_spmv = nullptr;     // P1 blocks of nonzero-split systems
    int2* d_map_rows = nullptr;     // P1 blocks of row-schedule systems (staged row kernel)
    int2* d_map_lr = nullptr;       // P1 blocks of lane-row systems
    int map_cap_lr = 0, nblk_lr = 0;
    int solo_lr = -1;               // the slot, when the lane-row blocks all belong to one system
    size_t lr_smem = 0;             // dynamic shared memory of the lane-row P1 launch (widest system)
    int2* d_map_vec = nullptr;
    int map_cap_spmv = 0, map_cap_rows = 0, map_cap_vec = 0;
    int nblk_spmv = 0, nblk_rows = 0, nblk_vec = 0;
    size_t rows_smem = 0;           // dynamic shared memory of the row P1 launch (widest system)
    std::vector<EngineSlot> slots;
    std::vector<SysDesc> h_sys;
    bool dirty = true;
    bool fresh = false;
    bool pending = false;           // a gse_engine_launch whose state copy is not yet waited for
    cudaEvent_t ev[2];
};


// Every engine call other than gse_engine_launch first settles a launch still
// in flight (gse_engine_wait), so host and device views of the states agree.
extern "C" int gse_engine_wait(gse_engine e, int* n_running);
#define ENGINE_SETTLE(e)                                      \
    do {                                                      \
        if ((e)->pending) {                                   \
            const int _rc = gse_engine_wait((e), nullptr);    \
            if (_rc != GSE_OK) return _rc;                    \
        }                                                     \
    } while (0)

// The engine's stream waits for the caller's stream (its b and x are ready) ...
static void engine_enter(gse_cg_engine* e) {
    cudaEventRecord(e->join, e->user);
    cudaStreamWaitEvent(e->stream, e->join, 0);
}
// ... and the caller's stream waits for the engine's work.
static void engine_leave(gse_cg_engine* e) {
    cudaEventRecord(e->join, e->stream);
    cudaStreamWaitEvent(e->user, e->join, 0);
}

extern "C" int gse_engine_create(int capacity, void* stream, gse_engine* out) {
    if (capacity < 1 || !out) return GSE_ERR_INVALID;
    gse_cg_engine* e = new gse_cg_engine();
    e->capacity = capacity;
    e->user = (cudaStream_t)stream;
    if (cudaStreamCreateWithFlags(&e->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&e->join, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        delete e;
        return GSE_ERR_CUDA;
    }
    cudaGetDevice(&e->device);
    cudaDeviceGetAttribute(&e->num_sms, cudaDevAttrMultiProcessorCount, e->device);
    p1_occupancy(P1_SPLIT, p1_smem());  // sets the P1 kernels' shared-memory limits on this device
    p1_occupancy(P1_ROWS, p1_rows_smem_max());
    p1_lr_occupancy(0);                 // sets the lane-row P1 kernel's shared-memory limit on this device
    e->slots.resize(capacity);
    e->h_sys.resize(capacity);
    if (cudaMalloc(&e->d_sys, capacity * sizeof(SysDesc)) != cudaSuccess ||
        cudaMalloc(&e->d_state, capacity * sizeof(CgState)) != cudaSuccess ||
        cudaMallocHost(&e->h_state, capacity * sizeof(CgState)) != cudaSuccess ||
        cudaMallocHost(&e->h_stage[0], capacity * sizeof(CgState)) != cudaSuccess ||
        cudaMallocHost(&e->h_stage[1], capacity * sizeof(CgState)) != cudaSuccess) {
        cudaGetLastError();
        gse_engine_destroy(e);
        return GSE_ERR_OOM;
    }
    memset(e->h_state, 0, capacity * sizeof(CgState));
    cudaEventCreateWithFlags(&e->ev[0], cudaEventDisableTiming);
    cudaEventCreateWithFlags(&e->ev[1], cudaEventDisableTiming);
    *out = e;
    return GSE_OK;
}

extern "C" void gse_engine_destroy(gse_engine e) {
    if (!e) return;
    cudaStreamSynchronize(e->stream);
    if (e->graph) cudaGraphExecDestroy(e->graph);
    cudaStreamDestroy(e->stream);
    if (e->join) cudaEventDestroy(e->join);
    if (e->d_sys) cudaFree(e->d_sys);
    if (e->d_state) cudaFree(e->d_state);
    if (e->h_state) cudaFreeHost(e->h_state);
    if (e->h_stage[0]) cudaFreeHost(e->h_stage[0]);
    if (e->h_stage[1]) cudaFreeHost(e->h_stage[1]);
    if (e->d_map_spmv) cudaFree(e->d_map_spmv);
    if (e->d_map_rows) cudaFree(e->d_map_rows);
    if (e->d_map_lr) cudaFree(e->d_map_lr);
    if (e->d_map_vec) cudaFree(e->d_map_vec);
    if (e->ev[0]) cudaEventDestroy(e->ev[0]);
    if (e->ev[1]) cudaEventDestroy(e->ev[1]);
    delete e;
}

static bool level_valid(const gse_matrix* h, int k) { return level_available(h, k); }

extern "C" int gse_engine_submit(gse_engine e, gse_handle h, const double* b, double* x, double tol,
                                 const gse_step_policy* pol, int* slot_out) {
    if (!e || !h || !b || !x || !pol || !(tol > 0)) return GSE_ERR_INVALID;
    if (!level_valid(h, pol->k_start) || !level_valid(h, pol->k_max)) return GSE_ERR_INVALID;
    ENGINE_SETTLE(e);
    const bool base = pol->k_start > 3 || pol->k_max > 3;
    if (base && pol->k_start != pol->k_max) return GSE_ERR_INVALID;
    if (!base && pol->k_start > pol->k_max) return GSE_ERR_INVALID;
    if (pol->t < 1 || pol->t > RING_MAX - 1 || pol->max_iter < 1) return GSE_ERR_INVALID;
    int slot = -1;
    for (int i = 0; i < e->capacity; i++)
        if (e->slots[i].active && e->slots[i].h == h) return GSE_ERR_INVALID;  // one workspace per handle
    for (int i = 0; i < e->capacity; i++)
        if (!e->slots[i].active && e->slots[i].done_reported) { slot = i; break; }
    if (slot < 0) return GSE_ERR_INVALID;
    engine_enter(e);
    int rc = ensure_cg_workspace(h, e->stream);
    if (rc != GSE_OK) return rc;
    cudaMemsetAsync(h->d_err, 0, sizeof(int), e->stream);   // this solve's bounded-wait record starts clear
    if ((pol->flags & GSE_POLICY_FLOOR) && !base) {
        rc = compute_eta(h, pol->k_max, e->stream);
        if (rc != GSE_OK) return rc;
    }
    Workspace* w = h->ws;
    SysDesc d;
    memset(&d, 0, sizeof(d));
    d.m = h->v;
    d.err = h->d_err;
    sys_partition(d, h, e->num_sms, pol->k_start, pol->k_max);
    if (d.nblk_spmv > w->partial_cap || d.nblk_vec > w->partial_cap) return GSE_ERR_INVALID;
    d.b = b;
    d.x = x;
    d.r = w->r;
    d.p = w->p;
    d.q = w->q;
    d.vec2 = vec2_aligned(d.x, d.r, d.p, d.q);
    d.ring = w->ring;
    d.st = e->d_state + slot;
    d.partial = w->partial;
    d.counter = w->counter;
    d.prm.l = pol->l;
    d.prm.t = pol->t;
    d.prm.m = pol->m;
    d.prm.ndec_limit = pol->ndec_limit;
    d.prm.max_iter = pol->max_iter;
    d.prm.flags = pol->flags;
    d.prm.kstart = pol->k_start;
    d.prm.kmax = pol->k_max;
    d.prm.rsd_limit = pol->rsd_limit;
    d.prm.reldec_limit = pol->reldec_limit;
    d.prm.tol = tol;
    for (int i = 0; i < 4; i++) d.prm.eta[i] = w->eta[i];
    e->h_sys[slot] = d;
    CgState s0;
    memset(&s0, 0, sizeof(s0));
    s0.mode = MODE_RESID_R;
    s0.k = pol->k_start;
    s0.j = -1;  // marks "needs init"
    s0.status = GSE_MAXITER;
    for (int i = 0; i < 4; i++) s0.sw[i] = -1;
    if (!base) s0.sw[pol->k_start - 1] = 0;
    e->h_state[slot] = s0;
    cudaMemcpyAsync(e->d_sys + slot, &e->h_sys[slot], sizeof(SysDesc), cudaMemcpyHostToDevice, e->stream);
    cudaMemcpyAsync(e->d_state + slot, &e->h_state[slot], sizeof(CgState), cudaMemcpyHostToDevice, e->stream);
    cudaStreamSynchronize(e->stream);   // pageable/pinned sources stay valid; cheap and rare
    e->slots[slot].active = true;
    e->slots[slot].done_reported = false;
    e->slots[slot].h = h;
    e->slots[slot].t0 = std::chrono::steady_clock::now();
    e->dirty = true;
    e->fresh = true;
    if (slot_out) *slot_out = slot;
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

static int rebuild_maps(gse_cg_engine* e) {
    std::vector<int2> ms, mr, ml, mv;
    size_t rsm = 0;
    size_t lsm = 0;
    for (int i = 0; i < e->capacity; i++) {
        if (!e->slots[i].active) continue;
        const SysDesc& d = e->h_sys[i];
        const bool rows = d.sched == GSE_SCHEDULE_ROWS && !d.lanerow;
        if (rows && p1_rows_smem(d.row_span, d.m.r_lo) > rsm) rsm = p1_rows_smem(d.row_span, d.m.r_lo);
        if (d.lanerow && (size_t)d.lr_smem > lsm) lsm = (size_t)d.lr_smem;
        for (int b = 0; b < d.nblk_spmv; b++) (d.lanerow ? ml : rows ? mr : ms).push_back(make_int2(i, b));
        for (int b = 0; b < d.nblk_vec; b++) mv.push_back(make_int2(i, b));
    }
    auto grow = [](int2** buf, int* cap, size_t need) -> int {
        if ((size_t)*cap >= need) return GSE_OK;
        if (*buf) cudaFree(*buf);
        size_t c = need + need / 2 + 16;
        if (cudaMalloc(buf, c * sizeof(int2)) != cudaSuccess) { cudaGetLastError(); *buf = nullptr; *cap = 0; return GSE_ERR_OOM; }
        *cap = (int)c;
        return GSE_OK;
    };
    cudaStreamSynchronize(e->stream);
    int rc = grow(&e->d_map_spmv, &e->map_cap_spmv, ms.size());
    if (rc == GSE_OK) rc = grow(&e->d_map_rows, &e->map_cap_rows, mr.size());
    if (rc == GSE_OK) rc = grow(&e->d_map_lr, &e->map_cap_lr, ml.size());
    if (rc == GSE_OK) rc = grow(&e->d_map_vec, &e->map_cap_vec, mv.size());
    if (rc != GSE_OK) return rc;
    if (!ms.empty()) cudaMemcpy(e->d_map_spmv, ms.data(), ms.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (!mr.empty()) cudaMemcpy(e->d_map_rows, mr.data(), mr.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (!ml.empty()) cudaMemcpy(e->d_map_lr, ml.data(), ml.size() * sizeof(int2), cudaMemcpyHostToDevice);
    if (!mv.empty()) cudaMemcpy(e->d_map_vec, mv.data(), mv.size() * sizeof(int2), cudaMemcpyHostToDevice);
    e->nblk_spmv = (int)ms.size();
    e->nblk_rows = (int)mr.size();
    e->nblk_lr = (int)ml.size();
    e->solo_lr = !ml.empty() && ml.front().x == ml.back().x ? ml.front().x : -1;
    e->lr_smem = lsm;
    e->nblk_vec = (int)mv.size();
    e->rows_smem = rsm;
    e->dirty = false;
    if (e->graph) {
        cudaGraphExecDestroy(e->graph);
        e->graph = nullptr;
    }
    return GSE_OK;
}

static void enqueue_slots(gse_cg_engine* e, int nslots) {
    for (int it = 0; it < nslots; it++) {
        if (e->nblk_lr && e->solo_lr >= 0)
            k_cg_p1_lr_solo<<<e->nblk_lr, ENG_LR_WARPS * 32, e->lr_smem, e->stream>>>(e->h_sys[e->solo_lr].m,
                                                                                     e->d_sys + e->solo_lr);
        else if (e->nblk_lr)
            k_cg_p1_lr<<<e->nblk_lr, ENG_LR_WARPS * 32, e->lr_smem, e->stream>>>(e->d_sys, e->d_map_lr);
        if (e->nblk_rows)
            k_cg_p1_rows<<<e->nblk_rows, ENG_ROW_WARPS * 32, e->rows_smem, e->stream>>>(e->d_sys, e->d_map_rows);
        if (e->nblk_spmv) {
            k_cg_p1<<<e->nblk_spmv, ENG_WARPS * 32, p1_smem(), e->stream>>>(e->d_sys, e->d_map_spmv);
            k_cg_fix<<<e->nblk_vec, 256, 0, e->stream>>>(e->d_sys, e->d_map_vec);   // split rows (nonzero split only)
        }
        k_cg_p2<<<e->nblk_vec, 256, 0, e->stream>>>(e->d_sys, e->d_map_vec);
        k_cg_p3<<<e->nblk_vec, 256, 0, e->stream>>>(e->d_sys, e->d_map_vec);
    }
}

// Runs nslots iteration slots: a full batch from the captured graph (captured
// on first use), anything else launched directly.
static void run_slots(gse_cg_engine* e, int nslots, int batch) {
    if (nslots == batch && e->graph_ok) {
        if (!e->graph || e->graph_slots != batch) {
            if (e->graph) {
                cudaGraphExecDestroy(e->graph);
                e->graph = nullptr;
            }
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(e->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                enqueue_slots(e, nslots);
                if (cudaStreamEndCapture(e->stream, &g) == cudaSuccess && g &&
                    cudaGraphInstantiate(&e->graph, g, 0) == cudaSuccess) {
                    e->graph_slots = batch;
                } else {
                    e->graph = nullptr;
                }
                if (g) cudaGraphDestroy(g);
            }
            if (!e->graph) {             // capture unavailable: launch directly from now on
                cudaGetLastError();
                e->graph_ok = false;
            }
        }
        if (e->graph && cudaGraphLaunch(e->graph, e->stream) == cudaSuccess) return;
        cudaGetLastError();
        e->graph_ok = false;
    }
    enqueue_slots(e, nslots);
}

static bool any_running(gse_cg_engine* e) {
    for (int i = 0; i < e->capacity; i++)
        if (e->slots[i].active && e->h_state[i].mode != MODE_DONE) return true;
    return false;
}

// Advances all active systems by up to max_slots iteration slots (batches of
// `batch`, double-buffered); returns early when every active system is done.
extern "C" int gse_engine_run(gse_engine e, int max_slots, int batch, int* n_running) {
    if (!e || max_slots < 0) return GSE_ERR_INVALID;
    ENGINE_SETTLE(e);
    if (batch < 1) batch = 8;
    engine_enter(e);
    if (e->dirty) {
        const int rc = rebuild_maps(e);
        if (rc != GSE_OK) return rc;
    }
    if (e->nblk_vec == 0) {
        if (n_running) *n_running = 0;
        return GSE_OK;
    }
    if (e->fresh) {
        k_cg_init<<<e->nblk_vec, 256, 0, e->stream>>>(e->d_sys, e->d_map_vec);
        k_cg_p3<<<e->nblk_vec, 256, 0, e->stream>>>(e->d_sys, e->d_map_vec);  // zero x for b = 0
        e->fresh = false;
    }
    const size_t sbytes = e->capacity * sizeof(CgState);
    int done_slots = 0, inflight = 0, cur = 0;
    bool running = true;
    while (done_slots < max_slots && running) {
        const int nb = max_slots - done_slots < batch ? max_slots - done_slots : batch;
        run_slots(e, nb, batch);
        done_slots += nb;
        cudaMemcpyAsync(e->h_stage[cur], e->d_state, sbytes, cudaMemcpyDeviceToHost, e->stream);
        cudaEventRecord(e->ev[cur], e->stream);
        inflight++;
        if (inflight == 2) {
            cudaEventSynchronize(e->ev[cur ^ 1]);
            memcpy(e->h_state, e->h_stage[cur ^ 1], sbytes);
            inflight = 1;
            running = any_running(e);
        }
        cur ^= 1;
    }
    cudaStreamSynchronize(e->stream);
    engine_leave(e);
    if (inflight) memcpy(e->h_state, e->h_stage[cur ^ 1], sbytes);
    running = any_running(e);
    if (cudaGetLastError() != cudaSuccess) return GSE_ERR_CUDA;
    if (n_running) {
        int c = 0;
        for (int i = 0; i < e->capacity; i++)
            if (e->slots[i].active && e->h_state[i].mode != MODE_DONE) c++;
        *n_running = c;
    }
    return GSE_OK;
}

// The asynchronous form of gse_engine_run: the slots and one copy of every
// system's state are queued on the engine's stream and the call returns; the
// host is free (to encode the next requests) until gse_engine_wait.
extern "C" int gse_engine_launch(gse_engine e, int max_slots, int batch) {
    if (!e || max_slots < 0) return GSE_ERR_INVALID;
    if (batch < 1) batch = 8;
    ENGINE_SETTLE(e);
    engine_enter(e);
    if (e->dirty) {
        const int rc = rebuild_maps(e);
        if (rc != GSE_OK) return rc;
    }
    if (e->nblk_vec == 0) return GSE_OK;
    if (e->fresh) {
        k_cg_init<<<e->nblk_vec, 256, 0, e->stream>>>(e->d_sys, e->d_map_vec);
        k_cg_p3<<<e->nblk_vec, 256, 0, e->stream>>>(e->d_sys, e->d_map_vec);  // zero x for b = 0
        e->fresh = false;
    }
    for (int done_slots = 0; done_slots < max_slots;) {
        const int nb = max_slots - done_slots < batch ? max_slots - done_slots : batch;
        run_slots(e, nb, batch);
        done_slots += nb;
    }
    cudaMemcpyAsync(e->h_stage[0], e->d_state, e->capacity * sizeof(CgState), cudaMemcpyDeviceToHost, e->stream);
    cudaEventRecord(e->ev[0], e->stream);
    e->pending = true;
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

extern "C" int gse_engine_wait(gse_engine e, int* n_running) {
    if (!e) return GSE_ERR_INVALID;
    if (e->pending) {
        e->pending = false;
        if (cudaEventSynchronize(e->ev[0]) != cudaSuccess) return GSE_ERR_CUDA;
        memcpy(e->h_state, e->h_stage[0], e->capacity * sizeof(CgState));
        engine_leave(e);
    }
    if (n_running) {
        int c = 0;
        for (int i = 0; i < e->capacity; i++)
            if (e->slots[i].active && e->h_state[i].mode != MODE_DONE) c++;
        *n_running = c;
    }
    return GSE_OK;
}

static void fill_info(gse_cg_engine* e, int slot, gse_solve_info* info, double rel_true) {
    const CgState& s = e->h_state[slot];
    info->status = s.mode == MODE_DONE ? s.status : GSE_MAXITER;
    int err = 0;
    cudaMemcpy(&err, e->slots[slot].h->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (err) info->status = GSE_TIMEOUT;   // a bounded device-side wait gave up
    info->iters = s.j < 0 ? 0 : s.j;
    const int base = e->h_sys[slot].prm.kmax > 3;
    info->k_final = base ? 0 : s.k;
    for (int i = 0; i < 3; i++) info->switch_iter[i] = base ? -1 : s.sw[i];
    info->rel_res_rec = s.res;
    info->rel_res_true = rel_true;
    info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - e->slots[slot].t0).count();
}

// Recomputes ||b - A_kmax x|| / ||b|| for a finished system (uses its q vector).
static double true_residual(gse_cg_engine* e, int slot) {
    const SysDesc& d = e->h_sys[slot];
    gse_matrix* h = e->slots[slot].h;
    const CgState& s = e->h_state[slot];
    if (!(s.nb > 0)) return 0.0;
    SpmvArgs a = {};
    a.x = d.x;
    a.y = d.q;
    a.b = d.b;
    launch_spmv(h, d.prm.kmax, EPI_RESID, a, e->stream);
    std::vector<double> qh((size_t)d.n);
    cudaMemcpyAsync(qh.data(), d.q, d.n * sizeof(double), cudaMemcpyDeviceToHost, e->stream);
    cudaStreamSynchronize(e->stream);
    double ss = 0.0;
    for (int64_t i = 0; i < d.n; i++) ss += qh[i] * qh[i];
    return sqrt(ss) / s.nb;
}

// Reports finished systems (slots and infos, up to max_done) and frees their slots.
extern "C" int gse_engine_poll(gse_engine e, int* done_slots, gse_solve_info* infos, int max_done, int* n_done) {
    if (!e) return GSE_ERR_INVALID;
    ENGINE_SETTLE(e);
    engine_enter(e);
    int c = 0;
    for (int i = 0; i < e->capacity && c < max_done; i++) {
        EngineSlot& sl = e->slots[i];
        if (!sl.active || e->h_state[i].mode != MODE_DONE) continue;
        gse_solve_info info;
        memset(&info, 0, sizeof(info));
        // a converged system's true residual was computed on the device when it
        // passed the check (x has not changed since); otherwise recompute it
        const CgState& st = e->h_state[i];
        const double tr = st.status == GSE_OK ? st.true_res : true_residual(e, i);
        fill_info(e, i, &info, tr);
        if (done_slots) done_slots[c] = i;
        if (infos) infos[c] = info;
        sl.active = false;
        sl.done_reported = true;
        e->dirty = true;
        c++;
    }
    if (n_done) *n_done = c;
    return GSE_OK;
}

// Cancels a slot (its system stays where it is; info reports MAXITER).
extern "C" int gse_engine_cancel(gse_engine e, int slot, gse_solve_info* info) {
    if (!e || slot < 0 || slot >= e->capacity || !e->slots[slot].active) return GSE_ERR_INVALID;
    ENGINE_SETTLE(e);
    engine_enter(e);
    cudaStreamSynchronize(e->stream);
    cudaMemcpy(&e->h_state[slot], e->d_state + slot, sizeof(CgState), cudaMemcpyDeviceToHost);
    if (info) fill_info(e, slot, info, true_residual(e, slot));
    e->slots[slot].active = false;
    e->slots[slot].done_reported = true;
    e->dirty = true;
    return GSE_OK;
}

static int solve_all(gse_cg_engine* e, int nsys, gse_solve_info* infos, int max_iter_total) {
    int running = 1;
    // generous slot budget: every restart and check costs one slot
    const int budget = max_iter_total + 64 * 4;
    int used = 0;
    while (running && used < budget) {
        const int chunk = budget - used < 256 ? budget - used : 256;
        const int rc = gse_engine_run(e, chunk, 16, &running);
        if (rc != GSE_OK) return rc;
        used += chunk;
    }
    std::vector<int> slots(nsys);
    std::vector<gse_solve_info> inf(nsys);
    int nd = 0;
    gse_engine_poll(e, slots.data(), inf.data(), nsys, &nd);
    int first_bad = GSE_OK;
    for (int i = 0; i < nd; i++) {
        if (infos) infos[slots[i]] = inf[i];
        if (inf[i].status != GSE_OK && first_bad == GSE_OK) first_bad = inf[i].status;
    }
    for (int i = 0; i < nsys; i++) {
        if (e->slots[i].active) {
            gse_solve_info info;
            gse_engine_cancel(e, i, &info);
            if (infos) infos[i] = info;
            if (first_bad == GSE_OK) first_bad = GSE_MAXITER;
        }
    }
    return first_bad;
}

extern "C" int gse_cg(gse_handle h, const double* b, double* x, double tol, const gse_step_policy* policy,
                      gse_solve_info* info, void* stream) {
    if (!h || !b || !x || !policy) return GSE_ERR_INVALID;
    const auto t0 = std::chrono::steady_clock::now();
    gse_engine e = nullptr;
    int rc = gse_engine_create(1, stream, &e);
    if (rc != GSE_OK) return rc;
    rc = gse_engine_submit(e, h, b, x, tol, policy, nullptr);
    if (rc != GSE_OK) {
        gse_engine_destroy(e);
        return rc;
    }
    gse_solve_info inf;
    memset(&inf, 0, sizeof(inf));
    rc = solve_all(e, 1, &inf, policy->max_iter);
    gse_engine_destroy(e);
    inf.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (info) *info = inf;
    return rc;
}

extern "C" int gse_batch_cg(int nsys, const gse_handle* hs, const double* const* b, double* const* x, double tol,
                            const gse_step_policy* policy, gse_solve_info* infos, void* stream) {
    if (nsys < 1 || !hs || !b || !x || !policy) return GSE_ERR_INVALID;
    gse_engine e = nullptr;
    int rc = gse_engine_create(nsys, stream, &e);
    if (rc != GSE_OK) return rc;
    for (int i = 0; i < nsys; i++) {
        rc = gse_engine_submit(e, hs[i], b[i], x[i], tol, policy, nullptr);
        if (rc != GSE_OK) {
            gse_engine_destroy(e);
            return rc;
        }
    }
    rc = solve_all(e, nsys, infos, policy->max_iter);
    gse_engine_destroy(e);
    return rc;
}
