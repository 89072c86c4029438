// solver_internal.cuh -- types of the device-resident CG engine (solver.cu)
// shared with other translation units that launch its kernels.
#pragma once

#include "spmv_lanerow.cuh"
#include "spmv_pipe.cuh"

namespace gse {

enum { MODE_ITER = 0, MODE_RESID_R = 1, MODE_RESID_T = 2, MODE_DONE = 3 };
enum { PA_NONE = 0, PA_UPDATE = 1, PA_XONLY = 2, PA_COPY_R = 3, PA_COPY_Q = 4, PA_ZERO_X = 5 };
constexpr int RING_MAX = 4096;
constexpr int ENG_WARPS = 4;
constexpr int ENG_ROW_STAGES = 2;   // stage ring of the row schedule (wide stages: fewer, more CTAs)
constexpr int ENG_ROW_WARPS = 8;    // row schedule: CTAs of 8 warps, 256-row super-blocks
constexpr int ENG_LR_WARPS = 8;     // lane-row schedule: CTAs of 8 warps, 64-row tiles per warp

struct CgState {
    int mode, k, status, j, p_action, hlen, hpos, brk;   // brk: p.Ap <= 0 or non-finite (set by P1)
    int sw[4];
    double rho, pq, alpha, beta, nb, res, true_res, pad;
};

struct CgParams {
    int l, t, m, ndec_limit, max_iter, flags, kstart, kmax;
    double rsd_limit, reldec_limit, tol;
    double eta[4];
};

struct SysDesc {
    MatView m;
    int upl, nblk_spmv, nblk_vec, sched;   // sched: 1 (nonzero split) or GSE_SCHEDULE_ROWS
    int row_span;              // staged row kernel: 256-row span
    int lanerow;               // row schedule through the lane-row loop (spmv_lanerow.cuh)
    int lr_smem;               // lane-row: dynamic shared memory of its P1 CTAs
    int lr_tbl;                // lane-row: 0 per-group format; 1 / 2 exponent table (general / fast decode)
    int vec2;                  // x, r, p, q 16-byte aligned: the vector phases load element pairs
    int64_t n, n_chunks;
    const double* b;
    double* x;
    double* r;
    double* p;
    double* q;
    double* ring;
    CgState* st;
    double* partial;
    unsigned* counter;
    int* err;                  // the handle's timeout word
    CgParams prm;
};

struct Workspace {
    double* r = nullptr;
    double* p = nullptr;
    double* q = nullptr;
    double* ring = nullptr;
    double* partial = nullptr;
    unsigned* counter = nullptr;
    int64_t n = 0;
    int partial_cap = 0;
    // GMRES
    double* V = nullptr;
    int V_cols = 0;
    double* gm_scratch = nullptr;   // GMRES partials, ring, state and counters
    size_t gm_scratch_n = 0;
    void* gm_host = nullptr;        // pinned host copy of the GMRES state
    bool eta_ready = false;
    double eta[4] = {0, 0, 0, 0};
};

// Engine kernels (solver.cu); one iteration slot is p1, fix, p2, p3.  Each processes the systems named by `map`
// (one int2 {system, block-within-system} per block).
__global__ void k_cg_init(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p1(const SysDesc* __restrict__ sys, const int2* __restrict__ map);        // nonzero split
__global__ void k_cg_p1_rows(const SysDesc* __restrict__ sys, const int2* __restrict__ map);   // row schedule
__global__ void k_cg_p1_lr(const SysDesc* __restrict__ sys, const int2* __restrict__ map);     // lane-row schedule
int p1_lr_occupancy(size_t smem);   // sets the lane-row P1 kernel's shared-memory limit; CTAs per SM at `smem`
__global__ void k_cg_fix(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p2(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p3(const SysDesc* __restrict__ sys, const int2* __restrict__ map);

// Shared memory of a P1 CTA on the nonzero split: none (direct loads).
inline size_t p1_smem() { return 0; }

// Shared memory of a P1 CTA on the row schedule for a stage span (nonzeros per
// 256-row super-block), again for the largest value source.
inline size_t p1_rows_smem(int span, int r_lo) {
    const int a = rows_block_smem<ENG_ROW_STAGES>(row_stage_layout<SRC_FP64, 0>(span, r_lo));
    const int b = rows_block_smem<ENG_ROW_STAGES>(row_stage_layout<3, -1>(span, r_lo));
    return (size_t)(a > b ? a : b);
}
inline size_t p1_rows_smem_max() { return p1_rows_smem(GSE_ROW_SPAN_MAX, 16); }

// Shared memory of a lane-row P1 CTA of a system that runs value sources
// kstart..kmax (GSE levels) or its baseline kmax: the widest of them.
inline size_t p1_lr_smem(int kstart, int kmax) {
    int b = 0;
    if (kmax > 3) b = lanerow_smem_k<1>(kmax, ENG_LR_WARPS);
    else
        for (int k = kstart < 1 ? 1 : kstart; k <= kmax; k++) {
            const int v = lanerow_smem_k<1>(k, ENG_LR_WARPS);
            b = v > b ? v : b;
        }
    return (size_t)b;
}

// P1 kernels: 0 nonzero split, 1 staged rows, 2 lane-row.
enum { P1_SPLIT = 0, P1_ROWS = 1, P1_LANEROW = 2 };

// P1 CTAs an SM holds for a dynamic shared-memory size (the kernel's
// shared-memory limit is set on the current device first).
inline int p1_occupancy(int which, size_t smem) {
    const void* fn = which == P1_ROWS ? (const void*)k_cg_p1_rows : (const void*)k_cg_p1;
    const size_t lim = which == P1_ROWS ? p1_rows_smem_max() : p1_smem();
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lim);
    const int threads = (which == P1_ROWS ? ENG_ROW_WARPS : ENG_WARPS) * 32;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess || nb < 1) {
        cudaGetLastError();
        nb = 1;
    }
    return nb;
}

// Fills the schedule-dependent part of a system descriptor (engine and
// allocation-free entry point use the same partition, so results match).
// Block counts depend on the system and the device only, never on what else
// is in a batch: P1 gets one wave of CTAs at the occupancy of the system's own
// stage ring (row schedule) or of the nonzero-split ring.
// 256-thread CTAs of the vector phases (P2, P3) an SM holds (the smaller).
inline int vec_occupancy() {
    int a = 0, b = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, (const void*)k_cg_p2, 256, 0) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, (const void*)k_cg_p3, 256, 0) != cudaSuccess) {
        cudaGetLastError();
        return 4;
    }
    const int v = a < b ? a : b;
    return v < 1 ? 1 : v;
}

// True when every vector the vector phases touch is 16-byte aligned.
inline int vec2_aligned(const void* a, const void* b, const void* c, const void* d) {
    return (((uintptr_t)a | (uintptr_t)b | (uintptr_t)c | (uintptr_t)d) & 15u) == 0 ? 1 : 0;
}

inline void sys_partition(SysDesc& d, const gse_matrix* h, int num_sms, int kstart, int kmax) {
    d.upl = 1;
    d.sched = (h->schedule_forced ? h->schedule_forced : h->schedule_auto) == GSE_SCHEDULE_ROWS &&
                      h->row_span256 <= GSE_ROW_SPAN_MAX ? GSE_SCHEDULE_ROWS : 1;
    d.lanerow = d.sched == GSE_SCHEDULE_ROWS && lanerow_ok(h, kstart) && lanerow_ok(h, kmax) ? 1 : 0;
    d.lr_tbl = d.lanerow ? lanerow_table_kind(h) : 0;
    d.row_span = h->row_span256;
    d.lr_smem = d.lanerow ? (int)p1_lr_smem(kstart, kmax) : 0;
    d.n = h->v.n_rows;
    d.n_chunks = (h->v.nnz + 255) / 256;
    const int64_t partial_cap = (int64_t)num_sms * 64;
    int64_t nbs;
    if (d.lanerow) {
        nbs = (d.n + 32 * ENG_LR_WARPS - 1) / (32 * ENG_LR_WARPS);   // a 32-row tile per warp
        const int64_t wave = (int64_t)num_sms * p1_lr_occupancy((size_t)d.lr_smem);
        if (nbs > wave) nbs = wave;
    } else if (d.sched == GSE_SCHEDULE_ROWS) {
        nbs = (d.n + 32 * ENG_ROW_WARPS - 1) / (32 * ENG_ROW_WARPS);
        const int64_t wave = (int64_t)num_sms * p1_occupancy(P1_ROWS, p1_rows_smem(d.row_span, d.m.r_lo));
        if (nbs > wave) nbs = wave;
    } else {
        nbs = (d.n_chunks + ENG_WARPS - 1) / ENG_WARPS;                // a chunk per warp
        const int64_t wave = (int64_t)num_sms * p1_occupancy(P1_SPLIT, p1_smem());
        if (nbs > wave) nbs = wave;
    }
    if (nbs < 1) nbs = 1;
    int64_t nbv = (d.n + 1023) / 1024;
    const int64_t vwave = (int64_t)num_sms * vec_occupancy();      // one wave of the vector phases at most
    if (nbv > vwave) nbv = vwave;
    if (nbv < 1) nbv = 1;
    if (nbs > partial_cap) nbs = partial_cap;
    if (nbv > partial_cap) nbv = partial_cap;
    d.nblk_spmv = (int)nbs;
    d.nblk_vec = (int)nbv;
}

}  // namespace gse
