// solver_internal.cuh -- types of the device-resident CG engine (solver.cu)
// shared with other translation units that launch its kernels.
#pragma once

#include "spmv_pipe.cuh"

namespace gse {

enum { MODE_ITER = 0, MODE_RESID_R = 1, MODE_RESID_T = 2, MODE_DONE = 3 };
enum { PA_NONE = 0, PA_UPDATE = 1, PA_XONLY = 2, PA_COPY_R = 3, PA_COPY_Q = 4, PA_ZERO_X = 5 };
constexpr int RING_MAX = 4096;
constexpr int ENG_WARPS = 4;
constexpr int ENG_STAGES = 3;

struct CgState {
    int mode, k, status, j, p_action, hlen, hpos, pad;
    int sw[4];
    double rho, pq, alpha, beta, nb, res, true_res, xnorm2;
};

struct CgParams {
    int l, t, m, ndec_limit, max_iter, flags, kstart, kmax;
    double rsd_limit, reldec_limit, tol;
    double eta[4];
};

struct SysDesc {
    MatView m;
    int upl, nblk_spmv, nblk_vec, sched;   // sched: 1 (nonzero split) or GSE_SCHEDULE_ROWS
    int row_span, pad2;
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
    double* gm_scratch = nullptr;
    size_t gm_scratch_n = 0;
    bool eta_ready = false;
    double eta[4] = {0, 0, 0, 0};
};

// Engine kernels (solver.cu); one iteration slot is p1, fix, p2, p3.  Each processes the systems named by `map`
// (one int2 {system, block-within-system} per block).
__global__ void k_cg_init(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p1(const SysDesc* __restrict__ sys, const int2* __restrict__ map, int warp_smem);
__global__ void k_cg_fix(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p2(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p3(const SysDesc* __restrict__ sys, const int2* __restrict__ map);

// Per-warp share of P1's shared memory on the nonzero split: the CTA's stage
// ring for the largest value source, divided over its warps.
inline int eng_chunks_warp_smem() {
    const int a = chunks_block_smem<ENG_STAGES, 1>(chunk_stage_layout<SRC_FP64, 0, 1>(ENG_WARPS, 16));
    const int b = chunks_block_smem<ENG_STAGES, 1>(chunk_stage_layout<3, -1, 1>(ENG_WARPS, 16));
    return ((a > b ? a : b) + ENG_WARPS - 1) / ENG_WARPS;
}
#define ENG_WARP_SMEM (eng_chunks_warp_smem())
inline size_t p1_smem() { return (size_t)ENG_WARPS * ENG_WARP_SMEM; }

// Largest per-warp shared memory P1 can need (row schedule at the widest span).
inline int eng_max_warp_smem() {
    const int r = rows_block_smem<ENG_STAGES>(row_stage_layout<SRC_FP64, 0>(GSE_ROW_SPAN_MAX, 16));
    const int q = rows_block_smem<ENG_STAGES>(row_stage_layout<3, -1>(GSE_ROW_SPAN_MAX, 16));
    const int m = (r > q ? r : q) / ENG_WARPS + 1;
    return m > ENG_WARP_SMEM ? m : ENG_WARP_SMEM;
}

// Per-warp shared memory P1 needs for a system (its schedule, any level).
// (The row schedule stages whole CTAs: its need is the CTA's, divided over the warps.)
inline int sys_warp_smem(const SysDesc& d) {
    if (d.sched != GSE_SCHEDULE_ROWS) return ENG_WARP_SMEM;
    const int a = rows_block_smem<ENG_STAGES>(row_stage_layout<SRC_FP64, 0>(d.row_span, d.m.r_lo));
    const int b = rows_block_smem<ENG_STAGES>(row_stage_layout<3, -1>(d.row_span, d.m.r_lo));
    const int need = (a > b ? a : b);
    return (need + ENG_WARPS - 1) / ENG_WARPS;
}

// Fills the schedule-dependent part of a system descriptor (engine and
// allocation-free entry point use the same partition, so results match).
inline void sys_partition(SysDesc& d, const gse_matrix* h, int num_sms, int p1_resident) {
    d.upl = 1;
    d.row_span = h->row_span128;   // super-blocks of 32 * ENG_WARPS = 128 rows
    d.sched = (h->schedule_forced ? h->schedule_forced : h->schedule_auto) == GSE_SCHEDULE_ROWS &&
                      h->row_span128 <= GSE_ROW_SPAN_MAX ? GSE_SCHEDULE_ROWS : 1;
    d.n = h->v.n_rows;
    d.n_chunks = (h->v.nnz + 255) / 256;
    const int64_t partial_cap = (int64_t)num_sms * 64;
    int64_t nbs;
    if (d.sched == GSE_SCHEDULE_ROWS) {
        nbs = (d.n + 32 * ENG_WARPS - 1) / (32 * ENG_WARPS);
        if (nbs > (int64_t)num_sms * 4) nbs = (int64_t)num_sms * 4;   // fixed cap: independent of the batch
    } else {
        nbs = (d.n_chunks + ENG_WARPS - 1) / ENG_WARPS;                // super-chunks
        if (nbs > (int64_t)num_sms * p1_resident) nbs = (int64_t)num_sms * p1_resident;
    }
    if (nbs < 1) nbs = 1;
    int64_t nbv = (d.n + 1023) / 1024;
    if (nbv > (int64_t)num_sms * 8) nbv = (int64_t)num_sms * 8;
    if (nbv < 1) nbv = 1;
    if (nbs > partial_cap) nbs = partial_cap;
    if (nbv > partial_cap) nbv = partial_cap;
    d.nblk_spmv = (int)nbs;
    d.nblk_vec = (int)nbv;
}

}  // namespace gse
