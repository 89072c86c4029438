// solver_internal.cuh -- types of the device-resident CG engine (solver.cu)
// shared with other translation units that launch its kernels.
#pragma once

#include "spmv_core.cuh"

namespace gse {

enum { MODE_ITER = 0, MODE_RESID_R = 1, MODE_RESID_T = 2, MODE_DONE = 3 };
enum { PA_NONE = 0, PA_UPDATE = 1, PA_XONLY = 2, PA_COPY_R = 3, PA_COPY_Q = 4, PA_ZERO_X = 5 };
constexpr int RING_MAX = 4096;
constexpr int ENG_WARPS = 8;

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
    int upl, nblk_spmv, nblk_vec, pad;
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

// Engine kernels (solver.cu).  Each processes the systems named by `map`
// (one int2 {system, block-within-system} per block).
__global__ void k_cg_init(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p1(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p2(const SysDesc* __restrict__ sys, const int2* __restrict__ map);
__global__ void k_cg_p3(const SysDesc* __restrict__ sys, const int2* __restrict__ map);

inline size_t p1_smem() { return (size_t)ENG_WARPS * 512 * sizeof(double) + 64 * sizeof(double); }

}  // namespace gse
