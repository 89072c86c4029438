// noalloc.cu -- gse_cg_noalloc: the stepped CG for callers that cannot
// allocate device memory at solve time.
//
// Some callers cannot call cudaMalloc once their set-up is over: a solver
// embedded in a real-time loop with a fixed memory budget, code running under
// an allocator that forbids new device allocations, or a host thread that must
// not synchronise the device the way cudaMalloc/cudaFree can.  gse_cg allocates
// its Krylov workspace and engine tables on first use; this entry point runs
// the same engine kernels with every piece of scratch (r, p, q, the residual
// history, reduction partials and counters, the system descriptor, its state
// and block maps) carved out of one file-scope device array of fixed size.  It
// calls no cudaMalloc, cudaFree or allocating library routine.  The encoded
// matrix itself comes from gse_encode, done beforehand.
//
// The array is part of the module, so every GPU that loads this library holds
// it until the process exits (about 1.7 MB).  All calls share it: calls whose
// work overlaps on the GPU (from two host threads, or on two streams) race and
// corrupt each other.  Each call re-initialises what must start from a known
// value (counters zeroed, state and descriptor rewritten).
#include <chrono>
#include <cmath>
#include <cstring>
#include <mutex>

#include "solver_internal.cuh"

namespace gse {
namespace {

constexpr int64_t NA_MAX_ROWS = 65536;      // largest system (rows) this entry point accepts
constexpr int NA_MAX_BLOCKS = 4096;         // grid-size cap of any engine phase

constexpr size_t na_align(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t NA_OFF_R = 0;
constexpr size_t NA_OFF_P = na_align(NA_OFF_R + NA_MAX_ROWS * sizeof(double));
constexpr size_t NA_OFF_Q = na_align(NA_OFF_P + NA_MAX_ROWS * sizeof(double));
constexpr size_t NA_OFF_RING = na_align(NA_OFF_Q + NA_MAX_ROWS * sizeof(double));
constexpr size_t NA_OFF_PARTIAL = na_align(NA_OFF_RING + (RING_MAX + 1) * sizeof(double));
constexpr size_t NA_OFF_COUNTER = na_align(NA_OFF_PARTIAL + NA_MAX_BLOCKS * sizeof(double));
constexpr size_t NA_OFF_SYS = na_align(NA_OFF_COUNTER + 8 * sizeof(unsigned));
constexpr size_t NA_OFF_STATE = na_align(NA_OFF_SYS + sizeof(SysDesc));
constexpr size_t NA_OFF_MAP_SPMV = na_align(NA_OFF_STATE + sizeof(CgState));
constexpr size_t NA_OFF_MAP_VEC = na_align(NA_OFF_MAP_SPMV + NA_MAX_BLOCKS * sizeof(int2));
constexpr size_t NA_OFF_NORM = na_align(NA_OFF_MAP_VEC + NA_MAX_BLOCKS * sizeof(int2));
constexpr size_t NA_BYTES = na_align(NA_OFF_NORM + 8 * sizeof(double));

// The scratch.  Host code must not use this name as an address (in host code
// it is only a stand-in); it takes the device address from
// cudaGetSymbolAddress, once per device, in na_scratch().
static __device__ __align__(256) unsigned char g_cg_scratch[NA_BYTES];

std::mutex g_na_mu;
unsigned char* g_na_ptr[128] = {nullptr};

// Device address of the scratch on the current device (set-up on first use).
int na_scratch(unsigned char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 128) return GSE_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_cg_scratch);
        if (e != cudaSuccess || !p) {
            cudaGetLastError();
            return GSE_ERR_CUDA;
        }
        g_na_ptr[dev] = (unsigned char*)p;
    }
    *out = g_na_ptr[dev];
    return GSE_OK;
}

__global__ void k_na_maps(int2* map_spmv, int nbs, int2* map_vec, int nbv) {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < nbs || i < nbv; i += gridDim.x * blockDim.x) {
        if (i < nbs) map_spmv[i] = make_int2(0, i);
        if (i < nbv) map_vec[i] = make_int2(0, i);
    }
}

// ||v||^2 with one block (n <= NA_MAX_ROWS), fixed summation order.
__global__ void k_na_norm2(const double* __restrict__ v, int64_t n, double* out) {
    __shared__ double red[32];
    double a = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a = fma(v[i], v[i], a);
    a = block_sum(a, red);
    if (threadIdx.x == 0) *out = a;
}

bool level_valid_na(const gse_matrix* h, int k) { return level_available(h, k); }

}  // namespace
}  // namespace gse

using namespace gse;

extern "C" int gse_cg_noalloc(gse_handle h, const double* b, double* x, double tol, const gse_step_policy* pol,
                              gse_solve_info* info, void* stream) {
    if (!h || !b || !x || !pol || !(tol > 0)) return GSE_ERR_INVALID;
    if (!level_valid_na(h, pol->k_start) || !level_valid_na(h, pol->k_max)) return GSE_ERR_INVALID;
    const bool base = pol->k_start > 3 || pol->k_max > 3;
    if (base && pol->k_start != pol->k_max) return GSE_ERR_INVALID;
    if (!base && pol->k_start > pol->k_max) return GSE_ERR_INVALID;
    if (pol->t < 1 || pol->t > RING_MAX - 1 || pol->max_iter < 1) return GSE_ERR_INVALID;
    if (h->v.n_rows > NA_MAX_ROWS) return GSE_ERR_UNSUPPORTED;   // beyond the fixed scratch
    if (pol->flags & GSE_POLICY_FLOOR) return GSE_ERR_UNSUPPORTED; // its coefficients need allocations
    const auto t0 = std::chrono::steady_clock::now();
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base_ptr = nullptr;
    int rc = na_scratch(&base_ptr);
    if (rc != GSE_OK) return rc;

    // the same partition the engine uses, so results match gse_cg bit for bit
    int dev = 0, num_sms = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev);
    SysDesc d;
    memset(&d, 0, sizeof(d));
    d.m = h->v;
    d.err = h->d_err;
    sys_partition(d, h, num_sms, pol->k_start, pol->k_max);
    const int64_t nbs = d.nblk_spmv, nbv = d.nblk_vec;
    if (nbs > NA_MAX_BLOCKS || 2 * nbv > NA_MAX_BLOCKS) return GSE_ERR_UNSUPPORTED;   // P2 keeps two sums per block
    const bool rows = d.sched == GSE_SCHEDULE_ROWS;
    const size_t p1sm = d.lanerow ? (size_t)d.lr_smem
                        : rows    ? p1_rows_smem(d.row_span, d.m.r_lo)
                                  : p1_smem();
    d.b = b;
    d.x = x;
    d.r = (double*)(base_ptr + NA_OFF_R);
    d.p = (double*)(base_ptr + NA_OFF_P);
    d.q = (double*)(base_ptr + NA_OFF_Q);
    d.vec2 = vec2_aligned(d.x, d.r, d.p, d.q);
    d.ring = (double*)(base_ptr + NA_OFF_RING);
    d.st = (CgState*)(base_ptr + NA_OFF_STATE);
    d.partial = (double*)(base_ptr + NA_OFF_PARTIAL);
    d.counter = (unsigned*)(base_ptr + NA_OFF_COUNTER);
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
    CgState s0;
    memset(&s0, 0, sizeof(s0));
    s0.mode = MODE_RESID_R;
    s0.k = pol->k_start;
    s0.j = -1;
    s0.status = GSE_MAXITER;
    for (int i = 0; i < 4; i++) s0.sw[i] = -1;
    if (!base) s0.sw[pol->k_start - 1] = 0;
    SysDesc* d_sys = (SysDesc*)(base_ptr + NA_OFF_SYS);
    int2* map_spmv = (int2*)(base_ptr + NA_OFF_MAP_SPMV);
    int2* map_vec = (int2*)(base_ptr + NA_OFF_MAP_VEC);
    double* d_norm = (double*)(base_ptr + NA_OFF_NORM);
    // re-initialise what the previous call left behind (host sources are on the
    // stack: pageable copies complete their host side before returning)
    cudaMemcpyAsync(d_sys, &d, sizeof(d), cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(d.st, &s0, sizeof(s0), cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(d.counter, 0, 8 * sizeof(unsigned), s);
    cudaMemsetAsync(h->d_err, 0, sizeof(int), s);   // this solve's bounded-wait record starts clear
    k_na_maps<<<16, 256, 0, s>>>(map_spmv, (int)nbs, map_vec, (int)nbv);
    k_cg_init<<<(unsigned)nbv, 256, 0, s>>>(d_sys, map_vec);
    k_cg_p3<<<(unsigned)nbv, 256, 0, s>>>(d_sys, map_vec);
    const int budget = pol->max_iter + 64 * 4;
    int used = 0;
    CgState hs;
    memset(&hs, 0, sizeof(hs));
    while (used < budget) {
        const int nb = budget - used < 16 ? budget - used : 16;
        for (int it = 0; it < nb; it++) {
            if (d.lanerow) {
                k_cg_p1_lr<<<(unsigned)nbs, ENG_LR_WARPS * 32, p1sm, s>>>(d_sys, map_spmv);
            } else if (rows) {
                k_cg_p1_rows<<<(unsigned)nbs, ENG_ROW_WARPS * 32, p1sm, s>>>(d_sys, map_spmv);
            } else {
                k_cg_p1<<<(unsigned)nbs, ENG_WARPS * 32, p1sm, s>>>(d_sys, map_spmv);
                k_cg_fix<<<(unsigned)nbv, 256, 0, s>>>(d_sys, map_vec);
            }
            k_cg_p2<<<(unsigned)nbv, 256, 0, s>>>(d_sys, map_vec);
            k_cg_p3<<<(unsigned)nbv, 256, 0, s>>>(d_sys, map_vec);
        }
        used += nb;
        cudaMemcpyAsync(&hs, d.st, sizeof(hs), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return GSE_ERR_CUDA;
        if (hs.mode == MODE_DONE) break;
    }
    // final true residual ||b - A_kmax x|| / ||b||: a converged solve's was
    // computed on the device when it passed the check (x has not changed
    // since), as gse_cg reports it; otherwise recompute it (q is free now)
    double true_res = 0.0;
    if (hs.mode == MODE_DONE && hs.status == GSE_OK) {
        true_res = hs.true_res;
    } else if (hs.nb > 0.0) {
        SpmvArgs a = {};
        a.x = x;
        a.y = d.q;
        a.b = b;
        launch_spmv(h, pol->k_max, EPI_RESID, a, s);
        k_na_norm2<<<1, 1024, 0, s>>>(d.q, d.n, d_norm);
        double nrm2 = 0.0;
        cudaMemcpyAsync(&nrm2, d_norm, sizeof(double), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return GSE_ERR_CUDA;
        true_res = sqrt(nrm2) / hs.nb;
    }
    if (cudaGetLastError() != cudaSuccess) return GSE_ERR_CUDA;
    int status = hs.mode == MODE_DONE ? hs.status : GSE_MAXITER;
    int err = 0;
    cudaMemcpyAsync(&err, h->d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
    cudaStreamSynchronize(s);
    if (err) status = GSE_TIMEOUT;   // a bounded device-side wait gave up
    if (info) {
        memset(info, 0, sizeof(*info));
        info->status = status;
        info->iters = hs.j < 0 ? 0 : hs.j;
        info->k_final = base ? 0 : hs.k;
        for (int i = 0; i < 3; i++) info->switch_iter[i] = base ? -1 : hs.sw[i];
        info->rel_res_rec = hs.res;
        info->rel_res_true = true_res;
        info->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return status;
}
