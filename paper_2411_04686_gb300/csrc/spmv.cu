// spmv.cu -- standalone GSE-SpMV (gse_spmv) and the plain FP64 / FP32 CSR
// baselines through the same chunk engine; schedule choice and autotuning.
#include <cstdio>
#include <mutex>

#include "spmv_core.cuh"

namespace gse {

constexpr int SPMV_WARPS = 8;

template <int UPL>
constexpr size_t spmv_smem() { return (size_t)SPMV_WARPS * 256 * UPL * sizeof(double) + 64 * sizeof(double); }

// Reduces one double per block (v, valid in thread 0) over the grid into
// *out; the last block to finish sums the block partials in block order.
__device__ __forceinline__ void grid_sum_last_block(double v, double* partial, unsigned* counter,
                                                    double* out, double* red) {
    __shared__ bool last;
    if (threadIdx.x == 0) {
        partial[blockIdx.x] = v;
        __threadfence();
        last = atomicAdd(counter, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    double s = 0.0;
    for (unsigned i = threadIdx.x; i < gridDim.x; i += blockDim.x) s += __ldcg(partial + i);
    s = block_sum(s, red);
    if (threadIdx.x == 0) {
        *out = s;
        *counter = 0;
    }
}

template <int K, int R, int UPL>
__global__ void __launch_bounds__(256) k_spmv(MatView m, const double* __restrict__ x, Epi e,
                                               int64_t n_chunks, double* red_partial,
                                               unsigned* red_counter, double* dot_out, const int* gate) {
    if (gate && *gate) return;
    extern __shared__ double smem[];
    constexpr int CH = 256 * UPL;
    const int warp = threadIdx.x >> 5;
    double* yb = smem + warp * CH;
    double* red = smem + SPMV_WARPS * CH;
    fill_empty_rows(m, e, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                    (int64_t)gridDim.x * blockDim.x);
    double dot = 0.0;
    for (int64_t c = (int64_t)blockIdx.x * SPMV_WARPS + warp; c < n_chunks;
         c += (int64_t)gridDim.x * SPMV_WARPS)
        dot += process_chunk<K, R, UPL>(m, x, e, c, yb);
    if (e.kind == EPI_CG_PQ) {
        const double s = block_sum(dot, red);
        grid_sum_last_block(s, red_partial, red_counter, dot_out, red);
    }
}

typedef void (*SpmvKernel)(MatView, const double*, Epi, int64_t, double*, unsigned*, double*, const int*);

template <int K, int R, int UPL>
SpmvKernel kernel_of() { return k_spmv<K, R, UPL>; }

template <int K, int R>
SpmvKernel pick_upl(int upl) {
    switch (upl) {
        case 1: return kernel_of<K, R, 1>();
        case 2: return kernel_of<K, R, 2>();
        default: return kernel_of<K, R, 4>();
    }
}

static SpmvKernel pick_kernel(int k, int r_lo, int upl) {
    switch (k) {
        case 1: return pick_upl<1, 0>(upl);
        case 2: return pick_upl<2, 0>(upl);
        case 3:
            switch (r_lo) {
                case 0: return pick_upl<3, 0>(upl);
                case 4: return pick_upl<3, 4>(upl);
                case 8: return pick_upl<3, 8>(upl);
                default: return pick_upl<3, 16>(upl);
            }
        case SRC_FP32: return pick_upl<SRC_FP32, 0>(upl);
        default: return pick_upl<SRC_FP64, 0>(upl);
    }
}

static size_t smem_of(int upl) {
    return upl == 1 ? spmv_smem<1>() : upl == 2 ? spmv_smem<2>() : spmv_smem<4>();
}

// Occupancy-derived resident blocks per SM for each kernel (cached).
static int resident_blocks(SpmvKernel kfn, int upl) {
    static std::mutex mu;
    static const void* keys[64];
    static int vals[64];
    static int nkeys = 0;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < nkeys; i++)
        if (keys[i] == (const void*)kfn) return vals[i];
    const size_t sm = smem_of(upl);
    if (sm > 48 * 1024)
        cudaFuncSetAttribute((const void*)kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kfn, 256, sm) != cudaSuccess || nb < 1) nb = 1;
    if (nkeys < 64) {
        keys[nkeys] = (const void*)kfn;
        vals[nkeys] = nb;
        nkeys++;
    }
    return nb;
}

int spmv_grid(gse_matrix* h, int upl) {
    const int64_t ch = 256 * upl;
    const int64_t n_chunks = (h->v.nnz + ch - 1) / ch;
    SpmvKernel kfn = pick_kernel(3, h->v.r_lo, upl);
    const int64_t resident = (int64_t)h->num_sms * resident_blocks(kfn, upl);
    int64_t g = (n_chunks + SPMV_WARPS - 1) / SPMV_WARPS;
    if (g > resident) g = resident;
    if (g < 1) g = 1;
    return (int)g;
}

int launch_spmv(gse_matrix* h, int k, int epi, const SpmvArgs& a, cudaStream_t s, int upl_override) {
    const int upl = upl_override ? upl_override : units_per_lane(h);
    SpmvKernel kfn = pick_kernel(k, h->v.r_lo, upl);
    const int64_t ch = 256 * upl;
    const int64_t n_chunks = (h->v.nnz + ch - 1) / ch;
    const int64_t resident = (int64_t)h->num_sms * resident_blocks(kfn, upl);
    int64_t g = (n_chunks + SPMV_WARPS - 1) / SPMV_WARPS;
    if (g > resident) g = resident;
    const int64_t gmin = (h->v.n_empty + 255) / 256;
    if (g < gmin) g = gmin < resident ? gmin : resident;
    if (g < 1) g = 1;
    if (epi == EPI_CG_PQ && g > h->red_capacity) g = h->red_capacity;
    Epi e;
    e.kind = epi;
    e.y = a.y;
    e.b = a.b;
    e.p = a.p;
    kfn<<<(unsigned)g, 256, smem_of(upl), s>>>(h->v, a.x, e, n_chunks, a.red_partial ? a.red_partial : h->red_partial,
                                              a.red_counter ? a.red_counter : h->red_counter, a.dot_out,
                                              a.skip_flag);
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

}  // namespace gse

using namespace gse;

static bool level_ok(gse_matrix* h, int k) {
    if (k >= 1 && k <= h->n_seg) return true;
    if (k == GSE_LEVEL_FP64) return h->v.val64 != nullptr;
    if (k == GSE_LEVEL_FP32) return h->v.val32 != nullptr;
    return false;
}

extern "C" int gse_spmv(gse_handle h, int k, const double* x, double* y, void* stream) {
    if (!h || !x || !y || !level_ok(h, k)) return GSE_ERR_INVALID;
    SpmvArgs a = {};
    a.x = x;
    a.y = y;
    return launch_spmv(h, k, EPI_STORE, a, (cudaStream_t)stream);
}

extern "C" int gse_set_schedule(gse_handle h, int upl) {
    if (!h || !(upl == 0 || upl == 1 || upl == 2 || upl == 4)) return GSE_ERR_INVALID;
    h->schedule_forced = upl;
    return GSE_OK;
}

extern "C" int gse_autotune(gse_handle h, int k, void* stream) {
    if (!h || !level_ok(h, k)) return GSE_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    double *x = nullptr, *y = nullptr;
    GSE_CUDA_TRY(cudaMallocAsync(&x, (size_t)(h->v.n_cols + 1) * sizeof(double), s));
    if (cudaMallocAsync(&y, (size_t)(h->v.n_rows + 1) * sizeof(double), s) != cudaSuccess) {
        cudaFreeAsync(x, s);
        return GSE_ERR_OOM;
    }
    cudaMemsetAsync(x, 0, (size_t)(h->v.n_cols + 1) * sizeof(double), s);
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const int cands[3] = {1, 2, 4};
    float best = 1e30f;
    int best_upl = units_per_lane(h);
    SpmvArgs a = {};
    a.x = x;
    a.y = y;
    for (int ci = 0; ci < 3; ci++) {
        const int upl = cands[ci];
        launch_spmv(h, k, EPI_STORE, a, s, upl);  // warm
        cudaEventRecord(e0, s);
        for (int r = 0; r < 5; r++) launch_spmv(h, k, EPI_STORE, a, s, upl);
        cudaEventRecord(e1, s);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) {
            best = ms;
            best_upl = upl;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFreeAsync(x, s);
    cudaFreeAsync(y, s);
    cudaStreamSynchronize(s);
    h->schedule_auto = best_upl;
    h->schedule_forced = 0;
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}
