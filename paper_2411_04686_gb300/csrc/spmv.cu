// spmv.cu -- standalone GSE-SpMV (gse_spmv) and the plain FP64 / FP32 / FP16 /
// BF16 CSR baselines through the same loops: the row schedule (k_spmv_rows),
// the direct-load nonzero split (k_spmv_direct) and the staged nonzero split
// (k_spmv); schedule choice and autotuning.
#include <cstdio>
#include <mutex>

#include "spmv_lanerow.cuh"
#include "spmv_pipe.cuh"

namespace gse {

// warps per CTA on the nonzero split: 8 / UPL, so a stage always holds 2048 nonzeros
template <int UPL>
constexpr int spmv_warps() { return 8 / UPL; }

// y = A_k x (or b - A_k x) on the nonzero split: CTAs of 8/UPL warps walk
// super-chunks of that many chunks through a TMA-filled ring of 2 or 3 stages
// (whichever keeps more warps resident).
template <int K, int R, int UPL, bool RESID, int STAGES, bool TBL = false>
__global__ void __launch_bounds__(spmv_warps<UPL>() * 32) k_spmv(MatView m, const double* __restrict__ x, Epi e,
                                                                  int64_t n_chunks, ChunkStage L, int* err,
                                                                  const int* gate) {
    if (gate && *gate) return;
    extern __shared__ __align__(128) unsigned char smem[];
    fill_empty_rows(m, e, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
    spmv_chunks_block<K, R, UPL, false, RESID, STAGES, TBL>(m, x, e, blockIdx.x, gridDim.x, n_chunks, L, smem, err);
}

// One unit of 8 per lane: the direct-load nonzero split (no stage ring), 8-warp CTAs.
template <int K, int R, bool RESID>
__global__ void __launch_bounds__(256) k_spmv_direct(MatView m, const double* __restrict__ x, Epi e, int64_t n_chunks,
                                                     ChunkStage L, int* err, const int* gate) {
    if (gate && *gate) return;
    (void)L;
    (void)err;
    fill_empty_rows(m, e, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    spmv_chunks_direct<K, R, false, RESID>(m, x, e, gw, ((int64_t)gridDim.x * blockDim.x) >> 5, n_chunks);
}

// The same at level 3 for a handle in the default layout (groups of 32,
// segments 16/16/20, no table): the decoder's widths are compile-time
// constants, and at 64 registers an SM holds 4 CTAs (the general level-3
// kernel: 3).  The values are the same bits.
template <bool RESID>
__global__ void __launch_bounds__(256, 4) k_spmv_direct_std3(MatView m, const double* __restrict__ x, Epi e,
                                                             int64_t n_chunks, ChunkStage L, int* err, const int* gate) {
    if (gate && *gate) return;
    (void)L;
    (void)err;
    fill_empty_rows(m, e, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, (int64_t)gridDim.x * blockDim.x);
    const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    spmv_chunks_direct<3, 4, false, RESID, true>(m, x, e, gw, ((int64_t)gridDim.x * blockDim.x) >> 5, n_chunks);
}

// Finishes the rows that cross chunk boundaries (after k_spmv, same stream).
template <int UPL>
__global__ void __launch_bounds__(256) k_spmv_fix(MatView m, Epi e, int64_t n_chunks, const int* gate) {
    if (gate && *gate) return;
    fix_split_rows<256 * UPL>(m, e, n_chunks, (int64_t)blockIdx.x * blockDim.x + threadIdx.x,
                              (int64_t)gridDim.x * blockDim.x);
}

// Row schedule: one row per lane, 256 consecutive rows per CTA and stage,
// staged by one producer thread with large bulk copies (short rows).  The ring
// has 2 or 3 stages, whichever keeps more warps resident (wide stages at k = 3
// and FP64 cap the CTAs an SM holds by shared memory).
constexpr int ROWS_WARPS = 8;

template <int K, int R, bool RESID, int STAGES, bool TBL = false>
__global__ void __launch_bounds__(ROWS_WARPS * 32) k_spmv_rows(MatView m, const double* __restrict__ x, Epi e,
                                                                int64_t nsb, RowStage L, int* err, const int* gate) {
    if (gate && *gate) return;
    extern __shared__ __align__(128) unsigned char smem[];
    spmv_rows_block<K, R, false, RESID, STAGES, TBL>(m, x, e, blockIdx.x, gridDim.x, nsb, L, smem, err);
}

// Lane-row schedule: one row per lane, two rows per lane in flight, each warp
// staging its own 64-row tiles (spmv_lanerow.cuh); 8-warp CTAs, warps take
// tiles round-robin.
constexpr int LR_WARPS = 8;

// TBL: 0 the per-group format; 1 the global table (index in the column word),
// general decode; 2 the same when every entry exceeds W_1 (fast decode).
template <int K, bool RESID, int TBL = 0>
__global__ void __launch_bounds__(LR_WARPS * 32) k_spmv_lanerow(MatView m, const double* __restrict__ x, Epi e,
                                                                 const int* gate) {
    if (gate && *gate) return;
    extern __shared__ __align__(128) unsigned char smem[];
    constexpr int R = lr_rows_per_lane<K>();
    const int warp = threadIdx.x >> 5;
    const int64_t ntile = (m.n_rows + 32 * R - 1) / (32 * R);
    lr_loop<K, false, RESID, R, TBL>(m, x, e, (int64_t)blockIdx.x * LR_WARPS + warp, (int64_t)gridDim.x * LR_WARPS,
                                     ntile, smem + warp * LR_STAGES * LrLayout<K, R>::BYTES);
}

typedef void (*LaneRowKernel)(MatView, const double*, Epi, const int*);

template <int K, bool RESID>
static LaneRowKernel pick_lr(int* smem, int* rows, int tbl) {
    *smem = lr_smem<K>(LR_WARPS);
    *rows = lr_rows_per_lane<K>();
    if (K > 3) return tbl ? k_spmv_lanerow<K, RESID, 1> : k_spmv_lanerow<K, RESID>;   // baselines: masked columns
    return tbl == 2 ? k_spmv_lanerow<K, RESID, 2> : tbl == 1 ? k_spmv_lanerow<K, RESID, 1> : k_spmv_lanerow<K, RESID>;
}

template <bool RESID>
static LaneRowKernel pick_lanerow_t(int k, int* smem, int* rows, int tbl) {
    switch (k) {
        case 1: return pick_lr<1, RESID>(smem, rows, tbl);
        case 2: return pick_lr<2, RESID>(smem, rows, tbl);
        case 3: return pick_lr<3, RESID>(smem, rows, tbl);
        case SRC_FP32: return pick_lr<SRC_FP32, RESID>(smem, rows, tbl);
        case SRC_FP16: return pick_lr<SRC_FP16, RESID>(smem, rows, tbl);
        case SRC_BF16: return pick_lr<SRC_BF16, RESID>(smem, rows, tbl);
        default: return pick_lr<SRC_FP64, RESID>(smem, rows, tbl);
    }
}

typedef void (*RowsKernel)(MatView, const double*, Epi, int64_t, RowStage, int*, const int*);

template <bool RESID, int STAGES>
static RowsKernel pick_rows_t(int k, int r_lo, RowStage* L, int span, bool tbl) {
    switch (k) {
        case 1:
            *L = row_stage_layout<1, 0>(span, r_lo);
            return tbl ? k_spmv_rows<1, 0, RESID, STAGES, true> : k_spmv_rows<1, 0, RESID, STAGES>;
        case 2:
            *L = row_stage_layout<2, 0>(span, r_lo);
            return tbl ? k_spmv_rows<2, 0, RESID, STAGES, true> : k_spmv_rows<2, 0, RESID, STAGES>;
        case 3:
            *L = row_stage_layout<3, -1>(span, r_lo);
            if (tbl) return r_lo == 4 ? k_spmv_rows<3, 4, RESID, STAGES, true> : k_spmv_rows<3, -1, RESID, STAGES, true>;
            if (r_lo == 4) return k_spmv_rows<3, 4, RESID, STAGES>;
            if (r_lo == 0) return k_spmv_rows<3, 0, RESID, STAGES>;
            return k_spmv_rows<3, -1, RESID, STAGES>;
        case SRC_FP32: *L = row_stage_layout<SRC_FP32, 0>(span, r_lo); return k_spmv_rows<SRC_FP32, 0, RESID, STAGES>;
        case SRC_FP16: *L = row_stage_layout<SRC_FP16, 0>(span, r_lo); return k_spmv_rows<SRC_FP16, 0, RESID, STAGES>;
        case SRC_BF16: *L = row_stage_layout<SRC_BF16, 0>(span, r_lo); return k_spmv_rows<SRC_BF16, 0, RESID, STAGES>;
        default: *L = row_stage_layout<SRC_FP64, 0>(span, r_lo); return k_spmv_rows<SRC_FP64, 0, RESID, STAGES>;
    }
}

// Resident CTAs per SM of a kernel with its block size and dynamic shared
// memory (0 on error), cached per (kernel, shared-memory size, device): the
// shared-memory attribute is set on each device before its first launch.
static int occupancy_cached(const void* fn, int threads, size_t smem) {
    static std::mutex mu;
    static const void* keys[512];
    static size_t sizes[512];
    static int devs[512];
    static int vals[512];
    static int nkeys = 0;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    std::lock_guard<std::mutex> lock(mu);
    for (int i = 0; i < nkeys; i++)
        if (keys[i] == fn && sizes[i] == smem && devs[i] == dev) return vals[i];
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    if (nkeys < 512) {
        keys[nkeys] = fn;
        sizes[nkeys] = smem;
        devs[nkeys] = dev;
        vals[nkeys] = nb;
        nkeys++;
    }
    return nb;
}

static int rows_resident(RowsKernel fn, size_t smem) { return occupancy_cached((const void*)fn, ROWS_WARPS * 32, smem); }

static int launch_rows(gse_matrix* h, int k, int epi, const SpmvArgs& a, cudaStream_t s) {
    RowStage L2, L3;
    const bool resid = epi == EPI_RESID;
    const bool tbl = h->v.tbl != 0;
    RowsKernel f3 = resid ? pick_rows_t<true, 3>(k, h->v.r_lo, &L3, h->row_span256, tbl)
                          : pick_rows_t<false, 3>(k, h->v.r_lo, &L3, h->row_span256, tbl);
    RowsKernel f2 = resid ? pick_rows_t<true, 2>(k, h->v.r_lo, &L2, h->row_span256, tbl)
                          : pick_rows_t<false, 2>(k, h->v.r_lo, &L2, h->row_span256, tbl);
    const size_t smem3 = (size_t)rows_block_smem<3>(L3), smem2 = (size_t)rows_block_smem<2>(L2);
    const int nb3 = rows_resident(f3, smem3), nb2 = rows_resident(f2, smem2);
    const bool two = nb2 >= nb3;      // equal occupancy: the smaller ring leaves more L1 for the x gathers
    RowsKernel fn = two ? f2 : f3;
    const size_t smem = two ? smem2 : smem3;
    const RowStage L = two ? L2 : L3;
    const int nb = (two ? nb2 : nb3) < 1 ? 1 : (two ? nb2 : nb3);
    const int64_t nsb = (h->v.n_rows + 32 * ROWS_WARPS - 1) / (32 * ROWS_WARPS);
    int64_t g = nsb;
    const int64_t resident = (int64_t)h->num_sms * nb;
    if (g > resident) g = resident;
    if (g < 1) g = 1;
    Epi e;
    e.kind = epi;
    e.y = a.y;
    e.b = a.b;
    e.p = a.p;
    fn<<<(unsigned)g, ROWS_WARPS * 32, smem, s>>>(h->v, a.x, e, nsb, L, h->d_err, a.skip_flag);
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

// The lane-row kernel serves a handle when every tile's slice fits its stage
// (32-row tiles within 256 nonzeros, 64-row tiles within 512), its rows are at
// most 64 long, and its level decodes with the lane-row decoders (or is a
// plain CSR baseline).
static bool lanerow_spans_ok(const gse_matrix* h) {
    return h->tile_span32 <= lr_cap_rows(1) && h->tile_span64 <= lr_cap_rows(2) && h->max_row_len <= 64 &&
           h->v.n_rows < (int64_t)1 << 30;
}

bool lanerow_ok(const gse_matrix* h, int k) {
    if (!lanerow_spans_ok(h)) return false;
    // the exponent table with its index in the column word: masked columns,
    // per-value table exponents (an index in the head stays on other kernels)
    if (h->v.tbl) return lanerow_format_tbl(h->v, h->n_seg);
    if (h->v.col_mask != 0xFFFFFFFFu) return false;
    return k > 3 || lanerow_format(h->v, h->group_size, h->n_seg);
}

// 0: per-group format; 1: table, general decode; 2: table, every entry above
// W_1 so a nonzero head holds the leading one (fast decode).
int lanerow_table_kind(const gse_matrix* h) {
    if (!h->v.tbl) return 0;
    for (int i = 0; i < h->num_exp; i++)
        if (h->etab_host[i] <= LR_W1) return 1;
    return 2;
}

static int launch_lanerow(gse_matrix* h, int k, int epi, const SpmvArgs& a, cudaStream_t s) {
    int smem = 0, R = 1;
    const int tbl = lanerow_table_kind(h);
    LaneRowKernel fn = epi == EPI_RESID ? pick_lanerow_t<true>(k, &smem, &R, tbl)
                                        : pick_lanerow_t<false>(k, &smem, &R, tbl);
    int nb = occupancy_cached((const void*)fn, LR_WARPS * 32, (size_t)smem);
    if (nb < 1) nb = 1;
    const int64_t ntile = (h->v.n_rows + 32 * R - 1) / (32 * R);
    int64_t g = (ntile + LR_WARPS - 1) / LR_WARPS;
    const int64_t resident = (int64_t)h->num_sms * nb;
    if (g > resident) g = resident;
    if (g < 1) g = 1;
    Epi e;
    e.kind = epi;
    e.y = a.y;
    e.b = a.b;
    e.p = a.p;
    fn<<<(unsigned)g, LR_WARPS * 32, (size_t)smem, s>>>(h->v, a.x, e, a.skip_flag);
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

typedef void (*SpmvKernel)(MatView, const double*, Epi, int64_t, ChunkStage, int*, const int*);

struct KernelPick {
    SpmvKernel fn;
    ChunkStage L;
    size_t smem;
    int warps;
};

template <int K, int R, int UPL, bool RESID, int STAGES, bool TBL = false>
KernelPick pick_stages(int r_lo) {
    KernelPick kp;
    kp.fn = k_spmv<K, R, UPL, RESID, STAGES, TBL>;
    kp.warps = spmv_warps<UPL>();
    kp.L = chunk_stage_layout<K, R, UPL>(kp.warps, r_lo);
    kp.smem = (size_t)chunks_block_smem<STAGES, UPL>(kp.L);
    return kp;
}

static int resident_blocks(const KernelPick& kp);

template <int K, int R, bool RESID>
KernelPick pick_direct(int r_lo) {
    KernelPick kp;
    kp.fn = k_spmv_direct<K, R, RESID>;
    kp.warps = 8;
    kp.L = chunk_stage_layout<K, R, 1>(8, r_lo);    // unused by the kernel
    kp.smem = 0;
    return kp;
}

template <int K, int R, int UPL, bool RESID, bool TBL = false>
KernelPick pick_one(int r_lo) {
    if constexpr (UPL == 1) {
        return pick_direct<K, R, RESID>(r_lo);   // the exponent source (group or table) is read per unit or value
    } else {
        const KernelPick a = pick_stages<K, R, UPL, RESID, 3, TBL>(r_lo), b = pick_stages<K, R, UPL, RESID, 2, TBL>(r_lo);
        return resident_blocks(b) >= resident_blocks(a) ? b : a;   // equal occupancy: 2 stages, more L1 for the gathers
    }
}

template <int K, int R, bool RESID>
KernelPick pick_upl(int upl, int r_lo) {
    switch (upl) {
        case 1: return pick_one<K, R, 1, RESID>(r_lo);
        case 2: return pick_one<K, R, 2, RESID>(r_lo);
        default: return pick_one<K, R, 4, RESID>(r_lo);
    }
}

// Table format: one unit per lane on the nonzero split (exponent per value).
template <bool RESID>
static KernelPick pick_kernel_tbl(int k, int r_lo) {
    switch (k) {
        case 1: return pick_one<1, 0, 1, RESID, true>(r_lo);
        case 2: return pick_one<2, 0, 1, RESID, true>(r_lo);
        case 3: return r_lo == 4 ? pick_one<3, 4, 1, RESID, true>(r_lo) : pick_one<3, -1, 1, RESID, true>(r_lo);
        case SRC_FP32: return pick_one<SRC_FP32, 0, 1, RESID>(r_lo);
        case SRC_FP16: return pick_one<SRC_FP16, 0, 1, RESID>(r_lo);
        case SRC_BF16: return pick_one<SRC_BF16, 0, 1, RESID>(r_lo);
        default: return pick_one<SRC_FP64, 0, 1, RESID>(r_lo);
    }
}

template <bool RESID>
static KernelPick pick_kernel_t(int k, int r_lo, int upl) {
    switch (k) {
        case 1: return pick_upl<1, 0, RESID>(upl, r_lo);
        case 2: return pick_upl<2, 0, RESID>(upl, r_lo);
        case 3:
            switch (r_lo) {
                case 0: return pick_upl<3, 0, RESID>(upl, r_lo);
                case 4: return pick_upl<3, 4, RESID>(upl, r_lo);
                case 8: return pick_upl<3, 8, RESID>(upl, r_lo);
                default: return pick_upl<3, 16, RESID>(upl, r_lo);
            }
        case SRC_FP32: return pick_upl<SRC_FP32, 0, RESID>(upl, r_lo);
        case SRC_FP16: return pick_one<SRC_FP16, 0, 1, RESID>(r_lo);     // 16-bit baselines: one unit per lane
        case SRC_BF16: return pick_one<SRC_BF16, 0, 1, RESID>(r_lo);
        default: return pick_upl<SRC_FP64, 0, RESID>(upl, r_lo);
    }
}

// The level-3 direct nonzero split for a handle in the default layout.
template <bool RESID>
static KernelPick pick_direct_std3() {
    KernelPick kp;
    kp.fn = k_spmv_direct_std3<RESID>;
    kp.warps = 8;
    kp.L = chunk_stage_layout<3, 4, 1>(8, 4);    // unused by the kernel
    kp.smem = 0;
    return kp;
}

static KernelPick pick_kernel(int k, int r_lo, int upl, bool resid, bool tbl) {
    if (tbl) return resid ? pick_kernel_tbl<true>(k, r_lo) : pick_kernel_tbl<false>(k, r_lo);
    return resid ? pick_kernel_t<true>(k, r_lo, upl) : pick_kernel_t<false>(k, r_lo, upl);
}

// Occupancy-derived resident blocks per SM for each kernel (cached per device).
static int resident_blocks(const KernelPick& kp) {
    const int nb = occupancy_cached((const void*)kp.fn, kp.warps * 32, kp.smem);
    return nb < 1 ? 1 : nb;
}

int launch_spmv(gse_matrix* h, int k, int epi, const SpmvArgs& a, cudaStream_t s, int upl_override) {
    int upl = upl_override ? upl_override : units_per_lane(h);
    if (upl == GSE_SCHEDULE_ROWS)
        return lanerow_ok(h, k) ? launch_lanerow(h, k, epi, a, s) : launch_rows(h, k, epi, a, s);
    if (h->v.tbl || src16(k)) upl = 1;         // the table format and the 16-bit baselines run one unit per lane
    const bool std3 = upl == 1 && k == 3 && h->n_seg == 3 && lanerow_format(h->v, h->group_size, h->n_seg) &&
                      h->v.col_mask == 0xFFFFFFFFu;
    const KernelPick kp = std3 ? (epi == EPI_RESID ? pick_direct_std3<true>() : pick_direct_std3<false>())
                               : pick_kernel(k, h->v.r_lo, upl, epi == EPI_RESID, h->v.tbl != 0);
    const int64_t ch = 256 * upl;
    const int64_t n_chunks = (h->v.nnz + ch - 1) / ch;
    const int64_t resident = (int64_t)h->num_sms * resident_blocks(kp);
    int64_t g = (n_chunks + kp.warps - 1) / kp.warps;          // super-chunks
    if (g > resident) g = resident;
    const int64_t gmin = (h->v.n_empty + kp.warps * 32 - 1) / (kp.warps * 32);
    if (g < gmin) g = gmin < resident ? gmin : resident;
    if (g < 1) g = 1;
    Epi e;
    e.kind = epi;
    e.y = a.y;
    e.b = a.b;
    e.p = a.p;
    kp.fn<<<(unsigned)g, kp.warps * 32, kp.smem, s>>>(h->v, a.x, e, n_chunks, kp.L, h->d_err, a.skip_flag);
    if (n_chunks > 1) {
        int64_t gf = (n_chunks + 255) / 256;
        if (gf > (int64_t)h->num_sms * 8) gf = (int64_t)h->num_sms * 8;
        if (upl == 1) k_spmv_fix<1><<<(unsigned)gf, 256, 0, s>>>(h->v, e, n_chunks, a.skip_flag);
        else if (upl == 2) k_spmv_fix<2><<<(unsigned)gf, 256, 0, s>>>(h->v, e, n_chunks, a.skip_flag);
        else k_spmv_fix<4><<<(unsigned)gf, 256, 0, s>>>(h->v, e, n_chunks, a.skip_flag);
    }
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

}  // namespace gse

using namespace gse;

static bool level_ok(gse_matrix* h, int k) { return level_available(h, k); }

extern "C" int gse_spmv(gse_handle h, int k, const double* x, double* y, void* stream) {
    if (!h || !x || !y || !level_ok(h, k)) return GSE_ERR_INVALID;
    SpmvArgs a = {};
    a.x = x;
    a.y = y;
    return launch_spmv(h, k, EPI_STORE, a, (cudaStream_t)stream);
}

extern "C" int gse_test_timeout(gse_handle h, int on) {
    if (!h || !h->d_err) return GSE_ERR_INVALID;
    const int v = on ? 1 : 0;
    if (cudaMemcpy(h->d_err + 2, &v, sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess) return GSE_ERR_CUDA;
    return GSE_OK;
}

extern "C" int gse_set_schedule(gse_handle h, int upl) {
    if (!h || !(upl == 0 || upl == 1 || upl == 2 || upl == 4 || upl == GSE_SCHEDULE_ROWS)) return GSE_ERR_INVALID;
    if (upl == GSE_SCHEDULE_ROWS && (h->row_span256 > GSE_ROW_SPAN_MAX || h->row_span128 > GSE_ROW_SPAN_MAX))
        return GSE_ERR_UNSUPPORTED;
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
    const int cands[4] = {GSE_SCHEDULE_ROWS, 1, 2, 4};
    float best = 1e30f;
    int best_upl = units_per_lane(h);
    SpmvArgs a = {};
    a.x = x;
    a.y = y;
    for (int ci = 0; ci < 4; ci++) {
        const int upl = cands[ci];
        if (upl == GSE_SCHEDULE_ROWS && (h->row_span256 > GSE_ROW_SPAN_MAX || h->row_span128 > GSE_ROW_SPAN_MAX))
            continue;
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
