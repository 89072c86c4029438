// encode.cu -- gse_encode (Sec. III-B, Alg. 1, Fig. 3) and the handle's life
// cycle: validation, the group-shared-exponent encoder, row-end mask and chunk
// metadata, row statistics, baseline values, export/decode, footprint.
#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "pool.cuh"
#include "spmv_core.cuh"

namespace gse {

// ---- validation -------------------------------------------------------------

__global__ void k_validate_rows(const int32_t* row_ptr, int64_t n, int64_t nnz, int* err,
                                int* max_len) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = row_ptr[r], t = row_ptr[r + 1];
        if (t < s || s < 0 || t > nnz) atomicOr(err, 1);
        else atomicMax(max_len, t - s);
        if (r == 0 && s != 0) atomicOr(err, 1);
        if (r == n - 1 && t != nnz) atomicOr(err, 1);
    }
}

__global__ void k_validate_cols(const int32_t* col, int64_t nnz, int64_t n_cols, int* err) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int32_t c = col[e];
        if (c < 0 || c >= n_cols) atomicOr(err, 1);
    }
}

// ---- the encoder ------------------------------------------------------------
// One thread per nonzero; a warp covers 32 consecutive nonzeros, i.e. 32/G
// whole groups.  Per group: E_g = max biased exponent + 1 (0 if all are zero
// or subnormal); per value: M = floor(|v| 2^(W - (E_g - 1023))) (round toward
// zero, as Alg. 1), then the head / tail1 / tail2 fields of Fig. 3.

struct EncParams {
    int G, s1, s2, s3, s3hi, r_lo, W, W1, W2, n_seg;
};

__global__ void k_encode(const double* __restrict__ val, const int32_t* __restrict__ col_in,
                         int64_t nnz, int64_t nnz_pad, EncParams p, int32_t* col, uint16_t* head,
                         uint16_t* tail1, uint16_t* t2hi, uint32_t* t2lo, uint16_t* gexp, int* err) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_pad; e += stride) {
        const bool real = e < nnz;
        const uint64_t b = real ? (uint64_t)__double_as_longlong(val[e]) : 0ull;
        const int ex = (int)((b >> 52) & 0x7FF);
        if (ex == 0x7FF) atomicOr(err, 2);
        int emax = ex;
        for (int o = 1; o < p.G; o <<= 1) emax = max(emax, __shfl_xor_sync(FULL, emax, o));
        const int Eg = emax == 0 ? 0 : emax + 1;
        uint64_t M = 0;
        if (ex != 0 && ex != 0x7FF) {
            const uint64_t S = (1ull << 52) | (b & 0xFFFFFFFFFFFFFull);
            const int sh = p.W - 52 - (Eg - ex);
            M = sh >= 0 ? (S << sh) : (-sh < 64 ? (S >> (-sh)) : 0ull);
        }
        const uint32_t sign = (uint32_t)(b >> 63);
        head[e] = (uint16_t)((sign << (p.s1 - 1)) | (uint32_t)(M >> (p.W - p.W1)));
        if (p.n_seg >= 2) tail1[e] = (uint16_t)((M >> (p.W - p.W2)) & ((1ull << p.s2) - 1));
        if (p.n_seg >= 3) {
            const uint32_t t2 = (uint32_t)(M & ((1ull << p.s3) - 1));
            t2hi[e] = (uint16_t)(t2 >> p.r_lo);
            if (p.r_lo > 0) {
                const int i = (int)(e & 7);
                const int bit = i * p.r_lo;
                uint32_t w = (t2 & ((1u << p.r_lo) - 1u)) << (bit & 31);
                const int lanes_per_word = 32 / p.r_lo;
                for (int o = 1; o < lanes_per_word; o <<= 1) w |= __shfl_xor_sync(FULL, w, o);
                if ((i % lanes_per_word) == 0)
                    t2lo[(e >> 3) * (p.r_lo / 4) + (bit >> 5)] = w;
            }
        }
        if ((lane & (p.G - 1)) == 0) gexp[e / p.G] = (uint16_t)Eg;
        col[e] = real ? col_in[e] : 0;
    }
}

// ---- global exponent table (Sec. III-B "Shared Exponents Extraction") -------

// Occurrences of every biased exponent among the values (counted per block in
// shared memory, then added to the global histogram).
__global__ void k_exp_hist(const double* __restrict__ val, int64_t nnz, unsigned long long* hist) {
    __shared__ unsigned int h[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) h[i] = 0;
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(&h[(unsigned)((uint64_t)__double_as_longlong(val[e]) >> 52) & 0x7FFu], 1u);
    __syncthreads();
    for (int i = threadIdx.x; i < 2048; i += blockDim.x)
        if (h[i]) atomicAdd(hist + i, (unsigned long long)h[i]);
}

// Largest biased exponent among the finite values (the sampled extraction
// still needs max + 1 of the whole matrix; Inf/NaN are flagged by the encoder).
__global__ void k_exp_max(const double* __restrict__ val, int64_t nnz, int* emax) {
    int m = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz; e += (int64_t)gridDim.x * blockDim.x) {
        const int ex = (int)(((uint64_t)__double_as_longlong(val[e]) >> 52) & 0x7FFu);
        if (ex != 0x7FF) m = max(m, ex);
    }
    for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xFFFFFFFFu, m, o));
    if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(emax, m);
}

// Sampled extraction (Sec. III-B): one warp per row block b reads the block's
// sampled row and counts each of its exponents once per row of the block.
__global__ void k_exp_hist_sampled(const int32_t* __restrict__ row_ptr, const double* __restrict__ val, int64_t n_rows,
                                   int64_t block_rows, const int64_t* __restrict__ sample, int64_t n_blocks,
                                   unsigned long long* hist) {
    const int lane = threadIdx.x & 31;
    const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
    for (int64_t b = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; b < n_blocks; b += warps) {
        const int64_t first = b * block_rows;
        const unsigned long long w = (unsigned long long)(first + block_rows <= n_rows ? block_rows : n_rows - first);
        const int64_t r = sample[b];
        for (int64_t j = row_ptr[r] + lane; j < row_ptr[r + 1]; j += 32) {
            const int ex = (int)(((uint64_t)__double_as_longlong(val[j]) >> 52) & 0x7FFu);
            if (ex != 0 && ex != 0x7FF) atomicAdd(hist + ex, w);
        }
    }
}

// Alg. 1 against the table through a per-exponent lookup: lut[e] = index | d << 8
// (the entry equal to e + 1 with d = 1, else the nearest larger entry T with
// d = T - e), then the segment split of k_encode.  The index is stored in the
// top bits of the column word (ei_shift < 32), or, with hb > 0, in the hb head
// bits right below the sign; p then carries the widths shortened by hb.
__global__ void k_encode_table(const double* __restrict__ val, const int32_t* __restrict__ col_in, int64_t nnz,
                               int64_t nnz_pad, EncParams p, const uint32_t* __restrict__ lut, int ei_shift, int hb,
                               int32_t* col, uint16_t* head, uint16_t* tail1, uint16_t* t2hi, uint32_t* t2lo,
                               int* err) {
    const unsigned FULL = 0xFFFFFFFFu;
    __shared__ uint32_t slut[2048];
    for (int i = threadIdx.x; i < 2048; i += blockDim.x) slut[i] = lut[i];
    __syncthreads();
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_pad; e += stride) {
        const bool real = e < nnz;
        const uint64_t b = real ? (uint64_t)__double_as_longlong(val[e]) : 0ull;
        const int ex = (int)((b >> 52) & 0x7FF);
        if (ex == 0x7FF) atomicOr(err, 2);
        const uint32_t l = slut[ex];
        const uint32_t idx = l & 0xFFu;
        const int d = (int)(l >> 8);
        uint64_t M = 0;
        if (ex != 0 && ex != 0x7FF) {
            const uint64_t S = (1ull << 52) | (b & 0xFFFFFFFFFFFFFull);
            const int sh = p.W - 52 - d;
            M = sh >= 0 ? (S << sh) : (-sh < 64 ? (S >> (-sh)) : 0ull);
        }
        const uint32_t sign = (uint32_t)(b >> 63);
        const uint32_t hidx = hb > 0 ? idx << (p.s1 - 1 - hb) : 0u;
        head[e] = (uint16_t)((sign << (p.s1 - 1)) | hidx | (uint32_t)(M >> (p.W - p.W1)));
        if (p.n_seg >= 2) tail1[e] = (uint16_t)((M >> (p.W - p.W2)) & ((1ull << p.s2) - 1));
        if (p.n_seg >= 3) {
            const uint32_t t2 = (uint32_t)(M & ((1ull << p.s3) - 1));
            t2hi[e] = (uint16_t)(t2 >> p.r_lo);
            if (p.r_lo > 0) {
                const int i = (int)(e & 7);
                const int bit = i * p.r_lo;
                uint32_t w = (t2 & ((1u << p.r_lo) - 1u)) << (bit & 31);
                const int lanes_per_word = 32 / p.r_lo;
                for (int o = 1; o < lanes_per_word; o <<= 1) w |= __shfl_xor_sync(FULL, w, o);
                if ((i % lanes_per_word) == 0)
                    t2lo[(e >> 3) * (p.r_lo / 4) + (bit >> 5)] = w;
            }
        }
        const uint32_t c = real ? (uint32_t)col_in[e] : 0u;
        col[e] = (int32_t)(ei_shift < 32 ? (c | (idx << ei_shift)) : c);
    }
}

// Host side of the table: the num_exp most frequent exponents (count
// descending, then exponent descending), each + 1, with max + 1 forced in
// place of the last kept entry when it did not make the cut; then the lookup
// of every exponent's entry and distance.  emax_all >= 0 gives the largest
// exponent when the histogram is a sample that may miss it.  Returns the number
// of entries.
static int build_table(const unsigned long long* hist, int emax_all, int num_exp, int16_t* table, uint32_t* lut) {
    int order[2047];
    int n_distinct = 0, emax = 0;
    for (int e = 2046; e >= 1; e--)
        if (hist[e]) {
            order[n_distinct++] = e;
            if (e > emax) emax = e;
        }
    if (emax_all >= 0) emax = emax_all;
    std::stable_sort(order, order + n_distinct, [&](int a, int b) { return hist[a] > hist[b]; });
    int n = 0;
    if (emax == 0) {
        table[n++] = 0;
    } else if (n_distinct == 0) {
        table[n++] = (int16_t)(emax + 1);         // an empty sample: max + 1 alone
    } else {
        bool has_max = false;
        for (int i = 0; i < n_distinct && n < num_exp; i++) {
            table[n++] = (int16_t)(order[i] + 1);
            has_max = has_max || order[i] == emax;
        }
        if (!has_max) table[n - 1] = (int16_t)(emax + 1);
    }
    for (int e = 0; e < 2048; e++) {
        uint32_t idx = 0, d = 1;
        if (e != 0) {
            int best = -1, bd = 1 << 30;
            for (int k = 0; k < n; k++) {
                const int diff = table[k] - e;
                if (diff == 1) { best = k; bd = 1; break; }
                if (diff > 0 && diff < bd) { bd = diff; best = k; }
            }
            if (best >= 0) { idx = (uint32_t)best; d = (uint32_t)bd; }
            else { idx = 0; d = 2047; }   // above every entry: cannot occur (max + 1 is in the table)
        }
        lut[e] = idx | (d << 8);
    }
    return n;
}

// ---- structure metadata -----------------------------------------------------

__global__ void k_rowend(const int32_t* row_ptr, int64_t n, uint32_t* rowend, int* flag_nonempty,
                         int* flag_empty) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = row_ptr[r], t = row_ptr[r + 1];
        if (t > s) atomicOr(rowend + ((t - 1) >> 5), 1u << ((t - 1) & 31));
        flag_nonempty[r] = t > s;
        flag_empty[r] = t == s;
    }
}

// Widest nonzero span of a block of RB consecutive rows, widened to whole
// groups of 32 nonzeros.
__global__ void k_row_span(const int32_t* row_ptr, int64_t n, int RB, int* out) {
    const int64_t nb = (n + RB - 1) / RB;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r1 = b * RB + RB < n ? b * RB + RB : n;
        const int64_t s = row_ptr[b * RB], t = row_ptr[r1];
        const int64_t span = (((t + 31) >> 5) << 5) - ((s >> 5) << 5);
        atomicMax(out, (int)(span < (1 << 30) ? span : (1 << 30)));
    }
}

// Widest slice of a tile of RB consecutive rows that the lane-row kernel
// stages: from its first nonzero rounded down to 8 to its end rounded up to 8.
__global__ void k_tile_span(const int32_t* row_ptr, int64_t n, int RB, int* out) {
    const int64_t nb = (n + RB - 1) / RB;
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nb; b += (int64_t)gridDim.x * blockDim.x) {
        const int64_t r1 = b * RB + RB < n ? b * RB + RB : n;
        const int64_t s = row_ptr[b * RB], t = row_ptr[r1];
        const int64_t span = (((t + 7) >> 3) << 3) - ((s >> 3) << 3);
        atomicMax(out, (int)(span < (1 << 30) ? span : (1 << 30)));
    }
}

__global__ void k_block_popc(const uint32_t* rowend, int64_t nblk, int* out) {
    for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < nblk; b += (int64_t)gridDim.x * blockDim.x) {
        int s = 0;
        for (int i = 0; i < 8; i++) s += __popc(rowend[b * 8 + i]);
        out[b] = s;
    }
}

// Exclusive scan of int32 (three passes: block sums, scan of the sums, apply).
constexpr int SCAN_BLOCK = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_BLOCK * SCAN_ITEMS;

__device__ int block_exclusive_scan(int v, int* sh, int* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += t;
    }
    __syncthreads();
    if (lane == 31) sh[w] = incl;
    __syncthreads();
    if (w == 0) {
        const int nw = blockDim.x >> 5;
        int x = lane < nw ? sh[lane] : 0;
        int xi = x;
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xFFFFFFFFu, xi, o);
            if (lane >= o) xi += t;
        }
        if (lane < nw) sh[lane] = xi - x;
        if (lane == 31) sh[32] = xi;
    }
    __syncthreads();
    const int res = incl - v + sh[w];
    if (total) *total = sh[32];
    return res;
}

__global__ void k_scan_reduce(const int* in, int64_t n, int* bsum) {
    __shared__ int sh[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int s = 0;
    for (int i = 0; i < SCAN_ITEMS; i++) {
        const int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        if (idx < n) s += in[idx];
    }
    int total;
    block_exclusive_scan(s, sh, &total);
    if (threadIdx.x == 0) bsum[blockIdx.x] = total;
}

__global__ void k_scan_bsum(int* bsum, int64_t nb, int* grand_total) {
    __shared__ int sh[33];
    int carry = 0;
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t i = base + threadIdx.x;
        const int v = i < nb ? bsum[i] : 0;
        int total;
        const int ex = block_exclusive_scan(v, sh, &total);
        if (i < nb) bsum[i] = ex + carry;
        carry += total;
        __syncthreads();
    }
    if (threadIdx.x == 0) *grand_total = carry;
}

__global__ void k_scan_apply(const int* in, int64_t n, const int* bsum, int* out) {
    __shared__ int sh[33];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    int v[SCAN_ITEMS];
    int s = 0;
    for (int i = 0; i < SCAN_ITEMS; i++) {
        const int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        v[i] = idx < n ? in[idx] : 0;
        s += v[i];
    }
    int ex = block_exclusive_scan(s, sh, nullptr) + bsum[blockIdx.x];
    for (int i = 0; i < SCAN_ITEMS; i++) {
        const int64_t idx = base + (int64_t)threadIdx.x * SCAN_ITEMS + i;
        if (idx < n) out[idx] = ex;
        ex += v[i];
    }
}

// out[i] = exclusive prefix of in[0..i); *total (device) = sum.  tmp: ceil(n/TILE) ints.
static void exclusive_scan(const int* in, int64_t n, int* out, int* tmp, int* total, cudaStream_t s) {
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb > 0) {
        k_scan_reduce<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, n, tmp);
        k_scan_bsum<<<1, SCAN_BLOCK, 0, s>>>(tmp, nb, total);
        k_scan_apply<<<(unsigned)nb, SCAN_BLOCK, 0, s>>>(in, n, tmp, out);
    } else {
        cudaMemsetAsync(total, 0, sizeof(int), s);
    }
}

__global__ void k_scatter_rows(const int* flag, const int* pos, int64_t n, int32_t* dst) {
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += (int64_t)gridDim.x * blockDim.x)
        if (flag[r]) dst[pos[r]] = (int32_t)r;
}

// 16-bit baselines: round to nearest even once from FP64 (cuda_fp16 /
// cuda_bf16 conversions); count finite values that became infinite.
__global__ void k_round16(const double* val, int64_t nnz, int64_t nnz_pad, int kind, uint16_t* out,
                          unsigned long long* n_overflow) {
    unsigned long long ov = 0;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_pad; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = e < nnz ? val[e] : 0.0;
        uint16_t b;
        if (kind == GSE_LEVEL_FP16) {
            b = __half_as_ushort(__double2half(v));
            ov += isfinite(v) && (b & 0x7C00u) == 0x7C00u;
        } else {
            b = __bfloat16_as_ushort(__double2bfloat16(v));
            ov += isfinite(v) && (b & 0x7F80u) == 0x7F80u;
        }
        out[e] = b;
    }
    if (ov) atomicAdd(n_overflow, ov);
}

__global__ void k_pad_values(const double* val, int64_t nnz, int64_t nnz_pad, double* v64, float* v32) {
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nnz_pad; e += (int64_t)gridDim.x * blockDim.x) {
        const double v = e < nnz ? val[e] : 0.0;
        if (v64) v64[e] = v;
        if (v32) v32[e] = __double2float_rn(v);
    }
}

template <int K, int R>
__global__ void k_decode(MatView m, double* out) {
    const int64_t nunits = (m.nnz + 7) / 8;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < nunits; u += (int64_t)gridDim.x * blockDim.x) {
        int col[8];
        double a[8];
        load_unit<K, R>(m, u, col, a);
        for (int i = 0; i < 8; i++)
            if (u * 8 + i < m.nnz) out[u * 8 + i] = a[i];
    }
}

static unsigned grid_for(int64_t n, int threads = 256) {
    int64_t g = (n + threads - 1) / threads;
    if (g > 65535LL * 16) g = 65535LL * 16;
    if (g < 1) g = 1;
    return (unsigned)g;
}

static void free_all(gse_matrix* h) {
    void* bufs[] = {h->buf_col, h->buf_head, h->buf_tail1, h->buf_t2hi, h->buf_t2lo, h->buf_gexp,
                    h->buf_rowend, h->buf_blk_row0, h->buf_nzrow, h->buf_empty, h->buf_row_ptr,
                    h->buf_val64, h->buf_val32, h->buf_val16, h->buf_valbf, h->buf_carry, h->buf_part, h->buf_etab,
                    h->red_partial, h->red_counter, h->red_result, h->d_err};
    for (void* b : bufs) pool_free(b);
}

}  // namespace gse

namespace gse {

cudaMemPool_t device_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof(props));
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t p = nullptr;
        if (cudaMemPoolCreate(&p, &props) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        uint64_t keep = UINT64_MAX;                  // freed blocks stay cached for the next matrix
        cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = p;
    }
    return pools[dev];
}

}  // namespace gse

using namespace gse;

void gse_free_workspace(gse_matrix* h);  // solver.cu

extern "C" const char* gse_strerror(int status) {
    switch (status) {
        case GSE_OK: return "ok";
        case GSE_MAXITER: return "maximum iterations reached";
        case GSE_BREAKDOWN: return "solver breakdown";
        case GSE_NONFINITE: return "non-finite value in the solver";
        case GSE_TIMEOUT: return "bounded wait timed out";
        case GSE_ERR_INVALID: return "invalid argument or malformed CSR";
        case GSE_ERR_NONFINITE: return "input value is Inf or NaN";
        case GSE_ERR_OOM: return "device allocation failed";
        case GSE_ERR_CUDA: return "CUDA runtime error";
        case GSE_ERR_UNSUPPORTED: return "unsupported parameter";
        default: return "unknown status";
    }
}

// A buffer the handle keeps (from the library's pool, ordered on stream s).
template <typename T>
static int dev_alloc(T** p, size_t count, size_t* acc, cudaStream_t s) {
    return pool_alloc(p, count, acc, s);
}

// Options of the table format (num_exp 0: the per-group format).
struct TableOpts {
    int num_exp = 0;
    int index_place = GSE_INDEX_AUTO;
    int64_t block_rows = 0;             // > 0: sampled extraction, one row per block
    const int64_t* sample_rows = nullptr;
};

// Encoder temporaries come from the library's pool and go back with
// cudaFreeAsync on the encoder's stream: allocating and releasing them never
// waits for other streams' work (cudaFree would wait for the whole device, e.g.
// a solver batch running while the next matrix encodes).
template <typename T>
static int tmp_alloc(T** p, size_t count, cudaStream_t s) {
    return pool_alloc(p, count, nullptr, s);
}

static int encode_impl(const gse_csr* csr, int G, const int* seg_bits, int n_seg, cudaStream_t s,
                       gse_matrix* h, const TableOpts& topt) {
    const int num_exp = topt.num_exp;
    const int64_t n = csr->n_rows, nnz = csr->nnz;
    h->group_size = G;
    h->n_seg = n_seg;
    int sb[3] = {0, 0, 0};
    for (int i = 0; i < n_seg; i++) sb[i] = seg_bits[i];
    memcpy(h->seg_bits, sb, sizeof(sb));
    MatView& v = h->v;
    v.nnz = nnz;
    v.n_rows = n;
    v.n_cols = csr->n_cols;
    v.nnz_pad = ((nnz + GSE_CHUNK_MAX - 1) / GSE_CHUNK_MAX) * GSE_CHUNK_MAX;
    if (v.nnz_pad == 0) v.nnz_pad = GSE_CHUNK_MAX;
    v.g_shift = G == 8 ? 3 : G == 16 ? 4 : 5;
    v.s1 = sb[0];
    v.s2 = n_seg >= 2 ? sb[1] : 0;
    v.s3 = n_seg >= 3 ? sb[2] : 0;
    v.s3hi = v.s3 > 16 ? 16 : v.s3;
    v.r_lo = v.s3 - v.s3hi;
    v.W1 = sb[0] - 1;
    v.W2 = v.W1 + v.s2;
    v.W3 = v.W2 + v.s3;
    const int64_t npad = v.nnz_pad, nblk = npad / 256;
    size_t acc = 0;
    int rc;
#define ALLOC(ptr, T, cnt) \
    do { T* _p; if ((rc = dev_alloc(&_p, (size_t)(cnt), &acc, s)) != GSE_OK) return rc; ptr = _p; } while (0)
    ALLOC(h->buf_row_ptr, int32_t, n + 1);
    ALLOC(h->buf_col, int32_t, npad);
    ALLOC(h->buf_head, uint16_t, npad);
    if (n_seg >= 2) ALLOC(h->buf_tail1, uint16_t, npad);
    if (n_seg >= 3) ALLOC(h->buf_t2hi, uint16_t, npad);
    if (n_seg >= 3 && v.r_lo > 0) ALLOC(h->buf_t2lo, uint32_t, npad / 8 * v.r_lo / 4);
    ALLOC(h->buf_gexp, uint16_t, npad / G);
    ALLOC(h->buf_rowend, uint32_t, npad / 32);
    ALLOC(h->buf_blk_row0, int32_t, nblk + 1);
    ALLOC(h->buf_carry, double, nblk);
    ALLOC(h->buf_part, double, nblk);
    h->red_capacity = h->num_sms * 32;
    ALLOC(h->red_partial, double, h->red_capacity);
    ALLOC(h->red_counter, unsigned, 4);
    ALLOC(h->red_result, double, 4);
    ALLOC(h->d_err, int, 4);
    v.inject = h->d_err + 2;     // the timeout test flag (gse_test_timeout), cleared below
    h->bytes_matrix = acc;
    // temporaries
    int *d_err = nullptr, *d_flag = nullptr, *d_flag2 = nullptr, *d_pos = nullptr;
    int *d_scan_tmp = nullptr, *d_total = nullptr;
    double* d_val = nullptr;
    const int32_t* d_colin = nullptr;
    int32_t* d_colin_own = nullptr;
    const int64_t nflags = n > nblk ? n : nblk;
    if ((rc = tmp_alloc(&d_err, 12, s)) != GSE_OK) return rc;
    bool ok = tmp_alloc(&d_flag, nflags + 1, s) == GSE_OK && tmp_alloc(&d_flag2, nflags + 1, s) == GSE_OK &&
              tmp_alloc(&d_pos, nflags + 1, s) == GSE_OK &&
              tmp_alloc(&d_scan_tmp, nflags / SCAN_TILE + 2, s) == GSE_OK &&
              tmp_alloc(&d_total, 4, s) == GSE_OK;
    if (ok && !csr->on_device) ok = tmp_alloc(&d_val, nnz, s) == GSE_OK && tmp_alloc(&d_colin_own, nnz, s) == GSE_OK;
    int status = GSE_OK;
    if (!ok) status = GSE_ERR_OOM;
    if (status == GSE_OK) {
        cudaMemsetAsync(d_err, 0, 12 * sizeof(int), s);
        int32_t* rp = (int32_t*)h->buf_row_ptr;
        if (csr->on_device) {
            cudaMemcpyAsync(rp, csr->row_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyDeviceToDevice, s);
            d_colin = csr->col_idx;
        } else {
            cudaMemcpyAsync(rp, csr->row_ptr, (n + 1) * sizeof(int32_t), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(d_colin_own, csr->col_idx, nnz * sizeof(int32_t), cudaMemcpyHostToDevice, s);
            cudaMemcpyAsync(d_val, csr->val, nnz * sizeof(double), cudaMemcpyHostToDevice, s);
            d_colin = d_colin_own;
        }
        const double* val = csr->on_device ? csr->val : d_val;
        // validation
        if (n > 0) k_validate_rows<<<grid_for(n), 256, 0, s>>>(rp, n, nnz, d_err, d_err + 1);
        if (nnz > 0) k_validate_cols<<<grid_for(nnz), 256, 0, s>>>(d_colin, nnz, v.n_cols, d_err);
        int herr[2] = {0, 0};
        cudaMemcpyAsync(herr, d_err, 2 * sizeof(int), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) status = GSE_ERR_CUDA;
        else if (herr[0]) status = GSE_ERR_INVALID;
        h->max_row_len = herr[1];
        if (status == GSE_OK) {
            EncParams p;
            p.G = G;
            p.s1 = v.s1;
            p.s2 = v.s2;
            p.s3 = v.s3;
            p.s3hi = v.s3hi;
            p.r_lo = v.r_lo;
            p.W = n_seg == 1 ? v.W1 : n_seg == 2 ? v.W2 : v.W3;
            p.W1 = v.W1;
            p.W2 = v.W2;
            p.n_seg = n_seg;
            v.tbl = 0;
            v.ei_shift = 32;
            v.col_mask = 0xFFFFFFFFu;
            v.hi_shift = 0;
            v.hi_mask = 0;
            h->num_exp = 0;
            h->index_in_head = 0;
            if (num_exp > 0) {
                // the table format: histogram on the device, table and lookup on the host
                unsigned long long* d_hist = nullptr;
                uint32_t* d_lut = nullptr;
                int64_t* d_sample = nullptr;
                const bool sampled = topt.block_rows > 0;
                const int64_t n_blocks = sampled ? (n + topt.block_rows - 1) / topt.block_rows : 0;
                if (tmp_alloc(&d_hist, 2048, s) != GSE_OK || tmp_alloc(&d_lut, 2048, s) != GSE_OK ||
                    (sampled && tmp_alloc(&d_sample, (size_t)n_blocks + 1, s) != GSE_OK)) {
                    status = GSE_ERR_OOM;
                } else {
                    cudaMemsetAsync(d_hist, 0, 2048 * sizeof(unsigned long long), s);
                    int emax_all = -1;
                    if (sampled) {
                        // the largest exponent over all values, then the sampled rows' counts
                        cudaMemsetAsync(d_err + 7, 0, sizeof(int), s);
                        if (nnz > 0) k_exp_max<<<h->num_sms * 4, 512, 0, s>>>(val, nnz, d_err + 7);
                        cudaMemcpyAsync(d_sample, topt.sample_rows, n_blocks * sizeof(int64_t), cudaMemcpyHostToDevice, s);
                        if (n_blocks > 0)
                            k_exp_hist_sampled<<<grid_for(n_blocks * 32), 256, 0, s>>>(rp, val, n, topt.block_rows,
                                                                                      d_sample, n_blocks, d_hist);
                        cudaMemcpyAsync(&emax_all, d_err + 7, sizeof(int), cudaMemcpyDeviceToHost, s);
                    } else if (nnz > 0) {
                        k_exp_hist<<<h->num_sms * 4, 512, 0, s>>>(val, nnz, d_hist);
                    }
                    std::vector<unsigned long long> hist(2048);
                    cudaMemcpyAsync(hist.data(), d_hist, 2048 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s);
                    if (cudaStreamSynchronize(s) != cudaSuccess) status = GSE_ERR_CUDA;
                    std::vector<uint32_t> lut(2048);
                    int16_t table[64] = {0};
                    const int nt = status == GSE_OK ? build_table(hist.data(), emax_all, num_exp, table, lut.data()) : 1;
                    int ei_bits = 0;
                    while ((1 << ei_bits) < nt) ei_bits++;
                    // where the index goes: the column word while its spare bits hold it
                    // (Sec. III-C), else the head right below the sign
                    const bool col_fits = ei_bits == 0 || v.n_cols <= (int64_t)(0xFFFFFFFFu >> ei_bits) + 1;
                    const bool in_head = ei_bits > 0 && (topt.index_place == GSE_INDEX_VALUE ||
                                                         (topt.index_place == GSE_INDEX_AUTO && !col_fits));
                    if (status == GSE_OK && !in_head && !col_fits) status = GSE_ERR_UNSUPPORTED;
                    if (status == GSE_OK && in_head && ei_bits > v.s1 - 2) status = GSE_ERR_UNSUPPORTED;
                    const int hb = in_head ? ei_bits : 0;
                    int16_t dtab[64] = {0};
                    for (int i = 0; i < nt; i++) dtab[i] = (int16_t)(table[i] + hb);
                    int16_t* d_etab = nullptr;
                    if (status == GSE_OK && dev_alloc(&d_etab, 64, &h->bytes_matrix, s) != GSE_OK) status = GSE_ERR_OOM;
                    if (status == GSE_OK) {
                        h->buf_etab = d_etab;
                        cudaMemcpyAsync(d_etab, dtab, sizeof(dtab), cudaMemcpyHostToDevice, s);
                        v.etab = d_etab;
                        v.tbl = 1;
                        if (in_head) {
                            v.hi_shift = v.s1 - 1 - hb;
                            v.hi_mask = (1u << hb) - 1u;
                        } else {
                            v.ei_shift = 32 - ei_bits;
                            v.col_mask = 0xFFFFFFFFu >> ei_bits;
                        }
                        memcpy(h->etab_host, table, sizeof(table));
                        h->num_exp = nt;
                        h->index_in_head = in_head;
                        EncParams pt = p;        // widths shortened by the index bits in the head
                        pt.W -= hb;
                        pt.W1 -= hb;
                        pt.W2 -= hb;
                        cudaMemcpyAsync(d_lut, lut.data(), 2048 * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
                        cudaMemsetAsync(h->buf_gexp, 0, npad / G * sizeof(uint16_t), s);
                        k_encode_table<<<grid_for(npad), 256, 0, s>>>(val, d_colin, nnz, npad, pt, d_lut, v.ei_shift, hb,
                                                                      (int32_t*)h->buf_col, (uint16_t*)h->buf_head,
                                                                      (uint16_t*)h->buf_tail1, (uint16_t*)h->buf_t2hi,
                                                                      (uint32_t*)h->buf_t2lo, d_err);
                        cudaStreamSynchronize(s);          // the lookup buffer is freed right below
                    }
                }
                if (d_hist) cudaFreeAsync(d_hist, s);
                if (d_lut) cudaFreeAsync(d_lut, s);
                if (d_sample) cudaFreeAsync(d_sample, s);
            } else {
                k_encode<<<grid_for(npad), 256, 0, s>>>(val, d_colin, nnz, npad, p, (int32_t*)h->buf_col,
                                                        (uint16_t*)h->buf_head, (uint16_t*)h->buf_tail1,
                                                        (uint16_t*)h->buf_t2hi, (uint32_t*)h->buf_t2lo,
                                                        (uint16_t*)h->buf_gexp, d_err);
            }
        }
        if (status == GSE_OK) {
            // row ends, empty rows
            cudaMemsetAsync(h->buf_rowend, 0, npad / 32 * sizeof(uint32_t), s);
            if (n > 0) k_rowend<<<grid_for(n), 256, 0, s>>>(rp, n, (uint32_t*)h->buf_rowend, d_flag, d_flag2);
            exclusive_scan(d_flag, n, d_pos, d_scan_tmp, d_total, s);
            int n_nonempty = 0;
            cudaMemcpyAsync(&n_nonempty, d_total, sizeof(int), cudaMemcpyDeviceToHost, s);
            cudaMemcpyAsync(herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) status = GSE_ERR_CUDA;
            else if (herr[0] & 2) status = GSE_ERR_NONFINITE;
            v.n_nonempty = n_nonempty;
            v.n_empty = n - n_nonempty;
            if (status == GSE_OK && v.n_empty > 0) {
                int32_t *nz, *em;
                if (dev_alloc(&nz, (size_t)n_nonempty, &h->bytes_matrix, s) != GSE_OK ||
                    (h->buf_nzrow = nz, dev_alloc(&em, (size_t)v.n_empty, &h->bytes_matrix, s)) != GSE_OK) {
                    status = GSE_ERR_OOM;
                } else {
                    h->buf_empty = em;
                    k_scatter_rows<<<grid_for(n), 256, 0, s>>>(d_flag, d_pos, n, nz);
                    exclusive_scan(d_flag2, n, d_pos, d_scan_tmp, d_total, s);
                    k_scatter_rows<<<grid_for(n), 256, 0, s>>>(d_flag2, d_pos, n, em);
                }
            }
            if (status == GSE_OK) {
                cudaMemsetAsync(d_err + 4, 0, 5 * sizeof(int), s);
                const int rbs[3] = {32, 128, 256};
                for (int q = 0; q < 3; q++)
                    if (n > 0) k_row_span<<<grid_for((n + rbs[q] - 1) / rbs[q]), 256, 0, s>>>(rp, n, rbs[q], d_err + 4 + q);
                if (n > 0) k_tile_span<<<grid_for((n + 31) / 32), 256, 0, s>>>(rp, n, 32, d_err + 7);
                if (n > 0) k_tile_span<<<grid_for((n + 63) / 64), 256, 0, s>>>(rp, n, 64, d_err + 8);
                int span[5] = {0, 0, 0, 0, 0};
                cudaMemcpyAsync(span, d_err + 4, 5 * sizeof(int), cudaMemcpyDeviceToHost, s);
                k_block_popc<<<grid_for(nblk), 256, 0, s>>>((uint32_t*)h->buf_rowend, nblk, d_flag);
                exclusive_scan(d_flag, nblk, (int*)h->buf_blk_row0, d_scan_tmp, d_total, s);
                cudaMemsetAsync(h->red_counter, 0, 4 * sizeof(unsigned), s);
                cudaMemsetAsync(h->d_err, 0, 4 * sizeof(int), s);
                if (cudaStreamSynchronize(s) != cudaSuccess) status = GSE_ERR_CUDA;
                h->row_span = span[0];
                h->row_span128 = span[1];
                h->row_span256 = span[2];
                h->tile_span32 = span[3];
                h->tile_span64 = span[4];
            }
        }
    }
    cudaFreeAsync(d_err, s);
    if (d_flag) cudaFreeAsync(d_flag, s);
    if (d_flag2) cudaFreeAsync(d_flag2, s);
    if (d_pos) cudaFreeAsync(d_pos, s);
    if (d_scan_tmp) cudaFreeAsync(d_scan_tmp, s);
    if (d_total) cudaFreeAsync(d_total, s);
    if (d_val) cudaFreeAsync(d_val, s);
    if (d_colin_own) cudaFreeAsync(d_colin_own, s);
    if (status != GSE_OK) return status;
    v.col = (const int32_t*)h->buf_col;
    v.head = (const uint16_t*)h->buf_head;
    v.tail1 = (const uint16_t*)h->buf_tail1;
    v.t2hi = (const uint16_t*)h->buf_t2hi;
    v.t2lo = (const uint32_t*)h->buf_t2lo;
    v.gexp = (const uint16_t*)h->buf_gexp;
    v.rowend = (const uint32_t*)h->buf_rowend;
    v.blk_row0 = (const int32_t*)h->buf_blk_row0;
    v.nzrow = (const int32_t*)h->buf_nzrow;
    v.empty = (const int32_t*)h->buf_empty;
    v.row_ptr = (const int32_t*)h->buf_row_ptr;
    v.carry = (double*)h->buf_carry;
    v.part = (double*)h->buf_part;
    h->mean_row_len = n > 0 ? (double)nnz / (double)n : 0.0;
    // schedule: short rows in every 256-row block -> one row per lane; otherwise
    // the nonzero split, one unit of 8 per lane, 8-warp CTAs (gse_autotune refines this)
    h->schedule_auto = h->row_span256 <= GSE_ROW_SPAN_MAX && h->max_row_len <= 64 ? GSE_SCHEDULE_ROWS : 1;
    h->schedule_forced = 0;
    return GSE_OK;
#undef ALLOC
}

static int encode_entry(const gse_csr* csr, int group_size, const int* seg_bits, int n_seg, void* stream,
                        gse_handle* out, const TableOpts& topt) {
    if (!csr || !seg_bits || !out) return GSE_ERR_INVALID;
    *out = nullptr;
    if (csr->n_rows < 0 || csr->n_cols < 0 || csr->nnz < 0 || csr->nnz >= (1LL << 31) ||
        csr->n_rows >= (1LL << 31) || csr->n_cols >= (1LL << 31))
        return GSE_ERR_INVALID;
    if (!csr->row_ptr || (csr->nnz > 0 && (!csr->col_idx || !csr->val))) return GSE_ERR_INVALID;
    if (n_seg < 1 || n_seg > 3) return GSE_ERR_INVALID;
    if (seg_bits[0] < 2 || seg_bits[0] > 16) return GSE_ERR_INVALID;
    if (n_seg >= 2 && (seg_bits[1] < 1 || seg_bits[1] > 16)) return GSE_ERR_INVALID;
    if (n_seg >= 3) {
        const int s3 = seg_bits[2];
        if (s3 < 1 || s3 > 32) return GSE_ERR_INVALID;
        if (s3 > 16 && s3 != 20 && s3 != 24 && s3 != 32) return GSE_ERR_UNSUPPORTED;
    }
    if (group_size != 8 && group_size != 16 && group_size != 32) return GSE_ERR_UNSUPPORTED;
    if (topt.block_rows > 0) {
        // one sampled row per block of block_rows rows, inside its block (host array)
        if (!topt.sample_rows && csr->n_rows > 0) return GSE_ERR_INVALID;
        const int64_t nb = (csr->n_rows + topt.block_rows - 1) / topt.block_rows;
        for (int64_t b = 0; b < nb; b++) {
            const int64_t r = topt.sample_rows[b], lo = b * topt.block_rows;
            if (r < lo || r >= lo + topt.block_rows || r >= csr->n_rows) return GSE_ERR_INVALID;
        }
    }
    gse_matrix* h = (gse_matrix*)calloc(1, sizeof(gse_matrix));
    if (!h) return GSE_ERR_OOM;
    cudaGetDevice(&h->device);
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
    if (h->num_sms < 1) h->num_sms = 1;
    const int rc = encode_impl(csr, group_size, seg_bits, n_seg, (cudaStream_t)stream, h, topt);
    if (rc != GSE_OK) {
        cudaStreamSynchronize((cudaStream_t)stream);     // nothing queued may still use the buffers
        free_all(h);
        free(h);
        return rc;
    }
    *out = h;
    return GSE_OK;
}

extern "C" int gse_encode(const gse_csr* csr, int group_size, const int* seg_bits, int n_seg,
                          void* stream, gse_handle* out) {
    return encode_entry(csr, group_size, seg_bits, n_seg, stream, out, TableOpts());
}

extern "C" int gse_encode_table_ex(const gse_csr* csr, int num_exp, const int* seg_bits, int n_seg, int index_place,
                                   int64_t block_rows, const int64_t* sample_rows, void* stream, gse_handle* out) {
    if (out) *out = nullptr;
    if (num_exp < 1 || num_exp > 64 || block_rows < 0) return GSE_ERR_INVALID;
    if (index_place != GSE_INDEX_AUTO && index_place != GSE_INDEX_COL && index_place != GSE_INDEX_VALUE)
        return GSE_ERR_INVALID;
    TableOpts t;
    t.num_exp = num_exp;
    t.index_place = index_place;
    t.block_rows = block_rows;
    t.sample_rows = sample_rows;
    // group_size only sizes the (unused) group-exponent array here
    return encode_entry(csr, 32, seg_bits, n_seg, stream, out, t);
}

extern "C" int gse_encode_table(const gse_csr* csr, int num_exp, const int* seg_bits, int n_seg, void* stream,
                                gse_handle* out) {
    return gse_encode_table_ex(csr, num_exp, seg_bits, n_seg, GSE_INDEX_AUTO, 0, nullptr, stream, out);
}

extern "C" int gse_export_table(gse_handle h, int16_t* table, int* n_table, uint8_t* idx) {
    if (!h || !h->v.tbl) return GSE_ERR_INVALID;
    cudaDeviceSynchronize();
    if (table) memcpy(table, h->etab_host, (size_t)h->num_exp * sizeof(int16_t));
    if (n_table) *n_table = h->num_exp;
    const int64_t nnz = h->v.nnz;
    if (idx && nnz) {
        if (h->index_in_head) {
            std::vector<uint16_t> hd(nnz);
            GSE_CUDA_TRY(cudaMemcpy(hd.data(), h->buf_head, nnz * sizeof(uint16_t), cudaMemcpyDeviceToHost));
            for (int64_t e = 0; e < nnz; e++) idx[e] = (uint8_t)((hd[e] >> h->v.hi_shift) & h->v.hi_mask);
        } else {
            std::vector<uint32_t> c(nnz);
            GSE_CUDA_TRY(cudaMemcpy(c.data(), h->buf_col, nnz * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            for (int64_t e = 0; e < nnz; e++)
                idx[e] = h->v.ei_shift < 32 ? (uint8_t)(c[e] >> h->v.ei_shift) : 0;
        }
    }
    return GSE_OK;
}

extern "C" int gse_attach_values(gse_handle h, const gse_csr* csr, int bits, void* stream) {
    if (!h || !csr || (bits != 64 && bits != 32 && bits != GSE_LEVEL_FP16 && bits != GSE_LEVEL_BF16))
        return GSE_ERR_INVALID;
    if (csr->nnz != h->v.nnz || csr->n_rows != h->v.n_rows || (csr->nnz > 0 && !csr->val)) return GSE_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const double* val = csr->val;
    double* tmp = nullptr;
    if (!csr->on_device) {
        if (tmp_alloc(&tmp, (size_t)h->v.nnz + 1, s) != GSE_OK) return GSE_ERR_OOM;
        cudaMemcpyAsync(tmp, csr->val, h->v.nnz * sizeof(double), cudaMemcpyHostToDevice, s);
        val = tmp;
    }
    double* v64 = nullptr;
    float* v32 = nullptr;
    int rc = GSE_OK;
    if (bits == GSE_LEVEL_FP16 || bits == GSE_LEVEL_BF16) {
        void*& buf = bits == GSE_LEVEL_FP16 ? h->buf_val16 : h->buf_valbf;
        uint16_t* v16 = nullptr;
        unsigned long long* d_ov = nullptr;
        if (!buf) rc = dev_alloc(&v16, (size_t)h->v.nnz_pad, &h->bytes_matrix, s);
        if (rc == GSE_OK && v16) buf = v16;
        if (rc == GSE_OK && tmp_alloc(&d_ov, 1, s) != GSE_OK) rc = GSE_ERR_OOM;
        if (rc == GSE_OK) {
            cudaMemsetAsync(d_ov, 0, sizeof(unsigned long long), s);
            k_round16<<<grid_for(h->v.nnz_pad), 256, 0, s>>>(val, h->v.nnz, h->v.nnz_pad, bits, (uint16_t*)buf, d_ov);
            unsigned long long ov = 0;
            cudaMemcpyAsync(&ov, d_ov, sizeof(ov), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) rc = GSE_ERR_CUDA;
            if (bits == GSE_LEVEL_FP16) h->overflow16 = (int64_t)ov;
            if (bits == GSE_LEVEL_FP16) h->v.val16 = (const uint16_t*)buf;
            else h->v.valbf = (const uint16_t*)buf;
        }
        if (d_ov) cudaFreeAsync(d_ov, s);
        if (tmp) cudaFreeAsync(tmp, s);
        if (rc == GSE_OK && cudaGetLastError() != cudaSuccess) rc = GSE_ERR_CUDA;
        return rc;
    }
    if (bits == 64 && !h->buf_val64) rc = dev_alloc(&v64, (size_t)h->v.nnz_pad, &h->bytes_matrix, s);
    if (bits == 32 && !h->buf_val32) rc = dev_alloc(&v32, (size_t)h->v.nnz_pad, &h->bytes_matrix, s);
    if (rc == GSE_OK) {
        if (v64) h->buf_val64 = v64;
        if (v32) h->buf_val32 = v32;
        k_pad_values<<<grid_for(h->v.nnz_pad), 256, 0, s>>>(val, h->v.nnz, h->v.nnz_pad,
                                                            bits == 64 ? (double*)h->buf_val64 : nullptr,
                                                            bits == 32 ? (float*)h->buf_val32 : nullptr);
        h->v.val64 = (const double*)h->buf_val64;
        h->v.val32 = (const float*)h->buf_val32;
    }
    if (tmp) cudaFreeAsync(tmp, s);
    if (cudaGetLastError() != cudaSuccess) return GSE_ERR_CUDA;
    return rc;
}

extern "C" int gse_export(gse_handle h, uint16_t* head, uint16_t* tail1, uint32_t* tail2, int16_t* gexp) {
    if (!h) return GSE_ERR_INVALID;
    const int64_t nnz = h->v.nnz;
    cudaDeviceSynchronize();
    if (head && nnz) GSE_CUDA_TRY(cudaMemcpy(head, h->buf_head, nnz * sizeof(uint16_t), cudaMemcpyDeviceToHost));
    if (tail1 && nnz) {
        if (h->n_seg >= 2) GSE_CUDA_TRY(cudaMemcpy(tail1, h->buf_tail1, nnz * sizeof(uint16_t), cudaMemcpyDeviceToHost));
        else memset(tail1, 0, nnz * sizeof(uint16_t));
    }
    if (tail2 && nnz) {
        if (h->n_seg >= 3) {
            std::vector<uint16_t> hi(nnz);
            GSE_CUDA_TRY(cudaMemcpy(hi.data(), h->buf_t2hi, nnz * sizeof(uint16_t), cudaMemcpyDeviceToHost));
            const int r = h->v.r_lo;
            std::vector<uint32_t> lo;
            if (r > 0) {
                lo.resize(h->v.nnz_pad / 8 * r / 4);
                GSE_CUDA_TRY(cudaMemcpy(lo.data(), h->buf_t2lo, lo.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost));
            }
            for (int64_t e = 0; e < nnz; e++) {
                uint32_t t = hi[e];
                if (r > 0) {
                    const int bit = (int)(e & 7) * r;
                    t = (t << r) | ((lo[(e >> 3) * (r / 4) + (bit >> 5)] >> (bit & 31)) & ((1u << r) - 1u));
                }
                tail2[e] = t;
            }
        } else {
            memset(tail2, 0, nnz * sizeof(uint32_t));
        }
    }
    const int64_t ng = (nnz + h->group_size - 1) / h->group_size;
    if (gexp && h->v.tbl) return GSE_ERR_INVALID;     // table format: gse_export_table
    if (gexp && ng) GSE_CUDA_TRY(cudaMemcpy(gexp, h->buf_gexp, ng * sizeof(int16_t), cudaMemcpyDeviceToHost));
    return GSE_OK;
}

extern "C" int gse_decode(gse_handle h, int k, double* vals, void* stream) {
    if (!h || !vals) return GSE_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nunits = (h->v.nnz + 7) / 8;
    const unsigned g = grid_for(nunits);
    if (k == 1) k_decode<1, 0><<<g, 256, 0, s>>>(h->v, vals);
    else if (k == 2 && h->n_seg >= 2) k_decode<2, 0><<<g, 256, 0, s>>>(h->v, vals);
    else if (k == 3 && h->n_seg >= 3) {
        switch (h->v.r_lo) {
            case 0: k_decode<3, 0><<<g, 256, 0, s>>>(h->v, vals); break;
            case 4: k_decode<3, 4><<<g, 256, 0, s>>>(h->v, vals); break;
            case 8: k_decode<3, 8><<<g, 256, 0, s>>>(h->v, vals); break;
            default: k_decode<3, 16><<<g, 256, 0, s>>>(h->v, vals); break;
        }
    } else if (k == GSE_LEVEL_FP64 && h->v.val64) k_decode<SRC_FP64, 0><<<g, 256, 0, s>>>(h->v, vals);
    else if (k == GSE_LEVEL_FP32 && h->v.val32) k_decode<SRC_FP32, 0><<<g, 256, 0, s>>>(h->v, vals);
    else if (k == GSE_LEVEL_FP16 && h->v.val16) k_decode<SRC_FP16, 0><<<g, 256, 0, s>>>(h->v, vals);
    else if (k == GSE_LEVEL_BF16 && h->v.valbf) k_decode<SRC_BF16, 0><<<g, 256, 0, s>>>(h->v, vals);
    else return GSE_ERR_INVALID;
    return cudaGetLastError() == cudaSuccess ? GSE_OK : GSE_ERR_CUDA;
}

extern "C" int gse_matrix_get_info(gse_handle h, gse_matrix_info* info) {
    if (!h || !info) return GSE_ERR_INVALID;
    memset(info, 0, sizeof(*info));
    info->n_rows = h->v.n_rows;
    info->n_cols = h->v.n_cols;
    info->nnz = h->v.nnz;
    info->n_groups = (h->v.nnz + h->group_size - 1) / h->group_size;
    info->n_empty_rows = h->v.n_empty;
    info->group_size = h->group_size;
    info->n_seg = h->n_seg;
    for (int i = 0; i < 3; i++) info->seg_bits[i] = h->seg_bits[i];
    info->max_row_len = h->max_row_len;
    info->mean_row_len = h->mean_row_len;
    info->schedule = units_per_lane(h);
    info->num_exp = h->num_exp;
    info->index_in_head = h->index_in_head;
    info->overflow16 = h->overflow16;
    // algorithmic bytes: col + live segments + group exponent per nonzero,
    // row_ptr, x read once, y written once
    const double nnz = (double)h->v.nnz, n = (double)h->v.n_rows, nc = (double)h->v.n_cols;
    const double base = nnz * 4.0 + nnz / h->group_size * 2.0 + 4.0 * (n + 1) + 8.0 * nc + 8.0 * n;
    double seg = 0.0;
    for (int k = 0; k < h->n_seg; k++) {
        seg += nnz * h->seg_bits[k] / 8.0;
        info->bytes_level[k] = (int64_t)(base + seg);
    }
    return GSE_OK;
}

extern "C" size_t gse_footprint(gse_handle h) {
    if (!h) return 0;
    return h->bytes_matrix + h->bytes_ws;
}

extern "C" void gse_free(gse_handle h) {
    if (!h) return;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != h->device) cudaSetDevice(h->device);
    cudaDeviceSynchronize();           // no queued work may still use the buffers
    gse_free_workspace(h);
    free_all(h);
    if (cur != h->device) cudaSetDevice(cur);
    free(h);
}
