// gse_internal.cuh -- handle layout and helpers shared by the library's .cu files.
//
// Device layout of an encoded matrix (all arrays padded to nnz_pad, a multiple
// of CHUNK_MAX = 1024 nonzeros, so every chunk of every schedule is full):
//   col     int32[nnz_pad]            column indices (padding: 0)
//   head    u16[nnz_pad]              sign | top W_1 magnitude bits
//   tail1   u16[nnz_pad]              next s2 bits           (n_seg >= 2)
//   t2hi    u16[nnz_pad]              top min(s3,16) bits of tail2 (n_seg = 3)
//   t2lo    u32[nnz_pad / 8 * r / 4]  low r = s3 - 16 bits, packed per unit of
//                                     8 nonzeros (r in {4, 8, 16}), r bytes each
//   gexp    u16[n_groups]             group exponent E_g = max e + 1 (0: all zero)
//                                     (group format only)
// Table format (gse_encode_table): one table etab[num_exp] of shared exponents
// for the whole matrix (each a frequent exponent + 1, max + 1 among them); the
// index of a nonzero's entry sits in the top ei_bits bits of its col word
// (col = index << (32 - ei_bits) | column), so every kernel masks col with
// col_mask (all ones in the group format) and reads E = etab[col >> ei_shift];
// with the index in the head instead, E = etab[head index bits] (tbl_index).
//   rowend  u32[nnz_pad / 32]         bit e: nonzero e is the last of its row
//   blk_row0 int32[nnz_pad / 256]     compact index (nonempty rows only) of the
//                                     row holding nonzero 256*b
//   nzrow   int32[n_nonempty]         compact -> actual row (only with empty rows)
//   empty   int32[n_empty]            the empty rows (zero-filled by every SpMV)
// Split-row scratch (rows spanning chunks), indexed by 256-nonzero block:
//   carry f64 (piece of the row open at a chunk's end), part f64 (piece of the
//   row open at its start); finished by a separate pass after each SpMV.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gse.h"

#define GSE_CHUNK_BASE 256   // nonzeros per lane-unit chunk with 1 unit per lane
#define GSE_CHUNK_MAX 1024   // with 4 units per lane
#define GSE_UNIT 8           // consecutive nonzeros per unit
#define GSE_ROW_SPAN_MAX 4096  // largest nonzero span of a row block the row schedule stages

namespace gse {

// Device-side view of an encoded matrix, passed to kernels by value.
struct MatView {
    const int32_t* col;
    const uint16_t* head;
    const uint16_t* tail1;
    const uint16_t* t2hi;
    const uint32_t* t2lo;
    const uint16_t* gexp;
    const uint32_t* rowend;
    const int32_t* blk_row0;
    const int32_t* nzrow;      // nullptr when every row is nonempty
    const int32_t* empty;
    const int32_t* row_ptr;
    const double* val64;
    const float* val32;
    const uint16_t* val16;     // FP16 baseline values (bit patterns)
    const uint16_t* valbf;     // BF16 baseline values (bit patterns)
    double* carry;
    double* part;
    int64_t nnz, nnz_pad, n_rows, n_cols, n_nonempty, n_empty;
    int g_shift;               // log2(group size)
    int s1, s2, s3, s3hi, r_lo; // segment widths; s3hi = min(s3,16), r_lo = s3 - s3hi
    int W1, W2, W3;
    int tbl;                   // 1: global exponent table (etab); 0: per-group gexp
    int ei_shift;              // index in the col word: col >> ei_shift (32 when it is not there)
    uint32_t col_mask;         // column = col & col_mask
    int hi_shift;              // index in the head: (head >> hi_shift) & hi_mask (hi_mask 0 when not)
    uint32_t hi_mask;
    const int* inject;         // device flag (gse_test_timeout): staged kernels issue no copy, short waits
    const int16_t* etab;       // the shared exponents (table format; device, 64 entries); with
                               // the index in the head each entry is stored + its bit count, so
                               // the head, read as a full-width head, decodes unchanged
};

// Column index of a stored col word (strips the exponent index of the table format).
__device__ __forceinline__ int32_t col_of(const MatView& m, int32_t c) { return (int32_t)((uint32_t)c & m.col_mask); }
// Exponent-table index of a table-format nonzero, from its col word or its head;
// the index bits are cleared from the head (h) on the way.
__device__ __forceinline__ int tbl_index(const MatView& m, int32_t c, uint32_t& h) {
    const uint32_t hidx = (h >> m.hi_shift) & m.hi_mask;
    h &= ~(m.hi_mask << m.hi_shift);
    return (int)((uint64_t)(uint32_t)c >> m.ei_shift) | (int)hidx;
}

struct Workspace;  // solver vectors, allocated on first solve (solver.cu)

}  // namespace gse

struct gse_matrix {
    gse::MatView v;
    int group_size;
    int n_seg;
    int seg_bits[3];
    int max_row_len;
    double mean_row_len;
    int schedule_auto;   // units per lane (1, 2, 4) or GSE_SCHEDULE_ROWS, from row statistics / autotune
    int row_span;        // max nonzeros of any 32-row block, widened to groups of 32
    int row_span128;     // ... of any 128-row block (engine: 4-warp CTAs)
    int row_span256;     // ... of any 256-row block (standalone SpMV: 8-warp CTAs)
    int tile_span32;     // max nonzeros of any 32-row tile, its ends rounded out to 8 (lane-row stages)
    int tile_span64;     // ... of any 64-row tile
    int num_exp;         // table format: entries of the exponent table (0: group format)
    int16_t etab_host[64]; // table format: host copy of the table
    int index_in_head;   // table format: 1 when the index sits in the head, 0 in the col word
    void* buf_etab;      // table format: the table on the device (64 entries)
    int schedule_forced; // 0: automatic
    int num_sms;
    int device;
    // owned device allocations
    void* buf_col;
    void* buf_head;
    void* buf_tail1;
    void* buf_t2hi;
    void* buf_t2lo;
    void* buf_gexp;
    void* buf_rowend;
    void* buf_blk_row0;
    void* buf_nzrow;
    void* buf_empty;
    void* buf_row_ptr;
    void* buf_val64;
    void* buf_val32;
    void* buf_val16;
    void* buf_valbf;
    int64_t overflow16;  // FP16 values that overflowed at attach
    void* buf_carry;
    void* buf_part;
    // small scratch for grid reductions
    double* red_partial;   // one per block
    unsigned* red_counter;
    double* red_result;
    int red_capacity;
    size_t bytes_matrix;
    int* d_err;            // bounded-wait timeouts recorded by kernels (GSE_TIMEOUT)
    gse::Workspace* ws;
    size_t bytes_ws;
};

namespace gse {

// Status helpers.
#define GSE_CUDA_TRY(expr)                                  \
    do {                                                    \
        cudaError_t _e = (expr);                            \
        if (_e != cudaSuccess) {                            \
            if (_e == cudaErrorMemoryAllocation) return GSE_ERR_OOM; \
            return GSE_ERR_CUDA;                            \
        }                                                   \
    } while (0)

inline int units_per_lane(const gse_matrix* h) {
    return h->schedule_forced ? h->schedule_forced : h->schedule_auto;
}

// A level the handle can run: a GSE level 1..n_seg or an attached baseline.
inline bool level_available(const gse_matrix* h, int k) {
    if (k >= 1 && k <= h->n_seg) return true;
    if (k == GSE_LEVEL_FP64) return h->v.val64 != nullptr;
    if (k == GSE_LEVEL_FP32) return h->v.val32 != nullptr;
    if (k == GSE_LEVEL_FP16) return h->v.val16 != nullptr;
    if (k == GSE_LEVEL_BF16) return h->v.valbf != nullptr;
    return false;
}

// SpMV launch (spmv.cu).  Epilogue kinds:
enum EpiKind { EPI_STORE = 0, EPI_CG_PQ = 1, EPI_RESID = 2 };

struct SpmvArgs {
    const double* x;     // gathered vector
    double* y;           // output (EPI_STORE / EPI_CG_PQ: y = A x; EPI_RESID: y = b - A x)
    const double* b;     // EPI_RESID
    const double* p;     // EPI_CG_PQ: dot partner (normally == x)
    double* dot_out;     // EPI_CG_PQ: result scalar (device)
    // grid-reduction scratch (EPI_CG_PQ)
    double* red_partial;
    unsigned* red_counter;
    const int* skip_flag; // if non-null and *skip_flag != 0 the kernel returns at once
};

int launch_spmv(gse_matrix* h, int k, int epi, const SpmvArgs& a, cudaStream_t s, int upl_override = 0);
// True when gse_spmv at level k runs the lane-row kernel on the row schedule.
bool lanerow_ok(const gse_matrix* h, int k);
// For a handle on the lane-row kernels: 0 the per-group format; 1 the exponent
// table with its index in the column word (general decode); 2 the same with
// every entry above W_1 (fast decode).
int lanerow_table_kind(const gse_matrix* h);

}  // namespace gse
