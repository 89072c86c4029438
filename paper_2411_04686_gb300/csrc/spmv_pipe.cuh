// spmv_pipe.cuh -- the GSE-SpMV main loops.
//
// The row schedule and the 2- and 4-unit nonzero split stage the matrix
// through a ring of shared-memory stages per CTA; the default 1-unit nonzero
// split (for scattered columns) loads straight from global memory instead, so
// that the SM's L1 stays free for the random x gathers (spmv_chunks_direct).
// In the staged loops one producer thread fills a stage with a few large 1-D
// bulk copies (cp.async.bulk, completion counted in bytes on a "full" mbarrier): column
// indices, the live segment arrays (or the CSR values of a baseline), row-end
// bits and group exponents -- contiguous, 16-byte aligned slices of the HBM
// arrays.  Every warp consumes its part, then arrives on the stage's "empty"
// barrier; the producer refills the stage once all warps have left it.  Large
// copies from one issuer per CTA keep the DRAM stream dense (on this GPU, many
// small per-warp copies reach only 2-3 TB/s).
//
// Every mbarrier wait is bounded; on expiry the kernel records GSE_TIMEOUT in
// *err and leaves the loop.
#pragma once

#include "spmv_core.cuh"

namespace gse {

constexpr uint32_t MBAR_SPIN_LIMIT = 1u << 22;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Spin bound of a launch whose handle has the timeout test flag set (no copy
// is issued, so every wait runs out, quickly, with nothing in flight).
constexpr uint32_t MBAR_SPIN_TEST = 1024u;

// Bounded wait for phase `parity` of the barrier; false if the bound ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity, uint32_t limit = MBAR_SPIN_LIMIT) {
    for (uint32_t it = 0; it < limit; it++)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
        "l"(src), "r"(bytes), "r"(bar)
        : "memory");
}

struct ChunkScalars {
    int64_t row0;
    bool starts_mid;
};

__device__ __forceinline__ ChunkScalars chunk_scalars(const MatView& m, int64_t c, int CH, int UPL) {
    ChunkScalars s;
    s.row0 = __ldg(m.blk_row0 + c * UPL);
    s.starts_mid = false;
    if (c > 0) {
        const int64_t pe = c * CH - 1;
        s.starts_mid = !((__ldg(m.rowend + (pe >> 5)) >> (pe & 31)) & 1u);
    }
    return s;
}

}  // namespace gse

namespace gse {

// ---- row schedule: one row per lane, 32 consecutive rows per warp ----------
// For matrices whose 32-row blocks span at most `span` nonzeros (short rows):
// a stage holds the block's nonzeros, widened to whole groups of 32 (and the
// group exponents to whole 8-group runs) so every bulk copy is 16-byte aligned.
// Each lane walks its own row from shared memory: no row-end bits, no lane
// scans, no rows crossing warps, so no scratch and no second pass.

struct RowStage {
    int span;          // nonzeros a stage can hold (multiple of 32)
    int off_v, off_gx, bytes;
};

template <int K, int R>
__host__ __device__ inline RowStage row_stage_layout(int span, int r_lo) {
    RowStage L;
    L.span = span;
    L.off_v = span * 4;
    int v;
    if (K == SRC_FP64) v = span * 8;
    else if (K == SRC_FP32) v = span * 4;
    else if (src16(K)) v = span * 2;
    else v = span * 2 * (K >= 3 ? 3 : K) + (K >= 3 ? span * (R < 0 ? r_lo : R) / 8 : 0);
    L.off_gx = L.off_v + ((v + 127) / 128) * 128;
    const int gx = (span / 8 + 16) * 2;    // group exponents of the span (groups >= 8), 8-group aligned ends
    L.bytes = ((L.off_gx + gx) + 127) / 128 * 128;
    return L;
}

struct RowBlock {
    int64_t e_lo, e_hi;   // nonzero range copied (group aligned)
    int64_t g_lo;         // first group exponent copied (8-group aligned)
};

__device__ __forceinline__ RowBlock row_block(int64_t s, int64_t t, int g_shift) {
    RowBlock rb;
    rb.e_lo = (s >> 5) << 5;
    rb.e_hi = ((t + 31) >> 5) << 5;
    rb.g_lo = ((rb.e_lo >> g_shift) >> 3) << 3;
    return rb;
}

template <int K, int R, bool TBL = false>
__device__ __forceinline__ void issue_rows(const MatView& m, const RowStage& L, RowBlock rb, unsigned char* stage,
                                           uint32_t bar) {
    const uint32_t n = (uint32_t)(rb.e_hi - rb.e_lo);
    if (n == 0) {
        mbar_expect_tx(bar, 0);
        return;
    }
    const int64_t g_hi = (((rb.e_hi >> m.g_shift) + 7) >> 3) << 3;
    const uint32_t gx_bytes = (uint32_t)((g_hi - rb.g_lo) * 2);
    const int r = R < 0 ? m.r_lo : R;
    uint32_t vbytes;
    if constexpr (K == SRC_FP64) vbytes = n * 8;
    else if constexpr (K == SRC_FP32) vbytes = n * 4;
    else if constexpr (src16(K)) vbytes = n * 2;
    else vbytes = n * 2 * (K >= 3 ? 3 : K) + (K >= 3 ? n * r / 8 : 0);
    const bool gse_src = K <= 3 && !TBL;     // the baselines and the table format have no group exponents
    mbar_expect_tx(bar, n * 4 + vbytes + (gse_src ? gx_bytes : 0));
    const uint32_t s = smem_u32(stage);
    bulk_g2s(s, m.col + rb.e_lo, n * 4, bar);
    if constexpr (K == SRC_FP64) {
        bulk_g2s(s + L.off_v, m.val64 + rb.e_lo, n * 8, bar);
    } else if constexpr (K == SRC_FP32) {
        bulk_g2s(s + L.off_v, m.val32 + rb.e_lo, n * 4, bar);
    } else if constexpr (src16(K)) {
        bulk_g2s(s + L.off_v, (K == SRC_FP16 ? m.val16 : m.valbf) + rb.e_lo, n * 2, bar);
    } else {
        const uint32_t sp2 = (uint32_t)L.span * 2;
        bulk_g2s(s + L.off_v, m.head + rb.e_lo, n * 2, bar);
        if constexpr (K >= 2) bulk_g2s(s + L.off_v + sp2, m.tail1 + rb.e_lo, n * 2, bar);
        if constexpr (K >= 3) {
            bulk_g2s(s + L.off_v + 2 * sp2, m.t2hi + rb.e_lo, n * 2, bar);
            if (r > 0) bulk_g2s(s + L.off_v + 3 * sp2, m.t2lo + rb.e_lo / 8 * r / 4, n * r / 8, bar);
        }
        if constexpr (!TBL) bulk_g2s(s + L.off_gx, m.gexp + rb.g_lo, gx_bytes, bar);
    }
}

// Value of the stage's nonzero i (stage-local index; its group is
// (i >> g_shift) + goff in the stage's exponent run; in the table format the
// shared exponent is etab[index in the col word cw or in the head]).
template <int K, int R, bool TBL = false>
__device__ __forceinline__ double row_value(const MatView& m, const RowStage& L, const unsigned char* stage, int i,
                                            int goff, int32_t cw = 0, const int16_t* etab = nullptr) {
    if constexpr (K == SRC_FP64) {
        return reinterpret_cast<const double*>(stage + L.off_v)[i];
    } else if constexpr (K == SRC_FP32) {
        return widen_f32(reinterpret_cast<const uint32_t*>(stage + L.off_v)[i]);
    } else if constexpr (src16(K)) {
        return widen16<K>(reinterpret_cast<const uint16_t*>(stage + L.off_v)[i]);
    } else {
        const uint16_t* hv = reinterpret_cast<const uint16_t*>(stage + L.off_v);
        uint32_t h = hv[i];
        const int Eg = TBL ? (int)etab[tbl_index(m, cw, h)]
                           : (int)reinterpret_cast<const uint16_t*>(stage + L.off_gx)[(i >> m.g_shift) + goff];
        if constexpr (K == 1) return decode_l1_f(h, Eg, (uint32_t)(Eg - m.W1 - 127) << 20, m);
        const uint32_t t1 = hv[L.span + i];
        if constexpr (K == 2) return decode_l2(h, t1, Eg, m);
        uint32_t t2 = hv[2 * L.span + i];
        const int r = R < 0 ? m.r_lo : R;
        if (r > 0) {
            const uint32_t* lw = reinterpret_cast<const uint32_t*>(stage + L.off_v + 6 * L.span);
            const int bit = i * r;
            t2 = (t2 << r) | ((lw[bit >> 5] >> (bit & 31)) & ((1u << r) - 1u));
        }
        if constexpr (R == 0 || R == 4) {
            // the row schedule serves matrices whose groups rarely hold values
            // 2^15 below their maximum: the head-only form, else the general one
            if (ok_l3_fast(h, Eg, m)) return decode_l3_fast(h, t1, t2, Eg, m);
            return decode_l3_sel(h, t1, t2, Eg, m);
        }
        return decode_l3(h, t1, t2, Eg, m);
    }
}

}  // namespace gse

namespace gse {

// ---- row schedule, block-level pipeline ------------------------------------
// A CTA of W warps owns "super-blocks" of 32*W consecutive rows (one row per
// lane).  One thread (the producer) fills a ring of STAGES stages with the
// super-block's nonzeros using a handful of large bulk copies; every warp
// consumes its 32 rows from the stage and then arrives on the stage's "empty"
// barrier, which the producer waits on before refilling it.  Large copies from
// one issuer per CTA keep the DRAM stream dense (many small per-warp copies do
// not).  All waits are bounded.

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

template <int K, int R, bool DOT, bool RESID, int STAGES, bool TBL = false>
__device__ __forceinline__ double spmv_rows_block(const MatView& m, const double* __restrict__ x, const Epi& e,
                                                  int64_t sb0, int64_t sbstride, int64_t nsb, const RowStage& L,
                                                  unsigned char* smem, int* err) {
    __shared__ int16_t etab[64];                                  // table format: the shared exponents
    if (TBL && threadIdx.x < 64) etab[threadIdx.x] = __ldg(m.etab + threadIdx.x);
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
    const int RB = 32 * W;                                        // rows per super-block
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + STAGES;
    unsigned char* stages = smem + 128;
    const bool producer = threadIdx.x == 0;
    const int64_t n = m.n_rows;
    // test flag (gse_test_timeout): issue no copy, wait with a short bound
    const bool inj = m.inject && __ldg(m.inject) != 0;
    const uint32_t lim = inj ? MBAR_SPIN_TEST : MBAR_SPIN_LIMIT;
    double dot = 0.0;
    if (sb0 >= nsb) return dot;
    auto bounds = [&](int64_t sb, int64_t* s0, int64_t* t0) {
        const int64_t r0 = sb * RB, r1 = r0 + RB < n ? r0 + RB : n;
        *s0 = __ldg(m.row_ptr + r0);
        *t0 = __ldg(m.row_ptr + r1);
    };
    auto lane_row = [&](int64_t sb, int64_t* rs, int64_t* rt) {
        const int64_t r = sb * RB + warp * 32 + lane;
        *rs = __ldg(m.row_ptr + (r < n ? r : n));
        *rt = __ldg(m.row_ptr + (r < n ? r + 1 : n));
    };
    if (producer) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(smem_u32(full + s), 1);
            mbar_init(smem_u32(empty + s), W);
        }
        fence_mbar_init();
        for (int s = 0; s < STAGES && !inj; s++) {
            const int64_t sb = sb0 + s * sbstride;
            if (sb >= nsb) break;
            int64_t bs, bt;
            bounds(sb, &bs, &bt);
            issue_rows<K, R, TBL>(m, L, row_block(bs, bt, m.g_shift), stages + s * L.bytes, smem_u32(full + s));
        }
    }
    __syncthreads();
    int64_t rs_n, rt_n, cb_s, cb_t, is_n = 0, it_n = 0;
    lane_row(sb0, &rs_n, &rt_n);
    bounds(sb0, &cb_s, &cb_t);
    if (producer && sb0 + (int64_t)STAGES * sbstride < nsb) bounds(sb0 + (int64_t)STAGES * sbstride, &is_n, &it_n);
    uint32_t fphase = 0, ephase = 0;
    bool ok = true;
    int64_t i = 0;
    for (int64_t sb = sb0; sb < nsb; sb += sbstride, i++) {
        const int s = (int)(i % STAGES);
        const int64_t rs = rs_n, rt = rt_n;
        const RowBlock rb = row_block(cb_s, cb_t, m.g_shift);
        const int64_t nxt = sb + sbstride, si = sb + (int64_t)STAGES * sbstride;
        const int64_t is = is_n, it = it_n;
        if (nxt < nsb) {
            lane_row(nxt, &rs_n, &rt_n);
            bounds(nxt, &cb_s, &cb_t);
        }
        if (producer && si + sbstride < nsb) bounds(si + sbstride, &is_n, &it_n);
        ok = __all_sync(FULL, mbar_wait_bounded(smem_u32(full + s), (fphase >> s) & 1u, lim));
        if (!ok) break;
        fphase ^= 1u << s;
        const unsigned char* st = stages + s * L.bytes;
        double acc = 0.0;
        const int32_t* scol = reinterpret_cast<const int32_t*>(st);
        const int ls = (int)(rs - rb.e_lo), lt = (int)(rt - rb.e_lo);
        const int goff = (int)((rb.e_lo >> m.g_shift) - rb.g_lo);
        // the row in batches of 8: all x gathers of a batch are in flight
        // together (one round trip per batch), then the values are rebuilt
        // and accumulated in order
        for (int li = ls; li < lt; li += 8) {
            const int cnt = lt - li;
            double xv[8];
#pragma unroll
            for (int u = 0; u < 8; u++) xv[u] = u < cnt ? __ldg(x + col_of(m, scol[li + u])) : 0.0;
#pragma unroll
            for (int u = 0; u < 8; u++)
                if (u < cnt)
                    acc = fma(row_value<K, R, TBL>(m, L, st, li + u, goff, TBL ? scol[li + u] : 0, etab), xv[u], acc);
        }
        const int64_t r = sb * RB + warp * 32 + lane;
        if (r < n) {
            if (DOT) dot = fma(__ldg(e.p + r), acc, dot);
            epi_finish_t<RESID>(e, r, acc);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(empty + s));      // this warp is done with stage s
        if (producer && si < nsb) {
            // all W warps must have left stage s before it is refilled
            const bool freed = mbar_wait_bounded(smem_u32(empty + s), (ephase >> s) & 1u, lim);
            if (!freed) atomicOr(err, 1);
            else {
                fence_proxy_async_smem();
                issue_rows<K, R, TBL>(m, L, row_block(is, it, m.g_shift), stages + s * L.bytes, smem_u32(full + s));
            }
        }
        ephase ^= 1u << s;
    }
    if (!ok) {
        if (lane == 0) atomicOr(err, 1);
    }
    // every issued fill has been consumed (the loop visits each super-block it
    // issued) unless a wait gave up; the CTA's barriers die with it
    return dot;
}

// Shared memory of a CTA on the block-level row schedule.
template <int STAGES>
__host__ __device__ inline int rows_block_smem(const RowStage& L) { return 128 + STAGES * L.bytes; }

}  // namespace gse

namespace gse {

// ---- nonzero-split schedule, block-level pipeline ---------------------------
// A CTA of W warps owns super-chunks of W consecutive chunks (W * 256 * UPL
// nonzeros); one producer thread stages a super-chunk with large bulk copies
// and each warp runs the chunk logic (row-end bits, lane scans, split-row
// pieces) on its own chunk c = super-chunk * W + warp.  Same chunk numbering as
// the per-warp variant, so the split-row pass is unchanged.

struct ChunkStage {
    int nch;                        // chunks per stage (W)
    int ch;                         // nonzeros per chunk
    int off_v, off_re, off_gx, bytes;
};

template <int K, int R, int UPL>
__host__ __device__ inline ChunkStage chunk_stage_layout(int W, int r_lo) {
    ChunkStage L;
    L.nch = W;
    L.ch = 256 * UPL;
    const int e = W * L.ch;
    L.off_v = e * 4;
    int v;
    if (K == SRC_FP64) v = e * 8;
    else if (K == SRC_FP32) v = e * 4;
    else if (src16(K)) v = e * 2;
    else v = e * 2 * (K >= 3 ? 3 : K) + (K >= 3 ? e * (R < 0 ? r_lo : R) / 8 : 0);
    L.off_re = L.off_v + ((v + 127) / 128) * 128;
    L.off_gx = L.off_re + ((e / 8 + 127) / 128) * 128;
    L.bytes = ((L.off_gx + e / 4) + 127) / 128 * 128;   // gexp: e / G * 2 <= e / 4 bytes
    return L;
}

template <int K, int R, int UPL, bool TBL = false>
__device__ __forceinline__ void issue_superchunk(const MatView& m, const ChunkStage& L, int64_t sc, int64_t nch_total,
                                                 unsigned char* stage, uint32_t bar) {
    // chunks sc*W .. min(sc*W + W, nch_total) - 1 (the tail super-chunk may be short)
    int64_t c0 = sc * L.nch, c1 = c0 + L.nch < nch_total ? c0 + L.nch : nch_total;
    const uint32_t e = (uint32_t)((c1 - c0) * L.ch);
    const int64_t e0 = c0 * L.ch;
    const int r = R < 0 ? m.r_lo : R;
    const uint32_t gx_bytes = (uint32_t)((e >> m.g_shift) * 2);
    uint32_t vbytes;
    if constexpr (K == SRC_FP64) vbytes = e * 8;
    else if constexpr (K == SRC_FP32) vbytes = e * 4;
    else if constexpr (src16(K)) vbytes = e * 2;
    else vbytes = e * 2 * (K >= 3 ? 3 : K) + (K >= 3 ? e * r / 8 : 0);
    const bool gse_src = K <= 3 && !TBL;
    mbar_expect_tx(bar, e * 4 + vbytes + e / 8 + (gse_src ? gx_bytes : 0));
    const uint32_t s = smem_u32(stage);
    const uint32_t E = (uint32_t)(L.nch * L.ch);    // full-stage stride of the segment arrays
    bulk_g2s(s, m.col + e0, e * 4, bar);
    if constexpr (K == SRC_FP64) {
        bulk_g2s(s + L.off_v, m.val64 + e0, e * 8, bar);
    } else if constexpr (K == SRC_FP32) {
        bulk_g2s(s + L.off_v, m.val32 + e0, e * 4, bar);
    } else if constexpr (src16(K)) {
        bulk_g2s(s + L.off_v, (K == SRC_FP16 ? m.val16 : m.valbf) + e0, e * 2, bar);
    } else {
        bulk_g2s(s + L.off_v, m.head + e0, e * 2, bar);
        if constexpr (K >= 2) bulk_g2s(s + L.off_v + E * 2, m.tail1 + e0, e * 2, bar);
        if constexpr (K >= 3) {
            bulk_g2s(s + L.off_v + E * 4, m.t2hi + e0, e * 2, bar);
            if (r > 0) bulk_g2s(s + L.off_v + E * 6, m.t2lo + e0 / 8 * r / 4, e * r / 8, bar);
        }
        if constexpr (!TBL) bulk_g2s(s + L.off_gx, m.gexp + (e0 >> m.g_shift), gx_bytes, bar);
    }
    bulk_g2s(s + L.off_re, m.rowend + e0 / 32, e / 8, bar);
}

// Values of unit u (stage-relative unit index) of a block-level stage; in the
// table format each value's shared exponent comes from its col word cw[i].
template <int K, int R, bool TBL = false>
__device__ __forceinline__ void unit_values_blk(const MatView& m, const ChunkStage& L, const unsigned char* stage,
                                                int u, double* a, const int32_t* cw = nullptr,
                                                const int16_t* etab = nullptr) {
    const int E = L.nch * L.ch;
    if constexpr (K == SRC_FP64) {
        const double2* v2 = reinterpret_cast<const double2*>(stage + L.off_v) + 4 * u;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const double2 d = v2[j];
            a[2 * j] = d.x;
            a[2 * j + 1] = d.y;
        }
    } else if constexpr (K == SRC_FP32) {
        const uint4* f4 = reinterpret_cast<const uint4*>(stage + L.off_v) + 2 * u;
        const uint4 fa = f4[0], fb = f4[1];
        a[0] = widen_f32(fa.x); a[1] = widen_f32(fa.y); a[2] = widen_f32(fa.z); a[3] = widen_f32(fa.w);
        a[4] = widen_f32(fb.x); a[5] = widen_f32(fb.y); a[6] = widen_f32(fb.z); a[7] = widen_f32(fb.w);
    } else if constexpr (src16(K)) {
        const uint4 w = reinterpret_cast<const uint4*>(stage + L.off_v)[u];
#pragma unroll
        for (int i = 0; i < 8; i++) a[i] = widen16<K>(u16_of(w, i));
    } else {
        const uint16_t* gx = reinterpret_cast<const uint16_t*>(stage + L.off_gx);
        const int Eg0 = TBL ? 0 : (int)gx[(u * GSE_UNIT) >> m.g_shift];
        const uint4 hw = reinterpret_cast<const uint4*>(stage + L.off_v)[u];
        uint4 t1w = make_uint4(0, 0, 0, 0), t2w = make_uint4(0, 0, 0, 0);
        uint32_t lo[4] = {0, 0, 0, 0};
        if constexpr (K >= 2) t1w = reinterpret_cast<const uint4*>(stage + L.off_v + E * 2)[u];
        const int r = R < 0 ? m.r_lo : R;
        if constexpr (K >= 3) {
            t2w = reinterpret_cast<const uint4*>(stage + L.off_v + E * 4)[u];
            const uint32_t* lw = reinterpret_cast<const uint32_t*>(stage + L.off_v + E * 6);
            if (r == 4) lo[0] = lw[u];
            else if (r == 8) { lo[0] = lw[2 * u]; lo[1] = lw[2 * u + 1]; }
            else if (r == 16) { const uint4 l4 = reinterpret_cast<const uint4*>(lw)[u]; lo[0] = l4.x; lo[1] = l4.y; lo[2] = l4.z; lo[3] = l4.w; }
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
            uint32_t h = u16_of(hw, i);
            const int Eg = TBL ? (int)etab[tbl_index(m, cw[i], h)] : Eg0;
            if constexpr (K == 1) {
                a[i] = decode_l1_f(h, Eg, (uint32_t)(Eg - m.W1 - 127) << 20, m);
            } else if constexpr (K == 2) {
                a[i] = decode_l2(h, u16_of(t1w, i), Eg, m);
            } else {
                uint32_t t2 = u16_of(t2w, i);
                if (r > 0) {
                    const int bit = i * r;
                    t2 = (t2 << r) | ((lo[bit >> 5] >> (bit & 31)) & ((1u << r) - 1u));
                }
                if constexpr (R == 0 || R == 4) a[i] = decode_l3_sel(h, u16_of(t1w, i), t2, Eg, m);
                else a[i] = decode_l3(h, u16_of(t1w, i), t2, Eg, m);
            }
        }
    }
}

// One warp's chunk c from a block-level stage (its units start at ub).
// Every finished row goes straight through the epilogue from the lane that
// finishes it: rows ending inside a lane after its first row end as soon as
// they end, the lane's first row end once the segmented scan has supplied the
// carries of the lanes before it.  No shared staging of row results, so a CTA
// needs only its stage ring.
template <int K, int R, int UPL, bool DOT, bool RESID, bool TBL = false>
__device__ __forceinline__ double compute_chunk_blk(const MatView& m, const Epi& e, int64_t c, const ChunkStage& L,
                                                    const unsigned char* stage, int ub, const double* __restrict__ x,
                                                    ChunkScalars sc, const int16_t* etab = nullptr) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const uint32_t* re = reinterpret_cast<const uint32_t*>(stage + L.off_re) + (ub >> 2);
    uint32_t bits;
    if constexpr (UPL == 4) bits = re[lane];
    else if constexpr (UPL == 2) bits = (re[lane >> 1] >> ((lane & 1) * 16)) & 0xFFFFu;
    else bits = (re[lane >> 2] >> ((lane & 3) * 8)) & 0xFFu;
    // x gathers for the lane's 8*UPL nonzeros, issued before the scans
    double xv[8 * UPL];
    int32_t cw[TBL ? 8 * UPL : 1];
    const int4* c4 = reinterpret_cast<const int4*>(stage) + 2 * (ub + UPL * lane);
#pragma unroll
    for (int q = 0; q < UPL; q++) {
        const int4 ca = c4[2 * q], cb = c4[2 * q + 1];
        xv[8 * q + 0] = __ldg(x + col_of(m, ca.x)); xv[8 * q + 1] = __ldg(x + col_of(m, ca.y));
        xv[8 * q + 2] = __ldg(x + col_of(m, ca.z)); xv[8 * q + 3] = __ldg(x + col_of(m, ca.w));
        xv[8 * q + 4] = __ldg(x + col_of(m, cb.x)); xv[8 * q + 5] = __ldg(x + col_of(m, cb.y));
        xv[8 * q + 6] = __ldg(x + col_of(m, cb.z)); xv[8 * q + 7] = __ldg(x + col_of(m, cb.w));
        if constexpr (TBL) {
            cw[8 * q + 0] = ca.x; cw[8 * q + 1] = ca.y; cw[8 * q + 2] = ca.z; cw[8 * q + 3] = ca.w;
            cw[8 * q + 4] = cb.x; cw[8 * q + 5] = cb.y; cw[8 * q + 6] = cb.z; cw[8 * q + 7] = cb.w;
        }
    }
    const int cnt = __popc(bits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - cnt;
    const int total_ends = __shfl_sync(FULL, incl, 31);
    double cur = 0.0, hp = 0.0, dot = 0.0;
    int j = 0;
#pragma unroll
    for (int q = 0; q < UPL; q++) {
        double a[8];
        unit_values_blk<K, R, TBL>(m, L, stage, ub + lane * UPL + q, a, TBL ? cw + 8 * q : nullptr, etab);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            cur = fma(a[i], xv[8 * q + i], cur);
            const bool end = (bits >> (q * 8 + i)) & 1u;
            if (end && j > 0) {     // a row that starts and ends in this lane: ordinal excl + j >= 1
                const int64_t Rw = actual_row(m, sc.row0 + excl + j);
                if (DOT) dot = fma(__ldg(e.p + Rw), cur, dot);
                epi_finish_t<RESID>(e, Rw, cur);
            }
            hp = end && j == 0 ? cur : hp;
            j += end ? 1 : 0;
            cur = end ? 0.0 : cur;
        }
    }
    const bool seen = j > 0;
    const double co = cur;
    double out;
    if (__all_sync(FULL, seen)) {
        out = co;
    } else {
        double v = co;
        bool f = seen;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double vu = __shfl_up_sync(FULL, v, o);
            const bool fu = __shfl_up_sync(FULL, (int)f, o) != 0;
            if (lane >= o) {
                if (!f) v += vu;
                f = f || fu;
            }
        }
        out = v;
    }
    double in = __shfl_up_sync(FULL, out, 1);
    if (lane == 0) in = 0.0;
    if (seen) {                     // the lane's first row end: ordinal excl
        const double v = in + hp;
        if (excl == 0 && sc.starts_mid) {
            // the piece of a row begun in an earlier chunk (summed by the fix pass)
            if (DOT) dot = fma(__ldg(e.p + actual_row(m, sc.row0)), v, dot);
            m.part[c] = v;
        } else {
            const int64_t Rw = actual_row(m, sc.row0 + excl);
            if (DOT) dot = fma(__ldg(e.p + Rw), v, dot);
            epi_finish_t<RESID>(e, Rw, v);
        }
    }
    const double out31 = __shfl_sync(FULL, out, 31);
    const bool last_end = __shfl_sync(FULL, (bits >> (8 * UPL - 1)) & 1u, 31) != 0;
    if (lane == 0) {
        if (total_ends == 0) {
            if (sc.row0 < m.n_nonempty) {
                if (DOT) dot = fma(__ldg(e.p + actual_row(m, sc.row0)), out31, dot);
                if (sc.starts_mid) m.part[c] = out31;
                else m.carry[c] = out31;
            }
        } else {
            const int64_t ro = sc.row0 + total_ends;
            if (!last_end && ro < m.n_nonempty) {
                if (DOT) dot = fma(__ldg(e.p + actual_row(m, ro)), out31, dot);
                m.carry[c] = out31;
            }
        }
    }
    return dot;
}

// The CTA's share of an SpMV on the nonzero split: super-chunks sc0, sc0 +
// scstride, ... of W chunks each (nch_total chunks in all).  smem: the STAGES
// stages.
template <int K, int R, int UPL, bool DOT, bool RESID, int STAGES, bool TBL = false>
__device__ __forceinline__ double spmv_chunks_block(const MatView& m, const double* __restrict__ x, const Epi& e,
                                                    int64_t sc0, int64_t scstride, int64_t nch_total,
                                                    const ChunkStage& L, unsigned char* smem, int* err) {
    __shared__ int16_t etab[64];                                  // table format: the shared exponents
    if (TBL && threadIdx.x < 64) etab[threadIdx.x] = __ldg(m.etab + threadIdx.x);
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = L.nch;
    constexpr int CH = 256 * UPL;
    uint64_t* full = reinterpret_cast<uint64_t*>(smem);
    uint64_t* empty = full + STAGES;
    unsigned char* stages = smem + 128;
    const bool producer = threadIdx.x == 0;
    const int64_t nsc = (nch_total + W - 1) / W;
    // test flag (gse_test_timeout): issue no copy, wait with a short bound
    const bool inj = m.inject && __ldg(m.inject) != 0;
    const uint32_t lim = inj ? MBAR_SPIN_TEST : MBAR_SPIN_LIMIT;
    double dot = 0.0;
    if (sc0 >= nsc) return dot;
    if (producer) {
        for (int s = 0; s < STAGES; s++) {
            mbar_init(smem_u32(full + s), 1);
            mbar_init(smem_u32(empty + s), W);
        }
        fence_mbar_init();
        for (int s = 0; s < STAGES && !inj; s++) {
            const int64_t sc = sc0 + s * scstride;
            if (sc >= nsc) break;
            issue_superchunk<K, R, UPL, TBL>(m, L, sc, nch_total, stages + s * L.bytes, smem_u32(full + s));
        }
    }
    __syncthreads();
    uint32_t fphase = 0, ephase = 0;
    bool ok = true;
    int64_t i = 0;
    ChunkScalars scn;
    {
        const int64_t c = sc0 * W + warp;
        if (c < nch_total) scn = chunk_scalars(m, c, CH, UPL);
    }
    for (int64_t sc = sc0; sc < nsc; sc += scstride, i++) {
        const int s = (int)(i % STAGES);
        const int64_t c = sc * W + warp;
        const ChunkScalars scs = scn;
        const int64_t cn = (sc + scstride) * W + warp;
        if (sc + scstride < nsc && cn < nch_total) scn = chunk_scalars(m, cn, CH, UPL);
        ok = __all_sync(FULL, mbar_wait_bounded(smem_u32(full + s), (fphase >> s) & 1u, lim));
        if (!ok) break;
        fphase ^= 1u << s;
        if (c < nch_total)
            dot += compute_chunk_blk<K, R, UPL, DOT, RESID, TBL>(m, e, c, L, stages + s * L.bytes, warp * 32 * UPL, x,
                                                                 scs, etab);
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(empty + s));
        const int64_t si = sc + (int64_t)STAGES * scstride;
        if (producer && si < nsc) {
            if (!mbar_wait_bounded(smem_u32(empty + s), (ephase >> s) & 1u, lim)) atomicOr(err, 1);
            else {
                fence_proxy_async_smem();
                issue_superchunk<K, R, UPL, TBL>(m, L, si, nch_total, stages + s * L.bytes, smem_u32(full + s));
            }
        }
        ephase ^= 1u << s;
    }
    if (!ok && lane == 0) atomicOr(err, 1);
    return dot;
}

// ---- nonzero split, direct loads (one unit of 8 per lane) ----------------
// The same chunk logic with no shared-memory staging: lane l of the warp that
// owns chunk c loads unit 32c + l (two int4 of columns, one 128-bit word per
// live segment, the group exponent, its byte of row-end bits) straight from
// global memory -- coalesced across the warp -- and gathers x.  Without a
// stage ring every SM keeps its whole L1 for the random x gathers, which is
// what matrices with scattered columns are bound by; this is the default
// nonzero-split kernel (the staged ring above serves 2 and 4 units per lane).
template <int K, int R, bool DOT, bool RESID, bool STD = false>
__device__ __forceinline__ double compute_chunk_direct(const MatView& m, const Epi& e, int64_t c,
                                                       const double* __restrict__ x) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const ChunkScalars sc = chunk_scalars(m, c, 256, 1);
    const uint32_t bits = (__ldg(m.rowend + ((c * 256) >> 5) + (lane >> 2)) >> ((lane & 3) * 8)) & 0xFFu;
    int col[8];
    double a[8];
    load_unit<K, R, STD>(m, c * 32 + lane, col, a);
    double xv[8];
#pragma unroll
    for (int i = 0; i < 8; i++) xv[i] = __ldg(x + col_of(m, col[i]));
    if (__ballot_sync(FULL, bits != 0u) == 0u) {
        // No row ends in the chunk: all 256 nonzeros belong to one row (begun
        // here or earlier, going on past the chunk).  Each lane sums its 8 in
        // two interleaved chains, the warp adds the lanes by a butterfly, and
        // the chunk's piece goes to part / carry for the split-row pass.
        double s0 = 0.0, s1 = 0.0;
#pragma unroll
        for (int i = 0; i < 8; i += 2) {
            s0 = fma(a[i], xv[i], s0);
            s1 = fma(a[i + 1], xv[i + 1], s1);
        }
        double v = s0 + s1;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
        double dot = 0.0;
        if (lane == 0 && sc.row0 < m.n_nonempty) {
            if (DOT) dot = __ldg(e.p + actual_row(m, sc.row0)) * v;
            if (sc.starts_mid) m.part[c] = v;
            else m.carry[c] = v;
        }
        return dot;
    }
    const int cnt = __popc(bits);
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, o);
        if (lane >= o) incl += t;
    }
    const int excl = incl - cnt;
    const int total_ends = __shfl_sync(FULL, incl, 31);
    double cur = 0.0, hp = 0.0, dot = 0.0;
    int j = 0;
#pragma unroll
    for (int i = 0; i < 8; i++) {
        cur = fma(a[i], xv[i], cur);
        const bool end = (bits >> i) & 1u;
        if (end && j > 0) {         // a row that starts and ends in this lane: ordinal excl + j >= 1
            const int64_t Rw = actual_row(m, sc.row0 + excl + j);
            if (DOT) dot = fma(__ldg(e.p + Rw), cur, dot);
            epi_finish_t<RESID>(e, Rw, cur);
        }
        hp = end && j == 0 ? cur : hp;
        j += end ? 1 : 0;
        cur = end ? 0.0 : cur;
    }
    const bool seen = j > 0;
    double out = cur;
    if (!__all_sync(FULL, seen)) {  // rows crossing lanes: segmented scan of the lane carries
        double v = cur;
        bool f = seen;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const double vu = __shfl_up_sync(FULL, v, o);
            const bool fu = __shfl_up_sync(FULL, (int)f, o) != 0;
            if (lane >= o) {
                if (!f) v += vu;
                f = f || fu;
            }
        }
        out = v;
    }
    double in = __shfl_up_sync(FULL, out, 1);
    if (lane == 0) in = 0.0;
    if (seen) {                     // the lane's first row end: ordinal excl
        const double v = in + hp;
        if (excl == 0 && sc.starts_mid) {
            if (DOT) dot = fma(__ldg(e.p + actual_row(m, sc.row0)), v, dot);
            m.part[c] = v;
        } else {
            const int64_t Rw = actual_row(m, sc.row0 + excl);
            if (DOT) dot = fma(__ldg(e.p + Rw), v, dot);
            epi_finish_t<RESID>(e, Rw, v);
        }
    }
    const double out31 = __shfl_sync(FULL, out, 31);
    const bool last_end = __shfl_sync(FULL, (bits >> 7) & 1u, 31) != 0;
    if (lane == 0) {
        if (total_ends == 0) {
            if (sc.row0 < m.n_nonempty) {
                if (DOT) dot = fma(__ldg(e.p + actual_row(m, sc.row0)), out31, dot);
                if (sc.starts_mid) m.part[c] = out31;
                else m.carry[c] = out31;
            }
        } else {
            const int64_t ro = sc.row0 + total_ends;
            if (!last_end && ro < m.n_nonempty) {
                if (DOT) dot = fma(__ldg(e.p + actual_row(m, ro)), out31, dot);
                m.carry[c] = out31;
            }
        }
    }
    return dot;
}

// Warps w0, w0 + wstride, ... of a launch take chunks w0, w0 + wstride, ...
// STD: the handle has the default layout (StdLayout), decoded with its widths
// as constants.
template <int K, int R, bool DOT, bool RESID, bool STD = false>
__device__ __forceinline__ double spmv_chunks_direct(const MatView& m, const double* __restrict__ x, const Epi& e,
                                                     int64_t w0, int64_t wstride, int64_t n_chunks) {
    double dot = 0.0;
    for (int64_t c = w0; c < n_chunks; c += wstride) dot += compute_chunk_direct<K, R, DOT, RESID, STD>(m, e, c, x);
    return dot;
}

template <int STAGES, int UPL>
__host__ __device__ inline int chunks_block_smem(const ChunkStage& L) {
    return 128 + STAGES * L.bytes;
}

}  // namespace gse
