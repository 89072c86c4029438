// spmv_lanerow.cuh -- GSE-SpMV with one row per lane and two rows per lane in
// flight, each warp staging its own 64-row tiles (Sec. III-C, Alg. 2 and the
// tail variants).
//
// For matrices with short rows (stencils, every batched system).  A warp owns
// tiles t0, t0 + stride, ... of 64 consecutive rows; lane l runs rows l and
// 32 + l of a tile.  The warp copies the tile's slice of the column array and
// of the live segment arrays (or of the plain CSR values of a baseline) into
// its own two-stage ring in shared memory with cp.async (16-byte pieces, every
// lane issuing, L1 bypassed) one tile ahead of the tile it computes: no
// CTA-wide barrier, no producer thread, no mbarrier.  Reading the slice back
// from shared memory turns the lane-strided row walk into conflict-free
// accesses.  Each lane gathers the x values of both its rows, then accumulates
// both rows in order with one DFMA per nonzero, the two rows' FMA chains
// interleaved.
//
// Why two rows: on GB300 a DFMA takes 64 cycles and the FP64 unit needs about
// four dependent chains per SM in flight to stay busy, while each warp spends
// most of a tile waiting for its loads.  Two independent chains per warp
// double the FP64 work in flight and halve the per-row share of the tile's
// fixed costs (copies, bounds, exponents, stores).  Each row is still summed in
// column order from 0, so the result is the same as the one-row order.
//
// Decoding, for the 16/16/20 segment layout with groups of 32 (W_1 = 15,
// W_2 = 31, W_3 = 51) and a row whose nonzeros share one group exponent E_g
// (any row within two groups of equal exponent): the value's leading one is
// the head's leading one at every level, so its exponent and top bits come from
// the FP32 image of the head magnitude (exact: < 2^15) shifted into the FP64
// high word plus a per-row offset, and the tails are shifted in below it with
// one funnel shift.  A batch holding a zero head magnitude at level 2 or 3
// (leading one in a tail) and any row with other exponents fall back to the
// general decoders of spmv_core.cuh with each nonzero's own group exponent;
// both give the exact value, so the result does not depend on the path.
#pragma once

#include "spmv_core.cuh"

namespace gse {

// ---- cp.async (asynchronous global -> shared copies) -----------------------
__device__ __forceinline__ void cpa16(uint32_t dst, const void* src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(src) : "memory");
}
__device__ __forceinline__ void cpa_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cpa_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// Standard layout of the fast decoders.
constexpr int LR_W1 = 15;
constexpr int LR_EBIAS = LR_W1 + 127;      // E_g - W_1 - 127: FP32 image -> FP64 exponent offset
constexpr int LR_STAGES = 2;               // the tile being computed, the next one in flight

// True when a handle's encoding is the one the lane-row decoders are written
// for (per-group exponents, G = 32, segments 16/16/20 or a prefix of them).
inline bool lanerow_format(const MatView& v, int group_size, int n_seg) {
    if (v.tbl || group_size != 32 || v.s1 != 16) return false;
    if (n_seg >= 2 && v.s2 != 16) return false;
    if (n_seg >= 3 && (v.s3 != 20 || v.r_lo != 4)) return false;
    return true;
}

// True when a table-format handle can run the lane-row kernels (standalone
// SpMV): the exponent index in the column word and the 16/16/20 segments.
inline bool lanerow_format_tbl(const MatView& v, int n_seg) {
    if (!v.tbl || v.hi_mask != 0 || v.s1 != 16) return false;
    if (n_seg >= 2 && v.s2 != 16) return false;
    if (n_seg >= 3 && (v.s3 != 20 || v.r_lo != 4)) return false;
    return true;
}

// Rows per lane at each value source: two at level 1 (the least decode work,
// so more chains per warp pay), one elsewhere (wider decode: one row per lane
// keeps more warps resident).
template <int K>
__host__ __device__ constexpr int lr_rows_per_lane() { return K == 1 ? 2 : 1; }

// Layout of one stage (one tile of 32 * R rows), fixed at compile time: the
// column slice, then the value arrays, each CAP = 256 * R elements.  A tile
// whose slice (its first nonzero rounded down to 8, its end rounded up to 8)
// is wider runs on the staged row kernel instead.  The slices start on a
// multiple of 8 nonzeros (t2lo: of 32 = 4 words), so every 16-byte copy is
// aligned, and every shared-memory offset below is a constant.
template <int K, int RR = lr_rows_per_lane<K>()>
struct LrLayout {
    static constexpr int R = RR;
    static constexpr int CAP = 256 * R;
    static constexpr int VB = K == SRC_FP64 ? 8 : K == SRC_FP32 ? 4 : 2;   // bytes per value (per segment)
    static constexpr int NSEG = K >= 3 && K <= 3 ? 3 : K == 2 ? 2 : 1;       // value arrays
    static constexpr int OFF_V = CAP * 4;
    static constexpr int OFF_LO = OFF_V + CAP * VB * NSEG;
    static constexpr int LO_BYTES = K == 3 ? CAP / 2 + 48 : 0;              // nibble words + alignment slack
    static constexpr int BYTES = (OFF_LO + LO_BYTES + 127) / 128 * 128;
};

// Shared memory of a CTA of W warps: LR_STAGES stages per warp plus a tail pad.
// A lane past its row reads up to 63 elements beyond its row (rows are at
// most 64 long); those values are never used, and the pad keeps the reads of
// the last stage's last array inside the allocation: 63 values of the widest
// source (FP64: 504 bytes), else a few nibble words or 16-bit values.
template <int K>
__host__ __device__ constexpr int lr_pad() {
    return K == SRC_FP64 ? 512 : K == SRC_FP32 ? 256 : 128;
}
template <int K, int R = lr_rows_per_lane<K>()>
__host__ __device__ constexpr int lr_smem(int W) {
    return W * LR_STAGES * LrLayout<K, R>::BYTES + lr_pad<K>();
}

// Copies `nc` 16-byte chunks from g to shared address st: lane l takes chunks
// l, l + 32, ... (consecutive lanes, consecutive chunks: each warp-wide copy
// covers 512 contiguous bytes).  ROUNDS, the most chunks a lane can get, is
// fixed by the layout; the rounds are unrolled and predicated.
template <int ROUNDS>
__device__ __forceinline__ void lr_copy(uint32_t st, const char* g, int nc, int lane) {
#pragma unroll
    for (int j = 0; j < ROUNDS; j++) {
        const int c = lane + 32 * j;
        if (c < nc) cpa16(st + c * 16, g + c * 16);
    }
}

// Copies slice [e0, e1) of the arrays level K reads into stage `st`.
template <int K, int R>
__device__ __forceinline__ void lr_issue(const MatView& m, uint32_t st, int e0, int e1, int lane) {
    using LY = LrLayout<K, R>;
    constexpr int C = LY::CAP;
    const int a8 = e0 & ~7, n8 = ((e1 + 7) & ~7) - a8;
    lr_copy<C / 128>(st, reinterpret_cast<const char*>(m.col + a8), n8 >> 2, lane);
    if constexpr (K == SRC_FP64) {
        lr_copy<C / 64>(st + LY::OFF_V, reinterpret_cast<const char*>(m.val64 + a8), n8 >> 1, lane);
    } else if constexpr (K == SRC_FP32) {
        lr_copy<C / 128>(st + LY::OFF_V, reinterpret_cast<const char*>(m.val32 + a8), n8 >> 2, lane);
    } else if constexpr (src16(K)) {
        lr_copy<C / 256>(st + LY::OFF_V, reinterpret_cast<const char*>((K == SRC_FP16 ? m.val16 : m.valbf) + a8),
                         n8 >> 3, lane);
    } else {
        lr_copy<C / 256>(st + LY::OFF_V, reinterpret_cast<const char*>(m.head + a8), n8 >> 3, lane);
        if constexpr (K >= 2)
            lr_copy<C / 256>(st + LY::OFF_V + 2 * C, reinterpret_cast<const char*>(m.tail1 + a8), n8 >> 3, lane);
        if constexpr (K >= 3) {
            lr_copy<C / 256>(st + LY::OFF_V + 4 * C, reinterpret_cast<const char*>(m.t2hi + a8), n8 >> 3, lane);
            // nibble words of the slice, 8 nonzeros per word, 4 words per chunk
            const int w0 = (e0 >> 5) << 2, w1 = ((e1 + 31) >> 5) << 2;
            lr_copy<1>(st + LY::OFF_LO, reinterpret_cast<const char*>(m.t2lo + w0), (w1 - w0) >> 2, lane);
        }
    }
}

// FP64 high word of a head whose magnitude is nonzero: exponent and top bits
// from the FP32 image of the magnitude, plus the row's exponent offset
// eoff = (E_g - W_1 - 127) << 20, plus the sign.  fb returns the image.
__device__ __forceinline__ uint32_t lr_head_hi(uint32_t h, uint32_t eoff, uint32_t& fb) {
    fb = __float_as_uint(__uint_as_float(0x4B000000u | (h & 0x7FFFu)) - 8388608.0f);
    return ((fb >> 3) + eoff) | ((h << 16) & 0x80000000u);
}

// Fast decode of one value (leading one in the head at K >= 2).  nib16: its
// low tail2 bits already at bits 16..19 (level 3).
template <int K>
__device__ __forceinline__ double lr_fast(uint32_t h, uint32_t t1, uint32_t t2, uint32_t nib16, uint32_t eoff) {
    const uint32_t fb = __float_as_uint(__uint_as_float(0x4B000000u | (h & 0x7FFFu)) - 8388608.0f);
    const uint32_t base = (fb >> 3) + eoff;                // exponent and the head's bits below its leading one
    const uint32_t hs = h << 16;                           // sign at bit 31
    uint32_t hi, lo = 0;
    if constexpr (K == 1) {
        hi = (h & 0x7FFFu) ? (base | (hs & 0x80000000u)) : (hs & 0x80000000u);
    } else {
        const uint32_t p = (fb >> 23) - 127u;              // leading one of the head magnitude
        uint32_t hiT, loT;
        if constexpr (K == 2) {
            hiT = t1 << 4;                                 // tail1 right below the head bits
            loT = 0;
        } else {
            // (tail1 << 20 | tail2) << 16 as hiT:loT, with W = tail1 << 16 | top 16 bits of tail2
            const uint32_t W = __byte_perm(t2, t1, 0x5410);
            hiT = W >> 12;
            loT = (W << 20) | nib16;
        }
        hi = ((base | (hiT >> p))) | (hs & 0x80000000u);
        lo = __funnelshift_r(loT, hiT, p);
    }
    return __hiloint2double((int)hi, (int)lo);
}

// General decode of one value with its own group exponent (any head).  A
// handle on this kernel has the default layout (lanerow_format), so the
// decoders take its widths as compile-time constants.
template <int K>
__device__ __forceinline__ double lr_general(const MatView& m, uint32_t h, uint32_t t1, uint32_t t2, uint32_t nib,
                                             int Eg) {
    (void)m;
    if constexpr (K == 1) return decode_l1(h, Eg, StdLayout{});
    else if constexpr (K == 2) return decode_l2(h, t1, Eg, StdLayout{});
    else return decode_l3(h, t1, (t2 << 4) | nib, Eg, StdLayout{});
}

// The rows of one lane within a staged tile (R of them: rows l, 32 + l, ...).
template <int R>
struct LrRows {
    int o[R];          // stage-local index of the row's first nonzero
    int len[R];        // nonzeros
    int rs[R];         // CSR index of the first nonzero
    uint32_t eoff[R];  // fast-decode exponent offset
};

// x[c] if `live`, else 0: a zeroed register and a predicated read-only load
// (no select after the load).
__device__ __forceinline__ double lr_ldx(const double* p, bool live) {
    double v;
    asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %2, 0;\n\tmov.b64 %0, 0;\n\t@q ld.global.nc.f64 %0, [%1];\n\t}"
        : "=d"(v)
        : "l"(p), "r"((unsigned)live));
    return v;
}

// Nonzeros u0 .. u0 + N - 1 of the lane's R rows: every gather first (all in
// flight), then the rows' FMA chains interleaved, each row in column order.
// TBL: the global exponent table with the index in the column word (Sec.
// III-C; 0: the per-group format): columns are masked, and each value's
// exponent is its table entry.
template <int K, int N, int R, bool FAST, int TBL = 0>
__device__ __forceinline__ void lr_batch(const MatView& m, const double* __restrict__ x, const unsigned char* st,
                                         const LrRows<R>& W, int u0, int wbase, double* acc) {
    using LY = LrLayout<K, R>;
    const int32_t* scol = reinterpret_cast<const int32_t*>(st);
    double xv[R][N];
#pragma unroll
    for (int r = 0; r < R; r++) {
#pragma unroll
        for (int u = 0; u < N; u++) {
            const int32_t c = scol[W.o[r] + u0 + u];
            xv[r][u] = lr_ldx(x + (TBL ? col_of(m, c) : c), u0 + u < W.len[r]);
        }
    }
    if constexpr (K == SRC_FP64) {
        const double* sv = reinterpret_cast<const double*>(st + LY::OFF_V);
#pragma unroll
        for (int u = 0; u < N; u++)
#pragma unroll
            for (int r = 0; r < R; r++)
                if (u0 + u < W.len[r]) acc[r] = fma(sv[W.o[r] + u0 + u], xv[r][u], acc[r]);
    } else if constexpr (K == SRC_FP32) {
        const uint32_t* sv = reinterpret_cast<const uint32_t*>(st + LY::OFF_V);
#pragma unroll
        for (int u = 0; u < N; u++)
#pragma unroll
            for (int r = 0; r < R; r++)
                if (u0 + u < W.len[r]) acc[r] = fma(widen_f32(sv[W.o[r] + u0 + u]), xv[r][u], acc[r]);
    } else if constexpr (src16(K)) {
        const uint16_t* sv = reinterpret_cast<const uint16_t*>(st + LY::OFF_V);
#pragma unroll
        for (int u = 0; u < N; u++)
#pragma unroll
            for (int r = 0; r < R; r++)
                if (u0 + u < W.len[r]) acc[r] = fma(widen16<K>(sv[W.o[r] + u0 + u]), xv[r][u], acc[r]);
    } else {
        const uint16_t* sh = reinterpret_cast<const uint16_t*>(st + LY::OFF_V);
        const uint32_t* lw = reinterpret_cast<const uint32_t*>(st + LY::OFF_LO);
        // the batch's low tail2 nibbles of each row, nonzero u at bits 4u.. of one word
        uint32_t nib[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            nib[r] = 0;
            if constexpr (K >= 3) {
                const int e = W.rs[r] + u0, w = (e >> 3) - wbase;
                nib[r] = __funnelshift_r(lw[w], lw[w + 1], (e & 7) * 4);
            }
        }
#pragma unroll
        for (int u = 0; u < N; u++) {
#pragma unroll
            for (int r = 0; r < R; r++) {
                const int i = W.o[r] + u0 + u;
                const uint32_t h = sh[i];
                const uint32_t t1 = K >= 2 ? (uint32_t)sh[LY::CAP + i] : 0u;
                const uint32_t t2 = K >= 3 ? (uint32_t)sh[2 * LY::CAP + i] : 0u;
                const uint32_t nb = (nib[r] >> (4 * u)) & 0xFu;
                double a;
                if constexpr (FAST) {
                    // the nibble placed at bits 16..19 with one shift and a mask
                    const uint32_t nb16 = (4 * u <= 16 ? nib[r] << (16 - 4 * u) : nib[r] >> (4 * u - 16)) & 0xF0000u;
                    uint32_t eoff = W.eoff[r];
                    if constexpr (TBL != 0) {          // the value's own table entry
                        const uint32_t ix = (uint32_t)((uint64_t)(uint32_t)scol[i] >> m.ei_shift);
                        eoff = (uint32_t)((int)__ldg(m.etab + ix) - LR_EBIAS) << 20;
                    }
                    a = lr_fast<K>(h, t1, t2, nb16, eoff);
                } else if constexpr (TBL != 0) {
                    // the index bits of the column word (past a row's end a
                    // stale word still gives an index below the table's 64)
                    const uint32_t ix = (uint32_t)((uint64_t)(uint32_t)scol[i] >> m.ei_shift);
                    a = lr_general<K>(m, h, t1, t2, nb, (int)__ldg(m.etab + ix));
                } else {
                    const int Eg = u0 + u < W.len[r] ? (int)__ldg(m.gexp + ((W.rs[r] + u0 + u) >> 5)) : 0;
                    a = lr_general<K>(m, h, t1, t2, nb, Eg);
                }
                // past the row's end x reads 0 and the group format's fast
                // decoders give a finite value, so the FMA adds an exact zero
                // (acc is never -0); a table entry read through a stale column
                // word may not, so the table format predicates the FMA
                if ((FAST && TBL == 0) || u0 + u < W.len[r]) acc[r] = fma(a, xv[r][u], acc[r]);
            }
        }
    }
}

// The lane's rows: batches of 8, then one batch of the warp's remaining length
// (the longest row of the warp's tile).
template <int K, int R, bool FAST, int TBL = 0>
__device__ __forceinline__ void lr_rows(const MatView& m, const double* __restrict__ x, const unsigned char* st,
                                        const LrRows<R>& W, int maxlen, int wbase, double* acc) {
    int u0 = 0;
    for (; u0 + 8 <= maxlen; u0 += 8) lr_batch<K, 8, R, FAST, TBL>(m, x, st, W, u0, wbase, acc);
    switch (maxlen - u0) {
#define GSE_LR_TAIL(NN) \
    case NN: lr_batch<K, NN, R, FAST, TBL>(m, x, st, W, u0, wbase, acc); break;
        GSE_LR_TAIL(7) GSE_LR_TAIL(6) GSE_LR_TAIL(5) GSE_LR_TAIL(4) GSE_LR_TAIL(3) GSE_LR_TAIL(2) GSE_LR_TAIL(1)
#undef GSE_LR_TAIL
        default: break;
    }
}

// The fast-decode test and exponent offset of one row (group format).
__device__ __forceinline__ bool lr_row_fast(const MatView& m, int rs, int rt, uint32_t* eoff) {
    if (rt == rs) {
        *eoff = 0;
        return true;
    }
    const int Ega = (int)__ldg(m.gexp + (rs >> 5)), Egb = (int)__ldg(m.gexp + ((rt - 1) >> 5));
    *eoff = (uint32_t)(Ega - LR_EBIAS) << 20;
    return ((rt - 1) >> 5) - (rs >> 5) <= 1 && Ega == Egb && Ega > LR_W1;
}

// True when no head of the staged slice (n8 heads) has a zero magnitude: every
// leading one is then in the head (levels 2 and 3 decode fast).  Eight heads
// per 16-byte word; a zero 15-bit field is found with the borrow test
// (v - 1) & ~v & 0x8000 per 16-bit lane.
template <int K, int R>
__device__ __forceinline__ bool lr_heads_nonzero(const unsigned char* st, int n8, int lane) {
    const uint4* hw = reinterpret_cast<const uint4*>(st + LrLayout<K, R>::OFF_V);
    uint32_t z = 0;
#pragma unroll
    for (int j = 0; j < LrLayout<K, R>::CAP / 256; j++) {
        const int c = lane + 32 * j;
        const uint4 w = c < n8 / 8 ? hw[c] : make_uint4(0x10001u, 0x10001u, 0x10001u, 0x10001u);
        const uint32_t v[4] = {w.x & 0x7FFF7FFFu, w.y & 0x7FFF7FFFu, w.z & 0x7FFF7FFFu, w.w & 0x7FFF7FFFu};
#pragma unroll
        for (int j = 0; j < 4; j++) z |= (v[j] - 0x00010001u) & ~v[j] & 0x80008000u;
    }
    return __all_sync(0xFFFFFFFFu, z == 0u);
}

// The R rows of every lane of one staged tile whose slice starts at CSR
// index e0 and ends at e1; rs[r], rt[r]: the lane's row r.
template <int K, int R, int TBL = 0>
__device__ __forceinline__ void lr_tile(const MatView& m, const double* __restrict__ x, const unsigned char* st, int e0, int e1, const int* rs, const int* rt,
                                        int lane, double* acc) {
    const unsigned FULL = 0xFFFFFFFFu;
    const int a8 = e0 & ~7;
    LrRows<R> W;
    int mx = 0;
#pragma unroll
    for (int r = 0; r < R; r++) {
        W.o[r] = rs[r] - a8;
        W.len[r] = rt[r] - rs[r];
        W.rs[r] = rs[r];
        W.eoff[r] = 0;
        mx = max(mx, W.len[r]);
        acc[r] = 0.0;
    }
    const int maxlen = __reduce_max_sync(FULL, mx);
    const int wbase = (e0 >> 5) << 2;
    if constexpr (K <= 3 && TBL == 1) {
        lr_rows<K, R, false, 1>(m, x, st, W, maxlen, wbase, acc);
    } else if constexpr (K <= 3 && TBL == 2) {
        // every table entry exceeds W_1 (checked at launch): a value's leading
        // one is in its head whenever the head magnitude is nonzero
        const bool fast = K < 2 || lr_heads_nonzero<K, R>(st, ((e1 + 7) & ~7) - a8, lane);
        if (fast) lr_rows<K, R, true, 2>(m, x, st, W, maxlen, wbase, acc);
        else lr_rows<K, R, false, 2>(m, x, st, W, maxlen, wbase, acc);
    } else if constexpr (K <= 3) {
        bool ok = true;
#pragma unroll
        for (int r = 0; r < R; r++) ok = lr_row_fast(m, rs[r], rt[r], &W.eoff[r]) && ok;
        bool fast = __all_sync(FULL, ok);
        if (K >= 2 && fast) fast = lr_heads_nonzero<K, R>(st, ((e1 + 7) & ~7) - a8, lane);
        if (fast) lr_rows<K, R, true>(m, x, st, W, maxlen, wbase, acc);
        else lr_rows<K, R, false>(m, x, st, W, maxlen, wbase, acc);
    } else {
        lr_rows<K, R, false, TBL>(m, x, st, W, maxlen, wbase, acc);
    }
}

// The warp's share of an SpMV: tiles of 32 * R rows t0, t0 + tstride, ...
// (ntile in all), through the warp's two stages at `wsm`.  Row and nonzero
// indices are 32-bit (the CSR's row pointers are int32).  Returns the lane's
// share of p.y (DOT) -- zero otherwise.
template <int K, bool DOT, bool RESID, int R = lr_rows_per_lane<K>(), int TBL = 0>
__device__ __forceinline__ double lr_loop(const MatView& m, const double* __restrict__ x, const Epi& e, int64_t t0_,
                                          int64_t tstride_, int64_t ntile_, unsigned char* wsm) {
    constexpr int TILE = 32 * R;
    constexpr int SB = LrLayout<K, R>::BYTES;
    const unsigned FULL = 0xFFFFFFFFu;
    const int lane = threadIdx.x & 31;
    const int n = (int)m.n_rows, t0 = (int)t0_, tstride = (int)tstride_, ntile = (int)ntile_;
    const int32_t* __restrict__ rp = m.row_ptr;
    double dot = 0.0;
    if (t0 >= ntile) return dot;
    // row starts of the lane's rows of tile t, and the tile's end
    struct Bounds { int a[R]; int end; };
    auto bounds = [&](int t) {
        Bounds bd;
#pragma unroll
        for (int r = 0; r < R; r++) bd.a[r] = __ldg(rp + min(t * TILE + 32 * r + lane, n));
        bd.end = __ldg(rp + min(t * TILE + TILE, n));
        return bd;
    };
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(wsm);
    Bounds cur = bounds(t0), nxt;
    lr_issue<K, R>(m, s0, __shfl_sync(FULL, cur.a[0], 0), cur.end, lane);
    cpa_commit();
    if (t0 + tstride < ntile) nxt = bounds(t0 + tstride);
    int s = 0;
    for (int t = t0; t < ntile; t += tstride) {
        if (t + tstride < ntile) lr_issue<K, R>(m, s0 + (s ^ 1) * SB, __shfl_sync(FULL, nxt.a[0], 0), nxt.end, lane);
        cpa_commit();
        Bounds nn;
        if (t + 2 * tstride < ntile) nn = bounds(t + 2 * tstride);
        // row ends: the next lane's start; lane 31's from the next row group / the tile end
        int rt[R];
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int d = __shfl_down_sync(FULL, cur.a[r], 1);
            const int nxt0 = r + 1 < R ? __shfl_sync(FULL, cur.a[r + 1 < R ? r + 1 : r], 0) : cur.end;
            rt[r] = lane == 31 ? nxt0 : d;
        }
        const int e0 = __shfl_sync(FULL, cur.a[0], 0);
        cpa_wait<1>();                      // tile t's copies (all but the newest group) have landed
        __syncwarp();
        double acc[R];
        lr_tile<K, R, TBL>(m, x, wsm + s * SB, e0, cur.end, cur.a, rt, lane, acc);
#pragma unroll
        for (int r = 0; r < R; r++) {
            const int row = t * TILE + 32 * r + lane;
            if (row < n) {
                if (DOT) dot = fma(__ldg(e.p + row), acc[r], dot);
                epi_finish_t<RESID>(e, row, acc[r]);
            }
        }
        __syncwarp();                       // stage s is refilled at the next iteration
        cur = nxt;
        nxt = nn;
        s ^= 1;
    }
    cpa_wait<0>();
    return dot;
}

// Shared memory of a lane-row CTA of W warps at value source k with R rows
// per lane.
template <int R>
inline int lanerow_smem_k(int k, int W) {
    switch (k) {
        case 1: return lr_smem<1, R>(W);
        case 2: return lr_smem<2, R>(W);
        case 3: return lr_smem<3, R>(W);
        case SRC_FP32: return lr_smem<SRC_FP32, R>(W);
        case SRC_FP16: return lr_smem<SRC_FP16, R>(W);
        case SRC_BF16: return lr_smem<SRC_BF16, R>(W);
        default: return lr_smem<SRC_FP64, R>(W);
    }
}

// Widest slice a lane-row stage holds with R rows per lane.
constexpr int lr_cap_rows(int R) { return 256 * R; }

}  // namespace gse
