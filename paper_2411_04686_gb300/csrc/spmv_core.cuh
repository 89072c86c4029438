// spmv_core.cuh -- building blocks of the GSE-SpMV (Sec. III-C, Alg. 2 and its
// tail variants): the integer-only decoders, value loads, epilogues and the pass
// that finishes rows crossing chunks.  The main loop is in spmv_pipe.cuh.
//
// Schedule: nonzero-split.  A chunk is CH = 256 * UPL consecutive nonzeros,
// processed by one warp; lane l owns UPL consecutive units of 8 nonzeros.  Each
// value is rebuilt in registers with integer operations only (leading one from
// the FP32 image of its segment or by CLZ, exponent from the shared exponent,
// mantissa by shifts; no int->double conversion and no FP64 scaling) and
// accumulated with exactly one DFMA.  Rows
// that end inside a lane are finished there; a row that crosses lanes is
// stitched by a segmented warp scan of the lane carries (skipped when every lane
// sees a row end, which holds whenever rows are at most 8 long); a row that
// crosses chunks leaves one piece per chunk in scratch and is summed, in chunk
// order, by fix_split_rows after the SpMV (deterministic).  Finished rows go
// through an epilogue from the lane that finishes them.
#pragma once

#include "gse_internal.cuh"

namespace gse {

// Value sources: K = 1, 2, 3 are GSE levels; K = 16 / 17 / 32 / 64 the plain CSR
// baselines in FP16 / BF16 / FP32 / FP64 (the level selectors of include/gse.h).
enum { SRC_FP16 = 16, SRC_BF16 = 17, SRC_FP32 = 32, SRC_FP64 = 64 };
// 16-bit value sources (the baselines stored in 2 bytes per nonzero).
__host__ __device__ constexpr bool src16(int K) { return K == SRC_FP16 || K == SRC_BF16; }

// The default layout (segments 16/16/20, groups of 32, no exponent table) with
// its widths as compile-time constants: the decoders read the same fields from
// it as from a MatView, so a kernel built on it decodes bit-identically with
// the shifts folded.
struct StdLayout {
    static constexpr int W1 = 15, s2 = 16, s3 = 20, W2 = 31, W3 = 51;
};
// The widths a decoder reads: the view's own (run time) or the default layout's.
template <bool STD>
struct WidthsOf {
    static __device__ __forceinline__ const MatView& get(const MatView& m) { return m; }
};
template <>
struct WidthsOf<true> {
    static __device__ __forceinline__ StdLayout get(const MatView&) { return StdLayout{}; }
};

// ---- decode (Alg. 2 and the concatenated tails) --------------------------------

// Subnormal results only: ldexp-style rounding (exact first scaling, one rounding).
static __device__ __noinline__ double decode_tiny(uint64_t M, int Eg, int Wk, uint32_t sign) {
    double v = (double)M * __longlong_as_double((uint64_t)(Eg - 1023 - Wk + 1023 + 200) << 52);
    v = v * __longlong_as_double((uint64_t)(1023 - 200) << 52);
    return sign ? -v : v;
}

// Level 1: M_1 = head magnitude (W_1 <= 15 bits).
template <class V>
__device__ __forceinline__ double decode_l1(uint32_t h, int Eg, const V& m) {
    const uint32_t mag = h & ((1u << m.W1) - 1u);
    const uint32_t sign = (h >> m.W1) & 1u;
    const int lz = __clz(mag);                       // leading one at bit 31 - lz
    const int expo = Eg - m.W1 + 31 - lz;
    if (mag != 0 && expo <= 0) return decode_tiny(mag, Eg, m.W1, sign);
    const uint32_t hi = (sign << 31) | ((uint32_t)expo << 20) | ((mag << (lz - 11)) & 0xFFFFFu);
    return __hiloint2double((int)(mag ? hi : (sign << 31)), 0);
}

// Level 1 for the row schedule: the leading one and the shifted mantissa come
// from the FP32 image of M_1 (exact: M_1 < 2^24, built by integer insertion and
// one FP32 subtraction), so the FP64 high word is that image shifted right by 3
// plus an exponent offset.  eoff = (E_g - W_1 - 127) << 20, per group.
template <class V>
__device__ __forceinline__ double decode_l1_f(uint32_t h, int Eg, uint32_t eoff, const V& m) {
    const uint32_t mag = h & ((1u << m.W1) - 1u);
    const uint32_t sign = (h >> m.W1) << 31;
    const float f = __uint_as_float(0x4B000000u | mag) - 8388608.0f;   // == (float)mag
    const uint32_t fb = __float_as_uint(f);
    if (mag != 0 && Eg <= m.W1) return decode_tiny(mag, Eg, m.W1, sign >> 31);
    const uint32_t hi = mag ? ((fb >> 3) + eoff) | sign : sign;
    return __hiloint2double((int)hi, 0);
}

// Level 2: M_2 = head magnitude << s2 | tail1 (W_2 <= 31 bits).
template <class V>
__device__ __forceinline__ double decode_l2(uint32_t h, uint32_t t1, int Eg, const V& m) {
    const uint32_t M = ((h & ((1u << m.W1) - 1u)) << m.s2) | t1;
    const uint32_t sign = (h >> m.W1) & 1u;
    const int lz = __clz(M);
    const int expo = Eg - m.W2 + 31 - lz;
    if (M != 0 && expo <= 0) return decode_tiny(M, Eg, m.W2, sign);
    const uint64_t mm = (uint64_t)M << (lz + 21);    // leading one lands on bit 52
    const uint32_t hi = (sign << 31) | ((uint32_t)expo << 20) | ((uint32_t)(mm >> 32) & 0xFFFFFu);
    return M ? __hiloint2double((int)hi, (int)(uint32_t)mm) : __hiloint2double((int)(sign << 31), 0);
}

// Level 3: M_3 = M_2 << s3 | tail2 (W_3 <= 63 bits).
template <class V>
__device__ __forceinline__ double decode_l3(uint32_t h, uint32_t t1, uint32_t t2, int Eg,
                                            const V& m) {
    const uint64_t M = ((uint64_t)((((h & ((1u << m.W1) - 1u)) << m.s2) | t1)) << m.s3) | t2;
    const uint32_t sign = (h >> m.W1) & 1u;
    const int lz = __clzll(M);
    const int expo = Eg - m.W3 + 63 - lz;
    if (M != 0 && expo <= 0) return decode_tiny(M, Eg, m.W3, sign);
    const int sh = lz - 11;                          // 52 - position of the leading one
    const uint64_t mm = sh >= 0 ? (M << sh) : (M >> (-sh));
    const uint64_t bits = ((uint64_t)sign << 63) | ((uint64_t)expo << 52) | (mm & 0xFFFFFFFFFFFFFull);
    return M ? __longlong_as_double((long long)bits) : __longlong_as_double((long long)((uint64_t)sign << 63));
}

// Level 3 when the leading one of M_3 lies in the head (head magnitude != 0)
// and the tails fit below bit 52 (W_3 <= 52): the FP32 image of the head gives
// the exponent and the top mantissa bits exactly as at level 1 (the value's
// leading one is the head's at every level), and the tails T = t1 << s3 | t2
// are shifted in right below it -- no 64-bit CLZ, no data-dependent shift
// direction.  Bit-identical to decode_l3 on the values it accepts; the caller
// checks ok_l3_fast and falls back to decode_l3 otherwise.
__device__ __forceinline__ bool ok_l3_fast(uint32_t h, int Eg, const MatView& m) {
    return (h & ((1u << m.W1) - 1u)) != 0u && Eg > m.W1;
}
__device__ __forceinline__ double decode_l3_fast(uint32_t h, uint32_t t1, uint32_t t2, int Eg, const MatView& m) {
    const uint32_t mag = h & ((1u << m.W1) - 1u);
    const uint32_t fb = __float_as_uint(__uint_as_float(0x4B000000u | mag) - 8388608.0f);
    // the leading one of M_3 sits at bit s2 + s3 + p, p = (fb >> 23) - 127; the
    // tails go to mantissa bits below 52 - p, i.e. T << (52 - s2 - s3 - p)
    const uint64_t T = ((uint64_t)t1 << m.s3) | t2;
    const uint64_t low = T << ((179 - m.s2 - m.s3) - (int)(fb >> 23));
    const uint32_t hi = (((fb >> 3) + ((uint32_t)(Eg - m.W1 - 127) << 20)) | ((h >> m.W1) << 31)) |
                        (uint32_t)(low >> 32);
    return __hiloint2double((int)hi, (int)(uint32_t)low);
}

// Level 3 without a data-dependent branch, for W_3 <= 52 and s3 <= 23: the
// leading one lies in the head, else in tail1, else in tail2; that segment's
// FP32 image gives the exponent and its bits below the leading one, and the
// segments after it are shifted in right below.  Bit-identical to decode_l3
// for every value (zero and, via the group test Eg <= W_3, subnormal results
// included).
template <class V>
__device__ __forceinline__ double decode_l3_sel(uint32_t h, uint32_t t1, uint32_t t2, int Eg, const V& m) {
    const uint32_t mag = h & ((1u << m.W1) - 1u);
    if (Eg <= m.W3) return decode_l3(h, t1, t2, Eg, m);          // results may be subnormal: exact path
    const bool in_h = mag != 0, in_1 = t1 != 0;
    const uint32_t lead = in_h ? mag : (in_1 ? t1 : t2);
    const int base = in_h ? m.s2 + m.s3 : (in_1 ? m.s3 : 0);        // bit position of the lead segment in M_3
    const uint64_t rest = in_h ? (((uint64_t)t1 << m.s3) | t2) : (in_1 ? (uint64_t)t2 : 0ull);
    const uint32_t fb = __float_as_uint(__uint_as_float(0x4B000000u | lead) - 8388608.0f);
    // leading one of M_3 at bit base + p, p = (fb >> 23) - 127; the rest goes to
    // the mantissa bits below 52 - p, i.e. rest << (52 - base - p)
    const uint64_t low = rest << (((179 - base) - (int)(fb >> 23)) & 63);   // in 1..52 whenever lead != 0
    const uint32_t hi = ((fb >> 3) + ((uint32_t)(Eg - m.W3 - 127 + base) << 20)) | ((h >> m.W1) << 31) |
                        (uint32_t)(low >> 32);
    const uint32_t sign = (h >> m.W1) << 31;
    return lead ? __hiloint2double((int)hi, (int)(uint32_t)low) : __hiloint2double((int)sign, 0);
}

// FP32 -> FP64 widening with integer operations (exact; no FP64 pipe use).
__device__ __forceinline__ double widen_f32(uint32_t f) {
    const uint32_t sign = f & 0x80000000u;
    const uint32_t e = (f >> 23) & 0xFFu;
    uint32_t man = f & 0x7FFFFFu;
    if (e == 0xFFu) return __hiloint2double((int)(sign | 0x7FF00000u | (man >> 3)), (int)(man << 29));
    if (e == 0) {
        if (man == 0) return __hiloint2double((int)sign, 0);
        const int lz = __clz(man) - 8;               // leading one at bit 23 - lz
        man = (man << lz) & 0x7FFFFFu;               // ... moved to bit 23 and dropped
        const uint32_t ed = 1023 - 126 - lz;         // man * 2^-149 = 1.f * 2^(-126 - lz)
        return __hiloint2double((int)(sign | (ed << 20) | (man >> 3)), (int)(man << 29));
    }
    return __hiloint2double((int)(sign | ((e + 896u) << 20) | (man >> 3)), (int)(man << 29));
}

// binary16 -> FP64 with integer operations (exact; subnormals normalised by CLZ).
__device__ __forceinline__ double widen_f16(uint32_t h) {
    const uint32_t sign = (h & 0x8000u) << 16;
    const uint32_t e = (h >> 10) & 0x1Fu;
    uint32_t man = h & 0x3FFu;
    if (e == 0x1Fu) return __hiloint2double((int)(sign | 0x7FF00000u | (man << 10)), 0);
    if (e == 0) {
        if (man == 0) return __hiloint2double((int)sign, 0);
        const int lz = __clz(man) - 21;              // leading one at bit 10 - lz
        man = (man << lz) & 0x3FFu;                  // ... moved to bit 10 and dropped
        // man * 2^-24 = 1.f * 2^(-14 - lz)
        return __hiloint2double((int)(sign | ((uint32_t)(1023 - 14 - lz) << 20) | (man << 10)), 0);
    }
    return __hiloint2double((int)(sign | ((e + 1008u) << 20) | (man << 10)), 0);
}
// bfloat16 -> FP64: bfloat16 is the top half of a binary32.
__device__ __forceinline__ double widen_bf16(uint32_t b) { return widen_f32(b << 16); }
template <int K>
__device__ __forceinline__ double widen16(uint32_t v) {
    if constexpr (K == SRC_FP16) return widen_f16(v);
    else return widen_bf16(v);
}

__device__ __forceinline__ uint32_t u16_of(const uint4& w, int i) {
    const uint32_t word = (i >> 1) == 0 ? w.x : (i >> 1) == 1 ? w.y : (i >> 1) == 2 ? w.z : w.w;
    return (i & 1) ? (word >> 16) : (word & 0xFFFFu);
}

// Loads unit u and rebuilds its 8 values.  R: bits of tail2 kept in the packed
// low array (0, 4, 8 or 16; -1 reads the width from the view at run time).
template <int K, int R, bool STD = false>
__device__ __forceinline__ void load_unit(const MatView& m, int64_t u, int* col, double* a) {
    const int4* c4 = reinterpret_cast<const int4*>(m.col) + 2 * u;
    const int4 ca = __ldg(c4), cb = __ldg(c4 + 1);
    col[0] = ca.x; col[1] = ca.y; col[2] = ca.z; col[3] = ca.w;
    col[4] = cb.x; col[5] = cb.y; col[6] = cb.z; col[7] = cb.w;
    if constexpr (K == SRC_FP64) {
        const double2* v2 = reinterpret_cast<const double2*>(m.val64) + 4 * u;
#pragma unroll
        for (int j = 0; j < 4; j++) {
            const double2 d = __ldcs(v2 + j);
            a[2 * j] = d.x;
            a[2 * j + 1] = d.y;
        }
    } else if constexpr (K == SRC_FP32) {
        const uint4* f4 = reinterpret_cast<const uint4*>(m.val32) + 2 * u;
        const uint4 fa = __ldcs(f4), fb = __ldcs(f4 + 1);
        a[0] = widen_f32(fa.x); a[1] = widen_f32(fa.y); a[2] = widen_f32(fa.z); a[3] = widen_f32(fa.w);
        a[4] = widen_f32(fb.x); a[5] = widen_f32(fb.y); a[6] = widen_f32(fb.z); a[7] = widen_f32(fb.w);
    } else if constexpr (src16(K)) {
        const uint4 w = __ldcs(reinterpret_cast<const uint4*>(K == SRC_FP16 ? m.val16 : m.valbf) + u);
#pragma unroll
        for (int i = 0; i < 8; i++) a[i] = widen16<K>(u16_of(w, i));
    } else {
        // STD: the default layout (checked at launch): groups of 32, no table
        const bool tbl = !STD && m.tbl;
        const int Eg0 = tbl ? 0 : (int)__ldg(m.gexp + ((u * GSE_UNIT) >> (STD ? 5 : m.g_shift)));
        const uint4 hw = __ldcs(reinterpret_cast<const uint4*>(m.head) + u);
        uint4 t1w = make_uint4(0, 0, 0, 0), t2w = make_uint4(0, 0, 0, 0);
        uint32_t lo[4] = {0, 0, 0, 0};
        if constexpr (K >= 2) t1w = __ldcs(reinterpret_cast<const uint4*>(m.tail1) + u);
        if constexpr (K >= 3) {
            t2w = __ldcs(reinterpret_cast<const uint4*>(m.t2hi) + u);
            if constexpr (R == 4) lo[0] = __ldcs(m.t2lo + u);
            if constexpr (R == 8) { const uint2 l2 = __ldcs(reinterpret_cast<const uint2*>(m.t2lo) + u); lo[0] = l2.x; lo[1] = l2.y; }
            if constexpr (R == 16) { const uint4 l4 = __ldcs(reinterpret_cast<const uint4*>(m.t2lo) + u); lo[0] = l4.x; lo[1] = l4.y; lo[2] = l4.z; lo[3] = l4.w; }
            if constexpr (R < 0) {
                if (m.r_lo == 4) lo[0] = __ldcs(m.t2lo + u);
                else if (m.r_lo == 8) { const uint2 l2 = __ldcs(reinterpret_cast<const uint2*>(m.t2lo) + u); lo[0] = l2.x; lo[1] = l2.y; }
                else if (m.r_lo == 16) { const uint4 l4 = __ldcs(reinterpret_cast<const uint4*>(m.t2lo) + u); lo[0] = l4.x; lo[1] = l4.y; lo[2] = l4.z; lo[3] = l4.w; }
            }
        }
        const auto& L = WidthsOf<STD>::get(m);
#pragma unroll
        for (int i = 0; i < 8; i++) {
            uint32_t h = u16_of(hw, i);
            const int Eg = tbl ? (int)__ldg(m.etab + tbl_index(m, col[i], h)) : Eg0;   // table format: per value
            if constexpr (K == 1) {
                a[i] = decode_l1_f(h, Eg, (uint32_t)(Eg - L.W1 - 127) << 20, L);
            } else if constexpr (K == 2) {
                a[i] = decode_l2(h, u16_of(t1w, i), Eg, L);
            } else {
                uint32_t t2 = u16_of(t2w, i);
                if constexpr (R > 0) {
                    const int bit = i * R;
                    t2 = (t2 << R) | ((lo[bit >> 5] >> (bit & 31)) & ((1u << R) - 1u));
                } else if constexpr (R < 0) {
                    if (m.r_lo > 0) {
                        const int bit = i * m.r_lo;
                        t2 = (t2 << m.r_lo) | ((lo[bit >> 5] >> (bit & 31)) & ((1u << m.r_lo) - 1u));
                    }
                }
                if constexpr (R == 0 || R == 4) a[i] = decode_l3_sel(h, u16_of(t1w, i), t2, Eg, L);
                else a[i] = decode_l3(h, u16_of(t1w, i), t2, Eg, L);
            }
        }
    }
}

// ---- epilogues ----------------------------------------------------------------
// EPI_STORE: y[R] = v.  EPI_RESID: y[R] = b[R] - v.  EPI_CG_PQ: y[R] = v and
// dot += p[R] * v (linear in v, so row pieces may be added separately).
struct Epi {
    int kind;
    double* y;
    const double* b;
    const double* p;
};

__device__ __forceinline__ void epi_finish(const Epi& e, int64_t R, double v) {
    if (e.kind == EPI_RESID) e.y[R] = e.b[R] - v;
    else e.y[R] = v;
}

// Same, with the kind fixed at compile time (no predicated-off FP64 work).
template <bool RESID>
__device__ __forceinline__ void epi_finish_t(const Epi& e, int64_t R, double v) {
    if constexpr (RESID) e.y[R] = e.b[R] - v;
    else e.y[R] = v;
}

// Maps a compact (nonempty) row index to the matrix row.
__device__ __forceinline__ int64_t actual_row(const MatView& m, int64_t rc) {
    return m.nzrow ? (int64_t)__ldg(m.nzrow + rc) : rc;
}

// Rows that cross chunk boundaries.  A chunk stores the piece of the row that
// was open when it began in part[c] (only if it began mid-row) and the piece of
// the row still open at its end in carry[c] (only if that row began inside it).
// fix_split_rows (a separate, later pass) adds carry[c1] + part[c1+1..c2] in
// chunk order for every such row: deterministic, and no fences or atomics in
// the SpMV itself.
template <int CH>
__device__ __forceinline__ void fix_split_rows(const MatView& m, const Epi& e, int64_t n_chunks,
                                               int64_t tid, int64_t nthreads) {
    for (int64_t c = tid + 1; c < n_chunks; c += nthreads) {
        const int64_t pe = c * CH - 1;
        if ((__ldg(m.rowend + (pe >> 5)) >> (pe & 31)) & 1u) continue;   // boundary on a row end
        const int64_t rc = __ldg(m.blk_row0 + c * (CH / 256));
        if (rc >= m.n_nonempty) continue;
        const int64_t R = actual_row(m, rc);
        const int64_t s = __ldg(m.row_ptr + R), t = __ldg(m.row_ptr + R + 1);
        const int64_t c2 = (t - 1) / CH;
        if (c2 != c) continue;            // a later boundary finishes this row
        const int64_t c1 = s / CH;
        double sum = m.carry[c1];
        for (int64_t cc = c1 + 1; cc <= c2; cc++) sum += m.part[cc];
        epi_finish(e, R, sum);
    }
}

// Zero rows (every SpMV writes them: y = 0, or y = b for the residual form).
__device__ __forceinline__ void fill_empty_rows(const MatView& m, const Epi& e, int64_t tid,
                                                int64_t nthreads) {
    for (int64_t i = tid; i < m.n_empty; i += nthreads) {
        const int64_t R = __ldg(m.empty + i);
        epi_finish(e, R, 0.0);
    }
}

// Deterministic sum of one double per thread of the block into red[0]
// (thread 0 holds the result).  red: >= blockDim/32 doubles of shared memory.
__device__ __forceinline__ double block_sum(double v, double* red) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if (lane == 0) red[w] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0) {
        for (int i = 0; i < (int)(blockDim.x >> 5); i++) s += red[i];
    }
    return s;
}

}  // namespace gse
