/*
 * gse_oracle.c -- plain, slow, single-threaded CPU oracle for the
 * group-shared-exponent (GSE) SpMV and the stepped mixed-precision CG/GMRES
 * of "Precision-Aware Iterative Algorithms Based on Group-Shared Exponents
 * of Floating-Point Numbers" (Gao et al., arXiv 2411.04686).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library calls, links or
 * includes this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or constant
 * generator with the CUDA path.
 *
 * Every routine follows the paper's definition in the paper's order, with no
 * blocking, fusion or reordering, so that it can be checked against the paper
 * by eye.  All floating point is IEEE binary64; build with -ffp-contract=off so
 * that x86_64 and aarch64 produce identical results (FMA appears only where it
 * is written out as fma()).
 *
 * Format variant (Sec. III-B applied to one group):  the set F of the paper is
 * one group of G consecutive CSR nonzeros, with numExp = 1.  The rule of the
 * denormalized representation (Sec. III-B, "Denormalized Representation") then
 * forces the single shared exponent of the group to be max(e) + 1, so every
 * value is denormalized against it and the exponent index takes 0 bits.
 *
 * Notation: seg_bits = {s1, s2, s3}; s1 includes the sign bit (the head keeps
 * the sign in its top bit, Alg. 2), so the head carries W_1 = s1 - 1 magnitude
 * bits and level k carries W_k = W_1 + s2 + ... + s_k.  E_g is the biased
 * group exponent, d = E_g - e >= 1 the alignment distance of one value.
 *
 * Table variant (the paper's default format): orc_table_* keep one table of
 * numExp shared exponents for the whole matrix (Sec. III-B) and an exponent
 * index per nonzero (Sec. III-C keeps it in the column index's top bits); a
 * value whose exponent plus 1 is not in the table is denormalized against the
 * nearest larger entry (Alg. 1).  The segment split is the same.
 * orc_table_build_sampled is the sampled extraction of Sec. III-B (one random
 * row per row block); orc_table_*_in_value keep the index in the top head bits
 * instead (Sec. III-C, for column counts without spare bits).
 *
 * 16-bit baselines: orc_round16 / orc_widen16 store the values as FP16 or
 * BF16 (round to nearest even, one rounding from FP64) for the baseline SpMV
 * and solvers of Sec. IV-C.
 *
 * Parity status: every function here is pinned by the CPU test suite (closed
 * forms, an independent transcription of Alg. 1/Alg. 2, brute force, exact
 * rational sums, textbook invariants, dense LU).  Nothing is unpinned.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Status codes (oracle-local; the product library defines its own).         */
enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_BREAKDOWN = 2, ORC_NONFINITE = 3,
       ORC_ERR_INVALID = -1 };

static uint64_t bits_of(double v) { uint64_t b; memcpy(&b, &v, 8); return b; }

/* Validates segment widths.  Returns the total magnitude width W_nseg or -1. */
static int total_width(const int* seg_bits, int nseg)
{
    if (nseg < 1 || nseg > 3) return -1;
    if (seg_bits[0] < 2 || seg_bits[0] > 16) return -1;
    int w = seg_bits[0] - 1;
    if (nseg >= 2) { if (seg_bits[1] < 1 || seg_bits[1] > 16) return -1; w += seg_bits[1]; }
    if (nseg >= 3) { if (seg_bits[2] < 1 || seg_bits[2] > 32) return -1; w += seg_bits[2]; }
    if (w > 63) return -1;
    return w;
}

/* Magnitude width of level k (k = 1..nseg). */
static int level_width(const int* seg_bits, int k)
{
    int w = seg_bits[0] - 1;
    for (int i = 1; i < k; i++) w += seg_bits[i];
    return w;
}

/*
 * Encode (Sec. III-B, Alg. 1, with the group rule of the denormalized
 * representation and the segmented storage of Fig. 3).
 *
 * For each group g of G consecutive values (the last one may be partial):
 *  1. e_i = biased exponent field of v_i.  E_g = max_i e_i + 1, or 0 when the
 *     whole group is zeros/subnormals.
 *  2. M_i = floor(|v_i| * 2^(W - (E_g - 1023))), W = W_nseg: the significand
 *     with its explicit leading 1, right-aligned so that a value with d = 1
 *     puts its leading 1 at bit W - 1.  Round toward zero, as Alg. 1 does.
 *     Zeros and subnormals give M = 0 (sign kept).
 *  3. head  = sign << (s1 - 1) | M >> (W - W_1)
 *     tail1 = (M >> (W - W_2)) & (2^s2 - 1)
 *     tail2 = M & (2^s3 - 1)
 * Rejects non-finite input with ORC_NONFINITE.
 */
int orc_encode(int64_t nnz, const double* val, int G, const int* seg_bits, int nseg,
               uint16_t* head, uint16_t* tail1, uint32_t* tail2, int16_t* gexp)
{
    int W = total_width(seg_bits, nseg);
    if (W < 0 || G < 1 || nnz < 0) return ORC_ERR_INVALID;
    int W1 = level_width(seg_bits, 1);
    int W2 = nseg >= 2 ? level_width(seg_bits, 2) : W1;
    int64_t ngroups = (nnz + G - 1) / G;
    for (int64_t g = 0; g < ngroups; g++) {
        int64_t lo = g * G, hi = lo + G < nnz ? lo + G : nnz;
        /* step 1: the group's shared exponent */
        int emax = 0;
        for (int64_t i = lo; i < hi; i++) {
            uint64_t b = bits_of(val[i]);
            int e = (int)((b >> 52) & 0x7FF);
            if (e == 0x7FF) return ORC_NONFINITE;
            if (e > emax) emax = e;
        }
        int Eg = emax == 0 ? 0 : emax + 1;
        gexp[g] = (int16_t)Eg;
        /* steps 2 and 3, one value at a time */
        for (int64_t i = lo; i < hi; i++) {
            uint64_t b = bits_of(val[i]);
            uint64_t sign = b >> 63;
            int e = (int)((b >> 52) & 0x7FF);
            uint64_t M = 0;
            if (e != 0) {
                uint64_t S = (1ULL << 52) | (b & ((1ULL << 52) - 1));
                int d = Eg - e;                 /* >= 1 */
                int shift = W - 52 - d;         /* M = S * 2^shift, truncated */
                if (shift >= 0) M = S << shift;
                else if (-shift < 64) M = S >> (-shift);
                else M = 0;
            }
            head[i] = (uint16_t)((sign << (seg_bits[0] - 1)) | (M >> (W - W1)));
            if (tail1) tail1[i] = nseg >= 2 ? (uint16_t)((M >> (W - W2)) & ((1ULL << seg_bits[1]) - 1)) : 0;
            if (tail2) tail2[i] = nseg >= 3 ? (uint32_t)(M & ((1ULL << seg_bits[2]) - 1)) : 0;
        }
    }
    return ORC_OK;
}

/*
 * Decode one value at level k (Alg. 2 for k = 1; the concatenation of head and
 * tails described after Alg. 2 for k = 2, 3):
 *   M_k = head_magnitude << (W_k - W_1) | tail1 << (W_k - W_2) | tail2
 *   value = (-1)^sign * M_k * 2^(E_g - 1023 - W_k)
 * (double)M_k is exact (M_k holds at most 53 significant bits); ldexp is exact
 * unless the result is subnormal, where it rounds to nearest even.
 */
static double decode_one(uint16_t h, uint16_t t1, uint32_t t2, int Eg,
                         const int* seg_bits, int k)
{
    int s1 = seg_bits[0];
    uint64_t sign = (h >> (s1 - 1)) & 1;
    uint64_t M = h & ((1u << (s1 - 1)) - 1);
    if (k >= 2) M = (M << seg_bits[1]) | t1;
    if (k >= 3) M = (M << seg_bits[2]) | t2;
    int Wk = level_width(seg_bits, k);
    double v = ldexp((double)M, Eg - 1023 - Wk);
    return sign ? -v : v;
}

int orc_decode(int64_t nnz, const uint16_t* head, const uint16_t* tail1, const uint32_t* tail2,
               const int16_t* gexp, int G, const int* seg_bits, int nseg, int k, double* out)
{
    if (total_width(seg_bits, nseg) < 0 || k < 1 || k > nseg || G < 1) return ORC_ERR_INVALID;
    for (int64_t i = 0; i < nnz; i++)
        out[i] = decode_one(head[i], k >= 2 ? tail1[i] : 0, k >= 3 ? tail2[i] : 0,
                            gexp[i / G], seg_bits, k);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Global shared-exponent table (the paper's default format): one table of   */
/* numExp shared exponents for the whole matrix (Sec. III-B), the exponent   */
/* index of each nonzero kept beside its column index (Sec. III-C).          */

/*
 * Sec. III-B, "Shared Exponents Extraction": count the nonzeros carrying each
 * exponent, order the exponents by count (descending; equal counts: the larger
 * exponent first), keep the first numExp and store each one plus 1 (Sec. III-B,
 * "Denormalized Representation": the hidden one becomes explicit).  The same
 * passage requires max(e) + 1 to be one of them; when the largest exponent did
 * not make the cut it replaces the last kept entry.  Zeros and subnormals
 * (e = 0) are not counted.  Returns the number of entries (at most numExp); a
 * matrix without a normal value gets the single entry 0.  Returns -ORC_NONFINITE
 * when a value is Inf or NaN, ORC_ERR_INVALID for bad arguments.
 */
static int select_entries(const int64_t* count, int emax, int num_exp, int16_t* table)
{
    int n = 0;
    int taken[2048] = {0};
    while (n < num_exp) {                 /* selection by (count desc, exponent desc) */
        int best = -1;
        for (int e = 2046; e >= 1; e--)
            if (count[e] > 0 && !taken[e] && (best < 0 || count[e] > count[best])) best = e;
        if (best < 0) break;
        taken[best] = 1;
        table[n++] = (int16_t)(best + 1);
    }
    if (n == 0) table[n++] = (int16_t)(emax + 1);   /* nothing counted: max + 1 alone */
    else if (!taken[emax]) table[n - 1] = (int16_t)(emax + 1);
    return n;
}

/* The exact extraction: every nonzero counted once. */
int orc_table_build(int64_t nnz, const double* val, int num_exp, int16_t* table)
{
    if (num_exp < 1 || nnz < 0) return ORC_ERR_INVALID;
    int64_t* count = calloc(2048, sizeof(int64_t));
    int emax = 0;
    for (int64_t i = 0; i < nnz; i++) {
        int e = (int)((bits_of(val[i]) >> 52) & 0x7FF);
        if (e == 0x7FF) { free(count); return -ORC_NONFINITE; }
        if (e == 0) continue;
        count[e]++;
        if (e > emax) emax = e;
    }
    if (emax == 0) { table[0] = 0; free(count); return 1; }
    int n = select_entries(count, emax, num_exp, table);
    free(count);
    return n;
}

/*
 * Sec. III-B, the sampled extraction: the rows are cut into blocks of
 * block_rows consecutive rows (the last may be shorter) and the exponent
 * distribution of one row per block, sample_rows[b] (drawn by the caller),
 * stands for the distribution of the whole block.  Reading: every row of block
 * b is taken to hold the sampled row's exponents, so each of that row's
 * nonzeros counts rows_in_block(b) times.  The selection is then that of
 * orc_table_build.  max(e) + 1 must stay in the table for the encoding to be
 * able to hold every value (Sec. III-B, "Denormalized Representation"), so the
 * maximum exponent is taken over all values, not over the sample.  Returns the
 * number of entries, -ORC_NONFINITE on Inf/NaN, ORC_ERR_INVALID for bad
 * arguments or a sample row outside its block.
 */
int orc_table_build_sampled(int64_t n_rows, const int32_t* row_ptr, const double* val, int num_exp,
                            int64_t block_rows, const int64_t* sample_rows, int16_t* table)
{
    if (num_exp < 1 || n_rows < 0 || block_rows < 1) return ORC_ERR_INVALID;
    int64_t nnz = n_rows > 0 ? row_ptr[n_rows] : 0;
    int emax = 0;
    for (int64_t i = 0; i < nnz; i++) {
        int e = (int)((bits_of(val[i]) >> 52) & 0x7FF);
        if (e == 0x7FF) return -ORC_NONFINITE;
        if (e > emax) emax = e;
    }
    int64_t n_blocks = (n_rows + block_rows - 1) / block_rows;
    for (int64_t b = 0; b < n_blocks; b++)
        if (sample_rows[b] < b * block_rows || sample_rows[b] >= b * block_rows + block_rows ||
            sample_rows[b] >= n_rows)
            return ORC_ERR_INVALID;
    if (emax == 0) { table[0] = 0; return 1; }
    int64_t* count = calloc(2048, sizeof(int64_t));
    for (int64_t b = 0; b < n_blocks; b++) {
        int64_t first = b * block_rows;
        int64_t rows_in_block = first + block_rows <= n_rows ? block_rows : n_rows - first;
        int64_t r = sample_rows[b];
        for (int64_t j = row_ptr[r]; j < row_ptr[r + 1]; j++) {
            int e = (int)((bits_of(val[j]) >> 52) & 0x7FF);
            if (e != 0) count[e] += rows_in_block;
        }
    }
    int n = select_entries(count, emax, num_exp, table);
    free(count);
    return n;
}

/* Alg. 1, the search for one value's shared exponent: the entry equal to
 * e + 1 (then minDiff = 1), else the nearest entry above e (minDiff = entry - e,
 * the smallest positive difference).  e = 0 (zero or subnormal) takes index 0;
 * its mantissa is 0 anyway. */
static void table_lookup(int e, const int16_t* table, int n_table, int* idx, int* d)
{
    *idx = 0;
    *d = 1;
    if (e == 0) return;
    for (int k = 0; k < n_table; k++)
        if (table[k] == e + 1) { *idx = k; *d = 1; return; }
    int min_diff = 1 << 30;
    for (int jj = 0; jj < n_table; jj++) {
        int diff = table[jj] - e;
        if (diff > 0 && diff < min_diff) { min_diff = diff; *idx = jj; }
    }
    *d = min_diff;
}

/* Alg. 1 for every nonzero against the table, then the segment split of
 * Fig. 3: M = floor(|v| * 2^(W - (T - 1023))) with T = table[index], i.e. the
 * 53-bit significand S shifted right by 52 + d - W (truncation, as Alg. 1;
 * M = 0 once the explicit one is shifted out).  idx receives the index. */
int orc_table_encode(int64_t nnz, const double* val, const int16_t* table, int n_table,
                     const int* seg_bits, int nseg, uint16_t* head, uint16_t* tail1, uint32_t* tail2,
                     uint8_t* idx)
{
    int W = total_width(seg_bits, nseg);
    if (W < 0 || n_table < 1 || nnz < 0) return ORC_ERR_INVALID;
    int W1 = level_width(seg_bits, 1);
    int W2 = nseg >= 2 ? level_width(seg_bits, 2) : W1;
    for (int64_t i = 0; i < nnz; i++) {
        uint64_t b = bits_of(val[i]);
        uint64_t sign = b >> 63;
        int e = (int)((b >> 52) & 0x7FF);
        if (e == 0x7FF) return ORC_NONFINITE;
        int k, d;
        table_lookup(e, table, n_table, &k, &d);
        uint64_t M = 0;
        if (e != 0) {
            uint64_t S = (1ULL << 52) | (b & ((1ULL << 52) - 1));
            int shift = W - 52 - d;
            if (shift >= 0) M = S << shift;
            else if (-shift < 64) M = S >> (-shift);
            else M = 0;
        }
        idx[i] = (uint8_t)k;
        head[i] = (uint16_t)((sign << (seg_bits[0] - 1)) | (M >> (W - W1)));
        if (tail1) tail1[i] = nseg >= 2 ? (uint16_t)((M >> (W - W2)) & ((1ULL << seg_bits[1]) - 1)) : 0;
        if (tail2) tail2[i] = nseg >= 3 ? (uint32_t)(M & ((1ULL << seg_bits[2]) - 1)) : 0;
    }
    return ORC_OK;
}

/* Decode at level k with the table: as decode_one, the shared exponent being
 * table[idx[i]] (Alg. 2 reads it from the exponent array by the index). */
int orc_table_decode(int64_t nnz, const uint16_t* head, const uint16_t* tail1, const uint32_t* tail2,
                     const uint8_t* idx, const int16_t* table, int n_table, const int* seg_bits, int nseg,
                     int k, double* out)
{
    if (total_width(seg_bits, nseg) < 0 || k < 1 || k > nseg || n_table < 1) return ORC_ERR_INVALID;
    for (int64_t i = 0; i < nnz; i++) {
        if (idx[i] >= n_table) return ORC_ERR_INVALID;
        out[i] = decode_one(head[i], k >= 2 ? tail1[i] : 0, k >= 3 ? tail2[i] : 0, table[idx[i]], seg_bits, k);
    }
    return ORC_OK;
}

/*
 * Sec. III-C, the index kept in the value array instead of the column index
 * (for matrices whose column count leaves no spare bits).  Reading: the
 * ceil(log2(n_table)) index bits b take the top magnitude bits of the head,
 * right below the sign, so every level has b magnitude bits fewer:
 *   head = sign << (s1 - 1) | index << (s1 - 1 - b) | M >> (W' - W'_1),
 * where M is the Alg. 1 mantissa for the widths {s1 - b, s2, s3}, i.e. the
 * segment split of orc_table_encode with a head of s1 - b bits whose sign is
 * then moved up past the index.  Requires b <= s1 - 2.
 */
static int index_bits(int n_table)
{
    int b = 0;
    while ((1 << b) < n_table) b++;
    return b;
}

int orc_table_encode_in_value(int64_t nnz, const double* val, const int16_t* table, int n_table,
                              const int* seg_bits, int nseg, uint16_t* head, uint16_t* tail1, uint32_t* tail2)
{
    if (total_width(seg_bits, nseg) < 0 || n_table < 1 || nnz < 0) return ORC_ERR_INVALID;
    int b = index_bits(n_table);
    if (b > seg_bits[0] - 2) return ORC_ERR_INVALID;
    int short_bits[3] = {seg_bits[0] - b, nseg >= 2 ? seg_bits[1] : 0, nseg >= 3 ? seg_bits[2] : 0};
    uint8_t* idx = malloc(nnz > 0 ? (size_t)nnz : 1);
    int rc = orc_table_encode(nnz, val, table, n_table, short_bits, nseg, head, tail1, tail2, idx);
    if (rc == ORC_OK) {
        int ws = short_bits[0] - 1;                     /* magnitude bits left in the head */
        for (int64_t i = 0; i < nnz; i++) {
            uint32_t sign = (head[i] >> ws) & 1u;
            uint32_t mag = head[i] & ((1u << ws) - 1u);
            head[i] = (uint16_t)((sign << (seg_bits[0] - 1)) | ((uint32_t)idx[i] << ws) | mag);
        }
    }
    free(idx);
    return rc;
}

/* Decode of that layout at level k: the index and the short head are taken
 * apart again and decoded as the table format with the widths {s1 - b, s2, s3}. */
int orc_table_decode_in_value(int64_t nnz, const uint16_t* head, const uint16_t* tail1, const uint32_t* tail2,
                              const int16_t* table, int n_table, const int* seg_bits, int nseg, int k, double* out)
{
    if (total_width(seg_bits, nseg) < 0 || k < 1 || k > nseg || n_table < 1) return ORC_ERR_INVALID;
    int b = index_bits(n_table);
    if (b > seg_bits[0] - 2) return ORC_ERR_INVALID;
    int short_bits[3] = {seg_bits[0] - b, nseg >= 2 ? seg_bits[1] : 0, nseg >= 3 ? seg_bits[2] : 0};
    int ws = short_bits[0] - 1;
    for (int64_t i = 0; i < nnz; i++) {
        uint32_t sign = (head[i] >> (seg_bits[0] - 1)) & 1u;
        uint32_t ix = (head[i] >> ws) & ((1u << b) - 1u);
        uint32_t mag = head[i] & ((1u << ws) - 1u);
        if ((int)ix >= n_table) return ORC_ERR_INVALID;
        uint16_t h = (uint16_t)((sign << ws) | mag);
        out[i] = decode_one(h, k >= 2 ? tail1[i] : 0, k >= 3 ? tail2[i] : 0, table[ix], short_bits, k);
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* 16-bit baselines (Sec. IV-C): the nonzeros stored as IEEE binary16 (FP16) */
/* or bfloat16 (BF16), converted once from FP64 by rounding to nearest, ties */
/* to even, and widened back to FP64 exactly for the multiply-accumulate.    */

/* Round |v| to a binary format with ebits exponent bits and mbits stored
 * mantissa bits (FP16: 5, 10; BF16: 8, 7).  The quantum of v's binade (of the
 * subnormal range below the smallest normal) divides |v| exactly; rint() in the
 * default mode rounds the quotient to nearest even.  A carry into the next
 * binade and overflow to infinity follow from the encoding. */
static uint16_t round_small(double v, int ebits, int mbits)
{
    uint16_t sign = signbit(v) ? (uint16_t)(1u << (ebits + mbits)) : 0;
    int bias = (1 << (ebits - 1)) - 1, emin = 1 - bias, emax = bias;
    uint16_t inf = (uint16_t)(((1u << ebits) - 1) << mbits);
    double a = fabs(v);
    if (isnan(v)) return (uint16_t)(sign | inf | (1u << (mbits - 1)));
    if (isinf(v)) return (uint16_t)(sign | inf);
    if (a == 0.0) return sign;
    int e;
    frexp(a, &e);
    int E = e - 1;                       /* a in [2^E, 2^(E+1)) */
    int qexp = (E < emin ? emin : E) - mbits;
    double n = rint(ldexp(a, -qexp));    /* integer, at most 2^(mbits+1) */
    uint32_t ni = (uint32_t)n;
    if (E < emin) return (uint16_t)(sign | ni);      /* n = 2^mbits lands on the smallest normal */
    if (ni == (1u << (mbits + 1))) { ni >>= 1; E++; }
    if (E > emax) return (uint16_t)(sign | inf);
    return (uint16_t)(sign | ((uint32_t)(E + bias) << mbits) | (ni - (1u << mbits)));
}

static double widen_small(uint16_t h, int ebits, int mbits)
{
    int bias = (1 << (ebits - 1)) - 1;
    int ef = (h >> mbits) & ((1 << ebits) - 1);
    uint32_t man = h & ((1u << mbits) - 1);
    double s = (h >> (ebits + mbits)) & 1 ? -1.0 : 1.0;
    if (ef == (1 << ebits) - 1) return man ? NAN : s * INFINITY;
    if (ef == 0) return s * ldexp((double)man, 1 - bias - mbits);
    return s * ldexp((double)(man | (1u << mbits)), ef - bias - mbits);
}

/* kind 16: FP16, 17: BF16.  n_overflow counts finite values that became
 * infinite (the FP16 arithmetic overflow the paper reports). */
int orc_round16(int64_t n, const double* val, int kind, uint16_t* out, int64_t* n_overflow)
{
    if (kind != 16 && kind != 17) return ORC_ERR_INVALID;
    int eb = kind == 16 ? 5 : 8, mb = kind == 16 ? 10 : 7;
    int64_t ov = 0;
    for (int64_t i = 0; i < n; i++) {
        out[i] = round_small(val[i], eb, mb);
        if (isfinite(val[i]) && ((out[i] >> mb) & ((1 << eb) - 1)) == (1 << eb) - 1) ov++;
    }
    if (n_overflow) *n_overflow = ov;
    return ORC_OK;
}

int orc_widen16(int64_t n, const uint16_t* in, int kind, double* out)
{
    if (kind != 16 && kind != 17) return ORC_ERR_INVALID;
    int eb = kind == 16 ? 5 : 8, mb = kind == 16 ? 10 : 7;
    for (int64_t i = 0; i < n; i++) out[i] = widen_small(in[i], eb, mb);
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* SpMV                                                                      */

/* y_i = sum_j a_ij x_{c(j)} in FP64, left to right in row order (Sec. III-C:
 * values are widened and multiplied/accumulated in double precision). */
void orc_spmv(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
              const double* x, double* y)
{
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; j++) s = s + a[j] * x[col[j]];
        y[i] = s;
    }
}

/* Row i of the GSE-SpMV at level k (Alg. 2 and the two tail variants after
 * it): each value is decoded to FP64 as it is read, then multiplied and
 * accumulated in FP64, left to right. */
static double gse_row(int64_t i, const int32_t* row_ptr, const int32_t* col,
                      const uint16_t* head, const uint16_t* tail1, const uint32_t* tail2,
                      const int16_t* gexp, int G, const int* seg_bits, int k, const double* x)
{
    double s = 0.0;
    for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; j++) {
        double v = decode_one(head[j], k >= 2 ? tail1[j] : 0, k >= 3 ? tail2[j] : 0,
                              gexp[j / G], seg_bits, k);
        s = s + v * x[col[j]];
    }
    return s;
}

/* GSE-SpMV at level k: y_i = row i for every row. */
int orc_gse_spmv(int64_t n, const int32_t* row_ptr, const int32_t* col,
                 const uint16_t* head, const uint16_t* tail1, const uint32_t* tail2,
                 const int16_t* gexp, int G, const int* seg_bits, int nseg, int k,
                 const double* x, double* y)
{
    if (total_width(seg_bits, nseg) < 0 || k < 1 || k > nseg || G < 1) return ORC_ERR_INVALID;
    for (int64_t i = 0; i < n; i++) y[i] = gse_row(i, row_ptr, col, head, tail1, tail2, gexp, G, seg_bits, k, x);
    return ORC_OK;
}

/* The same GSE-SpMV over rows [r0, r1) only (y indexed by row), with the rows
 * shared among `threads` OpenMP threads when threads > 1.  Every row is summed
 * exactly as in orc_gse_spmv; only which thread computes it changes.  Used for
 * the timed CPU baselines (a row sample; all host cores). */
int orc_gse_spmv_rows(int64_t r0, int64_t r1, const int32_t* row_ptr, const int32_t* col,
                      const uint16_t* head, const uint16_t* tail1, const uint32_t* tail2,
                      const int16_t* gexp, int G, const int* seg_bits, int nseg, int k,
                      const double* x, double* y, int threads)
{
    if (total_width(seg_bits, nseg) < 0 || k < 1 || k > nseg || G < 1 || r0 < 0 || r1 < r0 || threads < 1)
        return ORC_ERR_INVALID;
#pragma omp parallel for num_threads(threads) schedule(dynamic, 4096) if (threads > 1)
    for (int64_t i = r0; i < r1; i++) y[i] = gse_row(i, row_ptr, col, head, tail1, tail2, gexp, G, seg_bits, k, x);
    return ORC_OK;
}

/* Compensated dot product Dot2 (Ogita, Rump, Oishi, "Accurate sum and dot
 * product", SIAM J. Sci. Comput. 26(6), 2005, Algorithm 5.3): TwoProduct by
 * fma, TwoSum (Knuth) for the running sum, error terms summed in FP64.  The
 * result is as accurate as if computed in twice the working precision and then
 * rounded.  yabs_i = sum_j |a_ij x_j| is the scale of the parity criterion. */
void orc_spmv_dot2(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
                   const double* x, double* y, double* yabs)
{
    for (int64_t i = 0; i < n; i++) {
        double p = 0.0, s = 0.0, sa = 0.0;
        for (int32_t j = row_ptr[i]; j < row_ptr[i + 1]; j++) {
            double h = a[j] * x[col[j]];
            double r = fma(a[j], x[col[j]], -h);      /* TwoProduct: a*x = h + r exactly */
            double q0 = p + h;                        /* TwoSum(p, h) = (q0, q) */
            double z = q0 - p;
            double q = (p - (q0 - z)) + (h - z);
            p = q0;
            s = s + (q + r);
            sa = sa + fabs(h);
        }
        y[i] = p + s;
        if (yabs) yabs[i] = sa;
    }
}

/* ------------------------------------------------------------------------ */
/* Dense helpers (plain loops).                                              */

static double dot(int64_t n, const double* u, const double* v)
{
    double s = 0.0;
    for (int64_t i = 0; i < n; i++) s = s + u[i] * v[i];
    return s;
}

static double nrm2(int64_t n, const double* u) { return sqrt(dot(n, u, u)); }

/* r = b - A x */
static void residual(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
                     const double* b, const double* x, double* r)
{
    orc_spmv(n, row_ptr, col, a, x, r);
    for (int64_t i = 0; i < n; i++) r[i] = b[i] - r[i];
}

typedef struct {
    int status, iters, k_final;
    int switch_iter[3];           /* iteration at which level k+1 began (-1: never) */
    double rel_res_rec, rel_res_true;
} orc_info;

typedef struct {
    int l, t, m;
    double rsd_limit;
    int ndec_limit;
    double reldec_limit;
    int max_iter, restart, k_start, k_max, flags;
} orc_policy;

/* Policy flag: evaluate only the convergence check, never Conditions 1-3. */
#define ORC_POLICY_NO_STAGNATION 1
#define ORC_POLICY_FLOOR 2          /* the perturbation-floor trigger (beyond the paper) */

/*
 * Plain FP64 CG (Hestenes-Stiefel), the FP64 baseline of Sec. IV.  Stops when
 * ||r_j|| / ||b|| < tol (recurrence residual).  Optional traces: r_j, p_j, x_j
 * for j = 0 .. trace_n - 1, each row n long.
 */
int orc_cg(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
           const double* b, double* x, double tol, int max_iter, orc_info* info,
           double* trace_r, double* trace_p, double* trace_x, int trace_n)
{
    double* r = malloc(n * sizeof(double));
    double* p = malloc(n * sizeof(double));
    double* q = malloc(n * sizeof(double));
    residual(n, row_ptr, col, a, b, x, r);
    memcpy(p, r, n * sizeof(double));
    double nb = nrm2(n, b);
    double rho = dot(n, r, r);
    int status = ORC_MAXITER, it = 0;
    double res = nb > 0 ? sqrt(rho) / nb : 0.0;
    if (nb == 0.0) { for (int64_t i = 0; i < n; i++) x[i] = 0.0; res = 0.0; }
    if (res < tol) status = ORC_OK;
    for (it = 0; status != ORC_OK && it < max_iter; ) {
        if (trace_n > it) {
            if (trace_r) memcpy(trace_r + it * n, r, n * sizeof(double));
            if (trace_p) memcpy(trace_p + it * n, p, n * sizeof(double));
            if (trace_x) memcpy(trace_x + it * n, x, n * sizeof(double));
        }
        orc_spmv(n, row_ptr, col, a, p, q);
        double pq = dot(n, p, q);
        if (!isfinite(pq)) { status = ORC_NONFINITE; break; }
        if (pq <= 0.0) { status = ORC_BREAKDOWN; break; }
        double alpha = rho / pq;
        for (int64_t i = 0; i < n; i++) x[i] = x[i] + alpha * p[i];
        for (int64_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
        double rho_new = dot(n, r, r);
        it++;
        res = sqrt(rho_new) / nb;
        if (!isfinite(res)) { status = ORC_NONFINITE; break; }
        if (res < tol) { status = ORC_OK; break; }
        double beta = rho_new / rho;
        for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
        rho = rho_new;
    }
    if (trace_n > it) {
        if (trace_r) memcpy(trace_r + it * n, r, n * sizeof(double));
        if (trace_p) memcpy(trace_p + it * n, p, n * sizeof(double));
        if (trace_x) memcpy(trace_x + it * n, x, n * sizeof(double));
    }
    if (info) {
        info->status = status; info->iters = it; info->k_final = 0;
        info->switch_iter[0] = info->switch_iter[1] = info->switch_iter[2] = -1;
        info->rel_res_rec = res;
        residual(n, row_ptr, col, a, b, x, q);
        info->rel_res_true = nb > 0 ? nrm2(n, q) / nb : 0.0;
    }
    free(r); free(p); free(q);
    return status;
}

/*
 * Restarted GMRES(restart) in FP64 with modified Gram-Schmidt Arnoldi and
 * Givens rotations; each cycle restarts from the true residual.  Stops when the
 * least-squares residual |g_{i+1}| / ||b|| < tol.  Optional outputs of the
 * first cycle: V (restart + 1 basis vectors of length n, vector-major) and the
 * Hessenberg matrix H ((restart + 1) x restart, row-major) before rotation.
 */
typedef struct {
    double *V, *H, *Hrot, *cs, *sn, *g, *y, *w;
} gmres_ws;

static int gmres_cycle(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
                       const double* b, double* x, int restart, double nb, double tol,
                       int* iters, int max_iter, gmres_ws* ws, double* hist, int* hist_len,
                       double* res_out, double* V_out, double* H_out)
{
    int m = restart;
    double* V = ws->V;
    residual(n, row_ptr, col, a, b, x, V);
    double beta = nrm2(n, V);
    *res_out = beta / nb;
    if (!isfinite(beta)) return ORC_NONFINITE;
    if (beta / nb < tol || beta == 0.0) return ORC_OK;
    for (int64_t t = 0; t < n; t++) V[t] = V[t] / beta;
    for (int i = 0; i <= m; i++) ws->g[i] = 0.0;
    ws->g[0] = beta;
    int done = 0, i;
    for (i = 0; i < m && !done; i++) {
        double* vi = V + (int64_t)i * n;
        double* w = V + (int64_t)(i + 1) * n;
        orc_spmv(n, row_ptr, col, a, vi, w);
        double* h = ws->H + (int64_t)i * (m + 1);     /* column i of H, length m+1 */
        for (int j = 0; j <= i; j++) {
            double* vj = V + (int64_t)j * n;
            h[j] = dot(n, w, vj);
            for (int64_t t = 0; t < n; t++) w[t] = w[t] - h[j] * vj[t];
        }
        h[i + 1] = nrm2(n, w);
        if (H_out) for (int j = 0; j <= i + 1; j++) H_out[(int64_t)j * m + i] = h[j];
        if (h[i + 1] != 0.0) for (int64_t t = 0; t < n; t++) w[t] = w[t] / h[i + 1];
        /* apply the previous rotations to column i, then make a new one */
        double* hr = ws->Hrot + (int64_t)i * (m + 1);
        for (int j = 0; j <= i + 1; j++) hr[j] = h[j];
        for (int j = 0; j < i; j++) {
            double t0 = ws->cs[j] * hr[j] + ws->sn[j] * hr[j + 1];
            hr[j + 1] = -ws->sn[j] * hr[j] + ws->cs[j] * hr[j + 1];
            hr[j] = t0;
        }
        double den = hypot(hr[i], hr[i + 1]);
        if (den == 0.0 || !isfinite(den)) return ORC_BREAKDOWN;
        ws->cs[i] = hr[i] / den;
        ws->sn[i] = hr[i + 1] / den;
        hr[i] = den;
        hr[i + 1] = 0.0;
        ws->g[i + 1] = -ws->sn[i] * ws->g[i];
        ws->g[i] = ws->cs[i] * ws->g[i];
        (*iters)++;
        double res = fabs(ws->g[i + 1]) / nb;
        *res_out = res;
        if (hist) hist[(*hist_len)++] = res;
        if (res < tol || h[i + 1] == 0.0 || *iters >= max_iter) done = 1;
    }
    if (V_out) memcpy(V_out, V, (size_t)(i + 1) * n * sizeof(double));
    /* back substitution R y = g, then x += V y */
    for (int j = i - 1; j >= 0; j--) {
        double s = ws->g[j];
        for (int c = j + 1; c < i; c++) s = s - ws->Hrot[(int64_t)c * (m + 1) + j] * ws->y[c];
        ws->y[j] = s / ws->Hrot[(int64_t)j * (m + 1) + j];
    }
    for (int j = 0; j < i; j++)
        for (int64_t t = 0; t < n; t++) x[t] = x[t] + ws->y[j] * V[(int64_t)j * n + t];
    return *res_out < tol ? ORC_OK : ORC_MAXITER;
}

static int gmres_ws_alloc(gmres_ws* ws, int64_t n, int m)
{
    ws->V = malloc((size_t)(m + 1) * n * sizeof(double));
    ws->H = calloc((size_t)(m + 1) * m, sizeof(double));
    ws->Hrot = calloc((size_t)(m + 1) * m, sizeof(double));
    ws->cs = malloc(m * sizeof(double));
    ws->sn = malloc(m * sizeof(double));
    ws->g = malloc((m + 1) * sizeof(double));
    ws->y = malloc((m + 1) * sizeof(double));
    ws->w = NULL;
    return ws->V && ws->H && ws->Hrot && ws->cs && ws->sn && ws->g && ws->y;
}

static void gmres_ws_free(gmres_ws* ws)
{
    free(ws->V); free(ws->H); free(ws->Hrot); free(ws->cs); free(ws->sn); free(ws->g); free(ws->y);
}

int orc_gmres(int64_t n, const int32_t* row_ptr, const int32_t* col, const double* a,
              const double* b, double* x, double tol, int restart, int max_iter, orc_info* info,
              double* V_out, double* H_out)
{
    gmres_ws ws;
    if (restart < 1 || !gmres_ws_alloc(&ws, n, restart)) return ORC_ERR_INVALID;
    double nb = nrm2(n, b);
    int iters = 0, status = ORC_MAXITER, cycle = 0;
    double res = 0.0;
    if (nb == 0.0) { for (int64_t i = 0; i < n; i++) x[i] = 0.0; status = ORC_OK; }
    while (status != ORC_OK && iters < max_iter) {
        int s = gmres_cycle(n, row_ptr, col, a, b, x, restart, nb, tol, &iters, max_iter, &ws,
                            NULL, NULL, &res, cycle == 0 ? V_out : NULL, cycle == 0 ? H_out : NULL);
        cycle++;
        if (s == ORC_OK) { status = ORC_OK; break; }
        if (s == ORC_BREAKDOWN || s == ORC_NONFINITE) { status = s; break; }
    }
    if (info) {
        info->status = status; info->iters = iters; info->k_final = 0;
        info->switch_iter[0] = info->switch_iter[1] = info->switch_iter[2] = -1;
        info->rel_res_rec = res;
        residual(n, row_ptr, col, a, b, x, ws.V);
        info->rel_res_true = nb > 0 ? nrm2(n, ws.V) / nb : 0.0;
    }
    gmres_ws_free(&ws);
    return status;
}

/* ------------------------------------------------------------------------ */
/* Step policy (Sec. III-D, Eqs. 3-6 and Conditions 1-3).                    */

/*
 * Metrics over the window ending at the newest entry resid[len-1] = resid[j]:
 *   Eq. 3  RSD    = sqrt( (1/t) sum_{i=j-t}^{j-1} (resid[i] - avg)^2 ) / avg,
 *                   avg = mean of resid[j-t .. j-1]
 *   Eqs. 4-5 nDec = #{ i in [j-t, j-1] : resid[i] > resid[i+1] }
 *   Eq. 6  relDec = (resid[j-t] - resid[j-1]) / resid[j-t]
 * Needs len >= t + 1.  Returns -1 if not.
 */
int orc_step_metrics(const double* resid, int len, int t, double* rsd, int* ndec, double* reldec)
{
    if (t < 1 || len < t + 1) return -1;
    int j = len - 1;
    double avg = 0.0;
    for (int i = j - t; i <= j - 1; i++) avg = avg + resid[i];
    avg = avg / t;
    double var = 0.0;
    for (int i = j - t; i <= j - 1; i++) var = var + (resid[i] - avg) * (resid[i] - avg);
    *rsd = sqrt(var / t) / avg;
    int nd = 0;
    for (int i = j - t; i <= j - 1; i++) if (resid[i] > resid[i + 1]) nd++;
    *ndec = nd;
    *reldec = (resid[j - t] - resid[j - 1]) / resid[j - t];
    return 0;
}

/*
 * Conditions 1-3 of Sec. III-D.  The paper's parameter list carries an nDec
 * limit (Sec. IV-D) that the conditions write as t/2; the limit takes t/2's
 * place when positive, and t/2 is used otherwise.  Returns a bit mask:
 * 1 = Condition 1, 2 = Condition 2, 4 = Condition 3.
 */
int orc_step_decide(double rsd, int ndec, double reldec, int t, const orc_policy* p)
{
    double thr = p->ndec_limit > 0 ? (double)p->ndec_limit : 0.5 * t;
    int c = 0;
    if (rsd > p->rsd_limit && (double)ndec < thr) c |= 1;
    if ((double)ndec >= thr && reldec < p->reldec_limit) c |= 2;
    if (ndec == 0) c |= 4;
    return c;
}

/* Whether a stagnation check is due at global iteration j (checks start after
 * the first l iterations and recur every m iterations). */
static int check_due(int j, const orc_policy* p)
{
    return j >= p->l && p->m > 0 && j % p->m == 0;
}

/*
 * Stepped mixed-precision CG (Alg. 3 with the policy of Sec. III-D).
 * a_levels[k-1] holds the FP64 values of A_k (k = 1 .. k_max), all on the
 * same CSR structure: the oracle decodes each level once.
 *
 * Readings where the paper is silent:
 *  - the monitored residual is the recurrence residual ||r_j|| / ||b||;
 *  - one level per step;
 *  - at a step: k += 1, r = b - A_k x, p = r, the history is cleared;
 *  - when the recurrence residual drops below tol, the true residual with
 *    A_kmax decides: below tol stops; otherwise the solver steps (or, at
 *    k_max, restarts from the true residual);
 *  - p.Ap <= 0 at k < k_max is treated as a step, at k_max as a breakdown.
 * With ORC_POLICY_FLOOR (an addition beyond the paper, reported apart from it):
 * A_k differs from A_kmax by a perturbation whose infinity norm is
 *   eta_k = max_i sum_j |a_kmax,ij - a_k,ij|,
 * so once the recurrence residual falls to eta_k ||x|| / ||b|| (x the current
 * iterate, 2-norms) level k has nothing more to give and the solver steps,
 * before the stagnation check of that iteration.
 * hist (optional, capacity hist_cap) receives every recurrence residual.
 */
static double level_gap(int64_t n, const int32_t* row_ptr, const double* hi, const double* lo)
{
    double eta = 0.0;
    for (int64_t i = 0; i < n; i++) {
        double s = 0.0;
        for (int32_t e = row_ptr[i]; e < row_ptr[i + 1]; e++) s += fabs(hi[e] - lo[e]);
        if (s > eta) eta = s;
    }
    return eta;
}

int orc_stepped_cg(int64_t n, const int32_t* row_ptr, const int32_t* col,
                   const double* const* a_levels, const double* b, double* x, double tol,
                   const orc_policy* pol, orc_info* info, double* hist, int hist_cap)
{
    int kmax = pol->k_max, k = pol->k_start;
    double* r = malloc(n * sizeof(double));
    double* p = malloc(n * sizeof(double));
    double* q = malloc(n * sizeof(double));
    double* win = malloc(((size_t)pol->max_iter + 2) * sizeof(double));
    int wlen = 0, j = 0, status = ORC_MAXITER, nh = 0;
    int sw[3] = {-1, -1, -1};
    sw[k - 1] = 0;
    double nb = nrm2(n, b), res = 0.0, rho;
    double eta[4] = {0.0, 0.0, 0.0, 0.0};
    if (pol->flags & ORC_POLICY_FLOOR)
        for (int kk = 1; kk < kmax; kk++) eta[kk] = level_gap(n, row_ptr, a_levels[kmax - 1], a_levels[kk - 1]);
    if (nb == 0.0) {
        for (int64_t i = 0; i < n; i++) x[i] = 0.0;
        status = ORC_OK;
    }
    /* (re)start at level k */
    residual(n, row_ptr, col, a_levels[k - 1], b, x, r);
    memcpy(p, r, n * sizeof(double));
    rho = dot(n, r, r);
    res = nb > 0 ? sqrt(rho) / nb : 0.0;
    while (status != ORC_OK && j < pol->max_iter) {
        int restart = 0;
        orc_spmv(n, row_ptr, col, a_levels[k - 1], p, q);
        double pq = dot(n, p, q);
        if (!isfinite(pq)) { status = ORC_NONFINITE; break; }
        if (pq <= 0.0) {
            if (k < kmax) { k++; sw[k - 1] = j; restart = 1; }
            else { status = ORC_BREAKDOWN; break; }
        }
        if (!restart) {
            double alpha = rho / pq;
            for (int64_t i = 0; i < n; i++) x[i] = x[i] + alpha * p[i];
            for (int64_t i = 0; i < n; i++) r[i] = r[i] - alpha * q[i];
            double rho_new = dot(n, r, r);
            j++;
            res = sqrt(rho_new) / nb;
            if (!isfinite(res)) { status = ORC_NONFINITE; break; }
            win[wlen++] = res;
            if (hist && nh < hist_cap) hist[nh++] = res;
            if (res < tol) {
                residual(n, row_ptr, col, a_levels[kmax - 1], b, x, q);
                double tr = nrm2(n, q) / nb;
                if (tr < tol) { status = ORC_OK; break; }
                if (k < kmax) { k++; sw[k - 1] = j; }
                restart = 1;
            } else if (k < kmax && (pol->flags & ORC_POLICY_FLOOR) && res <= eta[k] * nrm2(n, x) / nb) {
                k++; sw[k - 1] = j; restart = 1;
            } else if (k < kmax && !(pol->flags & ORC_POLICY_NO_STAGNATION) &&
                       check_due(j, pol) && wlen >= pol->t + 1) {
                double rsd, reldec; int ndec;
                orc_step_metrics(win, wlen, pol->t, &rsd, &ndec, &reldec);
                if (orc_step_decide(rsd, ndec, reldec, pol->t, pol)) {
                    k++; sw[k - 1] = j; restart = 1;
                }
            }
            if (!restart) {
                double beta = rho_new / rho;
                for (int64_t i = 0; i < n; i++) p[i] = r[i] + beta * p[i];
                rho = rho_new;
            }
        }
        if (restart) {
            residual(n, row_ptr, col, a_levels[k - 1], b, x, r);
            memcpy(p, r, n * sizeof(double));
            rho = dot(n, r, r);
            wlen = 0;
        }
    }
    if (info) {
        info->status = status; info->iters = j; info->k_final = k;
        for (int i = 0; i < 3; i++) info->switch_iter[i] = sw[i];
        info->rel_res_rec = res;
        residual(n, row_ptr, col, a_levels[kmax - 1], b, x, q);
        info->rel_res_true = nb > 0 ? nrm2(n, q) / nb : 0.0;
    }
    free(r); free(p); free(q); free(win);
    return status;
}

/*
 * Stepped mixed-precision GMRES(restart).  Same readings as the stepped CG,
 * except that the level changes only at restart boundaries (changing A inside
 * an Arnoldi cycle would break A V = V H): after each cycle, if a check fell
 * due during the cycle (a multiple of m at or after l was crossed) and the
 * history holds t + 1 entries, Eqs. 3-6 and Conditions 1-3 are evaluated.
 * Inner-iteration residuals |g_{i+1}| / ||b|| feed the history.
 */
int orc_stepped_gmres(int64_t n, const int32_t* row_ptr, const int32_t* col,
                      const double* const* a_levels, const double* b, double* x, double tol,
                      const orc_policy* pol, orc_info* info, double* hist, int hist_cap)
{
    gmres_ws ws;
    int m = pol->restart;
    if (m < 1 || !gmres_ws_alloc(&ws, n, m)) return ORC_ERR_INVALID;
    int kmax = pol->k_max, k = pol->k_start;
    double* win = malloc(((size_t)pol->max_iter + m + 2) * sizeof(double));
    int wlen = 0, j = 0, status = ORC_MAXITER, nh = 0;
    int sw[3] = {-1, -1, -1};
    sw[k - 1] = 0;
    double nb = nrm2(n, b), res = 0.0;
    if (nb == 0.0) { for (int64_t i = 0; i < n; i++) x[i] = 0.0; status = ORC_OK; }
    while (status != ORC_OK && j < pol->max_iter) {
        int j_before = j, wlen_before = wlen;
        int s = gmres_cycle(n, row_ptr, col, a_levels[k - 1], b, x, m, nb, tol, &j,
                            pol->max_iter, &ws, win, &wlen, &res, NULL, NULL);
        if (hist) for (int i = wlen_before; i < wlen && nh < hist_cap; i++) hist[nh++] = win[i];
        if (s == ORC_NONFINITE) { status = s; break; }
        if (s == ORC_BREAKDOWN) {
            if (k < kmax) { k++; sw[k - 1] = j; wlen = 0; continue; }
            status = s; break;
        }
        if (s == ORC_OK) {
            residual(n, row_ptr, col, a_levels[kmax - 1], b, x, ws.V);
            double tr = nrm2(n, ws.V) / nb;
            if (tr < tol) { status = ORC_OK; break; }
            if (k < kmax) { k++; sw[k - 1] = j; wlen = 0; }
            continue;
        }
        if (k < kmax && !(pol->flags & ORC_POLICY_NO_STAGNATION) && pol->m > 0 &&
            j >= pol->l && j / pol->m > j_before / pol->m && wlen >= pol->t + 1) {
            double rsd, reldec; int ndec;
            orc_step_metrics(win, wlen, pol->t, &rsd, &ndec, &reldec);
            if (orc_step_decide(rsd, ndec, reldec, pol->t, pol)) { k++; sw[k - 1] = j; wlen = 0; }
        }
    }
    if (info) {
        info->status = status; info->iters = j; info->k_final = k;
        for (int i = 0; i < 3; i++) info->switch_iter[i] = sw[i];
        info->rel_res_rec = res;
        residual(n, row_ptr, col, a_levels[kmax - 1], b, x, ws.V);
        info->rel_res_true = nb > 0 ? nrm2(n, ws.V) / nb : 0.0;
    }
    gmres_ws_free(&ws);
    free(win);
    return status;
}
